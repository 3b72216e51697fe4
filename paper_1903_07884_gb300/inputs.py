"""Seeded synthetic inputs: voxel permittivity fields, incident fields, partition
boxes and the serving request stream.

This module is shared by the CUDA path's tests/bench and by the CPU oracle.  It
holds none of the solver's arithmetic: it only *describes* a scatterer (the
complex relative permittivity per voxel, Sec. 2, eps_r = eps' - j eps'') and a
source field sampled at voxel centres.  The material operator M, the Green's
generators, the preconditioner and the solver are computed separately by each
side.

Geometries stand in for the paper's straight waveguide (Sec. 3, Sec. 5.1),
Bragg grating (Sec. 5.2, Fig. "Bragg") and directional coupler (Sec. 5.3.2).
Materials follow Table 1 (Si 12.11, SiO2 2.085).  Time dependence is
e^{+j omega t} (Sec. 2), so a wave travelling towards +x is exp(-j k x) and a
lossy material has eps = eps' - j eps'' with eps'' >= 0.

Conventions
-----------
* Arrays are C-ordered ``[nz][ny][nx]`` (x fastest); vector fields are
  ``[3][nz][ny][nx]`` with component order (x, y, z).
* Voxel centres sit at ``(i + 1/2) h``.
* Lengths are in micrometres; k0 = 2 pi / lambda in 1/um.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

EPS_SI = 12.11        # silicon, Table 1 (12.1) at the precision the workloads state
EPS_SIO2 = 2.085      # silicon dioxide, Table 1
N_EFF_INC = 3.48      # phase index of the synthetic incident wave (sqrt(12.11))
SIGMA_INC = 0.15      # Gaussian half-width of the incident profile, um

Box = Tuple[int, ...]   # (x0, y0, z0, nx, ny, nz[, levels]); levels 2 = 2-level circulant


@dataclasses.dataclass
class Problem:
    """One scattering problem on a uniform voxel grid."""
    name: str
    nx: int
    ny: int
    nz: int
    h: float                 # voxel edge, um
    wavelength: float        # free-space wavelength, um
    eps_bg: float            # background (cladding) relative permittivity
    eps: np.ndarray          # complex128 [nz][ny][nx], relative permittivity
    e_inc: np.ndarray        # complex128 [3][nz][ny][nx], incident field
    boxes: List[Box]         # preconditioner partition; [] = whole grid
    homog: int = 3           # homogenisation variant (1 mode, 2 mean, 3 real mean)
    kind: str = "straight"

    @property
    def k0(self) -> float:
        return 2.0 * math.pi / self.wavelength

    @property
    def n_vox(self) -> int:
        return self.nx * self.ny * self.nz


def absorber_ramp(nx: int, la: int, both_ends: bool = True) -> np.ndarray:
    """eps'' per x-slab: quadratic ramp (s/la)^2, s = 1..la counted from the
    inner edge of each absorber, so the outermost slab reaches 1."""
    out = np.zeros(nx)
    if la <= 0:
        return out
    s = np.arange(1, la + 1, dtype=np.float64)
    ramp = (s / la) ** 2
    out[nx - la:] = ramp                  # right end: inner edge first
    if both_ends:
        out[:la] = np.maximum(out[:la], ramp[::-1])   # left end: outermost at x=0
    return out


def incident_field(nx: int, ny: int, nz: int, h: float, wavelength: float,
                   yc: float, zc: float, sigma: float = SIGMA_INC,
                   n_eff: float = N_EFF_INC) -> np.ndarray:
    """y-polarised travelling wave exp(-j k0 n_eff x) with a Gaussian y-z
    profile centred at (yc, zc), sampled at voxel centres."""
    k0 = 2.0 * math.pi / wavelength
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    z = (np.arange(nz) + 0.5) * h
    phase = np.exp(-1j * k0 * n_eff * x)                        # [nx]
    prof = np.exp(-((y[None, :] - yc) ** 2 + (z[:, None] - zc) ** 2) / (2.0 * sigma ** 2))  # [nz][ny]
    e = np.zeros((3, nz, ny, nx), dtype=np.complex128)
    e[1] = prof[:, :, None] * phase[None, None, :]
    return e


def _core_mask_field(nx, ny, nz, y_lo, y_hi, z_lo=0, z_hi=None):
    z_hi = nz if z_hi is None else z_hi
    m = np.zeros((nz, ny, nx), dtype=bool)
    m[z_lo:z_hi, y_lo:y_hi, :] = True
    return m


def _fill(mask: np.ndarray, eps_core: float, eps_bg: float, loss_x: np.ndarray) -> np.ndarray:
    eps = np.full(mask.shape, eps_bg, dtype=np.complex128)
    core = np.broadcast_to(eps_core - 1j * loss_x[None, None, :], mask.shape)
    eps[mask] = core[mask]
    return eps


def straight_guide(nx: int, ny: int, nz: int, h: float, wavelength: float,
                   core_ny: Optional[int] = None, core_nz: Optional[int] = None,
                   eps_core: float = EPS_SI, eps_bg: float = 1.0,
                   absorber: Optional[int] = None, name: str = "straight") -> Problem:
    """Straight waveguide along x with a centred rectangular core and
    quadratic absorbing ramps at both ends (absorber slabs default 10% of nx)."""
    core_ny = ny if core_ny is None else core_ny
    core_nz = nz if core_nz is None else core_nz
    la = int(0.1 * nx) if absorber is None else absorber
    y0 = (ny - core_ny) // 2
    z0 = (nz - core_nz) // 2
    mask = _core_mask_field(nx, ny, nz, y0, y0 + core_ny, z0, z0 + core_nz)
    eps = _fill(mask, eps_core, eps_bg, absorber_ramp(nx, la))
    yc = (y0 + core_ny / 2.0) * h
    zc = (z0 + core_nz / 2.0) * h
    e = incident_field(nx, ny, nz, h, wavelength, yc, zc)
    return Problem(name, nx, ny, nz, h, wavelength, eps_bg, eps, e, [], 3, "straight")


def bragg_grating(nx: int, ny: int, nz: int, h: float, wavelength: float,
                  wide: int = 16, narrow: int = 12, period: int = 32,
                  eps_core: float = EPS_SI, eps_bg: float = EPS_SIO2,
                  nboxes: int = 2, absorber: Optional[int] = None,
                  name: str = "bragg") -> Problem:
    """Bragg grating (Sec. 5.2): core width alternating wide/narrow with the
    given period (50% duty, wide first at x = 0), centred in y, filling z;
    partitioned into ``nboxes`` equal x-slices."""
    la = int(0.1 * nx) if absorber is None else absorber
    mask = np.zeros((nz, ny, nx), dtype=bool)
    x = np.arange(nx)
    is_wide = (x % period) < (period // 2)
    for w, sel in ((wide, is_wide), (narrow, ~is_wide)):
        y0 = (ny - w) // 2
        mask[:, y0:y0 + w, sel] = True
    eps = _fill(mask, eps_core, eps_bg, absorber_ramp(nx, la))
    yc = ny * h / 2.0
    zc = nz * h / 2.0
    e = incident_field(nx, ny, nz, h, wavelength, yc, zc)
    boxes: List[Box] = []
    if nboxes > 1:
        edges = [round(i * nx / nboxes) for i in range(nboxes + 1)]
        boxes = [(edges[i], 0, 0, edges[i + 1] - edges[i], ny, nz) for i in range(nboxes)]
    return Problem(name, nx, ny, nz, h, wavelength, eps_bg, eps, e, boxes, 3, "bragg")


def directional_coupler(nx: int, h: float, wavelength: float, ny: int = 48, nz: int = 8,
                        core_w: int = 16, gap: int = 8, margin: int = 4,
                        eps_core: float = EPS_SI, eps_bg: float = EPS_SIO2,
                        absorber: Optional[int] = None, name: str = "coupler") -> Problem:
    """Two parallel cores (Sec. 5.3.2 straight section): margin + core + gap +
    core + margin voxels in y, cores fill z, one box per core, Gaussian
    incidence centred on the first core only."""
    assert 2 * margin + 2 * core_w + gap == ny
    la = int(0.1 * nx) if absorber is None else absorber
    mask = np.zeros((nz, ny, nx), dtype=bool)
    c0 = margin
    c1 = margin + core_w + gap
    mask[:, c0:c0 + core_w, :] = True
    mask[:, c1:c1 + core_w, :] = True
    eps = _fill(mask, eps_core, eps_bg, absorber_ramp(nx, la))
    yc = (c0 + core_w / 2.0) * h
    zc = nz * h / 2.0
    e = incident_field(nx, ny, nz, h, wavelength, yc, zc)
    boxes = [(0, c0, 0, nx, core_w, nz), (0, c1, 0, nx, core_w, nz)]
    return Problem(name, nx, ny, nz, h, wavelength, eps_bg, eps, e, boxes, 3, "coupler")


def disk_resonator(radius: int, h: float = 0.02, wavelength: float = 1.545, nz: int = 11,
                   bus_w: int = 20, gap: int = 10, margin: int = 4, lead: int = 16,
                   eps_core: float = EPS_SI, eps_bg: float = EPS_SIO2,
                   absorber: Optional[int] = None, disk_levels: int = 2, name: str = "disk") -> Problem:
    """Disk resonator beside a bus waveguide (Sec. 5.3.1, Fig. "disk"): a
    straight bus core of ``bus_w`` voxels along x, a gap of ``gap`` voxels and
    a disk of ``radius`` voxels (voxel centres inside the circle are core),
    both filling the slab of nz voxels, in SiO2.  The bus runs ``lead`` voxels
    past the disk at each end and carries the absorbing ramps (default
    ``lead - 4`` slabs, applied to core voxels, so the disk stays lossless).
    Two boxes: the bus (1-level) and the disk's bounding square (2-level by
    default), with the modal homogenisation the paper uses for the disk."""
    d = 2 * radius
    nx = d + 2 * lead
    ny = margin + bus_w + gap + d + margin
    la = max(lead - 4, 0) if absorber is None else absorber
    mask = np.zeros((nz, ny, nx), dtype=bool)
    mask[:, margin:margin + bus_w, :] = True
    y_d0 = margin + bus_w + gap
    xc, yc = nx / 2.0, y_d0 + radius
    xs = np.arange(nx) + 0.5
    ys = np.arange(ny) + 0.5
    inside = (xs[None, :] - xc) ** 2 + (ys[:, None] - yc) ** 2 <= radius * radius
    mask[:, inside] = True
    eps = _fill(mask, eps_core, eps_bg, absorber_ramp(nx, la))
    e = incident_field(nx, ny, nz, h, wavelength, (margin + bus_w / 2.0) * h, nz * h / 2.0)
    boxes = [(0, margin, 0, nx, bus_w, nz), (lead, y_d0, 0, d, d, nz, disk_levels)]
    return Problem(name, nx, ny, nz, h, wavelength, eps_bg, eps, e, boxes, 1, "disk")


# ----------------------------------------------------------------------------
# The five workloads (small straight guide, long straight guide, Bragg grating,
# directional coupler at 16 wavelengths, serving stream).
# ----------------------------------------------------------------------------

def workload_small_straight() -> Problem:
    """64x8x4 silicon bar in air, h = 0.05 um, lambda = 1.55 um, 8-slab
    absorbers at both ends (6144 unknowns)."""
    return straight_guide(64, 8, 4, 0.05, 1.55, absorber=8, name="straight_64x8x4")


def workload_long_straight(nx: int = 1024) -> Problem:
    """1024x16x8 silicon wire in air, h = 0.025 um, 10% absorbers."""
    return straight_guide(nx, 16, 8, 0.025, 1.55, name=f"straight_{nx}x16x8")


def workload_bragg(nx: int = 4096) -> Problem:
    """4096x24x8 Bragg grating in SiO2, widths 16/12, period 32, 2 x-boxes."""
    return bragg_grating(nx, 24, 8, 0.025, 1.55, name=f"bragg_{nx}x24x8")


def coupler_wavelengths(n: int = 16) -> np.ndarray:
    return 1.50 + np.arange(n) * (0.10 / (n - 1) if n > 1 else 0.0)


def workload_coupler(nx: int = 2048, wavelength: float = 1.55) -> Problem:
    """2048x48x8 directional coupler in SiO2, one box per core."""
    return directional_coupler(nx, 0.025, wavelength, name=f"coupler_{nx}x48x8")


@dataclasses.dataclass
class Request:
    idx: int
    t_arrival: float         # seconds from stream start
    kind: str                # "straight" or "bragg"
    nx: int
    ny: int
    nz: int
    wavelength: float

    def problem(self) -> Problem:
        if self.kind == "straight":
            if self.ny == 16:
                return straight_guide(self.nx, 16, 8, 0.025, self.wavelength,
                                      name=f"req{self.idx}")
            return straight_guide(self.nx, self.ny, 8, 0.025, self.wavelength,
                                  core_ny=16, core_nz=8, name=f"req{self.idx}")
        wide = 16
        narrow = 12
        return bragg_grating(self.nx, self.ny, 8, 0.025, self.wavelength, wide=wide,
                             narrow=narrow, name=f"req{self.idx}")


def serving_stream(n: int = 256, rate_hz: float = 50.0, seed: int = 0,
                   nx_range: Tuple[int, int] = (256, 8192)) -> List[Request]:
    """Poisson arrivals (exponential gaps, mean 1/rate), kind 50/50, nx uniform
    integer in ``nx_range`` (inclusive), cross-section 16x8 or 24x8 (50/50),
    lambda uniform in [1.50, 1.60] um.  numpy PCG64 with the given seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    t = np.cumsum(gaps) - gaps[0]
    kinds = rng.integers(0, 2, size=n)
    nxs = rng.integers(nx_range[0], nx_range[1] + 1, size=n)
    nys = np.where(rng.integers(0, 2, size=n) == 0, 16, 24)
    lams = rng.uniform(1.50, 1.60, size=n)
    return [Request(i, float(t[i]), "straight" if kinds[i] == 0 else "bragg",
                    int(nxs[i]), int(nys[i]), 8, float(lams[i])) for i in range(n)]


def random_field(shape: Sequence[int], seed: int) -> np.ndarray:
    """Seeded complex test vector with N(0,1) real and imaginary parts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_permittivity(nz: int, ny: int, nx: int, seed: int, lo: float = 1.5,
                        hi: float = 12.11, loss: float = 0.5) -> np.ndarray:
    """Seeded inhomogeneous permittivity field for parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.uniform(lo, hi, size=(nz, ny, nx))
    im = rng.uniform(0.0, loss, size=(nz, ny, nx))
    return re - 1j * im
