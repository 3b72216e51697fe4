"""GPU parity: libvie (through its C ABI) against the CPU oracle on the same
seeded inputs.

Tolerances: the complex-FP64 matvec matches to 1e-12 relative (element-wise
against the largest entry, and in norm); the FP64 preconditioner apply to
1e-11 (LU + explicit inverse vs. LU solves, condition numbers of D_f ~ 1e2);
complex-FP32 paths in norm and element-wise to the single-precision rounding
of their arithmetic: 1e-6 for the matvec (unit roundoff 6e-8 times the ~15
rounding steps of an FFT chain and the product) and, for the preconditioner,
whose blocks are factored and inverted in complex FP32, 2e-6 where every
block is well conditioned (kappa(D_f) up to ~600: the measured error is
2e-7 to 7e-7), and bounds that follow the worst block elsewhere: the
elimination's FP32 rounding reaches the small pivots of a near-singular
block with relative error ~ u32 kappa.  The 24x8 box of m = 576
(kappa ~ 530, m three times larger) measures 5.3e-6 and takes 1.5e-5; the
16x8-voxel Si core in air has one x-frequency block with kappa ~ 1e5
(oracle blocks, numpy cond), measures 4.2e-5 and takes 1e-4.  Solutions to
1e-6 relative error.
"""
import dataclasses
import math

import numpy as np
import pytest

from gpu_common import cuda_or_fail, maxerr, relerr
from oracle import operator as op
from oracle import precond as pc
from oracle import solve as osolve
from paper_1903_07884_gb300 import inputs, vie
from paper_1903_07884_gb300.solver import Plan, make_opts, to_device

pytestmark = pytest.mark.gpu

K0 = 2 * math.pi / 1.55

# complex-FP32 preconditioner bounds of the cases with an ill-conditioned
# block (module docstring); 2e-6 for the others
C64_PRECOND_BOUND = {"wide_box_m576": 1.5e-5, "si_core_16x8": 1e-4}


def _oracle_matvec(nx, ny, nz, h, k0, eps_bg, eps, x):
    M = op.material(eps, eps_bg)
    k = op.background_k(k0, eps_bg)
    spec = op.generator_spectra(nx, ny, nz, h, k)
    return op.fft_matvec(x, M, spec)


@pytest.mark.parametrize("shape,eps_bg", [((1, 1, 1), 1.0), ((2, 1, 1), 1.0), ((3, 2, 2), 2.085), ((5, 3, 2), 1.0),
                                          ((7, 4, 3), 2.085), ((37, 5, 3), 1.0), ((64, 8, 4), 1.0),
                                          ((33, 12, 2), 2.085), ((6, 40, 40), 1.0), ((16, 100, 11), 2.085),
                                          ((1, 130, 17), 1.0)])
def test_matvec_fp64_matches_oracle(shape, eps_bg):
    """The last three shapes have Py Pz > 4096 (separate y and z line passes;
    (1, 130, 17) also a single x column, Py = 2 * 135 = 270)."""
    torch = cuda_or_fail()
    nx, ny, nz = shape
    h = 0.05
    eps = inputs.random_permittivity(nz, ny, nx, seed=nx * 7 + ny)
    x = inputs.random_field((3, nz, ny, nx), seed=3 + nx)
    ref = _oracle_matvec(nx, ny, nz, h, K0, eps_bg, eps, x)
    plan = Plan(nx, ny, nz, h, K0, eps_bg, make_opts(precision=vie.VIE_FP64, precond=vie.VIE_PREC_NONE))
    plan.set_permittivity(eps)
    y = plan.matvec(to_device(x), vie.VIE_FP64).cpu().numpy()
    plan.close()
    assert maxerr(y, ref) <= 1e-12
    assert relerr(y, ref) <= 1e-12
    if nx * ny * nz <= 120:   # brute force against the dense matrix too
        A = op.dense_matrix(nx, ny, nz, h, op.background_k(K0, eps_bg), op.material(eps, eps_bg))
        assert relerr(y, op.dense_matvec(A, x)) <= 1e-12


@pytest.mark.parametrize("shape", [(5, 3, 2), (64, 8, 4), (100, 12, 4), (1013, 3, 2), (2031, 3, 2), (2048, 4, 2),
                                   (16, 100, 11), (1, 128, 33)])
def test_matvec_mixed_matches_oracle(shape):
    """(1013, 3, 2) and (2031, 3, 2): ragged nx whose embeddings are L = 2048
    and 4096, the compile-time radix-16 x passes (zero padding and crop at a
    non-aligned edge); (2048, 4, 2) the full 4096 line.  The last two have
    Py Pz > 4096 (split y and z passes; with nx = 1 the y-lines of Py = 256
    are contiguous and take the warp-register FFT)."""
    cuda_or_fail()
    nx, ny, nz = shape
    eps = inputs.random_permittivity(nz, ny, nx, seed=11)
    x = inputs.random_field((3, nz, ny, nx), seed=12)
    ref = _oracle_matvec(nx, ny, nz, 0.025, K0, 1.0, eps, x)
    plan = Plan(nx, ny, nz, 0.025, K0, 1.0, make_opts(precision=vie.VIE_MIXED, precond=vie.VIE_PREC_NONE))
    plan.set_permittivity(eps)
    y = plan.matvec(to_device(x), vie.VIE_MIXED).cpu().numpy()
    plan.close()
    assert relerr(y, ref) <= 1e-6
    assert maxerr(y, ref) <= 1e-6


def test_matvec_long_guide_full_size():
    """1024x16x8 long straight guide: element-wise against the oracle."""
    cuda_or_fail()
    p = inputs.workload_long_straight()
    x = inputs.random_field((3, p.nz, p.ny, p.nx), seed=5)
    ref = _oracle_matvec(p.nx, p.ny, p.nz, p.h, p.k0, p.eps_bg, p.eps, x)
    plan = Plan.for_problem(p, precision=vie.VIE_FP64, precond=vie.VIE_PREC_NONE)
    plan.set_permittivity(p.eps)
    y64 = plan.matvec(to_device(x), vie.VIE_FP64).cpu().numpy()
    y32 = plan.matvec(to_device(x), vie.VIE_MIXED).cpu().numpy()
    plan.close()
    assert maxerr(y64, ref) <= 1e-12
    assert relerr(y32, ref) <= 1e-6
    assert maxerr(y32, ref) <= 1e-6


def test_matvec_bragg_full_size_sampled_rows():
    """4096x24x8 Bragg grating (unfused x pass): 24 sampled outputs against
    rows of A evaluated one by one from the generator definition."""
    cuda_or_fail()
    p = inputs.workload_bragg()
    x = inputs.random_field((3, p.nz, p.ny, p.nx), seed=6)
    plan = Plan.for_problem(p, precision=vie.VIE_FP64, precond=vie.VIE_PREC_NONE)
    plan.set_permittivity(p.eps)
    y = plan.matvec(to_device(x), vie.VIE_FP64).cpu().numpy().ravel()
    plan.close()
    M = op.material(p.eps, p.eps_bg)
    k = op.background_k(p.k0, p.eps_bg)
    rng = np.random.default_rng(0)
    n3 = 3 * p.n_vox
    rows = list(rng.integers(0, n3, size=20)) + [0, n3 - 1, p.n_vox, 2 * p.n_vox + 12345]
    xv = x.ravel()
    for r in rows:
        ref = op.matrix_row(int(r), p.nx, p.ny, p.nz, p.h, k, M) @ xv
        scale = max(abs(ref), np.abs(xv).max())
        assert abs(y[r] - ref) <= 1e-12 * scale * 10


def _precond_case(name):
    if name == "straight_full":
        p = inputs.straight_guide(40, 4, 2, 0.05, 1.55, absorber=4)
        return p, 0.0, 3
    if name == "small_reduced":
        return inputs.workload_small_straight(), 1e-3, 3
    if name == "prime_nx_bluestein":
        return inputs.straight_guide(37, 3, 2, 0.05, 1.55, absorber=3), 0.0, 2
    if name == "bragg_boxes_mode":
        return inputs.bragg_grating(96, 12, 4, 0.025, 1.55, wide=8, narrow=6, period=16), 1e-3, 1
    if name == "wide_box_m576":
        return inputs.straight_guide(24, 24, 8, 0.025, 1.55, core_ny=16, core_nz=8, absorber=2), 0.0, 3
    if name == "coupler_boxes":
        return inputs.directional_coupler(64, 0.025, 1.55, ny=24, nz=4, core_w=8, gap=4, margin=2), 0.0, 3
    # 2-level boxes (Sec. 4, the 2-level paragraph; Sec. 5.3.1)
    if name == "disk_blocked_2level":
        return inputs.disk_resonator(6, nz=3, bus_w=4, gap=2, margin=2, lead=6), 1e-3, 1
    if name == "two_level_prime_bluestein":
        p = inputs.straight_guide(13, 11, 2, 0.05, 1.55, core_ny=7, absorber=2)
        return dataclasses.replace(p, boxes=[(0, 0, 0, 13, 11, 2, 2)]), 0.0, 2
    if name == "two_level_even":
        p = inputs.straight_guide(32, 20, 4, 0.025, 1.55, core_ny=12, absorber=3)
        return dataclasses.replace(p, boxes=[(0, 0, 0, 32, 20, 4, 2)]), 0.0, 3
    if name == "two_level_nz11":     # m2 = 33: two rows per lane, the disk's slab thickness
        p = inputs.straight_guide(12, 10, 11, 0.02, 1.545, core_ny=6, absorber=2)
        return dataclasses.replace(p, boxes=[(0, 0, 0, 12, 10, 11, 2)]), 0.0, 1
    if name == "two_level_m96":
        p = inputs.straight_guide(8, 6, 32, 0.025, 1.55, core_ny=4, core_nz=24, absorber=1)
        return dataclasses.replace(p, boxes=[(0, 0, 0, 8, 6, 32, 2)]), 0.0, 2
    raise KeyError(name)


@pytest.mark.parametrize("name", ["straight_full", "small_reduced", "prime_nx_bluestein", "bragg_boxes_mode",
                                  "coupler_boxes", "wide_box_m576", "disk_blocked_2level",
                                  "two_level_prime_bluestein", "two_level_even", "two_level_nz11", "two_level_m96"])
def test_precond_fp64_matches_oracle(name):
    cuda_or_fail()
    p, tau, variant = _precond_case(name)
    M = op.material(p.eps, p.eps_bg)
    k = op.background_k(p.k0, p.eps_bg)
    P = pc.Preconditioner(p.nx, p.ny, p.nz, p.h, k, M, p.boxes, variant, tau)
    r = inputs.random_field((3, p.nz, p.ny, p.nx), seed=21)
    ref = P.apply(r)
    plan = Plan.for_problem(p, precision=vie.VIE_FP64, reduce_tol=tau, homog=variant)
    plan.set_permittivity(p.eps)
    plan.build()
    z = plan.precond(to_device(r), vie.VIE_FP64).cpu().numpy()
    plan.close()
    assert relerr(z, ref) <= 1e-11
    assert maxerr(z, ref) <= 1e-11


@pytest.mark.parametrize("name", ["straight_full", "small_reduced", "bragg_boxes_mode", "wide_box_m576",
                                  "disk_blocked_2level", "two_level_prime_bluestein", "two_level_even",
                                  "two_level_nz11", "two_level_m96"])
def test_precond_mixed_matches_oracle(name):
    cuda_or_fail()
    p, tau, variant = _precond_case(name)
    M = op.material(p.eps, p.eps_bg)
    k = op.background_k(p.k0, p.eps_bg)
    P = pc.Preconditioner(p.nx, p.ny, p.nz, p.h, k, M, p.boxes, variant, tau)
    r = inputs.random_field((3, p.nz, p.ny, p.nx), seed=22)
    ref = P.apply(r)
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED, reduce_tol=tau, homog=variant)
    plan.set_permittivity(p.eps)
    plan.build()
    z = plan.precond(to_device(r), vie.VIE_MIXED).cpu().numpy()
    plan.close()
    bound = C64_PRECOND_BOUND.get(name, 2e-6)
    assert relerr(z, ref) <= bound
    assert maxerr(z, ref) <= bound


def test_precond_mixed_tensor_core_block_product():
    """The discarded-frequency product with the representative block (Sec. 4.2)
    runs on the tensor cores in the mixed path (3xTF32 split, FP32-level
    accuracy): the 16x8 cross-section gives m = 384, and the discarded
    frequencies fill 128-frequency tiles with a ragged last one.  The bound is
    that of the 16x8 Si core's near-singular block (module docstring)."""
    cuda_or_fail()
    p = inputs.straight_guide(320, 16, 8, 0.025, 1.55)
    tau = 1e-3
    M = op.material(p.eps, p.eps_bg)
    k = op.background_k(p.k0, p.eps_bg)
    P = pc.Preconditioner(p.nx, p.ny, p.nz, p.h, k, M, p.boxes, 3, tau)
    assert 0 < len(P.boxes[0].kept) < p.nx // 2   # most frequencies take the representative block
    r = inputs.random_field((3, p.nz, p.ny, p.nx), seed=23)
    ref = P.apply(r)
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED, reduce_tol=tau, homog=3)
    plan.set_permittivity(p.eps)
    plan.build()
    vie.vie_profile_enable(1)
    vie.vie_profile_reset()
    z = plan.precond(to_device(r), vie.VIE_MIXED).cpu().numpy()
    table = vie.profile_table()
    vie.vie_profile_enable(0)
    plan.close()
    assert table.get("rep_gemm_tc", (0, 0.0))[0] == 1, table
    assert relerr(z, ref) <= C64_PRECOND_BOUND["si_core_16x8"]
    assert maxerr(z, ref) <= C64_PRECOND_BOUND["si_core_16x8"]


@pytest.mark.parametrize("nx", [256, 512, 1024])
def test_precond_mixed_power_of_two_lines(nx):
    """Power-of-two box lengths of 256..1024 take the warp-register x-transform
    in the mixed path (Sec. 4: the x-FFT of every line of the box, then the
    blocks, then the inverse x-FFT); ragged line counts per warp included
    (m = 3 * 3 * 2 = 18 lines)."""
    cuda_or_fail()
    p = inputs.straight_guide(nx, 3, 2, 0.05, 1.55)
    tau = 1e-3
    M = op.material(p.eps, p.eps_bg)
    k = op.background_k(p.k0, p.eps_bg)
    P = pc.Preconditioner(p.nx, p.ny, p.nz, p.h, k, M, p.boxes, 3, tau)
    r = inputs.random_field((3, p.nz, p.ny, p.nx), seed=24)
    ref = P.apply(r)
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED, reduce_tol=tau, homog=3)
    plan.set_permittivity(p.eps)
    plan.build()
    vie.vie_profile_enable(1)
    vie.vie_profile_reset()
    z = plan.precond(to_device(r), vie.VIE_MIXED).cpu().numpy()
    table = vie.profile_table()
    vie.vie_profile_enable(0)
    plan.close()
    assert table.get("fft_warp_c64", (0, 0.0))[0] == 2, table
    assert relerr(z, ref) <= 2e-6
    assert maxerr(z, ref) <= 2e-6


@pytest.mark.parametrize("precision,tol,bound", [(vie.VIE_FP64, 1e-11, 1e-7), (vie.VIE_MIXED, 1e-10, 1e-6)])
def test_solve_small_straight_matches_dense_lu(precision, tol, bound):
    """64x8x4 bar with absorbers: GPU solution against the oracle's direct LU."""
    cuda_or_fail()
    p = inputs.workload_small_straight()
    ref = osolve.dense_solve(p)
    plan = Plan.for_problem(p, precision=precision, tol=tol)
    plan.set_permittivity(p.eps)
    w, info = plan.solve(p.e_inc)
    plan.close()
    assert info["relres"] <= tol
    assert relerr(w.cpu().numpy(), ref) <= bound


def test_solve_tiny_cases_match_dense_lu():
    cuda_or_fail()
    for p in (inputs.straight_guide(1, 1, 1, 0.05, 1.55, absorber=0),
              inputs.straight_guide(9, 2, 1, 0.05, 1.55, absorber=2),
              inputs.directional_coupler(12, 0.025, 1.55, ny=12, nz=2, core_w=3, gap=2, margin=2)):
        ref = osolve.dense_solve(p)
        for prec in (vie.VIE_FP64, vie.VIE_MIXED):
            plan = Plan.for_problem(p, precision=prec, tol=1e-11, reduce_tol=0.0)
            plan.set_permittivity(p.eps)
            w, info = plan.solve(p.e_inc)
            plan.close()
            assert relerr(w.cpu().numpy(), ref) <= 1e-6, (p.name, prec, info)


@pytest.mark.parametrize("precision", [vie.VIE_FP64, vie.VIE_MIXED])
def test_solve_disk_blocked_two_level_matches_dense_lu(precision):
    """Disk beside a bus (Sec. 5.3.1) with the blocked-circulant preconditioner:
    1-level bus box, 2-level disk box, modal M~."""
    cuda_or_fail()
    p = inputs.disk_resonator(4, nz=2, bus_w=3, gap=2, margin=2, lead=5)
    ref = osolve.dense_solve(p)
    plan = Plan.for_problem(p, precision=precision, tol=1e-11, reduce_tol=0.0)
    plan.set_permittivity(p.eps)
    w, info = plan.solve(p.e_inc)
    plan.close()
    assert info["relres"] <= 1e-11
    assert info["precond_blocks"] == (p.nx // 2 + 1) + (4 + 1) * (4 + 1)
    assert relerr(w.cpu().numpy(), ref) <= 1e-6


def test_matvec_fp64_long_line_split():
    """x-embedding longer than one shared-memory line in FP64 (L = 13122 >
    12736): the split path against the oracle, element-wise."""
    cuda_or_fail()
    nx, ny, nz = 6500, 2, 2
    eps = inputs.random_permittivity(nz, ny, nx, seed=77)
    x = inputs.random_field((3, nz, ny, nx), seed=78)
    ref = _oracle_matvec(nx, ny, nz, 0.025, K0, 1.0, eps, x)
    plan = Plan(nx, ny, nz, 0.025, K0, 1.0, make_opts(precision=vie.VIE_FP64, precond=vie.VIE_PREC_NONE))
    plan.set_permittivity(eps)
    y = plan.matvec(to_device(x), vie.VIE_FP64).cpu().numpy()
    y32 = plan.matvec(to_device(x), vie.VIE_MIXED).cpu().numpy()
    plan.close()
    assert maxerr(y, ref) <= 1e-12
    assert relerr(y32, ref) <= 1e-6
    assert maxerr(y32, ref) <= 1e-6


def test_precond_fp64_long_prime_box_bluestein_split():
    """Prime box length 6379: Bluestein through a 16384-point transform,
    split once in FP64 (Chan eigenvalues and the FP64 apply)."""
    cuda_or_fail()
    p = inputs.straight_guide(6379, 1, 1, 0.025, 1.55, absorber=300)
    M = op.material(p.eps, p.eps_bg)
    k = op.background_k(p.k0, p.eps_bg)
    P = pc.Preconditioner(p.nx, p.ny, p.nz, p.h, k, M, None, 3, 0.0)
    r = inputs.random_field((3, p.nz, p.ny, p.nx), seed=31)
    ref = P.apply(r)
    plan = Plan.for_problem(p, precision=vie.VIE_FP64, reduce_tol=0.0)
    plan.set_permittivity(p.eps)
    plan.build()
    z = plan.precond(to_device(r), vie.VIE_FP64).cpu().numpy()
    plan.close()
    assert relerr(z, ref) <= 1e-11


def test_solve_rejects_non_finite_permittivity():
    cuda_or_fail()
    p = inputs.straight_guide(16, 4, 2, 0.05, 1.55, absorber=2)
    eps = p.eps.copy()
    eps[0, 1, 3] = np.nan
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED)
    plan.set_permittivity(eps)
    with pytest.raises(vie.VieError) as e:
        plan.solve(p.e_inc)
    assert e.value.status == vie.VIE_EINVAL
    plan.close()
