"""The autotuner (GPU): at plan creation it times the x-pass variants of the
matvec -- the compile-time radix-16 kernel where one exists and the generic
Stockham kernel with three radix orders -- and at preconditioner build the
kept-block product's CTAs per block; it reports candidates, times and the
choice, caches the choice per shape, and the tuned plan still matches the
oracle."""
import math
import re

import numpy as np
import pytest

from gpu_common import cuda_or_fail, maxerr, relerr
from oracle import operator as op
from paper_1903_07884_gb300 import inputs, vie
from paper_1903_07884_gb300.solver import Plan, make_opts, to_device

pytestmark = pytest.mark.gpu

K0 = 2 * math.pi / 1.55


def _xpass_lines(report, tag):
    return [ln for ln in report.splitlines() if ln.startswith(tag)]


@pytest.mark.parametrize("nx,ct", [(1024, True), (2031, True), (700, False)])
def test_x_pass_candidates_timed_and_chosen(nx, ct):
    cuda_or_fail()
    ny, nz = 4, 2
    eps = inputs.random_permittivity(nz, ny, nx, seed=nx)
    x = inputs.random_field((3, nz, ny, nx), seed=nx + 1)
    plan = Plan(nx, ny, nz, 0.025, K0, 1.0, make_opts(precision=vie.VIE_MIXED, precond=vie.VIE_PREC_NONE))
    rep = vie.vie_plan_tuning(plan.handle)
    lines = _xpass_lines(rep, "x_pass_c64")
    assert len(lines) == 1, rep
    names = re.findall(r" (radix16x16x\d+|stockham\[[0-9.]+\]) ([0-9.]+) ms;", lines[0])
    # distinct radix orders only (a palindromic order is timed once)
    assert len(names) == len(set(n for n, _ in names)) and len(names) >= (3 if ct else 2), lines[0]
    assert (names[0][0].startswith("radix16")) == ct
    assert all(float(t) > 0 for _, t in names)
    chosen = int(re.search(r"chosen (\d+)", lines[0]).group(1))
    assert (0 if ct else 1) <= chosen <= 3
    assert _xpass_lines(rep, "x_pass_c128"), rep
    # the choice is cached per shape: a second plan reports the same
    plan2 = Plan(nx, ny, nz, 0.025, K0, 1.0, make_opts(precision=vie.VIE_MIXED, precond=vie.VIE_PREC_NONE))
    assert _xpass_lines(vie.vie_plan_tuning(plan2.handle), "x_pass_c64") == lines
    plan2.close()
    # whatever variant was chosen, the matvec matches the oracle
    plan.set_permittivity(eps)
    y = plan.matvec(to_device(x), vie.VIE_MIXED).cpu().numpy()
    plan.close()
    M = op.material(eps, 1.0)
    ref = op.fft_matvec(x, M, op.generator_spectra(nx, ny, nz, 0.025, op.background_k(K0, 1.0)))
    assert relerr(y, ref) <= 1e-6 and maxerr(y, ref) <= 1e-6


def test_gemv_split_tuned_at_build():
    cuda_or_fail()
    p = inputs.straight_guide(320, 16, 8, 0.025, 1.55)
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED, reduce_tol=1e-3)
    plan.set_permittivity(p.eps)
    plan.build()
    rep = vie.vie_plan_tuning(plan.handle)
    lines = _xpass_lines(rep, "block_gemv_c64")
    plan.close()
    assert len(lines) == 1, rep
    splits = re.findall(r"split (\d) ([0-9.]+) ms;", lines[0])
    assert [int(s) for s, _ in splits] == [1, 2, 4, 8]
    assert int(re.search(r"chosen (\d+)", lines[0]).group(1)) in (1, 2, 4, 8)


def test_yz_columns_per_cta_tuned_for_register_cross_sections():
    """16x8-voxel cross-sections (Py = 32, Pz = 16) take the register yz
    passes; the tuner times 16, 8 and 4 x-columns per CTA and the matvec
    stays within the complex-FP32 bound of the oracle for the choice made."""
    cuda_or_fail()
    nx, ny, nz = 300, 16, 8
    plan = Plan(nx, ny, nz, 0.025, K0, 1.0, make_opts(precision=vie.VIE_MIXED, precond=vie.VIE_PREC_NONE))
    rep = vie.vie_plan_tuning(plan.handle)
    lines = _xpass_lines(rep, "yz_passes_c64")
    assert len(lines) == 1, rep
    cols = re.findall(r" (\d+) columns/CTA ([0-9.]+) ms;", lines[0])
    assert [int(c) for c, _ in cols] == [16, 8, 4]
    assert int(re.search(r"chosen (\d+)", lines[0]).group(1)) in (16, 8, 4)
    eps = inputs.random_permittivity(nz, ny, nx, seed=17)
    x = inputs.random_field((3, nz, ny, nx), seed=18)
    plan.set_permittivity(eps)
    y = plan.matvec(to_device(x), vie.VIE_MIXED).cpu().numpy()
    plan.close()
    ref = op.fft_matvec(x, op.material(eps, 1.0),
                        op.generator_spectra(nx, ny, nz, 0.025, op.background_k(K0, 1.0)))
    assert relerr(y, ref) <= 1e-6 and maxerr(y, ref) <= 1e-6


@pytest.mark.parametrize("nx,variants", [(1013, [0, 1, 2, 3]), (2031, [0, 1, 2, 3, 4]), (4073, [1, 2, 3, 4]),
                                         (700, [1, 2, 3]), (2200, [1, 2, 3, 5, 6, 7]), (4500, [6, 7]),
                                         (7803, [6, 7])])
def test_every_x_pass_variant_matches_oracle(nx, variants):
    """Every candidate the tuner may choose, forced in turn through the test
    hook: three-pass (L = 2048, 4096) and four-pass (L = 4096, 8192)
    compile-time kernels, the generic kernel with each radix order, and the
    kernel split over a cluster of 2, 4 or 8 CTAs (nx = 2200: L = 4480, where
    one CTA still holds the three lines; nx = 4500 and 7803: L = 9000 and
    15680, where it needs at least four), on ragged lengths (zero padding and
    crop at non-aligned edges)."""
    cuda_or_fail()
    ny, nz = 3, 2
    eps = inputs.random_permittivity(nz, ny, nx, seed=nx + 5)
    x = inputs.random_field((3, nz, ny, nx), seed=nx + 6)
    ref = op.fft_matvec(x, op.material(eps, 1.0),
                        op.generator_spectra(nx, ny, nz, 0.025, op.background_k(K0, 1.0)))
    plan = Plan(nx, ny, nz, 0.025, K0, 1.0, make_opts(precision=vie.VIE_MIXED, precond=vie.VIE_PREC_NONE))
    plan.set_permittivity(eps)
    xd = to_device(x)
    for v in variants:
        assert vie.vie_plan_set_tuning(plan.handle, "x_pass_c64", v) == vie.VIE_OK, (v, vie.last_error())
        y = plan.matvec(xd, vie.VIE_MIXED).cpu().numpy()
        assert relerr(y, ref) <= 1e-6 and maxerr(y, ref) <= 1e-6, (nx, v, relerr(y, ref))
    for v in (1, 2, 3):
        assert vie.vie_plan_set_tuning(plan.handle, "x_pass_c128", v) == vie.VIE_OK
        y = plan.matvec(xd, vie.VIE_FP64).cpu().numpy()
        assert maxerr(y, ref) <= 1e-12, (nx, v)
    # a variant the shape does not have is refused
    bad = {1013: 4, 700: 4, 4073: 0, 2031: 5, 2200: 4, 4500: 5, 7803: 1}[nx]
    assert vie.vie_plan_set_tuning(plan.handle, "x_pass_c64", bad) == vie.VIE_EINVAL
    plan.close()


@pytest.mark.parametrize("nx,q", [(2200, 2), (4500, 4)])
def test_cluster_split_x_pass_is_a_tuned_candidate(nx, q):
    """Embeddings whose three complex-FP32 lines exceed one CTA's shared
    memory are timed with the x pass split over a cluster of q CTAs (and, where
    one CTA still fits them, against the generic kernel)."""
    cuda_or_fail()
    plan = Plan(nx, 4, 2, 0.025, K0, 1.0, make_opts(precision=vie.VIE_MIXED, precond=vie.VIE_PREC_NONE))
    lines = _xpass_lines(vie.vie_plan_tuning(plan.handle), "x_pass_c64")
    plan.close()
    assert len(lines) == 1 and f" cluster{q}x" in lines[0], lines


def test_every_yz_and_gemv_choice_matches_oracle():
    cuda_or_fail()
    p = inputs.straight_guide(320, 16, 8, 0.025, 1.55)
    M = op.material(p.eps, p.eps_bg)
    k = op.background_k(p.k0, p.eps_bg)
    x = inputs.random_field((3, p.nz, p.ny, p.nx), seed=41)
    ref = op.fft_matvec(x, M, op.generator_spectra(p.nx, p.ny, p.nz, p.h, k))
    from oracle import precond as pc
    P = pc.Preconditioner(p.nx, p.ny, p.nz, p.h, k, M, p.boxes, 3, 1e-3)
    zref = P.apply(x)
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED, reduce_tol=1e-3)
    plan.set_permittivity(p.eps)
    plan.build()
    xd = to_device(x)
    for xg in (16, 8, 4):
        assert vie.vie_plan_set_tuning(plan.handle, "yz_passes_c64", xg) == vie.VIE_OK
        y = plan.matvec(xd, vie.VIE_MIXED).cpu().numpy()
        assert relerr(y, ref) <= 1e-6 and maxerr(y, ref) <= 1e-6, xg
    outs = []
    for sp in (1, 2, 4, 8):
        assert vie.vie_plan_set_tuning(plan.handle, "block_gemv", sp) == vie.VIE_OK
        z = plan.precond(xd, vie.VIE_MIXED).cpu().numpy()
        # the 16x8 Si core's near-singular block bounds the complex-FP32
        # preconditioner (test_gpu_parity module docstring)
        assert relerr(z, zref) <= 1e-4 and maxerr(z, zref) <= 1e-4, sp
        outs.append(z)
    for z in outs[1:]:   # the split does not change a single bit
        np.testing.assert_array_equal(z, outs[0])
    # the tensor-core product of the discarded frequencies: both N tiles run
    # the same K chunks in the same order for every output element
    rep = vie.vie_plan_tuning(plan.handle)
    lines = _xpass_lines(rep, "rep_gemm_tc")
    assert len(lines) == 1, rep
    assert [int(t) for t in re.findall(r"N tile (\d+) ", lines[0])] == [64, 32], lines[0]
    tiles = []
    for tn in (64, 32):
        assert vie.vie_plan_set_tuning(plan.handle, "rep_gemm_tc", tn) == vie.VIE_OK
        z = plan.precond(xd, vie.VIE_MIXED).cpu().numpy()
        assert relerr(z, zref) <= 1e-4 and maxerr(z, zref) <= 1e-4, tn
        tiles.append(z)
    np.testing.assert_array_equal(tiles[1], tiles[0])
    assert vie.vie_plan_set_tuning(plan.handle, "rep_gemm_tc", 48) == vie.VIE_EINVAL
    plan.close()


def test_generic_yz_columns_tuned_and_every_choice_matches_oracle():
    """A 24x4-voxel cross-section (Py = 48, Pz = 8) has no register yz kernel:
    the tuner times 1..16 x-columns per CTA of the generic shared-memory
    passes; every choice gives bitwise the same matvec, within 1e-6 of the
    oracle."""
    cuda_or_fail()
    nx, ny, nz = 96, 24, 4
    plan = Plan(nx, ny, nz, 0.025, K0, 2.085, make_opts(precision=vie.VIE_MIXED, precond=vie.VIE_PREC_NONE))
    rep = vie.vie_plan_tuning(plan.handle)
    lines = _xpass_lines(rep, "yz_generic_c64")
    assert len(lines) == 1, rep
    cols = [int(c) for c, _ in re.findall(r" (\d+) columns/CTA ([0-9.]+) ms;", lines[0])]
    assert cols[:3] == [1, 2, 4], lines[0]
    eps = inputs.random_permittivity(nz, ny, nx, seed=19)
    x = inputs.random_field((3, nz, ny, nx), seed=20)
    plan.set_permittivity(eps)
    ref = op.fft_matvec(x, op.material(eps, 2.085),
                        op.generator_spectra(nx, ny, nz, 0.025, op.background_k(K0, 2.085)))
    xd = to_device(x)
    outs = []
    for xg in cols:
        assert vie.vie_plan_set_tuning(plan.handle, "yz_generic_c64", xg) == vie.VIE_OK
        y = plan.matvec(xd, vie.VIE_MIXED).cpu().numpy()
        assert relerr(y, ref) <= 1e-6 and maxerr(y, ref) <= 1e-6, xg
        outs.append(y)
    for y in outs[1:]:
        np.testing.assert_array_equal(y, outs[0])
    plan.close()
