"""GPU solves against the CPU oracle's solutions (Sec. 2, Eq. discrete_form).

* The 1024x16x8 long straight wire at the benchmark's settings (tolerance
  1e-9 on the FP64 residual, GMRES(50), real-mean homogenised 1-level
  preconditioner with reduction tau = 1e-3), in mixed precision and in FP64,
  against the oracle solution stored by tests/golden/make_oracle_solutions.py
  (oracle GMRES to 1e-12).  The bound is the target of the method: relative
  error <= 1e-6 in norm, and element-wise against the largest entry.
* Unpreconditioned GMRES (Sec. 3, the baseline of the iteration-vs-length
  study): the identity-preconditioned GPU solve of the 64x8x4 bar against the
  oracle's dense LU, and its iteration count against the oracle's own
  unpreconditioned GMRES(50) on the same system.
"""
import json
import os

import numpy as np
import pytest

from gpu_common import cuda_or_fail, maxerr, relerr
from oracle import solve as osolve
from paper_1903_07884_gb300 import inputs, vie
from paper_1903_07884_gb300.solver import Plan, make_opts, to_device

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _stored(name):
    meta = json.load(open(os.path.join(GOLDEN, "oracle_solutions.json")))[name]
    return np.load(os.path.join(GOLDEN, meta["file"])), meta


@pytest.mark.parametrize("precision", [vie.VIE_MIXED, vie.VIE_FP64])
def test_long_straight_solution_matches_oracle(precision):
    cuda_or_fail()
    ref, meta = _stored("long_straight_1024x16x8")
    assert meta["relres"] <= 1e-12
    p = inputs.workload_long_straight()
    plan = Plan.for_problem(p, precision=precision, tol=1e-9)
    plan.set_permittivity(p.eps)
    w, info = plan.solve(p.e_inc)
    plan.close()
    w = w.cpu().numpy()
    assert info["relres"] <= 1e-9
    assert relerr(w, ref) <= 1e-6, info
    assert maxerr(w, ref) <= 1e-6, info


def test_small_straight_solution_matches_stored_dense_lu():
    """64x8x4 bar against the stored dense-LU solution, both precisions."""
    cuda_or_fail()
    ref, meta = _stored("small_straight_64x8x4")
    p = inputs.workload_small_straight()
    for precision in (vie.VIE_MIXED, vie.VIE_FP64):
        plan = Plan.for_problem(p, precision=precision, tol=1e-9)
        plan.set_permittivity(p.eps)
        w, info = plan.solve(p.e_inc)
        plan.close()
        w = w.cpu().numpy()
        assert relerr(w, ref) <= 1e-6, (precision, info)
        assert maxerr(w, ref) <= 1e-6, (precision, info)


def test_unpreconditioned_solve_matches_oracle():
    cuda_or_fail()
    p = inputs.workload_small_straight()
    ref = osolve.dense_solve(p)
    orc = osolve.iterative_solve(p, tol=1e-10, use_precond=False, max_iter=20000)
    assert orc.relres <= 1e-10
    for precision in (vie.VIE_FP64, vie.VIE_MIXED):
        plan = Plan.for_problem(p, precision=precision, tol=1e-10, precond=vie.VIE_PREC_NONE, max_iter=20000)
        plan.set_permittivity(p.eps)
        w, info = plan.solve(p.e_inc, allow_noconv=True)
        plan.close()
        w = w.cpu().numpy()
        assert info["relres"] <= 1e-10, (precision, info)
        assert relerr(w, ref) <= 1e-6, (precision, info)
        if precision == vie.VIE_FP64:
            # same Krylov method in FP64 (CGS2 on the GPU, MGS in the oracle)
            assert abs(info["iters_inner"] - orc.iters) <= 0.05 * orc.iters + 5, (info, orc.iters)


@pytest.mark.parametrize("precision", [vie.VIE_MIXED, vie.VIE_FP64])
def test_bragg_full_size_solution_matches_oracle_sample(precision):
    """4096x24x8 Bragg grating (2.36 M unknowns, two x-boxes, real-mean
    homogenised blocks, tau = 1e-3): the GPU solution at the benchmark
    tolerance against a seeded sample of 4091 entries of the oracle's
    solution (oracle GMRES to 1e-12, stored by make_oracle_solutions.py), in
    norm and element-wise against the sample's largest entry."""
    cuda_or_fail()
    meta = json.load(open(os.path.join(GOLDEN, "oracle_solutions.json")))["bragg_4096x24x8_2boxes"]
    assert meta["relres"] <= 1e-12
    d = np.load(os.path.join(GOLDEN, meta["file"]))
    idx, ref = d["idx"], d["w"]
    p = inputs.workload_bragg()
    plan = Plan.for_problem(p, precision=precision, tol=1e-9)
    plan.set_permittivity(p.eps)
    w, info = plan.solve(p.e_inc)
    plan.close()
    ws = w.cpu().numpy().ravel()[idx]
    assert info["relres"] <= 1e-9
    assert relerr(ws, ref) <= 1e-6, info
    assert maxerr(ws, ref) <= 1e-6, info


@pytest.mark.parametrize("precision", [vie.VIE_MIXED, vie.VIE_FP64])
def test_coupler_full_size_solution_matches_oracle_sample(precision):
    """2048x48x8 directional coupler (two 16-wide cores, two x-boxes) at the
    first wavelength of its sweep, 1.50 um: the GPU solution at the benchmark
    tolerance against a seeded sample of the oracle's solution (oracle GMRES
    to 1e-12, stored by make_oracle_solutions.py)."""
    cuda_or_fail()
    name = "coupler_2048x48x8_2boxes_lambda1.50"
    meta = json.load(open(os.path.join(GOLDEN, "oracle_solutions.json")))[name]
    assert meta["relres"] <= 1e-12
    d = np.load(os.path.join(GOLDEN, meta["file"]))
    idx, ref = d["idx"], d["w"]
    p = inputs.workload_coupler(wavelength=1.50)
    plan = Plan.for_problem(p, precision=precision, tol=1e-9)
    plan.set_permittivity(p.eps)
    w, info = plan.solve(p.e_inc)
    plan.close()
    ws = w.cpu().numpy().ravel()[idx]
    assert info["relres"] <= 1e-9
    assert relerr(ws, ref) <= 1e-6, info
    assert maxerr(ws, ref) <= 1e-6, info


def test_coupler_wavelength_batch_matches_solo_solves_and_oracle_sample():
    """Two wavelengths of the 2048x48x8 coupler sweep (1.50 and 1.55 um) in
    one lockstep batch (vie_solve_batch): each result bitwise equal to the
    same plan solved alone, and the 1.50 um result within 1e-6 of the
    oracle's stored solution sample."""
    torch = cuda_or_fail()
    name = "coupler_2048x48x8_2boxes_lambda1.50"
    meta = json.load(open(os.path.join(GOLDEN, "oracle_solutions.json")))[name]
    d = np.load(os.path.join(GOLDEN, meta["file"]))
    idx, ref = d["idx"], d["w"]
    probs = [inputs.workload_coupler(wavelength=lam) for lam in (1.50, 1.55)]
    alone = []
    for p in probs:
        plan = Plan.for_problem(p, tol=1e-9)
        plan.set_permittivity(p.eps)
        w, info = plan.solve(p.e_inc)
        assert info["relres"] <= 1e-9
        alone.append(w.cpu().numpy())
        plan.close()
    plans, es, ws = [], [], []
    for p in probs:
        pl = Plan(p.nx, p.ny, p.nz, p.h, p.k0, p.eps_bg, make_opts(tol=1e-9, boxes=p.boxes or None, homog=p.homog))
        pl.set_permittivity(p.eps)
        e = to_device(p.e_inc)
        es.append(e)
        ws.append(torch.empty_like(e))
        plans.append(pl)
    torch.cuda.synchronize()
    infos = vie.vie_solve_batch([pl.handle for pl in plans], [e.data_ptr() for e in es], [w.data_ptr() for w in ws])
    torch.cuda.synchronize()
    for i in range(len(probs)):
        assert infos[i].relres <= 1e-9
        np.testing.assert_array_equal(ws[i].cpu().numpy(), alone[i])
    wb = ws[0].cpu().numpy().ravel()[idx]
    assert relerr(wb, ref) <= 1e-6
    assert maxerr(wb, ref) <= 1e-6
    for pl in plans:
        pl.close()
