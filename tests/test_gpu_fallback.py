"""FP64 fallback of the mixed-precision solve.

A straight wire of 1676x16x8 voxels at lambda = 1.52985 um (a length that is
not 2-3-5-7 smooth, so the x-blocks of the circulant preconditioner,
Sec. 5.1, are built on Bluestein transforms) is a system on which the
complex-FP32 inner GMRES cycles of the GMRES-IR solve stop gaining: its FP64
residual stalls near 0.6 ||b|| with the default 100-step inner cycles, while
FP64 GMRES(50) converges in about 425 iterations.  The mixed solve must then
go on in FP64 from its iterate and reach the tolerance, with the same
solution as the FP64 solve, and do so bitwise alike alone and in a lockstep
batch.  The benchmark workloads must not need the fallback.
"""
import numpy as np
import pytest

from gpu_common import cuda_or_fail, relerr
from paper_1903_07884_gb300 import inputs, vie
from paper_1903_07884_gb300.solver import Plan, make_opts, to_device

pytestmark = pytest.mark.gpu

LAMBDA = 1.5298507272502448


def _stalling_wire():
    return inputs.straight_guide(1676, 16, 8, 0.025, LAMBDA, name="straight_1676x16x8")


def test_stalled_refinement_falls_back_to_fp64_and_converges():
    cuda_or_fail()
    p = _stalling_wire()
    plan = Plan.for_problem(p, precision=vie.VIE_FP64, tol=1e-9)
    plan.set_permittivity(p.eps)
    w64, info64 = plan.solve(p.e_inc)
    plan.close()
    assert info64["relres"] <= 1e-9
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED, tol=1e-9)
    plan.set_permittivity(p.eps)
    w, info = plan.solve(p.e_inc)
    plan.close()
    assert info["relres"] <= 1e-9, info
    assert info["iters_fp64_fallback"] > 0, info
    assert info["iters_fp64_fallback"] <= info["iters_inner"]
    assert relerr(w.cpu().numpy(), w64.cpu().numpy()) <= 1e-6, info


def test_fallback_inside_a_batch_is_bitwise_the_solo_result():
    torch = cuda_or_fail()
    probs = [_stalling_wire(), inputs.straight_guide(131, 8, 4, 0.025, 1.52, core_ny=6, core_nz=4, name="u1")]
    alone, infos_alone = [], []
    for p in probs:
        plan = Plan.for_problem(p, tol=1e-9)
        plan.set_permittivity(p.eps)
        w, info = plan.solve(p.e_inc)
        alone.append(w.cpu().numpy())
        infos_alone.append(info)
        plan.close()
    assert infos_alone[0]["iters_fp64_fallback"] > 0
    assert infos_alone[1]["iters_fp64_fallback"] == 0
    plans, es, ws = [], [], []
    for p in probs:
        pl = Plan(p.nx, p.ny, p.nz, p.h, p.k0, p.eps_bg,
                  make_opts(tol=1e-9, boxes=p.boxes or None, homog=p.homog))
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
        assert infos[i].iters_fp64_fallback == infos_alone[i]["iters_fp64_fallback"]
        np.testing.assert_array_equal(ws[i].cpu().numpy(), alone[i])
    for pl in plans:
        pl.close()


@pytest.mark.parametrize("make", [inputs.workload_long_straight, inputs.workload_bragg])
def test_benchmark_workloads_need_no_fallback(make):
    cuda_or_fail()
    p = make()
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED, tol=1e-9)
    plan.set_permittivity(p.eps)
    w, info = plan.solve(p.e_inc)
    plan.close()
    assert info["relres"] <= 1e-9
    assert info["iters_fp64_fallback"] == 0, info
