"""Degenerate systems of (I - M N) w = M e_inc (Sec. 2, Eq. discrete_form)
and arguments the library must refuse, through the C ABI.

* A zero incident field gives b = 0 and the solution w = 0 exactly, with no
  GMRES iteration, in both precisions.
* A grid that is all background (eps = eps_b everywhere) has M = 0, so
  b = M e_inc = 0 and w = 0 whatever the incident field.
* Empty grids and out-of-range options are rejected with VIE_EINVAL before
  anything is allocated.
"""
import numpy as np
import pytest

from gpu_common import cuda_or_fail
from paper_1903_07884_gb300 import inputs, vie
from paper_1903_07884_gb300.solver import Plan, make_opts

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [vie.VIE_MIXED, vie.VIE_FP64])
def test_zero_incident_field_gives_zero_solution(precision):
    cuda_or_fail()
    p = inputs.straight_guide(96, 8, 4, 0.05, 1.55, absorber=8)
    plan = Plan.for_problem(p, precision=precision, tol=1e-9)
    plan.set_permittivity(p.eps)
    w, info = plan.solve(np.zeros_like(p.e_inc))
    plan.close()
    assert info["iters_inner"] == 0 and info["relres"] == 0.0
    assert not np.any(w.cpu().numpy())


@pytest.mark.parametrize("precision", [vie.VIE_MIXED, vie.VIE_FP64])
def test_all_background_grid_gives_zero_solution(precision):
    cuda_or_fail()
    p = inputs.straight_guide(64, 8, 4, 0.05, 1.55, absorber=0)
    eps = np.full(p.eps.shape, p.eps_bg, dtype=np.complex128)
    plan = Plan.for_problem(p, precision=precision, tol=1e-9)
    plan.set_permittivity(eps)
    w, info = plan.solve(p.e_inc)
    plan.close()
    assert info["iters_inner"] == 0 and info["relres"] == 0.0
    assert not np.any(w.cpu().numpy())


@pytest.mark.parametrize("dims", [(0, 4, 2), (8, 0, 2), (8, 4, 0), (-1, 4, 2)])
def test_empty_grid_is_rejected(dims):
    cuda_or_fail()
    with pytest.raises(vie.VieError) as e:
        vie.vie_plan_create(*dims, 0.05, 2 * np.pi / 1.55, 1.0, make_opts())
    assert e.value.status == vie.VIE_EINVAL


@pytest.mark.parametrize("field,value", [("restart", 0), ("restart", 129), ("tol", 0.0), ("max_iter", 0),
                                         ("inner_restart", 129), ("precision", 7)])
def test_out_of_range_options_are_rejected(field, value):
    cuda_or_fail()
    opts = make_opts()
    setattr(opts, field, value)
    with pytest.raises(vie.VieError) as e:
        vie.vie_plan_create(16, 4, 2, 0.05, 2 * np.pi / 1.55, 1.0, opts)
    assert e.value.status == vie.VIE_EINVAL
