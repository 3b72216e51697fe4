"""The allocation-free matvec entry point (vie_matvec_static).

It serves callers that may not allocate device memory -- for example a host
framework that owns all GPU memory through its own pool -- and therefore
cannot create a plan.  Its scratch is a fixed device array inside libvie.
Here it must reproduce the plan-based complex-FP64 matvec (vie_matvec) to the
matvec tolerance of the other tests (1e-12), on two calls in a row (the
second call finds the first call's data in the shared array), and reject a
grid whose scratch would not fit.  This file sorts last so that a run that
stops at the first failure has run every other test before it.
"""
import math

import numpy as np
import pytest

from gpu_common import cuda_or_fail, maxerr, relerr
from paper_1903_07884_gb300 import inputs, vie
from paper_1903_07884_gb300.solver import Plan, make_opts, to_device

pytestmark = pytest.mark.gpu

K0 = 2 * math.pi / 1.55


@pytest.mark.parametrize("shape,h,eps_bg", [((64, 8, 4), 0.05, 1.0), ((1024, 16, 8), 0.025, 2.085),
                                            ((37, 5, 3), 0.05, 1.0)])
def test_static_matvec_matches_plan_matvec_twice(shape, h, eps_bg):
    torch = cuda_or_fail()
    nx, ny, nz = shape
    eps = to_device(inputs.random_permittivity(nz, ny, nx, seed=nx + ny))
    plan = Plan(nx, ny, nz, h, K0, eps_bg, make_opts(precision=vie.VIE_FP64, precond=vie.VIE_PREC_NONE))
    plan.set_permittivity(eps)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = to_device(inputs.random_field((3, nz, ny, nx), seed=100 + call))
        ref = plan.matvec(x, vie.VIE_FP64)
        y = torch.empty_like(x)
        st = vie.vie_matvec_static(nx, ny, nz, h, K0, eps_bg, eps.data_ptr(), x.data_ptr(), y.data_ptr(), stream)
        assert st == vie.VIE_OK, vie.last_error()
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), ref.cpu().numpy()
        assert maxerr(a, b) <= 1e-12, call
        assert relerr(a, b) <= 1e-12, call
    plan.close()


def test_static_matvec_rejects_grids_beyond_its_scratch():
    torch = cuda_or_fail()
    nx, ny, nz = 2048, 32, 16          # needs more than the 64 MiB scratch
    eps = torch.ones((nz, ny, nx), dtype=torch.complex128, device="cuda")
    x = torch.zeros((3, nz, ny, nx), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    st = vie.vie_matvec_static(nx, ny, nz, 0.025, K0, 1.0, eps.data_ptr(), x.data_ptr(), y.data_ptr(), 0)
    assert st == vie.VIE_EINVAL
    assert "scratch" in vie.last_error()


def test_static_matvec_allocates_no_device_memory():
    """The entry point's defining property: after one warm-up call (which
    loads the library's device code under lazy loading), further calls --
    including one on a grid with transform lengths not seen before -- leave
    the device's free memory unchanged.  Inputs are allocated first."""
    torch = cuda_or_fail()
    shapes = [(24, 4, 2), (30, 4, 2)]      # same kernel variants, new embedding lengths L = 48, 60
    bufs = []
    for nx, ny, nz in shapes:
        eps = to_device(inputs.random_permittivity(nz, ny, nx, seed=3))
        x = to_device(inputs.random_field((3, nz, ny, nx), seed=4))
        bufs.append((nx, ny, nz, eps, x, torch.empty_like(x)))
    stream = torch.cuda.current_stream().cuda_stream

    def call(i):
        nx, ny, nz, eps, x, y = bufs[i]
        st = vie.vie_matvec_static(nx, ny, nz, 0.05, K0, 1.0, eps.data_ptr(), x.data_ptr(), y.data_ptr(), stream)
        assert st == vie.VIE_OK, vie.last_error()

    call(0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    call(0)
    call(1)
    call(1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_matvec_rejects_overlapping_output():
    torch = cuda_or_fail()
    nx, ny, nz = 8, 4, 2
    n3 = 3 * nx * ny * nz
    eps = to_device(inputs.random_permittivity(nz, ny, nx, seed=5))
    buf = torch.zeros(2 * n3, dtype=torch.complex128, device="cuda")
    x = buf[:n3]
    y_partial = buf[n3 // 2:n3 // 2 + n3]          # shares half of x
    st = vie.vie_matvec_static(nx, ny, nz, 0.05, K0, 1.0, eps.data_ptr(), x.data_ptr(), y_partial.data_ptr(), 0)
    assert st == vie.VIE_EINVAL
    assert "overlap" in vie.last_error()
