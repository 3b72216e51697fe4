"""PyTorch-facing convenience around the libvie C ABI.

PyTorch provides device memory (complex128 tensors, whose layout is double2)
and the stream; every computation runs in libvie's kernels.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import vie


def _require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libvie needs a CUDA device")
    return torch


def to_device(a: np.ndarray, device="cuda"):
    torch = _require_cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to(device)


def make_opts(precision=vie.VIE_MIXED, precond=vie.VIE_PREC_CIRCULANT, homog=vie.VIE_HOM_REALMEAN,
              reduce_tol=1e-3, tol=1e-9, restart=50, max_iter=5000, inner_tol=1e-6, max_refine=1000,
              boxes: Optional[Sequence] = None, inner_restart=0) -> vie.vie_opts:
    return vie.default_opts(precision=precision, precond=precond, homog=homog, reduce_tol=reduce_tol, tol=tol,
                            restart=restart, max_iter=max_iter, inner_tol=inner_tol, max_refine=max_refine,
                            boxes=list(boxes) if boxes else None, inner_restart=inner_restart)


class Plan:
    """One grid + physics; owns a libvie plan on the current torch stream."""

    def __init__(self, nx, ny, nz, h, k0, eps_bg, opts: Optional[vie.vie_opts] = None, stream=None):
        torch = _require_cuda()
        self.shape = (3, nz, ny, nx)
        self.N = nx * ny * nz
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.opts = opts
        self.handle = vie.vie_plan_create(nx, ny, nz, h, k0, eps_bg, opts, self.stream.cuda_stream)
        self._eps = None

    @classmethod
    def for_problem(cls, p, **kw):
        boxes = kw.pop("boxes", p.boxes if p.boxes else None)
        homog = kw.pop("homog", p.homog)
        opts = make_opts(boxes=boxes, homog=homog, **kw)
        return cls(p.nx, p.ny, p.nz, p.h, p.k0, p.eps_bg, opts)

    def set_permittivity(self, eps) -> None:
        if isinstance(eps, np.ndarray):
            eps = to_device(eps)
        self._eps = eps.contiguous()
        vie.vie_set_permittivity(self.handle, self._eps.data_ptr())

    def build(self) -> None:
        vie.vie_build_preconditioner(self.handle)

    def matvec(self, x, precision=vie.VIE_FP64):
        torch = _require_cuda()
        x = x.contiguous()
        y = torch.empty_like(x)
        vie.vie_matvec(self.handle, x.data_ptr(), y.data_ptr(), precision)
        return y

    def precond(self, r, precision=vie.VIE_FP64):
        torch = _require_cuda()
        r = r.contiguous()
        z = torch.empty_like(r)
        vie.vie_precond_apply(self.handle, r.data_ptr(), z.data_ptr(), precision)
        return z

    def solve(self, e_inc, allow_noconv=False):
        torch = _require_cuda()
        if isinstance(e_inc, np.ndarray):
            e_inc = to_device(e_inc)
        e_inc = e_inc.contiguous()
        w = torch.empty_like(e_inc)
        info = vie.vie_solve(self.handle, e_inc.data_ptr(), w.data_ptr(), allow_noconv)
        return w, info.as_dict()

    def close(self) -> None:
        if self.handle is not None:
            vie.vie_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
