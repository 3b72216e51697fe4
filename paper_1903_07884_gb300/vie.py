"""Thin ctypes binding of libvie (include/vie.h): argument marshalling only.

Every entry point keeps its C name.  Device buffers are passed as raw
pointers (for example ``tensor.data_ptr()`` of a ``torch.complex128`` CUDA
tensor, whose layout equals double2); streams as ``cudaStream_t`` integers.
There is no fallback: if libvie.so is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvie.so")

VIE_OK, VIE_ENOCONV, VIE_PENDING = 0, 1, 2
VIE_EINVAL, VIE_ENOMEM, VIE_ECUDA, VIE_ETIMEOUT, VIE_EREJECTED, VIE_ESTATE = -1, -2, -3, -4, -5, -6
VIE_FP64, VIE_MIXED = 0, 1
VIE_HOM_MODE, VIE_HOM_MEAN, VIE_HOM_REALMEAN = 1, 2, 3
VIE_PREC_NONE, VIE_PREC_CIRCULANT = 0, 1


class vie_box(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_int), ("y0", ctypes.c_int), ("z0", ctypes.c_int),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("levels", ctypes.c_int)]


class vie_opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("precision", ctypes.c_int), ("precond", ctypes.c_int), ("homog", ctypes.c_int),
                ("reduce_tol", ctypes.c_double), ("boxes", ctypes.POINTER(vie_box)),
                ("nboxes", ctypes.c_int), ("inner_restart", ctypes.c_int)]


class vie_info(ctypes.Structure):
    _fields_ = [("iters_inner", ctypes.c_int), ("iters_outer", ctypes.c_int),
                ("relres", ctypes.c_double), ("precond_bytes", ctypes.c_size_t),
                ("kept_fraction", ctypes.c_double), ("t_setup_ms", ctypes.c_float),
                ("t_solve_ms", ctypes.c_float), ("precond_blocks", ctypes.c_longlong),
                ("precond_discarded", ctypes.c_longlong), ("reorth_passes", ctypes.c_int),
                ("iters_fp64_fallback", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class VieError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libvie status {status}: {msg}")
        self.status = status


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "vie_default_opts": (None, [ctypes.POINTER(vie_opts)]),
    "vie_plan_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.POINTER(vie_opts),
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "vie_plan_destroy": (None, [ctypes.c_void_p]),
    "vie_set_permittivity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "vie_build_preconditioner": (ctypes.c_int, [ctypes.c_void_p]),
    "vie_matvec": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "vie_precond_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "vie_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(vie_info)]),
    "vie_solve_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.POINTER(vie_info)]),
    "vie_solve_batch": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(vie_info)]),
    "vie_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "vie_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.POINTER(vie_opts), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "vie_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(vie_info)]),
    "vie_server_drain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "vie_server_reserved_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "vie_estimate_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vie_opts)]),
    "vie_server_destroy": (None, [ctypes.c_void_p]),
    "vie_matvec_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "vie_plan_tuning": (ctypes.c_char_p, [ctypes.c_void_p]),
    "vie_plan_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int]),
    "vie_last_error": (ctypes.c_char_p, []),
    "vie_kernel_launches": (ctypes.c_int64, []),
    "vie_profile_enable": (None, [ctypes.c_int]),
    "vie_profile_reset": (None, []),
    "vie_profile_query": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_double)]),
    "vie_profile_kernels": (ctypes.c_int, [ctypes.POINTER(ctypes.c_char_p), ctypes.c_int]),
}


def lib():
    """Load libvie.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libvie.so not built ({LIB_PATH}); run paper_1903_07884_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> Sequence[str]:
    return list(_SIGS)


def last_error() -> str:
    return lib().vie_last_error().decode()


def check(status: int, allow: Sequence[int] = (VIE_OK,)) -> int:
    if status in allow:
        return status
    if status < 0 or status not in allow:
        raise VieError(status, last_error())
    return status


def default_opts(**kw) -> vie_opts:
    o = vie_opts()
    lib().vie_default_opts(ctypes.byref(o))
    boxes = kw.pop("boxes", None)
    for k, v in kw.items():
        setattr(o, k, v)
    if boxes:
        arr = (vie_box * len(boxes))(*[vie_box(*b) for b in boxes])
        o.boxes = ctypes.cast(arr, ctypes.POINTER(vie_box))
        o.nboxes = len(boxes)
        o._keep = arr           # keep the array alive with the struct
    return o


# --- same-name wrappers (status codes returned unchanged) -------------------

def vie_plan_create(nx, ny, nz, h, k0, eps_bg, opts: Optional[vie_opts], stream: int = 0) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    check(lib().vie_plan_create(nx, ny, nz, h, k0, eps_bg, ctypes.byref(opts) if opts is not None else None,
                                ctypes.c_void_p(stream), ctypes.byref(out)))
    return out


def vie_plan_destroy(plan) -> None:
    lib().vie_plan_destroy(plan)


def vie_set_permittivity(plan, eps_ptr: int) -> int:
    return check(lib().vie_set_permittivity(plan, ctypes.c_void_p(eps_ptr)))


def vie_build_preconditioner(plan) -> int:
    return check(lib().vie_build_preconditioner(plan))


def vie_matvec(plan, x_ptr: int, y_ptr: int, precision: int) -> int:
    return check(lib().vie_matvec(plan, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), precision))


def vie_precond_apply(plan, r_ptr: int, z_ptr: int, precision: int) -> int:
    return check(lib().vie_precond_apply(plan, ctypes.c_void_p(r_ptr), ctypes.c_void_p(z_ptr), precision))


def vie_solve(plan, e_ptr: int, w_ptr: int, allow_noconv: bool = False) -> vie_info:
    info = vie_info()
    allow = (VIE_OK, VIE_ENOCONV) if allow_noconv else (VIE_OK,)
    check(lib().vie_solve(plan, ctypes.c_void_p(e_ptr), ctypes.c_void_p(w_ptr), ctypes.byref(info)), allow)
    return info


def vie_solve_host(plan, eps_host: int, e_host: int, w_host: int, allow_noconv: bool = False) -> vie_info:
    info = vie_info()
    allow = (VIE_OK, VIE_ENOCONV) if allow_noconv else (VIE_OK,)
    check(lib().vie_solve_host(plan, ctypes.c_void_p(eps_host), ctypes.c_void_p(e_host),
                               ctypes.c_void_p(w_host), ctypes.byref(info)), allow)
    return info


def vie_solve_batch(plans, e_ptrs, w_ptrs, allow_noconv: bool = False):
    n = len(plans)
    P = (ctypes.c_void_p * n)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    E = (ctypes.c_void_p * n)(*e_ptrs)
    W = (ctypes.c_void_p * n)(*w_ptrs)
    infos = (vie_info * n)()
    allow = (VIE_OK, VIE_ENOCONV) if allow_noconv else (VIE_OK,)
    check(lib().vie_solve_batch(P, n, E, W, infos), allow)
    return list(infos)


def vie_server_create(budget_bytes: int, max_inflight: int):
    out = ctypes.c_void_p()
    check(lib().vie_server_create(budget_bytes, max_inflight, ctypes.byref(out)))
    return out


def vie_server_submit(srv, nx, ny, nz, h, k0, eps_bg, opts, eps_host: int, e_host: int, w_host: int) -> tuple:
    t = ctypes.c_int64()
    st = lib().vie_server_submit(srv, nx, ny, nz, h, k0, eps_bg, ctypes.byref(opts) if opts is not None else None,
                                 ctypes.c_void_p(eps_host), ctypes.c_void_p(e_host), ctypes.c_void_p(w_host),
                                 ctypes.byref(t))
    return st, t.value


def vie_server_poll(srv, ticket: int):
    info = vie_info()
    st = lib().vie_server_poll(srv, ticket, ctypes.byref(info))
    return st, info


def vie_server_drain(srv, timeout_ms: float) -> int:
    return lib().vie_server_drain(srv, timeout_ms)


def vie_server_reserved_bytes(srv) -> int:
    return lib().vie_server_reserved_bytes(srv)


def vie_estimate_bytes(nx, ny, nz, opts=None) -> int:
    return lib().vie_estimate_bytes(nx, ny, nz, ctypes.byref(opts) if opts is not None else None)


def vie_server_destroy(srv) -> None:
    lib().vie_server_destroy(srv)


def vie_matvec_static(nx, ny, nz, h, k0, eps_bg, eps_ptr: int, x_ptr: int, y_ptr: int, stream: int = 0) -> int:
    """Allocation-free complex-FP64 matvec (all scratch in a fixed array inside
    libvie); returns the status code unchanged."""
    return lib().vie_matvec_static(nx, ny, nz, h, k0, eps_bg, ctypes.c_void_p(eps_ptr), ctypes.c_void_p(x_ptr),
                                   ctypes.c_void_p(y_ptr), ctypes.c_void_p(stream))


def vie_plan_tuning(plan) -> str:
    """The autotuner's report for the plan (candidates, times, choices)."""
    return (lib().vie_plan_tuning(plan) or b"").decode()


def vie_plan_set_tuning(plan, kernel: str, choice: int) -> int:
    """Override one autotuner choice (test hook); returns the status code."""
    return lib().vie_plan_set_tuning(plan, kernel.encode(), choice)


def vie_kernel_launches() -> int:
    return lib().vie_kernel_launches()


def vie_profile_enable(on: bool) -> None:
    lib().vie_profile_enable(1 if on else 0)


def vie_profile_reset() -> None:
    lib().vie_profile_reset()


def vie_profile_query(kernel: str):
    n = ctypes.c_int64()
    t = ctypes.c_double()
    check(lib().vie_profile_query(kernel.encode(), ctypes.byref(n), ctypes.byref(t)))
    return n.value, t.value


def vie_profile_kernels():
    cap = 64
    arr = (ctypes.c_char_p * cap)()
    n = lib().vie_profile_kernels(arr, cap)
    return [arr[i].decode() for i in range(min(n, cap))]


def profile_table() -> dict:
    """{kernel: (launches, total_ms)} for every kernel recorded since the last reset."""
    return {k: vie_profile_query(k) for k in vie_profile_kernels()}
