"""ctypes binding of libpexsi_gb300.so (argument marshalling only).

Every function carries the name of the C entry point it calls and does no
arithmetic of the method: all numeric work runs in the library's CUDA
kernels. There is no CPU fallback; if the library is missing the first call
raises.

Host arrays are numpy arrays; device buffers are passed as integer addresses
(for example ``tensor.data_ptr()`` of a CUDA torch tensor) and streams as
integer ``cudaStream_t`` handles (``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_int64_p = ctypes.POINTER(ctypes.c_int64)
c_double_p = ctypes.POINTER(ctypes.c_double)

ERR_NAMES = {0: "PEXSI_OK", -1: "PEXSI_ERR_INVALID_ARG", -2: "PEXSI_ERR_NOT_SYMMETRIC", -3: "PEXSI_ERR_NOMEM",
             -4: "PEXSI_ERR_CUDA", -5: "PEXSI_ERR_BREAKDOWN", -6: "PEXSI_ERR_INTERNAL", -7: "PEXSI_ERR_CANCELLED",
             -8: "PEXSI_ERR_TIMEOUT", 1: "PEXSI_PENDING"}
PEXSI_PENDING = 1
PEXSI_ERR_INVALID_ARG = -1
PEXSI_ERR_NOMEM = -3
PEXSI_ERR_CANCELLED = -7
PEXSI_ERR_TIMEOUT = -8
PEXSI_ERR_BREAKDOWN = -5


class PexsiError(RuntimeError):
    def __init__(self, code: int, detail: str = ""):
        self.code = code
        super().__init__(f"{ERR_NAMES.get(code, code)}: {detail}")


class pexsi_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("panel", ctypes.c_int32), ("leaf_cols", ctypes.c_int32),
                ("amalgamate", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("split_slices", ctypes.c_int32),
                ("hbm_budget", ctypes.c_int64), ("wait_ns", ctypes.c_int64), ("inject", ctypes.c_int32),
                ("split_block", ctypes.c_int32)]


class pexsi_plan_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nsuper", ctypes.c_int64),
                ("nlevels", ctypes.c_int64), ("nnz_L", ctypes.c_int64), ("front_elems", ctypes.c_int64),
                ("max_front", ctypes.c_int64), ("max_width", ctypes.c_int64),
                ("factor_gemm_flops", ctypes.c_double), ("selinv_gemm_flops", ctypes.c_double),
                ("diag_flops", ctypes.c_double), ("gather_bytes", ctypes.c_double),
                ("batch", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64)]


class pexsi_dm_info(ctypes.Structure):
    _fields_ = [("trace_dm_s", ctypes.c_double), ("trace_edm_s", ctypes.c_double),
                ("trace_fdm_s", ctypes.c_double), ("min_pivot_ratio", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("gemm_flops", ctypes.c_double),
                ("n_poles", ctypes.c_int32), ("breakdown_front", ctypes.c_int32),
                ("trace_ddm_s", ctypes.c_double)]


class pexsi_schedule(ctypes.Structure):
    _fields_ = [("wave", ctypes.c_int32), ("oz_block", ctypes.c_int32), ("ms_per_pole", ctypes.c_double),
                ("from_cache", ctypes.c_int32), ("candidates", ctypes.c_int32)]


class pexsi_kernel_profile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double), ("tensor_flops", ctypes.c_double)]


PROFILE_CLASSES = 12


class pexsi_mu_opts(ctypes.Structure):
    _fields_ = [("mu_lo", ctypes.c_double), ("mu_hi", ctypes.c_double), ("n_electrons", ctypes.c_double),
                ("tol_ne", ctypes.c_double), ("delta_n", ctypes.c_double), ("n_shifts", ctypes.c_int32),
                ("max_inertia", ctypes.c_int32), ("max_newton", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


class pexsi_mu_info(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("n_e", ctypes.c_double), ("dn_dmu", ctypes.c_double),
                ("mu_inertia", ctypes.c_double), ("bracket_lo", ctypes.c_double), ("bracket_hi", ctypes.c_double),
                ("inertia_cycles", ctypes.c_int32), ("newton_iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("reserved0", ctypes.c_int32)]


class pexsi_server_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("slots", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("hbm_budget", ctypes.c_int64)]


class pexsi_request(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("H", c_double_p), ("S", c_double_p), ("mu", ctypes.c_double),
                ("beta", ctypes.c_double), ("delta_e", ctypes.c_double), ("n_poles", ctypes.c_int32),
                ("n_shifts", ctypes.c_int32), ("shifts", c_double_p), ("dm", c_double_p), ("edm", c_double_p),
                ("fdm", c_double_p), ("counts", c_int64_p)]


class pexsi_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("breakdown_front", ctypes.c_int32), ("trace_dm_s", ctypes.c_double),
                ("trace_edm_s", ctypes.c_double), ("trace_fdm_s", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("footprint_bytes", ctypes.c_int64),
                ("batch", ctypes.c_int32), ("max_concurrent", ctypes.c_int32)]


class pexsi_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("peak_bytes", ctypes.c_int64), ("budget", ctypes.c_int64),
                ("peak_concurrent", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


def _as_dict(st: ctypes.Structure) -> dict:
    return {name: getattr(st, name) for name, _ in st._fields_}


# (name, restype, argtypes) of every entry point declared in include/pexsi_gb300.h
SIGNATURES = [
    ("pexsi_opts_default", ctypes.c_int, [ctypes.POINTER(pexsi_opts)]),
    ("pexsi_setup", ctypes.c_int, [ctypes.c_int64, c_int64_p, c_int32_p, c_int32_p, ctypes.POINTER(pexsi_opts),
                                   ctypes.POINTER(ctypes.c_void_p)]),
    ("pexsi_plan_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("pexsi_plan_get_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pexsi_plan_stats)]),
    ("pexsi_plan_get_perm", ctypes.c_int, [ctypes.c_void_p, c_int32_p]),
    ("pexsi_plan_get_supernodes", ctypes.c_int, [ctypes.c_void_p, c_int32_p, c_int64_p, c_int32_p, c_int32_p]),
    ("pexsi_pole_table", ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                                        c_double_p, c_double_p, c_double_p, c_double_p]),
    ("pexsi_dm", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int32, ctypes.c_double, c_double_p, c_double_p, c_double_p,
                                ctypes.POINTER(pexsi_dm_info)]),
    ("pexsi_dm_poles", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      c_double_p, c_double_p, c_double_p, ctypes.POINTER(pexsi_dm_info)]),
    ("pexsi_profile_enable", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("pexsi_profile_read", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pexsi_kernel_profile)]),
    ("pexsi_profile_reset", ctypes.c_int, [ctypes.c_void_p]),
    ("pexsi_dm_device", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(pexsi_dm_info)]),
    ("pexsi_selinv", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, ctypes.c_double, ctypes.c_double,
                                    c_double_p]),
    ("pexsi_inertia", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, c_double_p, ctypes.c_int32,
                                     c_int64_p]),
    ("pexsi_inertia_device", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, c_double_p,
                                            ctypes.c_int32, c_int64_p, ctypes.c_void_p]),
    ("pexsi_dm_hermitian", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int32, ctypes.c_double, c_double_p, c_double_p,
                                          c_double_p, ctypes.POINTER(pexsi_dm_info)]),
    ("pexsi_dm_hermitian_device", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(pexsi_dm_info)]),
    ("pexsi_selinv_hermitian", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, ctypes.c_double,
                                              ctypes.c_double, c_double_p]),
    ("pexsi_inertia_hermitian", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, c_double_p, ctypes.c_int32,
                                               c_int64_p]),
    ("pexsi_group_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                          ctypes.POINTER(pexsi_opts), ctypes.POINTER(ctypes.c_void_p)]),
    ("pexsi_group_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("pexsi_group_get_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pexsi_plan_stats)]),
    ("pexsi_group_get_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pexsi_schedule)]),
    ("pexsi_group_set_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pexsi_schedule)]),
    ("pexsi_group_dm_device", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(ctypes.c_void_p), c_double_p, c_double_p, ctypes.c_int32,
                                             c_double_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                             ctypes.POINTER(pexsi_dm_info)]),
    ("pexsi_group_dm", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_void_p), c_double_p, c_double_p, ctypes.c_int32,
                                      c_double_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(pexsi_dm_info)]),
    ("pexsi_group_tune", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p), c_double_p, c_double_p, ctypes.c_int32,
                                        c_double_p, ctypes.c_char_p, ctypes.c_int32, ctypes.POINTER(pexsi_schedule)]),
    ("pexsi_group_last_error_detail", ctypes.c_char_p, [ctypes.c_void_p]),
    ("pexsi_trace_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    ("pexsi_mu_opts_default", ctypes.c_int, [ctypes.POINTER(pexsi_mu_opts)]),
    ("pexsi_mu_solve", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, ctypes.c_double, ctypes.c_int32,
                                      ctypes.c_double, ctypes.POINTER(pexsi_mu_opts), c_double_p, c_double_p,
                                      c_double_p, ctypes.POINTER(pexsi_mu_info)]),
    ("pexsi_dos", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int32, c_double_p, c_double_p, c_double_p]),
    ("pexsi_ldos", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, ctypes.c_double, ctypes.c_double,
                                  c_double_p]),
    ("pexsi_server_opts_default", ctypes.c_int, [ctypes.POINTER(pexsi_server_opts)]),
    ("pexsi_server_create", ctypes.c_int, [ctypes.POINTER(pexsi_server_opts), ctypes.POINTER(ctypes.c_void_p)]),
    ("pexsi_server_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pexsi_request), c_int64_p]),
    ("pexsi_server_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(pexsi_result)]),
    ("pexsi_server_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(pexsi_result)]),
    ("pexsi_server_cancel", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    ("pexsi_server_release", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    ("pexsi_server_get_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pexsi_server_stats)]),
    ("pexsi_server_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("pexsi_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("pexsi_last_error_detail", ctypes.c_char_p, [ctypes.c_void_p]),
]

_LIB = None


def library_path() -> str:
    return _build.lib_path()


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1405_0194_gb300.build.build(); "
                               "this package has no CPU fallback")
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(rc: int, plan=None):
    if rc != 0:
        detail = ""
        if plan is not None:
            d = lib().pexsi_last_error_detail(plan)
            detail = d.decode() if d else ""
        if not detail:
            detail = lib().pexsi_strerror(rc).decode()
        raise PexsiError(rc, detail)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.shape[0] != n:
        raise ValueError(f"expected {n} values, got {a.shape[0]}")
    return a


# ---------------------------------------------------------------- calls
def pexsi_opts_default(**overrides) -> pexsi_opts:
    o = pexsi_opts()
    _check(lib().pexsi_opts_default(ctypes.byref(o)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def pexsi_setup(n, colptr, rowind, perm=None, opts: pexsi_opts | None = None):
    """Returns an opaque plan handle (int)."""
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(rowind, dtype=np.int32)
    perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    h = ctypes.c_void_p()
    rc = lib().pexsi_setup(int(n), _ptr(colptr, ctypes.c_int64), _ptr(rowind, ctypes.c_int32),
                           _ptr(perm, ctypes.c_int32), None if opts is None else ctypes.byref(opts), ctypes.byref(h))
    _check(rc)
    return h.value


def pexsi_plan_destroy(plan):
    _check(lib().pexsi_plan_destroy(plan))


def pexsi_plan_get_stats(plan) -> dict:
    st = pexsi_plan_stats()
    _check(lib().pexsi_plan_get_stats(plan, ctypes.byref(st)), plan)
    return _as_dict(st)


def pexsi_plan_get_perm(plan) -> np.ndarray:
    n = pexsi_plan_get_stats(plan)["n"]
    perm = np.empty(n, dtype=np.int32)
    _check(lib().pexsi_plan_get_perm(plan, _ptr(perm, ctypes.c_int32)), plan)
    return perm


def pexsi_plan_get_supernodes(plan):
    """(first, rptr, rows, parent) of the supernodal structure."""
    ns = pexsi_plan_get_stats(plan)["nsuper"]
    first = np.empty(ns + 1, dtype=np.int32)
    rptr = np.empty(ns + 1, dtype=np.int64)
    parent = np.empty(ns, dtype=np.int32)
    _check(lib().pexsi_plan_get_supernodes(plan, _ptr(first, ctypes.c_int32), _ptr(rptr, ctypes.c_int64), None,
                                           _ptr(parent, ctypes.c_int32)), plan)
    rows = np.empty(int(rptr[-1]), dtype=np.int32)
    _check(lib().pexsi_plan_get_supernodes(plan, _ptr(first, ctypes.c_int32), _ptr(rptr, ctypes.c_int64),
                                           _ptr(rows, ctypes.c_int32), _ptr(parent, ctypes.c_int32)), plan)
    return first, rptr, rows, parent


def pexsi_pole_table(beta, delta_e, n_poles, mu=0.0) -> dict:
    """Shifts z_l + mu and weights (complex numpy arrays of length n_poles)."""
    bufs = [np.empty(2 * n_poles) for _ in range(4)]
    rc = lib().pexsi_pole_table(float(beta), float(delta_e), int(n_poles), float(mu),
                                *[_ptr(b, ctypes.c_double) for b in bufs])
    _check(rc)
    z, wr, we, wf = [b.view(np.complex128) for b in bufs]
    return {"z": z, "w_rho": wr, "w_E": we, "w_F": wf}


def pexsi_dm(plan, H, S, mu, beta, n_poles, delta_e, want=("dm", "edm", "fdm")):
    """Host-buffer DM/EDM/FDM. Returns (dm, edm, fdm, info); unwanted outputs are None."""
    nnz = pexsi_plan_get_stats(plan)["nnz"]
    H = _f64(H, nnz)
    S = None if S is None else _f64(S, nnz)
    outs = {k: (np.empty(nnz) if k in want else None) for k in ("dm", "edm", "fdm")}
    info = pexsi_dm_info()
    rc = lib().pexsi_dm(plan, _ptr(H, ctypes.c_double), _ptr(S, ctypes.c_double), float(mu), float(beta),
                        int(n_poles), float(delta_e), _ptr(outs["dm"], ctypes.c_double),
                        _ptr(outs["edm"], ctypes.c_double), _ptr(outs["fdm"], ctypes.c_double), ctypes.byref(info))
    _check(rc, plan)
    return outs["dm"], outs["edm"], outs["fdm"], _as_dict(info)


def pexsi_dm_poles(plan, H, S, mu, beta, n_poles, delta_e, pole_begin, pole_end, accumulate=0, dm=None, edm=None,
                   fdm=None):
    """Host-buffer DM/EDM/FDM over a pole subrange. ``dm``/``edm``/``fdm`` are
    float64 numpy arrays of nnz (or None to skip); they are written (or added
    to when ``accumulate``). Returns the info dict."""
    nnz = pexsi_plan_get_stats(plan)["nnz"]
    H = _f64(H, nnz) if not (isinstance(H, np.ndarray) and H.flags.c_contiguous and H.dtype == np.float64) else H
    if S is not None and not (isinstance(S, np.ndarray) and S.flags.c_contiguous and S.dtype == np.float64):
        S = _f64(S, nnz)
    for a in (dm, edm, fdm):
        if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous or a.shape[0] != nnz):
            raise ValueError("outputs must be contiguous float64 arrays of nnz")
    info = pexsi_dm_info()
    rc = lib().pexsi_dm_poles(plan, _ptr(H, ctypes.c_double), _ptr(S, ctypes.c_double), float(mu), float(beta),
                              int(n_poles), float(delta_e), int(pole_begin), int(pole_end), int(accumulate),
                              _ptr(dm, ctypes.c_double), _ptr(edm, ctypes.c_double), _ptr(fdm, ctypes.c_double),
                              ctypes.byref(info))
    _check(rc, plan)
    return _as_dict(info)


def pexsi_profile_enable(plan, on=True):
    _check(lib().pexsi_profile_enable(plan, int(bool(on))), plan)


def pexsi_profile_reset(plan):
    _check(lib().pexsi_profile_reset(plan), plan)


def pexsi_profile_read(plan) -> list:
    """Per-kernel-class totals: list of dicts (name, launches, ms, flops, bytes)."""
    arr = (pexsi_kernel_profile * PROFILE_CLASSES)()
    _check(lib().pexsi_profile_read(plan, arr), plan)
    return [{"name": a.name.decode(), "launches": a.launches, "ms": a.ms, "flops": a.flops, "bytes": a.bytes,
             "tensor_flops": a.tensor_flops} for a in arr]


def pexsi_dm_device(plan, dH, dS, mu, beta, n_poles, delta_e, pole_begin, pole_end, accumulate, d_dm, d_edm, d_fdm,
                    stream=0, want_info=False):
    """Device-buffer form; pointers and stream are integers (0 / None = NULL)."""
    info = pexsi_dm_info() if want_info else None
    rc = lib().pexsi_dm_device(plan, dH or None, dS or None, float(mu), float(beta), int(n_poles), float(delta_e),
                               int(pole_begin), int(pole_end), int(accumulate), d_dm or None, d_edm or None,
                               d_fdm or None, stream or None, None if info is None else ctypes.byref(info))
    _check(rc, plan)
    return None if info is None else _as_dict(info)


def pexsi_selinv(plan, H, S, z) -> np.ndarray:
    """Selected elements of (H - z S)^{-1} on the pattern (complex, CSC order)."""
    nnz = pexsi_plan_get_stats(plan)["nnz"]
    H = _f64(H, nnz)
    S = None if S is None else _f64(S, nnz)
    out = np.empty(2 * nnz)
    rc = lib().pexsi_selinv(plan, _ptr(H, ctypes.c_double), _ptr(S, ctypes.c_double), float(np.real(z)),
                            float(np.imag(z)), _ptr(out, ctypes.c_double))
    _check(rc, plan)
    return out.view(np.complex128)


def pexsi_inertia(plan, H, S, shifts) -> np.ndarray:
    nnz = pexsi_plan_get_stats(plan)["nnz"]
    H = _f64(H, nnz)
    S = None if S is None else _f64(S, nnz)
    shifts = _f64(np.atleast_1d(shifts))
    counts = np.empty(shifts.shape[0], dtype=np.int64)
    rc = lib().pexsi_inertia(plan, _ptr(H, ctypes.c_double), _ptr(S, ctypes.c_double), _ptr(shifts, ctypes.c_double),
                             int(shifts.shape[0]), _ptr(counts, ctypes.c_int64))
    _check(rc, plan)
    return counts


def pexsi_inertia_device(plan, dH, dS, shifts, stream=0) -> np.ndarray:
    shifts = _f64(np.atleast_1d(shifts))
    counts = np.empty(shifts.shape[0], dtype=np.int64)
    rc = lib().pexsi_inertia_device(plan, dH or None, dS or None, _ptr(shifts, ctypes.c_double),
                                    int(shifts.shape[0]), _ptr(counts, ctypes.c_int64), stream or None)
    _check(rc, plan)
    return counts


def pexsi_trace_noalloc(d_dm, d_edm, d_fdm, d_S, nnz, d_out3, stream=0):
    """Allocation-free (Tr[DM S], Tr[EDM S], Tr[FDM S]) into the device array
    at d_out3; all arguments are device addresses (0 / None = NULL)."""
    rc = lib().pexsi_trace_noalloc(d_dm or None, d_edm or None, d_fdm or None, d_S or None, int(nnz),
                                   d_out3 or None, stream or None)
    _check(rc)


# ---------------------------------------------------------------- complex Hermitian H and S
def _c128(a, n):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.shape[0] != n:
        raise ValueError(f"expected {n} values, got {a.shape[0]}")
    return a


def _cptr(a):
    return None if a is None else a.ctypes.data_as(c_double_p)


def pexsi_dm_hermitian(plan, H, S, mu, beta, n_poles, delta_e, want=("dm", "edm", "fdm")):
    """Complex Hermitian H, S (complex128 arrays of nnz, CSC order; S None =
    identity). Returns complex (dm, edm, fdm, info); unwanted outputs None."""
    nnz = pexsi_plan_get_stats(plan)["nnz"]
    H = _c128(H, nnz)
    S = None if S is None else _c128(S, nnz)
    outs = {k: (np.empty(nnz, dtype=np.complex128) if k in want else None) for k in ("dm", "edm", "fdm")}
    info = pexsi_dm_info()
    rc = lib().pexsi_dm_hermitian(plan, _cptr(H), _cptr(S), float(mu), float(beta), int(n_poles), float(delta_e),
                                  _cptr(outs["dm"]), _cptr(outs["edm"]), _cptr(outs["fdm"]), ctypes.byref(info))
    _check(rc, plan)
    return outs["dm"], outs["edm"], outs["fdm"], _as_dict(info)


def pexsi_dm_hermitian_device(plan, dH, dS, mu, beta, n_poles, delta_e, pole_begin, pole_end, accumulate, d_dm,
                              d_edm, d_fdm, stream=0, want_info=False):
    """Device form (addresses of complex128 device arrays of nnz)."""
    info = pexsi_dm_info() if want_info else None
    rc = lib().pexsi_dm_hermitian_device(plan, dH or None, dS or None, float(mu), float(beta), int(n_poles),
                                         float(delta_e), int(pole_begin), int(pole_end), int(accumulate),
                                         d_dm or None, d_edm or None, d_fdm or None, stream or None,
                                         None if info is None else ctypes.byref(info))
    _check(rc, plan)
    return None if info is None else _as_dict(info)


def pexsi_selinv_hermitian(plan, H, S, z) -> np.ndarray:
    """G[r, c] of (H - z S)^{-1} at every CSC entry (complex128, nnz)."""
    nnz = pexsi_plan_get_stats(plan)["nnz"]
    H = _c128(H, nnz)
    S = None if S is None else _c128(S, nnz)
    out = np.empty(nnz, dtype=np.complex128)
    rc = lib().pexsi_selinv_hermitian(plan, _cptr(H), _cptr(S), float(np.real(z)), float(np.imag(z)), _cptr(out))
    _check(rc, plan)
    return out


def pexsi_inertia_hermitian(plan, H, S, shifts) -> np.ndarray:
    nnz = pexsi_plan_get_stats(plan)["nnz"]
    H = _c128(H, nnz)
    S = None if S is None else _c128(S, nnz)
    shifts = _f64(np.atleast_1d(shifts))
    counts = np.empty(shifts.shape[0], dtype=np.int64)
    rc = lib().pexsi_inertia_hermitian(plan, _cptr(H), _cptr(S), _ptr(shifts, ctypes.c_double),
                                       int(shifts.shape[0]), _ptr(counts, ctypes.c_int64))
    _check(rc, plan)
    return counts


# ---------------------------------------------------------------- groups of systems
def _ptrs(vals):
    """ctypes array of void* from integers / numpy arrays / None."""
    arr = (ctypes.c_void_p * len(vals))()
    for i, v in enumerate(vals):
        if v is None or (isinstance(v, int) and v == 0):
            arr[i] = None
        elif isinstance(v, np.ndarray):
            arr[i] = v.ctypes.data
        else:
            arr[i] = int(v)
    return arr


def _gcheck(rc, group):
    if rc != 0:
        d = lib().pexsi_group_last_error_detail(group) if group else b""
        raise PexsiError(rc, (d.decode() if d else "") or lib().pexsi_strerror(rc).decode())


def pexsi_group_create(plans, opts: pexsi_opts | None = None):
    """A group over the systems of `plans` (plan handles). Returns a handle."""
    arr = (ctypes.c_void_p * len(plans))(*plans)
    h = ctypes.c_void_p()
    rc = lib().pexsi_group_create(arr, len(plans), None if opts is None else ctypes.byref(opts), ctypes.byref(h))
    _check(rc)
    return h.value


def pexsi_group_destroy(group):
    _check(lib().pexsi_group_destroy(group))


def pexsi_group_get_stats(group) -> dict:
    st = pexsi_plan_stats()
    _gcheck(lib().pexsi_group_get_stats(group, ctypes.byref(st)), group)
    return _as_dict(st)


def pexsi_group_get_schedule(group) -> dict:
    sc = pexsi_schedule()
    _gcheck(lib().pexsi_group_get_schedule(group, ctypes.byref(sc)), group)
    return _as_dict(sc)


def pexsi_group_set_schedule(group, wave=0, oz_block=4):
    sc = pexsi_schedule(int(wave), int(oz_block), 0.0, 0, 0)
    _gcheck(lib().pexsi_group_set_schedule(group, ctypes.byref(sc)), group)


def pexsi_group_dm_device(group, dH, dS, mu, beta, n_poles, delta_e, pole_begin, pole_end, accumulate, d_dm, d_edm,
                          d_fdm, stream=0, want_info=False):
    """Device form: dH, dS, d_dm, d_edm, d_fdm are lists of device addresses
    (one per system; dS may be None); mu, beta, delta_e lists of floats.
    Returns a list of info dicts when want_info."""
    n = len(dH)
    mu_a, beta_a, de_a = (np.ascontiguousarray(x, dtype=np.float64) for x in (mu, beta, delta_e))
    infos = (pexsi_dm_info * n)() if want_info else None
    rc = lib().pexsi_group_dm_device(group, _ptrs(dH), None if dS is None else _ptrs(dS), _ptr(mu_a, ctypes.c_double),
                                     _ptr(beta_a, ctypes.c_double), int(n_poles), _ptr(de_a, ctypes.c_double),
                                     int(pole_begin), int(pole_end), int(accumulate), _ptrs(d_dm), _ptrs(d_edm),
                                     _ptrs(d_fdm), stream or None, infos)
    _gcheck(rc, group)
    return None if infos is None else [_as_dict(x) for x in infos]


def pexsi_group_dm(group, H, S, mu, beta, n_poles, delta_e):
    """Host form: H, S lists of float64 arrays (S may be None). Returns
    (dm, edm, fdm, infos): lists per system."""
    n = len(H)
    H = [_f64(h) for h in H]
    S = None if S is None else [None if x is None else _f64(x) for x in S]
    outs = [[np.empty(h.shape[0]) for h in H] for _ in range(3)]
    mu_a, beta_a, de_a = (np.ascontiguousarray(x, dtype=np.float64) for x in (mu, beta, delta_e))
    infos = (pexsi_dm_info * n)()
    rc = lib().pexsi_group_dm(group, _ptrs(H), None if S is None else _ptrs(S), _ptr(mu_a, ctypes.c_double),
                              _ptr(beta_a, ctypes.c_double), int(n_poles), _ptr(de_a, ctypes.c_double),
                              _ptrs(outs[0]), _ptrs(outs[1]), _ptrs(outs[2]), infos)
    _gcheck(rc, group)
    return outs[0], outs[1], outs[2], [_as_dict(x) for x in infos]


def pexsi_group_tune(group, dH, dS, mu, beta, n_poles, delta_e, cache_path=None, force=False) -> dict:
    mu_a, beta_a, de_a = (np.ascontiguousarray(x, dtype=np.float64) for x in (mu, beta, delta_e))
    sc = pexsi_schedule()
    rc = lib().pexsi_group_tune(group, _ptrs(dH), None if dS is None else _ptrs(dS), _ptr(mu_a, ctypes.c_double),
                                _ptr(beta_a, ctypes.c_double), int(n_poles), _ptr(de_a, ctypes.c_double),
                                None if cache_path is None else str(cache_path).encode(), int(bool(force)),
                                ctypes.byref(sc))
    _gcheck(rc, group)
    return _as_dict(sc)


# ---------------------------------------------------------------- mu search
def pexsi_mu_opts_default(**overrides) -> pexsi_mu_opts:
    o = pexsi_mu_opts()
    _check(lib().pexsi_mu_opts_default(ctypes.byref(o)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def pexsi_mu_solve(plan, H, S, beta, n_poles, delta_e, opts: pexsi_mu_opts, want=("dm", "edm", "fdm")):
    """Returns (dm, edm, fdm, info) at the chemical potential found."""
    nnz = pexsi_plan_get_stats(plan)["nnz"]
    H = _f64(H, nnz)
    S = None if S is None else _f64(S, nnz)
    outs = {k: (np.empty(nnz) if k in want else None) for k in ("dm", "edm", "fdm")}
    info = pexsi_mu_info()
    rc = lib().pexsi_mu_solve(plan, _ptr(H, ctypes.c_double), _ptr(S, ctypes.c_double), float(beta), int(n_poles),
                              float(delta_e), ctypes.byref(opts), _ptr(outs["dm"], ctypes.c_double),
                              _ptr(outs["edm"], ctypes.c_double), _ptr(outs["fdm"], ctypes.c_double),
                              ctypes.byref(info))
    _check(rc, plan)
    return outs["dm"], outs["edm"], outs["fdm"], _as_dict(info)


# ---------------------------------------------------------------- DOS / LDOS
def pexsi_dos(plan, H, S, e_lo, e_hi, n_points):
    """(eps, cdos, dos) arrays of n_points."""
    nnz = pexsi_plan_get_stats(plan)["nnz"]
    H = _f64(H, nnz)
    S = None if S is None else _f64(S, nnz)
    eps, cdos, dos = (np.empty(int(n_points)) for _ in range(3))
    rc = lib().pexsi_dos(plan, _ptr(H, ctypes.c_double), _ptr(S, ctypes.c_double), float(e_lo), float(e_hi),
                         int(n_points), _ptr(eps, ctypes.c_double), _ptr(cdos, ctypes.c_double),
                         _ptr(dos, ctypes.c_double))
    _check(rc, plan)
    return eps, cdos, dos


def pexsi_ldos(plan, H, S, eps, eta) -> np.ndarray:
    nnz = pexsi_plan_get_stats(plan)["nnz"]
    H = _f64(H, nnz)
    S = None if S is None else _f64(S, nnz)
    out = np.empty(nnz)
    rc = lib().pexsi_ldos(plan, _ptr(H, ctypes.c_double), _ptr(S, ctypes.c_double), float(eps), float(eta),
                          _ptr(out, ctypes.c_double))
    _check(rc, plan)
    return out


# ---------------------------------------------------------------- server
def pexsi_server_opts_default(**overrides) -> pexsi_server_opts:
    o = pexsi_server_opts()
    _check(lib().pexsi_server_opts_default(ctypes.byref(o)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def pexsi_server_create(opts: pexsi_server_opts | None = None):
    h = ctypes.c_void_p()
    _check(lib().pexsi_server_create(None if opts is None else ctypes.byref(opts), ctypes.byref(h)))
    return h.value


class ServerRequest:
    """Keeps the numpy buffers of one submitted request alive until it is
    collected (the server copies H, S and shifts at submit, but writes the
    outputs into these arrays when the request completes)."""

    def __init__(self, plan, H, S, mu=0.0, beta=1.0, n_poles=0, delta_e=1.0, shifts=None, want=("dm", "edm", "fdm")):
        nnz = pexsi_plan_get_stats(plan)["nnz"]
        self.H = _f64(H, nnz)
        self.S = None if S is None else _f64(S, nnz)
        self.shifts = None if shifts is None else _f64(np.atleast_1d(shifts))
        nsh = 0 if self.shifts is None else self.shifts.shape[0]
        self.dm = np.zeros(nnz) if (n_poles and "dm" in want) else None
        self.edm = np.zeros(nnz) if (n_poles and "edm" in want) else None
        self.fdm = np.zeros(nnz) if (n_poles and "fdm" in want) else None
        self.counts = np.zeros(nsh, dtype=np.int64) if nsh else None
        self.c = pexsi_request(plan, _ptr(self.H, ctypes.c_double), _ptr(self.S, ctypes.c_double), float(mu),
                               float(beta), float(delta_e), int(n_poles), int(nsh), _ptr(self.shifts, ctypes.c_double),
                               _ptr(self.dm, ctypes.c_double), _ptr(self.edm, ctypes.c_double),
                               _ptr(self.fdm, ctypes.c_double), _ptr(self.counts, ctypes.c_int64))
        self.ticket = None


def pexsi_server_submit(server, request: ServerRequest) -> int:
    t = ctypes.c_int64()
    _check(lib().pexsi_server_submit(server, ctypes.byref(request.c), ctypes.byref(t)))
    request.ticket = t.value
    return t.value


def pexsi_server_poll(server, ticket):
    """None while pending, else the result dict."""
    r = pexsi_result()
    rc = lib().pexsi_server_poll(server, int(ticket), ctypes.byref(r))
    if rc == PEXSI_PENDING:
        return None
    _check(rc)
    return _as_dict(r)


def pexsi_server_wait(server, ticket) -> dict:
    r = pexsi_result()
    _check(lib().pexsi_server_wait(server, int(ticket), ctypes.byref(r)))
    return _as_dict(r)


def pexsi_server_cancel(server, ticket):
    _check(lib().pexsi_server_cancel(server, int(ticket)))


def pexsi_server_release(server, ticket):
    _check(lib().pexsi_server_release(server, int(ticket)))


def pexsi_server_get_stats(server) -> dict:
    st = pexsi_server_stats()
    _check(lib().pexsi_server_get_stats(server, ctypes.byref(st)))
    return _as_dict(st)


def pexsi_server_destroy(server):
    _check(lib().pexsi_server_destroy(server))


def pexsi_strerror(code: int) -> str:
    return lib().pexsi_strerror(int(code)).decode()


def pexsi_last_error_detail(plan) -> str:
    d = lib().pexsi_last_error_detail(plan)
    return d.decode() if d else ""
