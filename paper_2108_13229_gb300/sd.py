"""Thin ctypes binding of the C ABI in include/sd.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Arrays may
be numpy float64 arrays (host) or contiguous float64 torch tensors (host or
CUDA); the library detects the memory type.  There is no Python fallback:
if libsd.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsd.so")
_lib = None

SD_OK, SD_PENDING = 0, 1
SD_E_INVAL, SD_E_NOMEM, SD_E_NOCONV, SD_E_NUMERIC, SD_E_TIMEOUT, SD_E_CUDA, SD_E_STATE = -1, -2, -3, -4, -5, -6, -7
SD_FP64, SD_MIXED = 0, 1
SD_TRI_SCHUR, SD_PV_BJ_I, SD_PV_BGS_I = 0, 1, 2
SD_BC_MMS, SD_BC_MMS_TRACTION, SD_BC_PAPER = 0, 1, 2
SD_PROF_APPLY, SD_PROF_CHEB_V, SD_PROF_MUPDATE, SD_PROF_MDOT = 0, 1, 2, 3
SD_NOALLOC_MAX_N = 256
SD_BATCH_LOCKSTEP = 1
SD_BATCH_GRAPH = 2
SD_SERVER_LOCKSTEP = 1
SD_MONOLITHIC, SD_PARTITIONED = 0, 1
SD_ORDER_AUTO, SD_ORDER_PM_FIRST, SD_ORDER_FF_FIRST = 0, 1, 2
SD_GEO_SQUARE, SD_GEO_CHANNEL = 0, 1


class SdError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, sd_strerror(code), code))


class sd_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32)]


class sd_options(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("rtol", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("precond", ctypes.c_int32), ("bc", ctypes.c_int32),
                ("cheb_degree", ctypes.c_int32), ("cheb_degree_coarse", ctypes.c_int32),
                ("schur_degree", ctypes.c_int32), ("coarsest", ctypes.c_int32), ("schur_gamma", ctypes.c_double),
                ("cheb_ratio", ctypes.c_double), ("schur_mass", ctypes.c_int32), ("fuse_coarse", ctypes.c_int32),
                ("orth", ctypes.c_int32), ("reorth_eta", ctypes.c_double), ("extrapolate", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("pdl", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("tile_rows", ctypes.c_int32),
                ("darcy_coupled", ctypes.c_int32), ("coupling", ctypes.c_int32),
                ("coupling_max", ctypes.c_int32), ("coupling_columns", ctypes.c_int32),
                ("coupling_eps", ctypes.c_double), ("coupling_omega", ctypes.c_double),
                ("coupling_order", ctypes.c_int32), ("coupling_rtol", ctypes.c_double),
                ("bc_dp", ctypes.c_double), ("bc_tend", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("geometry", ctypes.c_int32), ("darcy_schur", ctypes.c_int32)]


class sd_step_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32), ("status", ctypes.c_int32),
                ("relres", ctypes.c_double), ("ms", ctypes.c_double), ("reorths", ctypes.c_int32),
                ("coupling_iters", ctypes.c_int32), ("relres_v", ctypes.c_double),
                ("relres_pff", ctypes.c_double), ("relres_pm", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sd_request(ctypes.Structure):
    _fields_ = [("grid", sd_grid), ("mu", ctypes.c_double), ("alpha_bj", ctypes.c_double), ("dt", ctypes.c_double),
                ("K", ctypes.POINTER(ctypes.c_double)), ("nsteps", ctypes.c_int32), ("keep_fields", ctypes.c_int32)]


class sd_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps_done", ctypes.c_int32), ("total_iters", ctypes.c_int32),
                ("max_relres", ctypes.c_double), ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("dof", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = ctypes.c_void_p
_SIGS = {
    "sd_options_default": (None, [ctypes.POINTER(sd_options)]),
    "sd_dof_count": (ctypes.c_int64, [ctypes.c_int32]),
    "sd_dof_count_geometry": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int32]),
    "sd_memory_estimate": (ctypes.c_int64, [ctypes.POINTER(sd_grid), ctypes.POINTER(sd_options)]),
    "sd_create": (ctypes.c_int, [ctypes.POINTER(sd_grid), ctypes.c_double, _vp, ctypes.c_double, ctypes.c_double,
                                 ctypes.POINTER(sd_options), ctypes.POINTER(_vp)]),
    "sd_step": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(sd_step_info)]),
    "sd_get_fields": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "sd_get_state": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), _vp, _vp]),
    "sd_set_state": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int64, _vp, _vp]),
    "sd_get_history": (ctypes.c_int, [_vp, _vp]),
    "sd_set_history": (ctypes.c_int, [_vp, _vp]),
    "sd_apply": (ctypes.c_int, [_vp, _vp, _vp]),
    "sd_rhs": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp]),
    "sd_solve": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(sd_step_info)]),
    "sd_sync": (ctypes.c_int, [_vp]),
    "sd_destroy": (None, [_vp]),
    "sd_solve_batch": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.POINTER(sd_step_info)), ctypes.c_int32]),
    "sd_solve_batch_ex": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.POINTER(sd_step_info)), ctypes.c_int32, ctypes.c_int32]),
    "sd_server_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(sd_options),
                                        ctypes.POINTER(_vp)]),
    "sd_server_create_ex": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(sd_options), ctypes.c_int32,
                                           ctypes.POINTER(_vp)]),
    "sd_submit": (ctypes.c_int, [_vp, ctypes.POINTER(sd_request), ctypes.POINTER(ctypes.c_uint64)]),
    "sd_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(sd_result), _vp]),
    "sd_server_drain": (ctypes.c_int, [_vp]),
    "sd_server_destroy": (None, [_vp]),
    "sd_profile": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "sd_profile_read": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "sd_launch_count": (ctypes.c_int64, []),
    "sd_struct_size": (ctypes.c_int64, [ctypes.c_int32]),
    "sd_apply_noalloc": (ctypes.c_int, [ctypes.POINTER(sd_grid), ctypes.c_double, _vp, ctypes.c_double,
                                        ctypes.c_double, _vp, _vp, _vp]),
    "sd_autotune": (ctypes.c_int, [ctypes.POINTER(sd_grid), ctypes.c_double, _vp, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(sd_options), ctypes.c_int32, ctypes.c_char_p,
                                   ctypes.POINTER(sd_options), ctypes.POINTER(ctypes.c_double)]),
    "sd_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}


def lib_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError("libsd.so is not built (run __graft_entry__.build() or "
                           "python -m paper_2108_13229_gb300.build)")
    lib = ctypes.CDLL(_LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code: int, where: str) -> int:
    if code < 0:
        raise SdError(code, where)
    return code


def _ptr(a, count=None):
    """Address of a float64 contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float64 numpy array")
        if count is not None and a.size < count:
            raise ValueError("array too small: %d < %d" % (a.size, count))
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        if count is not None and a.numel() < count:
            raise ValueError("tensor too small")
        if a.is_cuda:
            torch.cuda.current_stream(a.device).synchronize()
        return a.data_ptr()
    raise TypeError("unsupported array type %r" % type(a))


# ------------------------------------------------------------------ API
def sd_strerror(code: int) -> str:
    return _load().sd_strerror(int(code)).decode()


def sd_options_default() -> sd_options:
    o = sd_options()
    _load().sd_options_default(ctypes.byref(o))
    return o


def sd_dof_count(n: int) -> int:
    return int(_load().sd_dof_count(int(n)))


def sd_dof_count_geometry(n: int, geometry: int) -> int:
    return int(_load().sd_dof_count_geometry(int(n), int(geometry)))


def sd_memory_estimate(n: int, opts: sd_options | None = None) -> int:
    g = sd_grid(n, n)
    return int(_load().sd_memory_estimate(ctypes.byref(g), ctypes.byref(opts) if opts is not None else None))


class Handle:
    """Owns one sd_handle; freed by sd_destroy() or garbage collection."""

    def __init__(self, ptr, n, geometry=SD_GEO_SQUARE):
        self.ptr = ptr
        self.n = n
        self.geometry = geometry
        self.nx = 3 * n if geometry == SD_GEO_CHANNEL else n  # free-flow cells across
        self.dof = sd_dof_count_geometry(n, geometry)

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                _load().sd_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def sd_create(n: int, mu: float, K, alpha_bj: float, dt: float, opts: sd_options | None = None) -> Handle:
    if isinstance(K, np.ndarray):
        K = np.ascontiguousarray(K, dtype=np.float64)
    out = ctypes.c_void_p()
    g = sd_grid(n, n)
    rc = _load().sd_create(ctypes.byref(g), float(mu), _ptr(K, n * n), float(alpha_bj), float(dt),
                           ctypes.byref(opts) if opts is not None else None, ctypes.byref(out))
    _check(rc, "sd_create")
    return Handle(out.value, n, opts.geometry if opts is not None else SD_GEO_SQUARE)


def sd_step(h: Handle, nsteps: int = 1, raise_on_error: bool = True):
    info = (sd_step_info * max(1, nsteps))()
    rc = _load().sd_step(h.ptr, int(nsteps), info)
    if raise_on_error:
        _check(rc, "sd_step")
    return [info[k].as_dict() for k in range(nsteps)]


def sd_get_fields(h: Handle, u=None, v=None, p_ff=None, p_pm=None):
    """Copy the fields out; numpy arrays are allocated for the ones not given."""
    n, nx = h.n, h.nx
    u = np.empty((n, nx + 1)) if u is None else u
    v = np.empty((n + 1, nx)) if v is None else v
    p_ff = np.empty((n, nx)) if p_ff is None else p_ff
    p_pm = np.empty((n, n)) if p_pm is None else p_pm
    _check(_load().sd_get_fields(h.ptr, _ptr(u, n * (nx + 1)), _ptr(v, nx * (n + 1)), _ptr(p_ff, n * nx),
                                 _ptr(p_pm, n * n)), "sd_get_fields")
    return {"u": u, "v": v, "p_ff": p_ff, "p_pm": p_pm}


def sd_get_state(h: Handle, x=None, xprev=None, with_prev: bool = False):
    """(t, step, x) or, with_prev=True, (t, step, x, xprev)."""
    x = np.empty(h.dof) if x is None else x
    if with_prev and xprev is None:
        xprev = np.empty(h.dof)
    t = ctypes.c_double()
    st = ctypes.c_int64()
    _check(_load().sd_get_state(h.ptr, ctypes.byref(t), ctypes.byref(st), _ptr(x, h.dof),
                                _ptr(xprev, h.dof) if xprev is not None else None), "sd_get_state")
    if with_prev or xprev is not None:
        return t.value, st.value, x, xprev
    return t.value, st.value, x


def sd_set_state(h: Handle, t: float, step: int, x, xprev=None) -> None:
    _check(_load().sd_set_state(h.ptr, float(t), int(step), _ptr(x, h.dof),
                                _ptr(xprev, h.dof) if xprev is not None else None), "sd_set_state")


def sd_get_history(h: Handle, xprev2=None):
    """x^{n-2} of the quadratic extrapolation, or None when the handle does not hold it."""
    xprev2 = np.empty(h.dof) if xprev2 is None else xprev2
    rc = _load().sd_get_history(h.ptr, _ptr(xprev2, h.dof))
    if rc == SD_E_STATE:
        return None
    _check(rc, "sd_get_history")
    return xprev2


def sd_set_history(h: Handle, xprev2) -> None:
    _check(_load().sd_set_history(h.ptr, _ptr(xprev2, h.dof)), "sd_set_history")


def sd_apply(h: Handle, x, y=None):
    y = np.empty(h.dof) if y is None else y
    _check(_load().sd_apply(h.ptr, _ptr(x, h.dof), _ptr(y, h.dof)), "sd_apply")
    return y


def sd_rhs(h: Handle, xprev, t: float, b=None):
    b = np.empty(h.dof) if b is None else b
    _check(_load().sd_rhs(h.ptr, _ptr(xprev, h.dof), float(t), _ptr(b, h.dof)), "sd_rhs")
    return b


def sd_solve(h: Handle, b, x, raise_on_error: bool = True):
    """Solve A x = b in place (x: initial guess in, solution out)."""
    info = sd_step_info()
    rc = _load().sd_solve(h.ptr, _ptr(b, h.dof), _ptr(x, h.dof), ctypes.byref(info))
    if raise_on_error:
        _check(rc, "sd_solve")
    return info.as_dict()


def sd_sync(h: Handle) -> None:
    _check(_load().sd_sync(h.ptr), "sd_sync")


def sd_destroy(h: Handle) -> None:
    if h.ptr:
        _load().sd_destroy(h.ptr)
        h.ptr = None


def sd_solve_batch(handles, nsteps, max_threads: int = 0, raise_on_error: bool = True, lockstep: bool = True):
    """Advance the handles together; lockstep=False: every instance on its own stream (sd_solve_batch_ex flags 0)."""
    return sd_solve_batch_ex(handles, nsteps, max_threads, SD_BATCH_LOCKSTEP if lockstep else 0, raise_on_error)


def sd_solve_batch_ex(handles, nsteps, max_threads: int = 0, flags: int = SD_BATCH_LOCKSTEP,
                      raise_on_error: bool = True):
    """Advance the handles together with the given SD_BATCH_* flags; per handle, a list of its step infos."""
    cnt = len(handles)
    hs = (ctypes.c_void_p * cnt)(*[h.ptr for h in handles])
    ns = (ctypes.c_int32 * cnt)(*[int(k) for k in nsteps])
    bufs = [(sd_step_info * max(1, int(k)))() for k in nsteps]
    infos = (ctypes.POINTER(sd_step_info) * cnt)(*[ctypes.cast(b, ctypes.POINTER(sd_step_info)) for b in bufs])
    rc = _load().sd_solve_batch_ex(hs, cnt, ns, infos, int(max_threads), int(flags))
    if raise_on_error:
        _check(rc, "sd_solve_batch_ex")
    return [[bufs[k][q].as_dict() for q in range(int(nsteps[k]))] for k in range(cnt)]


class Server:
    def __init__(self, ptr):
        self.ptr = ptr
        self._keep = {}

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                _load().sd_server_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def sd_server_create(hbm_budget_bytes: int, max_running: int = 4, opts: sd_options | None = None,
                     lockstep: bool = False) -> Server:
    """lockstep=True: small runs served by size class in lockstep ticks (sd_server_create_ex SD_SERVER_LOCKSTEP)."""
    out = ctypes.c_void_p()
    _check(_load().sd_server_create_ex(int(hbm_budget_bytes), int(max_running),
                                       ctypes.byref(opts) if opts is not None else None,
                                       SD_SERVER_LOCKSTEP if lockstep else 0, ctypes.byref(out)),
           "sd_server_create")
    return Server(out.value)


def sd_server_create_ex(hbm_budget_bytes: int, max_running: int = 4, opts: sd_options | None = None,
                        flags: int = 0) -> Server:
    return sd_server_create(hbm_budget_bytes, max_running, opts, lockstep=bool(flags & SD_SERVER_LOCKSTEP))


def sd_submit(server: Server, n: int, mu: float, K, alpha_bj: float, dt: float, nsteps: int,
              keep_fields: bool = False) -> int:
    K = np.ascontiguousarray(K, dtype=np.float64).reshape(-1)
    req = sd_request(sd_grid(n, n), float(mu), float(alpha_bj), float(dt),
                     K.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(nsteps), int(bool(keep_fields)))
    ticket = ctypes.c_uint64()
    _check(_load().sd_submit(server.ptr, ctypes.byref(req), ctypes.byref(ticket)), "sd_submit")
    server._keep[ticket.value] = 4 * n * n + 2 * n
    return ticket.value


def sd_poll(server: Server, ticket: int, want_x: bool = False):
    """(status, result dict, x or None); status SD_PENDING while not finished."""
    res = sd_result()
    dof = server._keep.get(ticket, 0)
    x = np.empty(dof) if (want_x and dof) else None
    rc = _load().sd_poll(server.ptr, ctypes.c_uint64(ticket), ctypes.byref(res), _ptr(x) if x is not None else None)
    if rc != SD_PENDING:
        server._keep.pop(ticket, None)
    return rc, res.as_dict(), x


def sd_server_drain(server: Server) -> None:
    _check(_load().sd_server_drain(server.ptr), "sd_server_drain")


def sd_server_destroy(server: Server) -> None:
    if server.ptr:
        _load().sd_server_destroy(server.ptr)
        server.ptr = None


def sd_profile(h: Handle, kernel: int, enable: bool = True) -> None:
    _check(_load().sd_profile(h.ptr, int(kernel), int(bool(enable))), "sd_profile")


def sd_profile_read(h: Handle):
    """(total device ms, launches, algorithmic bytes, algorithmic flops) of the profiled kernel class."""
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    by = ctypes.c_double()
    fl = ctypes.c_double()
    _check(_load().sd_profile_read(h.ptr, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(by), ctypes.byref(fl)),
           "sd_profile_read")
    return ms.value, cnt.value, by.value, fl.value


def sd_launch_count() -> int:
    return int(_load().sd_launch_count())


def sd_apply_noalloc(n: int, mu: float, K, alpha_bj: float, dt: float, x, y, stream=None) -> None:
    """y = A x without allocating (see include/sd.h).

    K, x and y are CUDA float64 tensors of one device (x and y of 4n^2+2n
    elements); the library refuses host memory with SD_E_INVAL.  The call
    runs with that device current; stream=None queues the work on its current
    torch stream, so later work on that stream sees y.  With an explicit
    cudaStream_t handle the caller orders its own reads of y after that
    stream."""
    dof = 4 * n * n + 2 * n
    g = sd_grid(n, n)
    cuda = [a for a in (K, x, y) if getattr(a, "is_cuda", False)]
    if not cuda:  # host arrays: passed through for the library to refuse
        _check(_load().sd_apply_noalloc(ctypes.byref(g), float(mu), _ptr(K, n * n), float(alpha_bj), float(dt),
                                        _ptr(x, dof), _ptr(y, dof), stream), "sd_apply_noalloc")
        return
    import torch
    dev = cuda[0].device
    if any(a.device != dev for a in cuda):
        raise ValueError("K, x and y must be on one device")
    with torch.cuda.device(dev):
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        _check(_load().sd_apply_noalloc(ctypes.byref(g), float(mu), _ptr(K, n * n), float(alpha_bj), float(dt),
                                        _ptr(x, dof), _ptr(y, dof), stream), "sd_apply_noalloc")


def sd_autotune(n: int, mu: float, K, alpha_bj: float, dt: float, base: sd_options | None = None,
                nsteps: int = 3, cache_path: str | None = None):
    """(tuned sd_options, mean device ms per step of the winner); see include/sd.h."""
    if isinstance(K, np.ndarray):
        K = np.ascontiguousarray(K, dtype=np.float64)
    g = sd_grid(n, n)
    best = sd_options()
    ms = ctypes.c_double()
    rc = _load().sd_autotune(ctypes.byref(g), float(mu), _ptr(K, n * n), float(alpha_bj), float(dt),
                             ctypes.byref(base) if base is not None else None, int(nsteps),
                             cache_path.encode() if cache_path else None, ctypes.byref(best), ctypes.byref(ms))
    _check(rc, "sd_autotune")
    return best, ms.value


def sd_struct_size(which: int) -> int:
    return int(_load().sd_struct_size(int(which)))
