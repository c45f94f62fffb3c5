"""FP64 CPU oracle for the coupled Stokes-Darcy step (arXiv 2108.13229, Sec. 2).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this module; the product library never
imports it.  The arithmetic lives in ``sd_oracle.c`` (plain C, FP64,
single-threaded); this file only builds it with gcc and marshals numpy
arrays through ctypes.

Vector layout of the whole system (the same order as the public C ABI uses
for its host buffers): ``u`` ((n+1) x n faces, row j*(n+1)+i), ``v``
(n x (n+1) faces, row j*n+i, j = 0 on the interface), ``p_ff`` (n x n),
``p_pm`` (n x n); DoF = 4n^2 + 2n (Table 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sd_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: it also builds on Arm)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    lib.or_create.restype = ctypes.c_void_p
    lib.or_create.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
    lib.or_create_bc.restype = ctypes.c_void_p
    lib.or_create_bc.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_double]
    lib.or_create_geo.restype = ctypes.c_void_p
    lib.or_create_geo.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int]
    lib.or_dof_count_geo.restype = ctypes.c_int64
    lib.or_dof_count_geo.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.or_exact_geo.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp]
    lib.or_p_in.restype = ctypes.c_double
    lib.or_p_in.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.or_destroy.argtypes = [ctypes.c_void_p]
    lib.or_ndof.restype = ctypes.c_int64
    lib.or_ndof.argtypes = [ctypes.c_void_p]
    lib.or_nnz.restype = ctypes.c_int64
    lib.or_nnz.argtypes = [ctypes.c_void_p]
    lib.or_dof_count.restype = ctypes.c_int64
    lib.or_dof_count.argtypes = [ctypes.c_int]
    lib.or_get_csr.argtypes = [ctypes.c_void_p, _i64p, _i32p, _dp]
    lib.or_apply.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.or_exact.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
    lib.or_rhs.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, _dp]
    lib.or_factor.restype = ctypes.c_int
    lib.or_factor.argtypes = [ctypes.c_void_p]
    lib.or_solve.restype = ctypes.c_int
    lib.or_solve.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.or_bandwidth.restype = ctypes.c_int
    lib.or_bandwidth.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.or_residual.restype = ctypes.c_double
    lib.or_residual.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
    lib.or_run.restype = ctypes.c_int
    lib.or_run.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_int]
    for name in ("or_mms_u", "or_mms_v", "or_mms_ppm"):
        f = getattr(lib, name)
        f.restype = ctypes.c_double
        f.argtypes = [ctypes.c_double] * 3
    for name in ("or_mms_pff", "or_mms_fx", "or_mms_fy"):
        f = getattr(lib, name)
        f.restype = ctypes.c_double
        f.argtypes = [ctypes.c_double] * 4
    _lib = lib
    return lib


def _ptr(a: np.ndarray, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def dof_count(n: int, geo: int = 0) -> int:
    """4n^2 + 2n (geo 0, Table 1); 10n^2 + 4n for the channel of Sec. 5's model problem (geo 1)."""
    return int(_load().or_dof_count_geo(n, geo))


def ff_width(n: int, geo: int = 0) -> int:
    """Free-flow cells across: n (square) or 3n (channel)."""
    return 3 * n if geo == 1 else n


def offsets(n: int, geo: int = 0) -> dict:
    """Start offset of each field in the whole-system vector."""
    nx = ff_width(n, geo)
    nu, nv, npf = n * (nx + 1), nx * (n + 1), nx * n
    return {"u": 0, "v": nu, "p_ff": nu + nv, "p_pm": nu + nv + npf, "end": nu + nv + npf + n * n}


def split(x: np.ndarray, n: int, geo: int = 0) -> dict:
    """Views of the four fields as 2-D arrays indexed [j, i]."""
    o = offsets(n, geo)
    nx = ff_width(n, geo)
    return {
        "u": x[o["u"]:o["v"]].reshape(n, nx + 1),
        "v": x[o["v"]:o["p_ff"]].reshape(n + 1, nx),
        "p_ff": x[o["p_ff"]:o["p_pm"]].reshape(n, nx),
        "p_pm": x[o["p_pm"]:o["end"]].reshape(n, n),
    }


def exact(n: int, t: float, mu: float = 1.0, geo: int = 0) -> np.ndarray:
    """Manufactured solution sampled at the DoF locations at time t."""
    x = np.zeros(dof_count(n, geo))
    _load().or_exact_geo(n, t, mu, geo, _ptr(x))
    return x


def mms(name: str, *args) -> float:
    """Evaluate one manufactured closed form: u, v, pff, ppm, fx, fy."""
    return float(getattr(_load(), "or_mms_" + name)(*[float(a) for a in args]))


def p_in(dp: float, t_end: float, t: float) -> float:
    """Inflow pressure of the paper's pressure-driven problem (bc 2): half cosine from 0 to dp over [0, t_end]."""
    return float(_load().or_p_in(float(dp), float(t_end), float(t)))


class Oracle:
    """Assembled FP64 system of one instance (n cells per side per subdomain).

    bc 0: manufactured solution, Dirichlet velocity on the free-flow sides;
    bc 1: manufactured solution with traction free-flow sides;
    bc 2: the paper's pressure-driven problem (inflow pressure p_in(t) with
    amplitude dp and ramp time t_end on the left, zero on the right).
    geo 0: free flow [0,1]x[1,2] over the porous medium (Table 1); geo 1: the
    channel [-1,2]x[1,2] of Sec. 5's model problem over the same porous
    medium, the interface the middle third of its floor, walls beside it.
    """

    def __init__(self, n: int, mu: float, alpha: float, dt: float, K, bc: int = 0, dp: float = 1.0,
                 t_end: float = 1.0, geo: int = 0):
        K = _f64(K).reshape(n, n)
        self.n, self.mu, self.alpha, self.dt = n, float(mu), float(alpha), float(dt)
        self.bc, self.dp, self.t_end, self.geo = int(bc), float(dp), float(t_end), int(geo)
        self._lib = _load()
        self._c = self._lib.or_create_geo(n, self.mu, self.alpha, self.dt, _ptr(K), self.bc, self.dp, self.t_end,
                                          self.geo)
        if not self._c:
            raise ValueError("oracle: invalid parameters")
        self.ndof = int(self._lib.or_ndof(self._c))
        self.nnz = int(self._lib.or_nnz(self._c))
        self.factored = False

    def __del__(self):
        c = getattr(self, "_c", None)
        if c:
            self._lib.or_destroy(c)
            self._c = None

    def csr(self):
        rowptr = np.zeros(self.ndof + 1, dtype=np.int64)
        col = np.zeros(self.nnz, dtype=np.int32)
        val = np.zeros(self.nnz)
        self._lib.or_get_csr(self._c, _ptr(rowptr, ctypes.c_int64), _ptr(col, ctypes.c_int32), _ptr(val))
        return rowptr, col, val

    def scipy_csr(self):
        import scipy.sparse as sp
        rowptr, col, val = self.csr()
        return sp.csr_matrix((val, col, rowptr), shape=(self.ndof, self.ndof))

    def apply(self, x) -> np.ndarray:
        x = _f64(x)
        y = np.zeros(self.ndof)
        self._lib.or_apply(self._c, _ptr(x), _ptr(y))
        return y

    def rhs(self, xprev, t: float) -> np.ndarray:
        xprev = _f64(xprev)
        b = np.zeros(self.ndof)
        self._lib.or_rhs(self._c, _ptr(xprev), float(t), _ptr(b))
        return b

    def factor(self) -> None:
        info = self._lib.or_factor(self._c)
        if info != 0:
            raise RuntimeError("oracle: banded LU failed (info=%d)" % info)
        self.factored = True

    def bandwidth(self):
        kl, ku = ctypes.c_int(), ctypes.c_int()
        self._lib.or_bandwidth(self._c, ctypes.byref(kl), ctypes.byref(ku))
        return kl.value, ku.value

    def solve(self, b) -> np.ndarray:
        if not self.factored:
            self.factor()
        b = _f64(b)
        x = np.zeros(self.ndof)
        if self._lib.or_solve(self._c, _ptr(b), _ptr(x)) != 0:
            raise RuntimeError("oracle: solve without factorisation")
        return x

    def residual(self, x, b):
        x, b = _f64(x), _f64(b)
        r = np.zeros(self.ndof)
        nrm = self._lib.or_residual(self._c, _ptr(x), _ptr(b), _ptr(r))
        return r, float(nrm)

    def run(self, x0, t0: float, nsteps: int) -> np.ndarray:
        """nsteps implicit-Euler steps from state x0 at time t0."""
        if not self.factored:
            self.factor()
        x = _f64(x0).copy()
        if self._lib.or_run(self._c, _ptr(x), float(t0), int(nsteps)) != 0:
            raise RuntimeError("oracle: run failed")
        return x
