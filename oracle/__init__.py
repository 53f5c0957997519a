"""TEST INFRASTRUCTURE ONLY: Python access to the plain FP64 C oracle.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It loads ``oracle/_build/libucp_oracle.so``
(compiled by :func:`build`) through ctypes and exposes the oracle's functions
on numpy arrays.  Nothing here shares code with the CUDA library.

The oracle follows the paper's Section V-A problem statement (Witsenhausen's
counterexample), Corollary 1 (pointwise minimisation of the marginal cost),
eq. (2) (partial exhaustion over neighbouring samples), Section IV-A (Jacobi
parallelism over the grid) and the closed-form u1 = E[x1 | y1] of Section IV-C.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ucp_oracle.c")
_SRC2 = os.path.join(_HERE, "ucp_oracle2d.c")
_OUT = os.path.join(_HERE, "_build", "libucp_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: FP64, no fused multiply-add, OpenMP."""
    srcs = (_SRC, _SRC[:-1] + "h", _SRC2, _SRC2[:-1] + "h")
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= max(os.path.getmtime(x) for x in srcs)):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC, _SRC2, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


class _Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("sigma", ctypes.c_double),
                ("delta", ctypes.c_double), ("x_half", ctypes.c_double),
                ("w_half", ctypes.c_double), ("y_half", ctypes.c_double),
                ("cand_half", ctypes.c_double), ("n_coarse", ctypes.c_int32),
                ("n_refine", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("n_nbr", ctypes.c_int32), ("problem", ctypes.c_int32)]


class Alg1Report(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("local_iters", ctypes.c_int32), ("exhaustion_iters", ctypes.c_int32),
                ("N_L", ctypes.c_int32), ("N_P", ctypes.c_int32),
                ("J", ctypes.c_double), ("I_L", ctypes.c_double), ("I_P", ctypes.c_double)]


_lib = None


def build_variant(src_text: str, out_path: str) -> str:
    """Compile a variant of the oracle source (tests plant mistakes this way
    to check that the pins catch them)."""
    src = out_path[:-3] + ".c"
    with open(src, "w") as fh:
        fh.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", "-fopenmp", "-I", _HERE, "-o", out_path, src, _SRC2,
                    "-lm"], check=True)
    return out_path


def source() -> str:
    return open(_SRC).read()


def load_library(path: str):
    """ctypes handle of an oracle library at `path`, argument types set."""
    return _configure(ctypes.CDLL(path))


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(L):
    P = ctypes.POINTER(_Params)
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    L.orc_sizes.argtypes = [P, i64p, i64p, i64p, i64p, i32p]
    L.orc_grids.argtypes = [P, dp, dp, dp, dp, dp]
    L.orc_value.argtypes = [P, ctypes.c_int64]
    L.orc_value.restype = ctypes.c_double
    L.orc_init.argtypes = [P, ctypes.c_int, dp, i64p]
    L.orc_S.argtypes = [P, dp, ctypes.c_int64]
    L.orc_S.restype = ctypes.c_double
    L.orc_cost.argtypes = [P, dp, ctypes.c_int64, ctypes.c_int64]
    L.orc_cost.restype = ctypes.c_double
    L.orc_search.argtypes = [P, i64p, dp, i64p, i32p, ctypes.c_int64,
                             ctypes.c_int64]
    L.orc_candidates.argtypes = [P, i64p, dp, ctypes.c_int64, i64p, dp]
    L.orc_mmse.argtypes = [P, i64p, dp, ctypes.c_int64, ctypes.c_int64]
    L.orc_J.argtypes = [P, i64p, dp]
    L.orc_J.restype = ctypes.c_double
    L.orc_solve.argtypes = [P, ctypes.c_int, dp, ctypes.c_int, i64p, dp,
                            dp, i32p]
    L.orc_derivs.argtypes = [P, dp, ctypes.c_int64, ctypes.c_int64, dp, dp]
    L.orc_local_update.argtypes = [P, i64p, dp, ctypes.c_double, i64p, ctypes.c_int64,
                                   ctypes.c_int64]
    L.orc_split.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    L.orc_split.restype = ctypes.c_int
    L.orc_algorithm1.argtypes = [P, ctypes.c_int, dp, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int, i64p, dp, dp, i32p,
                                 ctypes.POINTER(Alg1Report)]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_get_threads.restype = ctypes.c_int
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


class Oracle:
    """One instance on the oracle: Witsenhausen's counterexample (problem 0,
    Section V-A) or zero-delay source-channel coding (problem 1, Section V-B).

    ``params`` is a mapping with keys k, sigma, delta, x_half, w_half, y_half,
    cand_half, n_coarse, n_refine, n_levels, n_nbr and optionally problem
    (default 0; extra keys are ignored).
    Controllers f are int64 lattice indices nu; ``value(nu)`` converts.
    """

    def __init__(self, params, library=None):
        self._L = library
        self.params = dict(params)
        self._p = _Params(*(float(params[k]) for k in
                            ("k", "sigma", "delta", "x_half", "w_half",
                             "y_half", "cand_half")),
                          *(int(params[k]) for k in
                            ("n_coarse", "n_refine", "n_levels", "n_nbr")),
                          int(params.get("problem", 0)))
        n = [ctypes.c_int64() for _ in range(4)]
        sh = ctypes.c_int32()
        if self._lib().orc_sizes(ctypes.byref(self._p), *(ctypes.byref(v) for v in n),
                           ctypes.byref(sh)) != 0:
            raise ValueError(f"invalid oracle parameters: {params}")
        self.n_x, self.n_w, self.n_y, self.n_cand = (v.value for v in n)
        self.shift = sh.value

    def _lib(self):
        return self._L if self._L is not None else lib()

    # -- grids ----------------------------------------------------------
    def grids(self):
        x = np.empty(self.n_x); px = np.empty(self.n_x)
        w = np.empty(self.n_w); phi = np.empty(self.n_w)
        y = np.empty(self.n_y)
        self._lib().orc_grids(ctypes.byref(self._p), _dp(x), _dp(px), _dp(w),
                        _dp(phi), _dp(y))
        return dict(x=x, px=px, w=w, phi=phi, y=y)

    def value(self, nu):
        nu = np.asarray(nu, dtype=np.int64)
        return np.ldexp(nu.astype(np.float64) * self.params["delta"], -self.shift)

    def init(self, kind: int, table=None):
        nu = np.empty(self.n_x, dtype=np.int64)
        tab = None if table is None else np.ascontiguousarray(table, np.float64)
        rc = self._lib().orc_init(ctypes.byref(self._p), int(kind),
                            _dp(tab) if tab is not None else None, _i64p(nu))
        if rc != 0:
            raise ValueError("oracle init failed")
        return nu

    # -- pieces of the sweep ------------------------------------------------
    def S(self, U, nu) -> float:
        U = np.ascontiguousarray(U, np.float64)
        return float(self._lib().orc_S(ctypes.byref(self._p), _dp(U), int(nu)))

    def cost(self, U, i, nu) -> float:
        U = np.ascontiguousarray(U, np.float64)
        return float(self._lib().orc_cost(ctypes.byref(self._p), _dp(U), int(i),
                                    int(nu)))

    def search(self, nu_pre, U, i0=0, i1=None):
        i1 = self.n_x if i1 is None else i1
        nu_pre = np.ascontiguousarray(nu_pre, np.int64)
        U = np.ascontiguousarray(U, np.float64)
        out = nu_pre.copy()
        idx = np.full(self.n_x, -1, dtype=np.int32)
        self._lib().orc_search(ctypes.byref(self._p), _i64p(nu_pre), _dp(U),
                         _i64p(out), _i32p(idx), int(i0), int(i1))
        return out, idx

    def candidates(self, nu_pre, U, i):
        nu_pre = np.ascontiguousarray(nu_pre, np.int64)
        U = np.ascontiguousarray(U, np.float64)
        nus = np.empty(self.n_cand, dtype=np.int64)
        gs = np.empty(self.n_cand)
        idx = self._lib().orc_candidates(ctypes.byref(self._p), _i64p(nu_pre), _dp(U),
                                   int(i), _i64p(nus), _dp(gs))
        return nus, gs, int(idx)

    def mmse(self, nu, j0=0, j1=None):
        j1 = self.n_y if j1 is None else j1
        nu = np.ascontiguousarray(nu, np.int64)
        U = np.full(self.n_y, np.nan)
        self._lib().orc_mmse(ctypes.byref(self._p), _i64p(nu), _dp(U), int(j0), int(j1))
        return U

    def J(self, nu, U) -> float:
        nu = np.ascontiguousarray(nu, np.int64)
        U = np.ascontiguousarray(U, np.float64)
        return float(self._lib().orc_J(ctypes.byref(self._p), _i64p(nu), _dp(U)))

    # -- Algorithm 1 (Sections III-B to III-D) ---------------------------
    def derivs(self, U, i, nu):
        """(g'/2, g''/2) of the marginal cost of u0 at x_i, u = value(nu)."""
        U = np.ascontiguousarray(U, np.float64)
        a, b = ctypes.c_double(), ctypes.c_double()
        if self._lib().orc_derivs(ctypes.byref(self._p), _dp(U), int(i), int(nu),
                                  ctypes.byref(a), ctypes.byref(b)) != 0:
            raise ValueError("invalid parameters")
        return a.value, b.value

    def local_update(self, nu_pre, U, tau=0.0, i0=0, i1=None):
        i1 = self.n_x if i1 is None else i1
        nu_pre = np.ascontiguousarray(nu_pre, np.int64)
        U = np.ascontiguousarray(U, np.float64)
        out = nu_pre.copy()
        self._lib().orc_local_update(ctypes.byref(self._p), _i64p(nu_pre), _dp(U),
                                     float(tau), _i64p(out), int(i0), int(i1))
        return out

    def split(self, I_L, I_P, N, n_l):
        return int(self._lib().orc_split(float(I_L), float(I_P), int(N), int(n_l)))

    def algorithm1(self, init_kind=0, N=20, precision=1e-10, tau=0.0, max_rounds=100,
                   table=None):
        nu = np.empty(self.n_x, dtype=np.int64)
        U = np.empty(self.n_y)
        Jp = np.full(1 + 2 * max_rounds, np.nan)
        NL = np.full(max_rounds, -1, dtype=np.int32)
        rep = Alg1Report()
        tab = None if table is None else np.ascontiguousarray(table, np.float64)
        rc = self._lib().orc_algorithm1(ctypes.byref(self._p), int(init_kind),
                                        _dp(tab) if tab is not None else None, int(N),
                                        float(precision), float(tau), int(max_rounds),
                                        _i64p(nu), _dp(U), _dp(Jp), _i32p(NL),
                                        ctypes.byref(rep))
        if rc != 0:
            raise ValueError("oracle algorithm1 failed")
        r = {k: getattr(rep, k) for k, _ in Alg1Report._fields_}
        n = r["rounds"]
        r.update(nu=nu, U=U, J_phase=Jp[:1 + 2 * n], N_L_rounds=NL[:n])
        return r

    def solve(self, init_kind: int, n_sweeps: int, table=None, want_idx=False):
        nu = np.empty(self.n_x, dtype=np.int64)
        U = np.empty(self.n_y)
        Jh = np.empty(n_sweeps + 1)
        idx = np.empty((n_sweeps, self.n_x), dtype=np.int32) if want_idx else None
        tab = None if table is None else np.ascontiguousarray(table, np.float64)
        rc = self._lib().orc_solve(ctypes.byref(self._p), int(init_kind),
                             _dp(tab) if tab is not None else None, int(n_sweeps),
                             _i64p(nu), _dp(U), _dp(Jh),
                             _i32p(idx) if idx is not None else None)
        if rc != 0:
            raise ValueError("oracle solve failed")
        return dict(nu=nu, U=U, J=Jh, idx=idx)


# ---- the 2-dimensional Witsenhausen counterexample (Section V-D) -----------

class _Params2(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("sigma", ctypes.c_double),
                ("delta", ctypes.c_double), ("x_half", ctypes.c_double),
                ("w_half", ctypes.c_double), ("y_half", ctypes.c_double),
                ("cand_half", ctypes.c_double), ("n_coarse", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("n_nbr", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


def _configure2(L):
    P = ctypes.POINTER(_Params2)
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    L.orc2_sizes.argtypes = [P, i64p, i64p, i64p, i64p, i32p]
    L.orc2_weights.argtypes = [P, dp, dp]
    L.orc2_init.argtypes = [P, ctypes.c_int, dp, i64p]
    L.orc2_S.argtypes = [P, dp, ctypes.c_int64, ctypes.c_int64]
    L.orc2_S.restype = ctypes.c_double
    L.orc2_cost.argtypes = [P, dp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
    L.orc2_cost.restype = ctypes.c_double
    L.orc2_search.argtypes = [P, i64p, dp, i64p, i32p, ctypes.c_int64, ctypes.c_int64]
    L.orc2_candidates.argtypes = [P, i64p, dp, ctypes.c_int64, i64p, dp]
    L.orc2_mmse.argtypes = [P, i64p, dp, ctypes.c_int64, ctypes.c_int64]
    L.orc2_J.argtypes = [P, i64p, dp]
    L.orc2_J.restype = ctypes.c_double
    return L


class Oracle2D:
    """One instance of the 2-D Witsenhausen counterexample on the oracle.
    ``params``: k, sigma, delta, x_half, w_half, y_half, cand_half, n_coarse,
    n_levels, n_nbr.  Controllers are int64 lattice indices of shape
    (n_x * n_x, 2); u1 tables are arrays of shape (n_y * n_y, 2)."""

    def __init__(self, params, library=None):
        self._L = library
        self.params = dict(params)
        self._p = _Params2(*(float(params[k]) for k in
                             ("k", "sigma", "delta", "x_half", "w_half", "y_half",
                              "cand_half")),
                           int(params["n_coarse"]), int(params["n_levels"]),
                           int(params["n_nbr"]), 0)
        n = [ctypes.c_int64() for _ in range(4)]
        sh = ctypes.c_int32()
        if self._lib().orc2_sizes(ctypes.byref(self._p), *(ctypes.byref(v) for v in n),
                                  ctypes.byref(sh)) != 0:
            raise ValueError(f"invalid 2-D oracle parameters: {params}")
        self.n_x, self.n_w, self.n_y, self.n_cand = (v.value for v in n)
        self.shift = sh.value
        self.N = self.n_x * self.n_x

    def _lib(self):
        L = self._L if self._L is not None else lib()
        if not getattr(L, "_orc2", False):
            _configure2(L)
            L._orc2 = True
        return L

    def value(self, nu):
        nu = np.asarray(nu, dtype=np.int64)
        return np.ldexp(nu.astype(np.float64) * self.params["delta"], -self.shift)

    def grid(self, n):
        return (np.arange(n) - (n - 1) // 2) * self.params["delta"]

    def weights(self):
        px = np.empty(self.N)
        phi = np.empty(self.n_w * self.n_w)
        self._lib().orc2_weights(ctypes.byref(self._p), _dp(px), _dp(phi))
        return px, phi

    def init(self, kind=0, table=None):
        nu = np.empty((self.N, 2), dtype=np.int64)
        tab = None if table is None else np.ascontiguousarray(table, np.float64)
        if self._lib().orc2_init(ctypes.byref(self._p), int(kind),
                                 _dp(tab) if tab is not None else None, _i64p(nu)) != 0:
            raise ValueError("2-D oracle init failed")
        return nu

    def S(self, U, nu1, nu2):
        U = np.ascontiguousarray(U, np.float64)
        return float(self._lib().orc2_S(ctypes.byref(self._p), _dp(U), int(nu1), int(nu2)))

    def cost(self, U, i, nu1, nu2):
        U = np.ascontiguousarray(U, np.float64)
        return float(self._lib().orc2_cost(ctypes.byref(self._p), _dp(U), int(i), int(nu1),
                                           int(nu2)))

    def search(self, nu_pre, U, i0=0, i1=None):
        i1 = self.N if i1 is None else i1
        nu_pre = np.ascontiguousarray(nu_pre, np.int64)
        U = np.ascontiguousarray(U, np.float64)
        out = nu_pre.copy()
        idx = np.full(self.N, -1, dtype=np.int32)
        self._lib().orc2_search(ctypes.byref(self._p), _i64p(nu_pre), _dp(U), _i64p(out),
                                _i32p(idx), int(i0), int(i1))
        return out, idx

    def candidates(self, nu_pre, U, i):
        nu_pre = np.ascontiguousarray(nu_pre, np.int64)
        U = np.ascontiguousarray(U, np.float64)
        nus = np.empty((self.n_cand, 2), dtype=np.int64)
        gs = np.empty(self.n_cand)
        k = self._lib().orc2_candidates(ctypes.byref(self._p), _i64p(nu_pre), _dp(U), int(i),
                                        _i64p(nus), _dp(gs))
        return nus, gs, int(k)

    def mmse(self, nu, t0=0, t1=None):
        t1 = self.n_y * self.n_y if t1 is None else t1
        nu = np.ascontiguousarray(nu, np.int64)
        U = np.full((self.n_y * self.n_y, 2), np.nan)
        self._lib().orc2_mmse(ctypes.byref(self._p), _i64p(nu), _dp(U), int(t0), int(t1))
        return U

    def J(self, nu, U):
        nu = np.ascontiguousarray(nu, np.int64)
        U = np.ascontiguousarray(U, np.float64)
        return float(self._lib().orc2_J(ctypes.byref(self._p), _i64p(nu), _dp(U)))

    def solve(self, n_sweeps, table=None):
        """init -> U = mmse(f) -> n_sweeps x {search, mmse, J}."""
        nu = self.init(0 if table is None else 2, table)
        U = self.mmse(nu)
        Jh = [self.J(nu, U)]
        idx = None
        for _ in range(n_sweeps):
            nu, idx = self.search(nu, U)
            U = self.mmse(nu)
            Jh.append(self.J(nu, U))
        return dict(nu=nu, U=U, J=np.array(Jh), idx=idx)
