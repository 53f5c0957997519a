"""Thin Python binding of libucp.so (C ABI in include/ucp.h).

Argument marshalling only: every step of the sweep runs in the library's CUDA
kernels.  PyTorch supplies the CUDA stream and, through the allocator hooks,
the device memory (its caching allocator).  The library must have been built
(``__graft_entry__.build()`` or ``python -m paper_1908_04489_gb300.build``);
if it is missing, loading raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

UCP_OK, UCP_PENDING = 0, 1
STATUS = {0: "UCP_OK", 1: "UCP_PENDING", -1: "UCP_E_ARG", -2: "UCP_E_NOMEM",
          -3: "UCP_E_BUDGET", -4: "UCP_E_CUDA", -5: "UCP_E_TIMEOUT",
          -6: "UCP_E_STATE", -7: "UCP_E_NOTFOUND"}


class UcpError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} {detail}".strip())


class Params(ctypes.Structure):
    """Mirror of ``ucp_params``."""
    _fields_ = [("k", ctypes.c_double), ("sigma", ctypes.c_double),
                ("delta", ctypes.c_double), ("x_half", ctypes.c_double),
                ("w_half", ctypes.c_double), ("y_half", ctypes.c_double),
                ("cand_half", ctypes.c_double), ("n_coarse", ctypes.c_int32),
                ("n_refine", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("n_nbr", ctypes.c_int32), ("init_kind", ctypes.c_int32),
                ("precision", ctypes.c_int32),
                ("init_table", ctypes.POINTER(ctypes.c_double)),
                ("init_len", ctypes.c_uint64), ("flags", ctypes.c_uint64),
                ("problem", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    @classmethod
    def from_dict(cls, p, table=None):
        obj = cls(float(p["k"]), float(p["sigma"]), float(p["delta"]),
                  float(p["x_half"]), float(p["w_half"]), float(p["y_half"]),
                  float(p["cand_half"]), int(p["n_coarse"]), int(p["n_refine"]),
                  int(p["n_levels"]), int(p["n_nbr"]), int(p.get("init_kind", 0)),
                  int(p.get("precision", 0)), None, 0, int(p.get("flags", 0)),
                  int(p.get("problem", 0)), 0)
        if table is not None:
            obj._table = np.ascontiguousarray(table, dtype=np.float64)
            obj.init_table = obj._table.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            obj.init_len = obj._table.size
        return obj


class Result(ctypes.Structure):
    """Mirror of ``ucp_result``."""
    _fields_ = [("J", ctypes.c_double), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("sweeps", ctypes.c_int32), ("status", ctypes.c_int32)]


class SrvInfo(ctypes.Structure):
    """Mirror of ``ucp_srv_info``."""
    _fields_ = [("queued", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("max_active", ctypes.c_int32), ("bytes_in_use", ctypes.c_uint64),
                ("now", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u64p = ctypes.POINTER(ctypes.c_uint64)
_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)


class SolveParams(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("precision", ctypes.c_double), ("tau", ctypes.c_double)]


class SolveReport(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("local_iters", ctypes.c_int32), ("exhaustion_iters", ctypes.c_int32),
                ("N_L", ctypes.c_int32), ("N_P", ctypes.c_int32),
                ("J", ctypes.c_double), ("I_L", ctypes.c_double), ("I_P", ctypes.c_double)]


class LaunchConfig(ctypes.Structure):
    _fields_ = [("search_lanes", ctypes.c_int32), ("u1_threads", ctypes.c_int32 * 5),
                ("defer_blocks", ctypes.c_int32)]

    @classmethod
    def from_dict(cls, d):
        c = cls()
        c.search_lanes = int(d.get("search_lanes", 0))
        for r, v in enumerate(d.get("u1_threads", [0] * 5)):
            c.u1_threads[r] = int(v)
        c.defer_blocks = int(d.get("defer_blocks", 0))
        return c


class Params2(ctypes.Structure):
    """ucp2_params: the 2-dimensional problem of Section V-D."""
    _fields_ = [("k", ctypes.c_double), ("sigma", ctypes.c_double), ("delta", ctypes.c_double),
                ("x_half", ctypes.c_double), ("w_half", ctypes.c_double),
                ("y_half", ctypes.c_double), ("cand_half", ctypes.c_double),
                ("n_coarse", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("n_nbr", ctypes.c_int32), ("direct", ctypes.c_int32)]

    @classmethod
    def from_dict(cls, d):
        c = cls()
        for name, _ in cls._fields_:
            setattr(c, name, d.get(name, 0) if name == "direct" else d[name])
        return c


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libucp.so; raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libucp.so is not built ({path}); run "
                           "__graft_entry__.build() first")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(Params)
    L.ucp_status_str.argtypes = [ctypes.c_int]
    L.ucp_status_str.restype = ctypes.c_char_p
    L.ucp_last_error.restype = ctypes.c_char_p
    L.ucp_version.restype = ctypes.c_char_p
    L.ucp_plan.argtypes = [P, _u64p, _u64p, _u64p, _u64p, _u64p]
    L.ucp_ctx_create.argtypes = [ctypes.c_int32, ALLOC_FN, FREE_FN, _vp,
                                 ctypes.POINTER(_vp)]
    L.ucp_ctx_destroy.argtypes = [_vp]
    L.ucp_create.argtypes = [_vp, P, _vp, ctypes.POINTER(_vp)]
    L.ucp_sizes.argtypes = [_vp, _u64p, _u64p, _u64p, _u64p, _u64p]
    L.ucp_sweep.argtypes = [_vp, ctypes.c_int32]
    L.ucp_eval_J.argtypes = [_vp, _dp]
    L.ucp_J_history.argtypes = [_vp, _dp, _u64, _u64p]
    L.ucp_get_controllers.argtypes = [_vp, _dp, _u64, _dp, _u64, ctypes.c_int32,
                                      _i32p]
    L.ucp_set_controllers.argtypes = [_vp, _dp, _u64, _dp, _u64]
    L.ucp_destroy.argtypes = [_vp]
    L.ucp_profile.argtypes = [_vp, ctypes.c_int32]
    L.ucp_kernel_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_char_p),
                                   ctypes.POINTER(ctypes.c_int64), _dp,
                                   ctypes.c_int32]
    L.ucp_kernel_times.restype = ctypes.c_int32
    L.ucp_tie_recosts.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
    L.ucp_get_tables.argtypes = [_vp, _dp, _dp, _dp, ctypes.c_int64,
                                 ctypes.POINTER(ctypes.c_float), ctypes.c_int64,
                                 ctypes.POINTER(ctypes.c_int64)]
    L.ucp_probe_alu.argtypes = [_dp, _dp, _dp, _vp]
    L.ucp_work_counters.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.c_int32]
    L.ucp_srv_create.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int32, _vp,
                                 ctypes.POINTER(_vp)]
    L.ucp_submit.argtypes = [_vp, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]
    L.ucp_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(Result), _dp, _u64,
                           _dp, _u64]
    L.ucp_srv_stats.argtypes = [_vp, ctypes.POINTER(SrvInfo)]
    L.ucp_srv_fail_next_step.argtypes = [_vp]
    L.ucp_srv_destroy.argtypes = [_vp]
    L.ucp_batch_create.argtypes = [_vp, P, ctypes.c_int32, _vp, ctypes.POINTER(_vp)]
    L.ucp_batch_sweep.argtypes = [_vp, ctypes.c_int32]
    L.ucp_batch_eval_J.argtypes = [_vp, _dp]
    L.ucp_batch_instance.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(_vp)]
    L.ucp_batch_destroy.argtypes = [_vp]
    L.ucp_batch_profile.argtypes = [_vp, ctypes.c_int32]
    L.ucp_batch_kernel_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_char_p),
                                         ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int32]
    L.ucp_batch_kernel_times.restype = ctypes.c_int32
    L.ucp_local_update.argtypes = [_vp, ctypes.c_int32, ctypes.c_double]
    L.ucp_sweep_part.argtypes = [_vp, ctypes.c_int64, ctypes.c_int64, _dp]
    L.ucp_set_launch_config.argtypes = [_vp, ctypes.POINTER(LaunchConfig)]
    L.ucp_ctx_set_launch_config.argtypes = [_vp, ctypes.POINTER(LaunchConfig)]
    L.ucp_batch_set_launch_config.argtypes = [_vp, ctypes.POINTER(LaunchConfig)]
    L.ucp_sweep_finish.argtypes = [_vp, _dp, _u64]
    L.ucp_solve.argtypes = [_vp, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveReport),
                            _dp, _i32p]
    P2 = ctypes.POINTER(Params2)
    L.ucp2_plan.argtypes = [P2, _u64p, _u64p, _u64p, _u64p]
    L.ucp2_create.argtypes = [_vp, P2, _dp, _vp, ctypes.POINTER(_vp)]
    L.ucp2_sweep.argtypes = [_vp, ctypes.c_int32]
    L.ucp2_J_history.argtypes = [_vp, _dp, _u64, _u64p]
    L.ucp2_get_controllers.argtypes = [_vp, _dp, _u64, _dp, _u64, _i32p, _u64]
    L.ucp2_set_controllers.argtypes = [_vp, _dp, _u64, _dp, _u64]
    L.ucp2_destroy.argtypes = [_vp]
    L.ucp2_profile.argtypes = [_vp, ctypes.c_int32]
    L.ucp2_kernel_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_char_p),
                                    ctypes.POINTER(ctypes.c_int64), _dp, ctypes.c_int32]
    L.ucp2_kernel_times.restype = ctypes.c_int32
    L.ucp2_work_counters.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
    _lib = L
    return L


def _check(st, where):
    if st != UCP_OK:
        detail = load().ucp_last_error().decode(errors="replace")
        raise UcpError(st, where, detail)


def _ptr(a, typ):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(typ))


def plan(params, table=None) -> dict:
    """Validate parameters on the host (no GPU needed): sizes and bytes.
    table: the initial controller table of an init_kind 2 start."""
    L = load()
    v = [ctypes.c_uint64() for _ in range(5)]
    _check(L.ucp_plan(ctypes.byref(Params.from_dict(params, table)),
                      *(ctypes.byref(x) for x in v)), "ucp_plan")
    return dict(zip(("n_x", "n_w", "n_y", "n_cand", "device_bytes"),
                    (x.value for x in v)))


def probe_alu(stream=None) -> dict:
    """Measured FP64 / FP32 FMA TFLOP/s and FP32 ex2 Gop/s of this GPU."""
    v = [ctypes.c_double() for _ in range(3)]
    sp = getattr(stream, "cuda_stream", stream)
    _check(load().ucp_probe_alu(*(ctypes.byref(x) for x in v), _vp(sp)),
           "ucp_probe_alu")
    return dict(zip(("fp64_tflops", "fp32_tflops", "ex2_gops"),
                    (x.value for x in v)))


class Context:
    """ucp_ctx bound to a CUDA device, with PyTorch's caching allocator."""

    def __init__(self, device: int | None = None, use_torch_allocator=True):
        import torch
        L = load()
        self.device = torch.cuda.current_device() if device is None else device
        self._alloc = self._free = None
        if use_torch_allocator:
            dev = self.device

            def _a(n, user):
                try:
                    return torch.cuda.caching_allocator_alloc(
                        int(n), dev, torch.cuda.current_stream(dev))
                except RuntimeError:
                    return None

            def _f(p, user):
                torch.cuda.caching_allocator_delete(p)

            self._alloc, self._free = ALLOC_FN(_a), FREE_FN(_f)
        else:
            self._alloc = ctypes.cast(None, ALLOC_FN)
            self._free = ctypes.cast(None, FREE_FN)
        h = _vp()
        _check(L.ucp_ctx_create(self.device, self._alloc, self._free, None,
                                ctypes.byref(h)), "ucp_ctx_create")
        self.h = h

    def set_launch_config(self, cfg: dict):
        """Launch shapes that instances and batches created on this context
        afterwards start with (``ucp_ctx_set_launch_config``)."""
        c = LaunchConfig.from_dict(cfg)
        _check(load().ucp_ctx_set_launch_config(self.h, ctypes.byref(c)),
               "ucp_ctx_set_launch_config")

    def close(self):
        if self.h:
            load().ucp_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx = None


def default_context() -> Context:
    global _default_ctx
    if _default_ctx is None:
        _default_ctx = Context()
    return _default_ctx


class Instance:
    """One Witsenhausen instance (``ucp_create`` ... ``ucp_destroy``)."""

    def __init__(self, params, table=None, stream=None, ctx: Context | None = None):
        import torch
        L = load()
        self.ctx = ctx or default_context()
        self.params = dict(params)
        if stream is None:
            stream = torch.cuda.current_stream(self.ctx.device)
        self.stream = stream
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        h = _vp()
        self._p = Params.from_dict(params, table)
        _check(L.ucp_create(self.ctx.h, ctypes.byref(self._p), _vp(sp),
                            ctypes.byref(h)), "ucp_create")
        self.h = h
        v = [ctypes.c_uint64() for _ in range(5)]
        _check(L.ucp_sizes(h, *(ctypes.byref(x) for x in v)), "ucp_sizes")
        self.n_x, self.n_w, self.n_y, self.n_cand, self.device_bytes = \
            (x.value for x in v)

    def sweep(self, n: int = 1):
        _check(load().ucp_sweep(self.h, int(n)), "ucp_sweep")

    def eval_J(self) -> float:
        J = ctypes.c_double()
        _check(load().ucp_eval_J(self.h, ctypes.byref(J)), "ucp_eval_J")
        return J.value

    def J_history(self, n: int = 1 << 20) -> np.ndarray:
        out = np.empty(n)
        m = ctypes.c_uint64()
        _check(load().ucp_J_history(self.h, _ptr(out, ctypes.c_double), n,
                                    ctypes.byref(m)), "ucp_J_history")
        return out[:m.value]

    def get_controllers(self, as_paper_u0=False, want=("f", "U", "idx")):
        f = np.empty(self.n_x) if "f" in want else None
        U = np.empty(self.n_y) if "U" in want else None
        idx = np.empty(self.n_x, dtype=np.int32) if "idx" in want else None
        _check(load().ucp_get_controllers(
            self.h, _ptr(f, ctypes.c_double), self.n_x,
            _ptr(U, ctypes.c_double), self.n_y, int(bool(as_paper_u0)),
            _ptr(idx, ctypes.c_int32)), "ucp_get_controllers")
        return dict(f=f, U=U, idx=idx)

    def set_controllers(self, f, U=None):
        f = np.ascontiguousarray(f, dtype=np.float64)
        U = None if U is None else np.ascontiguousarray(U, dtype=np.float64)
        _check(load().ucp_set_controllers(
            self.h, _ptr(f, ctypes.c_double), f.size, _ptr(U, ctypes.c_double),
            0 if U is None else U.size), "ucp_set_controllers")

    def profile(self, on=True):
        _check(load().ucp_profile(self.h, int(bool(on))), "ucp_profile")

    def kernel_times(self) -> dict:
        L = load()
        cap = 64
        names = (ctypes.c_char_p * cap)()
        launches = (ctypes.c_int64 * cap)()
        ms = (ctypes.c_double * cap)()
        n = L.ucp_kernel_times(self.h, names, launches, ms, cap)
        return {names[k].decode(): (launches[k], ms[k]) for k in range(min(n, cap))}

    COUNTERS = ("recosts", "u1_pairs", "u1_boxes", "u1_df_terms", "u1_f32_terms",
                "direct_costs")

    def work_counters(self) -> dict:
        out = (ctypes.c_int64 * len(self.COUNTERS))()
        _check(load().ucp_work_counters(self.h, out, len(self.COUNTERS)),
               "ucp_work_counters")
        return dict(zip(self.COUNTERS, (int(v) for v in out)))

    def get_tables(self) -> dict:
        """Correlation tables P, Q, R of the current u1 table, the per-column
        error bound of the table identity, and the index offsets (c_lo: lattice
        cell of position 0; jlo: y-index of E-index 0)."""
        L = load()
        sz = (ctypes.c_int64 * 4)()
        _check(L.ucp_get_tables(self.h, None, None, None, 0, None, 0, sz), "ucp_get_tables")
        n_pos, n_cols = int(sz[0]), int(sz[1])
        P, Q, R = (np.empty(n_pos) for _ in range(3))
        bt = np.empty(n_cols, dtype=np.float32)
        _check(L.ucp_get_tables(self.h, _ptr(P, ctypes.c_double), _ptr(Q, ctypes.c_double),
                                _ptr(R, ctypes.c_double), n_pos,
                                bt.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                n_cols, sz), "ucp_get_tables")
        return {"P": P, "Q": Q, "R": R, "bound": bt, "c_lo": int(sz[2]), "jlo": int(sz[3])}

    def set_launch_config(self, cfg: dict):
        """Launch shapes of later sweeps (``ucp_set_launch_config``): keys
        search_lanes, u1_threads (5 entries), defer_blocks; 0 = the rule."""
        c = LaunchConfig.from_dict(cfg)
        _check(load().ucp_set_launch_config(self.h, ctypes.byref(c)), "ucp_set_launch_config")

    def sweep_part(self, i0: int, i1: int) -> np.ndarray:
        """The search of x0 points i0..i1-1; their new f (``ucp_sweep_part``)."""
        out = np.empty(max(0, int(i1) - int(i0)))
        _check(load().ucp_sweep_part(self.h, int(i0), int(i1), _ptr(out, ctypes.c_double)),
               "ucp_sweep_part")
        return out

    def sweep_finish(self, f):
        """The whole new f, then the rest of the sweep (``ucp_sweep_finish``)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        _check(load().ucp_sweep_finish(self.h, _ptr(f, ctypes.c_double), f.size),
               "ucp_sweep_finish")

    def local_update(self, n: int = 1, tau: float = 0.0):
        """n local-update iterations of Algorithm 1 (``ucp_local_update``)."""
        _check(load().ucp_local_update(self.h, int(n), float(tau)), "ucp_local_update")

    def solve(self, N=20, precision=1e-10, tau=0.0, max_rounds=100) -> dict:
        """Algorithm 1's outer loop from the current state (``ucp_solve``):
        the report, J after every phase and N_L of every round."""
        sp = SolveParams(int(N), int(max_rounds), float(precision), float(tau))
        rep = SolveReport()
        cap = max(0, int(max_rounds))       # the library rejects a negative count
        Jp = np.full(1 + 2 * cap, np.nan)
        NL = np.full(max(1, cap), -1, dtype=np.int32)
        _check(load().ucp_solve(self.h, ctypes.byref(sp), ctypes.byref(rep),
                                _ptr(Jp, ctypes.c_double), _ptr(NL, ctypes.c_int32)),
               "ucp_solve")
        r = {k: getattr(rep, k) for k, _ in SolveReport._fields_}
        n = r["rounds"]
        r.update(J_phase=Jp[:1 + 2 * n], N_L_rounds=NL[:n])
        return r

    def tie_recosts(self) -> int:
        v = ctypes.c_int64()
        _check(load().ucp_tie_recosts(self.h, ctypes.byref(v)), "ucp_tie_recosts")
        return v.value

    def close(self):
        if getattr(self, "h", None):
            _check(load().ucp_destroy(self.h), "ucp_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan2(params) -> dict:
    """Sizes of a 2-dimensional instance (host only)."""
    v = [ctypes.c_uint64() for _ in range(4)]
    _check(load().ucp2_plan(ctypes.byref(Params2.from_dict(params)),
                            *(ctypes.byref(x) for x in v)), "ucp2_plan")
    return dict(zip(("n_x", "n_w", "n_y", "n_cand"), (x.value for x in v)))


class Instance2D:
    """One instance of the 2-dimensional counterexample (``ucp2_create`` ...
    ``ucp2_destroy``).  f has shape (n_x^2, 2), the u1 tables (n_y^2, 2),
    both over flat grid indices a n + b."""

    def __init__(self, params, init_f=None, stream=None, ctx: Context | None = None):
        import torch
        L = load()
        self.ctx = ctx or default_context()
        self.params = dict(params)
        if stream is None:
            stream = torch.cuda.current_stream(self.ctx.device)
        self.stream = stream
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        sizes = plan2(params)
        self.n_x, self.n_w, self.n_y, self.n_cand = (sizes[k] for k in
                                                      ("n_x", "n_w", "n_y", "n_cand"))
        f0 = None
        if init_f is not None:
            f0 = np.ascontiguousarray(init_f, dtype=np.float64).reshape(-1)
            if f0.size != 2 * self.n_x ** 2:
                raise ValueError(f"init_f needs {2 * self.n_x ** 2} values, got {f0.size}")
        h = _vp()
        self._p = Params2.from_dict(params)
        _check(L.ucp2_create(self.ctx.h, ctypes.byref(self._p), _ptr(f0, ctypes.c_double),
                             _vp(sp), ctypes.byref(h)), "ucp2_create")
        self.h = h

    def sweep(self, n: int = 1):
        _check(load().ucp2_sweep(self.h, int(n)), "ucp2_sweep")

    def J_history(self, n: int = 1 << 16) -> np.ndarray:
        out = np.empty(n)
        m = ctypes.c_uint64()
        _check(load().ucp2_J_history(self.h, _ptr(out, ctypes.c_double), n,
                                     ctypes.byref(m)), "ucp2_J_history")
        return out[:m.value]

    def get_controllers(self, want=("f", "U", "idx")):
        nx2, ny2 = self.n_x ** 2, self.n_y ** 2
        f = np.empty((nx2, 2)) if "f" in want else None
        U = np.empty((ny2, 2)) if "U" in want else None
        idx = np.empty(nx2, dtype=np.int32) if "idx" in want else None
        _check(load().ucp2_get_controllers(
            self.h, _ptr(f, ctypes.c_double), 2 * nx2, _ptr(U, ctypes.c_double), 2 * ny2,
            _ptr(idx, ctypes.c_int32), nx2), "ucp2_get_controllers")
        return dict(f=f, U=U, idx=idx)

    def profile(self, on=True):
        _check(load().ucp2_profile(self.h, int(bool(on))), "ucp2_profile")

    def kernel_times(self, cap=32) -> dict:
        """{group: (launches, total ms)} of the profiled sweeps."""
        names = (ctypes.c_char_p * cap)()
        launches = (ctypes.c_int64 * cap)()
        ms = (ctypes.c_double * cap)()
        n = load().ucp2_kernel_times(self.h, names, launches, ms, cap)
        if n < 0:
            raise UcpError(-4, "ucp2_kernel_times", "")
        return {names[k].decode(): (launches[k], ms[k]) for k in range(min(n, cap))}

    def work_counters(self) -> dict:
        v = ctypes.c_int64()
        _check(load().ucp2_work_counters(self.h, ctypes.byref(v)), "ucp2_work_counters")
        return {"u1_live_pairs": v.value}

    def set_controllers(self, f, U=None):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        U = None if U is None else np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
        _check(load().ucp2_set_controllers(
            self.h, _ptr(f, ctypes.c_double), f.size, _ptr(U, ctypes.c_double),
            0 if U is None else U.size), "ucp2_set_controllers")

    def close(self):
        if getattr(self, "h", None):
            load().ucp2_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Member(Instance):
    """A batch member viewed as an instance (owned by the batch)."""

    def __init__(self, handle, params):
        self.h = handle
        self.params = dict(params)
        v = [ctypes.c_uint64() for _ in range(5)]
        _check(load().ucp_sizes(handle, *(ctypes.byref(x) for x in v)), "ucp_sizes")
        self.n_x, self.n_w, self.n_y, self.n_cand, self.device_bytes = \
            (x.value for x in v)

    def close(self):
        self.h = None   # the batch destroys its members


class Batch:
    """Many instances swept together (``ucp_batch_*``)."""

    def __init__(self, params_list, stream=None, ctx: Context | None = None, tables=None):
        """tables: None, or one entry per member: None or the member's initial
        controller table (members with init_kind 2)."""
        import torch
        L = load()
        self.ctx = ctx or default_context()
        self.params = [dict(p) for p in params_list]
        if stream is None:
            stream = torch.cuda.current_stream(self.ctx.device)
        self.stream = stream
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        tables = tables or [None] * len(self.params)
        # the Params objects own the table arrays until the call returns
        objs = [Params.from_dict(p, t) for p, t in zip(self.params, tables)]
        arr = (Params * len(self.params))(*objs)
        h = _vp()
        _check(L.ucp_batch_create(self.ctx.h, arr, len(self.params), _vp(sp),
                                  ctypes.byref(h)), "ucp_batch_create")
        self.h = h
        self.members = []
        for k, p in enumerate(self.params):
            m = _vp()
            _check(L.ucp_batch_instance(h, k, ctypes.byref(m)), "ucp_batch_instance")
            self.members.append(_Member(m, p))

    def sweep(self, n: int = 1):
        _check(load().ucp_batch_sweep(self.h, int(n)), "ucp_batch_sweep")

    def profile(self, on=True):
        _check(load().ucp_batch_profile(self.h, int(bool(on))), "ucp_batch_profile")

    def kernel_times(self) -> dict:
        cap = 64
        names = (ctypes.c_char_p * cap)()
        launches = (ctypes.c_int64 * cap)()
        ms = (ctypes.c_double * cap)()
        n = load().ucp_batch_kernel_times(self.h, names, launches, ms, cap)
        return {names[k].decode(): (launches[k], ms[k]) for k in range(min(n, cap))}

    def set_launch_config(self, cfg: dict):
        """Launch shapes of later batched sweeps (``ucp_batch_set_launch_config``)."""
        c = LaunchConfig.from_dict(cfg)
        _check(load().ucp_batch_set_launch_config(self.h, ctypes.byref(c)),
               "ucp_batch_set_launch_config")

    def eval_J(self) -> np.ndarray:
        out = np.empty(len(self.params))
        _check(load().ucp_batch_eval_J(self.h, _ptr(out, ctypes.c_double)),
               "ucp_batch_eval_J")
        return out

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.h = None
            _check(load().ucp_batch_destroy(self.h), "ucp_batch_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (``ucp_srv_*``, ``ucp_submit``,
    ``ucp_poll``)."""

    def __init__(self, hbm_budget_bytes=8 << 30, max_slots=256, stream=None,
                 ctx: Context | None = None):
        import torch
        L = load()
        self.ctx = ctx or default_context()
        if stream is None:
            stream = torch.cuda.Stream(self.ctx.device)
        self.stream = stream
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        h = _vp()
        _check(L.ucp_srv_create(self.ctx.h, int(hbm_budget_bytes), int(max_slots),
                                _vp(sp), ctypes.byref(h)), "ucp_srv_create")
        self.h = h
        self._sizes = {}

    def submit(self, params, sweeps=None, table=None) -> int:
        p = Params.from_dict(params, table)
        t = ctypes.c_uint64()
        n = int(params.get("sweeps", 0) if sweeps is None else sweeps)
        _check(load().ucp_submit(self.h, ctypes.byref(p), n, ctypes.byref(t)),
               "ucp_submit")
        pl = plan(params, table)
        self._sizes[t.value] = (pl["n_x"], pl["n_y"])
        return t.value

    def poll(self, ticket, want_arrays=True):
        """None while pending; else a dict with J, times, f, U."""
        nx, ny = self._sizes.get(ticket, (0, 0))
        f = np.empty(nx) if want_arrays else None
        U = np.empty(ny) if want_arrays else None
        res = Result()
        st = load().ucp_poll(self.h, ticket, ctypes.byref(res), _ptr(f, ctypes.c_double),
                             nx, _ptr(U, ctypes.c_double), ny)
        if st == UCP_PENDING:
            return None
        self._sizes.pop(ticket, None)
        _check(st, "ucp_poll")
        return dict(J=res.J, t_submit=res.t_submit, t_admit=res.t_admit,
                    t_done=res.t_done, sweeps=res.sweeps, f=f, U=U)

    def stats(self) -> dict:
        info = SrvInfo()
        _check(load().ucp_srv_stats(self.h, ctypes.byref(info)), "ucp_srv_stats")
        return {k: getattr(info, k) for k, _ in SrvInfo._fields_}

    def fail_next_step(self):
        _check(load().ucp_srv_fail_next_step(self.h), "ucp_srv_fail_next_step")

    def close(self):
        if getattr(self, "h", None):
            st = load().ucp_srv_destroy(self.h)
            self.h = None
            return st
        return 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
