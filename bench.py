"""Benchmark: UCP solves/s of the Witsenhausen sweep on GB300.

Workload (default): the fine single instance -- k = 0.2, sigma = 5,
delta = 0.005 (10001 x0 / 2401 w / 14001 y points), odd 3-step staircase init,
64 coarse candidates then 4 levels of 16, 50 sweeps.  One step = one whole
solve: setup (grids, weights, init, u1, J) + 50 sweeps, every step of the
path in the library's kernels.

  value        -- solves/s with the instance set up on the device inside the
                  timed region (CUDA events on the instance stream; L2 flushed
                  between steps by a 512 MiB write outside the events).
  e2e          -- solves/s through the C ABI from host buffers: the initial
                  controller table goes host->device, f and u1 come back, J is
                  read.
  parity       -- the FP64 C oracle's own whole solve of the same workload
                  (all host cores) against the GPU's: J after every sweep,
                  the final controllers.
  cpu_baseline -- that oracle solve's time (a whole solve, not a sample).
  --impl reference -- the oracle on the host cores, each step a bounded
                  sample of one solve (its share of the solve stated).
  roofline     -- the dominant kernel's algorithmic work (the method's
                  arithmetic, not the instructions that emulate its precision)
                  per CUDA-event-timed launch, against the measured peak of
                  the pipe it runs on; "issued" gives the emulation count.

Under torchrun every rank solves its own copy (independent problems, no
collective): weak scaling, value = all solves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("UCP solves/s at |ΔJ|≤1e-9 vs FP64 oracle (batched vs plain GPU); "
          "p50/p99 latency")
UNIT = "solves/s"


def workload(name: str, precision: int):
    from paper_1908_04489_gb300 import workloads as W
    if name == "c2":
        return W.c2(precision=precision), (
            "c2: single Witsenhausen instance k=0.2 sigma=5, delta=0.005 "
            "(10001 x0 / 2401 w / 14001 y), staircase init, 64 coarse + 4x16 "
            "refine, 50 sweeps")
    if name == "c1":
        return W.c1() | {"precision": precision}, (
            "c1: k=0.2 sigma=5, delta=0.05 (1001/241/1401), identity init, "
            "10 sweeps")
    if name == "sc":
        return W.source_channel(), (
            "zero-delay source-channel coding (Section V-B): lambda=2, x0 ~ N(0,1), "
            "w ~ U(-1,1), delta=0.02 (501/101/701), identity init, 20 sweeps, plain FP64")
    if name == "c5":
        return W.c5(precision=precision), (
            "c5: k=0.2 sigma=10, delta=0.001 (100001/14001/120001), 6 levels, "
            "identity init, 20 sweeps")
    raise SystemExit(f"unknown workload {name}")


def init_table(p):
    """Host-side initial controller f of the workload's start (identity for
    init_kind 0, the staircase for init_kind 1) for the end-to-end leg, which
    passes it through init_kind 2 (the same lattice values)."""
    d = p["delta"]
    n = int(round(2 * p["x_half"] / d)) + 1
    a = np.arange(n) - (n - 1) // 2
    if p["init_kind"] == 0:
        return a * d
    m = np.minimum(np.abs(a) // int(round(7.0 / d)), 2)
    return np.where(a == 0, 0.0, np.sign(a) * 3.5 * (2 * m + 1))


# ---- work per kernel launch -------------------------------------------------
# Two counts per kernel.  "algorithmic": the method's own arithmetic as this
# path formulates it, 2 flops per multiply-add:
#   search  per (x_i, candidate) 19: S(u) from the three correlation tables at
#           the candidate's position (1 - t, the two P terms, the three Q/R
#           products and their weights, the sums: 15) plus k^2 (u - x)^2 and
#           the sum (4);
#   tables  per (table, position, tap) 2: P, Q and R are three correlations of
#           n_pos positions over n_w taps;
#   u1 sums per Taylor term evaluated 2 (one Horner step), per directly summed
#           (source, target) pair 8 (the weight's exponent, two accumulations)
#           plus one exp counted apart; the terms come from device counters.
# "issued": what the precision emulation costs on the pipe it runs on --
#   tables  bf16 tensor products as issued: 21 products of the six 8-bit
#           slices per operand, per table, 64-column group and 128-tap chunk,
#           M = 128 x N = 64 x K = 128;
#   double-float kernels in FP32 flops of their double-float operations
#           (FADD/FMUL 1, FFMA 2; df_add 11, df_mul 10, product-accumulate 18):
#           search 104 per candidate (the screened evaluation and its bound);
#           u1 per direct pair 39 and per (source, run) 130, per Taylor
#           (box, run) 130 + 63 per target, per Taylor term 21 (double-float)
#           or 2 (FP32).
# The plain FP64 path counts FP64 flops: 6 per quadrature term.
TC_PRODUCTS = 21
ALG_SEARCH_CAND = 19.0
ALG_TABLE_TAP = 2.0
ALG_U1_TERM = 2.0
ALG_U1_PAIR = 8.0
FLOPS_U1_PAIR = 39.0
FLOPS_U1_ANCHOR = 130.0
FLOPS_U1_BOX_TARGET = 63.0
FLOPS_U1_TERM_DF = 21.0
FLOPS_U1_TERM_F32 = 2.0
FLOPS_SEARCH_CAND = 104.0

# DRAM bytes per launch from one-kernel ncu captures of the current kernels
# (dram__bytes_read.sum + dram__bytes_write.sum; cold cache), keyed by the
# profiled kernel group; None where the kernel changed since its capture.
TRAFFIC_BYTES = {"c2": {"search": 0.264e6, "tables": 1.70e6, "mmse_main": 0.074e6}}
TRAFFIC_SOURCE = "profiles/hot_kernels_c2_ncu_full.md"

# kernels launched per timed group of the library's profiler (the groups not
# listed launch one kernel), and the instance set-up launches of one solve
# (weights 3, coarse list, fast set-up, filter slices and W2, init, the first
# u1 step 4, tables 3, J), which run before the profiler is switched on
KERNELS_PER_GROUP = {"search": 2}
SETUP_LAUNCHES = 15

WORK_MODEL = {
    "search": "19 flops per (x0 point, candidate): S(u) from the three correlation "
              "tables (15) + k^2 (u - x)^2 and the sum (4)",
    "tables": "2 flops per (table, position, tap): 3 n_pos n_w multiply-adds",
    "mmse_main": "2 flops per Taylor term evaluated + 8 per directly summed "
                 "(source, target) pair, from device counters",
}
DTYPE = {
    1: ("f32x2", "double-float (pairs of FP32, ~48 bits) on the FP32 pipe for the "
                 "screened search, the u1 sums and J's terms; exact 8-bit integer "
                 "slices in bf16 on the tensor cores (FP32 accumulation, exact) for "
                 "the correlation tables; FP64 for near-tie re-costs, the u1 ratio and "
                 "J's sum; decisions equal the FP64 oracle's"),
    0: ("f64", "FP64 throughout (plain path)"),
}


def kernel_work(p, sizes, counters, launches):
    """{kernel group: (algorithmic flops, issued flops, pipe)} per launch."""
    nx, nw, ny = sizes["n_x"], sizes["n_w"], sizes["n_y"]
    if p["precision"] == 0:
        q = nx * sizes["n_cand"] * nw * 6.0
        return {"search": (q, q, "fp64"), "mmse": (nx * ny * 8.0, nx * ny * 8.0, "fp64")}
    run = sizes.get("run", 16)
    per = 1.0 / max(1, launches.get("mmse_main", 1))
    terms = counters.get("u1_df_terms", 0) + counters.get("u1_f32_terms", 0)
    u1_alg = (terms * ALG_U1_TERM + counters.get("u1_pairs", 0) * run * ALG_U1_PAIR) * per
    u1 = (counters.get("u1_pairs", 0) * (run * FLOPS_U1_PAIR + FLOPS_U1_ANCHOR) +
          counters.get("u1_boxes", 0) * (run * FLOPS_U1_BOX_TARGET + FLOPS_U1_ANCHOR) +
          counters.get("u1_df_terms", 0) * FLOPS_U1_TERM_DF +
          counters.get("u1_f32_terms", 0) * FLOPS_U1_TERM_F32) * per
    tab = 3 * sizes["tc_ng"] * sizes["tc_nch"] * TC_PRODUCTS * 2.0 * 128 * 64 * 128
    tab_alg = 3.0 * sizes["n_pos"] * nw * ALG_TABLE_TAP
    return {
        "tables": (tab_alg, tab, "bf16"),
        "mmse_main": (u1_alg, u1, "fp32"),
        "search": (nx * sizes["n_cand"] * ALG_SEARCH_CAND,
                   nx * sizes["n_cand"] * FLOPS_SEARCH_CAND, "fp32"),
    }


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


# ---- clocks ---------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"ucp_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# ---- CPU oracle sample ----------------------------------------------------

def oracle_sample(p, budget_s=12.0, threads=None, seed=0):
    """Time the oracle on a bounded sample of one solve and extrapolate:
    64-point blocks of x_i for the search and, on grids whose u1 step alone
    would take long, 64-row blocks of y_j for the u1 step, each spread over
    the grid; one J.  Returns (solves/s, threads, description, seconds
    spent); seconds * solves/s is the share of one solve the sample did."""
    import oracle
    threads = threads or os.cpu_count() or 1
    oracle.set_threads(threads)
    o = oracle.Oracle(p)
    nu = o.init(p["init_kind"]) if p["init_kind"] != 2 else o.init(2, init_table(p))
    rng = np.random.default_rng(seed)
    if o.n_x * o.n_y <= 4e8:
        t0 = time.perf_counter()
        U = o.mmse(nu)
        t_mmse = time.perf_counter() - t0
        rows = o.n_y
    else:
        U = np.interp(np.linspace(-1, 1, o.n_y), [-1, 1], [-1, 1]) * p["y_half"]
        rows, t_u = 0, 0.0
        for j0 in rng.permutation(np.arange(0, max(1, o.n_y - 63), 64)):
            t0 = time.perf_counter()
            o.mmse(nu, int(j0), int(min(o.n_y, j0 + 64)))
            t_u += time.perf_counter() - t0
            rows += int(min(o.n_y, j0 + 64) - j0)
            if t_u >= budget_s * 0.2:
                break
        t_mmse = t_u / rows * o.n_y
    t0 = time.perf_counter()
    o.J(nu, U)
    t_J = time.perf_counter() - t0
    starts = rng.permutation(np.arange(0, max(1, o.n_x - 63), 64))
    done_i, t_search = 0, 0.0
    for s0 in starts:
        t0 = time.perf_counter()
        o.search(nu, U, int(s0), int(min(o.n_x, s0 + 64)))
        t_search += time.perf_counter() - t0
        done_i += int(min(o.n_x, s0 + 64) - s0)
        if t_search >= budget_s * 0.7:
            break
    per_sweep = t_search / done_i * o.n_x + t_mmse + t_J
    solve_s = t_mmse + t_J + p["sweeps"] * per_sweep
    oracle.set_threads(1)
    spent = t_search + t_J + (t_mmse if rows == o.n_y else t_mmse * rows / o.n_y)
    sample = (f"{done_i} of {o.n_x} x0 searches (64-point blocks spread over "
              f"the grid), {rows} of {o.n_y} u1 rows, one J; extrapolated to "
              f"set-up + {p['sweeps']} sweeps")
    return 1.0 / solve_s, threads, sample, spent


def oracle_parity(p, inst, args):
    """The oracle's own whole solve of the workload on every host core
    (init, u1, then every sweep) against the GPU's solve held by `inst`: J
    after every sweep, the final controllers.  Its wall time is the CPU
    baseline (a whole solve, not a sample)."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    o = oracle.Oracle(p)
    t0 = time.perf_counter()
    r = o.solve(int(p["init_kind"]), int(p["sweeps"]))
    secs = time.perf_counter() - t0
    oracle.set_threads(1)
    Jh = inst.J_history()
    st = inst.get_controllers()
    fo = o.value(r["nu"])
    ndiff = int(np.sum(st["f"] != fo))
    dJ = float(np.max(np.abs(Jh - r["J"])))
    dU = float(np.max(np.abs(st["U"] - r["U"])))
    parity = {"compared": f"the oracle's own solve (set-up + {p['sweeps']} sweeps) "
                          "against the GPU's: J after every sweep, final f and u1",
              "max_abs_dJ": dJ, "tol_J": 1e-9, "J": float(Jh[-1]),
              "J_oracle": float(r["J"][-1]), "final_f_points_differing": ndiff,
              "controllers_bit_identical": ndiff == 0, "max_abs_dU": dU, "tol_U": 1e-6,
              "pass": bool(dJ <= 1e-9 and dU <= 1e-6)}
    cpu = {"value": 1.0 / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"one whole solve of the workload (set-up + {p['sweeps']} sweeps) "
                     f"on {cores} host cores, not extrapolated",
           "seconds": round(secs, 2)}
    return parity, cpu


# ---- multi-rank aggregation -------------------------------------------------

def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over the ranks (x itself when world == 1)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, max_seconds: float) -> float:
    """Units all ranks processed per second of the slowest rank."""
    return world * units_per_rank / max_seconds


# ---- GPU arm --------------------------------------------------------------

def fast_sizes(p, binding):
    """Table positions, tensor-core grid and u1 run length of the fast path
    (mirrors the library's plan: reach of the candidate lattice, 64-column
    groups of 128 positions, 128-tap chunks, run length rule)."""
    d = p["delta"]
    hx = round(p["x_half"] / d); hw = round(p["w_half"] / d)
    hy = round(p["y_half"] / d); hr = round(p["cand_half"] / d)
    q = 2 * max(1, -(-hr // (p["n_coarse"] - 1)))
    reach = (p["n_coarse"] - 1) * (q // 2) + 2 * q
    ext = max(reach, hx + 2 * q) + 2
    s = dict(binding.plan(p))
    s["n_pos"] = 2 * ext + 2
    na = -(-s["n_pos"] // 128)
    s["tc_ng"] = -(-na // 64)
    s["tc_nch"] = -(-(s["n_w"] + 127) // 128)
    F = max(hr + 2 * q, hx) * d
    slope = d * (hy * d + F)
    run = 16
    while run > 1 and (run - 1) * slope > 15.0:
        run //= 2
    s["run"] = run
    return s


def batched_work(ps, b, binding, sweeps):
    """Work of one batched sweep per modelled kernel group, summed over the
    members (the single-instance model of kernel_work).  The u1 counters
    cover the set-up's u1 step and the sweeps; they are scaled to one sweep
    by 1 / (sweeps + 1)."""
    tot = {}
    for p, m in zip(ps, b.members):
        sz = fast_sizes(p, binding)
        c = {k: v / (sweeps + 1) for k, v in m.work_counters().items()}
        for k, (a, i, pp) in kernel_work(p, sz, c, {"mmse_main": 1}).items():
            ta, ti, _ = tot.get(k, (0.0, 0.0, pp))
            tot[k] = (ta + a, ti + i, pp)
    return tot


def roofline_entries(work, kern, pipe_peak):
    """Per modelled kernel group: ms per launch (CUDA events), algorithmic and
    issued TFLOP/s and their fractions of the pipe's measured peak."""
    out = {}
    for k, (alg, iss, pp) in work.items():
        if k in kern and kern[k][0]:
            ms_l = kern[k][1] / kern[k][0]
            pk, bound, _ = pipe_peak[pp]
            a_, i_ = alg / (ms_l / 1e3) / 1e12, iss / (ms_l / 1e3) / 1e12
            out[k] = {"bound": bound, "pipe": pp, "ms_per_launch": ms_l,
                      "algorithmic_tflops": a_, "frac": a_ / pk,
                      "issued_tflops": i_, "issued_frac": i_ / pk}
    return out


def pipe_peaks(peaks):
    mp = load_peaks()
    return {
        "fp32": (peaks["fp32_tflops"], "alu",
                 "of measured FP32 FMA throughput (ucp_probe_alu, this run)"),
        "fp64": (peaks["fp64_tflops"], "alu",
                 "of measured FP64 FMA throughput (ucp_probe_alu, this run)"),
        "bf16": (mp.get("bf16_tflops_sustained", 1700.0), "tensor",
                 "of measured dense bf16 cuBLAS throughput, sustained (MEASURED_PEAKS.json)"
                 if "bf16_tflops_sustained" in mp else "of fallback dense bf16 1.7 PFLOP/s"),
    }


def measure_batched(args, binding, torch, stream, flush, world=1, rank=0):
    """c3: 256 uneven instances solved (setup + 10 sweeps + J) as one batch,
    one at a time on the same fast path, and one at a time on the plain FP64
    path (a sample, extrapolated by grid work).  Under torchrun the instances
    are partitioned over the ranks by estimated work (no collective on the
    data path); each rank solves its part as one batch, the time is the
    slowest rank's, and only the one-GPU comparisons are skipped."""
    from paper_1908_04489_gb300 import workloads as W
    ps_all = W.c3()
    n = len(ps_all)
    parts = W.partition(ps_all, world)
    ps = [ps_all[k] for k in parts[rank]]

    # launch shapes tuned on a scratch batch of the same members (untimed;
    # every shape gives the same results), then every timed batch starts
    # with them through the context
    from paper_1908_04489_gb300 import autotune
    tuned, table = autotune.tuned_batch_config(
        binding, ps, stream, torch.cuda.get_device_name(), retune=True,
        path=os.path.join(tempfile.gettempdir(), f"ucp_tune_{os.getpid()}.json"))
    ctx = binding.default_context()
    ctx.set_launch_config(tuned)

    def batch_solve():
        b = binding.Batch(ps, stream=stream)
        b.sweep(10)
        return b

    for _ in range(2):
        b = batch_solve(); b.eval_J(); b.close()
    times = []
    for _ in range(max(1, args.batch_steps)):
        flush.fill_(1)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b = batch_solve()
        e1.record(stream)
        e1.synchronize()
        times.append(max_over_ranks(e0.elapsed_time(e1), world, "cuda"))
        Jb = b.eval_J()
        b.close()
    t_batch = float(np.median(times)) / 1e3
    default_ms = table[0][1] if table else None
    tuned_ms = min(ms for _, ms in table) if table else None
    tuning = {"config": tuned, "default_ms_per_sweep": default_ms,
              "tuned_ms_per_sweep": tuned_ms, "configs_timed": len(table) if table else 0,
              "how": "coordinate descent over search lanes, u1 threads per run and deferred "
                     "blocks on a scratch batch (CUDA events over 3 sweeps, median of 3); "
                     "every shape gives the same results"}
    if world > 1:
        ctx.set_launch_config(autotune.default_config())
        est = [sum(W.work_estimate(ps_all[k]) for k in part) for part in parts]
        return {
            "workload": "c3: 256 Witsenhausen instances (seed 1908) partitioned over "
                        f"{world} GPUs by estimated work, one batch per GPU, 10 sweeps",
            "solves_per_s": n / t_batch, "ms_per_batch": t_batch * 1e3,
            "scaling": "strong", "instances_per_rank": [len(q) for q in parts],
            "work_estimate_imbalance": max(est) / (sum(est) / world),
        }
    # one more batch, untimed, with per-kernel CUDA events around each kernel
    # group of the 10 batched sweeps (kernel by kernel, no graph replay)
    flush.fill_(1)
    b = binding.Batch(ps, stream=stream)
    b.profile(True)
    b.sweep(10)
    kern = b.kernel_times()
    work = batched_work(ps, b, binding, sweeps=10)
    b.close()
    per_kernel = roofline_entries(work, kern, pipe_peaks(binding.probe_alu(stream)))
    ctx.set_launch_config(autotune.default_config())   # the rules for every other leg
    # one at a time, same fast path
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    flush.fill_(1)
    e0.record(stream)
    insts = []
    for p in ps:
        inst = binding.Instance(p, stream=stream)
        inst.sweep(10)
        insts.append(inst)
    e1.record(stream)
    e1.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    Js = np.array([i.eval_J() for i in insts])
    for i in insts:
        i.close()
    # plain FP64 path on a sample, extrapolated by sum of n_x * n_w
    pick = list(range(0, n, max(1, n // args.plain_sample)))[:args.plain_sample]
    work = lambda p: binding.plan(p)["n_x"] * binding.plan(p)["n_w"]
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in pick:
        inst = binding.Instance(dict(ps[k], precision=0), stream=stream)
        inst.sweep(10)
        inst.close()
    e1.record(stream)
    e1.synchronize()
    t_plain_sample = e0.elapsed_time(e1) / 1e3
    t_plain = t_plain_sample * sum(work(p) for p in ps) / sum(work(ps[k]) for k in pick)
    return {
        "workload": "c3: 256 Witsenhausen instances (seed 1908), k log-U[0.05,0.5], "
                    "sigma U[1,10], delta in {0.01,0.02}, 533..9959 x0 points, "
                    "identity init, 10 sweeps",
        "solves_per_s": n / t_batch, "ms_per_batch": t_batch * 1e3,
        "one_at_a_time_fast_solves_per_s": n / t_seq,
        "plain_fp64_solves_per_s": n / t_plain,
        "plain_fp64_sample": f"{len(pick)} of {n} instances, extrapolated by n_x*n_w",
        "batched_vs_one_at_a_time": t_seq / t_batch,
        "batched_vs_plain_fp64": t_plain / t_batch,
        "max_abs_J_batched_vs_one_at_a_time": float(np.max(np.abs(Jb - Js))),
        "kernels_ms_per_batch": {k: v[1] for k, v in kern.items()},
        "roofline_per_kernel": per_kernel,
        "launch_tuning": tuning,
    }


def time_solves(binding, torch, stream, flush, p, steps):
    """Median seconds of whole solves (set-up + p["sweeps"] sweeps) timed
    with CUDA events on `stream`, after two untimed solves; the last solve's
    J and controllers."""
    for _ in range(2):
        with binding.Instance(p, stream=stream) as inst:
            inst.sweep(p["sweeps"])
            inst.eval_J()
    times = []
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inst = binding.Instance(p, stream=stream)
        inst.sweep(p["sweeps"])
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        J = inst.eval_J()
        st = inst.get_controllers()
        Jh = inst.J_history()
        inst.close()
    return float(np.median(times)) / 1e3, J, st, Jh


def measure_source_channel(args, binding, torch, stream, flush):
    """Section V-B's second problem on the same sweep (zero-delay
    source-channel coding, lambda = 2, w ~ U(-1, 1)): whole solves (set-up +
    20 sweeps) timed with CUDA events on the plain FP64 path and in the fast
    mode (precision 1: screened search on three tables, warp u1 step), J
    checked against the oracle recomputing it from the GPU's final state and
    against the oracle's own solve."""
    from paper_1908_04489_gb300 import workloads as W
    pf = W.source_channel(precision=1)
    tf, Jf, _, Jhf = time_solves(binding, torch, stream, flush, pf, max(3, args.batch_steps))
    with binding.Instance(pf, stream=stream) as inst:
        inst.profile(True)
        inst.sweep(pf["sweeps"])
        kern_f = {k: v[1] for k, v in inst.kernel_times().items()}
    p = W.source_channel()
    for _ in range(2):
        with binding.Instance(p, stream=stream) as inst:
            inst.sweep(p["sweeps"])
            inst.eval_J()
    times = []
    for _ in range(max(3, args.batch_steps)):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inst = binding.Instance(p, stream=stream)
        inst.sweep(p["sweeps"])
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        J = inst.eval_J()
        st = inst.get_controllers()
        inst.close()
    t = float(np.median(times)) / 1e3
    # one more solve with per-kernel events (kernel by kernel on the stream)
    with binding.Instance(p, stream=stream) as inst:
        inst.profile(True)
        inst.sweep(p["sweeps"])
        kern = {k: v[1] for k, v in inst.kernel_times().items()}
    out = {"workload": "zero-delay source-channel coding (Section V-B): lambda = 2, "
                       "x0 ~ N(0,1), w ~ U(-1,1), delta = 0.02 (501 x0 / 101 w / 701 y), "
                       "identity start, 20 sweeps, plain FP64 path",
           "solves_per_s": 1.0 / t, "ms_per_solve": t * 1e3, "J": J,
           "J_paper": 0.890756, "kernels_ms_per_solve": kern,
           "fast_mode": {"solves_per_s": 1.0 / tf, "ms_per_solve": tf * 1e3, "J": Jf,
                         "vs_plain": t / tf, "kernels_ms_per_solve": kern_f}}
    # FP64 work of the plain search: 6 flops per quadrature term, every
    # candidate of every x0 point each sweep (the u1 and J passes are small)
    sz = binding.plan(p)
    flops = sz["n_x"] * sz["n_cand"] * sz["n_w"] * 6.0 * p["sweeps"]
    fp64 = binding.probe_alu(stream)["fp64_tflops"]
    out["search_fp64_tflops"] = flops / t / 1e12
    out["search_fp64_frac"] = flops / t / 1e12 / fp64
    if not args.no_cpu:
        import oracle
        o = oracle.Oracle(p)
        Jo = o.J(o.init(2, st["f"]), st["U"])
        out["abs_dJ_oracle_from_gpu_state"] = abs(J - Jo)
        cores = os.cpu_count() or 1
        oracle.set_threads(cores)
        t0 = time.perf_counter()
        ref = o.solve(0, p["sweeps"])
        tc = time.perf_counter() - t0
        oracle.set_threads(1)
        out["cpu_oracle"] = {"solves_per_s": 1.0 / tc, "cores": cores,
                             "sample": "one whole solve (20 sweeps) from the identity"}
        out["abs_dJ_vs_oracle_trajectory"] = abs(J - float(ref["J"][-1]))
        out["fast_mode"]["max_abs_dJ_vs_oracle_trajectory"] = float(
            np.max(np.abs(np.asarray(Jhf) - np.asarray(ref["J"]))))
    return out


def measure_serving(args, binding, torch):
    """c4-style stream: requests (k log-U[0.05,0.5], sigma U[1,10], delta in
    {0.05, 0.01, 0.005}, 20 sweeps) submitted at Poisson arrival times at each
    rate; latency = result on the host - submission."""
    from paper_1908_04489_gb300 import workloads as W
    out = []
    for rate in args.serve_rates:
        reqs, times = W.c4(n=args.serve_requests, rate=rate)
        srv = binding.Server(hbm_budget_bytes=args.serve_budget_gb << 30,
                             max_slots=args.serve_slots)
        # warm the server's memory pool with a few requests
        warm = [srv.submit(r) for r in reqs[:8]]
        while warm:
            warm = [t for t in warm if srv.poll(t, want_arrays=False) is None]
        pending, lat, done_t = {}, [], []
        t0 = time.perf_counter()
        k = 0
        while k < len(reqs) or pending:
            now = time.perf_counter() - t0
            while k < len(reqs) and times[k] <= now:
                pending[srv.submit(reqs[k])] = k
                k += 1
            for t in list(pending):
                r = srv.poll(t, want_arrays=False)
                if r is not None:
                    lat.append(r["t_done"] - r["t_submit"])
                    done_t.append(r["t_done"])
                    del pending[t]
            if k < len(reqs) and not pending:
                time.sleep(max(0.0, min(0.001, times[k] - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = np.array(lat) * 1e3
        out.append({"rate_per_s": rate, "requests": len(reqs),
                    "solves_per_s": len(reqs) / wall,
                    "p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99)),
                    "max_batch": st["max_active"], "steps": st["steps"]})
    cap = max(r["solves_per_s"] for r in out)
    kept = [r["rate_per_s"] for r in out if r["solves_per_s"] >= 0.95 * r["rate_per_s"]]
    return {"workload": "c4: Poisson stream, 20 sweeps per request, delta in "
                        "{0.05,0.01,0.005}, k log-U[0.05,0.5], sigma U[1,10] "
                        f"({args.serve_requests} requests per rate)",
            "rates": out, "capacity_solves_per_s": cap,
            "knee_rate_per_s": max(kept) if kept else None,
            "knee": "the highest offered rate served at >= 95% of the rate"}


def measure_c5(args, binding, torch, stream, flush):
    """c5, the large single instance (k = 0.2, sigma = 10, delta = 0.001:
    100001 x0 / 14001 w / 120001 y points, 6 levels, identity start, 20
    sweeps): whole solves timed with CUDA events, the per-kernel roofline of
    a profiled solve, the oracle on a sample, and J after every sweep against
    the oracle's stored 20-sweep solve."""
    from paper_1908_04489_gb300 import workloads as W
    p = W.c5()
    sizes = fast_sizes(p, binding)
    with binding.Instance(p, stream=stream) as inst:
        inst.sweep(p["sweeps"])
        inst.eval_J()
    times, counters = [], dict.fromkeys(binding.Instance.COUNTERS, 0)
    for _ in range(max(1, args.c5_steps)):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inst = binding.Instance(p, stream=stream)
        inst.sweep(p["sweeps"])
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        Jh = inst.J_history()
        for k, v in inst.work_counters().items():
            counters[k] += v / max(1, args.c5_steps)
        inst.close()
    with binding.Instance(p, stream=stream) as inst:
        inst.profile(True)
        inst.sweep(p["sweeps"])
        kern = {k: list(v) for k, v in inst.kernel_times().items()}
    work = kernel_work(p, sizes, counters, {k: v[0] for k, v in kern.items()})
    per_kernel = roofline_entries(work, kern, pipe_peaks(binding.probe_alu(stream)))
    t = float(np.median(times)) / 1e3
    out = {"workload": "c5: k=0.2 sigma=10, delta=0.001 (100001 x0 / 14001 w / 120001 y), "
                       "6 levels, identity init, 20 sweeps",
           "solves_per_s": 1.0 / t, "ms_per_solve": t * 1e3, "J": float(Jh[-1]),
           "kernels_ms_per_solve": {k: v[1] for k, v in kern.items()},
           "roofline_per_kernel": per_kernel,
           "work_per_solve": counters}
    gold = os.path.join(ROOT, "tests", "golden", "oracle_c5.json")
    if os.path.exists(gold):
        ref = json.load(open(gold))["solve"]["J"]
        out["parity"] = {"compared": "J after every sweep against the oracle's own "
                                     "20-sweep solve (stored by the oracle-only script "
                                     "tests/golden/make_oracle_trajectories.py)",
                         "max_abs_dJ": float(np.max(np.abs(Jh - np.asarray(ref)))),
                         "tol_J": 1e-9}
    if not args.no_cpu:
        v, cores, sample, spent = oracle_sample(p, 8.0)
        out["cpu_oracle"] = {"solves_per_s": v, "cores": cores, "sample": sample,
                             "seconds": round(spent, 2)}
    return out


P2D = dict(k=0.2, sigma=5.0, delta=0.3125, x_half=25.0, w_half=5.0, y_half=35.0,
           cand_half=30.0, n_coarse=13, n_levels=8, n_nbr=2)
P2D_SWEEPS = 40
P2D_PAPER_J = 0.166719   # Section V-D, 160 x 160 samples (other grids and list)


def measure_2d(args, binding, torch, stream, flush):
    """The 2-dimensional counterexample of Section V-D (k = 0.2, sigma = 5):
    161 x 161 x0 points over [-25, 25]^2 (delta = 0.3125), 33 x 33 noise
    points, 225 x 225 y points, 13 x 13 coarse values and 8 levels; a solve is
    the identity start and 40 sweeps.  Whole solves timed with CUDA events;
    the last sweep checked against the oracle on sampled points (decisions
    from the GPU's own pre-sweep state, u1 at sampled targets, J of the
    state); the oracle's sweep rate estimated from the same samples."""
    import oracle
    p = dict(P2D)
    with binding.Instance2D(p, stream=stream) as g:
        g.sweep(2)
    times = []
    for _ in range(max(1, args.twod_steps)):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g = binding.Instance2D(p, stream=stream)
        g.sweep(P2D_SWEEPS - 1)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        if _ + 1 < max(1, args.twod_steps):
            g.close()
    pre = g.get_controllers()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.sweep(1)
    e1.record(stream)
    e1.synchronize()
    last_ms = e0.elapsed_time(e1)
    post = g.get_controllers()
    Jh = g.J_history()
    g.close()
    t = (float(np.median(times)) + last_ms) / 1e3
    # one more solve with per-kernel-group events, for the dominant kernel's
    # roofline: the u1 sums, 6 flops per (target, source) pair of the method
    # (product, denominator, two numerators); issued as about 45 FP32-pipe
    # instructions per pair slot of the stages it evaluates (not skipped)
    with binding.Instance2D(p, stream=stream) as gp:
        gp.profile(True)
        gp.sweep(P2D_SWEEPS)
        kern = gp.kernel_times()
        live = gp.work_counters()["u1_live_pairs"]
    peaks = pipe_peaks(binding.probe_alu(stream))
    n_src = (2 * round(p["x_half"] / p["delta"]) + 1) ** 2
    n_tgt = (2 * round(p["y_half"] / p["delta"]) + 1) ** 2
    su = kern.get("u1_sums", (0, 0.0))
    roof = None
    if su[0]:
        sec = su[1] / su[0] / 1e3
        alg = 6.0 * n_src * n_tgt / sec / 1e12
        live_per = live / (P2D_SWEEPS + 1)
        issued = 45.0 * live_per / sec / 1e12
        roof = {"kernel": "k2_u1_sums", "bound": "alu", "unit": "TFLOP/s",
                "ms_per_launch": sec * 1e3, "pairs_per_launch": n_src * n_tgt,
                "evaluated_pair_slots_per_pair": live_per / (n_src * n_tgt),
                "achieved": alg, "peak": peaks["fp32"][0], "frac": alg / peaks["fp32"][0],
                "peak_source": peaks["fp32"][2],
                "work_model": "6 flops per (target, source) pair: the weight product, the "
                              "denominator and two numerators",
                "vs_fp64_peak": alg / peaks["fp64"][0],
                "issued": {"fp32_pipe_instr_per_pair_slot": 45, "achieved_tinstr_per_s": issued,
                           "frac_of_fp32_issue_peak": issued / (peaks["fp32"][0] / 2.0)}}
    out_kern = {k: v[1] / P2D_SWEEPS for k, v in kern.items()}
    out = {"workload": "2-D Witsenhausen (Section V-D): k=0.2 sigma=5, 161x161 x0 over "
                       "[-25,25]^2 (delta=0.3125), 33x33 w, 225x225 y, 13x13 coarse + "
                       "8 levels, window radius 2, identity init, 40 sweeps",
           "solves_per_s": 1.0 / t, "ms_per_solve": t * 1e3,
           "ms_per_sweep": t * 1e3 / P2D_SWEEPS, "J": float(Jh[-1]),
           "J_paper": P2D_PAPER_J,
           "J_note": "plausibility band only: the paper's 160x160 samples, interpolation "
                     "and candidate scheme differ",
           "kernels_ms_per_sweep": out_kern, "roofline": roof}
    if args.no_cpu:
        return out
    import time as _t
    o = oracle.Oracle2D(p)
    d, sh = p["delta"], o.shift
    lat = lambda f: np.rint(np.ldexp(f / d, sh)).astype(np.int64)
    nu_pre, nu_post = lat(pre["f"]), lat(post["f"])
    rng = np.random.default_rng(1908)
    pts = rng.choice(o.N, 48, replace=False)
    t0 = _t.perf_counter()
    differ, gap = 0, 0.0
    for i in pts:
        a, b = o.search(nu_pre, pre["U"], int(i), int(i) + 1)
        if not (np.array_equal(a[i], nu_post[i]) and b[i] == post["idx"][i]):
            differ += 1
            gap = max(gap, o.cost(pre["U"], int(i), *nu_post[i]) -
                      o.cost(pre["U"], int(i), *a[i]))
    t_search = (_t.perf_counter() - t0) / len(pts)
    tg = rng.choice(o.n_y ** 2, 48, replace=False)
    t0 = _t.perf_counter()
    dU = 0.0
    for tt in tg:
        Uo = o.mmse(nu_post, int(tt), int(tt) + 1)
        dU = max(dU, float(np.max(np.abs(post["U"][tt] - Uo[tt]))))
    t_u1 = (_t.perf_counter() - t0) / len(tg)
    t0 = _t.perf_counter()
    Jo = o.J(nu_post, post["U"])
    t_J = _t.perf_counter() - t0
    out["parity"] = {"compared": "last sweep: 48 sampled x0 points' decisions from the "
                                 "GPU's own pre-sweep state, u1 at 48 sampled targets, "
                                 "J of the GPU's state (FP64 2-D oracle)",
                     "decisions_differing": differ, "max_cost_gap_of_differing": gap,
                     "max_abs_dU": dU, "dJ": float(Jh[-1] - Jo), "tol_U": 1e-11}
    sweep_s = t_search * o.N + t_u1 * o.n_y ** 2 + t_J
    out["cpu_oracle"] = {"solves_per_s": 1.0 / (sweep_s * P2D_SWEEPS), "cores": 1,
                         "sample": "48 points' searches, 48 targets' u1, one J, "
                                   "scaled to a 40-sweep solve",
                         "s_per_sweep": sweep_s}
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1908_04489_gb300 import binding, build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    binding.load()

    p, desc = workload(args.workload, args.precision)
    sizes = fast_sizes(p, binding)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    peaks = binding.probe_alu(stream)

    for _ in range(args.warmup):
        inst = binding.Instance(p, stream=stream)
        inst.sweep(p["sweeps"])
        inst.eval_J()
        inst.close()
    torch.cuda.synchronize()

    # ---- device-timed steps
    clocks = Clocks(local)
    clocks.start()
    step_ms, Js, kern = [], [], {}
    counters = dict.fromkeys(binding.Instance.COUNTERS, 0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inst = binding.Instance(p, stream=stream)
        inst.sweep(p["sweeps"])
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        Js.append(inst.eval_J())
        for k, v in inst.work_counters().items():
            counters[k] += v
        inst.close()
    # one more solve, untimed, with per-kernel CUDA events for the breakdown
    flush.fill_(1)
    inst = binding.Instance(p, stream=stream)
    inst.profile(True)
    inst.sweep(p["sweeps"])
    for k, (nl, ms) in inst.kernel_times().items():
        kern[k] = [nl * args.steps, ms * args.steps]
    last = inst
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(float(np.sum(step_ms)), world, "cuda")
    value = whole_job_rate(world, args.steps, total_ms / 1e3)

    # ---- end-to-end through the C ABI with host buffers
    table = init_table(p)
    pe = dict(p, init_kind=2)
    e2e_s = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        inst = binding.Instance(pe, table=table, stream=stream)
        inst.sweep(pe["sweeps"])
        out = inst.get_controllers(want=("f", "U"))
        Je = inst.eval_J()
        inst.close()
        e2e_s.append(time.perf_counter() - t0)
    assert abs(Je - Js[-1]) <= 1e-9, (Je, Js[-1])
    e2e_total = max_over_ranks(float(np.sum(e2e_s)), world, "cuda")
    e2e = {"value": whole_job_rate(world, args.steps, e2e_total), "unit": UNIT,
           "h2d_bytes_per_step": int(table.nbytes),
           "d2h_bytes_per_step": int(out["f"].nbytes + out["U"].nbytes + 8)}

    # ---- roofline of the dominant kernel, and of every modelled kernel
    launches = {k: v[0] for k, v in kern.items()}
    work = kernel_work(p, sizes, {k: v / args.steps for k, v in counters.items()},
                       {k: v / args.steps for k, v in launches.items()})
    pp_ = pipe_peaks(peaks)
    per_kernel = roofline_entries(work, kern, pp_)
    dom = max(per_kernel, key=lambda k: kern[k][1])
    d = per_kernel[dom]
    peak, bound, src = pp_[d["pipe"]]
    traffic = TRAFFIC_BYTES.get(args.workload, {}).get(dom)
    roofline = {"bound": bound, "kernel": dom, "achieved": d["algorithmic_tflops"],
                "peak": peak, "unit": "TFLOP/s", "frac": d["frac"],
                "traffic": traffic,
                "traffic_source": TRAFFIC_SOURCE if traffic is not None else None,
                "work_model": WORK_MODEL.get(dom, ""),
                "issued": {"achieved": d["issued_tflops"], "frac": d["issued_frac"]},
                "peak_source": src, "share_of_step": kern[dom][1] / total_ms,
                "per_kernel": per_kernel}

    batched = None
    if not args.no_batched:   # every rank: the instances are partitioned
        batched = measure_batched(args, binding, torch, stream, flush, world, rank)
    source_channel = None
    if rank == 0 and not args.no_batched:
        source_channel = measure_source_channel(args, binding, torch, stream, flush)
    serving = None
    if rank == 0 and not args.no_serving:
        serving = measure_serving(args, binding, torch)
    large = None
    if rank == 0 and not args.no_c5 and args.workload != "c5":
        large = measure_c5(args, binding, torch, stream, flush)
    twod = None
    if rank == 0 and not args.no_2d:
        twod = measure_2d(args, binding, torch, stream, flush)
    # the oracle's own solve last: no host load while the GPU legs run
    parity, cpu = None, None
    if rank == 0 and not args.no_cpu:
        parity, cpu = oracle_parity(p, last, args)
    last.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[p["precision"]][0],
        "dtype_detail": DTYPE[p["precision"]][1],
        "data": "synthetic (analytic Witsenhausen instance, Section V-A)",
        "config": {"workload": desc, "precision": p["precision"],
                   "l2": "flushed between steps (512 MiB write outside the events)",
                   "parallelism": f"independent solves x{world}"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "gpu_launches": int(sum(v[0] * KERNELS_PER_GROUP.get(k, 1)
                                for k, v in kern.items()) + SETUP_LAUNCHES * args.steps),
        "kernels_ms_per_step": {k: v[1] / args.steps for k, v in kern.items()},
        "roofline": roofline, "e2e": e2e, "clocks": clk, "parity": parity,
        "work_per_solve": {k: v / args.steps for k, v in counters.items()},
        "alu_peaks_measured": peaks,
    }
    if batched is not None:
        line["batched"] = batched
    if source_channel is not None:
        line["source_channel"] = source_channel
    if serving is not None:
        line["serving"] = serving
    if large is not None:
        line["large"] = large
    if twod is not None:
        line["two_dim"] = twod
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_profile(args):
    """One instance of the workload, then --profile-sweeps sweeps: the launch
    sequence the ncu summaries under profiles/ were captured from."""
    import torch
    from paper_1908_04489_gb300 import binding, build
    build.build()
    if args.search_lanes:
        binding.load()
        binding.default_context().set_launch_config({"search_lanes": args.search_lanes})
    if args.workload == "c3":
        # the first --batch-n instances of the batched workload, swept as one
        # batch (captured-graph sweeps on a non-default stream)
        from paper_1908_04489_gb300 import workloads as W
        ps = W.c3()[:args.batch_n]
        stream = torch.cuda.Stream() if args.profile_graph else None
        with binding.Batch(ps, stream=stream) as b:
            b.sweep(args.profile_sweeps)
            J = b.eval_J()
        print(json.dumps({"workload": "c3", "instances": len(ps), "J_mean": float(np.mean(J)),
                          "sweeps": args.profile_sweeps, "graph": bool(args.profile_graph)}))
        torch.cuda.synchronize()
        return
    if args.workload == "2d":
        # the 2-dimensional instance of Section V-D (the bench's 2-D leg)
        with binding.Instance2D(P2D) as g:
            g.sweep(args.profile_sweeps)
            J = g.J_history()
        print(json.dumps({"workload": "2d", "J": float(J[-1]), "sweeps": args.profile_sweeps}))
        torch.cuda.synchronize()
        return
    if args.workload == "sc":
        # Section V-B's problem (source-channel coding), --precision selects the mode
        from paper_1908_04489_gb300 import workloads as W
        p = W.source_channel(precision=args.precision)
        with binding.Instance(p) as inst:
            inst.sweep(args.profile_sweeps)
            J = inst.eval_J()
        print(json.dumps({"workload": "sc", "precision": args.precision, "J": J,
                          "sweeps": args.profile_sweeps}))
        torch.cuda.synchronize()
        return
    p, _ = workload(args.workload, args.precision)
    # on a non-default stream the sweeps replay captured graphs (the bench's
    # timed path); on the default stream they launch kernel by kernel
    stream = torch.cuda.Stream() if args.profile_graph else None
    with binding.Instance(p, stream=stream) as inst:
        inst.sweep(args.profile_sweeps)
        print(json.dumps({"workload": args.workload, "J": inst.eval_J(),
                          "sweeps": args.profile_sweeps,
                          "graph": bool(args.profile_graph)}))
    torch.cuda.synchronize()


def run_reference(args):
    """The oracle as it stands on the host cores, on the workload of the GPU
    arm.  A whole c2 oracle solve takes tens of seconds, so each step is a
    bounded sample of one solve (different blocks of x0 points each step);
    ms_per_step is the sample's measured time and solves_per_step the share
    of one solve it did, so value = solves done / time taken."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p, desc = workload(args.workload, args.precision)
    secs, shares = [], []
    for s in range(args.warmup + args.steps):
        v, cores, sample, spent = oracle_sample(p, args.ref_step_s, seed=s)
        if s >= args.warmup:
            secs.append(spent)
            shares.append(spent * v)
    value = float(np.sum(shares) / np.sum(secs))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "solves_per_step": float(np.mean(shares)),
        "config": {"workload": desc, "precision": "oracle FP64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "kind": "oracle",
                         "sample": "each step: " + sample + " (a share "
                                   f"{float(np.mean(shares)):.4f} of one solve)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ucp", choices=["ucp", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--ref-step-s", type=float, default=1.5,
                    help="--impl reference: seconds of oracle work per step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--batch-n", type=int, default=256,
                    help="with --workload c3 --profile-sweeps: batch size")
    ap.add_argument("--plain-sample", type=int, default=8)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-c5", action="store_true")
    ap.add_argument("--search-lanes", type=int, default=0,
                    help="with --profile-sweeps: lanes per x0 point of the search")
    ap.add_argument("--serving-only", action="store_true",
                    help="only the serving leg (with --serve-requests 20000: the c4 "
                         "workload at its own size), one JSON line")
    ap.add_argument("--c5-steps", type=int, default=2)
    ap.add_argument("--no-2d", action="store_true")
    ap.add_argument("--twod-steps", type=int, default=2)
    ap.add_argument("--serve-requests", type=int, default=600)
    ap.add_argument("--serve-rates", type=float, nargs="+",
                    default=[100.0, 200.0, 500.0, 1000.0, 2000.0, 5000.0])
    ap.add_argument("--serve-slots", type=int, default=512)
    ap.add_argument("--serve-budget-gb", type=int, default=64)
    ap.add_argument("--profile-sweeps", type=int, default=0,
                    help="only build one instance and run this many sweeps "
                         "(a short, fixed launch sequence for ncu)")
    ap.add_argument("--profile-graph", action="store_true",
                    help="with --profile-sweeps: run on a non-default stream "
                         "(captured-graph sweeps, as in the timed steps)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.serving_only:
        import torch
        from paper_1908_04489_gb300 import binding, build
        build.build()
        binding.load()
        print(json.dumps(measure_serving(args, binding, torch)))
    elif args.profile_sweeps:
        run_profile(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
