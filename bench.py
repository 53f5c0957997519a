"""Benchmark: UCP solves/s of the Witsenhausen sweep on GB300.

Workload (default): the fine single instance -- k = 0.2, sigma = 5,
delta = 0.005 (10001 x0 / 2401 w / 14001 y points), odd 3-step staircase init,
64 coarse candidates then 4 levels of 16, 50 sweeps.  One step = one whole
solve: setup (grids, weights, init, u1, J) + 50 sweeps, every step of the
path in the library's kernels.

  value  -- solves/s with the instance set up on the device inside the timed
            region (CUDA events on the instance stream; L2 flushed between
            steps by a 512 MiB write outside the events).
  e2e    -- solves/s through the C ABI from host buffers: the initial
            controller table goes host->device, f and u1 come back, J is read.
  cpu_baseline / --impl reference -- the FP64 C oracle timed on the host
            cores on a bounded sample of the same solve, extrapolated.

Under torchrun every rank solves its own copy (independent problems, no
collective): weak scaling, value = all solves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
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
    if name == "c5":
        return W.c5(precision=precision), (
            "c5: k=0.2 sigma=10, delta=0.001 (100001/14001/120001), 6 levels, "
            "identity init, 20 sweeps")
    raise SystemExit(f"unknown workload {name}")


def init_table(p):
    """Host-side initial controller f (the staircase of init_kind 1) for the
    end-to-end leg, which passes it through init_kind 2."""
    d = p["delta"]
    n = int(round(2 * p["x_half"] / d)) + 1
    a = np.arange(n) - (n - 1) // 2
    m = np.minimum(np.abs(a) // int(round(7.0 / d)), 2)
    return np.where(a == 0, 0.0, np.sign(a) * 3.5 * (2 * m + 1))


# ---- algorithmic work per kernel launch (FP64 flops) ----------------------

def kernel_work(p, sizes):
    """Algorithmic FP64 flops per launch of each kernel.

    search: one quadrature term per (x_i, refinement candidate, w_l) =
    lerp mul + add, residual sub, square, weight mul, accumulate = 6 flops.
    mmse:   per (y_j, x_i): residual, square, halve, prior add, shift,
    numerator multiply-add, denominator add = 8 flops (+ one exp).
    S lists: 6 flops per (value, w_l).  J: 5 flops per x_i.
    """
    nx, nw, ny = sizes["n_x"], sizes["n_w"], sizes["n_y"]
    L, R = p["n_levels"], p["n_refine"]
    return {
        "search": nx * L * R * nw * 6.0,
        "mmse": nx * ny * 8.0,
        "mmse_main": nx * ny * 8.0,
        "tables": sizes.get("n_pos", 0) * nw * 6.0,
        "S_f": nx * nw * 6.0,
        "S_coarse": p["n_coarse"] * nw * 6.0,
        "J": nx * 5.0,
    }


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (dense), from the platform table


# ---- clocks ---------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
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

def oracle_sample(p, budget_s=12.0, threads=None):
    """Time the oracle on a bounded sample of one solve and extrapolate:
    strided x_i for the search, strided y_j for the u1 step, full J."""
    import oracle
    threads = threads or os.cpu_count() or 1
    oracle.set_threads(threads)
    o = oracle.Oracle(p)
    nu = o.init(p["init_kind"]) if p["init_kind"] != 2 else o.init(2, init_table(p))
    t0 = time.perf_counter()
    U = o.mmse(nu)
    t_mmse_full = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.J(nu, U)
    t_J = time.perf_counter() - t0
    # search: blocks of 64 consecutive x_i spread over the grid, added until
    # the budget is used (OpenMP splits each block over the host cores)
    rng = np.random.default_rng(0)
    starts = rng.permutation(np.arange(0, max(1, o.n_x - 63), 64))
    done_i, t_search = 0, 0.0
    for s0 in starts:
        t0 = time.perf_counter()
        o.search(nu, U, int(s0), int(min(o.n_x, s0 + 64)))
        t_search += time.perf_counter() - t0
        done_i += int(min(o.n_x, s0 + 64) - s0)
        if t_search >= budget_s * 0.7:
            break
    per_sweep = t_search / done_i * o.n_x + t_mmse_full + t_J
    solve_s = t_mmse_full + t_J + p["sweeps"] * per_sweep
    oracle.set_threads(1)
    sample = (f"{done_i} of {o.n_x} x0 searches (64-point blocks spread over "
              f"the grid) + one full u1 step "
              f"({o.n_y} y points) + one J, extrapolated to {p['sweeps']} sweeps")
    return 1.0 / solve_s, threads, sample, t_search + t_mmse_full + t_J


# ---- GPU arm --------------------------------------------------------------

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
    sizes = binding.plan(p)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def solve(profile=False):
        inst = binding.Instance(p, stream=stream)
        if profile:
            inst.profile(True)
        inst.sweep(p["sweeps"])
        return inst

    # cpu baseline first (host only, before any timing)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, sample, spent = oracle_sample(p, args.cpu_budget)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": sample, "seconds": round(spent, 2)}

    for _ in range(args.warmup):
        inst = solve()
        inst.eval_J()
        inst.close()
    torch.cuda.synchronize()

    # ---- device-timed steps
    clocks = Clocks(local)
    clocks.start()
    step_ms, Js, kern = [], [], {}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inst = binding.Instance(p, stream=stream)
        inst.profile(True)
        inst.sweep(p["sweeps"])
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for k, (n, ms) in inst.kernel_times().items():
            a = kern.setdefault(k, [0, 0.0])
            a[0] += n
            a[1] += ms
        Js.append(inst.eval_J())
        recosts = inst.tie_recosts()
        last = inst
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = float(np.sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1e3)

    # parity of the reported J: recompute J with the oracle from the GPU state
    parity = None
    if rank == 0 and not args.no_cpu:
        import oracle
        st = last.get_controllers()
        o = oracle.Oracle(p)
        oracle.set_threads(os.cpu_count() or 1)
        Jo = o.J(o.init(2, st["f"]), st["U"])
        oracle.set_threads(1)
        parity = {"J": Js[-1], "J_oracle_from_gpu_state": Jo,
                  "abs_dJ": abs(Js[-1] - Jo), "tol": 1e-9}
    last.close()

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
    e2e_total = float(np.sum(e2e_s))
    if world > 1:
        t = torch.tensor([e2e_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    e2e = {"value": world * args.steps / e2e_total, "unit": UNIT,
           "h2d_bytes_per_step": int(table.nbytes),
           "d2h_bytes_per_step": int(out["f"].nbytes + out["U"].nbytes + 8)}

    # ---- roofline of the dominant kernel (FP64 ALU bound)
    work = kernel_work(p, sizes)
    dom = max(kern, key=lambda k: kern[k][1])
    launches, ms = kern[dom]
    avg_s = ms / launches / 1e3
    achieved = work.get(dom, 0.0) / avg_s / 1e12
    peak = FP64_NOMINAL_TFLOPS
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": "FP64 dense nominal (no measured FP64 peak)",
                "share_of_step": ms / total_ms}
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (analytic Witsenhausen instance, Section V-A)",
        "config": {"workload": desc, "precision": p["precision"],
                   "l2": "flushed between steps (512 MiB write outside the events)",
                   "parallelism": f"independent solves x{world}"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "gpu_launches": int(sum(v[0] for v in kern.values())),
        "kernels_ms_per_step": {k: v[1] / args.steps for k, v in kern.items()},
        "roofline": roofline, "e2e": e2e, "clocks": clk, "parity": parity,
        "tie_recosts_per_solve": recosts,
    }
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
    p, _ = workload(args.workload, args.precision)
    with binding.Instance(p) as inst:
        inst.sweep(args.profile_sweeps)
        print(json.dumps({"workload": args.workload, "J": inst.eval_J(),
                          "sweeps": args.profile_sweeps}))
    torch.cuda.synchronize()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p, desc = workload(args.workload, args.precision)
    vals = []
    for s in range(args.warmup + args.steps):
        v, cores, sample, spent = oracle_sample(p, args.cpu_budget / 2)
        if s >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": desc, "precision": "oracle FP64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ucp", choices=["ucp", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-sweeps", type=int, default=0,
                    help="only build one instance and run this many sweeps "
                         "(a short, fixed launch sequence for ncu)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_sweeps:
        run_profile(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
