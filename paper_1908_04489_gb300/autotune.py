"""Launch-shape autotuner for the sweep.

The library exposes three knobs that only change how the same work is spread
over threads (``ucp_launch_config``): lanes per x0 point in the screened
search (4, 8, 16), threads sharing a u1 run of targets (1, 2, 4, per run
length) and blocks of the deferred near-tie search per instance.  Every
choice gives the same results bit for bit, so the tuner may pick freely by
speed.  (The u1 tile size and run length would also change speed, but they
change the summation structure of the u1 sums and hence the last bits of
u1, so they stay fixed by the library's rules.)

Search: coordinate descent from the library's rules -- one knob at a time
over its values, a value kept when it is at least ``gain`` faster -- each
configuration timed on the target itself by CUDA events over whole sweeps
(graph replays on a non-default stream).  The winners are cached in a JSON
file keyed by device name and a workload key: the batch size bucket and the
set of (delta, n_w) of the members.
"""
from __future__ import annotations

import json
import os

import numpy as np

KNOBS = ("search_lanes", "u1_threads", "defer_blocks")
LANES = (8, 4, 16)
THREADS = (4, 2, 1)
DEFER = (4, 2, 8, 16, 64)


def default_config() -> dict:
    return {"search_lanes": 0, "u1_threads": [0] * 5, "defer_blocks": 0}


def run_slots(params_list) -> list:
    """Run-length slots (R = 1, 2, 4, 8, 16 -> 0..4) the members use, from
    the library's run-length rule: the exponent change along a run of R
    targets, R delta (Y + max |f|), stays below 15."""
    out = set()
    for p in params_list:
        d = p["delta"]
        hy, hx = round(p["y_half"] / d), round(p["x_half"] / d)
        hr = round(p["cand_half"] / d)
        q = 2 * max(1, -(-hr // (p["n_coarse"] - 1)))
        F = max(hr + 2 * q, hx) * d
        slope = d * (hy * d + F)
        R = 16
        while R > 1 and (R - 1) * slope > 15.0:
            R //= 2
        out.add(R.bit_length() - 1)
    return sorted(out)


def workload_key(params_list) -> str:
    n = len(params_list)
    bucket = 1 << max(0, int(np.ceil(np.log2(max(1, n)))))
    dw = sorted({(round(p["delta"], 9), 2 * round(p["w_half"] / p["delta"]) + 1)
                 for p in params_list})
    return f"n<={bucket}|" + ",".join(f"{d}:{w}" for d, w in dw)


def candidates(cfg: dict, knob: str, slot: int | None = None):
    """Configurations that change one knob of cfg."""
    out = []
    if knob == "search_lanes":
        for v in LANES:
            c = json.loads(json.dumps(cfg))
            c["search_lanes"] = v
            out.append(c)
    elif knob == "u1_threads":
        for v in THREADS:
            if v > (1 << slot):
                continue
            c = json.loads(json.dumps(cfg))
            c["u1_threads"][slot] = v
            out.append(c)
    else:
        for v in DEFER:
            c = json.loads(json.dumps(cfg))
            c["defer_blocks"] = v
            out.append(c)
    return out


def time_config(target, cfg, stream, sweeps=3, reps=3) -> float:
    """Median milliseconds per sweep of `target` (an Instance or a Batch)
    under cfg: one warm-up sweep (graph capture), then reps timed runs of
    `sweeps` sweeps bracketed by CUDA events on the target's stream."""
    import torch
    target.set_launch_config(cfg)
    target.sweep(1)
    ms = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        target.sweep(sweeps)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1) / sweeps)
    return float(np.median(ms))


def tune(target, params_list, stream, sweeps=3, reps=3, gain=0.01):
    """Coordinate descent over the knobs on `target` (swept while tuning;
    use a scratch copy of the workload).  Returns (best config, table of
    (config, ms per sweep) in the order measured)."""
    best = default_config()
    table = []
    best_ms = time_config(target, best, stream, sweeps, reps)
    table.append((json.loads(json.dumps(best)), best_ms))
    steps = [("search_lanes", None)] + [("u1_threads", r) for r in run_slots(params_list)] + \
        [("defer_blocks", None)]
    for knob, slot in steps:
        for c in candidates(best, knob, slot):
            if c == best:
                continue
            ms = time_config(target, c, stream, sweeps, reps)
            table.append((c, ms))
            if ms < best_ms * (1.0 - gain):
                best, best_ms = c, ms
    target.set_launch_config(best)
    return best, table


def cache_path() -> str:
    return os.environ.get("UCP_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ucp",
                                       "launch_shapes.json"))


def load_cache(path=None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def store(device: str, key: str, cfg: dict, ms: float, path=None):
    path = path or cache_path()
    data = load_cache(path)
    data.setdefault(device, {})[key] = {"config": cfg, "ms_per_sweep": ms}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(device: str, key: str, path=None):
    return load_cache(path).get(device, {}).get(key)


def tuned_batch_config(binding, params_list, stream, device: str, retune=False, path=None,
                       sweeps=3, reps=3):
    """The cached configuration of this batch workload on this device, or a
    fresh tuning on a scratch batch of the same members (then cached).
    Returns (config, table or None when it came from the cache)."""
    key = workload_key(params_list)
    hit = None if retune else lookup(device, key, path)
    if hit is not None:
        return hit["config"], None
    with binding.Batch(params_list, stream=stream) as scratch:
        best, table = tune(scratch, params_list, stream, sweeps, reps)
    store(device, key, best, min(ms for _, ms in table), path)
    return best, table
