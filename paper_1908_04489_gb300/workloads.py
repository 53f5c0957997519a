"""Seeded synthetic Witsenhausen workloads (inputs only, no solver arithmetic).

Both the CUDA path and the FP64 oracle take the parameter dicts produced here,
so their inputs are identical.  Every instance is the analytic problem of the
paper's Section V-A: x0 ~ N(0, sigma^2), w ~ N(0, 1); no dataset is involved.

Parameter dict keys: k, sigma, delta, x_half, w_half, y_half, cand_half,
n_coarse, n_refine, n_levels, n_nbr, init_kind (0 identity, 1 odd staircase,
2 table), sweeps, precision (0 plain FP64, 1 fast).

Random draws use splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state advances by the golden
gamma 0x9E3779B97F4A7C15 and each output is the variant-13 mix of the state.
Stream s of seed S starts from state S ^ (s * 0xD1B54A32D192ED03).
"""
from __future__ import annotations

import math

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


class SplitMix64:
    def __init__(self, seed: int, stream: int = 0):
        self.state = (seed ^ ((stream * 0xD1B54A32D192ED03) & MASK)) & MASK

    def next_u64(self) -> int:
        self.state = (self.state + GAMMA) & MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def _snap(v: float, delta: float) -> float:
    """Nearest multiple of delta (grid half widths must be multiples)."""
    return round(v / delta) * delta


def base(**kw):
    p = dict(k=0.2, sigma=5.0, delta=0.05, x_half=25.0, w_half=6.0,
             y_half=35.0, cand_half=30.0, n_coarse=64, n_refine=16,
             n_levels=4, n_nbr=2, init_kind=0, sweeps=10, precision=0)
    p.update(kw)
    return p


def c1():
    """Plain FP64 single instance: k=0.2, sigma=5, delta=0.05 (1001 x0,
    241 w, 1401 y points), identity init, 4 levels, 10 sweeps."""
    return base()


def c2(precision: int = 1):
    """Fine single instance: delta=0.005 (10001 x0, 2401 w, 14001 y points),
    odd 3-step staircase init, 4 levels, 50 sweeps."""
    return base(delta=0.005, init_kind=1, sweeps=50, precision=precision)


def c5(precision: int = 1):
    """Large single instance: k=0.2, sigma=10, delta=0.001 (100001 x0,
    14001 w, 120001 y points), 6 levels, identity init, 20 sweeps."""
    return base(sigma=10.0, delta=0.001, x_half=50.0, w_half=7.0, y_half=60.0,
                cand_half=53.0, n_levels=6, sweeps=20, precision=precision)


def random_instance(rng: SplitMix64, deltas, sweeps: int, precision: int):
    """k log-uniform in [0.05, 0.5], sigma uniform in [1, 10], delta drawn
    uniformly from ``deltas``; x half width 5 sigma, coarse range 6 sigma,
    w half width 6, y half width = coarse range + 6 (all snapped to delta)."""
    k = math.exp(math.log(0.05) + rng.uniform() * (math.log(0.5) - math.log(0.05)))
    sigma = 1.0 + 9.0 * rng.uniform()
    delta = deltas[min(int(rng.uniform() * len(deltas)), len(deltas) - 1)]
    x_half = _snap(5.0 * sigma, delta)
    cand = _snap(6.0 * sigma, delta)
    return base(k=k, sigma=sigma, delta=delta, x_half=x_half, w_half=6.0,
                y_half=_snap(cand + 6.0, delta), cand_half=cand,
                sweeps=sweeps, precision=precision)


def source_channel(precision: int = 0, **kw):
    """Zero-delay source-channel coding (Section V-B): lambda = 2 (k = sqrt 2,
    the control cost k^2 u0^2), x0 ~ N(0, 1), w ~ U(-1, 1); x0 grid [-5, 5],
    w grid [-1, 1], y grid [-7, 7] at delta = 0.02, coarse candidates in
    [-6, 6], 4 levels of 16, identity start, 20 sweeps; plain FP64 path."""
    p = base(k=math.sqrt(2.0), sigma=1.0, delta=0.02, x_half=5.0, w_half=1.0,
             y_half=7.0, cand_half=6.0, problem=1, sweeps=20, precision=precision)
    p.update(kw)
    return p


def work_estimate(p) -> float:
    """Relative cost of one solve of instance p on the fast path, from its
    grid sizes alone: the search and the box step grow with the x0 points,
    the u1 sums with the y points, the correlation tables with both times the
    taps (used to balance instances across GPUs)."""
    d = p["delta"]
    n_x = 2 * round(p["x_half"] / d) + 1
    n_w = 2 * round(p["w_half"] / d) + 1
    n_y = 2 * round(p["y_half"] / d) + 1
    return float(p.get("sweeps", 1)) * (n_x + n_y + (n_x + n_y) * n_w / 256.0)


def partition(ps, parts: int):
    """Split instances over `parts` GPUs by estimated work: longest first to
    the least loaded part (ties to the lower part and the lower index), each
    part's indices in increasing order.  Deterministic."""
    order = sorted(range(len(ps)), key=lambda k: (-work_estimate(ps[k]), k))
    load = [0.0] * parts
    out = [[] for _ in range(parts)]
    for k in order:
        r = min(range(parts), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += work_estimate(ps[k])
    return [sorted(o) for o in out]


def c3(n: int = 256, seed: int = 1908, precision: int = 1):
    """Batched: n instances, seed 1908 stream 0, delta in {0.01, 0.02},
    identity init, 10 sweeps."""
    rng = SplitMix64(seed, 0)
    return [random_instance(rng, (0.01, 0.02), 10, precision) for _ in range(n)]


def c4(n: int = 20000, rate: float = 1000.0, seed: int = 1908,
       precision: int = 1):
    """Serving: n requests (params from stream 1, delta in {0.05, 0.01,
    0.005}, 20 sweeps) with exponential inter-arrival times at ``rate``/s
    (stream 2).  Returns (list of params, list of arrival times in s)."""
    rp = SplitMix64(seed, 1)
    ra = SplitMix64(seed, 2)
    reqs, t, times = [], 0.0, []
    for _ in range(n):
        reqs.append(random_instance(rp, (0.05, 0.01, 0.005), 20, precision))
        t += -math.log(1.0 - ra.uniform()) / rate
        times.append(t)
    return reqs, times


def c4_sample(n_sample: int = 200, n: int = 20000, seed: int = 1908):
    """Indices of a seeded sample of the c4 request stream (the parameters of
    c4 do not depend on the arrival rate): ``n_sample`` distinct request
    numbers in [0, n), drawn by a partial Fisher-Yates shuffle on seed 1908
    stream 3, returned in increasing order."""
    rng = SplitMix64(seed, 3)
    perm = list(range(n))
    for k in range(n_sample):
        r = k + min(int(rng.uniform() * (n - k)), n - k - 1)
        perm[k], perm[r] = perm[r], perm[k]
    return sorted(perm[:n_sample])


def small(**kw):
    """A small instance for unit tests: delta=0.1 and narrow grids."""
    p = base(delta=0.1, x_half=12.0, w_half=4.0, y_half=20.0, cand_half=15.0,
             n_levels=3, sweeps=3)
    p.update(kw)
    return p


CONFIGS = {"c1": c1, "c2": c2, "c5": c5}
