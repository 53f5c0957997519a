"""Writes the oracle's trajectories of the batched, served and large workloads
to small JSON fixtures beside this script.  It calls only ``oracle/`` (and the
seeded parameter generators of ``workloads``); no value comes from the GPU.

The oracle's solve of these workloads costs minutes to an hour of host cores
(c3: 1.5e12 quadrature terms over 256 instances; the c4 sample: 200 requests
of up to 20001 x 2401 points for 20 sweeps; c5: 2.2e11 terms per sweep), too
long for a test run, so the tests compare the GPU against what this script
stored.  Per solve it records:

  J        J of the initial state and after every sweep (Section V-A's
           objective, FP64, as the oracle computes it);
  nu_sha   the first 16 hex digits of SHA-256 over the controller's lattice
           indices (int64, little endian) for the initial state and after
           every sweep: equal digests mean bit-identical controllers;
  idx_sha  the same digest over the winners' list positions of the last sweep
           (int32, little endian);
  U_j, U   the final u1 table at 16 seeded y points.

Usage (from the repository root):
  python tests/golden/make_oracle_trajectories.py c3 c4 c5 [--procs N]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"))
                          .tobytes()).hexdigest()[:16]


def trajectory(p, n_sweeps, threads, seed):
    """The oracle's solve, one sweep at a time (the same calls orc_solve
    makes): init -> U = mmse(f) -> J, then per sweep search -> mmse -> J."""
    import oracle
    oracle.set_threads(threads)
    o = oracle.Oracle(p)
    nu = o.init(int(p.get("init_kind", 0)))
    U = o.mmse(nu)
    J = [o.J(nu, U)]
    sha = [digest(nu)]
    idx = None
    for _ in range(n_sweeps):
        nu, idx = o.search(nu, U)
        U = o.mmse(nu)
        J.append(o.J(nu, U))
        sha.append(digest(nu))
    rng = np.random.default_rng(seed)
    js = np.unique(np.concatenate([[0, o.n_y - 1, (o.n_y - 1) // 2],
                                   rng.integers(0, o.n_y, 13)]))
    return dict(J=J, nu_sha=sha, idx_sha=digest(idx) if idx is not None else None,
                U_j=[int(j) for j in js], U=[float(U[j]) for j in js])


def _job(args):
    key, p, n_sweeps, threads, seed = args
    t = time.time()
    r = trajectory(p, n_sweeps, threads, seed)
    r.update(key=key, k=p["k"], sigma=p["sigma"], delta=p["delta"],
             oracle_s=round(time.time() - t, 2))
    return r


def run_pool(jobs, procs):
    ctx = mp.get_context("spawn")
    out = {}
    with ctx.Pool(procs) as pool:
        for r in pool.imap_unordered(_job, jobs):
            out[r["key"]] = r
            print(f"  {r['key']}: {r['oracle_s']} s", flush=True)
    return [out[j[0]] for j in jobs]


def header(what, recipe):
    return dict(what=what, recipe=recipe,
                written_by="tests/golden/make_oracle_trajectories.py (oracle only)",
                oracle="oracle/ucp_oracle.c, FP64, -ffp-contract=off",
                host=f"{platform.machine()} {platform.system()}",
                written=time.strftime("%Y-%m-%d"))


def main():
    from paper_1908_04489_gb300 import workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("which", nargs="+", choices=["c3", "c4", "c5"])
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    for which in a.which:
        t0 = time.time()
        print(which, flush=True)
        if which == "c3":
            ps = W.c3()
            jobs = [(k, p, p["sweeps"], 1, k) for k, p in enumerate(ps)]
            # largest first, so the pool's tail is short
            jobs.sort(key=lambda j: -W.work_estimate(j[1]))
            res = sorted(run_pool(jobs, a.procs), key=lambda r: r["key"])
            doc = header("c3: 256 Witsenhausen instances, seed 1908 stream 0, 10 sweeps, "
                         "identity start", "workloads.c3()")
            doc["members"] = res
        elif which == "c4":
            reqs, _ = W.c4()
            sample = W.c4_sample()
            jobs = [(r, reqs[r], reqs[r]["sweeps"], 1, r) for r in sample]
            jobs.sort(key=lambda j: -W.work_estimate(j[1]))
            res = sorted(run_pool(jobs, a.procs), key=lambda r: r["key"])
            doc = header("c4: the seeded 200-request sample of the 20000-request stream "
                         "(seed 1908 stream 1), 20 sweeps each, identity start",
                         "workloads.c4() at the indices workloads.c4_sample()")
            doc["requests"] = res
        else:
            p = W.c5()
            res = _job(("c5", p, p["sweeps"], a.procs, 5))
            doc = header("c5: k = 0.2, sigma = 10, delta = 0.001 (100001 / 14001 / "
                         "120001 points), 6 levels, identity start, 20 sweeps",
                         "workloads.c5()")
            doc["solve"] = res
        doc["seconds"] = round(time.time() - t0, 1)
        path = os.path.join(HERE, f"oracle_{which}.json")
        with open(path, "w") as fh:
            json.dump(doc, fh, indent=0, separators=(",", ":"))
            fh.write("\n")
        print(f"{which}: wrote {path} in {doc['seconds']} s", flush=True)


if __name__ == "__main__":
    main()
