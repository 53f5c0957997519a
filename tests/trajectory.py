"""Helpers of the trajectory parity tests: whole solves on the GPU against the
FP64 oracle's own solves (not the oracle re-evaluating the GPU's state).

A trajectory is a list of states, one per sweep (entry 0 = the start after
the first u1 step): f values, the u1 table U, J, and the winners' list
positions of the sweep that produced the state.

Where both sides make the same decisions the controllers are bit-identical at
every sweep.  The u1 tables of the two sides differ by exp() ulps and by the
GPU's summation order (max |dU| = eps, ~1e-13), and a decision between two
candidates whose costs are that close can go either way.  With |U - U'| <= eps
the marginal cost of one candidate (Section V-A) moves by at most
2 eps sqrt(S) + eps^2, S the quadrature part of the cost (Cauchy-Schwarz over
the normalised weights).  A near-tie at one refinement level changes the
centre of the next, so a flipped decision can end anywhere along another
branch of the coarse-to-fine search.  At the first sweep whose decisions
differ (the controllers before it bit-identical, the tables within rounding)
first_divergence() replays the oracle's search for every x_i where the new f
differ, under the oracle's table, branching at every stage over the
candidates within that allowance of the stage minimum, and asserts that the
GPU's (value, list position) is one of the reachable winners.  Later sweeps
start from different controllers and are counted, not replayed; J is bounded
by |dJ| <= 1e-9 after every sweep throughout, and where every decision
agreed, U within 1e-6.  (A near-tie between two distant values -- f at the
edge of a step of the staircase -- moves U by up to the step height in the
thin transition zones where that source dominates, which J weighs by ~1e-9
or less.)
"""
from __future__ import annotations

import numpy as np

import oracle

TOL_J = 1e-9


def oracle_trajectory(p, n_sweeps, threads=None, table=None):
    """The oracle's solve one sweep at a time (the calls orc_solve makes)."""
    import os
    oracle.set_threads(threads or os.cpu_count() or 1)
    try:
        o = oracle.Oracle(p)
        nu = o.init(int(p.get("init_kind", 0)), table)
        U = o.mmse(nu)
        out = [dict(nu=nu, U=U, J=o.J(nu, U), idx=None)]
        for _ in range(n_sweeps):
            nu, idx = o.search(nu, U)
            U = o.mmse(nu)
            out.append(dict(nu=nu, U=U, J=o.J(nu, U), idx=idx))
    finally:
        oracle.set_threads(1)
    return o, out


def gpu_trajectory_instance(binding, p, n_sweeps, stream=None, table=None):
    """One GPU instance swept one sweep at a time, its state read after each."""
    out = []
    with binding.Instance(p, table=table, stream=stream) as inst:
        st = inst.get_controllers()
        out.append(dict(f=st["f"], U=st["U"], idx=None))
        for _ in range(n_sweeps):
            inst.sweep(1)
            st = inst.get_controllers()
            out.append(dict(f=st["f"], U=st["U"], idx=st["idx"]))
        Jh = inst.J_history()
    for s, J in enumerate(Jh):
        out[s]["J"] = float(J)
    return out


def allow_of(g, eps):
    """Largest gap between two candidates' oracle costs (the larger one g) that
    a table difference eps can reverse: each cost moves by at most
    2 eps sqrt(S) + eps^2 with S <= g, plus both sides' rounding of the
    fixed-order quadrature (< 40 ulps of g each)."""
    g = max(g, 0.0)
    return 2.0 * (2.0 * eps * np.sqrt(g) + eps * eps) + 1e-14 * g


def _first_minima(cands, eps):
    """Candidates (nu, g, pos) in list order that can be the first strict
    minimum when every cost may move by half the allowance: those within the
    allowance of the minimum, each value at its first position."""
    gmin = min(c[1] for c in cands)
    out, seen = [], set()
    for c in cands:
        if c[1] - gmin <= allow_of(c[1], eps) and c[0] not in seen:
            out.append(c)
            seen.add(c[0])
    return out


def possible_winners(o, U, nu_pre, i, eps):
    """Every (lattice value, list position) the candidate search of x_i can
    end on when the costs it compares are the oracle's under table U, each
    moved by at most the allowance for eps: the search replayed with every
    near-tie branched (stage 0 = incumbent, neighbours and coarse values; then
    each level refines around the best so far)."""
    p = o.params
    r, nc, nr, L = p["n_nbr"], p["n_coarse"], p["n_refine"], p["n_levels"]
    nus, gs, _ = o.candidates(nu_pre, U, i)
    n0 = 1 + 2 * r + nc
    states = _first_minima([(int(nus[k]), float(gs[k]), k) for k in range(n0)], eps)
    bits = int(round(np.log2(nr // 2)))
    hr = round(p["cand_half"] / p["delta"])
    q = 2 * max(1, -(-hr // (nc - 1)))
    pos = n0
    ms = list(range(-nr // 2, 0)) + list(range(1, nr // 2 + 1))
    for lv in range(1, L + 1):
        h = q << (bits * (L - lv))
        nxt = {}
        for b in states:
            cands = [b] + [(b[0] + m * h, o.cost(U, i, b[0] + m * h), pos + k)
                           for k, m in enumerate(ms)]
            for c in _first_minima(cands, eps):
                nxt[(c[0], c[2])] = c
        states = list(nxt.values())
        pos += nr
    return {(c[0], c[2]) for c in states}


def first_divergence(o, pre, post, what="", threads=None):
    """The first sweep whose decisions differ: `pre` is the GPU's state
    before it (controller bit-identical to the oracle's, u1 table within
    rounding), `post` the GPU's state after it.  The oracle recomputes its own
    table from that controller and its own decisions; every x_i where the
    GPU's winner differs must be one the oracle's search can end on when its
    costs move within what the tables' difference eps allows.  Returns a
    report (points, eps, the oracle's cost gaps of the GPU's winners)."""
    import os
    oracle.set_threads(threads or os.cpu_count() or 1)
    try:
        nu_pre = o.init(2, pre["f"])
        U_o = o.mmse(nu_pre)
        nu_o, _ = o.search(nu_pre, U_o)
    finally:
        oracle.set_threads(1)
    eps = float(np.max(np.abs(pre["U"] - U_o)))
    nu_g = o.init(2, post["f"])
    diff = np.nonzero(nu_g != nu_o)[0]
    gaps = []
    for i in diff:
        win = possible_winners(o, U_o, nu_pre, int(i), eps)
        got = (int(nu_g[i]), int(post["idx"][i]))
        assert got in win, (what, int(i), got, sorted(win), eps)
        gaps.append(o.cost(U_o, int(i), got[0]) - o.cost(U_o, int(i), int(nu_o[i])))
    return dict(points=int(diff.size), eps=eps,
                max_abs_gap=float(max((abs(x) for x in gaps), default=0.0)),
                max_df=float(np.max(np.abs(o.value(nu_g) - o.value(nu_o)))) if diff.size else 0.0)


def check(o, gpu, orc, what=""):
    """Assert |dJ| <= 1e-9 per sweep; where every decision agreed, U within
    1e-6; at the first sweep whose decisions differ, that each differing
    decision is a near-tie the tables' difference can reverse (later sweeps
    start from different controllers and are counted, not replayed).
    Returns a report."""
    assert len(gpu) == len(orc)
    dJ = [abs(g["J"] - c["J"]) for g, c in zip(gpu, orc)]
    rep = dict(what=what, sweeps=len(orc) - 1, max_dJ=max(dJ), first_diff_sweep=None,
               diff_points=[], first=None, max_dU=0.0)
    assert max(dJ) <= TOL_J, (what, max(dJ), int(np.argmax(dJ)))
    np.testing.assert_array_equal(gpu[0]["f"], o.value(orc[0]["nu"]))
    for s in range(1, len(orc)):
        diff = np.nonzero(gpu[s]["f"] != o.value(orc[s]["nu"]))[0]
        rep["diff_points"].append(int(diff.size))
        if diff.size and rep["first_diff_sweep"] is None:
            rep["first_diff_sweep"] = s
            rep["first"] = first_divergence(o, gpu[s - 1], gpu[s], what)
    rep["max_dU"] = float(np.max(np.abs(gpu[-1]["U"] - orc[-1]["U"])))
    rep["max_df"] = float(np.max(np.abs(gpu[-1]["f"] - o.value(orc[-1]["nu"]))))
    rep["final_diff_points"] = rep["diff_points"][-1] if rep["diff_points"] else 0
    if rep["first_diff_sweep"] is None:
        # the same decisions throughout: the controllers are bit-identical
        # and u1 differs only by the rounding of its sums
        assert rep["max_dU"] <= 1e-6, (what, rep["max_dU"])
    return rep
