"""Algorithm 1's outer loop on the GPU (Sections III-B to III-D) against the
FP64 oracle, through the C ABI (ucp_local_update, ucp_solve).

  - lockstep: from the oracle's state, one local-update iteration (Newton's
    step for every x0 point, then the u1 step and J) gives bit-identical
    controller values, u1 within 1e-11 and J within 1e-11 -- on c1 from three
    starts, edge configurations and the source-channel problem, both paths;
  - whole runs: ucp_solve (N = 20, p = 1e-10, Section IV) from the identity
    against the oracle's Algorithm 1: the same rounds and splits, J after
    every phase within 1e-9, and the paper's value for its problem within a
    plausibility band.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1908_04489_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_U = 1e-11
TOL_J = 1e-11


@pytest.fixture(scope="module")
def binding():
    import torch
    assert torch.cuda.is_available()
    from paper_1908_04489_gb300 import binding as b, build
    build.build()
    b.load()
    return b


def lockstep_local(binding, p, nu, U, iters=2):
    o = oracle.Oracle(p)
    with binding.Instance(p) as inst:
        for _ in range(iters):
            inst.set_controllers(o.value(nu), U)
            inst.local_update(1)
            got = inst.get_controllers(want=("f", "U"))
            Jg = inst.eval_J()
            nu1 = o.local_update(nu, U)
            np.testing.assert_array_equal(got["f"], o.value(nu1))
            U1 = o.mmse(nu1)
            assert np.max(np.abs(got["U"] - U1)) <= TOL_U
            assert abs(Jg - o.J(nu1, U1)) <= TOL_J
            nu, U = nu1, U1


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("start", ["identity", "staircase", "noisy"])
def test_local_update_lockstep_c1(binding, precision, start):
    p = dict(W.c1(), precision=precision)
    o = oracle.Oracle(p)
    if start == "noisy":
        rng = np.random.default_rng(17)
        nu = o.init(2, o.grids()["x"] * 0.8 + rng.normal(0, 0.5, o.n_x))
    else:
        nu = o.init(0 if start == "identity" else 1)
    U = o.mmse(nu)
    if start == "staircase":          # a state partway through a solve
        nu, _ = o.search(nu, U)
        U = o.mmse(nu)
    lockstep_local(binding, p, nu, U)


EDGE = [dict(y_half=3.0), dict(cand_half=40.0), dict(n_levels=0, n_refine=2),
        dict(x_half=0.1, w_half=0.1, y_half=0.1, cand_half=0.0)]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("extra", EDGE, ids=[str(e) for e in EDGE])
def test_local_update_lockstep_edge_cases(binding, precision, extra):
    p = W.small(precision=precision, **extra)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(19)
    nu = o.init(2, o.grids()["x"] * 1.1 + rng.normal(0, 1.0, o.n_x))
    lockstep_local(binding, p, nu, o.mmse(nu))


def test_local_update_lockstep_source_channel(binding):
    p = W.source_channel()
    o = oracle.Oracle(p)
    nu = o.init(0)
    U = o.mmse(nu)
    nu, _ = o.search(nu, U)
    lockstep_local(binding, p, nu, o.mmse(nu))


def paper_value(key):
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_values.json")))
    return gold[key]["value"]


def compare_runs(o, got, ref):
    assert got["rounds"] == ref["rounds"] and got["converged"] == ref["converged"]
    np.testing.assert_array_equal(got["N_L_rounds"], ref["N_L_rounds"])
    assert got["local_iters"] == ref["local_iters"]
    assert got["exhaustion_iters"] == ref["exhaustion_iters"]
    assert np.max(np.abs(got["J_phase"] - ref["J_phase"])) <= 1e-9
    assert abs(got["J"] - ref["J"]) <= 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_algorithm1_c1_against_the_oracle(binding, precision):
    """Algorithm 1 from the identity (Section III-D) with N = 20 and
    p = 1e-10 (Section IV) on the c1 grid: the GPU's rounds, splits and J
    after every phase against the oracle's; the converged J near the value
    Section V-A prints for k = 0.2, sigma = 5."""
    p = dict(W.c1(), precision=precision)
    o = oracle.Oracle(p)
    oracle.set_threads(os.cpu_count() or 1)
    try:
        ref = o.algorithm1(0, N=20, precision=1e-10, max_rounds=60)
    finally:
        oracle.set_threads(1)
    with binding.Instance(p) as inst:
        got = inst.solve(N=20, precision=1e-10, max_rounds=60)
        f = inst.get_controllers(want=("f",))["f"]
    compare_runs(o, got, ref)
    assert got["converged"] == 1
    assert np.max(np.abs(f - o.value(ref["nu"]))) <= 1e-6
    assert abs(got["J"] - paper_value("witsenhausen_k0.2_sigma5_J")) < 1e-4
    print(f"c1 Algorithm 1 (precision {precision}): {got['rounds']} rounds, "
          f"{got['local_iters']} local updates, {got['exhaustion_iters']} sweeps, "
          f"J = {got['J']:.9f}")


def test_algorithm1_source_channel_against_the_oracle(binding):
    """The same loop on zero-delay source-channel coding (Section V-B, plain
    FP64 path) against the oracle; the paper's value within 0.01."""
    p = W.source_channel()
    o = oracle.Oracle(p)
    oracle.set_threads(os.cpu_count() or 1)
    try:
        ref = o.algorithm1(0, N=20, precision=1e-10, max_rounds=40)
    finally:
        oracle.set_threads(1)
    with binding.Instance(p) as inst:
        got = inst.solve(N=20, precision=1e-10, max_rounds=40)
    compare_runs(o, got, ref)
    assert abs(got["J"] - paper_value("source_channel_lambda2_J")) < 0.01
    print(f"source-channel Algorithm 1: {got['rounds']} rounds, J = {got['J']:.9f}, "
          f"converged {got['converged']}")


def test_solve_rejects_bad_parameters(binding):
    with binding.Instance(W.small()) as inst:
        for kw in (dict(N=1), dict(max_rounds=-1), dict(precision=-1.0),
                   dict(precision=float("nan"))):
            with pytest.raises(binding.UcpError):
                inst.solve(**kw)
        with pytest.raises(binding.UcpError):
            inst.local_update(-1)
        inst.solve(max_rounds=0)          # no round: nothing changes
        inst.local_update(0)
        assert np.isfinite(inst.eval_J())
