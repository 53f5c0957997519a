"""GPU parity of the second problem on the same sweep: zero-delay
source-channel coding (Section V-B; x1 = u0(x0) + w, w ~ U(-1, 1),
J = E[lambda u0^2 + (u1(x1) - x0)^2], f = u0), plain FP64 path, through the
C ABI, against the FP64 oracle.

As for Witsenhausen's problem: from the same state the winner list positions
and new controller values are bit-exact, U and J agree within 1e-11 (exp
ulps only); independent trajectories agree to |dJ| <= 1e-9.
"""
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


def lockstep(binding, p, nu, U, sweeps, tol_u=TOL_U):
    o = oracle.Oracle(p)
    with binding.Instance(p) as inst:
        for _ in range(sweeps):
            inst.set_controllers(o.value(nu), U)
            inst.sweep(1)
            got = inst.get_controllers()
            Jg = inst.eval_J()
            nu1, idx = o.search(nu, U)
            np.testing.assert_array_equal(got["idx"], idx)
            np.testing.assert_array_equal(got["f"], o.value(nu1))
            U1 = o.mmse(nu1)
            assert np.max(np.abs(got["U"] - U1)) <= tol_u
            assert abs(Jg - o.J(nu1, got["U"])) <= TOL_J
            nu, U = nu1, U1


@pytest.mark.parametrize("precision", [0, 1], ids=["plain", "fast"])
@pytest.mark.parametrize("start", ["identity", "noisy", "flat"])
def test_lockstep_source_channel(binding, start, precision):
    """precision 1: the screened search on the three tables (decisions bit
    for bit, the weights being equal and exp-free) and the warp u1 step."""
    p = W.source_channel(precision=precision)
    o = oracle.Oracle(p)
    g = o.grids()
    if start == "identity":
        nu = o.init(0)
    elif start == "noisy":
        rng = np.random.default_rng(11)
        nu = o.init(2, np.clip(1.3 * g["x"] + rng.normal(0, 0.4, o.n_x), -5.5, 5.5))
    else:   # a two-level start: windows beyond both levels use the nearest sources
        nu = o.init(2, np.where(g["x"] < 0, -0.8, 0.8))
    lockstep(binding, p, nu, o.mmse(nu), sweeps=3)


@pytest.mark.parametrize("extra", [dict(n_nbr=0), dict(n_refine=4, n_levels=3),
                                   dict(y_half=2.0), dict(cand_half=9.0, y_half=9.0)],
                         ids=["no neighbours", "n_refine 4", "clamped y", "wide candidates"])
@pytest.mark.parametrize("precision", [0, 1], ids=["plain", "fast"])
def test_lockstep_source_channel_edges(binding, extra, precision):
    p = W.source_channel(precision=precision, **extra)
    o = oracle.Oracle(p)
    g = o.grids()
    rng = np.random.default_rng(5)
    nu = o.init(2, g["x"] + rng.normal(0, 0.5, o.n_x))
    lockstep(binding, p, nu, o.mmse(nu), sweeps=2)


def test_trajectory_source_channel(binding):
    """Independent 20-sweep solves from the identity: J within 1e-9 per
    sweep, the same final decisions, and the value of Section V-B (0.890756)
    within 0.01."""
    p = W.source_channel()
    o = oracle.Oracle(p)
    ref = o.solve(0, p["sweeps"], want_idx=True)
    with binding.Instance(p) as inst:
        inst.sweep(p["sweeps"])
        Jh = inst.J_history()
        got = inst.get_controllers()
        u0 = inst.get_controllers(as_paper_u0=True)["f"]
    assert np.max(np.abs(Jh - ref["J"])) <= 1e-9
    np.testing.assert_array_equal(got["idx"], ref["idx"][-1])
    assert np.max(np.abs(got["f"] - o.value(ref["nu"]))) <= 1e-6
    assert np.max(np.abs(got["U"] - ref["U"])) <= 1e-6
    np.testing.assert_array_equal(u0, got["f"])        # f is u0 itself here
    assert abs(Jh[-1] - 0.890756) < 0.01


def test_fast_mode_makes_the_plain_decisions(binding):
    """From the same controllers and u1 table the fast mode's screened search
    returns the plain search's values and list positions bit for bit, sweep
    after sweep of a 20-sweep run (each sweep restarted from the plain
    instance's state)."""
    p0 = W.source_channel()
    p1 = W.source_channel(precision=1)
    with binding.Instance(p0) as a, binding.Instance(p1) as b:
        for s in range(p0["sweeps"]):
            st = a.get_controllers()
            b.set_controllers(st["f"], st["U"])
            a.sweep(1)
            b.sweep(1)
            ga, gb = a.get_controllers(), b.get_controllers()
            np.testing.assert_array_equal(ga["idx"], gb["idx"])
            np.testing.assert_array_equal(ga["f"], gb["f"])
            assert np.max(np.abs(ga["U"] - gb["U"])) <= TOL_U


def test_fast_mode_trajectory(binding):
    """Independent 20-sweep solves, fast mode against the oracle's own: J
    within 1e-9 per sweep up to and including the first sweep whose decisions
    differ (u1 differs from the oracle's by roundings only); the final J near
    Section V-B's value."""
    p = W.source_channel(precision=1)
    o = oracle.Oracle(p)
    fs = []
    with binding.Instance(p) as inst:
        for _ in range(p["sweeps"]):
            inst.sweep(1)
            fs.append(inst.get_controllers(want=("f",))["f"])
        Jh = inst.J_history()
    nu = o.init(0)
    U = o.mmse(nu)
    assert abs(Jh[0] - o.J(nu, U)) <= 1e-9
    for s in range(p["sweeps"]):
        nu, _ = o.search(nu, U)
        U = o.mmse(nu)
        assert abs(Jh[s + 1] - o.J(nu, U)) <= 1e-9, s
        if not np.array_equal(fs[s], o.value(nu)):
            break
    assert abs(Jh[-1] - 0.890756) < 0.01


def test_batches_and_the_server_refuse_problem_1(binding):
    p = W.source_channel(precision=1)
    with pytest.raises(binding.UcpError) as e:
        binding.Batch([p, p])
    assert "problem 0" in str(e.value)
