"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Decisions (winner list positions and the new controller values) must be
bit-exact when both sides start a sweep from the same state; the u1 table and
J must agree within tolerances derived from the FP64 arithmetic (the only
differing operations are exp() ulps and the summation order of the J
reduction).  Independent trajectories must agree to |dJ| <= 1e-9 and
controllers to 1e-6.
"""
import numpy as np
import pytest

import oracle
from paper_1908_04489_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# u1 step: each weight differs by at most a few ulps between exp
# implementations, so U_j moves by <= ~1e-15 * spread(f) ~ 1e-13.
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


def lockstep(binding, p, nu, U, sweeps=1):
    """Run `sweeps` single sweeps, each from the oracle's state."""
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
            assert np.max(np.abs(got["U"] - U1)) <= TOL_U
            assert abs(Jg - o.J(nu1, U1)) <= TOL_J
            nu, U = nu1, U1
    return nu, U


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("init", [0, 1])
def test_lockstep_c1(binding, precision, init):
    p = W.c1()
    p["precision"] = precision
    o = oracle.Oracle(p)
    nu = o.init(init)
    lockstep(binding, p, nu, o.mmse(nu), sweeps=3)


def test_lockstep_plain_path_on_a_grid_that_fills_the_gpu(binding):
    """The plain search takes n_refine lanes per x0 point on grids of more
    than 16 warps per SM (small grids get a warp per point with the
    quadrature split over it); 5001 x0 points take the former."""
    import os
    p = dict(W.c1(), delta=0.01, precision=0)
    o = oracle.Oracle(p)
    assert o.n_x == 5001
    nu = o.init(0)
    oracle.set_threads(os.cpu_count() or 1)
    try:
        lockstep(binding, p, nu, o.mmse(nu), sweeps=1)
    finally:
        oracle.set_threads(1)


@pytest.mark.parametrize("precision", [0, 1])
def test_trajectory_c1(binding, precision):
    """Independent 10-sweep solves of config c1 (identity init)."""
    p = W.c1()
    p["precision"] = precision
    o = oracle.Oracle(p)
    oracle.set_threads(8)
    ref = o.solve(0, p["sweeps"], want_idx=True)
    oracle.set_threads(1)
    with binding.Instance(p) as inst:
        inst.sweep(p["sweeps"])
        Jh = inst.J_history()
        got = inst.get_controllers()
    assert Jh.shape == ref["J"].shape
    assert np.max(np.abs(Jh - ref["J"])) <= 1e-9
    np.testing.assert_array_equal(got["idx"], ref["idx"][-1])
    assert np.max(np.abs(got["f"] - o.value(ref["nu"]))) <= 1e-6
    assert np.max(np.abs(got["U"] - ref["U"])) <= 1e-6


EDGE = [
    dict(n_levels=0),
    dict(n_nbr=0),
    dict(n_refine=2, n_levels=5),
    dict(n_refine=4, n_levels=3),
    dict(n_refine=32, n_levels=2),
    dict(n_coarse=2),
    dict(n_coarse=7),
    dict(x_half=0.1, w_half=0.1, y_half=0.1, cand_half=0.0),   # 3 points each
    dict(cand_half=40.0),                                       # beyond the y range
    dict(y_half=3.0),                                           # heavy clamping
    dict(k=0.05, sigma=1.0, x_half=5.0, cand_half=6.0, y_half=12.0),
    dict(n_nbr=8, x_half=0.5),                                  # neighbours past both ends
]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("extra", EDGE, ids=[str(e) for e in EDGE])
def test_lockstep_edge_cases(binding, precision, extra):
    p = W.small(precision=precision, **extra)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(7)
    g = o.grids()
    nu = o.init(2, g["x"] * 0.9 + rng.normal(0, 0.7, o.n_x))
    lockstep(binding, p, nu, o.mmse(nu), sweeps=2)


@pytest.mark.parametrize("precision", [0, 1])
def test_table_init_and_u0_output(binding, precision):
    p = W.small(precision=precision, init_kind=2)
    o = oracle.Oracle(p)
    g = o.grids()
    table = np.round(g["x"] / 3.0) * 3.0 + 0.123456789
    nu = o.init(2, table)
    with binding.Instance(p, table=table) as inst:
        got = inst.get_controllers(as_paper_u0=True)
        np.testing.assert_array_equal(got["f"], o.value(nu) - g["x"])
        assert np.max(np.abs(got["U"] - o.mmse(nu))) <= TOL_U
        assert np.all(got["idx"] == -1)
        assert abs(inst.eval_J() - o.J(nu, o.mmse(nu))) <= TOL_J


@pytest.mark.parametrize("precision", [0, 1])
def test_staircase_start_equals_the_oracle(binding, precision):
    """The odd staircase start of the c2 workload, set up by the GPU
    (init_kind 1), equals the oracle's start value for value before any
    sweep, at full c2 size (10001 x0 points)."""
    p = W.c2(precision=precision)
    o = oracle.Oracle(p)
    with binding.Instance(p) as inst:
        got = inst.get_controllers()
    np.testing.assert_array_equal(got["f"], o.value(o.init(1)))
    assert np.all(got["idx"] == -1)


def test_full_size_c2_sampled(binding):
    """Config c2 at full size (10001 / 2401 / 14001 points), as the bench runs
    it: after two sweeps, a sampled subset of x_i and y_j is recomputed by the
    oracle from the GPU's own pre-sweep state."""
    p = W.c2(precision=1)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(11)
    with binding.Instance(p) as inst:
        inst.sweep(2)
        pre = inst.get_controllers()
        inst.sweep(1)
        post = inst.get_controllers()
        Jg = inst.eval_J()
    nu_pre = o.init(2, pre["f"])
    assert np.array_equal(o.value(nu_pre), pre["f"])
    oracle.set_threads(8)
    sel = np.unique(np.concatenate([[0, 1, o.n_x - 1], rng.integers(0, o.n_x, 61)]))
    for i in sel:
        nu1, idx = o.search(nu_pre, pre["U"], i, i + 1)
        assert idx[i] == post["idx"][i]
        assert o.value(nu1[i]) == post["f"][i]
    nu_post = o.init(2, post["f"])
    for j in np.unique(np.concatenate([[0, o.n_y - 1], rng.integers(0, o.n_y, 30)])):
        assert abs(o.mmse(nu_post, j, j + 1)[j] - post["U"][j]) <= TOL_U
    assert abs(o.J(nu_post, post["U"]) - Jg) <= TOL_J
    oracle.set_threads(1)


def test_history_and_profile(binding):
    p = W.small(sweeps=3)
    with binding.Instance(p) as inst:
        inst.profile(True)
        inst.sweep(3)
        times = inst.kernel_times()
        Jh = inst.J_history()
    assert len(Jh) == 4 and np.all(np.isfinite(Jh))
    assert times["search"][0] == 3 and times["search"][1] > 0


def test_history_grows_past_initial_capacity(binding):
    p = W.small(x_half=2.0, w_half=2.0, y_half=4.0, cand_half=3.0)
    with binding.Instance(p) as inst:
        inst.sweep(100)
        Jh = inst.J_history()
    assert len(Jh) == 101 and np.all(np.diff(Jh) <= 1e-12)


def test_errors_leave_instance_usable(binding):
    p = W.small()
    with binding.Instance(p) as inst:
        with pytest.raises(binding.UcpError):
            inst.set_controllers(np.zeros(3))
        with pytest.raises(binding.UcpError):
            inst.sweep(-1)
        inst.sweep(1)
        assert np.isfinite(inst.eval_J())


def test_full_size_c5_sampled(binding):
    """Config c5 at full size (100001 / 14001 / 120001 points, 6 levels): after
    one sweep, sampled x_i and y_j are recomputed by the oracle from the
    GPU's own pre-sweep state; decisions must match exactly."""
    p = W.c5(precision=1)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(13)
    with binding.Instance(p) as inst:
        inst.sweep(1)
        pre = inst.get_controllers()
        inst.sweep(1)
        post = inst.get_controllers()
        Jg = inst.eval_J()
        recosts = inst.tie_recosts()
    nu_pre = o.init(2, pre["f"])
    assert np.array_equal(o.value(nu_pre), pre["f"])
    oracle.set_threads(16)
    sel = np.unique(np.concatenate([[0, o.n_x - 1, (o.n_x - 1) // 2],
                                    rng.integers(0, o.n_x, 29)]))
    for i in sel:
        nu1, idx = o.search(nu_pre, pre["U"], i, i + 1)
        assert idx[i] == post["idx"][i]
        assert o.value(nu1[i]) == post["f"][i]
    nu_post = o.init(2, post["f"])
    for j in np.unique(np.concatenate([[0, o.n_y - 1], rng.integers(0, o.n_y, 12)])):
        assert abs(o.mmse(nu_post, j, j + 1)[j] - post["U"][j]) <= TOL_U
    assert abs(o.J(nu_post, post["U"]) - Jg) <= TOL_J
    oracle.set_threads(1)
    assert recosts > 0     # level-6 gaps reach the rounding scale
