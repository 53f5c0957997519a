"""The 2-dimensional Witsenhausen counterexample (Section V-D) on the GPU
against the FP64 2-D oracle, through the ucp2_* C-ABI.

  - lockstep: before every sweep the GPU's own state (f, U) is handed to the
    oracle, whose search from that state must reproduce the GPU's decisions
    (lattice values and list positions) bit for bit except at near-ties,
    where the GPU's result must be one the oracle's search reaches with the
    tie broken either way; the GPU's u1 tables must equal the oracle's u1
    step of the GPU's controllers and the GPU's J the oracle's J of the
    GPU's state;
  - whole solves: the GPU's trajectory against the oracle's own solve, J
    within 1e-9 up to and including the first sweep whose decisions differ;
  - J: exact (1e-13) with the direct forms; from the correlation tables in
    the screened mode, within half the prior-weighted certified bound;
  - a start from a table, set_controllers, argument errors;
  - a grid of several warps' worth of candidates (the list longer than 32)
    with the window leaving the grid, sampled points against the oracle.
The only differences between the two sides are the exp() of the weights and
of the u1 step (ulps); everything else is the same FP64 arithmetic in the
same order, so decisions agree except where two candidates' costs are equal
to within ~1e-14 of the cost.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P2 = dict(k=0.2, sigma=5.0, delta=1.25, x_half=12.5, w_half=5.0, y_half=20.0,
          cand_half=15.0, n_coarse=7, n_levels=6, n_nbr=2)
# Finer axis, more coarse values than a warp has lanes, window radius 3.
P2B = dict(k=0.25, sigma=4.0, delta=0.625, x_half=10.0, w_half=3.75, y_half=17.5,
           cand_half=13.75, n_coarse=9, n_levels=8, n_nbr=3)


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1908_04489_gb300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="module")
def O():
    import oracle
    oracle.build()
    return oracle


def allow(g):
    """Cost gap two FP64 evaluations of one candidate can differ by when the
    only difference is the weights' exp() ulps (each of the fixed-order sum's
    terms moves by a few ulps of itself)."""
    return 1e-14 * max(g, 1e-300)


def q_of(p):
    hr = round(p["cand_half"] / p["delta"])
    return 2 * max(1, -(-hr // (p["n_coarse"] - 1)))


def first_minima(cands):
    gmin = min(c[1] for c in cands)
    out, seen = [], set()
    for c in cands:
        if c[1] - gmin <= allow(c[1]) and c[0] not in seen:
            out.append(c)
            seen.add(c[0])
    return out


def possible_winners(o, U, nu_pre, i):
    """Every (value pair, list position) the oracle's search of point i ends
    on with each near-tie broken either way: stage 0 (incumbent, window,
    coarse grid) as listed, then each level's 8 neighbours around every
    surviving best."""
    p = o.params
    nus, gs, _ = o.candidates(nu_pre, U, i)
    side = 2 * p["n_nbr"] + 1
    n0 = side * side + p["n_coarse"] ** 2
    states = first_minima([((int(nus[k, 0]), int(nus[k, 1])), float(gs[k]), k)
                           for k in range(n0)])
    q, L = q_of(p), p["n_levels"]
    pos = n0
    moves = [(s, t) for s in (-1, 0, 1) for t in (-1, 0, 1) if (s, t) != (0, 0)]
    for lv in range(1, L + 1):
        h = q << (L - lv)
        nxt = {}
        for b in states:
            cands = [b]
            for k, (s, t) in enumerate(moves):
                v = (b[0][0] + s * h, b[0][1] + t * h)
                cands.append((v, o.cost(U, i, *v), pos + k))
            for c in first_minima(cands):
                nxt[(c[0], c[2])] = c
        states = list(nxt.values())
        pos += 8
    return {(c[0], c[2]) for c in states}


def J_bound(o, nu, U, J):
    """How far the screened mode's J (table costs) may be from the exact J:
    half the prior-weighted certified bound of the table costs,
    eps_k (M_i + g_i) with eps_k = (4 n_w + 512) 2^-53 and M_i =
    |u_i|^2 + 2 |u_i|_1 max|U| + 2 max|U|^2, plus the sums' rounding."""
    px, _ = o.weights()
    u = o.value(nu)
    um = float(np.max(np.abs(U)))
    M = (u * u).sum(1) + 2.0 * np.abs(u).sum(1) * um + 2.0 * um * um
    eps_k = (4 * o.n_w + 512) * 2.0 ** -53
    return 0.5 * eps_k * (float(px @ M) + 2.0 * J) + 1e-13 * J


def close_J(o, nu, U, J_gpu, J_or, exact):
    if exact:
        return abs(J_gpu - J_or) <= 1e-13 * J_or
    return abs(J_gpu - J_or) <= J_bound(o, nu, U, J_or)


def lattice(o, f):
    """Lattice indices of GPU f values (exact: they are lattice values)."""
    nu = np.rint(np.ldexp(f / o.params["delta"], o.shift)).astype(np.int64)
    assert np.array_equal(o.value(nu), f)
    return nu


def check_sweep(o, nu_pre, U_pre, f_post, idx_post, points=None):
    """The oracle's search from the GPU's pre-sweep state against the GPU's
    decisions; returns the number of near-tie differences."""
    nu_gpu = lattice(o, f_post)
    if points is None:
        nu_o, idx_o = o.search(nu_pre, U_pre)
        points = np.arange(o.N)
    else:
        nu_o = np.empty((o.N, 2), dtype=np.int64)
        idx_o = np.full(o.N, -1, dtype=np.int32)
        for i in points:
            a, b = o.search(nu_pre, U_pre, int(i), int(i) + 1)
            nu_o[i], idx_o[i] = a[i], b[i]
    ties = 0
    for i in points:
        if np.array_equal(nu_o[i], nu_gpu[i]) and idx_o[i] == idx_post[i]:
            continue
        win = possible_winners(o, U_pre, nu_pre, int(i))
        key = ((int(nu_gpu[i, 0]), int(nu_gpu[i, 1])), int(idx_post[i]))
        assert key in win, (i, key, nu_o[i], idx_o[i], win)
        ties += 1
    return ties


def test_start_equals_the_oracle(B, O):
    o = O.Oracle2D(P2)
    with B.Instance2D(P2) as g:
        assert (g.n_x, g.n_w, g.n_y, g.n_cand) == (o.n_x, o.n_w, o.n_y, o.n_cand)
        st = g.get_controllers()
        nu0 = o.init(0)
        assert np.array_equal(st["f"], o.value(nu0))
        assert np.all(st["idx"] == -1)
        U0 = o.mmse(nu0)
        assert np.max(np.abs(st["U"] - U0)) <= 1e-12
        J = g.J_history()
        assert len(J) == 1
        assert close_J(o, nu0, st["U"], J[0], o.J(nu0, st["U"]), exact=False)
    with B.Instance2D(dict(P2, direct=1)) as g:
        J = g.J_history()
        st = g.get_controllers()
        assert close_J(o, nu0, st["U"], J[0], o.J(nu0, st["U"]), exact=True)
        assert abs(J[0] - o.J(nu0, U0)) <= 1e-12 * J[0]


@pytest.mark.parametrize("direct", [0, 3], ids=["fast", "direct"])
@pytest.mark.parametrize("p,sweeps", [(P2, 8), (P2B, 3)], ids=["P2", "P2B"])
def test_lockstep(B, O, p, sweeps, direct):
    o = O.Oracle2D(p)
    ties = 0
    with B.Instance2D(dict(p, direct=direct)) as g:
        for s in range(sweeps):
            pre = g.get_controllers()
            nu_pre = lattice(o, pre["f"])
            g.sweep(1)
            post = g.get_controllers()
            ties += check_sweep(o, nu_pre, pre["U"], post["f"], post["idx"])
            nu_post = lattice(o, post["f"])
            assert np.max(np.abs(post["U"] - o.mmse(nu_post))) <= 1e-11, s
            J = g.J_history()
            assert len(J) == s + 2
            assert close_J(o, nu_post, post["U"], J[-1], o.J(nu_post, post["U"]),
                           exact=bool(direct & 1)), s
    # Mirror-image candidates have equal costs up to rounding, and the
    # weights' exp() ulps decide some of those ties the other way.
    assert ties <= max(2, o.N * sweeps // 50), ties


def test_whole_solve_matches_the_oracle(B, O):
    o = O.Oracle2D(P2)
    n = 10
    ref = o.solve(n)
    traj = []
    with B.Instance2D(P2) as g:
        traj.append(g.get_controllers())
        for _ in range(n):
            g.sweep(1)
            traj.append(g.get_controllers())
        J = g.J_history()
    assert len(J) == n + 1
    # Oracle states one sweep at a time (the same calls solve() makes).
    nu = o.init(0)
    U = o.mmse(nu)
    for s in range(n + 1):
        if s:
            nu, _ = o.search(nu, U)
            U = o.mmse(nu)
        Jo = o.J(nu, U)
        assert abs(J[s] - Jo) <= 1e-9, (s, J[s], Jo)
        nu_gpu = lattice(o, traj[s]["f"])
        if not np.array_equal(nu_gpu, nu):
            # The first differing sweep: its differences are near-ties of the
            # oracle's search from the GPU's previous state.
            nu_pre = lattice(o, traj[s - 1]["f"])
            check_sweep(o, nu_pre, traj[s - 1]["U"], traj[s]["f"], traj[s]["idx"])
            break
    else:
        assert abs(J[-1] - ref["J"][-1]) <= 1e-9
    assert J[-1] < J[0]


def test_table_start_and_set_controllers(B, O):
    o = O.Oracle2D(P2)
    xs = o.grid(o.n_x)
    h = np.sign(xs) * np.minimum(np.abs(xs), 7.5) * 1.5   # a saturating affine map
    tab = np.stack([np.repeat(h, o.n_x), np.tile(h, o.n_x)], axis=1)
    nu = o.init(2, tab)
    with B.Instance2D(P2, init_f=tab) as g:
        st = g.get_controllers()
        assert np.array_equal(st["f"], o.value(nu))
        assert np.max(np.abs(st["U"] - o.mmse(nu))) <= 1e-11
        J0 = g.J_history()[0]
        assert close_J(o, nu, st["U"], J0, o.J(nu, st["U"]), exact=False)
        # set_controllers without U runs the u1 step; with U keeps it.
        g.set_controllers(o.value(o.init(0)))
        st2 = g.get_controllers()
        assert np.array_equal(st2["f"], o.value(o.init(0)))
        assert np.max(np.abs(st2["U"] - o.mmse(o.init(0)))) <= 1e-11
        U_any = np.full((o.n_y ** 2, 2), 0.5)
        g.set_controllers(st["f"], U_any)
        st3 = g.get_controllers()
        assert np.array_equal(st3["U"], U_any)
        J3 = g.J_history()[-1]
        assert close_J(o, nu, U_any, J3, o.J(nu, U_any), exact=False)
        g.sweep(2)
        assert len(g.J_history()) == 3


def test_argument_errors(B):
    bad = dict(P2, x_half=12.4)
    with pytest.raises(B.UcpError):
        B.Instance2D(bad)
    with pytest.raises(B.UcpError):
        B.Instance2D(dict(P2, n_coarse=1))
    with B.Instance2D(P2) as g:
        with pytest.raises(B.UcpError):
            g.set_controllers(np.zeros(5))
        f = np.zeros((g.n_x ** 2, 2))
        f[3, 1] = np.inf
        with pytest.raises(B.UcpError):
            g.set_controllers(f)
        with pytest.raises(B.UcpError):
            g.sweep(-1)
        g.sweep(1)   # the instance is still usable after rejected calls
        assert len(g.J_history()) == 2


def test_larger_grid_sampled(B, O):
    """n_x = 41, a list of 25 + 81 + 64 = 170 candidates per point (window
    radius 3 leaving the grid at the border): sampled points, three sweeps."""
    p = dict(k=0.2, sigma=5.0, delta=0.625, x_half=12.5, w_half=3.75, y_half=20.0,
             cand_half=15.0, n_coarse=9, n_levels=8, n_nbr=2)
    o = O.Oracle2D(p)
    rng = np.random.default_rng(1908)
    n = o.N
    border = [0, o.n_x - 1, n - 1, n - o.n_x, o.n_x * (o.n_x // 2) + o.n_x // 2, 1, o.n_x + 1]
    with B.Instance2D(p) as g:
        for s in range(3):
            pre = g.get_controllers()
            nu_pre = lattice(o, pre["f"])
            g.sweep(1)
            post = g.get_controllers()
            pts = np.unique(np.concatenate([border, rng.choice(n, 60, replace=False)]))
            check_sweep(o, nu_pre, pre["U"], post["f"], post["idx"], points=pts)
            nu_post = lattice(o, post["f"])
            t = rng.choice(o.n_y ** 2, 40, replace=False)
            for tt in t:
                Uo = o.mmse(nu_post, int(tt), int(tt) + 1)
                assert np.max(np.abs(post["U"][tt] - Uo[tt])) <= 1e-11


# n_w^2 = 16641 taps: the exact quadratures of the screened search run on one
# lane (more chunk sums than a warp keeps in shared memory).
P2W = dict(k=0.2, sigma=0.6, delta=0.0625, x_half=1.0, w_half=4.0, y_half=6.0,
           cand_half=2.0, n_coarse=5, n_levels=3, n_nbr=1)


def staircase_table(o, step):
    """A quantised start (f = step round(x / step) per axis): whole windows of
    equal values, so the list is full of duplicates and exact ties."""
    xs = o.grid(o.n_x)
    h = step * np.round(xs / step)
    return np.stack([np.repeat(h, o.n_x), np.tile(h, o.n_x)], axis=1)


@pytest.mark.parametrize("case", ["P2B", "P2W", "staircase", "levels26", "huge"])
def test_screened_equals_direct(B, O, case):
    """The screened search makes the direct search's decisions bit for bit
    (values and list positions) at every sweep.  levels26: fractions of more
    than 24 bits, so the FP64 table costs screen; huge: one incumbent beyond
    2^44 lattice steps, whose table cost falls back to FP64 inside the
    double-float screening."""
    p, sweeps, tab = {"P2B": (P2B, 4, None), "P2W": (P2W, 2, None),
                      "staircase": (P2, 6, "stairs"),
                      "levels26": (dict(P2, n_levels=26), 3, None),
                      "huge": (P2, 2, "huge")}[case]
    o = O.Oracle2D(p)
    init = None
    if tab == "stairs":
        init = staircase_table(o, 5.0)
    elif tab == "huge":
        init = o.value(o.init(0)).astype(float)
        init[o.N // 3] = (1.0e13, -1.0e13)
    with B.Instance2D(dict(p, direct=0), init_f=init) as a, \
            B.Instance2D(dict(p, direct=1), init_f=init) as b:
        for s in range(sweeps):
            a.sweep(1)
            b.sweep(1)
            sa, sb = a.get_controllers(), b.get_controllers()
            assert np.array_equal(sa["f"], sb["f"]), s
            assert np.array_equal(sa["idx"], sb["idx"]), s
            assert np.array_equal(sa["U"], sb["U"]), s
            # J: the table costs' J against the exact one of the same state
            Ja, Jb = a.J_history()[-1], b.J_history()[-1]
            assert close_J(o, lattice(o, sa["f"]), sa["U"], Ja, Jb, exact=False), s
    if case == "P2W":
        # and the oracle's decisions from the same state
        with B.Instance2D(p) as g:
            pre = g.get_controllers()
            g.sweep(1)
            post = g.get_controllers()
            pts = np.arange(0, o.N, 7)
            check_sweep(o, lattice(o, pre["f"]), pre["U"], post["f"], post["idx"], points=pts)


def two_clusters(o, L):
    """f = (L, -L) on the left half of the x0 grid, (-L, L) on the right:
    at the target y = (L, L) each source is near in one component only, so
    the per-axis minima of the factorised weights sum far below the joint
    one (every factorised weight underflows there)."""
    a = np.repeat(np.arange(o.n_x), o.n_x)
    left = a < o.n_x // 2
    return np.stack([np.where(left, L, -L), np.where(left, -L, L)], axis=1).astype(float)


@pytest.mark.parametrize("case", ["identity", "clusters", "clusters_wide"])
def test_factorised_u1_matches_direct(B, O, case):
    """identity: every target on the double-float sums; clusters (L = 20):
    the corner target's factors underflow even in FP64 (gap 2 L^2 = 800), so
    the direct form runs there; clusters_wide (L = 6.25, gap ~78): beyond
    FP32's range, inside FP64's -- the FP64 pass."""
    p = dict(P2B, y_half=30.0) if case.startswith("clusters") else P2B
    o = O.Oracle2D(p)
    init = {"identity": None, "clusters": two_clusters(o, 20.0),
            "clusters_wide": two_clusters(o, 6.25)}[case]
    with B.Instance2D(dict(p, direct=0), init_f=init) as a, \
            B.Instance2D(dict(p, direct=2), init_f=init) as b:
        Ua, Ub = a.get_controllers()["U"], b.get_controllers()["U"]
        nu = lattice(o, a.get_controllers()["f"])
        Uo = o.mmse(nu)
        assert np.max(np.abs(Ua - Ub)) <= 1e-11
        assert np.max(np.abs(Ua - Uo)) <= 1e-11
        if case == "clusters":
            # the corner target (L, L) itself (where the fallback ran)
            j = o.n_y // 2 + round(20.0 / p["delta"])
            t = j * o.n_y + j
            assert np.array_equal(Ua[t], Ub[t])


def test_profile_and_work_counters(B, O):
    """Per-kernel-group timing and the evaluated-pair counter of the u1 sums:
    every group of a sweep is timed once per sweep, and the counter stays
    within the stages four u1 steps can evaluate (the first at creation)."""
    o = O.Oracle2D(P2)
    with B.Instance2D(P2) as g:
        g.profile(True)
        g.sweep(3)
        kt = g.kernel_times()
        for name in ("search", "u1_shifts", "u1_factors", "u1_sums", "u1_finish", "tables_J"):
            assert kt[name][0] == 3 and kt[name][1] > 0.0, (name, kt)
        live = g.work_counters()["u1_live_pairs"]
        # a stage is 32 sources x 32 x 32 targets (padding included); over all
        # source splits a tile has at most ceil(N / 32) + 64 stages per u1 step
        tiles = -(-o.n_y // 32)
        assert 0 < live <= 4 * tiles * tiles * (-(-o.N // 32) + 64) * 32 ** 3
        g.profile(False)
        assert g.kernel_times() == {}
