"""Pins of the FP64 oracle against facts other than itself (no GPU).

Each test checks the oracle against something the mathematics or a library
routine fixes: closed forms for affine controllers (Section V-A problem),
numpy's linear interpolation with constant extension, a weighted mean, brute
force over the candidate list, and invariants of the sweep (Corollary 1's
pointwise minimisation never raises the cost).  A dropped term, a wrong sign,
a shifted index or a transposed operand in the oracle fails at least one.
"""
import numpy as np
import pytest

import oracle
from paper_1908_04489_gb300 import workloads as W


def wide(**kw):
    # x0 to 10 sigma, w to 9, y to 60: grid truncation below 1e-15
    p = W.base(x_half=50.0, w_half=9.0, y_half=60.0, cand_half=30.0)
    p.update(kw)
    return p


def np_phi(o):
    w = (np.arange(o.n_w) - (o.n_w - 1) // 2) * o.params["delta"]
    phi = np.exp(-w * w / 2)
    return w, phi / phi.sum()


def np_S(o, U, u):
    """S(u) = sum_l phi_l (u - U^(u + w_l))^2 with numpy's interpolation
    (linear inside, constant beyond the ends) and float positions."""
    w, phi = np_phi(o)
    y = (np.arange(o.n_y) - (o.n_y - 1) // 2) * o.params["delta"]
    return float(np.sum(phi * (u - np.interp(u + w, y, U)) ** 2))


def test_grids_weights_normalised_and_symmetric():
    o = oracle.Oracle(wide())
    g = o.grids()
    assert abs(g["px"].sum() - 1) < 1e-14 and abs(g["phi"].sum() - 1) < 1e-14
    for a in ("x", "w", "y"):
        assert np.array_equal(g[a], -g[a][::-1])
    # prior variance sigma^2 and unit noise variance (rectangle rule is exact
    # to rounding for Gaussians at this spacing)
    assert abs(np.sum(g["px"] * g["x"] ** 2) - 25.0) < 1e-11
    assert abs(np.sum(g["phi"] * g["w"] ** 2) - 1.0) < 1e-13
    assert o.n_x == 2001 and o.n_w == 361 and o.n_y == 2401


def test_c1_sizes_and_candidate_count():
    o = oracle.Oracle(W.c1())
    assert (o.n_x, o.n_w, o.n_y) == (1001, 241, 1401)
    assert o.n_cand == 1 + 4 + 64 + 4 * 16
    assert o.shift == 12


@pytest.mark.parametrize("c", [0.0, 25.0 / 26.0, 0.5, 1.0])
def test_S_closed_form_for_linear_u1(c):
    """U = c y  =>  S(u) = (1 - c)^2 u^2 + c^2 sum phi w^2 = (1-c)^2 u^2 + c^2."""
    o = oracle.Oracle(wide())
    y = o.grids()["y"]
    U = c * y
    rng = np.random.default_rng(0)
    for nu in rng.integers(-40 << o.shift, 40 << o.shift, size=64) // 20:
        u = float(o.value(nu))
        ref = (1 - c) ** 2 * u * u + c * c
        assert abs(o.S(U, nu) - ref) <= 1e-12 * max(1.0, ref)


def test_S_matches_library_interpolation_with_clamping():
    o = oracle.Oracle(W.small())
    y = o.grids()["y"]
    rng = np.random.default_rng(1)
    U = 0.8 * y + np.cumsum(rng.normal(0, 0.3, o.n_y))
    lim = int((o.params["y_half"] + o.params["w_half"] + 3) / o.params["delta"])
    nus = rng.integers(-lim << o.shift, lim << o.shift, size=300)
    for nu in nus:
        u = float(o.value(nu))
        assert abs(o.S(U, nu) - np_S(o, U, u)) <= 1e-11 * max(1.0, np_S(o, U, u))


def test_cost_adds_control_term():
    o = oracle.Oracle(W.small(k=0.37))
    g = o.grids()
    U = np.tanh(g["y"]) * 3
    for i, nu in [(0, 5 << o.shift), (57, -(13 << o.shift) + 77), (120, 3)]:
        u = float(o.value(nu))
        ref = 0.37 ** 2 * (u - g["x"][i]) ** 2 + np_S(o, U, u)
        assert abs(o.cost(U, i, nu) - ref) <= 1e-11 * max(1.0, ref)


@pytest.mark.parametrize("lam", [1.0, 0.5, 1.25])
def test_mmse_affine_closed_form(lam):
    """f = lam x0  =>  E[x1 | y1 = y] = lam^2 s^2 / (1 + lam^2 s^2) y."""
    p = wide()
    o = oracle.Oracle(p)
    g = o.grids()
    nu = o.init(2, lam * g["x"])
    U = o.mmse(nu)
    c = lam * lam * 25.0 / (1 + lam * lam * 25.0)
    inner = np.abs(g["y"]) <= 35.0 * lam
    err = np.abs(U[inner] - c * g["y"][inner])
    assert err.max() <= 1e-12 * 40


def test_mmse_is_weighted_mean_and_newton_fixed_point():
    """U_j minimises C_1(v, y_j) = sum_i p_i phi(y_j - f_i) (f_i - v)^2: it is
    numpy's weighted average, and a Newton step on C_1 from U_j stays put."""
    o = oracle.Oracle(W.small())
    g = o.grids()
    rng = np.random.default_rng(2)
    f = np.round(3.5 * np.sign(g["x"]) * (1 + (np.abs(g["x"]) > 6))) + \
        rng.normal(0, 0.2, o.n_x)
    nu = o.init(2, f)
    fv = o.value(nu)
    U = o.mmse(nu)
    for j in range(0, o.n_y, 7):
        wgt = g["px"] * np.exp(-(g["y"][j] - fv) ** 2 / 2)
        ref = np.average(fv, weights=wgt)
        assert abs(U[j] - ref) <= 1e-12 * max(1.0, abs(ref))
        d1 = -2 * np.sum(wgt * (fv - U[j]))
        d2 = 2 * np.sum(wgt)
        assert abs(d1 / d2) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("lam", [1.0, 0.5, 0.75])
def test_J_affine_closed_form(lam):
    """J = k^2 (1-lam)^2 s^2 + lam^2 s^2 / (1 + lam^2 s^2) for f = lam x0 with
    the MMSE u1 (Section V-A objective)."""
    p = wide()
    o = oracle.Oracle(p)
    g = o.grids()
    nu = o.init(2, lam * g["x"])
    U = o.mmse(nu)
    J = o.J(nu, U)
    s2 = 25.0
    ref = 0.04 * (1 - lam) ** 2 * s2 + lam * lam * s2 / (1 + lam * lam * s2)
    assert abs(J - ref) <= 1e-12


def test_search_linear_u1_finds_continuous_minimiser():
    """For U = c y the cost is a strict quadratic with minimiser
    u* = k^2 x / (k^2 + (1 - c)^2); the coarse-to-fine search must land within
    half a finest-level step of it."""
    p = wide()
    o = oracle.Oracle(p)
    g = o.grids()
    c = 25.0 / 26.0
    U = c * g["y"]
    nu0 = o.init(0)
    sel = np.arange(500, 1501, 25)
    nu1, idx = o.search(nu0, U, sel[0], sel[-1] + 1)
    k2 = p["k"] ** 2
    h_fine = 20 * p["delta"] / 8 ** p["n_levels"]
    for i in sel:
        ustar = k2 * g["x"][i] / (k2 + (1 - c) ** 2)
        assert abs(o.value(nu1[i]) - ustar) <= h_fine / 2 + 1e-12


def _np_candidates(o, nu_pre, i):
    p = o.params
    one = 1 << o.shift
    hr = round(p["cand_half"] / p["delta"])
    q = 2 * max(1, -(-hr // (p["n_coarse"] - 1)))
    lst = [nu_pre[i]]
    for d in list(range(-p["n_nbr"], 0)) + list(range(1, p["n_nbr"] + 1)):
        ii = i + d
        lst.append(nu_pre[ii] if 0 <= ii < o.n_x else nu_pre[i])
    for j in range(p["n_coarse"]):
        lst.append((2 * j - (p["n_coarse"] - 1)) * (q // 2) * one)
    return lst, q


def test_search_matches_brute_force_over_the_list():
    """Rebuild the list independently, cost every entry with numpy's
    interpolation, and take the first minimum: same winner, same index.  A
    different winner is accepted only at a tie to rounding (both costs equal
    within 1e-12 in the independent evaluation)."""
    p = W.small(k=0.3, n_levels=2, n_refine=8)
    o = oracle.Oracle(p)
    g = o.grids()
    rng = np.random.default_rng(3)
    U = 0.9 * g["y"] + np.sin(g["y"]) * 1.5 + 0.1
    nu_pre = o.init(2, g["x"] + rng.normal(0, 0.5, o.n_x))
    nu1, idx = o.search(nu_pre, U)
    k2 = p["k"] ** 2
    bits = int(np.log2(p["n_refine"] // 2))
    ties = 0
    for i in range(0, o.n_x, 3):
        nus, gs, oi = o.candidates(nu_pre, U, i)
        base_list, q = _np_candidates(o, nu_pre, i)
        cost = lambda nu: k2 * (float(o.value(nu)) - g["x"][i]) ** 2 + \
            np_S(o, U, float(o.value(nu)))
        lst = list(base_list)
        costs = [cost(nu) for nu in lst]
        for lv in range(1, p["n_levels"] + 2):
            mine = int(np.argmin(costs))
            theirs = int(np.argmin(gs[:len(lst)]))
            if mine != theirs:
                assert abs(costs[mine] - costs[theirs]) <= 1e-12
                ties += 1
            if lv > p["n_levels"]:
                break
            h = q << (bits * (p["n_levels"] - lv))
            for m in list(range(-p["n_refine"] // 2, 0)) + \
                    list(range(1, p["n_refine"] // 2 + 1)):
                lst.append(lst[theirs] + m * h)
                costs.append(cost(lst[-1]))
        assert list(nus) == lst
        assert np.allclose(gs, costs, rtol=1e-11, atol=1e-12)
        assert oi == idx[i] and nu1[i] == lst[oi]
    assert ties <= 2


def test_half_step_never_raises_J():
    """Corollary 1: replacing f_i by the list minimiser (the list contains
    f_i itself) cannot raise J for fixed u1; holds exactly in FP64."""
    p = W.c1()
    o = oracle.Oracle(p)
    nu = o.init(1)
    U = o.mmse(nu)
    for _ in range(3):
        nu1, _ = o.search(nu, U)
        assert o.J(nu1, U) <= o.J(nu, U)
        nu = nu1
        U = o.mmse(nu)


def test_sweeps_keep_odd_symmetry_and_do_not_raise_J():
    """From the odd identity init every sweep keeps f and U odd (to rounding)
    and J does not rise.  From the odd staircase, x0 = 0 sits on a jump of U
    where +u and -u tie exactly and the first-in-list rule picks one side, so
    only the first sweep away from x0 = 0 is checked there."""
    p = W.small(sweeps=4)
    o = oracle.Oracle(p)
    c = (o.n_x - 1) // 2
    mask = np.arange(o.n_x) != c
    r = o.solve(0, 4)
    f = o.value(r["nu"])
    assert np.max(np.abs(f + f[::-1])) <= 1e-12
    assert np.max(np.abs(r["U"] + r["U"][::-1])) <= 1e-12
    assert np.all(np.diff(r["J"]) <= 1e-12)
    nu = o.init(1)
    U = o.mmse(nu)
    assert np.max(np.abs(U + U[::-1])) <= 1e-12
    nu1, _ = o.search(nu, U)
    f = o.value(nu1)
    assert np.max(np.abs(f + f[::-1])[mask]) <= 1e-12
    assert f[c] != 0.0  # the tie at x0 = 0 moved the centre off zero


def test_thread_count_does_not_change_results():
    p = W.c1()
    o = oracle.Oracle(p)
    oracle.set_threads(1)
    a = o.solve(1, 2, want_idx=True)
    oracle.set_threads(4)
    b = o.solve(1, 2, want_idx=True)
    oracle.set_threads(1)
    assert np.array_equal(a["nu"], b["nu"]) and np.array_equal(a["idx"], b["idx"])
    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["J"], b["J"])


def test_paper_converged_value_band():
    """Section V-A prints J = 0.166897 for k = 0.2, sigma = 5 after the full
    Algorithm 1 on unstated grids: a plausibility band, not a parity pin."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_values.json")))
    ref = gold["witsenhausen_k0.2_sigma5_J"]["value"]
    p = W.c1()
    o = oracle.Oracle(p)
    oracle.set_threads(4)
    r = o.solve(1, 12)
    oracle.set_threads(1)
    assert abs(r["J"][-1] - ref) < 0.006
    assert r["J"][-1] < r["J"][1]


def staircase_level(x_units, delta):
    """The odd three-step staircase start, f(x) = 3.5 sgn(x) (2 min(floor(|x|/7),
    2) + 1) with f(0) = 0, evaluated in exact rational arithmetic at
    x = x_units * delta (so that floor(|x|/7) is not at the mercy of a rounded
    quotient at the jumps)."""
    from fractions import Fraction
    x = Fraction(int(x_units)) * Fraction(repr(delta))
    if x == 0:
        return 0.0
    m = min(int(abs(x) / 7), 2)
    return float((1 if x > 0 else -1) * Fraction(7, 2) * (2 * m + 1))


@pytest.mark.parametrize("delta", [0.05, 0.005])
def test_staircase_start_values(delta):
    """The odd staircase start (the garbled "3.5 sign-rounded(x0/7)" read as
    three steps per side: levels +-3.5, +-10.5, +-17.5, jumps at |x0| = 7 and
    14, f(0) = 0): the oracle's lattice values equal the formula at every x0
    point, and at the named points on both sides of each jump."""
    p = W.base(delta=delta)
    o = oracle.Oracle(p)
    f = o.value(o.init(1))
    hx = (o.n_x - 1) // 2
    ref = np.array([staircase_level(i - hx, delta) for i in range(o.n_x)])
    assert np.max(np.abs(f - ref)) <= 1e-12
    named = {0.0: 0.0, 7.0 - delta: 3.5, 7.0: 10.5, 14.0 - delta: 10.5, 14.0: 17.5,
             25.0: 17.5}
    for xv, level in named.items():
        for sgn in (1, -1):
            i = hx + sgn * int(round(xv / delta))
            assert abs(f[i] - sgn * level) <= 1e-12, (xv, sgn, f[i])
    # odd, three levels per side
    assert np.array_equal(f, -f[::-1])
    assert sorted(set(np.round(f, 9))) == [-17.5, -10.5, -3.5, 0.0, 3.5, 10.5, 17.5]
