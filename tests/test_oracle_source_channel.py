"""Pins of the oracle's second problem, zero-delay source-channel coding
(Section V-B): x1 = u0(x0) + w, w ~ U(-W, W), J = E[lambda u0^2 +
(u1(x1) - x0)^2], lambda = k^2, the first controller carried as f = u0.

Each test checks the oracle against something other than itself: the mean of
a truncated normal (the u1 update with the identity controller), the prior's
second moment (J with u0 = 0), numpy's interpolation (the marginal cost),
brute force over the candidate list, invariants of the sweep, and the value
the paper prints (a plausibility band).  Planted mistakes in the new code
must fail one of them.  No GPU.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1908_04489_gb300 import workloads as W


def sc(**kw):
    return W.source_channel(**kw)


def np_cost(o, U, i, u):
    """k^2 u^2 + sum_l phi_l (U^(u + w_l) - x_i)^2 with numpy's interpolation
    (linear inside, constant beyond the ends) and equal weights."""
    d = o.params["delta"]
    w = (np.arange(o.n_w) - (o.n_w - 1) // 2) * d
    y = (np.arange(o.n_y) - (o.n_y - 1) // 2) * d
    x = (i - (o.n_x - 1) // 2) * d
    phi = np.full(o.n_w, 1.0 / o.n_w)
    return o.params["k"] ** 2 * u * u + float(np.sum(phi * (np.interp(u + w, y, U) - x) ** 2))


def truncated_normal_mean(a, b, s):
    """E[X | a <= X <= b] for X ~ N(0, s^2)."""
    pdf = lambda z: math.exp(-z * z / 2) / math.sqrt(2 * math.pi)
    cdf = lambda z: 0.5 * (1 + math.erf(z / math.sqrt(2)))
    al, be = a / s, b / s
    return s * (pdf(al) - pdf(be)) / (cdf(be) - cdf(al))


def test_equal_quadrature_weights():
    o = oracle.Oracle(sc())
    g = o.grids()
    assert np.all(g["phi"] == g["phi"][0]) and abs(g["phi"].sum() - 1) < 1e-14
    assert g["w"][0] == -1.0 and g["w"][-1] == 1.0


def u1_of_linear(o, a, yv):
    """U(y) for f = a x0 (a > 0) at y = yv, from the oracle."""
    g = o.grids()
    nu = o.init(2, a * g["x"])
    j = int(round(yv / o.params["delta"])) + (o.n_y - 1) // 2
    return o.mmse(nu, j, j + 1)[j]


@pytest.mark.parametrize("a,yv", [(1.0, 0.0), (1.0, 0.37), (1.0, -1.25), (0.5, 0.37),
                                  (0.5, -0.8), (2.0, 2.5)])
def test_u1_of_a_linear_controller_is_a_truncated_normal_mean(a, yv):
    """f = a x0: the sources within W of y are the x0 in [(y - W)/a, (y + W)/a],
    so U(y) = E[x0 | (y - W)/a <= x0 <= (y + W)/a] (rectangle rule, error
    O(delta))."""
    o = oracle.Oracle(sc(delta=0.001, x_half=5.0, y_half=7.0, cand_half=6.0))
    ref = truncated_normal_mean((yv - 1.0) / a, (yv + 1.0) / a, 1.0)
    got = u1_of_linear(o, a, yv)
    assert abs(got - ref) < 2e-3, (got, ref)


def test_u1_uses_the_nearest_sources_beyond_the_window():
    """f = 0 everywhere: every y beyond W sees all sources at the same
    distance, so U = the prior mean 0; within W too."""
    o = oracle.Oracle(sc())
    U = o.mmse(np.zeros(o.n_x, dtype=np.int64))
    assert np.max(np.abs(U)) < 1e-15


def three_level(o):
    """f = 3 for x0 > 0, -5 for x0 < 0, 0.5 at x0 = 0 (lattice values), and
    the prior-weighted means of x0 over each side."""
    g = o.grids()
    x = g["x"]
    f = np.where(x > 0, 3.0, np.where(x < 0, -5.0, 0.5))
    nu = o.init(2, f)
    wgt = np.exp(-x * x / (2 * o.params["sigma"] ** 2))
    pos, neg = x > 0, x < 0
    return nu, np.sum(wgt[pos] * x[pos]) / np.sum(wgt[pos]), \
        np.sum(wgt[neg] * x[neg]) / np.sum(wgt[neg])


@pytest.mark.parametrize("yv,which", [(6.5, "pos"), (4.5, "pos"), (2.2, "pos"),
                                      (1.6, "zero"), (-7.0, "neg"), (-4.2, "neg")])
def test_u1_takes_the_nearest_group_of_sources(yv, which):
    """Section V-B's likelihood is flat on |y - f(x0)| <= W.  With three
    groups of sources (f = 3 on x0 > 0, f = -5 on x0 < 0, f = 0.5 at x0 = 0)
    and W = 1: y = 2.2 and -4.2 see one group inside the window; y = 6.5, 4.5
    and -7 see none and take the nearest group (the limit of a slightly
    wider window); y = 1.6 is 1.1 from the lone source at x0 = 0 and 1.4 from
    the f = 3 group, so U = 0 there, where averaging all groups, or widening
    the window by W, would not give 0."""
    o = oracle.Oracle(sc())
    nu, mpos, mneg = three_level(o)
    j = int(round(yv / o.params["delta"])) + (o.n_y - 1) // 2
    got = o.mmse(nu, j, j + 1)[j]
    ref = {"pos": mpos, "neg": mneg, "zero": 0.0}[which]
    assert abs(got - ref) <= 1e-13, (yv, got, ref)


def test_J_without_transmission_is_the_prior_variance():
    """u0 = 0: u1 = E[x0] = 0 and J = E[x0^2] = sigma^2."""
    for s in (1.0, 1.7):
        o = oracle.Oracle(sc(sigma=s, x_half=round(8 * s / 0.02) * 0.02))
        nu = np.zeros(o.n_x, dtype=np.int64)
        assert abs(o.J(nu, o.mmse(nu)) - s * s) < 1e-9


@pytest.mark.parametrize("a", [0.6, 1.0, 1.7])
def test_search_with_a_linear_u1_finds_the_continuous_minimiser(a):
    """U = a y (inside the grid): with symmetric equal weights,
    g(u; x) = k^2 u^2 + a^2 (u^2 + E w^2) - 2 a x u + x^2, minimised at
    u* = a x / (k^2 + a^2); the search lands within the finest step of it."""
    p = sc(y_half=9.0, cand_half=6.0)
    o = oracle.Oracle(p)
    g = o.grids()
    U = a * g["y"]
    nu0 = o.init(0)
    sel = np.arange(100, 401, 25)
    out, _ = o.search(nu0, U, sel[0], sel[-1] + 1)
    k2 = p["k"] ** 2
    q = 2 * -(-round(p["cand_half"] / p["delta"]) // (p["n_coarse"] - 1))
    h_fine = q * p["delta"] / (p["n_refine"] // 2) ** p["n_levels"]
    for i in sel:
        u_star = a * g["x"][i] / (k2 + a * a)
        assert abs(o.value(out[i]) - u_star) <= h_fine / 2 + 1e-12, (i, o.value(out[i]), u_star)


@pytest.mark.parametrize("c,a", [(0.5, 0.8), (1.2, 0.3)])
def test_J_closed_form_for_linear_controllers(c, a):
    """f = c x0 and U = a y (inside the grid): J = sum_i p_i [k^2 f_i^2 +
    a^2 (f_i^2 + E w^2) - 2 a f_i x_i + x_i^2] = (k^2 c^2 + a^2 c^2 - 2 a c + 1) s2
    + a^2 E w^2, with s2 = sigma^2 (wide x grid) and E w^2 the second moment of
    the equal-weight w grid, delta^2 hw (hw + 1) / 3."""
    p = sc(x_half=8.0, y_half=20.0, cand_half=6.0)
    o = oracle.Oracle(p)
    g = o.grids()
    nu = o.init(2, c * g["x"])
    U = a * g["y"]
    hw = round(p["w_half"] / p["delta"])
    ew2 = p["delta"] ** 2 * hw * (hw + 1) / 3.0
    k2 = p["k"] ** 2
    fx = o.value(nu)                      # c x0 rounded to the candidate lattice
    s_ff = float(np.sum(g["px"] * fx * fx)); s_fx = float(np.sum(g["px"] * fx * g["x"]))
    ref = k2 * s_ff + a * a * (s_ff + ew2) - 2 * a * s_fx + 1.0
    assert abs(o.J(nu, U) - ref) < 1e-10
    # and against the exact moments of the continuous prior (lattice rounding of f)
    cont = (k2 * c * c + a * a * c * c - 2 * a * c + 1.0) + a * a * ew2
    assert abs(o.J(nu, U) - cont) < 1e-3


def test_cost_against_library_interpolation():
    o = oracle.Oracle(sc())
    g = o.grids()
    U = 0.8 * np.tanh(2 * g["y"]) + 0.05 * g["y"]
    for i, nu in [(10, 5 << o.shift), (250, -(13 << o.shift) + 77), (400, 3), (0, 300 << o.shift)]:
        u = float(o.value(nu))
        ref = np_cost(o, U, i, u)
        assert abs(o.cost(U, i, nu) - ref) < 1e-12 * max(1.0, ref)


def test_search_is_the_first_minimum_of_its_list():
    o = oracle.Oracle(sc())
    g = o.grids()
    rng = np.random.default_rng(7)
    nu_pre = o.init(2, np.clip(g["x"] + rng.normal(0, 0.3, o.n_x), -4, 4))
    U = o.mmse(nu_pre)
    out, idx = o.search(nu_pre, U)
    for i in (0, 1, 77, 250, 499, 500):
        nus, gs, k = o.candidates(nu_pre, U, i)
        first = int(np.argmin(gs))          # numpy returns the first minimum
        assert k == first and out[i] == nus[first] and idx[i] == first


def test_sweeps_do_not_raise_J_and_keep_odd_symmetry():
    o = oracle.Oracle(sc())
    r = o.solve(0, 8)
    assert np.all(np.diff(r["J"]) <= 1e-12)
    f = o.value(r["nu"])
    assert np.max(np.abs(f + f[::-1])) <= 1e-12
    U = r["U"]
    assert np.max(np.abs(U + U[::-1])) <= 1e-12


def test_paper_value_band():
    """Section V-B prints J = 0.890756 for lambda = 2 (grids not stated); the
    sweep from the identity settles within 0.01 of it."""
    o = oracle.Oracle(sc())
    r = o.solve(0, 20)
    assert abs(r["J"][-1] - 0.890756) < 0.01
    assert abs(r["J"][-1] - r["J"][-2]) < 1e-9


MUTANTS = {
    "u1 numerator uses f": ("num = num + wgt * xi;",
                            "num = num + wgt * value_of(g, nu[i]);"),
    "window from x": ("if (fabs(yj - value_of(g, nu[i])) > reach) continue;\n"
                      "            double wgt",
                      "if (fabs(yj - xi) > reach) continue;\n"
                      "            double wgt"),
    "estimate against f": ("double d = uh - x;", "double d = uh - u;"),
    "control on u - x": ("return g->kk * (u * u) + acc;",
                         "return g->kk * ((u - x) * (u - x)) + acc;"),
    "Gaussian weights": ("if (g->p.problem == 1) phi[l] = 1.0;", ""),
    "no nearest-source fallback": ("double reach = dmin <= W ? W : dmin;",
                                   "double reach = W;"),
    "fallback window widened by W": ("double reach = dmin <= W ? W : dmin;",
                                     "double reach = dmin <= W ? W : dmin + W;"),
    "fallback takes every source": ("double reach = dmin <= W ? W : dmin;",
                                    "double reach = dmin <= W ? W : INFINITY;"),
}


def pin_failures(L):
    bad = []
    o = oracle.Oracle(sc(), library=L)
    g = o.grids()
    if not np.all(g["phi"] == g["phi"][0]):
        bad.append("weights")
    t = oracle.Oracle(sc(delta=0.001, x_half=5.0, y_half=7.0, cand_half=6.0), library=L)
    if abs(u1_of_linear(t, 0.5, 0.37) - truncated_normal_mean(-1.26, 2.74, 1.0)) > 2e-3:
        bad.append("u1 truncated mean")
    nu3, mpos, mneg = three_level(o)
    for yv, ref in ((6.5, mpos), (1.6, 0.0), (-7.0, mneg)):
        j = int(round(yv / o.params["delta"])) + (o.n_y - 1) // 2
        got = o.mmse(nu3, j, j + 1)[j]
        if not abs(got - ref) <= 1e-13:
            bad.append("nearest sources")
            break
    Uc = 0.8 * np.tanh(2 * g["y"]) + 0.05 * g["y"]
    for i, nu in [(10, 5 << o.shift), (250, -(13 << o.shift) + 77)]:
        ref = np_cost(o, Uc, i, float(o.value(nu)))
        if abs(o.cost(Uc, i, nu) - ref) > 1e-12 * max(1.0, ref):
            bad.append("cost")
            break
    return bad


def test_the_unmodified_oracle_passes_the_source_channel_pins():
    assert pin_failures(oracle.lib()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_planted_mistake_fails_a_source_channel_pin(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) >= 1, f"mutation anchor missing: {old}"
    path = oracle.build_variant(src.replace(old, new), str(tmp_path / "libmut.so"))
    assert pin_failures(oracle.load_library(path)), f"'{name}' went unnoticed"
