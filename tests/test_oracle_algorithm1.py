"""Pins of the oracle's Algorithm 1 (Sections III-B to III-D): the local
update's derivatives, Newton's step, the adaptive split and the outer loop.
No GPU.

  - g' and g'' against central differences of the oracle's own cost inside a
    y-cell (where the discretised cost is exactly quadratic in u), for both
    problems;
  - one Newton step on a cost that is quadratic everywhere (a linear u1 with
    no clamping) lands on its minimiser k^2 x / (k^2 + (1 - c)^2), to half a
    lattice step;
  - the split N_L = min(max(floor(I_L N / (I_L + I_P)), 1), N - 1) on cases
    worked out by hand;
  - the loop on the c1 grid from the identity: terminates at p = 1e-10 with
    the paper's converged value for k = 0.2, sigma = 5 within 1e-4 (a
    plausibility band: the paper's grids are not stated), every round's
    split the formula applied to the recorded improvements, partial
    exhaustion never raising J;
  - planted mistakes in the new code each fail one of these.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1908_04489_gb300 import workloads as W


def fd_derivs(o, U, i, nu, steps=64):
    """Central first and second differences of g(.; x_i) over +-steps lattice
    points around nu (all inside nu's y-cell)."""
    h = steps * o.params["delta"] / (1 << o.shift)
    gm, g0, gp = (o.cost(U, i, nu + d * steps) for d in (-1, 0, 1))
    return (gp - gm) / (2 * h), (gp - 2 * g0 + gm) / (h * h)


def inner_nu(o, u):
    """A lattice point near u whose neighbours +-64 lie in the same cell."""
    one = 1 << o.shift
    nu = int(round(u / o.params["delta"] * one))
    cell_pos = nu % one
    return nu - cell_pos + one // 2          # the middle of its cell


@pytest.mark.parametrize("problem", [0, 1])
def test_derivatives_match_central_differences_inside_a_cell(problem):
    p = W.small(k=0.3) if problem == 0 else W.source_channel(delta=0.05, x_half=4.0,
                                                            y_half=6.0, cand_half=5.0)
    o = oracle.Oracle(p)
    g = o.grids()
    rng = np.random.default_rng(4)
    U = (0.9 * g["y"] + np.sin(g["y"]) * 1.5 + 0.1) if problem == 0 else \
        0.8 * np.tanh(2 * g["y"]) + 0.05 * g["y"] + rng.normal(0, 0.01, o.n_y)
    for i in (3, o.n_x // 3, o.n_x // 2, o.n_x - 5):
        for u in (-3.3, -0.71, 0.4, 2.9):
            nu = inner_nu(o, u)
            h1, h2 = o.derivs(U, i, nu)
            d1, d2 = fd_derivs(o, U, i, nu)
            assert abs(2 * h1 - d1) <= 1e-7 * max(1.0, abs(d1)), (i, u, 2 * h1, d1)
            assert abs(2 * h2 - d2) <= 1e-5 * max(1.0, abs(d2)), (i, u, 2 * h2, d2)
            assert h2 >= o.params["k"] ** 2 - 1e-15       # g'' >= 2 k^2


@pytest.mark.parametrize("c", [25.0 / 26.0, 0.5, 0.0])
def test_one_newton_step_lands_on_the_minimiser_of_a_quadratic_cost(c):
    """U = c y inside the table (wide grids, no clamping): g(u; x) =
    k^2 (u - x)^2 + (1 - c)^2 u^2 + c^2 W2 is quadratic in u, so Newton's step
    from anywhere lands on u* = k^2 x / (k^2 + (1 - c)^2)."""
    p = W.base(x_half=50.0, w_half=9.0, y_half=60.0, cand_half=30.0)
    o = oracle.Oracle(p)
    g = o.grids()
    U = c * g["y"]
    rng = np.random.default_rng(5)
    sel = np.arange(800, 1201, 40)
    nu_pre = o.init(2, g["x"] + rng.normal(0, 3.0, o.n_x))
    nu1 = o.local_update(nu_pre, U, tau=0.1, i0=sel[0], i1=sel[-1] + 1)
    k2 = p["k"] ** 2
    h = p["delta"] / (1 << o.shift)
    for i in sel:
        ustar = k2 * g["x"][i] / (k2 + (1 - c) ** 2)
        assert abs(o.value(nu1[i]) - ustar) <= h / 2 + 1e-12, (i, o.value(nu1[i]), ustar)
    # the minimiser (on the lattice) is a fixed point
    nu2 = o.local_update(nu1, U, i0=sel[0], i1=sel[-1] + 1)
    assert np.array_equal(nu2[sel], nu1[sel])


@pytest.mark.parametrize("I_L,I_P,N,n_l,want", [
    (3.0, 1.0, 20, 10, 15),      # floor(60 / 4) = 15
    (1.0, 3.0, 20, 10, 5),       # floor(20 / 4) = 5
    (1.0, 2.0, 20, 10, 6),       # floor(20 / 3) = 6.67 -> 6
    (0.0, 1.0, 20, 10, 1),       # at least one local update
    (1.0, 0.0, 20, 10, 19),      # at most N - 1
    (1e-12, 1e-3, 20, 7, 1),
    (2.0, 2.0, 7, 3, 3),         # floor(14 / 4) = 3
    (0.0, 0.0, 20, 7, 7),        # no improvement at all: split kept
])
def test_split_on_hand_worked_cases(I_L, I_P, N, n_l, want):
    o = oracle.Oracle(W.small())
    assert o.split(I_L, I_P, N, n_l) == want


@pytest.fixture(scope="module")
def c1_run():
    o = oracle.Oracle(W.c1())
    oracle.set_threads(os.cpu_count() or 1)
    try:
        r = o.algorithm1(0, N=20, precision=1e-10, max_rounds=60)
    finally:
        oracle.set_threads(1)
    return o, r


def test_algorithm1_converges_near_the_papers_value(c1_run):
    """Section V-A prints J = 0.166897 for k = 0.2, sigma = 5 after
    Algorithm 1 with N = 20, p = 1e-10 (Section IV) from the identity
    (Section III-D); the same loop on the c1 grid lands within 1e-4."""
    o, r = c1_run
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_values.json")))
    ref = gold["witsenhausen_k0.2_sigma5_J"]["value"]
    assert r["converged"] == 1 and r["I_L"] + r["I_P"] <= 1e-10
    assert abs(r["J"] - ref) < 1e-4, r["J"]
    assert r["J"] < r["J_phase"][0]


def test_algorithm1_bookkeeping(c1_run):
    """Every round's split is the formula applied to the improvements the
    recorded J values give; the loop ran while I_L + I_P > p; partial
    exhaustion never raised J."""
    o, r = c1_run
    Jp, NL = r["J_phase"], r["N_L_rounds"]
    assert NL[0] == 10
    for k in range(len(NL)):
        IL = abs(Jp[2 * k] - Jp[2 * k + 1])
        IP = abs(Jp[2 * k + 1] - Jp[2 * k + 2])
        assert Jp[2 * k + 2] <= Jp[2 * k + 1] + 1e-15
        nxt = NL[k + 1] if k + 1 < len(NL) else r["N_L"]
        assert nxt == o.split(IL, IP, 20, NL[k])
        if k + 1 < len(NL):
            assert IL + IP > 1e-10
    assert r["local_iters"] == int(np.sum(NL))
    assert r["exhaustion_iters"] == int(np.sum(20 - NL))


MUTANTS = {
    "local update descends the wrong way": ("a[l] = phi[l] * (e * c);",
                                            "a[l] = phi[l] * (-e * c);"),
    "g' without the control term": ("double lin = g->p.problem == 1 ? g->kk * u : g->kk * (u - x);",
                                    "double lin = 0.0;"),
    "g'' missing a factor 1/delta": ("*h2 = g->kk + s2 / (dl * dl);", "*h2 = g->kk + s2 / dl;"),
    "slope ignores the cell step": ("double e = u - uh, c = dl - d;",
                                    "double e = u - uh, c = dl;"),
    "split rounds instead of flooring": ("double r = floor(I_L * (double)N / (I_L + I_P));",
                                         "double r = round(I_L * (double)N / (I_L + I_P));"),
    "split without its upper clamp": (
        "int nl = r < 1.0 ? 1 : (r > (double)(N - 1) ? N - 1 : (int)r);",
        "int nl = r < 1.0 ? 1 : (int)r;"),
}


def pin_failures(L):
    bad = []
    o = oracle.Oracle(W.small(k=0.3), library=L)
    g = o.grids()
    U = 0.9 * g["y"] + np.sin(g["y"]) * 1.5 + 0.1
    for i, u in ((50, 0.4), (120, -2.9)):
        nu = inner_nu(o, u)
        h1, h2 = o.derivs(U, i, nu)
        d1, d2 = fd_derivs(o, U, i, nu)
        if abs(2 * h1 - d1) > 1e-7 * max(1.0, abs(d1)) or \
                abs(2 * h2 - d2) > 1e-5 * max(1.0, abs(d2)):
            bad.append("derivatives")
            break
    w = oracle.Oracle(W.base(x_half=50.0, w_half=9.0, y_half=60.0, cand_half=30.0), library=L)
    gw = w.grids()
    c = 0.5
    nu1 = w.local_update(w.init(2, gw["x"] + 1.0), c * gw["y"], i0=1000, i1=1001)
    ustar = 0.04 * gw["x"][1000] / (0.04 + (1 - c) ** 2)
    if abs(w.value(nu1[1000]) - ustar) > 0.05 / (1 << w.shift):
        bad.append("newton")
    for I_L, I_P, N, n_l, want in ((1.0, 2.0, 20, 10, 6), (1.0, 0.0, 20, 10, 19)):
        if w.split(I_L, I_P, N, n_l) != want:
            bad.append("split")
            break
    return bad


def test_the_unmodified_oracle_passes_the_algorithm1_pins():
    assert pin_failures(oracle.lib()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_planted_mistake_fails_an_algorithm1_pin(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) >= 1, f"mutation anchor missing: {old}"
    path = oracle.build_variant(src.replace(old, new), str(tmp_path / "libmut.so"))
    assert pin_failures(oracle.load_library(path)), f"'{name}' went unnoticed"
