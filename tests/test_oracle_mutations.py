"""Planted mistakes in the oracle (CPU only): each mutant of the oracle source
must fail at least one pin.  The mutants are built from a copy of the source
in a temporary directory; the oracle itself is not touched."""
import numpy as np
import pytest

import oracle
from paper_1908_04489_gb300 import workloads as W

MUTANTS = {
    "drop control term": ("return g->kk * (a * a) + S_of(g, phi, U, nu);",
                          "return S_of(g, phi, U, nu);"),
    "wrong residual sign": ("double e = u - uh;", "double e = u + uh;"),
    "shifted y index": ("int64_t jb = cell - g->hw + g->hy;",
                        "int64_t jb = cell - g->hw + g->hy + 1;"),
    "transposed interpolation": ("double uh = U[jl] + t * (U[jr] - U[jl]);",
                                 "double uh = U[jr] + t * (U[jl] - U[jr]);"),
    "wrong noise variance": ("phi[l] = exp(-(w * w) / 2.0);",
                             "phi[l] = exp(-(w * w));"),
    "u1 update without the prior": (
        "double e = (xi * xi) / two_s2 + ((yj - fi) * (yj - fi)) / 2.0;",
        "double e = ((yj - fi) * (yj - fi)) / 2.0;"),
    "u1 numerator uses x0": ("num = num + wgt * fi;", "num = num + wgt * xi;"),
    "mirrored neighbours": ("int64_t ii = i + d;", "int64_t ii = i - d;"),
    "coarse levels one step too coarse": (
        "int64_t h = g->q * ((int64_t)1 << (bits * (p->n_levels - lv)));",
        "int64_t h = g->q * ((int64_t)1 << (bits * (p->n_levels - lv + 1)));"),
    "J without prior weights": ("J = J + px[i] * terms[i];", "J = J + terms[i];"),
    "staircase steps 3.5 wide": ("if (half_steps(7.0, p->delta, &n7) || n7 < 1) return -1;",
                                 "if (half_steps(3.5, p->delta, &n7) || n7 < 1) return -1;"),
    "staircase levels 3.5 (m + 1)": (
        "double v = 3.5 * (double)(2 * m + 1) / p->delta * (double)g.one;",
        "double v = 3.5 * (double)(m + 1) / p->delta * (double)g.one;"),
    "staircase without its cap": ("if (m > 2) m = 2;", ""),
}


def np_S(o, U, u):
    w = (np.arange(o.n_w) - (o.n_w - 1) // 2) * o.params["delta"]
    phi = np.exp(-w * w / 2)
    phi /= phi.sum()
    y = (np.arange(o.n_y) - (o.n_y - 1) // 2) * o.params["delta"]
    return float(np.sum(phi * (u - np.interp(u + w, y, U)) ** 2))


def pin_failures(L):
    """Names of the pins (a compact subset of test_oracle_pins) that fail."""
    bad = []
    wide = W.base(x_half=50.0, w_half=9.0, y_half=60.0, cand_half=30.0)
    o = oracle.Oracle(wide, library=L)
    g = o.grids()
    if abs(g["phi"].sum() - 1) > 1e-13 or abs(np.sum(g["phi"] * g["w"] ** 2) - 1) > 1e-12:
        bad.append("noise weights")
    c = 25.0 / 26.0
    U = c * g["y"]
    for nu in (3 << o.shift, -(7 << o.shift) + 123, 11):
        u = float(o.value(nu))
        if abs(o.S(U, nu) - ((1 - c) ** 2 * u * u + c * c)) > 1e-10:
            bad.append("S closed form")
            break
    lam = 0.5                              # f = lam x0 (lam = 1 hides x0 vs f)
    cl = lam * lam * 25.0 / (1 + lam * lam * 25.0)
    nu1 = o.init(2, lam * g["x"])
    U1 = o.mmse(nu1)
    inner = np.abs(g["y"]) <= 35 * lam
    if np.max(np.abs(U1[inner] - cl * g["y"][inner])) > 1e-9:
        bad.append("u1 closed form")
    if abs(o.J(nu1, U1) - (0.04 * (1 - lam) ** 2 * 25.0 + cl)) > 1e-10:
        bad.append("J closed form")
    nu0 = o.init(0)
    sel = np.arange(600, 1401, 100)
    nus, _ = o.search(nu0, U, sel[0], sel[-1] + 1)
    k2 = wide["k"] ** 2
    h_fine = 20 * wide["delta"] / 8 ** wide["n_levels"]
    for i in sel:
        if abs(o.value(nus[i]) - k2 * g["x"][i] / (k2 + (1 - c) ** 2)) > h_fine / 2 + 1e-12:
            bad.append("search minimiser")
            break
    small = W.small(k=0.3)
    s = oracle.Oracle(small, library=L)
    gs = s.grids()
    Us = 0.9 * gs["y"] + np.sin(gs["y"]) * 1.5 + 0.1
    for i, nu in [(3, 5 << s.shift), (57, -(13 << s.shift) + 77), (120, 3)]:
        u = float(s.value(nu))
        ref = 0.09 * (u - gs["x"][i]) ** 2 + np_S(s, Us, u)
        if abs(s.cost(Us, i, nu) - ref) > 1e-10 * max(1.0, ref):
            bad.append("cost vs library interpolation")
            break
    # the odd staircase start: levels +-3.5, +-10.5, +-17.5 with jumps at 7, 14
    c1 = oracle.Oracle(W.c1(), library=L)
    fs = c1.value(c1.init(1))
    hx = (c1.n_x - 1) // 2
    for xv, level in ((0.0, 0.0), (6.95, 3.5), (7.0, 10.5), (13.95, 10.5), (14.0, 17.5),
                      (25.0, 17.5)):
        i = hx + int(round(xv / 0.05))
        if abs(fs[i] - level) > 1e-12 or abs(fs[2 * hx - i] + level) > 1e-12:
            bad.append("staircase start")
            break
    rng = np.random.default_rng(3)
    nu_pre = s.init(2, gs["x"] + rng.normal(0, 0.5, s.n_x))
    for i in (10, 50):
        nus_l, _, _ = s.candidates(nu_pre, Us, i)
        expect = [nu_pre[i], nu_pre[i - 2], nu_pre[i - 1], nu_pre[i + 1], nu_pre[i + 2]]
        if list(nus_l[:5]) != expect:
            bad.append("neighbour list")
            break
    return bad


@pytest.fixture(scope="module")
def clean_failures():
    return pin_failures(oracle.lib())


def test_the_unmodified_oracle_passes_the_compact_pins(clean_failures):
    assert clean_failures == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_planted_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) >= 1, f"mutation anchor missing: {old}"
    mutant = src.replace(old, new)
    path = oracle.build_variant(mutant, str(tmp_path / "libmutant.so"))
    failures = pin_failures(oracle.load_library(path))
    assert failures, f"planted mistake '{name}' went unnoticed"
