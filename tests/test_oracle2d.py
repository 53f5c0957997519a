"""Pins of the 2-D oracle (Section V-D) against facts other than itself (no
GPU):
  - separable controllers: with f(x) = (h(x_a), h(x_b)) the problem splits
    into two copies of the one-dimensional one, so u1, the marginal cost and
    J must equal the (separately pinned) one-dimensional oracle's: U(y) =
    (U1(y_1), U1(y_2)), g(u; x) = g1(u_1; x_a) + g1(u_2; x_b), J = J1 (the
    objective carries a factor 1/2);
  - affine controllers f = lam x: J = k^2 (1 - lam)^2 s^2 + lam^2 s^2 /
    (1 + lam^2 s^2), as in one dimension;
  - S(u) against scipy's linear interpolation on the grid with clamping;
  - the search against brute force over an independently built list;
  - u1 against numpy's weighted mean;
  - the u0 half step never raises J (Corollary 1);
  - planted mistakes each fail one of these.
"""
import numpy as np
import pytest

import oracle
from paper_1908_04489_gb300 import workloads as W

P2 = dict(k=0.2, sigma=5.0, delta=1.25, x_half=12.5, w_half=5.0, y_half=20.0,
          cand_half=15.0, n_coarse=7, n_levels=6, n_nbr=2)


def one_d(p2, levels=3):
    """The one-dimensional instance on the same axis grids (n_refine 4, so
    the lattices of both sides contain the multiples of delta / 8)."""
    return W.base(k=p2["k"], sigma=p2["sigma"], delta=p2["delta"], x_half=p2["x_half"],
                  w_half=p2["w_half"], y_half=p2["y_half"], cand_half=p2["cand_half"],
                  n_refine=4, n_levels=levels)


def separable(o2, o1, h):
    """2-D lattice controller (h(x_a), h(x_b)) from 1-D values h."""
    n = o2.n_x
    tab = np.stack([np.repeat(h, n), np.tile(h, n)], axis=1)
    return o2.init(2, tab)


def test_separable_controllers_reduce_to_one_dimension():
    o2 = oracle.Oracle2D(P2)
    o1 = oracle.Oracle(one_d(P2))
    x = o2.grid(o2.n_x)
    step = P2["delta"] / 8                      # on both oracles' lattices
    h = np.round((0.8 * x + 2.0 * np.tanh(x / 3)) / step) * step
    nu1 = o1.init(2, h)
    U1 = o1.mmse(nu1)
    nu2 = separable(o2, o1, h)
    U2 = o2.mmse(nu2)
    ny = o2.n_y
    assert np.max(np.abs(U2[:, 0] - np.repeat(U1, ny))) <= 1e-12
    assert np.max(np.abs(U2[:, 1] - np.tile(U1, ny))) <= 1e-12
    # the cost splits, with the separable table built from U1 exactly
    Us = np.stack([np.repeat(U1, ny), np.tile(U1, ny)], axis=1)
    rng = np.random.default_rng(2)
    one2, one1 = 1 << o2.shift, 1 << o1.shift
    for _ in range(12):
        i = int(rng.integers(0, o2.N))
        a, b = divmod(i, o2.n_x)
        v1, v2 = rng.integers(-60, 60, 2) / 4.0 * P2["delta"]
        g2 = o2.cost(Us, i, round(v1 / P2["delta"] * one2), round(v2 / P2["delta"] * one2))
        g1 = o1.cost(U1, a, round(v1 / P2["delta"] * one1)) + \
            o1.cost(U1, b, round(v2 / P2["delta"] * one1))
        assert abs(g2 - g1) <= 1e-12 * max(1.0, g1), (i, g2, g1)
    assert abs(o2.J(nu2, Us) - o1.J(nu1, U1)) <= 1e-12


def test_affine_closed_form():
    """f = lam x with wide grids (sigma = 1): J = k^2 (1 - lam)^2 + lam^2 /
    (1 + lam^2), the one-dimensional value (Section V-D's factor 1/2 against
    two components)."""
    p = dict(k=0.2, sigma=1.0, delta=0.25, x_half=8.0, w_half=7.0, y_half=10.0,
             cand_half=6.0, n_coarse=5, n_levels=2, n_nbr=1)
    o = oracle.Oracle2D(p)
    lam = 0.5
    x = o.grid(o.n_x)
    tab = lam * np.stack([np.repeat(x, o.n_x), np.tile(x, o.n_x)], axis=1)
    nu = o.init(2, tab)
    oracle.set_threads(8)
    try:
        U = o.mmse(nu)
        J = o.J(nu, U)
    finally:
        oracle.set_threads(1)
    ref = 0.04 * (1 - lam) ** 2 + lam * lam / (1 + lam * lam)
    assert abs(J - ref) <= 1e-9, (J, ref)


def np_S(o, U, u):
    from scipy.interpolate import RegularGridInterpolator
    d = o.params["delta"]
    y = o.grid(o.n_y)
    w = o.grid(o.n_w)
    phi1 = np.exp(-w * w / 2)
    phi1 /= phi1.sum()
    pts = np.stack(np.meshgrid(u[0] + w, u[1] + w, indexing="ij"), axis=-1).reshape(-1, 2)
    pts = np.clip(pts, y[0], y[-1])
    tot = 0.0
    for k in range(2):
        f = RegularGridInterpolator((y, y), U[:, k].reshape(o.n_y, o.n_y), method="linear")
        e = u[k] - f(pts)
        tot = tot + (np.outer(phi1, phi1).ravel() * e * e)
    return float(np.sum(tot)) if np.ndim(tot) else float(tot)


def test_S_matches_library_bilinear_interpolation_with_clamping():
    o = oracle.Oracle2D(P2)
    y = o.grid(o.n_y)
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    U = np.stack([0.8 * Y1 + np.sin(Y2), 0.7 * Y2 - 0.3 * np.cos(Y1 * Y2 / 9)],
                 axis=-1).reshape(-1, 2)
    rng = np.random.default_rng(3)
    one = 1 << o.shift
    lim = int((P2["y_half"] + P2["w_half"] + 3) / P2["delta"])
    for _ in range(20):
        n1, n2 = (int(v) for v in rng.integers(-lim * one, lim * one, 2))
        ref = np_S(o, U, (float(o.value(n1)), float(o.value(n2))))
        assert abs(o.S(U, n1, n2) - ref) <= 1e-11 * max(1.0, ref)


def np_list(o, nu_pre, i):
    p = o.params
    n, r, nc = o.n_x, p["n_nbr"], p["n_coarse"]
    one = 1 << o.shift
    hr = round(p["cand_half"] / p["delta"])
    q = 2 * max(1, -(-hr // (nc - 1)))
    a, b = divmod(i, n)
    lst = [tuple(nu_pre[i])]
    for da in range(-r, r + 1):
        for db in range(-r, r + 1):
            if da == 0 and db == 0:
                continue
            aa, bb = a + da, b + db
            j = aa * n + bb if 0 <= aa < n and 0 <= bb < n else i
            lst.append(tuple(nu_pre[j]))
    for j1 in range(nc):
        for j2 in range(nc):
            lst.append(((2 * j1 - (nc - 1)) * (q // 2) * one, (2 * j2 - (nc - 1)) * (q // 2) * one))
    return lst, q


def test_search_matches_brute_force_over_the_list():
    o = oracle.Oracle2D(P2)
    y = o.grid(o.n_y)
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    U = np.stack([0.9 * Y1 + 1.5 * np.sin(Y1 / 2), 0.9 * Y2 + 0.1], axis=-1).reshape(-1, 2)
    x = o.grid(o.n_x)
    rng = np.random.default_rng(5)
    tab = np.stack([np.repeat(x, o.n_x), np.tile(x, o.n_x)], axis=1) + rng.normal(0, 0.5, (o.N, 2))
    nu_pre = o.init(2, tab)
    nu1, idx = o.search(nu_pre, U)
    k2 = P2["k"] ** 2
    X1, X2 = np.repeat(x, o.n_x), np.tile(x, o.n_x)
    for i in range(0, o.N, 37):
        base, q = np_list(o, nu_pre, i)
        cost = lambda v: k2 * ((float(o.value(v[0])) - X1[i]) ** 2 +
                               (float(o.value(v[1])) - X2[i]) ** 2) + \
            np_S(o, U, (float(o.value(v[0])), float(o.value(v[1]))))
        lst = list(base)
        costs = [cost(v) for v in lst]
        for lv in range(1, P2["n_levels"] + 1):
            best = lst[int(np.argmin(costs))]
            h = q << (P2["n_levels"] - lv)
            for s in (-1, 0, 1):
                for t in (-1, 0, 1):
                    if s == 0 and t == 0:
                        continue
                    lst.append((best[0] + s * h, best[1] + t * h))
                    costs.append(cost(lst[-1]))
        nus, gs, k = o.candidates(nu_pre, U, i)
        assert [tuple(v) for v in nus] == lst
        assert np.allclose(gs, costs, rtol=1e-11, atol=1e-12)
        assert k == int(np.argmin(costs)) == idx[i]
        assert tuple(nu1[i]) == lst[k]


def test_mmse_is_the_weighted_mean():
    o = oracle.Oracle2D(P2)
    x = o.grid(o.n_x)
    X1, X2 = np.repeat(x, o.n_x), np.tile(x, o.n_x)
    f = np.stack([X1 + np.sign(X2) * 2.0, 0.5 * X2], axis=1)
    nu = o.init(2, f)
    fv = o.value(nu)
    U = o.mmse(nu)
    y = o.grid(o.n_y)
    px, _ = o.weights()
    for t in range(0, o.n_y * o.n_y, 97):
        y1, y2 = y[t // o.n_y], y[t % o.n_y]
        w = px * np.exp(-((y1 - fv[:, 0]) ** 2 + (y2 - fv[:, 1]) ** 2) / 2)
        ref = (w @ fv) / w.sum()
        assert np.max(np.abs(U[t] - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


def test_half_step_never_raises_J():
    o = oracle.Oracle2D(P2)
    nu = o.init(0)
    U = o.mmse(nu)
    for _ in range(3):
        nu1, _ = o.search(nu, U)
        assert o.J(nu1, U) <= o.J(nu, U)
        nu = nu1
        U = o.mmse(nu)


MUTANTS = {
    "axes of the bilinear interpolation swapped": (
        "double r0 = u00 + t2 * (u01 - u00);\n    double r1 = u10 + t2 * (u11 - u10);\n"
        "    return r0 + t1 * (r1 - r0);",
        "double r0 = u00 + t1 * (u01 - u00);\n    double r1 = u10 + t1 * (u11 - u10);\n"
        "    return r0 + t2 * (r1 - r0);"),
    "second component dropped from the residual": (
        "phi2[c * m + d] * (e1 * e1 + e2 * e2)", "phi2[c * m + d] * (e1 * e1)"),
    "u1 numerator uses x0": ("n1 = n1 + w * f1;", "n1 = n1 + w * xa;"),
    "J without its factor 1/2": ("return 0.5 * J;", "return J;"),
    "neighbour window transposed": ("int64_t aa = a + da, bb = b + db;",
                                    "int64_t aa = a + db, bb = b + da;"),
}


def pin_failures(L):
    bad = []
    o2 = oracle.Oracle2D(P2, library=L)
    o1 = oracle.Oracle(one_d(P2))
    x = o2.grid(o2.n_x)
    step = P2["delta"] / 8
    h = np.round((0.8 * x + 2.0 * np.tanh(x / 3)) / step) * step
    nu1 = o1.init(2, h)
    U1 = o1.mmse(nu1)
    nu2 = separable(o2, o1, h)
    U2 = o2.mmse(nu2)
    ny = o2.n_y
    if np.max(np.abs(U2[:, 0] - np.repeat(U1, ny))) > 1e-12:
        bad.append("separable u1")
    Us = np.stack([np.repeat(U1, ny), np.tile(U1, ny)], axis=1)
    if abs(o2.J(nu2, Us) - o1.J(nu1, U1)) > 1e-12:
        bad.append("separable J")
    y = o2.grid(ny)
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    U = np.stack([0.8 * Y1 + np.sin(Y2), 0.7 * Y2 - 0.3 * np.cos(Y1 * Y2 / 9)],
                 axis=-1).reshape(-1, 2)
    one = 1 << o2.shift
    for n1, n2 in ((3 * one + 17, -5 * one + 3), (-7 * one + 40, 2 * one + 9)):
        ref = np_S(o2, U, (float(o2.value(n1)), float(o2.value(n2))))
        if abs(o2.S(U, n1, n2) - ref) > 1e-11 * max(1.0, ref):
            bad.append("S")
            break
    rng = np.random.default_rng(5)
    tab = np.stack([np.repeat(x, o2.n_x), np.tile(x, o2.n_x)], axis=1) + \
        rng.normal(0, 0.5, (o2.N, 2))
    nu_pre = o2.init(2, tab)
    for i in (o2.n_x + 3, 2 * o2.n_x + 5):
        nus, _, _ = o2.candidates(nu_pre, U, i)
        base, _ = np_list(o2, nu_pre, i)
        if [tuple(v) for v in nus[:len(base)]] != base:
            bad.append("list")
            break
    return bad


def test_the_unmodified_oracle_passes_the_2d_pins():
    assert pin_failures(oracle.lib()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_planted_mistake_fails_a_2d_pin(name, tmp_path):
    import os
    import subprocess
    old, new = MUTANTS[name]
    here = os.path.dirname(oracle.__file__)
    src = open(os.path.join(here, "ucp_oracle2d.c")).read()
    assert src.count(old) >= 1, f"mutation anchor missing: {old}"
    mut = tmp_path / "ucp_oracle2d.c"
    mut.write_text(src.replace(old, new))
    (tmp_path / "ucp_oracle2d.h").write_text(open(os.path.join(here, "ucp_oracle2d.h")).read())
    out = str(tmp_path / "libmut.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", "-fopenmp", "-I", here, "-o", out,
                    os.path.join(here, "ucp_oracle.c"), str(mut), "-lm"], check=True)
    assert pin_failures(oracle.load_library(out)), f"'{name}' went unnoticed"
