"""GPU: the tensor-core correlation tables against their exact values.

The fast path evaluates the w quadrature of Section V-A's cost through three
correlations of the Gaussian weights against E = U^(y) - y:
  P_p = sum_l phi_l w_l E_{p+l},  Q_p = sum_l phi_l E_{p+l}^2,
  R_p = sum_l phi_l E_{p+l} E_{p+l+1}.
The library builds them with exact bf16 slice products on the tensor cores and
reports, per table column, a bound on the error they cause in
S = W2 + 2[(1-t)P_p + t P_{p+1}] + (1-t)^2 Q_p + 2t(1-t) R_p + t^2 Q_{p+1}.
Here the exact correlations are formed on the CPU from the oracle's u1 table
(every product split into two doubles without error, each sum correctly
rounded by math.fsum), and every cell's table error must lie within the bound.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1908_04489_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    import torch
    assert torch.cuda.is_available()
    from paper_1908_04489_gb300 import binding as b, build
    build.build()
    b.load()
    return b


def two_prod(a, b):
    """a * b = p + e exactly (Dekker's product with Veltkamp splitting)."""
    p = a * b
    c = 134217729.0  # 2^27 + 1
    t = c * a
    ah = t - (t - a)
    al = a - ah
    t = c * b
    bh = t - (t - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def signal(p, U, jlo, n_e):
    """E_m = U^(y_{jlo+m}) - y_{jlo+m} (U constant beyond the table) and
    E_{m+1}, in FP64, for m < n_e."""
    d = p["delta"]
    hy = int(round(p["y_half"] / d))
    jj = jlo + np.arange(n_e + 1)
    e = U[np.clip(jj, 0, len(U) - 1)] - (jj - hy).astype(np.float64) * d
    return e[:n_e], e[1:n_e + 1]


def correlations(h, x, n_pos, n_w, x2=None):
    """sum_l h_l x_{p+l} (x2: times x2_{p+l}) for p < n_pos, exactly rounded."""
    out = np.empty(n_pos)
    for p0 in range(0, n_pos, 512):
        p1 = min(n_pos, p0 + 512)
        idx = np.arange(p0, p1)[:, None] + np.arange(n_w)[None, :]
        xs = x[idx]
        if x2 is None:
            a, b = two_prod(np.broadcast_to(h, xs.shape), xs)
            parts = (a, b)
        else:
            s, se = two_prod(xs, x2[idx])
            a, b = two_prod(np.broadcast_to(h, xs.shape), s)
            parts = (a, b, np.broadcast_to(h, xs.shape) * se)
        for k in range(p1 - p0):
            out[p0 + k] = math.fsum(np.concatenate([q[k] for q in parts]))
    return out


def check_tables(binding, p, nu, U, o):
    with binding.Instance(p) as inst:
        inst.set_controllers(o.value(nu), U)
        T = inst.get_tables()
    n_pos, jlo = len(T["P"]), T["jlo"]
    g = o.grids()
    w, phi = g["w"], g["phi"]
    n_w = len(w)
    e0, e1 = signal(p, U, jlo, n_pos + n_w + 1)
    a = phi * w
    P = correlations(a, e0, n_pos, n_w)
    Q = correlations(phi, e0, n_pos, n_w, x2=e0)
    R = correlations(phi, e0, n_pos, n_w, x2=e1)
    dP = np.abs(T["P"] - P)
    dQ = np.abs(T["Q"] - Q)
    dR = np.abs(T["R"] - R)
    bt = T["bound"].astype(np.float64)
    # every cell (p, p + 1): the error of S at any t in [0, 1]
    pc = np.arange(n_pos - 1)
    err = 2 * np.maximum(dP[pc], dP[pc + 1]) + np.maximum(np.maximum(dQ[pc], dR[pc]), dQ[pc + 1])
    a1, a2 = pc >> 7, (pc + 1) >> 7
    bound = bt[a1] + np.where(a2 != a1, bt[a2], 0.0)
    ratio = err / bound
    assert np.all(err <= bound), (float(ratio.max()), int(ratio.argmax()))
    # the bound is a table-precision bound, not a loose one
    Mq = np.maximum(1.0, np.maximum(Q[pc], Q[pc + 1]))
    assert np.all(bound <= 1e-10 * Mq), float((bound / Mq).max())
    print(f"max err/bound {ratio.max():.3e}  max bound/M {(bound / Mq).max():.3e}")
    return float(ratio.max()), float((bound / Mq).max())


@pytest.mark.parametrize("init", [0, 1])
def test_tables_c1(binding, init):
    p = W.c1()
    p["precision"] = 1
    o = oracle.Oracle(p)
    nu = o.init(init)
    check_tables(binding, p, nu, o.mmse(nu), o)


def test_tables_c1_after_sweeps(binding):
    """Tables of a converging state (three oracle sweeps from the staircase)."""
    p = W.c1()
    p["precision"] = 1
    o = oracle.Oracle(p)
    nu = o.init(1)
    U = o.mmse(nu)
    for _ in range(3):
        nu, _ = o.search(nu, U)
        U = o.mmse(nu)
    check_tables(binding, p, nu, U, o)


def test_tables_c2_full_size(binding):
    """Full c2 grids (10001 x0 / 2401 w / 14001 y, staircase init): 20 tap
    chunks and two column groups, as in the bench."""
    p = W.c2(precision=1)
    o = oracle.Oracle(p)
    oracle.set_threads(8)
    nu = o.init(1)
    U = o.mmse(nu)
    oracle.set_threads(1)
    check_tables(binding, p, nu, U, o)
