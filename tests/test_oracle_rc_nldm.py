"""Pins for the oracle's net RC (Eqs. 1-3) and NLDM interpolation (Section 3.1.2).

Each check compares the oracle with something other than itself: Elmore
moments written through shared-path resistances (the textbook definition, a
different formula from the oracle's two-pass recursion), closed forms on RC
chains and stars, and tables filled with exactly bilinear functions.
"""
import numpy as np
import pytest

import netgen
import oracle

KRC = 1e-3  # Ohm * fF in ps


def _shared_path_resistance(parent, res):
    n = len(parent)
    paths = []
    for u in range(n):
        s, v = set(), u
        while v > 0:
            s.add(v)
            v = parent[v]
        paths.append(s)
    R = np.zeros((n, n))
    for u in range(n):
        for i in range(n):
            R[u, i] = sum(res[v] for v in paths[u] & paths[i])
    return R


def test_elmore_rc_chain_closed_form():
    # n equal segments: D_k = R C (k n - k (k - 1) / 2), Load_k = (n - k + 1) C
    n, R, C = 12, 37.0, 2.5
    parent = [-1] + list(range(n))
    res = [0.0] + [R] * n
    cap = [0.0] + [C] * n
    load, delay, imp = oracle.elmore_tree(parent, res, cap)
    k = np.arange(n + 1, dtype=np.float64)
    np.testing.assert_allclose(delay, R * C * (k * n - k * (k - 1) / 2) * KRC, rtol=1e-13)
    np.testing.assert_allclose(load[1:], (n - k[1:] + 1) * C, rtol=1e-14)
    assert load[0] == pytest.approx(n * C)
    # second moment m2_k = sum_i R_ki C_i D_i with R_ki = R min(i, k)
    D = delay
    m2 = (R * np.minimum.outer(k, k) * C * D[None, :])[:, 1:].sum(1) * KRC
    np.testing.assert_allclose(imp, np.sqrt(np.maximum(0, 2 * m2 - D ** 2)), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_elmore_random_tree_matches_shared_path_definition(seed):
    rng = np.random.default_rng(seed)
    n = 40
    parent = [-1] + [int(rng.integers(0, u)) for u in range(1, n)]
    res = np.concatenate([[0.0], rng.uniform(1, 100, n - 1)])
    cap = rng.uniform(0.1, 5, n)
    load, delay, imp = oracle.elmore_tree(parent, res, cap)
    Rs = _shared_path_resistance(parent, res)
    D = Rs @ cap * KRC
    np.testing.assert_allclose(delay, D, rtol=1e-12)
    m2 = Rs @ (cap * D) * KRC
    np.testing.assert_allclose(imp, np.sqrt(np.maximum(0, 2 * m2 - D ** 2)), rtol=1e-10, atol=1e-14)
    # Load(u) = subtree capacitance
    sub = np.zeros(n)
    for u in range(n):
        v = u
        while v >= 0:
            sub[v] += cap[u]
            v = parent[v]
    np.testing.assert_allclose(load, sub, rtol=1e-13)


def test_star_net_closed_form_and_impulse_equals_delay():
    b = netgen.NetlistBuilder(r_per_um=0.1, c_per_um=0.2)
    d = b.pin(cap=0.7, x=10, y=20)
    sinks = [b.pin(cap=c, x=x, y=y) for c, x, y in
             [(1.0, 110, 20), (2.5, 10, -30), (0.5, 60, 70), (3.0, 10, 20)]]
    b.net(d, sinks)
    b.start(d)
    for s in sinks:
        b.end(s)
    nl, xy = b.build()
    lib = netgen.bilinear_library(1, (1, 0, 0, 0))
    r = oracle.sta(nl, lib, xy)
    dist = np.abs(xy[sinks] - xy[d]).sum(1).astype(np.float64)
    caps = nl.pin_cap[sinks].astype(np.float64)
    np.testing.assert_allclose(r["wdelay"][sinks], 0.1 * dist * (caps + 0.2 * dist / 2) * KRC, rtol=1e-12)
    np.testing.assert_allclose(r["impulse"][sinks], r["wdelay"][sinks], rtol=1e-12)
    assert r["net_load"][0] == pytest.approx(np.float64(np.float32(0.7)) + (caps + 0.2 * dist).sum(), rel=1e-13)
    # the coincident sink has zero wire delay
    assert r["wdelay"][sinks[3]] == 0.0


# ---------------------------------------------------------------------------
# NLDM
# ---------------------------------------------------------------------------
S_IDX = np.array([5, 10, 20, 50, 100, 200, 500], np.float32)
L_IDX = np.array([1, 2, 5, 10, 20, 50, 200], np.float32)
COEF = (3.0, 0.25, 1.5, 0.0625)  # dyadic: every table entry is exact in float32


def _bilinear_table(coef=COEF):
    a, b, c, e = coef
    S = S_IDX.astype(np.float64)[:, None]
    L = L_IDX.astype(np.float64)[None, :]
    t = a + b * S + c * L + e * S * L
    assert np.all(t.astype(np.float32) == t)
    return t.astype(np.float32)


def test_nldm_reproduces_bilinear_function_inside_and_outside():
    a, b, c, e = COEF
    tab = _bilinear_table()
    rng = np.random.default_rng(5)
    pts = np.concatenate([rng.uniform(0.5, 2000, (200, 2)),
                          [[1, 0.01], [1000, 1000], [5, 1], [500, 200], [4.99, 200.01]]])
    for s, l in pts:
        v, dds, ddl, _, _ = oracle.nldm(tab, S_IDX, L_IDX, s, l)
        exact = a + b * s + c * l + e * s * l
        assert v == pytest.approx(exact, rel=1e-12, abs=1e-9)
        assert dds == pytest.approx(b + e * l, rel=1e-12, abs=1e-12)
        assert ddl == pytest.approx(c + e * s, rel=1e-12, abs=1e-12)


def test_nldm_axes_not_transposed_and_grid_points_exact():
    # a table that depends on slew only must ignore the load and vice versa
    only_s = _bilinear_table((0.0, 1.0, 0.0, 0.0))
    only_l = _bilinear_table((0.0, 0.0, 1.0, 0.0))
    assert oracle.nldm(only_s, S_IDX, L_IDX, 37.0, 3.0)[0] == pytest.approx(37.0)
    assert oracle.nldm(only_l, S_IDX, L_IDX, 37.0, 3.0)[0] == pytest.approx(3.0)
    rng = np.random.default_rng(1)
    tab = rng.uniform(0, 100, (7, 7)).astype(np.float32)
    for i in range(7):
        for j in range(7):
            v, _, _, ks, kl = oracle.nldm(tab, S_IDX, L_IDX, float(S_IDX[i]), float(L_IDX[j]))
            assert v == pytest.approx(float(tab[i, j]), rel=1e-12)
            assert ks == min(i, 5) and kl == min(j, 5)  # right-continuous segments


def test_nldm_segment_choice_below_and_above_range():
    tab = _bilinear_table()
    assert oracle.nldm(tab, S_IDX, L_IDX, 1.0, 0.1)[3:] == (0, 0)
    assert oracle.nldm(tab, S_IDX, L_IDX, 1e4, 1e6)[3:] == (5, 5)
    assert oracle.nldm(tab, S_IDX, L_IDX, 10.0, 2.0)[3:] == (1, 1)
    assert oracle.nldm(tab, S_IDX, L_IDX, 9.999, 1.999)[3:] == (0, 0)


def test_nldm_monotone_table_gives_monotone_values():
    w = netgen.tiny_design(3)
    lib = w.library
    rng = np.random.default_rng(0)
    for t in range(3):
        tab = lib.delay_tab[t, 0, 0]
        s = np.sort(rng.uniform(1, 800, 30))
        vals = [oracle.nldm(tab, lib.slew_index[t], lib.load_index[t], x, 50.0)[0] for x in s]
        assert np.all(np.diff(vals) >= -1e-12)


# ---------------------------------------------------------------------------
# LSE (Eq. 4)
# ---------------------------------------------------------------------------
def test_lse_limits_and_stability():
    x = np.array([3.0, -1.0, 2.5, 2.9])
    assert oracle.lse(x, 1e-6) == pytest.approx(3.0, abs=1e-9)
    assert oracle.lse(np.full(5, 7.0), 2.0) == pytest.approx(7.0 + 2.0 * np.log(5))
    assert oracle.lse(x + 1e6, 0.5) == pytest.approx(oracle.lse(x, 0.5) + 1e6, rel=1e-15)
    assert np.isfinite(oracle.lse(np.array([1e7, 1e7 - 1]), 1e-3))
    assert oracle.lse(np.array([4.0]), 10.0) == 4.0
    # upper bound max + gamma ln n, lower bound max
    for g in (0.1, 1.0, 10.0):
        v = oracle.lse(x, g)
        assert 3.0 <= v <= 3.0 + g * np.log(4) + 1e-12
