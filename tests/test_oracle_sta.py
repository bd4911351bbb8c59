"""Pins for the oracle's propagation, slack, smoothed loss and gradient.

- arrival and required times equal brute-force enumeration of every path on
  tiny DAGs (slew-independent tables, so every edge delay is fixed);
- a hand-wired buffer chain with slew-dependent tables is followed step by step;
- slack / WNS / TNS invariants, the critical path's slack equals WNS, early <=
  late, LSE arrival >= max arrival and -> max as gamma -> 0;
- gradients equal FP64 central finite differences, and sum to zero under
  translation;
- levels equal the constructed levels and satisfy their defining recursion.
"""
import numpy as np
import pytest

import netgen
import oracle
from tests import _tinydag as td


@pytest.mark.parametrize("clocked", [0, 1])
@pytest.mark.parametrize("seed", range(6))
def test_at_rat_equal_path_enumeration(seed, clocked):
    w = td.tiny_netlist(seed, clock_nets=clocked)
    nl = w.netlist
    lib, A, B = td.linear_library(5, [1, 2, 3, 4, 1], seed=seed)
    r = oracle.sta(nl, lib, w.xy)
    arr, req = td.enumerate_paths(nl, lib, A, B, w.xy)
    # required times of clocked endpoints move with the capturing clock's arrival
    # (hold: latest rising edge, setup: earliest); unclocked ones are constants
    hold_shift = np.zeros(nl.end_pins.shape[0])
    setup_shift = np.zeros(nl.end_pins.shape[0])
    if nl.end_clock is not None:
        for e, k in enumerate(nl.end_clock):
            if k >= 0:
                hold_shift[e] = max(arr[(int(k), 0)])
                setup_shift[e] = min(arr[(int(k), 0)])
        assert np.count_nonzero(setup_shift) > 0
    for p in range(nl.num_pins):
        for rf in range(2):
            vals = arr[(p, rf)]
            assert r["at"][p, 2 + rf] == pytest.approx(max(vals), rel=1e-12, abs=1e-9)
            assert r["at"][p, rf] == pytest.approx(min(vals), rel=1e-12, abs=1e-9)
            paths = req[(p, rf)]
            if not paths:
                assert r["rat"][p, 2 + rf] == np.inf and r["rat"][p, rf] == -np.inf
                continue
            late = min(float(nl.end_rat[e, 2 + rfe]) + setup_shift[e] - d for e, rfe, d in paths)
            early = max(float(nl.end_rat[e, rfe]) + hold_shift[e] - d for e, rfe, d in paths)
            assert r["rat"][p, 2 + rf] == pytest.approx(late, rel=1e-12, abs=1e-9)
            assert r["rat"][p, rf] == pytest.approx(early, rel=1e-12, abs=1e-9)


def test_buffer_chain_slews_followed_by_hand():
    # PI -> buf0 (positive unate) -> inv1 (negative unate) -> PO, tables a + b s + c l + e s l
    b = netgen.NetlistBuilder(r_per_um=0.5, c_per_um=0.25)
    pi = b.pin(0.0, 0, 0)
    i0 = b.pin(1.0, 40, 0)
    o0 = b.pin(0.0, 40, 0)
    i1 = b.pin(2.0, 40, 60)
    o1 = b.pin(0.0, 40, 60)
    po = b.pin(1.5, 0, 60)
    b.net(pi, [i0])
    b.net(o0, [i1])
    b.net(o1, [po])
    b.cell(0, [i0], o0)
    b.cell(1, [i1], o1)
    b.start(pi, at=(1.0, 2.0, 3.0, 4.0), slew=(10.0, 11.0, 12.0, 13.0))
    b.end(po, rat=(0.0, 0.0, 500.0, 400.0))
    nl, xy = b.build()
    lib, coef = _two_type_library()
    lib.arc_unate[0, :] = 1
    lib.arc_unate[1, :] = -1
    r = oracle.sta(nl, lib, xy)

    def wire(d, cap):  # star: delay = impulse = r d (cap + c d / 2) k
        return 0.5 * d * (cap + 0.25 * d / 2) * 1e-3

    def table(t, rf, kind, s, l):
        a, bb, c, e = coef[(t, rf, kind)]
        return a + bb * s + c * l + e * s * l

    at = {0: 1.0, 1: 2.0, 2: 3.0, 3: 4.0}
    sl = {0: 10.0, 1: 11.0, 2: 12.0, 3: 13.0}
    # wire pi -> i0 (40 um)
    w0 = wire(40, 1.0)
    at = {q: v + w0 for q, v in at.items()}
    sl = {q: np.hypot(v, w0) for q, v in sl.items()}
    np.testing.assert_allclose(r["at"][i0], [at[q] for q in range(4)], rtol=1e-13)
    np.testing.assert_allclose(r["slew"][i0], [sl[q] for q in range(4)], rtol=1e-13)
    # buf0 drives 60 um to i1 (cap 2): load = 2 + 0.25 * 60
    load0 = 2.0 + 0.25 * 60
    at = {q: at[q] + table(0, q % 2, "d", sl[q], load0) for q in range(4)}
    sl = {q: table(0, q % 2, "s", sl[q], load0) for q in range(4)}
    np.testing.assert_allclose(r["at"][o0], [at[q] for q in range(4)], rtol=1e-13)
    w1 = wire(60, 2.0)
    at = {q: v + w1 for q, v in at.items()}
    sl = {q: np.hypot(v, w1) for q, v in sl.items()}
    # inv1 is negative unate: output rise comes from input fall
    load1 = 1.5 + 0.25 * 40
    at2, sl2 = {}, {}
    for el in range(2):
        for rf in range(2):
            q_in = 2 * el + (1 - rf)
            at2[2 * el + rf] = at[q_in] + table(1, rf, "d", sl[q_in], load1)
            sl2[2 * el + rf] = table(1, rf, "s", sl[q_in], load1)
    np.testing.assert_allclose(r["at"][o1], [at2[q] for q in range(4)], rtol=1e-13)
    np.testing.assert_allclose(r["slew"][o1], [sl2[q] for q in range(4)], rtol=1e-13)
    w2 = wire(40, 1.5)
    np.testing.assert_allclose(r["at"][po], [at2[q] + w2 for q in range(4)], rtol=1e-13)
    # endpoint slacks: early = AT - RAT_c, late = RAT_c - AT, min over rise/fall
    late = min(500.0 - (at2[2] + w2), 400.0 - (at2[3] + w2))
    early = min(at2[0] + w2, at2[1] + w2)
    assert r["ep_slack"][0, 1] == pytest.approx(late, rel=1e-13)
    assert r["ep_slack"][0, 0] == pytest.approx(early, rel=1e-13)
    # a single-arc cell makes the LSE arrival equal to the late arrival
    np.testing.assert_allclose(r["ats"][po], r["at"][po, 2:], rtol=1e-13)


def _two_type_library():
    s_idx = np.tile(np.array([5, 10, 20, 50, 100, 200, 500], np.float32), (2, 1))
    l_idx = np.tile(np.array([1, 2, 5, 10, 20, 50, 200], np.float32), (2, 1))
    S = s_idx[0].astype(np.float64)[:, None]
    L = l_idx[0].astype(np.float64)[None, :]
    coef = {}
    delay = np.zeros((2, 4, 2, 7, 7), np.float32)
    slew = np.zeros((2, 4, 2, 7, 7), np.float32)
    vals = [(3.0, 0.25, 1.5, 0.0625), (5.0, 0.125, 2.0, 0.03125), (2.5, 0.5, 0.75, 0.015625),
            (4.0, 0.375, 1.25, 0.0078125), (6.0, 0.0625, 3.0, 0.0), (7.5, 0.25, 0.5, 0.0625),
            (1.0, 0.75, 1.0, 0.03125), (8.0, 0.125, 2.5, 0.015625)]
    k = 0
    for t in range(2):
        for rf in range(2):
            for kind, tab in (("d", delay), ("s", slew)):
                coef[(t, rf, kind)] = vals[k]
                a, b, c, e = vals[k]
                tab[t, :, rf] = (a + b * S + c * L + e * S * L)[None]
                k += 1
    lib = netgen.Library(np.array([1, 1], np.int32), np.ones((2, 4), np.int8), s_idx, l_idx,
                         delay, slew)
    return lib, coef


@pytest.fixture(scope="module")
def tiny():
    w = netgen.tiny_design(0)
    return w, oracle.sta(w.netlist, w.library, w.xy, gamma=10.0)


def test_slack_wns_tns_invariants(tiny):
    w, r = tiny
    nl = w.netlist
    at, rat, ps, es = r["at"], r["rat"], r["pin_slack"], r["ep_slack"]
    np.testing.assert_allclose(ps[:, 1], np.min(rat[:, 2:] - at[:, 2:], axis=1), rtol=0, atol=1e-9)
    np.testing.assert_allclose(ps[:, 0], np.min(at[:, :2] - rat[:, :2], axis=1), rtol=0, atol=1e-9)
    s = r["summary"]
    assert s["tns_late"] == pytest.approx(np.minimum(es[:, 1], 0).sum(), rel=1e-12)
    assert s["wns_late"] == pytest.approx(es[:, 1].min(), rel=1e-12)
    assert s["tns_early"] == pytest.approx(np.minimum(es[:, 0], 0).sum(), abs=1e-9)
    assert s["wns_early"] == pytest.approx(es[:, 0].min(), rel=1e-12)
    assert s["late_violations"] == (es[:, 1] < 0).sum()
    # early <= late for arrival times and slews (monotone tables), LSE >= max
    assert np.all(at[:, :2] <= at[:, 2:] + 1e-9)
    assert np.all(r["slew"][:, :2] <= r["slew"][:, 2:] + 1e-9)
    assert np.all(r["ats"] >= at[:, 2:] - 1e-9)
    # every endpoint pin has no fanout here, so its propagated RAT is its constraint
    np.testing.assert_allclose(rat[nl.end_pins], nl.end_rat.astype(np.float64), rtol=0, atol=0)


def test_critical_path_slack_equals_wns(tiny):
    w, r = tiny
    nl = w.netlist
    wns = r["summary"]["wns_late"]
    e = int(np.argmin(r["ep_slack"][:, 1]))
    p = int(nl.end_pins[e])
    rf = int(np.argmin(nl.end_rat[e, 2:] - r["at"][p, 2:]))
    sink_of = {}
    for n in range(nl.num_nets):
        for s in nl.net_pins[nl.net_ptr[n] + 1:nl.net_ptr[n + 1]]:
            sink_of[int(s)] = int(nl.net_pins[nl.net_ptr[n]])
    out_cell = {int(o): c for c, o in enumerate(nl.cell_out_pin)}
    steps = 0
    while True:
        assert r["pin_slack"][p, 1] == pytest.approx(wns, abs=1e-6 * abs(wns))
        steps += 1
        if p in sink_of:
            p = sink_of[p]
        elif p in out_cell:
            c = out_cell[p]
            t = nl.cell_type[c]
            best, nxt = -np.inf, None
            for ai, i in enumerate(nl.cell_in_pins[nl.cell_in_ptr[c]:nl.cell_in_ptr[c + 1]]):
                a = nl.cell_in_ptr[c] + ai
                rfi = rf if w.library.arc_unate[t, ai] > 0 else 1 - rf
                v = r["at"][i, 2 + rfi] + r["adel"][a, 2 + rf]
                if v > best:
                    best, nxt = v, (int(i), rfi)
            p, rf = nxt
        else:
            break
    assert steps > 10


def test_lse_arrival_tends_to_max(tiny):
    w, _ = tiny
    r = oracle.sta(w.netlist, w.library, w.xy, gamma=1e-7)
    np.testing.assert_allclose(r["ats"], r["at"][:, 2:], rtol=1e-9, atol=1e-6)


def test_levels_match_construction_and_recursion(tiny):
    w, _ = tiny
    nl = w.netlist
    lv = oracle.levels(nl)
    np.testing.assert_array_equal(lv, w.info["net_level"])
    sink_net = np.full(nl.num_pins, -1)
    for n in range(nl.num_nets):
        sink_net[nl.net_pins[nl.net_ptr[n] + 1:nl.net_ptr[n + 1]]] = n
    out_cell = {int(o): c for c, o in enumerate(nl.cell_out_pin)}
    for n in range(nl.num_nets):
        d = int(nl.net_pins[nl.net_ptr[n]])
        if d not in out_cell:
            assert lv[n] == 0
            continue
        c = out_cell[d]
        feeds = [sink_net[i] for i in nl.cell_in_pins[nl.cell_in_ptr[c]:nl.cell_in_ptr[c + 1]]]
        assert lv[n] == 1 + max([lv[m] for m in feeds if m >= 0], default=-1)


def test_cycle_and_invalid_netlists_are_rejected():
    b = netgen.NetlistBuilder()
    i0, o0, i1, o1 = (b.pin(1.0) for _ in range(4))
    b.net(o0, [i1])
    b.net(o1, [i0])
    b.cell(0, [i0], o0)
    b.cell(0, [i1], o1)
    nl, xy = b.build()
    lib = netgen.bilinear_library(1, (1, 0, 0, 0))
    lib.type_num_arcs[:] = 1
    with pytest.raises(oracle.OracleError, match="cycle"):
        oracle.sta(nl, lib, xy)
    with pytest.raises(oracle.OracleError, match="cycle"):
        oracle.levels(nl)
    # a pin with two sources (asserted and a net sink)
    b2 = netgen.NetlistBuilder()
    d, s = b2.pin(), b2.pin(1.0)
    b2.net(d, [s])
    b2.start(d)
    b2.start(s)
    nl2, xy2 = b2.build()
    with pytest.raises(oracle.OracleError, match="invalid"):
        oracle.sta(nl2, lib, xy2)


# ---------------------------------------------------------------------------
# gradient
# ---------------------------------------------------------------------------
def _check_fd(nl, lib, xy, pins, gamma, w_tns, w_wns, tol):
    r = oracle.sta(nl, lib, xy, gamma, w_tns, w_wns)
    fd, ok = oracle.finite_difference(nl, lib, xy, pins, gamma, w_tns, w_wns, h=1e-3)
    g = r["grad"][pins]
    scale = max(1.0, np.abs(r["grad"]).max())
    assert ok.mean() > 0.8
    err = np.abs(g - fd)[ok]
    assert err.max() <= tol * scale, (err.max(), scale)
    return r


@pytest.mark.parametrize("clocked", [0, 1])
@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("weights", [(1.0, 0.0), (0.0, 1.0), (0.7, 0.3)])
def test_gradient_matches_finite_differences_tiny(seed, weights, clocked):
    w = td.tiny_netlist(seed, n_comb=12, depth=5, clock_nets=clocked)
    gamma = 5.0
    r = _check_fd(w.netlist, w.library, w.xy, np.arange(w.netlist.num_pins), gamma,
                  weights[0], weights[1], tol=2e-6)
    assert np.abs(r["grad"]).max() > 0


def test_gradient_matches_finite_differences_design():
    w = netgen.tiny_design(0)
    rng = np.random.default_rng(7)
    pins = rng.choice(w.netlist.num_pins, size=60, replace=False)
    _check_fd(w.netlist, w.library, w.xy, pins, 10.0, 1.0, 0.5, tol=2e-6)


def test_gradient_translation_invariance():
    w = netgen.tiny_design(1)
    r = oracle.sta(w.netlist, w.library, w.xy, 10.0, 1.0, 1.0)
    g = r["grad"]
    assert abs(g[:, 0].sum()) <= 1e-9 * np.abs(g).sum()
    assert abs(g[:, 1].sum()) <= 1e-9 * np.abs(g).sum()
    moved = w.xy.astype(np.float64) + np.array([123.25, -45.5])
    r2 = oracle.sta(w.netlist, w.library, moved, 10.0, 1.0, 1.0)
    assert r2["summary"]["loss"] == pytest.approx(r["summary"]["loss"], rel=1e-12)


# ---------------------------------------------------------------------------
# propagated clock
# ---------------------------------------------------------------------------
def _clock_pair():
    """Clock source c -> (ck1, ck2); flop F1 (ck1 -> q1) launches into d2, the
    D pin captured by flop F2 (ck2 -> q2 -> po).  Slew-independent tables."""
    b = netgen.NetlistBuilder(r_per_um=0.5, c_per_um=0.25)
    c = b.pin(0.0, 5, 7)
    ck1 = b.pin(1.0, 25, 3)
    q1 = b.pin(0.0, 27, 6)
    d2 = b.pin(1.5, 60, 20)
    ck2 = b.pin(2.0, 9, 45)
    q2 = b.pin(0.0, 12, 47)
    po = b.pin(1.0, 80, 31)
    b.net(c, [ck1, ck2])
    b.net(q1, [d2])
    b.net(q2, [po])
    b.cell(0, [ck1], q1)
    b.cell(0, [ck2], q2)
    b.start(c, at=(1.0, 1.0, 4.0, 4.0), slew=(20.0,) * 4)
    b.end(d2, rat=(2.0, 2.0, 15.0, 15.0), clock=ck2)
    b.end(po, rat=(0.0, 0.0, 1000.0, 1000.0))
    nl, xy = b.build()
    lib, A, B = td.linear_library(1, [1], seed=3)
    lib.arc_unate[:] = 1
    return nl, xy, lib, A, B, dict(c=c, ck1=ck1, q1=q1, d2=d2, ck2=ck2)


def test_propagated_clock_followed_by_hand():
    nl, xy, lib, A, B, p = _clock_pair()
    r = oracle.sta(nl, lib, xy, gamma=5.0)

    x = xy.astype(np.float64)

    def wire(drv, snk, cap):
        d = abs(x[snk, 0] - x[drv, 0]) + abs(x[snk, 1] - x[drv, 1])
        return 0.5 * d * (cap + 0.25 * d / 2) * 1e-3, d

    w1, _ = wire(p["c"], p["ck1"], 1.0)
    w2, _ = wire(p["c"], p["ck2"], 2.0)
    wd2, dist = wire(p["q1"], p["d2"], 1.5)
    load1 = 1.5 + 0.25 * dist
    q = [A[0, 0, rf] + B[0, 0, rf] * load1 for rf in range(2)]
    at_late = [4.0 + w1 + q[rf] + wd2 for rf in range(2)]
    at_early = [1.0 + w1 + q[rf] + wd2 for rf in range(2)]
    np.testing.assert_allclose(r["at"][p["d2"]], at_early + at_late, rtol=1e-13)
    rat_hold = 2.0 + 4.0 + w2     # latest capture edge
    rat_setup = 15.0 + 1.0 + w2   # earliest capture edge
    np.testing.assert_allclose(r["rat"][p["d2"]], [rat_hold, rat_hold, rat_setup, rat_setup], rtol=1e-13)
    assert r["ep_slack"][0, 1] == pytest.approx(min(rat_setup - a for a in at_late), rel=1e-13)
    assert r["ep_slack"][0, 0] == pytest.approx(min(a - rat_hold for a in at_early), rel=1e-13)
    assert r["ep_slack"][0, 1] < 0  # the capture term must reach the gradient below


def test_propagated_clock_gradient_by_finite_differences():
    nl, xy, lib, _, _, p = _clock_pair()
    r = _check_fd(nl, lib, xy, np.arange(nl.num_pins), 5.0, 1.0, 0.5, tol=2e-6)
    assert np.abs(r["grad"][p["ck2"]]).max() > 0


def test_zero_length_clock_wires_equal_ideal_clock():
    """With every CK pin at its clock source the wires vanish: the design equals
    the ideal-clock one with CK asserted at the clock arrival and D bounds moved
    by the capture edge (hold +late, setup +early)."""
    wc = netgen.tiny_design(0, clock_nets=2)
    wi = netgen.tiny_design(0)
    nc, ni = wc.netlist, wi.netlist
    P0 = ni.num_pins
    xy = wc.xy.astype(np.float64).copy()
    for n in range(ni.num_nets, nc.num_nets):
        pins = nc.net_pins[nc.net_ptr[n]:nc.net_ptr[n + 1]]
        xy[pins[1:]] = xy[pins[0]]
    clock_at = nc.start_at[-1]
    ideal = netgen.Netlist(**{f.name: getattr(ni, f.name) for f in netgen.dataclasses.fields(ni)})
    ideal.start_at = ni.start_at.copy()
    ck = np.isin(ni.start_pins, wc.info["ck_pins"])
    ideal.start_at[ck] = clock_at
    ideal.end_rat = ni.end_rat.copy()
    clocked = nc.end_clock >= 0
    ideal.end_rat[clocked] += np.array([clock_at[2], clock_at[2], clock_at[0], clock_at[0]], np.float32)
    rc = oracle.sta(nc, wc.library, xy, 10.0, 1.0, 0.5)
    ri = oracle.sta(ideal, wi.library, xy[:P0], 10.0, 1.0, 0.5)
    for k in ("at", "slew", "rat", "ats", "pin_slack"):
        np.testing.assert_array_equal(rc[k][:P0], ri[k], err_msg=k)
    np.testing.assert_array_equal(rc["ep_slack"], ri["ep_slack"])
    np.testing.assert_allclose(rc["grad"][:P0], ri["grad"], rtol=1e-12, atol=1e-12)
    for k in ri["summary"]:
        assert rc["summary"][k] == pytest.approx(ri["summary"][k], rel=1e-13)


def test_clocked_design_gradient_matches_finite_differences():
    w = netgen.tiny_design(1, clock_nets=2)
    nl = w.netlist
    rng = np.random.default_rng(11)
    pins = np.concatenate([nl.start_pins[-2:], rng.choice(w.info["ck_pins"], 20, replace=False),
                           rng.choice(nl.num_pins, 20, replace=False)])
    _check_fd(nl, w.library, w.xy, pins, 10.0, 1.0, 0.5, tol=2e-6)


def test_capturing_clock_must_hang_on_a_startpoint_net():
    nl, xy, lib, _, _, p = _clock_pair()
    bad = netgen.Netlist(**{f.name: getattr(nl, f.name) for f in netgen.dataclasses.fields(nl)})
    bad.end_clock = np.array([p["q1"], -1], np.int32)  # a cell output, not a clock-net sink
    with pytest.raises(oracle.OracleError, match="invalid"):
        oracle.sta(bad, lib, xy)
