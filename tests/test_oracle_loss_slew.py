"""Pins for the oracle's multi-arc slew merge and for the value of the smoothed loss.

- cells with two and three arcs, slew-dependent tables different for every arc
  and transition, positive and negative unate, followed by hand: the late output
  slew is the largest arc slew, the early one the smallest, independently of the
  arc that sets the arrival time (reading c8);
- a tie between two arcs' late slews gives its gradient to the first arc: the
  oracle's gradient equals the one-sided derivative in which the first arc wins;
- TNS_gamma and WNS_gamma (Section 3.2, Eq. 4 applied to slacks) by hand on a
  design whose LSE arrival times are known in closed form, including the zero
  term of the TNS soft-min (an endpoint at zero slack contributes -gamma ln 3),
  and their gamma -> 0 limits, the hard TNS and WNS.
"""
import numpy as np
import pytest

import netgen
import oracle

S_IDX = np.array([5, 10, 20, 50, 100, 200, 500], np.float32)
L_IDX = np.array([1, 2, 5, 10, 20, 50, 200], np.float32)
KRC = 1e-3


def _library(coef, arcs, unate):
    """Tables a + b s + c l + e s l per (type, arc, rf_out, kind) from ``coef``;
    dyadic coefficients on integer grid points, so every entry is exact in
    float32 and bilinear interpolation reproduces the function exactly."""
    T = len(arcs)
    S = S_IDX.astype(np.float64)[:, None]
    L = L_IDX.astype(np.float64)[None, :]
    delay = np.zeros((T, 4, 2, 7, 7), np.float32)
    slew = np.zeros((T, 4, 2, 7, 7), np.float32)
    for (t, a, rf, kind), (ca, cb, cc, ce) in coef.items():
        tab = delay if kind == "d" else slew
        tab[t, a, rf] = ca + cb * S + cc * L + ce * S * L
    un = np.ones((T, 4), np.int8)
    for t, u in enumerate(unate):
        un[t, :] = u
    return netgen.Library(np.asarray(arcs, np.int32), un, np.tile(S_IDX, (T, 1)),
                          np.tile(L_IDX, (T, 1)), delay, slew)


def _table(coef, t, a, rf, kind, s, l):
    ca, cb, cc, ce = coef[(t, a, rf, kind)]
    return ca + cb * s + cc * l + ce * s * l


def _wire(xy, r, c, drv, snk, cap):
    """star net: (delay = impulse, wire length) of the wire drv -> snk (Eqs. 1-3)"""
    d = abs(float(xy[snk, 0]) - float(xy[drv, 0])) + abs(float(xy[snk, 1]) - float(xy[drv, 1]))
    return r * d * (cap + c * d / 2) * KRC, d


def _multi_arc_design():
    """PIs a, b, c -> cell X (type 0, two arcs, positive unate) and cell Y
    (type 1, three arcs, negative unate); X's output also feeds Y."""
    r, c = 2.0, 0.5
    bld = netgen.NetlistBuilder(r_per_um=r, c_per_um=c)
    pa = bld.pin(0.0, 0, 0)
    pb = bld.pin(0.0, 0, 40)
    pc = bld.pin(0.0, 0, 90)
    x0 = bld.pin(1.0, 30, 5)     # X arc 0
    x1 = bld.pin(2.0, 25, 45)    # X arc 1
    xo = bld.pin(0.0, 35, 20)
    y0 = bld.pin(1.5, 70, 10)    # Y arc 0 (from X)
    y1 = bld.pin(0.5, 60, 60)    # Y arc 1 (from b)
    y2 = bld.pin(2.5, 50, 95)    # Y arc 2 (from c)
    yo = bld.pin(0.0, 75, 50)
    po = bld.pin(1.0, 100, 45)
    bld.net(pa, [x0])
    bld.net(pb, [x1, y1])
    bld.net(pc, [y2])
    bld.net(xo, [y0])
    bld.net(yo, [po])
    bld.cell(0, [x0, x1], xo)
    bld.cell(1, [y0, y1, y2], yo)
    bld.start(pa, at=(1.0, 2.0, 6.0, 3.0), slew=(8.0, 30.0, 12.0, 40.0))
    bld.start(pb, at=(4.0, 1.0, 5.0, 9.0), slew=(25.0, 6.0, 60.0, 14.0))
    bld.start(pc, at=(0.5, 3.5, 2.0, 7.0), slew=(15.0, 15.0, 35.0, 22.0))
    bld.end(po, rat=(0.0, 0.0, 900.0, 800.0))
    nl, xy = bld.build()
    # different per arc and per output transition; slew tables cross (a large
    # intercept with a small slope against the opposite), so the slew max and
    # min land on different arcs from the arrival-time max
    coef = {
        (0, 0, 0, "d"): (10.0, 0.25, 1.5, 0.0), (0, 0, 0, "s"): (40.0, 0.0625, 1.0, 0.0),
        (0, 0, 1, "d"): (12.0, 0.125, 1.25, 0.0), (0, 0, 1, "s"): (6.0, 0.75, 2.0, 0.0),
        (0, 1, 0, "d"): (30.0, 0.5, 0.5, 0.0), (0, 1, 0, "s"): (5.0, 0.5, 2.5, 0.015625),
        (0, 1, 1, "d"): (8.0, 0.375, 2.0, 0.0), (0, 1, 1, "s"): (35.0, 0.125, 0.75, 0.0),
        (1, 0, 0, "d"): (6.0, 0.125, 1.0, 0.0), (1, 0, 0, "s"): (9.0, 0.25, 3.0, 0.0),
        (1, 0, 1, "d"): (14.0, 0.25, 0.75, 0.0), (1, 0, 1, "s"): (50.0, 0.0625, 0.5, 0.0),
        (1, 1, 0, "d"): (25.0, 0.0625, 1.25, 0.0), (1, 1, 0, "s"): (20.0, 0.625, 1.0, 0.0),
        (1, 1, 1, "d"): (3.0, 0.5, 1.5, 0.0078125), (1, 1, 1, "s"): (4.0, 0.875, 1.25, 0.0),
        (1, 2, 0, "d"): (16.0, 0.375, 0.25, 0.0), (1, 2, 0, "s"): (60.0, 0.03125, 0.25, 0.0),
        (1, 2, 1, "d"): (20.0, 0.125, 1.0, 0.0), (1, 2, 1, "s"): (12.0, 0.5, 2.0, 0.0),
    }
    lib = _library(coef, [2, 3], [1, -1])
    return nl, xy, lib, coef, r, c, dict(pa=pa, pb=pb, pc=pc, x0=x0, x1=x1, xo=xo, y0=y0, y1=y1,
                                         y2=y2, yo=yo, po=po)


def _after_wire(at, sl, w):
    return at + w, np.sqrt(sl * sl + w * w)


def _cell_by_hand(coef, t, unate, ins, load):
    """ins: list over arcs of (at[4], slew[4]) at the input pins.  Returns the
    output (at[4], slew[4]) and, per condition, the arcs that set the arrival
    time and the slew."""
    at = np.zeros(4)
    sl = np.zeros(4)
    at_arc, sl_arc = {}, {}
    for el in range(2):
        for rf in range(2):
            q = 2 * el + rf
            rfi = rf if unate > 0 else 1 - rf
            cand_at, cand_sl = [], []
            for k, (ai, si) in enumerate(ins):
                s_in = si[2 * el + rfi]
                cand_at.append(ai[2 * el + rfi] + _table(coef, t, k, rf, "d", s_in, load))
                cand_sl.append(_table(coef, t, k, rf, "s", s_in, load))
            pick = np.argmax if el else np.argmin
            at_arc[q], sl_arc[q] = int(pick(cand_at)), int(pick(cand_sl))
            at[q], sl[q] = cand_at[at_arc[q]], cand_sl[sl_arc[q]]
    return at, sl, at_arc, sl_arc


def test_multi_arc_slew_merge_followed_by_hand():
    nl, xy, lib, coef, r, c, p = _multi_arc_design()
    res = oracle.sta(nl, lib, xy, gamma=5.0)
    start = {int(q): k for k, q in enumerate(nl.start_pins)}
    A = {q: nl.start_at[k].astype(np.float64) for q, k in start.items()}
    Sl = {q: nl.start_slew[k].astype(np.float64) for q, k in start.items()}
    cap = nl.pin_cap.astype(np.float64)

    def sink(drv, snk, at, sl):
        w, _ = _wire(xy, r, c, drv, snk, cap[snk])
        return _after_wire(at, sl, w)

    ax0, sx0 = sink(p["pa"], p["x0"], A[p["pa"]], Sl[p["pa"]])
    ax1, sx1 = sink(p["pb"], p["x1"], A[p["pb"]], Sl[p["pb"]])
    ld_x = cap[p["y0"]] + c * _wire(xy, r, c, p["xo"], p["y0"], 0.0)[1]
    at_x, sl_x, atx_arc, slx_arc = _cell_by_hand(coef, 0, 1, [(ax0, sx0), (ax1, sx1)], ld_x)
    np.testing.assert_allclose(res["at"][p["xo"]], at_x, rtol=1e-13)
    np.testing.assert_allclose(res["slew"][p["xo"]], sl_x, rtol=1e-13)

    ay0, sy0 = sink(p["xo"], p["y0"], at_x, sl_x)
    ay1, sy1 = sink(p["pb"], p["y1"], A[p["pb"]], Sl[p["pb"]])
    ay2, sy2 = sink(p["pc"], p["y2"], A[p["pc"]], Sl[p["pc"]])
    ld_y = cap[p["po"]] + c * _wire(xy, r, c, p["yo"], p["po"], 0.0)[1]
    at_y, sl_y, aty_arc, sly_arc = _cell_by_hand(coef, 1, -1, [(ay0, sy0), (ay1, sy1), (ay2, sy2)], ld_y)
    np.testing.assert_allclose(res["at"][p["yo"]], at_y, rtol=1e-13)
    np.testing.assert_allclose(res["slew"][p["yo"]], sl_y, rtol=1e-13)
    apo, spo = sink(p["yo"], p["po"], at_y, sl_y)
    np.testing.assert_allclose(res["slew"][p["po"]], spo, rtol=1e-13)

    # the design discriminates: the late slew comes from another arc than the
    # late arrival, and the early slew from another arc than the late slew
    assert any(slx_arc[q] != atx_arc[q] for q in (2, 3)) and any(sly_arc[q] != aty_arc[q] for q in (2, 3))
    assert any(slx_arc[q] != slx_arc[q - 2] for q in (2, 3)) and any(sly_arc[q] != sly_arc[q - 2] for q in (2, 3))


def _tie_design():
    """Two PIs with equal assertions drive the two inputs of cell X (type 0:
    both arcs have the same tables) over equal wires, so X's two late slews tie
    exactly; X drives a buffer whose delay depends strongly on its input slew."""
    r, c = 20.0, 2.0
    bld = netgen.NetlistBuilder(r_per_um=r, c_per_um=c)
    p0 = bld.pin(0.0, 0, 0)
    p1 = bld.pin(0.0, 0, 50)
    i0 = bld.pin(1.0, 30, 0)
    i1 = bld.pin(1.0, 30, 50)
    xo = bld.pin(0.0, 30, 25)
    bi = bld.pin(1.0, 34, 25)
    bo = bld.pin(0.0, 34, 30)
    po = bld.pin(1.0, 36, 30)
    bld.net(p0, [i0])
    bld.net(p1, [i1])
    bld.net(xo, [bi])
    bld.net(bo, [po])
    bld.cell(0, [i0, i1], xo)
    bld.cell(1, [bi], bo)
    for q in (p0, p1):
        bld.start(q, at=(0.0, 0.0, 5.0, 5.0), slew=(10.0, 10.0, 10.0, 10.0))
    bld.end(po, rat=(0.0, 0.0, 50.0, 50.0))
    nl, xy = bld.build()
    coef = {}
    for rf in range(2):
        for k in range(2):
            coef[(0, k, rf, "d")] = (6.0 + 2 * rf, 0.25, 0.5, 0.0)
            coef[(0, k, rf, "s")] = (4.0 + rf, 0.75, 1.0, 0.0)
        coef[(1, 0, rf, "d")] = (3.0, 2.0, 0.25, 0.0)
        coef[(1, 0, rf, "s")] = (5.0, 0.5, 0.5, 0.0)
    lib = _library(coef, [2, 1], [1, 1])
    return nl, xy, lib, dict(i0=i0, i1=i1)


def test_late_slew_tie_gives_its_gradient_to_the_first_arc():
    nl, xy, lib, p = _tie_design()
    gamma, wt, ww = 5.0, 1.0, 0.5
    r = oracle.sta(nl, lib, xy, gamma, wt, ww)
    assert np.array_equal(r["slew"][p["i0"]], r["slew"][p["i1"]])  # the tie is exact
    base = xy.astype(np.float64)
    f0, _ = oracle.loss(nl, lib, base, gamma, wt, ww)
    h = 1e-6

    def one_sided(pin, sign):
        x = base.copy()
        x[pin, 0] += sign * h
        f, _ = oracle.loss(nl, lib, x, gamma, wt, ww)
        return sign * (f - f0) / h

    scale = np.abs(r["grad"]).max()
    # moving i0 right raises its slew, so arc 0 wins: the right derivative has
    # arc 0's slew term; moving i1 left lowers its slew, so arc 0 still wins
    right0, left0 = one_sided(p["i0"], +1), one_sided(p["i0"], -1)
    right1, left1 = one_sided(p["i1"], +1), one_sided(p["i1"], -1)
    assert abs(right0 - left0) > 0.05 * scale and abs(right1 - left1) > 0.05 * scale
    assert r["grad"][p["i0"], 0] == pytest.approx(right0, abs=1e-4 * scale)
    assert r["grad"][p["i1"], 0] == pytest.approx(left1, abs=1e-4 * scale)


# ---------------------------------------------------------------------------
# smoothed loss values
# ---------------------------------------------------------------------------
def _softmin(x, gamma):
    x = np.asarray(x, np.float64)
    m = x.min()
    return m - gamma * np.log(np.exp(-(x - m) / gamma).sum())


def _fanout_design(rats):
    """One PI driving endpoints directly: the LSE arrival time of an endpoint
    is the PI's late arrival plus the wire delay (no cell on the way)."""
    r, c = 1.0, 0.5
    bld = netgen.NetlistBuilder(r_per_um=r, c_per_um=c)
    pi = bld.pin(0.0, 10, 10)
    ends = []
    places = [(10, 10), (40, 10), (10, 70), (25, 35), (60, 60)]
    for k, rat in enumerate(rats):
        q = bld.pin(0.5 + 0.5 * k, *places[k])
        ends.append(q)
        bld.end(q, rat=rat)
    bld.net(pi, ends)
    bld.start(pi, at=(0.0, 0.0, 20.0, 30.0), slew=(10.0,) * 4)
    nl, xy = bld.build()
    lib = netgen.bilinear_library(1, (1.0, 0.0, 0.0, 0.0))
    return nl, xy, lib, r, c


def test_smoothed_tns_wns_by_hand():
    # endpoint 0 sits on the PI (zero wire) with its late bounds equal to the
    # PI's late arrivals: zero slack on both transitions
    rats = [(0.0, 0.0, 20.0, 30.0), (0.0, 0.0, 15.0, 45.0), (0.0, 0.0, 60.0, 10.0),
            (0.0, 0.0, 900.0, 950.0), (0.0, 0.0, 22.0, 31.0)]
    nl, xy, lib, r, c = _fanout_design(rats)
    gamma, wt, ww = 4.0, 0.75, 0.25
    res = oracle.sta(nl, lib, xy, gamma, wt, ww)
    pi = int(nl.start_pins[0])
    s = []
    for e, q in enumerate(nl.end_pins):
        w, _ = _wire(xy, r, c, pi, int(q), float(nl.pin_cap[q]))
        s.append([rats[e][2] - (20.0 + w), rats[e][3] - (30.0 + w)])
    s = np.array(s)
    assert s[0, 0] == 0.0 and s[0, 1] == 0.0
    tns_g = sum(-gamma * np.log(np.exp(-s[e, 0] / gamma) + np.exp(-s[e, 1] / gamma) + 1.0)
                for e in range(len(rats)))
    wns_g = -gamma * np.log(np.exp(-s.reshape(-1) / gamma).sum())
    sm = res["summary"]
    assert sm["tns_gamma"] == pytest.approx(tns_g, rel=1e-12)
    assert sm["wns_gamma"] == pytest.approx(wns_g, rel=1e-12)
    assert sm["loss"] == pytest.approx(wt * tns_g + ww * wns_g, rel=1e-12)
    # the endpoint far inside its bounds contributes (almost) nothing: the 0 of
    # the soft-min {s_rise, s_fall, 0} is there
    only_far = _fanout_design([rats[3]])
    r3 = oracle.sta(only_far[0], only_far[2], only_far[1], gamma, 1.0, 0.0)
    assert abs(r3["summary"]["tns_gamma"]) < 1e-50


def test_zero_slack_endpoint_gives_minus_gamma_log3():
    nl, xy, lib, _, _ = _fanout_design([(0.0, 0.0, 20.0, 30.0)])
    for gamma in (1.0, 10.0):
        res = oracle.sta(nl, lib, xy, gamma, 1.0, 1.0)
        assert res["summary"]["tns_gamma"] == pytest.approx(-gamma * np.log(3.0), rel=1e-14)
        assert res["summary"]["wns_gamma"] == pytest.approx(-gamma * np.log(2.0), rel=1e-14)
        assert res["summary"]["tns_late"] == 0.0 and res["summary"]["wns_late"] == 0.0


def test_smoothed_loss_tends_to_hard_tns_wns():
    w = netgen.tiny_design(0)
    hard = oracle.sta(w.netlist, w.library, w.xy, gamma=10.0)["summary"]
    assert hard["tns_late"] < 0 and hard["late_violations"] > 10
    res = oracle.sta(w.netlist, w.library, w.xy, gamma=1e-6)["summary"]
    E = w.netlist.end_pins.shape[0]
    # |TNS_g - TNS| <= E gamma ln 3 + the LSE arrival excess (depth gamma ln 4)
    assert res["tns_gamma"] == pytest.approx(hard["tns_late"], abs=E * 1e-6 * 2 + 1e-3)
    assert res["wns_gamma"] == pytest.approx(hard["wns_late"], abs=1e-3)
    # at gamma = 10 ps the smoothed values sit below the hard ones (soft-min <= min)
    s10 = oracle.sta(w.netlist, w.library, w.xy, gamma=10.0)["summary"]
    assert s10["tns_gamma"] < hard["tns_late"] and s10["wns_gamma"] < hard["wns_late"]
