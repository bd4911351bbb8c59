"""The synthetic inputs follow their stated recipe (CPU only).

The contest designs the paper measures on (ICCAD 2015 superblue, ICCAD 2025
aes_cipher_top) are not available, so every test and the bench run on seeded
netlists from ``netgen``.  These tests check the generated netlists against the
shapes the recipe states: cell, flop, primary-input and primary-output counts,
logic depth, the fanout law and its cap, the placement box, pin capacitances,
the wire constants and the NLDM tables (7x7, monotone in input slew and load,
over 5-500 ps and 1-200 fF), and that jittered placements have the stated
spread.  The level count is the oracle's own levelization.
"""
import numpy as np
import pytest

import netgen
import oracle


def _sinks_per_net(nl):
    return np.diff(np.asarray(nl.net_ptr)) - 1


def _check_library(lib, num_types):
    assert lib.num_types == num_types
    s_idx = np.asarray(lib.slew_index).reshape(num_types, -1)
    l_idx = np.asarray(lib.load_index).reshape(num_types, -1)
    assert s_idx.shape[1] == 7 and l_idx.shape[1] == 7
    assert np.all(np.diff(s_idx, axis=1) > 0) and np.all(np.diff(l_idx, axis=1) > 0)
    assert np.allclose(s_idx[:, 0], 5.0) and np.allclose(s_idx[:, -1], 500.0)
    assert np.allclose(l_idx[:, 0], 1.0) and np.allclose(l_idx[:, -1], 200.0)
    assert set(np.asarray(lib.type_num_arcs).tolist()) <= {1, 2, 3, 4}
    for tab in (lib.delay_tab, lib.slew_tab):
        t = np.asarray(tab, np.float64).reshape(-1, 7, 7)
        assert np.all(t > 0)
        assert np.all(np.diff(t, axis=1) > 0), "monotone in input slew"
        assert np.all(np.diff(t, axis=2) > 0), "monotone in load"


def test_tiny_design_recipe():
    w = netgen.tiny_design(0)
    nl = w.netlist
    # 2,000 combinational cells and 200 flops; 100 PIs + 200 flop outputs start
    # paths, 100 POs + 200 flop D pins end them
    assert nl.num_cells == 2200
    assert len(nl.start_pins) == 300 and len(nl.end_pins) == 300
    assert 6000 <= nl.num_pins <= 12000
    levels = oracle.levels(nl)
    assert int(np.max(levels)) + 1 in (30, 31, 32)  # 30 logic levels, plus flop / PI / PO ends
    k = _sinks_per_net(nl)
    assert k.max() <= 16 + 1  # geometric(0.4) capped at 16 (plus a sink-less net's endpoint)
    assert 1.8 <= k.mean() <= 3.2  # the geometric law's mean 1 / 0.4 = 2.5, before the cap
    xy = np.asarray(w.xy)
    assert xy.min() >= 0.0 and xy.max() <= 500.0
    assert xy[:, 0].max() > 450.0 and xy[:, 1].max() > 450.0  # the whole box is used
    assert nl.r_per_um == pytest.approx(0.1) and nl.c_per_um == pytest.approx(0.2)
    sinks = np.asarray(nl.net_pins)[np.setdiff1d(np.arange(len(nl.net_pins)),
                                                 np.asarray(nl.net_ptr)[:-1])]
    caps = np.asarray(nl.pin_cap)[sinks]
    assert caps.min() >= 0.5 and caps.max() <= 3.0
    _check_library(w.library, 16 + 1)  # 16 combinational types and the flop


def test_superblue_like_recipe_small_scale():
    scale = 0.01
    w = netgen.superblue_like(3, scale=scale, depth=40)
    nl = w.netlist
    n_comb = int(round(613_000 * scale))
    assert nl.num_cells == n_comb + n_comb // 10
    levels = oracle.levels(nl)
    assert int(np.max(levels)) + 1 in (40, 41, 42)
    k = _sinks_per_net(nl)
    huge = int(round(20_000 * scale))
    # eight primary-input nets with 20k * scale sinks each, the rest power-law
    # (exponent 2.2, capped at 2,000): most nets drive one sink
    ptr, pins = np.asarray(nl.net_ptr), np.asarray(nl.net_pins)
    pi_net = np.isin(pins[ptr[:-1]], np.asarray(nl.start_pins))
    assert np.sum(pi_net & (k == huge)) == 8
    rest = k[~(pi_net & (k == huge))]
    assert rest.max() <= 2000 + 1
    assert np.mean(rest == 1) > 0.5
    xy = np.asarray(w.xy)
    assert xy.min() >= 0.0 and xy.max() <= 3000.0 and xy.max() > 2500.0
    _check_library(w.library, 64 + 1)


def test_jittered_placements_have_the_stated_spread():
    w = netgen.tiny_design(1)
    xy = np.asarray(w.xy, np.float64)
    xyb = netgen.jitter_positions(w.xy, 8, 5.0, 11)
    assert xyb.shape == (8,) + xy.shape and xyb.dtype == np.float32
    d = xyb.astype(np.float64) - xy[None]
    assert abs(d.mean()) < 0.2
    assert d.std() == pytest.approx(5.0, rel=0.05)
    assert not np.array_equal(xyb[0], xyb[1])
