"""Batched schedule: many placements of one netlist per call (lane per
placement).  Every placement is compared with the FP64 oracle at the parity
tolerances, and a placement's results must be bit-identical alone and in a
batch (the per-placement arithmetic does not depend on the batch)."""
import numpy as np
import pytest

import netgen
import oracle
from tests import _parity as tp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _placements(w, B, sigma=5.0, seed=7):
    return netgen.jitter_positions(w.xy, B, sigma, seed)


def _weights(B, seed=3):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0.5, 1.5, B), rng.uniform(0.0, 1.0, B)], 1).astype(np.float32)


def _check_all(nl, lib, xyb, W, gamma, res, which=None):
    for b in (range(len(res)) if which is None else which):
        ora = oracle.sta(nl, lib, xyb[b], gamma, float(W[b, 0]), float(W[b, 1]))
        tp.assert_parity(res[b], ora)


SWEEPS = ["levels", "dataflow", "wide"]


@pytest.mark.parametrize("sweep", SWEEPS)
@pytest.mark.parametrize("B", [1, 5, 33])
def test_tiny_design_batches(B, sweep):
    w = netgen.tiny_design(0)
    xyb, W = _placements(w, B), _weights(B)
    res = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, sweep=sweep)
    _check_all(w.netlist, w.library, xyb, W, 10.0, res)


@pytest.mark.parametrize("sweep", SWEEPS)
@pytest.mark.parametrize("tile_pins,chunk", [(1, 1), (16, 8), (4, 64), (64, 200)])
def test_task_shapes_mid_size(tile_pins, chunk, sweep):
    # power-law fanout and 400-sink primary-input nets: packed nets, single nets
    # and chunked large nets, two placement groups with a ragged second group
    w = netgen.superblue_like(3, scale=0.02, depth=40)
    B = 40
    xyb, W = _placements(w, B), _weights(B)
    res = tp.run_gpu_batch(w.netlist, w.library, xyb, 20.0, W, tile_pins=tile_pins, chunk=chunk, sweep=sweep)
    _check_all(w.netlist, w.library, xyb, W, 20.0, res, which=[0, 17, 31, 32, 39])


@pytest.mark.parametrize("sweep", SWEEPS)
@pytest.mark.parametrize("idx", range(3))
def test_edge_netlists_batched(idx, sweep):
    name, nl, xy, lib = tp.edge_netlists()[idx]
    B = 3
    xyb = netgen.jitter_positions(xy, B, 2.0, 5)
    W = _weights(B)
    res = tp.run_gpu_batch(nl, lib, xyb, 10.0, W, sweep=sweep)
    _check_all(nl, lib, xyb, W, 10.0, res)


def test_alone_equals_in_batch_bitwise():
    w = netgen.superblue_like(5, scale=0.01, depth=30)
    B = 37
    xyb, W = _placements(w, B, seed=11), _weights(B, seed=12)
    full = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W)
    for b in (0, 21, 36):
        alone = tp.run_gpu_batch(w.netlist, w.library, xyb[b:b + 1], 10.0, W[b:b + 1])[0]
        for k in ("at", "slew", "rat", "ats", "slack", "ep_slack", "grad"):
            assert np.array_equal(alone[k], full[b][k]), (b, k)
        assert alone["summary"] == full[b]["summary"]


def test_sweeps_bit_identical():
    w = netgen.superblue_like(8, scale=0.01, depth=30)
    B = 12
    xyb, W = _placements(w, B), _weights(B)
    a = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, sweep="levels", chunk=8)
    b = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, sweep="dataflow", chunk=8)
    for r, s in zip(a, b):
        for k in ("at", "slew", "rat", "ats", "slack", "ep_slack", "grad"):
            assert np.array_equal(r[k], s[k]), k
        assert r["summary"] == s["summary"]


def test_host_buffers_graphs_and_repeats():
    import torch
    import paper_2603_28381_gb300 as sta
    w = netgen.superblue_like(6, scale=0.01, depth=30)
    B = 8
    xyb, W = _placements(w, B), _weights(B)
    a = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W)
    b = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, host_xy=True, use_graphs=False)
    for r, s in zip(a, b):
        for k in ("at", "rat", "grad"):
            assert np.array_equal(r[k], s[k])
    # one engine, repeated steps with different positions, host gradient output
    eng = sta.StaEngine(w.netlist, w.library, schedule="batch", num_placements=B)
    for rep in range(3):
        xr = _placements(w, B, seed=100 + rep)
        eng.set_positions(torch.as_tensor(xr).cuda())
        eng.forward(gamma=10.0)
        g = eng.backward_grad(W, out=torch.empty(B, w.netlist.num_pins, 2))
        ora = oracle.sta(w.netlist, w.library, xr[rep], 10.0, float(W[rep, 0]), float(W[rep, 1]))
        gmax = np.abs(ora["grad"]).max()
        assert np.abs(g[rep].numpy() - ora["grad"]).max() <= tp.GRAD_RTOL * gmax
    eng.close()


@pytest.mark.parametrize("sweep", SWEEPS)
def test_batched_full_size_500k_64_placements(sweep):
    # the batched workload: ~500k pins, depth 100, 64 placements with 5 um jitter;
    # sampled placements against the oracle
    w = netgen.superblue_like(2, scale=0.2, depth=100)
    B = 64
    xyb, W = _placements(w, B), _weights(B)
    res = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, sweep=sweep)
    _check_all(w.netlist, w.library, xyb, W, 10.0, res, which=[0, 63])


def test_batched_wait_expiry_reported():
    import paper_2603_28381_gb300 as sta
    w = netgen.tiny_design(2)
    B = 4
    xyb, W = _placements(w, B), _weights(B)
    import torch
    eng = sta.StaEngine(w.netlist, w.library, schedule="batch", num_placements=B, batch_sweep="dataflow")
    eng.set_positions(torch.as_tensor(xyb).cuda())
    eng._debug_expire_wait()
    eng.forward(gamma=10.0)
    with pytest.raises(sta.StaError) as ei:
        eng.summary()
    assert ei.value.status == 5
    res = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, engine=eng)
    _check_all(w.netlist, w.library, xyb, W, 10.0, res, which=[0, 3])


def test_autotune_picks_a_candidate_and_stays_exact():
    import torch
    import paper_2603_28381_gb300 as sta
    w = netgen.superblue_like(9, scale=0.01, depth=30)
    B = 16
    xyb, W = _placements(w, B), _weights(B)
    eng = sta.StaEngine(w.netlist, w.library, schedule="batch", num_placements=B)
    eng.set_positions(torch.as_tensor(xyb).cuda())
    best, table = eng.autotune(tile_pins=(1, 4), chunks=(4, 32), sweeps=("levels", "dataflow"), reps=2)
    assert len(table) == 8 and all(np.isfinite(v) and v > 0 for v in table.values())
    assert best in table and table[best] == min(table.values())
    res = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, engine=eng)
    _check_all(w.netlist, w.library, xyb, W, 10.0, res, which=[0, 15])
    eng.close()


# ---------------------------------------------------------------------------
# lanes: the placements as independent lanes of the single-placement sweeps
# ---------------------------------------------------------------------------
def _same_as_single(nl, lib, xyb, W, gamma, res, which):
    for b in which:
        one = tp.run_gpu(nl, lib, xyb[b], gamma, (float(W[b, 0]), float(W[b, 1])))
        for k in ("at", "slew", "rat", "ats", "slack", "ep_slack", "grad"):
            assert np.array_equal(res[b][k], one[k], equal_nan=True), (b, k)
        assert res[b]["summary"] == one["summary"], b


@pytest.mark.parametrize("make,B", [(lambda: netgen.superblue_like(3, scale=0.02, depth=40), 5),
                                    (lambda: netgen.tiny_design(1, clock_nets=2), 3),
                                    (lambda: netgen.tiny_design(0), 33)],
                         ids=["sb_50k_x5", "tiny_clocked_x3", "tiny_x33"])
def test_lanes_equal_single_placements_bitwise(make, B):
    # each lane's every output is bit-identical to the same placement in a
    # single-placement handle; one lane is also checked against the oracle
    w = make()
    xyb, W = _placements(w, B, seed=21), _weights(B, seed=22)
    res = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, sweep="lanes")
    _same_as_single(w.netlist, w.library, xyb, W, 10.0, res, sorted({0, B // 2, B - 1}))
    _check_all(w.netlist, w.library, xyb, W, 10.0, res, which=[B - 1])


def test_lanes_host_buffers_repeats_and_edge_netlists():
    import torch
    import paper_2603_28381_gb300 as sta
    w = netgen.superblue_like(6, scale=0.01, depth=30)
    B = 4
    xyb, W = _placements(w, B), _weights(B)
    a = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, sweep="lanes")
    b = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, sweep="lanes", host_xy=True, use_graphs=False)
    for r, s in zip(a, b):
        for k in ("at", "rat", "grad", "ep_slack"):
            assert np.array_equal(r[k], s[k])
        assert r["summary"] == s["summary"]
    eng = sta.StaEngine(w.netlist, w.library, schedule="batch", num_placements=B, batch_sweep="lanes")
    for rep in range(2):
        xr = _placements(w, B, seed=200 + rep)
        got = tp.run_gpu_batch(w.netlist, w.library, xr, 10.0, W, engine=eng)
        _same_as_single(w.netlist, w.library, xr, W, 10.0, got, [rep, B - 1])
    eng.close()
    # fewer lanes than the handle holds (sta_set_active), then all again
    eng = sta.StaEngine(w.netlist, w.library, schedule="batch", num_placements=B, batch_sweep="lanes")
    for k in (2, 1, B):
        eng.set_active(k)
        xr = _placements(w, k, seed=300 + k)
        got = tp.run_gpu_batch(w.netlist, w.library, xr, 10.0, W[:k], engine=eng)
        assert len(got) == k
        _same_as_single(w.netlist, w.library, xr, W[:k], 10.0, got, sorted({0, k - 1}))
    eng.close()
    for idx in range(3):  # ragged and degenerate netlists
        name, nl, xy, lib = tp.edge_netlists()[idx]
        xe = netgen.jitter_positions(xy, 2, 2.0, 5)
        We = _weights(2)
        res = tp.run_gpu_batch(nl, lib, xe, 10.0, We, sweep="lanes")
        _check_all(nl, lib, xe, We, 10.0, res)


def _edge(name):
    return next((nl, xy, lib) for n, nl, xy, lib in tp.edge_netlists() if n == name)


@pytest.mark.parametrize("case", ["sb_50k_x5", "tiny_clocked_x3", "ragged_x40", "sb_50k_chunk8_x70"])
def test_wide_sweep_equals_narrow_bitwise(case):
    # a lane per placement (all four conditions in one lane) gives every output
    # bit-identical to the 8-placement x 4-condition sweep: padding lanes of a
    # 32-placement group, several groups, a propagated clock, and the large
    # nets' partial / driver / gradient tasks (8-sink chunks)
    if case == "ragged_x40":
        nl, xy, lib = _edge("ragged")
        xyb = netgen.jitter_positions(np.asarray(xy, np.float32), 40, 5.0, 3)
        W, chunk = _weights(40, seed=9), 0
    else:
        w = {"sb_50k_x5": lambda: netgen.superblue_like(3, scale=0.02, depth=40),
             "tiny_clocked_x3": lambda: netgen.tiny_design(1, clock_nets=2),
             "sb_50k_chunk8_x70": lambda: netgen.superblue_like(4, scale=0.02, depth=40)}[case]()
        nl, lib = w.netlist, w.library
        B = {"sb_50k_x5": 5, "tiny_clocked_x3": 3, "sb_50k_chunk8_x70": 70}[case]
        xyb, W = _placements(w, B, seed=13), _weights(B, seed=14)
        chunk = 8 if case.endswith("chunk8_x70") else 0
    narrow = tp.run_gpu_batch(nl, lib, xyb, 10.0, W, sweep="dataflow", chunk=chunk)
    wide = tp.run_gpu_batch(nl, lib, xyb, 10.0, W, sweep="wide", chunk=chunk)
    for b in range(len(narrow)):
        for k in ("at", "slew", "rat", "ats", "slack", "ep_slack", "grad"):
            assert np.array_equal(wide[b][k], narrow[b][k], equal_nan=True), (case, b, k)
        assert wide[b]["summary"] == narrow[b]["summary"], (case, b)
    _check_all(nl, lib, xyb, W, 10.0, wide, which=[len(wide) - 1])


@pytest.mark.parametrize("sweep", ["dataflow", "wide"])
def test_repeated_forward_without_new_positions(sweep):
    # the sweeps' polled words are reset with the positions; a second forward on
    # the same positions (here with another gamma, so every LSE arrival changes)
    # resets them itself, and an autotuned handle resets inside each candidate:
    # every result equals the one-forward sequence bit for bit
    import torch
    import paper_2603_28381_gb300 as sta
    w = netgen.superblue_like(3, scale=0.02, depth=40)
    B = 12
    xyb, W = _placements(w, B), _weights(B)
    ref = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, sweep=sweep, tile_pins=1, chunk=16)
    eng = sta.StaEngine(w.netlist, w.library, schedule="batch", num_placements=B, tile_pins=1, chunk=16,
                        batch_sweep=sweep)
    eng.set_positions(torch.as_tensor(xyb).cuda())
    eng.forward(gamma=3.0, lse=True, rat=True)
    eng.backward_grad(torch.as_tensor(W).cuda())
    eng.forward(gamma=10.0, lse=True, rat=True)  # no new positions: resets on its own stream
    g2 = eng.backward_grad(torch.as_tensor(W).cuda()).cpu().numpy()
    pins, ep, summ = eng.pins(), eng.endpoints(), eng.summary()
    for b in range(B):
        for k in ("at", "slew", "rat", "ats", "slack"):
            assert np.array_equal(pins[k][b], ref[b][k], equal_nan=True), (b, k)
        assert np.array_equal(ep[b], ref[b]["ep_slack"], equal_nan=True), b
        assert summ[b] == ref[b]["summary"], b
        assert np.array_equal(g2[b], ref[b]["grad"]), b
    eng.forward(gamma=3.0, lse=True, rat=True)
    res = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, engine=eng)  # new positions: reset beside them
    for b in range(B):
        for k in ("at", "slew", "rat", "ats", "slack", "ep_slack", "grad"):
            assert np.array_equal(res[b][k], ref[b][k], equal_nan=True), (b, k)
        assert res[b]["summary"] == ref[b]["summary"], b
    eng.autotune(tile_pins=(1, 2), chunks=(16,), sweeps=(sweep,), reps=2)
    eng.forward(gamma=10.0, lse=True, rat=True)
    g3 = eng.backward_grad(torch.as_tensor(W).cuda()).cpu().numpy()
    eng.close()
    _check_all(w.netlist, w.library, xyb, W, 10.0,
               [dict(ref[b], grad=g3[b]) for b in range(B)], which=[0, 11])
