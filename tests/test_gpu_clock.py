"""Propagated clock through the C ABI: flop clock pins hang on clock nets and
each flop D endpoint names the clock pin that captures it (hold bound + late
rising clock arrival, setup bound + early rising arrival).  Every schedule is
compared with the FP64 oracle element by element, gradients included (the
setup term's adjoint reaches the clock wires)."""
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


@pytest.mark.parametrize("use_graphs", [True, False])
@pytest.mark.parametrize("schedule", ["dataflow", "levels"])
def test_tiny_clocked_design(schedule, use_graphs):
    w = netgen.tiny_design(0, clock_nets=2)
    ora = oracle.sta(w.netlist, w.library, w.xy, 10.0, 1.0, 0.5)
    gpu = tp.run_gpu(w.netlist, w.library, w.xy, 10.0, (1.0, 0.5), use_graphs=use_graphs, schedule=schedule)
    tp.assert_parity(gpu, ora)
    ck = w.info["ck_pins"]
    assert np.abs(ora["grad"][ck]).max() > 0  # the clock wires carry gradient


@pytest.mark.parametrize("schedule", ["dataflow", "levels"])
def test_mid_size_clocked_design(schedule):
    # ~60k pins, power-law fanout, 8 clock nets of ~190 flop clock pins each
    w = netgen.superblue_like(4, scale=0.02, depth=40, clock_nets=8)
    ora = oracle.sta(w.netlist, w.library, w.xy, 20.0, 1.0, 0.5)
    gpu = tp.run_gpu(w.netlist, w.library, w.xy, 20.0, (1.0, 0.5), schedule=schedule)
    tp.assert_parity(gpu, ora)


@pytest.mark.parametrize("sweep", ["levels", "dataflow"])
def test_clocked_batches(sweep):
    w = netgen.tiny_design(1, clock_nets=2)
    B = 5
    xyb = netgen.jitter_positions(w.xy, B, 5.0, 9)
    rng = np.random.default_rng(2)
    W = np.stack([rng.uniform(0.5, 1.5, B), rng.uniform(0.0, 1.0, B)], 1).astype(np.float32)
    res = tp.run_gpu_batch(w.netlist, w.library, xyb, 10.0, W, sweep=sweep)
    for b in range(B):
        ora = oracle.sta(w.netlist, w.library, xyb[b], 10.0, float(W[b, 0]), float(W[b, 1]))
        tp.assert_parity(res[b], ora)


def test_zero_length_clock_wires_match_ideal_clock_handle():
    """Both handles on the GPU: a propagated clock whose wires have length zero
    gives the ideal-clock results with the capture edges folded into the bounds."""
    wc = netgen.tiny_design(0, clock_nets=2)
    wi = netgen.tiny_design(0)
    nc, ni = wc.netlist, wi.netlist
    P0 = ni.num_pins
    xy = wc.xy.copy()
    for n in range(ni.num_nets, nc.num_nets):
        pins = nc.net_pins[nc.net_ptr[n]:nc.net_ptr[n + 1]]
        xy[pins[1:]] = xy[pins[0]]
    clock_at = nc.start_at[-1]
    ideal = netgen.Netlist(**{f.name: getattr(ni, f.name) for f in netgen.dataclasses.fields(ni)})
    ideal.start_at = ni.start_at.copy()
    ideal.start_at[np.isin(ni.start_pins, wc.info["ck_pins"])] = clock_at
    ideal.end_rat = ni.end_rat.copy()
    ideal.end_rat[nc.end_clock >= 0] += np.array([clock_at[2], clock_at[2], clock_at[0], clock_at[0]], np.float32)
    gc = tp.run_gpu(nc, wc.library, xy, 10.0, (1.0, 0.5))
    gi = tp.run_gpu(ideal, wi.library, xy[:P0], 10.0, (1.0, 0.5))
    for k in ("at", "slew", "rat", "ats", "slack"):
        np.testing.assert_array_equal(gc[k][:P0], gi[k], err_msg=k)
    np.testing.assert_array_equal(gc["ep_slack"], gi["ep_slack"])
    gmax = float(np.abs(gi["grad"]).max())
    assert np.abs(gc["grad"][:P0] - gi["grad"]).max() <= 1e-5 * gmax


def test_served_clocked_netlists_match_oracle():
    import torch
    from paper_2603_28381_gb300.serving import StaServer
    designs = [netgen.tiny_design(2, clock_nets=3), netgen.superblue_like(5, scale=0.01, depth=30, clock_nets=4)]
    srv = StaServer(slots=2)
    ids = [srv.add_netlist(w.netlist, w.library) for w in designs]
    pending = {}
    for i, w in enumerate(designs):
        xy = torch.from_numpy(netgen.jitter_positions(w.xy, 1, 3.0, 50 + i)[0]).pin_memory()
        g = torch.zeros(xy.shape, dtype=torch.float32).pin_memory()
        rid = srv.submit(ids[i], xy, gradient=True, gamma=10.0, w=(1.0, 0.5), grad_out=g)
        pending[rid] = (w, xy, g)
    done = {}
    while len(done) < len(pending):
        for c in srv.poll(wait_ms=200):
            done[c["id"]] = c
    srv.close()
    for rid, (w, xy, g) in pending.items():
        assert done[rid]["status"] == 0
        ora = oracle.sta(w.netlist, w.library, xy.numpy(), 10.0, 1.0, 0.5)
        gmax = np.abs(ora["grad"]).max()
        assert np.abs(g.numpy() - ora["grad"]).max() <= tp.GRAD_RTOL * gmax
        s = done[rid]["summary"].tolist()
        scale = float(np.abs(ora["at"][:, 2:][np.isfinite(ora["at"][:, 2:])]).max())
        assert abs(s[2] - ora["summary"]["wns_late"]) <= tp.AT_RTOL * scale
        assert abs(s[3] - ora["summary"]["tns_late"]) <= tp.AT_RTOL * max(abs(ora["summary"]["tns_late"]), scale)
