"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle,
element by element, at the tolerances stated in tests/_parity.py."""
import numpy as np
import pytest

import netgen
import oracle
from tests import _parity as tp
from tests import _tinydag as td

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _check(w_or_parts, gamma=10.0, weights=(1.0, 0.5), **kw):
    """Oracle vs CUDA path through the C ABI on the same seeded inputs."""
    if isinstance(w_or_parts, tuple):
        nl, xy, lib = w_or_parts
    else:
        nl, xy, lib = w_or_parts.netlist, w_or_parts.xy, w_or_parts.library
    ora = oracle.sta(nl, lib, xy, gamma, *weights)
    gpu = tp.run_gpu(nl, lib, xy, gamma, weights, **kw)
    return tp.assert_parity(gpu, ora), gpu, ora


SCHEDULES = ["dataflow", "levels"]


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_design(seed, schedule):
    _check(netgen.tiny_design(seed), schedule=schedule)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("seed", range(6))
def test_tiny_dags_slew_independent_library(seed, schedule):
    w = td.tiny_netlist(seed)
    lib, _, _ = td.linear_library(5, [1, 2, 3, 4, 1], seed=seed)
    _check((w.netlist, w.xy, lib), gamma=3.0, schedule=schedule)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("idx", range(3))
def test_edge_netlists(idx, schedule):
    name, nl, xy, lib = tp.edge_netlists()[idx]
    errs, gpu, ora = _check((nl, xy, lib), schedule=schedule)
    if name == "no_endpoints":
        assert gpu["summary"]["tns_late"] == 0.0 and np.isinf(gpu["summary"]["wns_late"])
        assert np.all(gpu["grad"] == 0.0)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("gamma", [1.0, 50.0])
def test_mid_size_many_tiles(gamma, schedule):
    # ~50k pins over 40 levels: thousands of warp tasks, large-net tasks for the
    # power-law nets above 32 pins and the 400-sink primary-input nets
    _check(netgen.superblue_like(3, scale=0.02, depth=40), gamma=gamma, weights=(0.8, 0.2),
           schedule=schedule)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_full_size_superblue_like(schedule):
    # the benchmark's workload and launch configuration (CUDA graphs), all outputs
    w = netgen.superblue_like(1)
    errs, gpu, ora = _check(w, schedule=schedule)
    assert gpu["summary"]["num_endpoints"] == w.netlist.end_pins.shape[0]


def test_deterministic_graphs_and_host_input():
    w = netgen.superblue_like(4, scale=0.01, depth=30)
    a = tp.run_gpu(w.netlist, w.library, w.xy)
    b = tp.run_gpu(w.netlist, w.library, w.xy)
    c = tp.run_gpu(w.netlist, w.library, w.xy, use_graphs=False)
    d = tp.run_gpu(w.netlist, w.library, w.xy, host_xy=True)
    for k in ("at", "slew", "rat", "ats", "slack", "ep_slack", "grad"):
        for other in (b, c, d):
            assert np.array_equal(a[k], other[k], equal_nan=True), k
    assert a["summary"] == b["summary"] == c["summary"] == d["summary"]


def test_required_times_queried_before_gradient():
    # required times queried right after the forward run on their own; the
    # gradient sweep then runs alone; both equal the fused sweep's results
    import torch

    import paper_2603_28381_gb300 as sta
    w = netgen.superblue_like(6, scale=0.01, depth=30)
    fused = tp.run_gpu(w.netlist, w.library, w.xy)
    eng = sta.StaEngine(w.netlist, w.library)
    eng.set_positions(torch.as_tensor(w.xy).cuda())
    eng.forward(gamma=10.0)
    early = eng.pins()
    g = eng.backward_grad((1.0, 0.5)).cpu().numpy()
    late = eng.pins()
    eng.close()
    for k in ("at", "slew", "rat", "ats", "slack"):
        assert np.array_equal(early[k], fused[k], equal_nan=True), k
        assert np.array_equal(late[k], fused[k], equal_nan=True), k
    assert np.array_equal(g, fused["grad"])


def test_schedules_agree():
    # arrival / slew / LSE / required times bit-identical across schedules;
    # gradients agree to rounding (large-net sums are reassociated)
    w = netgen.superblue_like(5, scale=0.01, depth=30)
    a = tp.run_gpu(w.netlist, w.library, w.xy, schedule="dataflow")
    b = tp.run_gpu(w.netlist, w.library, w.xy, schedule="levels")
    for k in ("at", "slew", "rat", "ats", "slack", "ep_slack"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    gmax = np.abs(b["grad"]).max()
    assert np.abs(a["grad"] - b["grad"]).max() <= 1e-5 * gmax


def test_repeated_calls_follow_new_positions():
    import paper_2603_28381_gb300 as sta
    w = netgen.tiny_design(2)
    eng = sta.StaEngine(w.netlist, w.library)
    rng = np.random.default_rng(0)
    for it in range(3):
        xy = (w.xy + rng.normal(0, 20, w.xy.shape)).astype(np.float32)
        gpu = tp.run_gpu(w.netlist, w.library, xy, engine=eng)
        tp.assert_parity(gpu, oracle.sta(w.netlist, w.library, xy, 10.0, 1.0, 0.5))
    eng.close()


def test_gradient_against_finite_differences():
    # FP64 central differences (h = 1e-3 um) on 200 random pins; entries whose
    # perturbation changes a table segment, slew argmax or sign are excluded
    w = netgen.tiny_design(0)
    gamma, wts = 10.0, (1.0, 0.5)
    gpu = tp.run_gpu(w.netlist, w.library, w.xy, gamma, wts)
    pins = np.random.default_rng(2).choice(w.netlist.num_pins, 200, replace=False)
    fd, ok = oracle.finite_difference(w.netlist, w.library, w.xy, pins, gamma, *wts)
    assert ok.mean() > 0.8
    scale = max(np.abs(fd[ok]).max(), 1e-20)
    err = np.abs(gpu["grad"][pins] - fd)[ok]
    assert err.max() <= tp.GRAD_RTOL * scale, (err.max(), scale)


def test_autograd_function_matches_engine():
    import torch

    import paper_2603_28381_gb300 as sta
    w = netgen.tiny_design(1)
    eng = sta.StaEngine(w.netlist, w.library)
    xy = torch.tensor(w.xy, device="cuda", requires_grad=True)
    tns_g, wns_g = sta.timing_loss(xy, eng, 10.0)
    loss = 2.0 * tns_g - 0.5 * wns_g
    loss.backward()
    ora = oracle.sta(w.netlist, w.library, w.xy, 10.0, 2.0, -0.5)
    assert abs(tns_g.item() - ora["summary"]["tns_gamma"]) <= 1e-4 * abs(ora["summary"]["tns_gamma"])
    g = xy.grad.cpu().numpy()
    assert np.abs(g - ora["grad"]).max() <= tp.GRAD_RTOL * np.abs(ora["grad"]).max()
    eng.close()


def test_call_order_and_argument_errors():
    import torch

    import paper_2603_28381_gb300 as sta
    w = netgen.tiny_design(0)
    eng = sta.StaEngine(w.netlist, w.library)
    with pytest.raises(sta.StaError) as e:
        eng.forward()
    assert e.value.status == 6  # STA_ERR_STATE: positions first
    eng.set_positions(w.xy)
    with pytest.raises(sta.StaError) as e:
        eng.backward_grad()
    assert e.value.status == 6  # gradient before an LSE forward
    with pytest.raises(sta.StaError) as e:
        eng.forward(gamma=0.0)
    assert e.value.status == 1
    eng.forward(gamma=10.0, lse=False, rat=False)
    with pytest.raises(sta.StaError) as e:
        eng.backward_grad()
    assert e.value.status == 6
    with pytest.raises(sta.StaError) as e:
        eng.pins(at=False, slew=False, rat=True, ats=False, slack=False)
    assert e.value.status == 6  # required times were not propagated
    torch.cuda.synchronize()
    eng.close()


def test_misaligned_device_pointers_refused_before_device_work():
    # the entry points whose kernels read or write caller device pointers as
    # float2 refuse pointers off their alignment on the host (INVALID_ARG);
    # the handle then runs a normal step
    import torch

    import paper_2603_28381_gb300 as sta
    w = netgen.tiny_design(0)
    P = w.netlist.num_pins
    eng = sta.StaEngine(w.netlist, w.library)
    stream = torch.cuda.current_stream().cuda_stream
    big = torch.zeros(2 * P + 2, dtype=torch.float32, device="cuda")
    odd = big[1:]  # 4 bytes past an 8-byte boundary
    with pytest.raises(sta.StaError) as e:
        sta._sta.sta_set_positions(eng.h, odd.data_ptr(), 1, stream)
    assert e.value.status == 1 and "aligned" in sta.sta_last_error()
    eng.set_positions(torch.as_tensor(w.xy).cuda())
    eng.forward(gamma=10.0)
    wts = torch.ones(2, dtype=torch.float32, device="cuda")
    with pytest.raises(sta.StaError) as e:
        sta._sta.sta_backward_grad(eng.h, wts.data_ptr(), 1, odd.data_ptr(), 1, stream)
    assert e.value.status == 1
    with pytest.raises(sta.StaError) as e:
        sta._sta.sta_query_pins(eng.h, None, None, None, None, odd.data_ptr(), 1, stream)
    assert e.value.status == 1
    res = tp.run_gpu(w.netlist, w.library, w.xy, engine=eng)
    ref = tp.run_gpu(w.netlist, w.library, w.xy)
    for k in ("at", "slew", "rat", "ats", "slack", "ep_slack", "grad"):
        assert np.array_equal(res[k], ref[k], equal_nan=True), k
    eng.close()


def test_query_slack_matches_the_other_queries():
    import torch
    import paper_2603_28381_gb300 as sta
    w = netgen.tiny_design(1)
    eng = sta.StaEngine(w.netlist, w.library)
    eng.set_positions(torch.as_tensor(w.xy.astype(np.float32)).cuda())
    eng.forward(gamma=10.0)
    wt, ps, es = eng.slack()
    summ = eng.summary()
    for k in ("wns_early", "tns_early", "wns_late", "tns_late"):
        assert wt[k] == np.float32(summ[k])
    assert np.array_equal(ps, eng.pins(at=False, slew=False, rat=False, ats=False)["slack"])
    assert np.array_equal(es, eng.endpoints())
    eng.close()


def test_latency_probe_l2_and_dram():
    import paper_2603_28381_gb300 as sta
    l2 = sta.sta_measure_latency(16 << 20, 4000)
    dram = sta.sta_measure_latency(512 << 20, 2000)
    assert 50.0 < l2 < 5000.0
    assert dram > 0.8 * l2
