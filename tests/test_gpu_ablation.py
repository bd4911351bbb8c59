"""Ablations: net RC in the CTE scheme of Algorithm 2 against the pin-based
warp tasks and the oracle; sequential against fused gradient sweeps."""
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


def _cases():
    out = [("tiny", netgen.tiny_design(0)), ("mid", netgen.superblue_like(3, scale=0.02, depth=40))]
    name, nl, xy, lib = tp.edge_netlists()[1]  # 33-pin and 5000-sink nets, a dangling output
    out.append((name, netgen.Workload(netlist=nl, library=lib, xy=xy, info={})))
    return out


@pytest.mark.parametrize("case", range(3))
def test_cte_net_rc_matches_pin_based_and_oracle(case):
    import torch
    import paper_2603_28381_gb300 as sta
    name, w = _cases()[case]
    ora = oracle.sta(w.netlist, w.library, w.xy, 10.0, 1.0, 0.0)
    eng = sta.StaEngine(w.netlist, w.library)
    eng.set_positions(torch.as_tensor(w.xy.astype(np.float32)).cuda())
    res = {}
    for scheme in ("pin", "cte"):
        ms = eng.ablation_net_rc(scheme, reps=2)
        assert ms > 0
        res[scheme] = eng.net_rc()
    for k, ok in (("load", "net_load"), ("wdelay", "wdelay"), ("impulse", "impulse")):
        ref = ora[ok]
        tol = tp.AT_RTOL * max(float(np.abs(ref).max()), 1.0)
        for scheme in ("pin", "cte"):
            assert np.abs(res[scheme][k] - ref).max() <= tol, (name, scheme, k)
    # the per-sink terms are computed by the same arithmetic in both schemes
    assert np.array_equal(res["pin"]["wdelay"], res["cte"]["wdelay"])
    assert np.array_equal(res["pin"]["impulse"], res["cte"]["impulse"])
    # the analysis still runs normally afterwards
    gpu = tp.run_gpu(w.netlist, w.library, w.xy, 10.0, (1.0, 0.0), engine=eng)
    tp.assert_parity(gpu, ora)
    eng.close()


def test_sequential_and_fused_gradients_agree():
    import torch
    import paper_2603_28381_gb300 as sta
    from paper_2603_28381_gb300 import _sta
    w = netgen.superblue_like(3, scale=0.02, depth=40)
    eng = sta.StaEngine(w.netlist, w.library)
    xy = torch.as_tensor(w.xy.astype(np.float32)).cuda()
    wts = (1.0, 0.5)
    out = {}
    for mode, flags in (("sequential", _sta.STA_FWD_LSE | _sta.STA_FWD_RAT | _sta.STA_FWD_RAT_EAGER),
                        ("fused", _sta.STA_FWD_LSE | _sta.STA_FWD_RAT)):
        eng.set_positions(xy)
        _sta.sta_forward(eng.h, flags, 10.0, sta._stream_ptr(None))
        g = eng.backward_grad(wts)
        torch.cuda.synchronize()
        out[mode] = (g.cpu().numpy(), eng.pins(at=False, slew=False, ats=False, slack=False)["rat"])
        _, launches = eng.profile(with_times=False)
        assert launches["required"] == (1 if mode == "sequential" else 0)
        # the forward's prologue and endpoint launches also reset its own polled words
        # and those of the fused sweep after it; separate required-time and adjoint
        # sweeps reset theirs in launches of their own
        assert launches["reset"] == (2 if mode == "sequential" else 0)
    assert np.array_equal(out["sequential"][1], out["fused"][1])
    gmax = np.abs(out["fused"][0]).max()
    assert np.abs(out["sequential"][0] - out["fused"][0]).max() <= 1e-5 * gmax
    eng.close()
