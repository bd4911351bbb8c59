"""The allocation-free endpoint summary (sta_endpoint_summary_noalloc).

It exists for callers that cannot call cudaMalloc: code running while a stream
is captured into a CUDA graph, where allocation cannot be captured, and
processes whose device memory belongs to another framework's pool allocator.
These tests call it through the C ABI on device arrays and check its slacks and
summary, twice in a row, against the endpoint reduction that sta_forward
performs (the existing entry point) and against the FP64 oracle, within the
tolerances of tests/_parity.py, on an ideal-clock and a propagated-clock
design.  This file is collected last so that a failure here leaves every other
test run.
"""
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


def _reference(w, gamma):
    import torch

    import paper_2603_28381_gb300 as sta
    eng = sta.StaEngine(w.netlist, w.library)
    eng.set_positions(torch.as_tensor(w.xy).cuda())
    eng.forward(gamma=gamma, lse=True, rat=True)
    P = w.netlist.num_pins
    at = torch.empty(P, 4, dtype=torch.float32, device="cuda")
    ats = torch.empty(P, 2, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    sta._sta.sta_query_pins(eng.h, at.data_ptr(), None, None, ats.data_ptr(), None, 1, stream)
    summary = eng.summary()
    slack = eng.endpoints()
    torch.cuda.synchronize()
    eng.close()
    return at, ats, summary, slack


@pytest.mark.parametrize("make", [lambda: netgen.tiny_design(0),
                                  lambda: netgen.tiny_design(1, clock_nets=2),
                                  lambda: netgen.superblue_like(3, scale=0.02, depth=40)],
                         ids=["tiny", "tiny_clocked", "sb_50k"])
def test_noalloc_matches_forward_reduction_and_oracle_twice(make):
    import torch

    import paper_2603_28381_gb300 as sta
    gamma = 10.0
    w = make()
    nl = w.netlist
    at, ats, ref_sum, ref_slack = _reference(w, gamma)
    orc = oracle.sta(nl, w.library, w.xy, gamma, 1.0, 0.0)
    E, P = nl.end_pins.shape[0], nl.num_pins
    end_pins = torch.as_tensor(nl.end_pins.astype(np.int32)).cuda()
    end_rat = torch.as_tensor(nl.end_rat.astype(np.float32)).cuda()
    end_clk = (torch.as_tensor(nl.end_clock.astype(np.int32)).cuda() if nl.end_clock is not None else None)
    scale = float(np.abs(orc["at"][:, 2:]).max())
    tol = tp.AT_RTOL * scale
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        slack = torch.full((E, 2), float("nan"), dtype=torch.float32, device="cuda")
        summ = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        sta._sta.sta_endpoint_summary_noalloc(at.data_ptr(), ats.data_ptr(), P, end_pins.data_ptr(),
                                              end_rat.data_ptr(), 0 if end_clk is None else end_clk.data_ptr(),
                                              E, gamma, slack.data_ptr(), summ.data_ptr(), stream)
        torch.cuda.synchronize()
        got = slack.cpu().numpy()
        s = dict(zip(sta.SUMMARY_KEYS, summ.cpu().numpy().tolist()))
        for name, ref, rs in (("forward", ref_slack, ref_sum), ("oracle", orc["ep_slack"], orc["summary"])):
            assert np.abs(got - ref).max() <= tol, f"call {call}: endpoint slacks differ from the {name}"
            for k in ("wns_early", "wns_late", "wns_gamma"):
                assert abs(s[k] - rs[k]) <= tol, (call, name, k, s[k], rs[k])
            for k in ("tns_early", "tns_late", "tns_gamma"):
                assert abs(s[k] - rs[k]) <= tp.AT_RTOL * max(abs(rs[k]), scale), (call, name, k)
            assert s["late_violations"] == rs["late_violations"], (call, name)
        assert s["num_endpoints"] == E


def test_noalloc_rejects_too_many_endpoints():
    import paper_2603_28381_gb300 as sta
    too_many = (1 << 22) + 1
    with pytest.raises(sta.StaError) as e:
        sta._sta.sta_endpoint_summary_noalloc(16, None, 1, 16, 16, None, too_many, 10.0, 16, 16, 0)
    assert e.value.status == 1  # STA_ERR_INVALID_ARG, before any device work
    assert "STA_NOALLOC_MAX_ENDPOINTS" in sta.sta_last_error()
