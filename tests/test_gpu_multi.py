"""Many netlists in one handle (sta_create_multi).

The union of several netlists is swept in one launch per sweep; the endpoint
reduction, the smoothed loss and its adjoint seeds stay per netlist.  Every
result of netlist k must be bit-identical to the same netlist in its own
handle (same positions, gamma and loss weights), and match the FP64 oracle at
the tolerances of tests/_parity.py.  The mix holds synthetic netlists of
different sizes and depths (one with a propagated clock) and the hand-wired
edge netlists (a single net, the ragged one with a 5000-sink net, one without
endpoints), all over one library.
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


def _mix():
    base = netgen.superblue_like(3, scale=0.01, depth=40)
    lib = base.library  # types 0-3 have 1-4 arcs, as the edge netlists expect
    edge = {name: (nl, xy) for name, nl, xy, _ in tp.edge_netlists()}
    parts = [(base.netlist, base.xy),
             edge["single_net"],
             (lambda w: (w.netlist, w.xy))(netgen.superblue_like(4, scale=0.004, depth=30, clock_nets=2)),
             edge["ragged"],
             edge["no_endpoints"],
             (lambda w: (w.netlist, w.xy))(netgen.superblue_like(5, scale=0.002, depth=20))]
    nls = [p[0] for p in parts]
    xys = [np.asarray(p[1], np.float32) for p in parts]
    rng = np.random.default_rng(41)
    W = rng.uniform(0.2, 1.5, size=(len(nls), 2)).astype(np.float32)
    return nls, xys, lib, W


def _run_multi(nls, xys, lib, W, gamma, host=False):
    import torch

    import paper_2603_28381_gb300 as sta
    eng = sta.StaEngine.multi(nls, lib)
    xy = np.concatenate(xys).astype(np.float32)
    eng.set_positions(xy if host else torch.as_tensor(xy).cuda())
    eng.forward(gamma=gamma, lse=True, rat=True)
    g = eng.backward_grad(W if host else torch.as_tensor(W).cuda())
    torch.cuda.synchronize()
    pins = eng.pins()
    ep = eng.endpoints()
    summ = eng.summary()
    g = g.cpu().numpy()
    out = []
    for k in range(len(nls)):
        p0, p1 = eng.pin_offsets[k], eng.pin_offsets[k + 1]
        e0, e1 = eng.end_offsets[k], eng.end_offsets[k + 1]
        r = {key: v[p0:p1] for key, v in pins.items()}
        r["ep_slack"] = ep[e0:e1]
        r["summary"] = summ[k]
        r["grad"] = g[p0:p1]
        out.append(r)
    eng.close()
    return out


def _same(a, b, k):
    for key in ("at", "slew", "rat", "ats", "slack", "ep_slack", "grad"):
        assert np.array_equal(a[key], b[key], equal_nan=True), (k, key)
    assert a["summary"] == b["summary"], k


def test_multi_equals_each_netlist_alone_bitwise_and_oracle():
    gamma = 10.0
    nls, xys, lib, W = _mix()
    res = _run_multi(nls, xys, lib, W, gamma)
    assert res[1]["summary"]["num_endpoints"] == nls[1].end_pins.shape[0]
    assert res[4]["summary"]["num_endpoints"] == 0
    for k, (nl, xy) in enumerate(zip(nls, xys)):
        alone = tp.run_gpu(nl, lib, xy, gamma, (float(W[k, 0]), float(W[k, 1])))
        _same(res[k], alone, k)
    for k in (0, 2, 3):  # the largest, the clocked and the ragged netlist against the oracle
        ora = oracle.sta(nls[k], lib, xys[k], gamma, float(W[k, 0]), float(W[k, 1]))
        tp.assert_parity(res[k], ora)


def test_multi_host_inputs_and_repeats():
    # host positions and weights; a second step with other positions and
    # weights gives the same results as a fresh handle
    gamma = 10.0
    nls, xys, lib, W = _mix()
    nls, xys, W = nls[:4], xys[:4], W[:4]
    first = _run_multi(nls, xys, lib, W, gamma, host=True)
    import torch

    import paper_2603_28381_gb300 as sta
    eng = sta.StaEngine.multi(nls, lib)
    rng = np.random.default_rng(5)
    xys2 = [x + rng.normal(0.0, 3.0, x.shape).astype(np.float32) for x in xys]
    W2 = W[::-1].copy()
    for xs, ws in ((xys, W), (xys2, W2)):
        eng.set_positions(np.concatenate(xs))
        eng.forward(gamma=gamma)
        g = eng.backward_grad(ws).cpu().numpy()
    summ = eng.summary()
    eng.close()
    again = _run_multi(nls, xys2, lib, W2, gamma)
    for k in range(len(nls)):
        p0, p1 = int(sum(x.shape[0] for x in xys2[:k])), int(sum(x.shape[0] for x in xys2[:k + 1]))
        assert np.array_equal(g[p0:p1], again[k]["grad"]), k
        assert summ[k] == again[k]["summary"], k
    assert any(first[k]["summary"] != again[k]["summary"] for k in range(len(nls)))
    torch.cuda.synchronize()
