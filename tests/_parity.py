"""Running the CUDA path through the C ABI and comparing it with the oracle.

Tolerances (written here once, used by every parity test):
  * arrival/required times, slews, slacks, WNS: |gpu - oracle| <= 1e-4 * max |late AT|
  * TNS (hard and smoothed): <= 1e-4 * max(|TNS|, max |late AT|)
  * gradients: per component <= 1e-3 * max(max |oracle gradient|, 1e-20)
Infinite required times / slacks (pins with no path to an endpoint) must match
exactly.
"""
import numpy as np

import netgen

AT_RTOL = 1e-4
GRAD_RTOL = 1e-3


def edge_netlists():
    """Small hand-wired netlists that hit the ragged and degenerate cases."""
    out = []
    rng = np.random.default_rng(11)
    lib = netgen.make_library(np.random.default_rng(3), [1, 2, 3, 4])

    # 1: one primary input driving one output
    b = netgen.NetlistBuilder()
    pi, po = b.pin(0.0, 0, 0), b.pin(1.0, 30, 40)
    b.net(pi, [po])
    b.start(pi)
    b.end(po)
    out.append(("single_net",) + b.build() + (lib,))

    # 2: dangling cell output, coincident pins (d = 0), nets of 32 / 33 pins,
    #    eight 2-pin nets, a 5000-sink net driven by a cell, a free clock pin
    b = netgen.NetlistBuilder()
    pi = b.pin(0.0, 10, 10)
    ins = [b.pin(1.0, *rng.uniform(0, 300, 2)) for _ in range(4)]
    o4 = b.pin(0.0, 50, 50)
    b.cell(3, ins, o4)                                   # 4-input cell
    b.net(pi, ins[:2] + [b.pin(1.5, 10, 10)])            # includes a coincident sink
    ck = b.pin(0.0, 0, 0)
    q = b.pin(0.0, 5, 5)
    b.cell(0, [ck], q)                                   # flop-like: CK is a free startpoint
    b.start(ck)
    b.net(q, ins[2:])
    # o4 drives 31 sinks (32 pins): a full warp task
    s31 = []
    for _ in range(31):
        p = b.pin(float(rng.uniform(0.5, 3)), *rng.uniform(0, 300, 2))
        s31.append(p)
    b.net(o4, s31)
    # 31 single-input cells on those sinks; one dangling, one driving a 33-pin net
    outs = []
    for k, p in enumerate(s31):
        o = b.pin(0.0, *rng.uniform(0, 300, 2))
        b.cell(0, [p], o)
        outs.append(o)
    # outs[0]: dangling output (drives no net)
    s32 = [b.pin(1.0, *rng.uniform(0, 300, 2)) for _ in range(32)]
    b.net(outs[1], s32)                                  # 33 pins: a block task
    for p in s32:
        b.end(p)
    big = [b.pin(float(rng.uniform(0.5, 3)), *rng.uniform(0, 300, 2)) for _ in range(5000)]
    b.net(outs[2], big)
    for p in big[:4000]:
        b.end(p)
    more = []
    for p in big[4000:]:                                 # 1000 cells fed by the big net
        o = b.pin(0.0, *rng.uniform(0, 300, 2))
        b.cell(0, [p], o)
        more.append(o)
    for k in range(3, 31):                               # 28 two-pin nets
        e = b.pin(2.0, *rng.uniform(0, 300, 2))
        b.net(outs[k], [e])
        b.end(e)
    for o in more:
        e = b.pin(1.0, *rng.uniform(0, 300, 2))
        b.net(o, [e])
        b.end(e, rat=(5.0, 6.0, 900.0, 950.0))
    b.start(pi, at=(1.0, 2.0, 3.0, 4.0), slew=(15.0, 16.0, 25.0, 26.0))
    out.append(("ragged",) + b.build() + (lib,))

    # 3: no endpoints at all
    b = netgen.NetlistBuilder()
    pi, a, o, s = b.pin(0.0, 0, 0), b.pin(1.0, 5, 0), b.pin(0.0, 5, 0), b.pin(1.0, 9, 9)
    b.net(pi, [a])
    b.cell(0, [a], o)
    b.net(o, [s])
    b.start(pi)
    nl, xy = b.build()
    # s has no source other than the net, fine; no endpoint anywhere
    out.append(("no_endpoints", nl, xy, lib))
    return out


def run_gpu(nl, lib, xy, gamma=10.0, w=(1.0, 0.5), use_graphs=True, host_xy=False, engine=None,
            schedule="dataflow"):
    """One set_positions + forward(LSE, RAT) + backward through the C ABI."""
    import torch

    import paper_2603_28381_gb300 as sta
    eng = engine or sta.StaEngine(nl, lib, use_graphs=use_graphs, schedule=schedule)
    if host_xy:
        eng.set_positions(np.asarray(xy, np.float32))
    else:
        eng.set_positions(torch.as_tensor(np.asarray(xy, np.float32)).cuda())
    eng.forward(gamma=gamma, lse=True, rat=True)
    g = eng.backward_grad(w)
    torch.cuda.synchronize()
    res = eng.pins()
    res["ep_slack"] = eng.endpoints()
    res["summary"] = eng.summary()
    res["grad"] = g.cpu().numpy()
    if engine is None:
        eng.close()
    return res


def run_gpu_batch(nl, lib, xyb, gamma=10.0, w=(1.0, 0.5), use_graphs=True, host_xy=False, engine=None,
                  tile_pins=0, chunk=0, sweep="levels"):
    """The batched schedule on B placements xyb [B,P,2]: one set_positions +
    forward(LSE, RAT) + backward; a list of B per-placement result dicts."""
    import torch

    import paper_2603_28381_gb300 as sta
    xyb = np.ascontiguousarray(np.asarray(xyb, np.float32))
    B = xyb.shape[0]
    eng = engine or sta.StaEngine(nl, lib, use_graphs=use_graphs, schedule="batch", num_placements=B,
                                  tile_pins=tile_pins, chunk=chunk, batch_sweep=sweep)
    if host_xy:
        eng.set_positions(xyb)
    else:
        eng.set_positions(torch.as_tensor(xyb).cuda())
    eng.forward(gamma=gamma, lse=True, rat=True)
    wb = np.broadcast_to(np.asarray(w, np.float32), (B, 2)) if np.ndim(w) < 2 else np.asarray(w, np.float32)
    g = eng.backward_grad(torch.as_tensor(np.ascontiguousarray(wb)).cuda())
    torch.cuda.synchronize()
    pins = eng.pins()
    ep = eng.endpoints()
    summ = eng.summary()
    g = g.cpu().numpy()
    out = []
    for b in range(B):
        r = {k: v[b] for k, v in pins.items()}
        r["ep_slack"] = ep[b]
        r["summary"] = summ[b]
        r["grad"] = g[b]
        out.append(r)
    if engine is None:
        eng.close()
    return out


def _close(name, gpu, ora, tol):
    gpu = np.asarray(gpu, np.float64)
    ora = np.asarray(ora, np.float64)
    assert gpu.shape == ora.shape, (name, gpu.shape, ora.shape)
    inf_o = ~np.isfinite(ora)
    assert np.array_equal(inf_o, ~np.isfinite(gpu)), f"{name}: infinite entries differ"
    assert np.array_equal(ora[inf_o], gpu[inf_o]), f"{name}: infinite signs differ"
    if not (~inf_o).any():
        return 0.0
    err = np.abs(gpu[~inf_o] - ora[~inf_o])
    k = int(np.argmax(err))
    assert err.max() <= tol, f"{name}: max err {err.max():.4g} > tol {tol:.4g} (index {k})"
    return float(err.max())


def assert_parity(gpu, ora, grad=True):
    """Element-by-element comparison at the tolerances of this module."""
    at_late = ora["at"][:, 2:]
    scale = float(np.max(np.abs(at_late[np.isfinite(at_late)]))) if at_late.size else 1.0
    scale = max(scale, 1.0)
    tol = AT_RTOL * scale
    errs = {}
    errs["at"] = _close("at", gpu["at"], ora["at"], tol)
    errs["slew"] = _close("slew", gpu["slew"], ora["slew"], AT_RTOL * max(scale, np.abs(ora["slew"]).max()))
    errs["rat"] = _close("rat", gpu["rat"], ora["rat"], tol)
    errs["ats"] = _close("ats", gpu["ats"], ora["ats"], tol)
    errs["slack"] = _close("slack", gpu["slack"], ora["pin_slack"], tol)
    errs["ep_slack"] = _close("ep_slack", gpu["ep_slack"], ora["ep_slack"], tol)
    gs, os_ = gpu["summary"], ora["summary"]
    for k in ("wns_early", "wns_late", "wns_gamma"):
        if np.isfinite(os_[k]) or np.isfinite(gs[k]):
            assert abs(gs[k] - os_[k]) <= tol, (k, gs[k], os_[k])
    for k in ("tns_early", "tns_late", "tns_gamma"):
        t = AT_RTOL * max(abs(os_[k]), scale)
        assert abs(gs[k] - os_[k]) <= t, (k, gs[k], os_[k], t)
    near = int((np.abs(ora["ep_slack"][:, 1]) <= tol).sum())
    assert abs(gs["late_violations"] - os_["late_violations"]) <= near
    if grad:
        gmax = float(np.abs(ora["grad"]).max())
        errs["grad"] = _close("grad", gpu["grad"], ora["grad"], GRAD_RTOL * max(gmax, 1e-20))
    return errs
