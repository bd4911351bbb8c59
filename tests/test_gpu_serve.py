"""Serving loop: netlists resident under a memory budget, requests admitted
onto stream slots as they free up.  Every request's results (summary and
gradient) must be bit-identical to the same request run alone, in any mix and
under evictions, and agree with the oracle."""
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


@pytest.fixture(scope="module")
def designs():
    return [netgen.tiny_design(0), netgen.superblue_like(3, scale=0.02, depth=40),
            netgen.superblue_like(5, scale=0.01, depth=30)]


def _requests(designs, n, seed=0):
    import torch
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        k = int(rng.integers(len(designs)))
        w = designs[k]
        xy = netgen.jitter_positions(w.xy, 1, 3.0, 1000 + i)[0]
        xt = torch.from_numpy(xy).pin_memory()
        grad = bool(rng.random() < 0.3)
        reqs.append(dict(net=k, xy=xt, gradient=grad, gamma=float(rng.choice([5.0, 10.0])),
                         w=(1.0, float(rng.uniform(0, 1)))))
    return reqs


def _run(server, ids, reqs, one_at_a_time=False):
    import torch
    out = {}
    pending = {}
    for i, r in enumerate(reqs):
        g = torch.zeros(r["xy"].shape, dtype=torch.float32).pin_memory() if r["gradient"] else None
        rid = server.submit(ids[r["net"]], r["xy"], gradient=r["gradient"], gamma=r["gamma"], w=r["w"], grad_out=g)
        pending[rid] = i
        if one_at_a_time:
            while pending:
                for c in server.poll(wait_ms=200):
                    out[pending.pop(c["id"])] = c
    while pending:
        for c in server.poll(wait_ms=200):
            out[pending.pop(c["id"])] = c
    return [out[i] for i in range(len(reqs))]


def _same(a, b):
    assert a["status"] == 0 and b["status"] == 0
    assert np.array_equal(a["summary"], b["summary"])
    if a["grad"] is not None:
        assert np.array_equal(a["grad"].numpy(), b["grad"].numpy())


def test_mixed_requests_equal_alone_and_oracle(designs):
    from paper_2603_28381_gb300.serving import StaServer
    reqs = _requests(designs, 30)
    mix = StaServer(slots=4)
    ids = [mix.add_netlist(w.netlist, w.library) for w in designs]
    res_mix = _run(mix, ids, reqs)
    st = mix.stats()
    mix.close()
    alone = StaServer(sequential=True)
    ids2 = [alone.add_netlist(w.netlist, w.library) for w in designs]
    res_alone = _run(alone, ids2, reqs, one_at_a_time=True)
    alone.close()
    assert st["resident"] == 3 and st["evictions"] == 0
    for a, b in zip(res_mix, res_alone):
        _same(a, b)
    # two requests against the oracle
    for i in (0, next(k for k, r in enumerate(reqs) if r["gradient"])):
        r, w = reqs[i], designs[reqs[i]["net"]]
        ora = oracle.sta(w.netlist, w.library, r["xy"].numpy(), r["gamma"], r["w"][0], r["w"][1])
        s = dict(zip(["wns_early", "tns_early", "wns_late", "tns_late", "tns_gamma", "wns_gamma",
                      "late_violations", "num_endpoints"], res_mix[i]["summary"].tolist()))
        scale = float(np.abs(ora["at"][:, 2:][np.isfinite(ora["at"][:, 2:])]).max())
        for k in ("wns_late", "wns_gamma"):
            assert abs(s[k] - ora["summary"][k]) <= tp.AT_RTOL * scale
        for k in ("tns_late", "tns_gamma"):
            assert abs(s[k] - ora["summary"][k]) <= tp.AT_RTOL * max(abs(ora["summary"][k]), scale)
        if r["gradient"]:
            gmax = np.abs(ora["grad"]).max()
            assert np.abs(res_mix[i]["grad"].numpy() - ora["grad"]).max() <= tp.GRAD_RTOL * gmax


def _check_oracle(reqs, res, designs, idx):
    for i in idx:
        r, w = reqs[i], designs[reqs[i]["net"]]
        ora = oracle.sta(w.netlist, w.library, r["xy"].numpy(), r["gamma"], r["w"][0], r["w"][1])
        s = dict(zip(["wns_early", "tns_early", "wns_late", "tns_late", "tns_gamma", "wns_gamma",
                      "late_violations", "num_endpoints"], res[i]["summary"].tolist()))
        scale = float(np.abs(ora["at"][:, 2:][np.isfinite(ora["at"][:, 2:])]).max())
        for k in ("wns_late", "wns_gamma"):
            assert abs(s[k] - ora["summary"][k]) <= tp.AT_RTOL * scale, (i, k)
        for k in ("tns_late", "tns_gamma"):
            assert abs(s[k] - ora["summary"][k]) <= tp.AT_RTOL * max(abs(ora["summary"][k]), scale), (i, k)
        assert s["late_violations"] == ora["summary"]["late_violations"]
        if r["gradient"]:
            gmax = np.abs(ora["grad"]).max()
            assert np.abs(res[i]["grad"].numpy() - ora["grad"]).max() <= tp.GRAD_RTOL * gmax, i


def test_merged_requests_equal_alone_and_oracle(designs):
    # merging server: pending requests of one netlist (same gamma and kind) run as
    # lanes of one call; submitted all at once most of them merge.  The same
    # requests one at a time, on a merging server (a call with one lane) and on the
    # plain loop (single-placement handles), must give bit-identical results, and
    # match the oracle.
    from paper_2603_28381_gb300.serving import StaServer
    reqs = _requests(designs, 40, seed=7)
    mrg = StaServer(slots=2, merge=8)
    ids = [mrg.add_netlist(w.netlist, w.library) for w in designs]
    res_m = _run(mrg, ids, reqs)
    mrg.close()
    alone = StaServer(slots=2, merge=8)
    ids2 = [alone.add_netlist(w.netlist, w.library) for w in designs]
    res_a = _run(alone, ids2, reqs, one_at_a_time=True)
    alone.close()
    plain = StaServer(sequential=True)
    ids3 = [plain.add_netlist(w.netlist, w.library) for w in designs]
    res_p = _run(plain, ids3, reqs, one_at_a_time=True)
    plain.close()
    assert max(c["merged"] for c in res_m) > 1, "no requests were merged"
    assert sum(c["merged"] > 1 for c in res_m) >= len(reqs) // 4
    assert all(c["merged"] == 1 for c in res_a)
    for a, b, c in zip(res_m, res_a, res_p):
        _same(a, b)
        _same(a, c)
    merged_grad = [i for i, c in enumerate(res_m) if c["merged"] > 1 and reqs[i]["gradient"]]
    merged_fwd = [i for i, c in enumerate(res_m) if c["merged"] > 1 and not reqs[i]["gradient"]]
    _check_oracle(reqs, res_m, designs, merged_grad[:2] + merged_fwd[:2])


def test_replicas_run_one_netlist_concurrently_results_unchanged(designs):
    # replicas: pending requests of one netlist run concurrently on separate
    # resident copies; results must be bit-identical to the same requests alone
    from paper_2603_28381_gb300.serving import StaServer
    reqs = _requests(designs, 30, seed=9)
    rep = StaServer(slots=4, replicas=3)
    ids = [rep.add_netlist(w.netlist, w.library) for w in designs]
    res_r = _run(rep, ids, reqs)
    st = rep.stats()
    rep.close()
    alone = StaServer(sequential=True)
    ids2 = [alone.add_netlist(w.netlist, w.library) for w in designs]
    res_a = _run(alone, ids2, reqs, one_at_a_time=True)
    alone.close()
    assert st["admissions"] > len(designs)  # copies beyond the first were made
    # two requests of one netlist in flight at the same time
    overlap = any(a["netlist"] == b["netlist"] and a["t_start"] < b["t_done"] and b["t_start"] < a["t_done"]
                  for i, a in enumerate(res_r) for b in res_r[i + 1:])
    assert overlap
    for a, b in zip(res_r, res_a):
        _same(a, b)


def test_budget_forces_evictions_results_unchanged(designs):
    from paper_2603_28381_gb300.serving import StaServer
    reqs = _requests(designs, 16, seed=4)
    big = StaServer(slots=2)
    ids = [big.add_netlist(w.netlist, w.library, preload=False) for w in designs]
    est = [big.netlist_bytes(k) for k in ids]  # estimates (nothing resident yet)
    ref = _run(big, ids, reqs)
    big.close()
    # room for the largest netlist and not much more: admissions evict idle netlists
    small = StaServer(slots=2, budget_bytes=int(max(est) * 1.05))
    ids2 = [small.add_netlist(w.netlist, w.library, preload=False) for w in designs]
    got = _run(small, ids2, reqs)
    st = small.stats()
    small.close()
    assert st["evictions"] > 0 and st["admissions"] > 3
    for a, b in zip(got, ref):
        _same(a, b)


def test_bad_requests_rejected(designs):
    from paper_2603_28381_gb300 import StaError
    from paper_2603_28381_gb300.serving import StaServer
    import torch
    s = StaServer(slots=1)
    k = s.add_netlist(designs[0].netlist, designs[0].library)
    xy = torch.from_numpy(designs[0].xy).pin_memory()
    with pytest.raises(StaError):
        s.submit(k + 5, xy)
    with pytest.raises(StaError):
        s.submit(k, xy, gamma=0.0)
    # the host layout is built at registration: a combinational loop is
    # reported there (STA_ERR_NOT_DAG), not when a request first needs it
    b = netgen.NetlistBuilder()
    i0, o0, i1, o1 = (b.pin(1.0) for _ in range(4))
    b.net(o0, [i1])
    b.net(o1, [i0])
    b.cell(0, [i0], o0)
    b.cell(0, [i1], o1)
    loop, _ = b.build()
    with pytest.raises(StaError) as e:
        s.add_netlist(loop, designs[0].library, preload=False)
    assert e.value.status == 2
    s.close()
