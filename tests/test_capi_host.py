"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point include/sta.h declares; the host-side levelization and layout
order are bit-exact against independent computations; malformed netlists are
rejected with the documented status codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import netgen
import oracle
from tests import _tinydag as td

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sta():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2603_28381_gb300 as mod
    return mod


def test_library_exports_every_declared_symbol(sta):
    header = open(os.path.join(ROOT, "include", "sta.h")).read()
    declared = set(re.findall(r"^\S.*?\b(sta_\w+)\s*\(", header, flags=re.M))
    assert {"sta_create", "sta_forward", "sta_backward_grad", "sta_set_positions",
            "sta_query_summary", "sta_destroy"} <= declared
    lib = ctypes.CDLL(sta._sta.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(lib, name), f"libsta.so does not export {name}"
    assert set(sta._sta.EXPORTS) == declared
    assert sta.sta_abi_version() == 5


@pytest.mark.parametrize("make", [lambda: netgen.tiny_design(0), lambda: netgen.tiny_design(5),
                                  lambda: td.tiny_netlist(3),
                                  lambda: netgen.superblue_like(2, scale=0.01, depth=25)])
def test_levelize_bit_exact_against_oracle_dfs(sta, make):
    w = make()
    nl = w.netlist
    lv, L, order, pins = sta.sta_levelize(nl)
    ref = oracle.levels(nl)
    np.testing.assert_array_equal(lv, ref)
    assert L == ref.max() + 1
    # processing order: level; within a level nets of > 32 pins after the others,
    # then the latest position of a net feeding the driver cell (-1: none), then id
    size = np.diff(nl.net_ptr)
    sink_net = np.full(nl.num_pins, -1, np.int64)
    for n in range(nl.num_nets):
        sink_net[nl.net_pins[nl.net_ptr[n] + 1:nl.net_ptr[n + 1]]] = n
    out_cell = {int(p): c for c, p in enumerate(nl.cell_out_pin)}
    pos = np.full(nl.num_nets, -1, np.int64)
    expect = []
    for lvl in range(L):
        nets = np.flatnonzero(ref == lvl)
        key = []
        for n in nets:
            c = out_cell.get(int(nl.net_pins[nl.net_ptr[n]]), -1)
            ins = nl.cell_in_pins[nl.cell_in_ptr[c]:nl.cell_in_ptr[c + 1]] if c >= 0 else []
            key.append(max([pos[sink_net[p]] for p in ins if sink_net[p] >= 0], default=-1))
        o = nets[np.lexsort((nets, np.asarray(key), size[nets] > 32))]
        pos[o] = len(expect) + np.arange(o.size)
        expect.extend(o.tolist())
    np.testing.assert_array_equal(order, np.asarray(expect))
    # device pin order: per net in processing order, driver then sinks ascending
    exp_pins = []
    for n in expect:
        seg = nl.net_pins[nl.net_ptr[n]:nl.net_ptr[n + 1]]
        exp_pins.append(seg[:1])
        exp_pins.append(np.sort(seg[1:]))
    np.testing.assert_array_equal(pins, np.concatenate(exp_pins))


def test_levelize_rejects_cycles_and_malformed_netlists(sta):
    b = netgen.NetlistBuilder()
    i0, o0, i1, o1 = (b.pin(1.0) for _ in range(4))
    b.net(o0, [i1])
    b.net(o1, [i0])
    b.cell(0, [i0], o0)
    b.cell(0, [i1], o1)
    nl, _ = b.build()
    with pytest.raises(sta.StaError) as e:
        sta.sta_levelize(nl)
    assert e.value.status == 2  # STA_ERR_NOT_DAG
    # a pin on two nets
    b = netgen.NetlistBuilder()
    d, s = b.pin(), b.pin(1.0)
    b.net(d, [s])
    b.net(d, [s])
    b.start(d)
    nl, _ = b.build()
    with pytest.raises(sta.StaError) as e:
        sta.sta_levelize(nl)
    assert e.value.status == 1  # STA_ERR_INVALID_ARG
    assert "two nets" in sta.sta_last_error()
    # an endpoint that is a cell input
    b = netgen.NetlistBuilder()
    d, s, o, t = b.pin(), b.pin(1.0), b.pin(), b.pin(1.0)
    b.net(d, [s])
    b.cell(0, [s], o)
    b.net(o, [t])
    b.start(d)
    b.end(s)
    nl, _ = b.build()
    with pytest.raises(sta.StaError) as e:
        sta.sta_levelize(nl)
    assert e.value.status == 1
    # an orphan pin (no arrival source)
    b = netgen.NetlistBuilder()
    b.pin()
    nl, _ = b.build()
    with pytest.raises(sta.StaError):
        sta.sta_levelize(nl)


def test_levelize_checks_capturing_clock_pins(sta):
    """A propagated clock's capturing pin must be a cell input on a net driven
    by a startpoint, and capture one endpoint at most."""
    w = netgen.tiny_design(0, clock_nets=2)
    nl = w.netlist
    lv, L, _, _ = sta.sta_levelize(nl)
    np.testing.assert_array_equal(lv, oracle.levels(nl))
    bad = []
    b1 = netgen.Netlist(**{f.name: getattr(nl, f.name) for f in netgen.dataclasses.fields(nl)})
    b1.end_clock = nl.end_clock.copy()
    b1.end_clock[np.flatnonzero(nl.end_clock >= 0)[0]] = nl.cell_out_pin[0]  # a cell output
    bad.append(b1)
    b2 = netgen.Netlist(**{f.name: getattr(nl, f.name) for f in netgen.dataclasses.fields(nl)})
    b2.end_clock = nl.end_clock.copy()
    j = np.flatnonzero(nl.end_clock >= 0)[:2]
    b2.end_clock[j[1]] = b2.end_clock[j[0]]  # one clock pin capturing two endpoints
    bad.append(b2)
    b3 = netgen.Netlist(**{f.name: getattr(nl, f.name) for f in netgen.dataclasses.fields(nl)})
    b3.end_clock = nl.end_clock.copy()
    b3.end_clock[0] = nl.num_pins  # out of range
    bad.append(b3)
    # a comb cell input on a net driven by a cell output (not a startpoint)
    b4 = netgen.Netlist(**{f.name: getattr(nl, f.name) for f in netgen.dataclasses.fields(nl)})
    b4.end_clock = nl.end_clock.copy()
    drv = set(nl.net_pins[nl.net_ptr[:-1]].tolist())
    starts = set(nl.start_pins.tolist())
    for n in range(nl.num_nets):
        if nl.net_pins[nl.net_ptr[n]] not in starts:
            s = nl.net_pins[nl.net_ptr[n] + 1:nl.net_ptr[n + 1]]
            s = [p for p in s if p in set(nl.cell_in_pins.tolist()) and p not in drv]
            if s:
                b4.end_clock[np.flatnonzero(nl.end_clock >= 0)[0]] = s[0]
                break
    bad.append(b4)
    # the input of a multi-input cell on a startpoint's net: the oracle's model
    # takes it, the C ABI wants the clock pin of a one-input (clock->Q) cell
    b5 = netgen.Netlist(**{f.name: getattr(nl, f.name) for f in netgen.dataclasses.fields(nl)})
    b5.end_clock = nl.end_clock.copy()
    width = np.diff(nl.cell_in_ptr)
    owner = np.repeat(np.arange(nl.num_cells), width)
    for n in range(nl.num_nets):
        if nl.net_pins[nl.net_ptr[n]] in starts:
            s = [p for p in nl.net_pins[nl.net_ptr[n] + 1:nl.net_ptr[n + 1]]
                 if p in set(nl.cell_in_pins.tolist())
                 and width[owner[np.flatnonzero(nl.cell_in_pins == p)[0]]] > 1]
            if s:
                b5.end_clock[np.flatnonzero(nl.end_clock >= 0)[0]] = s[0]
                break
    assert not np.array_equal(b5.end_clock, nl.end_clock)
    bad.append(b5)
    for b in bad:
        with pytest.raises(sta.StaError) as e:
            sta.sta_levelize(b)
        assert e.value.status == 1
        with pytest.raises(oracle.OracleError) if b is not b2 and b is not b5 else _nothing():
            oracle.sta(b, w.library, w.xy)


class _nothing:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def test_product_path_fails_loudly_without_gpu(sta):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    w = netgen.tiny_design(0)
    with pytest.raises(RuntimeError):
        sta.StaEngine(w.netlist, w.library)
    with pytest.raises(sta.StaError) as e:
        sta._sta.sta_create(w.netlist, w.library)
    assert e.value.status == 4  # STA_ERR_CUDA, no CPU fallback


@pytest.mark.parametrize("tile_pins,tile_nets,chunk", [(32, 8, 32), (1, 1, 1), (4, 1 << 20, 16), (64, 4, 200)])
def test_task_plans_cover_every_sink_in_dependency_order(tile_pins, tile_nets, chunk):
    # the builder rejects any plan whose tasks depend on later tasks or leave a
    # sink without a forward task; here the counts are checked against the netlist
    import numpy as np
    import netgen
    from paper_2603_28381_gb300 import _sta
    w = netgen.superblue_like(3, scale=0.02, depth=40)
    nl = w.netlist
    plan = _sta.sta_plan_tasks(nl, w.library, tile_pins, tile_nets, chunk)
    fan = np.diff(nl.net_ptr) - 1  # sinks per description net
    big = fan + 1 > chunk + 1
    assert plan["split_nets"] == int(big.sum())
    assert plan["chunks"] == int(np.ceil(fan[big] / chunk).sum())
    assert plan["partials"] == plan["chunks"]                       # one partial per backward chunk
    # backward: a task per packed group, a partial, a driver and a gradient task per chunked net
    assert plan["backward_tasks"] == (plan["forward_tasks"] - plan["chunks"]) + 2 * plan["chunks"] + plan["split_nets"]
    assert plan["max_nets"] <= tile_nets
    assert plan["max_pins"] <= max(tile_pins, chunk + 1)


def test_latency_probe_checks_its_arguments(sta):
    for nbytes, steps in ((0, 10), (1 << 20, 0), (1 << 40, 10)):
        with pytest.raises(sta.StaError) as e:
            sta.sta_measure_latency(nbytes, steps)
        assert e.value.status == 1


def test_noalloc_summary_refuses_misaligned_pointers(sta):
    # the allocation-free summary reads at / end_rat as float4 and ats / ep_slack
    # as float2; a misaligned view is refused on the host, before any device work
    # (these pointer values are never dereferenced)
    good = dict(at=1 << 20, ats=1 << 20, end_pins=1 << 20, end_rat=1 << 20, end_clk=0,
                ep_slack=1 << 20, summary=1 << 20)
    for name, off in (("at", 4), ("at", 8), ("end_rat", 8), ("ats", 4), ("ep_slack", 4), ("summary", 4),
                      ("end_pins", 2), ("end_clk", 2)):
        a = dict(good)
        a[name] = (1 << 21) + off
        with pytest.raises(sta.StaError) as e:
            sta._sta.sta_endpoint_summary_noalloc(a["at"], a["ats"], 10, a["end_pins"], a["end_rat"],
                                                  a["end_clk"], 4, 10.0, a["ep_slack"], a["summary"], 0)
        assert e.value.status == 1, name  # STA_ERR_INVALID_ARG
        assert "misaligned" in sta.sta_last_error(), name


def test_multi_rejects_bad_unions_before_any_device_use(sta):
    # sta_create_multi checks the netlists and builds the union's layout on the
    # host; these are refused there, with the documented status codes
    from paper_2603_28381_gb300 import _sta
    a = netgen.superblue_like(3, scale=0.002, depth=10)
    b = netgen.superblue_like(4, scale=0.002, depth=10)
    with pytest.raises(sta.StaError) as e:
        _sta.sta_create_multi([], a.library)
    assert e.value.status == 1 and "count" in sta.sta_last_error()
    odd = netgen.superblue_like(4, scale=0.002, depth=10).netlist
    odd.r_per_um = 0.25
    with pytest.raises(sta.StaError) as e:
        _sta.sta_create_multi([a.netlist, odd], a.library)
    assert e.value.status == 1 and "r_per_um" in sta.sta_last_error()
    # a combinational loop in the second netlist: the union is not a DAG
    bl = netgen.NetlistBuilder()
    i0, o0, i1, o1 = (bl.pin(1.0) for _ in range(4))
    bl.net(o0, [i1])
    bl.net(o1, [i0])
    bl.cell(0, [i0], o0)
    bl.cell(0, [i1], o1)
    loop, _ = bl.build()
    with pytest.raises(sta.StaError) as e:
        _sta.sta_create_multi([a.netlist, loop, b.netlist], a.library)
    assert e.value.status == 2  # STA_ERR_NOT_DAG
