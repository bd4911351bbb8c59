"""Seeded synthetic netlist and cell-library generator.

This module produces the inputs that both the CUDA path and the FP64 oracle
consume: a CSR netlist (pins, nets whose first pin is the driver, cells with
input pins and one output pin), per-pin capacitances and positions, startpoint
assertions, endpoint constraints and a liberty-like library of 7x7 NLDM tables.
It holds none of the timing arithmetic (no delay, load, slew or slack is
computed here): it only draws topology and numbers from a seeded generator.

The shapes follow the paper's workloads (ICCAD 2015 superblue / ICCAD 2025
aes_cipher_top statistics, Table 1), which are not available here; synthetic
netlists of the same size, depth and fanout law stand in for them.

Conventions shared by every consumer:
  * units: ps, fF, Ohm, um.
  * condition index ``cond = 2*el + rf`` with el 0 = early / 1 = late and
    rf 0 = rise / 1 = fall (four timing conditions, Section 3.1.1).
  * library tables are laid out ``[type][arc][rf_out][slew_i][load_j]`` with
    7 slew and 7 load index points per type.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Tuple

import numpy as np

LUT = 7          # table points per axis
MAX_ARCS = 4     # arcs (input pins) per cell type

# Timing-constraint constants of the synthetic designs (ideal clock).
PERIOD_PS = 1000.0
SETUP_PS = 20.0
HOLD_PS = 10.0
PI_SLEW_PS = 20.0


@dataclasses.dataclass
class Netlist:
    """A netlist in the layout the C-ABI's ``StaNetlistDesc`` takes."""
    num_pins: int
    net_ptr: np.ndarray        # int32 [N+1]
    net_pins: np.ndarray       # int32 [net_ptr[N]]; first pin of a net = driver
    cell_type: np.ndarray      # int32 [C]
    cell_in_ptr: np.ndarray    # int32 [C+1]
    cell_in_pins: np.ndarray   # int32 [cell_in_ptr[C]]
    cell_out_pin: np.ndarray   # int32 [C]
    pin_cap: np.ndarray        # float32 [P] fF
    start_pins: np.ndarray     # int32 [S]
    start_at: np.ndarray       # float32 [S,4] ps
    start_slew: np.ndarray     # float32 [S,4] ps
    end_pins: np.ndarray       # int32 [E]
    end_rat: np.ndarray        # float32 [E,4] ps
    r_per_um: float
    c_per_um: float
    name: str = ""
    end_clock: Optional[np.ndarray] = None  # int32 [E] capturing clock pin, -1 none

    @property
    def num_nets(self) -> int:
        return int(self.net_ptr.shape[0] - 1)

    @property
    def num_cells(self) -> int:
        return int(self.cell_type.shape[0])

    def stats(self) -> Dict[str, int]:
        fan = np.diff(self.net_ptr) - 1
        return dict(pins=self.num_pins, nets=self.num_nets, cells=self.num_cells,
                    sinks=int(fan.sum()), arcs=int(self.cell_in_pins.shape[0]),
                    startpoints=int(self.start_pins.shape[0]),
                    endpoints=int(self.end_pins.shape[0]),
                    max_fanout=int(fan.max()) if fan.size else 0)


@dataclasses.dataclass
class Library:
    """A cell library in the layout the C-ABI's ``StaLibrary`` takes."""
    type_num_arcs: np.ndarray  # int32 [T]
    arc_unate: np.ndarray      # int8 [T,4]: +1 positive unate, -1 negative unate
    slew_index: np.ndarray     # float32 [T,7] ps
    load_index: np.ndarray     # float32 [T,7] fF
    delay_tab: np.ndarray      # float32 [T,4,2,7,7] ps
    slew_tab: np.ndarray       # float32 [T,4,2,7,7] ps

    @property
    def num_types(self) -> int:
        return int(self.type_num_arcs.shape[0])


@dataclasses.dataclass
class Workload:
    netlist: Netlist
    library: Library
    xy: np.ndarray             # float32 [P,2] um
    info: Dict[str, object]


# ----------------------------------------------------------------------------
# library
# ----------------------------------------------------------------------------

def geometric_index(lo: float, hi: float) -> np.ndarray:
    """Seven geometrically spaced index points lo .. hi."""
    k = np.arange(LUT, dtype=np.float64)
    return (lo * (hi / lo) ** (k / (LUT - 1))).astype(np.float32)


def make_library(rng: np.random.Generator, arcs_per_type: List[int],
                 unate: Optional[List[int]] = None, noise: float = 0.05) -> Library:
    """Tables ``a + b*slew + c*load + eps`` with eps a 2-D cumulative sum of
    non-negative increments, so that every table is monotone in both indices."""
    T = len(arcs_per_type)
    s_idx = np.tile(geometric_index(5.0, 500.0), (T, 1))
    l_idx = np.tile(geometric_index(1.0, 200.0), (T, 1))
    if unate is None:
        unate = [(-1 if rng.random() < 0.5 else 1) for _ in range(T)]
    arc_unate = np.zeros((T, MAX_ARCS), np.int8)
    for t in range(T):
        arc_unate[t, :] = unate[t]
    delay = np.zeros((T, MAX_ARCS, 2, LUT, LUT), np.float32)
    slew = np.zeros((T, MAX_ARCS, 2, LUT, LUT), np.float32)
    S = s_idx[0].astype(np.float64)[:, None]
    L = l_idx[0].astype(np.float64)[None, :]
    for t in range(T):
        for a in range(MAX_ARCS):
            for rf in range(2):
                for tab, (alo, ahi), (blo, bhi), (clo, chi) in (
                        (delay, (5, 30), (0.05, 0.3), (0.5, 5)),
                        (slew, (5, 20), (0.02, 0.2), (1, 8))):
                    a0 = rng.uniform(alo, ahi)
                    b0 = rng.uniform(blo, bhi)
                    c0 = rng.uniform(clo, chi)
                    inc = rng.uniform(0.0, noise, size=(LUT, LUT))
                    inc[0, 0] = 0.0
                    eps = np.cumsum(np.cumsum(inc, axis=0), axis=1)
                    tab[t, a, rf] = (a0 + b0 * S + c0 * L + eps).astype(np.float32)
    return Library(np.asarray(arcs_per_type, np.int32), arc_unate, s_idx, l_idx,
                   delay, slew)


def bilinear_library(num_types: int, coef: Tuple[float, float, float, float],
                     unate: int = 1) -> Library:
    """A library whose every table is the exact bilinear function
    ``a + b*slew + c*load + e*slew*load`` of its index points (used to pin the
    interpolation: it must reproduce the function everywhere)."""
    a, b, c, e = coef
    s_idx = np.tile(geometric_index(5.0, 500.0), (num_types, 1))
    l_idx = np.tile(geometric_index(1.0, 200.0), (num_types, 1))
    S = s_idx[0].astype(np.float64)[:, None]
    L = l_idx[0].astype(np.float64)[None, :]
    tab = (a + b * S + c * L + e * S * L).astype(np.float32)
    full = np.broadcast_to(tab, (num_types, MAX_ARCS, 2, LUT, LUT)).copy()
    return Library(np.full(num_types, MAX_ARCS, np.int32),
                   np.full((num_types, MAX_ARCS), unate, np.int8),
                   s_idx, l_idx, full, full.copy())


# ----------------------------------------------------------------------------
# a small hand-wiring helper (tests build tiny DAGs with it)
# ----------------------------------------------------------------------------

class NetlistBuilder:
    """Incremental construction of small netlists by hand."""

    def __init__(self, r_per_um: float = 0.1, c_per_um: float = 0.2):
        self.r, self.c = r_per_um, c_per_um
        self.caps: List[float] = []
        self.xy: List[Tuple[float, float]] = []
        self.nets: List[List[int]] = []
        self.cells: List[Tuple[int, List[int], int]] = []
        self.starts: List[Tuple[int, List[float], List[float]]] = []
        self.ends: List[Tuple[int, List[float], int]] = []

    def pin(self, cap: float = 0.0, x: float = 0.0, y: float = 0.0) -> int:
        self.caps.append(cap)
        self.xy.append((x, y))
        return len(self.caps) - 1

    def net(self, driver: int, sinks: List[int]) -> int:
        self.nets.append([driver] + list(sinks))
        return len(self.nets) - 1

    def cell(self, ctype: int, inputs: List[int], output: int) -> int:
        self.cells.append((ctype, list(inputs), output))
        return len(self.cells) - 1

    def start(self, p: int, at=(0.0,) * 4, slew=(PI_SLEW_PS,) * 4) -> None:
        self.starts.append((p, list(at), list(slew)))

    def end(self, p: int, rat=(0.0, 0.0, PERIOD_PS, PERIOD_PS), clock: int = -1) -> None:
        """``clock``: the clock pin of the flop that captures ``p`` (propagated clock)."""
        self.ends.append((p, list(rat), clock))

    def build(self, name: str = "hand") -> Tuple[Netlist, np.ndarray]:
        net_ptr = np.zeros(len(self.nets) + 1, np.int32)
        net_ptr[1:] = np.cumsum([len(n) for n in self.nets])
        net_pins = np.asarray([p for n in self.nets for p in n], np.int32)
        cin_ptr = np.zeros(len(self.cells) + 1, np.int32)
        cin_ptr[1:] = np.cumsum([len(c[1]) for c in self.cells])
        nl = Netlist(
            num_pins=len(self.caps), net_ptr=net_ptr, net_pins=net_pins,
            cell_type=np.asarray([c[0] for c in self.cells], np.int32),
            cell_in_ptr=cin_ptr,
            cell_in_pins=np.asarray([p for c in self.cells for p in c[1]], np.int32),
            cell_out_pin=np.asarray([c[2] for c in self.cells], np.int32),
            pin_cap=np.asarray(self.caps, np.float32),
            start_pins=np.asarray([s[0] for s in self.starts], np.int32),
            start_at=np.asarray([s[1] for s in self.starts], np.float32).reshape(-1, 4),
            start_slew=np.asarray([s[2] for s in self.starts], np.float32).reshape(-1, 4),
            end_pins=np.asarray([e[0] for e in self.ends], np.int32),
            end_rat=np.asarray([e[1] for e in self.ends], np.float32).reshape(-1, 4),
            r_per_um=float(self.r), c_per_um=float(self.c), name=name,
            end_clock=(np.asarray([e[2] for e in self.ends], np.int32)
                       if any(e[2] >= 0 for e in self.ends) else None))
        return nl, np.asarray(self.xy, np.float32).reshape(-1, 2)


# ----------------------------------------------------------------------------
# levelled random netlists
# ----------------------------------------------------------------------------

def _fanout_targets(rng, n, law):
    kind = law[0]
    if kind == "geom":
        _, p, cap = law
        return np.minimum(rng.geometric(p, size=n), cap).astype(np.int64)
    if kind == "power":
        _, alpha, cap = law
        k = np.arange(1, cap + 1, dtype=np.float64)
        pk = k ** (-alpha)
        pk /= pk.sum()
        return rng.choice(np.arange(1, cap + 1), size=n, p=pk).astype(np.int64)
    raise ValueError(kind)


def make_netlist(seed: int, *, n_comb: int, arcs_per_type: List[int], n_ff: int,
                 n_pi: int, n_po: int, depth: int, fanout, box: float,
                 n_huge: int = 0, huge_sinks: int = 0, r_per_um: float = 0.1,
                 c_per_um: float = 0.2, name: str = "", clock_nets: int = 0,
                 clock_at=(0.0, 0.0, 0.0, 0.0)) -> Workload:
    """A levelled random netlist.

    Combinational cells get a logic level 1..depth (every level non-empty); the
    first input of a level-l cell is wired to a net of level l-1 and its other
    inputs to nets of lower levels, drawn in proportion to each net's remaining
    target fanout (``fanout`` = ("geom", p, cap) or ("power", alpha, cap)).
    Flops are a one-arc clock-to-Q cell whose CK pin is an ideal-clock
    startpoint; their D pins and the primary outputs are endpoints. ``n_huge``
    primary-input nets receive ``huge_sinks`` sinks each on random cell inputs.
    With ``clock_nets`` > 0 the clock is propagated instead: that many clock
    sources (startpoints asserted at ``clock_at``) each drive a net whose sinks
    are the CK pins of a share of the flops, and every flop D endpoint names its
    own flop's CK pin as its capturing clock (the random draws for this come
    after all others, so the rest of the design is the ideal-clock one).
    Pins are numbered cell by cell (inputs, then output), then flop D pins,
    primary inputs and primary outputs, so that net order and pin order differ.
    """
    rng = np.random.default_rng(seed)
    n_types_comb = len(arcs_per_type)
    lib = make_library(rng, list(arcs_per_type) + [1],
                       unate=[(-1 if rng.random() < 0.5 else 1) for _ in arcs_per_type] + [1])
    ff_type = n_types_comb

    # --- cells, types, levels ---
    ctype = rng.integers(0, n_types_comb, size=n_comb)
    k_in = np.asarray(arcs_per_type, np.int64)[ctype]
    lvl = np.concatenate([np.arange(1, depth + 1),
                          rng.integers(1, depth + 1, size=max(0, n_comb - depth))])[:n_comb]
    rng.shuffle(lvl)

    n_cells = n_comb + n_ff
    cell_type = np.concatenate([ctype, np.full(n_ff, ff_type)]).astype(np.int32)
    cell_k = np.concatenate([k_in, np.ones(n_ff, np.int64)])
    cell_lvl = np.concatenate([lvl, np.zeros(n_ff, np.int64)])  # flop Q nets: level 0

    # pin numbering: per cell, inputs then output
    cell_first_pin = np.zeros(n_cells + 1, np.int64)
    cell_first_pin[1:] = np.cumsum(cell_k + 1)
    n_cell_pins = int(cell_first_pin[-1])
    cell_in_ptr = np.zeros(n_cells + 1, np.int64)
    cell_in_ptr[1:] = np.cumsum(cell_k)
    owner = np.repeat(np.arange(n_cells), cell_k)
    pos_in_cell = np.arange(int(cell_in_ptr[-1])) - cell_in_ptr[owner]
    cell_in_pins = cell_first_pin[owner] + pos_in_cell
    cell_out_pin = cell_first_pin[1:] - 1
    d_pin0 = n_cell_pins
    pi_pin0 = d_pin0 + n_ff
    po_pin0 = pi_pin0 + n_pi
    num_pins = po_pin0 + n_po

    # --- nets: one per cell output (comb + flop) then one per PI ---
    n_nets = n_cells + n_pi
    net_driver = np.concatenate([cell_out_pin, pi_pin0 + np.arange(n_pi)])
    net_lvl = np.concatenate([cell_lvl, np.zeros(n_pi, np.int64)])
    target = _fanout_targets(rng, n_nets, fanout)
    rem = target.astype(np.float64)
    sink_net = np.full(num_pins, -1, np.int64)   # net that a sink pin hangs on

    # huge PI nets: wire huge_sinks random non-first cell inputs each
    is_first = pos_in_cell == 0
    is_ff_in = owner >= n_comb
    cand_huge = np.flatnonzero(~is_first & ~is_ff_in)
    if n_huge:
        pick = rng.choice(cand_huge, size=n_huge * huge_sinks, replace=False)
        huge_nets = n_cells + rng.choice(n_pi, size=n_huge, replace=False)
        sink_net[cell_in_pins[pick]] = np.repeat(huge_nets, huge_sinks)
        rem[huge_nets] = 0.0

    # nets grouped by level for sampling
    order = np.argsort(net_lvl, kind="stable")
    lvl_sorted = net_lvl[order]
    lvl_start = np.searchsorted(lvl_sorted, np.arange(depth + 2))
    in_lvl = cell_lvl[owner]
    eps = 1e-3
    for l in range(1, depth + 1):
        sel = np.flatnonzero((in_lvl == l) & ~is_ff_in)
        sel = sel[sink_net[cell_in_pins[sel]] < 0]
        if sel.size == 0:
            continue
        first = sel[is_first[sel]]
        other = sel[~is_first[sel]]
        prev = order[lvl_start[l - 1]:lvl_start[l]]
        below = order[:lvl_start[l]]
        if first.size:
            w = np.maximum(rem[prev], eps)
            ch = prev[rng.choice(prev.size, size=first.size, p=w / w.sum())]
            sink_net[cell_in_pins[first]] = ch
            np.subtract.at(rem, ch, 1.0)
        if other.size:
            w = np.maximum(rem[below], eps)
            ch = below[rng.choice(below.size, size=other.size, p=w / w.sum())]
            sink_net[cell_in_pins[other]] = ch
            np.subtract.at(rem, ch, 1.0)

    # endpoints: flop D pins and POs; sink-less nets are served first
    ends = np.concatenate([d_pin0 + np.arange(n_ff), po_pin0 + np.arange(n_po)])
    rng.shuffle(ends)
    nsink = np.bincount(sink_net[sink_net >= 0], minlength=n_nets)
    empty = np.flatnonzero(nsink == 0)
    rng.shuffle(empty)
    extra_po = 0
    if empty.size > ends.size:
        extra_po = int(empty.size - ends.size)
        ends = np.concatenate([ends, num_pins + np.arange(extra_po)])
        sink_net = np.concatenate([sink_net, np.full(extra_po, -1, np.int64)])
        num_pins += extra_po
    sink_net[ends[:empty.size]] = empty
    rest = ends[empty.size:]
    if rest.size:
        w = np.maximum(rem, eps)
        sink_net[rest] = rng.choice(n_nets, size=rest.size, p=w / w.sum())

    # flop CK pins are the flop's single input: ideal-clock startpoints, no net
    ck_pins = cell_in_pins[is_ff_in]

    # --- CSR of nets: driver first, sinks in random order ---
    sinks = np.flatnonzero(sink_net >= 0)
    rng.shuffle(sinks)
    sinks = sinks[np.argsort(sink_net[sinks], kind="stable")]
    cnt = np.bincount(sink_net[sinks], minlength=n_nets)
    net_ptr = np.zeros(n_nets + 1, np.int64)
    net_ptr[1:] = np.cumsum(cnt + 1)
    net_pins = np.empty(int(net_ptr[-1]), np.int64)
    net_pins[net_ptr[:-1]] = net_driver
    offs = np.arange(sinks.size) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    net_pins[net_ptr[sink_net[sinks]] + 1 + offs] = sinks

    # --- electrical values ---
    pin_cap = rng.uniform(0.5, 3.0, size=num_pins).astype(np.float32)
    pin_cap[net_driver] = 0.0
    pin_cap[ck_pins] = 0.0
    xy = rng.uniform(0.0, box, size=(num_pins, 2)).astype(np.float32)

    pi_pins = pi_pin0 + np.arange(n_pi)
    start_pins = np.concatenate([pi_pins, ck_pins]).astype(np.int32)
    start_at = np.zeros((start_pins.size, 4), np.float32)
    start_slew = np.full((start_pins.size, 4), PI_SLEW_PS, np.float32)
    is_d = (ends >= d_pin0) & (ends < pi_pin0)
    end_rat = np.empty((ends.size, 4), np.float32)
    end_rat[:, 0:2] = np.where(is_d, HOLD_PS, 0.0)[:, None]
    end_rat[:, 2:4] = np.where(is_d, PERIOD_PS - SETUP_PS, PERIOD_PS)[:, None]

    nl = Netlist(num_pins=int(num_pins), net_ptr=net_ptr.astype(np.int32),
                 net_pins=net_pins.astype(np.int32), cell_type=cell_type,
                 cell_in_ptr=cell_in_ptr.astype(np.int32),
                 cell_in_pins=cell_in_pins.astype(np.int32),
                 cell_out_pin=cell_out_pin.astype(np.int32), pin_cap=pin_cap,
                 start_pins=start_pins, start_at=start_at, start_slew=start_slew,
                 end_pins=ends.astype(np.int32), end_rat=end_rat,
                 r_per_um=r_per_um, c_per_um=c_per_um, name=name)
    info = dict(seed=seed, depth=depth, box=box, fanout=fanout, extra_po=extra_po,
                net_level=net_lvl.astype(np.int32),
                n_comb=n_comb, n_ff=n_ff, n_pi=n_pi, n_po=n_po, n_huge=n_huge,
                huge_sinks=huge_sinks, clock_nets=clock_nets)
    if clock_nets > 0:
        nl, xy = _propagate_clock(rng, nl, xy, ck_pins, d_pin0, clock_nets, clock_at, box)
        info["net_level"] = None  # the clock nets add a level below the flops
        info["ck_pins"] = ck_pins.astype(np.int32)
    return Workload(nl, lib, xy, info)


def _propagate_clock(rng, nl: Netlist, xy: np.ndarray, ck_pins: np.ndarray, d_pin0: int,
                     clock_nets: int, clock_at, box: float) -> Tuple[Netlist, np.ndarray]:
    """Turn ideal-clock flop CK startpoints into sinks of ``clock_nets`` clock
    nets driven by new clock-source pins; D endpoints name their flop's CK pin."""
    n_ff = ck_pins.shape[0]
    if n_ff < clock_nets:
        raise ValueError("fewer flops than clock nets")
    P0 = nl.num_pins
    src = P0 + np.arange(clock_nets)
    assign = np.arange(n_ff) % clock_nets
    rng.shuffle(assign)
    nets = [np.concatenate([[src[j]], ck_pins[assign == j]]) for j in range(clock_nets)]
    net_pins = np.concatenate([nl.net_pins.astype(np.int64)] + nets)
    net_ptr = np.concatenate([nl.net_ptr.astype(np.int64),
                              nl.net_ptr[-1] + np.cumsum([len(n) for n in nets])])
    pin_cap = np.concatenate([nl.pin_cap, np.zeros(clock_nets, np.float32)])
    pin_cap[ck_pins] = rng.uniform(0.5, 3.0, size=n_ff).astype(np.float32)
    xy = np.concatenate([xy, rng.uniform(0.0, box, size=(clock_nets, 2)).astype(np.float32)])
    keep = ~np.isin(nl.start_pins, ck_pins)
    start_pins = np.concatenate([nl.start_pins[keep], src]).astype(np.int32)
    start_at = np.concatenate([nl.start_at[keep],
                               np.tile(np.asarray(clock_at, np.float32), (clock_nets, 1))])
    start_slew = np.concatenate([nl.start_slew[keep],
                                 np.full((clock_nets, 4), PI_SLEW_PS, np.float32)])
    ends = nl.end_pins.astype(np.int64)
    is_d = (ends >= d_pin0) & (ends < d_pin0 + n_ff)
    end_clock = np.where(is_d, ck_pins[np.clip(ends - d_pin0, 0, n_ff - 1)], -1).astype(np.int32)
    out = dataclasses.replace(nl, num_pins=int(P0 + clock_nets), net_ptr=net_ptr.astype(np.int32),
                              net_pins=net_pins.astype(np.int32), pin_cap=pin_cap,
                              start_pins=start_pins, start_at=start_at.astype(np.float32),
                              start_slew=start_slew, end_clock=end_clock,
                              name=nl.name + f"_clk{clock_nets}")
    return out, xy


# ----------------------------------------------------------------------------
# the paper-shaped workloads
# ----------------------------------------------------------------------------

def tiny_design(seed: int = 0, clock_nets: int = 0) -> Workload:
    """~8k pins, 30 levels, 16 types with 1-4 inputs, geometric(0.4) fanout
    capped at 16, 100 PIs / 100 POs / 200 flops, 500x500 um."""
    return make_netlist(seed, n_comb=2000, arcs_per_type=[1, 2, 3, 4] * 4, n_ff=200,
                        n_pi=100, n_po=100, depth=30, fanout=("geom", 0.4, 16),
                        box=500.0, name="tiny_2k_cells_d30", clock_nets=clock_nets,
                        clock_at=(0.0, 0.0, 3.0, 3.0))


def superblue_like(seed: int = 1, scale: float = 1.0, depth: int = 150,
                   huge: bool = True, clock_nets: int = 0) -> Workload:
    """~2.5M pins (superblue4-sized at scale 1), 150 levels, 64 types with
    1-4 inputs, power-law(2.2) fanout capped at 2000, 8 primary-input nets with
    20k sinks each (20k * scale below scale 1), 3000x3000 um."""
    n_comb = max(depth, int(round(613_000 * scale)))
    huge_sinks = int(round(20_000 * min(scale, 1.0)))
    return make_netlist(seed, n_comb=n_comb, arcs_per_type=[1, 2, 3, 4] * 16,
                        n_ff=max(1, n_comb // 10), n_pi=max(16, n_comb // 20),
                        n_po=max(1, n_comb // 20), depth=depth,
                        fanout=("power", 2.2, 2000), box=3000.0,
                        n_huge=(8 if huge and huge_sinks > 0 else 0),
                        huge_sinks=(huge_sinks if huge else 0),
                        name=f"superblue_like_x{scale:g}_d{depth}", clock_nets=clock_nets)


def jitter_positions(xy: np.ndarray, batch: int, sigma: float, seed: int) -> np.ndarray:
    """``batch`` placements = base positions + N(0, sigma) jitter, float32 [B,P,2]."""
    rng = np.random.default_rng(seed)
    j = rng.normal(0.0, sigma, size=(batch,) + xy.shape).astype(np.float32)
    return (xy[None].astype(np.float32) + j).astype(np.float32)
