"""Tiny random netlists and brute-force path enumeration (test helpers).

The enumeration walks every startpoint-to-pin path explicitly, carrying the
rise/fall transition through each arc's unateness, with edge delays written
from the closed forms of a star net and a slew-independent linear library. It
shares nothing with the oracle's topological sweep.
"""
import numpy as np

import netgen

KRC = 1e-3


def linear_library(num_types, arcs_per_type, seed=0):
    """Slew-independent tables T = A[t,a,rf] + B[t,a,rf] * load, exact in
    float32, different for every type, arc and output transition."""
    rng = np.random.default_rng(seed)
    T = num_types
    A = rng.integers(1, 64, size=(T, 4, 2)).astype(np.float64) / 4.0
    B = rng.integers(1, 32, size=(T, 4, 2)).astype(np.float64) / 8.0
    A2 = rng.integers(1, 64, size=(T, 4, 2)).astype(np.float64) / 4.0
    B2 = rng.integers(1, 32, size=(T, 4, 2)).astype(np.float64) / 8.0
    s_idx = np.tile(np.array([5, 10, 20, 50, 100, 200, 500], np.float32), (T, 1))
    l_idx = np.tile(np.array([1, 2, 5, 10, 20, 50, 200], np.float32), (T, 1))
    L = l_idx[0].astype(np.float64)
    delay = np.zeros((T, 4, 2, 7, 7), np.float32)
    slew = np.zeros((T, 4, 2, 7, 7), np.float32)
    for t in range(T):
        for a in range(4):
            for rf in range(2):
                delay[t, a, rf] = (A[t, a, rf] + B[t, a, rf] * L)[None, :]
                slew[t, a, rf] = (A2[t, a, rf] + B2[t, a, rf] * L)[None, :]
    unate = np.where(rng.random(T) < 0.5, -1, 1).astype(np.int8)
    lib = netgen.Library(np.asarray(arcs_per_type, np.int32), np.repeat(unate[:, None], 4, 1),
                         s_idx, l_idx, delay, slew)
    return lib, A, B


def tiny_netlist(seed, n_comb=10, depth=4, clock_nets=0):
    w = netgen.make_netlist(seed, n_comb=n_comb, arcs_per_type=[1, 2, 3, 4], n_ff=2, n_pi=3,
                            n_po=2, depth=depth, fanout=("geom", 0.5, 4), box=100.0,
                            name=f"tiny{seed}", clock_nets=clock_nets)
    return w


def star_quantities(nl, xy):
    xy = xy.astype(np.float64)
    cap = nl.pin_cap.astype(np.float64)
    P = nl.num_pins
    load = np.zeros(nl.num_nets)
    wd = np.zeros(P)
    for n in range(nl.num_nets):
        pins = nl.net_pins[nl.net_ptr[n]:nl.net_ptr[n + 1]]
        d = pins[0]
        load[n] = cap[d]
        for s in pins[1:]:
            dist = abs(xy[s, 0] - xy[d, 0]) + abs(xy[s, 1] - xy[d, 1])
            load[n] += cap[s] + nl.c_per_um * dist
            wd[s] = nl.r_per_um * dist * (cap[s] + nl.c_per_um * dist / 2) * KRC
    return load, wd


def edges(nl, lib, A, B, xy):
    """Timing edges (u, rf_u) -> (v, rf_v) with their delays."""
    load, wd = star_quantities(nl, xy)
    drv_net = {int(nl.net_pins[nl.net_ptr[n]]): n for n in range(nl.num_nets)}
    out = {}
    for n in range(nl.num_nets):
        pins = nl.net_pins[nl.net_ptr[n]:nl.net_ptr[n + 1]]
        for s in pins[1:]:
            for rf in range(2):
                out.setdefault((int(pins[0]), rf), []).append(((int(s), rf), wd[s]))
    for c in range(nl.num_cells):
        t = nl.cell_type[c]
        o = int(nl.cell_out_pin[c])
        ld = load[drv_net[o]] if o in drv_net else float(nl.pin_cap[o])
        for ai, i in enumerate(nl.cell_in_pins[nl.cell_in_ptr[c]:nl.cell_in_ptr[c + 1]]):
            for rf_out in range(2):
                rf_in = rf_out if lib.arc_unate[t, ai] > 0 else 1 - rf_out
                dly = A[t, ai, rf_out] + B[t, ai, rf_out] * ld
                out.setdefault((int(i), rf_in), []).append(((o, rf_out), dly))
    return out


def enumerate_paths(nl, lib, A, B, xy):
    """All-paths arrival and required times: dict (pin, rf) -> list of values."""
    E = edges(nl, lib, A, B, xy)
    arrivals = {}

    def walk(node, t):
        arrivals.setdefault(node, []).append(t)
        for nxt, d in E.get(node, []):
            walk(nxt, t + d)

    for k, p in enumerate(nl.start_pins):
        for rf in range(2):
            walk((int(p), rf), float(nl.start_at[k, 2 + rf]))
    ends = {int(p): k for k, p in enumerate(nl.end_pins)}
    required = {}

    def back(node):
        """list of (endpoint index, rf at endpoint, path delay) reachable from node"""
        res = []
        if node[0] in ends:
            res.append((ends[node[0]], node[1], 0.0))
        for nxt, d in E.get(node, []):
            for e, rf, dd in back(nxt):
                res.append((e, rf, dd + d))
        return res

    for p in range(nl.num_pins):
        for rf in range(2):
            required[(p, rf)] = back((p, rf))
    return arrivals, required
