"""FP64 CPU oracle for levelized static timing analysis (Warp-STAR, arXiv 2603.28381).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The CUDA path never
imports, links or runs anything in this directory, and this directory imports
nothing from the CUDA path.

The arithmetic lives in ``sta_oracle.c`` (plain C, double precision, a single
thread, pin graph walked in Kahn topological order).  This module compiles it
with gcc on first use and marshals numpy arrays through ctypes.

Every function is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``
(closed-form Elmore moments, exact bilinear tables, brute-force path
enumeration, slack/TNS invariants, LSE limits, finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sta_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

# summary layout returned by sta(): early (hold) and late (setup) WNS/TNS, then
# the smoothed terms of the loss.
SUMMARY_KEYS = ("wns_early", "tns_early", "wns_late", "tns_late",
                "tns_gamma", "wns_gamma", "loss", "late_violations")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so``."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Netlist(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int), ("N", ctypes.c_int), ("C", ctypes.c_int),
                ("net_ptr", ctypes.c_void_p), ("net_pins", ctypes.c_void_p),
                ("cell_type", ctypes.c_void_p), ("cell_in_ptr", ctypes.c_void_p),
                ("cell_in_pins", ctypes.c_void_p), ("cell_out_pin", ctypes.c_void_p),
                ("pin_cap", ctypes.c_void_p),
                ("S", ctypes.c_int), ("start_pins", ctypes.c_void_p),
                ("start_at", ctypes.c_void_p), ("start_slew", ctypes.c_void_p),
                ("E", ctypes.c_int), ("end_pins", ctypes.c_void_p), ("end_rat", ctypes.c_void_p),
                ("r_per_um", ctypes.c_double), ("c_per_um", ctypes.c_double),
                ("T", ctypes.c_int), ("type_num_arcs", ctypes.c_void_p),
                ("arc_unate", ctypes.c_void_p), ("slew_index", ctypes.c_void_p),
                ("load_index", ctypes.c_void_p), ("delay_tab", ctypes.c_void_p),
                ("slew_tab", ctypes.c_void_p), ("end_clk", ctypes.c_void_p)]


class _Out(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("at", "slew", "rat", "ats", "pin_slack", "ep_slack", "summary", "grad",
                 "net_load", "wdelay", "impulse", "adel", "decision_hash")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_SO lets the mutation tests load a deliberately broken copy
            lib = ctypes.CDLL(os.environ.get("ORACLE_SO") or build())
            lib.oracle_sta.restype = ctypes.c_int
            lib.oracle_sta.argtypes = [ctypes.POINTER(_Netlist), ctypes.c_void_p, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.POINTER(_Out)]
            lib.oracle_levels.restype = ctypes.c_int
            lib.oracle_levels.argtypes = [ctypes.POINTER(_Netlist), ctypes.c_void_p]
            lib.oracle_elmore_tree.restype = None
            lib.oracle_elmore_tree.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 7
            lib.oracle_nldm.restype = ctypes.c_double
            lib.oracle_nldm.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_lse.restype = ctypes.c_double
            lib.oracle_lse.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_double]
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class _Pack:
    """Keeps the contiguous copies alive while the C call runs."""

    def __init__(self, nl, lib):
        self.keep = []

        def ptr(a, dt):
            arr = _c(a, dt)
            self.keep.append(arr)
            return arr.ctypes.data

        self.s = _Netlist(
            P=int(nl.num_pins), N=int(nl.net_ptr.shape[0] - 1), C=int(nl.cell_type.shape[0]),
            net_ptr=ptr(nl.net_ptr, np.int32), net_pins=ptr(nl.net_pins, np.int32),
            cell_type=ptr(nl.cell_type, np.int32), cell_in_ptr=ptr(nl.cell_in_ptr, np.int32),
            cell_in_pins=ptr(nl.cell_in_pins, np.int32), cell_out_pin=ptr(nl.cell_out_pin, np.int32),
            pin_cap=ptr(nl.pin_cap, np.float32),
            S=int(nl.start_pins.shape[0]), start_pins=ptr(nl.start_pins, np.int32),
            start_at=ptr(nl.start_at, np.float32), start_slew=ptr(nl.start_slew, np.float32),
            E=int(nl.end_pins.shape[0]), end_pins=ptr(nl.end_pins, np.int32),
            end_rat=ptr(nl.end_rat, np.float32),
            r_per_um=float(nl.r_per_um), c_per_um=float(nl.c_per_um),
            T=0 if lib is None else int(lib.type_num_arcs.shape[0]),
            type_num_arcs=None if lib is None else ptr(lib.type_num_arcs, np.int32),
            arc_unate=None if lib is None else ptr(lib.arc_unate, np.int8),
            slew_index=None if lib is None else ptr(lib.slew_index, np.float32),
            load_index=None if lib is None else ptr(lib.load_index, np.float32),
            delay_tab=None if lib is None else ptr(lib.delay_tab, np.float32),
            slew_tab=None if lib is None else ptr(lib.slew_tab, np.float32),
            end_clk=(None if getattr(nl, "end_clock", None) is None else ptr(nl.end_clock, np.int32)))


class OracleError(RuntimeError):
    pass


def levels(nl) -> np.ndarray:
    """Net levels by memoised depth-first search (int32 [N])."""
    L = _load()
    pk = _Pack(nl, None)
    out = np.zeros(nl.net_ptr.shape[0] - 1, np.int32)
    rc = L.oracle_levels(ctypes.byref(pk.s), out.ctypes.data)
    if rc < 0:
        raise OracleError({-1: "invalid netlist", -2: "cycle", -3: "out of memory"}.get(rc, str(rc)))
    return out


def sta(nl, lib, xy, gamma: float = 10.0, w_tns: float = 1.0, w_wns: float = 0.0,
        want: Optional[set] = None) -> Dict[str, np.ndarray]:
    """Full FP64 STA, smoothed loss and its gradient with respect to ``xy``.

    Returns arrays in the netlist's own pin order: ``at``/``slew``/``rat`` [P,4],
    ``ats`` [P,2] (late rise/fall LSE arrival), ``pin_slack`` and ``ep_slack``
    [.,2] (early, late), ``grad`` [P,2], ``net_load`` [N], ``wdelay``/``impulse``
    [P], ``adel`` [A,4] and ``summary`` (dict with SUMMARY_KEYS) plus
    ``decision_hash`` (changes whenever a segment, argmax or sign changes).
    """
    L = _load()
    P = int(nl.num_pins)
    N = int(nl.net_ptr.shape[0] - 1)
    E = int(nl.end_pins.shape[0])
    A = int(nl.cell_in_pins.shape[0])
    shapes = dict(at=(P, 4), slew=(P, 4), rat=(P, 4), ats=(P, 2), pin_slack=(P, 2),
                  ep_slack=(E, 2), grad=(P, 2), net_load=(N,), wdelay=(P,), impulse=(P,),
                  adel=(A, 4))
    if want is None:
        want = set(shapes)
    res = {k: np.zeros(s, np.float64) for k, s in shapes.items() if k in want}
    summ = np.zeros(8, np.float64)
    h = np.zeros(1, np.uint64)
    pk = _Pack(nl, lib)
    xyd = _c(xy, np.float64).reshape(-1)
    if xyd.shape[0] != 2 * P:
        raise ValueError("xy must be [P,2]")
    o = _Out(**{k: (res[k].ctypes.data if k in res else None) for k in shapes},
             summary=summ.ctypes.data, decision_hash=h.ctypes.data)
    rc = L.oracle_sta(ctypes.byref(pk.s), xyd.ctypes.data, float(gamma), float(w_tns),
                      float(w_wns), ctypes.byref(o))
    if rc < 0:
        raise OracleError({-1: "invalid netlist", -2: "cycle", -3: "out of memory"}.get(rc, str(rc)))
    res["summary"] = dict(zip(SUMMARY_KEYS, summ.tolist()))
    res["decision_hash"] = int(h[0])
    return res


def loss(nl, lib, xy, gamma=10.0, w_tns=1.0, w_wns=0.0):
    """(loss, decision_hash) at positions ``xy`` (FP64)."""
    r = sta(nl, lib, xy, gamma, w_tns, w_wns, want=set())
    return r["summary"]["loss"], r["decision_hash"]


def elmore_tree(parent, res, cap):
    """Eqs. 1-3 on an RC tree (parents before children): (load, delay, impulse)."""
    L = _load()
    n = len(parent)
    parent = _c(parent, np.int32)
    res = _c(res, np.float64)
    cap = _c(cap, np.float64)
    load = np.zeros(n)
    delay = np.zeros(n)
    imp = np.zeros(n)
    work = np.zeros(2 * n)
    L.oracle_elmore_tree(n, parent.ctypes.data, res.ctypes.data, cap.ctypes.data,
                         load.ctypes.data, delay.ctypes.data, imp.ctypes.data, work.ctypes.data)
    return load, delay, imp


def nldm(tab, s_idx, l_idx, s, l):
    """One bilinear table lookup: (value, d/dslew, d/dload, seg_s, seg_l)."""
    L = _load()
    tab = _c(tab, np.float32).reshape(-1)
    s_idx = _c(s_idx, np.float32)
    l_idx = _c(l_idx, np.float32)
    dds = ctypes.c_double()
    ddl = ctypes.c_double()
    ks = ctypes.c_int()
    kl = ctypes.c_int()
    v = L.oracle_nldm(tab.ctypes.data, s_idx.ctypes.data, l_idx.ctypes.data, float(s), float(l),
                      ctypes.byref(dds), ctypes.byref(ddl), ctypes.byref(ks), ctypes.byref(kl))
    return v, dds.value, ddl.value, ks.value, kl.value


def lse(x, gamma):
    """Eq. 4 (stabilised LogSumExp) of a vector."""
    L = _load()
    x = _c(x, np.float64)
    return L.oracle_lse(int(x.shape[0]), x.ctypes.data, float(gamma))


def finite_difference(nl, lib, xy, pins, gamma=10.0, w_tns=1.0, w_wns=0.0, h=1e-3):
    """FP64 central differences of the loss at the given pins (both coordinates).

    Returns (fd [len(pins),2], valid [len(pins),2]); an entry is invalid when the
    +-h perturbation changes any discrete decision (table segment, slew argmax,
    sign of a coordinate difference), where the loss is not differentiable.
    """
    base = _c(xy, np.float64).copy()
    _, h0 = loss(nl, lib, base, gamma, w_tns, w_wns)
    fd = np.zeros((len(pins), 2))
    ok = np.zeros((len(pins), 2), bool)
    for i, p in enumerate(pins):
        for k in range(2):
            xp = base.copy()
            xp[p, k] += h
            lp, hp = loss(nl, lib, xp, gamma, w_tns, w_wns)
            xp[p, k] -= 2 * h
            lm, hm = loss(nl, lib, xp, gamma, w_tns, w_wns)
            fd[i, k] = (lp - lm) / (2 * h)
            ok[i, k] = (hp == h0) and (hm == h0)
    return fd, ok
