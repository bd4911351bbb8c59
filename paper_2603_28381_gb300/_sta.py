"""ctypes binding of libsta (include/sta.h): same names, argument marshalling only.

Every computation happens inside libsta's CUDA kernels.  If the library is not
built this module raises ImportError: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libsta.so")

STA_OK = 0
STATUS = {0: "STA_OK", 1: "STA_ERR_INVALID_ARG", 2: "STA_ERR_NOT_DAG", 3: "STA_ERR_OOM",
          4: "STA_ERR_CUDA", 5: "STA_ERR_TIMEOUT", 6: "STA_ERR_STATE"}
STA_FWD_LSE = 1
STA_FWD_RAT = 2
STA_FWD_RAT_EAGER = 4
SUMMARY_KEYS = ("wns_early", "tns_early", "wns_late", "tns_late", "tns_gamma", "wns_gamma",
                "late_violations", "num_endpoints")

_p = ctypes.c_void_p
_i32 = ctypes.c_int32


class StaNetlistDesc(ctypes.Structure):
    _fields_ = [("num_pins", _i32), ("num_nets", _i32), ("num_cells", _i32),
                ("net_ptr", _p), ("net_pins", _p), ("cell_type", _p), ("cell_in_ptr", _p),
                ("cell_in_pins", _p), ("cell_out_pin", _p), ("pin_cap", _p),
                ("num_start", _i32), ("start_pins", _p), ("start_at", _p), ("start_slew", _p),
                ("num_end", _i32), ("end_pins", _p), ("end_rat", _p),
                ("r_per_um", ctypes.c_float), ("c_per_um", ctypes.c_float),
                ("end_clock", _p)]


class StaLibrary(ctypes.Structure):
    _fields_ = [("num_types", _i32), ("type_num_arcs", _p), ("arc_unate", _p),
                ("slew_index", _p), ("load_index", _p), ("delay_tab", _p), ("slew_tab", _p)]


class StaOptions(ctypes.Structure):
    _fields_ = [("use_graphs", _i32), ("profile", _i32), ("schedule", _i32), ("num_placements", _i32),
                ("tile_pins", _i32), ("chunk", _i32), ("batch_sweep", _i32), ("grid_blocks", _i32)]


PROF_KINDS = ("positions", "net_rc", "forward", "endpoints", "required", "seed", "adjoint", "output", "reset")
SCHED_DATAFLOW = 0
SCHED_LEVELS = 1
SCHED_BATCH = 2
BATCH_LEVELS = 0
BATCH_DATAFLOW = 1
BATCH_LANES = 2
BATCH_WIDE = 3


class StaServerOptions(ctypes.Structure):
    _fields_ = [("slots", _i32), ("sequential", _i32), ("budget_bytes", ctypes.c_int64), ("merge", _i32),
                ("replicas", _i32), ("reserved", _i32 * 2)]


class StaServerRequest(ctypes.Structure):
    _fields_ = [("netlist", _i32), ("gradient", _i32), ("gamma", ctypes.c_float), ("w_tns", ctypes.c_float),
                ("w_wns", ctypes.c_float), ("xy", _p), ("grad", _p), ("summary", _p)]


class StaServerCompletion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", _i32), ("netlist", _i32), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double), ("merged", _i32), ("reserved", _i32)]


class StaError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsta.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    sig = {
        "sta_create": ([ctypes.POINTER(StaNetlistDesc), ctypes.POINTER(StaLibrary),
                        ctypes.POINTER(StaOptions), ctypes.POINTER(H)], ctypes.c_int),
        "sta_create_multi": ([ctypes.POINTER(ctypes.POINTER(StaNetlistDesc)), _i32, ctypes.POINTER(StaLibrary),
                              ctypes.POINTER(StaOptions), ctypes.POINTER(H)], ctypes.c_int),
        "sta_set_positions": ([H, _p, ctypes.c_int, _p], ctypes.c_int),
        "sta_forward": ([H, ctypes.c_uint32, ctypes.c_float, _p], ctypes.c_int),
        "sta_backward_grad": ([H, _p, ctypes.c_int, _p, ctypes.c_int, _p], ctypes.c_int),
        "sta_query_summary": ([H, _p, ctypes.c_int, _p], ctypes.c_int),
        "sta_stream_wait": ([H, _p], ctypes.c_int),
        "sta_synchronize": ([H], ctypes.c_int),
        "sta_query_net_rc": ([H, _p, _p, _p], ctypes.c_int),
        "sta_ablation_net_rc": ([H, _i32, _i32, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "sta_autotune": ([H, _p, _i32, _p, _i32, _p, _i32, _i32, ctypes.c_float, _p, _p], ctypes.c_int),
        "sta_debug_expire_wait": ([H], ctypes.c_int),
        "sta_query_pins": ([H, _p, _p, _p, _p, _p, ctypes.c_int, _p], ctypes.c_int),
        "sta_query_endpoints": ([H, _p, ctypes.c_int, _p], ctypes.c_int),
        "sta_query_slack": ([H, _p, _p, _p], ctypes.c_int),
        "sta_measure_latency": ([ctypes.c_int64, ctypes.c_int32, _p], ctypes.c_int),
        "sta_levelize": ([ctypes.POINTER(StaNetlistDesc), _p, _p, _p, _p], ctypes.c_int),
        "sta_query_sizes": ([H, _p], ctypes.c_int),
        "sta_plan_tasks": ([ctypes.POINTER(StaNetlistDesc), ctypes.POINTER(StaLibrary), _i32, _i32, _i32, _p],
                           ctypes.c_int),
        "sta_query_profile": ([H, _p, _p], ctypes.c_int),
        "sta_endpoint_summary_noalloc": ([_p, _p, _i32, _p, _p, _p, _i32, ctypes.c_float, _p, _p, _p],
                                         ctypes.c_int),
        "sta_set_active": ([H, _i32], ctypes.c_int),
        "sta_destroy": ([H], None),
        "sta_server_create": ([ctypes.POINTER(StaServerOptions), ctypes.POINTER(H)], ctypes.c_int),
        "sta_server_add_netlist": ([H, ctypes.POINTER(StaNetlistDesc), ctypes.POINTER(StaLibrary), _i32,
                                    ctypes.POINTER(_i32)], ctypes.c_int),
        "sta_server_submit": ([H, ctypes.POINTER(StaServerRequest), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "sta_server_poll": ([H, ctypes.POINTER(StaServerCompletion), _i32, ctypes.POINTER(_i32), _i32],
                            ctypes.c_int),
        "sta_server_stats": ([H, _p], ctypes.c_int),
        "sta_server_netlist_bytes": ([H, _i32, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "sta_server_destroy": ([H], None),
        "sta_server_clock": ([], ctypes.c_double),
        "sta_last_error": ([], ctypes.c_char_p),
        "sta_abi_version": ([], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()

# the header's entry points, for the export check
EXPORTS = ("sta_create", "sta_create_multi", "sta_set_positions", "sta_forward", "sta_backward_grad",
           "sta_query_summary", "sta_query_pins", "sta_query_endpoints", "sta_levelize",
           "sta_query_sizes", "sta_query_profile", "sta_stream_wait", "sta_destroy",
           "sta_synchronize", "sta_debug_expire_wait", "sta_autotune", "sta_server_create",
           "sta_server_add_netlist", "sta_server_submit", "sta_server_poll", "sta_server_stats",
           "sta_server_destroy", "sta_server_clock", "sta_server_netlist_bytes", "sta_query_net_rc",
           "sta_ablation_net_rc", "sta_plan_tasks", "sta_query_slack", "sta_measure_latency",
           "sta_last_error", "sta_abi_version", "sta_endpoint_summary_noalloc", "sta_set_active")


def _check(status: int, where: str) -> None:
    if status != STA_OK:
        raise StaError(status, where, (_lib.sta_last_error() or b"").decode())


def sta_last_error() -> str:
    return (_lib.sta_last_error() or b"").decode()


def sta_abi_version() -> int:
    return int(_lib.sta_abi_version())


def sta_measure_latency(nbytes: int, steps: int) -> float:
    """Nanoseconds per dependent load through L2 over a random cycle of nbytes."""
    out = ctypes.c_double()
    _check(_lib.sta_measure_latency(int(nbytes), int(steps), ctypes.byref(out)), "sta_measure_latency")
    return float(out.value)


class _Keep:
    """Contiguous host copies of the description arrays, alive while in use."""

    def __init__(self):
        self.arrs = []

    def __call__(self, a, dt):
        arr = np.ascontiguousarray(a, dtype=dt)
        self.arrs.append(arr)
        return arr.ctypes.data if arr.size else None


def netlist_desc(nl, keep: _Keep) -> StaNetlistDesc:
    return StaNetlistDesc(
        num_pins=int(nl.num_pins), num_nets=int(nl.net_ptr.shape[0] - 1),
        num_cells=int(nl.cell_type.shape[0]),
        net_ptr=keep(nl.net_ptr, np.int32), net_pins=keep(nl.net_pins, np.int32),
        cell_type=keep(nl.cell_type, np.int32), cell_in_ptr=keep(nl.cell_in_ptr, np.int32),
        cell_in_pins=keep(nl.cell_in_pins, np.int32), cell_out_pin=keep(nl.cell_out_pin, np.int32),
        pin_cap=keep(nl.pin_cap, np.float32),
        num_start=int(nl.start_pins.shape[0]), start_pins=keep(nl.start_pins, np.int32),
        start_at=keep(nl.start_at, np.float32), start_slew=keep(nl.start_slew, np.float32),
        num_end=int(nl.end_pins.shape[0]), end_pins=keep(nl.end_pins, np.int32),
        end_rat=keep(nl.end_rat, np.float32),
        r_per_um=float(nl.r_per_um), c_per_um=float(nl.c_per_um),
        end_clock=(None if getattr(nl, "end_clock", None) is None else keep(nl.end_clock, np.int32)))


def library_desc(lib, keep: _Keep) -> StaLibrary:
    return StaLibrary(num_types=int(lib.type_num_arcs.shape[0]),
                      type_num_arcs=keep(lib.type_num_arcs, np.int32),
                      arc_unate=keep(lib.arc_unate, np.int8),
                      slew_index=keep(lib.slew_index, np.float32),
                      load_index=keep(lib.load_index, np.float32),
                      delay_tab=keep(lib.delay_tab, np.float32),
                      slew_tab=keep(lib.slew_tab, np.float32))


def sta_levelize(nl):
    """Host-only levelization: (net_level [N], num_levels, net_order [N], pin_order)."""
    keep = _Keep()
    d = netlist_desc(nl, keep)
    N = d.num_nets
    lv = np.zeros(max(N, 1), np.int32)
    order = np.zeros(max(N, 1), np.int32)
    npins = int(nl.net_ptr[-1]) if N else 0
    pins = np.zeros(max(npins, 1), np.int32)
    nlev = np.zeros(1, np.int32)
    _check(_lib.sta_levelize(ctypes.byref(d), lv.ctypes.data, nlev.ctypes.data, order.ctypes.data,
                             pins.ctypes.data), "sta_levelize")
    return lv[:N], int(nlev[0]), order[:N], pins[:npins]


def sta_create(nl, lib, use_graphs: bool = True, profile: bool = False,
               schedule: int = SCHED_DATAFLOW, num_placements: int = 0, tile_pins: int = 0,
               chunk: int = 0, batch_sweep: int = BATCH_LEVELS, grid_blocks: int = 0) -> int:
    keep = _Keep()
    d = netlist_desc(nl, keep)
    l = library_desc(lib, keep)
    opts = StaOptions(use_graphs=1 if use_graphs else 0, profile=1 if profile else 0,
                      schedule=int(schedule), num_placements=int(num_placements),
                      tile_pins=int(tile_pins), chunk=int(chunk), batch_sweep=int(batch_sweep),
                      grid_blocks=int(grid_blocks))
    h = ctypes.c_void_p()
    _check(_lib.sta_create(ctypes.byref(d), ctypes.byref(l), ctypes.byref(opts), ctypes.byref(h)),
           "sta_create")
    return h.value


def sta_create_multi(nls, lib, use_graphs: bool = True, profile: bool = False, grid_blocks: int = 0) -> int:
    """One handle over the disjoint union of the netlists `nls` (sta_create_multi)."""
    keep = _Keep()
    descs = [netlist_desc(nl, keep) for nl in nls]
    arr = (ctypes.POINTER(StaNetlistDesc) * max(len(descs), 1))(*[ctypes.pointer(d) for d in descs])
    l = library_desc(lib, keep)
    opts = StaOptions(use_graphs=1 if use_graphs else 0, profile=1 if profile else 0, schedule=SCHED_DATAFLOW,
                      grid_blocks=int(grid_blocks))
    h = ctypes.c_void_p()
    _check(_lib.sta_create_multi(arr, len(descs), ctypes.byref(l), ctypes.byref(opts), ctypes.byref(h)),
           "sta_create_multi")
    return h.value


def sta_set_active(h: int, lanes: int) -> None:
    _check(_lib.sta_set_active(h, int(lanes)), "sta_set_active")


def sta_destroy(h: int) -> None:
    _lib.sta_destroy(h)


def sta_set_positions(h: int, xy_ptr: int, on_device: int, stream: int) -> None:
    _check(_lib.sta_set_positions(h, xy_ptr, on_device, stream), "sta_set_positions")


def sta_forward(h: int, flags: int, gamma: float, stream: int) -> None:
    _check(_lib.sta_forward(h, flags, gamma, stream), "sta_forward")


def sta_backward_grad(h: int, w_ptr: int, w_on_device: int, grad_ptr: int, on_device: int,
                      stream: int) -> None:
    _check(_lib.sta_backward_grad(h, w_ptr, w_on_device, grad_ptr, on_device, stream),
           "sta_backward_grad")


def sta_stream_wait(h: int, stream: int) -> None:
    _check(_lib.sta_stream_wait(h, stream), "sta_stream_wait")


def sta_autotune(h: int, tile_pins, chunks, sweeps, reps: int, gamma: float):
    """(best (tile_pins, chunk, sweep), ms table [n_tile, n_chunk, n_sweep])."""
    tp_ = np.ascontiguousarray(tile_pins, np.int32)
    ch = np.ascontiguousarray(chunks, np.int32)
    sw = np.ascontiguousarray(sweeps, np.int32)
    ms = np.zeros((tp_.size, ch.size, sw.size), np.float32)
    best = np.zeros(3, np.int32)
    _check(_lib.sta_autotune(h, tp_.ctypes.data, tp_.size, ch.ctypes.data, ch.size, sw.ctypes.data, sw.size,
                             int(reps), float(gamma), ms.ctypes.data, best.ctypes.data), "sta_autotune")
    return tuple(int(v) for v in best), ms


def sta_synchronize(h: int) -> None:
    _check(_lib.sta_synchronize(h), "sta_synchronize")


def sta_debug_expire_wait(h: int) -> None:
    _check(_lib.sta_debug_expire_wait(h), "sta_debug_expire_wait")


def sta_query_summary(h: int, out_ptr: int, on_device: int, stream: int) -> None:
    _check(_lib.sta_query_summary(h, out_ptr, on_device, stream), "sta_query_summary")


def sta_query_pins(h: int, at: int, slew: int, rat: int, ats: int, slack: int, on_device: int,
                   stream: int) -> None:
    _check(_lib.sta_query_pins(h, at, slew, rat, ats, slack, on_device, stream), "sta_query_pins")


def sta_query_endpoints(h: int, out_ptr: int, on_device: int, stream: int) -> None:
    _check(_lib.sta_query_endpoints(h, out_ptr, on_device, stream), "sta_query_endpoints")


def sta_plan_tasks(nl, lib, tile_pins: int, tile_nets: int, chunk: int):
    """Host-only task plan of a netlist for a task shape (no device use)."""
    keep = _Keep()
    d = netlist_desc(nl, keep)
    l = library_desc(lib, keep)
    out = np.zeros(8, np.int64)
    _check(_lib.sta_plan_tasks(ctypes.byref(d), ctypes.byref(l), int(tile_pins), int(tile_nets), int(chunk),
                               out.ctypes.data), "sta_plan_tasks")
    return dict(zip(("forward_tasks", "backward_tasks", "partials", "chunks", "max_pins", "max_nets",
                     "forward_edges", "split_nets"), out.tolist()))


def sta_query_sizes(h: int):
    out = np.zeros(8, np.int64)
    _check(_lib.sta_query_sizes(h, out.ctypes.data), "sta_query_sizes")
    return dict(zip(("pins", "nets", "levels", "arcs", "endpoints", "warp_tasks", "block_tasks",
                     "device_bytes"), out.tolist()))


def sta_query_profile(h: int, with_times: bool = True):
    """({kind: ms}, {kind: launches}) of the latest step (ms empty if not profiling)."""
    ms = np.zeros(len(PROF_KINDS), np.float64)
    n = np.zeros(len(PROF_KINDS), np.int32)
    _check(_lib.sta_query_profile(h, ms.ctypes.data if with_times else None, n.ctypes.data),
           "sta_query_profile")
    return (dict(zip(PROF_KINDS, ms.tolist())) if with_times else {},
            dict(zip(PROF_KINDS, n.tolist())))


def sta_endpoint_summary_noalloc(at_ptr: int, ats_ptr: int, num_pins: int, end_pins_ptr: int,
                                 end_rat_ptr: int, end_clk_ptr: int, num_end: int, gamma: float,
                                 ep_slack_ptr: int, summary_ptr: int, stream: int) -> None:
    """Allocation-free endpoint summary on device arrays (see include/sta.h)."""
    _check(_lib.sta_endpoint_summary_noalloc(at_ptr, ats_ptr, num_pins, end_pins_ptr, end_rat_ptr,
                                             end_clk_ptr, num_end, gamma, ep_slack_ptr, summary_ptr,
                                             stream),
           "sta_endpoint_summary_noalloc")
