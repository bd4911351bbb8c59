"""Request loop over resident netlists (libsta's sta_server_* entry points).

The loop itself is native (``csrc/serve.cu``): a worker thread admits requests
onto CUDA-stream slots as they free up, keeps netlists resident under a device
memory budget and reports completions with timestamps.  This module only
marshals arguments and keeps request buffers alive until their completion.

    srv = StaServer(slots=4, replicas=2)              # same-netlist requests concurrent on 2 copies
    k = srv.add_netlist(netlist, library)             # copied, made resident
    rid = srv.submit(k, xy_pinned, gradient=True, grad_out=g_pinned)
    done = srv.poll(wait_ms=100)                      # [{"id", "status", "t_submit", ...}]
"""
from __future__ import annotations

import ctypes
from typing import Dict, List, Optional

import numpy as np

from . import _sta


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class StaServer:
    """One server on the current CUDA device (sta_server_create)."""

    def __init__(self, slots: int = 4, sequential: bool = False, budget_bytes: int = 0, merge: int = 0,
                 replicas: int = 0):
        opts = _sta.StaServerOptions(slots=int(slots), sequential=1 if sequential else 0,
                                     budget_bytes=int(budget_bytes), merge=int(merge), replicas=int(replicas))
        h = ctypes.c_void_p()
        _sta._check(_sta._lib.sta_server_create(ctypes.byref(opts), ctypes.byref(h)), "sta_server_create")
        self.h = h.value
        self._keep: Dict[int, tuple] = {}
        self._pins: List[int] = []

    def add_netlist(self, netlist, library, preload: bool = True) -> int:
        keep = _sta._Keep()
        d = _sta.netlist_desc(netlist, keep)
        l = _sta.library_desc(library, keep)
        k = ctypes.c_int32()
        _sta._check(_sta._lib.sta_server_add_netlist(self.h, ctypes.byref(d), ctypes.byref(l),
                                                     1 if preload else 0, ctypes.byref(k)),
                    "sta_server_add_netlist")
        self._pins.append(int(netlist.num_pins))
        return int(k.value)

    def submit(self, netlist: int, xy, gradient: bool = False, gamma: float = 10.0, w=(1.0, 0.0),
               grad_out=None, summary_out: Optional[np.ndarray] = None) -> int:
        """Queue one request.  xy (and grad_out) are host arrays of [num_pins, 2]
        float32 (torch pinned tensors keep the copies asynchronous); they must
        stay unchanged until the request completes."""
        if summary_out is None:
            summary_out = np.zeros(8, np.float64)
        r = _sta.StaServerRequest(netlist=int(netlist), gradient=1 if gradient else 0, gamma=float(gamma),
                                  w_tns=float(w[0]), w_wns=float(w[1]), xy=_ptr(xy),
                                  grad=_ptr(grad_out) if gradient else None, summary=_ptr(summary_out))
        rid = ctypes.c_int64()
        _sta._check(_sta._lib.sta_server_submit(self.h, ctypes.byref(r), ctypes.byref(rid)), "sta_server_submit")
        self._keep[int(rid.value)] = (xy, grad_out, summary_out)
        return int(rid.value)

    def poll(self, max_n: int = 256, wait_ms: int = 0) -> List[dict]:
        buf = (_sta.StaServerCompletion * max(max_n, 1))()
        n = ctypes.c_int32()
        _sta._check(_sta._lib.sta_server_poll(self.h, buf, int(max_n), ctypes.byref(n), int(wait_ms)),
                    "sta_server_poll")
        out = []
        for i in range(n.value):
            c = buf[i]
            xy, g, s = self._keep.pop(int(c.id), (None, None, None))
            out.append({"id": int(c.id), "status": int(c.status), "netlist": int(c.netlist),
                        "t_submit": c.t_submit, "t_start": c.t_start, "t_done": c.t_done, "summary": s,
                        "grad": g, "merged": int(c.merged)})
        return out

    def netlist_bytes(self, netlist: int) -> int:
        b = ctypes.c_int64()
        _sta._check(_sta._lib.sta_server_netlist_bytes(self.h, int(netlist), ctypes.byref(b)),
                    "sta_server_netlist_bytes")
        return int(b.value)

    def stats(self) -> dict:
        o = np.zeros(4, np.int64)
        _sta._check(_sta._lib.sta_server_stats(self.h, o.ctypes.data), "sta_server_stats")
        return {"resident": int(o[0]), "resident_bytes": int(o[1]), "admissions": int(o[2]),
                "evictions": int(o[3])}

    @staticmethod
    def clock() -> float:
        return float(_sta._lib.sta_server_clock())

    def close(self) -> None:
        if getattr(self, "h", None):
            _sta._lib.sta_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
