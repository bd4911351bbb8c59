"""GB300-native levelized, differentiable static timing analysis (Warp-STAR, arXiv 2603.28381).

The whole analysis runs in libsta's sm_103a kernels (``csrc/``), behind the C
ABI of ``include/sta.h``; ``_sta`` binds it with ctypes under the same names.
PyTorch provides device memory, streams and autograd plumbing only.

    eng = StaEngine(netlist, library)        # sta_create: validate, levelize, upload
    eng.set_positions(xy)                    # sta_set_positions
    eng.forward(gamma=10.0)                  # sta_forward: RC, AT/slew, LSE-AT, slack, RAT
    g = eng.backward_grad((1.0, 0.0))        # sta_backward_grad: d(TNS_gamma)/d(x, y)
    tns_g, wns_g = timing_loss(xy_tensor, eng, 10.0)   # autograd wrapper
"""
from __future__ import annotations

from typing import Dict, Optional, Tuple, Union

import numpy as np

from . import _sta
from ._sta import (STA_FWD_LSE, STA_FWD_RAT, SUMMARY_KEYS, StaError, sta_abi_version,
                   sta_last_error, sta_levelize, sta_measure_latency)

__all__ = ["StaEngine", "timing_loss", "TimingLoss", "StaError", "sta_levelize", "STA_FWD_LSE",
           "STA_FWD_RAT", "SUMMARY_KEYS", "sta_abi_version", "sta_last_error", "sta_measure_latency"]


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class StaEngine:
    """One netlist resident on the current CUDA device.

    schedule "batch" analyses ``num_placements`` position sets B at once: every
    per-pin array gains a leading placement dimension ([B, P, 2] positions and
    gradients, [B, E, 2] endpoint slacks, one summary per placement) and the
    loss weights are per placement ([B, 2]).  batch_sweep "lanes" runs the B
    placements as independent lanes of the single-placement sweeps (results
    bit-identical to one placement per handle)."""

    def __init__(self, netlist, library, use_graphs: bool = True, profile: bool = False,
                 schedule: str = "dataflow", num_placements: int = 1, tile_pins: int = 0,
                 chunk: int = 0, batch_sweep: str = "levels", grid_blocks: int = 0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("StaEngine needs a CUDA device (there is no CPU path)")
        torch.cuda.init()
        self.num_pins = int(netlist.num_pins)
        self.num_end = int(netlist.end_pins.shape[0])
        self.device = torch.device("cuda", torch.cuda.current_device())
        sched = {"dataflow": _sta.SCHED_DATAFLOW, "levels": _sta.SCHED_LEVELS,
                 "batch": _sta.SCHED_BATCH}[schedule]
        self.schedule = schedule
        self.batched = schedule == "batch"
        self.B = int(num_placements) if self.batched else 1
        self.h = _sta.sta_create(netlist, library, use_graphs, profile, sched,
                                 self.B if self.batched else 0, tile_pins, chunk,
                                 {"levels": _sta.BATCH_LEVELS, "dataflow": _sta.BATCH_DATAFLOW,
                                  "lanes": _sta.BATCH_LANES, "wide": _sta.BATCH_WIDE}[batch_sweep],
                                 grid_blocks)
        self.sizes = _sta.sta_query_sizes(self.h)
        self.sizes["nets_desc"] = int(netlist.num_nets)
        self.gamma = None
        self.groups = 1

    @classmethod
    def multi(cls, netlists, library, use_graphs: bool = True, profile: bool = False, grid_blocks: int = 0):
        """Many netlists in one handle (sta_create_multi): positions, pins,
        endpoint slacks and gradients are over the netlists concatenated in
        order (`pin_offsets`, `end_offsets`); summary() is a list with one dict
        per netlist and backward_grad takes one weight pair per netlist."""
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("StaEngine needs a CUDA device (there is no CPU path)")
        torch.cuda.init()
        self = cls.__new__(cls)
        nls = list(netlists)
        self.pin_offsets = np.concatenate([[0], np.cumsum([int(n.num_pins) for n in nls])]).astype(np.int64)
        self.end_offsets = np.concatenate([[0], np.cumsum([int(n.end_pins.shape[0]) for n in nls])]).astype(np.int64)
        self.num_pins = int(self.pin_offsets[-1])
        self.num_end = int(self.end_offsets[-1])
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.schedule = "dataflow"
        self.batched = False
        self.B = 1
        self.h = _sta.sta_create_multi(nls, library, use_graphs, profile, grid_blocks)
        self.sizes = _sta.sta_query_sizes(self.h)
        self.sizes["nets_desc"] = int(sum(int(n.num_nets) for n in nls))
        self.gamma = None
        self.groups = len(nls)
        return self

    # -- lifetime --
    def close(self) -> None:
        if getattr(self, "h", None):
            _sta.sta_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls --
    def set_active(self, lanes: int) -> None:
        """batch_sweep "lanes": run placements [0, lanes) from the next
        set_positions on (sta_set_active); arrays then have `lanes` rows."""
        _sta.sta_set_active(self.h, lanes)
        self.B = int(lanes)

    def profile(self, with_times: bool = True):
        """(ms by kernel kind, launches by kind) of the latest step (sta_query_profile)."""
        return _sta.sta_query_profile(self.h, with_times)

    def set_positions(self, xy, stream=None) -> None:
        torch = _torch()
        if isinstance(xy, torch.Tensor):
            t = xy.detach()
            assert t.dtype == torch.float32 and t.is_contiguous() and t.numel() == 2 * self.num_pins * self.B
            _sta.sta_set_positions(self.h, t.data_ptr(), 1 if t.is_cuda else 0, _stream_ptr(stream))
            self._xy_keep = t
        else:
            a = np.ascontiguousarray(np.asarray(xy, np.float32)).reshape(-1)
            assert a.size == 2 * self.num_pins * self.B
            _sta.sta_set_positions(self.h, a.ctypes.data, 0, _stream_ptr(stream))

    def forward(self, gamma: float = 10.0, lse: bool = True, rat: bool = True, stream=None) -> None:
        flags = (STA_FWD_LSE if lse else 0) | (STA_FWD_RAT if rat else 0)
        _sta.sta_forward(self.h, flags, float(gamma), _stream_ptr(stream))
        self.gamma = gamma

    def backward_grad(self, w: Union[Tuple[float, float], "object"] = (1.0, 0.0), out=None,
                      stream=None):
        """d(w[0] TNS_gamma + w[1] WNS_gamma)/d(x, y) as a [P,2] float32 CUDA tensor."""
        torch = _torch()
        shape = (self.B, self.num_pins, 2) if self.batched else (self.num_pins, 2)
        if out is None:
            out = torch.empty(*shape, dtype=torch.float32, device=self.device)
        assert out.dtype == torch.float32 and out.is_contiguous() and out.numel() == 2 * self.num_pins * self.B
        on_dev = 1 if out.is_cuda else 0
        if isinstance(w, torch.Tensor) and w.is_cuda:
            wt = w.detach().to(torch.float32).contiguous()
            _sta.sta_backward_grad(self.h, wt.data_ptr(), 1, out.data_ptr(), on_dev, _stream_ptr(stream))
            self._w_keep = wt
        else:
            wa = np.ascontiguousarray(np.asarray(w, np.float32))
            if self.batched:
                wa = np.ascontiguousarray(np.broadcast_to(wa, (self.B, 2)))
            elif self.groups > 1:  # one pair per netlist
                wa = np.ascontiguousarray(np.broadcast_to(wa, (self.groups, 2)))
            _sta.sta_backward_grad(self.h, wa.ctypes.data, 0, out.data_ptr(), on_dev, _stream_ptr(stream))
        return out

    def stream_wait(self, stream=None) -> None:
        """Order `stream` after all queued work of the handle (sta_stream_wait)."""
        _sta.sta_stream_wait(self.h, _stream_ptr(stream))

    def synchronize(self) -> None:
        """Wait for the handle's sweeps; raises StaError (STA_ERR_TIMEOUT) if a
        bounded dependency wait expired since the last report (sta_synchronize)."""
        _sta.sta_synchronize(self.h)

    def autotune(self, tile_pins=(1, 2, 4), chunks=(8, 16, 32), sweeps=("levels", "dataflow"), reps: int = 3,
                 gamma: float = 10.0):
        """Pick the batched schedule's task shape by timing each candidate on the
        current positions (sta_autotune).  Returns (best, table): best =
        (tile_pins, chunk, sweep name), table = {(tile_pins, chunk, sweep): ms}."""
        names = {"levels": _sta.BATCH_LEVELS, "dataflow": _sta.BATCH_DATAFLOW, "wide": _sta.BATCH_WIDE}
        inv = {v: k for k, v in names.items()}
        best, ms = _sta.sta_autotune(self.h, list(tile_pins), list(chunks), [names[s] for s in sweeps], reps, gamma)
        table = {(int(a), int(c), s): float(ms[i, j, k]) for i, a in enumerate(tile_pins)
                 for j, c in enumerate(chunks) for k, s in enumerate(sweeps)}
        return (best[0], best[1], inv[best[2]]), table

    def net_rc(self) -> Dict[str, np.ndarray]:
        """Net RC results (sta_query_net_rc): load [nets], wdelay / impulse [pins]."""
        load = np.zeros(self.sizes["nets_desc"], np.float32)
        wd = np.zeros(self.num_pins, np.float32)
        im = np.zeros(self.num_pins, np.float32)
        _sta._check(_sta._lib.sta_query_net_rc(self.h, load.ctypes.data if load.size else None,
                                               wd.ctypes.data if wd.size else None,
                                               im.ctypes.data if im.size else None), "sta_query_net_rc")
        return {"load": load, "wdelay": wd, "impulse": im}

    def ablation_net_rc(self, scheme: str = "cte", reps: int = 10) -> float:
        """Mean ms of the net RC of every net in one scheme ("pin" or "cte")."""
        import ctypes as _ct
        ms = _ct.c_float()
        _sta._check(_sta._lib.sta_ablation_net_rc(self.h, {"pin": 0, "cte": 1}[scheme], int(reps), _ct.byref(ms)),
                    "sta_ablation_net_rc")
        return float(ms.value)

    def _debug_expire_wait(self) -> None:
        """Test hook: in the next forward one task's wait never succeeds and
        runs into its budget (sta_debug_expire_wait)."""
        _sta.sta_debug_expire_wait(self.h)

    def summary(self, stream=None):
        """Summary dict (a list of B dicts for the batched schedule, one per
        netlist for a handle of several netlists)."""
        out = np.zeros((max(self.B, self.groups), 8), np.float64)
        _sta.sta_query_summary(self.h, out.ctypes.data, 0, _stream_ptr(stream))
        rows = [dict(zip(SUMMARY_KEYS, r.tolist())) for r in out]
        return rows if (self.batched or self.groups > 1) else rows[0]

    def summary_device(self, out, stream=None):
        _sta.sta_query_summary(self.h, out.data_ptr(), 1, _stream_ptr(stream))
        return out

    def pins(self, at=True, slew=True, rat=True, ats=True, slack=True, stream=None) -> Dict[str, np.ndarray]:
        P = self.num_pins
        res = {}
        bufs = {}
        for k, want, width in (("at", at, 4), ("slew", slew, 4), ("rat", rat, 4), ("ats", ats, 2),
                               ("slack", slack, 2)):
            if want:
                bufs[k] = np.zeros((self.B, P, width) if self.batched else (P, width), np.float32)
        ptr = lambda k: bufs[k].ctypes.data if k in bufs else None
        _sta.sta_query_pins(self.h, ptr("at"), ptr("slew"), ptr("rat"), ptr("ats"), ptr("slack"), 0,
                            _stream_ptr(stream))
        res.update(bufs)
        return res

    def slack(self, pins: bool = True, endpoints: bool = True):
        """sta_query_slack: ({early_wns, early_tns, late_wns, late_tns}, pin slack [P,2] or None,
        endpoint slack [E,2] or None)."""
        wt = np.zeros(4, np.float32)
        ps = np.zeros((max(self.num_pins, 1), 2), np.float32) if pins else None
        es = np.zeros((max(self.num_end, 1), 2), np.float32) if endpoints else None
        _sta._check(_sta._lib.sta_query_slack(self.h, wt.ctypes.data, ps.ctypes.data if ps is not None else None,
                                              es.ctypes.data if es is not None else None), "sta_query_slack")
        return (dict(zip(("wns_early", "tns_early", "wns_late", "tns_late"), wt.tolist())),
                ps[:self.num_pins] if ps is not None else None, es[:self.num_end] if es is not None else None)

    def endpoints(self, stream=None) -> np.ndarray:
        out = np.zeros((self.B, self.num_end, 2), np.float32)
        _sta.sta_query_endpoints(self.h, out.ctypes.data if self.num_end else None, 0, _stream_ptr(stream))
        return out if self.batched else out[0]


class TimingLoss:
    """torch.autograd.Function: xy [P,2] -> (TNS_gamma, WNS_gamma).

    The forward leaves the required-time sweep running on libsta's own stream,
    so the adjoint sweep queued by the backward on the caller's stream overlaps
    it on the GPU (the paper's operation fusion, Section 3.2)."""

    _fn = None

    @classmethod
    def fn(cls):
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, xy, engine, gamma):
                    engine.set_positions(xy)
                    engine.forward(gamma=gamma, lse=True, rat=True)
                    summ = torch.empty(8, dtype=torch.float64, device=xy.device)
                    engine.summary_device(summ)
                    ctx.engine = engine
                    return summ[4].to(torch.float32), summ[5].to(torch.float32)

                @staticmethod
                def backward(ctx, g_tns, g_wns):
                    eng = ctx.engine
                    w = torch.stack([g_tns.reshape(()), g_wns.reshape(())]).to(torch.float32)
                    grad = eng.backward_grad(w)
                    return grad, None, None

            cls._fn = _F
        return cls._fn


def timing_loss(xy, engine: StaEngine, gamma: float = 10.0):
    """(TNS_gamma, WNS_gamma) of positions ``xy`` (a CUDA tensor), differentiable."""
    return TimingLoss.fn().apply(xy, engine, gamma)
