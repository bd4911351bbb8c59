#!/usr/bin/env python
"""Throughput of one differentiable STA step on a ~2.5M-pin netlist.

A step is the whole hot path on one placement: sta_set_positions (device
positions), sta_forward with LSE arrival times and required times, and
sta_backward_grad (d(TNS_gamma + WNS_gamma)/d(x, y)).  The workload is the
superblue4-shaped synthetic netlist (seed 1: ~2.5M pins, 150 levels,
power-law fanout capped at 2000, eight 20k-sink nets, 3000x3000 um, gamma =
10 ps).  The metric is pins per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  On one GPU the default line also carries the metric's
second half as two sub-records, each with its own clock record: `batch` (64
jittered placements of a ~500k-pin netlist per step, against the same
placements one per call) and `serve` (a Poisson stream of 2,000 requests over
ten resident netlists of 20k-3M pins, continuous admission against the plain
one-request-at-a-time loop, measured in a process of its own), and `multi` (64
small netlists in one handle); `--no-sub` leaves them out.  `--impl reference`
times the FP64 CPU oracle (the only reference this method has) on the box's
host cores on the same workload; the default line's `cpu_baseline` gives the
oracle on one core and, as `all_cores`, one concurrent call per host core.

The roofline's `achieved` bytes follow the per-unit algorithmic count (116 P +
16 N + 52 S + 84 A per step, split into forward, required times and
gradient); `per_kind_formula` gives every kernel kind's own reads and writes.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pins/s fwd+grad at 2.5M pins (% HBM roofline); served p50/p99 latency vs plain"
GAMMA = 10.0
WEIGHTS = (1.0, 1.0)
L2_BYTES = 129 * 2 ** 20
FLUSH_BYTES = 512 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--schedule", default="dataflow", choices=["dataflow", "levels"])
    ap.add_argument("--grid-blocks", type=int, default=0,
                    help="blocks of the persistent sweeps (0: every block that fits)")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serve", "multi", "ablation"],
                    help="single: one placement of the ~2.5M-pin netlist per step (the headline); "
                         "batch: 64 placements of a ~500k-pin netlist per step")
    ap.add_argument("--placements", type=int, default=64)
    ap.add_argument("--multi-netlists", type=int, default=64,
                    help="multi: netlists of 5k-40k pins in one handle (sta_create_multi)")
    ap.add_argument("--verbose", action="store_true", help="per-step times on stderr")
    ap.add_argument("--no-sub", action="store_true",
                    help="single: leave out the batched and served sub-records of the default line")
    ap.add_argument("--no-plain", action="store_true", help="batch: skip the one-placement-per-call comparison")
    ap.add_argument("--requests", type=int, default=2000, help="serve: requests in the stream")
    ap.add_argument("--netlists", type=int, default=10, help="serve: distinct netlists (20k to 3M pins)")
    ap.add_argument("--load", type=float, default=0.8,
                    help="serve: arrival rate as a fraction of the plain loop's service rate")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--replicas", type=int, default=2,
                    help="serve: resident copies per netlist in the replicas mode")
    ap.add_argument("--merge", type=int, default=8,
                    help="serve: requests of one netlist merged into one batched launch in the merged mode")
    ap.add_argument("--tile-pins", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--batch-sweep", default="levels", choices=["levels", "dataflow", "wide"])
    ap.add_argument("--clock-nets", type=int, default=0,
                    help="single: propagate the clock over this many clock nets (0: ideal clock)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batch: use --tile-pins/--chunk/--batch-sweep instead of the autotuner's choice")
    return ap.parse_args()


def workload(args):
    import netgen
    return netgen.superblue_like(args.seed, scale=args.scale, clock_nets=args.clock_nets)


def config_of(w, args, extra=None):
    st = w.netlist.stats()
    cfg = {"workload": f"superblue4-shaped synthetic netlist, seed {args.seed}: {st['pins']} pins, "
                       f"{st['nets']} nets, {st['cells']} cells, depth {w.info['depth']}, "
                       f"power-law(2.2) fanout <= 2000 plus 8 x {w.info['huge_sinks']}-sink nets, "
                       f"3000x3000 um, gamma {GAMMA} ps, fwd (AT+LSE+RAT) + gradient, "
                       + (f"clock propagated over {w.info['clock_nets']} clock nets to the flop clock pins"
                          if w.info.get("clock_nets") else "ideal clock"),
           "pins": st["pins"], "nets": st["nets"], "arcs": st["arcs"], "endpoints": st["endpoints"],
           "levels": int(w.info["depth"]) + 1, "gamma_ps": GAMMA}
    if extra:
        cfg.update(extra)
    return cfg


# --------------------------------------------------------------------------
# algorithmic bytes per kernel kind (each array crosses HBM once per producer
# and once per consumer; tables, level pointers and constants not counted)
# --------------------------------------------------------------------------
def algorithmic_bytes(sizes, S, schedule="dataflow", big=(0, 0), clocked=0):
    """Algorithmic bytes of one step by kernel kind.  big = (nets, sinks) of the
    nets of more than 32 pins (their RC runs in a prologue kernel in the
    dataflow schedule; every other net's RC runs inside the forward kernel).
    clocked = endpoints captured by a propagated clock."""
    P, N, A = sizes["pins"], sizes["nets"], sizes["arcs"]

    def rc(n, s):  # pin xy 8 + cap 4 per net pin, (delay, impulse) write 8 per sink, topology + load 8 per net
        return 12 * (n + s) + 8 * s + 8 * n

    fwd = 60 * A + 60 * N + 48 * S
    out = {
        # marking the words the dataflow sweeps poll: overhead, no algorithmic bytes
        "reset": 0,
        # xy gather: index 4P + positions read 8P + write 8P
        "positions": 20 * P,
        # per endpoint: pin 4, constraint 16, AT 16, LSE-AT 8, slack write 8
        "endpoints": 52 * sizes["endpoints"],
        # per sink: RAT 16 + delay 8; per net: RAT write 16 + topology 16; per arc: pin 4,
        # arc delay 16, RAT write 16
        "required": 24 * S + 32 * N + 36 * A,
        "seed": 36 * sizes["endpoints"] if schedule == "levels" else 8,
        # per sink: adjoints 16, late slew 8, (delay, impulse) 8, xy 8, cap 4, pin id 4, grad 8;
        # per net: topology 16, driver slew 8 + LSE-AT 8 + xy 8 + load 4 + grad 8 + pin id 4;
        # per arc: pin id 4, late slew 8, LSE-AT 8, arc delay 16, adjoint writes 16
        "adjoint": 56 * S + 56 * N + 52 * A,
    }
    # forward, per arc: pin id 4, fanin AT+slew+LSE-AT 40, arc delay write 16; per net:
    # topology 16, load 4, driver AT+slew+LSE-AT write 40; per sink: (delay, impulse) 8,
    # AT+slew+LSE-AT write 40
    if schedule == "levels":
        out["net_rc"] = rc(N, S)
        out["forward"] = fwd
    else:
        out["net_rc"] = rc(big[0], big[1])
        out["forward"] = fwd + rc(N - big[0], S - big[1])
    if clocked:
        # per clocked endpoint: the clock pin's AT 16 + the required-time seed write 16; its
        # adjoint seed: clock pin 4, constraint 16, pin 4, clock AT 16, LSE-AT 8, seed write 4;
        # the adjoint sweep reads a seed word per arc
        out["endpoints"] += 32 * clocked
        out["seed"] += 52 * clocked
        out["adjoint"] += 4 * A
    return out


def unit_bytes(sizes, S):
    """Algorithmic bytes of one forward + gradient call by the per-unit
    count (P pins, N nets, S sinks, A arcs; each array crosses HBM once per
    producer and once per consumer):
      forward  xy + cap 12P, net_ptr 4N, arc topology 6A, AT + slew write 32P,
               read by the arcs 32S, load 4N, wire delay 4S, arc delay 16A
      required wire delay 4S, arc delay 16A, topology 4N + 6A, RAT write + read 32P
      gradient LSE-AT write 8P + read 8S, late arc delay 8A, wire delay 4S,
               adjoint write + read 16P, stored partials 32A, xy reread 8P,
               gradient write 8P, d loss / d load 4N
    i.e. 116P + 16N + 52S + 84A per step.  The fused backward sweep carries the
    required times and the gradient."""
    P, N, A = sizes["pins"], sizes["nets"], sizes["arcs"]
    fwd = 44 * P + 8 * N + 36 * S + 22 * A
    req = 32 * P + 4 * N + 4 * S + 22 * A
    grad = 40 * P + 4 * N + 12 * S + 40 * A
    return {"forward": fwd, "required": req, "gradient": grad, "step": fwd + req + grad}


def algorithmic_bytes_batch(sizes, S, B, big=(0, 0)):
    """Algorithmic bytes of one batched step (B placements) by kernel kind.
    Per placement every per-pin value crosses HBM once per producer and once per
    consumer; topology and capacitances are read once per warp of 32 placements."""
    P, N, A, E = sizes["pins"], sizes["nets"], sizes["arcs"], sizes["endpoints"]
    topo = (16 * N + 8 * A + 4 * P) * -(-B // 32)
    # forward, per sink: xy 8, AT+slew+LSE-AT write 40; per net: driver xy 8, load write 4,
    # driver AT+slew+LSE-AT write 40; per arc: fanin AT+slew+LSE-AT 40
    fwd = B * (48 * S + 52 * N + 40 * A) + topo
    # fused backward, per sink: RAT 16, adjoints 16, late slew 8, xy 8, grad write 8; per net:
    # driver LSE-AT 8 + late slew 8 + xy 8 + load 4, RAT write 16, grad write 8; per arc: fanin
    # slews 16, LSE-AT 8, RAT + adjoint writes 32
    bwd = B * (56 * S + 52 * N + 56 * A) + topo
    return {"reset": 0, "positions": 16 * B * P + 4 * P, "net_rc": B * (8 * big[1] + 12 * big[0]),
            "forward": fwd, "endpoints": B * 32 * E + 20 * E, "required": 0, "seed": 8 * B,
            "adjoint": bwd, "output": 16 * B * P + 4 * P}


def measured_traffic(kind, args):
    """DRAM bytes per launch of kernel kind `kind` from the committed ncu capture
    (profiles/dram_traffic_dataflow_superblue_2p5M.json), or None when the
    capture does not apply: another workload or schedule, or kernel sources
    changed since the counters were taken (a digest of the sources is kept)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic_dataflow_superblue_2p5M.json")
    if (args.schedule != "dataflow" or args.scale != 1.0 or args.seed != 1 or args.clock_nets
            or not os.path.exists(path)):
        return None
    with open(path) as f:
        rec = json.load(f)
    h = hashlib.sha256()
    for name in rec["sources"]:
        with open(os.path.join(ROOT, name), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != rec["sources_sha256"]:
        return None
    v = rec["per_launch_bytes"].get(kind)
    return None if v is None else float(v)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = gpu_index
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(seconds, dist, device):
    """The job's time: the slowest rank's.  Ranks are independent replicas (no
    data-path collective); this scalar is the only value they exchange."""
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world * units_per_rank / seconds


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# --------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# --------------------------------------------------------------------------
def cpu_model():
    """The host CPU's model name (lscpu / /proc/cpuinfo), for the CPU baseline."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def time_oracle(w, budget_s=20.0, max_calls=5):
    import oracle
    oracle.build()
    t_calls = []
    t0 = time.perf_counter()
    while len(t_calls) < max_calls:
        t = time.perf_counter()
        oracle.sta(w.netlist, w.library, w.xy, GAMMA, *WEIGHTS, want={"grad"})
        t_calls.append(time.perf_counter() - t)
        if time.perf_counter() - t0 > budget_s:
            break
    return t_calls


def time_oracle_all_cores(w, threads):
    """The oracle as it stands on every host core at once: `threads` concurrent
    calls on the same netlist (the C oracle keeps no shared state, and ctypes
    releases the interpreter lock during a call).  Returns the wall time."""
    import concurrent.futures

    import oracle
    oracle.build()
    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        t = time.perf_counter()
        list(ex.map(lambda _: oracle.sta(w.netlist, w.library, w.xy, GAMMA, *WEIGHTS, want={"grad"}),
                    range(threads)))
        return time.perf_counter() - t


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(args)
    import oracle
    oracle.build()
    P = w.netlist.num_pins
    sample = w
    sample_note = "the whole netlist per step"
    # bound the run: the whole --steps/--warmup run should end within a few minutes
    t = time.perf_counter()
    oracle.sta(w.netlist, w.library, w.xy, GAMMA, *WEIGHTS, want={"grad"})
    t_full = time.perf_counter() - t
    if t_full * (args.steps + args.warmup) > 200.0:
        import netgen
        scale = max(0.002, 200.0 / ((args.steps + args.warmup) * t_full) * args.scale * 0.8)
        sample = netgen.superblue_like(args.seed, scale=scale, clock_nets=args.clock_nets)
        sample_note = (f"a {sample.netlist.num_pins}-pin netlist from the same generator "
                       f"(scale {scale:.3g}) per step, to bound the run")
    Ps = sample.netlist.num_pins
    for _ in range(max(0, args.warmup - 1)):
        oracle.sta(sample.netlist, sample.library, sample.xy, GAMMA, *WEIGHTS, want={"grad"})
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.sta(sample.netlist, sample.library, sample.xy, GAMMA, *WEIGHTS, want={"grad"})
        times.append(time.perf_counter() - t)
    tot = sum(times)
    value = Ps * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pins/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, args, {"reference": "FP64 CPU oracle (oracle/sta_oracle.c), "
                                                       "single thread, as it stands",
                                          "levels": int(oracle.levels(w.netlist).max()) + 1}),
            "cpu_baseline": {"value": value, "unit": "pins/s", "cores": 1, "kind": "oracle",
                             "cpu_model": cpu_model(), "host_cores": os.cpu_count(), "sample": sample_note},
            "e2e": {"value": value, "unit": "pins/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import paper_2603_28381_gb300 as sta

    w = workload(args)
    nl = w.netlist
    P = nl.num_pins
    S = int(nl.net_ptr[-1]) - nl.num_nets
    dev = torch.device("cuda", local)
    xy = torch.as_tensor(w.xy).to(dev)
    wts = torch.tensor(WEIGHTS, dtype=torch.float32, device=dev)
    grad = torch.empty(P, 2, dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(eng, out=grad):
        eng.set_positions(xy)
        eng.forward(gamma=GAMMA, lse=True, rat=True)
        eng.backward_grad(wts, out=out)
        eng.stream_wait()      # the step ends when the required-time sweep has ended too

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    eng = sta.StaEngine(nl, w.library, schedule=args.schedule, grid_blocks=args.grid_blocks)
    for _ in range(args.warmup):
        step(eng)
    cur = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = Clocks(local)
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()          # evict L2 (512 MB > 129 MB) between steps, outside the events
        ev[k][0].record(cur)
        step(eng)
        ev[k][1].record(cur)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    if args.verbose:
        print("step ms:", " ".join(f"{m:.3f}" for m in ms), file=sys.stderr)
    total_s = max_over_ranks(sum(ms) / 1e3, dist, dev)
    value = job_throughput(P * args.steps, world, total_s)
    _, launches = eng.profile(with_times=False)
    launches_per_step = int(sum(launches.values()))

    # end to end through the public API with host buffers: pinned positions in,
    # gradient and summary out, every step
    e2e = None
    if not args.no_e2e:
        xy_h = torch.as_tensor(w.xy).pin_memory()
        g_h = torch.empty(P, 2, dtype=torch.float32).pin_memory()
        for _ in range(2):
            eng.set_positions(xy_h)
            eng.forward(gamma=GAMMA)
            eng.backward_grad(WEIGHTS, out=g_h)
            eng.summary()
        barrier()
        t = time.perf_counter()
        for _ in range(args.steps):
            eng.set_positions(xy_h)
            eng.forward(gamma=GAMMA)
            eng.backward_grad(WEIGHTS, out=g_h)
            eng.summary()
        barrier()
        te = max_over_ranks(time.perf_counter() - t, dist, dev)
        e2e = {"value": job_throughput(P * args.steps, world, te), "unit": "pins/s",
               "h2d_bytes_per_step": 8 * P, "d2h_bytes_per_step": 8 * P + 64}
    eng.close()

    # roofline of the dominant kernel kind, from CUDA events around every launch of
    # the same steps (a handle with StaOptions.profile = 1)
    prof_eng = sta.StaEngine(nl, w.library, profile=True, schedule=args.schedule, grid_blocks=args.grid_blocks)
    for _ in range(2):
        step(prof_eng)
    acc = {}
    nprof = min(args.steps, 10)
    for _ in range(nprof):
        flush.zero_()
        step(prof_eng)
        msk, launches = prof_eng.profile()
        for k, v in msk.items():
            acc[k] = acc.get(k, 0.0) + v / nprof
    prof_eng.close()
    sizes = dict(pins=P, nets=prof_eng.sizes["nets"], arcs=prof_eng.sizes["arcs"],
                 endpoints=prof_eng.sizes["endpoints"])
    fan = np.diff(nl.net_ptr)
    clocked = 0 if nl.end_clock is None else int((nl.end_clock >= 0).sum())
    abytes = algorithmic_bytes(sizes, S, args.schedule,
                               big=(int((fan > 32).sum()), int((fan[fan > 32] - 1).sum())), clocked=clocked)
    if launches.get("required", 1) == 0:  # required times ran inside the adjoint sweep
        abytes["adjoint"] += abytes["required"]
        abytes["required"] = 0
    dom = max(acc, key=lambda k: acc[k])
    peak, peak_src = load_peaks()
    # the dominant kernel's algorithmic bytes by the per-unit count: the
    # forward sweep the forward's, the backward sweep the required times' and
    # (adjoint) the gradient's
    sb = unit_bytes(sizes, S)
    sweep_bytes = {"forward": sb["forward"], "required": sb["required"],
                   "adjoint": sb["gradient"] + (sb["required"] if launches.get("required", 1) == 0 else 0)}
    dom_bytes = sweep_bytes.get(dom, abytes[dom])
    achieved = dom_bytes / (acc[dom] / 1e3) / 1e9 if acc[dom] > 0 else 0.0
    traffic = measured_traffic(dom, args)
    step_s = total_s / args.steps
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                "traffic": None if traffic is None else float(traffic),
                "bytes_per_launch": int(dom_bytes), "bytes_formula": "per-unit count 116P + 16N + 52S + 84A per step",
                "launches_per_step": launches[dom],
                "avg_launch_us": 1e3 * acc[dom] / max(launches[dom], 1),
                "ms_by_kind": {k: round(v, 4) for k, v in acc.items()},
                "step_algorithmic_bytes": int(sb["step"]),
                "step_frac": sb["step"] / step_s / 1e9 / peak,
                "per_kind_formula": {
                    "how": "every kernel kind's own reads and writes (bench.py algorithmic_bytes), "
                           "including positions, net RC of large nets and endpoints",
                    "dominant_frac": (abytes[dom] / (acc[dom] / 1e3) / 1e9 / peak) if acc[dom] > 0 else 0.0,
                    "step_algorithmic_bytes": int(sum(abytes.values())),
                    "step_frac": sum(abytes.values()) / step_s / 1e9 / peak}}
    # depth floor: the forward and the fused backward sweep each need at least one
    # dependent round trip through L2 per level (a task reads what its producers stored)
    lat_l2 = sta.sta_measure_latency(32 << 20, 20000)
    lat_dram = sta.sta_measure_latency(512 << 20, 5000)
    levels = int(prof_eng.sizes["levels"])
    floor_ms = 2 * levels * lat_l2 / 1e6
    sweeps_ms = acc.get("forward", 0.0) + acc.get("adjoint", 0.0) + acc.get("required", 0.0)
    roofline["depth_floor"] = {"levels": levels, "dependent_steps": 2 * levels,
                               "l2_dependent_load_ns": round(lat_l2, 1),
                               "dram_dependent_load_ns": round(lat_dram, 1),
                               "floor_ms": round(floor_ms, 4),
                               "sweeps_ms": round(sweeps_ms, 4),
                               "sweeps_over_floor": round(sweeps_ms / floor_ms, 2)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        tc = time_oracle(w, budget_s=20.0, max_calls=8)
        cpu = {"value": P / (sum(tc) / len(tc)), "unit": "pins/s", "cores": 1, "kind": "oracle",
               "cpu_model": cpu_model(), "host_cores": os.cpu_count(),
               "sample": f"{len(tc)} full FP64 oracle calls (forward, required times, gradient) "
                         f"on the same {P}-pin netlist, single thread (mean)"}
        nt = max(1, os.cpu_count() or 1)
        ta = time_oracle_all_cores(w, nt)
        cpu["all_cores"] = {"value": nt * P / ta, "unit": "pins/s", "cores": nt,
                            "sample": f"{nt} concurrent full oracle calls on the same netlist, one per host "
                                      f"core (threads), wall time {ta:.2f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pins/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_of(w, args, {"levels": int(prof_eng.sizes["levels"]),
                                              "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                              "schedule": args.schedule,
                                              "l2": "flushed between steps (512 MB write)",
                                              "wall_s": round(t_wall, 3)}),
                "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
                "roofline": roofline, "cpu_baseline": cpu, "clocks": clk}
        if world == 1 and not args.no_sub:
            # the metric's second half: batched placements and the served stream,
            # each measured here with its own clock record
            import copy
            ba = copy.copy(args)
            ba.steps, ba.warmup, ba.scale = min(args.steps, 20), max(3, min(args.warmup, 5)), 1.0
            line["batch"] = run_batch(ba, emit=False)
            line["serve"] = serve_own_process(args)
            ma = copy.copy(args)
            ma.steps, ma.warmup = min(args.steps, 20), max(3, min(args.warmup, 5))
            line["multi"] = run_multi(ma, emit=False)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# batched placements: B position sets of one netlist per step
# --------------------------------------------------------------------------
def batch_workload(args):
    import netgen
    w = netgen.superblue_like(args.seed + 1, scale=0.2 * args.scale, depth=100)
    xyb = netgen.jitter_positions(w.xy, args.placements, 5.0, args.seed)
    return w, xyb


def run_batch(args, emit=True):
    import torch

    import paper_2603_28381_gb300 as sta
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    w, xyb_np = batch_workload(args)
    nl = w.netlist
    P, B = nl.num_pins, args.placements
    S = int(nl.net_ptr[-1]) - nl.num_nets
    dev = torch.device("cuda", local)
    xyb = torch.as_tensor(xyb_np).to(dev)
    W = torch.ones(B, 2, dtype=torch.float32, device=dev)
    grad = torch.empty(B, P, 2, dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(eng):
        eng.set_positions(xyb)
        eng.forward(gamma=GAMMA, lse=True, rat=True)
        eng.backward_grad(W, out=grad)
        eng.stream_wait()

    def timed(eng, fn, steps):
        for _ in range(args.warmup):
            fn(eng)
        cur = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(cur)
            fn(eng)
            ev[k][1].record(cur)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        if args.verbose:
            print("step ms:", " ".join(f"{m:.3f}" for m in ms), file=sys.stderr)
        return sum(ms) / 1e3

    eng = sta.StaEngine(nl, w.library, schedule="batch", num_placements=B, tile_pins=args.tile_pins,
                        chunk=args.chunk, batch_sweep=args.batch_sweep)
    tune = None
    if not args.no_autotune:  # untimed: pick the task shape on this workload
        eng.set_positions(xyb)
        best, table = eng.autotune(tile_pins=(1, 2, 4), chunks=(8, 16, 32), sweeps=("levels", "dataflow", "wide"),
                                   reps=3, gamma=GAMMA)
        args.tile_pins, args.chunk, args.batch_sweep = best
        tune = {"best": {"tile_pins": best[0], "chunk": best[1], "batch_sweep": best[2]},
                "ms": {f"{a}/{c}/{s}": round(v, 3) for (a, c, s), v in table.items()}}
    clocks = Clocks(local)
    total_s = timed(eng, step, args.steps)
    clk = clocks.stop()
    value = B * P * args.steps / total_s
    _, launches = eng.profile(with_times=False)
    eng.close()

    # the same placements as lanes of the single-placement sweeps (results equal
    # to one placement per handle), and their latency for small groups
    lanes = {}
    ln = sta.StaEngine(nl, w.library, schedule="batch", num_placements=B, batch_sweep="lanes")
    lanes_s = timed(ln, step, max(1, min(args.steps, 10)))
    lanes["ms_per_step"] = 1e3 * lanes_s / max(1, min(args.steps, 10))
    lanes["value"] = B * P / (lanes["ms_per_step"] / 1e3)
    lanes["small_groups_ms"] = {}
    for k in (1, 2, 4, 8):
        if k > B:
            break
        ln.set_active(k)
        xk = xyb[:k].contiguous()
        wk = W[:k].contiguous()
        gk = torch.empty(k, P, 2, dtype=torch.float32, device=dev)

        def stepk(e):
            e.set_positions(xk)
            e.forward(gamma=GAMMA, lse=True, rat=True)
            e.backward_grad(wk, out=gk)
            e.stream_wait()
        lanes["small_groups_ms"][str(k)] = round(1e3 * timed(ln, stepk, 5) / 5, 4)
    ln.close()

    # the plain path on the same placements: one placement per call, one after another
    one = sta.StaEngine(nl, w.library, schedule="dataflow")
    xs = [xyb[b].contiguous() for b in range(B)]
    g1 = torch.empty(P, 2, dtype=torch.float32, device=dev)
    w1 = torch.ones(2, dtype=torch.float32, device=dev)

    def plain(e):
        for b in range(B):
            e.set_positions(xs[b])
            e.forward(gamma=GAMMA, lse=True, rat=True)
            e.backward_grad(w1, out=g1)
        e.stream_wait()

    plain_steps = max(1, min(args.steps, 5))
    plain_s = timed(one, plain, plain_steps) if not args.no_plain else float("nan")
    one.close()
    plain_value = B * P * plain_steps / plain_s

    prof = sta.StaEngine(nl, w.library, schedule="batch", num_placements=B, profile=True,
                         tile_pins=args.tile_pins, chunk=args.chunk, batch_sweep=args.batch_sweep)
    for _ in range(2):
        step(prof)
    acc = {}
    nprof = min(args.steps, 5)
    for _ in range(nprof):
        flush.zero_()
        step(prof)
        msk, _ = prof.profile()
        for k, v in msk.items():
            acc[k] = acc.get(k, 0.0) + v / nprof
    sizes = dict(pins=P, nets=prof.sizes["nets"], arcs=prof.sizes["arcs"], endpoints=prof.sizes["endpoints"])
    prof.close()
    chunk = args.chunk or 16
    fan = np.diff(nl.net_ptr)
    bigm = fan > chunk + 1
    abytes = algorithmic_bytes_batch(sizes, S, B, big=(int(bigm.sum()), int((fan[bigm] - 1).sum())))
    peak, peak_src = load_peaks()
    dom = max(acc, key=lambda k: acc[k])
    achieved = abytes[dom] / (acc[dom] / 1e3) / 1e9 if acc[dom] > 0 else 0.0
    st = nl.stats()
    line = {"metric": "pins/s fwd+grad, batched placements", "value": value, "unit": "pins/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{B} placements (base + N(0, 5 um) jitter) of a {st['pins']}-pin "
                                   f"synthetic netlist, depth {w.info['depth']}, gamma {GAMMA} ps, "
                                   f"fwd (AT+LSE+RAT) + gradient per placement",
                       "pins": st["pins"], "placements": B, "tile_pins": args.tile_pins or 4,
                       "chunk": chunk, "batch_sweep": args.batch_sweep, "autotune": tune,
                       "l2": "flushed between steps (512 MB write)"},
            "plain": {"value": plain_value, "unit": "pins/s",
                      "how": "the same placements one per call on the single-placement dataflow schedule",
                      "ms_per_step": 1e3 * plain_s / plain_steps},
            "speedup_vs_plain": value / plain_value,
            "lanes": {"how": "the same placements as lanes of the single-placement sweeps in one launch "
                             "(STA_BATCH_LANES; results bit-identical to one placement per handle); "
                             "small_groups_ms: a call on the first 1, 2, 4, 8 placements",
                      **lanes},
            "gpu_launches": int(sum(launches.values())) * args.steps,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src, "traffic": None,
                         "ms_by_kind": {k: round(v, 4) for k, v in acc.items()},
                         "step_algorithmic_bytes": int(sum(abytes.values())),
                         "step_frac": sum(abytes.values()) / (total_s / args.steps) / 1e9 / peak},
            "clocks": clk}
    if emit:
        print(json.dumps(line), flush=True)
    return line


# --------------------------------------------------------------------------
# serving: a Poisson stream of requests over resident netlists of 20k-3M pins
# --------------------------------------------------------------------------
def serve_workload(args):
    import netgen
    rng = np.random.default_rng(args.seed + 17)
    lo, hi = np.log(20e3), np.log(3e6)
    pins = np.exp(np.linspace(lo, hi, args.netlists))  # log-spaced sizes, in random order
    rng.shuffle(pins)
    designs = []
    for i, p in enumerate(pins):
        depth = int(np.clip(30 + 120 * (np.log(p) - lo) / (hi - lo), 30, 150))
        designs.append(netgen.superblue_like(100 + i, scale=float(p / 2.5e6), depth=depth))
    return designs


def serve_own_process(args):
    """The serving record of the default line, measured in a process of its own
    (a fresh interpreter and CUDA context, as a serving process would have, with
    none of the earlier records' objects): `bench.py --workload serve` with the
    same stream arguments."""
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", "serve", "--seed", str(args.seed),
           "--requests", str(args.requests), "--netlists", str(args.netlists), "--load", str(args.load),
           "--slots", str(args.slots), "--replicas", str(args.replicas), "--merge", str(args.merge)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"serving record failed ({r.returncode}): {r.stderr[-2000:]}")
    rec = json.loads(r.stdout.strip().splitlines()[-1])
    rec["process"] = "own process: bench.py --workload serve with the same stream arguments"
    return rec


def run_serve(args, emit=True):
    import torch

    import netgen
    from paper_2603_28381_gb300.serving import StaServer
    designs = serve_workload(args)
    rng = np.random.default_rng(args.seed + 29)
    R = args.requests
    which = rng.integers(0, len(designs), R)
    grad = rng.random(R) < 0.3
    # two position sets per netlist (pinned), alternated: every request uploads a
    # full position array; gradients go to one pinned buffer per netlist
    xs = [[torch.from_numpy(netgen.jitter_positions(w.xy, 1, 5.0, 7 + j)[0]).pin_memory() for j in range(2)]
          for w in designs]
    gs = [torch.zeros(w.netlist.num_pins, 2).pin_memory() for w in designs]
    pins = np.array([w.netlist.num_pins for w in designs])

    def play(server, ids, arrivals):
        """Submit at the arrival times, collect completions; latencies in ms and
        how many requests ran in each request's launch."""
        done, lat, t_first, t_last = 0, np.zeros(R), None, 0.0
        merged = np.ones(R)
        rid_of = {}
        t0 = StaServer.clock() + 0.05
        i = 0
        while done < R:
            now = StaServer.clock()
            while i < R and now >= t0 + arrivals[i]:
                k = int(which[i])
                rid = server.submit(ids[k], xs[k][i & 1], gradient=bool(grad[i]), gamma=GAMMA, w=WEIGHTS,
                                    grad_out=gs[k])
                rid_of[rid] = i
                i += 1
            wait = 0 if i < R else 50
            for c in server.poll(wait_ms=wait):
                j = rid_of.pop(c["id"])
                if c["status"] != 0:
                    raise RuntimeError(f"request {j} failed with status {c['status']}")
                lat[j] = (c["t_done"] - (t0 + arrivals[j])) * 1e3
                merged[j] = c.get("merged", 1)
                t_last = max(t_last, c["t_done"])
                done += 1
            if i < R and wait == 0:
                # until the next arrival: a short sleep while it is more than a
                # millisecond away, then a spin on the clock (a late wake-up of the
                # load generator would count as latency; completions carry the
                # server's own stamps, so polling them later changes nothing)
                dt = t0 + arrivals[i] - StaServer.clock()
                if dt > 1e-3:
                    time.sleep(min(dt - 8e-4, 5e-4))
                else:
                    while StaServer.clock() < t0 + arrivals[i]:
                        pass
        span = t_last - t0
        return lat, span, merged

    # service times of the plain loop, request by request, to set the arrival rate
    calib = StaServer(sequential=True)
    ids = [calib.add_netlist(w.netlist, w.library) for w in designs]
    cal = []
    for k in range(len(designs)):
        for gflag in (False, True):
            for _ in range(3):
                rid = calib.submit(ids[k], xs[k][0], gradient=gflag, gamma=GAMMA, w=WEIGHTS, grad_out=gs[k])
                c = []
                while not c:
                    c = calib.poll(wait_ms=100)
                cal.append((k, gflag, c[0]["t_done"] - c[0]["t_start"]))
    calib.close()
    svc = {}
    for k, gflag, t in cal:
        svc.setdefault((k, gflag), []).append(t)
    mean_svc = float(np.mean([np.median(svc[(int(which[i]), bool(grad[i]))]) for i in range(R)]))
    rate = args.load / mean_svc
    arrivals = np.cumsum(rng.exponential(1.0 / rate, R))

    out = {}
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", 0)))
    sizes = None
    for mode in ("plain", "continuous", "replicas", "merged", "budget_bound"):
        budget = 0  # the server's default (150 GiB): every netlist stays resident
        if mode == "budget_bound":
            # half of what all netlists hold resident, and room for the largest:
            # idle netlists are evicted in LRU order and brought back at rate
            # (device allocation and upload from the layout built at registration)
            budget = int(max(0.5 * sum(sizes), 1.1 * max(sizes)))
        srv = StaServer(sequential=(mode == "plain"), slots=args.slots,
                        merge=args.merge if mode == "merged" else 0,
                        replicas=args.replicas if mode == "replicas" else 0, budget_bytes=budget)
        ids = [srv.add_netlist(w.netlist, w.library, preload=(mode != "budget_bound")) for w in designs]
        stats0 = srv.stats()
        if mode == "continuous":
            sizes = [srv.netlist_bytes(k) for k in ids]
        # the client loop is the load generator, not the system measured: no
        # collector pass of the process's older objects inside it (in the default
        # line those include the earlier records' netlists)
        gc.collect()
        gc.freeze()
        gc.disable()
        try:
            lat, span, merged = play(srv, ids, arrivals)
        finally:
            gc.enable()
            gc.unfreeze()
        st = srv.stats()
        srv.close()
        out[mode] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_ms": float(lat.mean()), "requests_per_s": R / span,
                     "pins_per_s": float(pins[which].sum() / span), "span_s": span,
                     "resident_netlists": stats0["resident"], "resident_bytes": stats0["resident_bytes"],
                     "evictions": st["evictions"]}
        if mode == "replicas":
            out[mode]["replicas"] = args.replicas
            out[mode]["copies_made"] = st["admissions"]
        if mode == "budget_bound":
            out[mode]["budget_bytes"] = budget
            out[mode]["all_resident_bytes"] = int(sum(sizes))
            out[mode]["admissions"] = st["admissions"]
        if mode == "merged":
            out[mode]["merge_lanes"] = args.merge
            out[mode]["requests_merged"] = float((merged > 1).mean())
            out[mode]["mean_requests_per_launch"] = float(R / np.sum(1.0 / merged))
    clk = clocks.stop()
    line = {"metric": "served p50/p99 latency vs plain", "value": out["continuous"]["p99_ms"], "unit": "ms p99",
            "n_gpus": 1, "steps": R, "warmup": 0, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{R} Poisson requests ({args.load:.0%} of the plain loop's capacity) over "
                                   f"{len(designs)} resident netlists of {int(pins.min())}-{int(pins.max())} "
                                   f"pins (log-spaced sizes), 70% forward (AT, LSE-AT, required times, "
                                   f"slacks), 30% forward + gradient, new positions per request",
                       "netlist_pins": pins.tolist(), "arrival_rate_per_s": rate,
                       "mean_plain_service_ms": mean_svc * 1e3, "slots": args.slots,
                       "budget": "150 GiB"},
            "continuous": out["continuous"], "plain": out["plain"], "replicas": out["replicas"],
            "merged": out["merged"], "budget_bound": out["budget_bound"],
            "p99_speedup_vs_plain": out["plain"]["p99_ms"] / out["continuous"]["p99_ms"],
            "p50_speedup_vs_plain": out["plain"]["p50_ms"] / out["continuous"]["p50_ms"],
            "replicas_p99_speedup_vs_plain": out["plain"]["p99_ms"] / out["replicas"]["p99_ms"],
            "merged_p99_speedup_vs_plain": out["plain"]["p99_ms"] / out["merged"]["p99_ms"],
            "clocks": clk}
    if emit:
        print(json.dumps(line), flush=True)
    return line


# --------------------------------------------------------------------------
# many small netlists per step in one handle (sta_create_multi)
# --------------------------------------------------------------------------
def multi_workload(args):
    """args.multi_netlists superblue-shaped netlists of log-uniform 5k-40k pins
    and depth 20-150, over the first one's library (every one has the same
    type structure)."""
    import netgen
    rng = np.random.default_rng(args.seed + 61)
    ws = []
    for k in range(args.multi_netlists):
        sc = float(np.exp(rng.uniform(np.log(0.002), np.log(0.016))))
        ws.append(netgen.superblue_like(args.seed + 100 + k, scale=sc, depth=int(rng.integers(20, 151))))
    return ws


def run_multi(args, emit=True):
    import torch

    import paper_2603_28381_gb300 as sta
    ws = multi_workload(args)
    lib = ws[0].library
    nls = [w.netlist for w in ws]
    K = len(nls)
    pins = np.array([nl.num_pins for nl in nls])
    P = int(pins.sum())
    dev = torch.device("cuda", 0)
    xy = torch.as_tensor(np.concatenate([w.xy for w in ws]).astype(np.float32)).to(dev)
    W = torch.ones(K, 2, dtype=torch.float32, device=dev)
    grad = torch.empty(P, 2, dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        cur = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(cur)
            fn()
            ev[k][1].record(cur)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    eng = sta.StaEngine.multi(nls, lib)

    def step():
        eng.set_positions(xy)
        eng.forward(gamma=GAMMA, lse=True, rat=True)
        eng.backward_grad(W, out=grad)
        eng.stream_wait()

    clocks = Clocks(0)
    total_s = timed(step, args.steps)
    clk = clocks.stop()
    _, launches = eng.profile(with_times=False)
    eng.close()

    # the plain path: one handle per netlist, called one after another
    ones = [sta.StaEngine(nl, lib) for nl in nls]
    offs = np.concatenate([[0], np.cumsum(pins)])

    def plain():
        for k, e in enumerate(ones):
            e.set_positions(xy[offs[k]:offs[k + 1]])
            e.forward(gamma=GAMMA, lse=True, rat=True)
            e.backward_grad(W[k], out=grad[offs[k]:offs[k + 1]])
        for e in ones:
            e.stream_wait()

    plain_steps = max(1, min(args.steps, 5))
    plain_s = timed(plain, plain_steps)
    for e in ones:
        e.close()
    sb = 0
    for nl in nls:
        st = nl.stats()
        sb += unit_bytes({"pins": st["pins"], "nets": st["nets"], "arcs": st["arcs"]},
                           int(nl.net_ptr[-1]) - st["nets"])["step"]
    peak, peak_src = load_peaks()
    value = P * args.steps / total_s
    plain_value = P * plain_steps / plain_s
    depths = [int(w.info["depth"]) for w in ws]
    line = {"metric": "pins/s fwd+grad, many netlists in one launch", "value": value, "unit": "pins/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{K} superblue-shaped synthetic netlists of {int(pins.min())}-{int(pins.max())} "
                                   f"pins (log-uniform), depth {min(depths)}-{max(depths)}, {P} pins in all, one "
                                   f"library, gamma {GAMMA} ps, fwd (AT+LSE+RAT) + gradient of each netlist's "
                                   f"own loss, in one handle (sta_create_multi)",
                       "netlists": K, "pins": P, "l2": "flushed between steps (512 MB write)"},
            "plain": {"value": plain_value, "unit": "pins/s", "ms_per_step": 1e3 * plain_s / plain_steps,
                      "how": "one handle per netlist, called one after another on one stream"},
            "speedup_vs_plain": value / plain_value,
            "gpu_launches": int(sum(launches.values())) * args.steps,
            "roofline": {"bound": "hbm", "step_algorithmic_bytes": int(sb), "peak": peak, "unit": "GB/s",
                         "peak_source": peak_src,
                         "step_frac": sb / (total_s / args.steps) / 1e9 / peak},
            "clocks": clk}
    if emit:
        print(json.dumps(line), flush=True)
    return line


# --------------------------------------------------------------------------
# ablations on the 2.5M-pin workload: CTE vs pin-based net RC (Algorithm 2),
# forward only vs sequential vs fused gradient (the Diff / Diff+Fusion ratio)
# --------------------------------------------------------------------------
def run_ablation(args):
    import torch

    import paper_2603_28381_gb300 as sta
    from paper_2603_28381_gb300 import _sta
    w = workload(args)
    nl = w.netlist
    P = nl.num_pins
    dev = torch.device("cuda", 0)
    xy = torch.as_tensor(w.xy).to(dev)
    wts = torch.tensor(WEIGHTS, dtype=torch.float32, device=dev)
    grad = torch.empty(P, 2, dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    eng = sta.StaEngine(nl, w.library)
    eng.set_positions(xy)
    rc = {s: eng.ablation_net_rc(s, reps=20) for s in ("pin", "cte", "pin", "cte")}  # second pass counts
    stream = sta._stream_ptr(None)
    fl = _sta.STA_FWD_LSE | _sta.STA_FWD_RAT

    def fwd_only():
        eng.set_positions(xy)
        _sta.sta_forward(eng.h, fl | _sta.STA_FWD_RAT_EAGER, GAMMA, stream)
        eng.stream_wait()

    def sequential():
        eng.set_positions(xy)
        _sta.sta_forward(eng.h, fl | _sta.STA_FWD_RAT_EAGER, GAMMA, stream)
        eng.backward_grad(wts, out=grad)
        eng.stream_wait()

    def fused():
        eng.set_positions(xy)
        _sta.sta_forward(eng.h, fl, GAMMA, stream)
        eng.backward_grad(wts, out=grad)
        eng.stream_wait()

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        cur = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(cur)
            fn()
            ev[k][1].record(cur)
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in ev]))

    t = {name: timed(fn, args.steps) for name, fn in (("forward", fwd_only), ("sequential", sequential),
                                                       ("fused", fused))}
    eng.close()
    line = {"metric": "ablations: CTE vs pin-based net RC; gradient sequential vs fused", "unit": "ms",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "f32", "data": "synthetic",
            "config": config_of(w, args, {"timing": "median of CUDA-event times per call, L2 flushed between"}),
            "net_rc_ms": {"pin_based": rc["pin"], "cte": rc["cte"], "cte_over_pin": rc["cte"] / rc["pin"]},
            "step_ms": t,
            "sequential_over_forward": t["sequential"] / t["forward"],
            "fused_over_forward": t["fused"] / t["forward"],
            "paper_context": "Table 3 (RTX 4090, superblue4): Diff 133%, Diff+Fusion 116% of the STA time"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "multi":
        run_multi(args)
    elif args.workload == "ablation":
        run_ablation(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
