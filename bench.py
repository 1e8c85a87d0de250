"""Benchmark of the PeriDEM hot path on one GB300 (replicas per GPU under torchrun).

A step is one velocity-Verlet step of the notched steel plate (Kalthoff-Winkler
geometry, 200 x 100 x 9 mm, h = 1 mm, 178,200 nodes, delta = 4h, 36.4 M directed
bonds): bond force with breaking, contact search and force, kick/drift.  Inputs
are resident in HBM when the timed region starts; the working set (~0.3 GB)
exceeds L2.  Prints one JSON line.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-steps/s & bond-updates/s vs FP64 GPU path; HBM roofline %; RVE surrogate err"
WORKLOAD = ("kalthoff notched steel plate 200x100x9 mm, h=1 mm, 178,200 nodes, delta=4h, "
            "E=190 GPa, G0=2.2e4 J/m^2, edge segment at 32 m/s, dt=0.8 dt_crit")
WORKLOADS = {
    "plate": WORKLOAD,
    "sphere": "glass sphere radius 1 mm, h=0.1 mm, 4,139 nodes, delta=3h, plates at 1 m/s, dt=0.8 dt_crit",
    "hollow": "glass hollow sphere R=1 mm, r=0.7 mm, h=0.02 mm, 343,846 nodes, delta=3h, plates at 5 m/s",
    "aggregate": "1000 star-shaped glass grains, h=R/12, ~7.6 M nodes, delta=3h, six walls, top wall at 10 m/s",
    "aggregate-125": ("125 star-shaped glass grains of the aggregate recipe (920,726 nodes; the case the aggregate's "
                      "DRAM traffic is captured on)"),
    "shape-sphere": "shape study: 125 solid glass spheres R=1 mm, h=R/8 (262,875 nodes), delta=3h, top wall 10 m/s",
    "shape-shell": "shape study: 125 glass shells R=1 mm, r=0.7R, h=R/8 (170,500 nodes), top wall 10 m/s",
    "shape-jack": "shape study: 125 glass jacks R=1 mm (arms R/3), h=R/8 (93,375 nodes), top wall 10 m/s",
    "double-hollow": "two stacked glass shells R=1 mm, r=0.7R, h=0.04 mm (85,084 nodes), top wall 10 m/s",
}


def cpu_sample(name, sc):
    """The workload the CPU baseline times: the full workload up to ~1 M nodes; for
    the 1000-grain aggregate a 64-grain aggregate of the same recipe (same grain
    shapes, h, material and box loading), so that the oracle's set-up and steps
    stay within a minute."""
    from paper_2506_05362_gb300 import scenarios as S
    if name == "aggregate":
        return S.aggregate(n_grains=64, seed=0), "64-grain aggregate of the same recipe"
    return sc, f"the full {name} workload"


def make_workload(name):
    from paper_2506_05362_gb300 import scenarios as S
    return {"plate": S.kalthoff, "sphere": S.sphere, "hollow": S.hollow,
            "aggregate": lambda: S.aggregate(n_grains=1000, seed=0),
            "aggregate-125": lambda: S.aggregate(n_grains=125, seed=0),
            "shape-sphere": lambda: S.shape_study("sphere"), "shape-shell": lambda: S.shape_study("shell"),
            "shape-jack": lambda: S.shape_study("jack"), "double-hollow": S.double_hollow}[name]()
KERNEL_NAMES = {0: "global gathers", 1: "shared-memory tiles", 2: "each bond once (two passes)"}
BYTES_PER_NODE = 170.0      # x, V, u (r/w), v (r/w), F, row pointers per node and step
BYTES_PER_BOND = 4.0 + 1.0 / 8.0  # neighbour index + broken bit per directed bond


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [q.strip() for q in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, val in zip(names, p[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reference_sample():
    """The bounded sample of the plate workload that the reference arm times: a
    40 x 60 x 9 mm cut (same h = 1 mm, delta = 4h, steel, notch geometry scaled,
    edge segment at 32 m/s), ~21,000 nodes, so that a step of the single-threaded
    FP64 oracle takes ~0.06 s and a 2000-step run a few minutes."""
    from paper_2506_05362_gb300 import scenarios as S
    return S.kalthoff(length=0.04, height=0.06, notch_len=0.02, notch_gap=0.02)


def reduce_max(x, ws, device=None):
    """Max over ranks of a float (the timed region's duration); identity for ws = 1."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def host_cores():
    """Cores this process may run on (sched_getaffinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    """The FP64 CPU oracle on the host's cores (its OpenMP build over the node
    loops): bounded sample of the same workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    sc = reference_sample()
    cores = oracle.set_threads(host_cores())
    m = oracle.Model.from_scenario(sc, parallel=True)
    dt = 0.8 * m.stable_dt()
    m.init()
    m.step(dt, max(args.warmup, 0))
    t0 = time.perf_counter()
    m.step(dt, args.steps)
    el = time.perf_counter() - t0
    n, B = sc.n, len(m.col)
    value = n * args.steps / el
    cpu = {"value": value, "unit": "node-steps/s", "cores": cores, "kind": "oracle",
           "sample": (f"{args.steps} velocity-Verlet steps, after {args.warmup} warm-up steps, of a 40x60x9 mm "
                      f"cut of the plate ({n} nodes, same h, delta, material and impact); OpenMP build of the "
                      f"FP64 C oracle on {cores} host cores")}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "node-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "nodes": n, "directed_bonds": B,
                                            "sample": "40x60x9 mm cut of the plate"},
            "bond_updates_per_s": B * args.steps / el, "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "node-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(sc, name="plate"):
    """The oracle on a bounded sample of the workload (8 steps; see cpu_sample): its
    OpenMP build on all host cores (the reported value), and the serial build on
    one core beside it.  Both builds give the same bits."""
    import oracle
    sc, what = cpu_sample(name, sc)
    steps = 8
    cores = oracle.set_threads(host_cores())
    rates = {}
    for par in (True, False):
        m = oracle.Model.from_scenario(sc, parallel=par)
        dt = 0.8 * m.stable_dt()
        m.init()
        t0 = time.perf_counter()
        m.step(dt, steps)
        el = time.perf_counter() - t0
        rates[par] = (sc.n * steps / el, len(m.col) * steps / el)
    return {"value": rates[True][0], "unit": "node-steps/s", "cores": cores, "kind": "oracle",
            "sample": (f"{steps} steps of {what} ({sc.n} nodes); FP64 C oracle, OpenMP build over the node "
                       f"loops on {cores} host cores (sched_getaffinity)"),
            "bond_updates_per_s": rates[True][1],
            "single_core": {"value": rates[False][0], "unit": "node-steps/s", "cores": 1,
                            "bond_updates_per_s": rates[False][1]}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=50, help="0 skips the end-to-end leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the all-FP64 comparison leg")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate-network leg")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per node (0 = autotune)")
    ap.add_argument("--tiles", default="auto", choices=["auto", "on", "off"])
    ap.add_argument("--pairs", default="auto", choices=["auto", "on", "off"],
                    help="each bond evaluated once (two passes)")
    ap.add_argument("--persistent", default="auto", choices=["auto", "on", "off"],
                    help="the steps between rebuilds in one cooperative launch")
    ap.add_argument("--workload", default="plate", choices=sorted(WORKLOADS),
                    help="workload of the timed steps (the headline figure is the plate)")
    ap.add_argument("--no-aggregate", action="store_true",
                    help="skip the 1000-grain aggregate leg (7.6 M nodes, one batched launch)")
    ap.add_argument("--surrogate-only", action="store_true",
                    help="time only the surrogate network (forward and training step) and print its figures")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.surrogate_only:
        import torch
        _, _, local = dist_env()
        torch.cuda.set_device(local)
        print(json.dumps(bench_surrogate(local, torch.cuda.Stream(local))))
        return 0

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2506_05362_gb300 import pd, scenarios as S

    sc = make_workload(args.workload)
    stream = torch.cuda.Stream(local)
    ctx = pd.Context.from_scenario(sc, precision=args.precision, device=local, stream=stream,
                                   lanes=args.lanes, tiles={"auto": 0, "on": 1, "off": -1}[args.tiles],
                                   pairs={"auto": 0, "on": 1, "off": -1}[args.pairs],
                                   persistent={"auto": 0, "on": 1, "off": -1}[args.persistent])
    lanes, kernel, tms = ctx.tuning()
    tuning = {"lanes_per_node": lanes, "kernel": KERNEL_NAMES[kernel],
              "ms_global_4_8_16_32": [round(float(t), 4) for t in tms[:4]],
              "ms_tiled_4_8_16_32": [round(float(t), 4) for t in tms[4:8]],
              "ms_pairs_4_8_16_32": [round(float(t), 4) for t in tms[8:]]}
    dt = 0.8 * ctx.stable_dt()
    n, B = sc.n, ctx.B
    # warm-up (captures the graphs)
    ctx.step(dt, args.warmup)

    def barrier():
        torch.cuda.synchronize(local)
        if ws > 1:
            torch.distributed.barrier()

    # ---- timed region: K steps, device time with CUDA events on the context's stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        ctx.step(dt, args.steps)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    _, _, launches = ctx.last_step_stats()
    steps_done, rebuilds, rollbacks = ctx.step_counters()
    ms = reduce_max(ms, ws, device=f"cuda:{local}")
    ms_step = ms / args.steps
    value = ws * n * args.steps / (ms * 1e-3)

    # ---- dominant kernel: fused force/update, each launch event-timed (no graph)
    ctx.set_profiling(True)
    prof_steps = min(args.steps, 400)
    ctx.step(dt, prof_steps)
    ms_force, ms_prof_total, _ = ctx.last_step_stats()
    ctx.set_profiling(False)
    force_ms_per_launch = ms_force / prof_steps
    alg_bytes = B * BYTES_PER_BOND + n * BYTES_PER_NODE
    hbm, peak_kind = peaks()
    achieved = alg_bytes / (force_ms_per_launch * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None, "kernel": "k_step (fused bond force + contact + walls + Verlet)",
            "peak_kind": peak_kind, "alg_bytes_per_launch": alg_bytes,
            "launch_ms": force_ms_per_launch}
    # DRAM traffic of one launch from an ncu capture, while the kernel source is
    # the one captured (profiles/k_step_traffic.json, one record per workload)
    traffic_file = os.path.join(ROOT, "profiles", "k_step_traffic.json")
    if os.path.exists(traffic_file):
        try:
            tr = json.load(open(traffic_file)).get(args.workload)
            if tr and tr.get("kernel_source_hash") == kernel_hash():
                roof["traffic"] = tr["bytes_per_launch"]
                roof["traffic_note"] = tr.get("note", "")
        except Exception:
            pass

    # ---- end to end through the C ABI with pinned host buffers: per step the whole
    # state (u, v and the bond memory, packed one bit per bond) goes host -> device,
    # one step runs, and the new state comes back
    nwords = (B + 31) // 32
    u_h = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    v_h = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    b_h = torch.empty(max(nwords, 1), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    u0, v0, b0, t0 = pd.pd_get_state_packed(ctx.h, n, B)
    u_h[:] = u0; v_h[:] = v0; b_h[:nwords] = b0
    sc0 = ctx.state_counters()
    barrier()
    te = time.perf_counter()
    for _ in range(args.e2e_steps):
        pd.pd_set_state_packed(ctx.h, u_h, v_h, b_h[:nwords])
        ctx.step(dt, 1)
        pd.pd_get_state_packed(ctx.h, n, B, u_h, v_h, b_h)
    barrier()
    e2e_s = time.perf_counter() - te
    sc1 = ctx.state_counters()
    e2e = None
    if args.e2e_steps > 0 and e2e_s > 0:
        e2e = {"value": ws * n * args.e2e_steps / e2e_s, "unit": "node-steps/s",
               "h2d_bytes_per_step": 48 * n + 4 * nwords, "d2h_bytes_per_step": 48 * n + 4 * nwords,
               "steps": args.e2e_steps,
               "set_state_applied": sc1[0] - sc0[0], "set_state_unchanged": sc1[1] - sc0[1],
               "path": "pd_set_state_packed + pd_step(dt,1) + pd_get_state_packed (u, v, bond memory at one "
                       "bit per bond), pinned host buffers"}

    # ---- all-FP64 GPU path on the same workload (comparison the metric asks for)
    fp64 = None
    if args.precision == "mixed" and not args.no_fp64:
        c64 = pd.Context.from_scenario(sc, precision="fp64", device=local, stream=stream)
        c64.step(dt, args.warmup)
        k64 = min(args.steps, 400 if n < 1_000_000 else 20)
        barrier()
        ev0.record(stream)
        c64.step(dt, k64)
        ev1.record(stream)
        barrier()
        m64 = ev0.elapsed_time(ev1)
        fp64 = {"value": n * k64 / (m64 * 1e-3), "unit": "node-steps/s", "steps": k64,
                "ms_per_step": m64 / k64, "bond_updates_per_s": B * k64 / (m64 * 1e-3)}
        c64.close()

    surrogate = None if args.no_surrogate else bench_surrogate(local, stream)
    aggregate = None if (args.no_aggregate or args.workload == "aggregate") else bench_aggregate(local, stream)
    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline else cpu_baseline(sc, args.workload)
    line = {"metric": METRIC, "value": value, "unit": "node-steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+df64" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "nodes": n, "directed_bonds": B, "precision": args.precision,
                       "l2": (f"inputs larger than L2: ~{alg_bytes / 1e9:.2f} GB streamed from HBM per step "
                              "(129 MB L2)"),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "bond_updates_per_s": ws * B * args.steps / (ms * 1e-3),
            "clocks": clk.summary(), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "fp64_gpu_path": fp64, "surrogate": surrogate, "aggregate": aggregate,
            "tuning": tuning, "contact_rebuilds": rebuilds, "rollbacks": rollbacks, "steps_run": steps_done}
    print(json.dumps(line), flush=True)
    ctx.close()


def bench_aggregate(local, stream, steps=200):
    """The 1000-grain aggregate (star-shaped glass grains, h = R/12, ~7.6 M nodes,
    ~0.8 G directed bonds) in one batched launch per step, autotuned: device time
    of `steps` steps with CUDA events on the context's stream."""
    import torch
    from paper_2506_05362_gb300 import pd, scenarios as S
    sc = S.aggregate(n_grains=1000, seed=0)
    ctx = pd.Context.from_scenario(sc, device=local, stream=stream)
    lanes, kernel, _ = ctx.tuning()
    dt = 0.8 * ctx.stable_dt()
    ctx.step(dt, 10)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(local)
    ev0.record(stream)
    ctx.step(dt, steps)
    ev1.record(stream)
    torch.cuda.synchronize(local)
    ms = ev0.elapsed_time(ev1)
    ctx.set_profiling(True)
    ctx.step(dt, 50)
    ms_force, _, _ = ctx.last_step_stats()
    ctx.set_profiling(False)
    n, B = sc.n, ctx.B
    force_ms = ms_force / 50
    alg = B * BYTES_PER_BOND + n * BYTES_PER_NODE
    hbm, kind = peaks()
    ctx.close()
    return {"workload": "1000 star-shaped glass grains, R ~ U(0.4, 0.6) mm, h = R/12 (0.5 mm/12), delta = 3h, "
                        "six walls, top wall at 10 m/s", "nodes": n, "directed_bonds": B, "steps": steps,
            "ms_per_step": ms / steps, "node_steps_per_s": n * steps / (ms * 1e-3),
            "bond_updates_per_s": B * steps / (ms * 1e-3), "lanes_per_node": lanes, "kernel": KERNEL_NAMES[kernel],
            "k_step_ms": force_ms, "k_step_hbm_frac": alg / (force_ms * 1e-3) / 1e9 / hbm, "peak_kind": kind}


def bench_surrogate(local, stream, reps=20):
    """MLP 109-256-256-256-256-6 at inference batch 65536 and one Adam training
    step at the same batch: device time with CUDA events, FLOP rate against the
    measured BF16 tensor peak."""
    import torch
    from paper_2506_05362_gb300 import pd
    dims = (109, 256, 256, 256, 256, 6)
    B = 65536
    net = pd.MLP(dims, seed=0, device=local, stream=stream)
    g = torch.Generator(device=f"cuda:{local}").manual_seed(0)
    X = torch.randn(B, dims[0], device=f"cuda:{local}", generator=g)
    T = torch.randn(B, dims[-1], device=f"cuda:{local}", generator=g)
    Y = torch.empty(B, dims[-1], device=f"cuda:{local}")
    flop_fwd = 2.0 * B * sum(dims[i] * dims[i + 1] for i in range(len(dims) - 1))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for _ in range(3):
            net.forward_device(X, Y)
            net.train_step_device(X, T, 1e-4)
        stream.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            net.forward_device(X, Y)
        ev1.record(stream)
        stream.synchronize()
        fwd_ms = ev0.elapsed_time(ev1) / reps
        ev0.record(stream)
        for _ in range(reps):
            net.train_step_device(X, T, 1e-4)
        ev1.record(stream)
        stream.synchronize()
        train_ms = ev0.elapsed_time(ev1) / reps
    net.close()
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, peak_s = float(mp["bf16_tflops"]), float(mp["bf16_tflops_sustained"])
        kind = "measured"
    except Exception:
        peak, peak_s, kind = 1900.0, 1700.0, "fallback"
    fwd_tf = flop_fwd / (fwd_ms * 1e-3) / 1e12
    train_tf = 3 * flop_fwd / (train_ms * 1e-3) / 1e12
    return {"dims": list(dims), "batch": B, "forward_ms": fwd_ms, "forward_samples_per_s": B / (fwd_ms * 1e-3),
            "train_step_ms": train_ms,
            "roofline": {"bound": "tensor", "achieved": fwd_tf, "peak": peak, "unit": "TFLOP/s",
                         "frac": fwd_tf / peak, "peak_kind": kind, "kernel": "k_mlp_fwd_tc (fused tcgen05 forward, all layers)"},
            "train_tflops": train_tf,
            # a training step (forward keeping activations, two backward GEMMs per
            # layer, reductions, Adam) against the sustained BF16 peak: the 3x
            # forward FLOPs of the GEMMs over the whole step's time
            "train_roofline": {"bound": "tensor", "achieved": train_tf, "peak": peak_s, "unit": "TFLOP/s",
                               "frac": train_tf / peak_s, "peak_kind": kind + " (sustained)",
                               "flop_per_step": 3 * flop_fwd}}


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ["pd_step.cu", "pd_internal.cuh", "pd_df.cuh"]:
        h.update(open(os.path.join(ROOT, "paper_2506_05362_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
