#!/usr/bin/env python
"""FGA forward-solve benchmark on GB300.

One step = one whole forward solve of the smooth heterogeneous workload through the C ABI
(fga_solve): wave-packet decomposition of the initial data, RK4 propagation of every P+, P-, S+
and S- beam (24^3 q x 8^3 p mesh points, 28.3 M beams, 400 steps of dt = 0.0025), seismograms at
400 surface receivers x 1,000 samples and a 64^3 snapshot at T = 1.  The medium is
c_p = 2 + 0.2 sin(2 pi x1) sin(2 pi x2) sin(2 pi x3), c_s = c_p/sqrt(3), on a 128^3 FP32 grid.

value = beam-steps/s (whole job, all ranks), with inputs resident in HBM; e2e = the same metric with
host buffers copied in and results copied out inside the timed region.  The reference arm
(--impl reference) times the FP64 CPU oracle on a strided sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP32 operations per beam-step and per Gaussian-sum pair, counted from the kernels' source (FMA = 2)
FLOP_PER_BEAM_STEP = {"P": 4180.0, "S": 4400.0}
FLOP_PER_PAIR_IN = 43.0       # dx, r^2, phase, exponent, e*(cos, sin), 3 complex multiply-adds
FLOP_PER_PAIR_OUT = 9.0       # dx, r^2, compare
MUFU_PER_PAIR_IN = 3.0        # exp2, sin, cos
FLOP_PER_LATTICE_PAIR_IN = 26.0   # window test (add, compare) + 3 complex multiply-adds
# DRAM bytes (dram__bytes_read + write) per launch of each category's kernel on the full smooth workload,
# from ncu captures summarised under profiles/; a category is absent until its current kernel is captured.
# gauss_sum: plane_tc_kernel<0, 10, 20>, 1.02 GB read + 4-6 MB written per launch (two launches of the timed solve);
# propagate: rk4_kernel, 1.5-1.8 GB read + 13.1-13.6 GB written per launch (the window's records; eight launches)
TRAFFIC_BYTES_PER_LAUNCH = {"gauss_sum": 1.025e9, "propagate": 1.49e10}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--size", default="full", choices=["full", "medium", "small"],
                    help="workload size: full = the benchmark; medium (16^3 q, 8.4 M beams, 1.5 GB of state) is "
                         "the profiler capture case; small is for debugging (neither is a bench line)")
    ap.add_argument("--serving", action="store_true",
                    help="the serving stream instead: 64 Poisson-arriving requests of mixed k and size on the resident "
                         "smooth model at 0.7 of the measured solo capacity; p50/p99 latency and beam-steps/s")
    ap.add_argument("--adjoint", action="store_true",
                    help="the crosswell gradient instead: 16 sources x 3.5 M beams, 200 steps, 256 receivers, L2 "
                         "misfit against data of the bumped model; time per gradient (forward + adjoint)")
    ap.add_argument("--point-source", action="store_true",
                    help="the paper's accuracy experiment instead: point force at (64,64,64) km, f = 1.4702 Hz; the FGA "
                         "starts at t0 = 3 s from the radiated field and is compared with the analytic solution at "
                         "6.93 s on a 697-receiver patch (time per solve, beam-steps/s, relative error)")
    ap.add_argument("--k", type=float, default=0.08, help="with --point-source: the FGA parameter k (1/km)")
    ap.add_argument("--layered", action="store_true",
                    help="the layered-crust workload instead: explosive source at 10 km depth, interfaces at 15 and "
                         "35 km, 10^3 q x 8^3 p x 4 classes (2.05 M beams) with psi selection 1e-6, 120 s at "
                         "dt = 0.01 s (12,000 steps), 256 surface stations (16 x 16 over +-300 km) every 0.1 s; "
                         "plus the FP32 error against FP64 on a 5^3 q x 4^3 p stride sample of it")
    ap.add_argument("--undulating", action="store_true",
                    help="with --layered: the interfaces undulate, x3 = 15 + 3 cos(2 pi x1/20) cos(2 pi x2/30) and "
                         "35 - 2 cos(...) cos(...) km (not parallel)")
    ap.add_argument("--shells", type=float, default=0.0, metavar="RC",
                    help="with --layered: the same crust bent into concentric spheres about (0, 0, RC) km (radii "
                         "RC - 15 and RC - 35; e.g. 6371 for the Earth), stations on the sphere r = RC")
    ap.add_argument("--policy", default="shortest", choices=["fifo", "shortest"],
                    help="with --serving: admission order (submission order, or least estimated work first with a "
                         "2 s age bound)")
    ap.add_argument("--requests", type=int, default=64, help="with --serving: requests in the stream")
    ap.add_argument("--nmax", type=float, default=2e7,
                    help="with --serving: largest drawn mesh size N (log-uniform in [1e5, nmax])")
    ap.add_argument("--misfit", default="l2", choices=["l2", "traveltime"],
                    help="with --adjoint: L2 waveform misfit, or cross-correlation traveltime misfit "
                         "(delays within +-20 samples) with its synthetic-only adjoint source")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the FP32-vs-FP64 comparison on the 8^3-q version of the workload")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def workload(size: str):
    from paper_1810_06760_gb300 import workloads as W
    if size == "small":
        return W.smooth(nq=8, np_=4, ny=48, nsteps=40, n_samples=100, rx_side=10, snap_side=16, grid_n=65)
    if size == "medium":
        return W.smooth(nq=16, nsteps=100, n_samples=250)
    return W.smooth()


METRIC = "FGA beam-steps/s and Gaussian-sum pts/s at fixed error; p50/p99 solve latency"


def workload_desc(w) -> str:
    """The forward-solve workload, named by its sizes (the same words in both arms' config)."""
    n = w.medium.grid_p.shape[0]
    snap = "x".join(str(len(a)) for a in w.snap_axes)
    return (f"smooth-heterogeneous: {n}^3 grid medium, k={w.k:g}, {w.mesh.nq}^3 q x {w.mesh.np_}^3 p mesh x "
            f"{len(w.classes)} classes ({w.n_beams} beams), {w.nsteps} RK4 steps, {len(w.receivers)} rx x "
            f"{len(w.times)} samples + {snap} snapshot")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                smax.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v: float, device=None) -> float:
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------------
# CPU oracle on a strided sample of the workload
# ------------------------------------------------------------------------------------------------

def oracle_sample(w, q_stride: int, p_stride: int, n_samples_cap=None):
    """Oracle propagation + seismogram sums of the beams of every q_stride-th q node and p_stride-th
    p node per axis (all four classes).  Returns (beam_steps, seconds, threads, description)."""
    from oracle import fga_oracle as O
    O.build()
    med = w.medium
    om = O.Model(med.kind, cp0=med.cp0, cs0=med.cs0, amp=med.amp, cs_ratio=med.cs_ratio, grid_p=med.grid_p,
                 grid_s=med.grid_s, origin=med.origin, spacing=med.spacing)
    m = w.mesh
    full = O.Mesh(m.nq, m.q0, m.dq, m.np_, m.p0, m.dp)
    sub = O.Mesh(len(range(0, m.nq, q_stride)), m.q0, m.dq * q_stride, len(range(0, m.np_, p_stride)), m.p0,
                 m.dp * p_stride)
    F = O.fbi(w.f, w.y0, w.dy, w.k, sub)           # untimed: the sample's wave-packet weights
    times = w.times if n_samples_cap is None else w.times[:n_samples_cap]
    s_step, s_th = O.sample_schedule(times, w.dt, w.nsteps)
    wgt = full.weight(w.k)
    beams = [O.beam_init(om, w.k, sub, F, None, c) for c in w.classes]
    t0 = time.perf_counter()
    for st, meta in beams:
        rec = O.propagate(om, st, meta, w.dt, w.nsteps, s_step, s_th, wgt)
        for j in range(len(times)):
            O.gauss_sum(rec[j], w.k, w.rw, w.receivers)
    dt = time.perf_counter() - t0
    nb = sub.M * len(w.classes)
    desc = (f"{nb} beams (q stride {q_stride}, p stride {p_stride} per axis, 4 classes) x {w.nsteps} RK4 steps "
            f"+ {len(w.receivers)} receivers x {len(times)} samples; decomposition untimed")
    return nb * w.nsteps, dt, O.get_threads(), desc


# ------------------------------------------------------------------------------------------------

def run_reference(args):
    # the oracle runs on rank 0's host cores only; other ranks exit at once (no process group needed)
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    w = workload(args.size)
    for _ in range(args.warmup):
        oracle_sample(w, 12, 8, n_samples_cap=50)
    vals = []
    for _ in range(args.steps):
        bs, secs, thr, desc = oracle_sample(w, 6, 2)
        vals.append((bs, secs))
    tot_bs = sum(v[0] for v in vals)
    tot_s = sum(v[1] for v in vals)
    value = tot_bs / tot_s
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "beam-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(w), "sample": desc},
            "cpu_baseline": {"value": value, "unit": "beam-steps/s", "cores": thr, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "beam-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_1810_06760_gb300 import fga

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = fga.PREC_FP32 if args.precision == "fp32" else fga.PREC_FP64
    w = workload(args.size)
    nb = w.n_beams
    beam_steps = nb * w.nsteps
    model = fga.model_from_medium(w.medium, dev)
    f = torch.as_tensor(w.f, device=dev)
    desc = fga.init_desc(w.k, f, None, w.y0, w.dy, w.mesh, w.classes, prec)
    cdt = torch.complex64 if prec == fga.PREC_FP32 else torch.complex128
    seis = torch.empty((len(w.times),) + tuple(len(a) for a in w.rx_axes) + (3,), dtype=cdt, device=dev)
    snap = torch.empty(tuple(len(a) for a in w.snap_axes) + (3,), dtype=cdt, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        fga.solve(model, desc, w.dt, w.nsteps, w.times, rw=w.rw, seis_out=seis, snap_out=snap, rx_axes=w.rx_axes,
                  snap_axes=w.snap_axes)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # timed region: device time with CUDA events on the launching stream, per-kernel event times live
    fga.profile_enable(2)
    fga.profile_read(reset=True)
    clk = Clocks(local)
    clk.start()
    barrier(pg)
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for i in range(args.steps):
        step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    clocks = clk.stop()
    prof = fga.profile_read(reset=True)
    # the in-window pair count of one solve (counting adds instructions, so it is not timed)
    fga.profile_enable(1)
    step()
    torch.cuda.synchronize()
    cnt = fga.profile_read(reset=True)
    # and of the same solve without the snapshot: the receivers' share
    fga.solve(model, desc, w.dt, w.nsteps, w.times, rw=w.rw, seis_out=seis, rx_axes=w.rx_axes)
    torch.cuda.synchronize()
    cnt_rx = fga.profile_read(reset=True)
    fga.profile_enable(0)
    prof["pairs_in_window"] = cnt["pairs_in_window"] * args.steps
    prof["pairs_in_window_rx"] = cnt_rx["pairs_in_window"] * args.steps
    prof["pairs_tested"] = cnt["pairs_tested"] * args.steps
    per_step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    total_ms = max_over_ranks(pg, total_ms, dev)
    value = world * args.steps * beam_steps / (total_ms / 1e3)
    assert torch.isfinite(torch.view_as_real(seis)).all() and torch.isfinite(torch.view_as_real(snap)).all()

    # dominant kernel and its roofline (FP32 ALU-bound: FP32 pipe peak from SM count x lanes x clock)
    pk, pk_kind = peaks()
    ms = dict(prof["ms"])
    # the receiver sums at the sample times (plane kernel on a receiver plane) and the snapshot (lattice
    # kernel) are separate kernels: rank them separately
    gauss_ms_total = ms["gauss_sum"] + ms["gauss_sum_state"]
    cnts = dict(prof["count"])
    by_kernel = {"propagate": ms["propagate"], "gauss_sum": ms["gauss_sum"], "gauss_sum_state": ms["gauss_sum_state"]}
    top = max(by_kernel, key=lambda c: by_kernel[c])
    pairs_of = {"gauss_sum": prof["pairs_in_window_rx"],
                "gauss_sum_state": prof["pairs_in_window"] - prof["pairs_in_window_rx"]}
    sm_clock = float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * sm_clock
    if prec == fga.PREC_FP32 and top == "propagate":
        nP = sum(1 for c in w.classes if c < 2) * w.mesh.M
        nS = sum(1 for c in w.classes if c >= 2) * w.mesh.M
        flops = (nP * FLOP_PER_BEAM_STEP["P"] + nS * FLOP_PER_BEAM_STEP["S"]) * w.nsteps * args.steps
    elif prec == fga.PREC_FP32 and top in pairs_of:
        # lattice sum: algorithmic work of the in-window pairs, one complex product per component and point
        # plus the window test (26 FLOP); the tensor-core kernels' extra (out-of-window, split) products are
        # not counted
        flops = pairs_of[top] * FLOP_PER_LATTICE_PAIR_IN
    else:
        flops = None
    launches = max(cnts[top], 1)
    per_launch_ms = ms[top] / launches
    roof = None
    if flops is not None:
        achieved = flops / (ms[top] / 1e3) / 1e12
        peak = fp32_peak / 1e12
        traffic = TRAFFIC_BYTES_PER_LAUNCH.get(top) if args.size == "full" else None
        roof = {"bound": "alu", "kernel": top, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_basis": f"FP32 pipe: {sms} SMs (device property) x 128 lanes x 2 x {sm_clock / 1e6:.0f} MHz "
                              f"(max SM clock of {pk_kind} peaks file)",
                "per_launch_ms": per_launch_ms, "launches": launches}
    gauss_s = gauss_ms_total / 1e3
    line = {
        "metric": METRIC,
        "value": value, "unit": "beam-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == fga.PREC_FP32 else "f64", "data": "synthetic",
        "config": {"workload": workload_desc(w),
                   "l2": "inputs larger than L2 (beam state 5.2 GB)", "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": statistics.median(per_step_ms),
                       "p99": sorted(per_step_ms)[min(len(per_step_ms) - 1, math.ceil(0.99 * len(per_step_ms)) - 1)]},
        "gauss_sum_pairs_per_s": prof["pairs_in_window"] / gauss_s if gauss_s > 0 else None,
        "receiver_samples_per_s": world * args.steps * (len(w.times) * len(w.receivers) + len(w.snapshot))
        / (total_ms / 1e3),
        "kernel_ms": {k: v / args.steps for k, v in prof["ms"].items() if v > 0},
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": prof["launches"],
    }

    if not args.no_e2e:
        # end to end through the public API from pinned host buffers: inputs in, solve, results out
        hf = torch.as_tensor(w.f).pin_memory()
        hgp = torch.as_tensor(w.medium.grid_p).pin_memory()
        hgs = torch.as_tensor(w.medium.grid_s).pin_memory()
        oseis = torch.empty(seis.shape, dtype=cdt).pin_memory()
        osnap = torch.empty(snap.shape, dtype=cdt).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in (hf, hgp, hgs))
        h2d += 8 * sum(len(a) for a in w.rx_axes + w.snap_axes)   # lattice axes, copied by the library
        d2h = oseis.numel() * oseis.element_size() + osnap.numel() * osnap.element_size()

        def e2e_step():
            df = hf.to(dev, non_blocking=True)
            gp = hgp.to(dev, non_blocking=True)
            gs = hgs.to(dev, non_blocking=True)
            m2 = fga.Model("grid", grid_p=gp, grid_s=gs, origin=w.medium.origin, spacing=w.medium.spacing)
            d2 = fga.init_desc(w.k, df, None, w.y0, w.dy, w.mesh, w.classes, prec)
            s_, n_ = fga.solve(m2, d2, w.dt, w.nsteps, w.times, rw=w.rw, rx_axes=w.rx_axes, snap_axes=w.snap_axes)
            oseis.copy_(s_, non_blocking=True)
            osnap.copy_(n_, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            m2.close()

        e2e_step()
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier(pg)
        e2e_s = max_over_ranks(pg, time.perf_counter() - t0, dev)
        line["e2e"] = {"value": world * args.steps * beam_steps / e2e_s, "unit": "beam-steps/s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if world == 1 and prec == fga.PREC_FP32 and not args.no_fp64:
        line["fp64_comparison"] = fp64_comparison(args, dev)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        bs, secs, thr, desc_s = oracle_sample(w, 6, 2) if args.size != "small" else oracle_sample(w, 4, 2)
        line["cpu_baseline"] = {"value": bs / secs, "unit": "beam-steps/s", "cores": thr, "kind": "oracle",
                                "sample": desc_s}
    if rank == 0:
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()
    return 0


def fp64_comparison(args, dev):
    """The FP32 split-precision path against the plain FP64 GPU path on the same inputs: the bench
    workload with its q mesh coarsened to 8^3 nodes over the same region (1,048,576 beams; every other
    size unchanged), one solve each, timed with CUDA events.  Reports both throughputs and the FP32
    results' error against the FP64 ones (relative L2, and element-wise on entries above 1e-2 of the
    peak)."""
    import numpy as np
    import torch

    from paper_1810_06760_gb300 import fga
    from paper_1810_06760_gb300 import workloads as W
    if args.size == "full":
        w = W.smooth(nq=8)
    elif args.size == "medium":
        w = W.smooth(nq=6, nsteps=100, n_samples=250)
    else:
        w = W.smooth(nq=4, np_=4, ny=48, nsteps=40, n_samples=100, rx_side=10, snap_side=16, grid_n=65)
    model = fga.model_from_medium(w.medium, dev)
    f = torch.as_tensor(w.f, device=dev)
    stream = torch.cuda.current_stream()
    out = {}
    res = {}
    for name, prec, reps in (("fp32", fga.PREC_FP32, 2), ("fp64", fga.PREC_FP64, 1)):
        desc = fga.init_desc(w.k, f, None, w.y0, w.dy, w.mesh, w.classes, prec)
        for r in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            seis, snap = fga.solve(model, desc, w.dt, w.nsteps, w.times, rw=w.rw, rx_axes=w.rx_axes,
                                   snap_axes=w.snap_axes)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[name] = (seis.cpu().numpy().astype(np.complex128), snap.cpu().numpy().astype(np.complex128))
        out[name] = {"ms_per_solve": ms, "beam_steps_per_s": w.n_beams * w.nsteps / (ms / 1e3)}
    model.close()

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    def elem(a, b, frac=1e-2):
        m = np.abs(b)
        sel = m >= frac * m.max()
        return float(np.max(np.abs(a[sel] - b[sel]) / m[sel]))
    (s32, n32), (s64, n64) = res["fp32"], res["fp64"]
    n_units = len(w.times) * len(w.receivers) + len(w.snapshot)
    return {"workload": f"the same workload with a {w.mesh.nq}^3 q mesh ({w.n_beams} beams)",
            "fp32": out["fp32"], "fp64": out["fp64"],
            "fp32_speedup": out["fp64"]["ms_per_solve"] / out["fp32"]["ms_per_solve"],
            "receiver_samples_per_solve": n_units,
            "err_fp32_vs_fp64": {"seismograms_rel_l2": rel(s32, s64), "snapshot_rel_l2": rel(n32, n64),
                                 "seismograms_max_rel_above_1e-2_of_peak": elem(s32, s64),
                                 "snapshot_max_rel_above_1e-2_of_peak": elem(n32, n64)}}


def run_serving(args):
    """Serving stream (the paper runs one solve at a time; this is the library's request loop)."""
    import numpy as np
    import torch

    from paper_1810_06760_gb300 import fga
    from paper_1810_06760_gb300 import workloads as W

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = fga.PREC_FP32 if args.precision == "fp32" else fga.PREC_FP64
    reqs = W.serving_requests(n=args.requests, seed=1, n_range=(1e5, args.nmax))
    policy = fga.SERVE_SHORTEST if args.policy == "shortest" else fga.SERVE_FIFO
    model = fga.model_from_medium(reqs[0].workload.medium, dev)
    # inputs resident before the timed region: per request its initial data, receivers, descriptor
    staged = []
    for r in reqs:
        w = r.workload
        f = torch.as_tensor(w.f, device=dev)
        rx = torch.as_tensor(w.receivers, device=dev)
        staged.append((w, fga.init_desc(w.k, f, None, w.y0, w.dy, w.mesh, w.classes, prec), f, rx))
    torch.cuda.synchronize()
    n_workers = 4

    def run(arrivals, workers):
        server = fga.Server(model, n_workers=workers, policy=policy)
        t0 = time.perf_counter()
        ids = []
        for (w, desc, f, rx), ta in zip(staged, arrivals):
            delay = t0 + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids.append(server.submit(desc, w.dt, w.nsteps, w.times, rw=w.rw, keep=(f,), rx_axes=w.rx_axes))
        infos = [server.wait(i)[1] for i in ids]
        wall = time.perf_counter() - t0
        st = server.stats()
        server.close()
        return infos, wall, st

    # warm-up (compilation of nothing, allocator and caches): the four smallest requests
    order = np.argsort([w.n_beams for w, *_ in staged])
    small = [staged[i] for i in order[:4]]
    sv = fga.Server(model, n_workers=1)
    for w, desc, f, rx in small:
        sv.wait(sv.submit(desc, w.dt, w.nsteps, w.times, rw=w.rw, keep=(f,), rx_axes=w.rx_axes))
    sv.close()
    # solo capacity: every request alone, back to back on one worker
    solo, solo_wall, _ = run([0.0] * len(staged), 1)
    service = [i["t_end"] - i["t_start"] for i in solo]
    capacity = 1.0 / float(np.mean(service))        # requests per second, one at a time
    rate = 0.7 * capacity
    arrivals = [r.arrival / rate for r in reqs]
    clk = Clocks(local)
    clk.start()
    infos, wall, st = run(arrivals, n_workers)
    clocks = clk.stop()
    lat = sorted(i["t_end"] - i["t_submit"] for i in infos)
    q = lambda p: float(np.percentile(lat, p))
    # slowdown: latency in the stream over the same request's service time alone
    slow = sorted((i["t_end"] - i["t_submit"]) / max(sv, 1e-9) for i, sv in zip(infos, service))
    beam_steps = sum(w.n_beams * w.nsteps for w, *_ in staged)
    line = {
        "metric": METRIC,
        "value": beam_steps / wall, "unit": "beam-steps/s", "n_gpus": world, "steps": len(reqs), "warmup": 4,
        "ms_per_step": 1e3 * wall / len(reqs), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == fga.PREC_FP32 else "f64", "data": "synthetic",
        "config": {"workload": f"serving stream: {len(reqs)} requests, Poisson arrivals (seed 1) at 0.7 x solo "
                               f"capacity, k in {{32,64,128}}, N log-uniform 1e5..{args.nmax:g} -> q n_q^3 x p 8^3 x 4 "
                               "classes, smooth 128^3 model resident, T=0.5 (200 steps), 256 rx (16x16 lattice) x 200 "
                               "samples",
                   "workers": n_workers, "policy": args.policy, "parallelism": f"replicas x{world}"},
        "latency_s": {"p50": q(50), "p99": q(99), "max": lat[-1], "mean": float(np.mean(lat))},
        "slowdown": {"p50": float(np.percentile(slow, 50)), "p99": float(np.percentile(slow, 99)),
                     "max": slow[-1]},
        "solo": {"capacity_req_per_s": capacity, "service_s_p50": float(np.median(service)),
                 "beam_steps_per_s": beam_steps / solo_wall},
        "offered_rate_req_per_s": rate,
        "server": {"peak_running": st["peak_running"], "peak_bytes": st["peak_bytes"],
                   "budget_bytes": st["budget_bytes"]},
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_adjoint(args):
    """Gradient of the L2 waveform misfit over 16 crosswell sources with respect to the 64^3 model grids."""
    import numpy as np
    import torch

    from paper_1810_06760_gb300 import fga
    from paper_1810_06760_gb300 import workloads as W

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = fga.PREC_FP32 if args.precision == "fp32" else fga.PREC_FP64
    if args.size == "full":
        ws, true = W.crosswell()
    elif args.size == "medium":   # one source, 8^3 q: the profiler capture case
        ws, true = W.crosswell(n_src_side=1, nq=8)
    else:
        ws, true = W.crosswell(n_src_side=1, nq=4, np_=4, ny=32, nsteps=40, grid_n=17, rx_side=4, n_times=20)
    model = fga.model_from_medium(ws[0].medium, dev)
    tmodel = fga.model_from_medium(true, dev)
    staged = []
    cdt = torch.complex64 if prec == fga.PREC_FP32 else torch.complex128
    for w in ws:
        f = torch.as_tensor(w.f, device=dev)
        rx = torch.as_tensor(w.receivers, device=dev)
        desc = fga.init_desc(w.k, f, None, w.y0, w.dy, w.mesh, w.classes, prec)
        # observed data (input, not timed): the FP64 path on the true model
        d64 = fga.init_desc(w.k, f, None, w.y0, w.dy, w.mesh, w.classes, fga.PREC_FP64)
        d, _ = fga.solve(tmodel, d64, w.dt, w.nsteps, w.times, rx, rw=w.rw)
        staged.append((w, desc, f, rx, d.to(cdt)))
    torch.cuda.synchronize()
    shape = tuple(ws[0].medium.grid_p.shape[:3]) + (10,)
    gp = torch.zeros(shape, dtype=torch.float64, device=dev)
    gs = torch.zeros(shape, dtype=torch.float64, device=dev)

    def gradient():
        gp.zero_()
        gs.zero_()
        misfit = 0.0
        for w, desc, f, rx, d in staged:
            u, _ = fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
            if args.misfit == "traveltime":
                _, r, mis = fga.traveltime_adjoint(u, d, float(w.times[1] - w.times[0]), 20)
                misfit += float(mis.item())
            else:
                r = u - d
                misfit += 0.5 * float(r.abs().pow(2).sum())
            fga.solve_vjp(model, desc, w.dt, w.nsteps, w.times, rx, r, grad_p=gp, grad_s=gs, rw=w.rw,
                          checkpoint_every=20)
        return misfit

    for _ in range(max(1, args.warmup)):
        gradient()
    fga.profile_enable(2)
    fga.profile_read(reset=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        misfit = gradient()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    prof = fga.profile_read(reset=True)
    fga.profile_enable(0)
    beam_steps = sum(w.n_beams * w.nsteps for w in ws)
    line = {
        "metric": ("crosswell traveltime-misfit gradient (forward + discrete adjoint)" if args.misfit == "traveltime"
                   else "crosswell L2-misfit gradient (forward + discrete adjoint)"),
        "value": wall / args.steps, "unit": "s/gradient", "higher_is_better": False, "n_gpus": world,
        "steps": args.steps, "warmup": max(1, args.warmup), "dtype": "f32" if prec == fga.PREC_FP32 else "f64",
        "data": "synthetic", "config": {"workload": f"crosswell ({args.size}): 64^3 smooth model, {len(ws)} sources x "
                                                     f"{ws[0].mesh.nq}^3 q x {ws[0].mesh.np_}^3 p x 4 classes, "
                                                     f"k={ws[0].k:g}, {ws[0].nsteps} steps, "
                                                     f"{len(ws[0].receivers)} rx x {len(ws[0].times)} samples, "
                                                     "checkpoints every 20 steps"},
        "per_source_s": wall / args.steps / len(ws),
        "beam_steps_per_s": 2 * beam_steps * args.steps / wall,
        "kernel_ms_per_gradient": {k: v / args.steps for k, v in prof["ms"].items() if v > 0},
        "misfit": misfit, "grad_norm": [float(gp.norm()), float(gs.norm())],
    }
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_point_source(args):
    """Eq. ex_anal's point force: field at t0 -> selected beams -> t1, timed with CUDA events."""
    import numpy as np
    import torch

    from paper_1810_06760_gb300 import fga
    from paper_1810_06760_gb300 import workloads as W

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = fga.PREC_FP32 if args.precision == "fp32" else fga.PREC_FP64
    c = W.e1_patch(k=args.k)
    model = fga.Model("const", cp0=c.cp, cs0=c.cs)
    src = fga.point_force(c.x0, c.force, c.rho, c.cp, c.cs, c.f, c.T0, c.sigma)
    rx = torch.as_tensor(c.receivers, device=dev)
    counts = {}

    def step():
        u, v = fga.point_force_field(src, c.ny, c.y0, c.dy, c.t0)
        desc = fga.init_desc(c.k, u, v, c.y0, c.dy, c.mesh, c.classes, prec, psi_rel_min=c.psi_rel_min)
        b = fga.decompose(model, desc)
        counts["beams"] = int(b.count().sum())
        fga.propagate(model, b, c.dt, c.nsteps)
        out = fga.reconstruct(b, rx, rw=c.rw)
        b.close()
        return out

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    fga.profile_enable(2)
    fga.profile_read(reset=True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(pg)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        u1 = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(pg, e0.elapsed_time(e1), dev) / args.steps
    prof = fga.profile_read(reset=True)
    fga.profile_enable(0)
    line = {"metric": "point-force FGA solve (field at t0, selection, RK4, sum) and error vs Eq. ex_anal",
            "value": world * counts["beams"] * c.nsteps / (ms / 1e3), "unit": "beam-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(1, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f32" if prec == fga.PREC_FP32 else "f64", "data": "synthetic",
            "config": {"workload": f"paper's point-force experiment: c_p 8, c_s 4.619 km/s, f 1.4702 Hz, FGA from "
                                   f"t0 = {c.t0} s to {c.t1} s, k = {c.k:g}/km, {c.mesh.nq}^3 q x {c.mesh.np_}^3 p "
                                   f"mesh x 4 classes with psi selection {c.psi_rel_min:g}, data grid "
                                   f"{'x'.join(str(int(n)) for n in c.ny)}, {len(c.receivers)} receivers",
                       "parallelism": f"replicas x{world}"},
            "beams": counts["beams"], "mesh_points_per_class": c.mesh.M, "nsteps": c.nsteps,
            "kernel_ms_per_step": {k: v / args.steps for k, v in prof["ms"].items() if v > 0}}
    # Eq. ex_anal at t1 on the receiver lattice, by the library's FP64 point-force kernel
    ax = c.rx_axes
    ref, _ = fga.point_force_field(src, [len(a) for a in ax], [a[0] for a in ax],
                                   [(a[1] - a[0]) if len(a) > 1 else 1.0 for a in ax], c.t1, velocity=False)
    ref = ref.reshape(-1, 3).real.cpu().numpy()
    got = u1.cpu().numpy()
    line["rel_l2_vs_analytic"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    line["paper_rel_error"] = 0.0384
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_layered(args):
    """Layered crust with interface events at its stated size, timed with CUDA events."""
    import numpy as np
    import torch

    from paper_1810_06760_gb300 import fga
    from paper_1810_06760_gb300 import workloads as W

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = fga.PREC_FP32 if args.precision == "fp32" else fga.PREC_FP64
    big = args.size == "full"
    sizes = dict(nq=10, np_=8, ny=48, nsteps=12000, dt=0.01, n_times=1200, rx_side=16, extent=600.0) if big else \
        dict(nq=5, np_=4, ny=32, nsteps=1200, dt=0.01, n_times=120, rx_side=16, extent=600.0)

    def solve(w, precision, growth=8.0):
        model = fga.model_from_medium(w.medium, dev)
        f = torch.as_tensor(w.f, device=dev)
        desc = fga.init_desc(w.k, f, None, w.y0, w.dy, w.mesh, w.classes, precision, psi_rel_min=1e-6)
        fga.set_layered_options(desc, max_interfaces=4, child_rel_min=1e-6, growth=growth)
        desc.psi_rel_min = 1e-6
        fga.profile_enable(2)
        fga.profile_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        rx = None if w.rx_axes is not None else torch.as_tensor(w.receivers, device=dev)
        seis, _ = fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw, rx_axes=w.rx_axes)
        e1.record()
        torch.cuda.synchronize()
        prof = fga.profile_read(reset=True)
        fga.profile_enable(0)
        model.close()
        return seis, e0.elapsed_time(e1), prof

    make = (lambda **kw: W.shells(rc=args.shells, **kw)) if args.shells > 0 else \
        (W.undulating if args.undulating else W.layered)
    w = make(**sizes)
    warm = make(**dict(sizes, nsteps=100, n_times=10))    # the same kernels and buffers, 100 steps
    for _ in range(args.warmup):
        solve(warm, prec)
    times = []
    for _ in range(args.steps):
        seis, ms, prof = solve(w, prec)
        times.append(ms)
    ms = max_over_ranks(pg, float(np.mean(times)), dev)
    # the population after the run: live beams and children lost to the reserved capacity
    model = fga.model_from_medium(w.medium, dev)
    f = torch.as_tensor(w.f, device=dev)
    desc = fga.init_desc(w.k, f, None, w.y0, w.dy, w.mesh, w.classes, prec, psi_rel_min=1e-6)
    fga.set_layered_options(desc, max_interfaces=4, child_rel_min=1e-6, growth=8.0)
    desc.psi_rel_min = 1e-6
    b = fga.decompose(model, desc)
    selected = int(b.count().sum())
    b.close()
    model.close()
    # FP32 against FP64 on a stride sample of the workload (5^3 q x 4^3 p), same times and stations
    ws = make(**dict(sizes, nq=5, np_=4))
    s32, ms32, _ = solve(ws, fga.PREC_FP32)
    s64, ms64, _ = solve(ws, fga.PREC_FP64)
    a, r = s32.cpu().numpy().astype(np.complex128), s64.cpu().numpy()
    line = {"metric": "layered-crust FGA solve with interface events (beam-steps/s, live beams)",
            "value": world * prof["beam_steps"] / (ms / 1e3), "unit": "beam-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f32" if prec == fga.PREC_FP32 else "f64", "data": "synthetic",
            "config": {"workload": (f"spherical crust (spheres r = {args.shells - 15:g}, {args.shells - 35:g} km about "
                                    f"(0, 0, {args.shells:g})), " if args.shells > 0 else
                                    "undulating crust (interfaces 15 + 3 cc, 35 - 2 cc km, cc = cos(2 pi x1/20) "
                                    "cos(2 pi x2/30)), " if args.undulating else
                                    "layered crust (interfaces 15, 35 km), ") +
                                   f"explosive source at 10 km, k = {w.k:.3f}/km, "
                                   f"{w.mesh.nq}^3 q x {w.mesh.np_}^3 p x 4 classes, psi selection 1e-6, "
                                   f"{w.nsteps} steps of {w.dt} s, {len(w.receivers)} stations x {len(w.times)} samples",
                       "parallelism": f"replicas x{world}"},
            "mesh_beams": 4 * w.mesh.M, "selected_beams": selected, "live_beam_steps": prof["beam_steps"],
            "mean_live_beams": prof["beam_steps"] / w.nsteps,
            "kernel_ms": {k: v for k, v in prof["ms"].items() if v > 0},
            "fp64_stride_sample": {"beams": 4 * ws.mesh.M, "ms_fp32": ms32, "ms_fp64": ms64,
                                   "seismograms_rel_l2_fp32_vs_fp64": float(np.linalg.norm(a - r) / np.linalg.norm(r))}}
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)
    if args.adjoint:
        return run_adjoint(args)
    if args.point_source:
        return run_point_source(args)
    if args.layered:
        return run_layered(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
