#!/usr/bin/env python3
"""Benchmark of the split-step turbulence path on one GB300 (or N, one process per GPU).

Workload: AR(1)-evolved phase screens and 8 Gaussian beams at N = 1024 (dx = 0.5 mm, L = 1 km,
16 screens of 62.5 m, Cn^2 = 1e-15, l0 = 5 mm, L0 = 10 m, alpha = 0.99, w0 = 1.0 + 0.25 b cm).
One step = one time step of the temporal-evolution workload: the AR update and synthesis of the
16 screens (Eq. 4-5, S16) followed by the propagation of all 8 beams through them (Eq. 1), i.e.
8 x 16 = 128 field-screen steps.  Metric: field-screen steps per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own independent realization (weak scaling, no data exchange);
the timed region is bracketed by a barrier and synchronisation and the max over ranks is taken.
--impl reference times the FP64 CPU oracle on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "field·screen steps/s at N=1024 (FP32 vs split-BF16 @ stated rel-L2), % HBM roofline"
UNIT = "field·screen steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1024)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0,
                    help="CPU-baseline sample budget (and the cap on one reference-arm sample)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline (profiling runs)")
    ap.add_argument("--overlap", action="store_true",
                    help="synthesise the next step's screens on a second stream while the current step propagates")
    ap.add_argument("--no-split-bf16", action="store_true",
                    help="skip the split-BF16 tensor-core comparison (profiling runs)")
    ap.add_argument("--workload", default="ar-evolution",
                    choices=["ar-evolution", "uneven", "monte-carlo", "d2nn", "single-path", "d2nn-train"],
                    help="ar-evolution: the headline N=1024 workload; uneven: 64-instance persistent batch")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.15)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def algorithmic_bytes(N, B, S, source_in_column=False):
    """Bytes one launch of each kernel kind must move (the roofline numerator), per the 2-pass model:
    column pass: field read + write; row passes: field read + write, screen read once (shared by the
    beams), the first pass writes only; screen synthesis: AR state read + write, column-transformed
    spectrum write + read, screen phasor write (8 B), PSD shape read once; fused propagation: the
    whole ts_propagate call (first row pass and S column + row passes, see propagate_bytes)."""
    px = N * N
    # averages over the launches of one call: with the sources generated in the first column pass,
    # that pass only writes and there is no first row pass
    col = (16 * S - (8 if source_in_column else 0)) * B * px / S
    row_first = 8 * B * px
    row_mid = 16 * B * px + 8 * px
    row_avg = row_mid if source_in_column else (row_first + S * row_mid) / (S + 1)
    screens = S * 40 * px + 4 * px
    fused = propagate_bytes(N, B, S, B)  # one launch = the whole propagation of the B fields
    return {0: col, 1: row_avg, 2: screens, 3: fused}


def tuning_summary(plan):
    """The autotuner's choice for a plan and its candidate table (us per column + row pass)."""
    t = plan.tuning()
    return {"points_per_thread": t[0], "col_variant": t[5], "row_variant": t[7], "streams": t[3],
            "us_streams_1_2_4": [round(x, 2) for x in t[4]],
            "fused": bool(plan.tuning_fused()[0]),
            "candidates_e_col_row_us": [[e, cv, rv, round(us, 2)] for e, cv, rv, us in plan.tuning_candidates() if us > 0]}


def hbm_peak():
    """(GB/s, source) of the HBM roofline denominator: the measured copy bandwidth, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def propagate_bytes(N, B, S, shared_screen_fields, intensity_only=False, source_in_column=False):
    """Algorithmic bytes of one ts_propagate call of B fields through S phasor screens, each screen
    set shared by `shared_screen_fields` fields: first row pass writes the field (8 B/px); every
    column pass reads + writes it (16); middle row passes read + write it (16) and read the phasor
    once per set (8); the last row pass reads the field and the phasor and writes the field (or
    only the 4-byte intensity).  With the sources generated in the first column pass there is no
    first row pass and that column pass only writes (8)."""
    px = N * N
    sets = B / shared_screen_fields
    last = (8 + 4) if intensity_only else (8 + 8)
    first = 0 if source_in_column else 8 * B
    cols = S * 16 * B - (8 * B if source_in_column else 0)
    return px * (first + cols + (S - 1) * 16 * B + last * B + S * 8 * sets)


def screen_bytes(N, n_screens, ar=False):
    """Algorithmic bytes of synthesising n_screens phasor screens: AR state read + write (16 B/px, AR
    only), column-transformed spectrum write + read (16), phasor write (8), PSD shape read once."""
    return N * N * (n_screens * ((16 if ar else 0) + 16 + 8) + 4)


def load_traffic(kind_name, variant=None):
    """(cold-cache DRAM bytes per launch, median warm-cache bytes per 4-field launch) of a kernel from
    the committed ncu summary, or (None, None) when any source file the kernel is built from changed
    since the counters were taken, or when the record is of another kernel variant than `variant`."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None, None
    try:
        k = json.load(open(path)).get("kernels", {}).get(kind_name)
    except (OSError, ValueError):
        return None, None
    from paper_2604_07248_gb300 import _build
    if k is None or k.get("sources_sha") != _build.files_sha(k.get("sources", [])):
        return None, None
    if variant is not None and k.get("variant") is not None and k.get("variant") != variant:
        return None, None
    warm = k.get("warm_dram_bytes_per_launch_4_fields")
    return k.get("dram_bytes_per_launch"), (int(statistics.median(warm)) if warm else None)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2604_07248_gb300 as ts
    from paper_2604_07248_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    wl = W.config3()
    N, S, B = wl.N, wl.S, len(wl.w0)
    plan = ts.Plan(W.LAMBDA, N, wl.dx, wl.dz, wl.cn2, l0=W.L0_INNER, L0=W.L0_OUTER, max_batch=B)
    plan.set_sources(wl.w0)
    spec = torch.zeros((S, N, N), dtype=torch.complex64, device=dev)
    # the screens go straight to their phasors exp(i phi): each screen's sincos is taken once, not
    # once per beam
    phasor = torch.zeros((S, N, N), dtype=torch.complex64, device=dev)
    U = torch.zeros((B, N, N), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    real = rank  # each rank evolves its own independent realization
    t_next = [0]

    def step_serial(p=plan):
        t = t_next[0]
        p.evolve_screens(spec, None, wl.seed, t, wl.alpha, real=real, phasor=phasor, stream=stream)
        p.propagate(U, B, phasor=phasor, phi_group=B, flags=ts.TS_PROP_SOURCE, stream=stream)
        t_next[0] = t + 1

    # overlapped steps: the screens of step t + 1 are synthesised on their own stream while step t
    # propagates; the phasors are double-buffered (step t reads buffer t mod 2; the AR state itself
    # is only touched by the screen stream, in step order)
    s_scr = torch.cuda.Stream(dev)
    phasors = [phasor, torch.zeros_like(phasor)] if args.overlap else [phasor]
    ev_scr = [torch.cuda.Event(), torch.cuda.Event()]
    ev_prop = [torch.cuda.Event(), torch.cuda.Event()]
    for ev in ev_prop:
        ev.record(stream)

    def step_overlap(p=plan):
        t = t_next[0]
        k = t % 2
        s_scr.wait_event(ev_prop[k])  # step t - 2 has finished reading this phasor buffer
        p.evolve_screens(spec, None, wl.seed, t, wl.alpha, real=real, phasor=phasors[k], stream=s_scr)
        ev_scr[k].record(s_scr)
        stream.wait_event(ev_scr[k])
        p.propagate(U, B, phasor=phasors[k], phi_group=B, flags=ts.TS_PROP_SOURCE, stream=stream)
        ev_prop[k].record(stream)
        t_next[0] = t + 1

    def step(p=plan):
        (step_overlap if args.overlap else step_serial)(p)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        if world == 1:
            return x
        tt = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        return float(tt.item())

    groups = plan.tuning()[3]  # concurrent field groups chosen by the autotuner
    fused = plan.tuning_fused()  # (fused persistent launch chosen, us per-pass, us fused)
    src_first = plan.tuning()[5] in (2, 3) and N in (512, 1024)  # no first row pass (sources in the column pass)
    launches_per_step = 2 + (1 if fused[0] else groups * ((0 if src_first else 1) + 2 * S))
    for _ in range(args.warmup):
        step()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    stream.wait_stream(s_scr)
    e1.record(stream)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    clk = clocks.stop()

    # per-kernel device time over a second pass of the same steps (events on the launching stream).
    # The kernels are timed alone: this pass uses a plan that keeps all fields on one stream, so no
    # launch overlaps another (the timed steps above run the autotuned number of concurrent groups).
    n_prof = 256  # whatever --steps is, so the per-kernel averages rest on 256 steps of launches
    # the same kernels as the timed steps (the main plan's autotuner choices), on one stream
    tune = plan.tuning()
    pinned = {"TS_PROP_STREAMS": "1", "TS_FFT_E": str(tune[0]), "TS_COL_VARIANT": str(tune[5]),
              "TS_ROW_VARIANT": str(tune[7]), "TS_FUSED": "1" if fused[0] else "0"}
    saved = {k: os.environ.get(k) for k in pinned}
    os.environ.update(pinned)
    prof_plan = ts.Plan(W.LAMBDA, N, wl.dx, wl.dz, wl.cn2, l0=W.L0_INNER, L0=W.L0_OUTER, max_batch=B)
    for k, v in saved.items():
        if v is None:
            del os.environ[k]
        else:
            os.environ[k] = v
    prof_plan.set_sources(wl.w0)
    prof_plan.timing(True, capacity=n_prof * (S + 1))
    barrier()
    for _ in range(n_prof):
        tt = t_next[0]
        prof_plan.evolve_screens(spec, None, wl.seed, tt, wl.alpha, real=real, phasor=phasor, stream=stream)
        prof_plan.propagate(U, B, phasor=phasor, phi_group=B, flags=ts.TS_PROP_SOURCE, stream=stream)
        t_next[0] = tt + 1
    barrier()
    plan_for_timing = prof_plan
    kinds = {0: "col_pass", 1: "row_pass", 2: "screen_synthesis", 3: "propagation_fused"}
    kt = {k: plan_for_timing.timing_read(k) for k in kinds}
    plan_for_timing.timing(False)
    # the first column pass generates the sources when the prefetching column pass runs per-pass
    src_col = (not fused[0]) and tune[5] in (2, 3) and N in (512, 1024)
    algo = algorithmic_bytes(N, B, S, source_in_column=src_col)
    measured = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    peak = float(measured["hbm_gbs"]) if measured else 6800.0
    peak_src = "measured" if measured else "fallback"
    per_kernel = {}
    for k, name in kinds.items():
        n, tot = kt[k]
        if n == 0:
            continue
        avg_ms = tot / n
        gbs = algo[k] / (avg_ms * 1e-3) / 1e9
        per_kernel[name] = {"launches": n, "avg_us": round(avg_ms * 1e3, 3), "share": None,
                            "algorithmic_bytes": int(algo[k]), "achieved_gbs": round(gbs, 1)}
    total = sum(kt[k][1] for k in kinds)
    for k, name in kinds.items():
        if name in per_kernel:
            per_kernel[name]["share"] = round(kt[k][1] / total, 4) if total > 0 else None
    dom = max(per_kernel, key=lambda n: per_kernel[n]["share"] or 0)
    dk = per_kernel[dom]
    # the record holds one column and one row variant: the one the autotuner picks at this workload
    traffic, traffic_warm = load_traffic(dom, {"col_pass": tune[5], "row_pass": tune[7]}.get(dom))
    roof = {"bound": "hbm", "kernel": dom, "achieved": dk["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": round(dk["achieved_gbs"] / peak, 4), "traffic": traffic,
            "traffic_note": "ncu dram read + write per 8-field launch, cold caches (ncu flushes before replay), from the "
                            "committed capture while the kernel's sources still hash to it; in the running pipeline "
                            "the fields stay L2-resident between the passes",
            "traffic_warm_4_fields": traffic_warm, "peak_source": peak_src,
            "timing": "per-launch CUDA events on the launching stream, each kernel alone (one stream)",
            "steps": n_prof, "kernels": per_kernel}

    # end to end through the public API with host buffers: per step, H2D of the 8 input fields from
    # pinned memory, the screen update and propagation, D2H of the 8 receiver fields.  Two device
    # field buffers and two copy streams let step t's copies overlap steps t-1 / t+1's compute.
    e2e = None
    if not args.no_e2e:
        n_e2e = min(args.steps, 256)
        host_in = torch.empty((B, N, N), dtype=torch.complex64, pin_memory=True)
        host_out = [torch.empty((B, N, N), dtype=torch.complex64, pin_memory=True) for _ in range(2)]
        dbuf = [torch.empty((B, N, N), dtype=torch.complex64, device=dev) for _ in range(2)]
        plan.make_sources(dbuf[0], B, stream=stream)  # the 8 source fields are the host-side input
        host_in.copy_(dbuf[0])
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        for k in range(2):
            ev_out[k].record(s_out)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s_in.wait_event(f0)
        for i in range(n_e2e):
            k = i % 2
            s_in.wait_event(ev_out[k])          # the buffer's previous result has left the device
            with torch.cuda.stream(s_in):
                dbuf[k].copy_(host_in, non_blocking=True)
            ev_in[k].record(s_in)
            stream.wait_event(ev_in[k])
            tt = t_next[0]
            plan.evolve_screens(spec, None, wl.seed, tt, wl.alpha, real=real, phasor=phasor, stream=stream)
            plan.propagate(dbuf[k], B, phasor=phasor, phi_group=B, stream=stream)
            t_next[0] = tt + 1
            ev_done[k].record(stream)
            s_out.wait_event(ev_done[k])
            with torch.cuda.stream(s_out):
                host_out[k].copy_(dbuf[k], non_blocking=True)
            ev_out[k].record(s_out)
        stream.wait_stream(s_out)
        f1.record(stream)
        barrier()
        ms_e2e = max_over_ranks(f0.elapsed_time(f1))
        e2e = {"value": round(n_e2e * B * S * world / (ms_e2e * 1e-3), 1), "unit": UNIT,
               "h2d_bytes_per_step": int(host_in.numel() * host_in.element_size()),
               "d2h_bytes_per_step": int(host_out[0].numel() * host_out[0].element_size()), "steps": n_e2e,
               "pipeline": "double-buffered fields, H2D and D2H on their own streams overlapping compute"}

    # the same workload with the split-BF16 tensor-core passes (TS_PLAN_SPLIT_BF16): device-timed
    # steps/s, and the per-frame rel-L2 of the 8 receiver fields against the FP32 passes through the
    # same screens (the FP32 passes are themselves within 1e-5 of the FP64 oracle)
    split = None
    if not args.no_split_bf16:
        tc_plan = ts.Plan(W.LAMBDA, N, wl.dx, wl.dz, wl.cn2, l0=W.L0_INNER, L0=W.L0_OUTER, max_batch=B,
                          flags=ts.TS_PLAN_SPLIT_BF16)
        tc_plan.set_sources(wl.w0)
        U_fp = torch.zeros_like(U)
        plan.propagate(U_fp, B, phasor=phasor, phi_group=B, flags=ts.TS_PROP_SOURCE, stream=stream)
        tc_plan.propagate(U, B, phasor=phasor, phi_group=B, flags=ts.TS_PROP_SOURCE, stream=stream)
        barrier()
        tc_plan.device_status()
        diff = (U.to(torch.complex128) - U_fp.to(torch.complex128)).abs().pow(2).sum(dim=(1, 2)).sqrt()
        rel = (diff / U_fp.to(torch.complex128).abs().pow(2).sum(dim=(1, 2)).sqrt()).cpu().tolist()
        # frames 0 and B - 1 of this step and the step's screens, for the CPU leg's FP64 oracle comparison
        oracle_input = None
        if rank == 0 and not args.no_cpu:
            oracle_input = (torch.angle(phasor.to(torch.complex128)).cpu().numpy(),
                            {b: (U[b].cpu().numpy(), U_fp[b].cpu().numpy()) for b in (0, B - 1)})
        del U_fp
        n_tc = min(args.steps, 256)
        for _ in range(args.warmup):
            step(tc_plan)
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(n_tc):
            step(tc_plan)
        g1.record(stream)
        barrier()
        tc_plan.device_status()
        ms_tc = max_over_ranks(g0.elapsed_time(g1))
        # per-launch device time of the tensor-core passes (CUDA events the library records on the
        # launching stream), averaged over the passes of 32 more steps
        n_tm = min(n_tc, 32)
        tc_plan.timing(True, capacity=n_tm * (S + 1))
        for _ in range(n_tm):
            step(tc_plan)
        barrier()
        tc_kernels = {}
        for k, name in ((0, "tc_col_pass"), (1, "tc_row_pass")):
            n, tot = tc_plan.timing_read(k)
            if n:
                tc_kernels[name] = {"launches": n, "avg_us": round(tot / n * 1e3, 3)}
        tc_plan.timing(False)
        split = {"value": round(n_tc * B * S * world / (ms_tc * 1e-3), 1), "unit": UNIT, "steps": n_tc,
                 "ms_per_step": round(ms_tc / n_tc, 5), "dtype": "bf16 hi+lo split, f32 accumulate",
                 "rel_l2_vs_fp32_per_frame_max": float(f"{max(rel):.3e}"),
                 "rel_l2_vs_fp32_per_frame": [float(f"{r:.3e}") for r in rel], "rel_l2_tolerance": 2e-3,
                 "rel_l2_vs_oracle_per_frame": None,  # filled by the CPU leg below
                 "streams": tc_plan.tuning()[3], "kernels": tc_kernels,
                 "note": "same workload and screens, AR update + 16 screens + 8 beams per step; column and "
                         "row passes on tcgen05 (32 x 32 four-step DFT)"}
        tc_plan.close()

    value = args.steps * B * S * world / (ms * 1e-3)
    # the split-step loop alone, as timed (the main plan's kernels and concurrent field groups): K'
    # ts_propagate calls of the B beams through the step's S resident phasor screens
    n_loop = min(args.steps, 256)
    for _ in range(2):
        plan.propagate(U, B, phasor=phasor, phi_group=B, flags=ts.TS_PROP_SOURCE, stream=stream)
    barrier()
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(n_loop):
        plan.propagate(U, B, phasor=phasor, phi_group=B, flags=ts.TS_PROP_SOURCE, stream=stream)
    h1.record(stream)
    barrier()
    ms_loop = max_over_ranks(h0.elapsed_time(h1)) / n_loop
    loop_bytes = propagate_bytes(N, B, S, B, source_in_column=src_col)
    loop_gbs = loop_bytes / (ms_loop * 1e-3) / 1e9
    roof["split_step_loop"] = {"algorithmic_bytes": int(loop_bytes), "us_per_call": round(ms_loop * 1e3, 2),
                               "achieved": round(loop_gbs, 1), "frac": round(loop_gbs / peak, 4), "calls": n_loop,
                               "note": "ts_propagate of the 8 beams through 16 resident phasor screens (16 column "
                                       "and row passes; the sources are generated in the first column pass), as "
                                       "configured by the autotuner"}

    # the whole timed step against the same peak: algorithmic bytes of one step (AR update + synthesis
    # of the S screens, propagation of the B beams) / device time per step
    step_bytes = screen_bytes(N, S, ar=True) + propagate_bytes(N, B, S, B, source_in_column=src_col)
    step_gbs = step_bytes / (ms / args.steps * 1e-3) / 1e9
    roof["step"] = {"algorithmic_bytes": int(step_bytes), "achieved": round(step_gbs, 1),
                    "frac": round(step_gbs / peak, 4),
                    "note": "whole timed step (screens + propagation, concurrent field groups as timed)"}
    res = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "N": N, "dx": wl.dx, "L": wl.L, "screens": S, "beams": B,
                   "cn2": wl.cn2[0], "alpha": wl.alpha, "field_screen_steps_per_step": B * S,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "screens_overlap_propagation": bool(args.overlap),
                   "autotune": dict(zip(("points_per_thread", "us_e16", "us_e32", "streams", "us_streams_1_2_4",
                                         "col_variant", "us_e32_warp_columns", "row_variant",
                                         "us_e32_shared_phasor_rows"),
                                        [round(x, 2) if isinstance(x, float) else
                                         ([round(y, 2) for y in x] if isinstance(x, list) else x)
                                         for x in plan.tuning()])),
                   "column_tiles": dict(zip(("col_variant", "us_variant2_grouped", "us_variant3_grouped"),
                                            [round(x, 2) if isinstance(x, float) else x
                                             for x in plan.tuning_columns()])),
                   "fused": {"chosen": fused[0], "us_per_pass": round(fused[1], 2), "us_fused": round(fused[2], 2)},
                   "l2": "working set 320 MiB (AR spectra 128 + screen phasors 128 + fields 64) > 126 MB L2; no flush"},
        "roofline": roof,
        "split_bf16": split,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    if rank == 0:
        res["cpu_baseline"] = None if args.no_cpu else cpu_baseline(args.cpu_seconds)
        if split is not None and oracle_input is not None:
            split["rel_l2_vs_oracle_per_frame"] = oracle_field_errors(wl, *oracle_input)
        print(json.dumps(res), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle as it stands, on one core and on all host cores
# ------------------------------------------------------------------------------------------------
def oracle_field_errors(wl, phi, frames):
    """CPU leg: per-frame rel-L2 of the split-BF16 and FP32 receiver fields (host copies) against the
    FP64 oracle propagated through the same screens (phi = arg of the step's phasor screens) from the
    same Gaussian sources."""
    import numpy as np

    import oracle as O
    from paper_2604_07248_gb300 import workloads as W

    t0 = time.perf_counter()
    md = O.medium(W.LAMBDA, wl.N, wl.dx, l0=W.L0_INNER, L0=W.L0_OUTER)
    out = {}
    for b, (u_tc, u_fp) in frames.items():
        ref = O.propagate(md, wl.dz, phi, O.source_gaussian(wl.N, wl.dx, wl.w0[b]))
        nr = np.linalg.norm(ref)
        out[str(b)] = {"split_bf16": float(f"{np.linalg.norm(u_tc - ref) / nr:.3e}"),
                       "fp32": float(f"{np.linalg.norm(u_fp - ref) / nr:.3e}")}
    out["oracle_seconds"] = round(time.perf_counter() - t0, 1)
    return out


def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in txt.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def oracle_rates(budget_s: float, threads: int = 1):
    """The oracle on a bounded sample of the temporal-evolution workload (N = 1024): `threads` host
    threads (the oracle's C code runs without the interpreter lock) first each evolve and synthesise
    screens of their own realization for 40 % of the budget, then each propagate a beam through their
    screens for 60 %.  Returns (seconds per screen update and per field-screen step on these threads,
    screens done, propagation steps done)."""
    import numpy as np

    import oracle as O
    from paper_2604_07248_gb300 import workloads as W

    wl = W.config3()
    md = O.medium(W.LAMBDA, wl.N, wl.dx, l0=W.L0_INNER, L0=W.L0_OUTER)
    dz, cn2 = wl.dz[0], wl.cn2[0]
    screens = [[] for _ in range(threads)]
    counts = [[0, 0] for _ in range(threads)]

    def run_screens(w, deadline):
        spec, _ = O.screen_spectrum(md, cn2, dz, 0, wl.seed, 0, w, 0)
        t = 0
        while True:
            t += 1
            spec, _ = O.ar_step(md, cn2, dz, 0, wl.seed, 0, w, t, wl.alpha, spec)
            screens[w].append(O.screen_from_spectrum(md, spec))
            counts[w][0] += 1
            if time.perf_counter() > deadline or t >= 16:
                break

    def run_prop(w, deadline):
        U = O.source_gaussian(wl.N, wl.dx, wl.w0[w % len(wl.w0)])
        k = 0
        while True:
            U = O.propagate(md, [dz], screens[w][k % len(screens[w])][None], U)
            counts[w][1] += 1
            k += 1
            if time.perf_counter() > deadline or k >= 128:
                break
        return np.abs(U).sum()

    def phase(fn, share):
        t0 = time.perf_counter()
        deadline = t0 + budget_s * share
        ts = [threading.Thread(target=fn, args=(w, deadline)) for w in range(threads)]
        for th in ts:
            th.start()
        for th in ts:
            th.join()
        return time.perf_counter() - t0

    wall_s = phase(run_screens, 0.4)
    wall_p = phase(run_prop, 0.6)
    n_scr = sum(c[0] for c in counts)
    n_prop = sum(c[1] for c in counts)
    return wall_s / n_scr, wall_p / n_prop, n_scr, n_prop


def cpu_baseline(budget_s: float):
    from paper_2604_07248_gb300 import workloads as W

    wl = W.config3()
    S, B = wl.S, len(wl.w0)
    cores, model = host_cpu()
    ts1, tp1, ns1, np1 = oracle_rates(budget_s * 0.4, 1)
    tsn, tpn, nsn, npn = oracle_rates(budget_s * 0.6, cores)
    one = B * S / (S * ts1 + B * S * tp1)
    alln = B * S / (S * tsn + B * S * tpn)
    return {"value": round(alln, 4), "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
            "single_thread": {"value": round(one, 4), "cores": 1, "screens": ns1, "propagation_steps": np1},
            "sample": (f"FP64 oracle, N=1024, {cores} host threads each on its own realization: {nsn} screen AR "
                       f"updates+syntheses ({tsn:.3f} s per screen on all cores) and {npn} single-beam propagation "
                       f"steps ({tpn:.3f} s per step on all cores), scaled to one time step (16 screens + 128 "
                       f"field-screen steps); single_thread: the same on one thread ({ns1} screens, {np1} steps)")}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2604_07248_gb300 import workloads as W

    wl = W.config3()
    S, B = wl.S, len(wl.w0)
    cores, model = host_cpu()
    budget_total = 150.0
    per_step_budget = min(args.cpu_seconds, max(2.0, budget_total / max(1, args.steps + args.warmup)))
    for _ in range(min(args.warmup, 1)):
        oracle_rates(2.0, cores)
    rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ts_, tp, _, _ = oracle_rates(per_step_budget, cores)
        rates.append(B * S / (S * ts_ + B * S * tp))
        if time.perf_counter() - t0 > budget_total:
            break
    wall = time.perf_counter() - t0
    value = statistics.median(rates)
    res = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "samples_timed": len(rates), "warmup": args.warmup,
           "ms_per_step": round(B * S / value * 1e3, 3),
           "ms_per_step_note": ("extrapolated: the time one full time step (16 screen updates + 128 field-screen "
                                "steps) would take at the sampled rates; each timed sample is a bounded part of a "
                                f"time step ({per_step_budget:.1f} s), not a full step"),
           "wall_seconds": round(wall, 1), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "N": wl.N, "screens": S, "beams": B},
           "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
                            "sample": f"per sample: {cores} host threads run FP64 oracle screen AR updates, then "
                                      "single-beam propagation steps at N=1024, each on its own realization; "
                                      "scaled to one time step"},
           "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def run_uneven(args):
    """64 instances, N in {256, 512, 1024, 2048}, 4..20 screens, Cn^2 log-uniform in [1e-16, 1e-14]
    (seeded), Gaussian w0 = 2 cm, dx = 2 mm, L = 1 km.  One step = one replay of the batch graph:
    screen synthesis for every instance plus ONE persistent propagation launch over all of them."""
    import torch

    import paper_2604_07248_gb300 as ts
    from paper_2604_07248_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = W.config4_instances()
    plans, fields, insts = [], [], []
    for i, d in enumerate(spec):
        p = ts.Plan(W.LAMBDA, d["N"], d["dx"], [d["L"] / d["S"]] * d["S"], [d["cn2"]] * d["S"], l0=W.L0_INNER,
                    L0=W.L0_OUTER, max_batch=1)
        p.set_sources([d["w0"]])
        f = torch.zeros((d["N"], d["N"]), dtype=torch.complex64, device=dev)
        plans.append(p)
        fields.append(f)
        insts.append(dict(plan=p, field=f, phasor=None, seed=W.SEED_BASE + 4, real=rank * len(spec) + i,
                          source=True))
    batch = ts.Batch(insts, timeout_s=10.0)
    units = sum(d["S"] for d in spec)
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        batch.run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    status = batch.status()
    counts = {}
    for d in spec:
        counts[d["N"]] = counts.get(d["N"], 0) + 1
    step_bytes = sum(screen_bytes(d["N"], d["S"]) + propagate_bytes(d["N"], 1, d["S"], 1) for d in spec)
    peak, peak_src = hbm_peak()
    gbs = step_bytes * world / (ms / args.steps * 1e-3) / 1e9
    res = {"metric": "field·screen steps/s, uneven batch (one persistent launch per step)",
           "value": round(args.steps * units * world / (ms * 1e-3), 1), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "uneven batch: 64 instances", "instances_by_N": counts,
                      "field_screen_steps_per_step": units, "batch": batch.info(), "status": status,
                      "autotune": batch.tuning()},
           "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(gbs / peak, 4), "traffic": None, "peak_source": peak_src,
                        "scope": "whole step (screen synthesis + the persistent launch), algorithmic bytes / time",
                        "algorithmic_bytes_per_step": int(step_bytes)}}
    if rank == 0:
        print(json.dumps(res), flush=True)


def run_monte_carlo(args):
    """Monte Carlo moments (N = 512, dx = 1 mm, L = 2 km, 10 screens with 3-level subharmonics, 8 Cn^2
    values 10^(-16 + 3i/7)): one step = one chunk of 32 realizations for one Cn^2 (cycling through
    the 8 values): synthesis of 32 x 10 screens (FFT part + subharmonics + piston), propagation of a
    plane wave and a 2 cm Gaussian through each realization's screens (64 fields, intensity and beam
    sums only), and the FP64 Welford merge of both groups' intensities.  Realization indices follow
    i * 1000 + r."""
    import torch

    import paper_2604_07248_gb300 as ts
    from paper_2604_07248_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cn2s = W.config2_cn2()
    wl = W.config2(cn2s[0])
    N, S, Rc = wl.N, wl.S, 32
    B = 2 * Rc
    plans = []
    for c in cn2s:
        p = ts.Plan(W.LAMBDA, N, wl.dx, wl.dz, [c] * S, l0=W.L0_INNER, L0=W.L0_OUTER, sh_levels=3, max_batch=B)
        p.set_sources([0.0, 0.02])  # field 2r: plane wave, 2r + 1: Gaussian, both through screens r
        plans.append(p)
    ph = torch.zeros((Rc, S, N, N), dtype=torch.complex64, device=dev)
    U = torch.zeros((B, N, N), dtype=torch.complex64, device=dev)
    I = torch.zeros((B, N, N), dtype=torch.float32, device=dev)
    sums = torch.zeros((B, 2), dtype=torch.float64, device=dev)
    mean = torch.zeros((len(cn2s), 2, N, N), dtype=torch.float64, device=dev)
    m2 = torch.zeros_like(mean)
    count = [0] * len(cn2s)
    chunk = [0] * len(cn2s)

    def step(k):
        i = k % len(cn2s)
        p = plans[i]
        r0 = rank * 100000 + i * 1000 + chunk[i] * Rc
        p.make_screens(None, wl.seed, real_base=r0, n_real=Rc, phasor=ph)
        p.propagate(U, B, phasor=ph, phi_group=2,
                    flags=ts.TS_PROP_SOURCE | ts.TS_PROP_INTENSITY | ts.TS_PROP_NO_FIELD, intensity=I, beam_sums=sums)
        p.moments_accumulate(I, B, 2, count[i], mean[i], m2[i])
        count[i] += Rc
        chunk[i] += 1

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    mean.zero_()
    m2.zero_()
    count = [0] * len(cn2s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        step(k)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    si = {}
    for i, c in enumerate(cn2s):
        if count[i] == 0:
            continue
        sm = torch.zeros(2, dtype=torch.float64, device=dev)
        plans[i].moments_finalize(mean[i], m2[i], 2, count[i], si_mean=sm)
        sig_r2 = 1.23 * c * (2 * 3.141592653589793 / W.LAMBDA) ** (7 / 6) * wl.L ** (11 / 6)
        si[f"{c:.3g}"] = {"realizations": count[i], "sigma_R2": round(sig_r2, 4),
                          "SI_plane_grid_mean": round(float(sm[0].item()), 4)}
    validation = mc_validation(plans, cn2s, wl, ph, U, I, sums, Rc, dev)
    units = args.steps * B * S * world
    step_bytes = (screen_bytes(N, Rc * S) + propagate_bytes(N, B, S, 2, intensity_only=True)
                  + N * N * (4 * B + 2 * 32))  # moments: intensities read, FP64 mean + M2 read + write
    peak, peak_src = hbm_peak()
    gbs = step_bytes / (ms / args.steps * 1e-3) / 1e9
    res = {"metric": "field·screen steps/s, Monte Carlo moments (screens with subharmonics, 2 sources, Welford)",
           "value": round(units / (ms * 1e-3), 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 (moments f64)", "data": "synthetic",
           "config": {"workload": "monte-carlo N=512 S=10 SH3, 8 Cn2, plane + Gaussian 2 cm", "N": N, "dx": wl.dx,
                      "L": wl.L, "screens": S, "realizations_per_step": Rc, "fields_per_step": B,
                      "screens_per_step": Rc * S, "field_screen_steps_per_step": B * S,
                      "autotune": tuning_summary(plans[0]),
                      "note": "SI of the plane wave over the whole grid; subharmonic screens are not periodic, "
                              "so the periodic grid adds seam scintillation above sigma_R^2 (informational)"},
           "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(gbs / peak, 4), "traffic": None, "peak_source": peak_src,
                        "scope": "whole step (all kernels), algorithmic bytes per step / device time per step",
                        "algorithmic_bytes_per_step": int(step_bytes)},
           "si": si, "validation": validation}
    if rank == 0:
        print(json.dumps(res), flush=True)


def mc_theory(cn2, wl, sh_levels):
    """Theory for the Monte Carlo workload's discrete model (numpy, from the phase PSD of S14 / S17 and
    the subharmonic cells of Eq. 2): the continuous sigma_R^2 (S19), the plane wave's first-order
    Rytov SI for thin screens (a screen d before the receiver adds 4 sum s^2 sin^2(kappa^2 d / 2k)),
    the 2 cm beam's long-term radius from the moment theorem (a screen adds its mean-square gradient
    / k^2 to the mean-square angle: W_LT^2 = W(L)^2 + 2 sum (d / k)^2 sum kappa^2 s^2), and Andrews'
    weak-turbulence W_LT = W sqrt(1 + 1.33 sigma_R^2 Lambda^(5/6))."""
    import numpy as np

    from paper_2604_07248_gb300 import workloads as W

    k = 2 * np.pi / W.LAMBDA
    N, dx, L, S = wl.N, wl.dx, wl.L, wl.S
    dz = L / S
    dk = 2 * np.pi / (N * dx)
    k0sq, kmsq = (2 * np.pi / W.L0_OUTER) ** 2, (2 * np.pi / W.L0_INNER) ** 2

    def phi_phi(kap2):
        return 2 * np.pi * k * k * dz * 0.033 * cn2 * (kap2 + k0sq) ** (-11 / 6) * np.exp(-kap2 / kmsq)

    f = np.fft.fftfreq(N, 1 / N) * dk
    k2 = f[None, :] ** 2 + f[:, None] ** 2
    s2 = phi_phi(k2) * dk * dk
    s2[0, 0] = 0.0
    d = [L - s * dz for s in range(1, S + 1)]
    rytov = float(sum(4 * np.sum(s2 * np.sin(k2 * ds / (2 * k)) ** 2) for ds in d))
    grad2 = float(np.sum(k2 * s2))
    if sh_levels:
        for p in range(1, 4):
            for m in (-1, 0, 1):
                for n in (-1, 0, 1):
                    if m or n:
                        kk = (m * m + n * n) * (dk / 3 ** p) ** 2
                        grad2 += kk * phi_phi(kk) * (dk / 3 ** p) ** 2
    zR = np.pi * 0.02 ** 2 / W.LAMBDA
    Wv = 0.02 * np.sqrt(1 + (L / zR) ** 2)
    sig_r2 = 1.23 * cn2 * k ** (7 / 6) * L ** (11 / 6)
    lam_ = 2 * L / (k * Wv ** 2)
    return {"sigma_R2": round(sig_r2, 5), "SI_rytov_discrete": round(rytov, 5),
            "W_LT_moment_m": round(float(np.sqrt(Wv ** 2 + 2 * sum((ds / k) ** 2 for ds in d) * grad2)), 6),
            "W_LT_andrews_m": round(float(Wv * np.sqrt(1 + 1.33 * sig_r2 * lam_ ** (5 / 6))), 6),
            "W_vacuum_m": round(float(Wv), 6)}


def mc_validation(plans, cn2s, wl, ph, U, I, sums, Rc, dev, R=1024):
    """R realizations per Cn^2 through the configured plans (subharmonics): the 2 cm beam's W_LT and
    on-axis SI; and through plans without subharmonics (periodic screens): the plane wave's SI over the
    grid against the discrete Rytov sum.  The configured subharmonic screens are not periodic, so on
    the periodic grid a plane wave picks up seam scintillation; that SI is listed as well."""
    import torch

    import paper_2604_07248_gb300 as ts
    from paper_2604_07248_gb300 import workloads as W

    N, S = wl.N, wl.S
    B = 2 * Rc
    out = {}
    for i, c in enumerate(cn2s):
        row = mc_theory(c, wl, 3)
        nosh = ts.Plan(W.LAMBDA, N, wl.dx, wl.dz, [c] * S, l0=W.L0_INNER, L0=W.L0_OUTER, max_batch=B)
        nosh.set_sources([0.0, 0.02])
        for tag, p in (("sh3", plans[i]), ("sh0", nosh)):
            mean = torch.zeros((2, N, N), dtype=torch.float64, device=dev)
            m2 = torch.zeros_like(mean)
            acc = torch.zeros((2, 2), dtype=torch.float64, device=dev)
            count = 0
            for ch in range(R // Rc):
                p.make_screens(None, wl.seed, real_base=900000 + i * 10000 + ch * Rc, n_real=Rc, phasor=ph)
                p.propagate(U, B, phasor=ph, phi_group=2,
                            flags=ts.TS_PROP_SOURCE | ts.TS_PROP_INTENSITY | ts.TS_PROP_NO_FIELD, intensity=I,
                            beam_sums=sums)
                p.moments_accumulate(I, B, 2, count, mean, m2, beam_sums=sums, beam_acc=acc)
                count += Rc
            sm = torch.zeros(2, dtype=torch.float64, device=dev)
            sc = torch.zeros(2, dtype=torch.float64, device=dev)
            w = torch.zeros(2, dtype=torch.float64, device=dev)
            p.moments_finalize(mean, m2, 2, count, si_mean=sm, si_center=sc, beam_acc=acc, w_lt=w)
            torch.cuda.synchronize(dev)
            if tag == "sh3":
                row.update({"W_LT_m": round(float(w[1].item()), 6), "SI_gauss_axis": round(float(sc[1].item()), 5),
                            "SI_plane_grid_with_subharmonic_seam": round(float(sm[0].item()), 5)})
            else:
                row.update({"SI_plane_grid_periodic_screens": round(float(sm[0].item()), 5),
                            "SI_gauss_axis_periodic_screens": round(float(sc[1].item()), 5)})
        nosh.close()
        row["realizations"] = R
        out[f"{c:.3g}"] = row
    return out


def run_d2nn(args):
    """Differentiable path (N = 512, dx = 1 mm, L = 1 km, 10 screens, Cn^2 = 5e-16, Gaussian 2 cm,
    batch 64, masks seeded N(0, 0.1 rad)): one step = forward propagation of the batch (screens
    regenerated from the seed), the two-mask receiver and its MAE loss against the apertured vacuum
    intensity, then the receiver adjoint (mask gradients) and the adjoint propagation (screens
    regenerated again).  Units: 64 x 10 forward + 64 x 10 adjoint field-screen steps."""
    import numpy as np
    import torch

    import paper_2604_07248_gb300 as ts
    from paper_2604_07248_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = W.config5()
    N, S, B, AP = wl.N, wl.S, wl.realizations, wl.extra["aperture"]
    plan = ts.Plan(W.LAMBDA, N, wl.dx, wl.dz, wl.cn2, l0=W.L0_INNER, L0=W.L0_OUTER, max_batch=B)
    plan.set_sources(wl.w0)
    vac = ts.Plan(W.LAMBDA, N, wl.dx, wl.dz, [0.0] * S, max_batch=1)
    vac.set_sources(wl.w0)
    th1 = torch.from_numpy(np.random.default_rng(wl.seed).normal(0, 0.1, (N, N)).astype(np.float32)).to(dev)
    th2 = torch.from_numpy(np.random.default_rng(wl.seed + 1).normal(0, 0.1, (N, N)).astype(np.float32)).to(dev)
    Uv = torch.zeros((1, N, N), dtype=torch.complex64, device=dev)
    vac.propagate(Uv, 1, flags=ts.TS_PROP_SOURCE)
    z = torch.zeros((N, N), dtype=torch.float32, device=dev)
    Iv = torch.zeros((1, N, N), dtype=torch.float32, device=dev)
    vac.d2nn_forward(Uv, 1, z, z, AP, z, 1, torch.zeros((3, 1, N, N), dtype=torch.complex64, device=dev), Iv,
                     torch.zeros(1, dtype=torch.float64, device=dev))
    Iref = Iv[0].contiguous()
    U = torch.zeros((B, N, N), dtype=torch.complex64, device=dev)
    ws = torch.zeros((3, B, N, N), dtype=torch.complex64, device=dev)
    I = torch.zeros((B, N, N), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g1, g2 = torch.zeros_like(z), torch.zeros_like(z)
    gU = torch.zeros_like(U)
    real0 = rank * 1000000

    def step(k):
        real = real0 + k * B
        plan.propagate(U, B, flags=ts.TS_PROP_SOURCE, seed=wl.seed, real_base=real)
        plan.d2nn_forward(U, B, th1, th2, AP, Iref, 0, ws, I, loss)
        plan.d2nn_backward(B, th1, th2, AP, Iref, 0, ws, I, g1, g2, gU)
        plan.propagate_backward(gU, B, seed=wl.seed, real_base=real)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        step(args.warmup + k)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    units = args.steps * 2 * B * S * world
    # forward and adjoint propagation regenerate one screen per field and step (24 B/px each, read
    # back as an 8-byte phasor by the row pass); the receiver passes move ~10 field-sized arrays each way
    step_bytes = (2 * propagate_bytes(N, B, S, 1) + 2 * S * screen_bytes(N, B)
                  + N * N * B * 8 * 20)
    peak, peak_src = hbm_peak()
    gbs = step_bytes / (ms / args.steps * 1e-3) / 1e9
    res = {"metric": "field·screen steps/s, differentiable path (forward + adjoint, two-mask receiver)",
           "value": round(units / (ms * 1e-3), 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 (loss f64)", "data": "synthetic",
           "config": {"workload": "d2nn N=512 S=10 B=64, MAE loss, screens regenerated from the seed", "N": N,
                      "dx": wl.dx, "L": wl.L, "screens": S, "batch": B, "aperture_m": AP,
                      "field_screen_steps_per_step": 2 * B * S, "autotune": tuning_summary(plan)},
           "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(gbs / peak, 4), "traffic": None, "peak_source": peak_src,
                        "scope": "whole step (all kernels), algorithmic bytes per step / device time per step",
                        "algorithmic_bytes_per_step": int(step_bytes)},
           "last_loss": float(loss.item()), "grad_norms": [float(g1.norm().item()), float(g2.norm().item())]}
    if rank == 0:
        print(json.dumps(res), flush=True)


def run_single_path(args):
    """One path (N = 128, dx = 2 mm, L = 1 km, 5 screens, Cn^2 = 1e-15, Gaussian w0 = 2 cm): one step
    = one ts_propagate call from the source with every screen regenerated from the seed (screen
    synthesis + column + row pass per step), captured once in a CUDA graph and replayed, so the
    number is the device latency of a whole path.  Also reported: the same call launched eagerly."""
    import torch

    import paper_2604_07248_gb300 as ts
    from paper_2604_07248_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = W.config1()
    N, S = wl.N, wl.S
    plan = ts.Plan(W.LAMBDA, N, wl.dx, wl.dz, wl.cn2, l0=W.L0_INNER, L0=W.L0_OUTER, max_batch=1)
    plan.set_sources(wl.w0)
    U = torch.zeros((1, N, N), dtype=torch.complex64, device=dev)
    side = torch.cuda.Stream(dev)
    real = [rank * 1000000]

    def path(stream):
        plan.propagate(U, 1, flags=ts.TS_PROP_SOURCE, seed=wl.seed, real_base=real[0], stream=stream)

    # eager launches
    for _ in range(args.warmup):
        path(torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    n_eager = min(args.steps, 256)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n_eager):
        path(torch.cuda.current_stream(dev))
    e1.record()
    torch.cuda.synchronize()
    eager_us = e0.elapsed_time(e1) * 1e3 / n_eager
    # the same call captured once in a CUDA graph
    side.wait_stream(torch.cuda.current_stream(dev))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        path(side)  # warm the side stream before capture
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=side):
            path(side)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / args.steps
    # the same path as a one-instance uneven batch: screen synthesis + ONE persistent propagation launch,
    # replayed as the batch's CUDA graph
    Ub = torch.zeros((N, N), dtype=torch.complex64, device=dev)
    batch = ts.Batch([dict(plan=plan, field=Ub, phasor=None, seed=wl.seed, real=real[0], source=True)], timeout_s=5.0)
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        batch.run()
    e1.record()
    torch.cuda.synchronize()
    batch_us = e0.elapsed_time(e1) * 1e3 / args.steps
    batch_ok = batch.status() == 0
    launches = 3 + 2 * S  # screen synthesis (column + row pass, all 5 screens), first row pass, 5 x (column, row)
    res = {"metric": "µs per path (device latency, CUDA-graph replay), N=128 single path", "value": round(us, 2),
           "unit": "us/path", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(us * 1e-3, 5), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "single path N=128 S=5 (config 1), screens regenerated from the seed", "N": N,
                      "dx": wl.dx, "L": wl.L, "screens": S, "launches_per_path": launches},
           "eager_us_per_path": round(eager_us, 2),
           "batch_us_per_path": round(batch_us, 2) if batch_ok else None,
           "field_screen_steps_per_s": round(S * world / (us * 1e-6), 1)}
    if rank == 0:
        print(json.dumps(res), flush=True)


def run_d2nn_train(args):
    """D2NN training (Sec. 2.5): 1024 x 1024 grid, 0.34 mm pixels, 1064 nm, 0.15 mrad beam (read as the
    full divergence: waist 4.5 mm), a 1500 m vertical HV5/7 path whose ground constant gives
    sigma_R^2 = 0.2, screens placed by the planner (Rytov limit 0.1 per interval, Eq. 7 steps), 12-inch
    aperture, two-mask receiver, MAE against the free-space intensity, Adam with a one-cycle schedule
    peaking at lr = 0.01 over 20 000 epochs, one turbulence realization per epoch.  One step = one
    epoch.  The paper's figure for this run: 20 000 epochs in 11 min on an RTX 4090."""
    import torch

    from paper_2604_07248_gb300 import training as tr
    from paper_2604_07248_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lam, N, dx, L, total = 1.064e-6, 1024, 0.34e-3, 1500.0, 20000
    w0 = lam / (3.141592653589793 * 0.075e-3)
    A, h, cn2p, dz, cn2 = tr.hv57_path(lam, L, 0.2, N, dx, 0.1)
    trainer = tr.D2nnTrainer(lam, N, dx, list(dz), list(cn2), w0, 0.3048, W.SEED_BASE + 6, total, l0=W.L0_INNER,
                             L0=W.L0_OUTER, device=dev)
    stream = torch.cuda.current_stream(dev)
    e0_epoch = rank * 10 ** 6
    for e in range(args.warmup):
        trainer.epoch(e0_epoch + e, stream=stream)
    torch.cuda.synchronize()
    first_loss = trainer.loss.item()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for e in range(args.warmup, args.warmup + args.steps):
        trainer.epoch(e0_epoch + e, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    value = args.steps * world / (ms * 1e-3)
    paper = 20000 / 660.0
    res = {"metric": "D2NN training epochs/s (Sec. 2.5 set-up, one realization per epoch)", "value": round(value, 2),
           "unit": "epochs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": round(value / paper, 2), "dtype": "f32 (loss f64)", "data": "synthetic",
           "config": {"workload": "d2nn-train N=1024 dx=0.34mm 1064nm HV5/7 1500m sigma_R2=0.2", "N": N, "dx": dx,
                      "lambda": lam, "w0_m": round(w0, 6), "L": L, "hv_A": float(f"{A:.4g}"), "screens": len(dz),
                      "dz_m": [round(float(x), 2) for x in dz], "aperture_m": 0.3048, "loss": "MAE",
                      "optimizer": "Adam, one-cycle lr (peak 0.01, 20000 epochs)",
                      "epochs_timed": [args.warmup, args.warmup + args.steps]},
           "projected_20000_epochs_s": round(20000 / value * world, 1),
           "baseline_note": "paper: 20 000 epochs in 11 min on an NVIDIA RTX 4090 (30.3 epochs/s); other hardware, "
                            "screen count not stated",
           "loss_first_timed_epoch_region": [first_loss, trainer.loss.item()]}
    if rank == 0:
        print(json.dumps(res), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "monte-carlo":
        run_monte_carlo(args)
    elif args.workload == "d2nn":
        run_d2nn(args)
    elif args.workload == "single-path":
        run_single_path(args)
    elif args.workload == "d2nn-train":
        run_d2nn_train(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
