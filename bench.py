#!/usr/bin/env python3
"""Throughput of the swept-source holographic OCT reconstruction on GB300.

One step = one whole reconstruction of a 1024 x 1024 x 256 volume from uint16
frames already resident in HBM: chromatic rescale (Eq. 5) + Fresnel transform
(Eq. 6) of all 256 frames, sweep-axis transform (Eq. 7), |V|^2 volume, and the
three orthogonal cuts.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ssoct|reference]

--impl reference times the FP64 CPU oracle on this host's cores on a bounded
sample of the same workload.  Under torchrun (N > 1) each rank reconstructs its
own volumes (replicas: the path has no exchange step between volumes).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gvoxel/s, 1024²×256 volume recon, FP32 vs tensor-core form; % of HBM roofline"
UNIT = "Gvoxel/s"
WORKLOAD = "paper_1024x1024x256"
PAPER_GVOXEL_PER_S = 10.0   # TITAN Xp, Table 1 of the paper (context only)
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1700.0  # sustained bf16 of one earlier GB300 measurement
TC_FLOP_PER_VOXEL = 768        # tensor-core axial form, see _tc_form


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def _bf16_peak():
    """Dense bf16 TFLOP/s for a kernel timed inside a long step (the sustained
    figure), and where it comes from."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if "bf16_tflops_sustained" in d:
            return float(d["bf16_tflops_sustained"]), "measured (sustained)"
    return FALLBACK_BF16_TFLOPS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 20 ms while running."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def mark(self, begin: bool):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(f[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + f[0].split(".")[1]) if "." in f[0] else 0.0
                rows.append((ts, float(f[2]), float(f[3]), f[5:]))
            except (ValueError, IndexError):
                continue
        if not rows:
            return None
        inside = [r for r in rows if self.t0 - 0.05 <= r[0] <= self.t1 + 0.05] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in inside:
            for n, v in zip(names, r[3][1:]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(local_ms: float, voxels_per_rank: int, world: int, dist=None, device="cpu"):
    """Whole-job throughput: every rank reconstructs its own volumes, the job's
    time per step is the slowest rank's, value = all ranks' voxels / that time.
    Returns (max ms over ranks, Gvoxel/s)."""
    ms = float(local_ms)
    if world > 1 and dist is not None:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * voxels_per_rank / (ms * 1e-3) / 1e9


def oracle_rate(w, n_frames: int):
    """FP64 oracle (as it stands) on a gate of the first n_frames frames of the
    workload: returns (voxels per second, seconds, threads)."""
    import oracle
    t = time.perf_counter()
    oracle.reconstruct(w.frames[:n_frames], w.pitch, w.z, w.lambdas[:n_frames], method="fft")
    dt = time.perf_counter() - t
    return w.nx * w.ny * n_frames / dt, dt, os.cpu_count()


def oracle_rate_single_core(w, budget_s: float = 8.0):
    """The same oracle with scipy.fft held to one thread, on a smaller sample:
    returns (voxels per second, frames, seconds)."""
    import oracle.ssoct_oracle as so
    old = so.WORKERS
    so.WORKERS = 1
    try:
        rate, dt, _ = oracle_rate(w, 2)
        n = int(max(2, min(w.nlambda, budget_s / (dt / 2.0))))
        rate, dt, _ = oracle_rate(w, n)
    finally:
        so.WORKERS = old
    return rate, n, dt


def _sample_frames(w, budget_s: float) -> int:
    rate, dt, _ = oracle_rate(w, 2)
    per_frame = dt / 2.0
    return int(max(2, min(w.nlambda, budget_s / per_frame)))


def run_reference(args):
    world, rank, local = _dist()
    if rank != 0:
        return
    import synth
    w = synth.workload(WORKLOAD)
    budget = max(0.5, 150.0 / (args.steps + args.warmup))
    n = _sample_frames(w, budget)
    for _ in range(args.warmup):
        oracle_rate(w, n)
    times = []
    for _ in range(args.steps):
        _, dt, cores = oracle_rate(w, n)
        times.append(dt)
    total = sum(times)
    vox = w.nx * w.ny * n
    value = vox * args.steps / total / 1e9
    sample = (f"oracle.reconstruct (float64 numpy/scipy.fft) of a {w.nx}x{w.ny}x{n} gate: the first {n} "
              f"frames of the {w.nx}x{w.ny}x{w.nlambda} workload, per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_GVOXEL_PER_S,
        "dtype": "f64", "data": "synthetic (seeded point scatterers, 12-bit, Gaussian read noise)",
        "config": {"workload": f"{w.nx}x{w.ny}x{w.nlambda} sweep, FP64 CPU oracle on a {n}-frame sample",
                   "window": [0, 0, w.nx, w.ny]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ssoct(args):
    import torch
    import torch.distributed as dist

    import paper_2003_08960_gb300 as ss
    import synth

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.size:
        nx, ny, nl = (int(v) for v in args.size.split("x"))
        w = synth.workload("custom", nx=nx, ny=ny, nlambda=nl, kind="points", seed=3 + rank)
    else:
        w = synth.workload(WORKLOAD, seed=3 + rank)
    flags = (ss.SSOCT_FLAG_TC_AXIAL if args.tc_axial else 0) | (ss.SSOCT_FLAG_AXIAL_FIRST if args.axial_first else 0)
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, flags=flags)
    h = plan.handle
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    frames = torch.from_numpy(w.frames.view(np.int16)).cuda()
    vol, _ = plan.empty_volume()
    nl, wy, wx = plan.volume_shape()
    # schedule of the persistent lateral kernel (and axial form, if --tc-axial
    # is not forcing it) chosen by the library's autotuner on these frames
    tune = None
    tune_cache = None
    if not args.no_autotune and not args.tc_axial:
        import tempfile
        fd, tune_cache = tempfile.mkstemp(suffix=".json", prefix="ssoct_tune_")
        os.close(fd)
        os.unlink(tune_cache)  # the tuner writes it; other plans of the bench read the choice back
        tune = plan.autotune(frames, tune_cache, stream)
    tc_main = args.tc_axial or bool(tune and tune["tc_axial"])
    af_main = args.axial_first or bool(tune and tune["axial_first"])
    xy = torch.empty((wy, wx), dtype=torch.float32, device="cuda")
    xz = torch.empty((nl, wx), dtype=torch.float32, device="cuda")
    yz = torch.empty((nl, wy), dtype=torch.float32, device="cuda")
    cut = (wx // 2 + wx // 4, wy // 2 + wy // 4, nl // 2)
    torch.cuda.synchronize()

    def step():
        st = ss.ssoct_reconstruct_frames(h, frames.data_ptr(), vol.data_ptr(), 0, sp)
        st |= ss.ssoct_get_cuts(h, vol.data_ptr(), cut[0], cut[1], cut[2], xy.data_ptr(), xz.data_ptr(),
                                yz.data_ptr(), sp)
        if st:
            raise RuntimeError(ss.ssoct_last_error(h))

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        step()
    if ss.ssoct_sync(h, sp) != 0:
        raise RuntimeError(ss.ssoct_last_error(h))
    ss.ssoct_profile(h, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark(True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark(False)
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    st = ss.ssoct_sync(h, sp)
    if st != 0:
        raise RuntimeError("kernel error: " + ss.ssoct_last_error(h))
    _, lat_ms, ax_ms, calls = ss.ssoct_profile_read(h)
    ss.ssoct_profile(h, False)
    clk = clocks.stop()
    # the spread of single steps (each between its own events), after the timed loop
    n_single = max(20, min(args.steps, 50))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_single)]
    for a, b in evs:
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    singles = sorted(a.elapsed_time(b) for a, b in evs)
    step_ms = {"median": statistics.median(singles), "min": singles[0], "max": singles[-1], "n": n_single,
               "note": "single steps, each between its own CUDA events, after the timed loop"}
    lat_ms /= max(calls, 1)
    ax_ms /= max(calls, 1)
    voxels = wx * wy * nl
    ms, value = aggregate(ms, voxels, world, dist if world > 1 else None, device="cuda")

    peak, peak_kind = _peaks()
    # single-GPU side lines (the N-GPU run keeps the main line and the end-to-end
    # line, which every rank measures as a replica)
    extra = not args.no_e2e and world == 1
    # end to end: pinned host frames -> ring (H2D) -> reconstruct -> volume to
    # pinned host (D2H); first of the extra lines, before the others fill the
    # device with their plans and graphs
    e2e = (_e2e(args, ss, torch, dist, w, plan, vol, nl, voxels, world, flags, frames, tune_cache)
           if not args.no_e2e else None)
    tc = _tc_form(args, ss, torch, w, frames, vol, stream, voxels, peak) if extra and not tc_main else None
    sliding = _sliding(args, ss, torch, plan, frames, vol, nl, voxels, stream) if extra else None
    if sliding is not None and args.size is None:
        sliding["push_stream"] = _push_stream(args, ss, torch, w, voxels)
    aberration = _aberration(args, ss, torch, synth, stream) if extra else None
    batched = _batched(args, ss, torch, synth, w, frames, stream) if extra else None

    # library-free comparison, last so that its buffers do not touch the lines above
    cufft = _cufft_chain(torch, frames, nl, w.ny, w.nx, voxels) if extra and not tc_main else None
    # error of each form against the FP64 oracle, per volume, outside every timed region
    parity = None
    tc_plan = tc.pop("_plan", None) if tc else None
    if rank == 0 and world == 1 and not args.no_parity:
        import oracle
        t_or = time.perf_counter()
        ref = oracle.reconstruct(w.frames, w.pitch, w.z, w.lambdas, method="fft")
        t_or = time.perf_counter() - t_or
        parity = _parity(ss, torch, plan, frames, ref, stream, 1e-3 if tc_main else 1e-5)
        parity["oracle_s"] = t_or
        parity["note"] = ("this line's form and schedule vs oracle.reconstruct (float64 scipy.fft) of the same "
                          "frames, whole volume")
        if tc_plan is not None:
            tc["rel_l2_vs_oracle"] = _parity(ss, torch, tc_plan, frames, ref, stream, 1e-3)
        del ref
    if tc_plan is not None:
        del tc_plan
    if af_main:
        # rescale-axial pass: uint16 frames in, half-spectrum planes out; lateral
        # pass: the planes in (each read once from HBM, its conjugate use from L2),
        # |V|^2 out
        plane_bytes = w.nx * w.ny * (nl // 2 + 1) * 8
        ax_bytes = w.nx * w.ny * nl * 2 + plane_bytes
        lat_bytes = plane_bytes + voxels * 4
    else:
        lat_bytes = w.nx * w.ny * nl * 2 + voxels * 8
        ax_bytes = voxels * (8 + 4)
    kernels = {
        "lateral": {"ms": lat_ms, "bytes": lat_bytes, "GBps": lat_bytes / (lat_ms * 1e-3) / 1e9},
        "axial": {"ms": ax_ms, "bytes": ax_bytes, "GBps": ax_bytes / (ax_ms * 1e-3) / 1e9},
    }
    for k in kernels.values():
        k["frac"] = k["GBps"] / peak
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    # stored counters of the kernel that dominates this line's form, taken at the
    # 1024x1024x256 workload (see profiles/traffic.json)
    if af_main:
        tkey = {"lateral": "lateral_af", "axial": "rescale_axial"}[dom]
    else:
        tkey = "axial_tc" if (tc_main and dom == "axial") else dom
    traffic = _traffic(tkey) if args.size is None else None
    whole_bytes = lat_bytes + ax_bytes
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "step_ms": step_ms, "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": value / PAPER_GVOXEL_PER_S, "dtype": "f32",
        "data": "synthetic (seeded point scatterers, 12-bit, Gaussian read noise)",
        "config": {"workload": f"{w.nx}x{w.ny}x{nl} sweep, uint16 frames resident in HBM, full window, "
                               "|V|^2 volume + 3 cuts per step",
                   "window": [0, 0, wx, wy],
                   "schedule": ({k: tune[k] for k in ("lag", "ring_slots", "tc_axial", "axial_first")} if tune
                                else f"plan default (lag {plan.info.ring_slots - 4}, {plan.info.ring_slots} ring slots)"),
                   "form": ("fp32, axial-first order (Eq. 5 + Eq. 7, then Eq. 6 per depth bin)" if af_main
                            else "tensor-core axial (bf16 hi+lo, fp32 accumulate)" if tc_main else "fp32 (paper order)"),
                   "l2": "inputs larger than L2 (512 MiB frames, 2 GiB intermediate per step)"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": kernels[dom]["GBps"], "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": kernels[dom]["frac"],
                     "traffic": traffic},
        "whole_step_hbm": {"bytes_per_voxel": whole_bytes / voxels,
                           "GBps": whole_bytes / (ms * 1e-3) / 1e9,
                           "frac": whole_bytes / (ms * 1e-3) / 1e9 / peak},
        "kernels": kernels,
        "rel_l2_vs_oracle": parity,
        "e2e": e2e,
        "sliding": sliding,
        "tc_axial": tc,
        "aberration": aberration,
        "batched": batched,
        "cufft_comparison": cufft,
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n = _sample_frames(w, 15.0)
        rate, dt, cores = oracle_rate(w, n)
        out["cpu_baseline"] = {"value": rate / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"FP64 oracle on the first {n} frames ({w.nx}x{w.ny}x{n} gate), {dt:.1f} s"}
        r1, n1, dt1 = oracle_rate_single_core(w)
        out["cpu_baseline"]["single_core"] = {
            "value": r1 / 1e9, "unit": UNIT, "cores": 1,
            "sample": f"the same oracle with scipy.fft on one thread, first {n1} frames, {dt1:.1f} s"}
    if tune_cache and os.path.exists(tune_cache):
        os.unlink(tune_cache)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _e2e(args, ss, torch, dist, w, plan, vol, nl, voxels, world, flags, frames, tune_cache):
    """Same metric through the C ABI with host buffers: every step pushes its
    frames from pinned host memory into a plan's ring (H2D), reconstructs the
    volume and reads it back to pinned host memory (D2H), all inside the timed
    region.  Two plans (two rings) and three streams let step k's H2D overlap
    step k-1's reconstruction and step k-2's D2H, as an acquisition pipeline
    would run; events keep each ring and volume buffer from being reused early.

    Right before the pipelined loop the same process times the host link on
    the same buffers: the H2D copy alone, the D2H copy alone, and both at once
    on two streams, so the record shows whether the two directions overlap.
    The loop runs twice, with the D2H as one copy and as four chunks (one
    cudaMemcpyAsync each), and the line keeps the faster."""
    plans = [plan, ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, flags=flags)]
    if tune_cache:
        plans[1].autotune(frames, tune_cache)  # the same choice as the main plan, from the cache
    vols = [vol, torch.empty_like(vol)]
    host_frames = torch.from_numpy(w.frames.view(np.int16)).pin_memory()
    host_vols = [torch.empty(vol.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    s_h2d, s_comp, s_d2h = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_h2d = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_d2h = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(3, min(args.steps, 20))
    h2d_bytes = int(host_frames.numel() * 2)
    d2h_bytes = int(host_vols[0].numel() * 4)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    dev_frames = torch.empty(host_frames.shape, dtype=host_frames.dtype, device="cuda")

    def link(h2d: bool, d2h: bool, reps: int = 5, chunks: int = 1):
        """ms per repetition of the H2D and/or D2H copy (both: concurrently on two
        streams; the D2H as `chunks` copies)."""
        def once(i):
            if h2d:
                with torch.cuda.stream(s_h2d):
                    dev_frames.copy_(host_frames, non_blocking=True)
            if d2h:
                src, dst = vols[i % 2].view(-1), host_vols[i % 2].view(-1)
                n = src.numel()
                with torch.cuda.stream(s_d2h):
                    for c in range(chunks):
                        lo, hi = n * c // chunks, n * (c + 1) // chunks
                        dst[lo:hi].copy_(src[lo:hi], non_blocking=True)
        once(0)
        torch.cuda.synchronize()
        e0.record(s_h2d)
        s_d2h.wait_event(e0)
        for i in range(reps):
            once(i)
        s_h2d.wait_stream(s_d2h)
        e1.record(s_h2d)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    h2d_ms, d2h_ms, both_ms = link(True, False), link(False, True), link(True, True)
    link_rec = {"h2d_ms": h2d_ms, "h2d_GBps": h2d_bytes / (h2d_ms * 1e-3) / 1e9,
                "d2h_ms": d2h_ms, "d2h_GBps": d2h_bytes / (d2h_ms * 1e-3) / 1e9,
                "both_ms": both_ms, "both_GBps": (h2d_bytes + d2h_bytes) / (both_ms * 1e-3) / 1e9,
                "overlap": (h2d_ms + d2h_ms) / both_ms,
                "note": "pinned host <-> device copies of one step's frames and volume, timed in this "
                        "process right before the pipelined loop; overlap = (H2D alone + D2H alone) / "
                        "both at once (1 = serialised, 2 = fully overlapped)"}

    def run_loop(chunks: int) -> float:
        flat = [v.view(-1) for v in vols]
        hflat = [v.view(-1) for v in host_vols]
        n = flat[0].numel()
        bounds = [n * c // chunks for c in range(chunks + 1)]

        def e2e_step(k):
            i = k % 2
            h = plans[i].handle
            if k >= 2:
                s_h2d.wait_event(ev_comp[i])      # the ring's previous gate has been read
            if ss.ssoct_push_frames(h, host_frames.data_ptr(), nl, False, -1, s_h2d.cuda_stream):
                raise RuntimeError(ss.ssoct_last_error(h))
            ev_h2d[i].record(s_h2d)
            s_comp.wait_event(ev_h2d[i])
            if k >= 2:
                s_comp.wait_event(ev_d2h[i])      # the volume buffer has been read back
            if ss.ssoct_reconstruct_volume(h, vols[i].data_ptr(), 0, s_comp.cuda_stream):
                raise RuntimeError(ss.ssoct_last_error(h))
            ev_comp[i].record(s_comp)
            s_d2h.wait_event(ev_comp[i])
            with torch.cuda.stream(s_d2h):
                for c in range(chunks):
                    hflat[i][bounds[c]:bounds[c + 1]].copy_(flat[i][bounds[c]:bounds[c + 1]], non_blocking=True)
            ev_d2h[i].record(s_d2h)

        for k in range(2):
            e2e_step(k)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0.record(s_h2d)
        for k in range(2, 2 + e2e_steps):
            e2e_step(k)
        s_d2h.wait_stream(s_h2d)
        s_d2h.wait_stream(s_comp)
        e1.record(s_d2h)
        torch.cuda.synchronize()
        for pl in plans:
            if ss.ssoct_sync(pl.handle, 0):
                raise RuntimeError("kernel error: " + ss.ssoct_last_error(pl.handle))
        return e0.elapsed_time(e1) / e2e_steps

    by_chunks = {1: run_loop(1), 4: run_loop(4)}
    chunks = min(by_chunks, key=by_chunks.get)
    e2e_ms = by_chunks[chunks]
    # the link's floor for the same bytes: the same H2D and D2H copies (the D2H
    # split as in the loop kept), with no kernels, on the same two streams, timed
    # again right after the loop; the faster of that and the timing before the
    # loop (long queues of whole-volume copies sometimes serialise the two
    # directions, which would make the floor look slower than the loop)
    copy_ms = min(link(True, True, reps=e2e_steps, chunks=chunks),
                  both_ms if chunks == 1 else link(True, True, chunks=chunks))
    e2e_ms, e2e_value = aggregate(e2e_ms, voxels, world, dist if world > 1 else None, device="cuda")
    return {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d_bytes,
            "d2h_bytes_per_step": d2h_bytes, "ms_per_step": e2e_ms,
            "ms_by_d2h_chunks": by_chunks, "d2h_chunks": chunks,
            "copy_floor_ms": copy_ms, "frac_of_copy_floor": copy_ms / e2e_ms,
            "link_before_loop": link_rec,
            "pipeline": "2 rings, H2D / reconstruct / D2H on 3 streams; copy floor = the same copies "
                        "alone on the same streams (pinned host memory, host link bound), the D2H split "
                        "as in the loop, the faster of two timings"}


def _sliding(args, ss, torch, plan, frames, vol, nl, voxels, stream, step_frames=13):
    """Sliding gates (streaming): each step pushes `step_frames` new frames (from
    device memory) into the ring and reconstructs the gate of the last nl frames,
    transforming only the new frames laterally.  13 frames per volume is the
    paper's ratio of 512 frames/s to about 38 volumes/s."""
    h = plan.handle
    sp = stream.cuda_stream
    fb = frames.element_size() * frames[0].numel()

    def push(k, start):
        for i in range(k):
            f = (start + i) % nl
            if ss.ssoct_push_frames(h, frames.data_ptr() + f * fb, 1, True, -1, sp):
                raise RuntimeError(ss.ssoct_last_error(h))

    push(nl, 0)
    if ss.ssoct_reconstruct_sliding(h, vol.data_ptr(), 0, sp):
        raise RuntimeError(ss.ssoct_last_error(h))
    pos = nl
    for _ in range(3):
        push(step_frames, pos)
        pos += step_frames
        ss.ssoct_reconstruct_sliding(h, vol.data_ptr(), 0, sp)
    steps = max(10, args.steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        push(step_frames, pos)
        pos += step_frames
        if ss.ssoct_reconstruct_sliding(h, vol.data_ptr(), 0, sp):
            raise RuntimeError(ss.ssoct_last_error(h))
    e1.record(stream)
    torch.cuda.synchronize()
    if ss.ssoct_sync(h, sp):
        raise RuntimeError("kernel error: " + ss.ssoct_last_error(h))
    ms = e0.elapsed_time(e1) / steps
    # display mode: the same gate updates, only the three cuts of each gate
    nl_, wy, wx = plan.volume_shape()
    xy = torch.empty((wy, wx), dtype=torch.float32, device="cuda")
    xz = torch.empty((nl_, wx), dtype=torch.float32, device="cuda")
    yz = torch.empty((nl_, wy), dtype=torch.float32, device="cuda")
    cut = (wx // 2 + wx // 4, wy // 2 + wy // 4, nl_ // 2)

    def cuts_step():
        nonlocal pos
        push(step_frames, pos)
        pos += step_frames
        if ss.ssoct_sliding_cuts(h, cut[0], cut[1], cut[2], xy.data_ptr(), xz.data_ptr(), yz.data_ptr(), sp):
            raise RuntimeError(ss.ssoct_last_error(h))

    for _ in range(3):
        cuts_step()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        cuts_step()
    e1.record(stream)
    torch.cuda.synchronize()
    if ss.ssoct_sync(h, sp):
        raise RuntimeError("kernel error: " + ss.ssoct_last_error(h))
    ms_cuts = e0.elapsed_time(e1) / steps
    return {"step_frames": step_frames, "ms_per_volume": ms, "volumes_per_s": 1000.0 / ms,
            "Gvoxel_per_s": voxels / (ms * 1e-3) / 1e9,
            "cuts_only": {"ms_per_gate": ms_cuts, "gates_per_s": 1000.0 / ms_cuts,
                          "note": "ssoct_sliding_cuts: xy, xz, yz of each gate, no volume; xy as a running "
                                  "sum over the gate (new holograms in, replaced ones out), summed in full "
                                  "again after every nlambda swapped-in frames"},
            "paper": "38 volumes/s (TITAN Xp, sliding 256-frame gate, 512 frames/s)"}


def _push_stream(args, ss, torch, w, voxels, step_frames=13, fps=512.0):
    """The paper's acquisition pattern (Table 1: 512 frames/s, about 38 volumes/s
    from a sliding 256-frame gate): frames arrive one at a time in pinned host
    memory, each is pushed on its own (ssoct_push_frames, one 2 MiB H2D copy),
    and after every `step_frames` frames the gate of the last nlambda frames is
    reconstructed (ssoct_reconstruct_sliding).  Run twice: paced by the host at
    `fps` frames per second, and as fast as the host can issue.  Latency is
    GPU time from the start of the gate's last frame copy to the end of its
    volume (CUDA events on the stream)."""
    import time
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas)
    h = plan.handle
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    host = torch.from_numpy(w.frames.view(np.int16)).pin_memory()
    fbytes = host[0].numel() * 2
    vol, _ = plan.empty_volume()
    nl = w.nlambda

    def run(n_frames, paced, seq0):
        marks = []
        t_start = time.perf_counter()
        for i in range(n_frames):
            if paced:
                due = t_start + i / fps
                while time.perf_counter() < due:
                    pass
            last = (i + 1) % step_frames == 0 and seq0 + i + 1 >= nl   # a full gate is in
            if last:
                a = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            if ss.ssoct_push_frames(h, host.data_ptr() + ((seq0 + i) % nl) * fbytes, 1, False, seq0 + i, sp):
                raise RuntimeError(ss.ssoct_last_error(h))
            if last:
                if ss.ssoct_reconstruct_sliding(h, vol.data_ptr(), 0, sp):
                    raise RuntimeError(ss.ssoct_last_error(h))
                b = torch.cuda.Event(enable_timing=True)
                b.record(stream)
                marks.append((a, b))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_start
        if ss.ssoct_sync(h, sp):
            raise RuntimeError("kernel error: " + ss.ssoct_last_error(h))
        lat = sorted(a.elapsed_time(b) for a, b in marks) or [float("nan")]
        return {"frames": n_frames, "wall_s": wall, "frames_per_s": n_frames / wall,
                "volumes_per_s": len(marks) / wall, "Gvoxel_per_s": len(marks) * voxels / wall / 1e9,
                "latency_ms": {"median": statistics.median(lat), "max": lat[-1]}}

    # fill the gate, then warm up
    run(nl + 2 * step_frames, False, 0)
    seq = nl + 2 * step_frames
    fast = run(2 * nl, False, seq)
    seq += 2 * nl
    paced = run(nl, True, seq)
    return {"step_frames": step_frames, "fast": fast, "paced_512fps": paced,
            "form": "one ssoct_push_frames per frame from pinned host memory (2 MiB H2D each), "
                    "ssoct_reconstruct_sliding after every step_frames frames; latency = GPU time from the "
                    "start of the gate's last frame copy to the end of its volume",
            "paper": "512 frames/s in, up to 38 volumes/s out (TITAN Xp)"}


def _tc_form(args, ss, torch, w, frames, vol, stream, voxels, peak):
    """The same step with the axial DFT on the tensor cores (SSOCT_FLAG_TC_AXIAL),
    on the same frames; its error against the FP64 oracle is added by the caller."""
    if w.nlambda != 256:
        return None
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, flags=ss.SSOCT_FLAG_TC_AXIAL)
    h, sp = plan.handle, stream.cuda_stream
    vt, _ = plan.empty_volume()

    def step():
        if ss.ssoct_reconstruct_frames(h, frames.data_ptr(), vt.data_ptr(), 0, sp):
            raise RuntimeError(ss.ssoct_last_error(h))

    for _ in range(args.warmup):
        step()
    if ss.ssoct_sync(h, sp) != 0:
        raise RuntimeError(ss.ssoct_last_error(h))
    ss.ssoct_profile(h, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    if ss.ssoct_sync(h, sp) != 0:
        raise RuntimeError(ss.ssoct_last_error(h))
    _, lat_ms, ax_ms, calls = ss.ssoct_profile_read(h)
    ax_ms /= max(calls, 1)
    ax_bytes = voxels * (8 + 4)
    # tensor work: per 32-pixel tile, 4 blocks x 3 products (hi.hi, hi.lo,
    # lo.hi) x 2 stages of a 128 x 32 x 32 real GEMM = 768 flop per voxel
    tflops = TC_FLOP_PER_VOXEL * voxels / (ax_ms * 1e-3) / 1e12
    tpeak, tkind = _bf16_peak()
    return {"value": voxels / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "axial_ms": ax_ms, "axial_GBps": ax_bytes / (ax_ms * 1e-3) / 1e9,
            "axial_frac": ax_bytes / (ax_ms * 1e-3) / 1e9 / peak,
            "tensor_roofline": {"bound": "tensor", "achieved": tflops, "peak": tpeak, "peak_kind": tkind,
                                "unit": "TFLOP/s", "frac": tflops / tpeak,
                                "flop_per_voxel": TC_FLOP_PER_VOXEL},
            "form": "axial DFT as two 16-point tcgen05 MMA stages, bf16 hi+lo operands, fp32 accumulate in TMEM",
            "_plan": plan}


def _parity(ss, torch, plan, frames, ref, stream, bound):
    """Relative L2 distance of one reconstruction from the FP64 oracle's volume
    ref [nl][ny][nx] (complex128): on the complex V and on |V|^2, summed over
    chunks of depth bins in float64."""
    vol, cplx = plan.reconstruct(frames, complex_out=True, stream=stream)
    torch.cuda.synchronize()
    if ss.ssoct_sync(plan.handle, stream.cuda_stream):
        raise RuntimeError("kernel error: " + ss.ssoct_last_error(plan.handle))
    v = cplx.cpu().numpy()
    p = vol.cpu().numpy()
    del vol, cplx
    acc = np.zeros(4)
    for q0 in range(0, v.shape[0], 16):
        r = ref[q0:q0 + 16]
        d = v[q0:q0 + 16].astype(np.complex128) - r
        rp = r.real ** 2 + r.imag ** 2
        dp = p[q0:q0 + 16].astype(np.float64) - rp
        acc += [(d.real ** 2 + d.imag ** 2).sum(), rp.sum(), (dp ** 2).sum(), (rp ** 2).sum()]
    return {"complex": float(np.sqrt(acc[0] / acc[1])), "intensity": float(np.sqrt(acc[2] / acc[3])),
            "bound_complex": bound}


def _cufft_chain(torch, frames, nl, ny, nx, voxels, steps=10):
    """Timing comparison only, outside the library: the same step's transforms
    done with cuFFT through torch.fft on the same GPU.  uint16 frames to complex
    times a unit-modulus chirp, the 2D DFT of every frame with the + sign of
    Eq. 6 (unnormalised), the DFT over the sweep (Eq. 7), |.|^2.  The Eq. 5
    resample has no matching library call and is left out, so the chain does
    less than the library's step."""
    f = frames.view(nl, ny, nx)
    phase = torch.rand((ny, nx), device="cuda", dtype=torch.float32) * 6.283185307179586
    chirp = torch.polar(torch.ones_like(phase), phase)
    h = torch.empty((nl, ny, nx), dtype=torch.complex64, device="cuda")
    g = torch.empty_like(h)
    p = torch.empty((nl, ny, nx), dtype=torch.float32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    acc = [0.0, 0.0, 0.0, 0.0]

    def step(timed):
        if timed:
            ev[0].record()
        torch.mul(f.float(), chirp, out=h)                    # frames x chirp
        if timed:
            ev[1].record()
        torch.fft.ifft2(h, norm="forward", out=g)            # + sign, unnormalised (Eq. 6)
        if timed:
            ev[2].record()
        torch.fft.fft(g, dim=0, out=h)                       # over the sweep (Eq. 7)
        if timed:
            ev[3].record()
        torch.abs(h, out=p)
        p.square_()
        if timed:
            ev[4].record()
            torch.cuda.synchronize()
            for i in range(4):
                acc[i] += ev[i].elapsed_time(ev[i + 1])

    for _ in range(3):
        step(False)
    torch.cuda.synchronize()
    for _ in range(steps):
        step(True)
    stages = [a / steps for a in acc]
    ms = sum(stages)
    out = {"ms_per_step": ms, "Gvoxel_per_s": voxels / (ms * 1e-3) / 1e9,
           "stages_ms": {"frames_x_chirp": stages[0], "fft2_cufft": stages[1], "fft_sweep_cufft": stages[2],
                         "abs2": stages[3]},
           "note": "timing comparison only (torch.fft = cuFFT), not part of the library; without the Eq. 5 "
                   "resample, full frames (no crop)"}
    del h, g, p
    torch.cuda.empty_cache()
    return out


def _aberration(args, ss, torch, synth, stream, steps=10):
    """Sharpness loss + gradient (dL/dz, dL/dc_1..15) per call of ssoct_sharpness on
    the 512x512x128 speckle sweep with 15 Zernike coefficients ~ N(0, 0.5 rad),
    reconstructed 5 mm beyond the generating distance.  Each call runs the forward
    and adjoint kernels and reads the 17 results back (it synchronises)."""
    import time
    w = synth.workload("mid_512x512x128")
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, flags=ss.SSOCT_FLAG_PUPIL)
    frames = torch.from_numpy(w.frames.view(np.int16)).cuda()
    vol, _ = plan.empty_volume()
    coeffs = np.random.default_rng(5).normal(0.0, 0.5, 15)
    for _ in range(max(args.warmup, 3)):
        loss, grad, _ = plan.sharpness(frames, coeffs, w.z + 5e-3, out=vol, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        loss, grad, _ = plan.sharpness(frames, coeffs, w.z + 5e-3, out=vol, stream=stream)
    ms = (time.perf_counter() - t0) * 1e3 / steps
    voxels = w.nx * w.ny * w.nlambda
    return {"workload": f"{w.nx}x{w.ny}x{w.nlambda} speckle, 15 Zernike coefficients, z + 5 mm",
            "ms_per_gradient": ms, "Gvoxel_per_s": voxels / (ms * 1e-3) / 1e9, "loss": loss,
            "grad_norm": float(np.linalg.norm(grad)),
            "note": "host wall time per ssoct_sharpness call (forward + adjoint + 17 doubles read back)"}


BATCH_SHAPES = [(256, 256, 64), (384, 384, 96), (512, 512, 128), (512, 512, 128), (640, 640, 160),
                (768, 768, 200), (1024, 1024, 256), (1024, 1024, 256)]


def _batched(args, ss, torch, synth, w_1024, frames_1024, stream, steps=10):
    """Eight uneven volumes (805.8 Mvoxel) reconstructed by one graph launch per
    step (ssoct_batch_run), against the same plans run one after another."""
    import tempfile
    fd, tune_cache = tempfile.mkstemp(suffix=".json", prefix="ssoct_batch_tune_")
    os.close(fd)
    os.unlink(tune_cache)
    plans, frames, vols, choices = [], [], [], []
    for i, (nx, ny, nl) in enumerate(BATCH_SHAPES):
        if (nx, ny, nl) == (w_1024.nx, w_1024.ny, w_1024.nlambda):
            w, f = w_1024, frames_1024
        else:
            w = synth.workload("custom", nx=nx, ny=ny, nlambda=nl, kind="points", seed=10 + i)
            f = torch.from_numpy(w.frames.view(np.int16)).cuda()
        plans.append(ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas))
        frames.append(f)
        vols.append(plans[-1].empty_volume()[0])
        # schedule, order and axial form chosen by the library's autotuner (the
        # two plans of a repeated shape time it once, through a cache file)
        choices.append(plans[-1].autotune(f, tune_cache, stream))
    voxels = sum(nx * ny * nl for nx, ny, nl in BATCH_SHAPES)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    lanes = {}
    for n_lanes in (1, 2, 4):
        batch = ss.Batch(plans, lanes=n_lanes)
        lanes[n_lanes] = timed(lambda: batch.run(frames, vols, stream=stream))
        batch.sync(stream)
        captures = batch.captures
        del batch
    best = min(lanes, key=lanes.get)
    ms_batch = lanes[best]

    def separate():
        for p, f, v in zip(plans, frames, vols):
            p.reconstruct(f, out=(v, None), stream=stream)

    ms_sep = timed(separate)
    if os.path.exists(tune_cache):
        os.unlink(tune_cache)
    return {"volumes": [f"{nx}x{ny}x{nl}" for nx, ny, nl in BATCH_SHAPES], "voxels": voxels,
            "autotuned": [{k: c[k] for k in ("lag", "ring_slots", "tc_axial", "axial_first")} for c in choices],
            "ms_per_batch": ms_batch, "Gvoxel_per_s": voxels / (ms_batch * 1e-3) / 1e9,
            "ms_separate": ms_sep, "Gvoxel_per_s_separate": voxels / (ms_sep * 1e-3) / 1e9,
            "lanes": best, "ms_by_lanes": lanes, "graph_captures": captures,
            "form": "one CUDA graph launch per batch, volume i on stream lane i mod lanes; "
                    "384/640/768 frames take the two-pass lateral path"}


# sources every kernel is built from besides its own .cu file
_COMMON_SOURCES = ("fft_codelets.cuh", "fft_common.cuh", "mbarrier.cuh", "ssoct_internal.h")


def kernel_source_hash(source: str) -> str:
    """sha256 (16 hex digits) over a kernel's .cu file and the headers every
    kernel includes, in a fixed order."""
    import hashlib
    h = hashlib.sha256()
    for name in (source,) + _COMMON_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2003_08960_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def _traffic(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current kernel sources (null otherwise)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d:
        return None
    return d["bytes_per_launch"] if kernel_source_hash(d["source"]) == d["source_sha256_16"] else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ssoct", choices=["ssoct", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-parity", action="store_true", help="skip the per-volume comparison with the FP64 oracle")
    ap.add_argument("--no-autotune", action="store_true", help="keep the plan's default schedule")
    ap.add_argument("--axial-first", action="store_true",
                    help="Eq. 5 + Eq. 7 before Eq. 6 (SSOCT_FLAG_AXIAL_FIRST) for the main line")
    ap.add_argument("--tc-axial", action="store_true", help="time the tensor-core axial form as the main line "
                                                            "(profiling captures)")
    ap.add_argument("--size", default=None, help="NXxNYxNLAMBDA instead of the 1024x1024x256 workload "
                                                 "(profiling captures; not a bench line)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ssoct(args)


if __name__ == "__main__":
    main()
