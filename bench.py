#!/usr/bin/env python
"""Throughput of the streaming TACAW time->energy stage on GB300.

One step = one segment of the realistic workload through the C ABI: reset, 64 pushes of
32 frames (64 probes, 256x256 k-ROI, complex64), finalize into I(k,E) (400 energies over
0-120 meV, Hann window, elastic mean removed) and the r=20 px aperture spectra.
Metric: complex MAC/s = P*K^2*T*Nw / step time (and EELS spectra/s = P*D / step time).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU (probe sets
are independent: no collective on the data path); value = all ranks' CMAC / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "complex MAC/s of streaming TACAW DFT and EELS spectra/s on 1 GB300 at stated error vs FP64"
UNIT = "CMAC/s"

# DRAM bytes per launch of the contraction kernel from an ncu capture, keyed by the hash of
# the kernel's source file at capture time (reported only while the source is unchanged).
KERNEL_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum of flush_tc_drain2_kernel on `bench.py
    # --small` (P=2, T=2048, 400 energies, default tiling): 2.461281 GB read + 0.203440 GB written per
    # launch of 1.0737e11 CMAC; key = hash of the code of k_tc_gemm.cu without its in-place section
    ("c496d2cc510ed277", "flush_tc_drain2_kernel"): 2.481715e-02,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="split_bf16", choices=["split_bf16", "split_fp16", "fp32"])
    ap.add_argument("--fp16-steps", type=int, default=2,
                    help="steps of the split-FP16 path for comparison (0: skip)")
    ap.add_argument("--fp32-steps", type=int, default=2, help="steps of the FP32 path for comparison (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="end-to-end steps from pinned host memory (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target seconds of the CPU oracle baseline")
    ap.add_argument("--small", action="store_true", help="small workload (profiling captures)")
    ap.add_argument("--pipeline", type=int, default=1,
                    help="segments in flight: one plan and CUDA stream each, steps alternate between them "
                         "(a segment's conversions overlap the previous segment's contraction)")
    ap.add_argument("--workload", default="realistic", choices=["realistic", "batched", "diff", "thick"],
                    help="batched: the 16 uneven partitions, autotuned tiles, one CUDA-graph replay per step; "
                         "diff: the differentiation workload, forward + adjoint per step; thick: one 32-probe "
                         "batch of the thick-sample workload per step")
    ap.add_argument("--in-place", dest="in_place", action="store_true", default=False,
                    help="the contraction reads pushed frames in place (no staging pass)")
    ap.add_argument("--staging", dest="in_place", action="store_false",
                    help="convert pushed frames into the library's staging area at push time (default)")
    ap.add_argument("--tc-omega-tile", type=int, default=0, help="tensor-core tiling override (0: plan default)")
    ap.add_argument("--tc-block-frames", type=int, default=0)
    ap.add_argument("--tc-drain-frames", type=int, default=0,
                    help="frames per drained hi*hi accumulator chunk (0: 512)")
    ap.add_argument("--accum", default="auto", choices=["auto", "kahan", "fp64", "fp32"],
                    help="Psi accumulators across flushes (only used when a segment needs several flushes)")
    ap.add_argument("--tc-max-ctas", type=int, default=0,
                    help="persistent contraction grid cap (0: every SM); with --pipeline 2 the free SMs "
                         "convert the next segment's pushes beside the current contraction")
    ap.add_argument("--trace", action="store_true",
                    help="add the per-CTA phase breakdown of one traced contraction (tacaw_flush_trace)")
    return ap.parse_args()


def stream_config(spec, P=None):
    from paper_2607_02236_gb300 import DetectorConfig, StreamConfig
    P = spec.P if P is None else P
    gx, gy = spec.full_grid
    rx, ry = spec.roi_origin
    return StreamConfig(
        n_probes=P, kx=spec.Kx, ky=spec.Ky, T=spec.T, dt_fs=spec.dt_fs,
        pitch_row=gx, pitch_frame=P * gx * gy, pitch_probe=gx * gy, roi_x0=rx, roi_y0=ry,
        E_meV=None if spec.fft_bins else [float(e) for e in spec.energies_meV()], fft_bins=spec.fft_bins,
        window=spec.window, window_param=spec.window_sigma() if spec.window == "gauss" else spec.window_param,
        subtract_mean=spec.subtract_mean, bose_T_K=spec.bose_T_K,
        detectors=[DetectorConfig(d.kind, d.cx, d.cy, d.r_in, d.r_out) for d in spec.detectors])


def workload(small: bool):
    import synth
    if small:
        s = synth.StreamSpec(P=2, Kx=256, Ky=256, T=2048, Tc=32, n_omega=400, E_max_meV=120.0, window="hann",
                             n_modes=32, amp_law="smooth", noise=1e-3)
        return "small-P2-K256-T2048-W400", s
    w = synth.realistic()
    return w.name, w.streams[0]


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value: float, dist, device) -> float:
    """The largest value over all ranks (the slowest replica sets the job's time)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput of independent replicas: all ranks' units over the slowest time."""
    return world * units_per_rank / seconds_max


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# sections of k_tc_gemm.cu that the staged kernels do not use: edits there keep their traffic
# figures valid (everything else in the file, shared helpers included, is hashed)
INPLACE_SECTION = (b"// In-place drained form (persistent)", b"// In-place variant:")


def file_hash(path, skip=None):
    """Hash of a source file's code: `//` comments and whitespace are left out, so that only
    code changes invalidate a capture."""
    with open(path, "rb") as f:
        data = f.read()
    if skip:
        a, b = data.find(skip[0]), data.find(skip[1])
        if 0 <= a < b:
            data = data[:a] + data[b:]
    data = re.sub(rb"//[^\n]*", b"", data)
    data = re.sub(rb"\s+", b"", data)
    return hashlib.sha256(data).hexdigest()[:16]


# ----------------------------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline leg and the reference arm)
# ----------------------------------------------------------------------------------------------
def oracle_rate(series, spec, seconds: float):
    """Times oracle.forward_pixels (as it stands) on pixel series [T, n]; CMAC/s and the sample used."""
    import numpy as np
    import oracle
    kw = dict(window_kind=spec.window, E_meV=spec.energies_meV(), dt_fs=spec.dt_fs,
              subtract_mean=spec.subtract_mean)
    T, n = series.shape
    oracle.forward_pixels(series[:, :min(n, 64)], **kw)      # warm-up
    k = min(1024, n)
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < seconds:
        s0 = (done // k) * k % max(1, n - k + 1)
        oracle.forward_pixels(series[:, s0:s0 + k], **kw)
        done += k
    dt = time.perf_counter() - t0
    return done * T * spec.Nw / dt, done, dt


def reference_arm(args):
    import numpy as np
    from synth import frames
    name, spec = workload(args.small)
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    rng = np.random.default_rng(0)
    n_px = 256
    pix = rng.integers(0, spec.Kx * spec.Ky, n_px)
    probe = 0
    series = frames.pixel_series(spec, 0, probe, pix // spec.Kx, pix % spec.Kx)
    import oracle
    kw = dict(window_kind=spec.window, E_meV=spec.energies_meV(), dt_fs=spec.dt_fs,
              subtract_mean=spec.subtract_mean)
    for _ in range(args.warmup):
        oracle.forward_pixels(series, **kw)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.forward_pixels(series, **kw)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    cm = n_px * spec.T * spec.Nw
    value = cm * len(times) / tot
    cores = os.cpu_count()
    sample = f"{n_px} pixels x T={spec.T} x Nw={spec.Nw} of {name} per step (FP64 NumPy oracle)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------------
# Batched partitions: 16 uneven streams in one plan (autotuned tiles, the last flushes of all
# streams in one persistent launch), a whole segment captured into a CUDA graph and replayed
# ----------------------------------------------------------------------------------------------
def batched_arm(args):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import synth
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = synth.batched()
    specs = list(w.streams)
    n_s = len(specs)
    cmac_step = sum(s.P * s.Kx * s.Ky * s.T * s.Nw for s in specs)
    # the segments (338 GB of frames) exceed HBM: each partition keeps R pushes resident and
    # cycles them (frame t of a segment is frame t mod (R*Tc) of the ring)
    R = 4
    main_st = torch.cuda.current_stream()
    bufs = []
    for i, s in enumerate(specs):
        fe = s.P * s.Kx * s.Ky
        b = torch.empty(R * s.Tc * fe, dtype=torch.complex64, device="cuda")
        sg.generate(s, 3000 + 97 * rank + i, b.data_ptr(), 0, R * s.Tc, pitch_row=s.Kx, pitch_frame=fe,
                    pitch_probe=s.Kx * s.Ky, stream=main_st.cuda_stream)
        bufs.append(b)
    # outputs before the plan: the plan takes its staging from what memory is left
    I = torch.empty(sum(s.P * s.Nw * s.Kx * s.Ky for s in specs), dtype=torch.float32, device="cuda")
    S = torch.empty(max(1, sum(s.P * len(s.detectors) * s.Nw for s in specs)), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = TacawPlan([stream_config(s) for s in specs], precision="split_bf16", tune="", accum=args.accum)
    plan_s = time.perf_counter() - t0
    info = plan.info()
    assert info["I_elems"] == I.numel() and info["S_elems"] <= S.numel()

    def enqueue(sth):
        plan.reset(sth)
        pushed = [0] * n_s
        while any(pushed[i] < s.T for i, s in enumerate(specs)):
            for i, s in enumerate(specs):
                if pushed[i] >= s.T:
                    continue
                n = min(s.Tc, s.T - pushed[i])
                slot = (pushed[i] // s.Tc) % R
                plan.push(i, bufs[i].data_ptr() + slot * s.Tc * s.P * s.Kx * s.Ky * 8, n, sth)
                pushed[i] += n
        plan.finalize_async(I, S, None, sth)

    # eager segments: launch count, contraction time, then the graph
    cap = torch.cuda.Stream()
    with torch.cuda.stream(cap):
        enqueue(cap.cuda_stream)
        plan.check_errors(cap.cuda_stream)
        l0 = plan.info()["kernel_launches"]
        plan.set_timing(True)
        plan.kernel_time_ms(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cap)
        enqueue(cap.cuda_stream)
        e1.record(cap)
        plan.check_errors(cap.cuda_stream)
        eager_ms = e0.elapsed_time(e1)
        k_ms, k_n = plan.kernel_time_ms(reset=True)
        plan.set_timing(False)
        launches = plan.info()["kernel_launches"] - l0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        enqueue(torch.cuda.current_stream().cuda_stream)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    e0.record(st)
    for _ in range(args.steps):
        g.replay()
    e1.record(st)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / args.steps
    plan.check_errors(st.cuda_stream)
    value = job_rate(cmac_step, world, ms * 1e-3)

    # stated error: two sampled series per partition, all energies, against the FP64 oracle
    rng = np.random.default_rng(rank)
    worst = 0.0
    for i, s in enumerate(specs):
        npx = s.Kx * s.Ky
        p = rng.integers(0, s.P, 2)
        k = rng.integers(0, npx, 2)
        ring = bufs[i].view(R * s.Tc, s.P, npx)[:, torch.as_tensor(p, device="cuda"), torch.as_tensor(k, device="cuda")]
        ring = ring.cpu().numpy()
        ser = ring[np.arange(s.T) % (R * s.Tc)]
        io, _ = plan.offsets(i)
        Ii = I[io:io + s.P * s.Nw * npx].view(s.P, s.Nw, npx)
        got = Ii[torch.as_tensor(p, device="cuda"), :, torch.as_tensor(k, device="cuda")].cpu().numpy().T
        kw = dict(window_kind=s.window, window_param=s.window_sigma() if s.window == "gauss" else s.window_param,
                  E_meV=s.energies_meV(), dt_fs=s.dt_fs, subtract_mean=s.subtract_mean)
        _, ref = oracle.forward_pixels(ser, **kw)
        worst = max(worst, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
    peaks, peak_src = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    achieved = cmac_step * 24 / (k_ms * 1e-3) / 1e12
    kname = "flush_tc_drain2_kernel"
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": {"workload": w.name, "partitions": n_s, "cmac_per_step": cmac_step,
                           "probes": [s.P for s in specs], "k_roi": [s.Kx for s in specs], "T": [s.T for s in specs],
                           "n_omega": specs[0].Nw, "frames_per_push": specs[0].Tc,
                           "k_stage": info["k_stage"], "tc_drain_frames": info["tc_drain_frames"],
                           "accumulators": ["kahan", "fp64", "fp32"][info["accum"]],
                           "tuned_streams": info["tuned_streams"], "tune_candidates": info["tune_candidates"],
                           "tune_ms": round(info["tune_ms"], 1), "plan_create_s": round(plan_s, 2),
                           "plan_device_GB": round(info["device_bytes"] / 1e9, 1),
                           "inputs": f"per-partition rings of {R} pushes resident in HBM, cycled over each segment",
                           "step": "one CUDA-graph replay of reset + all pushes + finalize_async",
                           "l2": "staged operands (>= 10 GB per step) larger than L2, no flush",
                           "parallelism": f"replicas x{world}"},
                "max_rel_err_I_vs_fp64": worst, "error_sample": "2 (probe, pixel) series per partition, all energies",
                "eager_ms_per_step": eager_ms, "gpu_launches": launches, "contraction_launches_per_step": k_n,
                "clocks": clocks, "e2e": None,
                "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": None, "kernel": kname, "flop_per_cmac": 24,
                             "kernel_ms": k_ms, "peak_source": f"{peak_src} bf16 sustained (MEASURED_PEAKS.json)"},
                "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    del g
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------------------------
# Thick sample: 32-probe batches of 1024^2 multislice frames, a centred 256^2 k-ROI cropped while
# the pushes are read, T = 8192 in 64-frame pushes, 1000 energies, compensated FP32 accumulators
# across flushes of 2048 frames.  One step = one probe batch (1/8 of the 256-probe scan).
# ----------------------------------------------------------------------------------------------
def thick_arm(args):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import synth
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = synth.thick()
    spec = w.streams[0]
    B = w.probe_batch
    K, T, Tc, Nw = spec.Kx, spec.T, spec.Tc, spec.Nw
    gx, gy = spec.full_grid
    rx, ry = spec.roi_origin
    npix = K * K
    fe = B * gx * gy                       # one full frame for each probe of the batch
    cmac_step = B * npix * T * Nw
    k_stage = 2048
    st_t = torch.cuda.current_stream()
    st = st_t.cuda_stream
    # a resident ring of R pushes (17.2 GB each), cycled over the segment: frame t of a step is
    # frame t mod (R * Tc) of the ring; only the ROI of the full grid is synthesised (and read)
    R = 2
    ring = torch.zeros(R * Tc * fe, dtype=torch.complex64, device="cuda")
    for r in range(R):
        sg.generate(spec, 33 + rank, ring.data_ptr() + r * Tc * fe * 8, r * Tc, Tc, pitch_row=gx, pitch_frame=fe,
                    pitch_probe=gx * gy, out_x0=rx, out_y0=ry, p0=0, P=B, stream=st)
    I = torch.empty(B * Nw * npix, dtype=torch.float32, device="cuda")
    S = torch.empty(max(1, B * len(spec.detectors) * Nw), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    plan = TacawPlan([stream_config(spec, P=B)], precision="split_bf16", k_stage=k_stage, accum="kahan")
    info = plan.info()
    n_push = T // Tc

    def step():
        plan.reset(st)
        for i in range(n_push):
            plan.push(0, ring.data_ptr() + (i % R) * Tc * fe * 8, Tc, st)
        plan.finalize_async(I, S if len(spec.detectors) else None, None, st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.check_errors(st)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    plan.set_timing(True)
    plan.kernel_time_ms(reset=True)
    l0 = plan.info()["kernel_launches"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st_t)
    for _ in range(args.steps):
        step()
    e1.record(st_t)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = clk.stop()
    plan.check_errors(st)
    launches = (plan.info()["kernel_launches"] - l0) // args.steps
    k_ms, k_n = plan.kernel_time_ms(reset=True)
    plan.set_timing(False)
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / args.steps
    value = job_rate(cmac_step, world, ms * 1e-3)

    # stated error: 8 (probe, pixel) series of the ring-cycled segment, all energies
    rng = np.random.default_rng(rank)
    pb = rng.integers(0, B, 8)
    c = (K // 2) * K + K // 2
    px = np.concatenate([[c, c + 3], rng.integers(0, npix, 6)])
    rows = torch.as_tensor(pb * gx * gy + (ry + px // K) * gx + (rx + px % K), device="cuda")
    cyc = ring.view(R * Tc, fe)[:, rows].cpu().numpy()
    ser = cyc[np.arange(T) % (R * Tc)]
    got = I.view(B, Nw, npix)[torch.as_tensor(pb, device="cuda"), :, torch.as_tensor(px, device="cuda")]
    got = got.cpu().numpy().T
    _, ref = oracle.forward_pixels(ser, window_kind=spec.window, E_meV=spec.energies_meV(), dt_fs=spec.dt_fs,
                                   subtract_mean=spec.subtract_mean)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))

    peaks, peak_src = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    flush_ms = k_ms / max(k_n, 1)
    achieved = (cmac_step * args.steps / max(k_n, 1)) * 24 / (flush_ms * 1e-3) / 1e12
    kname = "flush_tc_drain2_kernel"
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": {"workload": w.name, "probes_per_step": B, "full_grid": f"{gx}x{gy}",
                           "k_roi": f"{K}x{K} at ({rx}, {ry})", "T": T, "frames_per_push": Tc, "n_omega": Nw,
                           "E_range_meV": [0, spec.E_max_meV], "window": spec.window,
                           "k_stage": info["k_stage"], "flushes_per_step": T // info["k_stage"],
                           "accumulators": ["kahan", "fp64", "fp32"][info["accum"]],
                           "omega_tile": info["omega_tile"], "tc_drain_frames": info["tc_drain_frames"],
                           "plan_device_GB": round(info["device_bytes"] / 1e9, 1),
                           "inputs": f"ring of {R} pushes of full frames ({R * Tc * fe * 8 / 1e9:.1f} GB) cycled",
                           "l2": "pushes (17.2 GB of full frames, 1.07 GB of ROI read) larger than L2, no flush",
                           "parallelism": f"replicas x{world}"},
                "max_rel_err_I_vs_fp64": err, "error_sample": "8 (probe, pixel) series, all energies",
                "clocks": clocks, "gpu_launches": launches, "e2e": None, "cpu_baseline": None,
                "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": None, "kernel": kname, "flop_per_cmac": 24,
                             "kernel_ms": flush_ms, "launches_per_step": k_n // max(args.steps, 1),
                             "peak_source": f"{peak_src} bf16 sustained (MEASURED_PEAKS.json)"}}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------------------------
# Differentiation: forward spectrum and the hand-written adjoint (tacaw_backward) per step
# ----------------------------------------------------------------------------------------------
def diff_arm(args):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import synth
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = synth.diff()
    spec = w.streams[0]
    P, K, T, Nw = spec.P, spec.Kx, spec.T, spec.Nw
    D = len(spec.detectors)
    npix = K * K
    mask = oracle.detector_masks(K, K, spec.detectors)          # [D, K*K] (host geometry only)
    n_ap = int(np.count_nonzero(mask.reshape(D, -1).any(axis=0)))
    # forward: the dense DFT of every ROI pixel; adjoint: Psi recomputed on the aperture pixels
    # (not stored) and projected back onto every frame (G = 0 outside the apertures)
    cmac_fwd = P * npix * T * Nw
    cmac_adj = 2 * P * n_ap * T * Nw
    st_t = torch.cuda.current_stream()
    st = st_t.cuda_stream
    x = torch.empty(T * P * npix, dtype=torch.complex64, device="cuda")
    sg.generate(spec, 4 + rank, x.data_ptr(), 0, T, pitch_row=K, pitch_frame=P * npix, pitch_probe=npix, stream=st)
    grad = torch.empty_like(x)
    c = torch.tensor(synth.loss_weights(Nw, seed=0), dtype=torch.float32, device="cuda")
    dLdS = c[None, None, :].expand(P, D, Nw).contiguous()
    I = torch.empty(P * Nw * npix, dtype=torch.float32, device="cuda")
    S = torch.empty(max(1, P * D * Nw), dtype=torch.float32, device="cuda")
    plan = TacawPlan([stream_config(spec)], precision=w.precision)
    info = plan.info()
    n_push = (T + spec.Tc - 1) // spec.Tc

    def step(ev=None):
        plan.reset(st)
        for i in range(n_push):
            plan.push(0, x.data_ptr() + i * spec.Tc * P * npix * 8, min(spec.Tc, T - i * spec.Tc), st)
        plan.finalize_async(I, S, None, st)
        if ev is not None:
            ev[0].record(st_t)
        plan.backward(0, dLdS, x, grad, st)
        if ev is not None:
            ev[1].record(st_t)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.check_errors(st)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    plan.set_timing(True)
    plan.kernel_time_ms(reset=True)
    l0 = plan.info()["kernel_launches"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st_t)
    for k in range(args.steps):
        step(evs[k])
    e1.record(st_t)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = clk.stop()
    plan.check_errors(st)
    launches = (plan.info()["kernel_launches"] - l0) // args.steps
    k_ms, k_n = plan.kernel_time_ms(reset=True)
    plan.set_timing(False)
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / args.steps
    adj_ms = statistics.median(a.elapsed_time(b) for a, b in evs)
    value = job_rate(cmac_fwd + cmac_adj, world, ms * 1e-3)

    # stated error: spectra of two probes and the gradient at 16 aperture pixels of two probes
    rng = np.random.default_rng(rank)
    kw = dict(window_kind=spec.window, E_meV=spec.energies_meV(), dt_fs=spec.dt_fs,
              subtract_mean=spec.subtract_mean)
    ap = np.nonzero(mask[0].reshape(-1))[0]
    xv = x.view(T, P, npix)
    gv = grad.view(T, P, npix)
    err_s, err_g = 0.0, 0.0
    for p in rng.choice(P, 2, replace=False):
        series = xv[:, int(p)][:, torch.as_tensor(ap, device="cuda")].cpu().numpy()
        _, Iref = oracle.forward_pixels(series, **kw)
        sref = Iref.sum(axis=1)
        sgot = S.view(P, D, Nw)[int(p), 0].cpu().numpy()
        err_s = max(err_s, float(np.max(np.abs(sgot - sref)) / np.max(np.abs(sref))))
        sel = rng.choice(len(ap), 16, replace=False)
        gref = oracle.gradient_pixels(series[:, sel], c.cpu().numpy().astype(np.float64)[None, :],
                                      np.ones((len(sel), 1)), **kw)
        ggot = gv[:, int(p)][:, torch.as_tensor(ap[sel], device="cuda")].cpu().numpy()
        err_g = max(err_g, float(np.linalg.norm(ggot - gref) / np.linalg.norm(gref)))

    mhz = clocks.get("sm_max_mhz") or 2070.0
    ffma_peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
    # kernel_time_ms: total over the timed launches and their count
    fwd_launch_ms = k_ms / max(k_n, 1)
    fwd_tflops = (cmac_fwd * args.steps / max(k_n, 1)) * 8 / (fwd_launch_ms * 1e-3) / 1e12
    adj_tflops = cmac_adj * 8 / (adj_ms * 1e-3) / 1e12
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.name, "probes": P, "k_roi": f"{K}x{K}", "T": T, "n_omega": Nw,
                           "window": spec.window, "aperture_pixels": n_ap,
                           "cmac_per_step": {"forward": cmac_fwd, "adjoint": cmac_adj},
                           "step": "reset + push + finalize_async (FP32 path) + tacaw_backward (dL/dS = c(E))",
                           "l2": "frames (%.2f GB) and gradient re-read every step, no flush" % (T * P * npix * 8 / 1e9),
                           "parallelism": f"replicas x{world}"},
                "max_rel_err_S_vs_fp64": err_s, "rel_l2_err_grad_vs_fp64": err_g,
                "error_sample": "spectra of 2 probes; gradient at 16 aperture pixels of 2 probes",
                "clocks": clocks, "gpu_launches": launches, "e2e": None, "cpu_baseline": None,
                "roofline": {"bound": "alu", "achieved": fwd_tflops, "peak": ffma_peak, "unit": "TFLOP/s",
                             "frac": fwd_tflops / ffma_peak, "traffic": None, "kernel": "flush_simt_kernel",
                             "flop_per_cmac": 8, "kernel_ms": fwd_launch_ms,
                             "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"},
                "adjoint": {"ms": adj_ms, "cmac": cmac_adj, "achieved": adj_tflops, "peak": ffma_peak,
                            "unit": "TFLOP/s", "frac": adj_tflops / ffma_peak, "bound": "alu",
                            "kernels": "zero_roi_kernel, adj_psi_kernel, adj_grad_kernel",
                            "timed": "CUDA events around the tacaw_backward call (median per step; includes "
                                     "its closing wait for the device error word)"}}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batched":
        return batched_arm(args)
    if args.workload == "diff":
        return diff_arm(args)
    if args.workload == "thick":
        return thick_arm(args)

    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_02236_gb300 import TacawPlan
    import synth.gpu as sg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    name, spec = workload(args.small)
    P, K, T, Tc, Nw = spec.P, spec.Kx, spec.T, spec.Tc, spec.Nw
    D = len(spec.detectors)
    npix = K * K
    frame_elems = P * npix
    cmac_step = P * npix * T * Nw
    stream = torch.cuda.current_stream()
    st = stream.cuda_stream

    # inputs resident in HBM: frames [T][P][K][K] complex64 (68.7 GB for the realistic workload)
    x = torch.empty(T * frame_elems, dtype=torch.complex64, device="cuda")
    base = x.data_ptr()
    for t0 in range(0, T, 64):
        n = min(64, T - t0)
        sg.generate(spec, 1000 + rank, base + t0 * frame_elems * 8, t0, n, pitch_row=K,
                    pitch_frame=frame_elems, pitch_probe=npix, stream=st)
    torch.cuda.synchronize()
    I = torch.empty(P * Nw * npix, dtype=torch.float32, device="cuda")
    S = torch.empty(max(1, P * D * Nw), dtype=torch.float32, device="cuda")
    n_push = (T + Tc - 1) // Tc

    def run_step(plan, out=None, sth=None, ev=None, sobj=None):
        """One segment through the public API: reset, all pushes, finalize (asynchronous).
        ev: a pair of CUDA events recorded on sobj around the reset and pushes (the conversions)."""
        I_, S_ = out if out is not None else (I, S)
        sth = st if sth is None else sth
        if ev is not None:
            ev[0].record(sobj)
        plan.reset(sth)
        for i in range(n_push):
            plan.push(0, base + i * Tc * frame_elems * 8, min(Tc, T - i * Tc), sth)
        if ev is not None:
            ev[1].record(sobj)
        plan.finalize_async(I_, S_, None, sth)

    def timed(plans, steps, warmup, sample_clocks=False, outs=None, streams=None):
        """Steps alternate over the plans, each on its own stream (one segment in flight per plan)."""
        plans = plans if isinstance(plans, list) else [plans]
        outs = outs or [(I, S)]
        streams = streams or [stream]
        n = len(plans)
        for k in range(warmup):
            run_step(plans[k % n], outs[k % n], streams[k % n].cuda_stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local) if sample_clocks else None
        for pl in plans:
            pl.set_timing(True)
            pl.kernel_time_ms(reset=True)
        l0 = sum(pl.info()["kernel_launches"] for pl in plans)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for sx in streams:
            sx.wait_event(e0)
        # one segment in flight: the pushes' span (reset, provisional mean, conversions) per step
        pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)] if n == 1 else None
        for k in range(steps):
            run_step(plans[k % n], outs[k % n], streams[k % n].cuda_stream,
                     ev=pev[k] if pev else None, sobj=streams[k % n])
        for sx in streams:
            ev = torch.cuda.Event()
            ev.record(sx)
            stream.wait_event(ev)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        for sx, pl in zip(streams, plans):
            pl.check_errors(sx.cuda_stream)
        clocks = clk.stop() if clk else None
        ms = e0.elapsed_time(e1)
        timed.push_ms = statistics.median(a.elapsed_time(b) for a, b in pev) if pev else None
        kms, kn = 0.0, 0
        for pl in plans:
            a, b = pl.kernel_time_ms(reset=True)
            kms, kn = kms + a, kn + b
            pl.set_timing(False)
        launches = (sum(pl.info()["kernel_launches"] for pl in plans) - l0) // steps
        ms = max_over_ranks(ms, dist, "cuda")
        return ms / steps, kms / max(kn, 1), kn // max(steps, 1), launches, clocks

    tiling = dict(tc_omega_tile=args.tc_omega_tile, tc_block_frames=args.tc_block_frames,
                  tc_drain_frames=args.tc_drain_frames, tc_max_ctas=args.tc_max_ctas,
                  frames_in_place=bool(args.in_place and args.precision == "split_bf16"))
    split = args.precision.startswith("split")
    # segments in flight: plan k and stream k take steps k, k + n, ...; the first plan writes I, S
    n_pipe = max(1, args.pipeline)
    plans = [TacawPlan([stream_config(spec)], precision=args.precision, accum=args.accum, **tiling)
             for _ in range(n_pipe)]
    plan = plans[0]
    info = plan.info()
    outs = [(I, S)] + [(torch.empty_like(I), torch.empty_like(S)) for _ in range(n_pipe - 1)]
    pipe_streams = [torch.cuda.Stream() for _ in range(n_pipe)] if n_pipe > 1 else [stream]
    ms_step, k_ms, k_per_step, launches, clocks = timed(plans, args.steps, args.warmup, sample_clocks=True,
                                                        outs=outs, streams=pipe_streams)
    push_ms = timed.push_ms
    for pl in plans[1:]:          # free the other segments' staging before the comparison legs
        pl.close()
    del outs[1:]
    value = job_rate(cmac_step, world, ms_step * 1e-3)
    spectra_per_s = world * P * D / (ms_step * 1e-3)

    phases = None
    tr = None
    if args.trace and split:
        plan.set_timing(2)
        run_step(plan)
        torch.cuda.synchronize()
        tr = plan.flush_trace().astype(np.int64)
        plan.set_timing(0)
        if info["tc_drain_frames"]:
            # persistent drained kernel: one row per launched CTA (see tacaw_set_timing)
            tr = tr[tr[:, 0] != 0]
            life = tr[:, 6] - tr[:, 0]
            phases = {"ctas": int(len(tr)), "lifetime_us": round(float(np.median(life)) / 1e3, 1),
                      "setup_us": round(float(np.median(tr[:, 1] - tr[:, 0])) / 1e3, 2),
                      "first_operands_us": round(float(np.median(tr[:, 2] - tr[:, 1])) / 1e3, 2),
                      "mma_span_us": round(float(np.median(tr[:, 3] - tr[:, 2])) / 1e3, 1),
                      "tiles_per_cta": int(np.median(tr[:, 4])), "chunks_per_cta": int(np.median(tr[:, 5])),
                      "mma_us_per_tile": round(float(np.median((tr[:, 3] - tr[:, 2]) / np.maximum(tr[:, 4], 1))) / 1e3, 2),
                      "tail_after_last_mma_us": round(float(np.median(tr[:, 6] - tr[:, 3])) / 1e3, 2),
                      "unit": "median per CTA"}
            tr = None
    if tr is not None and args.trace and split:
        names = ["setup", "fill", "main_loop", "drain", "epilogue", "exit"]
        phases = {n: round(float(np.median(tr[:, i + 1] - tr[:, i])) / 1e3, 3) for i, n in enumerate(names)}
        gaps = []
        for sm in np.unique(tr[:, 7]):
            r = tr[tr[:, 7] == sm]
            r = r[np.argsort(r[:, 0])]
            gaps.extend((r[1:, 0] - r[:-1, 6]).tolist())
        phases["gap_between_ctas"] = round(float(np.median(gaps)) / 1e3, 3) if gaps else None
        phases["ctas"] = int(len(tr))
        phases["unit"] = "us (median per CTA)"

    # stated error vs FP64 at sampled pixels (all energies), incl. the bright centre
    import oracle
    rng = np.random.default_rng(rank)
    probes = rng.integers(0, P, 24)
    pix = np.concatenate([[K // 2 * K + K // 2, (K // 2 + 3) * K + K // 2 - 5],
                          rng.integers(0, npix, 22)])
    xv = x.view(T, P, npix)
    series = xv[:, torch.as_tensor(probes, device="cuda"), torch.as_tensor(pix, device="cuda")].cpu().numpy()
    Iv = I.view(P, Nw, npix)
    got = Iv[torch.as_tensor(probes, device="cuda"), :, torch.as_tensor(pix, device="cuda")].cpu().numpy().T
    _, ref = oracle.forward_pixels(series, window_kind=spec.window, E_meV=spec.energies_meV(), dt_fs=spec.dt_fs,
                                   subtract_mean=spec.subtract_mean)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


    # split-FP16 pieces (scaled frames) on the same input: same kernels and tiling, other operand type
    fp16 = None
    if args.fp16_steps > 0 and args.precision == "split_bf16":
        with TacawPlan([stream_config(spec)], precision="split_fp16", accum=args.accum, **tiling) as p16:
            ms16, k16, _, _, _ = timed(p16, args.fp16_steps, 1)
        got16 = Iv[torch.as_tensor(probes, device="cuda"), :, torch.as_tensor(pix, device="cuda")].cpu().numpy().T
        err16 = float(np.max(np.abs(got16 - ref)) / np.max(np.abs(ref)))
        fp16 = {"value": world * cmac_step / (ms16 * 1e-3), "unit": UNIT, "ms_per_step": ms16, "flush_ms": k16,
                "max_rel_err_I_vs_fp64": err16, "fp16_scale": 4096,
                "flush_tflops": cmac_step * 24 / (k16 * 1e-3) / 1e12}

    # FP32 CUDA-core path on the same input, for comparison at equal stated accuracy
    fp32 = None
    if args.fp32_steps > 0 and args.precision != "fp32":
        with TacawPlan([stream_config(spec)], precision="fp32") as p32:
            ms32, k32, _, _, _ = timed(p32, args.fp32_steps, 1)
        got32 = Iv[torch.as_tensor(probes, device="cuda"), :, torch.as_tensor(pix, device="cuda")].cpu().numpy().T
        err32 = float(np.max(np.abs(got32 - ref)) / np.max(np.abs(ref)))
        fp32 = {"value": world * cmac_step / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32,
                "flush_ms": k32, "max_rel_err_I_vs_fp64": err32}

    # end to end through the public API from pinned host memory (host ring of pushes, cycled);
    # last, because it overwrites the device input with the cycled ring
    e2e = None
    if args.e2e_steps > 0:
        ring = min(16, n_push)
        push_elems = Tc * frame_elems
        host = torch.empty(ring * push_elems, dtype=torch.complex64, pin_memory=True)
        host.copy_(x[: ring * push_elems])
        S_host = [torch.empty(S.numel(), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        cs = torch.cuda.Stream()
        in_place = bool(info["frames_in_place"])
        # a staged plan converts each push when it is enqueued, so device slices form a ring that
        # the next copies reuse as soon as that conversion is done (copies of the next step run
        # under this step's contraction); an in-place plan reads every slice until finalize
        n_slots = n_push if in_place else ring
        copied = [torch.cuda.Event() for _ in range(n_slots)]
        consumed = [None] * n_slots

        def e2e_step(k):
            plan.reset(st)
            for i in range(n_push):
                slot = i % n_slots
                n = min(Tc, T - i * Tc)
                with torch.cuda.stream(cs):
                    if consumed[slot] is not None:
                        cs.wait_event(consumed[slot])
                    x[slot * push_elems:slot * push_elems + n * frame_elems].copy_(
                        host[(i % ring) * push_elems:(i % ring) * push_elems + n * frame_elems], non_blocking=True)
                    copied[slot].record(cs)
                stream.wait_event(copied[slot])
                plan.push(0, base + slot * push_elems * 8, n, st)
                if not in_place:
                    consumed[slot] = torch.cuda.Event()
                    consumed[slot].record(stream)
            plan.finalize_async(I, S, None, st)
            S_host[k % 2].copy_(S, non_blocking=True)
            done = torch.cuda.Event()
            done.record(stream)
            if in_place:
                for slot in range(n_slots):
                    consumed[slot] = done
            return done

        e2e_step(0).synchronize()
        plan.check_errors(st)
        barrier()
        t0 = time.perf_counter()
        prev = None
        checksum = 0.0
        for k in range(args.e2e_steps):
            ev = e2e_step(k)
            if prev is not None:                 # the host reads each step's result, one step behind
                prev[0].synchronize()
                checksum += float(S_host[prev[1] % 2][0])
            prev = (ev, k)
        prev[0].synchronize()
        checksum += float(S_host[prev[1] % 2][0])
        plan.check_errors(st)
        el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": world * cmac_step * args.e2e_steps / el, "unit": UNIT,
               "h2d_bytes_per_step": T * frame_elems * 8, "d2h_bytes_per_step": S.numel() * 4,
               "ms_per_step": 1e3 * el / args.e2e_steps,
               "input": f"pinned host ring of {ring} pushes ({ring * push_elems * 8 / 1e9:.1f} GB) cycled",
               "ingest": "copy engines: cudaMemcpyAsync of each push into a device ring, then the push",
               "overlap": "copies of the next step overlap this step's contraction" if not in_place else "none"}

        # zero-copy ingest (staged plans): each push passes its pinned host address and the push
        # kernels read the frames over the host link, no separate copy
        if not in_place:
            def zc_step(k):
                plan.reset(st)
                for i in range(n_push):
                    n = min(Tc, T - i * Tc)
                    plan.push(0, host.data_ptr() + (i % ring) * push_elems * 8, n, st)
                plan.finalize_async(I, S, None, st)
                S_host[k % 2].copy_(S, non_blocking=True)
                done = torch.cuda.Event()
                done.record(stream)
                return done

            zc_step(0).synchronize()
            plan.check_errors(st)
            barrier()
            t0 = time.perf_counter()
            prev = None
            for k in range(args.e2e_steps):
                ev = zc_step(k)
                if prev is not None:
                    prev[0].synchronize()
                    checksum += float(S_host[prev[1] % 2][0])
                prev = (ev, k)
            prev[0].synchronize()
            checksum += float(S_host[prev[1] % 2][0])
            plan.check_errors(st)
            el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
            zc = {"value": world * cmac_step * args.e2e_steps / el, "unit": UNIT,
                  "h2d_bytes_per_step": T * frame_elems * 8, "d2h_bytes_per_step": S.numel() * 4,
                  "ms_per_step": 1e3 * el / args.e2e_steps, "input": e2e["input"],
                  "ingest": "zero-copy: the push kernels read each push from pinned host memory",
                  "overlap": "none (reads happen inside the conversions)"}
            # the faster ingest is the end-to-end figure; the other one is kept beside it
            if zc["value"] > e2e["value"]:
                zc["other_ingest"], e2e = e2e, zc
            else:
                e2e["other_ingest"] = zc
        del host
    plan.close()

    # roofline of the dominant kernel (the contraction) from its live CUDA-event duration
    peaks, peak_src = measured_peaks()
    cmac_launch = cmac_step / max(k_per_step, 1)
    if split:
        # 3 bf16 (or fp16) products (hi*hi, hi*lo, lo*hi) x 4 real MAC per complex MAC = 24 flop per CMAC
        achieved = cmac_launch * 24 / (k_ms * 1e-3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        src = os.path.join(ROOT, "paper_2607_02236_gb300", "csrc", "k_tc_gemm.cu")
        kname = "flush_tc_inplace_kernel" if info["frames_in_place"] else "flush_tc_drain2_kernel"
        tr = KERNEL_TRAFFIC.get((file_hash(src, None if info["frames_in_place"] else INPLACE_SECTION), kname))
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": (tr * cmac_launch if tr else None),
                "kernel": kname, "flop_per_cmac": 24,
                "peak_source": f"{peak_src} bf16 sustained (MEASURED_PEAKS.json)" +
                               (" x 1 (fp16 and bf16 have the same dense tensor rate)" if args.precision == "split_fp16" else ""),
                "kernel_ms": k_ms, "launches_per_step": k_per_step}
    else:
        achieved = cmac_launch * 8 / (k_ms * 1e-3) / 1e12
        sm = 152
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        peak = sm * 128 * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "flush_simt_kernel", "flop_per_cmac": 8,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock", "kernel_ms": k_ms,
                "launches_per_step": k_per_step}

    # HBM roofline of the pushes (staged plans): each conversion reads a complex64 sample (8 B)
    # and writes its two 16-bit pieces of Re and Im (or a float2 on the FP32 path, 8 B)
    conv = None
    if push_ms and not info["frames_in_place"]:
        conv_bytes = 16.0 * P * npix * T
        hbm = peaks.get("hbm_gbs")
        conv = {"bound": "hbm", "achieved": conv_bytes / (push_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": conv_bytes / (push_ms * 1e-3) / 1e9 / hbm if hbm else None, "traffic": None,
                "kernel": "convert_split_tiled_kernel" if split else "convert_fp32_kernel",
                "bytes_per_step": conv_bytes, "ms_per_step": push_ms,
                "timed": "CUDA events around reset + all pushes of each timed step (median); the span also "
                         "holds the provisional-mean kernel of the first push, whose 8 B per sample of "
                         "that push are not counted",
                "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json)"}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        n_cpu = 4096
        cp = rng.integers(0, P, n_cpu)
        cx = rng.integers(0, npix, n_cpu)
        ser = xv[:, torch.as_tensor(cp, device="cuda"), torch.as_tensor(cx, device="cuda")].cpu().numpy()
        rate, m, dt = oracle_rate(ser, spec, args.cpu_seconds)
        import multiprocessing
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else multiprocessing.cpu_count()
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{m} random (probe, pixel) series x T={T} x Nw={Nw} ({dt:.1f} s, FP64 NumPy)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"split_bf16": "bf16", "split_fp16": "f16"}.get(args.precision, "f32"),
                "data": "synthetic",
                "config": {"workload": name, "probes": P, "k_roi": f"{K}x{K}", "T": T, "frames_per_push": Tc,
                           "n_omega": Nw, "E_range_meV": [0, spec.E_max_meV], "window": spec.window,
                           "precision": args.precision + (" (hi*hi+hi*lo+lo*hi, fp32 accumulate, fp64 phase)"
                                                          if split else ""),
                           "k_stage": info["k_stage"], "omega_tile": info["omega_tile"],
                           "tc_block_frames": info["tc_block_frames"], "tc_drain_frames": info["tc_drain_frames"],
                           "frames_in_place": bool(info["frames_in_place"]),
                           "smem_stages": info["stages"], "plan_device_GB": round(info["device_bytes"] / 1e9, 2),
                           "l2": "inputs (%.1f GB) larger than L2, no flush" % (T * frame_elems * 8 / 1e9),
                           "segments_in_flight": n_pipe, "contraction_ctas_max": args.tc_max_ctas or None,
                           "parallelism": f"replicas x{world}"},
                "max_rel_err_I_vs_fp64": err, "error_sample": "24 (probe, pixel) series, all energies",
                "spectra_per_s": spectra_per_s, "clocks": clocks, "gpu_launches": launches, "e2e": e2e,
                "roofline": roof, "conversion_roofline": conv, "cpu_baseline": cpu, "fp32_path": fp32,
                "split_fp16_path": fp16}
        if phases:
            line["flush_phases"] = phases
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
