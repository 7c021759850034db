#!/usr/bin/env python
"""Throughput of the streaming TACAW time->energy stage on GB300.

Headline (default): the thick-sample workload, one step = the whole 256-probe scan through the
C ABI in 8 batches of 32 probes.  Each batch: reset, 128 pushes of 64 full 1024x1024 frames
(the centred 256x256 k-ROI is cropped while the pushes are read), finalize into I(k,E) (1000
energies over 0-150 meV, Hann window, elastic mean removed) and the r=20 px aperture spectra.
Metric: complex MAC/s = P*K^2*T*Nw / step time (and EELS spectra/s = P*D / step time).

The same line carries, as extra keys, the realistic stream (64 probes, 256^2, T=2048, 400
energies; with the FP32 and split-FP16 paths beside it), the 16 batched uneven partitions
(one CUDA-graph replay per step) and the differentiation workload (forward + adjoint), each
with its own error against the FP64 oracle and its own roofline.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--workload thick|realistic|batched|diff] [--no-extras]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU (probe sets are
independent: no collective on the data path); value = all ranks' CMAC / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "complex MAC/s of streaming TACAW DFT and EELS spectra/s on 1 GB300 at stated error vs FP64"
UNIT = "CMAC/s"
FLOP_PER_CMAC_SPLIT = 24      # hi*hi + hi*lo + lo*hi, each 4 real MAC (8 flop) per complex MAC
FLOP_PER_CMAC_FP32 = 8

# DRAM bytes per CMAC of a contraction kernel from an ncu capture at one workload's shape, keyed by
# the hash of the kernel's source file (code only) at capture time, the kernel and the workload:
# reported only for that workload and while the source is unchanged.
KERNEL_TRAFFIC = {
    # ncu --set full of flush_tc_drain2_kernel on `bench.py --small --no-extras` (the thick workload with
    # 1 probe: 65536 rows, T = 8192, 1000 energies, 5.369e11 CMAC per launch): 8.588006 GB read +
    # 0.263809 GB written per launch
    ("c203f07464ecfede", "flush_tc_drain2_kernel", "thick"): 1.648779e-02,
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="thick", choices=["thick", "thick_pipelined", "realistic", "batched",
                                                            "diff"],
                    help="thick (default): the 256-probe thick-sample scan per step; the others print their "
                         "own line (they are extra keys of the default line)")
    ap.add_argument("--no-extras", dest="extras", action="store_false", default=True,
                    help="thick line without the realistic / batched / differentiation legs")
    ap.add_argument("--small", action="store_true",
                    help="small case of the chosen workload (profiling captures): thick = 1 probe in 1 batch; "
                         "realistic = 2 probes")
    ap.add_argument("--k-stage", type=int, default=0,
                    help="frames staged per flush (0: as many as the HBM budget allows)")
    ap.add_argument("--accum", default="auto", choices=["auto", "kahan", "fp64", "fp32"])
    ap.add_argument("--precision", default="split_bf16", choices=["split_bf16", "split_fp16", "fp32"],
                    help="realistic workload: precision of the main leg")
    ap.add_argument("--in-place", action="store_true", help="realistic workload: frames read in place")
    ap.add_argument("--tc-omega-tile", type=int, default=0)
    ap.add_argument("--tc-block-frames", type=int, default=0)
    ap.add_argument("--tc-drain-frames", type=int, default=0)
    ap.add_argument("--tc-max-ctas", type=int, default=0)
    ap.add_argument("--fp32-steps", type=int, default=2, help="realistic: FP32-path comparison steps (0: skip)")
    ap.add_argument("--fp16-steps", type=int, default=2, help="realistic: split-FP16 comparison steps (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=1, help="end-to-end steps from pinned host memory (0: skip)")
    ap.add_argument("--e2e-free-sms", type=int, default=16,
                    help="thick e2e with two half-batch plans: SMs their contraction grids leave free for the "
                         "other half's pushes (0: skip that ingest)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target seconds of the CPU oracle baseline")
    ap.add_argument("--trace", action="store_true", help="per-CTA phase breakdown of one contraction")
    return ap.parse_args(argv)


def tiling(args):
    return dict(tc_omega_tile=args.tc_omega_tile, tc_block_frames=args.tc_block_frames,
                tc_drain_frames=args.tc_drain_frames, tc_max_ctas=args.tc_max_ctas)


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


def thick_spec(small: bool):
    """(name, spec, probes per batch) of the thick-sample workload (or its 1-probe small case)."""
    import synth
    w = synth.thick()
    spec, B = w.streams[0], w.probe_batch
    if small:
        return w.name + "-small-P1", synth.workloads.with_(spec, P=1), 1
    return w.name, spec, B


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


TC_SRC = os.path.join(ROOT, "paper_2607_02236_gb300", "csrc", "k_tc_gemm.cu")


def tensor_roofline(cmac_launch, kernel_ms, kname, launches_per_step, precision="split_bf16", workload=None):
    """Roofline of a tensor-core contraction launch: algorithmic flops (24 per CMAC) over its
    CUDA-event duration, against the measured burst bf16 rate (fp16 has the same dense rate)."""
    peaks, src = measured_peaks()
    achieved = cmac_launch * FLOP_PER_CMAC_SPLIT / (kernel_ms * 1e-3) / 1e12
    peak = peaks.get("bf16_tflops")
    sus = peaks.get("bf16_tflops_sustained")
    tr = KERNEL_TRAFFIC.get((file_hash(TC_SRC), kname, workload))
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": tr * cmac_launch if tr else None, "kernel": kname, "flop_per_cmac": FLOP_PER_CMAC_SPLIT,
            "kernel_ms": kernel_ms, "launches_per_step": launches_per_step,
            "frac_of_sustained": achieved / sus if sus else None,
            "peak_source": f"{src} bf16 burst (MEASURED_PEAKS.json bf16_tflops)" +
                           ("; fp16 and bf16 have the same dense tensor rate" if precision == "split_fp16" else "")}


def ffma_roofline(cmac_launch, kernel_ms, kname, launches_per_step, sm_max_mhz):
    """FP32 CUDA-core path: 8 flop per CMAC against 152 SMs x 128 FP32 lanes x 2 flop x clock."""
    mhz = sm_max_mhz or 2070.0
    peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
    achieved = cmac_launch * FLOP_PER_CMAC_FP32 / (kernel_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": kname, "flop_per_cmac": FLOP_PER_CMAC_FP32, "kernel_ms": kernel_ms,
            "launches_per_step": launches_per_step,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}


def step_spread(per_step):
    """Median, min and max of the timed steps' own durations (ms)."""
    if not per_step:
        return None
    return {"median": statistics.median(per_step), "min": min(per_step), "max": max(per_step), "n": len(per_step)}


def conversion_roofline(bytes_per_step, ms_per_step, split=True):
    """HBM roofline of the pushes: each conversion reads a complex64 sample (8 B) and writes its two
    16-bit pieces of Re and Im (or a float2 on the FP32 path): 16 B per (row, frame)."""
    peaks, src = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    ach = bytes_per_step / (ms_per_step * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm if hbm else None,
            "traffic": None, "kernel": "convert_split_tiled_kernel" if split else "convert_fp32_kernel",
            "bytes_per_step": bytes_per_step, "ms_per_step": ms_per_step,
            "timed": "CUDA events around reset + all pushes of each batch or segment (the span also holds the "
                     "provisional-mean kernel of the first push, whose reads are not counted)",
            "peak_source": f"{src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}


def host_cores():
    import multiprocessing
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else multiprocessing.cpu_count()


# ----------------------------------------------------------------------------------------------
# The FP64 oracle on the host cores: the cpu_baseline leg, which on the same sampled series of
# the GPU's own input also gives the stated error of the GPU result, and the reference arm
# ----------------------------------------------------------------------------------------------
def oracle_kw(spec):
    return dict(window_kind=spec.window,
                window_param=spec.window_sigma() if spec.window == "gauss" else spec.window_param,
                E_meV=spec.energies_meV(), dt_fs=spec.dt_fs, subtract_mean=spec.subtract_mean,
                bose_T_K=spec.bose_T_K)


def cpu_leg(series, got, spec, seconds=0.0):
    """series [T, n]: the GPU's input at n sampled (probe, pixel) places; got [Nw, m] (m <= n): the
    GPU's I at the first m of them.  Returns the max error relative to the peak against the FP64
    oracle there and, when seconds > 0, the oracle's throughput timed for about that long on the
    host cores over batches of the n series."""
    import numpy as np
    import oracle
    m = got.shape[1]
    _, ref = oracle.forward_pixels(series[:, :m], **oracle_kw(spec))
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    if seconds <= 0:
        return err, None
    T, n = series.shape
    k = min(256, n)
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < seconds:
        s0 = (done // k) * k % max(1, n - k + 1)
        oracle.forward_pixels(series[:, s0:s0 + k], **oracle_kw(spec))
        done += k
    dt = time.perf_counter() - t0
    cpu = {"value": done * T * spec.Nw / dt, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
           "sample": f"{done} (probe, pixel) series of the timed input x T={T} x Nw={spec.Nw} in {dt:.1f} s "
                     f"(FP64 NumPy oracle, threaded BLAS), scaled to CMAC/s"}
    return err, cpu


def reference_arm(args):
    """The oracle as it stands on the host cores, on a bounded sample of the headline workload."""
    import oracle
    import numpy as np
    from synth import frames
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    name, spec, _ = thick_spec(args.small)
    rng = np.random.default_rng(0)
    n_px = 32 if args.small else 256
    pix = rng.integers(0, spec.Kx * spec.Ky, n_px)
    series = frames.pixel_series(spec, 0, 0, pix // spec.Kx, pix % spec.Kx)
    kw = oracle_kw(spec)
    for _ in range(args.warmup):
        oracle.forward_pixels(series, **kw)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.forward_pixels(series, **kw)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = n_px * spec.T * spec.Nw * len(times) / tot
    sample = f"{n_px} pixel series x T={spec.T} x Nw={spec.Nw} of {name} per step (FP64 NumPy oracle)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------------
# GPU context and helpers
# ----------------------------------------------------------------------------------------------
class Ctx:
    def __init__(self):
        import torch
        import __graft_entry__
        __graft_entry__.build()
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(self.local)
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max_ms(self, ms):
        return max_over_ranks(ms, self.dist, "cuda")

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def free_device():
    import gc
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def link_peak_gbs(nbytes=4 << 30):
    """Host -> device bandwidth of one plain copy from pinned memory (cudaMemcpyAsync through
    torch), best of three, CUDA events."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h.fill_(1)
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        d.copy_(h, non_blocking=True)
        e1.record(st)
        e1.synchronize()
        best = max(best, nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    del h, d
    return best


def timed_steps(ctx, plan_list, step, steps, warmup, sample_clocks=True, per_step=None):
    """Runs `warmup` untimed and `steps` timed calls of step(k); CUDA events on the current stream,
    a barrier and a synchronize on both sides.  Returns (ms per step max over ranks, contraction
    ms per launch, contraction launches per step, kernel launches per step, clocks); a list given
    as per_step receives each timed step's own duration (events between the steps)."""
    import torch
    st = torch.cuda.current_stream()
    for k in range(warmup):
        step(k)
    torch.cuda.synchronize()
    for pl in plan_list:
        pl.check_errors(st.cuda_stream)
    ctx.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(ctx.local) if sample_clocks else None
    for pl in plan_list:
        pl.set_timing(True)
        pl.kernel_time_ms(reset=True)
    l0 = sum(pl.info()["kernel_launches"] for pl in plan_list)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    marks = []
    e0.record(st)
    for k in range(steps):
        step(warmup + k)
        if per_step is not None and k + 1 < steps:
            m = torch.cuda.Event(enable_timing=True)
            m.record(st)
            marks.append(m)
    e1.record(st)
    torch.cuda.synchronize()
    ctx.barrier()
    clocks = clk.stop() if clk else None
    if per_step is not None:
        bounds = [e0] + marks + [e1]
        per_step.extend(a.elapsed_time(b) for a, b in zip(bounds[:-1], bounds[1:]))
    for pl in plan_list:
        pl.check_errors(st.cuda_stream)
    kms, kn = 0.0, 0
    for pl in plan_list:
        a, b = pl.kernel_time_ms(reset=True)
        kms, kn = kms + a, kn + b
        pl.set_timing(False)
    launches = (sum(pl.info()["kernel_launches"] for pl in plan_list) - l0) // steps
    ms = ctx.max_ms(e0.elapsed_time(e1)) / steps
    return ms, kms / max(kn, 1), kn // max(steps, 1), launches, clocks


def sample_series(x_frames, rows, T, period=None):
    """[T, n] series of the device frame buffer x_frames viewed as [frames, elems] at element
    indices `rows` (frame t of a cycled ring is frame t mod period)."""
    import numpy as np
    import torch
    cyc = x_frames[:, torch.as_tensor(rows, device="cuda")].cpu().numpy()
    if period is None:
        return cyc[:T]
    return cyc[np.arange(T) % period]


def gather_I(I_view, probes, pix):
    """[Nw, n] of an output I viewed as [P, Nw, npix] at the sampled (probe, pixel) places."""
    import torch
    return I_view[torch.as_tensor(probes, device="cuda"), :, torch.as_tensor(pix, device="cuda")].cpu().numpy().T


def flush_phases(plan, step):
    """Per-CTA phase stamps of one traced contraction (persistent kernel: one row per CTA)."""
    import numpy as np
    import torch
    plan.set_timing(2)
    step(0)
    torch.cuda.synchronize()
    tr = plan.flush_trace().astype(np.int64)
    plan.set_timing(0)
    tr = tr[tr[:, 0] != 0]
    if not len(tr):
        return None
    return {"ctas": int(len(tr)), "lifetime_us": round(float(np.median(tr[:, 6] - tr[:, 0])) / 1e3, 1),
            "setup_us": round(float(np.median(tr[:, 1] - tr[:, 0])) / 1e3, 2),
            "first_operands_us": round(float(np.median(tr[:, 2] - tr[:, 1])) / 1e3, 2),
            "mma_span_us": round(float(np.median(tr[:, 3] - tr[:, 2])) / 1e3, 1),
            "tiles_per_cta": int(np.median(tr[:, 4])), "chunks_per_cta": int(np.median(tr[:, 5])),
            "mma_us_per_tile": round(float(np.median((tr[:, 3] - tr[:, 2]) / np.maximum(tr[:, 4], 1))) / 1e3, 2),
            "tail_after_last_mma_us": round(float(np.median(tr[:, 6] - tr[:, 3])) / 1e3, 2),
            "last_cta_exit_minus_first_us": round(float(tr[:, 6].max() - tr[:, 6].min()) / 1e3, 1),
            "unit": "median per CTA"}


# ----------------------------------------------------------------------------------------------
# Thick sample (the headline): 256 probes in 8 batches of 32, 1024^2 frames cropped to 256^2,
# T = 8192 in 64-frame pushes, 1000 energies; one plan reused with tacaw_reset per batch
# ----------------------------------------------------------------------------------------------
def thick_leg(ctx, args):
    import numpy as np
    import torch
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan
    name, spec, B = thick_spec(args.small)
    n_batch = spec.P // B
    K, T, Tc, Nw = spec.Kx, spec.T, spec.Tc, spec.Nw
    D = len(spec.detectors)
    gx, gy = spec.full_grid
    rx, ry = spec.roi_origin
    npix = K * K
    fe = B * gx * gy                       # one full frame for each probe of a batch
    cmac_step = B * npix * T * Nw * n_batch
    st_t = torch.cuda.current_stream()
    st = st_t.cuda_stream
    # a resident ring of R pushes of full frames (17.2 GB each), cycled over each segment: frame t
    # of a batch is frame t mod (R * Tc) of the ring; only the ROI of the full grid is synthesised
    # (and read); every batch reads the same ring
    R = 2
    ring = torch.zeros(R * Tc * fe, dtype=torch.complex64, device="cuda")
    for r in range(R):
        sg.generate(spec, 33 + ctx.rank, ring.data_ptr() + r * Tc * fe * 8, r * Tc, Tc, pitch_row=gx,
                    pitch_frame=fe, pitch_probe=gx * gy, out_x0=rx, out_y0=ry, p0=0, P=B, stream=st)
    I = torch.empty(spec.P * Nw * npix, dtype=torch.float32, device="cuda")        # all probes
    S = torch.empty(max(1, spec.P * D * Nw), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    plan = TacawPlan([stream_config(spec, P=B)], precision="split_bf16", k_stage=args.k_stage, accum=args.accum,
                     **tiling(args))
    info = plan.info()
    n_push = T // Tc
    i_b, s_b = B * Nw * npix, B * D * Nw
    pev = {}

    def batch(b, frames_base, k=None):
        if k is not None:
            pev[(k, b)] = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            pev[(k, b)][0].record(st_t)
        plan.reset(st)
        for i in range(n_push):
            plan.push(0, frames_base + (i % R) * Tc * fe * 8, Tc, st)
        if k is not None:
            pev[(k, b)][1].record(st_t)
        plan.finalize_async(I[b * i_b:(b + 1) * i_b], S[b * s_b:(b + 1) * s_b] if D else None, None, st)

    def step(k):
        for b in range(n_batch):
            batch(b, ring.data_ptr(), k if k >= args.warmup else None)

    f0 = plan.info()["flush_launches"]
    per_step = []
    ms, flush_ms, k_per_step, launches, clocks = timed_steps(ctx, [plan], step, args.steps, args.warmup,
                                                             per_step=per_step)
    flushes = (plan.info()["flush_launches"] - f0) // (args.steps + args.warmup)
    push_ms = statistics.median(sum(pev[(k, b)][0].elapsed_time(pev[(k, b)][1]) for b in range(n_batch))
                                for k in range(args.warmup, args.warmup + args.steps))
    value = job_rate(cmac_step, ctx.world, ms * 1e-3)
    phases = flush_phases(plan, lambda k: batch(0, ring.data_ptr())) if args.trace else None

    # sampled (probe, pixel) series of the ring-cycled input: the stated error at the first and
    # the last batch's I, and the CPU oracle baseline on the same series
    rng = np.random.default_rng(ctx.rank)
    n_s, n_chk = 256, 16
    pb = rng.integers(0, B, n_s)
    c = (K // 2) * K + K // 2
    px = np.concatenate([[c, c + 3, c - 5 * K + 2], rng.integers(0, npix, n_s - 3)])
    rows = pb * gx * gy + (ry + px // K) * gx + (rx + px % K)
    series = sample_series(ring.view(R * Tc, fe), rows, T, R * Tc)
    err, cpu = 0.0, None
    for b in sorted({0, n_batch - 1}):
        got = gather_I(I[b * i_b:(b + 1) * i_b].view(B, Nw, npix), pb[:n_chk], px[:n_chk])
        want_cpu = b == n_batch - 1 and ctx.rank == 0 and ctx.world == 1
        e, cb = cpu_leg(series, got, spec, args.cpu_seconds if want_cpu else 0.0)
        err = max(err, e)
        cpu = cb or cpu

    roof = tensor_roofline(cmac_step / max(k_per_step, 1), flush_ms, "flush_tc_drain2_kernel", k_per_step,
                           workload="thick")
    conv = conversion_roofline(16.0 * B * npix * T * n_batch, push_ms)

    # end to end through the public API from pinned host memory: the same step with the ring in
    # host memory -- the push kernels read each push's ROI rows over the host link (zero-copy
    # ingest) -- and each batch's spectra read back
    e2e = None
    if args.e2e_steps > 0:
        link = link_peak_gbs()
        host = torch.empty(ring.numel(), dtype=torch.complex64, pin_memory=True)
        host.copy_(ring)
        S_host = torch.empty(S.numel(), dtype=torch.float32, pin_memory=True)
        batch(0, host.data_ptr())                  # warm-up of the host path
        torch.cuda.synchronize()
        plan.check_errors(st)
        ctx.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for b in range(n_batch):
                batch(b, host.data_ptr())
                S_host[b * s_b:(b + 1) * s_b].copy_(S[b * s_b:(b + 1) * s_b], non_blocking=True)
        torch.cuda.synchronize()
        el = ctx.max_ms((time.perf_counter() - t0) * 1e3) * 1e-3
        plan.check_errors(st)
        h2d = B * npix * T * 8 * n_batch
        e2e = {"value": job_rate(cmac_step * args.e2e_steps, ctx.world, el), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": S.numel() * 4,
               "ms_per_step": 1e3 * el / args.e2e_steps, "steps": args.e2e_steps,
               "link_gbs_measured": link, "link_gbs_achieved": h2d / (el / args.e2e_steps) / 1e9,
               "frac": h2d / (el / args.e2e_steps) / 1e9 / link,
               "link_measure": "one 4 GiB cudaMemcpyAsync from pinned host memory to the device (best of 3, "
                               "CUDA events)",
               "input": f"pinned host ring of {R} pushes of full frames ({R * Tc * fe * 8 / 1e9:.1f} GB) cycled",
               "ingest": "zero-copy: the push kernels read each push's ROI rows straight from pinned host "
                         "memory over the host link (only the ROI crosses it)",
               "timed": "host wall clock around the step, device synchronized on both sides"}
        del ring
        plan.close()
        free_device()
        # the same step with two plans of half a batch each on two CUDA streams: one plan's pushes
        # (reading the host link) run while the other plan's contraction runs, its grid capped so
        # that SMs stay free for the pushes; the faster of the two ingests is the e2e figure
        if B % 2 == 0 and args.e2e_free_sms > 0:
            pipe = thick_e2e_pipelined(ctx, args, spec, B, n_batch, host, I, S, S_host, R)
            pipe["link_gbs_measured"] = link
            pipe["link_gbs_achieved"] = h2d / (pipe["ms_per_step"] * 1e-3) / 1e9
            pipe["frac"] = pipe["link_gbs_achieved"] / link
            pipe["input"] = e2e["input"]
            pipe["link_measure"] = e2e["link_measure"]
            if pipe["value"] > e2e["value"]:
                pipe["other_ingest"], e2e = e2e, pipe
            else:
                e2e["other_ingest"] = pipe
        del host
    else:
        del ring
        plan.close()
    del I, S
    free_device()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ctx.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "step_ms": step_spread(per_step),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": name, "probes_per_step": spec.P, "probe_batch": B, "batches_per_step": n_batch,
                       "full_grid": f"{gx}x{gy}", "k_roi": f"{K}x{K} at ({rx}, {ry})", "T": T,
                       "frames_per_push": Tc, "n_omega": Nw, "E_range_meV": [0, spec.E_max_meV],
                       "window": spec.window, "detectors": D,
                       "precision": "split_bf16: hi*hi + hi*lo + lo*hi, fp32 accumulate in tensor memory, hi*hi "
                                    f"drained into fp32 registers every {info['tc_drain_frames']} frames, fp64 phase",
                       "k_stage": info["k_stage"], "flushes_per_batch": -(-T // info["k_stage"]),
                       "accumulators": ["kahan", "fp64", "fp32"][info["accum"]] if info["k_stage"] < T else "none",
                       "omega_tile": info["omega_tile"], "tc_block_frames": info["tc_block_frames"],
                       "smem_stages": info["stages"], "plan_device_GB": round(info["device_bytes"] / 1e9, 1),
                       "inputs": f"ring of {R} pushes of full frames ({R * Tc * fe * 8 / 1e9:.1f} GB) resident in "
                                 "HBM, cycled over each batch; every batch reads the same ring",
                       "outputs": "I of all probes resident in HBM (%.1f GB), spectra" % (spec.P * Nw * npix * 4 / 1e9),
                       "l2": "pushes (17.2 GB of full frames, 1.07 GB of ROI read each) and the staging larger "
                             "than L2, no flush",
                       "parallelism": f"replicas x{ctx.world}"},
            "max_rel_err_I_vs_fp64": err,
            "error_sample": f"{n_chk} (probe, pixel) series of the first and the last batch, all energies",
            "spectra_per_s": job_rate(spec.P * D, ctx.world, ms * 1e-3),
            "clocks": clocks, "gpu_launches": launches, "contraction_launches_per_step": flushes,
            "e2e": e2e, "roofline": roof, "conversion_roofline": conv, "cpu_baseline": cpu}
    if phases:
        line["flush_phases"] = phases
    return line


def thick_e2e_pipelined(ctx, args, spec, B, n_batch, host, I, S, S_host, R):
    """End-to-end thick step with two plans of B/2 probes (probes 0..B/2-1 and B/2..B-1 of every
    pushed frame, read from the same pinned host ring): their half batches alternate on two CUDA
    streams, each half's pushes ordered after the other half's pushes, so that one half's
    zero-copy ingest runs beside the other half's contraction; the contraction grids leave
    args.e2e_free_sms SMs free for it.  Host wall clock over args.e2e_steps steps."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    K, T, Tc, Nw = spec.Kx, spec.T, spec.Tc, spec.Nw
    D = len(spec.detectors)
    gx, gy = spec.full_grid
    npix = K * K
    H = B // 2
    fe = B * gx * gy
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    cap = max(1, sms - args.e2e_free_sms)
    cfg = stream_config(spec, P=H)
    cfg.pitch_frame = fe                               # frames of the host ring hold all B probes
    plans = [TacawPlan([cfg], precision="split_bf16", accum=args.accum, tc_max_ctas=cap, **{
        k: v for k, v in tiling(args).items() if k != "tc_max_ctas"}) for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pushed = [torch.cuda.Event(), torch.cuda.Event()]
    i_h, s_h = H * Nw * npix, H * D * Nw
    n_push = T // Tc
    prev = [None]

    def half(b, h):
        pl, sx = plans[h], streams[h]
        st = sx.cuda_stream
        if prev[0] is not None:
            sx.wait_event(prev[0])                    # the other half's pushes are done
        pl.reset(st)
        base = host.data_ptr() + h * H * gx * gy * 8
        for i in range(n_push):
            pl.push(0, base + (i % R) * Tc * fe * 8, Tc, st)
        pushed[h].record(sx)
        prev[0] = pushed[h]
        o = (b * B + h * H)
        pl.finalize_async(I[o * Nw * npix:o * Nw * npix + i_h], S[o * D * Nw:o * D * Nw + s_h] if D else None,
                          None, st)
        if D:
            with torch.cuda.stream(sx):
                S_host[o * D * Nw:o * D * Nw + s_h].copy_(S[o * D * Nw:o * D * Nw + s_h], non_blocking=True)

    half(0, 0)                                         # warm-up of both plans' host paths
    half(0, 1)
    torch.cuda.synchronize()
    for pl, sx in zip(plans, streams):
        pl.check_errors(sx.cuda_stream)
    ctx.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        for b in range(n_batch):
            half(b, 0)
            half(b, 1)
    torch.cuda.synchronize()
    el = ctx.max_ms((time.perf_counter() - t0) * 1e3) * 1e-3
    for pl, sx in zip(plans, streams):
        pl.check_errors(sx.cuda_stream)
        pl.close()
    cmac_step = B * npix * T * Nw * n_batch
    return {"value": job_rate(cmac_step * args.e2e_steps, ctx.world, el), "unit": UNIT,
            "h2d_bytes_per_step": B * npix * T * 8 * n_batch, "d2h_bytes_per_step": S.numel() * 4,
            "ms_per_step": 1e3 * el / args.e2e_steps, "steps": args.e2e_steps,
            "ingest": f"zero-copy pushes; two plans of {H} probes alternate on two CUDA streams, one half's "
                      f"pushes beside the other half's contraction (grids capped at {cap} of {sms} SMs)",
            "timed": "host wall clock around the step, device synchronized on both sides"}


# ----------------------------------------------------------------------------------------------
# Realistic stream: 64 probes, 256^2, T = 2048 in 32-frame pushes, 400 energies, resident input
# ----------------------------------------------------------------------------------------------
def realistic_leg(ctx, args, sample_clocks=True):
    import numpy as np
    import torch
    import synth
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan
    spec = synth.realistic().streams[0]
    name = synth.realistic().name
    if args.small:
        spec, name = synth.workloads.with_(spec, P=2), "small-P2-K256-T2048-W400"
    P, K, T, Tc, Nw = spec.P, spec.Kx, spec.T, spec.Tc, spec.Nw
    D = len(spec.detectors)
    npix = K * K
    fe = P * npix
    cmac_step = P * npix * T * Nw
    st_t = torch.cuda.current_stream()
    st = st_t.cuda_stream
    x = torch.empty(T * fe, dtype=torch.complex64, device="cuda")        # 68.7 GB: [T][P][K][K]
    for t0 in range(0, T, 64):
        sg.generate(spec, 1000 + ctx.rank, x.data_ptr() + t0 * fe * 8, t0, min(64, T - t0), pitch_row=K,
                    pitch_frame=fe, pitch_probe=npix, stream=st)
    I = torch.empty(P * Nw * npix, dtype=torch.float32, device="cuda")
    S = torch.empty(max(1, P * D * Nw), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    n_push = (T + Tc - 1) // Tc
    split = args.precision.startswith("split")
    pev = {}

    def run(plan, k=None):
        if k is not None:
            pev[k] = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            pev[k][0].record(st_t)
        plan.reset(st)
        for i in range(n_push):
            plan.push(0, x.data_ptr() + i * Tc * fe * 8, min(Tc, T - i * Tc), st)
        if k is not None:
            pev[k][1].record(st_t)
        plan.finalize_async(I, S if D else None, None, st)

    rng = np.random.default_rng(ctx.rank)
    probes = rng.integers(0, P, 24)
    pix = np.concatenate([[K // 2 * K + K // 2, (K // 2 + 3) * K + K // 2 - 5], rng.integers(0, npix, 22)])
    series = sample_series(x.view(T, fe), probes * npix + pix, T)

    def error():
        e, _ = cpu_leg(series, gather_I(I.view(P, Nw, npix), probes, pix), spec)
        return e

    plan = TacawPlan([stream_config(spec)], precision=args.precision, accum=args.accum,
                     frames_in_place=bool(args.in_place), **tiling(args))
    info = plan.info()
    ms, flush_ms, k_per_step, launches, clocks = timed_steps(
        ctx, [plan], lambda k: run(plan, k if k >= args.warmup else None), args.steps, args.warmup, sample_clocks)
    push_ms = statistics.median(pev[k][0].elapsed_time(pev[k][1]) for k in range(args.warmup, args.warmup + args.steps))
    err = error()
    phases = flush_phases(plan, lambda k: run(plan)) if args.trace and split else None
    plan.close()
    if split:
        kname = "flush_tc_inplace_kernel" if info["frames_in_place"] else "flush_tc_drain2_kernel"
        roof = tensor_roofline(cmac_step / max(k_per_step, 1), flush_ms, kname, k_per_step, args.precision)
    else:
        roof = ffma_roofline(cmac_step / max(k_per_step, 1), flush_ms, "flush_simt_kernel", k_per_step,
                             (clocks or {}).get("sm_max_mhz"))
    conv = None if info["frames_in_place"] else conversion_roofline(16.0 * P * npix * T, push_ms, split)

    def comparison(precision, steps):
        with TacawPlan([stream_config(spec)], precision=precision) as pc:
            m, kf, kn, _, _ = timed_steps(ctx, [pc], lambda k: run(pc), steps, 1, sample_clocks=False)
        e = error()
        out = {"value": job_rate(cmac_step, ctx.world, m * 1e-3), "unit": UNIT, "ms_per_step": m,
               "flush_ms": kf, "max_rel_err_I_vs_fp64": e}
        if precision == "fp32":
            out["roofline"] = ffma_roofline(cmac_step / max(kn, 1), kf, "flush_simt_kernel", kn,
                                            (clocks or {}).get("sm_max_mhz"))
        else:
            out["roofline"] = tensor_roofline(cmac_step / max(kn, 1), kf, "flush_tc_drain2_kernel", kn, precision)
        return out

    fp16 = comparison("split_fp16", args.fp16_steps) if args.fp16_steps > 0 and args.precision == "split_bf16" else None
    fp32 = comparison("fp32", args.fp32_steps) if args.fp32_steps > 0 and args.precision != "fp32" else None
    del x, I, S
    free_device()
    out = {"workload": name, "value": job_rate(cmac_step, ctx.world, ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "steps": args.steps, "warmup": args.warmup, "precision": args.precision,
           "dtype": {"split_bf16": "bf16", "split_fp16": "f16"}.get(args.precision, "f32"),
           "config": {"probes": P, "k_roi": f"{K}x{K}", "T": T, "frames_per_push": Tc, "n_omega": Nw,
                      "E_range_meV": [0, spec.E_max_meV], "window": spec.window, "k_stage": info["k_stage"],
                      "omega_tile": info["omega_tile"], "tc_block_frames": info["tc_block_frames"],
                      "tc_drain_frames": info["tc_drain_frames"], "frames_in_place": bool(info["frames_in_place"]),
                      "plan_device_GB": round(info["device_bytes"] / 1e9, 1),
                      "l2": "inputs (%.1f GB) resident in HBM, larger than L2, no flush" % (T * fe * 8 / 1e9)},
           "max_rel_err_I_vs_fp64": err, "error_sample": "24 (probe, pixel) series, all energies",
           "spectra_per_s": job_rate(P * D, ctx.world, ms * 1e-3), "gpu_launches": launches, "clocks": clocks,
           "roofline": roof, "conversion_roofline": conv, "split_fp16_path": fp16, "fp32_path": fp32}
    if phases:
        out["flush_phases"] = phases
    return out


# ----------------------------------------------------------------------------------------------
# Batched partitions: 16 uneven streams in one plan (autotuned tiles, the flushes of all streams
# that fall due together in one persistent launch), a whole segment captured into a CUDA graph
# ----------------------------------------------------------------------------------------------
def batched_leg(ctx, args, sample_clocks=True):
    import numpy as np
    import torch
    import synth
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan
    w = synth.batched()
    specs = list(w.streams)
    n_s = len(specs)
    cmac_step = sum(s.P * s.Kx * s.Ky * s.T * s.Nw for s in specs)
    # the segments (338 GB of frames) exceed HBM: each partition keeps R pushes resident and
    # cycles them (frame t of a segment is frame t mod (R*Tc) of the ring)
    R = 4
    st_t = torch.cuda.current_stream()
    bufs = []
    for i, s in enumerate(specs):
        fe = s.P * s.Kx * s.Ky
        b = torch.empty(R * s.Tc * fe, dtype=torch.complex64, device="cuda")
        sg.generate(s, 3000 + 97 * ctx.rank + i, b.data_ptr(), 0, R * s.Tc, pitch_row=s.Kx, pitch_frame=fe,
                    pitch_probe=s.Kx * s.Ky, stream=st_t.cuda_stream)
        bufs.append(b)
    # outputs before the plan: the plan takes its staging from what memory is left
    I = torch.empty(sum(s.P * s.Nw * s.Kx * s.Ky for s in specs), dtype=torch.float32, device="cuda")
    S = torch.empty(max(1, sum(s.P * len(s.detectors) * s.Nw for s in specs)), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = TacawPlan([stream_config(s) for s in specs], precision="split_bf16", tune="", accum=args.accum)
    plan_s = time.perf_counter() - t0
    info = plan.info()

    def enqueue(sth):
        # one group push per round: every partition with frames left pushes its next chunk
        plan.reset(sth)
        pushed = [0] * n_s
        while any(pushed[i] < s.T for i, s in enumerate(specs)):
            ids, ptrs, cnt = [], [], []
            for i, s in enumerate(specs):
                if pushed[i] >= s.T:
                    continue
                n = min(s.Tc, s.T - pushed[i])
                slot = (pushed[i] // s.Tc) % R
                ids.append(i)
                ptrs.append(bufs[i].data_ptr() + slot * s.Tc * s.P * s.Kx * s.Ky * 8)
                cnt.append(n)
                pushed[i] += n
            plan.push_group(ids, ptrs, cnt, sth)
        plan.finalize_async(I, S, None, sth)

    # one eager segment (launch counts, contraction time), then the captured graph is timed
    cap = torch.cuda.Stream()
    with torch.cuda.stream(cap):
        enqueue(cap.cuda_stream)
        plan.check_errors(cap.cuda_stream)
        l0, f0 = plan.info()["kernel_launches"], plan.info()["flush_launches"]
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
        flushes = plan.info()["flush_launches"] - f0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        enqueue(torch.cuda.current_stream().cuda_stream)
    ms, _, _, _, clocks = timed_steps(ctx, [], lambda k: g.replay(), args.steps, args.warmup, sample_clocks)
    plan.check_errors(st_t.cuda_stream)

    # stated error: two sampled series per partition, all energies, against the FP64 oracle
    rng = np.random.default_rng(ctx.rank)
    worst = 0.0
    for i, s in enumerate(specs):
        npx = s.Kx * s.Ky
        p = rng.integers(0, s.P, 2)
        k = rng.integers(0, npx, 2)
        ser = sample_series(bufs[i].view(R * s.Tc, s.P * npx), p * npx + k, s.T, R * s.Tc)
        io, _ = plan.offsets(i)
        got = gather_I(I[io:io + s.P * s.Nw * npx].view(s.P, s.Nw, npx), p, k)
        e, _ = cpu_leg(ser, got, s)
        worst = max(worst, e)
    del g
    plan.close()
    del bufs, I, S
    free_device()
    return {"workload": w.name, "value": job_rate(cmac_step, ctx.world, ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "steps": args.steps, "warmup": args.warmup, "dtype": "bf16",
            "config": {"partitions": n_s, "cmac_per_step": cmac_step, "probes": [s.P for s in specs],
                       "k_roi": [s.Kx for s in specs], "T": [s.T for s in specs], "n_omega": specs[0].Nw,
                       "frames_per_push": specs[0].Tc, "k_stage": info["k_stage"],
                       "tc_drain_frames": info["tc_drain_frames"],
                       "accumulators": ["kahan", "fp64", "fp32"][info["accum"]],
                       "tuned_streams": info["tuned_streams"], "tune_candidates": info["tune_candidates"],
                       "tune_ms": round(info["tune_ms"], 1), "plan_create_s": round(plan_s, 2),
                       "plan_device_GB": round(info["device_bytes"] / 1e9, 1),
                       "inputs": f"per-partition rings of {R} pushes resident in HBM, cycled over each segment",
                       "step": "one CUDA-graph replay of reset + one group push per round (every partition's "
                               "next chunk, tacaw_push_frames_group) + finalize_async",
                       "l2": "staged operands (>= 10 GB per step) larger than L2, no flush"},
            "max_rel_err_I_vs_fp64": worst, "error_sample": "2 (probe, pixel) series per partition, all energies",
            "eager_ms_per_step": eager_ms, "gpu_launches": launches, "contraction_launches_per_step": flushes,
            "clocks": clocks,
            "roofline": tensor_roofline(cmac_step / max(k_n, 1), k_ms / max(k_n, 1), "flush_tc_drain2_kernel", k_n)}


# ----------------------------------------------------------------------------------------------
# Differentiation: forward spectrum and the hand-written adjoint (tacaw_backward) per step
# ----------------------------------------------------------------------------------------------
def diff_leg(ctx, args, sample_clocks=True):
    import numpy as np
    import torch
    import synth
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan
    w = synth.diff()
    spec = w.streams[0]
    P, K, T, Nw = spec.P, spec.Kx, spec.T, spec.Nw
    D = len(spec.detectors)
    npix = K * K
    st_t = torch.cuda.current_stream()
    st = st_t.cuda_stream
    x = torch.empty(T * P * npix, dtype=torch.complex64, device="cuda")
    sg.generate(spec, 4 + ctx.rank, x.data_ptr(), 0, T, pitch_row=K, pitch_frame=P * npix, pitch_probe=npix, stream=st)
    grad = torch.empty_like(x)
    c = torch.tensor(synth.loss_weights(Nw, seed=0), dtype=torch.float32, device="cuda")
    dLdS = c[None, None, :].expand(P, D, Nw).contiguous()
    I = torch.empty(P * Nw * npix, dtype=torch.float32, device="cuda")
    S = torch.empty(max(1, P * D * Nw), dtype=torch.float32, device="cuda")
    plan = TacawPlan([stream_config(spec)], precision=w.precision)
    info = plan.info()
    n_ap = int(info["aperture_pixels"])
    # forward: the dense DFT of every ROI pixel; adjoint: Psi recomputed on the aperture pixels
    # (not stored) and projected back onto every frame (G = 0 outside the apertures)
    cmac_fwd = P * npix * T * Nw
    cmac_adj = 2 * P * n_ap * T * Nw
    n_push = (T + spec.Tc - 1) // spec.Tc
    aev = {}

    def step(k):
        plan.reset(st)
        for i in range(n_push):
            plan.push(0, x.data_ptr() + i * spec.Tc * P * npix * 8, min(spec.Tc, T - i * spec.Tc), st)
        plan.finalize_async(I, S, None, st)
        aev[k] = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        aev[k][0].record(st_t)
        plan.backward(0, dLdS, x, grad, st)
        aev[k][1].record(st_t)

    ms, fwd_ms, k_n, launches, clocks = timed_steps(ctx, [plan], step, args.steps, args.warmup, sample_clocks)
    adj_ms = statistics.median(aev[k][0].elapsed_time(aev[k][1]) for k in range(args.warmup, args.warmup + args.steps))

    # the FP32 CUDA-core adjoint on the same input, the call alone (the baseline of the tensor-core one)
    def adjoint_call_ms(precision, reps):
        plan.set_adjoint_precision(precision)
        out = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st_t)
            plan.backward(0, dLdS, x, grad, st)
            e1.record(st_t)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        plan.set_adjoint_precision("split_bf16")
        return statistics.median(out)

    adj32_ms = adjoint_call_ms("fp32", max(3, args.steps))

    # stated error: spectra of two probes (all aperture pixels) and the gradient at 16 aperture
    # pixels of those probes, against the FP64 oracle
    import oracle
    rng = np.random.default_rng(ctx.rank)
    kw = oracle_kw(spec)
    kw.pop("window_param")
    kw.pop("bose_T_K")
    ap = np.asarray(oracle.detector_masks(K, K, spec.detectors)[0].reshape(-1).nonzero()[0])
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
    plan.close()
    del x, grad, I, S
    free_device()
    fwd = ffma_roofline(cmac_fwd, fwd_ms, "flush_simt_kernel", k_n, (clocks or {}).get("sm_max_mhz"))
    # the tensor-core adjoint call: its floor is the larger of the tensor time of its two
    # contractions and the HBM time of the bytes it must move (the gradient over the whole ROI of
    # every frame written once, the aperture rows' frames read once)
    adj_bytes = P * T * npix * 8 + P * n_ap * T * 8
    tc = tensor_roofline(cmac_adj, adj_ms, "tacaw_backward call (split BF16, tensor cores)", 1)
    peaks, psrc = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    mem_gbs = adj_bytes / (adj_ms * 1e-3) / 1e9
    adj = {"bound": "hbm", "achieved": mem_gbs, "peak": hbm, "unit": "GB/s", "frac": mem_gbs / hbm, "traffic": None,
           "kernel": "tacaw_backward call: ROI zero fill, aperture-row staging, two flush_tc_drain2_kernel "
                     "contractions, scatter into the frame layout",
           "bytes_per_call": adj_bytes, "tensor": {k: tc[k] for k in ("achieved", "peak", "unit", "frac")},
           "floor_ms": {"hbm": adj_bytes / (hbm * 1e9) * 1e3, "tensor": cmac_adj * FLOP_PER_CMAC_SPLIT / (tc["peak"] * 1e12) * 1e3},
           "peak_source": f"{psrc} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
           "timed": ("CUDA events around the tacaw_backward call (median per step; includes its zeroing kernel and "
                     "its closing wait for the device error word)")}
    if adj["floor_ms"]["tensor"] > adj["floor_ms"]["hbm"]:
        adj["bound"] = "tensor"
    adj32 = ffma_roofline(cmac_adj, adj32_ms, "adj_psi_kernel + adj_grad_kernel", 1, (clocks or {}).get("sm_max_mhz"))
    adj32["timed"] = "CUDA events around the tacaw_backward call alone (median), same input"
    return {"workload": w.name, "value": job_rate(cmac_fwd + cmac_adj, ctx.world, ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
            "config": {"probes": P, "k_roi": f"{K}x{K}", "T": T, "n_omega": Nw, "window": spec.window,
                       "aperture_pixels": n_ap, "cmac_per_step": {"forward": cmac_fwd, "adjoint": cmac_adj},
                       "step": "reset + push + finalize_async (FP32 path) + tacaw_backward (dL/dS = c(E); "
                               "adjoint on the tensor cores, split BF16)",
                       "l2": "frames (%.2f GB) and gradient re-read every step, no flush" % (T * P * npix * 8 / 1e9)},
            "max_rel_err_S_vs_fp64": err_s, "rel_l2_err_grad_vs_fp64": err_g,
            "error_sample": "spectra of 2 probes; gradient at 16 aperture pixels of those probes",
            "gpu_launches": launches, "clocks": clocks, "roofline": fwd, "adjoint": dict(adj, ms=adj_ms),
            "adjoint_fp32": dict(adj32, ms=adj32_ms, speedup_of_tensor_cores=adj32_ms / adj_ms)}


# ----------------------------------------------------------------------------------------------
# Thick sample with pipelined segments: the same 256 probes per step as 16 segments of 16 probes
# (two staging areas of 16 probes fit in HBM, two of 32 do not); each segment's contraction runs
# with the conversion of the next segment's pushes (tacaw_set_pipelined_segments)
# ----------------------------------------------------------------------------------------------
def thick_pipelined_leg(ctx, args, sample_clocks=True):
    import numpy as np
    import torch
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan
    name, spec, B = thick_spec(args.small)
    n_batch = spec.P // B
    K, T, Tc, Nw = spec.Kx, spec.T, spec.Tc, spec.Nw
    D = len(spec.detectors)
    gx, gy = spec.full_grid
    rx, ry = spec.roi_origin
    npix = K * K
    fe = B * gx * gy
    H = max(1, B // 2)
    n_seg = spec.P // H
    cmac_step = spec.P * npix * T * Nw
    st_t = torch.cuda.current_stream()
    st = st_t.cuda_stream
    R = 2
    ring = torch.zeros(R * Tc * fe, dtype=torch.complex64, device="cuda")
    for r in range(R):
        sg.generate(spec, 33 + ctx.rank, ring.data_ptr() + r * Tc * fe * 8, r * Tc, Tc, pitch_row=gx,
                    pitch_frame=fe, pitch_probe=gx * gy, out_x0=rx, out_y0=ry, p0=0, P=B, stream=st)
    I = torch.empty(spec.P * Nw * npix, dtype=torch.float32, device="cuda")
    S = torch.empty(max(1, spec.P * D * Nw), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    cfg = stream_config(spec, P=H)
    cfg.pitch_frame = fe                       # frames of the ring hold all B probes of a batch
    plan = TacawPlan([cfg], precision="split_bf16")
    plan.set_pipelined_segments(True)
    info = plan.info()
    n_push = T // Tc
    i_h, s_h = H * Nw * npix, H * D * Nw

    def step(k):
        for g in range(n_seg):
            b, h = divmod(g, B // H)
            plan.reset(st)
            base = ring.data_ptr() + h * H * gx * gy * 8
            for i in range(n_push):
                plan.push(0, base + (i % R) * Tc * fe * 8, Tc, st)
            o = b * B + h * H
            plan.finalize_async(I[o * Nw * npix:o * Nw * npix + i_h], S[o * D * Nw:o * D * Nw + s_h] if D else None,
                                None, st)
        plan.drain(st)

    ms, flush_ms, k_per_step, launches, clocks = timed_steps(ctx, [plan], step, args.steps, args.warmup,
                                                             sample_clocks)
    # stated error: 16 sampled (probe, pixel) series of the first and the last segment
    rng = np.random.default_rng(ctx.rank + 7)
    c = (K // 2) * K + K // 2
    err = 0.0
    for g in (0, n_seg - 1):
        b, h = divmod(g, B // H)
        pb = rng.integers(0, H, 16)
        px = np.concatenate([[c, c + 3], rng.integers(0, npix, 14)])
        rows = (h * H + pb) * gx * gy + (ry + px // K) * gx + (rx + px % K)
        series = sample_series(ring.view(R * Tc, fe), rows, T, R * Tc)
        o = b * B + h * H
        got = gather_I(I[o * Nw * npix:o * Nw * npix + i_h].view(H, Nw, npix), pb, px)
        e, _ = cpu_leg(series, got, spec, 0.0)
        err = max(err, e)
    plan.close()
    del ring, I, S
    free_device()
    roof = tensor_roofline(cmac_step / max(k_per_step, 1), flush_ms, "flush_tc_drain2_kernel + conversion warps",
                           k_per_step)
    return {"workload": name + "-pipelined-16", "value": job_rate(cmac_step, ctx.world, ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup, "dtype": "bf16",
            "config": {"probes_per_step": spec.P, "segment_probes": H, "segments_per_step": n_seg,
                       "k_roi": f"{K}x{K} at ({rx}, {ry})", "T": T, "frames_per_push": Tc, "n_omega": Nw,
                       "plan_device_GB": round(info["device_bytes"] / 1e9, 1),
                       "step": "per segment: reset + pushes (recorded) + finalize_async, which launches the "
                               "previous segment's contraction with this segment's conversion in its extra "
                               "warps; tacaw_drain after the last",
                       "why_16": "two staging areas of 32 probes (2 x 137 GB) do not fit beside the input ring "
                                 "and I; two of 16 probes do"},
            "max_rel_err_I_vs_fp64": err, "error_sample": "16 (probe, pixel) series of the first and the last "
                                                          "segment, all energies",
            "gpu_launches": launches, "contraction_launches_per_step": k_per_step, "clocks": clocks,
            "roofline": roof}


LEGS = {"realistic": realistic_leg, "batched": batched_leg, "diff": diff_leg, "thick_pipelined": thick_pipelined_leg}


def standalone_line(ctx, args, d):
    """The JSON line of a non-headline workload run on its own (--workload realistic|batched|diff)."""
    line = {"metric": METRIC, "value": d["value"], "unit": UNIT, "n_gpus": ctx.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": d["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": d.get("dtype", "bf16"), "data": "synthetic",
            "config": dict(d["config"], workload=d["workload"], parallelism=f"replicas x{ctx.world}"),
            "clocks": d.get("clocks"), "gpu_launches": d.get("gpu_launches"), "roofline": d.get("roofline"),
            "e2e": None, "cpu_baseline": None}
    for k, v in d.items():
        if k not in line and k not in ("workload", "steps", "warmup"):
            line[k] = v
    return line


def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        return reference_arm(args)
    ctx = Ctx()
    if args.workload != "thick":
        d = LEGS[args.workload](ctx, args)
        if ctx.rank == 0:
            print(json.dumps(standalone_line(ctx, args, d)), flush=True)
        ctx.close()
        return 0
    line = thick_leg(ctx, args)
    if args.extras and not args.small:
        # the differentiation step is ~5 ms: more steps for a stable time
        for name, leg in LEGS.items():
            steps = "20" if name == "diff" else ("2" if name == "thick_pipelined" else "3")
            extra_args = parse(["--steps", steps, "--warmup", "3", "--fp32-steps", str(args.fp32_steps),
                                "--fp16-steps", str(args.fp16_steps)])
            line[name] = leg(ctx, extra_args, sample_clocks=True)
    if ctx.rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
