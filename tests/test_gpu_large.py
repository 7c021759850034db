"""Full-size workloads through the C ABI, checked against the FP64 oracle on sampled outputs.

Pixels are independent in the definition, so the oracle recomputes I(k, E) for sampled
(probe, pixel) series, which are read back from the very frames the GPU consumed.  The
aperture spectra of a few probes are checked from all aperture pixels.

  realistic  64 probes, 256^2 ROI, T=2048 in 32-frame pushes, 400 E over 0-120 meV (both paths)
  thick      256 probes in batches of 32, 1024^2 frames cropped to the centred 256^2 ROI,
             T=8192 in 64-frame pushes, 1000 E over 0-150 meV, K_stage=2048 (four flushes,
             compensated FP32 accumulators), split BF16
  batched    16 partitions with uneven P, K^2, T, windows; 16-frame pushes interleaved
             round-robin; 300 E; split BF16, tiles picked by the autotuner, the final
             flushes of all partitions in one launch
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import oracle_kw, stream_config

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 1e-5, "split_inplace": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


def forward_kw(spec):
    kw = oracle_kw(spec)
    kw.pop("detectors")
    return kw


def sample_pixels(spec, n, rng):
    K = spec.Kx
    c = (spec.Ky // 2) * K + K // 2
    near = [c, c + 3, c - 5 * K + 2, c + 9 * K - 7]
    return np.concatenate([near, rng.integers(0, spec.Kx * spec.Ky, n - len(near))])


@pytest.mark.parametrize("precision", ["split_bf16", "fp32", "split_inplace"])
def test_realistic_full_size(precision):
    import torch
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan
    spec = synth.realistic().streams[0]
    P, K, T, Tc, Nw = spec.P, spec.Kx, spec.T, spec.Tc, spec.Nw
    npix = K * K
    fe = P * npix
    x = torch.empty(T * fe, dtype=torch.complex64, device="cuda")
    for t0 in range(0, T, 128):
        sg.generate(spec, 21, x.data_ptr() + t0 * fe * 8, t0, 128, pitch_row=K, pitch_frame=fe, pitch_probe=npix)
    I = torch.empty(P * Nw * npix, dtype=torch.float32, device="cuda")
    S = torch.empty(P * Nw, dtype=torch.float32, device="cuda")
    kw = dict(precision="split_bf16", frames_in_place=True) if precision == "split_inplace" else dict(
        precision=precision)
    with TacawPlan([stream_config(spec)], **kw) as plan:
        for i in range(T // Tc):
            plan.push(0, x.data_ptr() + i * Tc * fe * 8, Tc)
        plan.finalize(I, S)
    rng = np.random.default_rng(5)
    probes = rng.integers(0, P, 48)
    pix = sample_pixels(spec, 48, rng)
    xv = x.view(T, P, npix)
    ser = xv[:, torch.as_tensor(probes, device="cuda"), torch.as_tensor(pix, device="cuda")].cpu().numpy()
    got = I.view(P, Nw, npix)[torch.as_tensor(probes, device="cuda"), :, torch.as_tensor(pix, device="cuda")]
    got = got.cpu().numpy().T
    _, ref = oracle.forward_pixels(ser, **forward_kw(spec))
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print(f"realistic {precision}: sampled max rel I error {err:.3g}")
    assert err <= TOL[precision]
    # spectra of two probes from all aperture pixels
    ap = np.nonzero(oracle.detector_masks(K, K, spec.detectors)[0].reshape(-1))[0]
    for p in (0, P - 1):
        ser = xv[:, p, torch.as_tensor(ap, device="cuda")].cpu().numpy()
        _, Ip = oracle.forward_pixels(ser, **forward_kw(spec))
        ref = Ip.sum(axis=1)
        got = S.view(P, Nw)[p].cpu().numpy()
        e = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert e <= TOL[precision], (p, e)


@pytest.mark.parametrize("k_stage", [0, 2048], ids=["one_flush_per_batch", "four_flushes_kahan"])
def test_thick_probe_batches_crop_and_accumulators(k_stage):
    """Config 5: 1024^2 frames cropped to the centred 256^2 ROI while read, T = 8192 in 64-frame
    pushes, 1000 energies, 32-probe batches through one plan.  k_stage 0 is the bench's launch
    configuration (the default HBM budget holds the whole segment: one flush per batch, no
    accumulators; the first and the last batch are checked); 2048 forces four flushes per batch with
    compensated accumulators (all 8 batches)."""
    import torch
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan
    w = synth.thick()
    spec = w.streams[0]
    B = w.probe_batch
    K, T, Tc, Nw = spec.Kx, spec.T, spec.Tc, spec.Nw
    gx, gy = spec.full_grid
    rx, ry = spec.roi_origin
    npix = K * K
    fe = B * gx * gy                          # one full 1024^2 frame for each probe of a batch
    buf = torch.zeros(Tc * fe, dtype=torch.complex64, device="cuda")
    I = torch.empty(B * Nw * npix, dtype=torch.float32, device="cuda")
    S = torch.empty(B * Nw, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(9)
    worst = 0.0
    batches = list(range(0, spec.P, B)) if k_stage else [0, spec.P - B]
    with TacawPlan([stream_config(spec, P=B)], precision="split_bf16", k_stage=k_stage, accum="kahan") as plan:
        assert plan.info()["k_stage"] == (k_stage or T)
        for b0 in batches:
            plan.reset()
            pb = rng.integers(0, B, 6)
            px = sample_pixels(spec, 6, rng)
            rows = torch.as_tensor((pb * gx * gy + (ry + px // K) * gx + (rx + px % K)), device="cuda")
            ser = np.empty((T, len(pb)), dtype=np.complex64)
            for t0 in range(0, T, Tc):
                # the multislice grid is 1024^2; only the ROI is ever read, so only it is synthesised
                sg.generate(spec, 33, buf.data_ptr(), t0, Tc, pitch_row=gx, pitch_frame=fe, pitch_probe=gx * gy,
                            out_x0=rx, out_y0=ry, p0=b0, P=B)
                ser[t0:t0 + Tc] = buf.view(Tc, -1)[:, rows].cpu().numpy()
                plan.push(0, buf.data_ptr(), Tc)
            plan.finalize(I, S)
            got = I.view(B, Nw, npix)[torch.as_tensor(pb, device="cuda"), :, torch.as_tensor(px, device="cuda")]
            got = got.cpu().numpy().T
            _, ref = oracle.forward_pixels(ser, **forward_kw(spec))
            err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
            worst = max(worst, err)
        info = plan.info()
    print(f"thick (k_stage {k_stage}): sampled max rel I error {worst:.3g}, flushes {info['flushes']}")
    assert info["flushes"] == len(batches) * (T // (k_stage or T))
    assert worst <= TOL["split_bf16"]


def test_batched_uneven_partitions():
    import torch
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan
    w = synth.batched()
    specs = list(w.streams)
    bufs = [torch.empty(s.Tc * s.P * s.Kx * s.Ky, dtype=torch.complex64, device="cuda") for s in specs]
    rng = np.random.default_rng(13)
    samples = []
    for s in specs:
        pb = rng.integers(0, s.P, 4)
        px = sample_pixels(s, 4, rng)
        samples.append((pb, px, np.empty((s.T, 4), dtype=np.complex64)))
    with TacawPlan([stream_config(s) for s in specs], precision="split_bf16",
                   hbm_budget_bytes=200 * 2 ** 30, tune="") as plan:
        info = plan.info()
        assert info["tuned_streams"] == len(specs)
        print(f"batched: autotuner timed {info['tune_candidates']} candidates in {info['tune_ms']:.0f} ms")
        I = torch.empty(info["I_elems"], dtype=torch.float32, device="cuda")
        S = torch.empty(info["S_elems"], dtype=torch.float32, device="cuda")
        pushed = [0] * len(specs)
        while any(pushed[i] < s.T for i, s in enumerate(specs)):
            for i, s in enumerate(specs):
                if pushed[i] >= s.T:
                    continue
                n = min(s.Tc, s.T - pushed[i])
                npx = s.Kx * s.Ky
                sg.generate(s, 44, bufs[i].data_ptr(), pushed[i], n, pitch_row=s.Kx, pitch_frame=s.P * npx,
                            pitch_probe=npx)
                pb, px, ser = samples[i]
                rows = torch.as_tensor(pb * npx + px, device="cuda")
                ser[pushed[i]:pushed[i] + n] = bufs[i].view(s.Tc, -1)[:n, rows].cpu().numpy()
                plan.push(i, bufs[i], n)
                pushed[i] += n
        before = plan.info()
        plan.finalize(I, S)
        offs = [plan.offsets(i) for i in range(len(specs))]
        info = plan.info()
    # one contraction launch for all partitions (plus per-partition prologue/aperture kernels)
    tails = sum(1 for s in specs if s.T % info["tc_block_frames"])
    assert info["kernel_launches"] - before["kernel_launches"] == 2 * len(specs) + tails + 1
    worst = 0.0
    for i, s in enumerate(specs):
        pb, px, ser = samples[i]
        npx = s.Kx * s.Ky
        Ii = I[offs[i][0]:offs[i][0] + s.P * s.Nw * npx].view(s.P, s.Nw, npx)
        got = Ii[torch.as_tensor(pb, device="cuda"), :, torch.as_tensor(px, device="cuda")].cpu().numpy().T
        _, ref = oracle.forward_pixels(ser, **forward_kw(s))
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        worst = max(worst, err)
        assert err <= TOL["split_bf16"], (i, s.window, err)
    print(f"batched: k_stage {info['k_stage']}, flushes {info['flushes']}, worst sampled error {worst:.3g}")
