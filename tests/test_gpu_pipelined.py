"""Pipelined segments: each segment's contraction is deferred and launched with the conversion of
the next segment's pushes (done by extra warps of the same launch).  Over several segments the
results are the same, bit for bit, as those of a plan that converts at push time and contracts at
finalize, and match the FP64 oracle; the refusals leave the plan usable."""
import numpy as np
import pytest

import oracle
from synth import Detector, StreamSpec, frames
from tests.helpers import oracle_kw, rel_err_peak, stream_config

pytestmark = pytest.mark.gpu

# 3 probes x 40 x 36 ROI pixels (ragged row tiles) cropped at (6, 5) from a 52 x 46 grid, T = 128
# in 32-frame pushes
SPEC = StreamSpec(P=3, Kx=40, Ky=36, T=128, Tc=32, n_omega=90, E_max_meV=120.0, window="hann", n_modes=6,
                  noise=1e-3, Gx=52, Gy=46, detectors=(Detector("circular", 0, 0, -1, 7.0),
                                                       Detector("annular", 1.0, -2.0, 3.0, 9.0)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


def full_frames(spec, fr):
    """[P, T, Ky, Kx] ROI frames -> [T, P, Gy, Gx] full frames (zero outside the ROI)."""
    gx, gy = spec.full_grid
    rx, ry = spec.roi_origin
    P, T = fr.shape[:2]
    out = np.zeros((T, P, gy, gx), dtype=np.complex64)
    out[:, :, ry:ry + spec.Ky, rx:rx + spec.Kx] = fr.transpose(1, 0, 2, 3)
    return out


def run_segments(spec, bufs, pipelined, want_psi=False, sync_last=False):
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    gx, gy = spec.full_grid
    fb = spec.P * gx * gy * 8
    n_el = spec.P * spec.Nw * spec.Ky * spec.Kx
    outs = [(torch.full((n_el,), -1.0, device="cuda"), torch.full((spec.P * 2 * spec.Nw,), -1.0, device="cuda"),
             torch.zeros(n_el, dtype=torch.complex64, device="cuda") if want_psi else None) for _ in bufs]
    st = torch.cuda.current_stream()
    with TacawPlan([stream_config(spec)], precision="split_bf16") as plan:
        if pipelined:
            plan.set_pipelined_segments(True)
        for k, buf in enumerate(bufs):
            plan.reset(st)
            for t in range(0, spec.T, spec.Tc):
                plan.push(0, buf.data_ptr() + t * fb, spec.Tc, st)
            I, S, Psi = outs[k]
            if sync_last and k == len(bufs) - 1:
                plan.finalize(I, S, Psi, st)
            else:
                plan.finalize_async(I, S, Psi, st)
        if pipelined and not sync_last:
            plan.drain(st)
        plan.check_errors(st)
        launches = plan.info()["flush_launches"]
    torch.cuda.synchronize()
    res = [(I.cpu().numpy().reshape(spec.P, spec.Nw, spec.Ky, spec.Kx), S.cpu().numpy().reshape(spec.P, 2, spec.Nw),
            Psi.cpu().numpy().reshape(spec.P, spec.Nw, spec.Ky, spec.Kx) if Psi is not None else None)
           for I, S, Psi in outs]
    return res, launches


@pytest.mark.parametrize("subtract_mean", [True, False])
@pytest.mark.parametrize("sync_last", [False, True], ids=["drain", "finalize"])
def test_pipelined_segments_match_unpipelined_and_oracle(subtract_mean, sync_last):
    import dataclasses
    import torch
    spec = dataclasses.replace(SPEC, subtract_mean=subtract_mean)
    roi = [frames.frames(spec, 60 + k, 0, spec.T) for k in range(4)]        # four segments
    bufs = [torch.from_numpy(full_frames(spec, fr)).cuda() for fr in roi]
    want_psi = not subtract_mean
    ref_gpu, n_plain = run_segments(spec, bufs, False, want_psi)
    got, n_pipe = run_segments(spec, bufs, True, want_psi, sync_last)
    assert n_plain == n_pipe == 4                                           # one contraction a segment
    for k, fr in enumerate(roi):
        I, S, Psi = got[k]
        I0, S0, Psi0 = ref_gpu[k]
        assert np.array_equal(I, I0) and np.array_equal(S, S0), k
        if want_psi:
            assert np.array_equal(Psi, Psi0)
        ref = oracle.forward(fr, **oracle_kw(spec))
        assert rel_err_peak(I, ref.I) <= 1e-5, k
        assert rel_err_peak(S, ref.S) <= 1e-5, k


def test_pipelined_segments_refusals():
    import torch
    from paper_2607_02236_gb300 import TacawError, TacawPlan
    from paper_2607_02236_gb300.tacaw import ERR_STATE, ERR_UNSUPPORTED
    other = StreamSpec(P=1, Kx=16, Ky=16, T=64, Tc=32, n_omega=20)
    cases = [([stream_config(SPEC), stream_config(other)], dict(precision="split_bf16")),   # two streams
             ([stream_config(SPEC)], dict(precision="fp32")),
             ([stream_config(SPEC)], dict(precision="split_fp16")),
             ([stream_config(SPEC)], dict(precision="split_bf16", tc_block_frames=16)),
             ([stream_config(SPEC)], dict(precision="split_bf16", k_stage=64))]              # two flushes
    for streams, kw in cases:
        with TacawPlan(streams, **kw) as plan:
            with pytest.raises(TacawError) as ei:
                plan.set_pipelined_segments(True)
            assert ei.value.status == ERR_UNSUPPORTED, kw
    gx, gy = SPEC.full_grid
    buf = torch.zeros(SPEC.T * SPEC.P * gx * gy, dtype=torch.complex64, device="cuda")
    fb = SPEC.P * gx * gy * 8
    I = torch.empty(SPEC.P * SPEC.Nw * SPEC.Ky * SPEC.Kx, device="cuda")
    with TacawPlan([stream_config(SPEC)], precision="split_bf16") as plan:
        plan.push(0, buf.data_ptr(), 32)
        with pytest.raises(TacawError) as ei:                       # mid-segment
            plan.set_pipelined_segments(True)
        assert ei.value.status == ERR_STATE
        plan.reset()
        plan.set_pipelined_segments(True)
        for t in range(0, SPEC.T, 32):
            plan.push(0, buf.data_ptr() + t * fb, 32)
        plan.finalize_async(I)                                     # deferred
        with pytest.raises(TacawError) as ei:                       # disabling with a deferred contraction
            plan.set_pipelined_segments(False)
        assert ei.value.status == ERR_STATE
        plan.reset()
        plan.push(0, buf.data_ptr(), 32)                           # recorded for the deferred launch
        with pytest.raises(TacawError) as ei:
            plan.drain()
        assert ei.value.status == ERR_STATE
        for t in range(32, SPEC.T, 32):
            plan.push(0, buf.data_ptr() + t * fb, 32)
        plan.finalize(I)                                           # launches both, waits
        plan.set_pipelined_segments(False)
    torch.cuda.synchronize()
    assert float(I.abs().max()) == 0.0                             # zero frames: zero spectrum


def test_pipelined_from_pinned_host_memory():
    """Pushes from pinned host memory: the conversion warps read the frames over the host link
    through the recorded addresses; bit-identical to the unpipelined plan on the same frames."""
    import torch
    roi = [frames.frames(SPEC, 70 + k, 0, SPEC.T) for k in range(3)]
    bufs = [torch.from_numpy(full_frames(SPEC, fr)).pin_memory() for fr in roi]
    ref_gpu, _ = run_segments(SPEC, bufs, False)
    got, _ = run_segments(SPEC, bufs, True)
    for k, fr in enumerate(roi):
        assert np.array_equal(got[k][0], ref_gpu[k][0]) and np.array_equal(got[k][1], ref_gpu[k][1]), k
        assert rel_err_peak(got[k][0], oracle.forward(fr, **oracle_kw(SPEC)).I) <= 1e-5


def test_pipelined_segments_in_a_cuda_graph():
    """Two pipelined segments and the drain captured into one CUDA graph and replayed with new frame
    contents in the same buffers: each replay bit-identical to an unpipelined plan, and the
    replays launch nothing through the library."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    gx, gy = SPEC.full_grid
    fb = SPEC.P * gx * gy * 8
    n_el = SPEC.P * SPEC.Nw * SPEC.Ky * SPEC.Kx
    bufs = [torch.zeros(SPEC.T * SPEC.P * gy * gx, dtype=torch.complex64, device="cuda") for _ in range(2)]
    Is = [torch.zeros(n_el, device="cuda") for _ in range(2)]
    Ss = [torch.zeros(SPEC.P * 2 * SPEC.Nw, device="cuda") for _ in range(2)]
    st = torch.cuda.Stream()

    def segments(plan, stream):
        for k in range(2):
            plan.reset(stream)
            for t in range(0, SPEC.T, SPEC.Tc):
                plan.push(0, bufs[k].data_ptr() + t * fb, SPEC.Tc, stream)
            plan.finalize_async(Is[k], Ss[k], None, stream)
        plan.drain(stream)

    with TacawPlan([stream_config(SPEC)], precision="split_bf16") as plan:
        plan.set_pipelined_segments(True)
        with torch.cuda.stream(st):                  # eager first (kernel attributes set outside capture)
            segments(plan, st)
            plan.check_errors(st)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            segments(plan, torch.cuda.current_stream())
        launches = plan.info()["kernel_launches"]
        for seed in (80, 90):
            roi = [frames.frames(SPEC, seed + k, 0, SPEC.T) for k in range(2)]
            for b, fr in zip(bufs, roi):
                b.copy_(torch.from_numpy(full_frames(SPEC, fr)).view(-1))
            for x in Is + Ss:
                x.fill_(-1.0)
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            plan.check_errors(torch.cuda.current_stream())
            ref_gpu, _ = run_segments(SPEC, [b.view(SPEC.T, SPEC.P, gy, gx) for b in bufs], False)
            for k in range(2):
                I = Is[k].cpu().numpy().reshape(SPEC.P, SPEC.Nw, SPEC.Ky, SPEC.Kx)
                S = Ss[k].cpu().numpy().reshape(SPEC.P, 2, SPEC.Nw)
                assert np.array_equal(I, ref_gpu[k][0]) and np.array_equal(S, ref_gpu[k][1]), (seed, k)
                assert rel_err_peak(I, oracle.forward(roi[k], **oracle_kw(SPEC)).I) <= 1e-5
        assert plan.info()["kernel_launches"] == launches
        del g


def test_pipelined_segments_at_the_thick_shape():
    """The headline's shape: 1024^2 frames cropped to the centred 256^2 ROI while read, T = 8192 in
    64-frame pushes, 1000 energies, read from a resident ring of two pushes of full frames (as the
    bench cycles it); two one-probe segments pipelined against an unpipelined plan (1e-6 of the
    peak: with 64-frame pushes the two paths add the per-block FP32 sums in another FP64 order) and
    against the FP64 oracle at sampled (probe, pixel) series (1e-5)."""
    import torch
    import synth
    import synth.gpu as sg
    from paper_2607_02236_gb300 import TacawPlan
    spec = synth.thick().streams[0]
    K, T, Tc, Nw = spec.Kx, spec.T, spec.Tc, spec.Nw
    gx, gy = spec.full_grid
    rx, ry = spec.roi_origin
    npix = K * K
    B, R = 2, 2                                   # probes in the ring, pushes in the ring
    fe = B * gx * gy
    ring = torch.zeros(R * Tc * fe, dtype=torch.complex64, device="cuda")
    for r in range(R):
        sg.generate(spec, 41, ring.data_ptr() + r * Tc * fe * 8, r * Tc, Tc, pitch_row=gx, pitch_frame=fe,
                    pitch_probe=gx * gy, out_x0=rx, out_y0=ry, p0=0, P=B)
    cfg = stream_config(spec, P=1)
    cfg.pitch_frame = fe
    st = torch.cuda.current_stream()

    def run(pipelined):
        Is = [torch.full((Nw * npix,), -1.0, device="cuda") for _ in range(B)]
        with TacawPlan([cfg], precision="split_bf16") as plan:
            if pipelined:
                plan.set_pipelined_segments(True)
            for h in range(B):
                plan.reset(st)
                for i in range(T // Tc):
                    plan.push(0, ring.data_ptr() + h * gx * gy * 8 + (i % R) * Tc * fe * 8, Tc, st)
                plan.finalize_async(Is[h], None, None, st)
            if pipelined:
                plan.drain(st)
            plan.check_errors(st)
        torch.cuda.synchronize()
        return [I.view(Nw, npix) for I in Is]

    plain, pipe = run(False), run(True)
    rng = np.random.default_rng(17)
    kw = oracle_kw(spec)
    kw.pop("detectors")
    for h in range(B):
        peak = float(plain[h].abs().max())
        assert float((pipe[h] - plain[h]).abs().max()) <= 1e-6 * peak, h
        px = np.concatenate([[(K // 2) * K + K // 2], rng.integers(0, npix, 7)])
        rows = torch.as_tensor(h * gx * gy + (ry + px // K) * gx + (rx + px % K), device="cuda")
        cyc = ring.view(R * Tc, fe)[:, rows].cpu().numpy()
        series = cyc[np.arange(T) % (R * Tc)]
        _, ref = oracle.forward_pixels(series, **kw)
        got = pipe[h][:, torch.as_tensor(px, device="cuda")].cpu().numpy()
        assert rel_err_peak(got, ref) <= 1e-5, h
    del ring
