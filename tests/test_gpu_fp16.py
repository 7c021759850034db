"""Split-FP16 tensor-core path (fp16 hi/lo pieces of the scaled frames and of the twiddles)
against the FP64 oracle, through the C ABI.

The frames' residual psi - mu_hat is multiplied by the plan's fp16_scale (a power of two,
default 2^12) before the split and the epilogue undoes it exactly, so I, S and Psi compare
with the oracle at the split path's tolerance.  A scaled value beyond the fp16 range is
reported (TACAW_ERR_OVERFLOW) instead of producing infinities.
"""
import zlib

import numpy as np
import pytest

import oracle
import synth
from synth import Detector, StreamSpec, frames
from tests.helpers import oracle_kw, rel_err_peak, run_gpu, stream_config
from tests.test_gpu_parity import CASES, TOL_SPLIT, random_frames

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


def check(spec, fr, **kw):
    out = run_gpu(spec, fr, "split_fp16", **kw)
    ref = oracle.forward(fr, **oracle_kw(spec))
    eI = rel_err_peak(out["I"], ref.I)
    assert eI <= TOL_SPLIT, f"I error {eI:.3g}"
    if len(spec.detectors):
        eS = rel_err_peak(out["S"], ref.S)
        assert eS <= TOL_SPLIT, f"S error {eS:.3g}"
    if kw.get("want_psi"):
        eP = rel_err_peak(out["Psi"], ref.Psi)
        assert eP <= TOL_SPLIT, f"Psi error {eP:.3g}"
    assert out["info"]["precision"] == 2
    return out, ref, eI


def test_tiny_config_whole_fp16_vs_bf16():
    """Tiny workload: I, S and Psi (the epilogue's unscaling) within tolerance; the error of
    the fp16 pieces is reported beside the bf16 one on the same frames."""
    s = synth.tiny().streams[0]
    fr = frames.frames(s, 0, 0, s.T)
    out, ref, e16 = check(s, fr, want_psi=True)
    e_bf = rel_err_peak(run_gpu(s, fr, "split_bf16")["I"], ref.I)
    print(f"tiny: max rel I error fp16 {e16:.3g}, bf16 {e_bf:.3g}")


@pytest.mark.parametrize("name", sorted(CASES))
def test_edge_cases_fp16(name):
    spec, pushes, k_stage = CASES[name]
    fr = random_frames(spec.P, spec.T, spec.Ky, spec.Kx, seed=zlib.crc32(name.encode()) % 1000)
    out, ref, e = check(spec, fr, pushes=pushes, k_stage=k_stage)
    if k_stage:
        assert out["info"]["flushes"] > 1


@pytest.mark.parametrize("accum", ["kahan", "fp64", "fp32"])
def test_streaming_flushes_fp16(accum):
    """K_stage < T: the cross-flush accumulators hold scaled sums; the last flush unscales."""
    spec = StreamSpec(P=2, Kx=32, Ky=16, T=200, Tc=24, n_omega=70, E_max_meV=120.0, window="hann",
                      n_modes=6, detectors=(Detector("circular", 0, 0, -1, 5.0),))
    fr = frames.frames(spec, 3, 0, spec.T)
    out, ref, e = check(spec, fr, k_stage=48, accum=accum, want_psi=True)
    assert out["info"]["flushes"] == 5


@pytest.mark.parametrize("kw", [dict(tc_block_frames=32),
                                dict(tc_omega_tile=112, tc_block_frames=16),
                                dict(tc_drain_frames=64, tc_block_frames=16),
                                dict(tc_drain_frames=32, tc_block_frames=8)],
                         ids=["bf32", "wide_bf16", "drain64_bf16", "drain32_bf8"])
def test_tilings_fp16(kw):
    """The staged tensor-core kernel takes the fp16 operand type (instruction descriptor) at every
    staging row width and drain length."""
    spec = StreamSpec(P=3, Kx=36, Ky=36, T=168, Tc=40, n_omega=150, E_max_meV=120.0, window="hann", n_modes=6,
                      noise=1e-3, detectors=(Detector("circular", 0, 0, -1, 6.0),))
    fr = frames.frames(spec, 11, 0, spec.T)
    check(spec, fr, **kw)


def test_fp16_range_is_checked_and_scale_is_honoured():
    """Frames whose residual is ~100: at the default scale 2^12 the scaled values leave the
    fp16 range and finalize reports OVERFLOW; at 2^4 the same frames match the oracle."""
    from paper_2607_02236_gb300 import TacawError
    from paper_2607_02236_gb300.tacaw import ERR_OVERFLOW
    spec = StreamSpec(P=2, Kx=16, Ky=16, T=64, Tc=32, n_omega=30, E_max_meV=120.0, window="hann",
                      detectors=(Detector("circular", 0, 0, -1, 4.0),))
    fr = random_frames(2, 64, 16, 16, seed=77, elastic=300.0, signal=100.0)
    with pytest.raises(TacawError) as ei:
        run_gpu(spec, fr, "split_fp16")
    assert ei.value.status == ERR_OVERFLOW
    check(spec, fr, fp16_scale=16.0, want_psi=True)


@pytest.mark.parametrize("N,stride,skip", [(5, 32, 0), (3, 20, 45)])
def test_welch_and_skip_init_fp16(N, stride, skip):
    """Welch lanes (each segment's mean residual at the operand scale, its last flush adding
    (1/N) 2^-2e B |Psi|^2 into the average) and skipped leading frames on fp16 pieces."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    from tests.test_gpu_welch import SPEC as WSPEC, make_frames, welch_config
    s = WSPEC
    n = skip + (N - 1) * stride + s.T
    fr = make_frames(s.P, n, s.Ky, s.Kx, seed=50 + N)
    buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).to("cuda")
    fb = s.P * s.Kx * s.Ky * 8
    with TacawPlan([welch_config(s, N, stride, skip)], precision="split_fp16") as plan:
        info = plan.info()
        I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
        S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
        for t0 in range(0, n, 40):
            plan.push(0, buf.data_ptr() + t0 * fb, min(40, n - t0))
        plan.finalize(I, S)
    ref = oracle.welch_forward(fr, s.T, stride, skip_init=skip, **oracle_kw(s))
    got = I.cpu().numpy().reshape(s.P, s.Nw, s.Ky, s.Kx)
    assert rel_err_peak(got, ref.I) <= TOL_SPLIT
    assert rel_err_peak(S.cpu().numpy().reshape(s.P, 1, s.Nw), ref.S) <= TOL_SPLIT


def test_grouped_launch_and_graph_replay_fp16():
    """Uneven partitions in one plan: the last flushes of all streams in one grouped launch of
    fp16 operands, then the whole segment captured into a CUDA graph and replayed over new
    frames, each time against the oracle."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    from tests.test_gpu_graph_batched import SPECS, check_all, device_frames, make_frames, push_all
    frames_ = [make_frames(s, 500 + i) for i, s in enumerate(SPECS)]
    bufs = [device_frames(f) for f in frames_]
    st = torch.cuda.Stream()
    with TacawPlan([stream_config(s) for s in SPECS], precision="split_fp16") as plan:
        info = plan.info()
        I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
        S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
        with torch.cuda.stream(st):
            plan.reset(st)
            push_all(plan, bufs, st)
            plan.finalize_async(I, S, cuda_stream=st)
            plan.check_errors(st)
        check_all(plan, I, S, frames_, TOL_SPLIT)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            cur = torch.cuda.current_stream()
            plan.reset(cur)
            push_all(plan, bufs, cur)
            plan.finalize_async(I, S, cuda_stream=cur)
        frames_ = [make_frames(s, 600 + i) for i, s in enumerate(SPECS)]
        for b, f in zip(bufs, frames_):
            b.copy_(device_frames(f))
        I.zero_()
        S.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        plan.check_errors(torch.cuda.current_stream())
        check_all(plan, I, S, frames_, TOL_SPLIT)
        del g
