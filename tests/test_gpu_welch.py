"""Welch averaging (Sec. II.B): N overlapping segments of L frames, each with its own mean,
window and phase origin, averaged as I = (1/N) sum_n I_n -- against the FP64 oracle element
by element.  Pushes cross segment boundaries; several segments are open at once (lanes)."""
import numpy as np
import pytest

import oracle
from synth import Detector, StreamSpec
from tests.helpers import oracle_kw, rel_err_peak, stream_config

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


def make_frames(P, n, Ky, Kx, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((P, 1, Ky, Kx)) + 1j * rng.standard_normal((P, 1, Ky, Kx))
    t = np.arange(n)[None, :, None, None]
    tone = 0.05 * np.exp(2j * np.pi * 0.0731 * t) * rng.standard_normal((P, 1, Ky, Kx))
    s = 1e-2 * (rng.standard_normal((P, n, Ky, Kx)) + 1j * rng.standard_normal((P, n, Ky, Kx)))
    return (e + tone + s).astype(np.complex64)


def welch_config(spec, N, stride, skip=0):
    c = stream_config(spec)
    c.welch_segments, c.welch_stride, c.skip_init = N, stride, skip
    return c


def run(specs_ws, frames, push, precision="split_bf16", **plan_kw):
    """specs_ws: [(spec, N, stride)], frames: [array [P, n, Ky, Kx]]. Returns I, S per stream."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    bufs = [torch.from_numpy(np.ascontiguousarray(f.transpose(1, 0, 2, 3))).to("cuda") for f in frames]
    with TacawPlan([welch_config(s, N, st) for s, N, st in specs_ws], precision=precision, **plan_kw) as plan:
        info = plan.info()
        I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
        S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
        pushed = [0] * len(frames)
        total = [f.shape[1] for f in frames]
        while any(pushed[i] < total[i] for i in range(len(frames))):
            for i, (s, _, _) in enumerate(specs_ws):
                if pushed[i] < total[i]:
                    n = min(push, total[i] - pushed[i])
                    fb = s.P * s.Kx * s.Ky * 8
                    plan.push(i, bufs[i].data_ptr() + pushed[i] * fb, n)
                    pushed[i] += n
        plan.finalize(I, S)
        out = []
        for i, (s, _, _) in enumerate(specs_ws):
            io, so = plan.offsets(i)
            D = len(s.detectors)
            out.append((I[io:io + s.P * s.Nw * s.Ky * s.Kx].cpu().numpy().reshape(s.P, s.Nw, s.Ky, s.Kx),
                        S[so:so + s.P * D * s.Nw].cpu().numpy().reshape(s.P, D, s.Nw)))
        return out, plan.info()


def check(spec, N, stride, push, precision="split_bf16", seed=0, **plan_kw):
    n = (N - 1) * stride + spec.T
    fr = make_frames(spec.P, n, spec.Ky, spec.Kx, seed)
    (I, S), = run([(spec, N, stride)], [fr], push, precision, **plan_kw)[0]
    ref = oracle.welch_forward(fr, spec.T, stride, **oracle_kw(spec))
    tol = TOL[precision]
    eI = rel_err_peak(I, ref.I)
    assert eI <= tol, f"I error {eI:.3g}"
    if len(spec.detectors):
        eS = rel_err_peak(S, ref.S)
        assert eS <= tol, f"S error {eS:.3g}"
    return eI


SPEC = StreamSpec(P=2, Kx=24, Ky=20, T=64, Tc=40, n_omega=40, E_max_meV=120.0, window="hann",
                  detectors=(Detector("circular", 0, 0, -1, 6.0),))


@pytest.mark.parametrize("precision,kw", [("fp32", {}), ("split_bf16", {}), ("split_bf16", {"tc_drain_frames": 64}),
                                          ("split_bf16", {"frames_in_place": True}),
                                          ("split_bf16", {"k_stage": 32})])
def test_welch_half_overlap(precision, kw):
    """nu = 2: L = 64, stride 32, 5 segments (192 frames) pushed 40 at a time."""
    e = check(SPEC, 5, 32, 40, precision, **kw)
    print(f"welch nu=2 {precision} {kw}: {e:.3g}")


@pytest.mark.parametrize("N,stride,push", [(6, 16, 7), (3, 64, 50), (4, 21, 64), (1, 0, 64)])
def test_welch_strides_and_pushes(N, stride, push):
    """Stride not dividing L (four lanes), no overlap (one lane), nu = 3, one segment."""
    spec = StreamSpec(P=1, Kx=16, Ky=16, T=64, Tc=16, fft_bins=32, window="hann", detectors=())
    check(spec, N, stride or spec.T, push)


def test_welch_stream_beside_a_plain_stream():
    """A Welch-averaged stream and a single-segment stream in one plan (its last flush grouped)."""
    a = SPEC
    b = StreamSpec(P=3, Kx=16, Ky=16, T=96, Tc=32, n_omega=24, E_max_meV=90.0, window="gauss",
                   detectors=(Detector("circular", 0, 0, -1, 4.0),))
    fa = make_frames(a.P, 4 * 20 + a.T, a.Ky, a.Kx, 3)
    fb = make_frames(b.P, b.T, b.Ky, b.Kx, 4)
    outs, info = run([(a, 5, 20), (b, 1, 0)], [fa, fb], 24)
    ra = oracle.welch_forward(fa, a.T, 20, **oracle_kw(a))
    rb = oracle.forward(fb, **oracle_kw(b))
    assert rel_err_peak(outs[0][0], ra.I) <= TOL["split_bf16"]
    assert rel_err_peak(outs[0][1], ra.S) <= TOL["split_bf16"]
    assert rel_err_peak(outs[1][0], rb.I) <= TOL["split_bf16"]
    assert rel_err_peak(outs[1][1], rb.S) <= TOL["split_bf16"]
    assert info["n_streams"] == 2


@pytest.mark.parametrize("N,stride,skip,push,kw", [(4, 32, 45, 40, {}), (1, 0, 70, 33, {}), (3, 20, 96, 96, {}),
                                                    (4, 32, 45, 40, {"frames_in_place": True}),
                                                    (1, 0, 64, 32, {"frames_in_place": True})])
def test_skip_init(N, stride, skip, push, kw):
    """Leading frames dropped before the first segment (one segment or Welch; pushes that end
    inside, at and after the skipped part; in place)."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    spec = SPEC
    n = skip + (N - 1) * (stride or spec.T) + spec.T
    fr = make_frames(spec.P, n, spec.Ky, spec.Kx, 9)
    fr[:, :skip] += 30.0                                            # a transient that must not leak in
    buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).to("cuda")
    with TacawPlan([welch_config(spec, N, stride, skip)], precision="split_bf16", **kw) as plan:
        I = torch.zeros(plan.info()["I_elems"], device="cuda")
        S = torch.zeros(max(1, plan.info()["S_elems"]), device="cuda")
        fb = spec.P * spec.Kx * spec.Ky * 8
        t = 0
        while t < n:
            k = min(push, n - t)
            plan.push(0, buf.data_ptr() + t * fb, k)
            t += k
        plan.finalize(I, S)
    ref = oracle.welch_forward(fr, spec.T, stride or spec.T, skip_init=skip, **oracle_kw(spec))
    got = I.cpu().numpy().reshape(ref.I.shape)
    assert rel_err_peak(got, ref.I) <= TOL["split_bf16"]
    assert rel_err_peak(S.cpu().numpy()[:ref.S.size].reshape(ref.S.shape), ref.S) <= TOL["split_bf16"]


def test_welch_errors():
    import torch
    from paper_2607_02236_gb300 import TacawPlan, TacawError
    n = 4 * 32 + SPEC.T
    buf = torch.zeros(n * SPEC.P * SPEC.Kx * SPEC.Ky, dtype=torch.complex64, device="cuda")
    with TacawPlan([welch_config(SPEC, 5, 32)]) as plan:
        with pytest.raises(TacawError, match="OVERFLOW"):
            plan.push(0, buf, n + 1)
        plan.push(0, buf, n)
        I = torch.zeros(plan.info()["I_elems"], device="cuda")
        Psi = torch.zeros(plan.info()["I_elems"], dtype=torch.complex64, device="cuda")
        with pytest.raises(TacawError, match="INVALID_ARG"):
            plan.finalize(I, None, Psi)
        plan.finalize(I)


@pytest.mark.parametrize("adjoint", ["split_bf16", "fp32"])
@pytest.mark.parametrize("N,stride,skip", [(4, 24, 10), (3, 64, 0), (1, 0, 17)])
def test_welch_gradient_through_autograd(N, stride, skip, adjoint):
    """The adjoint of the averaged spectrum (segments weighted 1/N, overlaps summed, skipped
    frames zero) through torch.autograd, against the FP64 oracle's Welch gradient."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    from paper_2607_02236_gb300.autograd import spectrum
    spec = StreamSpec(P=2, Kx=16, Ky=12, T=64, Tc=32, n_omega=24, E_max_meV=120.0, window="hann",
                      detectors=(Detector("circular", 0, 0, -1, 3.5), Detector("annular", 1.0, 0.0, 2.0, 5.0)))
    n = skip + (N - 1) * (stride or spec.T) + spec.T
    fr = make_frames(spec.P, n, spec.Ky, spec.Kx, 21)
    rng = np.random.default_rng(5)
    c = rng.standard_normal((spec.P, len(spec.detectors), spec.Nw))
    x = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).to("cuda").requires_grad_(True)
    with TacawPlan([welch_config(spec, N, stride, skip)], precision="fp32") as plan:
        plan.set_adjoint_precision(adjoint)
        S = spectrum(x, plan, 0, 20)
        L = (S * torch.tensor(c, dtype=torch.float32, device="cuda")).sum()
        L.backward()
        torch.cuda.synchronize()
    g = x.grad.cpu().numpy().transpose(1, 0, 2, 3)               # [P, n, Ky, Kx]
    ref = oracle.welch_gradient(fr, c, spec.T, stride or spec.T, skip_init=skip, **oracle_kw(spec))
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel <= 1e-4, rel
    assert np.all(g[:, :skip] == 0)
    refS = oracle.welch_forward(fr, spec.T, stride or spec.T, skip_init=skip, **oracle_kw(spec)).S
    assert rel_err_peak(S.detach().cpu().numpy(), refS) <= TOL["fp32"]
