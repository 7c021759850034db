"""Differentiation workload: 8 probes, 128x128 ROI, T=512, 200 energies over 0-120 meV, Hann,
FP32.  L = sum_p sum_E c(E) S_p(E) with S the r=20 px aperture spectrum and c ~ N(0,1) seeded.

The adjoint (tacaw_backward behind torch.autograd), on the tensor cores (split BF16, the default)
and on the FP32 CUDA cores, is checked against the FP64 oracle gradient (relative L2 <= 1e-4 on
sampled aperture pixels, exact zeros outside the aperture) and against FP64 central finite
differences (h = 1e-6) of the oracle loss on 64 random entries; ragged sizes (row tiles, frames
and energies that fill no whole block) against the oracle's full gradient.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import frames as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["split_bf16", "fp32"])
def case(request):
    import torch
    from paper_2607_02236_gb300 import TacawPlan, build
    from paper_2607_02236_gb300.autograd import spectrum
    from tests.helpers import stream_config
    import synth.gpu as sg
    build.build_all()
    spec = synth.diff().streams[0]
    P, K, T, Nw = spec.P, spec.Kx, spec.T, spec.Nw
    x = torch.empty(T * P * K * K, dtype=torch.complex64, device="cuda")
    sg.generate(spec, 4, x.data_ptr(), 0, T, pitch_row=K, pitch_frame=P * K * K, pitch_probe=K * K)
    x = x.view(T, P, K, K).requires_grad_(True)
    plan = TacawPlan([stream_config(spec)], precision="fp32")
    plan.set_adjoint_precision(request.param)
    c = torch.tensor(synth.loss_weights(Nw, seed=0), dtype=torch.float32, device="cuda")
    S = spectrum(x, plan)
    L = (S * c[None, None, :]).sum()
    L.backward()
    torch.cuda.synchronize()
    xh = x.detach().cpu().numpy()                  # [T, P, K, K]
    g = x.grad.cpu().numpy()
    out = dict(spec=spec, x=xh, g=g, S=S.detach().cpu().numpy(), c=c.cpu().numpy().astype(np.float64))
    plan.close()
    return out


def aperture(spec):
    M = oracle.detector_masks(spec.Kx, spec.Ky, spec.detectors)[0].reshape(-1)
    return np.nonzero(M)[0]


def kw(spec):
    return dict(window_kind=spec.window, E_meV=spec.energies_meV(), dt_fs=spec.dt_fs,
                subtract_mean=spec.subtract_mean)


def test_forward_spectrum_matches_oracle(case):
    spec, x = case["spec"], case["x"]
    ap = aperture(spec)
    T = spec.T
    for p in range(spec.P):
        series = x[:, p].reshape(T, -1)[:, ap]
        _, I = oracle.forward_pixels(series, **kw(spec))
        ref = I.sum(axis=1)
        err = np.max(np.abs(case["S"][p, 0] - ref)) / np.max(np.abs(ref))
        assert err <= 1e-5, (p, err)


def test_gradient_matches_oracle_gradient(case):
    spec, x, g = case["spec"], case["x"], case["g"]
    T, K = spec.T, spec.Kx
    ap = aperture(spec)
    rng = np.random.default_rng(1)
    dLdS = case["c"][None, :]
    for p in range(spec.P):
        sel = rng.choice(ap, 16, replace=False)
        series = x[:, p].reshape(T, -1)[:, sel]
        ref = oracle.gradient_pixels(series, dLdS, np.ones((len(sel), 1)), **kw(spec))
        got = g[:, p].reshape(T, -1)[:, sel]
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 1e-4, (p, rel)
    # outside every aperture the gradient is exactly zero
    out = np.setdiff1d(np.arange(K * K), ap)
    assert np.all(g[:, :, :, :].reshape(T, spec.P, -1)[:, :, out] == 0)


def test_gradient_matches_fp64_finite_differences(case):
    spec, x, g = case["spec"], case["x"], case["g"]
    T = spec.T
    ap = aperture(spec)
    rng = np.random.default_rng(2)
    dLdS = case["c"][None, :]
    h = 1e-6
    scale = 0.0
    rows = []
    for _ in range(64):
        p = int(rng.integers(0, spec.P))
        k = int(rng.choice(ap))
        t = int(rng.integers(0, T))
        series = x[:, p].reshape(T, -1)[:, [k]].astype(np.complex128)
        for unit, part in ((1.0, "re"), (1j, "im")):
            a = series.copy()
            b = series.copy()
            a[t, 0] += h * unit
            b[t, 0] -= h * unit
            fd = (oracle.loss_pixels(a, dLdS, [[1.0]], **kw(spec)) -
                  oracle.loss_pixels(b, dLdS, [[1.0]], **kw(spec))) / (2 * h)
            gv = g[t, p].reshape(-1)[k]
            an = gv.real if part == "re" else gv.imag
            rows.append((fd, an))
            scale = max(scale, abs(fd))
    for fd, an in rows:
        assert abs(fd - an) <= 1e-4 * scale, (fd, an, scale)


def ragged_frames(P, T, Ky, Kx, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((P, 1, Ky, Kx)) + 1j * rng.standard_normal((P, 1, Ky, Kx))
    t = np.arange(T)[None, :, None, None]
    tone = 0.05 * np.exp(2j * np.pi * 0.0731 * t) * rng.standard_normal((P, 1, Ky, Kx))
    s = 1e-2 * (rng.standard_normal((P, T, Ky, Kx)) + 1j * rng.standard_normal((P, T, Ky, Kx)))
    return (e + tone + s).astype(np.complex64)


@pytest.mark.parametrize("adjoint", ["split_bf16", "fp32"])
@pytest.mark.parametrize("mean,window,bose_T_K", [(True, "gauss", 300.0), (False, "hann", 0.0)])
def test_adjoint_ragged_sizes(adjoint, mean, window, bose_T_K):
    """3 probes x 182 aperture pixels (row tiles of 128 with a ragged tail), T = 50 frames and
    37 signed off-grid energies (neither fills whole 32-wide staging blocks), a centred disk and
    an off-axis annulus, the mean removed or kept, Bose factor on or off: the whole gradient
    against the FP64 oracle's, and exactly zero outside the apertures."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan, build
    from synth import Detector, StreamSpec
    from tests.helpers import oracle_kw, stream_config
    build.build_all()
    spec = StreamSpec(P=3, Kx=20, Ky=20, T=50, Tc=50, n_omega=37, window=window, subtract_mean=mean,
                      bose_T_K=bose_T_K,
                      detectors=(Detector("circular", 0, 0, -1, 7.5), Detector("annular", 2.0, -1.0, 3.0, 6.0)))
    E = np.linspace(-40.0, 60.0, 37) + 0.137
    fr = ragged_frames(spec.P, spec.T, spec.Ky, spec.Kx, 8)
    rng = np.random.default_rng(9)
    c = rng.standard_normal((spec.P, 2, 37))
    cfg = stream_config(spec)
    cfg.E_meV = [float(e) for e in E]
    buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).to("cuda")   # [T][P][Ky][Kx]
    grad = torch.full_like(buf, complex(7.0, -7.0))
    with TacawPlan([cfg], precision="fp32") as plan:
        plan.set_adjoint_precision(adjoint)
        plan.backward(0, torch.tensor(c, dtype=torch.float32, device="cuda"), buf, grad)
    g = grad.cpu().numpy().transpose(1, 0, 2, 3)
    kw = oracle_kw(spec)
    kw["E_meV"] = E
    ref = oracle.gradient(fr, c, **kw)
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel <= 1e-4, rel
    inside = oracle.detector_masks(spec.Kx, spec.Ky, spec.detectors).sum(axis=0) > 0
    assert inside.sum() == 182
    assert np.all(g[:, :, ~inside] == 0)


@pytest.mark.parametrize("adjoint", ["split_bf16", "fp32"])
@pytest.mark.parametrize("shape", ["narrow", "wide"])
def test_adjoint_long_segment_and_many_energies(adjoint, shape):
    """T = 1100 frames and 600 energies: both tensor-core contractions of the adjoint run longer
    than one 512-deep accumulator chunk (Psi over 35 staging blocks of frames, the back-projection
    over 19 of energies), so their mid-tile drains into FP32 registers are exercised, with narrow
    tiles (58 aperture rows: one row tile, 8-wide tiles) and wide ones (4 probes x 1257 aperture
    pixels: 40 row tiles, 88-wide tiles); against the FP64 oracle's gradient (whole, or at 48
    sampled aperture pixels a probe), exactly zero outside the aperture."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan, build
    from synth import Detector, StreamSpec
    from tests.helpers import oracle_kw, stream_config
    build.build_all()
    if shape == "narrow":
        spec = StreamSpec(P=2, Kx=12, Ky=10, T=1100, Tc=1100, n_omega=600, E_max_meV=150.0, window="hann",
                          detectors=(Detector("circular", 0, 0, -1, 3.0),))
    else:
        spec = StreamSpec(P=4, Kx=48, Ky=48, T=1100, Tc=1100, n_omega=600, E_max_meV=150.0, window="hann",
                          detectors=(Detector("circular", 0, 0, -1, 20.0),))
    fr = ragged_frames(spec.P, spec.T, spec.Ky, spec.Kx, 11)
    c = np.random.default_rng(12).standard_normal((spec.P, 1, spec.Nw))
    buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).to("cuda")
    grad = torch.empty_like(buf)
    with TacawPlan([stream_config(spec)], precision="split_bf16") as plan:
        plan.set_adjoint_precision(adjoint)
        for _ in range(2):                          # the plan's scratch reused by the second call
            plan.backward(0, torch.tensor(c, dtype=torch.float32, device="cuda"), buf, grad)
    g = grad.cpu().numpy().transpose(1, 0, 2, 3)
    inside = oracle.detector_masks(spec.Kx, spec.Ky, spec.detectors)[0] > 0
    assert np.all(g[:, :, ~inside] == 0)
    kw = oracle_kw(spec)
    if shape == "narrow":
        ref = oracle.gradient(fr, c, **kw)
        rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        assert rel <= 1e-4, rel
        return
    kw.pop("detectors")
    kw.pop("window_param")
    ap = np.nonzero(inside.reshape(-1))[0]
    assert len(ap) == 1257
    rng = np.random.default_rng(13)
    for p in range(spec.P):
        sel = rng.choice(ap, 48, replace=False)
        series = fr[p].reshape(spec.T, -1)[:, sel]
        ref = oracle.gradient_pixels(series, c[p], np.ones((len(sel), 1)), **kw)
        got = g[p].reshape(spec.T, -1)[:, sel]
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 1e-4, (p, rel)


def test_adjoint_on_each_stream_of_a_multi_stream_plan():
    """A plan of two streams of different shapes (ROI, T, energies, apertures): backward on
    stream 0, then on the larger stream 1 (the plan's adjoint scratch grows), then on stream 0
    again (the grown scratch is reused, stream 0's tables kept): each against the FP64 oracle's
    gradient of its own stream."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan, build
    from synth import Detector, StreamSpec
    from tests.helpers import oracle_kw, stream_config
    build.build_all()
    specs = [StreamSpec(P=2, Kx=20, Ky=16, T=96, Tc=96, n_omega=40, E_max_meV=120.0, window="hann",
                        detectors=(Detector("circular", 0, 0, -1, 5.0),)),
             StreamSpec(P=3, Kx=40, Ky=36, T=200, Tc=200, n_omega=130, E_max_meV=150.0, window="gauss",
                        detectors=(Detector("circular", 0, 0, -1, 9.0), Detector("annular", 0, 0, 4.0, 12.0)))]
    data = []
    for i, sp in enumerate(specs):
        fr = ragged_frames(sp.P, sp.T, sp.Ky, sp.Kx, 40 + i)
        c = np.random.default_rng(50 + i).standard_normal((sp.P, len(sp.detectors), sp.Nw))
        buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).to("cuda")
        data.append((fr, c, buf))
    with TacawPlan([stream_config(sp) for sp in specs], precision="split_bf16") as plan:
        for sid in (0, 1, 0):
            sp = specs[sid]
            fr, c, buf = data[sid]
            grad = torch.empty_like(buf)
            plan.backward(sid, torch.tensor(c, dtype=torch.float32, device="cuda"), buf, grad)
            g = grad.cpu().numpy().transpose(1, 0, 2, 3)
            ref = oracle.gradient(fr, c, **oracle_kw(sp))
            rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
            assert rel <= 1e-4, (sid, rel)


def test_adjoint_precision_choices():
    """tacaw_set_adjoint_precision takes split BF16 (tensor cores) or FP32 (CUDA cores); split FP16
    or an unknown value is INVALID_ARG and leaves the plan usable."""
    from paper_2607_02236_gb300 import TacawError, TacawPlan, build
    from paper_2607_02236_gb300.tacaw import ERR_INVALID_ARG
    from synth import StreamSpec
    from tests.helpers import stream_config
    build.build_all()
    spec = StreamSpec(P=1, Kx=8, Ky=8, T=32, Tc=32, n_omega=8)
    with TacawPlan([stream_config(spec)], precision="split_bf16") as plan:
        plan.set_adjoint_precision("fp32")
        plan.set_adjoint_precision("split_bf16")
        for bad in ("split_fp16", "nope"):
            with pytest.raises(TacawError) as ei:
                plan.set_adjoint_precision(bad)
            assert ei.value.status == ERR_INVALID_ARG
        plan.set_adjoint_precision("fp32")
