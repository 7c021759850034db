"""Differentiation workload: 8 probes, 128x128 ROI, T=512, 200 energies over 0-120 meV, Hann,
FP32.  L = sum_p sum_E c(E) S_p(E) with S the r=20 px aperture spectrum and c ~ N(0,1) seeded.

The adjoint (tacaw_backward behind torch.autograd) is checked against the FP64 oracle gradient
(relative L2 <= 1e-4 on sampled aperture pixels, exact zeros outside the aperture) and
against FP64 central finite differences (h = 1e-6) of the oracle loss on 64 random entries.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import frames as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
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
