"""tacaw_detector_spectra_noalloc: detector spectra for callers that may not allocate device
memory (it uses the library's fixed device array instead of plan memory).

Checked through the C ABI against the spectra the plan path (tacaw_finalize) produces from
the same intensities, within the FP32 test tolerance, on two calls in a row; the second call
uses fewer aperture entries than the first, so stale entries left in the shared array by
the first call would show up.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from synth import Detector, StreamSpec
from tests.helpers import stream_config

pytestmark = pytest.mark.gpu

TOL = 1e-5


def run_plan(spec, x):
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    P, K, Nw, D = spec.P, spec.Kx, spec.Nw, len(spec.detectors)
    I = torch.empty(P * Nw * K * K, dtype=torch.float32, device="cuda")
    S = torch.empty(P * D * Nw, dtype=torch.float32, device="cuda")
    with TacawPlan([stream_config(spec)], precision="fp32") as plan:
        plan.push(0, x, spec.T)
        plan.finalize(I, S)
    torch.cuda.synchronize()
    return I, S.cpu().numpy().reshape(P, D, Nw)


def test_noalloc_spectra_match_plan_spectra_two_calls():
    import torch
    from paper_2607_02236_gb300 import build
    build.build_all()
    from paper_2607_02236_gb300.tacaw import DetectorConfig, detector_spectra_noalloc
    dets_a = (Detector("circular", 0, 0, -1, 9.0), Detector("annular", 0, 0, 4.0, 15.0),
              Detector("circular", 7, -5, -1, 4.0))
    dets_b = (Detector("annular", 2, 1, 1.0, 3.0),)
    base = dict(P=3, Kx=40, Ky=40, T=64, Tc=64, n_omega=70, E_max_meV=120.0, window="hann")
    spec_a = StreamSpec(detectors=dets_a, **base)
    spec_b = StreamSpec(detectors=dets_b, **base)
    rng = np.random.default_rng(3)
    f = (rng.standard_normal((64, 3, 40, 40)) + 1j * rng.standard_normal((64, 3, 40, 40))).astype(np.complex64)
    x = torch.from_numpy(f).cuda()
    I, S_a = run_plan(spec_a, x)
    _, S_b = run_plan(spec_b, x)
    for spec, S_ref in ((spec_a, S_a), (spec_b, S_b)):
        dets = [DetectorConfig(d.kind, d.cx, d.cy, d.r_in, d.r_out) for d in spec.detectors]
        S = torch.full((spec.P * len(dets) * spec.Nw,), float("nan"), dtype=torch.float32, device="cuda")
        detector_spectra_noalloc(I, spec.P, spec.Nw, spec.Kx, spec.Ky, dets, S)
        torch.cuda.synchronize()
        got = S.cpu().numpy().reshape(S_ref.shape)
        err = np.max(np.abs(got - S_ref)) / np.max(np.abs(S_ref))
        assert err <= TOL, err


def test_noalloc_rejects_oversize_requests():
    import torch
    from paper_2607_02236_gb300 import build
    build.build_all()
    from paper_2607_02236_gb300.tacaw import DetectorConfig, TacawError, ERR_INVALID_ARG, detector_spectra_noalloc
    I = torch.zeros(1, dtype=torch.float32, device="cuda")
    S = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(TacawError) as ei:
        detector_spectra_noalloc(I, 1, 1, 8, 8, [DetectorConfig()] * 1025, S)
    assert ei.value.status == ERR_INVALID_ARG and "maximum of 1024" in str(ei.value)
    # 2048 x 1024 pixels all inside one aperture: 2^21 entries > 2^20
    with pytest.raises(TacawError) as ei:
        detector_spectra_noalloc(I, 1, 1, 2048, 1024, [DetectorConfig(r_out=1e9)], S)
    assert ei.value.status == ERR_INVALID_ARG and "fixed device array" in str(ei.value)
