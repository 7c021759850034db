"""tacaw_detector_spectra_noalloc: detector spectra for callers that may not allocate device
memory (it keeps the aperture lists in the library's fixed device array instead of plan
memory).

Checked through the C ABI against the FP64 oracle: the oracle's I (rounded to float32) goes in,
and the spectra that come out must match the oracle's S within the FP32 test tolerance, with
circular, annular, off-axis and weighted-mask detectors, on two calls in a row.  The second
call uses fewer aperture entries than the first, so stale entries left in the shared array by
the first call would show up.  The refusals (pointers kernels cannot read, a capturing stream,
oversize requests) are checked before any device work.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from synth import Detector

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


def oracle_case(P=3, K=40, T=64, Nw=70, seed=3):
    rng = np.random.default_rng(seed)
    f = (rng.standard_normal((P, T, K, K)) + 1j * rng.standard_normal((P, T, K, K))).astype(np.complex64)
    E = np.arange(Nw) * (120.0 / Nw)
    return f, E


def test_noalloc_spectra_match_oracle_two_calls():
    import torch
    from paper_2607_02236_gb300.tacaw import DetectorConfig, detector_spectra_noalloc
    P, K, T, Nw = 3, 40, 64, 70
    f, E = oracle_case(P, K, T, Nw)
    rng = np.random.default_rng(11)
    mask = (rng.random((K, K)) * (rng.random((K, K)) < 0.25)).astype(np.float32)
    d_mask = torch.from_numpy(mask).cuda()
    dets_a = (Detector("circular", 0, 0, -1, 9.0), Detector("annular", 0, 0, 4.0, 15.0),
              Detector("circular", 7, -5, -1, 4.0))
    dets_b = (Detector("annular", 2, 1, 1.0, 3.0),)
    ref_a = oracle.forward(f, window_kind="hann", E_meV=E, dt_fs=5.0, detectors=list(dets_a))
    ref_b = oracle.forward(f, window_kind="hann", E_meV=E, dt_fs=5.0, detectors=list(dets_b))
    I = torch.from_numpy(np.ascontiguousarray(ref_a.I, dtype=np.float32)).cuda()   # [P][E][ky][kx]
    # first call: three geometric apertures and a weighted mask (S of the mask from its definition)
    S_mask = np.einsum("pjyx,yx->pj", ref_a.I, mask.astype(np.float64))[:, None, :]
    calls = [([DetectorConfig(d.kind, d.cx, d.cy, d.r_in, d.r_out) for d in dets_a] +
              [DetectorConfig("mask", 0, 0, 0, 0, mask_ptr=d_mask.data_ptr())],
              np.concatenate([ref_a.S, S_mask], axis=1)),
             ([DetectorConfig(d.kind, d.cx, d.cy, d.r_in, d.r_out) for d in dets_b], ref_b.S)]
    for dets, S_ref in calls:
        S = torch.full((P * len(dets) * Nw,), float("nan"), dtype=torch.float32, device="cuda")
        detector_spectra_noalloc(I, P, Nw, K, K, dets, S)
        torch.cuda.synchronize()
        got = S.cpu().numpy().reshape(S_ref.shape)
        err = np.max(np.abs(got - S_ref)) / np.max(np.abs(S_ref))
        assert err <= TOL, err


def test_noalloc_refusals_before_device_work():
    import torch
    from paper_2607_02236_gb300.tacaw import DetectorConfig, TacawError, ERR_INVALID_ARG, detector_spectra_noalloc
    I = torch.zeros(64, dtype=torch.float32, device="cuda")
    S = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(TacawError) as ei:
        detector_spectra_noalloc(I, 1, 1, 8, 8, [DetectorConfig()] * 1025, S)
    assert ei.value.status == ERR_INVALID_ARG and "maximum of 1024" in str(ei.value)
    # 2048 x 1024 pixels all inside one aperture: 2^21 entries > 2^20
    big = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(TacawError) as ei:
        detector_spectra_noalloc(big, 1, 1, 2048, 1024, [DetectorConfig(r_out=1e9)], S)
    assert ei.value.status == ERR_INVALID_ARG and "fixed device array" in str(ei.value)
    with pytest.raises(TacawError) as ei:
        detector_spectra_noalloc(big, 1, 1, 65536, 65536, [DetectorConfig(r_out=1.0)], S)
    assert ei.value.status == ERR_INVALID_ARG and "2^31" in str(ei.value)
    # pageable host memory for d_I or d_S: no kernel may read it
    host = np.zeros(64, dtype=np.float32)
    with pytest.raises(TacawError) as ei:
        detector_spectra_noalloc(host.ctypes.data, 1, 1, 8, 8, [DetectorConfig(r_out=2.0)], S)
    assert ei.value.status == ERR_INVALID_ARG and "d_I" in str(ei.value)
    with pytest.raises(TacawError) as ei:
        detector_spectra_noalloc(I, 1, 1, 8, 8, [DetectorConfig(r_out=2.0)], host.ctypes.data)
    assert ei.value.status == ERR_INVALID_ARG and "d_S" in str(ei.value)
    # a stream that is capturing a graph: refused, and the capture itself is left intact
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        with pytest.raises(TacawError) as ei:
            detector_spectra_noalloc(I, 1, 1, 8, 8, [DetectorConfig(r_out=2.0)], S, cuda_stream=st)
        S.add_(1.0)
    assert ei.value.status == ERR_INVALID_ARG and "capturing" in str(ei.value)
    g.replay()
    torch.cuda.synchronize()
    assert float(S[0]) == 1.0


def test_noalloc_matches_oracle_after_a_plan_run():
    """The entry point after the other tests of the process (and a plan's own spectra path):
    the same oracle comparison on a fresh case."""
    import torch
    from paper_2607_02236_gb300.tacaw import DetectorConfig, detector_spectra_noalloc
    P, K, T, Nw = 2, 24, 32, 40
    f, E = oracle_case(P, K, T, Nw, seed=9)
    dets = (Detector("circular", 0, 0, -1, 6.0), Detector("annular", -2, 3, 2.0, 8.0))
    ref = oracle.forward(f, window_kind="hann", E_meV=E, dt_fs=5.0, detectors=list(dets))
    I = torch.from_numpy(np.ascontiguousarray(ref.I, dtype=np.float32)).cuda()
    for _ in range(2):
        S = torch.full((P * len(dets) * Nw,), float("nan"), dtype=torch.float32, device="cuda")
        detector_spectra_noalloc(I, P, Nw, K, K, [DetectorConfig(d.kind, d.cx, d.cy, d.r_in, d.r_out) for d in dets], S)
        torch.cuda.synchronize()
        got = S.cpu().numpy().reshape(ref.S.shape)
        assert np.max(np.abs(got - ref.S)) / np.max(np.abs(ref.S)) <= TOL
