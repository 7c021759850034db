"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (max |GPU - oracle| / max |oracle|, per output):
  FP32 CUDA-core path:    1e-5 of peak intensity (and of peak spectrum)
  split tensor-core path: the same 1e-5 (TOL_SPLIT): hi*hi + hi*lo + lo*hi with FP32 accumulation
                          in tensor memory, hi*hi drained into FP32 registers every 512 frames
                          (each operand carries ~2^-17 relative error; measured 2-7e-6 on the
                          realistic, batched and thick workloads), so the split path is held to the
                          FP32 path's accuracy.
  white-noise edge cases: TOL_SPLIT_NOISE = 2e-5 for the split path on random_frames inputs in
                          test_edge_cases (no tones: every bin is an incoherent sum).  Each bf16 hi + lo
                          operand carries up to 2^-18 relative error (the rounding of lo), so a real MAC
                          of the three products is off by up to ~3 * 2^-18 |a||b|; over an incoherent sum
                          the peak bin's |Psi|^2 then moves by up to ~2 * 3 * 2^-18 = 2.3e-5 of itself
                          (measured 1.2e-5 at T = 48 and 600 energies, under 1e-5 elsewhere).
"""
import zlib

import numpy as np
import pytest

import oracle
import synth
from synth import Detector, StreamSpec, frames
from tests.helpers import oracle_kw, rel_err_peak, run_gpu

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_SPLIT = 1e-5
TOL_SPLIT_NOISE = 2e-5
TOL = {"fp32": TOL_FP32, "split_bf16": TOL_SPLIT, "split_inplace": TOL_SPLIT}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


def random_frames(P, T, Ky, Kx, seed=0, elastic=1.0, signal=1e-2):
    """Elastic offset per pixel plus small fluctuations (the regime the mean removal targets)."""
    rng = np.random.default_rng(seed)
    e = elastic * (rng.standard_normal((P, 1, Ky, Kx)) + 1j * rng.standard_normal((P, 1, Ky, Kx)))
    s = signal * (rng.standard_normal((P, T, Ky, Kx)) + 1j * rng.standard_normal((P, T, Ky, Kx)))
    return (e + s).astype(np.complex64)


def check(spec, fr, precision, tol=None, **kw):
    if precision == "split_inplace":      # pushed frames read in place by the contraction
        out = run_gpu(spec, fr, "split_bf16", frames_in_place=True, **kw)
    else:
        out = run_gpu(spec, fr, precision, **kw)
    ref = oracle.forward(fr, **oracle_kw(spec))
    eI = rel_err_peak(out["I"], ref.I)
    tol = TOL[precision] if tol is None else tol
    assert eI <= tol, f"I error {eI:.3g} > {tol}"
    if len(spec.detectors):
        eS = rel_err_peak(out["S"], ref.S)
        assert eS <= tol, f"S error {eS:.3g} > {tol}"
    if "want_psi" in kw:
        eP = rel_err_peak(out["Psi"], ref.Psi)
        assert eP <= tol, f"Psi error {eP:.3g}"
    return out, ref, eI


@pytest.mark.parametrize("precision", ["fp32", "split_bf16", "split_inplace"])
def test_tiny_config_whole(precision):
    """4 probes, 64x64, T=256 in one push, first 128 FFT bins, Hann, mean removed, r=20 aperture."""
    s = synth.tiny().streams[0]
    fr = frames.frames(s, 0, 0, s.T)
    out, ref, e = check(s, fr, precision, want_psi=True)
    print(f"tiny {precision}: max rel I error {e:.3g}")


CASES = {
    # ragged rows (M=105 < 128), T not a multiple of 8, uneven pushes
    "ragged": (StreamSpec(P=3, Kx=5, Ky=7, T=37, Tc=5, n_omega=19, E_max_meV=150.0, window="hann",
                          detectors=(Detector("circular", 0, 0, -1, 2.0),)), [5, 11, 8, 13], 0),
    # rows straddle probes (npix=144), several flushes with the accumulator
    "multiflush": (StreamSpec(P=3, Kx=12, Ky=12, T=100, Tc=10, n_omega=40, E_max_meV=120.0, window="hann",
                              detectors=(Detector("annular", 0, 0, 1.0, 4.0),)), None, 16),
    "rect_nomean": (StreamSpec(P=2, Kx=16, Ky=16, T=64, Tc=64, fft_bins=64, window="rect", subtract_mean=False,
                               detectors=(Detector("circular", 2, -3, -1, 3.0),)), None, 0),
    "gauss_bose": (StreamSpec(P=2, Kx=16, Ky=8, T=96, Tc=32, n_omega=33, E_max_meV=100.0, window="gauss",
                              bose_T_K=300.0, detectors=(Detector(), Detector("annular", 0, 0, 2, 5))), None, 0),
    "tukey": (StreamSpec(P=1, Kx=32, Ky=32, T=80, Tc=16, n_omega=50, E_max_meV=90.0, window="tukey",
                         window_param=0.1), None, 0),
    "many_omega": (StreamSpec(P=1, Kx=16, Ky=16, T=48, Tc=48, n_omega=600, E_max_meV=400.0, window="hann",
                              detectors=(Detector("circular", 0, 0, -1, 3.0),)), None, 0),
    "one_omega_one_frame": (StreamSpec(P=2, Kx=8, Ky=8, T=1, Tc=1, n_omega=1, E_max_meV=10.0, window="hann",
                                       subtract_mean=False), None, 0),
}


@pytest.mark.parametrize("precision", ["fp32", "split_bf16", "split_inplace"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_edge_cases(name, precision):
    spec, pushes, k_stage = CASES[name]
    fr = random_frames(spec.P, spec.T, spec.Ky, spec.Kx, seed=zlib.crc32(name.encode()) % 1000)
    if precision == "split_inplace" and name == "ragged":
        # 105 rows: an odd row count cannot be read in place (16-byte row copies); the plan is refused
        from paper_2607_02236_gb300 import TacawError
        from paper_2607_02236_gb300.tacaw import ERR_UNSUPPORTED
        with pytest.raises(TacawError) as ei:
            run_gpu(spec, fr, "split_bf16", frames_in_place=True, pushes=pushes, k_stage=k_stage)
        assert ei.value.status == ERR_UNSUPPORTED
        return
    if precision == "split_inplace" and k_stage % 32:
        k_stage = 32                      # in-place flushes are whole 32-frame blocks
    out, ref, e = check(spec, fr, precision, tol=TOL_FP32 if precision == "fp32" else TOL_SPLIT_NOISE,
                        pushes=pushes, k_stage=k_stage)
    if k_stage:
        assert out["info"]["flushes"] > 1


@pytest.mark.parametrize("accum", ["kahan", "fp64", "fp32"])
@pytest.mark.parametrize("precision", ["fp32", "split_bf16", "split_inplace"])
def test_streaming_flushes_match_single_flush(precision, accum):
    """K_stage < T (accumulators in HBM) gives the oracle's result too."""
    spec = StreamSpec(P=2, Kx=32, Ky=16, T=200, Tc=24, n_omega=70, E_max_meV=120.0, window="hann",
                      n_modes=6, detectors=(Detector("circular", 0, 0, -1, 5.0),))
    fr = frames.frames(spec, 3, 0, spec.T)
    k_stage = 64 if precision == "split_inplace" else 48      # in place: whole 32-frame blocks
    out, ref, e = check(spec, fr, precision, k_stage=k_stage, accum=accum)
    assert out["info"]["flushes"] == -(-spec.T // k_stage)


@pytest.mark.parametrize("k_stage,expect", [(16, 2), (8, 0), (0, 2)])
def test_auto_accumulators(k_stage, expect):
    """accum="auto": plain FP32 cross-flush sums up to 16 flushes a segment (13 here at
    K_stage = 16), compensated beyond (25 at K_stage = 8); irrelevant for one flush."""
    spec = StreamSpec(P=2, Kx=16, Ky=16, T=200, Tc=24, n_omega=40, E_max_meV=120.0, window="hann",
                      detectors=(Detector("circular", 0, 0, -1, 4.0),))
    fr = frames.frames(spec, 5, 0, spec.T)
    out, ref, e = check(spec, fr, "split_bf16", k_stage=k_stage, accum="auto")
    assert out["info"]["accum"] == expect, out["info"]["accum"]


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_elastic_only_input_gives_zero(precision):
    """Frames constant in time (pure elastic part): nothing is left after the mean removal."""
    spec = StreamSpec(P=2, Kx=24, Ky=16, T=72, Tc=24, n_omega=40, E_max_meV=120.0, window="hann",
                      detectors=(Detector("circular", 0, 0, -1, 5.0),))
    rng = np.random.default_rng(4)
    c = (rng.standard_normal((2, 1, 16, 24)) + 1j * rng.standard_normal((2, 1, 16, 24))).astype(np.complex64)
    fr = np.repeat(c, spec.T, axis=1)
    out = run_gpu(spec, fr, precision)
    scale = (np.abs(fr) ** 2).sum(axis=(1, 2, 3)).max() * spec.T
    assert np.abs(out["I"]).max() <= 1e-12 * scale ** 2 / spec.T, np.abs(out["I"]).max()
    assert np.abs(out["S"]).max() <= 1e-12 * scale ** 2 / spec.T


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_signed_energies_bose_and_custom_mask(precision):
    """Energy-gain and -loss sides (a signed +-60 meV grid) with the Bose factor of Eq. 1, and a
    caller-supplied weighted mask detector next to circular and annular ones."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan, DetectorConfig
    from tests.helpers import stream_config
    P, K, T, Nw = 2, 20, 64, 41
    rng = np.random.default_rng(12)
    fr = random_frames(P, T, K, K, seed=12)
    E = np.linspace(-60.0, 60.0, Nw)
    mask = (rng.random((K, K)) * (rng.random((K, K)) < 0.3)).astype(np.float32)
    d_mask = torch.from_numpy(mask).cuda()
    spec = StreamSpec(P=P, Kx=K, Ky=K, T=T, Tc=T, n_omega=Nw, window="hann", bose_T_K=300.0)
    cfg = stream_config(spec)
    cfg.E_meV = [float(e) for e in E]
    cfg.detectors = [DetectorConfig("circular", 0, 0, -1, 4.0), DetectorConfig("annular", 1, 0, 2.0, 6.0),
                     DetectorConfig("mask", 0, 0, 0, 0, mask_ptr=d_mask.data_ptr())]
    buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).cuda()
    I = torch.empty(P * Nw * K * K, device="cuda")
    S = torch.empty(P * 3 * Nw, device="cuda")
    with TacawPlan([cfg], precision=precision) as plan:
        plan.push(0, buf, T)
        plan.finalize(I, S)
    ref = oracle.forward(fr, window_kind="hann", E_meV=E, dt_fs=5.0, subtract_mean=True, bose_T_K=300.0,
                         detectors=[Detector("circular", 0, 0, -1, 4.0), Detector("annular", 1, 0, 2.0, 6.0)])
    got_I = I.cpu().numpy().reshape(P, Nw, K, K)
    assert rel_err_peak(got_I, ref.I) <= TOL[precision]
    S_mask = np.einsum("pjyx,yx->pj", ref.I, mask.astype(np.float64))
    S_ref = np.concatenate([ref.S, S_mask[:, None, :]], axis=1)
    assert rel_err_peak(S.cpu().numpy().reshape(P, 3, Nw), S_ref) <= TOL[precision]


def test_errors_overflow_and_state():
    import torch
    from paper_2607_02236_gb300 import TacawPlan, TacawError
    from paper_2607_02236_gb300.tacaw import ERR_OVERFLOW, ERR_STATE
    from tests.helpers import stream_config
    spec = StreamSpec(P=1, Kx=8, Ky=8, T=16, Tc=8, n_omega=4)
    buf = torch.zeros(32 * 64, dtype=torch.complex64, device="cuda")
    with TacawPlan([stream_config(spec)], precision="fp32") as plan:
        plan.push(0, buf, 8)
        I = torch.empty(4 * 64, device="cuda")
        with pytest.raises(TacawError) as ei:
            plan.finalize(I)
        assert ei.value.status == ERR_STATE
        with pytest.raises(TacawError) as ei:
            plan.push(0, buf, 9)
        assert ei.value.status == ERR_OVERFLOW
        plan.push(0, buf, 8)
        plan.finalize(I)
        with pytest.raises(TacawError) as ei:
            plan.push(0, buf, 1)
        assert ei.value.status == ERR_STATE
        plan.reset()
        plan.push(0, buf, 16)
        plan.finalize(I)


@pytest.mark.parametrize("wt,bf,drain,k_stage", [(0, 8, 0, 0), (0, 16, 0, 0), (0, 32, 0, 0), (16, 16, 0, 0),
                                                 (24, 8, 0, 0), (112, 16, 0, 0), (40, 32, 0, 0), (0, 8, 32, 0),
                                                 (0, 32, 64, 0), (0, 16, 1024, 0), (112, 16, 16, 0),
                                                 (40, 8, 24, 0), (0, 32, 32, 64), (72, 16, 64, 96)])
def test_staged_tilings(wt, bf, drain, k_stage):
    """Staged split path at every energy-tile width (16 .. 112 energies, a narrower last tile),
    staging row width (8, 16, 32 frames) and drain length (chunks that do not divide the flush, a
    single chunk, several flushes on top of the cross-flush accumulators): 31 ragged row tiles,
    T = 168 (not a multiple of 32: the last block has a zeroed tail)."""
    spec = StreamSpec(P=3, Kx=36, Ky=36, T=168, Tc=40, n_omega=150, E_max_meV=120.0, window="hann", n_modes=6,
                      noise=1e-3, detectors=(Detector("circular", 0, 0, -1, 6.0),))
    fr = frames.frames(spec, 10, 0, spec.T)
    out, ref, e = check(spec, fr, "split_bf16", tc_drain_frames=drain, tc_omega_tile=wt, tc_block_frames=bf,
                        k_stage=k_stage)
    info = out["info"]
    assert info["tc_drain_frames"] == max(bf, (drain or 512) // bf * bf)
    assert info["tc_block_frames"] == bf and info["frames_in_place"] == 0
    if wt:
        assert info["omega_tile"] == wt


@pytest.mark.parametrize("wt,drain", [(0, 0), (80, 64), (40, 32), (24, 1024)])
def test_inplace_tilings(wt, drain):
    """Pushed frames read in place by the contraction (operand A converted into tensor memory):
    energy-tile widths up to the in-place limit of 80, drain lengths, T = 168."""
    spec = StreamSpec(P=2, Kx=64, Ky=48, T=168, Tc=40, n_omega=150, E_max_meV=120.0, window="hann", n_modes=6,
                      noise=1e-3, detectors=(Detector("circular", 0, 0, -1, 6.0),))
    fr = frames.frames(spec, 8, 0, spec.T)
    out, ref, e = check(spec, fr, "split_inplace", tc_omega_tile=wt, tc_drain_frames=drain)
    info = out["info"]
    assert info["frames_in_place"] == 1 and info["tc_block_frames"] == 32


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
@pytest.mark.parametrize("win,param", [("blackmanharris", 0.0), ("kaiser", 3 * np.pi), ("kaiser", 5 * np.pi),
                                       ("chebwin", 100.0)])
def test_appendix_windows(win, param, precision):
    """App. A's windows (Blackman-Harris, Kaiser beta = 3 pi / 5 pi, Dolph-Chebyshev 100 dB) on a
    ragged segment (T = 150) and an off-grid energy list."""
    spec = StreamSpec(P=2, Kx=20, Ky=24, T=150, Tc=48, n_omega=60, E_max_meV=120.0, window=win, window_param=param,
                      detectors=(Detector("circular", 0, 0, -1, 5.0),))
    fr = random_frames(2, 150, 24, 20, seed=31)
    out, ref, e = check(spec, fr, precision)
    print(f"{win} {param:.3g} {precision}: {e:.3g}")
