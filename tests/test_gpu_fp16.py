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
from tests.helpers import oracle_kw, rel_err_peak, run_gpu
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


@pytest.mark.parametrize("kw", [dict(tc_accumulators=3, tc_cluster=2, tc_block_frames=32),
                                dict(tc_accumulators=1, tc_cluster=2, tc_omega_tile=200, tc_block_frames=16),
                                dict(tc_accumulators=3, tc_pair=1, tc_block_frames=32),
                                dict(tc_accumulators=1, tc_drain_frames=64, tc_block_frames=16),
                                dict(tc_accumulators=2, tc_drain_frames=32, tc_block_frames=8)],
                         ids=["classic3", "classic1_wide", "pair", "drain1", "drain2_bf8"])
def test_tilings_fp16(kw):
    """Every staged tensor-core kernel takes the fp16 operand type (instruction descriptor)."""
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
