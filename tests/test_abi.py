"""The C-ABI library loads and exports every entry point include/tacaw.h declares;
argument validation answers before any device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2607_02236_gb300 import build
    build.build_all()
    import paper_2607_02236_gb300.tacaw as t
    return t.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tacaw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tacaw_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("tacaw_plan_create", "tacaw_push_frames", "tacaw_finalize", "tacaw_backward", "tacaw_destroy",
              "tacaw_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    import paper_2607_02236_gb300.tacaw as t
    names = declared_functions()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(t.EXPORTS) == names


def test_synth_library_loads():
    from paper_2607_02236_gb300 import build
    build.build_all()
    import synth.gpu as g
    assert hasattr(g.lib(), "synth_frames")


def test_invalid_descriptors_rejected_without_device_work(L):
    import paper_2607_02236_gb300.tacaw as t
    base = dict(n_probes=2, kx=8, ky=8, T=16, dt_fs=5.0, pitch_row=8, pitch_frame=128, pitch_probe=64,
                fft_bins=8)
    bad = [dict(n_probes=0), dict(T=0), dict(dt_fs=0.0), dict(fft_bins=32), dict(pitch_row=4),
           dict(window="nope")]
    for b in bad:
        cfg = dict(base)
        cfg.update(b)
        with pytest.raises((t.TacawError, KeyError)) as ei:
            t.TacawPlan([t.StreamConfig(**cfg)], precision="fp32")
        if isinstance(ei.value, t.TacawError):
            assert ei.value.status == t.ERR_INVALID_ARG, (b, str(ei.value))
    # k_stage not a multiple of 8
    with pytest.raises(t.TacawError) as ei:
        t.TacawPlan([t.StreamConfig(**base)], precision="fp32", k_stage=12)
    assert ei.value.status == t.ERR_INVALID_ARG
    assert "multiple of 8" in L.tacaw_last_error().decode()


def test_null_plan_calls_are_errors(L):
    import paper_2607_02236_gb300.tacaw as t
    assert L.tacaw_push_frames(None, 0, None, 1, None) == t.ERR_INVALID_ARG
    assert L.tacaw_finalize(None, None, None, None, None) == t.ERR_INVALID_ARG
    assert L.tacaw_destroy(None) == t.OK


def test_split_fp16_options_rejected_without_device_work(L):
    import paper_2607_02236_gb300.tacaw as t
    cfg = t.StreamConfig(n_probes=2, kx=8, ky=8, T=16, dt_fs=5.0, pitch_row=8, pitch_frame=128, pitch_probe=64,
                         fft_bins=8)
    for bad in (3.0, -4.0, 2.0 ** 61, float("nan")):
        with pytest.raises(t.TacawError) as ei:
            t.TacawPlan([cfg], precision="split_fp16", fp16_scale=bad)
        assert ei.value.status == t.ERR_INVALID_ARG, bad
        assert "power of two" in L.tacaw_last_error().decode()
    with pytest.raises(t.TacawError) as ei:
        t.TacawPlan([cfg], precision="split_fp16", frames_in_place=True)
    assert ei.value.status == t.ERR_UNSUPPORTED
