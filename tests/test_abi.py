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
    assert L.tacaw_push_frames_group(None, 1, None, None, None, None) == t.ERR_INVALID_ARG
    assert L.tacaw_finalize(None, None, None, None, None) == t.ERR_INVALID_ARG
    assert L.tacaw_set_adjoint_precision(None, t.PRECISIONS["split_bf16"]) == t.ERR_INVALID_ARG
    assert L.tacaw_set_pipelined_segments(None, 1) == t.ERR_INVALID_ARG
    assert L.tacaw_drain(None, None) == t.ERR_INVALID_ARG
    n = ctypes.c_int64(-1)
    assert L.tacaw_state_size(None, ctypes.byref(n)) == t.ERR_INVALID_ARG and n.value == -1
    buf = ctypes.create_string_buffer(64)
    assert L.tacaw_save_state(None, buf, 64, None) == t.ERR_INVALID_ARG
    assert L.tacaw_restore_state(None, buf, 64, None) == t.ERR_INVALID_ARG
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


_BASE = dict(n_probes=2, kx=8, ky=8, T=16, dt_fs=5.0, pitch_row=8, pitch_frame=128, pitch_probe=64, fft_bins=8)

# (stream fields, plan options, message fragment): each is refused with INVALID_ARG before the
# plan touches the device
_REFUSED = [
    (dict(window="kaiser", window_param=61.0), {}, "Kaiser beta"),
    (dict(window="chebwin", window_param=0.0), {}, "Chebyshev attenuation"),
    (dict(roi_x0=-1, pitch_row=9), {}, "negative ROI origin"),
    (dict(pitch_frame=32), {}, "pitch_frame"),
    (dict(bose_T_K=-1.0), {}, "bose_T_K"),
    (dict(welch_segments=-1), {}, "welch_segments"),
    (dict(skip_init=-3), {}, "skip_init"),
    (dict(fft_bins=0, E_meV=None, n_omega=4), {}, "E_meV is NULL"),
    ({}, dict(tc_drain_frames=12), "tc_drain_frames"),
    ({}, dict(tc_omega_tile=12), "tc_omega_tile"),
    ({}, dict(tc_block_frames=24), "tc_block_frames"),
    ({}, dict(k_stage=40, tc_block_frames=32), "multiple of tc_block_frames"),
]


@pytest.mark.parametrize("stream_kw,plan_kw,msg", _REFUSED, ids=[r[2] for r in _REFUSED])
def test_plan_options_refused_before_device_work(L, stream_kw, plan_kw, msg):
    import paper_2607_02236_gb300.tacaw as t
    cfg = dict(_BASE)
    cfg.update(stream_kw)
    with pytest.raises(t.TacawError) as ei:
        t.TacawPlan([t.StreamConfig(**cfg)], precision="split_bf16", **plan_kw)
    assert ei.value.status == t.ERR_INVALID_ARG, str(ei.value)
    assert msg in L.tacaw_last_error().decode()


def test_bad_enums_refused_before_device_work(L):
    import ctypes
    import paper_2607_02236_gb300.tacaw as t
    s = t.CStreamDesc()
    s.n_probes, s.kx, s.ky, s.T, s.dt_fs = 1, 8, 8, 16, 5.0
    s.pitch_row, s.pitch_frame, s.pitch_probe, s.fft_bins, s.n_omega = 8, 64, 64, 1, 8
    for field_name, value, msg in (("precision", 7, "bad precision"), ("accum", 9, "bad accum")):
        d = t.CPlanDesc()
        d.n_streams, d.streams = 1, ctypes.pointer(s)
        d.precision, d.accum = 1, 3
        setattr(d, field_name, value)
        h = ctypes.c_void_p()
        assert L.tacaw_plan_create(ctypes.byref(d), ctypes.byref(h)) == t.ERR_INVALID_ARG
        assert msg in L.tacaw_last_error().decode()
        assert not h.value


def test_log_callback_receives_errors_and_can_be_removed(L):
    import paper_2607_02236_gb300.tacaw as t
    got = []
    t.set_log_callback(lambda level, msg: got.append((level, msg)))
    try:
        with pytest.raises(t.TacawError):
            t.TacawPlan([t.StreamConfig(**dict(_BASE, T=0))], precision="fp32")
        assert L.tacaw_push_frames(None, 0, None, 1, None) == t.ERR_INVALID_ARG
    finally:
        t.set_log_callback(None)
    assert [lvl for lvl, _ in got] == [t.LOG_ERROR, t.LOG_ERROR]
    assert "T must be >= 1" in got[0][1]
    assert got[1][1] == L.tacaw_last_error().decode()
    n = len(got)
    with pytest.raises(t.TacawError):
        t.TacawPlan([t.StreamConfig(**dict(_BASE, T=0))], precision="fp32")
    assert len(got) == n                                   # removed: no further calls


# in-place layouts the in-place kernel cannot take: refused with UNSUPPORTED before device work
_INPLACE_REFUSED = [
    (dict(kx=16, ky=16, pitch_row=20, pitch_frame=640, pitch_probe=320, roi_x0=2), {}, "contiguous"),
    (dict(kx=8, ky=8, pitch_row=16, pitch_frame=256, pitch_probe=128), {}, "contiguous"),
    (dict(kx=128, ky=2, pitch_row=129, pitch_frame=1024, pitch_probe=512, roi_x0=1), {}, "contiguous"),
    (dict(kx=128, ky=2, pitch_row=128, pitch_frame=512, pitch_probe=256), dict(tc_block_frames=16), "32-frame"),
    (dict(kx=128, ky=2, pitch_row=128, pitch_frame=512, pitch_probe=256), dict(k_stage=48), "32-frame"),
]


@pytest.mark.parametrize("stream_kw,plan_kw,msg", _INPLACE_REFUSED, ids=[f"{i}-{r[2]}" for i, r in
                                                                            enumerate(_INPLACE_REFUSED)])
def test_inplace_layouts_refused_before_device_work(L, stream_kw, plan_kw, msg):
    import paper_2607_02236_gb300.tacaw as t
    cfg = dict(_BASE, T=64)
    cfg.update(stream_kw)
    with pytest.raises(t.TacawError) as ei:
        t.TacawPlan([t.StreamConfig(**cfg)], precision="split_bf16", frames_in_place=True, **plan_kw)
    assert ei.value.status == t.ERR_UNSUPPORTED, str(ei.value)
    assert msg in L.tacaw_last_error().decode()
    with pytest.raises(t.TacawError) as ei:
        t.TacawPlan([t.StreamConfig(**cfg)], precision="fp32", frames_in_place=True)
    assert ei.value.status == t.ERR_UNSUPPORTED
