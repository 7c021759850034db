"""Checkpoint and resume of a segment in progress: a plan created from the same descriptor that
loads a checkpoint and takes the remaining pushes gives the same I, S and Psi, bit for bit, as
the plan that was never interrupted, whose results match the FP64 oracle (Eq. 1, the detector
sum, and the Welch average of Sec. II.B).  Checkpoints are taken mid-ring, at a full ring whose
flush is still deferred, before the first and after the last push; bad checkpoints are refused
with the plan left as it was."""
import numpy as np
import pytest

import oracle
from synth import Detector, StreamSpec, frames
from tests.helpers import oracle_kw, rel_err_peak, stream_config

pytestmark = pytest.mark.gpu

TOL = 1e-5

# 3 probes x 40 x 36 ROI pixels (4320 rows: a ragged last row tile), T = 256 in pushes of 24
SPEC = StreamSpec(P=3, Kx=40, Ky=36, T=256, Tc=24, n_omega=90, E_max_meV=120.0, window="hann", n_modes=6,
                  noise=1e-3, detectors=(Detector("circular", 0, 0, -1, 7.0), Detector("annular", 1.0, -2.0, 3.0, 9.0)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


@pytest.fixture(scope="module")
def data():
    import torch
    fr = frames.frames(SPEC, 71, 0, SPEC.T)                                   # [P, T, Ky, Kx]
    buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).cuda()
    other = frames.frames(SPEC, 72, 0, SPEC.T)
    obuf = torch.from_numpy(np.ascontiguousarray(other.transpose(1, 0, 2, 3))).cuda()
    return fr, buf, obuf


def frame_bytes(spec):
    return spec.P * spec.Kx * spec.Ky * 8


def push_range(plan, buf, spec, a, b, step, sid=0):
    t = a
    while t < b:
        n = min(step, b - t)
        plan.push(sid, buf.data_ptr() + t * frame_bytes(spec), n)
        t += n


def outputs(plan, spec, want_psi=True):
    import torch
    info = plan.info()
    I = torch.full((info["I_elems"],), -1.0, device="cuda")
    S = torch.full((max(1, info["S_elems"]),), -1.0, device="cuda")
    Psi = torch.zeros(info["I_elems"], dtype=torch.complex64, device="cuda") if want_psi else None
    plan.finalize(I, S, Psi)
    torch.cuda.synchronize()
    return (I.cpu().numpy(), S.cpu().numpy(), Psi.cpu().numpy() if want_psi else None)


def assert_identical(a, b):
    for x, y in zip(a, b):
        if x is None:
            continue
        assert np.array_equal(x, y), f"max difference {np.max(np.abs(x - y)):.3g}"


def check_oracle(res, fr, spec):
    ref = oracle.forward(fr, **oracle_kw(spec))
    I, S, Psi = res
    P, Nw, D = spec.P, spec.Nw, len(spec.detectors)
    assert rel_err_peak(I.reshape(P, Nw, spec.Ky, spec.Kx), ref.I) <= TOL
    assert rel_err_peak(S[:P * D * Nw].reshape(P, D, Nw), ref.S) <= TOL
    if Psi is not None:
        assert rel_err_peak(Psi.reshape(P, Nw, spec.Ky, spec.Kx), ref.Psi) <= TOL


CONFIGS = {
    "split_bf16-kahan": ("split_bf16", dict(accum="kahan", k_stage=64)),
    "split_bf16-fp64": ("split_bf16", dict(accum="fp64", k_stage=64)),
    "split_bf16-fp32": ("split_bf16", dict(accum="fp32", k_stage=64)),
    "split_fp16-kahan": ("split_fp16", dict(accum="kahan", k_stage=64)),
    "fp32-kahan": ("fp32", dict(accum="kahan", k_stage=64)),
    "split_bf16-one-flush": ("split_bf16", dict()),
}


def resume_case(data, precision, kw, cut, dirty=False):
    """Plan A takes frames [0, cut), is checkpointed, and finishes; plan B (optionally after a
    whole segment of other frames) loads the checkpoint and takes frames [cut, T)."""
    from paper_2607_02236_gb300 import TacawPlan
    fr, buf, obuf = data
    with TacawPlan([stream_config(SPEC)], precision=precision, **kw) as A:
        push_range(A, buf, SPEC, 0, cut, SPEC.Tc)
        state = A.save_state()
        assert state.size == A.state_size()
        push_range(A, buf, SPEC, cut, SPEC.T, SPEC.Tc)
        ref = outputs(A, SPEC)
    with TacawPlan([stream_config(SPEC)], precision=precision, **kw) as B:
        if dirty:
            push_range(B, obuf, SPEC, 0, SPEC.T, 40)
            outputs(B, SPEC)
        B.restore_state(state)
        push_range(B, buf, SPEC, cut, SPEC.T, SPEC.Tc)
        got = outputs(B, SPEC)
    assert_identical(got, ref)
    check_oracle(ref, fr, SPEC)
    return state


@pytest.mark.parametrize("cfg", list(CONFIGS))
def test_resume_mid_ring_is_bit_identical(data, cfg):
    """Checkpoint after 120 of 256 frames: with 64-frame rings one flush folded into the
    accumulators and 56 frames staged (a partial block)."""
    precision, kw = CONFIGS[cfg]
    resume_case(data, precision, kw, 120)


@pytest.mark.parametrize("cut", [0, 24, 192, 256], ids=["before-first", "first-push", "full-ring-due", "all-pushed"])
def test_resume_at_segment_edges(data, cut):
    """Before any push; inside the first ring; after 192 frames (a full ring whose flush waits for
    the next push); after the last push (finalize follows the restore)."""
    resume_case(data, "split_bf16", dict(accum="kahan", k_stage=64), cut, dirty=cut == 192)


def test_state_size_formula(data):
    """Header 48 + 48 per internal stream + 8 per stream; mean (8 B) and residual sums (16 B) per
    row; the staged blocks (8 B per row and frame); Kahan accumulators (16 B per row and energy)."""
    from paper_2607_02236_gb300 import TacawPlan
    fr, buf, _ = data
    M = SPEC.P * SPEC.Kx * SPEC.Ky
    M_pad = (M + 127) // 128 * 128
    with TacawPlan([stream_config(SPEC)], precision="split_bf16", accum="kahan", k_stage=64) as plan:
        bf = plan.info()["tc_block_frames"]
        base = 48 + 48 + 8 + M * 24
        assert plan.state_size() == base
        push_range(plan, buf, SPEC, 0, 120, SPEC.Tc)                      # 1 flush, 56 staged
        blocks = (56 + bf - 1) // bf
        assert plan.state_size() == base + blocks * M_pad * bf * 8 + SPEC.Nw * M_pad * 16


def test_rollback_on_the_same_plan(data, tmp_path):
    """A plan that finished its segment loads an earlier checkpoint of its own (read back from a
    file) and takes the same remaining pushes again: the same results, bit for bit."""
    from paper_2607_02236_gb300 import TacawPlan
    fr, buf, _ = data
    with TacawPlan([stream_config(SPEC)], precision="split_bf16", accum="kahan", k_stage=64) as plan:
        push_range(plan, buf, SPEC, 0, 120, SPEC.Tc)
        path = tmp_path / "segment.ckpt"
        plan.save_state().tofile(path)
        push_range(plan, buf, SPEC, 120, SPEC.T, SPEC.Tc)
        first = outputs(plan, SPEC)
        plan.restore_state(np.fromfile(path, dtype=np.uint8))
        push_range(plan, buf, SPEC, 120, SPEC.T, SPEC.Tc)
        second = outputs(plan, SPEC)
        # other push sizes: the FP64 mean sums add in another order, so equal within rounding
        plan.restore_state(np.fromfile(path, dtype=np.uint8))
        push_range(plan, buf, SPEC, 120, SPEC.T, 40)
        third = outputs(plan, SPEC)
    assert_identical(second, first)
    check_oracle(first, fr, SPEC)
    for x, y in zip(third, first):
        assert rel_err_peak(x, y) <= 1e-6


def welch_frames(P, n, Ky, Kx, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((P, 1, Ky, Kx)) + 1j * rng.standard_normal((P, 1, Ky, Kx))
    t = np.arange(n)[None, :, None, None]
    tone = 0.05 * np.exp(2j * np.pi * 0.0731 * t) * rng.standard_normal((P, 1, Ky, Kx))
    s = 1e-2 * (rng.standard_normal((P, n, Ky, Kx)) + 1j * rng.standard_normal((P, n, Ky, Kx)))
    return (e + tone + s).astype(np.complex64)


@pytest.mark.parametrize("precision", ["split_bf16", "fp32"])
def test_resume_welch_average(precision):
    """Welch averaging, L = 64, stride 32, 5 segments after 8 skipped frames, pushed 40 at a
    time: checkpoint after 128 frames (two lanes mid-segment, two segments in the average)."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    spec = StreamSpec(P=2, Kx=24, Ky=20, T=64, Tc=40, n_omega=40, E_max_meV=120.0, window="hann",
                      detectors=(Detector("circular", 0, 0, -1, 6.0),))
    N, stride, skip = 5, 32, 8
    n = skip + (N - 1) * stride + spec.T
    fr = welch_frames(spec.P, n, spec.Ky, spec.Kx, 5)
    buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).cuda()
    cfg = stream_config(spec)
    cfg.welch_segments, cfg.welch_stride, cfg.skip_init = N, stride, skip
    with TacawPlan([cfg], precision=precision, k_stage=32) as A:
        push_range(A, buf, spec, 0, 128, 40)
        state = A.save_state()
        push_range(A, buf, spec, 128, n, 40)
        ref = outputs(A, spec, want_psi=False)
    with TacawPlan([cfg], precision=precision, k_stage=32) as B:
        B.restore_state(state.tobytes())
        push_range(B, buf, spec, 128, n, 40)
        got = outputs(B, spec, want_psi=False)
    assert_identical(got, ref)
    w = oracle.welch_forward(fr, spec.T, stride, skip_init=skip, **oracle_kw(spec))
    assert rel_err_peak(ref[0].reshape(spec.P, spec.Nw, spec.Ky, spec.Kx), w.I) <= TOL
    assert rel_err_peak(ref[1][:spec.P * spec.Nw].reshape(spec.P, 1, spec.Nw), w.S) <= TOL


def test_in_place_checkpoint_at_ring_boundaries(data):
    """frames_in_place plans hold pushed frames by address until their ring's flush: a
    checkpoint is refused until the pushes fill whole rings, and taken there it resumes."""
    from paper_2607_02236_gb300 import TacawPlan, TacawError
    from paper_2607_02236_gb300.tacaw import ERR_STATE
    fr, buf, _ = data
    kw = dict(frames_in_place=True, k_stage=64, accum="kahan")
    with TacawPlan([stream_config(SPEC)], precision="split_bf16", **kw) as A:
        push_range(A, buf, SPEC, 0, 96, 32)
        with pytest.raises(TacawError) as ei:
            A.state_size()
        assert ei.value.status == ERR_STATE and "in-place" in str(ei.value)
        push_range(A, buf, SPEC, 96, 128, 32)
        state = A.save_state()
        push_range(A, buf, SPEC, 128, SPEC.T, 32)
        ref = outputs(A, SPEC)
    with TacawPlan([stream_config(SPEC)], precision="split_bf16", **kw) as B:
        B.restore_state(state)
        push_range(B, buf, SPEC, 128, SPEC.T, 32)
        got = outputs(B, SPEC)
    assert_identical(got, ref)
    check_oracle(ref, fr, SPEC)


def fnv1a64(b: bytes) -> int:
    """64-bit FNV-1a (offset basis 0xcbf29ce484222325, prime 0x100000001b3)."""
    h = 0xcbf29ce484222325
    for x in b:
        h = ((h ^ x) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def test_bad_checkpoints_are_refused_and_leave_the_plan_usable(data):
    import dataclasses
    import torch
    from paper_2607_02236_gb300 import TacawPlan, TacawError
    from paper_2607_02236_gb300 import tacaw as t
    fr, buf, _ = data
    kw = dict(accum="kahan", k_stage=64)
    with TacawPlan([stream_config(SPEC)], precision="split_bf16", **kw) as A:
        push_range(A, buf, SPEC, 0, 120, SPEC.Tc)
        good = A.save_state()
        L = t.lib()
        small = np.empty(good.size - 1, np.uint8)
        assert L.tacaw_save_state(A._h, small.ctypes.data, small.size, None) == t.ERR_INVALID_ARG
        dev = torch.empty(good.size, dtype=torch.uint8, device="cuda")
        assert L.tacaw_save_state(A._h, dev.data_ptr(), dev.numel(), None) == t.ERR_INVALID_ARG
        assert "host memory" in L.tacaw_last_error().decode()
        push_range(A, buf, SPEC, 120, SPEC.T, SPEC.Tc)
        ref = outputs(A, SPEC)
        with pytest.raises(TacawError) as ei:
            A.state_size()
        assert ei.value.status == t.ERR_STATE and "finalized" in str(ei.value)
    bad = {}
    b = good.copy(); b[0] ^= 1; bad["magic"] = (b, "not a plan checkpoint")
    b = good.copy(); b[8] = 99; bad["version"] = (b, "version 99")
    b = good.copy(); b[56] ^= 1; bad["counters"] = (b, "corrupted")      # staged frames of stream 0
    # counters that no push sequence gives (pushed beyond T), with a matching hash
    b = good.copy()
    b[48:56] = np.frombuffer(np.int64(999).tobytes(), np.uint8)
    b[40:48] = np.frombuffer(np.uint64(fnv1a64(b[48:48 + 48 + 8].tobytes())).tobytes(), np.uint8)
    bad["inconsistent"] = (b, "inconsistent")
    bad["truncated"] = (good[:-1], "truncated")
    bad["short"] = (good[:40], "too short")
    with TacawPlan([stream_config(SPEC)], precision="split_bf16", **kw) as B:
        push_range(B, buf, SPEC, 0, 120, SPEC.Tc)                         # where the checkpoint was taken
        for name, (blob, msg) in bad.items():
            with pytest.raises(TacawError) as ei:
                B.restore_state(blob)
            assert ei.value.status == t.ERR_INVALID_ARG and msg in str(ei.value), (name, str(ei.value))
        for other_spec, other_kw in [(dataclasses.replace(SPEC, n_omega=91), kw),
                                     (SPEC, dict(accum="kahan", k_stage=128)),
                                     (SPEC, dict(accum="fp64", k_stage=64)),
                                     (dataclasses.replace(SPEC, window="gauss"), kw)]:
            with TacawPlan([stream_config(other_spec)], precision="split_bf16", **other_kw) as C:
                with pytest.raises(TacawError) as ei:
                    C.restore_state(good)
                assert ei.value.status == t.ERR_INVALID_ARG and "another configuration" in str(ei.value)
        push_range(B, buf, SPEC, 120, SPEC.T, SPEC.Tc)
        got = outputs(B, SPEC)
    assert_identical(got, ref)


def test_pipelined_segments_checkpoint_after_drain(data):
    """With pipelined segments a finalized segment's contraction waits for the next finalize:
    checkpoints and restores are refused until tacaw_drain has launched it."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan, TacawError
    from paper_2607_02236_gb300.tacaw import ERR_STATE
    fr, buf, _ = data
    with TacawPlan([stream_config(SPEC)], precision="split_bf16") as A:
        A.set_pipelined_segments(True)
        push_range(A, buf, SPEC, 0, 128, 32)
        mid = A.save_state()
        push_range(A, buf, SPEC, 128, SPEC.T, 32)
        info = A.info()
        I = torch.full((info["I_elems"],), -1.0, device="cuda")
        S = torch.full((info["S_elems"],), -1.0, device="cuda")
        A.finalize_async(I, S, None)
        A.reset()
        for call in (A.state_size, lambda: A.restore_state(mid)):
            with pytest.raises(TacawError) as ei:
                call()
            assert ei.value.status == ERR_STATE and "tacaw_drain" in str(ei.value)
        A.drain()
        A.check_errors()
        ref = (I.cpu().numpy(), S.cpu().numpy(), None)
        A.restore_state(mid)
        push_range(A, buf, SPEC, 128, SPEC.T, 32)
        got = outputs(A, SPEC, want_psi=False)
    assert_identical(got, ref)
    check_oracle(ref, fr, SPEC)


# three partitions pushed one group per round of 32 frames; K_stage = 64 (rings of 64 frames)
ROUND_SPECS = [StreamSpec(P=2, Kx=24, Ky=24, T=160, Tc=32, n_omega=50, E_max_meV=120.0, window="hann",
                          detectors=(Detector(r_out=6.0),)),
               StreamSpec(P=3, Kx=16, Ky=20, T=96, Tc=32, n_omega=30, E_max_meV=90.0, window="gauss",
                          detectors=(Detector(r_out=4.0),), stream_id=1),
               StreamSpec(P=1, Kx=32, Ky=32, T=224, Tc=32, n_omega=70, E_max_meV=150.0, window="hann",
                          detectors=(), stream_id=2)]


def group_rounds(plan, specs, bufs, r0, r1):
    for r in range(r0, r1):
        ids, ptrs, cnt = [], [], []
        for i, s in enumerate(specs):
            t = 32 * r
            if t < s.T:
                ids.append(i)
                ptrs.append(bufs[i].data_ptr() + t * frame_bytes(s))
                cnt.append(min(32, s.T - t))
        if ids:
            plan.push_group(ids, ptrs, cnt)


@pytest.mark.parametrize("cut", [2, 3], ids=["all-rings-due", "mid-ring"])
def test_resume_grouped_partitions(cut):
    """Three partitions fed by tacaw_push_frames_group: after two push rounds every ring is full
    and its flush deferred to the next grouped launch; after three the rings are half full.  A plan
    that loads the checkpoint and takes the remaining rounds matches the uninterrupted plan bit
    for bit, and the oracle for each partition."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    frs = [frames.frames(s, 100 + i, 0, s.T) for i, s in enumerate(ROUND_SPECS)]
    bufs = [torch.from_numpy(np.ascontiguousarray(f.transpose(1, 0, 2, 3))).cuda() for f in frs]
    n_rounds = max((s.T + 31) // 32 for s in ROUND_SPECS)
    kw = dict(precision="split_bf16", k_stage=64, accum="kahan")
    res = []
    for resume in (False, True):
        with TacawPlan([stream_config(s) for s in ROUND_SPECS], **kw) as A:
            group_rounds(A, ROUND_SPECS, bufs, 0, cut)
            state = A.save_state()
            if not resume:
                group_rounds(A, ROUND_SPECS, bufs, cut, n_rounds)
                res.append((outputs(A, ROUND_SPECS[0]), [A.offsets(i) for i in range(3)]))
                continue
        with TacawPlan([stream_config(s) for s in ROUND_SPECS], **kw) as B:
            B.restore_state(state)
            group_rounds(B, ROUND_SPECS, bufs, cut, n_rounds)
            res.append((outputs(B, ROUND_SPECS[0]), [B.offsets(i) for i in range(3)]))
    (ref, offs), (got, _) = res
    assert_identical(got, ref)
    I, S, Psi = ref
    for i, s in enumerate(ROUND_SPECS):
        o = oracle.forward(frs[i], **oracle_kw(s))
        io, so = offs[i]
        n = s.P * s.Nw * s.Ky * s.Kx
        assert rel_err_peak(I[io:io + n].reshape(s.P, s.Nw, s.Ky, s.Kx), o.I) <= TOL
        assert rel_err_peak(Psi[io:io + n].reshape(s.P, s.Nw, s.Ky, s.Kx), o.Psi) <= TOL
        D = len(s.detectors)
        if D:
            assert rel_err_peak(S[so:so + s.P * D * s.Nw].reshape(s.P, D, s.Nw), o.S) <= TOL
