"""Device-side waits that run out, tested without a GPU fault.

Every wait of the tensor-core contraction kernels on a pipeline event is bounded by the GPU's
global timer.  tacaw_set_wait_limit_ns shortens that bound; at 1 us it is far shorter than the
work a tile takes (tens of microseconds of MMAs at T = 1024), so the epilogue warps' wait for a
finished accumulator chunk runs out deterministically.  The kernel then stops: its copies in
flight are waited for, its issued MMAs complete and its tensor memory is freed before it exits.
The host reads the error word: finalize returns TACAW_ERR_TIMEOUT and the plan is poisoned.
A fresh plan on the same device then matches the FP64 oracle, so the context stayed usable.
The tensor-core adjoint runs the same kernel: its backward reports the timeout the same way.
"""
import numpy as np
import pytest

import oracle
from synth import Detector, StreamSpec, frames
from tests.helpers import oracle_kw, rel_err_peak, run_gpu, stream_config

pytestmark = pytest.mark.gpu

SPEC = StreamSpec(P=2, Kx=64, Ky=64, T=1024, Tc=256, n_omega=100, E_max_meV=120.0, window="hann", n_modes=6,
                  detectors=(Detector("circular", 0, 0, -1, 8.0),))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


@pytest.mark.parametrize("in_place", [False, True], ids=["staged", "in_place"])
def test_wait_limit_reports_timeout_and_poisons_the_plan(in_place):
    import torch
    from paper_2607_02236_gb300 import TacawPlan, TacawError
    from paper_2607_02236_gb300.tacaw import ERR_STATE, ERR_TIMEOUT
    fr = frames.frames(SPEC, 5, 0, SPEC.T)
    buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).cuda()      # [T][P][K][K]
    P, K, Nw = SPEC.P, SPEC.Kx, SPEC.Nw
    I = torch.zeros(P * Nw * K * K, device="cuda")
    S = torch.zeros(P * Nw, device="cuda")
    fb = P * K * K * 8
    plan = TacawPlan([stream_config(SPEC)], precision="split_bf16", frames_in_place=in_place)
    try:
        plan.set_wait_limit_ns(1000)
        for t in range(0, SPEC.T, SPEC.Tc):
            plan.push(0, buf.data_ptr() + t * fb, SPEC.Tc)
        with pytest.raises(TacawError) as ei:
            plan.finalize(I, S)
        assert ei.value.status == ERR_TIMEOUT, str(ei.value)
        assert "timed out" in str(ei.value)
        # poisoned: every later call but destroy is refused
        with pytest.raises(TacawError) as ei:
            plan.reset()
        assert ei.value.status == ERR_STATE and "poisoned" in str(ei.value)
    finally:
        plan.close()
    torch.cuda.synchronize()
    # the context is intact: a fresh plan on the same device gives the oracle's result
    out = run_gpu(SPEC, fr, "split_bf16", frames_in_place=in_place)
    ref = oracle.forward(fr, **oracle_kw(SPEC))
    assert rel_err_peak(out["I"], ref.I) <= 1e-5
    assert rel_err_peak(out["S"], ref.S) <= 1e-5


def test_default_limit_restored():
    """Limit 0 restores the default: a plan given a short limit and then 0 runs normally."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    fr = frames.frames(SPEC, 6, 0, SPEC.T)
    buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).cuda()
    P, K, Nw = SPEC.P, SPEC.Kx, SPEC.Nw
    I = torch.zeros(P * Nw * K * K, device="cuda")
    with TacawPlan([stream_config(SPEC)], precision="split_bf16") as plan:
        plan.set_wait_limit_ns(1000)
        plan.set_wait_limit_ns(0)
        plan.push(0, buf, SPEC.T)
        plan.finalize(I)
    torch.cuda.synchronize()
    ref = oracle.forward(fr, **oracle_kw(SPEC))
    assert rel_err_peak(I.cpu().numpy().reshape(ref.I.shape), ref.I) <= 1e-5


def test_adjoint_wait_limit_reports_timeout():
    """tacaw_backward on the tensor cores with a 1 us wait limit: its Psi contraction (32 staging
    blocks a tile) runs out of a wait, the call returns TACAW_ERR_TIMEOUT and poisons the plan;
    a fresh plan's backward then matches the oracle's gradient."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan, TacawError
    from paper_2607_02236_gb300.tacaw import ERR_STATE, ERR_TIMEOUT
    fr = frames.frames(SPEC, 7, 0, SPEC.T)
    buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).cuda()      # [T][P][K][K]
    c = np.random.default_rng(3).standard_normal((SPEC.P, 1, SPEC.Nw))
    dLdS = torch.tensor(c, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(buf)
    plan = TacawPlan([stream_config(SPEC)], precision="split_bf16")
    try:
        plan.set_wait_limit_ns(1000)
        with pytest.raises(TacawError) as ei:
            plan.backward(0, dLdS, buf, grad)
        assert ei.value.status == ERR_TIMEOUT, str(ei.value)
        with pytest.raises(TacawError) as ei:
            plan.backward(0, dLdS, buf, grad)
        assert ei.value.status == ERR_STATE and "poisoned" in str(ei.value)
    finally:
        plan.close()
    torch.cuda.synchronize()
    with TacawPlan([stream_config(SPEC)], precision="split_bf16") as plan:
        plan.backward(0, dLdS, buf, grad)
    g = grad.cpu().numpy().transpose(1, 0, 2, 3)
    ref = oracle.gradient(fr, c, **oracle_kw(SPEC))
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) <= 1e-4
