"""Frames pushed from pinned host memory: the push kernels read them where they are (no
separate host-to-device copy) and the result matches the FP64 oracle exactly as a push from
device memory does.  Memory the device cannot read (pageable host memory) and in-place
plans given host memory are refused before any work is enqueued."""
import numpy as np
import pytest

import oracle
from synth import Detector, StreamSpec, frames
from tests.helpers import oracle_kw, rel_err_peak, stream_config
from tests.test_gpu_parity import TOL_FP32, TOL_SPLIT

pytestmark = pytest.mark.gpu

SPEC = StreamSpec(P=2, Kx=48, Ky=40, T=136, Tc=24, n_omega=90, E_max_meV=120.0, window="hann", n_modes=6,
                  noise=1e-3, detectors=(Detector("circular", 0, 0, -1, 6.0),))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


def _run(precision, fr_host_pinned, pushes, **kw):
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    s = SPEC
    fb = s.P * s.Ky * s.Kx * 8
    I = torch.empty(s.P * s.Nw * s.Ky * s.Kx, dtype=torch.float32, device="cuda")
    S = torch.empty(s.P * s.Nw, dtype=torch.float32, device="cuda")
    with TacawPlan([stream_config(s)], precision=precision, **kw) as plan:
        t = 0
        for n in pushes:
            plan.push(0, fr_host_pinned.data_ptr() + t * fb, n, torch.cuda.current_stream())
            t += n
        plan.finalize(I, S, None, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return I.cpu().numpy().reshape(s.P, s.Nw, s.Ky, s.Kx), S.cpu().numpy().reshape(s.P, 1, s.Nw)


@pytest.mark.parametrize("precision,k_stage", [("split_bf16", 0), ("split_bf16", 48), ("fp32", 0),
                                               ("split_fp16", 0)])
def test_push_from_pinned_host_memory(precision, k_stage):
    import torch
    fr = frames.frames(SPEC, 21, 0, SPEC.T)                         # [P, T, Ky, Kx]
    host = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).pin_memory()
    I, S = _run(precision, host, [24, 40, 8, 64], k_stage=k_stage)
    ref = oracle.forward(fr, **oracle_kw(SPEC))
    tol = TOL_FP32 if precision == "fp32" else TOL_SPLIT
    assert rel_err_peak(I, ref.I) <= tol
    assert rel_err_peak(S, ref.S) <= tol


def test_unreadable_or_in_place_host_frames_are_refused():
    import torch
    from paper_2607_02236_gb300 import TacawPlan, TacawError
    n = SPEC.P * SPEC.Kx * SPEC.Ky
    pageable = np.zeros(SPEC.T * n, dtype=np.complex64)
    pinned = torch.zeros(SPEC.T * n, dtype=torch.complex64).pin_memory()
    with TacawPlan([stream_config(SPEC)], precision="split_bf16") as plan:
        with pytest.raises(TacawError, match="INVALID_ARG"):
            plan.push(0, pageable.ctypes.data, 8)
        assert plan.info()["kernel_launches"] == 0
        plan.push(0, pinned.data_ptr(), SPEC.T)                     # accepted afterwards
    with TacawPlan([stream_config(SPEC)], precision="split_bf16", frames_in_place=True) as plan:
        with pytest.raises(TacawError, match="INVALID_ARG"):
            plan.push(0, pinned.data_ptr(), 8)


def test_pageable_outputs_and_gradient_buffers_are_refused():
    """finalize's outputs and backward's buffers are written by kernels: pageable host memory
    is refused before any work is enqueued, device memory then completes the same calls."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan, TacawError
    s = SPEC
    n = s.P * s.Kx * s.Ky
    fr = torch.zeros(s.T * n, dtype=torch.complex64, device="cuda")
    I_host = np.zeros(s.P * s.Nw * s.Kx * s.Ky, dtype=np.float32)
    grad_host = np.zeros(s.T * n, dtype=np.complex64)
    dLdS = torch.ones(s.P * s.Nw, dtype=torch.float32, device="cuda")
    with TacawPlan([stream_config(s)], precision="fp32") as plan:
        plan.push(0, fr, s.T)
        with pytest.raises(TacawError, match="INVALID_ARG"):
            plan.finalize(I_host.ctypes.data)
        I = torch.empty(I_host.size, dtype=torch.float32, device="cuda")
        plan.finalize(I)
        with pytest.raises(TacawError, match="INVALID_ARG"):
            plan.backward(0, dLdS, fr, grad_host.ctypes.data)
        grad = torch.empty_like(fr)
        plan.backward(0, dLdS, fr, grad)
    torch.cuda.synchronize()
    assert float(I.abs().max()) == 0.0 and float(grad.abs().max()) == 0.0
