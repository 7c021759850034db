"""torch.autograd.Function over the C ABI: spectra S[p, d, E] from a segment of frames,
with the hand-written adjoint (tacaw_backward) as its backward.

Gradient convention: PyTorch's for real losses of complex inputs,
grad = dL/dRe(psi) + i dL/dIm(psi), which is what tacaw_backward returns.
"""
from __future__ import annotations

import torch

from .tacaw import TacawPlan


def _dims(plan: TacawPlan, sid: int):
    s = plan.streams[sid]
    nw = int(s.fft_bins) if s.fft_bins else len(s.E_meV)
    return s, nw, len(s.detectors)


class TacawSpectrum(torch.autograd.Function):
    """S = TacawSpectrum.apply(frames, plan, stream_id, frames_per_push).

    frames: complex64 CUDA tensor holding the whole push sequence of `stream_id` in the
    pushed layout of the plan's stream descriptor (pitches): one segment, or with skip_init /
    Welch averaging skip_init + (N - 1) * stride + T frames.  The plan must have a single stream
    (finalize completes every stream).  Returns S as a float32 tensor [P, D, Nw].
    """

    @staticmethod
    def forward(ctx, frames, plan: TacawPlan, stream_id: int = 0, frames_per_push: int = 0):
        if len(plan.streams) != 1:
            raise ValueError("TacawSpectrum needs a single-stream plan")
        s, nw, D = _dims(plan, stream_id)
        cs = torch.cuda.current_stream()
        plan.reset(cs)
        n_seg = max(1, int(s.welch_segments))
        total = int(s.skip_init) + (n_seg - 1) * (int(s.welch_stride) or s.T) + s.T
        chunk = frames_per_push or total
        base = frames.data_ptr()
        for t0 in range(0, total, chunk):
            plan.push(stream_id, base + t0 * s.pitch_frame * 8, min(chunk, total - t0), cs)
        info = plan.info()
        I = torch.empty(info["I_elems"], dtype=torch.float32, device=frames.device)
        S = torch.empty(max(1, info["S_elems"]), dtype=torch.float32, device=frames.device)
        plan.finalize(I, S, None, cs)
        _, s_off = plan.offsets(stream_id)
        ctx.plan, ctx.sid = plan, stream_id
        ctx.save_for_backward(frames)
        return S[s_off:s_off + s.n_probes * D * nw].view(s.n_probes, D, nw)

    @staticmethod
    def backward(ctx, gS):
        (frames,) = ctx.saved_tensors
        grad = torch.zeros_like(frames)
        ctx.plan.backward(ctx.sid, gS.contiguous().to(torch.float32), frames, grad, torch.cuda.current_stream())
        return grad, None, None, None


def spectrum(frames, plan: TacawPlan, stream_id: int = 0, frames_per_push: int = 0):
    return TacawSpectrum.apply(frames, plan, stream_id, frames_per_push)
