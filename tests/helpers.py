"""Shared helpers of the GPU tests: descriptors from synthetic specs, GPU runs, oracle runs."""
from __future__ import annotations

import numpy as np

import oracle
from synth import StreamSpec


def stream_config(spec: StreamSpec, P: int = None):
    """Frame-major push layout [t][p][Gy][Gx] with the ROI at roi_origin of the full grid."""
    from paper_2607_02236_gb300 import StreamConfig, DetectorConfig
    P = spec.P if P is None else P
    gx, gy = spec.full_grid
    rx, ry = spec.roi_origin
    return StreamConfig(
        n_probes=P, kx=spec.Kx, ky=spec.Ky, T=spec.T, dt_fs=spec.dt_fs,
        pitch_row=gx, pitch_frame=P * gx * gy, pitch_probe=gx * gy, roi_x0=rx, roi_y0=ry,
        E_meV=None if spec.fft_bins else [float(e) for e in spec.energies_meV()], fft_bins=spec.fft_bins,
        window=spec.window, window_param=spec.window_sigma() if spec.window == "gauss" else spec.window_param,
        subtract_mean=spec.subtract_mean, bose_T_K=spec.bose_T_K,
        detectors=[DetectorConfig(d.kind, d.cx, d.cy, d.r_in, d.r_out) for d in spec.detectors])


def oracle_kw(spec: StreamSpec):
    kw = dict(window_kind=spec.window,
              window_param=spec.window_sigma() if spec.window == "gauss" else spec.window_param,
              dt_fs=spec.dt_fs, subtract_mean=spec.subtract_mean, bose_T_K=spec.bose_T_K,
              detectors=list(spec.detectors))
    if spec.fft_bins:
        kw["fft_bins"] = spec.fft_bins
    else:
        kw["E_meV"] = spec.energies_meV()
    return kw


def run_gpu(spec: StreamSpec, frames: np.ndarray, precision: str, pushes=None, k_stage: int = 0,
            accum: str = "kahan", want_psi: bool = False, **plan_kw):
    """frames: [P, T, Ky, Kx] complex64 host array (ROI only). Returns I, S, Psi (numpy)."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    P, T, Ky, Kx = frames.shape
    assert spec.full_grid == (Kx, Ky)
    buf = torch.from_numpy(np.ascontiguousarray(frames.transpose(1, 0, 2, 3))).to("cuda")
    pushes = pushes or [spec.Tc] * (T // spec.Tc) + ([T % spec.Tc] if T % spec.Tc else [])
    assert sum(pushes) == T
    Nw = spec.Nw
    D = len(spec.detectors)
    I = torch.empty(P * Nw * Ky * Kx, dtype=torch.float32, device="cuda")
    S = torch.empty(max(1, P * D * Nw), dtype=torch.float32, device="cuda")
    Psi = torch.empty(P * Nw * Ky * Kx, dtype=torch.complex64, device="cuda") if want_psi else None
    with TacawPlan([stream_config(spec)], precision=precision, accum=accum, k_stage=k_stage, **plan_kw) as plan:
        t = 0
        fb = P * Ky * Kx * 8
        for n in pushes:
            plan.push(0, buf.data_ptr() + t * fb, n)
            t += n
        plan.finalize(I, S if D else None, Psi)
        info = plan.info()
    torch.cuda.synchronize()
    out = dict(I=I.cpu().numpy().reshape(P, Nw, Ky, Kx), S=S.cpu().numpy()[:P * D * Nw].reshape(P, D, Nw),
               info=info)
    if want_psi:
        out["Psi"] = Psi.cpu().numpy().reshape(P, Nw, Ky, Kx)
    return out


def rel_err_peak(got, ref):
    """max |got - ref| / max |ref|"""
    g = np.asarray(got)
    g = g.astype(np.complex128) if np.iscomplexobj(g) else g.astype(np.float64)
    return float(np.max(np.abs(g - ref)) / max(np.max(np.abs(ref)), 1e-300))
