"""NumPy twin of the synthetic exit-wave generator (the CUDA twin is synth/csrc/synth.cu).

Model of one stream, probe p, ROI pixel k=(ix,iy), frame t (global index in the segment):

    psi[p,t,k] = psi0[p,k] + sum_m a[p,k,m] * exp(2*pi*i*(f_m*t + phi[p,k,m]))  + n[p,t,k]

* psi0: Gaussian envelope exp(-r^2/(2 sigma^2)) about the DC pixel of the full grid,
  normalised to unit norm over the full grid, times a per-(probe, pixel) random phase.
* f_m = E_m * dt / h cycles per frame, E_m ~ U(E_lo, E_hi), shared by all pixels/probes.
* phi ~ U(0,1) cycles per (probe, pixel, mode).
* a = amp*|psi0| * U(0.5,1)              (amp_law "uniform")
  a = amp*|psi0| * (0.5 + 0.5*s_m(k))    (amp_law "smooth"; s_m a seeded plane-wave cosine in [0,1])
* n: circular complex Gaussian, per-component std noise/sqrt(2).

Random numbers come from Philox4x32-10 keyed by (seed, stream_id), counters
(index, probe, purpose | mode<<8, frame).  Parameters are computed in FP64 on
both twins; the CUDA twin evaluates the sum in FP32, so the twins agree to
float rounding, not bit for bit.  Parity tests feed the oracle the frames the
GPU actually consumed.

Holds input synthesis only: none of the TACAW arithmetic.
"""
from __future__ import annotations

import numpy as np

from .philox import philox4x32_10, u01
from .workloads import H_MEV_PS, StreamSpec

PURPOSE_PSI0 = 1
PURPOSE_OMEGA = 2
PURPOSE_MODE = 3
PURPOSE_SMOOTH = 4
PURPOSE_NOISE = 5


def _key(seed: int, spec: StreamSpec):
    return (np.uint32(seed & 0xFFFFFFFF), np.uint32(0x5EED0000 ^ spec.stream_id))


def mode_energies(spec: StreamSpec, seed: int) -> np.ndarray:
    k0, k1 = _key(seed, spec)
    m = np.arange(spec.n_modes, dtype=np.uint32)
    r = philox4x32_10(m, 0, PURPOSE_OMEGA, 0, k0, k1)
    lo, hi = spec.E_modes
    return lo + (hi - lo) * u01(r[0])


def mode_cycles(spec: StreamSpec, seed: int) -> np.ndarray:
    """f_m in cycles per frame."""
    return mode_energies(spec, seed) * (spec.dt_fs * 1e-3) / H_MEV_PS


def envelope_norm(spec: StreamSpec) -> float:
    gx, gy = spec.full_grid
    x = np.arange(gx, dtype=np.float64) - gx // 2
    y = np.arange(gy, dtype=np.float64) - gy // 2
    ex = np.exp(-(x * x) / (2 * spec.sigma_env ** 2))
    ey = np.exp(-(y * y) / (2 * spec.sigma_env ** 2))
    # sum over the grid of env^2 = (sum_x ex^2) * (sum_y ey^2)
    return float(np.sqrt(np.sum(ex * ex) * np.sum(ey * ey)))


def smooth_params(spec: StreamSpec, seed: int):
    k0, k1 = _key(seed, spec)
    m = np.arange(spec.n_modes, dtype=np.uint32)
    r = philox4x32_10(m, 0, PURPOSE_SMOOTH, 0, k0, k1)
    u = np.floor(u01(r[0]) * 3.0)
    v = np.floor(u01(r[1]) * 3.0)
    chi = u01(r[2])
    return u, v, chi


def pixel_params(spec: StreamSpec, seed: int, probes, iy, ix):
    """Per-(probe, pixel) parameters on broadcastable index arrays (ROI coordinates).

    Returns psi0 (complex128), amp [..., M] (float64), phi [..., M] (cycles, float64).
    """
    k0, k1 = _key(seed, spec)
    p = np.asarray(probes, dtype=np.int64)
    iy = np.asarray(iy, dtype=np.int64)
    ix = np.asarray(ix, dtype=np.int64)
    p, iy, ix = np.broadcast_arrays(p, iy, ix)
    gx, gy = spec.full_grid
    ox, oy = spec.roi_origin
    X = ix + ox                      # full-grid coordinates
    Y = iy + oy
    pix = (Y * gx + X).astype(np.uint32)
    pu = p.astype(np.uint32)
    r = philox4x32_10(pix, pu, PURPOSE_PSI0, 0, k0, k1)
    dx = (X - gx // 2).astype(np.float64)
    dy = (Y - gy // 2).astype(np.float64)
    env = np.exp(-(dx * dx + dy * dy) / (2 * spec.sigma_env ** 2)) / envelope_norm(spec)
    psi0 = env * np.exp(2j * np.pi * u01(r[0]))
    M = spec.n_modes
    amp = np.empty(p.shape + (M,), dtype=np.float64)
    phi = np.empty(p.shape + (M,), dtype=np.float64)
    if spec.amp_law == "smooth":
        su, sv, schi = smooth_params(spec, seed)
    for m in range(M):
        rm = philox4x32_10(pix, pu, PURPOSE_MODE | (m << 8), 0, k0, k1)
        phi[..., m] = u01(rm[0])
        if spec.amp_law == "smooth":
            s = 0.5 + 0.5 * np.cos(2 * np.pi * ((su[m] * dx + sv[m] * dy) / spec.Kx + schi[m]))
        else:
            s = u01(rm[1])
        amp[..., m] = spec.amp * env * (0.5 + 0.5 * s)
    return psi0, amp, phi


def noise(spec: StreamSpec, seed: int, probes, t, iy, ix):
    k0, k1 = _key(seed, spec)
    p, t, iy, ix = np.broadcast_arrays(*(np.asarray(a, dtype=np.int64) for a in (probes, t, iy, ix)))
    gx, _ = spec.full_grid
    ox, oy = spec.roi_origin
    pix = ((iy + oy) * gx + (ix + ox)).astype(np.uint32)
    r = philox4x32_10(pix, p.astype(np.uint32), PURPOSE_NOISE, t.astype(np.uint32), k0, k1)
    rho = np.sqrt(-2.0 * np.log(u01(r[0])))
    ang = 2.0 * np.pi * u01(r[1])
    return (spec.noise / np.sqrt(2.0)) * rho * (np.cos(ang) + 1j * np.sin(ang))


def frames(spec: StreamSpec, seed: int, t0: int, n: int, probes=None, dtype=np.complex64):
    """Frames [P, n, Ky, Kx] for global frame indices t0..t0+n-1 (all ROI pixels)."""
    probes = np.arange(spec.P) if probes is None else np.asarray(probes)
    iy = np.arange(spec.Ky)[:, None]
    ix = np.arange(spec.Kx)[None, :]
    out = np.empty((len(probes), n, spec.Ky, spec.Kx), dtype=dtype)
    f = mode_cycles(spec, seed)
    for a, p in enumerate(probes):
        psi0, amp, phi = pixel_params(spec, seed, p, iy, ix)
        for b in range(n):
            t = t0 + b
            cyc = np.mod(f[None, None, :] * t + phi, 1.0)
            s = psi0 + np.sum(amp * np.exp(2j * np.pi * cyc), axis=-1)
            s = s + noise(spec, seed, p, t, iy, ix)
            out[a, b] = s
    return out


def pixel_series(spec: StreamSpec, seed: int, probe: int, iy, ix, t0: int = 0, n: int = None,
                 dtype=np.complex64):
    """Time series [n, len(iy)] for selected pixels of one probe (for sampled checks)."""
    n = spec.T - t0 if n is None else n
    iy = np.asarray(iy)
    ix = np.asarray(ix)
    psi0, amp, phi = pixel_params(spec, seed, probe, iy, ix)
    f = mode_cycles(spec, seed)
    t = (t0 + np.arange(n))[:, None]
    out = np.empty((n, iy.size), dtype=np.complex128)
    for j in range(iy.size):
        cyc = np.mod(f[None, :] * t + phi[j][None, :], 1.0)
        out[:, j] = psi0[j] + np.sum(amp[j][None, :] * np.exp(2j * np.pi * cyc), axis=-1)
        out[:, j] += noise(spec, seed, probe, t[:, 0], iy[j], ix[j])
    return out.astype(dtype)
