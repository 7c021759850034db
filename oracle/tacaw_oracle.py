"""FP64 CPU oracle for the streaming TACAW time->energy stage.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this module.  The CUDA
library never calls it and shares no code with it.

What is computed (per stream, probe p, ROI pixel k), all in float64:

  mu[k]     = (1/T) sum_n psi[n,k]                   (only if subtract_mean; the
                                                      elastic, time-mean part)
  y[n,k]    = w_n * (psi[n,k] - mu[k])               (window, Sec. II.B "Welch
                                                      method", Sec. III.A)
  theta_jn  = 2*pi*frac(c_j * n),  c_j = E_j*dt/h   (time->energy Fourier kernel;
                                                      energy scale of App. B, eps=h/(2 tau))
  Psi[k,j]  = sum_n y[n,k] * exp(-i theta_jn)        (the Fourier transform of Eq. 1)
  I[k,j]    = B(E_j) * |Psi[k,j]|^2,  B(E) = beta E / (1 - exp(-beta E))   (Eq. 1)
  S[d,j]    = sum_k M_d(k) * I[k,j]                  (DetectorSet apertures, Sec. II.B)

Welch averaging (Sec. II.B, "Welch method: trajectory chunk overlap & windowing" and the
1/N average of "Processing of a batch"): segments of L frames start at s_0 = 0 and
s_{n+1} = s_n + stride (stride = L // nu for the overlap nu), N = (n_frames - L) // stride + 1
of them; each is a segment of the definition above (its own mean, the window over its L
frames, phases counted from its first frame) and

  I_welch = (1/N) sum_n I_n,   S_welch = (1/N) sum_n S_n

and, for a real loss L = sum_{p,d,j} (dL/dS)[p,d,j] * S[p,d,j], the gradient in
PyTorch's convention for real losses of complex inputs, g = dL/dRe(psi) +
i dL/dIm(psi) = 2 dL/dconj(psi):

  G[k,j] = B(E_j) * sum_d (dL/dS)[d,j] M_d(k) * Psi[k,j]
  A[n,k] = sum_j exp(+i theta_jn) G[k,j]
  g[n,k] = 2 * ( w_n A[n,k] - (1/T) sum_n' w_n' A[n',k] )   (second term only with mean subtraction)

Readings of points the paper leaves open (each also listed in the design notes):
  * the mean is over the whole segment (the paper's "chunk" of L snapshots);
  * windows are scipy's periodic (fftbins=True) forms, the paper pointing to scipy
    for their definitions (App. A);
  * the kernel sign is exp(-i omega t), E > 0 is energy loss;
  * no normalisation: raw |Psi|^2 (the paper's per-voxel normalisation is not
    recoverable from its text);
  * the DC pixel of a Kx x Ky ROI is (Kx//2, Ky//2); a pixel is inside a circular
    aperture when its squared distance to the centre is <= r^2, inside an annular one
    when r_in^2 < d^2 <= r_out^2.

Every function here is pinned by tests/test_oracle_pins.py against something
other than itself (numpy.fft, scipy.signal windows, closed forms, brute force
in C with long double, finite differences, torch autograd).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

H_MEV_PS = 4.135667696          # Planck constant in meV*ps
KB_MEV_PER_K = 0.08617333262    # Boltzmann constant in meV/K


# ----------------------------------------------------------------------------------------------
# Windows (Sec. III.A: rectangular = Tukey alpha 0, Hann = Tukey alpha 1; App. A: scipy forms)
# ----------------------------------------------------------------------------------------------
def window(kind: str, T: int, param: float = 0.0) -> np.ndarray:
    """Periodic window of length T in float64.

    rect:  w_n = 1
    hann:  w_n = 1/2 - 1/2 cos(2 pi n / T)
    gauss: w_n = exp(-1/2 ((n - T/2)/sigma)^2), sigma = param (default T/6)
    tukey: cosine tapers of total fractional width alpha = param on a flat top
           (periodic form: the symmetric window of length T+1 with its last sample dropped)
    blackmanharris: 4-term cosine sum (Harris 1978), a = 0.35875, 0.48829, 0.14128, 0.01168
    kaiser: I0(beta sqrt(1 - (2n/T - 1)^2)) / I0(beta), beta = param (App. A: 3 pi, 5 pi)
    chebwin: Dolph-Chebyshev with side lobes param dB down (App. A: 100 dB)
    The last three are App. A's "more aggressive" windows, in scipy's periodic forms (the
    symmetric window of length T+1 without its last sample).
    T = 1 gives [1] for every kind (scipy's convention for length-1 windows).
    """
    n = np.arange(T, dtype=np.float64)
    if T == 1:
        return np.ones(1)  # scipy's convention: every length-1 window is [1]
    if kind == "rect":
        return np.ones(T)
    if kind == "hann":
        return 0.5 - 0.5 * np.cos(2.0 * np.pi * n / T)
    if kind == "gauss":
        sigma = param if param > 0 else T / 6.0
        return np.exp(-0.5 * ((n - T / 2.0) / sigma) ** 2)
    if kind == "tukey":
        alpha = float(param)
        if alpha <= 0:
            return np.ones(T)
        if alpha >= 1:
            return window("hann", T)
        L = T  # symmetric window of length T+1 spans indices 0..T
        w = np.ones(T)
        edge = alpha * L / 2.0
        for i in range(T):
            if i < edge:
                w[i] = 0.5 * (1 - np.cos(np.pi * i / edge))
            elif i > L - edge:
                w[i] = 0.5 * (1 - np.cos(np.pi * (L - i) / edge))
        return w
    if kind == "blackmanharris":
        a = (0.35875, 0.48829, 0.14128, 0.01168)
        x = 2.0 * np.pi * n / T
        return a[0] - a[1] * np.cos(x) + a[2] * np.cos(2 * x) - a[3] * np.cos(3 * x)
    if kind == "kaiser":
        beta = float(param)
        r = np.clip(1.0 - (2.0 * n / T - 1.0) ** 2, 0.0, None)
        return _bessel_i0(beta * np.sqrt(r)) / _bessel_i0(np.array([beta]))[0]
    if kind == "chebwin":
        return _dolph_chebyshev(T + 1, float(param))[:T]
    raise ValueError(f"unknown window {kind!r}")


def _bessel_i0(x) -> np.ndarray:
    """Modified Bessel function I0 by its power series sum_k ((x/2)^k / k!)^2 (x <= ~50)."""
    x = np.asarray(x, dtype=np.float64)
    term = np.ones_like(x)
    total = np.ones_like(x)
    q = (x / 2.0) ** 2
    for k in range(1, 200):
        term = term * q / (k * k)
        total = total + term
        if np.all(term <= 1e-18 * total):
            break
    return total


def _chebyshev_t(order: int, x) -> np.ndarray:
    """Chebyshev polynomial T_order(x) for real x (cos / cosh forms)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(order * np.arccos(x[inside]))
    big = x > 1.0
    out[big] = np.cosh(order * np.arccosh(x[big]))
    neg = x < -1.0
    out[neg] = (-1.0) ** order * np.cosh(order * np.arccosh(-x[neg]))
    return out


def _dolph_chebyshev(M: int, at_db: float) -> np.ndarray:
    """Symmetric Dolph-Chebyshev window of M taps, side lobes at_db below the main lobe: its
    frequency response is T_{M-1}(x0 cos(theta/2)) with T_{M-1}(x0) = 10^(at/20); the taps are
    the inverse DFT of M samples of that response about the window's centre, scaled to max 1."""
    if M == 1:
        return np.ones(1)
    r = 10.0 ** (at_db / 20.0)
    x0 = np.cosh(np.arccosh(r) / (M - 1))
    k = np.arange(M)
    W = _chebyshev_t(M - 1, x0 * np.cos(np.pi * k / M))
    n = np.arange(M)[:, None]
    w = np.real(np.exp(2j * np.pi * k[None, :] * (n - (M - 1) / 2.0) / M) @ W) / M
    return w / np.max(w)


# ----------------------------------------------------------------------------------------------
# Energy grid and Fourier kernel (App. B: energies up to eps = h/(2 tau); resolution h/(L tau))
# ----------------------------------------------------------------------------------------------
def cycles_per_frame(E_meV, dt_fs: float) -> np.ndarray:
    """c_j = E_j * dt / h (cycles per frame)."""
    return np.asarray(E_meV, dtype=np.float64) * (dt_fs * 1e-3) / H_MEV_PS


def fft_energies(T: int, dt_fs: float, n: int) -> np.ndarray:
    """First n bins of the T-point time FFT: E_j = j * h / (T dt)."""
    return np.arange(n, dtype=np.float64) * H_MEV_PS / (T * dt_fs * 1e-3)


def phase(T: int, *, E_meV=None, dt_fs=None, fft_bins: int = 0) -> np.ndarray:
    """theta[n, j] in radians.

    FFT grid (fft_bins > 0): exact integer form 2 pi ((j n) mod T) / T.
    Otherwise: 2 pi frac(c_j n) with the fractional part taken in FP64.
    """
    n = np.arange(T, dtype=np.int64)[:, None]
    if fft_bins:
        j = np.arange(fft_bins, dtype=np.int64)[None, :]
        return 2.0 * np.pi * ((j * n) % T).astype(np.float64) / T
    c = cycles_per_frame(E_meV, dt_fs)[None, :]
    x = c * n.astype(np.float64)
    return 2.0 * np.pi * (x - np.floor(x))


def bose(E_meV, T_K: float) -> np.ndarray:
    """Quantum-statistics factor of Eq. 1: beta E / (1 - exp(-beta E)); 1 at E = 0; 1 if T_K = 0 (off)."""
    E = np.asarray(E_meV, dtype=np.float64)
    if T_K <= 0:
        return np.ones_like(E)
    x = E / (KB_MEV_PER_K * T_K)
    out = np.ones_like(x)
    nz = x != 0
    out[nz] = x[nz] / (-np.expm1(-x[nz]))
    return out


# ----------------------------------------------------------------------------------------------
# Detector apertures (Sec. II.B DetectorSet: circular and annular with arbitrary centre and radii)
# ----------------------------------------------------------------------------------------------
def detector_masks(Kx: int, Ky: int, detectors: Sequence) -> np.ndarray:
    """M[d, iy, ix] in {0, 1}; centres are offsets from the DC pixel (Kx//2, Ky//2)."""
    iy = np.arange(Ky, dtype=np.float64)[:, None]
    ix = np.arange(Kx, dtype=np.float64)[None, :]
    out = np.zeros((len(detectors), Ky, Kx))
    for d, det in enumerate(detectors):
        dx = ix - (Kx // 2 + det.cx)
        dy = iy - (Ky // 2 + det.cy)
        r2 = dx * dx + dy * dy
        inside = r2 <= det.r_out * det.r_out
        if det.kind == "annular" and det.r_in >= 0:
            inside &= r2 > det.r_in * det.r_in
        out[d] = inside
    return out


# ----------------------------------------------------------------------------------------------
# Forward definition
# ----------------------------------------------------------------------------------------------
@dataclass
class Result:
    mu: np.ndarray        # [P, Ky, Kx] complex128
    Psi: np.ndarray       # [P, Nw, Ky, Kx] complex128
    I: np.ndarray         # [P, Nw, Ky, Kx] float64
    S: np.ndarray         # [P, D, Nw] float64


def forward(psi, *, window_kind="hann", window_param=0.0, E_meV=None, dt_fs=5.0, fft_bins=0,
            subtract_mean=True, bose_T_K=0.0, detectors=()) -> Result:
    """psi: [P, T, Ky, Kx] complex (upcast to complex128). Returns the Result of the definition above."""
    psi = np.asarray(psi).astype(np.complex128)
    P, T, Ky, Kx = psi.shape
    w = window(window_kind, T, window_param)
    if fft_bins:
        E = fft_energies(T, dt_fs, fft_bins)
    else:
        E = np.asarray(E_meV, dtype=np.float64)
    theta = phase(T, E_meV=E, dt_fs=dt_fs, fft_bins=fft_bins)        # [T, Nw]
    F = np.exp(-1j * theta)                                            # [T, Nw]
    x = psi.reshape(P, T, Ky * Kx)
    mu = x.mean(axis=1) if subtract_mean else np.zeros((P, Ky * Kx), dtype=np.complex128)
    y = w[None, :, None] * (x - mu[:, None, :])                        # [P, T, K]
    Psi = np.einsum("ptk,tj->pjk", y, F, optimize=True)                # [P, Nw, K]
    B = bose(E, bose_T_K)
    I = (Psi.real ** 2 + Psi.imag ** 2) * B[None, :, None]
    M = detector_masks(Kx, Ky, detectors).reshape(len(detectors), Ky * Kx)
    S = np.einsum("pjk,dk->pdj", I, M) if len(detectors) else np.zeros((P, 0, len(E)))
    return Result(mu.reshape(P, Ky, Kx), Psi.reshape(P, -1, Ky, Kx), I.reshape(P, -1, Ky, Kx), S)


def welch_segments(n_frames: int, L: int, stride: int) -> np.ndarray:
    """Start frames of the Welch segments: 0, stride, 2*stride, ... while a whole segment fits."""
    if L < 1 or stride < 1 or n_frames < L:
        return np.zeros(0, dtype=np.int64)
    return np.arange((n_frames - L) // stride + 1, dtype=np.int64) * stride


def welch_stride(L: int, nu: float) -> int:
    """Frames between segment starts for the overlap parameter nu (remainder-less division)."""
    return int(L // nu)


def welch_forward(psi, L: int, stride: int, skip_init: int = 0, **kw) -> Result:
    """Welch average of the segments of psi [P, n_frames, Ky, Kx] (see the module header).
    The first `skip_init` frames are dropped before the first segment (the configuration's
    `trajectory_chunks_skip_init`, App. listing, read as a frame count).
    Result.I and Result.S are the averages; mu and Psi are those of the last segment."""
    psi = np.asarray(psi)[:, skip_init:]
    starts = welch_segments(psi.shape[1], L, stride)
    if len(starts) == 0:
        raise ValueError("no whole segment of L frames")
    I = S = None
    for s0 in starts:
        r = forward(psi[:, s0:s0 + L], **kw)
        I = r.I if I is None else I + r.I
        S = r.S if S is None else S + r.S
    N = float(len(starts))
    return Result(r.mu, r.Psi, I / N, S / N)


def welch_gradient(psi, dLdS, L: int, stride: int, skip_init: int = 0, **kw) -> np.ndarray:
    """Gradient of sum dLdS * S_welch, S_welch = (1/N) sum_n S_n (welch_forward), with respect
    to the whole push sequence psi [P, n_frames, Ky, Kx]: each segment's gradient (gradient())
    weighted 1/N at its frames, summed where segments overlap, zero on dropped frames."""
    psi = np.asarray(psi)
    starts = welch_segments(psi.shape[1] - skip_init, L, stride) + skip_init
    if len(starts) == 0:
        raise ValueError("no whole segment of L frames")
    g = np.zeros(psi.shape, dtype=np.complex128)
    for s0 in starts:
        g[:, s0:s0 + L] += gradient(psi[:, s0:s0 + L], dLdS, **kw) / len(starts)
    return g


def gradient(psi, dLdS, *, window_kind="hann", window_param=0.0, E_meV=None, dt_fs=5.0,
             fft_bins=0, subtract_mean=True, bose_T_K=0.0, detectors=()) -> np.ndarray:
    """g = 2 dL/dconj(psi) for L = sum dLdS * S.  psi [P,T,Ky,Kx], dLdS [P,D,Nw]. Returns [P,T,Ky,Kx]."""
    psi = np.asarray(psi).astype(np.complex128)
    P, T, Ky, Kx = psi.shape
    r = forward(psi, window_kind=window_kind, window_param=window_param, E_meV=E_meV, dt_fs=dt_fs,
                fft_bins=fft_bins, subtract_mean=subtract_mean, bose_T_K=bose_T_K,
                detectors=detectors)
    w = window(window_kind, T, window_param)
    E = fft_energies(T, dt_fs, fft_bins) if fft_bins else np.asarray(E_meV, dtype=np.float64)
    theta = phase(T, E_meV=E, dt_fs=dt_fs, fft_bins=fft_bins)         # [T, Nw]
    B = bose(E, bose_T_K)
    M = detector_masks(Kx, Ky, detectors).reshape(len(detectors), Ky * Kx)
    Psi = r.Psi.reshape(P, len(E), Ky * Kx)
    coef = np.einsum("pdj,dk->pjk", np.asarray(dLdS, dtype=np.float64), M) * B[None, :, None]
    G = coef * Psi                                                     # [P, Nw, K]
    A = np.einsum("tj,pjk->ptk", np.exp(1j * theta), G, optimize=True)  # [P, T, K]
    g = w[None, :, None] * A
    if subtract_mean:
        g = g - g.mean(axis=1, keepdims=True)
    return (2.0 * g).reshape(P, T, Ky, Kx)


def loss(psi, dLdS, **kw) -> float:
    """L = sum dLdS * S for the forward above."""
    r = forward(psi, **kw)
    return float(np.sum(np.asarray(dLdS) * r.S))


def forward_pixels(series, *, window_kind="hann", window_param=0.0, E_meV=None, dt_fs=5.0,
                   fft_bins=0, subtract_mean=True, bose_T_K=0.0):
    """Psi and I for independent pixel time series: series [T, n] -> (Psi [Nw, n], I [Nw, n]).

    Pixels are independent in the definition, so sampled outputs of a large run can be
    checked one pixel at a time.
    """
    x = np.asarray(series).astype(np.complex128)
    T = x.shape[0]
    w = window(window_kind, T, window_param)
    E = fft_energies(T, dt_fs, fft_bins) if fft_bins else np.asarray(E_meV, dtype=np.float64)
    F = np.exp(-1j * phase(T, E_meV=E, dt_fs=dt_fs, fft_bins=fft_bins))
    mu = x.mean(axis=0, keepdims=True) if subtract_mean else 0.0
    y = w[:, None] * (x - mu)
    Psi = F.T @ y
    I = (Psi.real ** 2 + Psi.imag ** 2) * bose(E, bose_T_K)[:, None]
    return Psi, I


def gradient_pixels(series, dLdS, mask_w, *, window_kind="hann", window_param=0.0, E_meV=None, dt_fs=5.0,
                    fft_bins=0, subtract_mean=True, bose_T_K=0.0):
    """The gradient above for independent pixel series: series [T, n], dLdS [D, Nw] (one probe),
    mask_w [n, D] = M_d(k_i).  Returns g [T, n] = 2 dL/dconj(psi) at those pixels."""
    x = np.asarray(series).astype(np.complex128)
    T = x.shape[0]
    E = fft_energies(T, dt_fs, fft_bins) if fft_bins else np.asarray(E_meV, dtype=np.float64)
    theta = phase(T, E_meV=E, dt_fs=dt_fs, fft_bins=fft_bins)        # [T, Nw]
    Psi, _ = forward_pixels(x, window_kind=window_kind, window_param=window_param, E_meV=E, dt_fs=dt_fs,
                            fft_bins=fft_bins, subtract_mean=subtract_mean, bose_T_K=0.0)   # [Nw, n]
    coef = np.asarray(dLdS, dtype=np.float64).T @ np.asarray(mask_w, dtype=np.float64).T     # [Nw, n]
    G = coef * bose(E, bose_T_K)[:, None] * Psi
    A = np.exp(1j * theta) @ G                                          # [T, n]
    g = window(window_kind, T, window_param)[:, None] * A
    if subtract_mean:
        g = g - g.mean(axis=0, keepdims=True)
    return 2.0 * g


def loss_pixels(series, dLdS, mask_w, *, bose_T_K=0.0, **kw):
    """sum over the given pixels of sum_{d,j} dLdS[d,j] M_d(k) I[k,j] (the pixels' share of L)."""
    x = np.asarray(series).astype(np.complex128)
    E = fft_energies(x.shape[0], kw.get("dt_fs", 5.0), kw["fft_bins"]) if kw.get("fft_bins") else \
        np.asarray(kw["E_meV"], dtype=np.float64)
    _, I = forward_pixels(x, bose_T_K=bose_T_K, **kw)
    coef = np.asarray(dLdS, dtype=np.float64).T @ np.asarray(mask_w, dtype=np.float64).T
    return float(np.sum(coef * I))
