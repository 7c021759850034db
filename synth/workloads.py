"""Synthetic workload shapes standing in for the paper's TiO2 exit-wave streams.

The paper's data (MD trajectories, multislice exit waves) are not available,
so every input is synthetic and seeded.  The shapes follow the paper's
workloads: k-ROIs of a few hundred pixels per side (Sec. III.A uses 383^2),
16x16 scan grids (Sec. IV), energies up to ~120-150 meV (the +-30 THz ROI of
Sec. III.A), chunk lengths of hundreds to thousands of snapshots.

A workload is a list of streams (one per supercell partition).  Each stream has
P probes, a Ky x Kx k-ROI, T frames per segment pushed Tc at a time, a frame
interval dt, an energy grid and a window.  The energy grid is an *input*: an
explicit list E_j (meV), or the first n FFT bins of the segment.

This module describes inputs only; it holds none of the TACAW arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

from .philox import philox4x32_10, u01

H_MEV_PS = 4.135667696  # Planck constant h in meV*ps (CODATA 2018, exact)


@dataclass(frozen=True)
class Detector:
    """Aperture in pixel units, centre given as an offset from the DC pixel (Kx/2, Ky/2).

    kind: "circular" (r_out, inclusive) or "annular" (r_in < d <= r_out).
    """
    kind: str = "circular"
    cx: float = 0.0
    cy: float = 0.0
    r_in: float = -1.0
    r_out: float = 20.0


@dataclass(frozen=True)
class StreamSpec:
    P: int
    Kx: int
    Ky: int
    T: int
    Tc: int
    dt_fs: float = 5.0
    # energy grid: either fft_bins (first n FFT bins) or (E_max, n_omega) uniform, end point excluded
    fft_bins: int = 0
    n_omega: int = 0
    E_max_meV: float = 120.0
    window: str = "hann"          # rect | hann | gauss | tukey | blackmanharris | kaiser | chebwin
    window_param: float = 0.0     # gauss: sigma in frames (0 -> T/6); tukey: alpha; kaiser: beta;
                                  # chebwin: side-lobe attenuation in dB
    subtract_mean: bool = True
    bose_T_K: float = 0.0
    detectors: Tuple[Detector, ...] = (Detector(),)
    # generator
    n_modes: int = 8
    E_modes: Tuple[float, float] = (5.0, 100.0)
    amp: float = 1e-2
    amp_law: str = "uniform"      # uniform: |psi0|*U(0.5,1); smooth: |psi0|*(0.5+0.5*s_m(k))
    noise: float = 1e-4
    sigma_env: float = 8.0
    # full multislice grid the ROI is cropped from (0 -> the ROI is the full grid)
    Gx: int = 0
    Gy: int = 0
    stream_id: int = 0

    @property
    def Nw(self) -> int:
        return self.fft_bins if self.fft_bins else self.n_omega

    @property
    def full_grid(self) -> Tuple[int, int]:
        return (self.Gx or self.Kx, self.Gy or self.Ky)

    @property
    def roi_origin(self) -> Tuple[int, int]:
        """Top-left corner of the centred crop inside the full grid."""
        gx, gy = self.full_grid
        return ((gx - self.Kx) // 2, (gy - self.Ky) // 2)

    def energies_meV(self) -> np.ndarray:
        """The energy grid E_j in meV (FP64)."""
        if self.fft_bins:
            return np.arange(self.fft_bins, dtype=np.float64) * (H_MEV_PS / (self.T * self.dt_fs * 1e-3))
        return np.arange(self.n_omega, dtype=np.float64) * (self.E_max_meV / self.n_omega)

    def window_sigma(self) -> float:
        if self.window == "gauss":
            return self.window_param if self.window_param > 0 else self.T / 6.0
        return self.window_param

    def cmac(self) -> int:
        return self.P * self.Kx * self.Ky * self.T * self.Nw


@dataclass(frozen=True)
class Workload:
    name: str
    streams: Tuple[StreamSpec, ...]
    precision: str = "fp32"       # fp32 | split_bf16
    seed: int = 0
    probe_batch: int = 0          # >0: probes are processed in batches of this many
    note: str = ""

    def cmac(self) -> int:
        return sum(s.cmac() for s in self.streams)


def tiny(seed: int = 0) -> Workload:
    """4 probes, 64x64 ROI, T=256 in one push, first 128 FFT bins, Hann, 8 modes."""
    s = StreamSpec(P=4, Kx=64, Ky=64, T=256, Tc=256, fft_bins=128, window="hann",
                   n_modes=8, amp_law="uniform", noise=1e-4)
    return Workload("tiny-P4-K64-T256-fft128", (s,), precision="fp32", seed=seed)


def realistic(seed: int = 0, precision: str = "split_bf16") -> Workload:
    """64 probes (8x8 scan), 256x256 ROI, T=2048 pushed 32 at a time, 400 bins over 0-120 meV."""
    s = StreamSpec(P=64, Kx=256, Ky=256, T=2048, Tc=32, n_omega=400, E_max_meV=120.0,
                   window="hann", n_modes=32, amp_law="smooth", noise=1e-3)
    return Workload("realistic-P64-K256-T2048-W400", (s,), precision=precision, seed=seed)


def batched(seed: int = 0, n_part: int = 16) -> Workload:
    """16 partitions with seeded uneven shapes, Nw=300 over 0-120 meV, Tc=16, split-BF16."""
    streams = []
    for i in range(n_part):
        r = philox4x32_10(i, 0, 0x0B47, 0, seed, 0xBA7C)
        u = [u01(x) for x in r]
        T = 512 * (1 + int(u[0] * 8))            # {512, ..., 4096}
        K = (128, 192, 256, 384)[int(u[1] * 4)]
        P = 4 + int(u[2] * 29)                   # 4..32
        win = "hann" if u[3] < 0.5 else "gauss"
        streams.append(StreamSpec(P=P, Kx=K, Ky=K, T=T, Tc=16, n_omega=300, E_max_meV=120.0,
                                  window=win, n_modes=16, amp_law="uniform", noise=1e-3,
                                  stream_id=i))
    return Workload("batched-16part-W300", tuple(streams), precision="split_bf16", seed=seed)


def diff(seed: int = 0) -> Workload:
    """8 probes, 128x128 ROI, T=512, 200 bins over 0-120 meV, Hann, FP32 (forward + adjoint)."""
    s = StreamSpec(P=8, Kx=128, Ky=128, T=512, Tc=512, n_omega=200, E_max_meV=120.0,
                   window="hann", n_modes=8, amp_law="uniform", noise=1e-4)
    return Workload("diff-P8-K128-T512-W200", (s,), precision="fp32", seed=seed)


def thick(seed: int = 0, probes: int = 256, T: int = 8192) -> Workload:
    """256 probes in batches of 32, 1024^2 grid cropped to a centred 256^2 ROI,
    T=8192 pushed 64 at a time, 1000 bins over 0-150 meV, 30 modes."""
    s = StreamSpec(P=probes, Kx=256, Ky=256, T=T, Tc=64, n_omega=1000, E_max_meV=150.0,
                   window="hann", n_modes=30, amp_law="smooth", noise=1e-3, Gx=1024, Gy=1024)
    return Workload("thick-P256-G1024-K256-T8192-W1000", (s,), precision="split_bf16",
                    seed=seed, probe_batch=32)


def loss_weights(Nw: int, seed: int = 0) -> np.ndarray:
    """Seeded N(0,1) weights c(omega), one per energy bin (Box-Muller on Philox draws)."""
    j = np.arange(Nw, dtype=np.uint32)
    r = philox4x32_10(j, 0, 0xC0E5, 0, seed, 0x10C0)
    u0, u1 = u01(r[0]), u01(r[1])
    return np.sqrt(-2.0 * np.log(u0)) * np.cos(2.0 * np.pi * u1)


WORKLOADS = {"tiny": tiny, "realistic": realistic, "batched": batched, "diff": diff, "thick": thick}


def with_(spec: StreamSpec, **kw) -> StreamSpec:
    return replace(spec, **kw)
