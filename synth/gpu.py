"""ctypes binding of synth/libsynth.so: the CUDA twin of synth.frames.

Writes seeded synthetic frames straight into device memory (frame-major layout
[t][p][ky][kx] inside a possibly larger full grid).  Input synthesis only.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import c_double, c_int, c_longlong, c_uint, c_void_p, POINTER

import numpy as np

from . import frames as F
from .workloads import StreamSpec

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsynth.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2607_02236_gb300.build.build_all()")
        L = ctypes.CDLL(LIB_PATH)
        dp = POINTER(c_double)
        L.synth_frames.argtypes = [c_void_p, c_longlong, c_longlong, c_longlong, c_int, c_int, c_int, c_int,
                                   c_int, c_int, c_int, c_int, c_int, c_int, c_int, c_int, c_double, c_double,
                                   c_uint, c_uint, c_int, dp, c_int, c_double, dp, dp, dp, c_int, c_double,
                                   c_void_p]
        L.synth_frames.restype = c_int
        _lib = L
    return _lib


def generate(spec: StreamSpec, seed: int, out_ptr: int, t0: int, n: int, *, pitch_row: int, pitch_frame: int,
             pitch_probe: int, out_x0: int = 0, out_y0: int = 0, p0: int = 0, P: int = None, stream: int = 0):
    """Frames t0..t0+n-1 of probes p0..p0+P-1 into out_ptr (complex64 element pitches)."""
    P = spec.P - p0 if P is None else P
    f = np.ascontiguousarray(F.mode_cycles(spec, seed), dtype=np.float64)
    if spec.amp_law == "smooth":
        su, sv, chi = (np.ascontiguousarray(a, dtype=np.float64) for a in F.smooth_params(spec, seed))
    else:
        su = sv = chi = np.zeros(max(1, spec.n_modes))
    gx, gy = spec.full_grid
    rx, ry = spec.roi_origin
    dp = POINTER(c_double)
    rc = lib().synth_frames(
        c_void_p(out_ptr), pitch_row, pitch_frame, pitch_probe, out_x0, out_y0, P, p0, spec.Kx, spec.Ky, t0, n,
        gx, gy, rx, ry, spec.sigma_env, F.envelope_norm(spec), seed & 0xFFFFFFFF, spec.stream_id, spec.n_modes,
        f.ctypes.data_as(dp), 1 if spec.amp_law == "smooth" else 0, spec.amp, su.ctypes.data_as(dp),
        sv.ctypes.data_as(dp), chi.ctypes.data_as(dp), spec.Kx, spec.noise, c_void_p(stream))
    if rc != 0:
        raise RuntimeError(f"synth_frames failed with CUDA error {rc}")
