"""Thin ctypes binding of libtacaw.so (include/tacaw.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module only
builds the C descriptors, passes device pointers (ints or tensors' data_ptr()) and
CUDA stream handles, and turns non-OK statuses into exceptions.  It raises if the
compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import CFUNCTYPE, POINTER, c_char_p, c_double, c_float, c_int, c_int64, c_void_p
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtacaw.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_STATE, ERR_OVERFLOW, ERR_TIMEOUT, ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["OK", "INVALID_ARG", "OOM", "CUDA", "STATE", "OVERFLOW", "TIMEOUT", "UNSUPPORTED"]
WINDOWS = {"rect": 0, "hann": 1, "gauss": 2, "tukey": 3, "blackmanharris": 4, "kaiser": 5, "chebwin": 6}
PRECISIONS = {"fp32": 0, "split_bf16": 1, "split_fp16": 2}
ACCUMS = {"kahan": 0, "fp64": 1, "fp32": 2, "auto": 3}
DET_KINDS = {"circular": 0, "annular": 1, "mask": 2}

# Every symbol include/tacaw.h declares (checked by the CPU test that loads the library).
EXPORTS = ["tacaw_plan_create", "tacaw_push_frames", "tacaw_finalize", "tacaw_output_offsets",
           "tacaw_backward", "tacaw_reset", "tacaw_plan_get_info", "tacaw_set_timing",
           "tacaw_kernel_time_ms", "tacaw_destroy", "tacaw_last_error", "tacaw_version",
           "tacaw_detector_spectra_noalloc", "tacaw_flush_trace", "tacaw_finalize_async",
           "tacaw_check_errors", "tacaw_set_log_callback", "tacaw_set_wait_limit_ns", "tacaw_push_frames_group",
           "tacaw_set_adjoint_precision", "tacaw_set_pipelined_segments", "tacaw_drain",
           "tacaw_state_size", "tacaw_save_state", "tacaw_restore_state"]


class TacawError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"TACAW_ERR_{name}: {msg}")


class CDetector(ctypes.Structure):
    _fields_ = [("kind", c_int), ("cx", c_float), ("cy", c_float), ("r_in", c_float), ("r_out", c_float),
                ("d_mask", c_void_p)]


class CStreamDesc(ctypes.Structure):
    _fields_ = [("n_probes", c_int), ("kx", c_int), ("ky", c_int),
                ("pitch_row", c_int64), ("pitch_frame", c_int64), ("pitch_probe", c_int64),
                ("roi_x0", c_int), ("roi_y0", c_int), ("T", c_int), ("dt_fs", c_double),
                ("n_omega", c_int), ("E_meV", POINTER(c_double)), ("fft_bins", c_int),
                ("window", c_int), ("window_param", c_double), ("subtract_mean", c_int),
                ("bose_T_K", c_double), ("n_detectors", c_int), ("detectors", POINTER(CDetector)),
                ("welch_segments", c_int), ("welch_stride", c_int), ("skip_init", c_int)]


class CPlanDesc(ctypes.Structure):
    _fields_ = [("n_streams", c_int), ("streams", POINTER(CStreamDesc)), ("precision", c_int),
                ("accum", c_int), ("hbm_budget_bytes", c_int64), ("k_stage", c_int),
                ("tune_cache_path", c_char_p), ("tc_omega_tile", c_int), ("tc_block_frames", c_int),
                ("frames_in_place", c_int), ("tc_drain_frames", c_int), ("tc_max_ctas", c_int),
                ("fp16_scale", c_double)]


class CPlanInfo(ctypes.Structure):
    _fields_ = [("device_bytes", c_int64), ("k_stage", c_int), ("n_streams", c_int), ("precision", c_int),
                ("I_elems", c_int64), ("S_elems", c_int64), ("flushes", c_int64), ("omega_tile", c_int),
                ("stages", c_int), ("kernel_launches", c_int64), ("tc_block_frames", c_int),
                ("frames_in_place", c_int), ("tc_drain_frames", c_int), ("tuned_streams", c_int),
                ("tune_candidates", c_int), ("tune_ms", c_double), ("accum", c_int), ("flush_launches", c_int64),
                ("aperture_pixels", c_int64)]


_lib = None


def lib():
    """Loads libtacaw.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2607_02236_gb300.build.build_all()")
    L = ctypes.CDLL(LIB_PATH)
    L.tacaw_plan_create.argtypes = [POINTER(CPlanDesc), POINTER(c_void_p)]
    L.tacaw_push_frames.argtypes = [c_void_p, c_int, c_void_p, c_int, c_void_p]
    L.tacaw_push_frames_group.argtypes = [c_void_p, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_void_p),
                                          ctypes.POINTER(c_int), c_void_p]
    L.tacaw_finalize.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.tacaw_finalize_async.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.tacaw_check_errors.argtypes = [c_void_p, c_void_p]
    L.tacaw_output_offsets.argtypes = [c_void_p, c_int, POINTER(c_int64), POINTER(c_int64)]
    L.tacaw_backward.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]
    L.tacaw_reset.argtypes = [c_void_p, c_void_p]
    L.tacaw_plan_get_info.argtypes = [c_void_p, POINTER(CPlanInfo)]
    L.tacaw_set_timing.argtypes = [c_void_p, c_int]
    L.tacaw_set_wait_limit_ns.argtypes = [c_void_p, ctypes.c_uint64]
    L.tacaw_set_adjoint_precision.argtypes = [c_void_p, c_int]
    L.tacaw_set_pipelined_segments.argtypes = [c_void_p, c_int]
    L.tacaw_drain.argtypes = [c_void_p, c_void_p]
    L.tacaw_state_size.argtypes = [c_void_p, POINTER(c_int64)]
    L.tacaw_save_state.argtypes = [c_void_p, c_void_p, c_int64, c_void_p]
    L.tacaw_restore_state.argtypes = [c_void_p, c_void_p, c_int64, c_void_p]
    L.tacaw_kernel_time_ms.argtypes = [c_void_p, POINTER(c_double), POINTER(c_int64), c_int]
    L.tacaw_destroy.argtypes = [c_void_p]
    L.tacaw_flush_trace.argtypes = [c_void_p, c_void_p, c_int64, POINTER(c_int64)]
    L.tacaw_detector_spectra_noalloc.argtypes = [c_void_p, c_int, c_int, c_int, c_int, POINTER(CDetector), c_int,
                                                 c_void_p, c_void_p]
    L.tacaw_set_log_callback.argtypes = [c_void_p, c_void_p]
    L.tacaw_last_error.restype = c_char_p
    L.tacaw_version.restype = c_char_p
    for name in EXPORTS:
        f = getattr(L, name)
        if f.restype is None or f.restype is c_int:
            if name not in ("tacaw_last_error", "tacaw_version"):
                f.restype = c_int
    _lib = L
    return L


def _check(status: int):
    if status != OK:
        raise TacawError(status, lib().tacaw_last_error().decode())


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


@dataclass
class DetectorConfig:
    kind: str = "circular"
    cx: float = 0.0
    cy: float = 0.0
    r_in: float = -1.0
    r_out: float = 20.0
    mask_ptr: int = 0


@dataclass
class StreamConfig:
    """One stream (supercell partition).  Pitches are in complex64 elements."""
    n_probes: int
    kx: int
    ky: int
    T: int
    dt_fs: float
    pitch_row: int
    pitch_frame: int
    pitch_probe: int
    roi_x0: int = 0
    roi_y0: int = 0
    E_meV: Optional[Sequence[float]] = None
    fft_bins: int = 0
    n_omega: int = 0
    window: str = "hann"
    window_param: float = 0.0
    subtract_mean: bool = True
    bose_T_K: float = 0.0
    detectors: List[DetectorConfig] = field(default_factory=list)
    # Welch averaging: N segments of T frames, `welch_stride` frames apart (0: T); 0/1: off
    welch_segments: int = 0
    welch_stride: int = 0
    # leading frames dropped before the first segment (the trajectory's initial part)
    skip_init: int = 0


class TacawPlan:
    """A streaming plan over one or more streams (see include/tacaw.h)."""

    def __init__(self, streams: Sequence[StreamConfig], precision: str = "split_bf16", accum: str = "auto",
                 hbm_budget_bytes: int = 0, k_stage: int = 0, tc_omega_tile: int = 0, tc_block_frames: int = 0,
                 frames_in_place: bool = False, tune: Optional[str] = None, tc_drain_frames: int = 0,
                 tc_max_ctas: int = 0, fp16_scale: float = 0.0):
        """tune: None uses the built-in tile rule; "" autotunes at creation; a file path
        autotunes through a text cache at that path.  fp16_scale: operand scale of the
        split_fp16 precision (a power of two; 0 selects 2^12)."""
        L = lib()
        self._keep = []
        descs = (CStreamDesc * len(streams))()
        for i, s in enumerate(streams):
            d = descs[i]
            d.n_probes, d.kx, d.ky = s.n_probes, s.kx, s.ky
            d.pitch_row, d.pitch_frame, d.pitch_probe = s.pitch_row, s.pitch_frame, s.pitch_probe
            d.roi_x0, d.roi_y0, d.T, d.dt_fs = s.roi_x0, s.roi_y0, s.T, s.dt_fs
            if s.fft_bins:
                d.fft_bins, d.n_omega = 1, int(s.fft_bins)
                d.E_meV = POINTER(c_double)()
            elif s.E_meV is None:              # no grid: the library reports it
                d.fft_bins, d.n_omega = 0, int(s.n_omega)
                d.E_meV = POINTER(c_double)()
            else:
                E = (c_double * len(s.E_meV))(*[float(e) for e in s.E_meV])
                self._keep.append(E)
                d.fft_bins, d.n_omega = 0, len(s.E_meV)
                d.E_meV = ctypes.cast(E, POINTER(c_double))
            d.window, d.window_param = WINDOWS[s.window], float(s.window_param)
            d.subtract_mean, d.bose_T_K = int(bool(s.subtract_mean)), float(s.bose_T_K)
            dets = (CDetector * max(1, len(s.detectors)))()
            for k, t in enumerate(s.detectors):
                dets[k].kind, dets[k].cx, dets[k].cy = DET_KINDS[t.kind], t.cx, t.cy
                dets[k].r_in, dets[k].r_out, dets[k].d_mask = t.r_in, t.r_out, t.mask_ptr or None
            self._keep.append(dets)
            d.n_detectors = len(s.detectors)
            d.detectors = ctypes.cast(dets, POINTER(CDetector))
            d.welch_segments, d.welch_stride = int(s.welch_segments), int(s.welch_stride)
            d.skip_init = int(s.skip_init)
        pd = CPlanDesc(len(streams), ctypes.cast(descs, POINTER(CStreamDesc)), PRECISIONS[precision],
                       ACCUMS[accum], int(hbm_budget_bytes), int(k_stage),
                       None if tune is None else os.fsencode(tune), int(tc_omega_tile), int(tc_block_frames),
                       int(bool(frames_in_place)), int(tc_drain_frames), int(tc_max_ctas), float(fp16_scale))
        h = c_void_p()
        _check(L.tacaw_plan_create(ctypes.byref(pd), ctypes.byref(h)))
        self._h = h
        self.streams = list(streams)
        self.precision = precision

    # ---------------------------------------------------------------------------------
    def push(self, stream_id: int, frames, n_frames: int, cuda_stream=None):
        _check(lib().tacaw_push_frames(self._h, int(stream_id), _ptr(frames), int(n_frames), _stream(cuda_stream)))

    def push_group(self, stream_ids, frames, n_frames, cuda_stream=None):
        """One push of each of several streams (tacaw_push_frames_group): lists of stream ids,
        frame buffers (tensors or addresses) and frame counts."""
        n = len(stream_ids)
        if len(frames) != n or len(n_frames) != n:
            raise ValueError("stream_ids, frames and n_frames must have the same length")
        ids = (c_int * n)(*[int(i) for i in stream_ids])
        ptrs = (c_void_p * n)(*[_ptr(f) for f in frames])
        cnt = (c_int * n)(*[int(k) for k in n_frames])
        _check(lib().tacaw_push_frames_group(self._h, n, ids, ptrs, cnt, _stream(cuda_stream)))

    def finalize(self, I=None, S=None, Psi=None, cuda_stream=None):
        _check(lib().tacaw_finalize(self._h, _ptr(I), _ptr(S), _ptr(Psi), _stream(cuda_stream)))

    def finalize_async(self, I=None, S=None, Psi=None, cuda_stream=None):
        """Enqueues the finalize work without waiting (capturable into a CUDA graph)."""
        _check(lib().tacaw_finalize_async(self._h, _ptr(I), _ptr(S), _ptr(Psi), _stream(cuda_stream)))

    def check_errors(self, cuda_stream=None):
        _check(lib().tacaw_check_errors(self._h, _stream(cuda_stream)))

    def backward(self, stream_id: int, dL_dS, frames, grad, cuda_stream=None):
        _check(lib().tacaw_backward(self._h, int(stream_id), _ptr(dL_dS), _ptr(frames), _ptr(grad),
                                    _stream(cuda_stream)))

    def reset(self, cuda_stream=None):
        _check(lib().tacaw_reset(self._h, _stream(cuda_stream)))

    def offsets(self, stream_id: int):
        a, b = c_int64(), c_int64()
        _check(lib().tacaw_output_offsets(self._h, int(stream_id), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def info(self) -> dict:
        i = CPlanInfo()
        _check(lib().tacaw_plan_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in CPlanInfo._fields_}

    def set_wait_limit_ns(self, limit_ns: int):
        """Device pipeline waits of later contraction launches give up after limit_ns (0: default)."""
        _check(lib().tacaw_set_wait_limit_ns(self._h, int(limit_ns)))

    def set_adjoint_precision(self, precision: str):
        """Arithmetic of backward(): "split_bf16" (tensor cores, the default) or "fp32"."""
        _check(lib().tacaw_set_adjoint_precision(self._h, PRECISIONS.get(precision, -1)))

    def set_pipelined_segments(self, enable: bool = True):
        """Defer each segment's contraction to the next segment's finalize_async, which converts
        that segment's pushes in the same launch (see include/tacaw.h)."""
        _check(lib().tacaw_set_pipelined_segments(self._h, 1 if enable else 0))

    def drain(self, cuda_stream=None):
        """Launches a deferred contraction (pipelined segments)."""
        _check(lib().tacaw_drain(self._h, _stream(cuda_stream)))

    def state_size(self) -> int:
        """Bytes of a checkpoint of the segment in progress."""
        n = c_int64()
        _check(lib().tacaw_state_size(self._h, ctypes.byref(n)))
        return n.value

    def save_state(self, cuda_stream=None):
        """Checkpoint of the segment in progress (numpy uint8; waits for the copies)."""
        import numpy as np
        out = np.empty(self.state_size(), dtype=np.uint8)
        _check(lib().tacaw_save_state(self._h, out.ctypes.data, out.size, _stream(cuda_stream)))
        return out

    def restore_state(self, state, cuda_stream=None):
        """Continues from a checkpoint of a plan built from the same descriptor (bytes-like)."""
        import numpy as np
        buf = np.frombuffer(state, dtype=np.uint8)
        _check(lib().tacaw_restore_state(self._h, buf.ctypes.data, buf.size, _stream(cuda_stream)))

    def set_timing(self, on):
        """on: False/True, or 2 to also record per-CTA phase stamps of tensor-core flushes."""
        _check(lib().tacaw_set_timing(self._h, int(on)))

    def flush_trace(self):
        """Per-CTA stamps of the last traced tensor-core flush: numpy uint64 [n_ctas, 8]."""
        import numpy as np
        n = c_int64()
        _check(lib().tacaw_flush_trace(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros((max(n.value, 0), 8), dtype=np.uint64)
        if n.value:
            _check(lib().tacaw_flush_trace(self._h, out.ctypes.data, n.value, ctypes.byref(n)))
        return out

    def kernel_time_ms(self, reset: bool = True):
        ms, n = c_double(), c_int64()
        _check(lib().tacaw_kernel_time_ms(self._h, ctypes.byref(ms), ctypes.byref(n), int(bool(reset))))
        return ms.value, n.value

    def close(self):
        if getattr(self, "_h", None):
            lib().tacaw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _c_detectors(dets):
    arr = (CDetector * max(1, len(dets)))()
    for k, t in enumerate(dets):
        arr[k].kind, arr[k].cx, arr[k].cy = DET_KINDS[t.kind], t.cx, t.cy
        arr[k].r_in, arr[k].r_out, arr[k].d_mask = t.r_in, t.r_out, t.mask_ptr or None
    return arr


def detector_spectra_noalloc(I, n_probes: int, n_omega: int, kx: int, ky: int, detectors, S, cuda_stream=None):
    """S[p, d, E] from I[p, E, ky, kx] (device) through tacaw_detector_spectra_noalloc: no plan and no
    device allocation (the aperture lists live in the library's fixed device array)."""
    arr = _c_detectors(list(detectors))
    _check(lib().tacaw_detector_spectra_noalloc(_ptr(I), int(n_probes), int(n_omega), int(kx), int(ky),
                                                ctypes.cast(arr, POINTER(CDetector)), len(detectors), _ptr(S),
                                                _stream(cuda_stream)))


def version() -> str:
    return lib().tacaw_version().decode()


LOG_ERROR, LOG_INFO = 0, 1
_LOG_FN = CFUNCTYPE(None, c_int, c_char_p, c_void_p)
_log_keep = None


def set_log_callback(fn=None):
    """Routes the library's log (tacaw_set_log_callback) to fn(level, message); None removes
    it.  Levels: LOG_ERROR (every error returned, with its message), LOG_INFO (the
    configuration of each plan created)."""
    global _log_keep
    if fn is None:
        _check(lib().tacaw_set_log_callback(None, None))
        _log_keep = None
        return
    cb = _LOG_FN(lambda level, msg, user: fn(int(level), msg.decode(errors="replace") if msg else ""))
    _check(lib().tacaw_set_log_callback(ctypes.cast(cb, c_void_p), None))
    _log_keep = cb
