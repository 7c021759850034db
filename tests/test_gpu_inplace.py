"""Frames read in place by the contraction (no staging pass), against the FP64 oracle element by
element.  The persistent in-place kernel copies each tile's 128 contiguous rows of every frame
into a raw ring and converts them into tensor memory; both of its copy paths (one 2-D tensor box
a block for evenly spaced frames, per-frame copies otherwise) are exercised.  Layouts it cannot
take are refused at plan creation (CPU tests in test_abi.py)."""
import numpy as np
import pytest

import oracle
from synth import Detector, StreamSpec
from tests.helpers import oracle_kw, rel_err_peak, stream_config

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the FP32 path's bound, as for the staged split path


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


def full_frames(spec, seed, elastic=1.0, signal=1e-2):
    """[P, T, Gy, Gx] complex64: elastic offset per pixel, small fluctuations, a weak tone."""
    gx, gy = spec.full_grid
    rng = np.random.default_rng(seed)
    P, T = spec.P, spec.T
    e = elastic * (rng.standard_normal((P, 1, gy, gx)) + 1j * rng.standard_normal((P, 1, gy, gx)))
    t = np.arange(T)[None, :, None, None]
    tone = 0.03 * np.exp(2j * np.pi * 0.0517 * t) * rng.standard_normal((P, 1, gy, gx))
    s = signal * (rng.standard_normal((P, T, gy, gx)) + 1j * rng.standard_normal((P, T, gy, gx)))
    return (e + tone + s).astype(np.complex64)


def roi(spec, full):
    rx, ry = spec.roi_origin
    return np.ascontiguousarray(full[:, :, ry:ry + spec.Ky, rx:rx + spec.Kx])


def run(spec, full, pushes=None, k_stage=0, want_psi=False, **plan_kw):
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    gx, gy = spec.full_grid
    P, T = spec.P, spec.T
    buf = torch.from_numpy(np.ascontiguousarray(full.transpose(1, 0, 2, 3))).to("cuda")   # [T][P][Gy][Gx]
    pushes = pushes or [spec.Tc] * (T // spec.Tc) + ([T % spec.Tc] if T % spec.Tc else [])
    assert sum(pushes) == T
    D, Nw, npix = len(spec.detectors), spec.Nw, spec.Kx * spec.Ky
    I = torch.empty(P * Nw * npix, dtype=torch.float32, device="cuda")
    S = torch.empty(max(1, P * D * Nw), dtype=torch.float32, device="cuda")
    Psi = torch.empty(P * Nw * npix, dtype=torch.complex64, device="cuda") if want_psi else None
    with TacawPlan([stream_config(spec)], precision="split_bf16", frames_in_place=True, k_stage=k_stage,
                   **plan_kw) as plan:
        t, fb = 0, P * gx * gy * 8
        for n in pushes:
            plan.push(0, buf.data_ptr() + t * fb, n)
            t += n
        plan.finalize(I, S if D else None, Psi)
        info = plan.info()
    torch.cuda.synchronize()
    out = dict(I=I.cpu().numpy().reshape(P, Nw, spec.Ky, spec.Kx), S=S.cpu().numpy()[:P * D * Nw].reshape(P, D, Nw),
               info=info)
    if want_psi:
        out["Psi"] = Psi.cpu().numpy().reshape(P, Nw, spec.Ky, spec.Kx)
    return out


def check(spec, seed, want_psi=False, **kw):
    full = full_frames(spec, seed)
    out = run(spec, full, want_psi=want_psi, **kw)
    assert out["info"]["frames_in_place"] == 1, out["info"]
    ref = oracle.forward(roi(spec, full), **oracle_kw(spec))
    eI = rel_err_peak(out["I"], ref.I)
    assert eI <= TOL, f"I error {eI:.3g}"
    if len(spec.detectors):
        eS = rel_err_peak(out["S"], ref.S)
        assert eS <= TOL, f"S error {eS:.3g}"
    if want_psi:
        eP = rel_err_peak(out["Psi"], ref.Psi)
        assert eP <= TOL, f"Psi error {eP:.3g}"
    return out, eI


DRAINED = {
    # ROI 128 wide cropped from a 160 x 24 grid (rows of a tile contiguous inside one image row);
    # T ragged against the 32-frame block, two energy tiles
    "crop128": (StreamSpec(P=2, Kx=128, Ky=20, T=150, Tc=40, n_omega=100, E_max_meV=120.0, window="hann",
                           Gx=160, Gy=24, detectors=(Detector("circular", 0, 0, -1, 6.0),)), {}),
    # 3 probes of 20 x 18 (npix = 360): tiles straddle adjacent probes, last tile 56 rows, uneven pushes
    "adjacent_probes": (StreamSpec(P=3, Kx=20, Ky=18, T=96, Tc=32, n_omega=40, E_max_meV=120.0, window="gauss",
                                   detectors=(Detector(), Detector("annular", 1.0, -2.0, 2.0, 6.0))),
                        {"pushes": [7, 33, 56]}),
    # several flushes with the HBM accumulators, drained every 64 frames
    "streaming": (StreamSpec(P=2, Kx=32, Ky=16, T=200, Tc=24, n_omega=70, E_max_meV=120.0, window="hann",
                             detectors=(Detector("circular", 0, 0, -1, 5.0),)),
                  {"k_stage": 64, "tc_drain_frames": 64}),
    # one frame: a single partial block
    "one_frame": (StreamSpec(P=2, Kx=8, Ky=8, T=1, Tc=1, n_omega=3, E_max_meV=10.0, window="hann",
                             subtract_mean=False), {}),
    # no mean removal, Bose factor, off-grid energies over four tiles of 88
    "wide_bose": (StreamSpec(P=1, Kx=16, Ky=16, T=64, Tc=64, n_omega=300, E_max_meV=400.0, window="tukey",
                             window_param=0.2, subtract_mean=False, bose_T_K=300.0,
                             detectors=(Detector("circular", 0, 0, -1, 3.0),)), {}),
    # H drained every 64 frames: chunks end inside the tile (after blocks 1, 3, .., 9 of 11)
    "long_drains": (StreamSpec(P=1, Kx=16, Ky=24, T=330, Tc=64, n_omega=70, E_max_meV=120.0, window="hann",
                               detectors=(Detector("circular", 0, 0, -1, 5.0),)), {"tc_drain_frames": 64}),
    # 256 tiles on at most 152 CTAs: each tile's final runs after the next tile's first block;
    # H drained after every block
    "many_tiles": (StreamSpec(P=4, Kx=64, Ky=64, T=96, Tc=32, n_omega=100, E_max_meV=120.0, window="hann",
                              detectors=(Detector("circular", 0, 0, -1, 8.0),)), {"tc_drain_frames": 32}),
    # the same over four flushes with the HBM accumulators, three energy tiles
    "many_tiles_streaming": (StreamSpec(P=4, Kx=64, Ky=64, T=200, Tc=40, n_omega=150, E_max_meV=120.0,
                                        window="hann", detectors=(Detector("circular", 0, 0, -1, 8.0),)),
                             {"k_stage": 64, "tc_drain_frames": 32}),
    # the caller's tiling: 40 energies a tile, 32-frame blocks, one chunk
    "fixed_tile": (StreamSpec(P=2, Kx=64, Ky=48, T=168, Tc=40, n_omega=150, E_max_meV=120.0, window="hann",
                              detectors=(Detector("circular", 0, 0, -1, 6.0),)),
                   {"tc_omega_tile": 40, "tc_block_frames": 32, "tc_drain_frames": 1024}),
}


@pytest.mark.parametrize("name", sorted(DRAINED))
def test_persistent_drained_in_place(name):
    spec, kw = DRAINED[name]
    out, e = check(spec, 40 + sorted(DRAINED).index(name), want_psi=name in ("crop128", "adjacent_probes"), **kw)
    if kw.get("k_stage"):
        assert out["info"]["flushes"] > 1
    print(f"in place, drained ({name}): {e:.3g}")


def test_scattered_pushes():
    """Pushes from separate allocations (frames not evenly spaced across them): the persistent
    kernel copies each frame's rows on its own instead of one 2-D tensor box per block."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    spec = StreamSpec(P=2, Kx=32, Ky=16, T=150, Tc=40, n_omega=60, E_max_meV=120.0, window="hann",
                      detectors=(Detector("circular", 0, 0, -1, 5.0),))
    full = full_frames(spec, 71)
    fr = full.transpose(1, 0, 2, 3)                              # [T][P][Ky][Kx]
    cuts = [0, 13, 40, 41, 100, 150]
    # each push a gap of 3 frames after the previous one inside one allocation
    big = torch.zeros((spec.T + 3 * len(cuts),) + fr.shape[1:], dtype=torch.complex64, device="cuda")
    bufs = []
    for i, (a, b) in enumerate(zip(cuts[:-1], cuts[1:])):
        big[a + 3 * i:b + 3 * i] = torch.from_numpy(np.ascontiguousarray(fr[a:b])).to("cuda")
        bufs.append(big[a + 3 * i:b + 3 * i])
    I = torch.empty(spec.P * spec.Nw * spec.Kx * spec.Ky, device="cuda")
    S = torch.empty(spec.P * spec.Nw, device="cuda")
    with TacawPlan([stream_config(spec)], precision="split_bf16", frames_in_place=True) as plan:
        assert plan.info()["frames_in_place"] == 1
        for b in bufs:
            plan.push(0, b, b.shape[0])
        plan.finalize(I, S)
    torch.cuda.synchronize()
    ref = oracle.forward(full, **oracle_kw(spec))
    assert rel_err_peak(I.cpu().numpy().reshape(ref.I.shape), ref.I) <= TOL
    assert rel_err_peak(S.cpu().numpy().reshape(ref.S.shape), ref.S) <= TOL


def test_unaligned_push_is_refused():
    """The persistent kernel's bulk copies need 16-byte aligned frames: an 8-byte aligned push
    is refused before anything runs, and an aligned one is accepted afterwards."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan, TacawError
    spec = DRAINED["adjacent_probes"][0]
    n = spec.P * spec.Kx * spec.Ky
    buf = torch.zeros((spec.T + 1) * n, dtype=torch.complex64, device="cuda")
    with TacawPlan([stream_config(spec)], precision="split_bf16", frames_in_place=True) as plan:
        assert plan.info()["frames_in_place"] == 1
        with pytest.raises(TacawError, match="INVALID_ARG"):
            plan.push(0, buf.data_ptr() + 8, 4)
        plan.push(0, buf.data_ptr(), spec.T)
        I = torch.empty(plan.info()["I_elems"], device="cuda")
        plan.finalize(I)
    torch.cuda.synchronize()
    assert float(I.abs().max()) == 0.0
