"""The seeded input generator: Philox4x32-10 known-answer vectors and the exit-wave model."""
import numpy as np

import synth
from synth import frames
from synth.philox import philox4x32_10


def test_philox_known_answers():
    # Known-answer vectors published with the Random123 library (Salmon et al., SC'11).
    kat = [((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
           ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
           ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
            (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1))]
    for c, k, want in kat:
        got = philox4x32_10(*c, *k)
        assert tuple(int(x) for x in got) == want


def test_generator_statistics_and_shapes():
    w = synth.tiny()
    s = w.streams[0]
    f = frames.frames(s, 0, 0, 4)
    assert f.shape == (4, 4, 64, 64) and f.dtype == np.complex64
    # psi0 has unit norm; signal amplitudes are ~1e-2 of |psi0|
    psi0, amp, phi = frames.pixel_params(s, 0, np.arange(4)[:, None, None], np.arange(64)[None, :, None],
                                          np.arange(64)[None, None, :])
    np.testing.assert_allclose((np.abs(psi0) ** 2).sum(axis=(1, 2)), 1.0, rtol=1e-12)
    ratio = amp / np.abs(psi0)[..., None]
    assert ratio.min() >= 0.5e-2 - 1e-12 and ratio.max() <= 1e-2 + 1e-12
    # the time mean of a frame block is close to psi0
    E = frames.mode_energies(s, 0)
    assert E.min() >= 5.0 and E.max() <= 100.0
    # deterministic
    np.testing.assert_array_equal(f, frames.frames(s, 0, 0, 4))
    # different seeds differ
    assert np.abs(f - frames.frames(s, 1, 0, 4)).max() > 1e-3


def test_pixel_series_matches_frames():
    s = synth.diff().streams[0]
    f = frames.frames(s, 3, 5, 6, probes=[2])
    iy, ix = np.array([64, 0, 127]), np.array([64, 127, 3])
    ser = frames.pixel_series(s, 3, 2, iy, ix, t0=5, n=6)
    np.testing.assert_array_equal(ser, f[0][:, iy, ix])


def test_noise_std():
    s = synth.StreamSpec(P=1, Kx=64, Ky=64, T=8, Tc=8, n_omega=4, noise=1e-3)
    n = frames.noise(s, 0, 0, np.arange(8)[:, None, None], np.arange(64)[None, :, None],
                     np.arange(64)[None, None, :])
    assert abs(np.std(n.real) - 1e-3 / np.sqrt(2)) < 0.03e-3
    assert abs(np.std(n.imag) - 1e-3 / np.sqrt(2)) < 0.03e-3


def test_workload_shapes_match_their_configurations():
    """The five workloads carry the stated shapes: complex MAC per segment (P K^2 T Nw), pushes,
    energy ranges, probe batching and the crop of the thick-sample grid."""
    from synth import workloads as W
    cm = lambda w: sum(s.P * s.Kx * s.Ky * s.T * s.Nw for s in w.streams)
    tiny, real, bat, diff, thick = (W.WORKLOADS[k]() for k in ("tiny", "realistic", "batched", "diff", "thick"))
    assert cm(tiny) == 4 * 64 * 64 * 256 * 128 and tiny.streams[0].fft_bins == 128
    assert cm(real) == 64 * 256 * 256 * 2048 * 400 and real.streams[0].Tc == 32
    assert real.streams[0].E_max_meV == 120.0 and real.streams[0].n_modes == 32
    assert cm(diff) == 8 * 128 * 128 * 512 * 200 and diff.precision == "fp32"
    assert cm(thick) == 256 * 256 * 256 * 8192 * 1000 and thick.probe_batch == 32
    ts = thick.streams[0]
    assert ts.full_grid == (1024, 1024) and ts.roi_origin == (384, 384) and ts.Tc == 64
    assert ts.E_max_meV == 150.0 and ts.n_modes == 30
    # batched: 16 partitions, frame counts in {512, ..., 4096}, ROIs from the four sizes,
    # 4-32 probes, 300 energies, 16-frame pushes, Hann or Gaussian windows
    assert len(bat.streams) == 16
    for s in bat.streams:
        assert s.T % 512 == 0 and 512 <= s.T <= 4096
        assert s.Kx == s.Ky and s.Kx in (128, 192, 256, 384)
        assert 4 <= s.P <= 32 and s.Nw == 300 and s.Tc == 16 and s.window in ("hann", "gauss")
    assert 0.5e13 < cm(bat) < 3e13
