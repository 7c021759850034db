"""Pins of the FP64 oracle against things other than itself.

Each test would catch a plausible slip in the oracle: a dropped window, a wrong
sign or index in the Fourier kernel, a mean over the wrong axis, a wrong phase
reduction, a missing factor 2 in the gradient, a wrong mask convention.
"""
import ctypes
import json
import os

import numpy as np
import pytest
import scipy.signal

import oracle
from oracle import build_brute
from synth import Detector

HERE = os.path.dirname(os.path.abspath(__file__))
RNG = np.random.default_rng(1234)


def rand_psi(P, T, Ky, Kx, rng=RNG):
    return rng.standard_normal((P, T, Ky, Kx)) + 1j * rng.standard_normal((P, T, Ky, Kx))


# ------------------------------------------------------------------------------------ windows
@pytest.mark.parametrize("T", [1, 2, 7, 64, 257, 2048])
def test_windows_match_scipy_periodic(T):
    pairs = [(("rect", 0.0), "boxcar"), (("hann", 0.0), "hann"),
             (("gauss", T / 6.0), ("gaussian", T / 6.0)),
             (("tukey", 0.1), ("tukey", 0.1)), (("tukey", 0.5), ("tukey", 0.5))]
    for (kind, p), sp in pairs:
        if kind == "gauss" and T < 2:
            continue
        ours = oracle.window(kind, T, p)
        ref = scipy.signal.get_window(sp, T, fftbins=True)
        np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-14, err_msg=f"{kind} T={T}")


@pytest.mark.parametrize("T", [1, 2, 7, 8, 64, 65, 257, 2048])
def test_appendix_windows_match_scipy_periodic(T):
    """App. A's high-dynamic-range windows, which the paper defines by scipy's forms."""
    pairs = [(("blackmanharris", 0.0), "blackmanharris"), (("kaiser", 3 * np.pi), ("kaiser", 3 * np.pi)),
             (("kaiser", 5 * np.pi), ("kaiser", 5 * np.pi)), (("chebwin", 100.0), ("chebwin", 100.0)),
             (("chebwin", 60.0), ("chebwin", 60.0))]
    for (kind, p), sp in pairs:
        ours = oracle.window(kind, T, p)
        ref = scipy.signal.get_window(sp, T, fftbins=True)
        np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-12, err_msg=f"{kind} T={T}")


def test_chebwin_sidelobes_at_the_stated_attenuation():
    """Dolph-Chebyshev: every side lobe of the symmetric window's response is at_db down."""
    M, at = 129, 100.0
    w = oracle.tacaw_oracle._dolph_chebyshev(M, at)
    H = np.abs(np.fft.fft(w, 64 * M))
    H /= H[0]
    # beyond the first null the response stays at -100 dB (equiripple), within rounding
    k0 = np.argmax(H < 10 ** (-at / 20) * 1.001)
    side = H[k0:len(H) // 2]
    assert np.max(side) <= 10 ** (-at / 20) * (1 + 1e-6)
    assert np.max(side) >= 10 ** (-at / 20) * (1 - 1e-3)


def test_tukey_limits_are_rect_and_hann():
    # Sec. III.A: rectangular = Tukey alpha 0, Hann = Tukey alpha 1
    np.testing.assert_array_equal(oracle.window("tukey", 100, 0.0), oracle.window("rect", 100))
    np.testing.assert_allclose(oracle.window("tukey", 100, 1.0), oracle.window("hann", 100), atol=0)


# ------------------------------------------------------------------------------- Fourier part
@pytest.mark.parametrize("kind", ["rect", "hann"])
@pytest.mark.parametrize("sub", [False, True])
def test_fft_grid_equals_numpy_fft(kind, sub):
    P, T, Ky, Kx, nb = 2, 96, 3, 5, 40
    psi = rand_psi(P, T, Ky, Kx)
    r = oracle.forward(psi, window_kind=kind, fft_bins=nb, dt_fs=5.0, subtract_mean=sub)
    w = scipy.signal.get_window("boxcar" if kind == "rect" else "hann", T, fftbins=True)
    x = psi - (psi.mean(axis=1, keepdims=True) if sub else 0)
    ref = np.fft.fft(w[None, :, None, None] * x, axis=1)[:, :nb]
    np.testing.assert_allclose(r.Psi, ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    np.testing.assert_allclose(r.I, np.abs(ref) ** 2, rtol=0, atol=1e-11 * (np.abs(ref) ** 2).max())


def test_explicit_grid_equal_to_fft_grid_energies():
    # The fractional-phase path at E_j = j h/(T dt) must equal the exact integer path.
    T, dt = 128, 5.0
    psi = rand_psi(1, T, 2, 2)
    E = oracle.fft_energies(T, dt, 64)
    a = oracle.forward(psi, window_kind="hann", E_meV=E, dt_fs=dt)
    b = oracle.forward(psi, window_kind="hann", fft_bins=64, dt_fs=dt)
    np.testing.assert_allclose(a.Psi, b.Psi, atol=1e-10 * np.abs(b.Psi).max())


def test_parseval_full_grid():
    P, T, K = 2, 64, 3
    psi = rand_psi(P, T, K, K)
    r = oracle.forward(psi, window_kind="rect", fft_bins=T, subtract_mean=False)
    lhs = r.I.sum(axis=1)
    rhs = T * (np.abs(psi) ** 2).sum(axis=1)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


def test_parseval_hann_with_mean():
    P, T, K = 1, 80, 2
    psi = rand_psi(P, T, K, K)
    r = oracle.forward(psi, window_kind="hann", fft_bins=T, subtract_mean=True)
    w = scipy.signal.get_window("hann", T, fftbins=True)
    x = psi - psi.mean(axis=1, keepdims=True)
    rhs = T * ((w[None, :, None, None] ** 2) * np.abs(x) ** 2).sum(axis=1)
    np.testing.assert_allclose(r.I.sum(axis=1), rhs, rtol=1e-12)


def dirichlet(phi, T):
    """sum_{n<T} exp(-i phi n) in closed form."""
    phi = np.asarray(phi, dtype=np.float64)
    out = np.empty(phi.shape, dtype=np.complex128)
    s = np.sin(phi / 2)
    small = np.abs(s) < 1e-14
    out[~small] = np.exp(-1j * phi[~small] * (T - 1) / 2) * np.sin(T * phi[~small] / 2) / s[~small]
    out[small] = T
    return out


@pytest.mark.parametrize("kind", ["rect", "hann"])
@pytest.mark.parametrize("sub", [False, True])
def test_pure_tone_closed_form(kind, sub):
    """psi_n = A exp(+i w0 n): Psi(w) = A W(w - w0) with W the window's DTFT (and - mu W(w) with the mean)."""
    T, dt = 200, 5.0
    E0 = 37.3                                    # meV, off any FFT bin
    E = np.linspace(0.0, 120.0, 97) + 0.0173     # explicit grid, off the FFT bins
    A = 0.3 - 0.2j
    c0 = oracle.cycles_per_frame(E0, dt)
    n = np.arange(T)
    psi = (A * np.exp(2j * np.pi * c0 * n))[None, :, None, None]
    r = oracle.forward(psi, window_kind=kind, E_meV=E, dt_fs=dt, subtract_mean=sub)
    phi = 2 * np.pi * (oracle.cycles_per_frame(E, dt) - c0)
    phiE = 2 * np.pi * oracle.cycles_per_frame(E, dt)
    if kind == "rect":
        W = lambda ph: dirichlet(ph, T)
    else:
        W = lambda ph: 0.5 * dirichlet(ph, T) - 0.25 * dirichlet(ph - 2 * np.pi / T, T) \
            - 0.25 * dirichlet(ph + 2 * np.pi / T, T)
    ref = A * W(phi)
    if sub:
        mu = A * dirichlet(np.array([-2 * np.pi * c0]), T)[0] / T   # (1/T) sum_n e^{+i w0 n}
        ref = ref - mu * W(phiE)
    np.testing.assert_allclose(r.Psi[0, :, 0, 0], ref, rtol=0, atol=1e-10 * T)


def test_tone_on_bin_lands_in_bin_and_hann_leaks_to_neighbours_only():
    T, j0 = 128, 17
    n = np.arange(T)
    psi = np.exp(2j * np.pi * j0 * n / T)[None, :, None, None]
    r = oracle.forward(psi, window_kind="hann", fft_bins=T, subtract_mean=False)
    I = r.I[0, :, 0, 0]
    assert np.argmax(I) == j0
    np.testing.assert_allclose(I[j0], (T / 2) ** 2, rtol=1e-12)
    np.testing.assert_allclose(I[[j0 - 1, j0 + 1]], (T / 4) ** 2, rtol=1e-12)
    mask = np.ones(T, bool)
    mask[[j0 - 1, j0, j0 + 1]] = False
    assert I[mask].max() < 1e-20 * I[j0]


@pytest.mark.parametrize("kind,slope", [("rect", -1.0), ("hann", -3.0)])
def test_side_lobe_decay_rates(kind, slope):
    """Far side lobes of an off-bin tone fall as 1/w (rectangular: a jump at the segment edges)
    and 1/w^3 (Hann: value and slope vanish there), measured at lobe peaks k + 1/2 bins away."""
    T, dt = 4096, 5.0
    c0 = 311.37 / T                                  # cycles per frame, off any bin
    k = np.array([16.5, 32.5, 64.5, 128.5])
    E = (c0 + k / T) / oracle.cycles_per_frame(1.0, dt)
    psi = np.exp(2j * np.pi * c0 * np.arange(T))[None, :, None, None]
    r = oracle.forward(psi, window_kind=kind, E_meV=E, dt_fs=dt, subtract_mean=False)
    a = np.abs(r.Psi[0, :, 0, 0])
    np.testing.assert_allclose(np.diff(np.log(a)) / np.diff(np.log(k)), slope, atol=0.02)


def test_hann_side_lobes_below_tukey_and_rect():
    """The Hann window's side lobes lie below those of Tukey (alpha = 0.1) and of the rectangular
    window at every offset from 4 to 200 bins (the window comparison of Sec. III.A)."""
    T, dt = 1024, 5.0
    c0 = 100.29 / T
    k = np.linspace(4.0, 200.0, 1571)
    E = (c0 + k / T) / oracle.cycles_per_frame(1.0, dt)
    psi = np.exp(2j * np.pi * c0 * np.arange(T))[None, :, None, None]
    env = {}
    for kind, par in (("hann", 0.0), ("tukey", 0.1), ("rect", 0.0)):
        a = np.abs(oracle.forward(psi, window_kind=kind, window_param=par, E_meV=E, dt_fs=dt,
                                  subtract_mean=False).Psi[0, :, 0, 0])
        env[kind] = np.array([a[(k >= b) & (k < b + 4)].max() for b in range(4, 200, 4)])   # lobe envelope
    assert np.all(env["hann"] < env["tukey"]) and np.all(env["hann"] < env["rect"])


def test_wiener_khinchin_off_grid():
    """|Psi(w)|^2 = sum_tau R(tau) exp(-i w tau), R(tau) = sum_n y_{n+tau} conj(y_n) (direct lag sums)."""
    T, dt = 60, 5.0
    psi = rand_psi(1, T, 1, 1)
    E = np.array([0.0, 3.3, 17.77, 55.5, 101.01, 333.0])
    r = oracle.forward(psi, window_kind="hann", E_meV=E, dt_fs=dt, subtract_mean=True)
    w = scipy.signal.get_window("hann", T, fftbins=True)
    x = psi[0, :, 0, 0]
    y = w * (x - x.mean())
    c = oracle.cycles_per_frame(E, dt)
    S = np.zeros(len(E))
    for tau in range(-(T - 1), T):
        R = sum(y[n + tau] * np.conj(y[n]) for n in range(max(0, -tau), min(T, T - tau)))
        S = S + (R * np.exp(-2j * np.pi * c * tau)).real
    np.testing.assert_allclose(r.I[0, :, 0, 0], S, rtol=1e-10, atol=1e-12 * S.max())


def test_elastic_only_gives_zero():
    T = 256
    const = rand_psi(3, 1, 4, 4)
    psi = np.repeat(const, T, axis=1)
    for kind in ("rect", "hann", "gauss"):
        r = oracle.forward(psi, window_kind=kind, E_meV=np.linspace(0, 120, 50), dt_fs=5.0,
                           subtract_mean=True)
        assert r.I.max() <= 1e-24 * (np.abs(psi) ** 2).sum() ** 2


def test_phase_ramp_shifts_one_bin():
    """A COM-drift-like phase ramp exp(2 pi i n/T) shifts the spectrum by one bin (Sec. III.B)."""
    T = 64
    psi = rand_psi(1, T, 2, 2)
    n = np.arange(T)
    ramp = np.exp(2j * np.pi * n / T)[None, :, None, None]
    a = oracle.forward(psi, window_kind="rect", fft_bins=T, subtract_mean=False)
    b = oracle.forward(psi * ramp, window_kind="rect", fft_bins=T, subtract_mean=False)
    np.testing.assert_allclose(b.Psi, np.roll(a.Psi, 1, axis=1), atol=1e-11 * np.abs(a.Psi).max())


def test_brute_force_c_long_double():
    lib = ctypes.CDLL(build_brute.build())
    f = lib.tacaw_brute_intensity
    dp = ctypes.POINTER(ctypes.c_double)
    f.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int, dp]
    T, dt = 37, 5.0
    E = np.array([0.0, 1.5, 7.0, 33.3, 89.9, 120.0])
    for kind, sub in (("hann", True), ("rect", False), ("gauss", True)):
        psi = rand_psi(1, T, 2, 2)
        r = oracle.forward(psi, window_kind=kind, E_meV=E, dt_fs=dt, subtract_mean=sub)
        x = psi[0].reshape(T, 4)
        re = np.ascontiguousarray(x.real)
        im = np.ascontiguousarray(x.imag)
        w = np.ascontiguousarray(oracle.window(kind, T))
        c = np.ascontiguousarray(E * dt * 1e-3 / 4.135667696)
        out = np.zeros(len(E) * 4)
        f(re.ctypes.data_as(dp), im.ctypes.data_as(dp), T, 4, w.ctypes.data_as(dp),
          c.ctypes.data_as(dp), len(E), int(sub), out.ctypes.data_as(dp))
        np.testing.assert_allclose(r.I[0].reshape(len(E), 4), out.reshape(len(E), 4), rtol=1e-12,
                                   atol=1e-13 * out.max())


def test_linearity_and_independence():
    P, T, K = 2, 48, 3
    E = np.linspace(0, 100, 20)
    kw = dict(window_kind="hann", E_meV=E, dt_fs=5.0, subtract_mean=True)
    a, b = rand_psi(P, T, K, K), rand_psi(P, T, K, K)
    alpha, beta = 0.7 - 0.2j, -1.3 + 0.5j
    ra, rb = oracle.forward(a, **kw), oracle.forward(b, **kw)
    rc = oracle.forward(alpha * a + beta * b, **kw)
    np.testing.assert_allclose(rc.Psi, alpha * ra.Psi + beta * rb.Psi, atol=1e-12 * np.abs(rc.Psi).max())
    # probe permutation
    rp = oracle.forward(a[::-1], **kw)
    np.testing.assert_allclose(rp.I, ra.I[::-1], rtol=1e-13)
    # changing one pixel changes only that pixel's outputs
    a2 = a.copy()
    a2[1, :, 2, 1] += rand_psi(1, T, 1, 1)[0, :, 0, 0]
    r2 = oracle.forward(a2, **kw)
    diff = np.abs(r2.I - ra.I).sum(axis=1)
    assert diff[1, 2, 1] > 0
    diff[1, 2, 1] = 0
    assert diff.max() == 0


# ------------------------------------------------------------------------------ Bose factor
def test_bose_factor_limits():
    T_K = 300.0
    beta = 1.0 / (oracle.KB_MEV_PER_K * T_K)
    assert oracle.bose(np.array([0.0]), T_K)[0] == 1.0
    E = np.array([0.5, 5.0, 50.0, 150.0])
    B = oracle.bose(E, T_K)
    Bm = oracle.bose(-E, T_K)
    # detailed balance: B(-E) = exp(-beta E) B(E)
    np.testing.assert_allclose(Bm, np.exp(-beta * E) * B, rtol=1e-13)
    # small beta E: 1 + beta E / 2 + (beta E)^2 / 12
    e = np.array([1e-3, 1e-2])
    np.testing.assert_allclose(oracle.bose(e, T_K), 1 + beta * e / 2 + (beta * e) ** 2 / 12, rtol=1e-9)
    # large beta E: -> beta E
    np.testing.assert_allclose(oracle.bose(np.array([2000.0]), 10.0), 2000.0 / (oracle.KB_MEV_PER_K * 10.0),
                               rtol=1e-12)
    np.testing.assert_array_equal(oracle.bose(E, 0.0), np.ones(4))


def test_bose_applied_in_intensity():
    T = 64
    psi = rand_psi(1, T, 2, 2)
    E = np.linspace(-60, 60, 25)
    a = oracle.forward(psi, window_kind="hann", E_meV=E, dt_fs=5.0, bose_T_K=0.0)
    b = oracle.forward(psi, window_kind="hann", E_meV=E, dt_fs=5.0, bose_T_K=300.0)
    np.testing.assert_allclose(b.I, a.I * oracle.bose(E, 300.0)[None, :, None, None], rtol=1e-14)


# ------------------------------------------------------------------------------- detectors
def golden():
    with open(os.path.join(HERE, "golden", "paper_numbers.json")) as f:
        return json.load(f)


def test_circular_mask_counts_gauss_circle():
    g = golden()["gauss_circle_counts"]["value"]
    for r, n in g.items():
        M = oracle.detector_masks(64, 64, [Detector("circular", 0, 0, -1, float(r))])
        assert int(M.sum()) == n, r
        assert M[0, 32, 32] == 1


def test_annular_partitions_disk_and_offaxis_centre():
    d = [Detector("circular", 0, 0, -1, 10), Detector("annular", 0, 0, 10, 30),
         Detector("circular", 0, 0, -1, 30)]
    M = oracle.detector_masks(96, 96, d)
    np.testing.assert_array_equal(M[0] + M[1], M[2])
    off = oracle.detector_masks(64, 64, [Detector("circular", 7, -3, -1, 2)])[0]
    assert off[32 - 3, 32 + 7] == 1 and off.sum() == 13


def test_detector_sum_parseval_full_cover():
    """A detector covering every pixel, rect window, full FFT grid: sum_j S_j = T sum |psi|^2."""
    P, T, K = 2, 32, 4
    psi = rand_psi(P, T, K, K)
    r = oracle.forward(psi, window_kind="rect", fft_bins=T, subtract_mean=False,
                       detectors=[Detector("circular", 0, 0, -1, 100.0)])
    np.testing.assert_allclose(r.S[:, 0, :].sum(axis=1), T * (np.abs(psi) ** 2).sum(axis=(1, 2, 3)),
                               rtol=1e-12)


# ------------------------------------------------------------------------- paper's numbers
def test_paper_worked_numbers():
    g = golden()
    h = oracle.H_MEV_PS
    e = g["energy_sampling_meV"]
    dE = oracle.fft_energies(e["inputs"]["L"], e["inputs"]["tau_fs"], 2)[1]
    assert abs(dE - e["value"]) <= e["rel_tol"] * e["value"]
    e = g["max_energy_rule_of_thumb_meV_at_1fs"]
    eps = h / (2 * e["inputs"]["tau_fs"] * 1e-3)
    assert abs(eps - e["value"]) <= e["rel_tol"] * e["value"]
    e = g["energy_bins_pm30THz"]
    L, tau = e["inputs"]["L"], e["inputs"]["tau_fs"]
    # signed FFT bins j in [-L/2, L/2): frequency j / (L tau)
    j = np.arange(-L // 2, L // 2)
    f_THz = j / (L * tau * 1e-3)
    assert int(np.sum(np.abs(f_THz) <= e["inputs"]["f_max_THz"] + 1e-9)) == e["value"]
    # energies of those bins are E = h f
    np.testing.assert_allclose(oracle.fft_energies(L, tau, 91)[90], h * 30.0, rtol=1e-12)
    e = g["thermalisation_skip_ps"]
    assert abs(e["inputs"]["skip_snapshots"] * e["inputs"]["tau_fs"] * 1e-3 - e["value"]) < 1e-12
    e = g["exit_wave_memory_GB"]
    i = e["inputs"]
    mem = i["sx"] * i["sy"] * i["kx"] * i["ky"] * i["c"] * i["p"] * 2 / 1e9
    assert abs(mem - e["value"]) <= e["rel_tol"] * e["value"]


# -------------------------------------------------------------------------------- gradient
def _grad_case(seed=5):
    rng = np.random.default_rng(seed)
    P, T, K = 2, 24, 5
    psi = rand_psi(P, T, K, K, rng)
    E = np.linspace(0, 150, 11) + 0.37
    dets = [Detector("circular", 0, 0, -1, 1.5), Detector("annular", 0, 0, 1.0, 2.5)]
    dLdS = rng.standard_normal((P, len(dets), len(E)))
    kw = dict(window_kind="hann", E_meV=E, dt_fs=5.0, subtract_mean=True, bose_T_K=300.0,
              detectors=dets)
    return psi, dLdS, kw


def test_gradient_central_differences():
    psi, dLdS, kw = _grad_case()
    g = oracle.gradient(psi, dLdS, **kw)
    rng = np.random.default_rng(7)
    h = 1e-6
    # central differences in FP64 carry a rounding floor of ~eps * sum|dLdS*S| / h
    r = oracle.forward(psi, **kw)
    floor = 16 * np.finfo(np.float64).eps * float(np.sum(np.abs(dLdS) * r.S)) / h
    for _ in range(64):
        idx = tuple(int(rng.integers(0, s)) for s in psi.shape)
        for comp, unit in (("re", 1.0), ("im", 1j)):
            a = psi.copy()
            b = psi.copy()
            a[idx] += h * unit
            b[idx] -= h * unit
            fd = (oracle.loss(a, dLdS, **kw) - oracle.loss(b, dLdS, **kw)) / (2 * h)
            an = g[idx].real if comp == "re" else g[idx].imag
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)) + floor, (idx, comp, fd, an, floor)


def test_welch_gradient_central_differences():
    """welch_gradient against central differences of the Welch loss sum dLdS * S_welch
    (overlapping segments, skipped leading frames), probed on frames of one, two and no segments."""
    psi, dLdS, kw = _grad_case()
    P, T, Ky, Kx = psi.shape
    L, stride, skip = 12, 5, 3
    rng = np.random.default_rng(11)
    n = skip + 3 * stride + L
    seq = (rng.standard_normal((P, n, Ky, Kx)) + 1j * rng.standard_normal((P, n, Ky, Kx)))
    g = oracle.welch_gradient(seq, dLdS, L, stride, skip_init=skip, **kw)

    def welch_loss(x):
        return float(np.sum(dLdS * oracle.welch_forward(x, L, stride, skip_init=skip, **kw).S))

    h = 1e-6
    floor = 16 * np.finfo(np.float64).eps * abs(welch_loss(seq)) / h + 1e-9
    assert np.all(g[:, :skip] == 0)
    for t in (0, skip, skip + 2, skip + 6, skip + 11, skip + 13, n - 1):
        for _ in range(4):
            idx = (int(rng.integers(0, P)), t, int(rng.integers(0, Ky)), int(rng.integers(0, Kx)))
            for comp, unit in (("re", 1.0), ("im", 1j)):
                a = seq.copy()
                b = seq.copy()
                a[idx] += h * unit
                b[idx] -= h * unit
                fd = (welch_loss(a) - welch_loss(b)) / (2 * h)
                an = g[idx].real if comp == "re" else g[idx].imag
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + floor, (idx, comp, fd, an, floor)


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    psi, dLdS, kw = _grad_case(9)
    g = oracle.gradient(psi, dLdS, **kw)
    P, T, Ky, Kx = psi.shape
    E = kw["E_meV"]
    x = torch.tensor(psi, dtype=torch.complex128, requires_grad=True)
    w = torch.tensor(scipy.signal.get_window("hann", T, fftbins=True))
    c = torch.tensor(E * 5.0e-3 / 4.135667696)
    n = torch.arange(T, dtype=torch.float64)
    F = torch.exp(-2j * torch.pi * torch.outer(n, c))                      # [T, Nw]
    y = w[None, :, None, None] * (x - x.mean(dim=1, keepdim=True))
    Psi = torch.einsum("ptyx,tj->pjyx", y, F)
    B = torch.tensor(oracle.bose(E, 300.0))
    I = (Psi.abs() ** 2) * B[None, :, None, None]
    M = torch.tensor(oracle.detector_masks(Kx, Ky, kw["detectors"]))
    S = torch.einsum("pjyx,dyx->pdj", I, M)
    L = (torch.tensor(dLdS) * S).sum()
    L.backward()
    np.testing.assert_allclose(x.grad.numpy(), g, rtol=1e-10, atol=1e-12 * np.abs(g).max())


def test_pixel_gradient_equals_full_gradient_on_pixels():
    """Pixels are independent: the per-pixel gradient is the full gradient restricted to them."""
    psi, dLdS, kw = _grad_case(11)
    g = oracle.gradient(psi, dLdS, **kw)
    P, T, Ky, Kx = psi.shape
    M = oracle.detector_masks(Kx, Ky, kw["detectors"]).reshape(len(kw["detectors"]), -1)
    kw2 = {k: v for k, v in kw.items() if k != "detectors"}
    for p in range(P):
        series = psi[p].reshape(T, -1)
        gp = oracle.gradient_pixels(series, dLdS[p], M.T, **kw2)
        np.testing.assert_allclose(gp, g[p].reshape(T, -1), rtol=1e-10, atol=1e-12 * np.abs(g).max())
        Lp = oracle.loss_pixels(series, dLdS[p], M.T, **kw2)
        Lfull = float(np.sum(dLdS[p] * oracle.forward(psi[p:p + 1], **kw).S[0]))
        assert abs(Lp - Lfull) <= 1e-10 * abs(Lfull)


@pytest.mark.parametrize("grid", ["fft", "offgrid"])
@pytest.mark.parametrize("mean", [True, False])
@pytest.mark.parametrize("bose_T", [0.0, 300.0])
@pytest.mark.parametrize("win", [("hann", 0.0), ("gauss", 7.0), ("kaiser", 3 * np.pi)])
def test_pixel_forward_equals_full_forward_on_pixels(grid, mean, bose_T, win):
    """forward_pixels, the checker of every sampled full-size parity test, equals the full-array
    forward (pinned above by numpy.fft, closed forms, Wiener-Khinchin and brute force) element by
    element: Psi and I at every pixel of every probe, with the Bose factor on and off, FFT and
    off-grid (signed) energies, the mean removed or kept."""
    rng = np.random.default_rng(31)
    P, T, Ky, Kx = 2, 40, 5, 6
    psi = rand_psi(P, T, Ky, Kx, rng) + 3.0
    kw = dict(window_kind=win[0], window_param=win[1], dt_fs=5.0, subtract_mean=mean, bose_T_K=bose_T)
    if grid == "fft":
        kw["fft_bins"] = 24
    else:
        kw["E_meV"] = np.linspace(-37.0, 111.0, 29)
    full = oracle.forward(psi, **kw)
    for p in range(P):
        Psi, I = oracle.forward_pixels(psi[p].reshape(T, -1), **kw)
        ref_Psi = full.Psi[p].reshape(full.Psi.shape[1], -1)
        ref_I = full.I[p].reshape(full.I.shape[1], -1)
        np.testing.assert_allclose(Psi, ref_Psi, rtol=1e-12, atol=1e-12 * np.abs(ref_Psi).max())
        np.testing.assert_allclose(I, ref_I, rtol=1e-12, atol=1e-12 * np.abs(ref_I).max())
    # and per selected pixel columns (the sampled form the large tests use)
    sel = [0, 7, 29]
    Psi, I = oracle.forward_pixels(psi[1].reshape(T, -1)[:, sel], **kw)
    np.testing.assert_allclose(I, full.I[1].reshape(full.I.shape[1], -1)[:, sel], rtol=1e-12,
                               atol=1e-12 * np.abs(full.I).max())


# ------------------------------------------------------------------------------------ Welch
def test_welch_segment_starts_and_stride():
    """s_{n+1} = s_n + L // nu (remainder-less); whole segments only."""
    assert oracle.welch_stride(200, 2.0) == 100 and oracle.welch_stride(200, 3.0) == 66
    st = oracle.welch_segments(3200, 200, 100)
    assert len(st) == 31 and st[0] == 0 and np.all(np.diff(st) == 100) and st[-1] + 200 == 3200
    assert len(oracle.welch_segments(3299, 200, 100)) == 31
    assert len(oracle.welch_segments(199, 200, 100)) == 0


def test_welch_single_segment_is_the_plain_definition():
    rng = np.random.default_rng(71)
    psi = rand_psi(2, 40, 3, 4, rng)
    kw = dict(window_kind="hann", E_meV=np.linspace(0, 90, 9) + 0.3, dt_fs=5.0, subtract_mean=True,
              detectors=[Detector("circular", 0, 0, -1, 1.5)])
    a = oracle.welch_forward(psi, 40, 13, **kw)
    b = oracle.forward(psi, **kw)
    np.testing.assert_allclose(a.I, b.I, rtol=0, atol=0)
    np.testing.assert_allclose(a.S, b.S, rtol=0, atol=0)


@pytest.mark.parametrize("L,stride,win", [(64, 32, "hann"), (60, 20, "hann"), (50, 50, "rect"),
                                          (64, 21, "tukey"), (48, 16, "rect")])
def test_welch_matches_scipy_welch(L, stride, win):
    """On the FFT grid, I_welch = scipy.signal.welch(..., detrend='constant', scaling='spectrum',
    two-sided) * (sum of the window)^2: per-segment mean removal, window, |DFT|^2, 1/N average."""
    rng = np.random.default_rng(72)
    n = 5 * L + 7
    t = np.arange(n)
    x = (0.7 + 0.2j + np.exp(2j * np.pi * 0.137 * t) + 0.4 * np.exp(-2j * np.pi * 0.31 * t)
         + 0.3 * (rng.standard_normal(n) + 1j * rng.standard_normal(n)))
    psi = np.broadcast_to(x[None, :, None, None], (1, n, 1, 1)).copy()
    param = 0.3 if win == "tukey" else 0.0
    r = oracle.welch_forward(psi, L, stride, window_kind=win, window_param=param, fft_bins=L, dt_fs=5.0)
    sw = {"hann": "hann", "rect": "boxcar", "tukey": ("tukey", 0.3)}[win]
    _, pxx = scipy.signal.welch(x, window=sw, nperseg=L, noverlap=L - stride, detrend="constant",
                                return_onesided=False, scaling="spectrum", average="mean")
    wsum = oracle.window(win, L, param).sum()
    np.testing.assert_allclose(r.I[0, :, 0, 0], pxx * wsum ** 2, rtol=1e-9, atol=1e-9 * np.max(pxx) * wsum ** 2)


@pytest.mark.parametrize("skip", [1, 37, 64])
def test_welch_skip_init_matches_scipy_on_the_remaining_frames(skip):
    """skip_init drops the leading frames (an initial transient here) before the first segment:
    the result is scipy's Welch estimate of the frames after them."""
    rng = np.random.default_rng(73)
    L, stride = 64, 32
    n = skip + 4 * stride + L
    t = np.arange(n)
    x = (0.5 - 0.1j + np.exp(2j * np.pi * 0.21 * t) + 0.2 * (rng.standard_normal(n) + 1j * rng.standard_normal(n)))
    x[:skip] += 50.0 * np.exp(-t[:skip] / 7.0)                       # transient that must not leak in
    psi = x[None, :, None, None].copy()
    r = oracle.welch_forward(psi, L, stride, skip_init=skip, window_kind="hann", fft_bins=L, dt_fs=5.0)
    _, pxx = scipy.signal.welch(x[skip:], window="hann", nperseg=L, noverlap=L - stride, detrend="constant",
                                return_onesided=False, scaling="spectrum", average="mean")
    wsum = oracle.window("hann", L).sum()
    np.testing.assert_allclose(r.I[0, :, 0, 0], pxx * wsum ** 2, rtol=1e-9, atol=1e-9 * np.max(pxx) * wsum ** 2)
    assert len(oracle.welch_segments(n - skip, L, stride)) == 5
