"""Pins for oracle.twopt: shell counts by brute force, identities of r_c/s/TF,
white-noise and linear-field spectra."""
import itertools

import numpy as np
import pytest

from oracle import cosmo, pm, twopt
from paper_1805_02247_gb300 import synth


def test_shell_counts_by_brute_force():
    N = 8
    a = synth.gaussian_vector((N, N, N), seed=1)
    counts, *_ = twopt.power_spectra(a, a, 10.0)
    freqs = range(-N // 2 + 1, N // 2 + 1)  # one representative per full-grid mode
    want = np.zeros(N // 2)
    for n in itertools.product(freqs, repeat=3):
        r = np.sqrt(sum(x * x for x in n))
        i = int(np.floor(r - 0.5))
        if 0 <= i < N // 2:
            want[i] += 1
    assert np.array_equal(counts, want)


def test_identities_of_the_statistics():
    N, L = 16, 50.0
    a = synth.gaussian_vector((N, N, N), seed=2).astype(np.float64)
    b = synth.gaussian_vector((N, N, N), seed=3).astype(np.float64)
    _, paa, pbb, pab = twopt.power_spectra(a, a, L)
    rc, s, tf = twopt.statistics(paa, pbb, pab)
    assert np.allclose(rc, 1.0, atol=1e-12) and np.allclose(s, 0.0, atol=1e-10) and np.allclose(tf, 1.0)
    _, paa, pbb, pab = twopt.power_spectra(a, -2.0 * a, L)
    rc, s, tf = twopt.statistics(paa, pbb, pab)
    assert np.allclose(rc, -1.0, atol=1e-12) and np.allclose(tf, 2.0)
    # independent fields: |r_c| ~ 1/sqrt(modes per shell)
    c, paa, pbb, pab = twopt.power_spectra(a, b, L)
    rc, _, _ = twopt.statistics(paa, pbb, pab)
    assert np.all(np.abs(rc[2:]) < 5.0 / np.sqrt(c[2:]))


def test_white_noise_spectrum_is_flat():
    # <|A_k|^2> = N^3 sigma^2  =>  P = L^3 sigma^2 / N^3
    N, L = 32, 80.0
    a = synth.gaussian_vector((N, N, N), seed=4).astype(np.float64)
    c, paa, _, _ = twopt.power_spectra(a, a, L)
    want = L**3 / N**3
    m = c > 100
    assert np.all(np.abs(paa[m] / want - 1.0) < 5.0 / np.sqrt(c[m]))


def test_linear_field_recovers_the_input_power():
    N, L = 64, 400.0
    setup = pm.PMSetup(N=N, L=L, nsteps=1)
    s = pm.linear_field(synth.white_noise(N, 7), setup)
    delta = pm.irfft3(s)
    c, p, _, _ = twopt.power_spectra(delta, delta, L)
    k = twopt.shell_k(N, L)
    # shells average P over |n| in [i + 1/2, i + 3/2); compare with the mode-weighted
    # mean of P_lin over the same modes
    sh = twopt.shell_index(N)
    kk = np.sqrt(pm.k_squared(N)) * N / L
    w = pm.half_weights(N)
    m = sh >= 0
    want = np.bincount(sh[m], weights=(w * cosmo.P_lin_array(kk))[m], minlength=N // 2) / c
    ok = c > 500
    assert np.all(np.abs(p[ok] / want[ok] - 1.0) < 5.0 * np.sqrt(2.0 / c[ok]))
    assert k[0] == pytest.approx(2 * np.pi / L)


def _orthogonal_pair(N, seed):
    """A field a and a field n whose Fourier modes are in quadrature mode by mode
    (n_k = i c(k) a_k with c real and odd: here a scaled x-derivative with its
    Nyquist plane zeroed), so Re(a_k conj(n_k)) = 0 for every mode and every
    shell sum of the cross term vanishes exactly, not only on average."""
    a = synth.gaussian_vector((N, N, N), seed=seed).astype(np.float64)
    A = np.fft.rfftn(a)
    kx = np.fft.fftfreq(N, d=1.0 / N)[:, None, None] * np.ones((1, N, N // 2 + 1))
    kx[N // 2] = 0.0
    n = np.fft.irfftn(1j * 0.3 * kx * A, s=(N, N, N), axes=(0, 1, 2))
    return a, n


def test_stochasticity_is_the_noise_power_when_data_is_signal_plus_orthogonal_noise():
    # h = a + n with n in quadrature with a: P_hm = P_mm = P_aa, P_hh = P_aa + P_nn
    # per shell exactly, so r_c = sqrt(P_aa / P_hh), TF = sqrt(P_aa / P_hh) and
    # the stochasticity s = P_hh (1 - r_c^2) = P_hh - P_aa is the noise power P_nn.
    # The noise grows with |k|, so r_c falls strictly inside (0, 1) and a missing
    # P_hh factor (s = 1 - r_c^2) or the wrong auto spectrum in front fails.
    N, L = 16, 50.0
    a, n = _orthogonal_pair(N, seed=8)
    h = a + n
    _, P_hh, P_mm, P_hm = twopt.power_spectra(h, a, L)
    rc, s, tf = twopt.statistics(P_hh, P_mm, P_hm)
    _, P_nn, _, _ = twopt.power_spectra(n, n, L)
    _, P_aa, _, _ = twopt.power_spectra(a, a, L)
    assert np.all((rc[1:] > 0.05) & (rc[1:] < 0.99))
    assert np.allclose(s, P_nn, rtol=1e-10, atol=0)
    assert np.allclose(rc, np.sqrt(P_aa / (P_aa + P_nn)), rtol=1e-10)
    assert np.allclose(tf, np.sqrt(P_aa / (P_aa + P_nn)), rtol=1e-10)
    # anti-correlated: the model is -a; r_c changes sign, s and TF do not
    _, P_hh2, P_mm2, P_hm2 = twopt.power_spectra(h, -a, L)
    rc2, s2, tf2 = twopt.statistics(P_hh2, P_mm2, P_hm2)
    assert np.allclose(rc2, -rc, rtol=1e-10) and np.allclose(s2, s, rtol=1e-10) and np.allclose(tf2, tf, rtol=1e-10)


def test_stochasticity_scales_with_the_data_amplitude():
    # s carries the units of a power spectrum: scaling the data by 3 scales s by
    # 9 and leaves r_c unchanged; TF = sqrt(P_mm / P_hh) drops by 3
    N, L = 16, 50.0
    a, n = _orthogonal_pair(N, seed=9)
    st1 = twopt.statistics(*twopt.power_spectra(a + n, a, L)[1:])
    st3 = twopt.statistics(*twopt.power_spectra(3.0 * (a + n), a, L)[1:])
    assert np.allclose(st3[0], st1[0], rtol=1e-12)
    assert np.allclose(st3[1], 9.0 * st1[1], rtol=1e-12)
    assert np.allclose(st3[2], st1[2] / 3.0, rtol=1e-12)
