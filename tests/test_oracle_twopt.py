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
