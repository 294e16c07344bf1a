"""Two-point statistics of Sec. 4.3 (FP64, numpy).

Cross-correlation r_c = P_hN / sqrt(P_hh P_NN), stochasticity s = P_hh (1 - r_c^2)
and transfer function TF = sqrt(P_NN / P_hh), with P_ab(k) the (cross) power
spectrum of two fields in shells of |k|.

Conventions (the paper does not fix a binning):
* P_ab(k) = V / N^6 < Re(A_k conj(B_k)) > over the modes of a shell, where
  A = rfftn(a) is the unnormalised DFT of a real mesh field and V = L^3; for the
  linear field this returns P(k) (<|s_k|^2> = P N^6 / V).
* Shell i holds the modes with integer wavevector n (k = 2 pi n / L) whose norm
  satisfies i + 1/2 <= |n| < i + 3/2, i = 0 .. N/2 - 1; k = 0 belongs to none.
* Modes are counted over the full grid: each half-array entry has the weight
  w = 2 for 0 < k_z < N/2 and 1 on the k_z = 0 and N/2 planes.
"""
from __future__ import annotations

import numpy as np

from . import pm


def shell_index(N: int) -> np.ndarray:
    """Shell of every half-array entry (-1 for k = 0 or beyond the last shell)."""
    n_full = np.fft.fftfreq(N, d=1.0 / N)
    n_half = np.arange(N // 2 + 1)
    n2 = n_full[:, None, None] ** 2 + n_full[None, :, None] ** 2 + n_half[None, None, :] ** 2
    shell = np.floor(np.sqrt(n2) - 0.5).astype(np.int64)
    shell[(shell < 0) | (shell >= N // 2)] = -1
    return shell


def power_spectra(a: np.ndarray, b: np.ndarray, L: float):
    """Returns (counts, P_aa, P_bb, P_ab), each of length N/2."""
    N = a.shape[0]
    A = np.fft.rfftn(np.asarray(a, np.float64))
    B = np.fft.rfftn(np.asarray(b, np.float64))
    w = pm.half_weights(N)
    sh = shell_index(N)
    m = sh >= 0
    nb = N // 2
    counts = np.bincount(sh[m], weights=w[m], minlength=nb)
    norm = L**3 / float(N) ** 6

    def binned(v):
        return np.bincount(sh[m], weights=(w * v)[m], minlength=nb) / np.maximum(counts, 1) * norm

    return counts, binned(np.abs(A) ** 2), binned(np.abs(B) ** 2), binned((A * np.conj(B)).real)


def shell_k(N: int, L: float) -> np.ndarray:
    """Nominal wavenumber of each shell, (i + 1) * 2 pi / L in h/Mpc."""
    return (np.arange(N // 2) + 1) * 2 * np.pi / L


def statistics(P_hh, P_NN, P_hN):
    """(r_c, s, TF) of Sec. 4.3 from binned spectra (h: truth/data, N: model)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        rc = P_hN / np.sqrt(P_hh * P_NN)
        s = P_hh * (1.0 - rc**2)
        tf = np.sqrt(P_NN / P_hh)
    return rc, s, tf
