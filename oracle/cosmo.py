"""Background cosmology, linear growth and the linear power spectrum (FP64).

Sec. 3 fixes a flat LCDM model with h = 0.6711 and Omega_m = 0.3175. The
paper's CAMB spectrum is not available; the linear spectrum here is the
BBKS fitting form with shape parameter Gamma = 0.21 and sigma_8 = 0.8 (the
synthetic workload), P(k) = A k T(k)^2.

Time variable is the scale factor a; H0 = 1 in code units, so E(a) = H/H0.
Growth follows the integral solution for a pressureless matter + Lambda
universe, D(a) proportional to E(a) * int_0^a da' / (a' E(a'))^3,
normalised to D(1) = 1. The momentum and force growth factors used by the
kick-drift stepping are G_p(a) = a^3 E(a) dD/da and G_f(a) = 1.5 Omega_m D(a),
which obey dG_p/da = G_f / (a^2 E) (the linear growth equation).
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
from scipy import integrate

OMEGA_M = 0.3175  # Sec. 3
H_LITTLE = 0.6711  # Sec. 3
GAMMA_BBKS = 0.21
SIGMA8 = 0.8


def E(a: float, om: float = OMEGA_M) -> float:
    return math.sqrt(om / a**3 + (1.0 - om))


def dEda(a: float, om: float = OMEGA_M) -> float:
    return -1.5 * om / a**4 / E(a, om)


def _growth_integral(a: float, om: float) -> float:
    val, _ = integrate.quad(lambda x: 1.0 / (x * E(x, om)) ** 3, 0.0, a, epsabs=0.0, epsrel=1e-13, limit=200)
    return val


@lru_cache(maxsize=None)
def _norm(om: float) -> float:
    return E(1.0, om) * _growth_integral(1.0, om)


def D(a: float, om: float = OMEGA_M) -> float:
    """Linear growth factor, D(1) = 1."""
    return E(a, om) * _growth_integral(a, om) / _norm(om)


def dDda(a: float, om: float = OMEGA_M) -> float:
    """Derivative of D by differentiating the integral form."""
    ea = E(a, om)
    return (dEda(a, om) * _growth_integral(a, om) + ea / (a * ea) ** 3) / _norm(om)


def Gp(a: float, om: float = OMEGA_M) -> float:
    """Momentum growth: p = G_p(a) psi for a Zel'dovich trajectory x = q + D psi."""
    return a**3 * E(a, om) * dDda(a, om)


def Gf(a: float, om: float = OMEGA_M) -> float:
    """Force growth: F = G_f(a) psi in the linear regime (Poisson: lap phi = 1.5 Om delta)."""
    return 1.5 * om * D(a, om)


def T_bbks(k: float, gamma: float = GAMMA_BBKS) -> float:
    """Bardeen, Bond, Kaiser & Szalay (1986) transfer-function fit, q = k / Gamma (k in h/Mpc)."""
    if k <= 0.0:
        return 1.0
    q = k / gamma
    return (math.log(1.0 + 2.34 * q) / (2.34 * q)
            * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25)


def tophat_window(x: float) -> float:
    """Fourier transform of a unit real-space top hat, 3 (sin x - x cos x) / x^3."""
    if x < 1e-3:
        return 1.0 - x * x / 10.0
    return 3.0 * (math.sin(x) - x * math.cos(x)) / x**3


def sigma_R_sq(amp: float, R: float, gamma: float = GAMMA_BBKS, ns: float = 1.0) -> float:
    """sigma^2(R) = 1/(2 pi^2) int k^2 P(k) W(kR)^2 dk, integrated in ln k."""
    def integrand(lnk):
        k = math.exp(lnk)
        return k**3 * amp * k**ns * T_bbks(k, gamma) ** 2 * tophat_window(k * R) ** 2
    val, _ = integrate.quad(integrand, math.log(1e-6), math.log(1e3), epsabs=0.0, epsrel=1e-12, limit=1000)
    return val / (2.0 * math.pi**2)


@lru_cache(maxsize=None)
def bbks_amplitude(sigma8: float = SIGMA8, gamma: float = GAMMA_BBKS) -> float:
    """A such that P(k) = A k T(k)^2 has sigma_8 = sigma8 (top hat of 8 Mpc/h)."""
    return sigma8**2 / sigma_R_sq(1.0, 8.0, gamma)


def P_lin(k: float, sigma8: float = SIGMA8, gamma: float = GAMMA_BBKS) -> float:
    """Linear power at a = 1 in (Mpc/h)^3, k in h/Mpc."""
    return bbks_amplitude(sigma8, gamma) * k * T_bbks(k, gamma) ** 2


def T_bbks_array(k: np.ndarray, gamma: float = GAMMA_BBKS) -> np.ndarray:
    """Vectorised T_bbks; T(0) = 1."""
    k = np.asarray(k, dtype=np.float64)
    q = np.where(k > 0, k, 1.0) / gamma
    t = (np.log1p(2.34 * q) / (2.34 * q)
         * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25)
    return np.where(k > 0, t, 1.0)


def P_lin_array(k: np.ndarray, sigma8: float = SIGMA8, gamma: float = GAMMA_BBKS) -> np.ndarray:
    k = np.asarray(k, dtype=np.float64)
    return bbks_amplitude(sigma8, gamma) * k * T_bbks_array(k, gamma) ** 2
