"""Pins for oracle.cosmo: closed forms, an independent ODE solve, quadrature."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import cosmo, pm


def test_einstein_de_sitter_closed_form():
    # Omega_m = 1: D = a, G_p = a^3 E dD/da = a^1.5, G_f = 1.5 a
    for a in (0.05, 0.1, 0.37, 1.0):
        assert cosmo.D(a, 1.0) == pytest.approx(a, rel=1e-11)
        assert cosmo.Gp(a, 1.0) == pytest.approx(a**1.5, rel=1e-10)
        assert cosmo.Gf(a, 1.0) == pytest.approx(1.5 * a, rel=1e-11)


def test_growth_matches_ode_solution():
    # Independent route: integrate D'' + (3/a + E'/E) D' - 1.5 Om D / (a^5 E^2) = 0
    om = cosmo.OMEGA_M
    E = lambda a: math.sqrt(om / a**3 + 1 - om)
    dE = lambda a: -1.5 * om / a**4 / E(a)

    def rhs(a, y):
        d, v = y
        return [v, -(3 / a + dE(a) / E(a)) * v + 1.5 * om * d / (a**5 * E(a) ** 2)]

    a_start = 1e-4  # deep in matter domination: D = a
    sol = solve_ivp(rhs, (a_start, 1.0), [a_start, 1.0], rtol=1e-12, atol=1e-16, dense_output=True)
    d1 = sol.sol(1.0)[0]
    for a in (0.1, 0.25, 0.5, 0.8):
        assert cosmo.D(a) == pytest.approx(sol.sol(a)[0] / d1, rel=2e-7)
        assert cosmo.dDda(a) == pytest.approx(sol.sol(a)[1] / d1, rel=2e-7)


def test_momentum_force_growth_identity():
    # linear growth equation: dG_p/da = G_f / (a^2 E)
    for a in (0.1, 0.3, 0.7, 1.0):
        h = 1e-5
        deriv = (cosmo.Gp(a + h) - cosmo.Gp(a - h)) / (2 * h)
        assert deriv == pytest.approx(cosmo.Gf(a) / (a**2 * cosmo.E(a)), rel=1e-8)


def test_bbks_limits():
    assert cosmo.T_bbks(1e-9) == pytest.approx(1.0, abs=1e-7)
    ks = np.logspace(-3, 1, 50)
    t = cosmo.T_bbks_array(ks)
    assert np.all(np.diff(t) < 0)
    # large-k asymptote: T ~ ln(2.34 q) / (2.34 q) / (6.71 q)
    q = 1e4 / cosmo.GAMMA_BBKS
    assert cosmo.T_bbks(1e4) == pytest.approx(math.log(2.34 * q) / (2.34 * q) / (6.71 * q), rel=1e-3)
    assert np.allclose(t, [cosmo.T_bbks(k) for k in ks], rtol=1e-14)


def test_sigma8_by_independent_quadrature():
    # trapezoid in ln k on a fine grid (a different rule than the adaptive quad)
    lnk = np.linspace(np.log(1e-6), np.log(1e3), 400001)
    k = np.exp(lnk)
    x = k * 8.0
    W = np.where(x < 1e-3, 1 - x**2 / 10, 3 * (np.sin(x) - x * np.cos(x)) / np.maximum(x, 1e-30) ** 3)
    integrand = k**3 * cosmo.P_lin_array(k) * W**2 / (2 * np.pi**2)
    s8 = np.sqrt(np.trapezoid(integrand, lnk))
    assert s8 == pytest.approx(0.8, rel=1e-6)


def test_linear_field_power_normalisation():
    # <|s_k|^2> = P(k) N^6 / L^3: the mean of |s|^2 / P~ over many modes is 1
    setup = pm.PMSetup(N=64, L=400.0, nsteps=1)
    white = np.random.default_rng(5).standard_normal((64, 64, 64))
    s = pm.linear_field(white, setup)
    P = pm.power_half(setup)
    w = pm.half_weights(64)
    m = P > 0
    ratio = np.sum((w * np.abs(s) ** 2)[m] / P[m]) / np.sum(w[m])
    assert ratio == pytest.approx(1.0, abs=0.01)
    assert s[0, 0, 0] == 0
