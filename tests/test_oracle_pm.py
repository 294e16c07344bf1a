"""Pins for oracle.pm: transposes, closed forms, conservation, brute force, ZA exactness."""
import numpy as np
import pytest

from oracle import cosmo, pm
from paper_1805_02247_gb300 import synth


def rdot(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.sum(a.real * b.real + a.imag * b.imag))


def test_irfft_transpose_on_arbitrary_half_arrays():
    # holds for non-Hermitian half arrays too: irfftn ignores the imaginary
    # parts of self-conjugate entries and averages k_z in {0, N/2} pairs
    rng = np.random.default_rng(1)
    N = 6
    u = rng.standard_normal((N, N, N // 2 + 1)) + 1j * rng.standard_normal((N, N, N // 2 + 1))
    lam = rng.standard_normal((N, N, N))
    assert rdot(pm.irfft3(u), lam) == pytest.approx(rdot(u, pm.irfft3_T(lam)), rel=1e-12)


def test_irfft_transpose_brute_force_entries():
    # directional derivative of <irfft(u), lam> along single real/imaginary entries
    rng = np.random.default_rng(2)
    N = 4
    lam = rng.standard_normal((N, N, N))
    g = pm.irfft3_T(lam)
    for idx in [(0, 0, 0), (1, 2, 0), (3, 1, 1), (2, 0, 2), (0, 0, 2), (2, 2, 2)]:
        for part in (1.0, 1j):
            e = np.zeros((N, N, N // 2 + 1), complex)
            e[idx] = part
            val = float(np.sum(pm.irfft3(e) * lam))
            want = g[idx].real if part == 1.0 else g[idx].imag
            assert val == pytest.approx(want, abs=1e-13)


def test_force_of_single_mode_is_closed_form():
    # delta = A cos(k.x) -> F = -1.5 Om A (k / k^2) sin(k.x)
    N, A, om = 16, 0.7, cosmo.OMEGA_M
    n = np.array([2, -3, 1])
    x = np.indices((N, N, N)).astype(float)
    phase = 2 * np.pi / N * (n[0] * x[0] + n[1] * x[1] + n[2] * x[2])
    F = pm.force(A * np.cos(phase), om)
    k = 2 * np.pi / N * n
    for j in range(3):
        want = -1.5 * om * A * k[j] / np.dot(k, k) * np.sin(phase)
        assert np.allclose(F[j], want, atol=1e-12)


def test_force_transpose():
    rng = np.random.default_rng(3)
    N = 8
    d = rng.standard_normal((N, N, N))
    G = rng.standard_normal((3, N, N, N))
    assert rdot(pm.force(d, 0.3), G) == pytest.approx(rdot(d, pm.force_T(G, 0.3)), rel=1e-12)


def test_smoothing_single_mode_and_self_adjoint():
    N, R = 16, 1.7
    n = np.array([1, 2, -2])
    x = np.indices((N, N, N)).astype(float)
    k = 2 * np.pi / N * n
    f = np.cos(k[0] * x[0] + k[1] * x[1] + k[2] * x[2])
    assert np.allclose(pm.smooth(f, R), np.exp(-0.5 * np.dot(k, k) * R * R) * f, atol=1e-13)
    rng = np.random.default_rng(4)
    a, b = rng.standard_normal((2, N, N, N))
    assert rdot(pm.smooth(a, R), b) == pytest.approx(rdot(a, pm.smooth(b, R)), rel=1e-12)


def test_cic_mass_conservation_and_special_positions():
    N = 8
    x = synth.uniform_positions(N, 1000, seed=7, lo=-3.0, hi=11.0).astype(np.float64)
    rho = pm.paint(x, N)
    assert rho.sum() == pytest.approx(1000.0, rel=1e-13)
    # integer position: all mass in one cell
    rho = pm.paint(np.array([[3.0], [5.0], [7.0]]), N)
    assert rho[3, 5, 7] == 1.0 and rho.sum() == 1.0
    # cell centre between grid points: 1/8 to each of 8 cells, across the periodic edge
    rho = pm.paint(np.array([[7.5], [0.5], [7.5]]), N)
    for ox in (7, 0):
        for oy in (0, 1):
            for oz in (7, 0):
                assert rho[ox, oy, oz] == pytest.approx(0.125)


def test_cic_paint_readout_transpose_and_linear_interpolation():
    rng = np.random.default_rng(5)
    N = 8
    x = rng.uniform(-N, 2 * N, size=(3, 300))
    m = rng.standard_normal(300)
    g = rng.standard_normal((N, N, N))
    assert rdot(pm.paint(x, N, m), g) == pytest.approx(rdot(m, pm.readout(g, x)), rel=1e-12)
    # readout of a field linear in x inside one cell interpolates exactly
    f = np.broadcast_to(np.arange(N, dtype=float)[:, None, None], (N, N, N)).copy()
    xi = np.array([[2.25, 5.5], [1.0, 3.3], [0.7, 7.0]])
    assert np.allclose(pm.readout(f, xi), [2.25, 5.5])


def test_readout_grad_by_finite_differences():
    rng = np.random.default_rng(6)
    N = 6
    g = rng.standard_normal((N, N, N))
    x = np.floor(rng.uniform(0, N, size=(3, 50))) + rng.uniform(0.1, 0.9, size=(3, 50))
    G = pm.readout_grad(g, x)
    h = 1e-6
    for a in range(3):
        e = np.zeros_like(x); e[a] = h
        fd = (pm.readout(g, x + e) - pm.readout(g, x - e)) / (2 * h)
        assert np.allclose(G[a], fd, atol=1e-8)


def test_wrap_and_keys_on_edge_values():
    N = 4
    f = np.float32
    cases = {
        0.0: 0, 1.0: 1, 3.5: 3, float(np.nextafter(f(4), f(0))): 3, 4.0: 0, 4.25: 0,
        -0.25: 3, -1e-8: 0, -1e-30: 0, -4.0: 0, 8.5: 0, 3.999999: 3,
    }
    for u, want in cases.items():
        x = np.array([[u], [0.0], [0.0]], dtype=np.float32)
        assert pm.cell_keys(x, N)[0] == want * N * N, u
    # -1e-8 + 4 rounds to 4.0 in float32, which the rule maps to 0
    assert pm.wrap_f32(np.float32(-1e-8), N) == 0.0
    assert pm.wrap_f32(np.float32(-0.25), N) == np.float32(3.75)


def test_counting_sort_is_stable_brute_force():
    N = 4
    x = synth.uniform_positions(N, 200, seed=8, lo=-2, hi=6)
    keys = pm.cell_keys(x, N)
    perm, start = pm.sort_by_cell(keys, N)
    want = sorted(range(200), key=lambda i: (int(keys[i]), i))
    assert list(perm) == want
    assert start[0] == 0 and start[-1] == 200
    for c in range(N**3):
        assert all(keys[perm[j]] == c for j in range(start[c], start[c + 1]))


def test_za_displacement_divergence_is_minus_delta():
    setup = pm.PMSetup(N=16, L=100.0, nsteps=1)
    s = pm.linear_field(synth.white_noise(16, 0), setup)
    psi = pm.za_displacement(s).reshape(3, 16, 16, 16)
    ks, nyq = pm.wavenumbers(16)
    div = sum(1j * ks[j] * pm.rfft3(psi[j]) for j in range(3))
    keep = ~(nyq[0] | nyq[1] | nyq[2])
    keep[0, 0, 0] = False
    assert np.allclose((-div)[keep], s[keep], rtol=1e-10, atol=1e-8 * np.abs(s).max())


def _plane_wave(N, amp):
    A = amp / (2 * np.pi / N)  # D(1) A k = amp
    s = np.zeros((N, N, N // 2 + 1), complex)
    # psi_x = A sin(k q)  <=>  delta_lin = -A k cos(k q): +-k entries of N^3 A k / 2
    s[1, 0, 0] = -A * (2 * np.pi / N) * N**3 / 2
    s[N - 1, 0, 0] = np.conj(s[1, 0, 0])
    return A, s


@pytest.mark.parametrize("amp", [0.5, 0.005])
def test_plane_wave_follows_zeldovich_until_shell_crossing(amp):
    # A 1D plane wave is exact in Zel'dovich until shell crossing (D A k < 1).
    # With kick/drift factors built from D and G_p, PM reproduces x = q + D(a) psi
    # for any number of steps, up to the CIC window of paint + readout,
    # sinc(k/2)^4 = 0.9936 at k = 2 pi / 32. The sign-dependent half-cell shift of
    # CIC on a displaced lattice only feeds higher harmonics, so compare the
    # fundamental-mode amplitude of the displacement.
    N = 32
    A, s = _plane_wave(N, amp)
    q = pm.lattice(N)
    basis = np.sin(2 * np.pi / N * q[0])
    assert np.allclose(pm.za_displacement(s)[0], A * basis, atol=1e-10)
    got = {}
    for nsteps in (2, 5, 40):
        x, _, _ = pm.pm_forward(s, pm.PMSetup(N=N, L=100.0, nsteps=nsteps))
        got[nsteps] = np.sum((x[0] - q[0]) * basis) / np.sum(basis**2) / A
        assert np.max(np.abs(x[1] - q[1])) < 1e-12 and np.max(np.abs(x[2] - q[2])) < 1e-12
    window = np.sinc(1.0 / N) ** 4  # np.sinc(t) = sin(pi t)/(pi t); k/2 = pi/N
    for nsteps, ratio in got.items():
        assert ratio == pytest.approx(cosmo.D(1.0) * window, abs=3e-3), (nsteps, ratio)
    assert abs(got[2] - got[40]) < 3e-3


def test_large_scale_growth_follows_D():
    # small-amplitude field: the large-scale overdensity grows by D(1)/D(a0)
    # between the ICs and the end of the PM run (both painted with CIC, so the
    # paint window cancels; the force windows leave < 1% at 6.25 Mpc/h cells)
    N, L = 64, 400.0
    setup = pm.PMSetup(N=N, L=L, nsteps=5)
    s = 0.01 * pm.linear_field(synth.white_noise(N, 3), setup)
    x0, _ = pm.za_ics(s, setup)
    d0 = pm.rfft3(pm.density(x0, N))
    d1 = pm.rfft3(pm.final_density(s, setup))
    k2 = pm.k_squared(N)
    for shell in (1.01, 2.01, 3.01):
        low = (k2 > 0) & (k2 <= (2 * np.pi / N * shell) ** 2)
        ratio = np.sqrt(np.sum(np.abs(d1[low]) ** 2) / np.sum(np.abs(d0[low]) ** 2))
        assert ratio == pytest.approx(cosmo.D(1.0) / cosmo.D(0.1), rel=0.01)


@pytest.mark.parametrize("N,nsteps", [(8, 2), (16, 3)])
def test_pm_adjoint_by_finite_differences(N, nsteps):
    setup = pm.PMSetup(N=N, L=100.0, nsteps=nsteps)
    s = pm.linear_field(synth.white_noise(N, 0), setup)
    rng = np.random.default_rng(11)
    g_delta = rng.standard_normal((N, N, N))
    x_fin, cps, _ = pm.pm_forward(s, setup)
    grad = pm.final_density_T(cps, x_fin, g_delta, setup)
    f = lambda ss: float(np.sum(g_delta * pm.final_density(ss, setup)))
    for trial in range(3):
        v = pm.rfft3(rng.standard_normal((N, N, N))) * np.sqrt(pm.power_half(setup) / N**3)
        v[0, 0, 0] = 0
        # CIC is piecewise linear: a step small enough that no particle crosses a
        # cell face sees the smooth branch (1e-4 already crosses faces here)
        eps = 1e-6
        fd = (f(s + eps * v) - f(s - eps * v)) / (2 * eps)
        assert rdot(grad, v) == pytest.approx(fd, rel=1e-6)


# ----------------------------------------------------------------------------- 2LPT

def test_lpt2_vanishes_for_a_plane_wave():
    # one Fourier direction: only phi_xx is nonzero, the second-order source is
    # zero, and 2LPT reduces to Zel'dovich (exact in 1D before shell crossing)
    N = 16
    _, s = _plane_wave(N, 0.5)
    assert np.max(np.abs(pm.lpt2_displacement(s))) < 1e-12 * np.max(np.abs(pm.za_displacement(s)))
    setup2 = pm.PMSetup(N=N, L=100.0, nsteps=1, lpt_order=2)
    x2, p2 = pm.lpt_ics(s, setup2)
    x1, p1 = pm.za_ics(s, setup2)
    assert np.allclose(x2, x1, rtol=0, atol=1e-12) and np.allclose(p2, p1, rtol=0, atol=1e-12)


@pytest.mark.parametrize("axes", [(0, 1), (0, 2), (1, 2)])
def test_lpt2_closed_form_for_a_product_of_two_cosines(axes):
    # phi1 = A cos(a u) cos(b v) on two axes u, v (lap phi1 = delta): the source
    # is A^2 a^2 b^2 (cos 2au + cos 2bv) / 2, so phi2 = -(A^2/8)(b^2 cos 2au +
    # a^2 cos 2bv) and psi2 = grad phi2 = (A^2 a b / 4)(b sin 2au, a sin 2bv)
    N = 16
    u, v = axes
    a, b = 2 * np.pi * 1 / N, 2 * np.pi * 2 / N
    A = 0.7
    q = pm.lattice(N)
    phi = A * np.cos(a * q[u]) * np.cos(b * q[v])
    s = pm.rfft3((-(a * a + b * b) * phi).reshape(N, N, N))
    want = np.zeros((3, N ** 3))
    want[u] = A * A * a * b / 4 * b * np.sin(2 * a * q[u])
    want[v] = A * A * a * b / 4 * a * np.sin(2 * b * q[v])
    assert np.allclose(pm.lpt2_displacement(s), want, rtol=0, atol=1e-12)


def test_lpt2_source_on_a_diagonal_hessian_is_the_sum_of_pair_products():
    H = np.zeros((6, 2, 2, 2))
    H[0], H[1], H[2] = 2.0, 3.0, 5.0
    assert np.allclose(pm.lpt2_source(H), 2 * 3 + 2 * 5 + 3 * 5)
    H[3] = 1.0  # phi_xy enters squared with a minus sign
    assert np.allclose(pm.lpt2_source(H), 31 - 1)


def test_lpt_ics_adjoint_is_exact_for_the_quadratic_map():
    # x(s) and p(s) are quadratic in s, so central differences are exact
    N = 8
    setup = pm.PMSetup(N=N, L=100.0, nsteps=1, lpt_order=2)
    s = pm.linear_field(synth.white_noise(N, 0), setup)
    rng = np.random.default_rng(12)
    lx, lp = rng.standard_normal((3, N ** 3)), rng.standard_normal((3, N ** 3))
    g = pm.lpt_ics_T(lx, lp, s, setup)
    for _ in range(3):
        v = pm.rfft3(rng.standard_normal((N, N, N))) * np.sqrt(pm.power_half(setup) / N ** 3)
        eps = 0.1
        xp, pp = pm.lpt_ics(s + eps * v, setup)
        xm, pmm = pm.lpt_ics(s - eps * v, setup)
        fd = (np.sum(lx * (xp - xm)) + np.sum(lp * (pp - pmm))) / (2 * eps)
        assert rdot(g, v) == pytest.approx(fd, rel=1e-10)


def test_lpt2_pm_adjoint_by_finite_differences():
    N, nsteps = 8, 2
    setup = pm.PMSetup(N=N, L=100.0, nsteps=nsteps, lpt_order=2)
    s = pm.linear_field(synth.white_noise(N, 0), setup)
    rng = np.random.default_rng(13)
    g_delta = rng.standard_normal((N, N, N))
    x_fin, cps, _ = pm.pm_forward(s, setup)
    grad = pm.final_density_T(cps, x_fin, g_delta, setup, s)
    f = lambda ss: float(np.sum(g_delta * pm.final_density(ss, setup)))
    for _ in range(3):
        v = pm.rfft3(rng.standard_normal((N, N, N))) * np.sqrt(pm.power_half(setup) / N ** 3)
        v[0, 0, 0] = 0
        eps = 1e-6
        fd = (f(s + eps * v) - f(s - eps * v)) / (2 * eps)
        assert rdot(grad, v) == pytest.approx(fd, rel=1e-6)


def _f2_kernel(k1, k2):
    # second-order kernel of Eulerian perturbation theory (Einstein-de Sitter)
    a, b = np.linalg.norm(k1), np.linalg.norm(k2)
    mu = k1 @ k2 / (a * b)
    return 5 / 7 + 0.5 * mu * (a / b + b / a) + 2 / 7 * mu * mu


@pytest.mark.parametrize("n1,n2", [((1, 0, 0), (0, 1, 0)), ((1, 0, 0), (1, 1, 0)), ((2, 1, 0), (0, 1, 1)),
                                   ((1, 0, 0), (0, 0, 2))])
def test_lpt2_density_has_the_second_order_kernel(n1, n2):
    # delta_lin = A cos(k1 q) + B cos(k2 q): the density of the displaced lattice
    # (a direct sum over particles, no mesh) has the cos((k1 + k2) x) amplitude
    # D1^2 F2(k1, k2) A B at second order; Zel'dovich gives a different kernel
    # (1/2 instead of 5/7 for perpendicular modes). The second-order part is the
    # even part in the amplitude, (d(e) + d(-e)) / (2 e^2).
    N = 16
    q = pm.lattice(N)
    k1, k2 = 2 * np.pi / N * np.array(n1, float), 2 * np.pi / N * np.array(n2, float)
    A, B, eps = 1.0, 0.8, 1e-3
    s = pm.rfft3((A * np.cos(k1 @ q) + B * np.cos(k2 @ q)).reshape(N, N, N))
    setup = pm.PMSetup(N=N, L=100.0, nsteps=1, a0=0.5, lpt_order=2)
    D1 = cosmo.D(setup.a0, setup.om)
    kk = k1 + k2
    d = [np.mean(np.exp(-1j * (kk @ pm.lpt_ics(e * s, setup)[0]))) for e in (eps, -eps)]
    second = (d[0] + d[1]).real / 2 / eps ** 2
    assert second / (D1 ** 2 * A * B / 2) == pytest.approx(_f2_kernel(k1, k2), rel=1e-5)
