"""Particle-mesh forward model and its hand-written adjoint (FP64, numpy).

Follows Sec. 3 (FastPM forward model: LPT initial conditions at a = 0.1, a few
PM steps) and Sec. 5.2 (gradients of the PM evolution, written here by hand).
Where the paper is silent the readings below are used; each is a stated
convention, identical on the CUDA side.

Conventions
-----------
* Mesh: N^3 cells, C order [x][y][z]; lengths in grid units (cell = L/N Mpc/h).
* Fourier: s(k) is the numpy ``rfftn`` half array [N][N][N/2+1]; the real field
  is ``irfftn(s)`` (1/N^3 on the inverse). Grid-unit wavenumber k = 2 pi n / N,
  n in (-N/2, N/2]. The linear field has <|s_k|^2> = P(k) N^6 / L^3.
* The half-array entries (real and imaginary parts) are the independent real
  variables of the problem (Sec. 5.1 treats real and imaginary parts as
  independent modes). Gradients are w.r.t. those entries; the prior weights a
  mode by w_k = 2 for 0 < k_z < N/2 and 1 on the k_z = 0 and k_z = N/2 planes
  so that it equals the full-grid sum for a Hermitian field.
* Particles: one per cell, index i = (ix N + iy) N + iz, Lagrangian position q
  at the integer grid point; SoA arrays [3][Np].
* Odd Fourier multipliers (gradients) are set to zero where that component of n
  is the Nyquist frequency N/2, and every multiplier is zero at k = 0.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import cosmo

OFFSETS = [(ox, oy, oz) for ox in (0, 1) for oy in (0, 1) for oz in (0, 1)]


@dataclass(frozen=True)
class PMSetup:
    N: int
    L: float
    nsteps: int
    a0: float = 0.1
    om: float = cosmo.OMEGA_M
    sigma8: float = cosmo.SIGMA8
    gamma: float = cosmo.GAMMA_BBKS
    lpt_order: int = 1  # 1: Zel'dovich initial conditions; 2: second-order LPT (Sec. 3)


# ----------------------------------------------------------------------------- Fourier mesh

def wavenumbers(N: int):
    """Grid-unit wavenumber components broadcastable to the half array, plus Nyquist masks."""
    n_full = np.fft.fftfreq(N, d=1.0 / N)
    n_half = np.arange(N // 2 + 1, dtype=np.float64)
    kx = (2 * np.pi / N * n_full)[:, None, None]
    ky = (2 * np.pi / N * n_full)[None, :, None]
    kz = (2 * np.pi / N * n_half)[None, None, :]
    nyq = [np.abs(n_full)[:, None, None] == N // 2,
           np.abs(n_full)[None, :, None] == N // 2,
           (n_half == N // 2)[None, None, :]]
    return (kx, ky, kz), nyq


def k_squared(N: int) -> np.ndarray:
    (kx, ky, kz), _ = wavenumbers(N)
    return kx**2 + ky**2 + kz**2


def half_weights(N: int) -> np.ndarray:
    w = np.full(N // 2 + 1, 2.0)
    w[0] = 1.0
    w[N // 2] = 1.0
    return np.broadcast_to(w[None, None, :], (N, N, N // 2 + 1))


def rfft3(f: np.ndarray) -> np.ndarray:
    return np.fft.rfftn(f)


def irfft3(s: np.ndarray) -> np.ndarray:
    N = s.shape[0]
    return np.fft.irfftn(s, s=(N, N, N), axes=(0, 1, 2))


def irfft3_T(lam: np.ndarray) -> np.ndarray:
    """Transpose of irfft3 w.r.t. the real inner products on both sides.

    irfft3 uses each interior half-array entry twice (it and its conjugate
    partner) and each k_z in {0, N/2} entry once, so the transpose is
    (w_k / N^3) rfftn(lam).
    """
    N = lam.shape[0]
    return half_weights(N) / N**3 * np.fft.rfftn(lam)


def odd_multiplier(N: int, j: int, scale: float = 1.0) -> np.ndarray:
    """scale * i k_j / k^2, zero at k = 0 and on the Nyquist plane of component j."""
    ks, nyq = wavenumbers(N)
    k2 = k_squared(N)
    with np.errstate(divide="ignore", invalid="ignore"):
        m = 1j * scale * ks[j] / k2
    m = np.where(k2 == 0, 0, m)
    return np.where(nyq[j], 0, m)


def gaussian_multiplier(N: int, R_cells: float) -> np.ndarray:
    """exp(-k^2 R^2 / 2) with R in grid units (a unit-integral Gaussian of width R)."""
    return np.exp(-0.5 * k_squared(N) * R_cells**2)


def smooth(field: np.ndarray, R_cells: float) -> np.ndarray:
    """Gaussian smoothing; R = 0 is the identity. Self-adjoint (real even kernel)."""
    if R_cells == 0:
        return field.copy()
    return irfft3(gaussian_multiplier(field.shape[0], R_cells) * rfft3(field))


# ----------------------------------------------------------------------------- linear field

def power_half(setup: PMSetup) -> np.ndarray:
    """Expected |s_k|^2 = P(k) N^6 / L^3 on the half array (k = 0 entry set to 0)."""
    N, L = setup.N, setup.L
    kphys = np.sqrt(k_squared(N)) * N / L
    P = cosmo.P_lin_array(kphys, setup.sigma8, setup.gamma) * N**6 / L**3
    P[0, 0, 0] = 0.0
    return P


def linear_field(white: np.ndarray, setup: PMSetup, amplitude: float = 1.0) -> np.ndarray:
    """s(k) = amplitude * sqrt(P~(k) / N^3) * rfftn(white), s(0) = 0.

    rfftn of unit white noise has <|.|^2> = N^3, so <|s|^2> = amplitude^2 P~.
    """
    N = setup.N
    s = amplitude * np.sqrt(power_half(setup) / N**3) * rfft3(np.asarray(white, np.float64))
    s[0, 0, 0] = 0
    return s


# ----------------------------------------------------------------------------- initial conditions

def lattice(N: int) -> np.ndarray:
    return np.indices((N, N, N), dtype=np.float64).reshape(3, -1)


def za_displacement(s: np.ndarray) -> np.ndarray:
    """psi_k = i k s_k / k^2 (so that -div psi = delta), returned as [3][N^3] at a = 1."""
    N = s.shape[0]
    return np.stack([irfft3(odd_multiplier(N, j) * s).ravel() for j in range(3)])


def za_ics(s: np.ndarray, setup: PMSetup):
    """Zel'dovich ICs at a0: x = q + D(a0) psi, p = G_p(a0) psi."""
    psi = za_displacement(s)
    x = lattice(setup.N) + cosmo.D(setup.a0, setup.om) * psi
    p = cosmo.Gp(setup.a0, setup.om) * psi
    return x, p


def hessian_multiplier(N: int, i: int, j: int) -> np.ndarray:
    """k_i k_j / k^2: takes delta_k to the Fourier modes of d_i d_j phi with
    lap phi = delta (phi_k = -delta_k / k^2). Zero at k = 0; for i != j also
    zero where component i or j is the Nyquist frequency (an odd factor there)."""
    ks, nyq = wavenumbers(N)
    k2 = k_squared(N)
    with np.errstate(divide="ignore", invalid="ignore"):
        m = ks[i] * ks[j] / k2
    m = np.where(k2 == 0, 0.0, m)
    if i != j:
        m = np.where(nyq[i] | nyq[j], 0.0, m)
    return m


HESS_PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def lpt2_hessian(s: np.ndarray) -> np.ndarray:
    """[6][N][N][N]: phi_xx, phi_yy, phi_zz, phi_xy, phi_xz, phi_yz of the
    first-order potential (lap phi = delta, the linear field at a = 1)."""
    N = s.shape[0]
    return np.stack([irfft3(hessian_multiplier(N, i, j) * s) for (i, j) in HESS_PAIRS])


def lpt2_source(H: np.ndarray) -> np.ndarray:
    """Second-order source sum_{i<j} (phi_ii phi_jj - phi_ij^2) (textbook 2LPT)."""
    xx, yy, zz, xy, xz, yz = H
    return xx * yy + xx * zz + yy * zz - xy**2 - xz**2 - yz**2


def lpt2_displacement(s: np.ndarray) -> np.ndarray:
    """psi2 = grad phi2 with lap phi2 = the second-order source, [3][N^3] at a = 1:
    psi2_k = -i k S_k / k^2 (odd multiplier with factor -1)."""
    N = s.shape[0]
    Sk = rfft3(lpt2_source(lpt2_hessian(s)))
    return np.stack([irfft3(odd_multiplier(N, j, -1.0) * Sk).ravel() for j in range(3)])


def lpt2_growth(setup: PMSetup):
    """(D1, D2, Gp, Gp2) at a0: D2 = -3/7 D1^2 (the usual approximation, exact in
    Einstein-de Sitter) and Gp2 = a^3 E dD2/da = -6/7 D1 Gp."""
    D1 = cosmo.D(setup.a0, setup.om)
    Gp = cosmo.Gp(setup.a0, setup.om)
    return D1, -3.0 / 7.0 * D1 * D1, Gp, -6.0 / 7.0 * D1 * Gp


def lpt_ics(s: np.ndarray, setup: PMSetup):
    """Initial conditions of order setup.lpt_order at a0.
    Order 2: x = q + D1 psi1 + D2 psi2, p = Gp psi1 + Gp2 psi2."""
    if setup.lpt_order == 1:
        return za_ics(s, setup)
    D1, D2, Gp, Gp2 = lpt2_growth(setup)
    psi1 = za_displacement(s)
    psi2 = lpt2_displacement(s)
    return lattice(setup.N) + D1 * psi1 + D2 * psi2, Gp * psi1 + Gp2 * psi2


def lpt_ics_T(lam_x: np.ndarray, lam_p: np.ndarray, s: np.ndarray, setup: PMSetup) -> np.ndarray:
    """Adjoint of lpt_ics at s: gradient w.r.t. the half-array entries of s."""
    g = za_ics_T(lam_x, lam_p, setup)
    if setup.lpt_order == 1:
        return g
    N = setup.N
    D1, D2, Gp, Gp2 = lpt2_growth(setup)
    mu = (D2 * lam_x + Gp2 * lam_p).reshape(3, N, N, N)
    # transpose of S -> psi2_j: irfft(conj(m_j) rfft(.)) summed over j
    acc = np.zeros((N, N, N // 2 + 1), dtype=np.complex128)
    for j in range(3):
        acc += np.conj(odd_multiplier(N, j, -1.0)) * rfft3(mu[j])
    sigma = irfft3(acc)
    xx, yy, zz, xy, xz, yz = lpt2_hessian(s)
    gH = [sigma * (yy + zz), sigma * (xx + zz), sigma * (xx + yy),
          -2.0 * sigma * xy, -2.0 * sigma * xz, -2.0 * sigma * yz]
    for (i, j), gh in zip(HESS_PAIRS, gH):
        g += hessian_multiplier(N, i, j) * irfft3_T(gh)
    return g


def za_ics_T(lam_x: np.ndarray, lam_p: np.ndarray, setup: PMSetup) -> np.ndarray:
    """Adjoint of za_ics: gradient w.r.t. the half-array entries of s."""
    N = setup.N
    lam_psi = cosmo.D(setup.a0, setup.om) * lam_x + cosmo.Gp(setup.a0, setup.om) * lam_p
    g = np.zeros((N, N, N // 2 + 1), dtype=np.complex128)
    for j in range(3):
        g += np.conj(odd_multiplier(N, j)) * irfft3_T(lam_psi[j].reshape(N, N, N))
    return g


# ----------------------------------------------------------------------------- cell indexing

def wrap_f32(u, N: int) -> np.ndarray:
    """The indexing rule, evaluated in float32 exactly as the kernels do.

    w = fmod(u, N) (exact); if w < 0 then w = w + N (float32 rounding);
    if w >= N then w = 0.
    """
    u = np.asarray(u, dtype=np.float32)
    n = np.float32(N)
    w = np.fmod(u, n)
    w = np.where(w < 0, (w + n).astype(np.float32), w)
    w = np.where(w >= n, np.float32(0), w)
    return w.astype(np.float32)


def cell_keys(x32: np.ndarray, N: int) -> np.ndarray:
    """key = (floor(wx) N + floor(wy)) N + floor(wz) of the wrapped float32 position."""
    w = wrap_f32(x32, N)
    i = np.floor(w).astype(np.int64)
    return ((i[0] * N + i[1]) * N + i[2]).astype(np.uint32)


def sort_by_cell(keys: np.ndarray, N: int):
    """Stable counting sort: perm orders particles by (key, original index)."""
    perm = np.argsort(keys, kind="stable").astype(np.uint32)
    counts = np.bincount(keys.astype(np.int64), minlength=N**3)
    cell_start = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)
    return perm, cell_start


# ----------------------------------------------------------------------------- CIC

def _cic_cells(x: np.ndarray, N: int, f32_wrap: bool = False):
    # f32_wrap: the positions are float32 values and the cell index, an integer
    # decision, is taken from their float32 wrap (wrap_f32), as the kernels do
    w = wrap_f32(x, N).astype(np.float64) if f32_wrap else np.mod(np.asarray(x, np.float64), N)
    i = np.floor(w)
    d = w - i
    return i.astype(np.int64) % N, d


def _offset_index_weight(i, d, o, N):
    idx = (((i[0] + o[0]) % N) * N + (i[1] + o[1]) % N) * N + (i[2] + o[2]) % N
    wts = [d[a] if o[a] else 1.0 - d[a] for a in range(3)]
    return idx, wts


def paint(x: np.ndarray, N: int, mass=None, f32_wrap: bool = False) -> np.ndarray:
    """Cloud-in-cell assignment (Sec. 2: fields are CIC-convolved onto the grid)."""
    i, d = _cic_cells(x, N, f32_wrap)
    m = np.ones(x.shape[1]) if mass is None else np.asarray(mass, np.float64)
    rho = np.zeros(N**3)
    for o in OFFSETS:
        idx, w = _offset_index_weight(i, d, o, N)
        rho += np.bincount(idx, weights=m * w[0] * w[1] * w[2], minlength=N**3)
    return rho.reshape(N, N, N)


def readout(field: np.ndarray, x: np.ndarray, f32_wrap: bool = False) -> np.ndarray:
    """CIC interpolation of a mesh field at particle positions (transpose of paint in mass)."""
    N = field.shape[0]
    i, d = _cic_cells(x, N, f32_wrap)
    f = field.ravel()
    out = np.zeros(x.shape[1])
    for o in OFFSETS:
        idx, w = _offset_index_weight(i, d, o, N)
        out += w[0] * w[1] * w[2] * f[idx]
    return out


def readout_grad(field: np.ndarray, x: np.ndarray, f32_wrap: bool = False) -> np.ndarray:
    """d/dx_a of readout(field, x): derivative of the CIC weights, [3][Np]."""
    N = field.shape[0]
    i, d = _cic_cells(x, N, f32_wrap)
    f = field.ravel()
    out = np.zeros((3, x.shape[1]))
    for o in OFFSETS:
        idx, w = _offset_index_weight(i, d, o, N)
        for a in range(3):
            dw = [w[b] if b != a else (1.0 if o[a] else -1.0) for b in range(3)]
            out[a] += dw[0] * dw[1] * dw[2] * f[idx]
    return out


def density(x: np.ndarray, N: int) -> np.ndarray:
    """Overdensity delta = rho / rho_bar - 1 of unit-mass particles."""
    rho_bar = x.shape[1] / N**3
    return paint(x, N) / rho_bar - 1.0


# ----------------------------------------------------------------------------- force

def force(delta: np.ndarray, om: float) -> np.ndarray:
    """F = -grad phi with lap phi = 1.5 Om delta: F_k = 1.5 Om i k delta_k / k^2, [3][N][N][N]."""
    N = delta.shape[0]
    dk = rfft3(delta)
    return np.stack([irfft3(odd_multiplier(N, j, 1.5 * om) * dk) for j in range(3)])


def force_T(G: np.ndarray, om: float) -> np.ndarray:
    """Transpose of force(): sum_j irfft(conj(m_j) rfft(G_j)) (odd kernels: A^T = -A)."""
    N = G.shape[1]
    acc = np.zeros((N, N, N // 2 + 1), dtype=np.complex128)
    for j in range(3):
        acc += np.conj(odd_multiplier(N, j, 1.5 * om)) * rfft3(G[j])
    return irfft3(acc)


# ----------------------------------------------------------------------------- time stepping

def scale_factors(setup: PMSetup) -> np.ndarray:
    """Steps uniform in a from a0 to 1."""
    return np.linspace(setup.a0, 1.0, setup.nsteps + 1)


def kdk_factors(setup: PMSetup):
    """Kick and drift coefficients that make Zel'dovich trajectories exact.

    Step i: kick p from a_{i-1/2} (a_0 for i = 0) to a_{i+1/2} with the force
    at a_i, k_i = [G_p(a_{i+1/2}) - G_p(a_{i-1/2})] / G_f(a_i); then drift x
    from a_i to a_{i+1}, d_i = [D(a_{i+1}) - D(a_i)] / G_p(a_{i+1/2}).
    """
    a = scale_factors(setup)
    om = setup.om
    kick, drift = [], []
    for i in range(setup.nsteps):
        ah = 0.5 * (a[i] + a[i + 1])
        ah_prev = a[0] if i == 0 else 0.5 * (a[i - 1] + a[i])
        kick.append((cosmo.Gp(ah, om) - cosmo.Gp(ah_prev, om)) / cosmo.Gf(a[i], om))
        drift.append((cosmo.D(a[i + 1], om) - cosmo.D(a[i], om)) / cosmo.Gp(ah, om))
    return np.array(kick), np.array(drift)


def pm_forward(s: np.ndarray, setup: PMSetup):
    """s(k) -> final positions. Returns (x_final, [x_i before step i], p_final)."""
    N = setup.N
    x, p = lpt_ics(s, setup)
    kick, drift = kdk_factors(setup)
    checkpoints = []
    for i in range(setup.nsteps):
        checkpoints.append(x.copy())
        F = force(density(x, N), setup.om)
        p = p + kick[i] * np.stack([readout(F[j], x) for j in range(3)])
        x = x + drift[i] * p
    return x, checkpoints, p


def pm_adjoint(checkpoints, lam_x: np.ndarray, lam_p: np.ndarray, setup: PMSetup, s=None) -> np.ndarray:
    """Reverse mode of pm_forward: gradients at (x_final, p_final) -> gradient w.r.t. s.

    Each step's force field is recomputed from the stored positions.
    """
    N, om = setup.N, setup.om
    kick, drift = kdk_factors(setup)
    rho_bar = checkpoints[0].shape[1] / N**3
    lam_x = lam_x.copy()
    lam_p = lam_p.copy()
    for i in reversed(range(setup.nsteps)):
        x = checkpoints[i]
        lam_p = lam_p + drift[i] * lam_x
        F = force(density(x, N), om)
        # kick, direct term: the readout weights move with the particle
        for j in range(3):
            lam_x += kick[i] * lam_p[j] * readout_grad(F[j], x)
        # kick, through the mesh: readout^T = paint, force^T, paint^T = readout_grad
        G = np.stack([kick[i] * paint(x, N, mass=lam_p[j]) for j in range(3)])
        g_delta = force_T(G, om)
        lam_x += readout_grad(g_delta / rho_bar, x)
    return lpt_ics_T(lam_x, lam_p, s, setup)


def final_density(s: np.ndarray, setup: PMSetup) -> np.ndarray:
    x, _, _ = pm_forward(s, setup)
    return density(x, setup.N)


def final_density_T(checkpoints, x_final: np.ndarray, g_delta: np.ndarray, setup: PMSetup, s=None) -> np.ndarray:
    """Gradient w.r.t. s of <g_delta, delta_final(s)>."""
    N = setup.N
    rho_bar = x_final.shape[1] / N**3
    lam_x = readout_grad(g_delta / rho_bar, x_final)
    return pm_adjoint(checkpoints, lam_x, np.zeros_like(lam_x), setup, s)
