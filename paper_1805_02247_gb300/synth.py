"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module draws random numbers and nothing else: it holds none of the
reconstruction's arithmetic (no power spectrum, no FFT, no forward model).
Every stochastic quantity the method needs is drawn here once, on the host,
with numpy's PCG64, and handed to both implementations as plain arrays, so
parity never depends on two random-number generators agreeing.

Workload shapes follow the paper's setting (Sec. 3 and Sec. 5.3): a periodic
cube of side L Mpc/h, an N^3 mesh with one particle per cell, a linear field
drawn from Gaussian white noise, Xavier-initialised weights for the
81-50-30-1 network of Sec. 2.1, and per-voxel log-normal scatter for the data.
"""
from __future__ import annotations

import numpy as np

# Network shape of Sec. 2.1: 3 fields x 27 neighbours -> 50 -> 30 -> 1.
N_IN, N_H1, N_H2 = 81, 50, 30
# Flat parameter vector layout: W1[50][81], b1[50], W2[30][50], b2[30], w3[30], b3[1].
N_WEIGHTS = N_H1 * N_IN + N_H1 + N_H2 * N_H1 + N_H2 + N_H2 + 1


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def white_noise(n: int, seed: int) -> np.ndarray:
    """Real N(0,1) white noise on an n^3 mesh, float32, C order [x][y][z].

    The linear field is this noise coloured by the linear power spectrum; the
    colouring is the method's arithmetic and lives in each implementation.
    """
    return rng(seed).standard_normal((n, n, n)).astype(np.float32)


def scatter_noise(n: int, seed: int) -> np.ndarray:
    """Per-voxel N(0,1) draws for the log-normal data scatter, float32.

    Drawn from the same seed's stream after the white noise of that seed, so a
    data realisation is fully fixed by one seed.
    """
    g = rng(seed)
    g.standard_normal((n, n, n))  # the white noise of this seed comes first
    return g.standard_normal((n, n, n)).astype(np.float32)


def xavier_weights(seed: int) -> np.ndarray:
    """Glorot-uniform weights U(+-sqrt(6/(fan_in+fan_out))), zero biases.

    Returns the flat float32 vector in the layout documented above.
    """
    g = rng(seed)
    out = []
    for fan_in, fan_out in ((N_IN, N_H1), (N_H1, N_H2), (N_H2, 1)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        out.append(g.uniform(-lim, lim, size=(fan_out, fan_in)).ravel())
        out.append(np.zeros(fan_out))
    w = np.concatenate(out).astype(np.float32)
    assert w.size == N_WEIGHTS
    return w


N_MASS_WEIGHTS = 20 * 3 + 20 + 10 * 20 + 10 + 10 + 1


def mass_net_weights(seed: int, out_bias: float = 5.0, scale: float = 0.25) -> np.ndarray:
    """Glorot-uniform weights of the 3-20-10-1 mass network times `scale`, zero hidden biases.

    Layout: Wm1[20][3], bm1[20], Wm2[10][20], bm2[10], wm3[10], bm3. An untrained
    linear output has no sign; the output bias (default 5) and the shrunken
    weights keep the synthetic mass positive, as a trained mass network is.
    """
    g = rng(seed)
    out = []
    for fan_in, fan_out in ((3, 20), (20, 10), (10, 1)):
        lim = scale * np.sqrt(6.0 / (fan_in + fan_out))
        out.append(g.uniform(-lim, lim, size=(fan_out, fan_in)).ravel())
        out.append(np.zeros(fan_out))
    w = np.concatenate(out)
    w[-1] = out_bias
    assert w.size == N_MASS_WEIGHTS
    return w.astype(np.float32)


def two_net_weights(seed: int) -> np.ndarray:
    """Weights of the two-network head: the trunk's 5661 then the mass network's 301."""
    return np.concatenate([xavier_weights(seed), mass_net_weights(seed)]).astype(np.float32)


def uniform_positions(n: int, npart: int, seed: int, lo: float = 0.0, hi: float | None = None) -> np.ndarray:
    """Particle positions in grid units, float32 SoA [3][npart], uniform in [lo, hi)."""
    hi = float(n) if hi is None else hi
    return rng(seed).uniform(lo, hi, size=(3, npart)).astype(np.float32)


def clustered_positions(n: int, npart: int, seed: int, ncentres: int = 20000, frac: float = 0.5,
                        sigma: float = 0.4) -> np.ndarray:
    """Particle positions in grid units, float32 SoA [3][npart], the crowded
    cells of an evolved field: a fraction `frac` of the particles in Gaussian
    clumps (width `sigma` cells) around uniform centres with log-normally
    distributed occupations, the rest uniform in [0, n)."""
    g = rng(seed)
    nc = int(frac * npart)
    w = g.lognormal(0.0, 1.5, size=ncentres)
    occ = np.floor(w / w.sum() * nc).astype(np.int64)
    occ[: nc - occ.sum()] += 1
    centres = g.uniform(0.0, n, size=(3, ncentres))
    clumps = np.repeat(centres, occ, axis=1) + g.normal(0.0, sigma, size=(3, int(occ.sum())))
    rest = g.uniform(0.0, n, size=(3, npart - clumps.shape[1]))
    x = np.concatenate([clumps, rest], axis=1)
    return x[:, g.permutation(npart)].astype(np.float32)


def edge_positions(n: int) -> np.ndarray:
    """Hand-picked positions that stress the wrap and floor rules, float32 [3][k].

    Includes exact integers, values just below n and 0, negative values, values
    at and beyond n, and values that round to n in float32 after wrapping.
    """
    f = np.float32
    eps = np.nextafter(f(n), f(0))
    vals = np.array([0.0, 1.0, 0.5, n - 1, eps, n, n + 0.25, -0.25, -1e-8, -1e-30,
                     -n, 2 * n + 0.5, np.nextafter(f(0), f(1)), 1.0 - 1e-7, n - 0.5, 3.999999],
                    dtype=np.float32)
    k = vals.size
    return np.stack([vals, np.roll(vals, 3), np.roll(vals, 7)]).astype(np.float32).reshape(3, k)


def lognormal_density(n: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """A float32 overdensity mesh with the one-sided, heavy-tailed values of an
    evolved density: delta = exp(sigma g - sigma^2/2) - 1, g a unit Gaussian
    field given short-range correlation by averaging each cell with its six
    neighbours (periodic) and rescaling to unit variance."""
    g = rng(seed).standard_normal((n, n, n))
    c = g.copy()
    for ax in range(3):
        c += np.roll(g, 1, axis=ax) + np.roll(g, -1, axis=ax)
    c /= c.std()
    return (np.exp(sigma * c - 0.5 * sigma * sigma) - 1.0).astype(np.float32)


def sample_voxels(n: int, count: int, seed: int) -> np.ndarray:
    """int [count][3] voxel indices: random ones plus every corner of the box, so
    periodic neighbours across each face are among them."""
    r = rng(seed).integers(0, n, size=(count, 3))
    corners = np.array([[x, y, z] for x in (0, n - 1) for y in (0, n - 1) for z in (0, n - 1)])
    return np.concatenate([corners, r]).astype(np.int64)


def gaussian_vector(shape, seed: int) -> np.ndarray:
    """N(0,1) float32 array of any shape (adjoint seeds, L-BFGS test vectors)."""
    return rng(seed).standard_normal(shape).astype(np.float32)
