"""The light-matter network of Sec. 2 (FP64, numpy), forward and adjoint.

Sec. 2.1: a fully connected network y = phi(W x + b) per layer (Eq. 1), two
hidden layers of 50 and 30 ReLU units (Eq. relu). Sec. 2.2: its input at a
grid point is the value of three density fields at the 27 points of the
3x3x3 cube around it (3 x 27 = 81 inputs).

Output head: the synthetic workload uses one network with a softplus output
scaled by M_scale (a positive halo-mass field), M = M_scale ln(1 + e^y).

Input ordering (any fixed order is equivalent; this one is shared by the
weights and both implementations): index = c*27 + (ox+1)*9 + (oy+1)*3 + (oz+1)
for field c and neighbour offset (ox, oy, oz) in {-1,0,1}^3, periodic.
Weights: flat vector W1[50][81], b1[50], W2[30][50], b2[30], w3[30], b3.
"""
from __future__ import annotations

import numpy as np
from scipy.special import expit

N_IN, N_H1, N_H2 = 81, 50, 30
STENCIL = [(ox, oy, oz) for ox in (-1, 0, 1) for oy in (-1, 0, 1) for oz in (-1, 0, 1)]


def unpack(w: np.ndarray):
    w = np.asarray(w, np.float64)
    o = 0
    W1 = w[o:o + N_H1 * N_IN].reshape(N_H1, N_IN); o += N_H1 * N_IN
    b1 = w[o:o + N_H1]; o += N_H1
    W2 = w[o:o + N_H2 * N_H1].reshape(N_H2, N_H1); o += N_H2 * N_H1
    b2 = w[o:o + N_H2]; o += N_H2
    w3 = w[o:o + N_H2]; o += N_H2
    b3 = w[o]; o += 1
    assert o == w.size
    return W1, b1, W2, b2, w3, b3


def relu(x):
    return np.maximum(x, 0.0)


def softplus(y):
    return np.logaddexp(0.0, y)


def stencil_gather(fields: np.ndarray) -> np.ndarray:
    """[3][N][N][N] -> [81][N^3]: v[c,o](x) = f_c(x + o), periodic."""
    rows = []
    for c in range(3):
        for (ox, oy, oz) in STENCIL:
            rows.append(np.roll(fields[c], (-ox, -oy, -oz), axis=(0, 1, 2)).ravel())
    return np.stack(rows)


def stencil_gather_T(gv: np.ndarray, N: int) -> np.ndarray:
    """Transpose of stencil_gather: g_c(y) = sum_o gv[c,o](y - o)."""
    out = np.zeros((3, N, N, N))
    r = 0
    for c in range(3):
        for (ox, oy, oz) in STENCIL:
            out[c] += np.roll(gv[r].reshape(N, N, N), (ox, oy, oz), axis=(0, 1, 2))
            r += 1
    return out


def stencil_at(fields: np.ndarray, vox: np.ndarray) -> np.ndarray:
    """The 81 inputs of the listed voxels only: [81][n], vox = int [n][3] (x, y, z).
    Same order and periodic wrap as stencil_gather, for meshes too large to gather whole."""
    N = fields.shape[1]
    rows = []
    for c in range(3):
        for (ox, oy, oz) in STENCIL:
            rows.append(fields[c][(vox[:, 0] + ox) % N, (vox[:, 1] + oy) % N, (vox[:, 2] + oz) % N])
    return np.stack(rows)


def mlp_at(fields: np.ndarray, vox: np.ndarray, weights: np.ndarray, M_scale: float) -> np.ndarray:
    """The softplus network of Sec. 2 evaluated at the listed voxels: M [n]."""
    W1, b1, W2, b2, w3, b3 = unpack(weights)
    v = stencil_at(fields, vox)
    z2 = relu(W2 @ relu(W1 @ v + b1[:, None]) + b2[:, None])
    return M_scale * softplus(w3 @ z2 + b3)


def mlp_backward_at(gM: np.ndarray, vox: np.ndarray, fields: np.ndarray, weights: np.ndarray,
                    M_scale: float) -> np.ndarray:
    """Gradient of sum_j gM[j] M(vox_j) w.r.t. the three input fields [3][N][N][N]:
    the network adjoint for a mass gradient that is zero off the listed voxels."""
    N = fields.shape[1]
    W1, b1, W2, b2, w3, b3 = unpack(weights)
    v = stencil_at(fields, vox)
    a1 = W1 @ v + b1[:, None]
    a2 = W2 @ relu(a1) + b2[:, None]
    y = w3 @ relu(a2) + b3
    gy = np.asarray(gM, np.float64) * M_scale * expit(y)
    ga2 = np.outer(w3, gy) * (a2 > 0)
    ga1 = (W2.T @ ga2) * (a1 > 0)
    gv = W1.T @ ga1
    out = np.zeros((3, N, N, N))
    r = 0
    for c in range(3):
        for (ox, oy, oz) in STENCIL:
            np.add.at(out[c], ((vox[:, 0] + ox) % N, (vox[:, 1] + oy) % N, (vox[:, 2] + oz) % N), gv[r])
            r += 1
    return out


def mlp_forward(fields: np.ndarray, weights: np.ndarray, M_scale: float):
    """Per-voxel network; returns (M [N][N][N], cache for the adjoint)."""
    N = fields.shape[1]
    W1, b1, W2, b2, w3, b3 = unpack(weights)
    v = stencil_gather(fields)
    a1 = W1 @ v + b1[:, None]
    z1 = relu(a1)
    a2 = W2 @ z1 + b2[:, None]
    z2 = relu(a2)
    y = w3 @ z2 + b3
    M = M_scale * softplus(y)
    return M.reshape(N, N, N), (a1, a2, y)


# ----------------------------------------------------------------------------- the paper's two-network head
#
# Sec. 2: model = NNp x NNm. NNp is the 81-50-30-1 ReLU trunk above with a
# logistic output of sharpness a (Eq. logistic); NNm is a 3-20-10-1 network
# with ELU hidden units (Eq. elu) and a linear output, fed with the three
# fields at the voxel itself (Sec. 2.2). M = M_scale * logistic(y_p, a) * m.
# Mass-net weights (flat, after the 5661 of NNp): Wm1[20][3], bm1[20],
# Wm2[10][20], bm2[10], wm3[10], bm3.

NM_IN, NM_H1, NM_H2 = 3, 20, 10
N_MASS_WEIGHTS = NM_H1 * NM_IN + NM_H1 + NM_H2 * NM_H1 + NM_H2 + NM_H2 + 1


def unpack_mass(w: np.ndarray):
    w = np.asarray(w, np.float64)
    o = 0
    W1 = w[o:o + NM_H1 * NM_IN].reshape(NM_H1, NM_IN); o += NM_H1 * NM_IN
    b1 = w[o:o + NM_H1]; o += NM_H1
    W2 = w[o:o + NM_H2 * NM_H1].reshape(NM_H2, NM_H1); o += NM_H2 * NM_H1
    b2 = w[o:o + NM_H2]; o += NM_H2
    w3 = w[o:o + NM_H2]; o += NM_H2
    b3 = w[o]; o += 1
    assert o == w.size
    return W1, b1, W2, b2, w3, b3


def elu(x):
    return np.where(x > 0, x, np.expm1(np.minimum(x, 0.0)))


def elu_grad(x):
    return np.where(x > 0, 1.0, np.exp(np.minimum(x, 0.0)))


def logistic(x, a):
    return expit(a * x)


def _trunk_logit(fields, wp):
    W1, b1, W2, b2, w3, b3 = unpack(wp)
    v = stencil_gather(fields)
    a1 = W1 @ v + b1[:, None]
    a2 = W2 @ relu(a1) + b2[:, None]
    return w3 @ relu(a2) + b3, (a1, a2)


def _mass_net(fields, wm):
    W1, b1, W2, b2, w3, b3 = unpack_mass(wm)
    u = fields.reshape(3, -1)
    h1 = W1 @ u + b1[:, None]
    h2 = W2 @ elu(h1) + b2[:, None]
    return w3 @ elu(h2) + b3, (u, h1, h2)


def two_net_forward(fields, wp, wm, M_scale, a):
    """M = M_scale * logistic(y_p, a) * NNm(fields at the voxel)."""
    N = fields.shape[1]
    y, _ = _trunk_logit(fields, wp)
    m, _ = _mass_net(fields, wm)
    return (M_scale * logistic(y, a) * m).reshape(N, N, N)


def two_net_backward(gM, fields, wp, wm, M_scale, a):
    N = fields.shape[1]
    W1, b1, W2, b2, w3, b3 = unpack(wp)
    y, (a1, a2) = _trunk_logit(fields, wp)
    m, (u, h1, h2) = _mass_net(fields, wm)
    p = logistic(y, a)
    g = gM.ravel() * M_scale
    # position net
    gy = g * m * a * p * (1.0 - p)
    ga2 = np.outer(w3, gy) * (a2 > 0)
    ga1 = (W2.T @ ga2) * (a1 > 0)
    out = stencil_gather_T(W1.T @ ga1, N)
    # mass net, on the voxel's own three values
    V1, c1, V2, c2, v3, c3 = unpack_mass(wm)
    gm = g * p
    gh2 = np.outer(v3, gm) * elu_grad(h2)
    gh1 = (V2.T @ gh2) * elu_grad(h1)
    out += (V1.T @ gh1).reshape(3, N, N, N)
    return out


def mlp_backward(gM: np.ndarray, fields: np.ndarray, weights: np.ndarray, M_scale: float) -> np.ndarray:
    """Gradient of <gM, M(fields)> w.r.t. the three input fields."""
    N = fields.shape[1]
    W1, b1, W2, b2, w3, b3 = unpack(weights)
    _, (a1, a2, y) = mlp_forward(fields, weights, M_scale)
    gy = gM.ravel() * M_scale * expit(y)
    ga2 = np.outer(w3, gy) * (a2 > 0)
    ga1 = (W2.T @ ga2) * (a1 > 0)
    gv = W1.T @ ga1
    return stencil_gather_T(gv, N)
