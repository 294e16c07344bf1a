"""The reconstruction loss of Sec. 5.1 and its gradient w.r.t. s(k) (FP64).

Eq. (loss): L(s) = 1/2 s S^-1 s^dagger
                 + f_eff sum_i ((mu_N + log(M^NN_R,i + M0) - log(M^data_R,i + M0)) / (2 sigma_N))^2

Readings (the paper is silent or ambiguous on these):
* log is the natural logarithm.
* The residual square is taken literally as printed, r^2 / (4 sigma_N^2);
  Sec. 5.3 fixes sigma_N^2 = 0.25, f_eff = 1 (Sec. 5.1).
* M_R is the model (or data) mass field smoothed with a Gaussian of R_M =
  3 Mpc/h (Sec. 4.2 smooths both fields at 3 Mpc/h before comparing).
* The annealed residual smoothing of Sec. 5.2 is a Gaussian of R_sm applied to
  the residual field before squaring; R_sm = 0 means none.
* mu_N defaults to 0 (the mass-dependent offsets of Fig. noise are not printed).
* The three network input fields are the final overdensity smoothed with
  Gaussians of R_feat = (1, 2, 4) Mpc/h (Sec. 2.2 uses multi-scale smoothed
  density; the scales are those of the synthetic workload), optionally mixed
  by a 3x3 matrix C, f_i = sum_j C_ij delta_Rj: the paper's own set delta_0,
  delta_R1, delta_R1 - delta_R2 is R_feat = (0, R1, R2) with C rows (1, 0, 0),
  (0, 1, 0), (0, 1, -1).
* The prior is 1/2 sum over the half array of w_k |s_k|^2 / P~(k), k != 0 (pm.py).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import nn, pm


@dataclass(frozen=True)
class LossSetup:
    R_feat: tuple = (1.0, 2.0, 4.0)  # Mpc/h; 0 = unsmoothed
    feat_mix: tuple | None = None  # row-major 3x3 C, f_i = sum_j C_ij delta_Rj; None = identity
    R_M: float = 3.0  # Mpc/h
    sigma_N2: float = 0.25
    mu_N: float = 0.0
    f_eff: float = 1.0
    M_scale: float = 1e12  # M_sun/h per unit network output
    head: str = "softplus"  # or "two_net": logistic(NNp, a) x NNm (Sec. 2.1)


@dataclass(frozen=True)
class Anneal:
    R_sm: float  # Mpc/h
    M0: float  # M_sun/h
    a: float = 3.0  # logistic sharpness of the two-network head (annealed 1, 2, 3 in Sec. 5.2)


def _head_forward(f, weights, ls: LossSetup, a: float):
    if ls.head == "two_net":
        w = np.asarray(weights)
        return nn.two_net_forward(f, w[:nn.N_H1 * nn.N_IN + nn.N_H1 + nn.N_H2 * nn.N_H1 + 2 * nn.N_H2 + 1],
                                  w[-nn.N_MASS_WEIGHTS:], ls.M_scale, a)
    return nn.mlp_forward(f, weights, ls.M_scale)[0]


def _head_backward(gM, f, weights, ls: LossSetup, a: float):
    if ls.head == "two_net":
        w = np.asarray(weights)
        return nn.two_net_backward(gM, f, w[:nn.N_H1 * nn.N_IN + nn.N_H1 + nn.N_H2 * nn.N_H1 + 2 * nn.N_H2 + 1],
                                   w[-nn.N_MASS_WEIGHTS:], ls.M_scale, a)
    return nn.mlp_backward(gM, f, weights, ls.M_scale)


def features(delta: np.ndarray, pms: pm.PMSetup, ls: LossSetup) -> np.ndarray:
    cell = pms.L / pms.N
    smoothed = np.stack([pm.smooth(delta, R / cell) for R in ls.R_feat])
    if ls.feat_mix is None:
        return smoothed
    C = np.asarray(ls.feat_mix, np.float64).reshape(3, 3)
    return np.einsum("ij,jxyz->ixyz", C, smoothed)


def features_T(g_fields: np.ndarray, pms: pm.PMSetup, ls: LossSetup) -> np.ndarray:
    cell = pms.L / pms.N
    if ls.feat_mix is not None:
        C = np.asarray(ls.feat_mix, np.float64).reshape(3, 3)
        g_fields = np.einsum("ij,ixyz->jxyz", C, g_fields)  # transpose of the mix
    return sum(pm.smooth(g_fields[c], R / cell) for c, R in enumerate(ls.R_feat))


def nn_halo_map(delta: np.ndarray, weights: np.ndarray, pms: pm.PMSetup, ls: LossSetup, a: float = 3.0) -> np.ndarray:
    """Final overdensity -> network halo-mass field M_NN."""
    return _head_forward(features(delta, pms, ls), weights, ls, a)


def nn_halo_map_T(g_M: np.ndarray, delta: np.ndarray, weights: np.ndarray, pms: pm.PMSetup, ls: LossSetup,
                  a: float = 3.0) -> np.ndarray:
    f = features(delta, pms, ls)
    return features_T(_head_backward(g_M, f, weights, ls, a), pms, ls)


def prior(s: np.ndarray, P: np.ndarray) -> float:
    N = s.shape[0]
    w = pm.half_weights(N)
    mask = P > 0
    return 0.5 * float(np.sum((w * np.abs(s) ** 2)[mask] / P[mask]))


def prior_inverse_hessian(pms: pm.PMSetup) -> np.ndarray:
    """Diagonal of the prior's inverse Hessian over the half-array entries,
    P~(k) / w_k (0 at k = 0): the initial L-BFGS inverse Hessian (lbfgs.py)."""
    P = pm.power_half(pms)
    return P / pm.half_weights(pms.N)


def prior_grad(s: np.ndarray, P: np.ndarray) -> np.ndarray:
    N = s.shape[0]
    w = pm.half_weights(N)
    g = np.zeros_like(s)
    mask = P > 0
    g[mask] = (w * s)[mask] / P[mask]
    return g


def residual_terms(M_nn: np.ndarray, data_M: np.ndarray, pms: pm.PMSetup, ls: LossSetup, an: Anneal):
    """Residual part of Eq. (loss) from the model mass field; returns (L_res, cache)."""
    cell = pms.L / pms.N
    M_R = pm.smooth(M_nn, ls.R_M / cell)
    D_R = pm.smooth(np.asarray(data_M, np.float64), ls.R_M / cell)
    r = ls.mu_N + np.log(M_R + an.M0) - np.log(D_R + an.M0)
    r_s = pm.smooth(r, an.R_sm / cell)
    L_res = ls.f_eff * float(np.sum(r_s**2)) / (4.0 * ls.sigma_N2)
    return L_res, (M_R, r_s)


def residual_grad(cache, pms: pm.PMSetup, ls: LossSetup, an: Anneal) -> np.ndarray:
    """Gradient of the residual term w.r.t. M_NN."""
    cell = pms.L / pms.N
    M_R, r_s = cache
    g_rs = ls.f_eff * 2.0 * r_s / (4.0 * ls.sigma_N2)
    g_r = pm.smooth(g_rs, an.R_sm / cell)
    g_MR = g_r / (M_R + an.M0)
    return pm.smooth(g_MR, ls.R_M / cell)


def loss(s, data_M, weights, pms: pm.PMSetup, ls: LossSetup, an: Anneal) -> dict:
    delta = pm.final_density(s, pms)
    M_nn = nn_halo_map(delta, weights, pms, ls, an.a)
    L_res, _ = residual_terms(M_nn, data_M, pms, ls, an)
    L_pri = prior(s, pm.power_half(pms))
    return {"loss": L_pri + L_res, "prior": L_pri, "residual": L_res}


def loss_and_grad(s, data_M, weights, pms: pm.PMSetup, ls: LossSetup, an: Anneal):
    """Returns (loss parts dict, gradient w.r.t. the half-array entries of s)."""
    N = pms.N
    x_fin, checkpoints, _ = pm.pm_forward(s, pms)
    delta = pm.density(x_fin, N)
    f = features(delta, pms, ls)
    M_nn = _head_forward(f, weights, ls, an.a)
    L_res, cache = residual_terms(M_nn, data_M, pms, ls, an)
    P = pm.power_half(pms)
    L_pri = prior(s, P)
    g_M = residual_grad(cache, pms, ls, an)
    g_delta = features_T(_head_backward(g_M, f, weights, ls, an.a), pms, ls)
    g_s = pm.final_density_T(checkpoints, x_fin, g_delta, pms, s) + prior_grad(s, P)
    g_s[0, 0, 0] = 0
    return {"loss": L_pri + L_res, "prior": L_pri, "residual": L_res}, g_s


def synthetic_data(white_true: np.ndarray, scatter: np.ndarray, weights, pms: pm.PMSetup, ls: LossSetup,
                   sigma_ln: float = 0.3, a: float = 3.0) -> np.ndarray:
    """Data mass field: the model on the true linear field times log-normal scatter exp(sigma g)."""
    s_true = pm.linear_field(white_true, pms)
    M = nn_halo_map(pm.final_density(s_true, pms), weights, pms, ls, a)
    return M * np.exp(sigma_ln * np.asarray(scatter, np.float64))
