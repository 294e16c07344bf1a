"""L-BFGS step of Sec. 5.2 (FP64, numpy).

The paper names L-BFGS and its stop rule (the loss per degree of freedom stops
decreasing by 0.1% between iterations, Sec. 5.3) but not its memory, initial
Hessian or line search. Readings:
* memory m = 10 correction pairs; a pair is stored only if s^T y > 1e-10 |s| |y|;
* initial inverse Hessian: for the reconstruction, a diagonal D = P~(k) / w_k,
  the exact inverse Hessian of the Gaussian prior of Eq. (priorpdf) (zero at
  k = 0), so the search runs in whitened variables. The first step is -D g;
  later ones scale it as gamma D with gamma = s^T y / y^T D y of the newest pair
  (the usual scaling of the initial matrix, Nocedal & Wright Sec. 7.2, with the
  preconditioner D in place of I), which lets unit steps pass the line search
  once the data term dominates the curvature. Without a diagonal, H0 = gamma I
  with gamma = s^T y / y^T y and the first step is -g / |g|. A non-descent
  direction clears the memory and falls back to the first step;
* backtracking Armijo line search: step 1, halved up to 20 times, accepted when
  L(s + t d) <= L(s) + c1 t g.d with c1 = 1e-4; failure is an error;
* converged when (L_old - L_new) / |L_old| < tol (tol = 1e-3).
Inner products are the plain real inner product over the half-array entries
(real and imaginary parts are independent variables, Sec. 5.1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def dot(a: np.ndarray, b: np.ndarray) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    if np.iscomplexobj(a) or np.iscomplexobj(b):
        return float(np.sum(a.real * b.real + a.imag * b.imag))
    return float(np.sum(a * b))


def two_loop(g: np.ndarray, S: list, Y: list, H0=None) -> np.ndarray:
    """Direction d = -H g from the stored pairs (oldest first in S, Y).

    H0: real diagonal D of the initial inverse Hessian (same shape as g), used
    as gamma D, or None for gamma I."""
    q = g.copy()
    alphas = []
    for s, y in zip(reversed(S), reversed(Y)):
        rho = 1.0 / dot(y, s)
        a = rho * dot(s, q)
        q = q - a * y
        alphas.append((a, rho))
    if H0 is None:
        r = dot(S[-1], Y[-1]) / dot(Y[-1], Y[-1]) * q
    else:
        r = dot(S[-1], Y[-1]) / dot(Y[-1], H0 * Y[-1]) * (H0 * q)
    for (s, y), (a, rho) in zip(zip(S, Y), reversed(alphas)):
        b = rho * dot(y, r)
        r = r + (a - b) * s
    return -r


@dataclass
class LBFGSState:
    x: np.ndarray
    f: float | None = None
    g: np.ndarray | None = None
    S: list = field(default_factory=list)
    Y: list = field(default_factory=list)


def step(fun, st: LBFGSState, m: int = 10, c1: float = 1e-4, max_ls: int = 20, tol: float = 1e-3, H0=None):
    """One L-BFGS iteration. fun(x) -> (f, g). Returns (status, converged, n_evals)."""
    evals = 0
    if st.g is None:
        st.f, st.g = fun(st.x)
        evals += 1
    g = st.g
    if st.S:
        d = two_loop(g, st.S, st.Y, H0)
        gd = dot(g, d)
        if not gd < 0:
            st.S.clear(); st.Y.clear()
    if not st.S:
        d = -g / np.sqrt(dot(g, g)) if H0 is None else -H0 * g
        gd = dot(g, d)
    t = 1.0
    for _ in range(max_ls):
        x_new = st.x + t * d
        f_new, g_new = fun(x_new)
        evals += 1
        if f_new <= st.f + c1 * t * gd:
            break
        t *= 0.5
    else:
        return "linesearch_failed", False, evals
    sk = x_new - st.x
    yk = g_new - g
    sy = dot(sk, yk)
    if sy > 1e-10 * np.sqrt(dot(sk, sk) * dot(yk, yk)):
        st.S.append(sk); st.Y.append(yk)
        if len(st.S) > m:
            st.S.pop(0); st.Y.pop(0)
    converged = (st.f - f_new) < tol * abs(st.f)
    st.x, st.f, st.g = x_new, f_new, g_new
    return "ok", converged, evals
