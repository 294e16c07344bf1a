"""Annealed reconstruction (Sec. 5.2-5.3) on the FP64 oracle: stages of
(R_sm, M0[, a]), each iterating the oracle L-BFGS step until the loss stops
decreasing by tol (relative) or max_iter iterations pass."""
from __future__ import annotations

from . import lbfgs, loss


def reconstruct(s, data, weights, pms, ls, stages, max_iter=100, tol=1e-3):
    """stages: iterable of (R_sm, M0) or (R_sm, M0, a). Returns (s_final, history of losses per stage)."""
    history = []
    x = s
    H0 = loss.prior_inverse_hessian(pms)
    for stage in stages:
        R_sm, M0 = stage[0], stage[1]
        a = stage[2] if len(stage) > 2 else 3.0
        an = loss.Anneal(R_sm=R_sm, M0=M0, a=a)

        def fun(v, an=an):
            parts, g = loss.loss_and_grad(v, data, weights, pms, ls, an)
            return parts["loss"], g

        st = lbfgs.LBFGSState(x=x.copy())
        losses = []
        for _ in range(max_iter):
            status, conv, _ = lbfgs.step(fun, st, tol=tol, H0=H0)
            if status != "ok":
                break
            losses.append(st.f)
            if conv:
                break
        history.append(losses)
        x = st.x
    return x, history
