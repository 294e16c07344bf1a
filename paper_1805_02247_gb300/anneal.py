"""Annealed reconstruction driver (Sec. 5.2-5.3), sequencing recon_step().

The paper anneals three knobs of the loss while L-BFGS runs: the Gaussian
smoothing of the residual (N_sm = 4, 2, 1, 0.5, 0 cells), the nuisance mass M0
(1e12 then 1e11 M_sun/h) and, for the logistic position head, its sharpness a
(1, 2, 3). Each stage iterates until the loss stops decreasing by 0.1% between
iterations. Every iteration is one recon_step() on the GPU; this module only
orders the stages.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

from .pmrecon import Context, PMRError


@dataclass(frozen=True)
class Stage:
    R_sm: float     # residual smoothing, Mpc/h
    M0: float       # M_sun/h
    a: float = 3.0  # logistic sharpness of the two-network head (unused by the single-network head)


def paper_schedule(cell: float) -> list[Stage]:
    """The schedule of Sec. 5.3 for a single-network head (no sharpness knob):
    M0 = 1e12 with N_sm = 4, 2, 1, 0.5, 0 cells, then M0 = 1e11 with N_sm = 1, 0.5, 0."""
    stages = [Stage(n * cell, 1e12) for n in (4, 2, 1, 0.5, 0)]
    stages += [Stage(n * cell, 1e11) for n in (1, 0.5, 0)]
    return stages


def two_network_schedule(cell: float) -> list[Stage]:
    """Sec. 5.3 with the two-network head: at M0 = 1e12 the smoothing steps
    through N_sm = 4, 2, 1, 0.5, 0 cells, and at each N_sm the logistic
    sharpness runs a = 1, 2, 3; then M0 = 1e11 with a = 3 at N_sm = 1, 0.5, 0."""
    stages = [Stage(n * cell, 1e12, a) for n in (4, 2, 1, 0.5, 0) for a in (1.0, 2.0, 3.0)]
    stages += [Stage(n * cell, 1e11, 3.0) for n in (1, 0.5, 0)]
    return stages


def smoothing_schedule(radii_mpc, M0: float) -> list[Stage]:
    """Residual smoothing annealed over the given radii (Mpc/h) at one M0."""
    return [Stage(float(r), M0) for r in radii_mpc]


def reconstruct(ctx: Context, s, data, stages, max_iter: int = 100, callback=None, min_iter: int = 1,
                stage_end=None):
    """Runs the stages on s (complex64 half array, updated in place).

    Returns a list of per-iteration records {stage, iter, loss, prior, residual,
    converged, seconds}. A stage ends when recon_step reports convergence (from
    its min_iter-th iteration on) or after max_iter iterations; a line-search
    failure ends the stage. stage_end(index, stage), if given, runs after each
    stage (per-stage dumps).
    """
    history = []
    for si, st in enumerate(stages):
        ctx.lbfgs_reset()
        for it in range(max_iter):
            t0 = time.perf_counter()
            try:
                parts, conv = ctx.recon_step(s, data, st.R_sm, st.M0, st.a)
            except PMRError as e:
                if e.code == -5:  # PMR_ELINESEARCH: no decrease left at this stage
                    break
                raise
            rec = {"stage": si, "iter": it, "loss": parts[0], "prior": parts[1], "residual": parts[2],
                   "converged": conv, "seconds": time.perf_counter() - t0}
            history.append(rec)
            if callback:
                callback(rec)
            if conv and it + 1 >= min_iter:
                break
        if stage_end:
            stage_end(si, st)
    return history
