"""Whole-gradient parity on the register-FFT code path, against the FP64 oracle.

Meshes of N in {64, 128, 192, 256, 512} run every FFT pass as the register
four-step kernels (column passes, z passes, and the fused x-passes that carry
the Fourier multipliers, including the three-to-one force transpose and the
2LPT Hessian accumulations of the adjoint); smaller meshes take the
shared-memory Stockham kernels. The benchmark's 256^3 evaluation runs only the
register kernels, so the hand-written adjoint of Sec. 5.2 (PM derivatives,
network, loss) is compared here element by element at sizes the oracle still
finishes in seconds to a minute:

* 64^3, L = 400 Mpc/h, 10 PM steps, Zel'dovich ICs (the benchmark's box and
  step count at 1/64 of its voxels);
* 128^3, L = 400 Mpc/h, 5 PM steps, second-order LPT ICs (the annealed
  reconstruction workload's shape, Sec. 3 and 5.3).

M0 = 1e11: at 64^3 in a 400 Mpc/h box the R_M = 3 Mpc/h smoothing is below a
cell, and the truncated Gaussian rings the smoothed data mass down to about
-2.6e10, so the 1e8 of the small workload would put a negative number inside
the log (the oracle returns NaN there too).

Tolerances are the float32 path's: 1e-5 relative on fields and loss parts,
1e-4 relative L2 on gradients.
"""
import numpy as np
import pytest
import torch

from oracle import loss as oloss
from oracle import pm as opm
from paper_1805_02247_gb300 import pmrecon, synth

from gpu_util import context, f32, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
GRAD_TOL = 1e-4


def _problem(N, L, nsteps, lpt_order):
    setup = opm.PMSetup(N=N, L=L, nsteps=nsteps, lpt_order=lpt_order)
    s = f32(np.sqrt(0.1) * opm.linear_field(f32(synth.white_noise(N, 0)), setup))
    w = synth.xavier_weights(1)
    data = f32(oloss.synthetic_data(f32(synth.white_noise(N, 2)), f32(synth.scatter_noise(N, 2)), w, setup,
                                    oloss.LossSetup()))
    return setup, s, w, data


@pytest.fixture(scope="module")
def za64():
    N, L, nsteps = 64, 400.0, 10
    setup, s, w, data = _problem(N, L, nsteps, 1)
    ctx, _ = context(N=N, L=L, nsteps=nsteps)
    yield dict(ctx=ctx, setup=setup, s=s, w=w, data=data, N=N)
    ctx.close()


@pytest.fixture(scope="module")
def lpt128():
    N, L, nsteps = 128, 400.0, 5
    setup, s, w, data = _problem(N, L, nsteps, 2)
    ctx, _ = context(N=N, L=L, nsteps=nsteps, lpt_order=2)
    yield dict(ctx=ctx, setup=setup, s=s, w=w, data=data, N=N)
    ctx.close()


def _loss_and_grad_parity(job, R_sm, M0):
    ctx, setup, s, w, data = job["ctx"], job["setup"], job["s"], job["w"], job["data"]
    parts, g = ctx.loss_and_grad(to_dev(s), to_dev(data), R_sm, M0)
    want, gwant = oloss.loss_and_grad(s, data, w, setup, oloss.LossSetup(), oloss.Anneal(R_sm=R_sm, M0=M0))
    assert np.isfinite(want["loss"])
    assert parts[0] == pytest.approx(want["loss"], rel=FIELD_TOL)
    assert parts[1] == pytest.approx(want["prior"], rel=FIELD_TOL)
    assert parts[2] == pytest.approx(want["residual"], rel=FIELD_TOL)
    # the residual's share of the gradient is not negligible next to the prior's
    gprior = oloss.prior_grad(s, opm.power_half(setup))
    assert np.linalg.norm(gwant - gprior) > 0.3 * np.linalg.norm(gwant)
    assert rel_l2(to_np(g), gwant) <= GRAD_TOL


def test_loss_and_grad_parity_64cubed_10_steps(za64):
    _loss_and_grad_parity(za64, R_sm=4.0, M0=1e11)


def test_loss_and_grad_parity_128cubed_2lpt_5_steps(lpt128):
    _loss_and_grad_parity(lpt128, R_sm=2.0, M0=1e11)


def test_pm_forward_and_adjoint_64cubed_10_steps(za64):
    ctx, setup, s, N = za64["ctx"], za64["setup"], za64["s"], za64["N"]
    delta = to_np(ctx.pm_forward(to_dev(s)))
    x_fin, cps, _ = opm.pm_forward(s, setup)
    assert rel_l2(delta, opm.density(x_fin, N)) <= FIELD_TOL
    gd = f32(synth.gaussian_vector((N, N, N), seed=23))
    got = to_np(ctx.pm_adjoint(to_dev(gd)))
    assert rel_l2(got, opm.final_density_T(cps, x_fin, gd, setup, s)) <= GRAD_TOL


@pytest.mark.parametrize("lpt_order", [1, 2])
def test_lpt_ics_and_adjoint_64cubed(lpt_order):
    # the Zel'dovich (and 2LPT) displacement and its transpose on the register
    # passes: odd multipliers, the six Hessian c2r's and their accumulating r2c's
    N, L = 64, 400.0
    setup = opm.PMSetup(N=N, L=L, nsteps=10, lpt_order=lpt_order)
    s = f32(opm.linear_field(f32(synth.white_noise(N, 0)), setup))
    ctx, _ = context(N=N, L=L, nsteps=10, lpt_order=lpt_order)
    disp, mom = ctx.lpt_ics(to_dev(s))
    x_want, p_want = opm.lpt_ics(s, setup)
    assert rel_l2(to_np(disp), x_want - opm.lattice(N)) <= FIELD_TOL
    assert rel_l2(to_np(mom), p_want) <= FIELD_TOL
    lx = f32(synth.gaussian_vector((3, N ** 3), seed=33))
    lp = f32(synth.gaussian_vector((3, N ** 3), seed=34))
    g = to_np(ctx.lpt_ics_adjoint(to_dev(s), to_dev(lx), to_dev(lp)))
    assert rel_l2(g, opm.lpt_ics_T(lx, lp, s, setup)) <= GRAD_TOL
    ctx.close()


def test_recon_loss_autograd_function_64cubed(za64):
    # the differentiation pattern: L(s) behind torch.autograd.Function, its
    # backward the hand-written adjoint; compared with the oracle's gradient
    ctx, setup, s, w, data = za64["ctx"], za64["setup"], za64["s"], za64["w"], za64["data"]
    R_sm, M0 = 4.0, 1e11
    s_dev = to_dev(s).requires_grad_(True)
    loss = pmrecon.ReconLoss.apply(s_dev, to_dev(data), ctx, R_sm, M0)
    (2.0 * loss).backward()
    want, gwant = oloss.loss_and_grad(s, data, w, setup, oloss.LossSetup(), oloss.Anneal(R_sm=R_sm, M0=M0))
    assert float(loss) == pytest.approx(want["loss"], rel=FIELD_TOL)
    assert s_dev.grad.dtype == torch.complex64
    assert rel_l2(to_np(s_dev.grad), 2.0 * gwant) <= GRAD_TOL


def test_pm_forward_autograd_function_64cubed(za64):
    ctx, setup, s, N = za64["ctx"], za64["setup"], za64["s"], za64["N"]
    s_dev = to_dev(s).requires_grad_(True)
    delta = pmrecon.PMForward.apply(s_dev, ctx)
    gd = f32(synth.gaussian_vector((N, N, N), seed=24))
    (delta * to_dev(gd)).sum().backward()
    x_fin, cps, _ = opm.pm_forward(s, setup)
    assert rel_l2(to_np(delta.detach()), opm.density(x_fin, N)) <= FIELD_TOL
    assert rel_l2(to_np(s_dev.grad), opm.final_density_T(cps, x_fin, gd, setup, s)) <= GRAD_TOL
