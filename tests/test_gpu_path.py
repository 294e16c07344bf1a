"""GPU parity of the whole path through the C ABI against the FP64 oracle:
pm_forward / pm_adjoint, nn_halo_map and its adjoint, loss_and_grad, recon_step.
"""
import numpy as np
import pytest
import torch

from oracle import lbfgs as olb
from oracle import loss as oloss
from oracle import nn as onn
from oracle import pm as opm
from paper_1805_02247_gb300 import synth

from gpu_util import context, f32, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
GRAD_TOL = 1e-4


def _problem(N, L, nsteps, amp=1.0):
    setup = opm.PMSetup(N=N, L=L, nsteps=nsteps)
    s = f32(amp * opm.linear_field(f32(synth.white_noise(N, 0)), setup))
    return setup, s


@pytest.mark.parametrize("N,L,nsteps", [(16, 100.0, 2), (32, 100.0, 3), (24, 400.0, 5)])
def test_pm_forward_parity(N, L, nsteps):
    ctx, _ = context(N=N, L=L, nsteps=nsteps)
    setup, s = _problem(N, L, nsteps)
    delta = to_np(ctx.pm_forward(to_dev(s)))
    assert rel_l2(delta, opm.final_density(s, setup)) <= FIELD_TOL


@pytest.mark.parametrize("N,L,nsteps", [(16, 100.0, 2), (32, 100.0, 3)])
def test_pm_adjoint_parity(N, L, nsteps):
    ctx, _ = context(N=N, L=L, nsteps=nsteps)
    setup, s = _problem(N, L, nsteps)
    g = synth.gaussian_vector((N, N, N), seed=21)
    ctx.pm_forward(to_dev(s))
    got = to_np(ctx.pm_adjoint(to_dev(g)))
    x_fin, cps, _ = opm.pm_forward(s, setup)
    want = opm.final_density_T(cps, x_fin, f32(g), setup)
    assert rel_l2(got, want) <= GRAD_TOL


@pytest.mark.parametrize("N,L,nsteps", [(16, 100.0, 2), (24, 400.0, 5)])
def test_pm_forward_and_adjoint_parity_with_2lpt(N, L, nsteps):
    ctx, _ = context(N=N, L=L, nsteps=nsteps, lpt_order=2)
    setup = opm.PMSetup(N=N, L=L, nsteps=nsteps, lpt_order=2)
    _, s = _problem(N, L, nsteps)
    delta = to_np(ctx.pm_forward(to_dev(s)))
    x_fin, cps, _ = opm.pm_forward(s, setup)
    assert rel_l2(delta, opm.density(x_fin, N)) <= FIELD_TOL
    g = synth.gaussian_vector((N, N, N), seed=22)
    got = to_np(ctx.pm_adjoint(to_dev(g)))
    assert rel_l2(got, opm.final_density_T(cps, x_fin, f32(g), setup, s)) <= GRAD_TOL
    # computing initial conditions on their own replaces the state the adjoint needs
    from paper_1805_02247_gb300.pmrecon import PMRError
    ctx.lpt_ics(to_dev(s))
    with pytest.raises(PMRError, match="ESTATE"):
        ctx.pm_adjoint(to_dev(g))


def test_pm_adjoint_needs_forward():
    from paper_1805_02247_gb300.pmrecon import PMRError
    ctx, _ = context(N=8)
    with pytest.raises(PMRError, match="ESTATE"):
        ctx.pm_adjoint(torch.zeros(8, 8, 8, device="cuda"))


def test_nn_halo_map_and_adjoint_parity():
    N, L = 32, 100.0
    ctx, _ = context(N=N, L=L)
    setup = opm.PMSetup(N=N, L=L, nsteps=3)
    ls = oloss.LossSetup()
    w = synth.xavier_weights(1)
    delta = f32(2.0 * synth.gaussian_vector((N, N, N), seed=31))
    M = to_np(ctx.nn_halo_map(to_dev(delta)))
    assert rel_l2(M, oloss.nn_halo_map(delta, w, setup, ls)) <= FIELD_TOL
    gM = f32(synth.gaussian_vector((N, N, N), seed=32))
    gd = to_np(ctx.nn_halo_map_adjoint(to_dev(delta), to_dev(gM)))
    assert rel_l2(gd, oloss.nn_halo_map_T(gM, delta, w, setup, ls)) <= GRAD_TOL


@pytest.mark.parametrize("nn_path,ftol,gtol", [(0, FIELD_TOL, GRAD_TOL), (2, FIELD_TOL, GRAD_TOL), (1, 1e-2, 5e-2),
                                               (3, 2e-2, 1e-1)])
@pytest.mark.parametrize("N,L", [(32, 100.0), (24, 60.0)])
def test_network_paths_against_oracle(nn_path, ftol, gtol, N, L):
    # 0: tcgen05 tensor cores with two-part TF32 operands (float32 accuracy),
    # 2: float32 CUDA cores, 1: plain TF32 tensor cores, 3: bfloat16 tensor
    # cores with float32 accumulation (8-bit mantissas, ~2^-9 per operand; the
    # backward also sees ReLU masks flip on near-zero units, observed 5.6% on the
    # input gradient at 32^3): percent-level bounds, the bench reports the errors.
    # N = 24 leaves partial voxel tiles (tiles are 2 x 4 x 16).
    ctx, _ = context(N=N, L=L, nn_path=nn_path)
    setup = opm.PMSetup(N=N, L=L, nsteps=3)
    ls = oloss.LossSetup()
    w = synth.xavier_weights(1)
    delta = f32(3.0 * synth.gaussian_vector((N, N, N), seed=51))
    M = to_np(ctx.nn_halo_map(to_dev(delta)))
    assert rel_l2(M, oloss.nn_halo_map(delta, w, setup, ls)) <= ftol
    gM = f32(synth.gaussian_vector((N, N, N), seed=52))
    gd = to_np(ctx.nn_halo_map_adjoint(to_dev(delta), to_dev(gM)))
    assert rel_l2(gd, oloss.nn_halo_map_T(gM, delta, w, setup, ls)) <= gtol


@pytest.mark.parametrize("nn_path", [2, 0])
@pytest.mark.parametrize("N,L,a", [(32, 100.0, 1.0), (24, 60.0, 3.0)])
def test_two_network_head_against_oracle(nn_path, N, L, a):
    # Sec. 2.1: M = M_scale logistic(y, a) NNm(f) on both network paths
    ctx, _ = context(N=N, L=L, nn_path=nn_path, head=1)
    setup = opm.PMSetup(N=N, L=L, nsteps=3)
    ls = oloss.LossSetup(head="two_net")
    w = synth.two_net_weights(1)
    delta = f32(3.0 * synth.gaussian_vector((N, N, N), seed=61))
    M = to_np(ctx.nn_halo_map(to_dev(delta), a))
    assert rel_l2(M, oloss.nn_halo_map(delta, w, setup, ls, a)) <= FIELD_TOL
    gM = f32(synth.gaussian_vector((N, N, N), seed=62))
    gd = to_np(ctx.nn_halo_map_adjoint(to_dev(delta), to_dev(gM), a))
    assert rel_l2(gd, oloss.nn_halo_map_T(gM, delta, w, setup, ls, a)) <= GRAD_TOL


def _data(N, L, nsteps, head="softplus"):
    setup = opm.PMSetup(N=N, L=L, nsteps=nsteps)
    two = head == "two_net"
    w = synth.two_net_weights(1) if two else synth.xavier_weights(1)
    return f32(oloss.synthetic_data(f32(synth.white_noise(N, 2)), f32(synth.scatter_noise(N, 2)), w, setup,
                                    oloss.LossSetup(head=head)))


@pytest.mark.parametrize("nn_path", [2, 0])
@pytest.mark.parametrize("a", [1.0, 3.0])
def test_two_network_loss_and_grad_parity(nn_path, a):
    N, L, nsteps, R_sm, M0 = 16, 50.0, 2, 4.0, 1e11
    ctx, _ = context(N=N, L=L, nsteps=nsteps, nn_path=nn_path, head=1)
    setup, s = _problem(N, L, nsteps, amp=np.sqrt(0.1))
    data = _data(N, L, nsteps, head="two_net")
    parts, g = ctx.loss_and_grad(to_dev(s), to_dev(data), R_sm, M0, a=a)
    want, gwant = oloss.loss_and_grad(s, data, synth.two_net_weights(1), setup, oloss.LossSetup(head="two_net"),
                                      oloss.Anneal(R_sm=R_sm, M0=M0, a=a))
    assert parts[0] == pytest.approx(want["loss"], rel=FIELD_TOL)
    assert parts[2] == pytest.approx(want["residual"], rel=FIELD_TOL)
    assert rel_l2(to_np(g), gwant) <= GRAD_TOL


@pytest.mark.parametrize("N,L,nsteps,R_sm,M0", [(32, 100.0, 3, 4.0, 1e8), (16, 100.0, 2, 0.0, 1e11),
                                                (24, 400.0, 5, 2.0, 1e12)])
def test_loss_and_grad_parity(N, L, nsteps, R_sm, M0):
    ctx, _ = context(N=N, L=L, nsteps=nsteps)
    setup, s = _problem(N, L, nsteps, amp=np.sqrt(0.1))
    data = _data(N, L, nsteps)
    parts, g = ctx.loss_and_grad(to_dev(s), to_dev(data), R_sm, M0)
    w = synth.xavier_weights(1)
    want, gwant = oloss.loss_and_grad(s, data, w, setup, oloss.LossSetup(), oloss.Anneal(R_sm=R_sm, M0=M0))
    assert parts[0] == pytest.approx(want["loss"], rel=FIELD_TOL)
    assert parts[1] == pytest.approx(want["prior"], rel=FIELD_TOL)
    assert parts[2] == pytest.approx(want["residual"], rel=FIELD_TOL)
    assert rel_l2(to_np(g), gwant) <= GRAD_TOL


def test_loss_and_grad_parity_with_2lpt():
    N, L, nsteps, R_sm, M0 = 16, 50.0, 2, 4.0, 1e8
    ctx, _ = context(N=N, L=L, nsteps=nsteps, lpt_order=2)
    setup = opm.PMSetup(N=N, L=L, nsteps=nsteps, lpt_order=2)
    _, s = _problem(N, L, nsteps, amp=np.sqrt(0.1))
    data = _data(N, L, nsteps)
    parts, g = ctx.loss_and_grad(to_dev(s), to_dev(data), R_sm, M0)
    want, gwant = oloss.loss_and_grad(s, data, synth.xavier_weights(1), setup, oloss.LossSetup(),
                                      oloss.Anneal(R_sm=R_sm, M0=M0))
    assert parts[0] == pytest.approx(want["loss"], rel=FIELD_TOL)
    assert rel_l2(to_np(g), gwant) <= GRAD_TOL


def test_bf16_network_loss_and_gradient_against_oracle():
    # the bf16 tensor-core path inside the whole loss and gradient
    N, L, nsteps, R_sm, M0 = 16, 50.0, 2, 4.0, 1e8
    ctx, _ = context(N=N, L=L, nsteps=nsteps, nn_path=3)
    setup, s = _problem(N, L, nsteps, amp=np.sqrt(0.1))
    data = _data(N, L, nsteps)
    parts, g = ctx.loss_and_grad(to_dev(s), to_dev(data), R_sm, M0)
    want, gwant = oloss.loss_and_grad(s, data, synth.xavier_weights(1), setup, oloss.LossSetup(),
                                      oloss.Anneal(R_sm=R_sm, M0=M0))
    assert parts[0] == pytest.approx(want["loss"], rel=1e-2)
    assert rel_l2(to_np(g), gwant) <= 1e-1


def test_loss_nan_is_reported():
    from paper_1805_02247_gb300.pmrecon import PMRError
    N = 16
    ctx, _ = context(N=N)
    _, s = _problem(N, 100.0, 3)
    data = np.full((N, N, N), np.nan, np.float32)
    with pytest.raises(PMRError, match="ENAN"):
        ctx.loss_and_grad(to_dev(s), to_dev(data), 0.0, 1e8)


@pytest.mark.parametrize("nn_path,later_loss_tol", [(2, 1e-4), (0, 1e-4)])
def test_recon_step_follows_oracle_lbfgs(nn_path, later_loss_tol):
    N, L, nsteps = 16, 50.0, 2  # R_M = 3 Mpc/h spans ~1 cell: resolved smoothing
    R_sm, M0 = 4.0, 1e8
    ctx, _ = context(N=N, L=L, nsteps=nsteps, nn_path=nn_path)
    setup, s0 = _problem(N, L, nsteps, amp=np.sqrt(0.1))
    data = _data(N, L, nsteps)
    w = synth.xavier_weights(1)
    ls, an = oloss.LossSetup(), oloss.Anneal(R_sm=R_sm, M0=M0)

    def fun(x):
        parts, g = oloss.loss_and_grad(x, data, w, setup, ls, an)
        return parts["loss"], g

    st = olb.LBFGSState(x=s0.copy())
    s_dev = to_dev(s0)
    d_dev = to_dev(data)
    # The first step's loss follows the oracle to 1e-5. The iterate is a float32
    # copy of a float64 master point built from float32 gradients; the L-BFGS
    # history multiplies their rounding by the conditioning of the recursion,
    # so the iterate bound (the gradient tolerance) applies to the first two
    # iterations and later losses, which sit on slightly different points of
    # the trajectory, are held to 1e-4 (observed: 1.1e-5 with the float32
    # CUDA-core network, 3.4e-5 with the two-part TF32 tensor-core network).
    H0 = oloss.prior_inverse_hessian(setup)
    for it in range(4):
        status, conv_o, _ = olb.step(fun, st, H0=H0)
        parts, conv_g = ctx.recon_step(s_dev, d_dev, R_sm, M0)
        assert status == "ok"
        assert parts[0] == pytest.approx(st.f, rel=1e-5 if it == 0 else later_loss_tol), it
        if it < 2:
            assert rel_l2(to_np(s_dev), st.x) <= 1e-4, it
        assert conv_g == conv_o


def test_annealed_reconstruction_follows_oracle():
    # Sec. 5.2 annealing: residual smoothing 2 -> 1 -> 0 cells, then M0 1e9 -> 1e8,
    # one L-BFGS iteration per stage, so every stage starts afresh from the last
    # iterate (memory reset, new loss). A longer stay in one stage is not compared
    # point by point: after a short backtracked first step the curvature pair
    # amplifies float32 gradient rounding (recon_step's own test bounds that).
    # Tolerance: on this problem the oracle's own four stage losses move by at
    # most 2e-6 when its gradients carry 1e-6 relative noise.
    from oracle import anneal as oanneal
    from paper_1805_02247_gb300 import anneal

    N, L, nsteps = 16, 50.0, 2
    ctx, _ = context(N=N, L=L, nsteps=nsteps)
    setup, s0 = _problem(N, L, nsteps, amp=np.sqrt(0.1))
    data = _data(N, L, nsteps)
    stages = [anneal.Stage(6.25, 1e9), anneal.Stage(3.125, 1e9), anneal.Stage(0.0, 1e9), anneal.Stage(0.0, 1e8)]
    s_dev = to_dev(s0)
    hist = anneal.reconstruct(ctx, s_dev, to_dev(data), stages, max_iter=1)
    _, ohist = oanneal.reconstruct(s0, data, synth.xavier_weights(1), setup, oloss.LossSetup(),
                                   [(st.R_sm, st.M0) for st in stages], max_iter=1)
    assert [r["stage"] for r in hist] == [0, 1, 2, 3]
    got = [r["loss"] for r in hist]
    want = [h[0] for h in ohist]
    assert got[0] == pytest.approx(want[0], rel=1e-5)
    assert np.allclose(got, want, rtol=1e-4)
    # a longer stage keeps decreasing its own loss
    more = anneal.reconstruct(ctx, s_dev, to_dev(data), [anneal.Stage(0.0, 1e8)], max_iter=4)
    assert np.all(np.diff([r["loss"] for r in more]) < 0)


def test_two_network_annealing_over_sharpness_follows_oracle():
    # Sec. 5.2: the logistic sharpness a is annealed between stages (1 -> 2),
    # one iteration per stage. The two-network loss is steeper: under 1e-6
    # relative gradient noise the oracle's second-stage loss moves by 6.4e-5
    # (7.4e-5 under 1e-5), so it is held to 5e-4; the first to the loss tolerance.
    from oracle import anneal as oanneal
    from paper_1805_02247_gb300 import anneal

    N, L, nsteps = 16, 50.0, 2
    ctx, _ = context(N=N, L=L, nsteps=nsteps, head=1)
    setup, s0 = _problem(N, L, nsteps, amp=np.sqrt(0.1))
    data = _data(N, L, nsteps, head="two_net")
    stages = [anneal.Stage(6.25, 1e11, 1.0), anneal.Stage(6.25, 1e11, 2.0)]
    hist = anneal.reconstruct(ctx, to_dev(s0), to_dev(data), stages, max_iter=1)
    _, ohist = oanneal.reconstruct(s0, data, synth.two_net_weights(1), setup, oloss.LossSetup(head="two_net"),
                                   [(st.R_sm, st.M0, st.a) for st in stages], max_iter=1)
    got = [r["loss"] for r in hist]
    assert got[0] == pytest.approx(ohist[0][0], rel=1e-5)
    assert got[1] == pytest.approx(ohist[1][0], rel=5e-4)


def test_graph_replay_matches_direct_launches():
    # pmr_use_graphs: the captured evaluation gives the same bits as direct launches,
    # and a change of the anneal parameters re-captures
    from paper_1805_02247_gb300 import pmrecon
    N, L, nsteps = 16, 50.0, 2
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        cfg = pmrecon.default_config(N=N, L=L, nsteps=nsteps)
        ctx = pmrecon.Context(cfg, torch.from_numpy(synth.xavier_weights(1)).cuda(), stream=stream)
        _, s = _problem(N, L, nsteps, amp=np.sqrt(0.1))
        s_dev, d_dev = to_dev(s), to_dev(_data(N, L, nsteps))
        direct = [ctx.loss_and_grad(s_dev, d_dev, R, 1e8) for R in (4.0, 2.0)]
        direct = [(p, g.clone()) for p, g in direct]
        ctx.use_graphs(True)
        for _ in range(2):  # capture, then replay
            for (p0, g0), R in zip(direct, (4.0, 2.0)):
                p1, g1 = ctx.loss_and_grad(s_dev, d_dev, R, 1e8)
                assert p1 == p0
                assert torch.equal(g1, g0)
        stream.synchronize()
        ctx.close()


def test_graphs_need_a_stream():
    from paper_1805_02247_gb300.pmrecon import PMRError
    ctx, _ = context(N=8)  # default (legacy) stream
    with pytest.raises(PMRError, match="EINVAL"):
        ctx.use_graphs(True)


def test_pm_forward_autograd_detects_a_replaced_trajectory():
    # the context stores one trajectory: a backward whose forward was followed
    # by another forward on the same context raises instead of differentiating
    # the wrong trajectory; the newest forward's backward still works
    from paper_1805_02247_gb300.pmrecon import PMForward, PMRError
    N, L, nsteps = 16, 100.0, 2
    ctx, _ = context(N=N, L=L, nsteps=nsteps)
    setup, s = _problem(N, L, nsteps)
    assert ctx.forward_id() == -1
    s1 = to_dev(s).requires_grad_(True)
    s2 = to_dev(0.5 * s).requires_grad_(True)
    d1 = PMForward.apply(s1, ctx)
    d2 = PMForward.apply(s2, ctx)
    with pytest.raises(PMRError, match="ESTATE"):
        d1.sum().backward()
    g = synth.gaussian_vector((N, N, N), seed=25)
    (d2 * to_dev(g)).sum().backward()
    x_fin, cps, _ = opm.pm_forward(f32(0.5 * s), setup)
    assert rel_l2(to_np(s2.grad), opm.final_density_T(cps, x_fin, f32(g), setup)) <= GRAD_TOL


@pytest.mark.parametrize("nn_path", [0, 3])
def test_tensor_core_wait_timeout_is_reported_and_the_context_recovers(nn_path):
    # failure detection without a GPU fault: the stall hook makes the tensor-core
    # kernels issue no MMAs, so their bounded accumulator waits run out; each
    # kernel records the timeout, frees its tensor memory and returns. The loss
    # call reports PMR_ETIMEOUT, an asynchronous call's timeout surfaces at
    # pmr_sync, and the same context then computes the oracle's loss and gradient.
    from paper_1805_02247_gb300.pmrecon import PMRError
    N, L, nsteps, R_sm, M0 = 16, 50.0, 2, 4.0, 1e8
    ctx, _ = context(N=N, L=L, nsteps=nsteps, nn_path=nn_path)
    setup, s = _problem(N, L, nsteps, amp=np.sqrt(0.1))
    data = _data(N, L, nsteps)
    s_dev, d_dev = to_dev(s), to_dev(data)
    ctx.test_stall_mma(True)
    with pytest.raises(PMRError, match="ETIMEOUT"):
        ctx.loss_and_grad(s_dev, d_dev, R_sm, M0)
    ctx.nn_halo_map(to_dev(f32(synth.gaussian_vector((N, N, N), seed=71))))
    with pytest.raises(PMRError, match="ETIMEOUT"):
        ctx.sync()
    ctx.sync()  # reported once, then cleared
    ctx.test_stall_mma(False)
    parts, g = ctx.loss_and_grad(s_dev, d_dev, R_sm, M0)
    want, gwant = oloss.loss_and_grad(s, data, synth.xavier_weights(1), setup, oloss.LossSetup(),
                                      oloss.Anneal(R_sm=R_sm, M0=M0))
    tol = (FIELD_TOL, GRAD_TOL) if nn_path == 0 else (1e-2, 1e-1)
    assert parts[0] == pytest.approx(want["loss"], rel=tol[0])
    assert rel_l2(to_np(g), gwant) <= tol[1]


def test_loss_into_a_device_buffer_without_a_host_read():
    # loss_out may be a device pointer: the parts land on the stream with no
    # synchronisation, equal to what the host read returns
    N, L, nsteps, R_sm, M0 = 16, 50.0, 2, 4.0, 1e8
    ctx, _ = context(N=N, L=L, nsteps=nsteps)
    _, s = _problem(N, L, nsteps, amp=np.sqrt(0.1))
    s_dev, d_dev = to_dev(s), to_dev(_data(N, L, nsteps))
    loss_dev = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    none, g1 = ctx.loss_and_grad(s_dev, d_dev, R_sm, M0, loss_dev=loss_dev)
    assert none is None
    g1 = g1.clone()
    parts, g2 = ctx.loss_and_grad(s_dev, d_dev, R_sm, M0)
    assert tuple(loss_dev.cpu().tolist()) == parts
    assert torch.equal(g1, g2)


@pytest.mark.parametrize("head", [0, 1])
def test_paper_feature_set_through_feat_mix(head):
    # Sec. 2.2's input fields delta_0, delta_R1, delta_R1 - delta_R2 as
    # R_feat = (0, R1, R2) and feat_mix C: folded into the first-layer weights by
    # pmr_create, against the oracle forming the mixed fields explicitly
    mix = (1, 0, 0, 0, 1, 0, 0, 1, -1)
    N, L, nsteps, R_sm, M0 = 16, 50.0, 2, 4.0, 1e11
    two = head == 1
    ctx, _ = context(N=N, L=L, nsteps=nsteps, head=head, R_feat=(0.0, 3.0, 6.0), feat_mix=mix)
    setup = opm.PMSetup(N=N, L=L, nsteps=nsteps)
    ls = oloss.LossSetup(R_feat=(0.0, 3.0, 6.0), feat_mix=mix, head="two_net" if two else "softplus")
    w = synth.two_net_weights(1) if two else synth.xavier_weights(1)
    delta = f32(2.0 * synth.gaussian_vector((N, N, N), seed=81))
    M = to_np(ctx.nn_halo_map(to_dev(delta), 2.0))
    assert rel_l2(M, oloss.nn_halo_map(delta, w, setup, ls, 2.0)) <= FIELD_TOL
    gM = f32(synth.gaussian_vector((N, N, N), seed=82))
    gd = to_np(ctx.nn_halo_map_adjoint(to_dev(delta), to_dev(gM), 2.0))
    assert rel_l2(gd, oloss.nn_halo_map_T(gM, delta, w, setup, ls, 2.0)) <= GRAD_TOL
    _, s = _problem(N, L, nsteps, amp=np.sqrt(0.1))
    data = f32(oloss.synthetic_data(f32(synth.white_noise(N, 2)), f32(synth.scatter_noise(N, 2)), w, setup, ls,
                                    a=2.0))
    parts, g = ctx.loss_and_grad(to_dev(s), to_dev(data), R_sm, M0, a=2.0)
    want, gwant = oloss.loss_and_grad(s, data, w, setup, ls, oloss.Anneal(R_sm=R_sm, M0=M0, a=2.0))
    assert parts[0] == pytest.approx(want["loss"], rel=FIELD_TOL)
    assert rel_l2(to_np(g), gwant) <= GRAD_TOL
