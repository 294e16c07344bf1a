"""Pins for oracle.nn, oracle.loss and oracle.lbfgs."""
import math

import numpy as np
import pytest

from oracle import lbfgs, loss, nn, pm
from paper_1805_02247_gb300 import synth


def rdot(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.sum(a.real * b.real + a.imag * b.imag))


# ----------------------------------------------------------------------------- network

def test_activation_special_values():
    assert nn.softplus(0.0) == pytest.approx(math.log(2.0), rel=1e-15)
    assert nn.softplus(800.0) == pytest.approx(800.0, rel=1e-15)  # no overflow
    assert nn.softplus(-800.0) == pytest.approx(math.exp(-800.0))
    assert nn.relu(-1e-300) == 0.0 and nn.relu(2.5) == 2.5


def test_stencil_order_on_a_delta_field():
    N = 5
    f = np.zeros((3, N, N, N))
    f[1, 2, 3, 4] = 1.0  # field 1, voxel (2,3,4)
    v = nn.stencil_gather(f)
    for r, (ox, oy, oz) in enumerate(nn.STENCIL):
        row = v[27 + r].reshape(N, N, N)
        # v[c,o](x) = f_c(x + o): nonzero at x = (2,3,4) - o
        want = np.zeros((N, N, N)); want[(2 - ox) % N, (3 - oy) % N, (4 - oz) % N] = 1.0
        assert np.array_equal(row, want)
    assert not v[:27].any() and not v[54:].any()
    assert nn.STENCIL[13] == (0, 0, 0)


def test_stencil_transpose():
    rng = np.random.default_rng(1)
    N = 4
    f = rng.standard_normal((3, N, N, N))
    gv = rng.standard_normal((81, N**3))
    assert rdot(nn.stencil_gather(f), gv) == pytest.approx(rdot(f, nn.stencil_gather_T(gv, N)), rel=1e-12)


def test_mlp_closed_form_with_hand_set_weights():
    # W1 picks the centre value of field 0, W2 and w3 pass it through:
    # M = M_scale * softplus(relu(relu(f0(x))) - 0.5)
    N = 4
    w = np.zeros(synth.N_WEIGHTS)
    W1, b1, W2, b2, w3, _ = nn.unpack(w)  # views into w
    W1[0, 13] = 1.0
    W2[0, 0] = 1.0
    w3[0] = 1.0
    w[-1] = -0.5  # b3
    f = np.random.default_rng(2).standard_normal((3, N, N, N))
    M, _ = nn.mlp_forward(f, w, 1e12)
    want = 1e12 * np.log1p(np.exp(np.maximum(f[0], 0.0) - 0.5))
    assert np.allclose(M, want, rtol=1e-14)


def test_mlp_backward_by_finite_differences():
    rng = np.random.default_rng(3)
    N = 4
    w = synth.xavier_weights(1).astype(np.float64)
    w[4050:4100] = rng.uniform(-0.3, 0.3, 50)  # nonzero biases exercise more branches
    f = rng.standard_normal((3, N, N, N))
    gM = rng.standard_normal((N, N, N))
    g = nn.mlp_backward(gM, f, w, 2.0)
    fun = lambda ff: float(np.sum(gM * nn.mlp_forward(ff, w, 2.0)[0]))
    for _ in range(5):
        v = rng.standard_normal(f.shape)
        eps = 1e-6
        fd = (fun(f + eps * v) - fun(f - eps * v)) / (2 * eps)
        assert rdot(g, v) == pytest.approx(fd, rel=1e-6)


def test_two_net_special_values_and_closed_form():
    assert nn.logistic(0.0, 3.0) == 0.5 and nn.logistic(0.0, 1.0) == 0.5
    assert nn.elu(-50.0) == pytest.approx(-1.0) and nn.elu(2.0) == 2.0
    assert nn.elu_grad(-1e-12) == pytest.approx(1.0) and nn.elu_grad(3.0) == 1.0
    # NNp: logit = relu(f0(x)) - 0.5; NNm: hidden 0 = elu(f1(x)), second layer
    # passes it on, output = elu(elu(f1)) + 2  =>  closed form
    N = 4
    wp = np.zeros(synth.N_WEIGHTS)
    W1, _, W2, _, w3, _ = nn.unpack(wp)
    W1[0, 13] = 1.0
    W2[0, 0] = 1.0
    w3[0] = 1.0
    wp[-1] = -0.5
    wm = np.zeros(synth.N_MASS_WEIGHTS)
    V1, _, V2, _, v3, _ = nn.unpack_mass(wm)
    V1[0, 1] = 1.0
    V2[0, 0] = 1.0
    v3[0] = 1.0
    wm[-1] = 2.0
    f = np.random.default_rng(9).standard_normal((3, N, N, N))
    a = 2.0
    M = nn.two_net_forward(f, wp, wm, 1e12, a)
    p = 1.0 / (1.0 + np.exp(-a * (np.maximum(f[0], 0.0) - 0.5)))
    m = nn.elu(nn.elu(f[1])) + 2.0
    assert np.allclose(M, 1e12 * p * m, rtol=1e-14)


def test_two_net_backward_by_finite_differences():
    rng = np.random.default_rng(10)
    N = 4
    wp = synth.xavier_weights(1).astype(np.float64)
    wm = synth.mass_net_weights(3).astype(np.float64)
    wm[:60] *= 12.0  # larger first-layer weights exercise both ELU branches
    f = rng.standard_normal((3, N, N, N))
    gM = rng.standard_normal((N, N, N))
    g = nn.two_net_backward(gM, f, wp, wm, 2.0, 1.5)
    fun = lambda ff: float(np.sum(gM * nn.two_net_forward(ff, wp, wm, 2.0, 1.5)))
    for _ in range(5):
        v = rng.standard_normal(f.shape)
        eps = 1e-6
        fd = (fun(f + eps * v) - fun(f - eps * v)) / (2 * eps)
        assert rdot(g, v) == pytest.approx(fd, rel=1e-6)


def test_two_net_loss_gradient_by_finite_differences():
    N = 8
    pms = pm.PMSetup(N=N, L=50.0, nsteps=2)
    ls = loss.LossSetup(head="two_net")
    # M0 = 1e11 (second stage of Sec. 5.3) dominates the ringing of the sub-cell
    # R_M smoothing of the spiky logistic-head mass field at this coarse mesh
    an = loss.Anneal(R_sm=3.0, M0=1e11, a=2.0)
    w = np.concatenate([synth.xavier_weights(1), synth.mass_net_weights(3)])
    data = loss.synthetic_data(synth.white_noise(N, 2), synth.scatter_noise(N, 2), w, pms, ls, a=2.0)
    s = 0.5 * pm.linear_field(synth.white_noise(N, 0), pms)
    parts, g = loss.loss_and_grad(s, data, w, pms, ls, an)
    assert np.isfinite(parts["loss"])
    f = lambda ss: loss.loss(ss, data, w, pms, ls, an)["loss"]
    rng = np.random.default_rng(11)
    for _ in range(3):
        v = pm.rfft3(rng.standard_normal((N, N, N))) * np.sqrt(pm.power_half(pms) / N**3)
        v[0, 0, 0] = 0
        eps = 2e-7  # below the nearest CIC cell-face crossing along these directions
        fd = (f(s + eps * v) - f(s - eps * v)) / (2 * eps)
        assert rdot(g, v) == pytest.approx(fd, rel=2e-5)


# ----------------------------------------------------------------------------- loss

def test_prior_equals_full_grid_sum_and_its_gradient():
    # for a Hermitian field the weighted half-array sum is the full-grid sum
    setup = pm.PMSetup(N=8, L=100.0, nsteps=1)
    s = pm.linear_field(synth.white_noise(8, 4), setup)
    P = pm.power_half(setup)
    full = np.fft.fftn(pm.irfft3(s))
    kphys = np.sqrt(sum(k**2 for k in np.meshgrid(*(2 * np.pi * np.fft.fftfreq(8, d=100.0 / 8),) * 3, indexing="ij")))
    from oracle import cosmo
    Pfull = cosmo.P_lin_array(kphys) * 8**6 / 100.0**3
    m = kphys > 0
    brute = 0.5 * np.sum(np.abs(full[m]) ** 2 / Pfull[m])
    assert loss.prior(s, P) == pytest.approx(brute, rel=1e-10)
    g = loss.prior_grad(s, P)
    w = pm.half_weights(8)
    assert np.allclose(g[P > 0], (w * s)[P > 0] / P[P > 0], rtol=0, atol=0)
    assert g[0, 0, 0] == 0


def test_residual_without_smoothing_is_closed_form():
    N = 4
    rng = np.random.default_rng(5)
    M = np.exp(rng.uniform(20, 30, (N, N, N)))
    Dm = np.exp(rng.uniform(20, 30, (N, N, N)))
    pms = pm.PMSetup(N=N, L=4.0, nsteps=1)
    ls = loss.LossSetup(R_M=0.0, sigma_N2=0.25, mu_N=0.1, f_eff=0.7)
    an = loss.Anneal(R_sm=0.0, M0=1e10)
    L, _ = loss.residual_terms(M, Dm, pms, ls, an)
    r = 0.1 + np.log(M + 1e10) - np.log(Dm + 1e10)
    assert L == pytest.approx(0.7 * np.sum((r / (2 * 0.5)) ** 2), rel=1e-13)


def test_loss_reduces_to_prior_when_noise_is_huge():
    N = 8
    pms = pm.PMSetup(N=N, L=100.0, nsteps=1)
    ls = loss.LossSetup(sigma_N2=1e30)
    an = loss.Anneal(R_sm=4.0, M0=1e8)
    s = pm.linear_field(synth.white_noise(N, 0), pms)
    w = synth.xavier_weights(1)
    data = np.full((N, N, N), 1e12)
    parts, g = loss.loss_and_grad(s, data, w, pms, ls, an)
    P = pm.power_half(pms)
    assert parts["loss"] == pytest.approx(loss.prior(s, P), rel=1e-12)
    assert np.allclose(g, loss.prior_grad(s, P), rtol=1e-9, atol=1e-20)


@pytest.mark.parametrize("R_sm,lpt_order", [(0.0, 1), (4.0, 1), (4.0, 2)])
def test_full_gradient_by_finite_differences(R_sm, lpt_order):
    N = 8
    pms = pm.PMSetup(N=N, L=100.0, nsteps=2, lpt_order=lpt_order)
    ls = loss.LossSetup()
    an = loss.Anneal(R_sm=R_sm, M0=1e8)
    w = synth.xavier_weights(1)
    data = loss.synthetic_data(synth.white_noise(N, 2), synth.scatter_noise(N, 2), w, pms, ls)
    s = 0.5 * pm.linear_field(synth.white_noise(N, 0), pms)
    parts, g = loss.loss_and_grad(s, data, w, pms, ls, an)
    f = lambda ss: loss.loss(ss, data, w, pms, ls, an)["loss"]
    rng = np.random.default_rng(7)
    for _ in range(3):
        v = pm.rfft3(rng.standard_normal((N, N, N))) * np.sqrt(pm.power_half(pms) / N**3)
        v[0, 0, 0] = 0
        eps = 1e-6
        fd = (f(s + eps * v) - f(s - eps * v)) / (2 * eps)
        assert rdot(g, v) == pytest.approx(fd, rel=1e-5)


# ----------------------------------------------------------------------------- L-BFGS

def _quadratic(n, seed):
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(np.linspace(1.0, 20.0, n)) @ Q.T
    b = rng.standard_normal(n)
    return A, b, (lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b))


def test_lbfgs_minimises_a_quadratic():
    A, b, fun = _quadratic(20, 1)
    st = lbfgs.LBFGSState(x=np.zeros(20))
    for _ in range(60):
        status, _, _ = lbfgs.step(fun, st, m=10, tol=0.0)
        assert status == "ok"
        if np.linalg.norm(st.g) < 1e-7:  # Armijo on f resolves |g| to ~1e-9 in fp64
            break
    assert np.allclose(st.x, np.linalg.solve(A, b), atol=1e-7)


def test_two_loop_with_diagonal_h0_equals_dense_bfgs_matrix():
    rng = np.random.default_rng(4)
    n, k = 10, 4
    S = [rng.standard_normal(n) for _ in range(k)]
    M = rng.standard_normal((n, n)); M = M @ M.T + n * np.eye(n)
    Y = [M @ s for s in S]
    g = rng.standard_normal(n)
    D = rng.uniform(0.5, 3.0, n)
    # initial matrix gamma D, gamma from the newest pair (Nocedal & Wright Sec. 7.2)
    H = (S[-1] @ Y[-1]) / (Y[-1] @ (D * Y[-1])) * np.diag(D)
    for s, y in zip(S, Y):
        rho = 1.0 / (y @ s)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    assert np.allclose(lbfgs.two_loop(g, S, Y, D), -H @ g, rtol=1e-12, atol=1e-12)


def test_diagonal_h0_scaling_is_exact_on_a_scaled_diagonal_quadratic():
    # f = 1/2 x^T A x with A = (c D)^-1: after one pair, gamma D = A^-1 exactly,
    # so the second direction is the Newton step and lands on x = 0
    rng = np.random.default_rng(6)
    n = 12
    D = rng.uniform(0.2, 5.0, n)
    A = 1.0 / (3.7 * D)
    fun = lambda x: (0.5 * float(x @ (A * x)), A * x)
    st = lbfgs.LBFGSState(x=rng.standard_normal(n))
    lbfgs.step(fun, st, H0=D, tol=0.0)
    status, _, _ = lbfgs.step(fun, st, H0=D, tol=0.0)
    assert status == "ok"
    assert np.max(np.abs(st.x)) < 1e-12


def test_prior_preconditioned_first_step_solves_the_prior():
    # with the residual switched off the loss is the Gaussian prior; the first
    # step -H0 g with H0 = diag(P~/w) lands exactly on its minimum s = 0
    N = 8
    pms = pm.PMSetup(N=N, L=100.0, nsteps=1)
    P = pm.power_half(pms)
    s0 = pm.linear_field(synth.white_noise(N, 5), pms)
    fun = lambda x: (loss.prior(x, P), loss.prior_grad(x, P))
    st = lbfgs.LBFGSState(x=s0.copy())
    status, _, _ = lbfgs.step(fun, st, H0=loss.prior_inverse_hessian(pms))
    assert status == "ok"
    assert np.max(np.abs(st.x)) < 1e-9 * np.max(np.abs(s0))


def test_two_loop_equals_dense_bfgs_matrix():
    # with every pair kept, the two-loop product is the BFGS inverse Hessian
    # built from H0 = gamma I by the rank-two update, applied to g
    rng = np.random.default_rng(2)
    n, k = 12, 5
    S = [rng.standard_normal(n) for _ in range(k)]
    M = rng.standard_normal((n, n)); M = M @ M.T + n * np.eye(n)
    Y = [M @ s for s in S]  # s.y > 0
    g = rng.standard_normal(n)
    gamma = S[-1] @ Y[-1] / (Y[-1] @ Y[-1])
    H = gamma * np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / (y @ s)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    assert np.allclose(lbfgs.two_loop(g, S, Y), -H @ g, rtol=1e-12, atol=1e-12)


def test_sampled_network_equals_full_network_at_those_voxels():
    # the sampled forms used at full mesh size agree with the whole-mesh forms
    N = 8
    f = np.stack([synth.gaussian_vector((N, N, N), seed=s) for s in (71, 72, 73)]).astype(np.float64)
    w = synth.xavier_weights(1).astype(np.float64)
    vox = synth.sample_voxels(N, 40, seed=74)
    M_full, _ = nn.mlp_forward(f, w, 1e12)
    assert np.allclose(nn.mlp_at(f, vox, w, 1e12), M_full[vox[:, 0], vox[:, 1], vox[:, 2]], rtol=1e-13)
    # sparse mass gradient (duplicates accumulate, as in the dense adjoint)
    gM = np.zeros((N, N, N))
    vals = synth.gaussian_vector(vox.shape[0], seed=75).astype(np.float64)
    np.add.at(gM, (vox[:, 0], vox[:, 1], vox[:, 2]), vals)
    dense = nn.mlp_backward(gM, f, w, 1e12)
    assert np.allclose(nn.mlp_backward_at(vals, vox, f, w, 1e12), dense, rtol=1e-12, atol=1e-12 * np.abs(dense).max())


PAPER_MIX = (1, 0, 0, 0, 1, 0, 0, 1, -1)  # delta_0, delta_R1, delta_R1 - delta_R2 (Sec. 2.2)


def test_paper_feature_set_by_explicit_smoothing():
    # the mixed features with R_feat = (0, R1, R2): the unsmoothed density, its
    # R1 smoothing, and the difference of the R1 and R2 smoothings, each formed here
    # straight from a Gaussian filter written out in this test
    N, L, R1, R2 = 16, 50.0, 3.0, 6.0
    setup = pm.PMSetup(N=N, L=L, nsteps=1)
    ls = loss.LossSetup(R_feat=(0.0, R1, R2), feat_mix=PAPER_MIX)
    delta = synth.gaussian_vector((N, N, N), seed=9).astype(np.float64)
    kf = 2 * np.pi * np.fft.fftfreq(N) * N / L   # h/Mpc per mode along each axis
    kz = 2 * np.pi * np.arange(N // 2 + 1) / L
    k2 = kf[:, None, None] ** 2 + kf[None, :, None] ** 2 + kz[None, None, :] ** 2
    D = np.fft.rfftn(delta)
    sm = lambda R: np.fft.irfftn(D * np.exp(-0.5 * k2 * R * R), s=(N, N, N), axes=(0, 1, 2))
    f = loss.features(delta, setup, ls)
    assert np.allclose(f[0], delta, atol=1e-12)
    assert np.allclose(f[1], sm(R1), atol=1e-12)
    assert np.allclose(f[2], sm(R1) - sm(R2), atol=1e-12)


def test_mixed_features_adjoint_by_dot_product():
    N, L = 16, 50.0
    setup = pm.PMSetup(N=N, L=L, nsteps=1)
    ls = loss.LossSetup(R_feat=(0.0, 3.0, 6.0), feat_mix=(0.5, -1.0, 2.0, 0.0, 1.5, 0.25, 1.0, 1.0, -3.0))
    x = synth.gaussian_vector((N, N, N), seed=10).astype(np.float64)
    y = synth.gaussian_vector((3, N, N, N), seed=11).astype(np.float64)
    lhs = float(np.sum(loss.features(x, setup, ls) * y))
    rhs = float(np.sum(x * loss.features_T(y, setup, ls)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
