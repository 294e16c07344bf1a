"""GPU parity of the single steps of the path (C ABI) against the FP64 oracle.

Tolerances: bit-exact for cell keys, sort order and segment offsets; relative
L2 <= 1e-5 for float32 fields; 1e-4 for gradients.
"""
import numpy as np
import pytest
import torch

from oracle import loss as oloss
from oracle import nn as onn
from oracle import pm as opm
from paper_1805_02247_gb300 import synth

from gpu_util import context, f32, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.mark.parametrize("N,np_,lo,hi", [(8, 512, -8.0, 16.0), (16, 3000, -3.0, 19.0), (32, 32**3, 0.0, 32.0),
                                         (24, 100, 0.0, 24.0)])
def test_cell_sort_bit_exact(N, np_, lo, hi):
    ctx, _ = context(N=N)
    x = synth.uniform_positions(N, np_, seed=N + np_, lo=lo, hi=hi)
    if np_ >= 16:
        e = synth.edge_positions(N)
        x[:, : e.shape[1]] = e
    keys, perm, start = ctx.cell_sort(to_dev(x))
    want_keys = opm.cell_keys(x, N)
    want_perm, want_start = opm.sort_by_cell(want_keys, N)
    assert np.array_equal(to_np(keys).view(np.uint32), want_keys)
    assert np.array_equal(to_np(perm).view(np.uint32), want_perm)
    assert np.array_equal(to_np(start).view(np.uint32), want_start)


def test_cell_sort_crowded_cells():
    # many particles in few cells exercises the long-segment path of the stable sort
    N = 8
    x = synth.uniform_positions(N, 400, seed=3, lo=2.0, hi=2.9)
    ctx, _ = context(N=N)
    keys, perm, start = ctx.cell_sort(to_dev(x))
    want_perm, want_start = opm.sort_by_cell(opm.cell_keys(x, N), N)
    assert np.array_equal(to_np(perm).view(np.uint32), want_perm)
    assert np.array_equal(to_np(start).view(np.uint32), want_start)


def test_cell_sort_overfull_block():
    # more particles in one block's 512 cells than its shared-memory stage holds
    # (the global-memory path), with long and short segments in that block
    N = 24
    rng = np.random.default_rng(11)
    dense = np.stack([rng.uniform(0.0, 0.9, 7000), rng.uniform(0.0, 2.0, 7000), rng.uniform(0.0, 24.0, 7000)])
    sparse = np.stack([rng.uniform(0.0, 0.9, 600), rng.uniform(2.0, 21.0, 600), rng.uniform(0.0, 24.0, 600)])
    rest = synth.uniform_positions(N, N**3 - 7600, seed=12, lo=0.0, hi=float(N))
    x = np.concatenate([dense, sparse, rest], axis=1).astype(np.float32)
    x = x[:, rng.permutation(x.shape[1])]
    ctx, _ = context(N=N)
    keys, perm, start = ctx.cell_sort(to_dev(x))
    want_perm, want_start = opm.sort_by_cell(opm.cell_keys(x, N), N)
    assert np.array_equal(to_np(perm).view(np.uint32), want_perm)
    assert np.array_equal(to_np(start).view(np.uint32), want_start)
    rho = to_np(ctx.paint(to_dev(x)))
    assert rel_l2(rho, opm.paint(f32(x), N, f32_wrap=True)) <= FIELD_TOL


def test_cell_sort_segment_length_classes():
    # cells of exactly the lengths where the segment sort changes method (8 | 9: one
    # thread / one warp in registers, 32 | 33: one warp in shared memory, 512 | 513:
    # the whole block), in a block of 512 cells staged in shared memory (keys 0-511)
    # and in one past the stage's capacity of 5120 (keys 1024-1535, the global-memory path)
    N = 32
    rng = np.random.default_rng(5)
    staged = [1, 2, 8, 9, 31, 32, 33, 100, 512, 513, 1200]
    overfull = [2, 8, 9, 32, 33, 511, 512, 513, 4100]
    parts = []
    for k0, counts in ((0, staged), (1024, overfull)):
        keys = k0 + rng.choice(512, size=len(counts), replace=False)
        for key, k in zip(keys, counts):
            corner = np.array([[key // (N * N)], [(key // N) % N], [key % N]], dtype=np.float64)
            parts.append(corner + rng.uniform(0.02, 0.98, size=(3, k)))
    parts.append(np.stack([rng.uniform(4.0, 32.0, 5000), rng.uniform(0.0, 32.0, 5000),
                           rng.uniform(0.0, 32.0, 5000)]))
    x = np.concatenate(parts, axis=1).astype(np.float32)
    x = x[:, rng.permutation(x.shape[1])]
    ctx, _ = context(N=N)
    keys, perm, start = ctx.cell_sort(to_dev(x))
    want_perm, want_start = opm.sort_by_cell(opm.cell_keys(x, N), N)
    counts = np.diff(want_start.astype(np.int64))
    assert all(k in counts[:512] for k in staged) and all(k in counts[1024:1536] for k in overfull)
    assert counts[:512].sum() <= 5120 < counts[1024:1536].sum()
    assert np.array_equal(to_np(perm).view(np.uint32), want_perm)
    assert np.array_equal(to_np(start).view(np.uint32), want_start)
    rho = to_np(ctx.paint(to_dev(x)))
    assert rel_l2(rho, opm.paint(f32(x), N, f32_wrap=True)) <= FIELD_TOL


@pytest.mark.parametrize("N", [16, 18])
def test_cell_sort_many_crowded_cells(N):
    # several cells of 33 to about 1000 particles inside one staged block (the block-wide
    # sort of long segments in shared memory), short segments beside them, and
    # for N = 18 a last block of fewer than 512 cells
    rng = np.random.default_rng(21 + N)
    centres = rng.integers(0, 2, size=(20, 3)) + np.array([0, 0, 0])
    counts = rng.integers(33, 300, size=20)
    parts = [np.stack([np.full(k, cx + 0.5), np.full(k, cy + 0.5), np.full(k, cz * 3 + 0.25)])
             + rng.uniform(-0.45, 0.45, size=(3, k)) * np.array([[1.0], [1.0], [0.2]])
             for (cx, cy, cz), k in zip(centres, counts)]
    dense = np.concatenate(parts, axis=1)
    rest = synth.uniform_positions(N, N**3 - dense.shape[1], seed=22 + N, lo=0.0, hi=float(N))
    x = np.concatenate([dense, rest], axis=1).astype(np.float32)
    x = x[:, rng.permutation(x.shape[1])]
    ctx, _ = context(N=N)
    keys, perm, start = ctx.cell_sort(to_dev(x))
    want_perm, want_start = opm.sort_by_cell(opm.cell_keys(x, N), N)
    assert np.array_equal(to_np(perm).view(np.uint32), want_perm)
    assert np.array_equal(to_np(start).view(np.uint32), want_start)
    assert np.diff(want_start).max() > 32
    rho = to_np(ctx.paint(to_dev(x)))
    assert rel_l2(rho, opm.paint(f32(x), N, f32_wrap=True)) <= FIELD_TOL


@pytest.mark.parametrize("N,np_", [(16, 4096), (32, 20000), (16, 0), (24, 9000), (48, 60000), (8, 100)])
def test_paint_parity_and_mass_conservation(N, np_):
    ctx, _ = context(N=N)
    x = synth.uniform_positions(N, max(np_, 1), seed=5, lo=-N, hi=2 * N)[:, :np_]
    rho = to_np(ctx.paint(to_dev(x)))
    if np_ == 0:
        assert not rho.any()
        return
    want = opm.paint(f32(x), N, f32_wrap=True)
    assert rel_l2(rho, want) <= FIELD_TOL
    assert abs(rho.sum(dtype=np.float64) - np_) <= 1e-6 * np_
    m = synth.gaussian_vector(np_, seed=6)
    rho_m = to_np(ctx.paint(to_dev(x), to_dev(m)))
    assert rel_l2(rho_m, opm.paint(f32(x), N, mass=f32(m), f32_wrap=True)) <= FIELD_TOL
    # deterministic: same bits twice
    assert np.array_equal(rho, to_np(ctx.paint(to_dev(x))))


def test_readout_and_grad_parity():
    N = 16
    ctx, _ = context(N=N)
    x = synth.uniform_positions(N, 5000, seed=7, lo=-N, hi=2 * N)
    g = synth.gaussian_vector((N, N, N), seed=8)
    r = to_np(ctx.readout(to_dev(g), to_dev(x)))
    assert rel_l2(r, opm.readout(f32(g), f32(x), f32_wrap=True)) <= FIELD_TOL
    rg = to_np(ctx.readout_grad(to_dev(g), to_dev(x)))
    assert rel_l2(rg, opm.readout_grad(f32(g), f32(x), f32_wrap=True)) <= FIELD_TOL


@pytest.mark.parametrize("N", [8, 16, 24, 32, 48, 64, 96, 128, 192, 384])
def test_rfft_irfft_parity(N):
    # 64, 128, 192 (and 256, 512) take the register four-step column passes
    ctx, _ = context(N=N)
    f = synth.gaussian_vector((N, N, N), seed=N)
    k = to_np(ctx.rfft(to_dev(f)))
    assert rel_l2(k, np.fft.rfftn(f32(f))) <= FIELD_TOL
    # inverse of an arbitrary (non-Hermitian) half array: imaginary parts of
    # self-conjugate entries are ignored, as by the oracle's irfftn
    u = synth.gaussian_vector((N, N, N // 2 + 1), seed=N + 1) + 1j * synth.gaussian_vector((N, N, N // 2 + 1), seed=N + 2)
    got = to_np(ctx.irfft(to_dev(u)))
    assert rel_l2(got, opm.irfft3(f32(u))) <= FIELD_TOL


def test_fft_and_force_parity_at_the_largest_mesh():
    # N = 512, the largest mesh a context accepts, has register plans of its own
    # (512-point columns as 16 x 32, 256-point rows as 16 x 16)
    N = 512
    ctx, cfg = context(N=N, L=800.0, nsteps=1)
    f = synth.gaussian_vector((N, N, N), seed=41)
    k = to_np(ctx.rfft(to_dev(f)))
    assert rel_l2(k, np.fft.rfftn(f32(f))) <= FIELD_TOL
    assert rel_l2(to_np(ctx.irfft(to_dev(f32(k)))), opm.irfft3(f32(k))) <= FIELD_TOL
    del f, k
    d = synth.lognormal_density(N, seed=42)
    assert rel_l2(to_np(ctx.force(to_dev(d))), opm.force(f32(d), cfg.omega_m)) <= FIELD_TOL
    ctx.close()


@pytest.mark.parametrize("N", [32, 64, 128, 192])
def test_force_and_smooth_parity(N):
    ctx, cfg = context(N=N, L=100.0)
    d = synth.gaussian_vector((N, N, N), seed=11)
    F = to_np(ctx.force(to_dev(d)))
    assert rel_l2(F, opm.force(f32(d), cfg.omega_m)) <= FIELD_TOL
    for R in (0.0, 1.0, 4.0):
        sm = to_np(ctx.smooth(to_dev(d), R))
        assert rel_l2(sm, opm.smooth(f32(d), R / (100.0 / N))) <= FIELD_TOL


@pytest.mark.parametrize("N,L", [(32, 100.0), (24, 400.0)])
def test_linear_field_and_za_parity(N, L):
    ctx, cfg = context(N=N, L=L)
    setup = opm.PMSetup(N=N, L=L, nsteps=3)
    white = synth.white_noise(N, 0)
    s = to_np(ctx.linear_field(to_dev(white), 1.0))
    want = opm.linear_field(f32(white), setup)
    assert rel_l2(s, want) <= FIELD_TOL
    s_in = f32(want)
    disp, mom = ctx.za_ics(to_dev(s_in))
    x_want, p_want = opm.za_ics(s_in, setup)
    assert rel_l2(to_np(disp), x_want - opm.lattice(N)) <= FIELD_TOL
    assert rel_l2(to_np(mom), p_want) <= FIELD_TOL


def test_growth_factors_match_oracle():
    from oracle import cosmo
    from paper_1805_02247_gb300 import pmrecon
    _, cfg = context(N=8)
    for a in (0.1, 0.35, 0.7, 1.0):
        D, Gp, Gf = pmrecon.growth(cfg, a)
        assert D == pytest.approx(cosmo.D(a), rel=1e-11)
        assert Gp == pytest.approx(cosmo.Gp(a), rel=1e-10)
        assert Gf == pytest.approx(cosmo.Gf(a), rel=1e-11)


def test_lbfgs_direction_parity():
    from oracle import lbfgs as olb
    ctx, _ = context(N=16)
    rng = np.random.default_rng(3)
    n, k = 1000, 6
    S = [rng.standard_normal(n) for _ in range(k)]
    Y = [s + 0.3 * rng.standard_normal(n) for s in S]
    g = rng.standard_normal(n)
    d = ctx.lbfgs_direction(torch.tensor(g, device="cuda"), torch.tensor(np.stack(S), device="cuda"),
                            torch.tensor(np.stack(Y), device="cuda"))
    assert rel_l2(to_np(d), olb.two_loop(g, S, Y)) <= 1e-12


@pytest.mark.parametrize("N,L", [(32, 100.0), (24, 60.0)])
def test_power_spectra_parity(N, L):
    from oracle import twopt
    ctx, _ = context(N=N, L=L)
    a = synth.gaussian_vector((N, N, N), seed=61)
    b = (0.5 * a + synth.gaussian_vector((N, N, N), seed=62)).astype(np.float32)
    got = [t.numpy() for t in ctx.power_spectra(to_dev(a), to_dev(b))]
    want = twopt.power_spectra(f32(a), f32(b), L)
    assert np.array_equal(got[0], want[0])  # shell membership is an integer decision
    for g, w in zip(got[1:], want[1:]):
        assert rel_l2(g, w) <= FIELD_TOL
    # deterministic: identical bits on a second call
    again = [t.numpy() for t in ctx.power_spectra(to_dev(a), to_dev(b))]
    assert all(np.array_equal(x, y) for x, y in zip(got, again))


@pytest.mark.parametrize("N,L", [(32, 100.0), (24, 400.0), (192, 400.0)])
def test_lpt2_ics_and_adjoint_parity(N, L):
    # second-order LPT initial conditions (Sec. 3) and their adjoint
    ctx, _ = context(N=N, L=L, lpt_order=2)
    setup = opm.PMSetup(N=N, L=L, nsteps=3, lpt_order=2)
    s = f32(opm.linear_field(f32(synth.white_noise(N, 0)), setup))
    disp, mom = ctx.lpt_ics(to_dev(s))
    x_want, p_want = opm.lpt_ics(s, setup)
    assert rel_l2(to_np(disp), x_want - opm.lattice(N)) <= FIELD_TOL
    assert rel_l2(to_np(mom), p_want) <= FIELD_TOL
    lx = f32(synth.gaussian_vector((3, N ** 3), seed=31))
    lp = f32(synth.gaussian_vector((3, N ** 3), seed=32))
    g = to_np(ctx.lpt_ics_adjoint(to_dev(s), to_dev(lx), to_dev(lp)))
    assert rel_l2(g, opm.lpt_ics_T(lx, lp, s, setup)) <= GRAD_TOL


def test_lpt_order_one_is_zeldovich():
    N = 16
    ctx, _ = context(N=N, L=100.0, lpt_order=1)
    s = f32(opm.linear_field(f32(synth.white_noise(N, 0)), opm.PMSetup(N=N, L=100.0, nsteps=1)))
    d1, p1 = ctx.lpt_ics(to_dev(s))
    d0, p0 = ctx.za_ics(to_dev(s))
    assert torch.equal(d1, d0) and torch.equal(p1, p0)


@pytest.mark.parametrize("N,L", [(32, 100.0), (64, 400.0)])
def test_two_point_statistics_parity(N, L):
    # r_c, stochasticity s = P_hh (1 - r_c^2) and TF = sqrt(P_mm / P_hh) of Sec. 4.3,
    # formed on the device, against the oracle on the same meshes: data = signal +
    # noise in quadrature with it (s = the noise power, r_c strictly inside (0, 1))
    from oracle import twopt
    ctx, _ = context(N=N, L=L)
    a = synth.gaussian_vector((N, N, N), seed=63)
    kx = np.fft.fftfreq(N, d=1.0 / N)[:, None, None] * np.ones((1, N, N // 2 + 1))
    kx[N // 2] = 0.0
    n = np.fft.irfftn(0.3j * kx * np.fft.rfftn(a.astype(np.float64)), s=(N, N, N), axes=(0, 1, 2))
    h = (a + n).astype(np.float32)
    got = ctx.two_point(to_dev(h), to_dev(a))
    counts, P_hh, P_mm, P_hm = twopt.power_spectra(f32(h), f32(a), L)
    rc, s, tf = twopt.statistics(P_hh, P_mm, P_hm)
    assert np.array_equal(got["counts"].numpy(), counts)
    for key, want in (("P_hh", P_hh), ("P_mm", P_mm), ("P_hm", P_hm), ("r_c", rc), ("s", s), ("TF", tf)):
        assert rel_l2(got[key].numpy(), want) <= FIELD_TOL, key
    _, P_nn, _, _ = twopt.power_spectra(f32(h) - f32(a), f32(h) - f32(a), L)
    assert rel_l2(got["s"].numpy(), P_nn) <= 1e-4  # the stochasticity is the noise power


def test_network_and_adjoint_on_ragged_z_lines():
    # 192 = 128 + 64: every z-line of the tensor-core forward is one full tile and
    # one ragged tile (64 of its 128 rows); sampled voxels, the rows on both sides
    # of the tile boundary and the line's last rows included, and the adjoint there
    N, L = 192, 300.0
    ctx, _ = context(N=N, L=L, nsteps=1)
    setup = opm.PMSetup(N=N, L=L, nsteps=1)
    ls = oloss.LossSetup()
    w = synth.xavier_weights(1)
    d = synth.lognormal_density(N, seed=121)
    M = to_np(ctx.nn_halo_map(to_dev(d)))
    feats = oloss.features(f32(d), setup, ls)
    edge = np.array([[x, y, z] for x in (0, 1, N - 1) for y in (0, 5, N - 1)
                     for z in (0, 1, 126, 127, 128, 129, 190, 191)], np.int64)
    vox = np.concatenate([synth.sample_voxels(N, 2048, seed=122), edge])
    assert rel_l2(M[vox[:, 0], vox[:, 1], vox[:, 2]], onn.mlp_at(feats, vox, w, ls.M_scale)) <= FIELD_TOL
    vals = f32(synth.gaussian_vector(vox.shape[0], seed=123))
    gM = np.zeros((N, N, N), np.float32)
    np.add.at(gM, (vox[:, 0], vox[:, 1], vox[:, 2]), vals.astype(np.float32))
    got = to_np(ctx.nn_halo_map_adjoint(to_dev(d), to_dev(gM)))
    want = oloss.features_T(onn.mlp_backward_at(vals, vox, feats, w, ls.M_scale), setup, ls)
    assert rel_l2(got, want) <= GRAD_TOL
    ctx.close()
