"""The allocation-free paint entry point, checked against the regular one.

pmr_paint_noalloc() is for callers that cannot call cudaMalloc: code running
while a CUDA graph is being captured, framework plug-ins whose host owns all
device memory, and loops that must not let an allocation synchronise the
device. It takes its scratch from one fixed device array, so this file also
checks that a second call, which finds the first call's leftovers in that
array, still paints exactly what the context-based pmr_paint() paints.

Collected last (file name) so that a stop-at-first-failure run has already run
every other test; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import pm as opm
from paper_1805_02247_gb300 import pmrecon, synth

from gpu_util import context, f32, lib, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5


def _noalloc(lib, N, x, mass=None):
    rho = torch.empty(N, N, N, device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.pmr_paint_noalloc(N, x.data_ptr(), x.shape[1], None if mass is None else mass.data_ptr(),
                               rho.data_ptr(), ctypes.c_void_p(stream))
    assert rc == pmrecon.PMR_OK, lib.pmr_last_error(None).decode()
    return rho


def test_noalloc_paint_matches_pmr_paint_on_two_calls_in_a_row():
    N = 32
    ctx, _ = context(N=N)
    lib_ = lib()
    # call 1: unit masses, many particles; call 2: fewer particles with masses,
    # so stale sort data from call 1 would show up if anything were not cleared
    x1 = to_dev(synth.uniform_positions(N, 30000, seed=41, lo=-N, hi=2 * N))
    x2 = to_dev(synth.uniform_positions(N, 5000, seed=42, lo=0.0, hi=N))
    m2 = to_dev(synth.gaussian_vector(5000, seed=43))
    for x, m in ((x1, None), (x2, m2)):
        got = to_np(_noalloc(lib_, N, x, m))
        want = to_np(ctx.paint(x, m))
        assert rel_l2(got, want) <= FIELD_TOL
        assert np.array_equal(got, want)  # same kernels, same order: identical bits


def test_noalloc_paint_at_its_size_limit():
    # N = 64 and np = N^3 = 2^18 with masses fill every region of the fixed
    # array; the result equals pmr_paint's bits and the oracle's CIC paint
    N, np_ = 64, 1 << 18
    ctx, _ = context(N=N)
    lib_ = lib()
    xh = synth.uniform_positions(N, np_, seed=44, lo=-N, hi=2 * N)
    mh = synth.gaussian_vector(np_, seed=45)
    x, m = to_dev(xh), to_dev(mh)
    got = to_np(_noalloc(lib_, N, x, m))
    assert np.array_equal(got, to_np(ctx.paint(x, m)))
    assert rel_l2(got, opm.paint(f32(xh), N, mass=f32(mh), f32_wrap=True)) <= FIELD_TOL
    ctx.close()


def test_noalloc_paint_rejects_sizes_beyond_its_limit():
    lib_ = lib()
    x = torch.zeros(3, 8, device="cuda")
    rho = torch.empty(65, 65, 65, device="cuda")
    rc = lib_.pmr_paint_noalloc(65, x.data_ptr(), 8, None, rho.data_ptr(), None)
    assert rc == -1 and b"N must be" in lib_.pmr_last_error(None)
    # below the smallest mesh the paint's tiles handle
    rc = lib_.pmr_paint_noalloc(7, x.data_ptr(), 8, None, rho.data_ptr(), None)
    assert rc == -1 and b"N must be" in lib_.pmr_last_error(None)
    # more particles than cells (pmr_paint's bound)
    rc = lib_.pmr_paint_noalloc(8, x.data_ptr(), 8 ** 3 + 1, None, rho.data_ptr(), None)
    assert rc == -1 and b"np" in lib_.pmr_last_error(None)
    rc = lib_.pmr_paint_noalloc(64, x.data_ptr(), (1 << 18) + 1, None, rho.data_ptr(), None)
    assert rc == -1 and b"np" in lib_.pmr_last_error(None)
