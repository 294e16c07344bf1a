"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

from paper_1805_02247_gb300 import build, pmrecon, synth


def lib():
    build.build()
    return pmrecon.load()


def rel_l2(got, want) -> float:
    got = np.asarray(got, dtype=np.complex128 if np.iscomplexobj(got) else np.float64)
    want = np.asarray(want)
    return float(np.linalg.norm((got - want).ravel()) / max(np.linalg.norm(np.asarray(want).ravel()), 1e-300))


def to_dev(a, dtype=None) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    if np.iscomplexobj(a):
        return torch.from_numpy(a.astype(np.complex64)).cuda()
    return torch.from_numpy(a.astype(dtype or np.float32)).cuda()


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()


def context(N=32, L=100.0, nsteps=3, seed_w=1, **kw):
    lib()
    cfg = pmrecon.default_config(N=N, L=L, nsteps=nsteps, **kw)
    w = synth.two_net_weights(seed_w) if kw.get("head", 0) == 1 else synth.xavier_weights(seed_w)
    w = torch.from_numpy(w).cuda()
    return pmrecon.Context(cfg, w), cfg


def f32(a):
    """Round an input to float32 so both sides see identical values."""
    if np.iscomplexobj(a):
        return a.astype(np.complex64).astype(np.complex128)
    return np.asarray(a, np.float32).astype(np.float64)
