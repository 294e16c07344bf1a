"""Thin Python binding of libpmrecon.so (the C ABI in include/pmrecon.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. PyTorch provides device memory and the stream. There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpmrecon.so")

PMR_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENAN", -5: "ELINESEARCH", -6: "ESTATE", -7: "ETIMEOUT"}
N_WEIGHTS = 5661  # trunk network; the two-network head adds the mass network's
N_MASS_WEIGHTS = 301


class PMRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"PMR_{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int), ("L", ctypes.c_double), ("nsteps", ctypes.c_int), ("a0", ctypes.c_double),
        ("omega_m", ctypes.c_double), ("sigma8", ctypes.c_double), ("gamma_bbks", ctypes.c_double),
        ("R_feat", ctypes.c_double * 3), ("feat_mix", ctypes.c_float * 9), ("R_M", ctypes.c_double), ("sigma_N2", ctypes.c_double),
        ("mu_N", ctypes.c_double), ("f_eff", ctypes.c_double), ("M_scale", ctypes.c_double),
        ("lbfgs_m", ctypes.c_int), ("lbfgs_tol", ctypes.c_double), ("nn_path", ctypes.c_int), ("head", ctypes.c_int),
        ("lpt_order", ctypes.c_int),
    ]


class Anneal(ctypes.Structure):
    _fields_ = [("R_sm", ctypes.c_double), ("M0", ctypes.c_double), ("a_logistic", ctypes.c_double)]


_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "pmr_default_config": (None, [_P]),
    "pmr_workspace_bytes": (ctypes.c_size_t, [_P]),
    "pmr_create": (ctypes.c_int, [_P, _P, _P, _P]),
    "pmr_destroy": (ctypes.c_int, [_P]),
    "pmr_set_stream": (ctypes.c_int, [_P, _P]),
    "pmr_last_error": (ctypes.c_char_p, [_P]),
    "pmr_linear_field": (ctypes.c_int, [_P, _P, ctypes.c_double, _P]),
    "pm_forward": (ctypes.c_int, [_P, _P, _P]),
    "pm_adjoint": (ctypes.c_int, [_P, _P, _P]),
    "nn_halo_map": (ctypes.c_int, [_P, _P, _P, _P]),
    "nn_halo_map_adjoint": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "loss_and_grad": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "recon_step": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "pmr_lbfgs_reset": (ctypes.c_int, [_P]),
    "pmr_cell_sort": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P]),
    "pmr_paint": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
    "pmr_paint_noalloc": (ctypes.c_int, [ctypes.c_int, _P, _I64, _P, _P, _P]),
    "pmr_readout": (ctypes.c_int, [_P, _P, _P, _I64, _P]),
    "pmr_readout_grad": (ctypes.c_int, [_P, _P, _P, _I64, _P]),
    "pmr_rfft": (ctypes.c_int, [_P, _P, _P]),
    "pmr_irfft": (ctypes.c_int, [_P, _P, _P]),
    "pmr_force": (ctypes.c_int, [_P, _P, _P]),
    "pmr_smooth": (ctypes.c_int, [_P, _P, ctypes.c_double, _P]),
    "pmr_za_ics": (ctypes.c_int, [_P, _P, _P, _P]),
    "pmr_lpt_ics": (ctypes.c_int, [_P, _P, _P, _P]),
    "pmr_use_graphs": (ctypes.c_int, [_P, ctypes.c_int]),
    "pmr_lpt_ics_adjoint": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "pmr_growth": (ctypes.c_int, [_P, ctypes.c_double, _P, _P, _P]),
    "pmr_lbfgs_direction": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, _I64, _P]),
    "pmr_power_spectra": (ctypes.c_int, [_P, _P, _P, _P]),
    "pmr_two_point": (ctypes.c_int, [_P, _P, _P, _P]),
    "pmr_launch_count": (ctypes.c_int64, [_P]),
    "pmr_forward_id": (ctypes.c_int64, [_P]),
    "pmr_sync": (ctypes.c_int, [_P]),
    "pmr_test_stall_mma": (ctypes.c_int, [_P, ctypes.c_int]),
    "pmr_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "pmr_timing_report": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
}
EXPORTS = tuple(_SIGS)


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads the library (built by paper_1805_02247_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpmrecon.so not found at {path}: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_config(**overrides) -> Config:
    cfg = Config()
    load().pmr_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "R_feat":
            cfg.R_feat = (ctypes.c_double * 3)(*v)
        elif k == "feat_mix":
            cfg.feat_mix = (ctypes.c_float * 9)(*[float(x) for x in v])
        else:
            setattr(cfg, k, v)
    return cfg


def workspace_bytes(cfg: Config) -> int:
    return int(load().pmr_workspace_bytes(ctypes.byref(cfg)))


def growth(cfg: Config, a: float):
    D, Gp, Gf = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = load().pmr_growth(ctypes.byref(cfg), a, ctypes.byref(D), ctypes.byref(Gp), ctypes.byref(Gf))
    if rc != PMR_OK:
        raise PMRError(rc, load().pmr_last_error(None).decode())
    return D.value, Gp.value, Gf.value


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("tensors passed to the library must be contiguous CUDA tensors")
    return t.data_ptr()


class Context:
    """One reconstruction job: owns a pmr_ctx (workspace, checkpoints, L-BFGS history)."""

    def __init__(self, cfg: Config, weights: torch.Tensor, stream: torch.cuda.Stream | None = None):
        lib = load()
        self.cfg = cfg
        self.N = cfg.N
        self.device = weights.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        w = weights.to(device=self.device, dtype=torch.float32).contiguous()
        want = N_WEIGHTS + (N_MASS_WEIGHTS if cfg.head == 1 else 0)
        if w.numel() != want:
            raise ValueError(f"weights must have {want} entries")
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.pmr_create(ctypes.byref(cfg), _ptr(w), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != PMR_OK:
            raise PMRError(rc, lib.pmr_last_error(None).decode())
        self._h = h
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pmr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ helpers
    def _check(self, rc: int):
        if rc != PMR_OK:
            raise PMRError(rc, self._lib.pmr_last_error(self._h).decode())

    def mesh(self, *lead) -> torch.Tensor:
        return torch.empty(*lead, self.N, self.N, self.N, device=self.device, dtype=torch.float32)

    def half(self) -> torch.Tensor:
        return torch.empty(self.N, self.N, self.N // 2 + 1, device=self.device, dtype=torch.complex64)

    # ------------------------------------------------------------------ the path
    def linear_field(self, white: torch.Tensor, amplitude: float = 1.0, out=None) -> torch.Tensor:
        s = self.half() if out is None else out
        self._check(self._lib.pmr_linear_field(self._h, _ptr(white), amplitude, _ptr(s)))
        return s

    def pm_forward(self, s: torch.Tensor, out=None) -> torch.Tensor:
        d = self.mesh() if out is None else out
        self._check(self._lib.pm_forward(self._h, _ptr(s), _ptr(d)))
        return d

    def pm_adjoint(self, grad_delta: torch.Tensor, out=None) -> torch.Tensor:
        g = self.half() if out is None else out
        self._check(self._lib.pm_adjoint(self._h, _ptr(grad_delta), _ptr(g)))
        return g

    def nn_halo_map(self, delta: torch.Tensor, a: float = 3.0, out=None) -> torch.Tensor:
        """Halo-mass map of the final density; a = logistic sharpness (two-network head only)."""
        m = self.mesh() if out is None else out
        an = Anneal(0.0, 0.0, a)
        self._check(self._lib.nn_halo_map(self._h, _ptr(delta), _ptr(m), ctypes.byref(an)))
        return m

    def nn_halo_map_adjoint(self, delta: torch.Tensor, grad_mass: torch.Tensor, a: float = 3.0,
                            out=None) -> torch.Tensor:
        g = self.mesh() if out is None else out
        an = Anneal(0.0, 0.0, a)
        self._check(self._lib.nn_halo_map_adjoint(self._h, _ptr(delta), _ptr(grad_mass), _ptr(g),
                                                  ctypes.byref(an)))
        return g

    def loss_and_grad(self, s, data, R_sm: float, M0: float, out=None, readback: bool = True,
                      a: float = 3.0, loss_dev: torch.Tensor | None = None):
        """Loss parts (total, prior, residual) and the gradient. readback: return the parts on
        the host (synchronises); loss_dev: a float64 CUDA tensor of 3 to receive them on the
        stream instead (no synchronisation)."""
        g = self.half() if out is None else out
        an = Anneal(R_sm, M0, a)
        host = (ctypes.c_double * 3)()
        if loss_dev is not None:
            if loss_dev.dtype != torch.float64 or loss_dev.numel() < 3:
                raise ValueError("loss_dev must be a float64 CUDA tensor with 3 entries")
            dst = _ptr(loss_dev)
        else:
            dst = host if readback else None
        self._check(self._lib.loss_and_grad(self._h, _ptr(s), _ptr(data), ctypes.byref(an), dst, _ptr(g)))
        return (tuple(host) if readback and loss_dev is None else None), g

    def sync(self):
        """Synchronise the stream; raises PMR_ETIMEOUT / PMR_ECUDA for failures of earlier async calls."""
        self._check(self._lib.pmr_sync(self._h))

    def test_stall_mma(self, enable: bool):
        """Failure-detection test hook: tensor-core network kernels issue no MMAs, so their waits run out."""
        self._check(self._lib.pmr_test_stall_mma(self._h, 1 if enable else 0))

    def recon_step(self, s, data, R_sm: float, M0: float, a: float = 3.0):
        an = Anneal(R_sm, M0, a)
        host = (ctypes.c_double * 3)()
        conv = ctypes.c_int(0)
        self._check(self._lib.recon_step(self._h, _ptr(s), _ptr(data), ctypes.byref(an), host, ctypes.byref(conv)))
        return tuple(host), bool(conv.value)

    def power_spectra(self, a: torch.Tensor, b: torch.Tensor):
        """(counts, P_aa, P_bb, P_ab) per |k| shell as float64 host tensors (Sec. 4.3)."""
        nb = self.N // 2
        out = (ctypes.c_double * (4 * nb))()
        self._check(self._lib.pmr_power_spectra(self._h, _ptr(a), _ptr(b), out))
        t = torch.tensor(list(out), dtype=torch.float64).view(4, nb)
        return t[0], t[1], t[2], t[3]

    def two_point(self, h: torch.Tensor, m: torch.Tensor) -> dict:
        """Per |k| shell (Sec. 4.3): counts, P_hh, P_mm, P_hm, r_c, stochasticity s, transfer function TF,
        as float64 host tensors; h = the truth or data field, m = the model field."""
        nb = self.N // 2
        out = (ctypes.c_double * (7 * nb))()
        self._check(self._lib.pmr_two_point(self._h, _ptr(h), _ptr(m), out))
        t = torch.tensor(list(out), dtype=torch.float64).view(7, nb)
        return dict(zip(("counts", "P_hh", "P_mm", "P_hm", "r_c", "s", "TF"), t))

    def launch_count(self) -> int:
        return int(self._lib.pmr_launch_count(self._h))

    def forward_id(self) -> int:
        """Identifier of the trajectory the next pm_adjoint differentiates (-1: none)."""
        return int(self._lib.pmr_forward_id(self._h))

    def timing(self, enable: bool):
        self._check(self._lib.pmr_timing(self._h, int(enable)))

    def timing_report(self) -> dict:
        """{kernel name: (launches, total_ms)} since timing(True) or the last report."""
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self._lib.pmr_timing_report(self._h, buf, len(buf)))
        out = {}
        for line in buf.value.decode().splitlines():
            name, n, ms = line.split()
            out[name] = (int(n), float(ms))
        return out

    def use_graphs(self, enable: bool = True):
        """Replay each loss evaluation as one captured CUDA graph (needs a non-default stream)."""
        self._check(self._lib.pmr_use_graphs(self._h, 1 if enable else 0))

    def lbfgs_reset(self):
        self._check(self._lib.pmr_lbfgs_reset(self._h))

    # ------------------------------------------------------------------ single steps
    def cell_sort(self, x: torch.Tensor):
        np_ = x.shape[1]
        keys = torch.empty(np_, device=self.device, dtype=torch.int32)
        perm = torch.empty(np_, device=self.device, dtype=torch.int32)
        start = torch.empty(self.N**3 + 1, device=self.device, dtype=torch.int32)
        self._check(self._lib.pmr_cell_sort(self._h, _ptr(x), np_, _ptr(keys), _ptr(perm), _ptr(start)))
        return keys, perm, start

    def paint(self, x: torch.Tensor, mass: torch.Tensor | None = None) -> torch.Tensor:
        rho = self.mesh()
        self._check(self._lib.pmr_paint(self._h, _ptr(x), x.shape[1], _ptr(mass), _ptr(rho)))
        return rho

    def readout(self, field: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
        out = torch.empty(x.shape[1], device=self.device, dtype=torch.float32)
        self._check(self._lib.pmr_readout(self._h, _ptr(field), _ptr(x), x.shape[1], _ptr(out)))
        return out

    def readout_grad(self, field: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
        out = torch.empty(3, x.shape[1], device=self.device, dtype=torch.float32)
        self._check(self._lib.pmr_readout_grad(self._h, _ptr(field), _ptr(x), x.shape[1], _ptr(out)))
        return out

    def rfft(self, f: torch.Tensor) -> torch.Tensor:
        out = self.half()
        self._check(self._lib.pmr_rfft(self._h, _ptr(f), _ptr(out)))
        return out

    def irfft(self, s: torch.Tensor) -> torch.Tensor:
        out = self.mesh()
        self._check(self._lib.pmr_irfft(self._h, _ptr(s), _ptr(out)))
        return out

    def force(self, delta: torch.Tensor) -> torch.Tensor:
        out = self.mesh(3)
        self._check(self._lib.pmr_force(self._h, _ptr(delta), _ptr(out)))
        return out

    def smooth(self, f: torch.Tensor, R: float) -> torch.Tensor:
        out = self.mesh()
        self._check(self._lib.pmr_smooth(self._h, _ptr(f), R, _ptr(out)))
        return out

    def za_ics(self, s: torch.Tensor):
        disp = torch.empty(3, self.N**3, device=self.device, dtype=torch.float32)
        mom = torch.empty_like(disp)
        self._check(self._lib.pmr_za_ics(self._h, _ptr(s), _ptr(disp), _ptr(mom)))
        return disp, mom

    def lpt_ics(self, s: torch.Tensor):
        """Initial conditions of the configured order: (displacement, momentum), [3][N^3] each."""
        disp = torch.empty(3, self.N**3, device=self.device, dtype=torch.float32)
        mom = torch.empty_like(disp)
        self._check(self._lib.pmr_lpt_ics(self._h, _ptr(s), _ptr(disp), _ptr(mom)))
        return disp, mom

    def lpt_ics_adjoint(self, s: torch.Tensor, lam_x: torch.Tensor, lam_p: torch.Tensor) -> torch.Tensor:
        g = self.half()
        self._check(self._lib.pmr_lpt_ics_adjoint(self._h, _ptr(s), _ptr(lam_x), _ptr(lam_p), _ptr(g)))
        return g

    def lbfgs_direction(self, g: torch.Tensor, S: torch.Tensor, Y: torch.Tensor) -> torch.Tensor:
        d = torch.empty_like(g)
        self._check(self._lib.pmr_lbfgs_direction(self._h, _ptr(g), _ptr(S), _ptr(Y), S.shape[0], g.numel(), _ptr(d)))
        return d


class ReconLoss(torch.autograd.Function):
    """L(s) of Eq. (loss) as a differentiable function of s (complex64 half array).

    Forward and backward both run in the library: the forward call computes the
    gradient with the hand-written adjoint and backward scales it.
    """

    @staticmethod
    def forward(ctx_, s: torch.Tensor, data: torch.Tensor, job: Context, R_sm: float, M0: float,
                a: float = 3.0):
        parts, g = job.loss_and_grad(s.detach().contiguous(), data.contiguous(), R_sm, M0, a=a)
        ctx_.save_for_backward(g)
        return torch.tensor(parts[0], dtype=torch.float64, device=s.device)

    @staticmethod
    def backward(ctx_, grad_out):
        (g,) = ctx_.saved_tensors
        return g * grad_out.to(torch.float32), None, None, None, None, None


class PMForward(torch.autograd.Function):
    """delta_final(s) of the PM model with the hand-written adjoint as its backward.

    The context stores one trajectory (the per-step particle positions of its
    last forward sweep). backward() differentiates the trajectory its own
    forward() left; if any later call on the same context replaced it (another
    PMForward, loss_and_grad, recon_step, ...), backward raises PMR_ESTATE
    instead of returning the gradient of a different trajectory.
    """

    @staticmethod
    def forward(ctx_, s: torch.Tensor, job: Context):
        ctx_.job = job
        delta = job.pm_forward(s.detach().contiguous())
        ctx_.fwd_id = job.forward_id()
        return delta

    @staticmethod
    def backward(ctx_, grad_delta):
        job = ctx_.job
        if job.forward_id() != ctx_.fwd_id:
            raise PMRError(-6, "PMForward.backward: the context's stored trajectory was replaced after this "
                               "forward (run backward before the next forward on the same context)")
        return job.pm_adjoint(grad_delta.contiguous().to(torch.float32)), None
