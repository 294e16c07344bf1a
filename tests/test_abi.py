"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every function include/pmrecon.h declares; the binding's signatures cover them.
No compute call is made (no GPU needed)."""
import ctypes
import os
import re

from paper_1805_02247_gb300 import build, pmrecon

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?[\s\*])([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "for", "while", "sizeof")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pm_forward", "pm_adjoint", "nn_halo_map", "loss_and_grad", "recon_step"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert sorted(pmrecon.EXPORTS) == declared_functions()


def test_config_struct_matches_defaults_and_layout():
    build.build()
    cfg = pmrecon.default_config()
    assert (cfg.N, cfg.L, cfg.nsteps, cfg.a0) == (32, 100.0, 3, 0.1)
    assert list(cfg.R_feat) == [1.0, 2.0, 4.0] and cfg.sigma_N2 == 0.25 and cfg.lbfgs_m == 10
    assert pmrecon.workspace_bytes(cfg) > 0
    assert pmrecon.workspace_bytes(pmrecon.default_config(N=10)) == 0  # 10/2 = 5 has no radix-2/3/4 plan


def test_workspace_grows_by_one_step_of_kept_state():
    """One more PM step keeps, per particle of the lattice, its position (12 B),
    its step's sort (perm 4 B, cell offsets 4 B) and sorted fractional offsets
    (12 B), and the step's force for the adjoint (12 B): the footprint query the
    server admits jobs by must grow by exactly that (each buffer rounded to 256 B)."""
    build.build()

    def r(b):
        return (b + 255) // 256 * 256

    N = 64
    N3 = N ** 3
    for k in (1, 5):
        a = pmrecon.workspace_bytes(pmrecon.default_config(N=N, nsteps=k))
        b = pmrecon.workspace_bytes(pmrecon.default_config(N=N, nsteps=k + 1))
        per_step = (
            r(12 * N3 * (k + 2)) - r(12 * N3 * (k + 1))        # positions
            + r(4 * N3 * (k + 2)) - r(4 * N3 * (k + 1))        # perm of each step
            + r(4 * (N3 + 1) * (k + 2)) - r(4 * (N3 + 1) * (k + 1))  # cell offsets of each step
            + r(12 * N3 * (k + 2)) - r(12 * N3 * (k + 1))      # sorted fractional offsets
            + r(12 * N3 * (k + 1)) - r(12 * N3 * k)            # forces kept for the adjoint
        )
        assert b - a == per_step


def test_growth_is_host_only_and_matches_oracle():
    # pmr_growth needs no device: the library's own quadrature vs the oracle's
    from oracle import cosmo
    build.build()
    cfg = pmrecon.default_config()
    for a in (0.1, 0.5, 1.0):
        D, Gp, Gf = pmrecon.growth(cfg, a)
        assert abs(D / cosmo.D(a) - 1) < 1e-11
        assert abs(Gp / cosmo.Gp(a) - 1) < 1e-10
        assert abs(Gf / cosmo.Gf(a) - 1) < 1e-11
