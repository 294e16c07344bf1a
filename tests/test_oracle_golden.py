"""Configuration pins against values the paper prints (tests/golden/, each line
with its passage): the annealing procedure of Sec. 5.3 and the simulation and
loss parameters of Secs. 3, 4.2, 5.1 and 5.3, as the oracle, the library's
defaults and the reconstruction driver use them. No GPU needed."""
import inspect
import os

import pytest

from oracle import anneal as oanneal
from oracle import cosmo
from oracle import loss as oloss

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def _params():
    return {r[0]: r[1] for r in _rows("simulation_parameters.txt")}


def test_two_network_schedule_is_the_printed_procedure():
    # N_sm outer, a inner at M0 = 1e12; then a = 3 at M0 = 1e11
    from paper_1805_02247_gb300 import anneal
    cell = 3.125  # 400 Mpc/h over 128 cells
    want = [(float(m0), float(nsm) * cell, float(a)) for m0, nsm, a in _rows("annealing_schedule.txt")]
    got = [(st.M0, st.R_sm, st.a) for st in anneal.two_network_schedule(cell)]
    assert got == want


def test_single_network_schedule_drops_only_the_sharpness_loop():
    from paper_1805_02247_gb300 import anneal
    cell = 3.125
    want = []
    for m0, nsm, _ in _rows("annealing_schedule.txt"):
        st = (float(m0), float(nsm) * cell)
        if st not in want:
            want.append(st)
    assert [(st.M0, st.R_sm) for st in anneal.paper_schedule(cell)] == want


def test_oracle_constants_are_the_printed_ones():
    p = _params()
    assert cosmo.OMEGA_M == float(p["Omega_M"]) and cosmo.H_LITTLE == float(p["h"])
    ls = oloss.LossSetup()
    assert ls.R_M == float(p["R_M"]) and ls.sigma_N2 == float(p["sigma_N2"]) and ls.f_eff == float(p["f_eff"])
    assert inspect.signature(oanneal.reconstruct).parameters["tol"].default == float(p["lbfgs_tol"])


def test_library_defaults_are_the_printed_ones():
    from paper_1805_02247_gb300 import build, pmrecon
    build.build()
    p = _params()
    cfg = pmrecon.default_config()
    assert cfg.omega_m == float(p["Omega_M"])
    assert cfg.a0 == pytest.approx(1.0 / (1.0 + float(p["z_init"])), rel=1e-15)
    assert (cfg.R_M, cfg.sigma_N2, cfg.f_eff, cfg.lbfgs_tol) == (float(p["R_M"]), float(p["sigma_N2"]),
                                                                 float(p["f_eff"]), float(p["lbfgs_tol"]))


def test_reconstruction_run_uses_the_printed_setting():
    from paper_1805_02247_gb300 import experiments
    p = _params()
    d = inspect.signature(experiments.full_reconstruction).parameters
    assert (d["N"].default, d["L"].default, d["nsteps"].default, d["nbar"].default) == (
        int(p["N"]), float(p["L"]), int(p["pm_steps"]), float(p["nbar"]))


def test_network_shapes_are_the_printed_ones():
    from oracle import nn
    p = _params()
    assert [nn.N_IN, nn.N_H1, nn.N_H2, 1] == [int(v) for v in p["NNp_layers"].split(",")]
    assert [nn.NM_IN, nn.NM_H1, nn.NM_H2, 1] == [int(v) for v in p["NNm_layers"].split(",")]
    assert len(nn.STENCIL) * 3 == nn.N_IN
    assert oloss.Anneal(1.0, 1e12).a == float(p["logistic_a"])


def test_reconstruction_run_can_take_the_printed_schedule():
    from paper_1805_02247_gb300 import anneal, experiments
    p = _params()
    N, L = int(p["N"]), float(p["L"])
    assert experiments.stages_for("paper", 1, N, L, (), 0.0) == anneal.two_network_schedule(L / N)
    assert experiments.stages_for("paper", 0, N, L, (), 0.0) == anneal.paper_schedule(L / N)
    assert [(st.R_sm, st.M0) for st in experiments.stages_for("radii", 0, N, L, (4.0, 2.0), 1e12)] == [
        (4.0, 1e12), (2.0, 1e12)]
