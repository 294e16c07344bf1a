"""Host logic of the annealed-reconstruction summary (no GPU): the per-stage
record written next to the results keeps every iteration's loss and the first
16 k bins of the two-point statistics, rounded, in the stage order of the run."""
import json

import numpy as np

from paper_1805_02247_gb300.experiments import summarize_recon


def _stats(nk, seed):
    rng = np.random.default_rng(seed)
    return {"k": list(np.arange(1, nk + 1) * 0.0157079632679),
            "modes": list(rng.integers(10, 1000, nk).astype(float)),
            "r_c": list(rng.uniform(-1, 1, nk)),
            "transfer": list(rng.uniform(0, 2, nk)),
            "stochasticity": list(rng.uniform(0, 5000, nk))}


def _result(nk=24):
    cfg = {"N": 32, "L": 400.0, "nsteps": 5, "schedule": "paper", "min_iter": 10, "max_iter": 100}
    stages = [{"R_sm": r, "M0": m, "a": 3.0, "iterations": it, "loss_first": 2.0, "loss_last": 1.0,
               "converged": True, "seconds": 0.123456, "losses": list(np.linspace(2.0, 1.0, it) * 1e5),
               "linear_after": _stats(nk, 10 + i)}
              for i, (r, m, it) in enumerate([(12.5, 1e12, 11), (0.0, 1e12, 12), (0.0, 1e11, 10)])]
    return {"config": cfg, "setup_seconds": 3.14159, "reconstruction_seconds": 1.23456, "iterations": 33,
            "stages": stages,
            "before": {"linear": _stats(nk, 1), "final": _stats(nk, 2)},
            "after": {"linear": _stats(nk, 3), "final": _stats(nk, 4)}}


def test_summary_keeps_every_loss_and_the_first_16_bins():
    res = _result()
    out = summarize_recon(res, "python -m paper_1805_02247_gb300.experiments recon --N 32")
    json.dumps(out)  # plain JSON
    assert out["command"].endswith("recon --N 32") and "Sec. 5.3" in out["what"]
    assert out["iterations"] == 33 and out["reconstruction_seconds"] == 1.235 and out["setup_seconds"] == 3.14
    assert len(out["k_h_per_Mpc"]) == len(out["modes"]) == len(out["start"]["linear_r_c"]) == 16
    assert out["start"]["linear_r_c"] == [round(v, 4) for v in res["before"]["linear"]["r_c"][:16]]
    assert [s["R_sm_Mpc_h"] for s in out["stages"]] == [12.5, 0.0, 0.0]
    assert [s["M0"] for s in out["stages"]] == [1e12, 1e12, 1e11]
    for got, st in zip(out["stages"], res["stages"]):
        assert got["iterations"] == st["iterations"] == len(got["loss_per_iteration"])
        assert got["loss_per_iteration"] == [round(v, 1) for v in st["losses"]]
        assert set(got["linear_after"]) == {"r_c", "transfer", "stochasticity"}
        assert all(len(v) == 16 for v in got["linear_after"].values())
    assert set(out["final"]) == {"linear", "final_density"}
    assert out["final"]["final_density"]["r_c"] == [round(v, 4) for v in res["after"]["final"]["r_c"][:16]]


def test_summary_of_another_schedule_names_no_procedure():
    res = _result()
    res["config"]["schedule"] = "radii"
    assert summarize_recon(res, "cmd")["what"] == "annealed reconstruction on the GPU"
