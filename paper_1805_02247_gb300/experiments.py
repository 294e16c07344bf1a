"""Reconstruction runs of the kind the paper reports (Sec. 5.3), on synthetic data.

  python -m paper_1805_02247_gb300.experiments recon [--N 128] [--iters 100] [--schedule radii|paper] [--out run.json]
  python -m paper_1805_02247_gb300.experiments precision [--N 256] [--iters 200] [--out run.json]

`full_reconstruction` builds a truth field, its halo-mass data, and runs the
annealed L-BFGS reconstruction on the GPU from a start at 10% of the fiducial
power. It reports the loss history and, per |k| shell, the cross-correlation,
transfer function and stochasticity of the reconstructed linear field and of
its final density against the truth (Sec. 4.3).

Data (Sec. 3 and 5.3, with the paper's FOF catalogue replaced by the model):
the network's halo-mass field of the truth, times log-normal scatter
exp(0.3 g), keeping only the ceil(8 n L^3) most massive voxels (a halo number
density n spread over its 8 CIC cells) and zeroing the rest, as the paper's
sparse halo mesh is mostly empty.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np
import torch

from . import anneal, pmrecon, synth


def _stats(ctx, a, b):
    """Sec. 4.3 statistics of field b (the model) against field a (the truth), per |k| shell."""
    t = ctx.two_point(a, b)
    kf = 2 * math.pi / ctx.cfg.L
    k = kf * (np.arange(len(t["counts"])) + 1.0)  # shell i holds i <= |n| - 0.5 < i + 1
    return {"k": k.tolist(), "modes": t["counts"].tolist(), "r_c": t["r_c"].tolist(), "transfer": t["TF"].tolist(),
            "stochasticity": t["s"].tolist()}


def stages_for(schedule: str, head: int, N: int, L: float, radii, M0: float):
    """The annealing stages of a run: "radii" anneals the residual smoothing
    over the given radii (Mpc/h) at one M0; "paper" is the procedure of
    Sec. 5.3 in grid cells of L/N (with the sharpness loop for the two-network head)."""
    if schedule == "paper":
        cell = L / N
        return anneal.two_network_schedule(cell) if head == 1 else anneal.paper_schedule(cell)
    if schedule == "radii":
        return [anneal.Stage(float(r), M0) for r in radii]
    raise ValueError(f"unknown schedule {schedule!r}")


def full_reconstruction(N=128, L=400.0, nsteps=5, lpt_order=2, nbar=1e-3, radii=(4.0, 2.0, 1.0, 0.5), M0=1e12,
                        iters=100, min_iter=10, nn_path=0, head=0, device="cuda", progress=None, schedule="radii"):
    cfg = pmrecon.default_config(N=N, L=L, nsteps=nsteps, lpt_order=lpt_order, nn_path=nn_path, head=head)
    w = synth.two_net_weights(1) if head == 1 else synth.xavier_weights(1)
    ctx = pmrecon.Context(cfg, torch.from_numpy(w).to(device))
    dev = torch.device(device)
    t0 = time.perf_counter()
    s_true = ctx.linear_field(torch.from_numpy(synth.white_noise(N, 2)).to(dev), 1.0)
    d_true = ctx.pm_forward(s_true).clone()
    m_true = ctx.nn_halo_map(d_true)
    data = m_true * torch.exp(0.3 * torch.from_numpy(synth.scatter_noise(N, 2)).to(dev))
    keep = min(N ** 3, math.ceil(8 * nbar * L ** 3))
    thr = torch.topk(data.flatten(), keep).values[-1]
    data = torch.where(data >= thr, data, torch.zeros_like(data)).contiguous()
    s = ctx.linear_field(torch.from_numpy(synth.white_noise(N, 0)).to(dev), math.sqrt(0.1))
    stages = stages_for(schedule, head, N, L, radii, M0)
    lin_true = ctx.irfft(s_true)
    before = {"linear": _stats(ctx, lin_true, ctx.irfft(s)), "final": _stats(ctx, d_true, ctx.pm_forward(s))}
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    dumps = []

    def stage_end(si, st):
        # the reconstructed linear field against the truth after each stage (the
        # per-stage panels of the paper's reconstruction figure, Sec. 5.3)
        dumps.append(_stats(ctx, lin_true, ctx.irfft(s)))

    hist = anneal.reconstruct(ctx, s, data, stages, max_iter=iters, callback=progress, min_iter=min_iter,
                              stage_end=stage_end)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    after = {"linear": _stats(ctx, lin_true, ctx.irfft(s)), "final": _stats(ctx, d_true, ctx.pm_forward(s))}
    per_stage = []
    for si, st in enumerate(stages):
        rec = [h for h in hist if h["stage"] == si]
        per_stage.append({"R_sm": st.R_sm, "M0": st.M0, "a": st.a, "iterations": len(rec),
                          "loss_first": rec[0]["loss"] if rec else None, "loss_last": rec[-1]["loss"] if rec else None,
                          "converged": bool(rec and rec[-1]["converged"]),
                          "seconds": sum(h["seconds"] for h in rec),
                          "losses": [h["loss"] for h in rec],
                          "linear_after": dumps[si]})
    out = {"config": {"N": N, "L": L, "nsteps": nsteps, "lpt_order": lpt_order, "nbar": nbar, "kept_voxels": keep,
                      "schedule": schedule, "radii": list(radii), "M0": M0, "max_iter": iters, "min_iter": min_iter,
                      "nn_path": nn_path, "head": head},
           "setup_seconds": t1 - t0, "reconstruction_seconds": t2 - t1,
           "iterations": len(hist), "stages": per_stage, "before": before, "after": after}
    ctx.close()
    return out


def _rel(a, b):
    a = torch.view_as_real(a) if a.is_complex() else a
    b = torch.view_as_real(b) if b.is_complex() else b
    return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))


def precision(N=256, L=400.0, nsteps=5, iters=200, R_sm=4.0, M0=1e8, device="cuda", schedule=None, min_iter=10,
              tol=1e-7):
    """The bf16 tensor-core network (nn_path 3) against the float32-accurate one
    (nn_path 0, itself within 1e-5 / 1e-4 of the FP64 oracle in the tests): the
    error of each stage on the same inputs, and the loss each path reaches from
    the same start on the same data: after `iters` L-BFGS iterations at (R_sm,
    M0); with schedule="paper", at the end of the annealing procedure of
    Sec. 5.3 run to its stop rule (a stage ends when an iteration lowers the loss
    by less than 0.1%, from its min_iter-th iteration on; at most `iters` per
    stage); with schedule="converged", at (R_sm, M0) until an iteration lowers
    the loss by less than tol (relative) or after `iters` iterations. Each path's
    final point is also evaluated with the float32-accurate loss, so the two
    solutions are compared on one yardstick."""
    dev = torch.device(device)
    w = torch.from_numpy(synth.xavier_weights(1)).to(dev)
    ltol = tol if schedule == "converged" else 1e-3
    # path 0: float32-accurate network; 3: bf16 network; "c": the float32 path again
    # from the start perturbed by one part in 10^6 (the control: how far two float32
    # trajectories drift apart from rounding-sized differences alone)
    ctx = {p: pmrecon.Context(pmrecon.default_config(N=N, L=L, nsteps=nsteps, nn_path=0 if p == "c" else p,
                                                     lbfgs_tol=ltol), w)
           for p in (0, 3, "c")}
    s_true = ctx[0].linear_field(torch.from_numpy(synth.white_noise(N, 2)).to(dev), 1.0)
    delta = ctx[0].pm_forward(s_true).clone()
    data = (ctx[0].nn_halo_map(delta) * torch.exp(0.3 * torch.from_numpy(synth.scatter_noise(N, 2)).to(dev)))
    data = data.contiguous()
    s0 = ctx[0].linear_field(torch.from_numpy(synth.white_noise(N, 0)).to(dev), math.sqrt(0.1))
    eps = torch.from_numpy(synth.gaussian_vector(tuple(s0.shape) + (2,), seed=6)).to(dev)
    s0c = (s0 * (1 + 1e-6 * torch.view_as_complex(eps))).contiguous()
    starts = {0: s0, 3: s0, "c": s0c}
    gM = torch.from_numpy(synth.gaussian_vector((N, N, N), seed=5)).to(dev)
    M = {p: ctx[p].nn_halo_map(delta).clone() for p in (0, 3)}
    gd = {p: ctx[p].nn_halo_map_adjoint(delta, gM).clone() for p in (0, 3)}
    lg = {p: ctx[p].loss_and_grad(s0, data, R_sm, M0) for p in (0, 3)}
    paths = (0, 3, "c")
    stages_err = {"network_output_M": _rel(M[3], M[0]), "network_adjoint_grad_delta": _rel(gd[3], gd[0]),
                  "loss": abs(lg[3][0][0] / lg[0][0][0] - 1), "loss_gradient": _rel(lg[3][1], lg[0][1])}
    runs = {}
    finals = {}

    def fp32_loss_at(s_final, st):
        parts, _ = ctx[0].loss_and_grad(s_final, data, st.R_sm, st.M0)
        return parts[0]

    if schedule in ("paper", "converged"):
        stages = anneal.paper_schedule(L / N) if schedule == "paper" else [anneal.Stage(R_sm, M0)]
        mi = min_iter if schedule == "paper" else 1
        for p in paths:
            s = starts[p].clone()
            t = time.perf_counter()
            hist = anneal.reconstruct(ctx[p], s, data, stages, max_iter=iters, min_iter=mi)
            torch.cuda.synchronize()
            finals[p] = s
            per = []
            for si, st in enumerate(stages):
                rec = [h for h in hist if h["stage"] == si]
                per.append({"R_sm": st.R_sm, "M0": st.M0, "iterations": len(rec),
                            "final_loss": rec[-1]["loss"] if rec else None,
                            "converged": bool(rec and rec[-1]["converged"])})
            runs[p] = {"iterations": len(hist), "final_loss": hist[-1]["loss"], "stages": per,
                       "seconds": time.perf_counter() - t}
        last = stages[-1]
        yard = {p: fp32_loss_at(finals[p], last) for p in paths}
        for c in ctx.values():
            c.close()
        gaps = [abs(b["final_loss"] / a["final_loss"] - 1) if a["final_loss"] and b["final_loss"] else None
                for a, b in zip(runs[0]["stages"], runs[3]["stages"])]
        gaps_c = [abs(b["final_loss"] / a["final_loss"] - 1) if a["final_loss"] and b["final_loss"] else None
                  for a, b in zip(runs[0]["stages"], runs["c"]["stages"])]
        return {"config": {"N": N, "L": L, "nsteps": nsteps, "schedule": schedule, "max_iter_per_stage": iters,
                           "stop": (f"decrease below 0.1% per iteration from iteration {mi} of a stage"
                                    if schedule == "paper" else f"decrease below {tol:g} per iteration"),
                           "stages": [(st.R_sm, st.M0) for st in stages]},
                "stage_rel_err_bf16_vs_fp32": stages_err, "fp32_path": runs[0], "bf16_path": runs[3],
                "stage_final_loss_rel_gap": gaps, "stage_final_loss_rel_gap_fp32_control": gaps_c,
                "final_loss_rel_diff": abs(runs[3]["final_loss"] / runs[0]["final_loss"] - 1),
                "final_points_on_the_fp32_loss": {"fp32_path": yard[0], "bf16_path": yard[3],
                                                  "rel_diff": abs(yard[3] / yard[0] - 1),
                                                  "fp32_control_from_start_x(1+1e-6)": yard["c"],
                                                  "control_rel_diff": abs(yard["c"] / yard[0] - 1)},
                "fp32_control_path": runs["c"]}
    for p in paths:
        s = starts[p].clone()
        ctx[p].lbfgs_reset()
        t = time.perf_counter()
        losses = []
        for _ in range(iters):
            try:
                parts, conv = ctx[p].recon_step(s, data, R_sm, M0)
            except pmrecon.PMRError as e:
                if e.code == -5:
                    break
                raise
            losses.append(parts[0])
        torch.cuda.synchronize()
        runs[p] = {"iterations": len(losses), "final_loss": losses[-1], "first_loss": losses[0],
                   "seconds": time.perf_counter() - t}
        finals[p] = s
    yard = {p: fp32_loss_at(finals[p], anneal.Stage(R_sm, M0)) for p in paths}
    for c in ctx.values():
        c.close()
    return {"config": {"N": N, "L": L, "nsteps": nsteps, "R_sm": R_sm, "M0": M0, "iters": iters},
            "stage_rel_err_bf16_vs_fp32": stages_err, "fp32_path": runs[0], "bf16_path": runs[3],
            "fp32_control_path": runs["c"],
            "final_loss_rel_diff": abs(runs[3]["final_loss"] / runs[0]["final_loss"] - 1),
            "final_points_on_the_fp32_loss": {"fp32_path": yard[0], "bf16_path": yard[3],
                                              "rel_diff": abs(yard[3] / yard[0] - 1),
                                              "fp32_control_from_start_x(1+1e-6)": yard["c"],
                                              "control_rel_diff": abs(yard["c"] / yard[0] - 1)}}


def summarize_recon(res: dict, command: str, nk: int = 16) -> dict:
    """The per-stage summary of full_reconstruction's result: the loss of every
    iteration, and r_c, TF and s (Sec. 4.3) of the linear field on the first nk
    k bins after each stage."""
    def stats(d, keys):
        return {k: [round(float(v), 4) for v in d[k][:nk]] for k in keys}

    cfg = res["config"]
    what = "annealed reconstruction on the GPU"
    if cfg.get("schedule") == "paper":
        what += (", the procedure of Sec. 5.3 (M0 = 1e12 with N_sm = 4, 2, 1, 0.5, 0 cells, then M0 = 1e11 with "
                 "N_sm = 1, 0.5, 0; a stage ends when an iteration lowers the loss by less than 0.1%, from its "
                 f"{cfg['min_iter']}th iteration on, at most {cfg['max_iter']} iterations)")
    return {
        "what": what,
        "command": command,
        "config": cfg,
        "setup_seconds": round(res["setup_seconds"], 2),
        "reconstruction_seconds": round(res["reconstruction_seconds"], 3),
        "iterations": res["iterations"],
        "k_h_per_Mpc": [round(float(v), 4) for v in res["before"]["linear"]["k"][:nk]],
        "modes": [float(v) for v in res["before"]["linear"]["modes"][:nk]],
        "start": {"linear_r_c": stats(res["before"]["linear"], ["r_c"])["r_c"]},
        "stages": [{
            "R_sm_Mpc_h": st["R_sm"],
            "M0": st["M0"],
            "iterations": st["iterations"],
            "converged": st["converged"],
            "seconds": round(st["seconds"], 3),
            "loss_per_iteration": [round(float(v), 1) for v in st["losses"]],
            "linear_after": stats(st["linear_after"], ["r_c", "transfer", "stochasticity"]),
        } for st in res["stages"]],
        "final": {"linear": stats(res["after"]["linear"], ["r_c", "transfer", "stochasticity"]),
                  "final_density": stats(res["after"]["final"], ["r_c", "transfer"])},
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("run", choices=["recon", "precision"])
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--L", type=float, default=400.0)
    ap.add_argument("--nsteps", type=int, default=5)
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--nn-path", type=int, default=0)
    ap.add_argument("--head", type=int, default=0)
    ap.add_argument("--schedule", choices=["radii", "paper", "converged"], default="radii",
                    help="recon: radii (R_sm = 4, 2, 1, 0.5 Mpc/h at M0 = 1e12) or paper (the procedure of Sec. 5.3); "
                         "precision: paper, or converged (one stage to a 1e-7 relative decrease)")
    ap.add_argument("--R-sm", type=float, default=4.0, help="precision: residual smoothing, Mpc/h")
    ap.add_argument("--M0", type=float, default=1e8, help="precision: M0")
    ap.add_argument("--out", default=None)
    ap.add_argument("--summary", default=None,
                    help="recon: also write the per-stage summary (first 16 k bins, rounded) to this path")
    args = ap.parse_args(argv)
    if args.run == "precision":
        res = precision(N=args.N or 256, L=args.L, nsteps=args.nsteps, iters=args.iters or 200,
                        schedule=args.schedule if args.schedule in ("paper", "converged") else None,
                        R_sm=args.R_sm, M0=args.M0)
        if args.out:
            with open(args.out, "w") as f:
                f.write(json.dumps(res))
        print(json.dumps(res))
        return
    res = full_reconstruction(N=args.N or 128, L=args.L, nsteps=args.nsteps, iters=args.iters or 100,
                              nn_path=args.nn_path, head=args.head, schedule=args.schedule)
    text = json.dumps(res)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    if args.summary:
        words = ["python -m paper_1805_02247_gb300.experiments"] + list(argv if argv is not None else sys.argv[1:])
        command = " ".join(w for i, w in enumerate(words)
                           if w not in ("--summary", "--out") and words[i - 1] not in ("--summary", "--out"))
        with open(args.summary, "w") as f:
            json.dump(summarize_recon(res, command), f, indent=1)
            f.write("\n")
    s = res["stages"]
    print(json.dumps({"iterations": res["iterations"], "seconds": res["reconstruction_seconds"],
                      "stages": [(x["R_sm"], x["iterations"], x["loss_first"], x["loss_last"]) for x in s],
                      "r_c_linear_first8": [round(v, 3) for v in res["after"]["linear"]["r_c"][:8]]}))


if __name__ == "__main__":
    main()
