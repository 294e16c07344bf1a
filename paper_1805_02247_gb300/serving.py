"""Serving many reconstruction jobs on one GPU with continuous batching.

Jobs of different mesh sizes arrive over time. The server admits a job as soon
as a slot is free and its device footprint (the context workspace of
pmr_workspace_bytes plus its own arrays) fits the memory budget, so requests
that arrive while others run join the running set instead of waiting for it
to drain. Every admitted job owns a context on its own CUDA stream, keeps its
s(k), L-BFGS history and annealing state on the device, and runs its annealed
L-BFGS iterations (recon_step) on its own host thread; the library releases
the interpreter lock in every call, so the jobs' kernels overlap on the GPU.
With graphs on, each job replays its loss evaluations as one captured CUDA
graph. The server reports jobs/s and percentiles of the time from arrival to
convergence.

  python -m paper_1805_02247_gb300.serving bench [--jobs 64] [--rate 2] [--slots 8]
"""
from __future__ import annotations

import argparse
import json
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class JobSpec:
    job_id: int
    N: int
    L: float
    nsteps: int
    data_seed: int
    arrival: float                       # seconds after the server starts
    stages: list = field(default_factory=list)  # anneal.Stage list; empty = one default stage
    max_iter: int = 25                   # L-BFGS iterations per stage at most
    nn_path: int = 0


@dataclass
class JobRecord:
    job_id: int
    N: int
    arrival: float
    admitted: float = math.nan
    finished: float = math.nan
    iterations: int = 0
    final_loss: float = math.nan
    footprint: int = 0
    error: str | None = None
    result: object = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def synthetic_stream(n_jobs=64, rate=2.0, sizes=(64, 128, 192, 256), L_range=(200.0, 400.0), steps=(3, 10),
                     seed=7, first_data_seed=100, max_iter=25):
    """Poisson arrivals at `rate` jobs/s; mesh side, box and step count drawn per job."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += rng.exponential(1.0 / rate)
        N = int(rng.choice(sizes))
        L = float(rng.uniform(*L_range))
        ns = int(rng.integers(steps[0], steps[1] + 1))
        jobs.append(JobSpec(j, N, L, ns, first_data_seed + j, t, max_iter=max_iter))
    return jobs


class Server:
    """Admission by slots and memory; `runner(spec, record)` runs one job to the end.

    footprint(spec) -> bytes. The budget and slot count bound what runs at once."""

    def __init__(self, runner, footprint, memory_budget: int, max_slots: int = 8, clock=time.perf_counter):
        self.runner = runner
        self.footprint = footprint
        self.budget = int(memory_budget)
        self.max_slots = max_slots
        self.clock = clock
        self._cv = threading.Condition()
        self._used = 0
        self._running = 0

    def run(self, specs):
        """Serves the jobs (arrival times relative to now); returns records in job order."""
        pending = sorted(specs, key=lambda s: (s.arrival, s.job_id))
        recs = {s.job_id: JobRecord(s.job_id, s.N, s.arrival) for s in specs}
        for s in specs:
            recs[s.job_id].footprint = self.footprint(s)
            if recs[s.job_id].footprint > self.budget:
                raise ValueError(f"job {s.job_id} needs {recs[s.job_id].footprint} bytes, over the budget")
        t0 = self.clock()
        threads = []

        def work(spec, rec):
            try:
                self.runner(spec, rec)
            except Exception as e:  # the job fails, the server goes on
                rec.error = repr(e)[-500:]
            finally:
                rec.finished = self.clock() - t0
                with self._cv:
                    self._used -= rec.footprint
                    self._running -= 1
                    self._cv.notify_all()

        with self._cv:
            while pending:
                now = self.clock() - t0
                head = pending[0]
                fits = self._running < self.max_slots and self._used + recs[head.job_id].footprint <= self.budget
                if head.arrival <= now and fits:
                    pending.pop(0)
                    rec = recs[head.job_id]
                    rec.admitted = now
                    self._used += rec.footprint
                    self._running += 1
                    th = threading.Thread(target=work, args=(head, rec), daemon=True)
                    threads.append(th)
                    th.start()
                    continue
                wait = None if head.arrival <= now else head.arrival - now
                self._cv.wait(timeout=wait)
        for th in threads:
            th.join()
        return [recs[s.job_id] for s in sorted(specs, key=lambda s: s.job_id)]


def summarize(records, wall: float | None = None):
    ok = [r for r in records if r.error is None]
    lat = np.array([r.latency for r in ok]) if ok else np.array([math.nan])
    span = wall if wall is not None else (max(r.finished for r in ok) - min(r.arrival for r in ok) if ok else math.nan)
    return {"jobs": len(records), "failed": len(records) - len(ok), "jobs_per_s": len(ok) / span if span else math.nan,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_iterations": float(np.mean([r.iterations for r in ok])) if ok else math.nan}


# ----------------------------------------------------------------------------- GPU jobs

def gpu_runner(device, use_graphs=True, keep_result=False):
    """The job body: synthetic truth and data from the job's seed, start at 10%
    of the fiducial power, annealed recon_step iterations on the job's stream."""
    import torch

    from . import anneal, pmrecon, synth

    w = torch.from_numpy(synth.xavier_weights(1))

    def run(spec: JobSpec, rec: JobRecord):
        stream = torch.cuda.Stream(device)
        with torch.cuda.device(device), torch.cuda.stream(stream):
            cfg = pmrecon.default_config(N=spec.N, L=spec.L, nsteps=spec.nsteps, nn_path=spec.nn_path)
            ctx = pmrecon.Context(cfg, w.to(device, non_blocking=False), stream=stream)
            try:
                if use_graphs:
                    ctx.use_graphs(True)
                N = spec.N
                s_true = ctx.linear_field(torch.from_numpy(synth.white_noise(N, spec.data_seed)).to(device), 1.0)
                scatter = torch.from_numpy(synth.scatter_noise(N, spec.data_seed)).to(device)
                data = (ctx.nn_halo_map(ctx.pm_forward(s_true)) * torch.exp(0.3 * scatter)).contiguous()
                s = ctx.linear_field(torch.from_numpy(synth.white_noise(N, spec.data_seed + 1000)).to(device),
                                     math.sqrt(0.1))
                cell = spec.L / N
                # the first M0 of the paper's schedule (Sec. 5.3): large enough that the
                # smoothed masses stay above -M0 on coarse meshes
                stages = spec.stages or [anneal.Stage(2 * cell, 1e12), anneal.Stage(1 * cell, 1e12)]
                hist = anneal.reconstruct(ctx, s, data, stages, max_iter=spec.max_iter)
                stream.synchronize()
                rec.iterations = len(hist)
                rec.final_loss = hist[-1]["loss"] if hist else math.nan
                if keep_result:
                    rec.result = s.cpu()
            finally:
                ctx.close()
                torch.cuda.empty_cache()  # return the job's arrays before the next admission

    return run


def gpu_footprint(spec: JobSpec) -> int:
    from . import pmrecon

    cfg = pmrecon.default_config(N=spec.N, L=spec.L, nsteps=spec.nsteps, nn_path=spec.nn_path)
    N = spec.N
    nh = N * N * (N // 2 + 1)
    # context workspace + s, s_true, gradient views (c64) + data, scatter, density, mass (float32)
    return int(pmrecon.workspace_bytes(cfg)) + 3 * 8 * nh + 6 * 4 * N ** 3


def main(argv=None):
    ap = argparse.ArgumentParser(description="serving benchmark")
    ap.add_argument("run", choices=["bench"])
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--rate", type=float, default=2.0)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--max-iter", type=int, default=25)
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--budget-frac", type=float, default=0.8)
    args = ap.parse_args(argv)
    import torch

    from . import build

    build.build()
    dev = torch.device("cuda", 0)
    free, _ = torch.cuda.mem_get_info(dev)
    specs = synthetic_stream(args.jobs, args.rate, max_iter=args.max_iter)
    server = Server(gpu_runner(dev, use_graphs=not args.no_graphs), gpu_footprint,
                    int(args.budget_frac * free), args.slots)
    t = time.perf_counter()
    recs = server.run(specs)
    wall = time.perf_counter() - t
    out = summarize(recs, wall=wall - min(s.arrival for s in specs))
    out.update({"wall_s": wall, "slots": args.slots, "graphs": not args.no_graphs, "rate_jobs_per_s": args.rate,
                "sizes": sorted({s.N for s in specs}),
                "errors": [r.error for r in recs if r.error][:3]})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
