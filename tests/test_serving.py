"""Serving: admission by slots and memory with continuous batching (host
logic on CPU with a fake job body), and on the GPU that every result is the
same alone and in the mix."""
import threading
import time

import pytest

from paper_1805_02247_gb300.serving import JobSpec, Server, summarize, synthetic_stream


class FakeJobs:
    """Job body that sleeps N/1000 s and tracks how many run at once."""

    def __init__(self):
        self.lock = threading.Lock()
        self.running = 0
        self.peak = 0
        self.order = []

    def __call__(self, spec, rec):
        with self.lock:
            self.running += 1
            self.peak = max(self.peak, self.running)
            self.order.append(spec.job_id)
        time.sleep(spec.N / 1000.0)
        rec.iterations = spec.N
        rec.final_loss = float(spec.job_id)
        with self.lock:
            self.running -= 1


def specs(sizes, arrivals):
    return [JobSpec(j, n, 100.0, 3, 100 + j, a) for j, (n, a) in enumerate(zip(sizes, arrivals))]


def test_slots_bound_the_running_set():
    jobs = FakeJobs()
    srv = Server(jobs, lambda s: 1, memory_budget=100, max_slots=3)
    recs = srv.run(specs([40] * 9, [0.0] * 9))
    assert jobs.peak == 3
    assert all(r.error is None for r in recs)


def test_memory_budget_bounds_the_running_set():
    jobs = FakeJobs()
    srv = Server(jobs, lambda s: s.N, memory_budget=100, max_slots=8)
    recs = srv.run(specs([40, 40, 40, 40], [0.0] * 4))  # two fit at a time
    assert jobs.peak == 2
    assert sorted(jobs.order) == [0, 1, 2, 3]


def test_arrivals_join_the_running_set():
    # job 1 arrives while job 0 runs and starts before job 0 ends (not a drained queue)
    jobs = FakeJobs()
    srv = Server(jobs, lambda s: 1, memory_budget=10, max_slots=4)
    recs = srv.run(specs([200, 20], [0.0, 0.05]))
    assert recs[1].admitted < recs[0].finished
    assert recs[1].finished < recs[0].finished


def test_admission_is_first_come_first_served_and_arrival_timed():
    jobs = FakeJobs()
    srv = Server(jobs, lambda s: 1, memory_budget=10, max_slots=1)
    recs = srv.run(specs([10, 10, 10], [0.06, 0.0, 0.03]))
    assert jobs.order == [1, 2, 0]
    for r in recs:
        assert r.admitted >= r.arrival - 1e-3


def test_a_failing_job_does_not_stop_the_others():
    def body(spec, rec):
        if spec.job_id == 1:
            raise RuntimeError("boom")
        rec.iterations = 1

    recs = Server(body, lambda s: 1, 10, 2).run(specs([10, 10, 10], [0.0, 0.0, 0.0]))
    assert recs[1].error and "boom" in recs[1].error
    assert recs[0].error is None and recs[2].error is None
    out = summarize(recs)
    assert out["failed"] == 1 and out["jobs"] == 3


def test_oversized_job_is_rejected_up_front():
    with pytest.raises(ValueError):
        Server(FakeJobs(), lambda s: 1000, 10, 2).run(specs([10], [0.0]))


def test_synthetic_stream_shapes():
    st = synthetic_stream(64, 2.0)
    assert len(st) == 64
    assert {s.N for s in st} <= {64, 128, 192, 256}
    assert all(200.0 <= s.L <= 400.0 and 3 <= s.nsteps <= 10 for s in st)
    arr = [s.arrival for s in st]
    assert arr == sorted(arr) and 16.0 < arr[-1] < 64.0  # ~2 jobs/s
    assert [s.data_seed for s in st] == list(range(100, 164))


@pytest.mark.gpu
@pytest.mark.parametrize("graphs", [False, True])
def test_results_are_the_same_alone_and_in_the_mix(graphs):
    import torch

    from paper_1805_02247_gb300.serving import gpu_footprint, gpu_runner
    from paper_1805_02247_gb300 import anneal

    dev = torch.device("cuda", 0)

    def mk():
        # a 64^3 job among them runs the register-FFT kernels of the full-size path
        out = specs([16, 24, 64, 32, 16], [0.0, 0.0, 0.005, 0.01, 0.02])
        for s in out:
            s.L = 50.0 * s.N / 16
            s.max_iter = 4
            s.stages = [anneal.Stage(2 * s.L / s.N, 1e10), anneal.Stage(s.L / s.N, 1e10)]
        return out

    alone = Server(gpu_runner(dev, use_graphs=graphs, keep_result=True), gpu_footprint, 8 << 30, 1).run(mk())
    mixed = Server(gpu_runner(dev, use_graphs=graphs, keep_result=True), gpu_footprint, 8 << 30, 4).run(mk())
    for a, m in zip(alone, mixed):
        assert a.error is None and m.error is None, (a.error, m.error)
        assert a.iterations == m.iterations
        assert a.final_loss == m.final_loss
        assert torch.equal(a.result, m.result)  # deterministic kernels, one context per job
    if graphs:  # replaying captured graphs gives the same iterates as direct launches
        direct = Server(gpu_runner(dev, use_graphs=False, keep_result=True), gpu_footprint, 8 << 30, 4).run(mk())
        for a, d in zip(mixed, direct):
            assert torch.equal(a.result, d.result)
