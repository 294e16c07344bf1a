"""Pins of the oracle's L-BFGS line search, stop rule and annealing driver
(Sec. 5.2-5.3) on toy objectives whose minimisers and iteration counts follow
by hand. No GPU needed."""
import numpy as np

from oracle import anneal as oanneal
from oracle import lbfgs
from oracle import loss as oloss


def test_armijo_halves_an_overshooting_first_step():
    # f = x.x, H0 = 1: the first trial x - 2x = -x keeps f (no sufficient
    # decrease), the halved step lands on the minimum
    x0 = np.array([1.0, -2.0, 0.5])
    calls = []

    def fun(x):
        calls.append(x.copy())
        return float(x @ x), 2.0 * x

    st = lbfgs.LBFGSState(x=x0.copy())
    status, conv, evals = lbfgs.step(fun, st, H0=np.ones(3), tol=0.0)
    assert status == "ok" and evals == 3
    assert np.array_equal(calls[1], -x0) and np.array_equal(st.x, np.zeros(3))
    assert st.f == 0.0 and not conv  # tol = 0: never converged by the rule


def test_line_search_failure_is_reported():
    # a gradient of the wrong sign: the "descent" direction climbs f = x.x for
    # every step length, so no trial passes Armijo and the state is untouched
    fun = lambda x: (float(x @ x), -2.0 * x)
    st = lbfgs.LBFGSState(x=np.ones(2))
    status, conv, evals = lbfgs.step(fun, st, H0=np.ones(2), max_ls=5)
    assert status == "linesearch_failed" and not conv and evals == 6
    assert np.array_equal(st.x, np.ones(2)) and st.f == 2.0


def test_stop_rule_is_the_relative_decrease():
    # f = c x^2 with H0 = 1/(2c): every step is exact after the first, so the
    # second iteration's decrease is 0 and the rule fires; the first's is all of f
    c = 3.0
    fun = lambda x: (float(c * x @ x), 2.0 * c * x)
    st = lbfgs.LBFGSState(x=np.array([4.0]))
    _, conv1, _ = lbfgs.step(fun, st, H0=np.array([1.0 / (2.0 * c)]), tol=1e-3)
    assert st.f == 0.0 and not conv1  # (f_old - f_new) = |f_old| is not below tol |f_old|
    st2 = lbfgs.LBFGSState(x=np.array([4.0]))
    fun2 = lambda x: (float(c * x @ x + 100.0), 2.0 * c * x)
    _, conv2, _ = lbfgs.step(fun2, st2, H0=np.array([1.0 / (2.0 * c)]), tol=0.5)
    # decrease 48 of |f_old| = 148: below 0.5 |f_old|, converged
    assert st2.f == 100.0 and conv2


def test_driver_runs_the_stages_in_order_and_stops_each_by_the_rule(monkeypatch):
    # a separable quadratic whose centre depends on the stage's (R_sm, M0, a):
    # each stage converges to its own centre, starting where the last one ended
    seen = []

    def fake_loss(v, data, weights, pms, ls, an):
        centre = an.R_sm + 10.0 * np.log10(an.M0) + 100.0 * an.a
        seen.append((an.R_sm, an.M0, an.a))
        r = v - centre
        return {"loss": float(r @ r) + 1.0}, 2.0 * r

    monkeypatch.setattr(oloss, "loss_and_grad", fake_loss)
    monkeypatch.setattr(oloss, "prior_inverse_hessian", lambda pms: np.full(4, 0.5))
    stages = [(4.0, 1e12, 1.0), (4.0, 1e12, 2.0), (2.0, 1e11, 3.0)]
    x, hist = oanneal.reconstruct(np.zeros(4), None, None, None, None, stages, max_iter=10, tol=1e-3)
    # H0 = 1/2 is the exact inverse Hessian: iteration 1 lands on the centre
    # (loss 1), iteration 2 decreases by 0 and stops the stage
    assert [len(h) for h in hist] == [2, 2, 2] and all(h == [1.0, 1.0] for h in hist)
    assert np.array_equal(x, np.full(4, 2.0 + 110.0 + 300.0))
    order = []
    for st in seen:
        if not order or order[-1] != st:
            order.append(st)
    assert order == stages
