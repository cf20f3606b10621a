"""The optimisation loop's host logic (paper_1612_04929_gb300.optimize) on the CPU: the same loop
that drives the GPU evaluation, here driven by the CPU FP64 oracle through a stand-in with the
Context interface.  Both methods reduce the gate infidelity of the two-qubit CNOT problem to the
target, and the returned controls are the ones whose cost was reported."""
import numpy as np
import pytest

import synthetic as sy
from oracle import qoc_oracle as orc
from paper_1612_04929_gb300.optimize import optimize


class OracleContext:
    """The evaluate() of Context, computed by the oracle (test stand-in; no GPU)."""

    def __init__(self, prob):
        self.prob = prob

    def evaluate(self, u):
        return orc.cost_and_grad(self.prob, u)


@pytest.mark.parametrize("method,kw", [("lbfgs", {}), ("adam", {"lr": 0.01})])
def test_optimizer_reaches_target_on_cnot(method, kw):
    prob = sy.cnot2q(N=40)
    ctx = OracleContext(prob)
    c0, _, t0 = orc.cost_and_grad(prob, prob.u)
    r = optimize(ctx, prob.u, method=method, max_iter=400, target_infidelity=1e-3, **kw)
    assert t0[0] > 0.1 and r.reached, (t0[0], r.terms[0], r.evaluations)
    c, _, terms = orc.cost_and_grad(prob, r.u)
    assert abs(c - r.cost) <= 1e-12 and terms[0] <= 1e-3
    assert r.evaluations == len(r.history) and r.history[-1][2] <= 1e-3


def test_optimizer_rejects_unknown_method():
    prob = sy.cnot2q(N=4)
    with pytest.raises(ValueError):
        optimize(OracleContext(prob), prob.u, method="sgd")
