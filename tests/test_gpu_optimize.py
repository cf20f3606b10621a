"""The optimisation loop over the GPU evaluation (Sec. II.B; the CNOT of Sec. V.A): L-BFGS-B
with the exact gradient of the CUDA path drives two coupled five-level transmons from small
random controls to a CNOT with infidelity <= 1e-3 (99.9 % fidelity, the paper's convergence
criterion), with the forbidden-level, amplitude and variation penalties on.  The final controls
are checked against the CPU FP64 oracle."""
import numpy as np
import pytest

import synthetic as sy
from oracle import qoc_oracle as orc

pytestmark = pytest.mark.gpu


def test_transmon_cnot_reaches_999_fidelity():
    from paper_1612_04929_gb300 import Context, build
    from paper_1612_04929_gb300.optimize import optimize
    build.build()
    prob = sy.transmon_cnot()
    with Context("fp64") as ctx:
        ctx.set_problem(prob)
        r = optimize(ctx, prob.u, method="lbfgs", max_iter=3000, target_infidelity=1e-3)
    assert r.reached, (r.terms, r.iterations)
    c_ref, _, t_ref = orc.cost_and_grad(prob, r.u)
    assert abs(r.cost - c_ref) <= 1e-10 * abs(c_ref) and t_ref[0] <= 1e-3


def test_adam_lowers_the_cost():
    from paper_1612_04929_gb300 import Context, build
    from paper_1612_04929_gb300.optimize import optimize
    build.build()
    prob = sy.cnot2q()
    with Context("fp64") as ctx:
        ctx.set_problem(prob)
        r = optimize(ctx, prob.u, method="adam", lr=0.01, max_iter=500, target_infidelity=1e-3)
    assert r.reached and r.history[0][1] > 10 * r.cost
