"""State mode (the paper's Eq. 12): the truncated series applied to the propagated columns by
Horner matrix-vector products, without forming U_j, against the CPU FP64 oracle (<= 1e-10 FP64,
<= 1e-5 FP32), against the oracle's derivative of the truncated series at forced (p, n), and
against the unitary form (the same truncated map evaluated in another order); the cat-state
workload of Sec. V.C (d = 154, 8000 slices) at reduced and at full length."""
import numpy as np
import pytest

import synthetic as sy
from oracle import qoc_oracle as orc
from test_gpu_parity import check, rel, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1612_04929_gb300 import build
    build.build()


STATE_CASES = [
    dict(d=3, M=2, N=17, S=1, seed=171, nF=1),
    dict(d=9, M=3, N=40, S=3, seed=172, nF=2, path=True, E=2),
    dict(d=24, M=2, N=31, S=2, seed=173, nF=3, E=3, weights=True),
    dict(d=40, M=2, N=50, S=1, seed=174, nF=13),
    dict(d=70, M=2, N=12, S=5, seed=175, nF=4),     # larger than the per-slice unitary kernels
    dict(d=120, M=2, N=6, S=2, seed=176, nF=2),     # X_j read from L2 (no room in shared memory)
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", STATE_CASES, ids=lambda c: f"d{c['d']}S{c['S']}N{c['N']}")
def test_state_mode_matches_oracle(case, precision):
    if precision == "fp64" and case["d"] > 70:
        pytest.skip("FP64 at d = 120 is covered by the FP32 case")
    prob = sy.random_problem(**case, dt=0.2, u_scale=0.8)
    cost, grad, terms, info = check(prob, precision, propagation="state")
    assert info["kernel_path"] == 2 and info["adjoint_form"] == 4


@pytest.mark.parametrize("pn", [(3, 1), (9, 0), (6, 3)])
def test_state_mode_differentiates_the_series_exactly(pn):
    """Forced (p, n): the state-mode gradient is the exact derivative of the truncated map."""
    p, n = pn
    prob = sy.random_problem(d=7, M=2, N=15, S=2, seed=177, nF=2, path=True, E=2, dt=0.2)
    cost, grad, terms, info = run(prob, "fp64", propagation="state", p_override=p, n_override=n)
    assert (info["p"], info["n"]) == (p, n)
    c_t, g_t, _ = orc.taylor_cost_and_grad(prob, prob.u, p, n)
    assert abs(cost - c_t) <= 1e-12 * abs(c_t)
    assert rel(grad, g_t) <= 1e-11


def test_state_mode_equals_unitary_mode_fp64():
    """The same truncated map, evaluated in another order: FP64 results agree to rounding."""
    prob = sy.random_problem(d=12, M=3, N=60, S=3, seed=178, nF=2, path=True, E=2, dt=0.2)
    a = run(prob, "fp64", propagation="state")
    b = run(prob, "fp64")
    assert (a[3]["p"], a[3]["n"]) != (0, 0)
    assert abs(a[0] - b[0]) <= 1e-12 * abs(b[0]) and rel(a[1], b[1]) <= 1e-11


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_state_mode_waves_and_first_order(precision):
    """Several waves (states regenerated from the wave checkpoints), and the paper's first-order
    gradient (Eq. 11) on the state-mode recursions."""
    prob = sy.random_problem(d=10, M=2, N=29, S=2, seed=179, nF=2, path=True, E=2, dt=0.2, u_scale=0.8)
    cost, grad, terms, info = check(prob, precision, propagation="state", wave_slices=7)
    assert info["n_waves"] == 5
    tol = 1e-10 if precision == "fp64" else 1e-5
    c1, g1, _, _ = run(prob, precision, propagation="state", gradient="first_order")
    c_ref, g_ref, _ = orc.cost_and_grad(prob, prob.u, exact=False)
    assert abs(c1 - c_ref) <= tol * abs(c_ref) and rel(g1, g_ref) <= tol


def test_state_mode_rejects_many_columns():
    from paper_1612_04929_gb300 import QocError
    prob = sy.random_problem(d=12, M=2, N=4, S=9, seed=180, nF=1)
    with pytest.raises(QocError) as e:
        run(prob, "fp32", propagation="state")
    assert e.value.status == 9                       # QOC_ERR_UNSUPPORTED


def test_cat_state_reduced_N():
    """The first 1000 of the cat-state workload's 8000 slices, FP32 state mode and FP32 unitary
    form, both against the oracle."""
    prob = sy.cat_state(N=1000)
    cost, grad, terms, info = check(prob, "fp32", propagation="state")
    assert info["kernel_path"] == 2
    check(prob, "fp32")


def test_cat_state_full_size_sampled():
    """The cat-state workload at full length (N = 8000) in FP32 state mode: the cost, and the
    gradient at every 400th slice, against the oracle (whose costate sweep covers every slice)."""
    prob = sy.cat_state()
    cost, grad, terms, info = run(prob, "fp32", propagation="state")
    cols = list(range(0, 8000, 400)) + [7999]
    c_ref, g_ref, _ = orc.cost_and_grad(prob, prob.u, slices=cols)
    assert abs(cost - c_ref) <= 1e-5 * abs(c_ref)
    assert rel(grad[:, cols], g_ref[:, cols]) <= 1e-5


# ------------------------------------------------------------------ Chebyshev expansion (state mode)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", STATE_CASES[:5], ids=lambda c: f"d{c['d']}S{c['S']}N{c['N']}")
def test_chebyshev_state_mode_matches_oracle(case, precision):
    """The Chebyshev expansion of exp(-i dt H_j) (no scaling) in place of the Taylor series: the
    degree is the least whose tail bound meets tol, and cost and gradient meet the oracle."""
    if precision == "fp64" and case["d"] > 40:
        pytest.skip("FP64 at d = 70: the gradient kernel's K + 6 blocks of 70 x 5 exceed shared memory")
    prob = sy.random_problem(**case, dt=0.04, u_scale=0.8)     # theta a few units per slice
    cost, grad, terms, info = check(prob, precision, propagation="state", exponential="chebyshev")
    theta = orc.theta_bound(prob, prob.u)
    assert info["n"] == 0 and theta < info["p"] <= theta + 40


def test_chebyshev_needs_state_mode():
    from paper_1612_04929_gb300 import Context, QocError
    with pytest.raises(QocError) as e:
        Context("fp32", exponential="chebyshev")
    assert e.value.status == 9


def test_chebyshev_cat_state_reduced_N():
    """The cat-state system (theta ~ 3.2 per slice): degree ~13 instead of p 2^n = 40 matrix-vector
    products for the Taylor series at theta_max = 1."""
    prob = sy.cat_state(N=1000)
    cost, grad, terms, info = check(prob, "fp32", propagation="state", exponential="chebyshev")
    assert info["p"] <= 16
