"""The Paterson-Stockmeyer evaluation of the Taylor polynomial (the default on the FP32 per-slice
path, d <= 57, and on the FP32 / BF16_SPLIT batched path) against the CPU FP64 oracle: at forced
(p, n) against the oracle's derivative of the truncated series itself (every residue of p mod 3,
the degenerate orders p = 1, 2, 3), with the dense and the low-rank reverse modes, the block
recursion when no operands are stored, and the first-order gradient; and against the Horner form
of the same polynomial."""
import numpy as np
import pytest

import synthetic as sy
from oracle import qoc_oracle as orc
from test_gpu_parity import check, rel, run

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1612_04929_gb300 import build
    build.build()


def against_truncated_series(prob, precision, p, n, **opt):
    cost, grad, terms, info = run(prob, precision, p_override=p, n_override=n, **opt)
    assert (info["p"], info["n"]) == (p, n) and info["taylor_scheme"] == 1
    c_t, g_t, _ = orc.taylor_cost_and_grad(prob, prob.u, p, n)
    assert abs(cost - c_t) <= TOL * abs(c_t), (cost, c_t)
    assert rel(grad, g_t) <= TOL, rel(grad, g_t)
    return info


@pytest.mark.parametrize("pn", [(1, 3), (2, 2), (3, 2), (4, 1), (5, 2), (6, 0), (7, 2), (12, 0), (14, 2), (16, 1)])
def test_per_slice_forced_orders_dense(pn):
    """Per-slice kernels, dense reverse mode (S = 3 columns: rank 3 2^n is too large for the
    low-rank form at d = 9)."""
    prob = sy.random_problem(d=9, M=2, N=21, S=3, seed=401, nF=2, path=True, E=2, dt=0.2, u_scale=0.8)
    info = against_truncated_series(prob, "fp32", *pn)
    assert info["kernel_path"] == 0 and info["adjoint_form"] == 0


@pytest.mark.parametrize("pn", [(3, 0), (5, 1), (9, 1), (13, 2)])
def test_per_slice_forced_orders_low_rank(pn):
    """Per-slice kernels, low-rank reverse mode (S = 1 at d = 40: rank 2^n <= 5)."""
    prob = sy.random_problem(d=40, M=2, N=13, S=1, seed=402, nF=3, dt=0.1, u_scale=0.8)
    info = against_truncated_series(prob, "fp32", *pn)
    assert info["adjoint_form"] == 3


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("pn", [(2, 1), (3, 0), (8, 1), (12, 0)])
def test_batched_forced_orders(precision, pn):
    """The batched path (d = 70 > 68): products as batched GEMMs with the block added in the
    epilogue; BF16_SPLIT runs the reverse mode's products on the tensor cores."""
    prob = sy.random_problem(d=70, M=2, N=6, S=2, seed=403, nF=2, dt=0.05, u_scale=0.8)
    info = against_truncated_series(prob, precision, *pn)
    assert info["kernel_path"] == 1 and info["adjoint_form"] == 0


@pytest.mark.parametrize("pn", [(2, 1), (3, 0), (4, 2), (8, 1), (12, 0)])
def test_batched_tensor_core_forward_forced_orders(pn):
    """BF16_SPLIT from d = 128: the forward's products on the tensor cores (six seven-bit slices,
    two exact levels), 130 = 128 + 2 rows and 2 x 64 + 2 columns of tiles: every tile edge ragged."""
    prob = sy.random_problem(d=130, M=2, N=4, S=2, seed=410, nF=2, dt=0.03, u_scale=0.8)
    info = against_truncated_series(prob, "bf16", *pn)
    assert info["kernel_path"] == 1 and info["adjoint_form"] == 0


@pytest.mark.parametrize("d", [9, 40, 70])
def test_default_orders_match_oracle_and_horner(d):
    """Default (p, n) (theta_max 2): the oracle bar, and the Horner form of the same polynomial
    within FP32 rounding of each other."""
    prob = sy.random_problem(d=d, M=2, N=30 if d < 64 else 8, S=1 if d == 40 else 2, seed=404 + d, nF=2,
                             dt=0.2, u_scale=0.8)
    cost, grad, terms, info = check(prob, "fp32")
    assert info["taylor_scheme"] == 1
    p, n = info["p"], info["n"]
    c_h, g_h, _, info_h = run(prob, "fp32", taylor_scheme="horner", p_override=p, n_override=n)
    assert info_h["taylor_scheme"] == 0 and (info_h["p"], info_h["n"]) == (p, n)
    assert abs(cost - c_h) <= 2e-6 * abs(c_h) and rel(grad, g_h) <= 2e-6


def test_recompute_adjoint_with_ps_forward():
    """No stored operands (adjoint = recompute): the block recursion differentiates the same
    polynomial that the Paterson-Stockmeyer forward evaluated."""
    prob = sy.random_problem(d=12, M=3, N=25, S=2, seed=405, nF=2, path=True, dt=0.2, u_scale=0.8)
    cost, grad, terms, info = check(prob, "fp32", adjoint="recompute")
    assert info["taylor_scheme"] == 1 and info["adjoint_form"] == 1


def test_first_order_gradient_with_ps_forward():
    prob = sy.random_problem(d=12, M=3, N=25, S=2, seed=406, nF=2, dt=0.2, u_scale=0.8)
    c1, g1, _, info = run(prob, "fp32", gradient="first_order")
    c_ref, g_ref, _ = orc.cost_and_grad(prob, prob.u, exact=False)
    assert info["taylor_scheme"] == 1
    assert abs(c1 - c_ref) <= TOL * abs(c_ref) and rel(g1, g_ref) <= TOL


def test_scheme_reporting():
    """Horner where the form is not built: FP64, plain FP32 exponentials, TF32_SPLIT, and d above
    the per-slice form's shared-memory limit but within the per-slice path."""
    small = sy.random_problem(d=6, M=1, N=5, S=1, seed=407, nF=1)
    assert run(small, "fp64")[3]["taylor_scheme"] == 0
    assert run(small, "fp32", plain_fp32_exp=True)[3]["taylor_scheme"] == 0
    assert run(small, "fp32", taylor_scheme="horner")[3]["taylor_scheme"] == 0
    mid = sy.random_problem(d=64, M=1, N=4, S=1, seed=408, nF=1)
    info = check(mid, "fp32")[3]
    assert info["kernel_path"] == 0 and info["taylor_scheme"] == 0
    big = sy.random_problem(d=70, M=1, N=3, S=1, seed=409, nF=1)
    assert run(big, "tf32")[3]["taylor_scheme"] == 0


# ------------------------------------------------------------------ autotuner
def test_autotune_chooses_a_configuration_and_caches_it():
    """qoc_options.autotune: the candidates (Taylor scheme, theta_max x {1/2, 1, 2}, sweep form, and
    on the per-slice path the split into two waves) are timed on the caller's inputs; whichever wins,
    the result meets the oracle bar, and a second context of the same shape takes the cached choice
    without timing and gives the same numbers."""
    prob = sy.random_problem(d=12, M=2, N=40, S=2, seed=411, nF=2, path=True, E=2, dt=0.2, u_scale=0.8)
    cost, grad, terms, info = check(prob, "fp32", autotune=True)
    assert info["autotune_candidates"] >= 6
    c2, g2, _, info2 = run(prob, "fp32", autotune=True)
    assert info2["autotune_candidates"] == 0
    assert c2 == cost and np.array_equal(g2, grad)


def test_autotune_batched_path_and_graph_replay():
    """The batched path under BF16_SPLIT, and a graph-replayed per-slice context (tuned before the
    capture)."""
    big = sy.random_problem(d=70, M=2, N=8, S=2, seed=412, nF=2, dt=0.05, u_scale=0.8)
    info = check(big, "bf16", autotune=True)[3]
    assert info["kernel_path"] == 1 and info["autotune_candidates"] >= 4
    from paper_1612_04929_gb300 import Context
    import torch
    small = sy.random_problem(d=8, M=2, N=30, S=1, seed=413, nF=1, dt=0.2)
    c_ref, g_ref, _ = orc.cost_and_grad(small, small.u)
    u = torch.tensor(small.u, dtype=torch.float64, device="cuda")
    g = torch.empty_like(u)
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    with Context("fp32", autotune=True, graph=True) as c:
        c.set_problem(small)
        for _ in range(2):
            c.evaluate_device(u.data_ptr(), g.data_ptr(), out.data_ptr())
        c.sync()
        assert c.info()["autotune_candidates"] >= 1
    assert abs(float(out[0]) - c_ref) <= TOL * abs(c_ref) and rel(g.cpu().numpy(), g_ref) <= TOL
