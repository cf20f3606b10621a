"""The batched evaluation of many independent problems of uneven (d, N, M, E) in one call
(qoc_evaluate_batch): each problem against the CPU FP64 oracle, and the batch against the
one-problem-at-a-time evaluation of the same contexts (same kernels: identical results)."""
import numpy as np
import pytest

import synthetic as sy
from oracle import qoc_oracle as orc
from test_gpu_parity import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1612_04929_gb300 import build
    build.build()


def _run_batch(probs, precision="fp32"):
    import torch
    from paper_1612_04929_gb300 import Context, qoc_evaluate_batch
    ctxs = [Context(precision) for _ in probs]
    for c, p in zip(ctxs, probs):
        c.set_problem(p)
    us = [torch.tensor(p.u, dtype=torch.float64, device="cuda") for p in probs]
    gs = [torch.empty_like(u) for u in us]
    outs = [torch.empty(6, dtype=torch.float64, device="cuda") for _ in probs]
    stream = torch.cuda.current_stream().cuda_stream
    qoc_evaluate_batch(ctxs, [u.data_ptr() for u in us], [g.data_ptr() for g in gs], [o.data_ptr() for o in outs],
                       stream)
    torch.cuda.synchronize()
    res = [(o.cpu().numpy(), g.cpu().numpy()) for o, g in zip(outs, gs)]
    single = [c.evaluate(p.u) for c, p in zip(ctxs, probs)]
    for c in ctxs:
        c.close()
    return res, single


def test_batch_of_uneven_problems_matches_oracle():
    probs = [sy.batch_problem(i, ensemble=(4 if i % 3 == 0 else 1), n_range=(12, 30)) for i in range(9)]
    assert len({p.d for p in probs}) >= 3
    res, single = _run_batch(probs)
    for p, (o, g), (c1, g1, t1) in zip(probs, res, single):
        c_ref, g_ref, t_ref = orc.cost_and_grad(p, p.u)
        assert abs(o[0] - c_ref) <= 1e-5 * abs(c_ref), p.name
        assert rel(g, g_ref) <= 1e-5, p.name
        assert o[0] == c1 and np.array_equal(g, g1), p.name      # batch == one at a time


def test_batch_fp64_small():
    probs = [sy.random_problem(d=d, M=2, N=9, S=2, seed=700 + d, nF=1, E=2) for d in (3, 8, 20, 50)]
    res, single = _run_batch(probs, "fp64")
    for p, (o, g), _ in zip(probs, res, single):
        c_ref, g_ref, _ = orc.cost_and_grad(p, p.u)
        assert abs(o[0] - c_ref) <= 1e-10 * abs(c_ref) and rel(g, g_ref) <= 1e-10
