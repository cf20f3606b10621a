"""The batched evaluation of many independent problems of uneven (d, N, M, E) in one call
(qoc_evaluate_batch): each problem against the CPU FP64 oracle, and the batch against the
one-problem-at-a-time evaluation of the same contexts (same kernels: identical results)."""
import os

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


def _run_batch(probs, precision="fp32", single=True):
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
    single = [c.evaluate(p.u) for c, p in zip(ctxs, probs)] if single else None
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


# ------------------------------------------------------------------ the batched sweep at full size
E32_SUBSET = (0, 1, 3, 5)     # d = 16, 4, 8 (per-slice kernels) and 81 (batched path), 32 members each


def _sampled_cols(N):
    """Every 100th slice and the last one."""
    return sorted(set(list(range(0, N, 100)) + [N - 1]))


def _oracle_sampled(job):
    """The oracle's cost and its gradient at the sampled slices of batch problem i with E members
    (its costate sweep covers every slice; only the per-slice contractions are sampled)."""
    i, E = job
    p = sy.batch_problem(i, ensemble=E)
    c, g, _ = orc.cost_and_grad(p, p.u, slices=_sampled_cols(p.N))
    return c, g


def test_batch_full_size_sampled():
    """The batched sweep as stated: all 128 problems (d in {4, 8, 16, 40, 81, 128}, N up to
    4000) in one qoc_evaluate_batch call, plus 32-member detuning ensembles on four of them in a
    second call, each against the oracle: the cost, and the gradient at every 100th slice.  The
    oracle references are computed by a spawned process pool while the GPU evaluates."""
    import multiprocessing as mp
    jobs = [(i, 1) for i in range(128)] + [(i, 32) for i in E32_SUBSET]
    jobs.sort(key=lambda j: -(sy.batch_problem(j[0]).N * sy.batch_problem(j[0]).d ** 2 * j[1]))  # longest first
    # one BLAS thread per worker (the workers are spawned with this environment), one worker per core
    threads = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({k: "1" for k in threads})
    try:
        pool = mp.get_context("spawn").Pool(max(1, os.cpu_count() or 1))
    finally:
        for k, v in threads.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    with pool:
        pending = pool.map_async(_oracle_sampled, jobs, chunksize=1)
        probs = [sy.batch_problem(i, ensemble=E) for i, E in
                 [(i, 1) for i in range(128)] + [(i, 32) for i in E32_SUBSET]]
        res1, _ = _run_batch(probs[:128], single=False)
        res32, _ = _run_batch(probs[128:], single=False)
        refs = pending.get(timeout=1500)
    assert sorted({p.d for p in probs}) == [4, 8, 16, 40, 81, 128] and max(p.N for p in probs) > 3900
    ref_of = dict(zip(jobs, refs))
    keys = [(i, 1) for i in range(128)] + [(i, 32) for i in E32_SUBSET]
    for p, (o, g), key in zip(probs, res1 + res32, keys):
        c_ref, g_ref = ref_of[key]
        cols = _sampled_cols(p.N)
        assert abs(o[0] - c_ref) <= 1e-5 * abs(c_ref), (p.name, p.E)
        assert rel(g[:, cols], g_ref[:, cols]) <= 1e-5, (p.name, p.E, rel(g[:, cols], g_ref[:, cols]))
