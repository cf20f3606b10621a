"""The evaluation entry point that allocates no memory (qoc_evaluate_static), checked against
the CPU FP64 oracle and against the regular context-based entry point on the same inputs, on
several calls in a row.

Callers that may not allocate when they evaluate (stream capture, real-time loops, pooled
memory) use this entry point; it keeps every intermediate in one fixed device array that all
calls share, so no call may see anything an earlier call left behind, even when the shape
changes between calls.  This file is collected last so that a run stopping at the first
failure has run every other test."""
import numpy as np
import pytest

import synthetic as sy
from oracle import qoc_oracle as orc

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the FP64 tolerance of the parity tests


class Static:
    """Device copies of one problem's inputs and outputs for qoc_evaluate_static."""

    def __init__(self, prob):
        import torch
        self.torch = torch
        self.prob = prob
        self.dev = torch.device("cuda", 0)
        torch.cuda.set_device(self.dev)
        c128 = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.complex128)).to(self.dev)
        self.H0, self.Hk = c128(prob.H0), c128(prob.Hk)
        self.psi0, self.psiT = c128(prob.psi0), c128(prob.psiT)
        self.fmask = torch.zeros(prob.d, dtype=torch.int32, device=self.dev)
        self.fmask[torch.from_numpy(prob.forbidden.astype(np.int64))] = 1
        self.grad = torch.empty((prob.M, prob.N), dtype=torch.float64, device=self.dev)
        self.out = torch.empty(6, dtype=torch.float64, device=self.dev)

    def __call__(self, u_np, sync=True):
        from paper_1612_04929_gb300 import qoc_evaluate_static
        torch, p = self.torch, self.prob
        self.u = torch.from_numpy(np.ascontiguousarray(u_np)).to(self.dev)
        self.grad.fill_(np.nan)
        self.out.fill_(np.nan)
        qoc_evaluate_static(p.d, p.M, p.N, p.S, p.dt, self.H0.data_ptr(), self.Hk.data_ptr(), self.u.data_ptr(),
                            self.psi0.data_ptr(), self.psiT.data_ptr(), self.fmask.data_ptr(), p.alpha,
                            self.grad.data_ptr(), self.out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        if sync:
            torch.cuda.synchronize()
            return self.out.cpu().numpy(), self.grad.cpu().numpy()


def assert_close(o, g, c_ref, g_ref, t_ref):
    assert abs(o[0] - c_ref) <= TOL * abs(c_ref), (o[0], c_ref)
    assert np.max(np.abs(o[1:] - t_ref) / np.maximum(np.abs(t_ref), 1.0)) <= TOL
    assert np.linalg.norm(g - g_ref) <= TOL * np.linalg.norm(g_ref)


@pytest.mark.parametrize("case", [dict(d=8, M=3, N=60, S=3, seed=901, nF=2),
                                  dict(d=44, M=2, N=12, S=41, seed=903, nF=3)],   # 8-column panels padded
                         ids=["d8S3", "d44S41"])                                   # past the d x d slot
def test_static_entry_point_matches_oracle_and_context_twice(case):
    from paper_1612_04929_gb300 import Context, build

    build.build()
    prob = sy.random_problem(**case, dt=0.2, u_scale=0.8)
    st = Static(prob)
    rng = np.random.default_rng(902)
    controls = [prob.u, prob.u + 0.3 * rng.standard_normal(prob.u.shape)]   # two calls in a row
    with Context("fp64") as ctx:
        ctx.set_problem(prob)
        for u_np in controls:
            o, g = st(u_np)
            c_ref, g_ref, t_ref = orc.cost_and_grad(prob, u_np)   # the oracle
            assert_close(o, g, c_ref, g_ref, t_ref)
            c1, g1, t1 = ctx.evaluate(u_np)                        # the context entry point
            assert_close(o, g, c1, g1, t1)


def test_static_entry_point_survives_shape_changes():
    """Calls with different (d, S) on one stream, back to back without synchronising: the
    arena's layout (panel width, padding, offsets) changes between them, so the padding columns,
    carries and masks must be cleared by each call.  Each result is checked against the oracle."""
    from paper_1612_04929_gb300 import build

    build.build()
    big = sy.random_problem(d=44, M=2, N=12, S=41, seed=911, nF=3, dt=0.2, u_scale=0.8)
    small = sy.random_problem(d=8, M=3, N=30, S=3, seed=912, nF=0, dt=0.2, u_scale=0.8)
    runs = [Static(big), Static(small), Static(big)]
    us = [big.u, small.u, big.u + 0.1]
    for r, u in zip(runs, us):
        r(u, sync=False)
    runs[0].torch.cuda.synchronize()
    # the first call's outputs stay valid: they live in the caller's buffers, not in the arena
    for r, u in zip(runs, us):
        o, g = r.out.cpu().numpy(), r.grad.cpu().numpy()
        c_ref, g_ref, t_ref = orc.cost_and_grad(r.prob, u)
        assert_close(o, g, c_ref, g_ref, t_ref)


def test_static_entry_point_runs_the_largest_admitted_size():
    """d = 48, S = 1: the largest N that the header's bound admits (441 slices) fits the array
    and evaluates correctly."""
    from paper_1612_04929_gb300 import build

    build.build()
    prob = sy.random_problem(d=48, M=2, N=441, S=1, seed=913, nF=2, dt=0.2, u_scale=0.8)
    o, g = Static(prob)(prob.u)
    c_ref, g_ref, t_ref = orc.cost_and_grad(prob, prob.u)
    assert_close(o, g, c_ref, g_ref, t_ref)


def test_static_entry_point_marks_a_device_side_failure_with_nan():
    """A NaN control cannot be seen by the host in device memory: the call returns QOC_OK and
    the cost comes back as NaN.  The next call with valid controls is correct again."""
    from paper_1612_04929_gb300 import build

    build.build()
    prob = sy.random_problem(d=6, M=2, N=20, S=2, seed=914, nF=1, dt=0.2, u_scale=0.8)
    st = Static(prob)
    bad = prob.u.copy()
    bad[1, 7] = np.nan
    o, _ = st(bad)
    assert np.isnan(o[0])
    o, g = st(prob.u)
    c_ref, g_ref, t_ref = orc.cost_and_grad(prob, prob.u)
    assert_close(o, g, c_ref, g_ref, t_ref)


def test_static_entry_point_rejects_oversized_problems():
    from paper_1612_04929_gb300 import QocError, build, qoc_evaluate_static
    build.build()
    with pytest.raises(QocError) as e:     # d beyond the FP64 per-slice kernels
        qoc_evaluate_static(49, 0, 4, 1, 0.1, 1, 0, 0, 1, 1, 0, [1, 0, 0, 0, 0], 0, 1)
    assert e.value.status == 2
    with pytest.raises(QocError) as e:     # N * d^2 beyond the fixed array
        qoc_evaluate_static(48, 0, 20000, 1, 0.1, 1, 0, 0, 1, 1, 0, [1, 0, 0, 0, 0], 0, 1)
    assert e.value.status == 2


def test_static_entry_point_replays_from_a_cuda_graph():
    """Captured once in a CUDA graph (where allocation is not permitted) and replayed with new
    controls written into the same device buffer: each replay matches the context evaluation."""
    import torch
    from paper_1612_04929_gb300 import Context, build, qoc_evaluate_static

    build.build()
    prob = sy.random_problem(d=6, M=2, N=40, S=2, seed=905, nF=1, dt=0.2, u_scale=0.8)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)

    def c128(a):
        return torch.from_numpy(np.ascontiguousarray(a, np.complex128)).to(dev)

    H0, Hk, psi0, psiT = c128(prob.H0), c128(prob.Hk), c128(prob.psi0), c128(prob.psiT)
    fmask = torch.zeros(prob.d, dtype=torch.int32, device=dev)
    fmask[torch.from_numpy(prob.forbidden.astype(np.int64))] = 1
    u = torch.from_numpy(np.ascontiguousarray(prob.u)).to(dev)
    grad = torch.empty((prob.M, prob.N), dtype=torch.float64, device=dev)
    out = torch.empty(6, dtype=torch.float64, device=dev)
    side = torch.cuda.Stream()

    def call():
        qoc_evaluate_static(prob.d, prob.M, prob.N, prob.S, prob.dt, H0.data_ptr(), Hk.data_ptr(), u.data_ptr(),
                            psi0.data_ptr(), psiT.data_ptr(), fmask.data_ptr(), prob.alpha, grad.data_ptr(),
                            out.data_ptr(), torch.cuda.current_stream().cuda_stream)

    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        call()                                   # first use outside the capture
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        call()
    rng = np.random.default_rng(906)
    with Context("fp64") as ctx:
        ctx.set_problem(prob)
        for u_np in (prob.u, prob.u + 0.3 * rng.standard_normal(prob.u.shape)):
            u.copy_(torch.from_numpy(np.ascontiguousarray(u_np)))
            graph.replay()
            torch.cuda.synchronize()
            c_ref, g_ref, _ = ctx.evaluate(u_np)
            assert abs(out[0].item() - c_ref) <= TOL * abs(c_ref)
            assert np.linalg.norm(grad.cpu().numpy() - g_ref) <= TOL * np.linalg.norm(g_ref)
