"""The evaluation entry point that allocates no memory (qoc_evaluate_static), checked against
the regular context-based entry point on the same inputs, on two calls in a row.

Callers that may not allocate when they evaluate (stream capture, real-time loops, pooled
memory) use this entry point; it keeps every intermediate in one fixed device array that all
calls share, so the second call must not see anything the first call left behind.  This file
is collected last so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

import synthetic as sy

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the FP64 tolerance of the parity tests


@pytest.mark.parametrize("case", [dict(d=8, M=3, N=60, S=3, seed=901, nF=2),
                                  dict(d=44, M=2, N=12, S=41, seed=903, nF=3)],   # 8-column panels padded
                         ids=["d8S3", "d44S41"])                                   # past the d x d slot
def test_static_entry_point_matches_context_entry_point_twice(case):
    import torch
    from paper_1612_04929_gb300 import Context, build, qoc_evaluate_static

    build.build()
    prob = sy.random_problem(**case, dt=0.2, u_scale=0.8)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)

    def tensor_c128(a):
        return torch.from_numpy(np.ascontiguousarray(a, np.complex128)).to(dev)

    H0 = tensor_c128(prob.H0)
    Hk = tensor_c128(prob.Hk)
    psi0 = tensor_c128(prob.psi0)
    psiT = tensor_c128(prob.psiT)
    fmask = torch.zeros(prob.d, dtype=torch.int32, device=dev)
    fmask[torch.from_numpy(prob.forbidden.astype(np.int64))] = 1
    grad = torch.empty((prob.M, prob.N), dtype=torch.float64, device=dev)
    out = torch.empty(6, dtype=torch.float64, device=dev)

    rng = np.random.default_rng(902)
    controls = [prob.u, prob.u + 0.3 * rng.standard_normal(prob.u.shape)]   # two calls in a row
    with Context("fp64") as ctx:
        ctx.set_problem(prob)
        for u_np in controls:
            c_ref, g_ref, t_ref = ctx.evaluate(u_np)
            u = torch.from_numpy(np.ascontiguousarray(u_np)).to(dev)
            grad.fill_(np.nan)
            out.fill_(np.nan)
            stream = torch.cuda.current_stream().cuda_stream
            qoc_evaluate_static(prob.d, prob.M, prob.N, prob.S, prob.dt, H0.data_ptr(), Hk.data_ptr(),
                                u.data_ptr(), psi0.data_ptr(), psiT.data_ptr(), fmask.data_ptr(),
                                prob.alpha, grad.data_ptr(), out.data_ptr(), stream)
            torch.cuda.synchronize()
            o = out.cpu().numpy()
            g = grad.cpu().numpy()
            assert abs(o[0] - c_ref) <= TOL * abs(c_ref)
            assert np.max(np.abs(o[1:] - t_ref) / np.maximum(np.abs(t_ref), 1.0)) <= TOL
            assert np.linalg.norm(g - g_ref) <= TOL * np.linalg.norm(g_ref)


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
