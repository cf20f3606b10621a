"""The batch captured into one CUDA graph (qoc_batch_create / qoc_batch_launch): replays equal
the plain batched evaluation bit for bit, follow controls rewritten in place (against the CPU
FP64 oracle), report controls that outgrow the frozen Taylor orders (QOC_ERR_STALE), and hold
their contexts until the batch is destroyed."""
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


def _problems():
    # d in {4, 8, 16, 40} on the per-slice path, 81 and 128 on the batched large-d path
    probs = [sy.batch_problem(i, ensemble=(2 if i % 3 == 0 else 1), n_range=(12, 30)) for i in range(9)]
    probs.append(sy.batch_problem(20, d_choices=(128,), n_range=(12, 30)))
    assert {81, 128} <= {p.d for p in probs} and min(p.d for p in probs) <= 16
    return probs


class _Setup:
    def __init__(self, probs):
        import torch
        from paper_1612_04929_gb300 import Context
        self.probs = probs
        self.ctxs = [Context("fp32") for _ in probs]
        for c, p in zip(self.ctxs, probs):
            c.set_problem(p)
        self.us = [torch.tensor(p.u, dtype=torch.float64, device="cuda") for p in probs]
        self.gs = [torch.empty_like(u) for u in self.us]
        self.outs = [torch.empty(6, dtype=torch.float64, device="cuda") for _ in probs]
        self.stream = torch.cuda.current_stream().cuda_stream

    def ptrs(self):
        return ([u.data_ptr() for u in self.us], [g.data_ptr() for g in self.gs], [o.data_ptr() for o in self.outs])

    def results(self):
        import torch
        torch.cuda.synchronize()
        return [(o.cpu().numpy().copy(), g.cpu().numpy().copy()) for o, g in zip(self.outs, self.gs)]

    def close(self):
        for c in self.ctxs:
            c.close()


def test_captured_batch_replays_the_plain_batch_bit_for_bit():
    from paper_1612_04929_gb300 import Batch, qoc_evaluate_batch
    s = _Setup(_problems())
    qoc_evaluate_batch(s.ctxs, *s.ptrs(), s.stream)
    plain = s.results()
    paths = [c.info()["kernel_path"] for c in s.ctxs]
    assert 0 in paths and 1 in paths
    with Batch(s.ctxs, *s.ptrs(), s.stream) as b:
        first = s.results()                       # the evaluation that qoc_batch_create runs
        for o, g in zip(s.outs, s.gs):
            o.zero_()
            g.zero_()
        for _ in range(2):
            b.launch(s.stream)
        b.sync()
        replay = s.results()
    for p, (o0, g0), (o1, g1), (o2, g2) in zip(s.probs, plain, first, replay):
        assert np.array_equal(o0, o1) and np.array_equal(g0, g1), p.name
        assert np.array_equal(o0, o2) and np.array_equal(g0, g2), p.name
    for i in (2, 7, 9):                           # d = 81, 40, 128 against the oracle
        p = s.probs[i]
        c_ref, g_ref, _ = orc.cost_and_grad(p, p.u)
        assert abs(replay[i][0][0] - c_ref) <= 1e-5 * abs(c_ref) and rel(replay[i][1], g_ref) <= 1e-5, p.name
    s.close()


def test_captured_batch_follows_controls_rewritten_in_place():
    import torch
    from paper_1612_04929_gb300 import Batch
    s = _Setup(_problems())
    rng = np.random.default_rng(11)
    with Batch(s.ctxs, *s.ptrs(), s.stream) as b:
        new_u = []
        for u in s.us:       # smaller amplitudes: the frozen orders still cover them
            v = u.cpu().numpy() * rng.uniform(0.5, 0.9, size=u.shape)
            u.copy_(torch.from_numpy(v))
            new_u.append(v)
        b.launch(s.stream)
        b.sync()
        res = s.results()
    for i in (1, 2, 5, 7, 9):
        p = s.probs[i]
        c_ref, g_ref, _ = orc.cost_and_grad(p, new_u[i])
        assert abs(res[i][0][0] - c_ref) <= 1e-5 * abs(c_ref) and rel(res[i][1], g_ref) <= 1e-5, p.name
    s.close()


def test_controls_beyond_the_frozen_orders_are_reported_stale():
    import torch
    from paper_1612_04929_gb300 import Batch, QocError
    probs = _problems()
    idx = [i for i, p in enumerate(probs) if p.d >= 81]
    s = _Setup(probs)
    b = Batch(s.ctxs, *s.ptrs(), s.stream)
    k = idx[0]
    s.us[k].mul_(2.5)                  # theta grows past the frozen (p, n): flagged, not faulted
    b.launch(s.stream)
    with pytest.raises(QocError, match="QOC_ERR_STALE"):
        b.sync()
    b.close()
    # unfrozen, the same context picks new orders and matches the oracle again
    torch.cuda.synchronize()
    u = s.us[k].cpu().numpy()
    cost, grad, _ = s.ctxs[k].evaluate(u)
    c_ref, g_ref, _ = orc.cost_and_grad(probs[k], u)
    assert abs(cost - c_ref) <= 1e-5 * abs(c_ref) and rel(grad, g_ref) <= 1e-5
    s.close()


def test_batch_holds_its_contexts():
    from paper_1612_04929_gb300 import Batch, Context, QocError
    probs = _problems()[:3]
    s = _Setup(probs)
    b = Batch(s.ctxs, *s.ptrs(), s.stream)
    with pytest.raises(QocError, match="QOC_ERR_STATE"):
        s.ctxs[0].set_problem(probs[0])
    with pytest.raises(QocError, match="QOC_ERR_STATE"):
        s.ctxs[1].close()
    b.close()
    s.ctxs[0].set_problem(probs[0])   # released with the batch
    # state mode and profiled contexts pick their orders on the host or time on it: refused
    for kw in ({"propagation": "state"}, {"profile": True}):
        c = Context("fp32", **kw)
        c.set_problem(sy.batch_problem(1, n_range=(12, 30)))
        with pytest.raises(QocError, match="QOC_ERR_UNSUPPORTED"):
            Batch([c], *[x[1:2] for x in s.ptrs()], s.stream)
        c.close()
    s.close()


def test_destroying_a_held_context_is_deferred_to_the_batch():
    from paper_1612_04929_gb300 import Batch, qoc_destroy
    probs = _problems()[:3]
    s = _Setup(probs)
    b = Batch([c.handle for c in s.ctxs], *s.ptrs(), s.stream)
    before = s.results()
    h = s.ctxs[2].handle
    qoc_destroy(h)                     # deferred: the batch's graph still uses the context's buffers
    s.ctxs[2]._ctx = None
    b.launch(s.stream)
    b.sync()
    after = s.results()
    for (o0, g0), (o1, g1) in zip(before, after):
        assert np.array_equal(o0, o1) and np.array_equal(g0, g1)
    b.close()                          # frees the context
    s.close()
