"""The seeded synthetic workloads are the configurations they are named for: sizes, time steps,
and physics read back from the operators (spectra, conserved quantities, targets), not from the
constants of the generator.  CPU only."""
import numpy as np
import pytest

import synthetic as sy

TWO_PI = 2 * np.pi


def herm(h):
    return np.max(np.abs(h - h.conj().T)) == 0.0


def control_spread_ok(u, sigma):
    # n draws of N(0, sigma^2): the sample mean has standard error sigma / sqrt(n) and the sample
    # standard deviation sigma / sqrt(2n); allow five of each
    n = u.size
    return abs(u.std() / sigma - 1) < 5 / np.sqrt(2 * n) and abs(u.mean()) < 5 * sigma / np.sqrt(n)


def test_cnot2q():
    p = sy.cnot2q()
    assert (p.d, p.N, p.M, p.dt, p.S) == (4, 200, 4, 0.5, 4)
    assert np.allclose(np.sort(np.linalg.eigvalsh(p.H0)), TWO_PI * 0.01 * np.array([-1, -1, 1, 1]))
    # target: the CNOT with the first factor as control: |10> <-> |11>, |0x> fixed
    for a, b in [(0, 0), (1, 1), (2, 3), (3, 2)]:
        assert p.psiT[b, a] == 1.0
    assert np.array_equal(p.psi0, np.eye(4))
    assert all(herm(h) for h in p.Hk)
    # the four drives are single-qubit x / y operators: traceless, squares equal the identity
    for h in p.Hk:
        assert abs(np.trace(h)) < 1e-15 and np.allclose(h @ h, np.eye(4))
    assert control_spread_ok(p.u, TWO_PI * 0.02)
    assert list(p.alpha) == [1, 0, 0, 0, 0]


def test_transmon_cavity():
    p = sy.transmon_cavity()
    nt, nc = 4, 10
    assert (p.d, p.N, p.M, p.dt, p.S) == (40, 2000, 2, 1.0, 1)
    E = np.real(np.diag(p.H0))
    assert np.allclose(p.H0, np.diag(E))            # rotating frame: diagonal drift
    lvl = lambda t, c: E[nc * t + c]
    assert lvl(2, 0) - 2 * lvl(1, 0) + lvl(0, 0) == pytest.approx(-TWO_PI * 0.225)   # anharmonicity
    assert lvl(1, 1) - lvl(1, 0) - lvl(0, 1) + lvl(0, 0) == pytest.approx(-TWO_PI * 0.002)  # chi
    # drives act on the transmon alone: they commute with the cavity photon number
    nphot = np.kron(np.eye(nt), np.diag(np.arange(nc)))
    for h in p.Hk:
        assert herm(h) and np.allclose(h @ nphot, nphot @ h)
    assert p.psi0[0, 0] == 1 and p.psiT[1, 0] == 1     # |g,0> -> |g,1>
    forb = {nc * t + c for t in range(nt) for c in range(nc) if t == nt - 1 or c == nc - 1}
    assert set(p.forbidden.tolist()) == forb and len(forb) == 13
    assert p.alpha[0] == 1 and p.alpha[3] == pytest.approx(1 / p.N)
    assert control_spread_ok(p.u, TWO_PI * 0.02)


def test_transmon4():
    p = sy.transmon4()
    assert (p.d, p.N, p.M, p.dt) == (81, 1000, 8, 0.5)
    dims = [3] * 4
    digits = np.array(np.unravel_index(np.arange(81), dims)).T
    ntot = np.diag(digits.sum(axis=1).astype(float))
    assert np.allclose(p.H0 @ ntot, ntot @ p.H0)    # exchange conserves the excitation number
    # single-excitation block: the open chain's hopping J between neighbouring transmons
    one = [int(np.ravel_multi_index(tuple(np.eye(4, dtype=int)[i]), dims)) for i in range(4)]
    blk = p.H0[np.ix_(one, one)]
    assert np.allclose(blk, TWO_PI * 0.005 * (np.eye(4, k=1) + np.eye(4, k=-1)))
    two = int(np.ravel_multi_index((2, 0, 0, 0), dims))
    assert np.real(p.H0[two, two]) == pytest.approx(-TWO_PI * 0.2)   # anharmonicity of level 2
    sub = np.where(p.col_weight > 0)[0]
    assert len(sub) == 16 and np.all(digits[sub] <= 1)
    V = p.psiT[np.ix_(sub, sub)]
    assert np.allclose(V.conj().T @ V, np.eye(16))
    assert set(p.forbidden.tolist()) == set(np.where((digits == 2).any(axis=1))[0].tolist())
    assert control_spread_ok(p.u, TWO_PI * 0.03)


def test_gue256():
    p = sy.gue256()
    assert (p.d, p.N, p.M, p.dt) == (256, 2000, 16, 0.25)
    assert herm(p.H0)
    assert np.abs(np.linalg.eigvalsh(p.H0)).max() == pytest.approx(TWO_PI * 0.05, rel=1e-12)
    assert np.allclose(p.psiT.conj().T @ p.psiT, np.eye(256))
    for h in p.Hk:
        assert herm(h) and np.allclose(h @ h, np.eye(256))
    assert control_spread_ok(p.u, TWO_PI * 0.02)


def test_batch_problems_span_the_stated_ranges():
    probs = sy.batch_problems(128)
    ds = {p.d for p in probs}
    assert ds <= {4, 8, 16, 40, 81, 128} and len(ds) == 6
    assert all(200 <= p.N <= 4000 and 2 <= p.M <= 8 and p.dt == 0.5 for p in probs)
    ens = sy.batch_problem(3, ensemble=32)
    assert ens.E == 32 and herm(ens.Hdet)
