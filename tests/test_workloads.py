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


def test_transmon_cnot():
    """Two five-level transmons in the frame of the first: the drift's single-excitation block
    holds the 400 MHz detuning and the 100 MHz exchange; the anharmonicity shows in the two-
    excitation energies; the target maps the four computational states by CNOT."""
    p = sy.transmon_cnot()
    assert (p.d, p.N, p.M, p.S) == (25, 250, 5, 4) and abs(p.dt - 0.04) < 1e-15
    assert herm(p.H0) and all(herm(h) for h in p.Hk)
    e01, e10 = 1, 5                                     # |0,1> and |1,0> (index 5 q1 + q2)
    blk = p.H0[np.ix_([e01, e10], [e01, e10])]
    assert np.isclose(blk[0, 0] - blk[1, 1], TWO_PI * 0.4) and np.isclose(abs(blk[0, 1]), TWO_PI * 0.1)
    assert np.isclose(p.H0[10, 10].real, TWO_PI * -0.225)   # |2,0>: 2 levels of transmon 1, alpha
    comp = [0, 1, 5, 6]
    for s, t in [(0, 0), (1, 1), (2, 3), (3, 2)]:
        assert p.psi0[comp[s], s] == 1.0 and p.psiT[comp[t], s] == 1.0
    assert all(i // 5 >= 3 or i % 5 >= 3 for i in p.forbidden) and len(p.forbidden) == 25 - 9


def test_cat_state():
    """The cat-state system: d = 7 x 22 in the lab frame, 8000 slices of 5 ps; the uncoupled
    spectrum holds the transmon and cavity frequencies; the target is the normalised cat of
    amplitude 2 in the cavity with the transmon in its ground state (even photon numbers only)."""
    p = sy.cat_state()
    assert (p.d, p.N, p.M, p.S) == (154, 8000, 2, 1) and abs(p.dt - 0.005) < 1e-15
    assert herm(p.H0) and all(herm(h) for h in p.Hk)
    diag = np.real(np.diag(p.H0))
    assert np.isclose(diag[22] - diag[0], TWO_PI * 3.5) and np.isclose(diag[1] - diag[0], TWO_PI * 3.9)
    assert np.isclose(diag[44] - 2 * diag[22], TWO_PI * -0.225)
    cat = p.psiT[:22, 0]
    assert np.isclose(np.linalg.norm(p.psiT), 1.0) and np.allclose(cat[1::2], 0.0)
    assert np.isclose(abs(cat[0]) ** 2, 2 * np.exp(-4) / (1 + np.exp(-8)), rtol=1e-6)
    assert np.array_equal(p.psi0[:, 0], np.eye(154)[0])
    assert 22 * 3 in p.forbidden and 20 in p.forbidden and 21 in p.forbidden and 22 * 2 not in p.forbidden
