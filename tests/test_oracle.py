"""Pins of the CPU FP64 oracle against facts that do not come from the oracle itself:
closed forms, invariants, scipy's expm, central finite differences, a brute-force O(N^2)
tangent sum, and the paper's Algorithms 1-3 (Appendix A).  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg

import synthetic as sy
from oracle import qoc_oracle as orc

SX, SY, SZ = sy.SX, sy.SY, sy.SZ


def single_qubit(u, alpha, forbidden=(), target=1, N=None, dt=0.37):
    """H0 = 0, one control sigma_x, Psi_0 = |0>, Psi_T = |target>."""
    u = np.atleast_2d(np.asarray(u, np.float64))
    N = u.shape[1]
    return sy.Problem("q1", np.zeros((2, 2), np.complex128), SX[None], dt, N,
                      sy.basis_state(2, 0), sy.basis_state(2, target),
                      np.array(forbidden, np.int32), np.ones(1), np.asarray(alpha, float), u)


# ---------------------------------------------------------------- Eq. 3: the exponential
@pytest.mark.parametrize("theta", [0.0, 0.3, 1.0, math.pi / 2, 2.7, 11.0])
def test_expm_sigma_x_closed_form(theta):
    # exp(-i theta sx) = cos(theta) I - i sin(theta) sx
    dt = 0.25
    U, _, _ = orc.expm_herm(SX * (theta / dt), dt)
    ref = math.cos(theta) * np.eye(2) - 1j * math.sin(theta) * SX
    assert np.max(np.abs(U - ref)) < 1e-14


@pytest.mark.parametrize("d", [2, 5, 16, 40])
def test_expm_matches_scipy_and_is_unitary(d):
    rng = np.random.default_rng(d)
    H = sy.random_hermitian(d, rng, 1.3)
    U, _, _ = orc.expm_herm(H, 0.7)
    ref = scipy.linalg.expm(-1j * 0.7 * H)
    assert np.max(np.abs(U - ref)) < 1e-13
    assert np.max(np.abs(U.conj().T @ U - np.eye(d))) < 1e-13


@pytest.mark.parametrize("degenerate", [False, True])
def test_dexpm_against_finite_differences(degenerate):
    rng = np.random.default_rng(7)
    d = 4
    if degenerate:   # repeated eigenvalues: the sinc form must stay exact
        H = np.diag([0.5, 0.5, -1.0, -1.0]).astype(np.complex128)
    else:
        H = sy.random_hermitian(d, rng, 1.0)
    dH = sy.random_hermitian(d, rng, 1.0)
    dt, h = 0.9, 1e-6
    _, V, lam = orc.expm_herm(H, dt)
    dU = orc.dexpm_herm(V, lam, dH, dt)
    fd = (scipy.linalg.expm(-1j * dt * (H + h * dH)) - scipy.linalg.expm(-1j * dt * (H - h * dH))) / (2 * h)
    assert np.max(np.abs(dU - fd)) < 1e-8
    # commuting direction: d/dx exp(-i (H + x H) dt) = -i dt H U exactly
    U, V, lam = orc.expm_herm(H, dt)
    assert np.max(np.abs(orc.dexpm_herm(V, lam, H, dt) - (-1j * dt * H @ U))) < 1e-13


# ---------------------------------------------------------------- closed-form costs
def test_single_qubit_state_transfer_closed_form():
    # all U_j commute: Psi_N = cos(T)|0> - i sin(T)|1>, T = dt sum_j u_j
    rng = np.random.default_rng(1)
    u = rng.normal(0, 0.8, size=7)
    p = single_qubit(u, [1, 0, 0, 0, 0])
    T = p.dt * u.sum()
    c, g, terms = orc.cost_and_grad(p, p.u)
    assert abs(c - (1 - math.sin(T) ** 2)) < 1e-14
    assert np.max(np.abs(g[0] - (-p.dt * math.sin(2 * T)))) < 1e-14


def test_single_qubit_forbidden_closed_form():
    # C5 = sum_J sin^2(T_J), dC5/du_j = dt sum_{J>=j} sin(2 T_J)
    rng = np.random.default_rng(2)
    u = rng.normal(0, 0.8, size=9)
    p = single_qubit(u, [0, 0, 0, 1, 0], forbidden=[1])
    TJ = p.dt * np.cumsum(u)
    c, g, _ = orc.cost_and_grad(p, p.u)
    assert abs(c - np.sum(np.sin(TJ) ** 2)) < 1e-13
    ref = p.dt * np.cumsum(np.sin(2 * TJ)[::-1])[::-1]
    assert np.max(np.abs(g[0] - ref)) < 1e-13


def test_single_qubit_time_optimal_closed_form():
    # C7 = 1 - (1/N) sum_J sin^2(T_J), dC7/du_j = -(dt/N) sum_{J>=j} sin(2 T_J)
    rng = np.random.default_rng(3)
    u = rng.normal(0, 0.8, size=6)
    p = single_qubit(u, [0, 0, 0, 0, 1])
    TJ = p.dt * np.cumsum(u)
    c, g, _ = orc.cost_and_grad(p, p.u)
    assert abs(c - (1 - np.mean(np.sin(TJ) ** 2))) < 1e-14
    ref = -(p.dt / len(u)) * np.cumsum(np.sin(2 * TJ)[::-1])[::-1]
    assert np.max(np.abs(g[0] - ref)) < 1e-14


def test_single_qubit_ensemble_closed_form():
    # detuning delta_e on H_det = sx shifts every slice: T_{J,e} = dt sum_{j<=J} (u_j + delta_e).
    # C_fid and C5 are means over the members: C_fid = mean_e cos^2(T_{N,e}),
    # C5 = mean_e sum_J sin^2(T_{J,e}), with gradients mean_e of the one-member closed forms.
    rng = np.random.default_rng(4)
    u = rng.normal(0, 0.8, size=8)
    p = single_qubit(u, [1, 0, 0, 0.5, 0], forbidden=[1])
    p.delta = np.array([-0.3, 0.0, 0.45])
    p.Hdet = SX.copy()
    TJ = p.dt * np.cumsum(u[None, :] + p.delta[:, None], axis=1)     # (E, N)
    c, g, terms = orc.cost_and_grad(p, p.u)
    assert abs(terms[0] - np.mean(np.cos(TJ[:, -1]) ** 2)) < 1e-14
    assert abs(terms[3] - np.mean(np.sum(np.sin(TJ) ** 2, axis=1))) < 1e-13
    assert abs(c - terms[0] - 0.5 * terms[3]) < 1e-14
    g_fid = -p.dt * np.mean(np.sin(2 * TJ[:, -1]))
    g5 = p.dt * np.mean(np.cumsum(np.sin(2 * TJ)[:, ::-1], axis=1)[:, ::-1], axis=0)
    assert np.max(np.abs(g[0] - (g_fid + 0.5 * g5))) < 1e-13


def test_single_qubit_per_slice_targets_closed_form():
    # per-slice targets |J mod 2> at slice J: |O_J|^2 = sin^2(T_J) for odd J, cos^2(T_J) for even J,
    # so C67 = 1 - (1/N) sum_J |O_J|^2 and dC67/du_j = -(dt/N) sum_{J>=j} s_J sin(2 T_J), s_J = +-1
    rng = np.random.default_rng(5)
    u = rng.normal(0, 0.8, size=7)
    N = len(u)
    p = single_qubit(u, [0, 0, 0, 0, 1])
    J = np.arange(1, N + 1)
    p.psiT_path = np.stack([sy.basis_state(2, int(k % 2)) for k in J])
    TJ = p.dt * np.cumsum(u)
    occ = np.where(J % 2 == 1, np.sin(TJ) ** 2, np.cos(TJ) ** 2)
    sgn = np.where(J % 2 == 1, 1.0, -1.0)
    c, g, _ = orc.cost_and_grad(p, p.u)
    assert abs(c - (1 - np.mean(occ))) < 1e-14
    ref = -(p.dt / N) * np.cumsum((sgn * np.sin(2 * TJ))[::-1])[::-1]
    assert np.max(np.abs(g[0] - ref)) < 1e-14


def test_single_qubit_weighted_columns_closed_form():
    # columns |0>, |1> both aimed at |1> with weights w0, w1: overlaps -i sin T and cos T, so
    # O = (-i w0 sin T + w1 cos T) / (w0 + w1), C_fid = 1 - (w0^2 sin^2 T + w1^2 cos^2 T) / (w0 + w1)^2,
    # dC_fid/du_j = -dt (w0^2 - w1^2) sin(2T) / (w0 + w1)^2
    rng = np.random.default_rng(6)
    u = rng.normal(0, 0.8, size=5)
    p = single_qubit(u, [1, 0, 0, 0, 0])
    p.psi0 = np.eye(2, dtype=np.complex128)
    p.psiT = np.hstack([sy.basis_state(2, 1), sy.basis_state(2, 1)])
    w0, w1 = 0.7, 2.3
    p.col_weight = np.array([w0, w1])
    T = p.dt * u.sum()
    W2 = (w0 + w1) ** 2
    c, g, _ = orc.cost_and_grad(p, p.u)
    assert abs(c - (1 - (w0 ** 2 * math.sin(T) ** 2 + w1 ** 2 * math.cos(T) ** 2) / W2)) < 1e-14
    assert np.max(np.abs(g[0] - (-p.dt * (w0 ** 2 - w1 ** 2) * math.sin(2 * T) / W2))) < 1e-14


def test_control_terms_closed_form():
    u = np.array([[1.0, -2.0, 0.5], [0.0, 3.0, 1.0]])
    p = single_qubit(u[:1], [0, 1, 1, 0, 0])
    p = sy.Problem("q", p.H0, np.stack([SX, SY]), 0.1, 3, p.psi0, p.psiT, p.forbidden,
                   p.col_weight, np.array([0, 1.0, 1.0, 0, 0]), u)
    c, g, terms = orc.cost_and_grad(p, u)
    assert terms[1] == pytest.approx(1 + 4 + 0.25 + 0 + 9 + 1)
    assert terms[2] == pytest.approx(9 + 6.25 + 9 + 4)
    g4 = np.array([[2 * (1 - (-2)), 2 * (-2 - 1) - 2 * (0.5 + 2), 2 * (0.5 + 2)],
                   [2 * (0 - 3), 2 * (3 - 0) - 2 * (1 - 3), 2 * (1 - 3)]])
    assert np.max(np.abs(g - (2 * u + g4))) < 1e-14


def test_diagonal_drift_zero_drive_gate_closed_form():
    # C1 = 1 - |sum_a exp(-i E_a N dt) / d|^2 for diagonal H0, no drive, identity target
    E = np.array([0.3, -1.1, 2.0, 0.7])
    N, dt = 11, 0.21
    p = sy.Problem("diag", np.diag(E).astype(np.complex128), SX[None][:, :1, :1].repeat(0, 0).reshape(0, 4, 4),
                   dt, N, np.eye(4, dtype=np.complex128), np.eye(4, dtype=np.complex128),
                   np.zeros(0, np.int32), np.ones(4), np.array([1.0, 0, 0, 0, 0]), np.zeros((0, N)))
    c, _ = orc.cost_terms(p, p.u)
    ref = 1 - abs(np.sum(np.exp(-1j * E * N * dt)) / 4) ** 2
    assert abs(c - ref) < 1e-14


def test_identity_target_zero_hamiltonian_has_unit_fidelity():
    d, N = 5, 4
    z = np.zeros((d, d), np.complex128)
    p = sy.Problem("zero", z, np.stack([z, z]), 0.3, N, np.eye(d, dtype=np.complex128),
                   np.eye(d, dtype=np.complex128), np.zeros(0, np.int32), np.ones(d),
                   np.array([1.0, 0, 0, 0, 1.0]), np.zeros((2, N)))
    c, g, terms = orc.cost_and_grad(p, p.u)
    assert abs(terms[0]) < 1e-15 and abs(terms[4]) < 1e-15 and abs(c) < 1e-15


# ---------------------------------------------------------------- invariances
def test_cost_invariant_under_energy_shift_and_global_phase():
    p = sy.random_problem(4, 2, 6, 4, seed=11, nF=1)
    p.psi0 = np.eye(4, dtype=np.complex128)
    p.psiT = sy.haar_unitary(4, np.random.default_rng(3))
    c0, g0, _ = orc.cost_and_grad(p, p.u)
    p.H0 = p.H0 + 0.77 * np.eye(4)
    c1, g1, _ = orc.cost_and_grad(p, p.u)
    p.psiT = p.psiT * np.exp(0.4j)
    c2, g2, _ = orc.cost_and_grad(p, p.u)
    assert abs(c0 - c1) < 1e-13 and abs(c0 - c2) < 1e-13
    assert np.max(np.abs(g0 - g1)) < 1e-12 and np.max(np.abs(g0 - g2)) < 1e-12


def test_unitarity_of_slice_propagators():
    p = sy.transmon_cavity(N=8)
    H = orc.slice_hamiltonians(p, p.u)
    for h in H:
        U, _, _ = orc.expm_herm(h, p.dt)
        assert np.max(np.abs(U.conj().T @ U - np.eye(p.d))) < 1e-13


def test_slice_hamiltonian_assembly():
    p = sy.random_problem(3, 3, 4, 1, seed=5)
    H = orc.slice_hamiltonians(p, p.u)
    for j in range(p.N):
        ref = p.H0 + p.u[0, j] * p.Hk[0] + p.u[1, j] * p.Hk[1] + p.u[2, j] * p.Hk[2]
        assert np.max(np.abs(H[j] - ref)) < 1e-15


# ---------------------------------------------------------------- gradients
def _fd_grad(p, h=1e-6):
    g = np.zeros_like(p.u)
    for k in range(p.M):
        for j in range(p.N):
            up, um = p.u.copy(), p.u.copy()
            step = h * max(1.0, abs(p.u[k, j]))
            up[k, j] += step
            um[k, j] -= step
            g[k, j] = (orc.cost_terms(p, up)[0] - orc.cost_terms(p, um)[0]) / (2 * step)
    return g


CASES = [
    dict(d=2, M=1, N=5, S=1, seed=21, nF=1),
    dict(d=3, M=2, N=7, S=2, seed=22, nF=1, weights=True),
    dict(d=4, M=2, N=6, S=4, seed=23, nF=2, path=True),
    dict(d=3, M=2, N=5, S=1, seed=24, nF=1, E=3),
    dict(d=4, M=3, N=12, S=2, seed=25, nF=2, path=True, E=2, weights=True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"d{c['d']}N{c['N']}S{c['S']}")
def test_gradient_matches_finite_differences(case):
    p = sy.random_problem(**case)
    _, g, _ = orc.cost_and_grad(p, p.u)
    gf = _fd_grad(p)
    assert np.max(np.abs(g - gf)) < 1e-7 * max(1.0, np.max(np.abs(g)))


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"d{c['d']}N{c['N']}S{c['S']}")
def test_adjoint_matches_bruteforce_tangents(case):
    p = sy.random_problem(**case)
    _, g, _ = orc.cost_and_grad(p, p.u)
    gb = orc.grad_bruteforce(p, p.u)
    assert np.max(np.abs(g - gb)) < 1e-12 * max(1.0, np.max(np.abs(g)))


def test_directional_derivative_of_constant_shift():
    # d/dx C(u + x * 1_k) = sum_j dC/du_{k,j}
    p = sy.random_problem(3, 2, 8, 2, seed=31, nF=1)
    _, g, _ = orc.cost_and_grad(p, p.u)
    h = 1e-6
    for k in range(p.M):
        up, um = p.u.copy(), p.u.copy()
        up[k] += h
        um[k] -= h
        dd = (orc.cost_terms(p, up)[0] - orc.cost_terms(p, um)[0]) / (2 * h)
        assert abs(dd - g[k].sum()) < 1e-7


def test_paper_algorithm1_gate():
    p = sy.random_problem(4, 2, 9, 4, seed=41, alpha=[1, 0, 0, 0, 0])
    p.psi0 = np.eye(4, dtype=np.complex128)
    p.psiT = sy.haar_unitary(4, np.random.default_rng(9))
    _, g, _ = orc.cost_and_grad(p, p.u)
    assert np.max(np.abs(orc.grad_paper_alg1(p, p.u) - g)) < 1e-13


def test_paper_algorithm2_state():
    p = sy.random_problem(5, 3, 10, 1, seed=42, alpha=[1, 0, 0, 0, 0])
    _, g, _ = orc.cost_and_grad(p, p.u)
    assert np.max(np.abs(orc.grad_paper_alg2(p, p.u) - g)) < 1e-13


def test_paper_algorithm3_forbidden():
    p = sy.random_problem(5, 2, 11, 1, seed=43, nF=2, alpha=[0, 0, 0, 1, 0])
    _, g, _ = orc.cost_and_grad(p, p.u)
    assert np.max(np.abs(orc.grad_paper_alg3(p, p.u) - g)) < 1e-13


def test_first_order_gradient_is_second_order_close():
    # Eq. 11 drops the non-commuting part of dU_j, a term O(dt^2 ||[H_j, H_k]||) against a
    # leading term O(dt): the relative gap is first order in dt and halves with dt.
    gaps = []
    for dt in (0.08, 0.04):
        p = sy.random_problem(4, 2, 6, 1, seed=44, dt=dt, alpha=[1, 0, 0, 0, 0])
        ge = orc.grad_paper_alg2(p, p.u, exact=True)
        ga = orc.grad_paper_alg2(p, p.u, exact=False)
        gaps.append(np.linalg.norm(ge - ga) / np.linalg.norm(ge))
    assert 1.7 < gaps[0] / gaps[1] < 2.4


# ---------------------------------------------------------------- Sec. III: Taylor + squaring
def test_taylor_series_within_remainder_bound():
    rng = np.random.default_rng(51)
    for d in (2, 6, 20):
        H = sy.random_hermitian(d, rng, 2.0)
        dt = 0.8
        theta = dt * np.max(np.sum(np.abs(H), axis=0))
        for theta_max, tol in ((0.25, 1e-15), (0.5, 1e-8), (1.0, 1e-5)):
            p, n = orc.pick_pn(theta, theta_max, tol)
            U = orc.taylor_expm(-1j * dt / 2 ** n * H, p, n)
            ref = scipy.linalg.expm(-1j * dt * H)
            assert np.linalg.norm(U - ref, 2) <= tol + 1e-13 * d


def test_pick_pn_is_minimal():
    for theta in (0.01, 0.3, 0.7, 3.0, 47.0):
        for theta_max, tol in ((0.25, 1e-15), (0.5, 1e-8)):
            p, n = orc.pick_pn(theta, theta_max, tol)
            assert theta / 2 ** n <= theta_max
            assert n == 0 or theta / 2 ** (n - 1) > theta_max
            ts = theta / 2 ** n

            def rem(q):
                return 2 ** n * ts ** (q + 1) / math.factorial(q + 1) / (1 - ts / (q + 2))
            assert rem(p) <= tol and (p == 1 or rem(p - 1) > tol)


def test_theta_bounds_the_spectral_radius():
    p = sy.transmon_cavity(N=50)
    theta = orc.theta_bound(p, p.u)
    H = orc.slice_hamiltonians(p, p.u)
    assert p.dt * max(np.max(np.abs(np.linalg.eigvalsh(h))) for h in H) <= theta


def test_truncated_series_gradient_matches_finite_differences():
    p = sy.random_problem(3, 2, 5, 2, seed=52, nF=1, path=True)
    pp, nn = 4, 2          # deliberately short series: its gradient differs from exp's
    _, g, _ = orc.taylor_cost_and_grad(p, p.u, pp, nn)
    h = 1e-6
    gf = np.zeros_like(g)
    for k in range(p.M):
        for j in range(p.N):
            up, um = p.u.copy(), p.u.copy()
            up[k, j] += h
            um[k, j] -= h
            gf[k, j] = (orc.taylor_cost_and_grad(p, up, pp, nn)[0] -
                        orc.taylor_cost_and_grad(p, um, pp, nn)[0]) / (2 * h)
    assert np.max(np.abs(g - gf)) < 1e-7
    _, ge, _ = orc.cost_and_grad(p, p.u)
    assert np.max(np.abs(g - ge)) > 1e-6   # the truncation is visible at this order


def test_truncated_series_converges_to_exact():
    p = sy.random_problem(4, 2, 6, 2, seed=53, nF=1)
    pp, nn = orc.pick_pn(orc.theta_bound(p, p.u), 0.25, 1e-15)
    c, g, t = orc.taylor_cost_and_grad(p, p.u, pp, nn)
    ce, ge, te = orc.cost_and_grad(p, p.u)
    assert abs(c - ce) < 1e-13 and np.max(np.abs(g - ge)) < 1e-12


# ---------------------------------------------------------------- sensitivity of the pins
def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant plausible mistakes in the oracle and check that a pin above fails on each."""
    p = sy.random_problem(3, 2, 5, 2, seed=61, nF=1, path=True)
    gf = _fd_grad(p)

    def fails():
        _, g, _ = orc.cost_and_grad(p, p.u)
        return np.max(np.abs(g - gf)) > 1e-6

    orig_gamma = orc._gamma
    monkeypatch.setattr(orc, "_gamma", lambda lam, dt: np.conj(orig_gamma(lam, dt)))   # sign
    assert fails()
    monkeypatch.setattr(orc, "_gamma", orig_gamma)
    orig_dexpm = orc.dexpm_herm

    def swapped_basis(V, lam, dH, dt):               # V and V^dag exchanged
        return orig_dexpm(V.conj().T, lam, dH, dt)
    monkeypatch.setattr(orc, "dexpm_herm", swapped_basis)
    assert fails()
    monkeypatch.setattr(orc, "dexpm_herm", orig_dexpm)
    orig_src = orc._sources

    def drop_time_term(prob, psi, oN, oj, scale):     # a dropped source term
        return orig_src(prob, psi, oN, 0 * oj, scale)
    monkeypatch.setattr(orc, "_sources", drop_time_term)
    assert fails()
    monkeypatch.setattr(orc, "_sources", orig_src)
    assert not fails()


def test_closed_form_pins_catch_planted_mistakes(monkeypatch):
    """A per-slice target read one slice late, every member seeing the first member's detuning,
    and column weights ignored in the overlap each make a closed-form pin above fail."""
    def off_by_one(prob, j):
        return prob.psiT_path[min(j, prob.N - 1)] if prob.psiT_path is not None else prob.psiT
    monkeypatch.setattr(orc, "_targets", off_by_one)
    with pytest.raises(AssertionError):
        test_single_qubit_per_slice_targets_closed_form()
    monkeypatch.undo()
    orig_h = orc.slice_hamiltonians
    monkeypatch.setattr(orc, "slice_hamiltonians", lambda prob, u, e=0: orig_h(prob, u, 0))
    with pytest.raises(AssertionError):
        test_single_qubit_ensemble_closed_form()
    monkeypatch.undo()
    orig_ov = orc._overlap
    monkeypatch.setattr(orc, "_overlap", lambda target, psi, w: orig_ov(target, psi, np.ones_like(w)))
    with pytest.raises(AssertionError):
        test_single_qubit_weighted_columns_closed_form()
    monkeypatch.undo()
    test_single_qubit_per_slice_targets_closed_form()
    test_single_qubit_ensemble_closed_form()
    test_single_qubit_weighted_columns_closed_form()


# ---------------------------------------------------------------- synthetic inputs
def test_workload_inputs_are_well_formed():
    for make in (sy.cnot2q, sy.transmon_cavity, sy.transmon4):
        p = make()
        for h in [p.H0, *p.Hk]:
            assert np.max(np.abs(h - h.conj().T)) == 0.0
        assert p.u.shape == (p.M, p.N)
    c2 = sy.transmon_cavity()
    assert c2.d == 40 and len(c2.forbidden) == 13 and c2.N == 2000
    c3 = sy.transmon4()
    assert c3.d == 81 and len(c3.forbidden) == 65 and int(c3.col_weight.sum()) == 16
    sub = np.where(c3.col_weight > 0)[0]
    V = c3.psiT[np.ix_(sub, sub)]
    assert np.max(np.abs(V.conj().T @ V - np.eye(16))) < 1e-13


def test_sampled_slices_match_full_gradient():
    p = sy.random_problem(3, 2, 9, 2, seed=71, nF=1, path=True, E=2)
    _, g, _ = orc.cost_and_grad(p, p.u)
    c, gs, _ = orc.cost_and_grad(p, p.u, slices=[0, 4, 8])
    assert np.all(np.isnan(gs[:, [1, 2, 3, 5, 6, 7]]))
    assert np.max(np.abs(gs[:, [0, 4, 8]] - g[:, [0, 4, 8]])) == 0.0
