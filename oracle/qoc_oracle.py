"""Plain, slow, FP64 CPU oracle for one forward + gradient evaluation of a piecewise-constant
quantum-control cost (Leung, Abdelhafez, Koch, Schuster, "Speedup for quantum optimal control
from automatic differentiation based on graphics processing units", arXiv:1612.04929).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and, in ``bench.py``, the
CPU-baseline leg and the oracle arm (``--impl reference``) may import this module.  It shares no
code with the CUDA path.

What it computes (notation of the paper, Sec. II):

* Eq. 1   H_j = H_0 + sum_k u_{k,j} H_k                      (slices j = 1..N)
* Eq. 3   U_j = exp(-i H_j dt), here by Hermitian eigendecomposition H_j = V diag(lam) V^dag
* Eq. 2/4 Psi_j = U_j Psi_{j-1}; Psi_0 is a d x S block of initial columns (Psi_0 = I for gates)
* Table I costs, with column weights w_s (all 1 unless a subspace is selected):
    O_j    = sum_s w_s <PsiT^s(j)|Psi_j^s> / sum_s w_s
    C_fid  = 1 - |O_N|^2                                    (C1 for Psi_0 = I, C2 / C2-Sigma)
    C3     = sum_{k,j} u_{k,j}^2
    C4     = sum_k sum_{j=2..N} (u_{k,j} - u_{k,j-1})^2
    C5     = sum_{j=1..N} sum_s w_s sum_{f in F} |Psi_j[f, s]|^2
    C67    = 1 - (1/N) sum_{j=1..N} |O_j|^2                   (C6 gate / C7 state)
    C      = sum_mu alpha_mu C_mu                             (Sec. II, weighted total)
  Ensemble members (H_j + delta_e H_det) average the state-dependent terms.
* Gradient (Appendix A, Eqs. A3-A7 and Algorithms 1-3): the explicit adjoint recursion
    G_N = dC/dPsi_N,  G_{j-1} = U_j^dag G_j + src_{j-1},
    dC/du_{k,j} = Re tr[(G_j Psi_{j-1}^dag)^dag dU_j/du_{k,j}]
  with the exact derivative of the exponential (Daleckii-Krein divided differences) in place
  of the first-order form of Eq. 11, which is kept as an option (``exact=False``).

Conventions.  For a real cost C of a complex matrix A the cotangent is
Abar = dC/dRe(A) + i dC/dIm(A), so dC = Re tr(Abar^dag dA).

Second, independent gradient forms used to pin the adjoint:
* ``grad_bruteforce`` -- forward-mode tangents propagated slice by slice, O(N^2 M) (the double
  sum of Eq. A7 written out),
* ``grad_paper_alg1/alg2/alg3`` -- the paper's Algorithms 1, 2, 3 (C1, C2, C5 backward sweeps)
  with the exact dU,
* central finite differences (in the tests).

Diagnostic mode: ``taylor_expm`` / ``taylor_cost_and_grad`` evaluate the truncated Taylor series
with scaling and squaring of Eqs. 9-10 in FP64 plain loops (power sum, then 2^n-th power) and
differentiate that truncated series by its definition, so that truncation error can be
separated from arithmetic error in comparisons.  ``pick_pn`` is the global (p, n) heuristic.

Parity status: every public function here is pinned by tests/test_oracle.py (closed forms,
invariants, scipy.linalg.expm, finite differences, brute force, the paper's Algorithms 1-3).
"""
from __future__ import annotations

import math
from typing import Dict, Optional, Tuple

import numpy as np

__all__ = [
    "slice_hamiltonians", "expm_herm", "dexpm_herm", "propagate", "cost_terms", "cost_and_grad",
    "grad_bruteforce", "grad_paper_alg1", "grad_paper_alg2", "grad_paper_alg3",
    "taylor_expm", "pick_pn", "theta_bound", "taylor_cost_and_grad", "TERM_NAMES",
]

TERM_NAMES = ("fid", "amp", "var", "forbid", "time")


# ----------------------------------------------------------------------------------------
# Eq. 1 and Eq. 3
# ----------------------------------------------------------------------------------------
def slice_hamiltonians(prob, u: np.ndarray, e: int = 0) -> np.ndarray:
    """H_j = H_0 + sum_k u[k, j] H_k (+ delta_e H_det) for j = 1..N, returned as (N, d, d)
    (Sec. II, Eq. 1)."""
    u = np.asarray(u, np.float64)
    H = np.einsum("kj,kab->jab", u, prob.Hk) + prob.H0[None, :, :]
    if prob.Hdet is not None and prob.delta[e] != 0.0:
        H = H + prob.delta[e] * prob.Hdet[None, :, :]
    return H


def expm_herm(H: np.ndarray, dt: float) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """U = exp(-i H dt) for Hermitian H (Sec. II, Eq. 3) by H = V diag(lam) V^dag.
    Returns (U, V, lam)."""
    lam, V = np.linalg.eigh(H)
    U = (V * np.exp(-1j * lam * dt)[None, :]) @ V.conj().T
    return U, V, lam


def dexpm_herm(V: np.ndarray, lam: np.ndarray, dH: np.ndarray, dt: float) -> np.ndarray:
    """Exact directional derivative of exp(-i H dt) along dH (Daleckii-Krein):
    V^dag dU V = (V^dag dH V) o Gamma with Gamma_ab the divided difference of
    g(x) = exp(-i x dt):  Gamma_ab = -i dt exp(-i (l_a + l_b) dt / 2) sinc((l_a - l_b) dt / 2).
    The sinc form is exact and stays well defined when l_a = l_b."""
    return V @ ((V.conj().T @ dH @ V) * _gamma(lam, dt)) @ V.conj().T


def _gamma(lam: np.ndarray, dt: float) -> np.ndarray:
    a = lam[:, None]
    b = lam[None, :]
    x = 0.5 * (a - b) * dt
    return -1j * dt * np.exp(-0.5j * (a + b) * dt) * np.sinc(x / math.pi)


# ----------------------------------------------------------------------------------------
# Eqs. 2 and 4: propagation
# ----------------------------------------------------------------------------------------
def propagate(psi0: np.ndarray, U: np.ndarray) -> np.ndarray:
    """Psi_j = U_j Psi_{j-1} for j = 1..N (Eqs. 2, 4); returns (N+1, d, S) with Psi_0 first."""
    N = U.shape[0]
    out = np.empty((N + 1,) + psi0.shape, np.complex128)
    out[0] = psi0
    for j in range(1, N + 1):
        out[j] = U[j - 1] @ out[j - 1]
    return out


# ----------------------------------------------------------------------------------------
# Table I costs
# ----------------------------------------------------------------------------------------
def _targets(prob, j: int) -> np.ndarray:
    """Target block used by the per-slice time cost at slice j (1-based)."""
    return prob.psiT_path[j - 1] if prob.psiT_path is not None else prob.psiT


def _overlap(target: np.ndarray, psi: np.ndarray, w: np.ndarray) -> complex:
    """sum_s w_s <target^s|psi^s> / sum_s w_s (Table I C1/C2, C2-Sigma of Sec. II.A)."""
    return complex(np.sum(w * np.sum(target.conj() * psi, axis=0)) / np.sum(w))


def _control_terms(u: np.ndarray) -> Tuple[float, float, np.ndarray, np.ndarray]:
    """C3 = |u|^2 and C4 = sum_{k, j>=2} (u_{k,j} - u_{k,j-1})^2 (Table I) with gradients."""
    c3 = float(np.sum(u * u))
    g3 = 2.0 * u
    du = np.diff(u, axis=1)
    c4 = float(np.sum(du * du))
    g4 = np.zeros_like(u)
    g4[:, 1:] += 2.0 * du
    g4[:, :-1] -= 2.0 * du
    return c3, c4, g3, g4


def _member_costs(prob, psi: np.ndarray) -> Tuple[float, float, float, complex, np.ndarray]:
    """(C_fid, C5, C67, O_N, O_j for j=1..N) of one trajectory Psi_0..Psi_N."""
    N, w = prob.N, prob.col_weight
    oN = _overlap(prob.psiT, psi[N], w)
    c_fid = 1.0 - abs(oN) ** 2
    F = prob.forbidden
    c5 = 0.0
    if len(F):
        for j in range(1, N + 1):
            c5 += float(np.sum(w[None, :] * np.abs(psi[j][F, :]) ** 2))
    oj = np.array([_overlap(_targets(prob, j), psi[j], w) for j in range(1, N + 1)])
    c67 = 1.0 - float(np.mean(np.abs(oj) ** 2))
    return c_fid, c5, c67, oN, oj


def cost_terms(prob, u: np.ndarray) -> Tuple[float, np.ndarray]:
    """Total cost C = sum_mu alpha_mu C_mu and the five unweighted terms
    [C_fid, C3, C4, C5, C67] (state terms averaged over ensemble members)."""
    u = np.asarray(u, np.float64)
    acc = np.zeros(3)
    for e in range(prob.E):
        H = slice_hamiltonians(prob, u, e)
        U = np.stack([expm_herm(h, prob.dt)[0] for h in H])
        psi = propagate(prob.psi0, U)
        c_fid, c5, c67, _, _ = _member_costs(prob, psi)
        acc += (c_fid, c5, c67)
    acc /= prob.E
    c3, c4, _, _ = _control_terms(u)
    terms = np.array([acc[0], c3, c4, acc[1], acc[2]])
    return float(np.dot(prob.alpha, terms)), terms


# ----------------------------------------------------------------------------------------
# cotangent sources of the state-dependent costs
# ----------------------------------------------------------------------------------------
def _sources(prob, psi: np.ndarray, oN: complex, oj: np.ndarray, scale: float) -> np.ndarray:
    """src[j] = dC/dPsi_j (cotangent convention of the module docstring) for j = 0..N.
    Eq. A5 / A7 structure: the fidelity term enters at j = N only; C5 and C67 at every slice."""
    N, w = prob.N, prob.col_weight
    W = np.sum(w)
    a_fid, _, _, a5, a67 = prob.alpha
    src = np.zeros_like(psi)
    src[N] += scale * a_fid * (-2.0) * oN * prob.psiT * (w / W)[None, :]
    if len(prob.forbidden) and a5 != 0.0:
        F = prob.forbidden
        for j in range(1, N + 1):
            src[j][F, :] += scale * a5 * 2.0 * psi[j][F, :] * w[None, :]
    if a67 != 0.0:
        for j in range(1, N + 1):
            src[j] += scale * a67 * (-2.0 / N) * oj[j - 1] * _targets(prob, j) * (w / W)[None, :]
    return src


def _dU_list(prob, V, lam, exact: bool, U: np.ndarray) -> list:
    """dU_j/du_{k,j} for all k (exact Daleckii-Krein, or the first-order Eq. 11 form
    -i dt H_k U_j when ``exact`` is False)."""
    if exact:
        return [dexpm_herm(V, lam, hk, prob.dt) for hk in prob.Hk]
    return [-1j * prob.dt * hk @ U for hk in prob.Hk]


# ----------------------------------------------------------------------------------------
# cost and gradient by the explicit adjoint
# ----------------------------------------------------------------------------------------
def cost_and_grad(prob, u: np.ndarray, exact: bool = True, slices=None) -> Tuple[float, np.ndarray, np.ndarray]:
    """Total cost, gradient dC/du (M, N) and terms, by one forward sweep and one backward sweep
    of the costate (Sec. II.B reverse mode; Appendix A, Algorithm 3 pattern with sources at every
    slice).  ``slices`` (0-based indices) restricts the gradient to those slices (the other
    columns are NaN); the costate sweep is unchanged, only the per-slice dU contractions are
    skipped (used to check large systems at full length)."""
    u = np.asarray(u, np.float64)
    M, N = prob.M, prob.N
    wanted = None if slices is None else set(int(s) for s in slices)
    grad = np.zeros((M, N))
    if wanted is not None:
        grad[:, [j for j in range(N) if j not in wanted]] = np.nan
    acc = np.zeros(3)
    for e in range(prob.E):
        H = slice_hamiltonians(prob, u, e)
        eig = [expm_herm(h, prob.dt) for h in H]
        U = np.stack([x[0] for x in eig])
        psi = propagate(prob.psi0, U)
        c_fid, c5, c67, oN, oj = _member_costs(prob, psi)
        acc += (c_fid, c5, c67)
        src = _sources(prob, psi, oN, oj, 1.0 / prob.E)
        G = src[N].copy()
        for j in range(N, 0, -1):
            if wanted is None or (j - 1) in wanted:
                Ubar = G @ psi[j - 1].conj().T
                _, V, lam = eig[j - 1]
                for k, dU in enumerate(_dU_list(prob, V, lam, exact, U[j - 1])):
                    grad[k, j - 1] += np.real(np.sum(Ubar.conj() * dU))
            G = U[j - 1].conj().T @ G + src[j - 1]
    acc /= prob.E
    c3, c4, g3, g4 = _control_terms(u)
    a = prob.alpha
    grad += a[1] * g3 + a[2] * g4
    terms = np.array([acc[0], c3, c4, acc[1], acc[2]])
    return float(np.dot(a, terms)), grad, terms


def grad_bruteforce(prob, u: np.ndarray) -> np.ndarray:
    """dC/du by forward-mode tangents: for every (k, j) the tangent dPsi_J = U_J...U_{j+1} dU_j
    Psi_{j-1} is carried to every J >= j and contracted with the source of slice J (the double
    sum of Eq. A7 written out; O(N^2 M) matrix products)."""
    u = np.asarray(u, np.float64)
    M, N = prob.M, prob.N
    grad = np.zeros((M, N))
    for e in range(prob.E):
        H = slice_hamiltonians(prob, u, e)
        eig = [expm_herm(h, prob.dt) for h in H]
        U = np.stack([x[0] for x in eig])
        psi = propagate(prob.psi0, U)
        _, _, _, oN, oj = _member_costs(prob, psi)
        src = _sources(prob, psi, oN, oj, 1.0 / prob.E)
        for j in range(1, N + 1):
            _, V, lam = eig[j - 1]
            for k in range(M):
                tang = dexpm_herm(V, lam, prob.Hk[k], prob.dt) @ psi[j - 1]
                total = np.real(np.sum(src[j].conj() * tang))
                for J in range(j + 1, N + 1):
                    tang = U[J - 1] @ tang
                    total += np.real(np.sum(src[J].conj() * tang))
                grad[k, j - 1] += total
    _, _, g3, g4 = _control_terms(u)
    return grad + prob.alpha[1] * g3 + prob.alpha[2] * g4


# ----------------------------------------------------------------------------------------
# The paper's backward-propagation algorithms (Appendix A), with the exact dU_j
# ----------------------------------------------------------------------------------------
def _setup_single(prob, u):
    H = slice_hamiltonians(prob, u, 0)
    eig = [expm_herm(h, prob.dt) for h in H]
    U = np.stack([x[0] for x in eig])
    return eig, U, propagate(prob.psi0, U)


def grad_paper_alg1(prob, u: np.ndarray, exact: bool = True) -> np.ndarray:
    """Algorithm 1 (C1 gradient via backward propagation): P = tr(K_T^dag K_N)^* K_T^dag,
    X = K_N; at each slice from N down to 1 the gradient is read from (P, X), then
    X <- U_j^dag X and P <- P U_j.  Includes the 1/D^2 of C1 = 1 - |tr(.)/D|^2 that the paper
    drops, and uses dU_j (exact, or -i dt H_k U_j with ``exact=False``) in place of H_k."""
    eig, U, K = _setup_single(prob, u)
    D, N = prob.d, prob.N
    KT = prob.psiT
    P = np.trace(KT.conj().T @ K[N]).conjugate() * KT.conj().T
    X = K[N].copy()
    grad = np.zeros((prob.M, N))
    for j in range(N, 0, -1):
        _, V, lam = eig[j - 1]
        for k, dU in enumerate(_dU_list(prob, V, lam, exact, U[j - 1])):
            grad[k, j - 1] = -2.0 * np.real(np.trace(P @ dU @ U[j - 1].conj().T @ X)) / D ** 2
        X = U[j - 1].conj().T @ X
        P = P @ U[j - 1]
    return grad


def grad_paper_alg2(prob, u: np.ndarray, exact: bool = True) -> np.ndarray:
    """Algorithm 2 (C2 gradient via backward propagation) for one initial state:
    P = <Psi_T|Psi_N>^* <Psi_T|, X = |Psi_N>; X <- U_j^dag X, P <- P U_j."""
    eig, U, psi = _setup_single(prob, u)
    N = prob.N
    tgt = prob.psiT[:, 0]
    X = psi[N][:, 0].copy()
    P = np.vdot(tgt, X).conjugate() * tgt.conj()
    grad = np.zeros((prob.M, N))
    for j in range(N, 0, -1):
        _, V, lam = eig[j - 1]
        for k, dU in enumerate(_dU_list(prob, V, lam, exact, U[j - 1])):
            grad[k, j - 1] = -2.0 * np.real(P @ dU @ U[j - 1].conj().T @ X)
        X = U[j - 1].conj().T @ X
        P = P @ U[j - 1]
    return grad


def grad_paper_alg3(prob, u: np.ndarray, exact: bool = True) -> np.ndarray:
    """Algorithm 3 (C5 gradient via backward propagation) for one initial state and the
    forbidden projector P_F = sum_{f in F} |f><f|: P = <Psi_N|P_F, X = |Psi_N>; after reading
    the gradient at slice j: X <- U_j^dag X, P <- P U_j + <X|P_F."""
    eig, U, psi = _setup_single(prob, u)
    N = prob.N
    PF = np.zeros((prob.d, prob.d))
    PF[prob.forbidden, prob.forbidden] = 1.0
    X = psi[N][:, 0].copy()
    P = X.conj() @ PF
    grad = np.zeros((prob.M, N))
    for j in range(N, 0, -1):
        _, V, lam = eig[j - 1]
        for k, dU in enumerate(_dU_list(prob, V, lam, exact, U[j - 1])):
            grad[k, j - 1] = 2.0 * np.real(P @ dU @ U[j - 1].conj().T @ X)
        X = U[j - 1].conj().T @ X
        P = P @ U[j - 1] + X.conj() @ PF
    return grad


# ----------------------------------------------------------------------------------------
# Sec. III: truncated Taylor series with scaling and squaring (diagnostic mode)
# ----------------------------------------------------------------------------------------
def taylor_expm(X: np.ndarray, p: int, n: int) -> np.ndarray:
    """[sum_{k=0..p} X^k / k!]^(2^n) for X already scaled by 2^-n (Eq. 10), by plain power
    sums followed by n squarings (Eq. 9)."""
    d = X.shape[0]
    T = np.eye(d, dtype=np.complex128)
    term = np.eye(d, dtype=np.complex128)
    for k in range(1, p + 1):
        term = term @ X / k
        T = T + term
    for _ in range(n):
        T = T @ T
    return T


def _taylor_adjoint(X: np.ndarray, p: int, n: int, Ubar: np.ndarray) -> np.ndarray:
    """Xbar for U = taylor_expm(X, p, n) and cotangent Ubar, from the definition:
    squarings S_{m+1} = S_m^2 give Sbar_m = Sbar_{m+1} S_m^dag + S_m^dag Sbar_{m+1};
    T = sum_k X^k/k! gives Xbar = sum_{k>=1} (1/k!) sum_{a=0}^{k-1} (X^dag)^a Tbar (X^dag)^{k-1-a}."""
    d = X.shape[0]
    T = taylor_expm(X, p, 0)
    S = [T]
    for _ in range(n):
        S.append(S[-1] @ S[-1])
    Sbar = Ubar
    for m in range(n - 1, -1, -1):
        Sbar = Sbar @ S[m].conj().T + S[m].conj().T @ Sbar
    Tbar = Sbar
    Xh = X.conj().T
    powers = [np.eye(d, dtype=np.complex128)]
    for _ in range(p):
        powers.append(powers[-1] @ Xh)
    Xbar = np.zeros_like(X)
    for k in range(1, p + 1):
        acc = np.zeros_like(X)
        for a in range(k):
            acc += powers[a] @ Tbar @ powers[k - 1 - a]
        Xbar += acc / math.factorial(k)
    return Xbar


def theta_bound(prob, u: np.ndarray) -> float:
    """theta = dt * max_{j,e} (||H_0||_1 + |delta_e| ||H_det||_1 + sum_k |u_{k,j}| ||H_k||_1),
    an upper bound on ||H_j dt|| from the triangle inequality in the induced 1-norm (max
    absolute column sum).  No per-slice spectral estimate (Sec. III)."""
    def n1(a):
        return float(np.max(np.sum(np.abs(a), axis=0)))
    base = n1(prob.H0)
    if prob.Hdet is not None:
        base += float(np.max(np.abs(prob.delta))) * n1(prob.Hdet)
    hk = np.array([n1(h) for h in prob.Hk]) if prob.M else np.zeros(0)
    per_slice = np.abs(np.asarray(u, np.float64)).T @ hk if prob.M else np.zeros(prob.N)
    return prob.dt * (base + float(np.max(per_slice)))


def pick_pn(theta: float, theta_max: float, tol: float, p_max: int = 40) -> Tuple[int, int]:
    """One conservative global (p, n) for all slices (Sec. III): n is the least non-negative
    integer with theta / 2^n <= theta_max; p is the least order whose Taylor remainder bound,
    amplified by the 2^n squarings,
        2^n * ts^(p+1) / (p+1)! / (1 - ts/(p+2)) <= tol,   ts = theta / 2^n,
    holds."""
    n = 0
    while theta / (2.0 ** n) > theta_max:
        n += 1
    ts = theta / (2.0 ** n)
    p = 1
    while p < p_max:
        rem = (2.0 ** n) * ts ** (p + 1) / math.factorial(p + 1) / (1.0 - ts / (p + 2))
        if rem <= tol:
            break
        p += 1
    return p, n


def taylor_cost_and_grad(prob, u: np.ndarray, p: int, n: int) -> Tuple[float, np.ndarray, np.ndarray]:
    """Cost and exact gradient of the truncated-series method of Sec. III at fixed (p, n):
    U_j = taylor_expm(-i dt 2^-n H_j, p, n), same costs and costate recursion as
    ``cost_and_grad``, and dC/du_{k,j} = Re tr(Xbar_j^dag (-i dt 2^-n H_k))."""
    u = np.asarray(u, np.float64)
    M, N = prob.M, prob.N
    scale = prob.dt / (2.0 ** n)
    grad = np.zeros((M, N))
    acc = np.zeros(3)
    for e in range(prob.E):
        H = slice_hamiltonians(prob, u, e)
        Xs = [-1j * scale * h for h in H]
        U = np.stack([taylor_expm(x, p, n) for x in Xs])
        psi = propagate(prob.psi0, U)
        c_fid, c5, c67, oN, oj = _member_costs(prob, psi)
        acc += (c_fid, c5, c67)
        src = _sources(prob, psi, oN, oj, 1.0 / prob.E)
        G = src[N].copy()
        for j in range(N, 0, -1):
            Ubar = G @ psi[j - 1].conj().T
            Xbar = _taylor_adjoint(Xs[j - 1], p, n, Ubar)
            for k in range(M):
                grad[k, j - 1] += np.real(np.sum(Xbar.conj() * (-1j * scale * prob.Hk[k])))
            G = U[j - 1].conj().T @ G + src[j - 1]
    acc /= prob.E
    c3, c4, g3, g4 = _control_terms(u)
    a = prob.alpha
    grad += a[1] * g3 + a[2] * g4
    terms = np.array([acc[0], c3, c4, acc[1], acc[2]])
    return float(np.dot(a, terms)), grad, terms
