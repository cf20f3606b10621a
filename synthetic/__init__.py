"""Seeded synthetic inputs for the quantum-control cost evaluation.

This module only *builds problem inputs*: Hamiltonian matrices of the physical systems the
paper studies (Sec. V and Sec. IV), control amplitudes, initial and target states.  It holds
none of the method's arithmetic (no exponentials, no propagation, no costs, no gradients), so
both the CPU oracle and the CUDA path can take their inputs from here.

Units: hbar = 1, energies in rad/ns (2*pi * frequency in GHz), time in ns, so that H*dt is
dimensionless.

Every generator is deterministic in its seed (numpy ``default_rng``).  The paper uses no
dataset: all of its workloads are physically specified systems, and the five workloads below
follow them:

* ``cnot2q``      -- two coupled qubits (d=4), CNOT gate, full unitary, FP64 form.
* ``transmon_cavity`` -- transmon(4) x cavity(10), d=40, |g,0> -> |g,1> with a forbidden-level
  penalty at every slice (Sec. V.C style system, Table I C2 + C5).
* ``transmon4``   -- four 3-level transmons in an open chain, d=81, Haar target on the qubit
  subspace with a leakage penalty (Sec. II.A C2-Sigma + C5).
* ``gue256``      -- eight qubits, d=256, GUE drift, 16 Pauli x/y controls, Haar target.
* ``batch``       -- 128 independent problems of uneven (d, N, M) with detuning ensembles.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

TWO_PI = 2.0 * math.pi

# cost weights are ordered [fid, C3 amplitude, C4 variation, C5 forbidden, C6/C7 time]
ALPHA_FID, ALPHA_AMP, ALPHA_VAR, ALPHA_FORBID, ALPHA_TIME = range(5)


@dataclass
class Problem:
    """One control problem: H_j = H0 + sum_k u[k, j] Hk[k] (+ delta_e * Hdet per ensemble member)."""

    name: str
    H0: np.ndarray                  # (d, d) complex128, Hermitian
    Hk: np.ndarray                  # (M, d, d) complex128, Hermitian
    dt: float
    N: int
    psi0: np.ndarray                # (d, S) complex128, initial columns
    psiT: np.ndarray                # (d, S) complex128, final targets
    forbidden: np.ndarray           # (nF,) int32 basis indices
    col_weight: np.ndarray          # (S,) float64 weights of the propagated columns
    alpha: np.ndarray               # (5,) float64 weights [fid, C3, C4, C5, C6/7]
    u: np.ndarray                   # (M, N) float64 controls (the evaluation point)
    psiT_path: Optional[np.ndarray] = None   # (N, d, S) per-slice targets, or None
    delta: np.ndarray = field(default_factory=lambda: np.zeros(1))  # (E,) detunings
    Hdet: Optional[np.ndarray] = None        # (d, d) detuning operator, or None
    precision: str = "fp64"

    @property
    def d(self) -> int:
        return self.H0.shape[0]

    @property
    def M(self) -> int:
        return self.Hk.shape[0]

    @property
    def S(self) -> int:
        return self.psi0.shape[1]

    @property
    def E(self) -> int:
        return len(self.delta)


# ----------------------------------------------------------------------------------------
# operator building blocks
# ----------------------------------------------------------------------------------------
SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)


def kron_all(ops) -> np.ndarray:
    out = np.array([[1.0 + 0j]])
    for op in ops:
        out = np.kron(out, op)
    return out


def embed(op: np.ndarray, site: int, dims: List[int]) -> np.ndarray:
    """Operator ``op`` acting on ``site`` of a tensor product with local dimensions ``dims``
    (site 0 is the most significant index of the basis)."""
    ops = [np.eye(n, dtype=np.complex128) for n in dims]
    ops[site] = op
    return kron_all(ops)


def lowering(n: int) -> np.ndarray:
    """Truncated annihilation operator b on n levels: b|m> = sqrt(m)|m-1>."""
    return np.diag(np.sqrt(np.arange(1, n, dtype=np.float64)), k=1).astype(np.complex128)


def number(n: int) -> np.ndarray:
    return np.diag(np.arange(n, dtype=np.float64)).astype(np.complex128)


def haar_unitary(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed unitary: QR of a complex Ginibre matrix with the phases of R's diagonal
    divided out (Mezzadri 2007)."""
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def gue(n: int, rng: np.random.Generator, spectral_norm: float) -> np.ndarray:
    """GUE matrix (G + G^dagger)/2 rescaled to the given spectral norm."""
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    h = 0.5 * (g + g.conj().T)
    s = np.max(np.abs(np.linalg.eigvalsh(h)))
    return h * (spectral_norm / s)


def pauli_controls(nq: int, m: int) -> np.ndarray:
    """The first m of [sx_0, sy_0, sx_1, sy_1, ...] on nq qubits."""
    dims = [2] * nq
    ops = []
    for q in range(nq):
        ops.append(embed(SX, q, dims))
        ops.append(embed(SY, q, dims))
    return np.stack(ops[:m])


def ladder_controls(dims: List[int], sites: List[int], m: int) -> np.ndarray:
    """The first m of [x_s, y_s for s in sites] with x = b + b^dag, y = i(b^dag - b)."""
    ops = []
    for s in sites:
        b = lowering(dims[s])
        ops.append(embed(b + b.conj().T, s, dims))
        ops.append(embed(1j * (b.conj().T - b), s, dims))
    return np.stack(ops[:m])


def basis_state(d: int, idx: int) -> np.ndarray:
    v = np.zeros((d, 1), dtype=np.complex128)
    v[idx, 0] = 1.0
    return v


def default_alpha(fid=1.0, amp=0.0, var=0.0, forbid=0.0, time=0.0) -> np.ndarray:
    return np.array([fid, amp, var, forbid, time], dtype=np.float64)


# ----------------------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------------------
def cnot2q(seed: int = 1000, N: int = 200) -> Problem:
    """Two coupled qubits, d=4: H0 = 2pi*0.01 sz(x)sz, controls sx(x)I, sy(x)I, I(x)sx, I(x)sy,
    dt = 0.5 ns, u ~ N(0, (2pi*0.02)^2), CNOT target (qubit 1 = first factor controls),
    full-unitary propagation, cost 1 - |tr(K_T^dag K_N)/4|^2 (Table I, C1)."""
    rng = np.random.default_rng(seed)
    H0 = TWO_PI * 0.01 * np.kron(SZ, SZ)
    Hk = np.stack([np.kron(SX, I2), np.kron(SY, I2), np.kron(I2, SX), np.kron(I2, SY)])
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
    u = rng.normal(0.0, TWO_PI * 0.02, size=(4, N))
    return Problem("cnot2q_d4", H0, Hk, 0.5, N, np.eye(4, dtype=np.complex128), cnot,
                   np.zeros(0, np.int32), np.ones(4), default_alpha(), u, precision="fp64")


def transmon_cavity(seed: int = 2000, N: int = 2000, nt: int = 4, nc: int = 10) -> Problem:
    """Transmon (nt levels) x cavity (nc levels) in the rotating frame, transmon-major basis
    (index = nc*t + c).  H0 = (alpha/2) n_t(n_t - 1) (x) I + chi n_t (x) n_c with
    alpha = -2pi*0.225, chi = -2pi*0.002; controls are the transmon x/y drives; dt = 1 ns;
    |g,0> -> |g,1> state transfer (C2) plus a forbidden-occupation penalty (C5) on transmon
    level nt-1 and cavity level nc-1 at every slice, weight 1/(N*S)."""
    rng = np.random.default_rng(seed)
    d = nt * nc
    al, chi = -TWO_PI * 0.225, -TWO_PI * 0.002
    nt_op, nc_op = number(nt), number(nc)
    H0 = 0.5 * al * np.kron(nt_op @ (nt_op - np.eye(nt)), np.eye(nc)) + chi * np.kron(nt_op, nc_op)
    Hk = ladder_controls([nt, nc], [0], 2)
    forb = sorted({nc * (nt - 1) + c for c in range(nc)} | {nc * t + (nc - 1) for t in range(nt)})
    u = rng.normal(0.0, TWO_PI * 0.02, size=(2, N))
    return Problem(f"transmon_cavity_d{d}", H0, Hk, 1.0, N, basis_state(d, 0), basis_state(d, 1),
                   np.array(forb, np.int32), np.ones(1),
                   default_alpha(forbid=1.0 / N), u, precision="fp32")


def transmon4(seed: int = 3000, N: int = 1000, levels: int = 3, nq: int = 4) -> Problem:
    """Four 3-level transmons, d=81, open chain with exchange J(b_i^dag b_{i+1} + h.c.),
    J = 2pi*0.005, anharmonicity alpha = -2pi*0.2, 8 x/y drives with u ~ N(0, (2pi*0.03)^2),
    dt = 0.5 ns.  All 81 columns are propagated (Psi_0 = I); the fidelity is taken on the 16
    columns of the qubit subspace against a Haar-random 16x16 target embedded there, and the
    leakage penalty (C5) counts every basis state with a transmon in level 2, summed over the
    16 subspace columns with weight 1/(16 N).  The other 65 columns carry weight 0."""
    rng = np.random.default_rng(seed)
    dims = [levels] * nq
    d = levels ** nq
    al, J = -TWO_PI * 0.2, TWO_PI * 0.005
    H0 = np.zeros((d, d), np.complex128)
    for i in range(nq):
        n = number(levels)
        H0 += embed(0.5 * al * n @ (n - np.eye(levels)), i, dims)
    for i in range(nq - 1):
        b = lowering(levels)
        hop = kron_all([np.eye(levels)] * i + [b.conj().T, b] + [np.eye(levels)] * (nq - i - 2))
        H0 += J * (hop + hop.conj().T)
    Hk = ladder_controls(dims, list(range(nq)), 2 * nq)
    digits = np.array(np.unravel_index(np.arange(d), dims)).T      # (d, nq) level of each transmon
    sub = np.where(np.all(digits <= 1, axis=1))[0]                  # 16 qubit-subspace states
    forb = np.where(np.any(digits == 2, axis=1))[0].astype(np.int32)
    V = haar_unitary(len(sub), rng)
    psiT = np.zeros((d, d), np.complex128)
    for a, sa in enumerate(sub):
        for b_, sb in enumerate(sub):
            psiT[sa, sb] = V[a, b_]
    w = np.zeros(d)
    w[sub] = 1.0
    u = rng.normal(0.0, TWO_PI * 0.03, size=(2 * nq, N))
    return Problem(f"transmon4_d{d}", H0, Hk, 0.5, N, np.eye(d, dtype=np.complex128), psiT,
                   forb, w, default_alpha(forbid=1.0 / (len(sub) * N)), u, precision="tf32")


def gue256(seed: int = 4000, N: int = 2000, nq: int = 8, M: int = 16) -> Problem:
    """Eight qubits, d=256: GUE drift with spectral norm 2pi*0.05, 16 Pauli x/y controls,
    u ~ N(0, (2pi*0.02)^2), dt = 0.25 ns, Haar-random 256x256 target, full unitary (C1)."""
    rng = np.random.default_rng(seed)
    d = 2 ** nq
    H0 = gue(d, rng, TWO_PI * 0.05)
    Hk = pauli_controls(nq, M)
    V = haar_unitary(d, rng)
    u = rng.normal(0.0, TWO_PI * 0.02, size=(M, N))
    return Problem(f"gue256_d{d}", H0, Hk, 0.25, N, np.eye(d, dtype=np.complex128), V,
                   np.zeros(0, np.int32), np.ones(d), default_alpha(), u, precision="bf16")


def batch_problem(idx: int, ensemble: int = 1, seed_base: int = 5000,
                  d_choices=(4, 8, 16, 40, 81, 128), n_range=(200, 4000)) -> Problem:
    """Problem ``idx`` of the batched sweep: d ~ U{4,8,16,40,81,128}, N ~ U[200, 4000],
    M ~ U[2, 8] (capped by the number of available drives), GUE drift at 2pi*0.05, Pauli x/y
    controls for d = 2^m and ladder x/y drives for 40 = 4x10 and 81 = 3^4, Haar target, full
    unitary, dt = 0.5 ns, u ~ N(0, (2pi*0.02)^2).  With ``ensemble`` > 1 the members share u and
    add delta_e * Hdet with delta ~ N(0, (2pi*0.001)^2) and Hdet = total excitation number."""
    rng = np.random.default_rng(seed_base + idx)
    d = int(rng.choice(d_choices))
    N = int(rng.integers(n_range[0], n_range[1] + 1))
    M = int(rng.integers(2, 9))
    if d in (40,):
        dims, sites = [4, 10], [0, 1]
    elif d == 81:
        dims, sites = [3, 3, 3, 3], [0, 1, 2, 3]
    else:
        nq = int(round(math.log2(d)))
        dims, sites = [2] * nq, list(range(nq))
    if all(n == 2 for n in dims):
        M = min(M, 2 * len(dims))
        Hk = pauli_controls(len(dims), M)
    else:
        M = min(M, 2 * len(sites))
        Hk = ladder_controls(dims, sites, M)
    H0 = gue(d, rng, TWO_PI * 0.05)
    V = haar_unitary(d, rng)
    u = rng.normal(0.0, TWO_PI * 0.02, size=(M, N))
    Hdet = sum(embed(number(n), s, dims) for s, n in enumerate(dims))
    delta = np.zeros(1) if ensemble <= 1 else rng.normal(0.0, TWO_PI * 0.001, size=ensemble)
    return Problem(f"batch{idx}_d{d}", H0, Hk, 0.5, N, np.eye(d, dtype=np.complex128), V,
                   np.zeros(0, np.int32), np.ones(d), default_alpha(), u,
                   delta=delta, Hdet=Hdet, precision="fp32")


def batch_problems(count: int = 128, ensemble: int = 1, **kw) -> List[Problem]:
    """The batched sweep: problems 0..count-1 (keyword arguments go to ``batch_problem``)."""
    return [batch_problem(i, ensemble=ensemble, **kw) for i in range(count)]


def dsweep_problem(d: int, seed: int = 6000, N: int = 2000) -> Problem:
    """One point of the per-d sweep, d a power of two: log2(d) qubits, GUE drift with spectral norm
    2pi*0.05, Pauli x/y controls on the first two qubits (one x control for d = 2), Haar target,
    full unitary, dt = 0.5 ns, u ~ N(0, (2pi*0.02)^2); FP32."""
    rng = np.random.default_rng(seed + d)
    nq = int(round(math.log2(d)))
    H0 = gue(d, rng, TWO_PI * 0.05)
    Hk = pauli_controls(nq, 1 if nq == 1 else 4)
    M = Hk.shape[0]
    V = haar_unitary(d, rng)
    u = rng.normal(0.0, TWO_PI * 0.02, size=(M, N))
    return Problem(f"dsweep_d{d}", H0, Hk, 0.5, N, np.eye(d, dtype=np.complex128), V, np.zeros(0, np.int32),
                   np.ones(d), default_alpha(), u, precision="fp32")


def transmon_cnot(seed: int = 7000, N: int = 250, T: float = 10.0, levels: int = 5) -> Problem:
    """Two coupled transmons with `levels` levels each (d = 25), the CNOT of Sec. V.A in the frame
    rotating at the first transmon's frequency: H0 = Delta n_2 + sum_j (alpha/2) n_j (n_j - 1)
    + J (b_1^dag b_2 + b_1 b_2^dag) with Delta = 2pi*0.4 (3.9 - 3.5 GHz), alpha = -2pi*0.225,
    J = 2pi*0.1; controls x_1, y_1, x_2, y_2 (the two drive quadratures of each transmon in the
    rotating frame) and z_2 = n_2; gate time T = 10 ns in N slices.  The four computational
    states |q1 q2> (levels 0, 1) are propagated and must reach CNOT|q1 q2> (qubit 1 controls);
    levels 3 and 4 of either transmon are forbidden (C5, weight 1/(4N)), with small amplitude
    and variation penalties (C3, C4).  The controls start small and random: an optimizer's
    starting point."""
    rng = np.random.default_rng(seed)
    dims = [levels, levels]
    d = levels * levels
    al, J, delta = -TWO_PI * 0.225, TWO_PI * 0.1, TWO_PI * 0.4
    n = number(levels)
    b = lowering(levels)
    H0 = delta * embed(n, 1, dims)
    for i in range(2):
        H0 = H0 + embed(0.5 * al * n @ (n - np.eye(levels)), i, dims)
    hop = np.kron(b.conj().T, b)
    H0 = H0 + J * (hop + hop.conj().T)
    Hk = np.concatenate([ladder_controls(dims, [0, 1], 4), embed(n, 1, dims)[None]])
    comp = [levels * q1 + q2 for q1 in (0, 1) for q2 in (0, 1)]      # |00>, |01>, |10>, |11>
    cnot_of = {0: 0, 1: 1, 2: 3, 3: 2}
    psi0 = np.zeros((d, 4), np.complex128)
    psiT = np.zeros((d, 4), np.complex128)
    for s_, idx in enumerate(comp):
        psi0[idx, s_] = 1.0
        psiT[comp[cnot_of[s_]], s_] = 1.0
    digits = np.array(np.unravel_index(np.arange(d), dims)).T
    forb = np.where(np.any(digits >= 3, axis=1))[0].astype(np.int32)
    u = rng.normal(0.0, TWO_PI * 0.01, size=(Hk.shape[0], N))
    alpha = default_alpha(fid=1.0, amp=1e-6, var=1e-4, forbid=0.1 / (4 * N))
    return Problem(f"transmon_cnot_d{d}", H0, Hk, T / N, N, psi0, psiT, forb, np.ones(4), alpha, u,
                   precision="fp64")


def cat_state(seed: int = 8000, N: int = 8000, dt: float = 0.005, nq: int = 7, nr: int = 22,
              lam: float = 2.0, ensemble: int = 1) -> Problem:
    """Schroedinger-cat state preparation (Sec. V.C): a transmon (nq = 7 levels) coupled to a
    cavity mode (nr = 22 levels), d = 154, in the lab frame without the rotating-wave
    approximation, transmon-major basis (index = nr * t + r):
    H0 = w_q n_b + (alpha/2) n_b (n_b - 1) + w_r n_a + g (a + a^dag)(b + b^dag) with
    w_q = 2pi*3.5, alpha = -2pi*0.225, w_r = 2pi*3.9, g = 2pi*0.1; controls on the transmon only,
    H_x = b + b^dag and H_z = n_b.  N = 8000 slices of dt = 5 ps (T = 40 ns).  State transfer
    |0>_q |0>_r -> |0>_q |cat>_r with |cat> = (|lam> + |-lam>) / norm, lam = 2, built from the
    coherent states of the truncated mode and normalised (C2); occupation of transmon levels 3..6
    and cavity levels 20, 21 is penalised (C5, weight 1/N), with a small variation penalty (C4).
    The controls start small and random.  With ensemble > 1 the members add delta_e n_b (a
    transmon frequency offset, delta ~ N(0, (2pi*0.001)^2)) for robust control."""
    rng = np.random.default_rng(seed)
    d = nq * nr
    wq, al, wr, g = TWO_PI * 3.5, -TWO_PI * 0.225, TWO_PI * 3.9, TWO_PI * 0.1
    b, a = lowering(nq), lowering(nr)
    nb, na = number(nq), number(nr)
    Iq, Ir = np.eye(nq), np.eye(nr)
    H0 = (np.kron(wq * nb + 0.5 * al * nb @ (nb - Iq), Ir) + np.kron(Iq, wr * na)
          + g * np.kron(b + b.conj().T, a + a.conj().T)).astype(np.complex128)
    Hk = np.stack([np.kron(b + b.conj().T, Ir), np.kron(nb, Ir)]).astype(np.complex128)
    fock = np.arange(nr)
    coh = lambda z: np.array([z ** k / math.sqrt(math.factorial(k)) for k in fock], np.complex128)
    cat = coh(lam) + coh(-lam)
    cat /= np.linalg.norm(cat)
    psiT = np.zeros((d, 1), np.complex128)
    psiT[:nr, 0] = cat                                  # transmon level 0
    forb = sorted({nr * t + r for t in range(3, nq) for r in range(nr)} |
                  {nr * t + r for t in range(nq) for r in (nr - 2, nr - 1)})
    u = rng.normal(0.0, TWO_PI * 0.02, size=(2, N))
    delta = np.zeros(1) if ensemble <= 1 else rng.normal(0.0, TWO_PI * 0.001, size=ensemble)
    return Problem(f"cat_state_d{d}" + (f"_E{ensemble}" if ensemble > 1 else ""), H0, Hk, dt, N,
                   basis_state(d, 0), psiT, np.array(forb, np.int32), np.ones(1),
                   default_alpha(var=1e-4, forbid=1.0 / N), u, delta=delta,
                   Hdet=np.kron(nb, Ir).astype(np.complex128), precision="fp32")


DSWEEP_D = (2, 4, 8, 16, 32, 64, 128, 256)

WORKLOADS = {
    "cnot2q": cnot2q,
    "transmon_cavity": transmon_cavity,
    "transmon4": transmon4,
    "gue256": gue256,
    "transmon_cnot": transmon_cnot,
    "cat_state": cat_state,
}


# ----------------------------------------------------------------------------------------
# small random problems for tests
# ----------------------------------------------------------------------------------------
def random_hermitian(d: int, rng: np.random.Generator, scale: float = 1.0) -> np.ndarray:
    g = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    return scale * 0.5 * (g + g.conj().T)


def random_states(d: int, S: int, rng: np.random.Generator) -> np.ndarray:
    """S orthonormal columns (the first S columns of a Haar unitary)."""
    return haar_unitary(d, rng)[:, :S]


def random_problem(d: int, M: int, N: int, S: int, seed: int, *, dt: float = 0.3,
                   h0_scale: float = 1.0, hk_scale: float = 0.5, u_scale: float = 1.0,
                   alpha=None, nF: int = 0, path: bool = False, E: int = 1,
                   weights: bool = False, precision: str = "fp64") -> Problem:
    """A dense random problem with every cost term switched on (unless ``alpha`` says otherwise)."""
    rng = np.random.default_rng(seed)
    H0 = random_hermitian(d, rng, h0_scale)
    Hk = np.stack([random_hermitian(d, rng, hk_scale) for _ in range(M)]) if M else \
        np.zeros((0, d, d), np.complex128)
    psi0 = random_states(d, S, rng)
    psiT = random_states(d, S, rng)
    forb = np.sort(rng.choice(d, size=min(nF, d), replace=False)).astype(np.int32)
    w = rng.uniform(0.5, 1.5, size=S) if weights else np.ones(S)
    if alpha is None:
        alpha = default_alpha(1.0, 0.05, 0.1, 0.5, 0.3)
    u = rng.normal(0.0, u_scale, size=(M, N))
    psiT_path = None
    if path:
        psiT_path = np.stack([random_states(d, S, rng) for _ in range(N)])
    delta = np.zeros(1) if E <= 1 else rng.normal(0.0, 0.3, size=E)
    Hdet = random_hermitian(d, rng, 0.5) if E > 1 else None
    return Problem(f"random_d{d}_M{M}_N{N}_S{S}", H0, Hk, dt, N, psi0, psiT, forb, w,
                   np.asarray(alpha, np.float64), u, psiT_path, delta, Hdet, precision)
