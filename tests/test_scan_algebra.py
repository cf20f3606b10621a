"""CPU check, in NumPy, of the exact reformulation of the two sequential recursions over
checkpoint segments that the CUDA path runs in parallel (the paper runs them one slice at a time):

* forward  Psi_j = U_j Psi_{j-1} (Eqs. 2, 4);
* costate  G_N = src_N, G_{j-1} = U_j^dag G_j + src_{j-1} (Appendix A, Alg. 1-3).

Slices are grouped in waves of W slices and each wave in segments z of c slices (the last ones
ragged).  Per segment the product P_z = U_b ... U_a is formed by a pairwise tree, the later factor
on the left.  Forward: a scan Psi_b = P_z Psi_{a-1} over segments gives the checkpoints, then every
segment replays its slices from its checkpoint.  Backward, per wave from the last: every segment
runs its costate from a zero in-carry, leaving h_z = U_a^dag G_a^(0); the scan
Y_{z-1} = P_z^dag Y_z + h_z gives each segment's in-carry (Y of the last segment of a wave is the
carry handed down from the wave after it); every segment then reruns from Y_z.  Both must give the
serial recursions' states and costates.  CPU only."""
import numpy as np
import pytest


def random_unitaries(n, d, rng):
    z = rng.normal(size=(n, d, d)) + 1j * rng.normal(size=(n, d, d))
    q, r = np.linalg.qr(z)
    dg = np.diagonal(r, axis1=1, axis2=2)
    return q * (dg / np.abs(dg))[:, None, :]


def serial(U, psi0, src):
    N = len(U)
    psi = [psi0]
    for j in range(N):
        psi.append(U[j] @ psi[-1])
    G = [None] * (N + 1)
    G[N] = src[N]
    for j in range(N, 1, -1):
        G[j - 1] = U[j - 1].conj().T @ G[j] + src[j - 1]
    return psi, G


def tree_product(Useg):
    """Pairwise tree over the slices of one segment: node i of level l is node 2i+1 times node
    2i of level l-1 (later factor on the left); an unpaired last node moves up unchanged."""
    nodes = list(Useg)
    while len(nodes) > 1:
        nodes = [nodes[i + 1] @ nodes[i] if i + 1 < len(nodes) else nodes[i]
                 for i in range(0, len(nodes), 2)]
    return nodes[0]


def segmented(U, psi0, src, W, c):
    N = len(U)
    waves = [(j0, min(W, N - j0)) for j0 in range(0, N, W)]
    psi = [None] * (N + 1)
    psi[0] = psi0
    for j0, wlen in waves:                          # forward: scan over segments, then replay
        segs = [(j0 + a, min(c, wlen - a)) for a in range(0, wlen, c)]
        P = [tree_product(U[a:a + n]) for a, n in segs]
        ck = psi[j0]
        starts = []
        for z, (a, n) in enumerate(segs):
            starts.append(ck)
            ck = P[z] @ ck
        for z, (a, n) in enumerate(segs):           # independent per segment
            x = starts[z]
            for j in range(a, a + n):
                x = U[j] @ x
                psi[j + 1] = x
    G = [None] * (N + 1)
    carry = np.zeros_like(src[N])                   # Y handed down from the wave after
    for j0, wlen in reversed(waves):
        segs = [(j0 + a, min(c, wlen - a)) for a in range(0, wlen, c)]
        P = [tree_product(U[a:a + n]) for a, n in segs]

        def run(a, n, y, store):
            # slices a+1 .. a+n (1-based), in-carry y on the last; returns U_{a+1}^dag G_{a+1}
            g = y + src[a + n]
            if store:
                G[a + n] = g
            for j in range(a + n, a + 1, -1):
                g = U[j - 1].conj().T @ g + src[j - 1]
                if store:
                    G[j - 1] = g
            return U[a].conj().T @ g

        h = [run(a, n, np.zeros_like(carry), False) for a, n in segs]   # zero in-carry
        Y = [None] * len(segs)
        Y[-1] = carry
        for z in range(len(segs) - 1, 0, -1):       # Y_{z-1} = P_z^dag Y_z + h_z
            Y[z - 1] = P[z].conj().T @ Y[z] + h[z]
        outs = [run(a, n, Y[z], True) for z, (a, n) in enumerate(segs)]
        carry = outs[0]                             # out of the wave's first segment
    return psi, G


@pytest.mark.parametrize("N,W,c,d,S", [(1, 1, 1, 3, 1), (17, 17, 5, 4, 2), (40, 20, 5, 3, 3),
                                       (61, 30, 6, 5, 2), (97, 45, 9, 6, 6), (13, 12, 4, 2, 1)])
def test_segmented_recursions_equal_serial(N, W, c, d, S):
    rng = np.random.default_rng(N * 100 + c)
    U = random_unitaries(N, d, rng)
    psi0 = rng.normal(size=(d, S)) + 1j * rng.normal(size=(d, S))
    src = [rng.normal(size=(d, S)) + 1j * rng.normal(size=(d, S)) for _ in range(N + 1)]
    ps, gs = serial(U, psi0, src)
    pz, gz = segmented(U, psi0, src, W, c)
    for j in range(N + 1):
        assert np.abs(pz[j] - ps[j]).max() < 1e-12
    for j in range(1, N + 1):
        assert np.abs(gz[j] - gs[j]).max() < 1e-12


def test_tree_orders_factors_later_on_the_left():
    rng = np.random.default_rng(9)
    for n in range(1, 12):
        U = random_unitaries(n, 3, rng)
        ref = np.eye(3)
        for j in range(n):
            ref = U[j] @ ref
        assert np.abs(tree_product(U) - ref).max() < 1e-13
        if n >= 2:   # the reversed order is a different matrix, so the test sees a swap
            swapped = np.eye(3)
            for j in range(n):
                swapped = swapped @ U[j]
            assert np.abs(swapped - ref).max() > 1e-3
