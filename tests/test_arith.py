"""CPU checks of two arithmetic facts the FP32 kernels rely on, written out in NumPy:

* grid split: with v1 = v rounded to the power-of-two grid 2^(e-12), where 2^e bounds the row
  (column) 2-norms, every partial sum of a row-times-column contraction of grid parts is exact in
  FP32 (products of 13-bit grid parts are exact and, by Cauchy-Schwarz, the sums stay below 2^24
  grid units), and grid sums plus FP32 cross terms reproduce the FP64 product to ~2^-36;
* low-rank reverse mode: for a cotangent Ubar = L R^dag of rank S, the reverse mode through the
  squarings and the Horner steps of the truncated series keeps it as factors (the rank doubles at
  each squaring, R stays fixed through Horner), and gives the same Xbar as the dense reverse mode,
  which itself matches a finite-difference derivative of the truncated series;
* block form: for the polynomial map f (Horner series, then squarings) with real coefficients, the
  same Xbar is the (1,2) block of f applied to [[X^dag, Ubar], [0, X^dag]];
* Paterson-Stockmeyer form: the same truncated series evaluated in blocks of three terms,
  T = B_0 + Y(B_1 + Y(B_2 + ...)) with Y = X^3 and B_q = c_3q I + c_3q+1 X + c_3q+2 X^2, and its
  reverse mode (dense and low-rank), in the order and with the stored operands the FP32 per-slice
  kernels use, agree with the Horner forms above.
"""
import numpy as np
import pytest

f32 = np.float32


def grid_split(v, e):
    """FP64 array -> (v1, v2) FP32 with v1 on the grid 2^(e-12) and v2 = v - v1 rounded."""
    g = 2.0 ** (e - 12)
    v1 = (np.rint(v / g) * g).astype(f32)
    v2 = (v - v1.astype(np.float64)).astype(f32)
    return v1, v2


def random_unitary(d, rng):
    q, r = np.linalg.qr(rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("d", [8, 40, 81])
def test_grid_sums_are_exact_and_products_accurate(d):
    rng = np.random.default_rng(d)
    A, B = random_unitary(d, rng), random_unitary(d, rng)   # row / column 2-norms 1 <= 2^1
    a1r, a2r = grid_split(A.real, 1)
    a1i, a2i = grid_split(A.imag, 1)
    b1r, b2r = grid_split(B.real, 1)
    b1i, b2i = grid_split(B.imag, 1)
    bfr, bfi = (b1r + b2r).astype(f32), (b1i + b2i).astype(f32)
    Sr = np.zeros((d, d), f32)
    Lr = np.zeros((d, d), f32)
    for k in range(d):   # FP32 accumulation in k order; each step's products are exact here
        Sr = (Sr + a1r[:, k:k + 1] * b1r[k]).astype(f32)
        Sr = (Sr - a1i[:, k:k + 1] * b1i[k]).astype(f32)
        Lr = (Lr + a1r[:, k:k + 1] * b2r[k]).astype(f32)
        Lr = (Lr - a1i[:, k:k + 1] * b2i[k]).astype(f32)
        Lr = (Lr + a2r[:, k:k + 1] * bfr[k]).astype(f32)
        Lr = (Lr - a2i[:, k:k + 1] * bfi[k]).astype(f32)
    exact_S = a1r.astype(float) @ b1r.astype(float) - a1i.astype(float) @ b1i.astype(float)
    assert np.array_equal(Sr.astype(float), exact_S)
    err = np.abs(Sr.astype(float) + Lr.astype(float) - (A @ B).real).max()
    assert err < 2e-9
    plain = np.abs((A.astype(np.complex64) @ B.astype(np.complex64)).real - (A @ B).real).max()
    assert err < plain / 50


def taylor_forward(X, p, n):
    """Horner T = I + X(I + X/2(... (I + X/p))) and n squarings; returns U and the right operand of
    every product in the order the forward meets them (Z_{i+1} for Horner step i = p-1..1, then
    S_m = T^(2^m))."""
    d = X.shape[0]
    I = np.eye(d)
    Z = I + X / p
    ops = []
    for i in range(p - 1, 0, -1):
        ops.append(Z)
        Z = I + X @ Z / i
    for _ in range(n):
        ops.append(Z)
        Z = Z @ Z
    return Z, ops


def reverse_dense(X, Ubar, p, n):
    _, ops = taylor_forward(X, p, n)
    XH = X.conj().T
    Sbar = Ubar
    for m in range(n - 1, -1, -1):
        S = ops[p - 1 + m]
        Sbar = Sbar @ S.conj().T + S.conj().T @ Sbar
    Zbar = Sbar
    Xbar = np.zeros_like(X)
    for i in range(1, p):
        Znext = ops[p - 1 - i]   # Z_{i+1}
        Xbar = Xbar + Zbar @ Znext.conj().T / i
        Zbar = XH @ Zbar / i
    return Xbar + Zbar / p


def reverse_low_rank(X, L, R, p, n):
    _, ops = taylor_forward(X, p, n)
    XH = X.conj().T
    for m in range(n - 1, -1, -1):   # Sbar = L R^dag -> [L, S^dag L] [S R, R]^dag
        S = ops[p - 1 + m]
        L, R = np.hstack([L, S.conj().T @ L]), np.hstack([S @ R, R])
    Xbar = np.zeros_like(X)
    for i in range(1, p):            # R fixed; L_{i+1} = X^dag L_i / i
        Znext = ops[p - 1 - i]
        Xbar = Xbar + L @ (Znext @ R).conj().T / i
        L = XH @ L / i
    return Xbar + L @ R.conj().T / p, L.shape[1]


@pytest.mark.parametrize("d,S,p,n", [(12, 1, 9, 3), (16, 2, 7, 2), (10, 3, 5, 0), (20, 1, 12, 4)])
def test_low_rank_reverse_mode_equals_dense(d, S, p, n):
    rng = np.random.default_rng(100 * d + S)
    H = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    H = (H + H.conj().T) / 2
    X = -1j * 0.4 * H / np.abs(H).sum(0).max()
    L = rng.normal(size=(d, S)) + 1j * rng.normal(size=(d, S))
    R = rng.normal(size=(d, S)) + 1j * rng.normal(size=(d, S))
    dense = reverse_dense(X, L @ R.conj().T, p, n)
    low, r = reverse_low_rank(X, L, R, p, n)
    assert r == S << n
    assert np.abs(low - dense).max() <= 1e-12 * np.abs(dense).max()
    # the dense reverse mode is the adjoint of the truncated series' derivative:
    # Re tr(Ubar^dag dU) = Re tr(Xbar^dag dX) for a direction dX (central differences)
    dX = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    h = 1e-6
    Up, _ = taylor_forward(X + h * dX, p, n)
    Um, _ = taylor_forward(X - h * dX, p, n)
    Ubar = L @ R.conj().T
    lhs = np.real(np.trace(Ubar.conj().T @ (Up - Um) / (2 * h)))
    rhs = np.real(np.trace(dense.conj().T @ dX))
    assert abs(lhs - rhs) <= 1e-7 * max(1.0, abs(rhs))


@pytest.mark.parametrize("d,p,n", [(6, 9, 3), (11, 5, 0), (8, 14, 5)])
def test_block_triangular_form_equals_reverse_mode(d, p, n):
    rng = np.random.default_rng(d + 17 * p)
    H = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    H = (H + H.conj().T) / 2
    X = -1j * 0.5 * H / np.abs(H).sum(0).max()
    Ubar = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    XH = X.conj().T
    B = np.block([[XH, Ubar], [np.zeros((d, d)), XH]])
    FB, _ = taylor_forward(B, p, n)
    dense = reverse_dense(X, Ubar, p, n)
    assert np.abs(FB[:d, d:] - dense).max() <= 1e-12 * np.abs(dense).max()
    assert np.abs(FB[:d, :d] - taylor_forward(XH, p, n)[0]).max() < 1e-13


# ------------------------------------------------------------------ Paterson-Stockmeyer form
def ps_coefficients(p):
    """c_k = 1/k! for k <= p and 0 beyond (indices up to p + 3 are read)."""
    c = np.zeros(p + 4)
    f = 1.0
    for k in range(p + 1):
        if k:
            f *= k
        c[k] = 1.0 / f
    return c


def ps_top(p):
    """Index qt of the top block, formed without a product: blocks q = 0 .. p // 3; when 3 divides
    p the last block is c_p I alone and is folded into the one below it as c_p X^3."""
    Q = p // 3
    return Q - 1 if (p % 3 == 0 and p >= 3) else Q


def ps_forward(X, p, n):
    """The order-p Taylor polynomial by Paterson-Stockmeyer with block size 3, then n squarings.
    Returns U and the operands the reverse mode reads, in store-slot order: X^2, X^3, then the
    right operands W_{q+1} of the chain products q = qt-1 .. 0, then S_m = T^(2^m)."""
    d = X.shape[0]
    I = np.eye(d)
    c = ps_coefficients(p)
    P2 = X @ X
    P3 = P2 @ X
    qt = ps_top(p)
    W = c[3 * qt] * I + c[3 * qt + 1] * X + c[3 * qt + 2] * P2 + c[3 * qt + 3] * P3
    ops = [P2, P3]
    for q in range(qt - 1, -1, -1):
        ops.append(W)
        W = c[3 * q] * I + c[3 * q + 1] * X + c[3 * q + 2] * P2 + P3 @ W
    for _ in range(n):
        ops.append(W)
        W = W @ W
    return W, ops


def ps_slots(p, n):
    return ps_top(p) + 2 + n


def ps_powers_reverse(X, P2, P3bar, P2bar, Xbar):
    """P3 = P2 X and P2 = X X in reverse: the four dense products that end both reverse modes."""
    XH = X.conj().T
    P2bar = P2bar + P3bar @ XH
    Xbar = Xbar + P2.conj().T @ P3bar
    return Xbar + P2bar @ XH + XH @ P2bar


def ps_reverse_dense(X, Ubar, p, n):
    _, ops = ps_forward(X, p, n)
    c = ps_coefficients(p)
    qt = ps_top(p)
    P2, P3 = ops[0], ops[1]
    Sbar = Ubar
    for m in range(n - 1, -1, -1):
        S = ops[qt + 2 + m]
        Sbar = Sbar @ S.conj().T + S.conj().T @ Sbar
    Wbar = Sbar
    Xbar = np.zeros_like(X)
    P2bar = np.zeros_like(X)
    P3bar = np.zeros_like(X)
    for q in range(qt):                      # chain products in reverse: W_q = B_q + P3 W_{q+1}
        Wnext = ops[2 + (qt - 1 - q)]
        Xbar = Xbar + c[3 * q + 1] * Wbar
        P2bar = P2bar + c[3 * q + 2] * Wbar
        P3bar = P3bar + Wbar @ Wnext.conj().T
        Wbar = P3.conj().T @ Wbar
    Xbar = Xbar + c[3 * qt + 1] * Wbar       # the top block
    P2bar = P2bar + c[3 * qt + 2] * Wbar
    P3bar = P3bar + c[3 * qt + 3] * Wbar
    return ps_powers_reverse(X, P2, P3bar, P2bar, Xbar)


def ps_reverse_low_rank(X, L, R, p, n):
    """Ubar = L R^dag: the squarings append blocks to the factors; through the chain R stays fixed
    and L_{q+1} = P3^dag L_q, so the X and X^2 cotangents are (sum c L_q) R^dag and the X^3
    cotangent is sum_q L_q (W_{q+1} R)^dag; the powers then go dense."""
    _, ops = ps_forward(X, p, n)
    c = ps_coefficients(p)
    qt = ps_top(p)
    P2, P3 = ops[0], ops[1]
    for m in range(n - 1, -1, -1):
        S = ops[qt + 2 + m]
        L, R = np.hstack([L, S.conj().T @ L]), np.hstack([S @ R, R])
    A1 = np.zeros_like(L)
    A2 = np.zeros_like(L)
    P3bar = np.zeros_like(X)
    for q in range(qt):
        Wnext = ops[2 + (qt - 1 - q)]
        A1 = A1 + c[3 * q + 1] * L
        A2 = A2 + c[3 * q + 2] * L
        P3bar = P3bar + L @ (Wnext @ R).conj().T
        L = P3.conj().T @ L
    A1 = A1 + c[3 * qt + 1] * L
    A2 = A2 + c[3 * qt + 2] * L
    P3bar = P3bar + c[3 * qt + 3] * L @ R.conj().T
    RH = R.conj().T
    return ps_powers_reverse(X, P2, P3bar, A2 @ RH, A1 @ RH), L.shape[1]


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 9, 11, 12, 14])
@pytest.mark.parametrize("n", [0, 2])
def test_paterson_stockmeyer_equals_horner(p, n):
    """Same polynomial, another evaluation order: U and the dense and low-rank reverse modes agree
    with the Horner forms to rounding, for every residue of p mod 3."""
    d, S = 14, 1
    rng = np.random.default_rng(7 * p + n)
    H = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    H = (H + H.conj().T) / 2
    X = -1j * 1.6 * H / np.abs(H).sum(0).max()       # theta_s = 1.6, the FP32 kernels' range
    U_ps, ops = ps_forward(X, p, n)
    U_h, _ = taylor_forward(X, p, n)
    assert np.abs(U_ps - U_h).max() <= 1e-13 * np.abs(U_h).max()
    assert len(ops) == ps_slots(p, n)
    L = rng.normal(size=(d, S)) + 1j * rng.normal(size=(d, S))
    R = rng.normal(size=(d, S)) + 1j * rng.normal(size=(d, S))
    Ubar = L @ R.conj().T
    ref = reverse_dense(X, Ubar, p, n)
    dense = ps_reverse_dense(X, Ubar, p, n)
    low, r = ps_reverse_low_rank(X, L, R, p, n)
    assert r == S << n
    scale = np.abs(ref).max()
    assert np.abs(dense - ref).max() <= 1e-12 * scale
    assert np.abs(low - ref).max() <= 1e-12 * scale
