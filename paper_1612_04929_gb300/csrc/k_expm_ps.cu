// Reverse-mode adjoints of the Paterson-Stockmeyer form of the FP32 per-slice exponential
// (k_expm_fwd_ps): the exact derivative of the same truncated series (Eq. 10, then the squarings
// of Eq. 9) taken through the products in the order the forward ran them.  With Y = X^3,
// B_q = c_3q I + c_3q+1 X + c_3q+2 X^2 and W_q = B_q + Y W_{q+1} (T = W_0), the cotangents are
//   squarings:   Sbar_m = Sbar_{m+1} S_m^dag + S_m^dag Sbar_{m+1},          Wbar_0 = Sbar_0
//   chain q:     Xbar += c_3q+1 Wbar_q,  X2bar += c_3q+2 Wbar_q,  Ybar += Wbar_q W_{q+1}^dag,
//                Wbar_{q+1} = Y^dag Wbar_q
//   top block:   Xbar += c_3qt+1 Wbar_qt, X2bar += c_3qt+2 Wbar_qt, Ybar += c_3qt+3 Wbar_qt
//   powers:      X2bar += Ybar X^dag, Xbar += X2^dag Ybar  (Y = X^2 X),
//                Xbar += X2bar X^dag + X^dag X2bar           (X^2 = X X)
// and dC/du_kj = Re tr(Xbar^dag (-i s H_k)) (Eq. A3).  At p = 14, n = 2 that is 16 products per
// slice against 30 for the Horner reverse mode at the same (p, n).
//
//  k_expm_adj_ps    : the dense form; the stored operand of the next product arrives by cp.async
//                     while the current one is multiplied; Y^dag stays resident for the chain.
//  k_expm_adj_ps_lr : the low-rank form, when the cotangent Ubar_j = G_j Psi_{j-1}^dag (rank S)
//                     keeps a small rank r = S 2^n after the squarings: Wbar_q = L_q R^dag with R
//                     fixed through the chain and L_{q+1} = Y^dag L_q, so the X and X^2 cotangents
//                     are (sum_q c L_q) R^dag and Ybar = sum_q L_q (W_{q+1} R)^dag; the chain costs
//                     d x d by d x r products, and only the four power products stay dense.
//
// Thread layout and shared-memory matrices as in qoc_slice.cuh; the wide tile of the FP32
// adjoints (slice_tile(d, true)).
#include "qoc_device.cuh"
#include "qoc_internal.h"
#include "qoc_slice.cuh"

namespace qoc {

namespace {

using C = float2;

// xb += scale * the thread's own elements of Z (shared, leading dimension LD)
template <int MT>
__device__ __forceinline__ void add_own(C (&xb)[MT][MT], const C* __restrict__ Z, float scale, int d, int LD,
                                        int ty, int tx, int G) {
#pragma unroll
    for (int a = 0; a < MT; ++a)
#pragma unroll
        for (int b = 0; b < MT; ++b) {
            const int r = ty + G * a, c = tx + G * b;
            if (r < d && c < d) {
                const C z = Z[r * LD + c];
                xb[a][b].x = fmaf(scale, z.x, xb[a][b].x);
                xb[a][b].y = fmaf(scale, z.y, xb[a][b].y);
            }
        }
}

// YH = conjugate transpose of the D x D block of X (both shared, leading dimension LD)
__device__ __forceinline__ void ct_smem(C* __restrict__ YH, const C* __restrict__ X, int D, int LD) {
    for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
        const int a = idx / D, b = idx - a * D;
        C v = X[b * LD + a];
        v.y = -v.y;
        YH[a * LD + b] = v;
    }
}

// The power products that end both reverse modes: P2bar += Ybar X^dag, Xbar += X2^dag Ybar
// (p >= 3), then Xbar += X2bar X^dag + X^dag X2bar (p >= 2).  XH = X^dag and P2H = (X^2)^dag are
// ready in shared memory; T1, T2 are free D x LD buffers.  Called by every thread.
template <int MT>
__device__ __forceinline__ void ps_powers(C (&xb)[MT][MT], C (&p2b)[MT][MT], const C (&p3b)[MT][MT],
                                          const C* XH, const C* P2H, C* T1, C* T2, int p, int d, int LD,
                                          int ty, int tx, int G, bool act) {
    if (p >= 3) {
        if (act) store_acc<C, float, MT>(T1, p3b, 1.f, 0.f, d, LD, ty, tx, G);
        __syncthreads();
        if (act) {
            mm_acc<C, MT>(p2b, T1, XH, d, LD, ty, tx, G);
            mm_acc<C, MT>(xb, P2H, T1, d, LD, ty, tx, G);
        }
    }
    if (p >= 2) {
        if (act) store_acc<C, float, MT>(T2, p2b, 1.f, 0.f, d, LD, ty, tx, G);
        __syncthreads();
        if (act) {
            mm_acc<C, MT>(xb, T2, XH, d, LD, ty, tx, G);
            mm_acc<C, MT>(xb, XH, T2, d, LD, ty, tx, G);
        }
    }
}

// dC/du_kj = s sum_ab (Xbar_re Hk_im - Xbar_im Hk_re): FP32 pairs of exact products per thread,
// FP64 block sum
template <int MT>
__device__ __forceinline__ void ps_contract(const C (&xb)[MT][MT], const SysView<float>& sys,
                                            const DevParams* __restrict__ prm, double* __restrict__ gpart, int e,
                                            int j, int ty, int tx, int G, bool act, double* red) {
    const int d = sys.d;
    const size_t dd = (size_t)d * d;
    for (int k = 0; k < sys.M; ++k) {
        double v = 0.0;
        if (act) {
            float hi = 0.f, lo = 0.f;
#pragma unroll
            for (int a = 0; a < MT; ++a)
#pragma unroll
                for (int b = 0; b < MT; ++b) {
                    const int r = ty + G * a, c = tx + G * b;
                    if (r < d && c < d) {
                        const C hk = sys.Hk[k * dd + (size_t)r * d + c];
                        pair_acc(hi, lo, xb[a][b].x, hk.y);
                        pair_acc(hi, lo, -xb[a][b].y, hk.x);
                    }
                }
            v = (double)hi + (double)lo;
        }
        v = block_sum(v, red);
        if (threadIdx.x == 0) gpart[((size_t)e * sys.M + k) * sys.N + j] = prm->s * v;
    }
}

// slot of the i-th operand the reverse mode reads: the squaring operands S_{n-1} .. S_0, then the
// chain operands W_1 .. W_qt, then X^2 (slot layout in qoc_internal.h)
__device__ __forceinline__ int ps_rev_slot(int i, int qt, int n) { return i < qt + n ? qt + 1 + n - i : 0; }

}  // namespace

template <int MT>
__global__ void __launch_bounds__(MT == 4 ? 320 : 512, MT <= 2 ? 2 : 1)
k_expm_adj_ps(const DevParams* __restrict__ prm, SysView<float> sys, StateView<float> st, int j0,
              const C* __restrict__ states, const C* __restrict__ Gbuf, int wmax, double* __restrict__ gpart,
              ZStore<float> zs, int G) {
    const int p = prm->p, n = prm->n;
    if (!zs.ps || !zs_fits(zs, p, n)) return;           // no stored operands: the block recursion
    if (adj_lowrank_applies(st.S, n, sys.d)) return;      // k_expm_adj_ps_lr handles this evaluation
    const int D = G * MT, LD = D + 1, SZ = D * LD;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ float us[kMaxControls];
    __shared__ float cf[kPsCoefs];
    __shared__ double red[32];
    C* YH = reinterpret_cast<C*>(smraw);   // Y^dag through the chain, X^dag after it
    C* ZA = YH + SZ;
    C* ZB = ZA + SZ;
    C* SB = ZB + SZ;                       // stored operand of the current product ...
    C* SN = SB + SZ;                       // ... and of the next one, arriving meanwhile
    const int jl = blockIdx.x, e = blockIdx.y, j = j0 + jl;
    const int tid = threadIdx.x, tx = tid % G, ty = tid / G;
    const bool act = tid < G * G;
    const int d = sys.d, Sr = st.S, cb = st.cb, pst = st.pstride;
    const int qt = ps_top(p);
    for (int k = tid; k < sys.M; k += blockDim.x) us[k] = (float)sys.u[(size_t)k * sys.N + j];
    for (int k = tid; k < kPsCoefs; k += blockDim.x) cf[k] = prm->ch[k];
    // G_j (ZB) and Psi_{j-1} (SB) as d x S row-major
    const size_t slice = st.slice();
    const C* Gj = Gbuf + ((size_t)e * wmax + jl) * slice;
    const C* Pj = states + ((size_t)e * (wmax + 1) + jl) * slice;
    for (int idx = tid; idx < d * Sr; idx += blockDim.x) {
        const int a = idx / Sr, sc = idx - a * Sr;
        const size_t off = (size_t)(sc / cb) * pst + (size_t)a * cb + (sc % cb);
        ZB[idx] = Gj[off];
        SB[idx] = Pj[off];
    }
    const C* zst = zs.Z + ((size_t)e * zs.wmax + jl) * zs.cap * zs.mstride;
    auto fetch = [&](int slot, C* dst) {
        const C* src = zst + (size_t)slot * zs.mstride;
        for_rc(d, d, [&](int idx, int a, int b) { cp_async_elem(&dst[a * LD + b], &src[idx]); });
    };
    const int L = qt + n + (p >= 3 ? 1 : 0);   // operands read in sequence
    int cur = 0;
    auto issue = [&]() {
        if (cur < L) fetch(ps_rev_slot(cur, qt, n), SN);
        ++cur;
        cp_async_commit();
    };
    auto next = [&]() {   // wait for the operand in SN, make it SB, start the following one into the old SB
        cp_async_wait<0>();
        __syncthreads();
        C* t = SB; SB = SN; SN = t;
        issue();
    };
    if (qt >= 1) fetch(1, YH);
    issue();
    __syncthreads();
    if (act) {   // Ubar = G Psi^dag, the cotangent of U_j
        C acc[MT][MT];
        zero_acc<C, MT>(acc);
        for (int sc = 0; sc < Sr; ++sc) {
            C g[MT], q[MT];
#pragma unroll
            for (int i = 0; i < MT; ++i) {
                const int r = ty + G * i, c = tx + G * i;
                g[i] = (r < d) ? ZB[r * Sr + sc] : czero<C>();
                q[i] = (c < d) ? SB[c * Sr + sc] : czero<C>();
            }
#pragma unroll
            for (int i = 0; i < MT; ++i)
#pragma unroll
                for (int jj = 0; jj < MT; ++jj) cfma_bcj(acc[i][jj], g[i], q[jj]);
        }
        store_acc<C, float, MT>(ZA, acc, 1.f, 0.f, d, LD, ty, tx, G);
    }
    C* zb = ZA;
    C* zo = ZB;
    for (int m = n - 1; m >= 0; --m) {          // squarings in reverse
        next();                                 // SB = S_m^dag
        if (act) {
            C acc[MT][MT];
            zero_acc<C, MT>(acc);
            mm_acc<C, MT>(acc, zb, SB, d, LD, ty, tx, G);
            mm_acc<C, MT>(acc, SB, zb, d, LD, ty, tx, G);
            store_acc<C, float, MT>(zo, acc, 1.f, 0.f, d, LD, ty, tx, G);
        }
        C* t = zb; zb = zo; zo = t;
    }
    C xb[MT][MT], p2b[MT][MT], p3b[MT][MT];     // cotangents of X, X^2, Y
    zero_acc<C, MT>(xb);
    zero_acc<C, MT>(p2b);
    zero_acc<C, MT>(p3b);
    for (int q = 0; q < qt; ++q) {              // chain products in reverse
        next();                                 // SB = W_{q+1}^dag
        if (act) {
            mm_acc<C, MT>(p3b, zb, SB, d, LD, ty, tx, G);         // Ybar += Wbar_q W_{q+1}^dag
            add_own<MT>(xb, zb, cf[3 * q + 1], d, LD, ty, tx, G);
            add_own<MT>(p2b, zb, cf[3 * q + 2], d, LD, ty, tx, G);
            C acc[MT][MT];
            zero_acc<C, MT>(acc);
            mm_acc<C, MT>(acc, YH, zb, d, LD, ty, tx, G);         // Wbar_{q+1} = Y^dag Wbar_q
            store_acc<C, float, MT>(zo, acc, 1.f, 0.f, d, LD, ty, tx, G);
        }
        C* t = zb; zb = zo; zo = t;
    }
    __syncthreads();
    if (act) {                                  // the top block
        add_own<MT>(xb, zb, cf[3 * qt + 1], d, LD, ty, tx, G);
        add_own<MT>(p2b, zb, cf[3 * qt + 2], d, LD, ty, tx, G);
        add_own<MT>(p3b, zb, cf[3 * qt + 3], d, LD, ty, tx, G);
    }
    if (p >= 2) {
        if (p >= 3) {
            next();                             // SB = (X^2)^dag
        } else {
            cp_async_wait<0>();
            __syncthreads();
        }
        const float de = sys.delta ? (float)sys.delta[e] : 0.f;
        assemble_X<C, float>(SN, d, D, LD, sys.M, sys.H0, sys.Hk, sys.Hdet, de, us, (float)prm->s);
        __syncthreads();
        ct_smem(YH, SN, D, LD);                 // X^dag
        __syncthreads();
        ps_powers<MT>(xb, p2b, p3b, YH, SB, SN, zo, p, d, LD, ty, tx, G, act);
    } else {
        cp_async_wait<0>();
    }
    ps_contract<MT>(xb, sys, prm, gpart, e, j, ty, tx, G, act, red);
}

template <int MT>
__global__ void __launch_bounds__(MT == 4 ? 320 : 512, MT <= 2 ? 2 : 1)
k_expm_adj_ps_lr(const DevParams* __restrict__ prm, SysView<float> sys, StateView<float> st, int j0,
                 const C* __restrict__ states, const C* __restrict__ Gbuf, int wmax, double* __restrict__ gpart,
                 ZStore<float> zs, int G) {
    const int p = prm->p, n = prm->n;
    if (!zs.ps || !zs_fits(zs, p, n)) return;
    const int d = sys.d, Sr = st.S, cb = st.cb, pst = st.pstride;
    if (!adj_lowrank_applies(Sr, n, d)) return;
    const int D = G * MT, LD = D + 1, SZ = D * LD, RL = kLrMax;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ float us[kMaxControls];
    __shared__ float cf[kPsCoefs];
    __shared__ double red[32];
    C* YH = reinterpret_cast<C*>(smraw);   // Y^dag through the chain, X^dag after it
    C* SB = YH + SZ;
    C* SN = SB + SZ;
    C* Lb = SN + SZ;       // L (d x r, leading dimension RL), ping-pong with Lt
    C* Lt = Lb + d * RL;
    C* Rb = Lt + d * RL;   // R
    C* Wb = Rb + d * RL;   // S R (squarings), W_{q+1} R (chain)
    C* A1 = Wb + d * RL;   // sum_q c_3q+1 L_q
    C* A2 = A1 + d * RL;   // sum_q c_3q+2 L_q
    const int jl = blockIdx.x, e = blockIdx.y, j = j0 + jl;
    const int tid = threadIdx.x, tx = tid % G, ty = tid / G;
    const bool act = tid < G * G;
    const int qt = ps_top(p);
    for (int k = tid; k < sys.M; k += blockDim.x) us[k] = (float)sys.u[(size_t)k * sys.N + j];
    for (int k = tid; k < kPsCoefs; k += blockDim.x) cf[k] = prm->ch[k];
    for (int idx = tid; idx < d * RL; idx += blockDim.x) {
        A1[idx] = czero<C>();
        A2[idx] = czero<C>();
    }
    // L = G_j and R = Psi_{j-1} (d x S, from the panel layout)
    const size_t slice = st.slice();
    const C* Gj = Gbuf + ((size_t)e * wmax + jl) * slice;
    const C* Pj = states + ((size_t)e * (wmax + 1) + jl) * slice;
    for (int idx = tid; idx < d * Sr; idx += blockDim.x) {
        const int a = idx / Sr, sc = idx - a * Sr;
        const size_t off = (size_t)(sc / cb) * pst + (size_t)a * cb + (sc % cb);
        Lb[a * RL + sc] = Gj[off];
        Rb[a * RL + sc] = Pj[off];
    }
    const C* zst = zs.Z + ((size_t)e * zs.wmax + jl) * zs.cap * zs.mstride;
    auto fetch = [&](int slot, C* dst) {
        const C* src = zst + (size_t)slot * zs.mstride;
        for_rc(d, d, [&](int idx, int a, int b) { cp_async_elem(&dst[a * LD + b], &src[idx]); });
    };
    const int L = qt + n + (p >= 3 ? 1 : 0);
    int cur = 0;
    auto issue = [&]() {
        if (cur < L) fetch(ps_rev_slot(cur, qt, n), SN);
        ++cur;
        cp_async_commit();
    };
    auto next = [&]() {
        cp_async_wait<0>();
        __syncthreads();
        C* t = SB; SB = SN; SN = t;
        issue();
    };
    if (qt >= 1) fetch(1, YH);
    issue();
    // The two d x r products of a step in one pass: Wo = M Rin with M = SB^dag (SB holds the
    // conjugate transpose of the stored operand), and Lo = A Lin (A = YH or SB, row-major).  A
    // thread owns rows a and a + H (H = ceil(d / 2)) of one column t of both outputs.
    auto step_products = [&](C* Wo, const C* Rin, C* Lo, const C* A, const C* Lin, int rr) {
        const int H = (d + 1) >> 1;
        for (int o = tid; o < H * rr; o += blockDim.x) {
            const int a0 = o / rr, tcol = o - a0 * rr;
            const int a1 = (a0 + H < d) ? a0 + H : a0;
            C w0 = czero<C>(), w1 = czero<C>(), l0 = czero<C>(), l1 = czero<C>();
            const C* A0 = A + a0 * LD;
            const C* A1r = A + a1 * LD;
#pragma unroll 1
            for (int b = 0; b < d; ++b) {
                const C rv = Rin[b * RL + tcol], lv = Lin[b * RL + tcol];
                const C s0 = SB[b * LD + a0], s1 = SB[b * LD + a1];
                cfma_cj(w0, s0, rv);
                cfma_cj(w1, s1, rv);
                cfma(l0, A0[b], lv);
                cfma(l1, A1r[b], lv);
            }
            Wo[a0 * RL + tcol] = w0;
            Lo[a0 * RL + tcol] = l0;
            if (a0 + H < d) {
                Wo[a1 * RL + tcol] = w1;
                Lo[a1 * RL + tcol] = l1;
            }
        }
    };
    // xb += scale * sum_t Lm[row][t] conj(Rm[col][t])
    auto rank_update = [&](C (&xb)[MT][MT], const C* Lm, const C* Rm, int rr, float scale) {
        if (!act) return;
        C acc[MT][MT];
        zero_acc<C, MT>(acc);
        for (int tcol = 0; tcol < rr; ++tcol) {
            C a[MT], b[MT];
#pragma unroll
            for (int i = 0; i < MT; ++i) {
                const int row = ty + G * i, col = tx + G * i;
                a[i] = row < d ? Lm[row * RL + tcol] : czero<C>();
                b[i] = col < d ? Rm[col * RL + tcol] : czero<C>();
            }
#pragma unroll
            for (int i = 0; i < MT; ++i)
#pragma unroll
                for (int jj = 0; jj < MT; ++jj) cfma_bcj(acc[i][jj], a[i], b[jj]);
        }
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
            for (int jj = 0; jj < MT; ++jj) {
                xb[i][jj].x = fmaf(scale, acc[i][jj].x, xb[i][jj].x);
                xb[i][jj].y = fmaf(scale, acc[i][jj].y, xb[i][jj].y);
            }
    };
    int r = Sr;
    for (int m = n - 1; m >= 0; --m) {          // squarings in reverse: L <- [L, S^dag L], R <- [S R, R]
        next();                                 // SB = S_m^dag
        step_products(Wb, Rb, Lb + r, SB, Lb, r);
        __syncthreads();
        for (int o = tid; o < d * r; o += blockDim.x) {
            const int a = o / r, tcol = o - a * r;
            Rb[a * RL + tcol + r] = Rb[a * RL + tcol];
            Rb[a * RL + tcol] = Wb[a * RL + tcol];
        }
        r *= 2;
    }
    C xb[MT][MT], p2b[MT][MT], p3b[MT][MT];
    zero_acc<C, MT>(xb);
    zero_acc<C, MT>(p2b);
    zero_acc<C, MT>(p3b);
    C* Lc = Lb;
    C* Ln = Lt;
    for (int q = 0; q < qt; ++q) {              // chain products in reverse, R fixed
        next();                                 // SB = W_{q+1}^dag
        step_products(Wb, Rb, Ln, YH, Lc, r);   // V_q = W_{q+1} R; L_{q+1} = Y^dag L_q
        const float c1 = cf[3 * q + 1], c2 = cf[3 * q + 2];
        for (int o = tid; o < d * r; o += blockDim.x) {
            const int a = o / r, tcol = o - a * r;
            const C l = Lc[a * RL + tcol];
            C& s1 = A1[a * RL + tcol];
            C& s2 = A2[a * RL + tcol];
            s1.x = fmaf(c1, l.x, s1.x);
            s1.y = fmaf(c1, l.y, s1.y);
            s2.x = fmaf(c2, l.x, s2.x);
            s2.y = fmaf(c2, l.y, s2.y);
        }
        __syncthreads();
        rank_update(p3b, Lc, Wb, r, 1.f);       // Ybar += L_q V_q^dag
        C* t = Lc; Lc = Ln; Ln = t;
    }
    __syncthreads();
    {                                           // the top block
        const float c1 = cf[3 * qt + 1], c2 = cf[3 * qt + 2];
        for (int o = tid; o < d * r; o += blockDim.x) {
            const int a = o / r, tcol = o - a * r;
            const C l = Lc[a * RL + tcol];
            C& s1 = A1[a * RL + tcol];
            C& s2 = A2[a * RL + tcol];
            s1.x = fmaf(c1, l.x, s1.x);
            s1.y = fmaf(c1, l.y, s1.y);
            s2.x = fmaf(c2, l.x, s2.x);
            s2.y = fmaf(c2, l.y, s2.y);
        }
    }
    __syncthreads();
    if (cf[3 * qt + 3] != 0.f) rank_update(p3b, Lc, Rb, r, cf[3 * qt + 3]);
    rank_update(xb, A1, Rb, r, 1.f);            // Xbar = (sum c L_q) R^dag + ...
    rank_update(p2b, A2, Rb, r, 1.f);
    if (p >= 2) {
        if (p >= 3) {
            next();                             // SB = (X^2)^dag
        } else {
            cp_async_wait<0>();
            __syncthreads();
        }
        const float de = sys.delta ? (float)sys.delta[e] : 0.f;
        assemble_X<C, float>(SN, d, D, LD, sys.M, sys.H0, sys.Hk, sys.Hdet, de, us, (float)prm->s);
        __syncthreads();
        ct_smem(YH, SN, D, LD);                 // X^dag
        __syncthreads();
        ps_powers<MT>(xb, p2b, p3b, YH, SB, SN, Lb, p, d, LD, ty, tx, G, act);   // Lb: D x LD fits the six blocks
    } else {
        cp_async_wait<0>();
    }
    ps_contract<MT>(xb, sys, prm, gpart, e, j, ty, tx, G, act, red);
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
// tile of the adjoint kernels: the wide one (more outputs per thread at equal padding)
constexpr bool kPsWide = true;

static size_t ps_adj_smem(int d) {
    const int D = slice_tile(d, kPsWide).D;
    return (size_t)5 * D * (D + 1) * sizeof(C);
}
static size_t ps_lr_smem(int d) {
    const int D = slice_tile(d, kPsWide).D;
    return (size_t)3 * D * (D + 1) * sizeof(C) + 6 * (size_t)d * kLrMax * sizeof(C);
}

template <int MT>
static cudaError_t launch_ps_adj_mt(const DevParams* prm, const SysView<float>& sys, const StateView<float>& sv,
                                    int j0, int wlen, int E, const C* states, const C* Gbuf, int wmax, double* gpart,
                                    const ZStore<float>& zs, int G, cudaStream_t st, int* launches) {
    const size_t smem = ps_adj_smem(sys.d);
    cudaError_t err = cudaFuncSetAttribute(k_expm_adj_ps<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_expm_adj_ps<MT><<<dim3(wlen, E), slice_threads(G), smem, st>>>(prm, sys, sv, j0, states, Gbuf, wmax, gpart,
                                                                       zs, G);
    ++*launches;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (!adj_lowrank_applies(sv.S, 0, sys.d)) return cudaSuccess;   // no squaring count makes it apply
    // the power products reuse the six d x r blocks as one D x LD matrix
    if ((size_t)6 * sys.d * kLrMax < (size_t)slice_tile(sys.d, kPsWide).D * (slice_tile(sys.d, kPsWide).D + 1))
        return cudaErrorInvalidValue;
    const size_t smem_l = ps_lr_smem(sys.d);
    err = cudaFuncSetAttribute(k_expm_adj_ps_lr<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l);
    if (err != cudaSuccess) return err;
    k_expm_adj_ps_lr<MT><<<dim3(wlen, E), slice_threads(G), smem_l, st>>>(prm, sys, sv, j0, states, Gbuf, wmax,
                                                                            gpart, zs, G);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_expm_adj_ps(const DevParams* prm, const SysView<float>& sys, const StateView<float>& sv, int j0,
                               int wlen, int E, const float2* states, const float2* Gbuf, int wmax, double* gpart,
                               const ZStore<float>& zs, cudaStream_t st, int* launches) {
    const SliceTile tl = slice_tile(sys.d, kPsWide);
    if (!zs.ps || !zs.Z || sys.d > ps_max_d()) return cudaErrorInvalidValue;
    switch (tl.MT) {
        case 1: return launch_ps_adj_mt<1>(prm, sys, sv, j0, wlen, E, states, Gbuf, wmax, gpart, zs, tl.G, st, launches);
        case 2: return launch_ps_adj_mt<2>(prm, sys, sv, j0, wlen, E, states, Gbuf, wmax, gpart, zs, tl.G, st, launches);
        case 3: return launch_ps_adj_mt<3>(prm, sys, sv, j0, wlen, E, states, Gbuf, wmax, gpart, zs, tl.G, st, launches);
        case 4: return launch_ps_adj_mt<4>(prm, sys, sv, j0, wlen, E, states, Gbuf, wmax, gpart, zs, tl.G, st, launches);
        default: return cudaErrorInvalidValue;
    }
}

int ps_adj_ctas_per_sm(int d) {
    const SliceTile tl = slice_tile(d, kPsWide);
    if (tl.MT <= 0) return 1;
    const size_t smem = ps_adj_smem(d);
    const int thr = slice_threads(tl.G);
    int n = 0;
    cudaError_t e;
    switch (tl.MT) {
        case 1: cudaFuncSetAttribute(k_expm_adj_ps<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_adj_ps<1>, thr, smem); break;
        case 2: cudaFuncSetAttribute(k_expm_adj_ps<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_adj_ps<2>, thr, smem); break;
        case 3: cudaFuncSetAttribute(k_expm_adj_ps<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_adj_ps<3>, thr, smem); break;
        default: cudaFuncSetAttribute(k_expm_adj_ps<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_adj_ps<4>, thr, smem); break;
    }
    return (e == cudaSuccess && n > 0) ? n : 1;
}

}  // namespace qoc
