// Fused per-slice kernels for small and medium Hilbert dimension d (d <= 64 in FP32, d <= 48 in
// FP64): one CTA owns one slice (and one ensemble member) and keeps every matrix of that slice
// in shared memory.
//
//  k_expm_fwd : X_j = -i s H_j (s = dt / 2^n; Eq. 1 assembly fused), Horner evaluation of the
//               order-p Taylor polynomial T_j = I + X(I + X/2(... (I + X/p))) (Eq. 10), then n
//               squarings U_j = T_j^(2^n) (Eq. 9).  Writes U_j.
//  k_expm_adj : exact adjoint of that same polynomial map X -> f(X).  For a polynomial f with
//               real coefficients the adjoint of its Frechet derivative is L_f(X^dag, .), and
//               L_f(A, E) is the (1,2) block of f([[A, E], [0, A]]).  So Xbar_j is obtained by
//               running the same Horner + squaring recursion on the block-upper-triangular
//               matrix [[X^dag, Ubar], [0, X^dag]] with Ubar_j = G_j Psi_{j-1}^dag (G_j the
//               costate, Appendix A), then dC/du_{k,j} = Re tr(Xbar^dag (-i s H_k)) (Eq. A3).
//               This differentiates the truncated series exactly (not the first-order Eq. 11)
//               without storing the p + n intermediate matrices.
//  k_expm_adj_rev : the same derivative in reverse mode over the forward products, when the
//               forward kernel stored their right operands (ZStore): per squaring
//               Sbar_m = Sbar_{m+1} S_m^dag + S_m^dag Sbar_{m+1}, per Horner step
//               Xbar += Zbar_i Z_{i+1}^dag / i and Zbar_{i+1} = X^dag Zbar_i / i, starting from
//               Ubar and ending with Xbar += Zbar_p / p: two products per step instead of three,
//               and five matrices in shared memory instead of six (the stored operand of the
//               next product arrives by cp.async while the current one is multiplied).
//  k_expm_adj_lr : the same reverse mode when the cotangent has low rank.  The cotangent
//               Ubar_j = G_j Psi_{j-1}^dag, with G_j and Psi_{j-1} both d x S (S propagated
//               states), has rank at most S, so it is kept as factors L R^dag: each squaring
//               appends a block to each factor (rank doubles), each Horner step maps
//               L -> X^dag L / i with R fixed, and the products become d x d by d x r ones
//               (r = S 2^n).  Taken when r <= 16 and 8 r <= d.
//
// Thread layout: a G x G grid of threads (slice_tile); thread (ty, tx) owns the MT x MT outputs
// (ty + G a, tx + G b).  Matrices sit in shared memory padded to D = G MT rows with a leading
// dimension of D + 1 complex elements (breaks bank conflicts between the rows a warp reads);
// padding rows and columns are kept at zero.
#include "qoc_device.cuh"
#include "qoc_internal.h"
#include "qoc_slice.cuh"

namespace qoc {

// acc11 += A11 B11 ;  acc12 += A11 B12 + A12 B11   (block-upper-triangular product)
template <typename C, int MT>
__device__ __forceinline__ void mm_block(C (&acc11)[MT][MT], C (&acc12)[MT][MT],
                                         const C* __restrict__ A11, const C* __restrict__ A12,
                                         const C* __restrict__ B11, const C* __restrict__ B12,
                                         int kd, int LD, int ty, int tx, int G) {
#pragma unroll 1
    for (int k = 0; k < kd; ++k) {
        C a1[MT], a2[MT], b1[MT], b2[MT];
#pragma unroll
        for (int i = 0; i < MT; ++i) {
            a1[i] = A11[(ty + G * i) * LD + k];
            a2[i] = A12[(ty + G * i) * LD + k];
        }
#pragma unroll
        for (int i = 0; i < MT; ++i) {
            b1[i] = B11[k * LD + tx + G * i];
            b2[i] = B12[k * LD + tx + G * i];
        }
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
            for (int jj = 0; jj < MT; ++jj) {
                cfma(acc11[i][jj], a1[i], b1[jj]);
                cfma(acc12[i][jj], a1[i], b2[jj]);
                cfma(acc12[i][jj], a2[i], b1[jj]);
            }
    }
}

template <typename R, int MT>
__global__ void __launch_bounds__(512)
k_expm_fwd(const DevParams* __restrict__ prm, SysView<R> sys, int j0, C_t<R>* __restrict__ Ubuf,
           long long ustride, int wmax, ZStore<R> zs, int G) {
    using C = C_t<R>;
    const int D = G * MT, LD = D + 1, SZ = D * LD;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ R us[kMaxControls];
    C* X = reinterpret_cast<C*>(smraw);
    C* Za = X + SZ;
    C* Zb = Za + SZ;
    const int jl = blockIdx.x, e = blockIdx.y, j = j0 + jl;
    const int tid = threadIdx.x, tx = tid % G, ty = tid / G;
    const bool act = tid < G * G;   // the block is rounded up to whole warps
    const int d = sys.d, p = prm->p, n = prm->n;
    const R s = (R)prm->s;
    for (int k = tid; k < sys.M; k += blockDim.x) us[k] = (R)sys.u[(size_t)k * sys.N + j];
    __syncthreads();
    const R de = sys.delta ? (R)sys.delta[e] : R(0);
    assemble_X<C, R>(X, d, D, LD, sys.M, sys.H0, sys.Hk, sys.Hdet, de, us, s);
    __syncthreads();
    {   // Z = I + X / p
        const R ip = R(1) / R(p);
        for (int idx = tid; idx < D * D; idx += blockDim.x) {
            const int a = idx / D, b = idx - a * D;
            C x = X[a * LD + b];
            C z;
            z.x = x.x * ip + ((a == b && a < d) ? R(1) : R(0));
            z.y = x.y * ip;
            Za[a * LD + b] = z;
        }
    }
    __syncthreads();
    C* zin = Za;
    C* zout = Zb;
    C* zst = (zs.Z && p - 1 + n <= zs.cap) ? zs.Z + ((size_t)e * zs.wmax + jl) * zs.cap * zs.mstride : nullptr;
    for (int i = p - 1; i >= 1; --i) {          // Horner: Z <- I + X Z / i
        if (zst) store_ct<C>(zst + (size_t)(p - 1 - i) * zs.mstride, zin, d, LD);
        if (act) {
            C acc[MT][MT];
            zero_acc<C, MT>(acc);
            mm_acc<C, MT>(acc, X, zin, d, LD, ty, tx, G);
            store_acc<C, R, MT>(zout, acc, R(1) / R(i), R(1), d, LD, ty, tx, G);
        }
        __syncthreads();
        C* t = zin; zin = zout; zout = t;
    }
    for (int m = 0; m < n; ++m) {               // squaring: Z <- Z Z
        if (zst) store_ct<C>(zst + (size_t)(p - 1 + m) * zs.mstride, zin, d, LD);
        if (act) {
            C acc[MT][MT];
            zero_acc<C, MT>(acc);
            mm_acc<C, MT>(acc, zin, zin, d, LD, ty, tx, G);
            store_acc<C, R, MT>(zout, acc, R(1), R(0), d, LD, ty, tx, G);
        }
        __syncthreads();
        C* t = zin; zin = zout; zout = t;
    }
    // a slice holds U_j at offset 0 and U_j^dag at offset ustride / 2 (rows of U^dag are what the
    // backward costate sweep streams)
    C* U = Ubuf + ((size_t)e * wmax + jl) * ustride;
    C* UH = U + ustride / 2;
    for (int idx = tid; idx < d * d; idx += blockDim.x) {
        const int a = idx / d, b = idx - a * d;
        U[idx] = zin[a * LD + b];
        C h = zin[b * LD + a];
        h.y = -h.y;
        UH[idx] = h;
    }
}

template <typename R, int MT>
__global__ void __launch_bounds__(512)
k_expm_adj(const DevParams* __restrict__ prm, SysView<R> sys, StateView<R> st, int j0,
           const C_t<R>* __restrict__ states, const C_t<R>* __restrict__ Gbuf, int wmax,
           double* __restrict__ gpart, ZStore<R> zs, int G) {
    using C = C_t<R>;
    if (zs_fits(zs, prm->p, prm->n)) return;   // a reverse-mode kernel handles this evaluation
    const int D = G * MT, LD = D + 1, SZ = D * LD;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ R us[kMaxControls];
    __shared__ double red[32];
    C* XH = reinterpret_cast<C*>(smraw);
    C* Ub = XH + SZ;
    C* Z11a = Ub + SZ;
    C* Z12a = Z11a + SZ;
    C* Z11b = Z12a + SZ;
    C* Z12b = Z11b + SZ;
    const int jl = blockIdx.x, e = blockIdx.y, j = j0 + jl;
    const int tid = threadIdx.x, tx = tid % G, ty = tid / G;
    const bool act = tid < G * G;   // the block is rounded up to whole warps
    // only the S propagated columns are staged (d x S <= d x d fits a matrix slot; the padding
    // columns of the panel layout are zero and add nothing to Ubar)
    const int d = sys.d, p = prm->p, n = prm->n, Sp = st.S, cb = st.cb, ps = st.pstride;
    const R s = (R)prm->s;
    for (int k = tid; k < sys.M; k += blockDim.x) us[k] = (R)sys.u[(size_t)k * sys.N + j];
    __syncthreads();
    const R de = sys.delta ? (R)sys.delta[e] : R(0);
    // X into Z11a, then XH = X^dag
    assemble_X<C, R>(Z11a, d, D, LD, sys.M, sys.H0, sys.Hk, sys.Hdet, de, us, s);
    // stage G_j (Z11b) and Psi_{j-1} (Z12b) as d x Sp row-major from the column-panel layout
    const size_t slice = st.slice();
    const C* Gj = Gbuf + ((size_t)e * wmax + jl) * slice;
    const C* Pj = states + ((size_t)e * (wmax + 1) + jl) * slice;
    for (int idx = tid; idx < d * Sp; idx += blockDim.x) {
        const int a = idx / Sp, sc = idx - a * Sp;
        const size_t off = (size_t)(sc / cb) * ps + (size_t)a * cb + (sc % cb);
        Z11b[idx] = Gj[off];
        Z12b[idx] = Pj[off];
    }
    __syncthreads();
    for (int idx = tid; idx < D * D; idx += blockDim.x) {
        const int a = idx / D, b = idx - a * D;
        C x = Z11a[b * LD + a];
        x.y = -x.y;
        XH[a * LD + b] = x;
    }
    if (act) {   // Ubar = G Psi^dag
        C acc[MT][MT];
        zero_acc<C, MT>(acc);
        for (int sc = 0; sc < Sp; ++sc) {
            C g[MT], q[MT];
#pragma unroll
            for (int i = 0; i < MT; ++i) {
                const int r = ty + G * i, c = tx + G * i;
                g[i] = (r < d) ? Z11b[r * Sp + sc] : czero<C>();
                q[i] = (c < d) ? Z12b[c * Sp + sc] : czero<C>();
            }
#pragma unroll
            for (int i = 0; i < MT; ++i)
#pragma unroll
                for (int jj = 0; jj < MT; ++jj) cfma_bcj(acc[i][jj], g[i], q[jj]);
        }
        store_acc<C, R, MT>(Ub, acc, R(1), R(0), d, LD, ty, tx, G);
    }
    __syncthreads();
    {   // Horner start: Z11 = I + XH / p, Z12 = Ubar / p
        const R ip = R(1) / R(p);
        for (int idx = tid; idx < D * D; idx += blockDim.x) {
            const int a = idx / D, b = idx - a * D;
            C x = XH[a * LD + b], u = Ub[a * LD + b];
            C z1, z2;
            z1.x = x.x * ip + ((a == b && a < d) ? R(1) : R(0));
            z1.y = x.y * ip;
            z2.x = u.x * ip;
            z2.y = u.y * ip;
            Z11a[a * LD + b] = z1;
            Z12a[a * LD + b] = z2;
        }
    }
    __syncthreads();
    C *z11 = Z11a, *z12 = Z12a, *o11 = Z11b, *o12 = Z12b;
    for (int i = p - 1; i >= 1; --i) {
        if (act) {
            C a11[MT][MT], a12[MT][MT];
            zero_acc<C, MT>(a11);
            zero_acc<C, MT>(a12);
            mm_block<C, MT>(a11, a12, XH, Ub, z11, z12, d, LD, ty, tx, G);
            const R ri = R(1) / R(i);
            store_acc<C, R, MT>(o11, a11, ri, R(1), d, LD, ty, tx, G);
            store_acc<C, R, MT>(o12, a12, ri, R(0), d, LD, ty, tx, G);
        }
        __syncthreads();
        C* t = z11; z11 = o11; o11 = t;
        t = z12; z12 = o12; o12 = t;
    }
    for (int m = 0; m < n; ++m) {
        if (act) {
            C a11[MT][MT], a12[MT][MT];
            zero_acc<C, MT>(a11);
            zero_acc<C, MT>(a12);
            mm_block<C, MT>(a11, a12, z11, z12, z11, z12, d, LD, ty, tx, G);
            store_acc<C, R, MT>(o11, a11, R(1), R(0), d, LD, ty, tx, G);
            store_acc<C, R, MT>(o12, a12, R(1), R(0), d, LD, ty, tx, G);
        }
        __syncthreads();
        C* t = z11; z11 = o11; o11 = t;
        t = z12; z12 = o12; o12 = t;
    }
    // dC/du_{k,j} = Re tr(Xbar^dag (-i s H_k)) = s sum_ab (Xbar_re Hk_im - Xbar_im Hk_re)
    const size_t dd = (size_t)d * d;
    // per-thread partials: FP32 form as (hi, lo) pairs of exact products, FP64 form in FP64; the
    // block sum in FP64
    for (int k = 0; k < sys.M; ++k) {
        double v = 0.0;
        if constexpr (sizeof(R) == 4) {
            float hi = 0.f, lo = 0.f;
            for (int idx = tid; idx < d * d; idx += blockDim.x) {
                const int a = idx / d, b = idx - a * d;
                const C xb = z12[a * LD + b];
                const C hk = sys.Hk[k * dd + idx];
                pair_acc(hi, lo, xb.x, hk.y);
                pair_acc(hi, lo, -xb.y, hk.x);
            }
            v = (double)hi + (double)lo;
        } else {
            for (int idx = tid; idx < d * d; idx += blockDim.x) {
                const int a = idx / d, b = idx - a * d;
                const C xb = z12[a * LD + b];
                const C hk = sys.Hk[k * dd + idx];
                v += (double)xb.x * (double)hk.y - (double)xb.y * (double)hk.x;
            }
        }
        v = block_sum(v, red);
        if (tid == 0) gpart[((size_t)e * sys.M + k) * sys.N + j] = prm->s * v;
    }
}

// Low-rank reverse mode.  The cotangent of U_j is Ubar = G_j Psi_{j-1}^dag, of rank S (the
// propagated columns).  Through the squarings in reverse, Sbar = L R^dag becomes
// Sbar S^dag + S^dag Sbar = [L, S^dag L] [S R, R]^dag: the rank doubles, so T = Z_1 receives a
// rank r = 2^n S cotangent.  Through the Horner steps in reverse R stays fixed and only
// L_{i+1} = X^dag L_i / i changes, with Xbar += L_i (Z_{i+1} R)^dag / i and, for Z_p = I + X / p,
// Xbar += L_p R^dag / p: the same exact derivative as the dense reverse mode, with d x d by d x r
// products (r <= kLrMax) in place of d x d by d x d ones.  Used when 8 r <= d (qoc_internal.h).

template <typename R, int MT>
__global__ void __launch_bounds__(512, (MT <= 2 && sizeof(R) == 4) ? 3 : 1)
k_expm_adj_lr(const DevParams* __restrict__ prm, SysView<R> sys, StateView<R> st, int j0,
              const C_t<R>* __restrict__ states, const C_t<R>* __restrict__ Gbuf, int wmax,
              double* __restrict__ gpart, ZStore<R> zs, int G) {
    using C = C_t<R>;
    const int p = prm->p, n = prm->n;
    if (zs.ps || !zs_fits(zs, p, n)) return;
    const int d = sys.d, Sr = st.S, cb = st.cb, ps = st.pstride;
    if (!adj_lowrank_applies(Sr, n, d)) return;
    const int D = G * MT, LD = D + 1, SZ = D * LD, RL = kLrMax;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ R us[kMaxControls];
    __shared__ double red[32];
    C* XH = reinterpret_cast<C*>(smraw);
    C* SB = XH + SZ;       // stored operand of the current product ...
    C* SN = SB + SZ;       // ... and of the next one, arriving by cp.async meanwhile
    C* Lb = SN + SZ;       // L (d x r, leading dimension RL)
    C* Lt = Lb + d * RL;   // X^dag L / i (next L), or the scratch of a squaring
    C* Rb = Lt + d * RL;   // R
    C* Wb = Rb + d * RL;   // Z R (Horner), S R (squaring)
    const int jl = blockIdx.x, e = blockIdx.y, j = j0 + jl;
    const int tid = threadIdx.x, tx = tid % G, ty = tid / G;
    const bool act = tid < G * G;
    const R s = (R)prm->s;
    for (int k = tid; k < sys.M; k += blockDim.x) us[k] = (R)sys.u[(size_t)k * sys.N + j];
    __syncthreads();
    const R de = sys.delta ? (R)sys.delta[e] : R(0);
    assemble_X<C, R>(SN, d, D, LD, sys.M, sys.H0, sys.Hk, sys.Hdet, de, us, s);
    // L = G_j and R = Psi_{j-1} (d x S, from the panel layout)
    const size_t slice = st.slice();
    const C* Gj = Gbuf + ((size_t)e * wmax + jl) * slice;
    const C* Pj = states + ((size_t)e * (wmax + 1) + jl) * slice;
    for (int idx = tid; idx < d * Sr; idx += blockDim.x) {
        const int a = idx / Sr, sc = idx - a * Sr;
        const size_t off = (size_t)(sc / cb) * ps + (size_t)a * cb + (sc % cb);
        Lb[a * RL + sc] = Gj[off];
        Rb[a * RL + sc] = Pj[off];
    }
    __syncthreads();
    for (int idx = tid; idx < D * D; idx += blockDim.x) {
        const int a = idx / D, b = idx - a * D;
        C x = SN[b * LD + a];
        x.y = -x.y;
        XH[a * LD + b] = x;
    }
    __syncthreads();   // SN is free again
    const C* zst = zs.Z + ((size_t)e * zs.wmax + jl) * zs.cap * zs.mstride;
    auto issue = [&](int r) {
        if (r >= 0) {
            const C* src = zst + (size_t)r * zs.mstride;
            for_rc(d, d, [&](int idx, int a, int b) { cp_async_elem(&SN[a * LD + b], &src[idx]); });
        }
        cp_async_commit();
    };
    auto next = [&](int r) {   // wait for operand r (in SN), make it SB, start r - 1 into the old SB
        cp_async_wait<0>();
        __syncthreads();
        C* tt = SB; SB = SN; SN = tt;
        issue(r - 1);
    };
    // The two d x r products of a step in one pass: Wo = M Rin with M = SB^dag (SB holds the
    // conjugate transpose of the stored operand), and Lo = A Lin * scale (A = XH or SB, row-major).
    // A thread owns rows a and a + H (H = ceil(d / 2)) of one column t of both outputs: four
    // independent accumulators sharing the operand loads.
    auto step_products = [&](C* Wo, const C* Rin, C* Lo, const C* A, const C* Lin, int rr, R scale) {
        const int H = (d + 1) >> 1;
        for (int o = tid; o < H * rr; o += blockDim.x) {
            const int a0 = o / rr, tcol = o - a0 * rr;
            const int a1 = (a0 + H < d) ? a0 + H : a0;
            C w0 = czero<C>(), w1 = czero<C>(), l0 = czero<C>(), l1 = czero<C>();
            const C* A0 = A + a0 * LD;
            const C* A1 = A + a1 * LD;
#pragma unroll 1
            for (int b = 0; b < d; ++b) {
                const C rv = Rin[b * RL + tcol], lv = Lin[b * RL + tcol];
                const C s0 = SB[b * LD + a0], s1 = SB[b * LD + a1];
                cfma_cj(w0, s0, rv);
                cfma_cj(w1, s1, rv);
                cfma(l0, A0[b], lv);
                cfma(l1, A1[b], lv);
            }
            l0.x *= scale;
            l0.y *= scale;
            l1.x *= scale;
            l1.y *= scale;
            Wo[a0 * RL + tcol] = w0;
            Lo[a0 * RL + tcol] = l0;
            if (a0 + H < d) {
                Wo[a1 * RL + tcol] = w1;
                Lo[a1 * RL + tcol] = l1;
            }
        }
    };
    issue(p - 2 + n);
    int r = Sr;
    for (int m = n - 1; m >= 0; --m) {          // squarings in reverse: L <- [L, S^dag L], R <- [S R, R]
        next(p - 1 + m);
        step_products(Wb, Rb, Lb + r, SB, Lb, r, R(1));   // S R; S^dag L into columns r .. 2r - 1
        __syncthreads();
        for (int o = tid; o < d * r; o += blockDim.x) {
            const int a = o / r, tcol = o - a * r;
            Rb[a * RL + tcol + r] = Rb[a * RL + tcol];
            Rb[a * RL + tcol] = Wb[a * RL + tcol];
        }
        r *= 2;
    }
    C xb[MT][MT];                               // Xbar
    zero_acc<C, MT>(xb);
    // Xbar += scale * sum_t Lm[row][t] conj(Rm[col][t])
    auto rank_update = [&](const C* Lm, const C* Rm, R scale) {
        if (!act) return;
        C acc[MT][MT];
        zero_acc<C, MT>(acc);
        for (int tcol = 0; tcol < r; ++tcol) {
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
                xb[i][jj].x += acc[i][jj].x * scale;
                xb[i][jj].y += acc[i][jj].y * scale;
            }
    };
    C* Lc = Lb;
    C* Ln = Lt;
    for (int i = 1; i <= p - 1; ++i) {          // Horner steps in reverse
        next(p - 1 - i);                        // SB = Z_{i+1}^dag
        const R ri = R(1) / R(i);
        step_products(Wb, Rb, Ln, XH, Lc, r, ri);   // W = Z_{i+1} R; L_{i+1} = X^dag L_i / i
        __syncthreads();
        rank_update(Lc, Wb, ri);                // Xbar += L_i (Z_{i+1} R)^dag / i
        C* tt = Lc; Lc = Ln; Ln = tt;
    }
    cp_async_wait<0>();
    __syncthreads();
    rank_update(Lc, Rb, R(1) / R(p));           // Z_p = I + X / p: Xbar += L_p R^dag / p
    const size_t dd = (size_t)d * d;
    for (int k = 0; k < sys.M; ++k) {   // partials: FP32 pairs of exact products (FP32 form); FP64 sum
        double v = 0.0;
        if (act) {
            float hi = 0.f, lo = 0.f;
#pragma unroll
            for (int a = 0; a < MT; ++a)
#pragma unroll
                for (int b = 0; b < MT; ++b) {
                    const int rr = ty + G * a, c = tx + G * b;
                    if (rr < d && c < d) {
                        const C hk = sys.Hk[k * dd + (size_t)rr * d + c];
                        if constexpr (sizeof(R) == 4) {
                            pair_acc(hi, lo, xb[a][b].x, hk.y);
                            pair_acc(hi, lo, -xb[a][b].y, hk.x);
                        } else {
                            v += (double)xb[a][b].x * (double)hk.y - (double)xb[a][b].y * (double)hk.x;
                        }
                    }
                }
            if constexpr (sizeof(R) == 4) v = (double)hi + (double)lo;
        }
        v = block_sum(v, red);
        if (tid == 0) gpart[((size_t)e * sys.M + k) * sys.N + j] = prm->s * v;
    }
}

template <typename R, int MT>
__global__ void __launch_bounds__(512, (MT <= 2 && sizeof(R) == 4) ? 3 : 1)
k_expm_adj_rev(const DevParams* __restrict__ prm, SysView<R> sys, StateView<R> st, int j0,
               const C_t<R>* __restrict__ states, const C_t<R>* __restrict__ Gbuf, int wmax,
               double* __restrict__ gpart, ZStore<R> zs, int G) {
    using C = C_t<R>;
    const int p = prm->p, n = prm->n;
    if (zs.ps || !zs_fits(zs, p, n)) return;              // another kernel handles this evaluation
    if (adj_lowrank_applies(st.S, n, sys.d)) return;        // k_expm_adj_lr handles this evaluation
    const int D = G * MT, LD = D + 1, SZ = D * LD;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ R us[kMaxControls];
    __shared__ double red[32];
    C* XH = reinterpret_cast<C*>(smraw);
    C* ZA = XH + SZ;
    C* ZB = ZA + SZ;
    C* SB = ZB + SZ;       // stored operand of the current product ...
    C* SN = SB + SZ;       // ... and of the next one, arriving by cp.async meanwhile
    const int jl = blockIdx.x, e = blockIdx.y, j = j0 + jl;
    const int tid = threadIdx.x, tx = tid % G, ty = tid / G;
    const bool act = tid < G * G;   // the block is rounded up to whole warps
    const int d = sys.d, Sr = st.S, cb = st.cb, ps = st.pstride;
    const R s = (R)prm->s;
    for (int k = tid; k < sys.M; k += blockDim.x) us[k] = (R)sys.u[(size_t)k * sys.N + j];
    __syncthreads();
    const R de = sys.delta ? (R)sys.delta[e] : R(0);
    assemble_X<C, R>(ZA, d, D, LD, sys.M, sys.H0, sys.Hk, sys.Hdet, de, us, s);
    // G_j (ZB) and Psi_{j-1} (SB) as d x S row-major; the padding columns are zero
    const size_t slice = st.slice();
    const C* Gj = Gbuf + ((size_t)e * wmax + jl) * slice;
    const C* Pj = states + ((size_t)e * (wmax + 1) + jl) * slice;
    for (int idx = tid; idx < d * Sr; idx += blockDim.x) {
        const int a = idx / Sr, sc = idx - a * Sr;
        const size_t off = (size_t)(sc / cb) * ps + (size_t)a * cb + (sc % cb);
        ZB[idx] = Gj[off];
        SB[idx] = Pj[off];
    }
    __syncthreads();
    for (int idx = tid; idx < D * D; idx += blockDim.x) {
        const int a = idx / D, b = idx - a * D;
        C x = ZA[b * LD + a];
        x.y = -x.y;
        XH[a * LD + b] = x;
    }
    __syncthreads();
    if (act) {   // Ubar = G Psi^dag, the cotangent of U_j = S_n
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
        store_acc<C, R, MT>(ZA, acc, R(1), R(0), d, LD, ty, tx, G);
    }
    __syncthreads();
    const C* zst = zs.Z + ((size_t)e * zs.wmax + jl) * zs.cap * zs.mstride;
    // the stored conjugate transpose of the right operand of product r; the products run in
    // reverse, r = p - 2 + n down to 0, and r - 1 is fetched while r is multiplied.  One barrier
    // per product: after it the copy of r is visible to every thread and every thread has
    // finished product r + 1, so its operand slot takes the copy of r - 1 and its input
    // matrix becomes the output of r.
    auto issue = [&](int r) {
        if (r >= 0) {
            const C* src = zst + (size_t)r * zs.mstride;
            for_rc(d, d, [&](int idx, int a, int b) { cp_async_elem(&SN[a * LD + b], &src[idx]); });
        }
        cp_async_commit();
    };
    auto next = [&](int r) {   // wait for operand r (in SN), make it SB, start r - 1 into the old SB
        cp_async_wait<0>();
        __syncthreads();
        C* t = SB; SB = SN; SN = t;
        issue(r - 1);
    };
    issue(p - 2 + n);          // the first product's operand into SN
    C* zb = ZA;
    C* zo = ZB;
    for (int m = n - 1; m >= 0; --m) {          // squarings in reverse
        next(p - 1 + m);
        if (act) {
            C acc[MT][MT];
            zero_acc<C, MT>(acc);
            mm_acc<C, MT>(acc, zb, SB, d, LD, ty, tx, G);      // Sbar S^dag
            mm_acc<C, MT>(acc, SB, zb, d, LD, ty, tx, G);      // S^dag Sbar
            store_acc<C, R, MT>(zo, acc, R(1), R(0), d, LD, ty, tx, G);
        }
        C* t = zb; zb = zo; zo = t;
    }
    C xb[MT][MT];                               // Xbar, accumulated over the Horner steps
    zero_acc<C, MT>(xb);
    for (int i = 1; i <= p - 1; ++i) {          // Horner steps in reverse
        next(p - 1 - i);
        if (act) {
            const R ri = R(1) / R(i);
            C acc[MT][MT];
            zero_acc<C, MT>(acc);
            mm_acc<C, MT>(acc, zb, SB, d, LD, ty, tx, G);      // Zbar_i Z_{i+1}^dag
#pragma unroll
            for (int a = 0; a < MT; ++a)
#pragma unroll
                for (int b = 0; b < MT; ++b) {
                    xb[a][b].x += acc[a][b].x * ri;
                    xb[a][b].y += acc[a][b].y * ri;
                }
            zero_acc<C, MT>(acc);
            mm_acc<C, MT>(acc, XH, zb, d, LD, ty, tx, G);      // X^dag Zbar_i
            store_acc<C, R, MT>(zo, acc, ri, R(0), d, LD, ty, tx, G);
        }
        C* t = zb; zb = zo; zo = t;
    }
    cp_async_wait<0>();
    __syncthreads();
    // Z_p = I + X / p: Xbar += Zbar_p / p; then dC/du_{k,j} = s sum_ab (Xbar_re Hk_im - Xbar_im Hk_re)
    const R rp = R(1) / R(p);
    if (act) {
#pragma unroll
        for (int a = 0; a < MT; ++a)
#pragma unroll
            for (int b = 0; b < MT; ++b) {
                const int r = ty + G * a, c = tx + G * b;
                if (r < d && c < d) {
                    const C z = zb[r * LD + c];
                    xb[a][b].x += z.x * rp;
                    xb[a][b].y += z.y * rp;
                }
            }
    }
    const size_t dd = (size_t)d * d;
    for (int k = 0; k < sys.M; ++k) {   // partials: FP32 pairs of exact products (FP32 form); FP64 sum
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
                        if constexpr (sizeof(R) == 4) {
                            pair_acc(hi, lo, xb[a][b].x, hk.y);
                            pair_acc(hi, lo, -xb[a][b].y, hk.x);
                        } else {
                            v += (double)xb[a][b].x * (double)hk.y - (double)xb[a][b].y * (double)hk.x;
                        }
                    }
                }
            if constexpr (sizeof(R) == 4) v = (double)hi + (double)lo;
        }
        v = block_sum(v, red);
        if (tid == 0) gpart[((size_t)e * sys.M + k) * sys.N + j] = prm->s * v;
    }
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
// the adjoint kernels of the FP32 form take the wide tile (equal padding, more outputs per thread)
template <typename R> constexpr bool adj_wide() { return sizeof(R) == 4; }

template <typename R>
static size_t fused_smem(int d, int nmat, bool wide = false) {
    const int D = slice_tile(d, wide).D;
    return (size_t)nmat * D * (D + 1) * sizeof(C_t<R>);
}

template <typename R>
size_t fused_adj_smem(int d) {
    return fused_smem<R>(d, 6, adj_wide<R>());
}

template <typename R>
int fused_max_d() {
    for (int d = kMaxD; d >= 1; --d)
        if (slice_tile(d).MT > 0 && fused_smem<R>(d, 6) <= kMaxDynSmem) return d;
    return 0;
}

template <typename R, int MT>
static cudaError_t launch_fwd_mt(const DevParams* prm, const SysView<R>& sys, int j0, int wlen, int E,
                                 C_t<R>* Ubuf, long long ustride, int wmax, const ZStore<R>& zs, int G,
                                 cudaStream_t st) {
    const size_t smem = fused_smem<R>(sys.d, 3);
    cudaError_t err = cudaFuncSetAttribute(k_expm_fwd<R, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_expm_fwd<R, MT><<<dim3(wlen, E), slice_threads(G), smem, st>>>(prm, sys, j0, Ubuf, ustride, wmax, zs, G);
    return cudaGetLastError();
}

template <typename R, int MT>
static cudaError_t launch_adj_mt(const DevParams* prm, const SysView<R>& sys, const StateView<R>& sv, int j0,
                                 int wlen, int E, const C_t<R>* states, const C_t<R>* Gbuf, int wmax,
                                 double* gpart, const ZStore<R>& zs, int G, cudaStream_t st, int* launches) {
    const size_t smem = fused_smem<R>(sys.d, 6, adj_wide<R>());
    cudaError_t err = cudaFuncSetAttribute(k_expm_adj<R, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_expm_adj<R, MT><<<dim3(wlen, E), slice_threads(G), smem, st>>>(prm, sys, sv, j0, states, Gbuf, wmax, gpart,
                                                                       zs, G);
    err = cudaGetLastError();
    *launches = 1;
    if (err != cudaSuccess || !zs.Z) return err;
    if constexpr (sizeof(R) == 4) {
        if (zs.ps) return launch_expm_adj_ps(prm, sys, sv, j0, wlen, E, states, Gbuf, wmax, gpart, zs, st, launches);
    }
    const size_t smem_r = fused_smem<R>(sys.d, 5, adj_wide<R>());
    err = cudaFuncSetAttribute(k_expm_adj_rev<R, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r);
    if (err != cudaSuccess) return err;
    k_expm_adj_rev<R, MT><<<dim3(wlen, E), slice_threads(G), smem_r, st>>>(prm, sys, sv, j0, states, Gbuf, wmax,
                                                                             gpart, zs, G);
    *launches = 2;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (!adj_lowrank_applies(sv.S, 0, sys.d)) return cudaSuccess;   // no squaring count makes it apply
    const size_t smem_l = fused_smem<R>(sys.d, 3, adj_wide<R>()) + 4 * (size_t)sys.d * kLrMax * sizeof(C_t<R>);
    err = cudaFuncSetAttribute(k_expm_adj_lr<R, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l);
    if (err != cudaSuccess) return err;
    k_expm_adj_lr<R, MT><<<dim3(wlen, E), slice_threads(G), smem_l, st>>>(prm, sys, sv, j0, states, Gbuf, wmax,
                                                                            gpart, zs, G);
    *launches = 3;
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_expm_fwd_fused(const DevParams* prm, const SysView<R>& sys, int j0, int wlen, int E,
                                  C_t<R>* Ubuf, long long ustride, int wmax, const ZStore<R>& zs, cudaStream_t st) {
    const SliceTile tl = slice_tile(sys.d);
    if (sys.d > fused_max_d<R>()) return cudaErrorInvalidValue;
    switch (tl.MT) {
        case 1: return launch_fwd_mt<R, 1>(prm, sys, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 2: return launch_fwd_mt<R, 2>(prm, sys, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 3: return launch_fwd_mt<R, 3>(prm, sys, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 4: return launch_fwd_mt<R, 4>(prm, sys, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename R>
cudaError_t launch_expm_adj_fused(const DevParams* prm, const SysView<R>& sys, const StateView<R>& sv, int j0,
                                  int wlen, int E, const C_t<R>* states, const C_t<R>* Gbuf, int wmax,
                                  double* gpart, const ZStore<R>& zs, cudaStream_t st, int* launches) {
    const SliceTile tl = slice_tile(sys.d, adj_wide<R>());
    *launches = 0;
    if (sys.d > fused_max_d<R>()) return cudaErrorInvalidValue;
    switch (tl.MT) {
        case 1: return launch_adj_mt<R, 1>(prm, sys, sv, j0, wlen, E, states, Gbuf, wmax, gpart, zs, tl.G, st, launches);
        case 2: return launch_adj_mt<R, 2>(prm, sys, sv, j0, wlen, E, states, Gbuf, wmax, gpart, zs, tl.G, st, launches);
        case 3: return launch_adj_mt<R, 3>(prm, sys, sv, j0, wlen, E, states, Gbuf, wmax, gpart, zs, tl.G, st, launches);
        case 4: return launch_adj_mt<R, 4>(prm, sys, sv, j0, wlen, E, states, Gbuf, wmax, gpart, zs, tl.G, st, launches);
        default: return cudaErrorInvalidValue;
    }
}

// resident CTAs per SM of the forward and adjoint kernels at dimension d (wave sizing)
template <typename R>
int fused_ctas_per_sm(int d, bool adjoint) {
    const SliceTile tl = slice_tile(d, adjoint && adj_wide<R>());
    if (tl.MT <= 0) return 1;
    int n = 0;
    const int thr = slice_threads(tl.G);
    cudaError_t e;
    if (!adjoint) {
        const size_t smem = fused_smem<R>(d, 3);
        switch (tl.MT) {
            case 1: cudaFuncSetAttribute(k_expm_fwd<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd<R, 1>, thr, smem); break;
            case 2: cudaFuncSetAttribute(k_expm_fwd<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd<R, 2>, thr, smem); break;
            case 3: cudaFuncSetAttribute(k_expm_fwd<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd<R, 3>, thr, smem); break;
            default: cudaFuncSetAttribute(k_expm_fwd<R, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd<R, 4>, thr, smem); break;
        }
    } else {
        const size_t smem = fused_smem<R>(d, 5, adj_wide<R>());
        switch (tl.MT) {
            case 1: cudaFuncSetAttribute(k_expm_adj_rev<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_adj_rev<R, 1>, thr, smem); break;
            case 2: cudaFuncSetAttribute(k_expm_adj_rev<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_adj_rev<R, 2>, thr, smem); break;
            case 3: cudaFuncSetAttribute(k_expm_adj_rev<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_adj_rev<R, 3>, thr, smem); break;
            default: cudaFuncSetAttribute(k_expm_adj_rev<R, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_adj_rev<R, 4>, thr, smem); break;
        }
    }
    return (e == cudaSuccess && n > 0) ? n : 1;
}

template int fused_ctas_per_sm<float>(int, bool);
template int fused_ctas_per_sm<double>(int, bool);
template size_t fused_adj_smem<float>(int);
template size_t fused_adj_smem<double>(int);
template int fused_max_d<float>();
template int fused_max_d<double>();
template cudaError_t launch_expm_fwd_fused<float>(const DevParams*, const SysView<float>&, int, int, int, float2*,
                                                  long long, int, const ZStore<float>&, cudaStream_t);
template cudaError_t launch_expm_fwd_fused<double>(const DevParams*, const SysView<double>&, int, int, int, double2*,
                                                   long long, int, const ZStore<double>&, cudaStream_t);
template cudaError_t launch_expm_adj_fused<float>(const DevParams*, const SysView<float>&, const StateView<float>&,
                                                  int, int, int, const float2*, const float2*, int, double*,
                                                  const ZStore<float>&, cudaStream_t, int*);
template cudaError_t launch_expm_adj_fused<double>(const DevParams*, const SysView<double>&, const StateView<double>&,
                                                   int, int, int, const double2*, const double2*, int, double*,
                                                   const ZStore<double>&, cudaStream_t, int*);

}  // namespace qoc
