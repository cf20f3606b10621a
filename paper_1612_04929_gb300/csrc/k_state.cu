// State-mode propagation (the paper's Eq. 12): the slice map Psi -> T_p(X_j)^(2^n) Psi applied
// to the propagated columns by Horner matrix-vector products, without forming U_j.
//
// For a block Psi of S << d columns the unitary form's O((p + n) d^3) per slice becomes
// O(p 2^n d^2 S): every application of T_p(X) = sum_{k <= p} X^k / k! is the Horner recursion
// z = v; z <- v + X z / i for i = p .. 1, and the 2^n applications replace the squarings.  It is
// the same truncated map as the unitary form, evaluated in another order, so its gradient is the
// same exact derivative of the truncated series.
//
// Three kernels:
//   k_state_x      X_j = -i s (H_0 + sum_k u_kj H_k + delta_e H_det) for the slices of a wave
//                  (FP32 form: unevaluated hi + lo pairs from the pairs s H_k; FP64 form plain);
//   k_state_chain  one CTA per (column panel, ensemble member) runs the serial recursion over the
//                  wave: dir 0 the forward Psi_j = T(X_j)^(2^n) Psi_{j-1}, dir 1 the costate
//                  G_{j-1} = T(X_j)^dag^(2^n) G_j + src_{j-1} with T(X)^dag = T(X^dag) = T(-X)
//                  (real coefficients; X is anti-Hermitian).  The block is carried in extended
//                  precision (FP32 form: pairs, every product of grid-split operands as in the
//                  unitary form's sweeps, so the coherent rounding of H_j dt stays out of long
//                  evolutions);
//   k_state_grad   one CTA per (slice, member), all slices in parallel: recomputes the 2^n
//                  application inputs from Psi_{j-1}, then runs the reverse mode of the Horner
//                  chain with the cotangent G_j of the slice's output, accumulating
//                  Xbar = sum (cotangent) (intermediate)^dag / i in shared memory, and contracts
//                  dC/du_kj = s Re tr(Xbar^dag (-i H_k)) (FP32 form: plain FP32 products, like the
//                  unitary form's adjoint; FP64 form: FP64).
#include <algorithm>

#include "qoc_device.cuh"
#include "qoc_internal.h"

namespace qoc {

namespace {

// ---- pair (hi + lo) helpers of the FP32 form ----
__device__ __forceinline__ void st_norm(float& hi, float& lo) {
    const float s = hi + lo;
    lo = lo - (s - hi);
    hi = s;
}
// (hi, lo) += u (b_hi + b_lo), u = (u_hi + u_lo) a pair of the control amplitude
__device__ __forceinline__ void st_pair_fma(float& hi, float& lo, float2 u, float bh, float bl) {
    const float p = u.x * bh;
    float e = fmaf(u.x, bh, -p);
    e = fmaf(u.x, bl, e);
    e = fmaf(u.y, bh, e);
    float s, r;
    two_sum(hi, p, s, r);
    hi = s;
    lo += r + e;
}
// a / i for a pair a
__device__ __forceinline__ void st_div(float& hi, float& lo, float fi) {
    const float q = hi / fi;
    const float r = fmaf(-q, fi, hi);
    lo = (r + lo) / fi;
    hi = q;
    st_norm(hi, lo);
}
__device__ __forceinline__ void st_add(float4& a, const float4 b) {   // pair complex a += b
    float s, r;
    two_sum(a.x, b.x, s, r);
    a.x = s;
    a.z += r + b.z;
    two_sum(a.y, b.y, s, r);
    a.y = s;
    a.w += r + b.w;
    st_norm(a.x, a.z);
    st_norm(a.y, a.w);
}
__device__ __forceinline__ unsigned st_maxbits(const float4 v) { return __float_as_uint(fmaxf(fabsf(v.x), fabsf(v.y))); }
// grid of a block whose largest component is m: column 2-norms are at most sqrt(2d) m
__device__ __forceinline__ float st_block_magic(unsigned mbits, int d) {
    const float b = sqrtf(2.0f * d) * __uint_as_float(mbits) * 1.0625f;
    int e = -100;
    if (b > 0.f) e = (b < 1e30f) ? ilogbf(b) + 1 : 100;
    return grid_magic(e < -100 ? -100 : e);
}

// element (a, c) of a d x Spad block in the panel layout
template <typename R>
__device__ __forceinline__ size_t pidx(const StateView<R>& sv, int a, int c) {
    return (size_t)(c / sv.cb) * sv.pstride + (size_t)a * sv.cb + (c % sv.cb);
}

}  // namespace

// ------------------------------------------------------------------------------------------
// X_j for the slices of a wave: item = e * wlen + jl at X + item * xs
// ------------------------------------------------------------------------------------------
__global__ void k_state_x32(const DevParams* __restrict__ prm, int d, int M, int N, const double* __restrict__ u,
                            const double* __restrict__ delta, int has_det, const float4* __restrict__ sH, int j0,
                            int wlen, float4* __restrict__ X, size_t xs) {
    __shared__ float2 us[kMaxControls + 1];
    const int item = blockIdx.y, jl = item % wlen, e = item / wlen, j = j0 + jl;
    const size_t dd = (size_t)d * d;
    for (int k = threadIdx.x; k <= M; k += blockDim.x) {
        const double v = (k < M) ? u[(size_t)k * N + j] : (delta ? delta[e] : 0.0);
        const float h = (float)v;
        us[k] = make_float2(h, (float)(v - (double)h));
    }
    __syncthreads();
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        const float4 h0 = sH[idx];
        float rh = h0.x, rl = h0.z, ih = h0.y, il = h0.w;
        for (int k = 0; k < M; ++k) {
            const float4 hk = sH[(size_t)(1 + k) * dd + idx];
            st_pair_fma(rh, rl, us[k], hk.x, hk.z);
            st_pair_fma(ih, il, us[k], hk.y, hk.w);
        }
        if (has_det) {
            const float4 hd = sH[(size_t)(M + 1) * dd + idx];
            st_pair_fma(rh, rl, us[M], hd.x, hd.z);
            st_pair_fma(ih, il, us[M], hd.y, hd.w);
        }
        st_norm(rh, rl);
        st_norm(ih, il);
        // X = -i (s H), stored grid-split on the grid of X (2^(ex - 12)) once per slice, so the
        // chain's products read their parts directly
        const float mu = grid_magic(prm->ex);
        float4 x;
        grid_split(ih, il, mu, x.x, x.z);
        grid_split(-rh, -rl, mu, x.y, x.w);
        X[(size_t)item * xs + idx] = x;
    }
}

__global__ void k_state_x64(const DevParams* __restrict__ prm, int d, int M, int N, const double* __restrict__ u,
                            const double* __restrict__ delta, int has_det, const double2* __restrict__ H64, int j0,
                            int wlen, double2* __restrict__ X, size_t xs) {
    const int item = blockIdx.y, jl = item % wlen, e = item / wlen, j = j0 + jl;
    const size_t dd = (size_t)d * d;
    const double s = prm->s;
    const double de = delta ? delta[e] : 0.0;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        double2 h = H64[idx];
        for (int k = 0; k < M; ++k) {
            const double uk = u[(size_t)k * N + j];
            const double2 hk = H64[(size_t)(1 + k) * dd + idx];
            h.x = fma(uk, hk.x, h.x);
            h.y = fma(uk, hk.y, h.y);
        }
        if (has_det) {
            const double2 hd = H64[(size_t)(M + 1) * dd + idx];
            h.x = fma(de, hd.x, h.x);
            h.y = fma(de, hd.y, h.y);
        }
        X[(size_t)item * xs + idx] = make_double2(s * h.y, -s * h.x);
    }
}

// carried-block helpers: FP32 pairs (float4) and FP64 (double2)
template <typename K> __device__ __forceinline__ K kzero_k();
template <> __device__ __forceinline__ float4 kzero_k<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double2 kzero_k<double2>() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ void st_kadd(float4& a, const float4 b) { st_add(a, b); }
__device__ __forceinline__ void st_kadd(float4& a, const float2 b) { st_add(a, make_float4(b.x, b.y, 0.f, 0.f)); }
__device__ __forceinline__ void st_kadd(double2& a, const double2 b) {
    a.x += b.x;
    a.y += b.y;
}
__device__ __forceinline__ void st_kdiv(float4& a, int i) {
    if (i == 1) return;
    st_div(a.x, a.z, (float)i);
    st_div(a.y, a.w, (float)i);
}
__device__ __forceinline__ void st_kdiv(double2& a, int i) {
    a.x /= i;
    a.y /= i;
}
__device__ __forceinline__ float2 st_round(const float4 a) { return make_float2(a.x + a.z, a.y + a.w); }
__device__ __forceinline__ double2 st_round(const double2 a) { return a; }
// pair times pair: (hi + lo)(bh + bl), the product's rounding error and the cross terms in lo
__device__ __forceinline__ void st_mul(float& hi, float& lo, float bh, float bl) {
    const float pr = hi * bh;
    float e = fmaf(hi, bh, -pr);
    e = fmaf(hi, bl, e);
    e = fmaf(lo, bh, e);
    hi = pr;
    lo = e;
    st_norm(hi, lo);
}
__device__ __forceinline__ void st_kscale(float4& a, double s) {
    const float sh = (float)s, sl = (float)(s - (double)sh);
    st_mul(a.x, a.z, sh, sl);
    st_mul(a.y, a.w, sh, sl);
}
__device__ __forceinline__ void st_kscale(double2& a, double s) {
    a.x *= s;
    a.y *= s;
}
// a <- (i s) a
__device__ __forceinline__ void st_kmul_i(float4& a, double s) {
    st_kscale(a, s);
    a = make_float4(-a.y, a.x, -a.w, a.z);
}
__device__ __forceinline__ void st_kmul_i(double2& a, double s) { a = make_double2(-s * a.y, s * a.x); }
__device__ __forceinline__ void st_ktwice(float4& a) { a = make_float4(2.f * a.x, 2.f * a.y, 2.f * a.z, 2.f * a.w); }
__device__ __forceinline__ void st_ktwice(double2& a) { a = make_double2(2.0 * a.x, 2.0 * a.y); }
__device__ __forceinline__ void st_kneg(float4& a) { a = make_float4(-a.x, -a.y, -a.z, -a.w); }
__device__ __forceinline__ void st_kneg(double2& a) { a = make_double2(-a.x, -a.y); }
// a <- i^r a (r = 0 .. 3)
__device__ __forceinline__ void st_krot(float4& a, int r) {
    if (r == 1) a = make_float4(-a.y, a.x, -a.w, a.z);
    else if (r == 2) a = make_float4(-a.x, -a.y, -a.z, -a.w);
    else if (r == 3) a = make_float4(a.y, -a.x, a.w, -a.z);
}
__device__ __forceinline__ void st_krot(double2& a, int r) {
    if (r == 1) a = make_double2(-a.y, a.x);
    else if (r == 2) a = make_double2(-a.x, -a.y);
    else if (r == 3) a = make_double2(a.y, -a.x);
}

// ------------------------------------------------------------------------------------------
// serial recursion over a wave: dir 0 forward, dir 1 costate
// ------------------------------------------------------------------------------------------
// Matrix element of X as read by the chain: FP32 grid-split pairs (float4: re and im grid parts on
// 2^(ex - 12), then the remainders; written so by k_state_x32); FP64 plain.
template <typename R> struct XElem;
template <> struct XElem<float> { using T = float4; };
template <> struct XElem<double> { using T = double2; };

// y = sgn X z for the d x cb panel.  A warp owns an output row a at a time, its lanes stride
// the columns b of X (coalesced reads of the row) for every panel column c, then a shuffle
// reduction; lane 0 writes the cb results.  FP32: z is given grid-split (zg), the grid parts'
// products are summed exactly and the cross terms rounded (the unitary form's sweep step);
// the result is an hi + lo pair.
template <int CB>
__device__ __forceinline__ void st_matvec32(const float4* __restrict__ X, const float4* __restrict__ zg,
                                            float4* __restrict__ y, int d, float mu, float sgn) {
    // RB rows per warp at a time and UB columns per lane per chunk, every load of a chunk issued
    // before its products: the chain is latency-bound, so loads in flight matter more than issue
    constexpr int RB = CB <= 2 ? 4 : 1, UB = 4;
    (void)mu;                                          // X arrives grid-split
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int a0 = warp * RB; a0 < d; a0 += nw * RB) {
        float acc[RB][CB][4];
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
            for (int c = 0; c < CB; ++c) acc[r][c][0] = acc[r][c][1] = acc[r][c][2] = acc[r][c][3] = 0.f;
        for (int b0 = 0; b0 < d; b0 += 32 * UB) {
            float4 xv[RB][UB];
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int q = 0; q < UB; ++q) {
                    const int a = a0 + r, b = b0 + q * 32 + lane;
                    xv[r][q] = (a < d && b < d) ? X[(size_t)a * d + b] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
            for (int q = 0; q < UB; ++q) {
                const int b = b0 + q * 32 + lane;
                if (b >= d) break;
                float4 zq[CB];
#pragma unroll
                for (int c = 0; c < CB; ++c) zq[c] = zg[b * CB + c];
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const float4 u = xv[r][q];        // grid part (x, y) and remainder (z, w)
                    const float2 uf = make_float2(u.x + u.z, u.y + u.w);
#pragma unroll
                    for (int c = 0; c < CB; ++c) {
                        const float4 x = zq[c];
                        float* s = acc[r][c];
                        s[0] = fmaf(u.x, x.x, s[0]);
                        s[0] = fmaf(-u.y, x.y, s[0]);
                        s[1] = fmaf(u.x, x.y, s[1]);
                        s[1] = fmaf(u.y, x.x, s[1]);
                        s[2] = fmaf(u.z, x.x, s[2]);
                        s[2] = fmaf(-u.w, x.y, s[2]);
                        s[2] = fmaf(uf.x, x.z, s[2]);
                        s[2] = fmaf(-uf.y, x.w, s[2]);
                        s[3] = fmaf(u.z, x.y, s[3]);
                        s[3] = fmaf(u.w, x.x, s[3]);
                        s[3] = fmaf(uf.x, x.w, s[3]);
                        s[3] = fmaf(uf.y, x.z, s[3]);
                    }
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int c = 0; c < CB; ++c)
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[r][c][i] += __shfl_xor_sync(0xffffffffu, acc[r][c][i], off);
        if (lane == 0) {
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const int a = a0 + r;
                if (a >= d) break;
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    float4 v;
                    two_sum(acc[r][c][0], acc[r][c][2], v.x, v.z);
                    two_sum(acc[r][c][1], acc[r][c][3], v.y, v.w);
                    y[a * CB + c] = make_float4(sgn * v.x, sgn * v.y, sgn * v.z, sgn * v.w);
                }
            }
        }
    }
}
template <int CB>
__device__ __forceinline__ void st_matvec64(const double2* __restrict__ X, const double2* __restrict__ z,
                                            double2* __restrict__ y, int d, double sgn) {
    constexpr int RB = CB <= 2 ? 4 : 1, UB = 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int a0 = warp * RB; a0 < d; a0 += nw * RB) {
        double2 acc[RB][CB];
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
            for (int c = 0; c < CB; ++c) acc[r][c] = make_double2(0.0, 0.0);
        for (int b0 = 0; b0 < d; b0 += 32 * UB) {
            double2 xv[RB][UB];
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int q = 0; q < UB; ++q) {
                    const int a = a0 + r, b = b0 + q * 32 + lane;
                    xv[r][q] = (a < d && b < d) ? X[(size_t)a * d + b] : make_double2(0.0, 0.0);
                }
#pragma unroll
            for (int q = 0; q < UB; ++q) {
                const int b = b0 + q * 32 + lane;
                if (b >= d) break;
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    const double2 zz = z[b * CB + c];
#pragma unroll
                    for (int r = 0; r < RB; ++r) cfma(acc[r][c], xv[r][q], zz);
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    acc[r][c].x += __shfl_xor_sync(0xffffffffu, acc[r][c].x, off);
                    acc[r][c].y += __shfl_xor_sync(0xffffffffu, acc[r][c].y, off);
                }
        if (lane == 0)
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const int a = a0 + r;
                if (a >= d) break;
#pragma unroll
                for (int c = 0; c < CB; ++c) y[a * CB + c] = make_double2(sgn * acc[r][c].x, sgn * acc[r][c].y);
            }
    }
}

// One CTA per (panel kb, member e), CB = the panel width.  Shared memory: the block v at the
// start of the current application, the Horner accumulator z, the product y, the grid-split z
// (FP32), and, when XS, X_j of the current slice (copied once per slice).
template <typename R, int CB, bool XS>
__global__ void __launch_bounds__(512) k_state_chain(StateChainArgs<R> A) {
    using C = C_t<R>;
    using K = K_t<R>;
    using XE = typename XElem<R>::T;
    extern __shared__ __align__(16) unsigned char sm[];
    const int kb = blockIdx.x, e = blockIdx.y, tid = threadIdx.x, nt = blockDim.x;
    const int d = A.d, P = d * CB;
    XE* Xs = reinterpret_cast<XE*>(sm);
    K* v = reinterpret_cast<K*>(sm + (XS ? (size_t)d * d * sizeof(XE) : 0));
    K* z = v + P;
    K* y = z + P;
    K* wacc = y + P;        // Chebyshev: the running sum and the previous term
    K* zprev = wacc + P;
    float4* zg = reinterpret_cast<float4*>(zprev + P);
    __shared__ unsigned zmax[2];
    const size_t slice = A.sv.slice(), poff = (size_t)kb * A.sv.pstride;
    const int p = A.prm->p, n = A.prm->n;
    float mu = 0.f;
    if constexpr (sizeof(R) == 4) mu = grid_magic(A.prm->ex);
    const bool fwd = A.dir == 0;
    const R sgn = fwd ? R(1) : R(-1);                  // costate: T(X^dag) = T(-X)
    if (tid == 0) zmax[0] = zmax[1] = 0u;
    __syncthreads();
    // starting block: forward from the checkpoint; costate from the in-carry (or zero) plus the
    // source of the wave's last slice
    for (int o = tid; o < P; o += nt) {
        const int a = o / CB, c = o - a * CB;
        const size_t gi = poff + (size_t)a * A.sv.cb + c;
        K x = kzero_k<K>();
        if (A.cin) x = A.cin[(size_t)e * A.cin_es + gi];
        if (!fwd) {
            st_kadd(x, A.src[(size_t)e * A.src_es + (size_t)(A.wlen - 1) * slice + gi]);
            A.out[(size_t)e * A.out_es + (size_t)(A.wlen - 1) * slice + gi] = st_round(x);
        } else {
            A.out[(size_t)e * A.out_es + gi] = st_round(x);
        }
        v[o] = x;
        if constexpr (sizeof(R) == 4) atomicMax(&zmax[0], st_maxbits(x));
    }
    int par = 0;   // zmax slot holding the current z's largest component
    const size_t nitems = (size_t)A.wlen;
#pragma unroll 1
    for (int t = 0; t < A.wlen; ++t) {
        const int jl = fwd ? t : A.wlen - 1 - t;
        const XE* Xg = reinterpret_cast<const XE*>(A.X) + ((size_t)e * nitems + jl) * A.xs;
        __syncthreads();                                // v complete; the previous slice is done
        if constexpr (XS) {
            for (int i = tid; i < d * d; i += nt) Xs[i] = Xg[i];
            __syncthreads();
        }
        const XE* Xj = XS ? Xs : Xg;
        // y = sgn X b for the block b whose largest component zmax[par] holds (FP32: b is split on
        // its grid first); barriers on both sides
        auto matvec = [&](const K* bsrc, R sg) {
            __syncthreads();                            // b written, y free
            if constexpr (sizeof(R) == 4) {
                const float mx = st_block_magic(zmax[par], d);
                for (int o = tid; o < P; o += nt) {
                    const float4 w = bsrc[o];
                    float4 q;
                    grid_split(w.x, w.z, mx, q.x, q.z);
                    grid_split(w.y, w.w, mx, q.y, q.w);
                    zg[o] = q;
                }
                if (tid == 0) zmax[par ^ 1] = 0u;
                __syncthreads();
                st_matvec32<CB>(reinterpret_cast<const float4*>(Xj), zg, reinterpret_cast<float4*>(y), d, mu, (float)sg);
            } else {
                st_matvec64<CB>(reinterpret_cast<const double2*>(Xj), reinterpret_cast<const double2*>(bsrc),
                                reinterpret_cast<double2*>(y), d, (double)sg);
            }
            __syncthreads();                            // y complete
        };
        if (!A.cheb) {
#pragma unroll 1
            for (int m = 0; m < (1 << n); ++m) {
                for (int o = tid; o < P; o += nt) z[o] = v[o];
                // zmax[par] holds the largest component of v (= z)
#pragma unroll 1
                for (int i = p; i >= 1; --i) {
                    matvec(z, sgn);
                    for (int o = tid; o < P; o += nt) {     // z = v + y / i
                        K w = y[o];
                        st_kdiv(w, i);
                        st_kadd(w, v[o]);
                        z[o] = w;
                        if constexpr (sizeof(R) == 4) atomicMax(&zmax[par ^ 1], st_maxbits(w));
                    }
                    par ^= 1;
                }
                __syncthreads();
                for (int o = tid; o < P; o += nt) v[o] = z[o];
            }
        } else {
            // Chebyshev: w = sum_k a_k rot_k(phi_k), phi_0 = v, phi_1 = A v, phi_{k+1} = 2 A phi_k -
            // phi_{k-1}, A = (i / theta) X (Hermitian); rot_k = (-i)^k forward, i^k for the adjoint
            const int Kc = A.cheb->K;
            for (int o = tid; o < P; o += nt) {
                zprev[o] = v[o];
                K w = v[o];
                st_kscale(w, A.cheb->a[0]);
                wacc[o] = w;
            }
#pragma unroll 1
            for (int k = 1; k <= Kc; ++k) {
                matvec(k == 1 ? v : z, R(1));
                const int rot = fwd ? ((4 - (k & 3)) & 3) : (k & 3);   // power of i
                for (int o = tid; o < P; o += nt) {
                    K a = y[o];
                    st_kmul_i(a, A.cheb->inv_theta);            // A phi = (i / theta) X phi
                    K nx = a;
                    if (k > 1) {
                        st_ktwice(nx);
                        K pm = zprev[o];
                        st_kneg(pm);
                        st_kadd(nx, pm);
                        zprev[o] = z[o];
                    }
                    if (k == 1) zprev[o] = v[o];
                    z[o] = nx;
                    K t = nx;
                    st_krot(t, rot);
                    st_kscale(t, A.cheb->a[k]);
                    K w = wacc[o];
                    st_kadd(w, t);
                    wacc[o] = w;
                    if constexpr (sizeof(R) == 4) atomicMax(&zmax[par ^ 1], st_maxbits(nx));
                }
                par ^= 1;
            }
            __syncthreads();
            for (int o = tid; o < P; o += nt) v[o] = wacc[o];
        }
        // the slice's result: forward Psi_{jl+1}; costate U_jl^dag G_jl, then + src_{jl-1}
        for (int o = tid; o < P; o += nt) {
            const int a = o / CB, c = o - a * CB;
            const size_t gi = poff + (size_t)a * A.sv.cb + c;
            K x = v[o];
            if (fwd) {
                A.out[(size_t)e * A.out_es + (size_t)(jl + 1) * slice + gi] = st_round(x);
                if (jl == A.wlen - 1 && A.cout) A.cout[(size_t)e * A.cout_es + gi] = x;
            } else if (jl >= 1) {
                st_kadd(x, A.src[(size_t)e * A.src_es + (size_t)(jl - 1) * slice + gi]);
                A.out[(size_t)e * A.out_es + (size_t)(jl - 1) * slice + gi] = st_round(x);
                v[o] = x;
            } else if (A.cout) {
                A.cout[(size_t)e * A.cout_es + gi] = x;
            }
        }
        // the next slice starts from v: its largest component (the costate's source was added)
        if constexpr (sizeof(R) == 4) {
            __syncthreads();
            if (tid == 0) zmax[par ^ 1] = 0u;
            __syncthreads();
            for (int o = tid; o < P; o += nt) atomicMax(&zmax[par ^ 1], st_maxbits(v[o]));
            par ^= 1;
        }
    }
}

// ------------------------------------------------------------------------------------------
// per-slice exact gradient of the truncated map (all slices of a wave in parallel)
// ------------------------------------------------------------------------------------------
constexpr int kStateMaxS = 8;

// y = sgn X z on d x S compact blocks (column c of row a at a * S + c), plain arithmetic in the
// compute precision (FP32 form: X's pair rounded to FP32)
template <typename R, typename XE>
__device__ __forceinline__ void st_mv_plain(const XE* __restrict__ X, const C_t<R>* __restrict__ z,
                                            C_t<R>* __restrict__ y, int d, int S, R sgn) {
    using C = C_t<R>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int a = warp; a < d; a += nw) {
        C acc[kStateMaxS];
#pragma unroll
        for (int c = 0; c < kStateMaxS; ++c) acc[c] = czero<C>();
        const XE* Xr = X + (size_t)a * d;
        for (int b = lane; b < d; b += 32) {
            const XE xv = Xr[b];
            C x;
            if constexpr (sizeof(R) == 4) x = make_float2(xv.x + xv.z, xv.y + xv.w);
            else x = xv;
#pragma unroll
            for (int c = 0; c < kStateMaxS; ++c)
                if (c < S) cfma(acc[c], x, z[b * S + c]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int c = 0; c < kStateMaxS; ++c) {
                acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, off);
                acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, off);
            }
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < kStateMaxS; ++c)
                if (c < S) {
                    C r;
                    r.x = sgn * acc[c].x;
                    r.y = sgn * acc[c].y;
                    y[a * S + c] = r;
                }
    }
}

// c <- (i s) c for a complex value of either precision
template <typename C, typename R>
__device__ __forceinline__ C cmul_i(const C c, R s) {
    C r;
    r.x = -s * c.y;
    r.y = s * c.x;
    return r;
}
template <typename C>
__device__ __forceinline__ C crot(const C c, int r) {   // i^r c
    C o = c;
    if (r == 1) { o.x = -c.y; o.y = c.x; }
    else if (r == 2) { o.x = -c.x; o.y = -c.y; }
    else if (r == 3) { o.x = c.y; o.y = -c.x; }
    return o;
}

// Exact gradient of the Chebyshev map w = sum_k c_k phi_k, phi_0 = v, phi_1 = A v,
// phi_{k+1} = 2 A phi_k - phi_{k-1}, A = (i / theta) X (so A^dag = A), c_k = (-i)^k a_k:
// cotangents b_k of phi_k from the top, b_k = conj(c_k) wbar + f A b_{k+1} - b_{k+2} (f = 2,
// or 1 for k = 0), Abar += f b_{k+1} phi_k^dag; then Xbar = (-i / theta) Abar into Xb.
template <typename R, typename XE>
__device__ void cheb_grad(const StateGradArgs<R>& A, const XE* X, const C_t<R>* Psi, const C_t<R>* Gj, C_t<R>* Xb,
                          C_t<R>* pool, C_t<R>* Phi) {
    using C = C_t<R>;
    const int tid = threadIdx.x, nt = blockDim.x, d = A.d, S = A.sv.S;
    const size_t dd = (size_t)d * d, blk = (size_t)d * S;
    const int Kc = A.cheb->K;
    const R th = (R)A.cheb->inv_theta;
    // Phi: the K + 1 terms, in the item's global scratch; the cotangent blocks in shared memory
    C* wb = pool;
    C* b2 = wb + blk;
    C* b1 = b2 + blk;
    C* b0 = b1 + blk;
    C* tmp = b0 + blk;
    for (int o = tid; o < (int)blk; o += nt) {
        const int a = o / S, c = o - a * S;
        Phi[o] = Psi[pidx(A.sv, a, c)];
        wb[o] = Gj[pidx(A.sv, a, c)];
    }
    for (int k = 1; k <= Kc; ++k) {                    // the forward terms
        __syncthreads();
        st_mv_plain<R, XE>(X, Phi + (size_t)(k - 1) * blk, tmp, d, S, R(1));
        __syncthreads();
        for (int o = tid; o < (int)blk; o += nt) {
            C a = cmul_i(tmp[o], th);
            if (k > 1) {
                a.x = R(2) * a.x - Phi[(size_t)(k - 2) * blk + o].x;
                a.y = R(2) * a.y - Phi[(size_t)(k - 2) * blk + o].y;
            }
            Phi[(size_t)k * blk + o] = a;
        }
    }
    for (int o = tid; o < (int)blk; o += nt) {         // b_{K+1} = 0, b_K = conj(c_K) wbar
        b2[o] = czero<C>();
        C t = crot(wb[o], Kc & 3);
        t.x *= (R)A.cheb->a[Kc];
        t.y *= (R)A.cheb->a[Kc];
        b1[o] = t;
    }
    for (int k = Kc - 1; k >= 0; --k) {
        const R f = k == 0 ? R(1) : R(2);
        __syncthreads();
        // Abar += f b_{k+1} phi_k^dag
        const C* ph = Phi + (size_t)k * blk;
        for (size_t idx = tid; idx < dd; idx += nt) {
            const int a = (int)(idx / d), b = (int)(idx - (size_t)a * d);
            C acc = Xb[idx];
            for (int c = 0; c < S; ++c) {
                C t = b1[a * S + c];
                t.x *= f;
                t.y *= f;
                cfma_bcj(acc, t, ph[b * S + c]);
            }
            Xb[idx] = acc;
        }
        st_mv_plain<R, XE>(X, b1, tmp, d, S, R(1));
        __syncthreads();
        for (int o = tid; o < (int)blk; o += nt) {
            C t = crot(wb[o], k & 3);
            t.x *= (R)A.cheb->a[k];
            t.y *= (R)A.cheb->a[k];
            const C am = cmul_i(tmp[o], th);
            t.x += f * am.x - b2[o].x;
            t.y += f * am.y - b2[o].y;
            b0[o] = t;
        }
        __syncthreads();
        for (int o = tid; o < (int)blk; o += nt) {     // shift: b_{k+2} <- b_{k+1}, b_{k+1} <- b_k
            b2[o] = b1[o];
            b1[o] = b0[o];
        }
    }
    __syncthreads();
    for (size_t idx = tid; idx < dd; idx += nt) Xb[idx] = cmul_i(Xb[idx], -th);   // Xbar = (-i / theta) Abar
}

template <typename R>
__global__ void __launch_bounds__(512) k_state_grad(StateGradArgs<R> A) {
    using C = C_t<R>;
    using XE = typename XElem<R>::T;
    extern __shared__ __align__(16) unsigned char sm[];
    const int item = blockIdx.x, jl = item % A.wlen, e = item / A.wlen, j = A.j0 + jl;
    const int tid = threadIdx.x, nt = blockDim.x, d = A.d, S = A.sv.S;
    const int p = A.prm->p, n = A.prm->n, napp = 1 << n;
    const size_t dd = (size_t)d * d, blk = (size_t)d * S, slice = A.sv.slice();
    C* Xb = reinterpret_cast<C*>(sm);                  // Xbar, d x d
    C* zb = Xb + dd;                                   // cotangent
    C* vb = zb + blk;                                  // cotangent of the application input
    C* tmp = vb + blk;
    // the napp + 1 application inputs and the Horner intermediates Z[1 .. p + 1] (or the Chebyshev
    // terms) in the item's global scratch
    C* V = A.scr + (size_t)item * A.scr_stride;
    C* Z = V + (size_t)(napp + 1) * blk;
    const XE* X = reinterpret_cast<const XE*>(A.X) + (size_t)item * A.xs;
    const C* Psi = A.states + ((size_t)e * (A.wmax + 1) + jl) * slice;
    const C* Gj = A.G + ((size_t)e * A.wmax + jl) * slice;
    for (size_t i = tid; i < dd; i += nt) Xb[i] = czero<C>();
    if (A.cheb) {
        cheb_grad(A, X, Psi, Gj, Xb, Xb + dd, A.scr + (size_t)item * A.scr_stride);
    } else {
    for (int o = tid; o < (int)blk; o += nt) {
        const int a = o / S, c = o - a * S;
        V[o] = Psi[pidx(A.sv, a, c)];
        vb[o] = Gj[pidx(A.sv, a, c)];
    }
    // one application z = T(X) v: Z[p + 1] = v, Z[i] = v + X Z[i + 1] / i (Z[1] the result)
    auto apply = [&](const C* v) {
        for (int o = tid; o < (int)blk; o += nt) Z[(size_t)(p + 1) * blk + o] = v[o];
        for (int i = p; i >= 1; --i) {
            __syncthreads();
            st_mv_plain<R, XE>(X, Z + (size_t)(i + 1) * blk, tmp, d, S, R(1));
            __syncthreads();
            const R ri = R(1) / R(i);
            for (int o = tid; o < (int)blk; o += nt) {
                C w = tmp[o];
                w.x = fma(w.x, ri, v[o].x);
                w.y = fma(w.y, ri, v[o].y);
                Z[(size_t)i * blk + o] = w;
            }
        }
        __syncthreads();
    };
    for (int m = 0; m < napp; ++m) {                    // inputs of the 2^n applications
        apply(V + (size_t)m * blk);
        for (int o = tid; o < (int)blk; o += nt) V[(size_t)(m + 1) * blk + o] = Z[blk + o];
    }
    for (int m = napp - 1; m >= 0; --m) {
        apply(V + (size_t)m * blk);                     // Z[i] of application m
        for (int o = tid; o < (int)blk; o += nt) {
            zb[o] = vb[o];
            vb[o] = czero<C>();
        }
        for (int i = 1; i <= p; ++i) {
            __syncthreads();
            const R ri = R(1) / R(i);
            for (int o = tid; o < (int)blk; o += nt) {     // v contributes directly to z_i
                vb[o].x += zb[o].x;
                vb[o].y += zb[o].y;
            }
            // Xbar += zbar Z[i + 1]^dag / i
            const C* Zi1 = Z + (size_t)(i + 1) * blk;
            for (size_t idx = tid; idx < dd; idx += nt) {
                const int a = (int)(idx / d), b = (int)(idx - (size_t)a * d);
                C acc = Xb[idx];
                for (int c = 0; c < S; ++c) {
                    C t = zb[a * S + c];
                    t.x *= ri;
                    t.y *= ri;
                    cfma_bcj(acc, t, Zi1[b * S + c]);
                }
                Xb[idx] = acc;
            }
            // zbar <- X^dag zbar / i = -X zbar / i
            st_mv_plain<R, XE>(X, zb, tmp, d, S, R(-1));
            __syncthreads();
            for (int o = tid; o < (int)blk; o += nt) {
                C w = tmp[o];
                w.x *= ri;
                w.y *= ri;
                zb[o] = w;
            }
        }
        __syncthreads();
        for (int o = tid; o < (int)blk; o += nt) {          // z_{p+1} = v
            vb[o].x += zb[o].x;
            vb[o].y += zb[o].y;
        }
    }
    }
    __syncthreads();
    // dC/du_kj = s Re tr(Xbar^dag (-i H_k)) = s sum (Xbar_re Hk_im - Xbar_im Hk_re)
    __shared__ double red[32];
    for (int k = 0; k < A.M; ++k) {
        const C* hk = A.Hk + (size_t)k * dd;
        double v = 0.0;
        for (size_t idx = tid; idx < dd; idx += nt)
            v += (double)Xb[idx].x * (double)hk[idx].y - (double)Xb[idx].y * (double)hk[idx].x;
        v = block_sum(v, red);
        if (tid == 0) A.gpart[((size_t)e * A.M + k) * A.N + j] = A.prm->s * v;
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
// shared memory of the gradient kernel: Xbar and five d x S blocks
template <typename R>
size_t state_grad_smem(int d, int S, int p, int n, int K) {
    (void)p;
    (void)n;
    (void)K;
    return sizeof(C_t<R>) * ((size_t)d * d + 5 * (size_t)d * S);
}
// global scratch per item (C elements): the application inputs and Horner intermediates, or the
// Chebyshev terms
size_t state_grad_scratch(int d, int S, int p, int n, int K) {
    const size_t blocks = K > 0 ? (size_t)K + 1 : (size_t)(1 << n) + 1 + p + 2;
    return blocks * (size_t)d * S;
}

template <typename R>
cudaError_t launch_state_x(const DevParams* prm, int d, int M, int N, const double* u, const double* delta, int has_det,
                           const void* Hsrc, int j0, int wlen, int E, void* X, size_t xs, cudaStream_t st) {
    const size_t dd = (size_t)d * d;
    const int eb = (int)std::min<size_t>(64, (dd + 255) / 256);
    if constexpr (sizeof(R) == 4)
        k_state_x32<<<dim3(eb, wlen * E), 256, 0, st>>>(prm, d, M, N, u, delta, has_det,
                                                        reinterpret_cast<const float4*>(Hsrc), j0, wlen,
                                                        reinterpret_cast<float4*>(X), xs);
    else
        k_state_x64<<<dim3(eb, wlen * E), 256, 0, st>>>(prm, d, M, N, u, delta, has_det,
                                                        reinterpret_cast<const double2*>(Hsrc), j0, wlen,
                                                        reinterpret_cast<double2*>(X), xs);
    return cudaGetLastError();
}

template <typename R, int CB, bool XS>
static cudaError_t chain_launch(const StateChainArgs<R>& a, cudaStream_t st) {
    using XE = typename XElem<R>::T;
    const size_t P = (size_t)a.d * CB;
    const size_t smem = (XS ? (size_t)a.d * a.d * sizeof(XE) : 0) + 5 * P * sizeof(K_t<R>) + P * sizeof(float4);
    if (smem > kMaxDynSmem) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_state_chain<R, CB, XS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int threads = a.d > 64 ? 512 : 256;   // a warp per matrix row in the products
    k_state_chain<R, CB, XS><<<dim3(a.sv.ncb, a.E), threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename R, int CB>
static cudaError_t chain_xs(const StateChainArgs<R>& a, cudaStream_t st) {
    using XE = typename XElem<R>::T;
    const size_t P = (size_t)a.d * CB;
    const size_t with_x = (size_t)a.d * a.d * sizeof(XE) + 5 * P * sizeof(K_t<R>) + P * sizeof(float4);
    if (with_x <= kMaxDynSmem) return chain_launch<R, CB, true>(a, st);   // X_j staged per slice
    return chain_launch<R, CB, false>(a, st);                              // rows read from L2
}

template <typename R>
cudaError_t launch_state_chain(const StateChainArgs<R>& a, cudaStream_t st) {
    switch (a.sv.cb) {
        case 1: return chain_xs<R, 1>(a, st);
        case 2: return chain_xs<R, 2>(a, st);
        case 3: return chain_xs<R, 3>(a, st);
        case 4: return chain_xs<R, 4>(a, st);
        case 5: return chain_xs<R, 5>(a, st);
        case 6: return chain_xs<R, 6>(a, st);
        case 7: return chain_xs<R, 7>(a, st);
        case 8: return chain_xs<R, 8>(a, st);
    }
    return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_state_grad(const StateGradArgs<R>& a, int p, int n, cudaStream_t st) {
    if (a.sv.S > kStateMaxS) return cudaErrorInvalidValue;
    const size_t smem = state_grad_smem<R>(a.d, a.sv.S, p, n, a.cheb ? a.K : 0);
    if (smem > kMaxDynSmem) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_state_grad<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (a.M == 0) return cudaSuccess;
    k_state_grad<R><<<a.wlen * a.E, 512, smem, st>>>(a);
    return cudaGetLastError();
}

template size_t state_grad_smem<float>(int, int, int, int, int);
template size_t state_grad_smem<double>(int, int, int, int, int);
template cudaError_t launch_state_x<float>(const DevParams*, int, int, int, const double*, const double*, int,
                                           const void*, int, int, int, void*, size_t, cudaStream_t);
template cudaError_t launch_state_x<double>(const DevParams*, int, int, int, const double*, const double*, int,
                                            const void*, int, int, int, void*, size_t, cudaStream_t);
template cudaError_t launch_state_chain<float>(const StateChainArgs<float>&, cudaStream_t);
template cudaError_t launch_state_chain<double>(const StateChainArgs<double>&, cudaStream_t);
template cudaError_t launch_state_grad<float>(const StateGradArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_state_grad<double>(const StateGradArgs<double>&, int, int, cudaStream_t);

}  // namespace qoc
