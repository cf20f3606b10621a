// Large-d slice exponentials and their exact adjoint as batched tiled GEMMs.
//
// When the matrices of one slice no longer fit one CTA's shared memory (d > 64 FP32, d > 48
// FP64), every Horner / squaring product of Eqs. 9-10 runs as one launch over all slices of the
// wave: CTA (tile, item) computes a T x T tile of C_item = A_item B_item with the operands
// streamed through shared memory in K-chunks.  The same arithmetic as the per-slice kernels:
//   * FP32 form: X_j grid-split (qoc_device.cuh) from an FP64 assembly, split products (exact
//     FP32 sums of the grid parts plus rounded cross terms) for the squarings and for the
//     Horner steps i <= m_split, plain FP32 products for the earlier steps; U_j is the rounded
//     sum of its two parts;
//   * adjoint: the block recursion on [[X^dag, Ubar], [0, X^dag]] (exact derivative of the
//     truncated series), FP32 (FP32 form) or FP64 (FP64 form);
//   * dC/du_{k,j} = Re tr(Xbar^dag (-i s H_k)) reduced in FP64.
// Matrices of item b sit at base + b * mstride, row-major d x d.
#include <cmath>
#include <type_traits>
#include <utility>

#include "qoc_device.cuh"
#include "qoc_internal.h"

namespace qoc {

// ------------------------------------------------------------------------------------------
// element helpers: E = float4 (pair), float2, double2
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void big_norm(float& hi, float& lo) {
    const float s = hi + lo;
    lo = lo - (s - hi);
    hi = s;
}
__device__ __forceinline__ void big_div(float& hi, float& lo, float fi) {
    const float q = hi / fi;
    const float r = fmaf(-q, fi, hi);
    lo = (r + lo) / fi;
    hi = q;
    big_norm(hi, lo);
}
__device__ __forceinline__ void big_add1(float& hi, float& lo) {
    const float t = hi + 1.0f;
    const float bv = t - hi;
    lo += (hi - (t - bv)) + (1.0f - bv);
    hi = t;
    big_norm(hi, lo);
}

template <typename E> __device__ __forceinline__ E ezero();
template <> __device__ __forceinline__ float4 ezero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ float2 ezero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 ezero<double2>() { return make_double2(0.0, 0.0); }

// Tile rows owned by a thread are ty + 16 x; rows at or past d (edge tiles) add nothing.  The
// number of x a warp has to run: the largest over its lanes, so that the skip is warp-uniform.
__device__ __forceinline__ int warp_rows(int valid, int ty, int MT) {
    int xs = 0;
    while (xs < MT && ty + 16 * xs < valid) ++xs;
    return __reduce_max_sync(0xffffffffu, (unsigned)xs);
}

// ------------------------------------------------------------------------------------------
// assembly: X = -i s H_j (+ delta_e H_det) from FP64 H; Z = I + X / p
// ------------------------------------------------------------------------------------------
// float4: grid-split with exponent e (e == kFullForm: the full FP32 value in .x, .y, zero .z, .w)
constexpr int kFullForm = 1000;
__device__ __forceinline__ void put(float4& o, double x, double y, int e) {
    if (e == kFullForm) {
        o = make_float4((float)x, (float)y, 0.f, 0.f);
        return;
    }
    o.x = (float)ldexp(rint(ldexp(x, 12 - e)), e - 12);
    o.y = (float)ldexp(rint(ldexp(y, 12 - e)), e - 12);
    o.z = (float)(x - (double)o.x);
    o.w = (float)(y - (double)o.y);
}
__device__ __forceinline__ void put(double2& o, double x, double y, int) { o = make_double2(x, y); }
__device__ __forceinline__ void put(float2& o, double x, double y, int) { o = make_float2((float)x, (float)y); }

template <typename E>
__global__ void k_big_assemble(const DevParams* __restrict__ prm, BigSys sys, int j0, int wlen, E* __restrict__ X,
                               E* __restrict__ Z, size_t mstride, int ex, int ezp) {
    const int item = blockIdx.y, jl = item % wlen, e = item / wlen, j = j0 + jl;
    const int d = sys.d, M = sys.M;
    const size_t dd = (size_t)d * d;
    const double s = prm->s;
    const double ip = 1.0 / prm->p;
    const double de = sys.delta ? sys.delta[e] : 0.0;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        double2 h = sys.H64[idx];
        for (int k = 0; k < M; ++k) {
            const double uk = sys.u[(size_t)k * sys.N + j];
            const double2 hk = sys.H64[(size_t)(1 + k) * dd + idx];
            h.x = fma(uk, hk.x, h.x);
            h.y = fma(uk, hk.y, h.y);
        }
        if (sys.has_det) {
            const double2 hd = sys.H64[(size_t)(M + 1) * dd + idx];
            h.x = fma(de, hd.x, h.x);
            h.y = fma(de, hd.y, h.y);
        }
        const double xr = s * h.y, xi = -s * h.x;
        const int a = (int)(idx / d), b = (int)(idx - (size_t)a * d);
        E xv, zv;
        put(xv, xr, xi, ex);
        put(zv, xr * ip + (a == b ? 1.0 : 0.0), xi * ip, ezp);
        X[(size_t)item * mstride + idx] = xv;
        Z[(size_t)item * mstride + idx] = zv;
    }
}

// FP32 split form: X = -i s H_j and Z = I + X / p in pair arithmetic from the pairs s H_0,
// s H_k, s H_det (as the per-slice split kernel assembles them), grid-split (ex; Z with ezp).
__device__ __forceinline__ float4 big_gsplit(float rh, float rl, float ih, float il, int e) {
    if (e == kFullForm) return make_float4(rh + rl, ih + il, 0.f, 0.f);
    const float m = grid_magic(e);
    float4 o;
    grid_split(rh, rl, m, o.x, o.z);
    grid_split(ih, il, m, o.y, o.w);
    return o;
}
__global__ void k_big_assemble_split(const DevParams* __restrict__ prm, BigSys sys, const float4* __restrict__ sH,
                                     int j0, int wlen, float4* __restrict__ X, float4* __restrict__ Z, size_t mstride,
                                     int ex, int ezp) {
    __shared__ float2 us[kMaxControls + 1];
    const int item = blockIdx.y, jl = item % wlen, e = item / wlen, j = j0 + jl;
    const int d = sys.d, M = sys.M;
    const size_t dd = (size_t)d * d;
    for (int k = threadIdx.x; k <= M; k += blockDim.x) {
        const double v = (k < M) ? sys.u[(size_t)k * sys.N + j] : (sys.delta ? sys.delta[e] : 0.0);
        const float h = (float)v;
        us[k] = make_float2(h, (float)(v - (double)h));
    }
    __syncthreads();
    const float fp = (float)prm->p;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        const float4 h0 = sH[idx];
        float rh = h0.x, rl = h0.z, ih = h0.y, il = h0.w;
        for (int k = 0; k < M; ++k) {
            const float4 hk = sH[(size_t)(1 + k) * dd + idx];
            pair_fma(rh, rl, us[k], hk.x, hk.z);
            pair_fma(ih, il, us[k], hk.y, hk.w);
        }
        if (sys.has_det) {
            const float4 hd = sH[(size_t)(M + 1) * dd + idx];
            pair_fma(rh, rl, us[M], hd.x, hd.z);
            pair_fma(ih, il, us[M], hd.y, hd.w);
        }
        big_norm(rh, rl);
        big_norm(ih, il);
        float xrh = ih, xrl = il, xih = -rh, xil = -rl;   // X = -i (s H)
        X[(size_t)item * mstride + idx] = big_gsplit(xrh, xrl, xih, xil, ex);
        if (prm->p > 1) {
            big_div(xrh, xrl, fp);
            big_div(xih, xil, fp);
        }
        if (!Z) continue;   // the Paterson-Stockmeyer form starts from X alone
        const int a = (int)(idx / d), b = (int)(idx - (size_t)a * d);
        if (a == b) big_add1(xrh, xrl);
        Z[(size_t)item * mstride + idx] = big_gsplit(xrh, xrl, xih, xil, ezp);
    }
}

// ------------------------------------------------------------------------------------------
// batched product C = A B (T x T tile per CTA), epilogue:
//   kind 0: C = I + AB / i     (Horner step i)
//   kind 1: C = AB             (squaring)
//   kind 2: C = AB + c0 I + c1 X + c2 X^2   (Paterson-Stockmeyer chain product; SPLIT and PLAIN32
//           only: the block terms in pair arithmetic (SPLIT) or FP32 (PLAIN32), from PsAdd)
// SPLIT: split product of grid-split float4 operands, the result grid-split with `magic`;
// PLAIN32: plain FP32 product of a grid-split A (X) and a full-form B, the result in full form
// (magic == 0) or grid-split; otherwise plain products of E = float2 / double2.
// ------------------------------------------------------------------------------------------
constexpr int KC = 16;

// the block B_q = c0 I + c1 X + c2 X^2 added by a Paterson-Stockmeyer chain product (kind 2); the
// coefficients as FP32 pairs, X and X^2 grid-split, item matrices mstride apart
struct PsAdd {
    const float4* X = nullptr;
    const float4* X2 = nullptr;
    float2 c0{0.f, 0.f}, c1{0.f, 0.f}, c2{0.f, 0.f};
};

template <typename E, int T, int MODE>   // MODE 0 plain, 1 split, 2 plain FP32 (E = float4)
__global__ void __launch_bounds__(256)
k_big_mm(int d, const E* __restrict__ A, const E* __restrict__ B, E* __restrict__ Cm, size_t mstride, int kind, int i,
         float magic, PsAdd ps) {
    constexpr int MT = T / 16;
    // two buffers of (As[T][KC + 1], Bs[KC][T + 1]): the next K-chunk is copied (cp.async) while
    // the current one is multiplied
    extern __shared__ __align__(16) unsigned char smraw[];
    typedef E ATile[T][KC + 1];
    typedef E BTile[KC][T + 1];
    ATile* Abuf = reinterpret_cast<ATile*>(smraw);
    BTile* Bbuf = reinterpret_cast<BTile*>(smraw + 2 * sizeof(ATile));
    const int item = blockIdx.y;
    const int ntn = (d + T - 1) / T;
    const int tm = blockIdx.x / ntn, tn = blockIdx.x - tm * ntn;
    const int r0 = tm * T, c0 = tn * T;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int xw = warp_rows(d - r0, ty, MT);
    const E* Ai = A + (size_t)item * mstride;
    const E* Bi = B + (size_t)item * mstride;
    // split accumulators: grid sums (re, im) exact, cross terms (re, im); MODE 2 uses [0], [1]
    float sa[MT][MT][4];
    E acc[MT][MT];
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y) {
            sa[x][y][0] = sa[x][y][1] = sa[x][y][2] = sa[x][y][3] = 0.f;
            acc[x][y] = ezero<E>();
        }
    auto issue = [&](int buf, int k0) {
        for (int idx = tid; idx < T * KC; idx += 256) {
            const int r = idx / KC, k = idx - r * KC;
            const int gr = r0 + r, gk = k0 + k;
            if (gr < d && gk < d) cp_async_elem(&Abuf[buf][r][k], &Ai[(size_t)gr * d + gk]);
            else Abuf[buf][r][k] = ezero<E>();
        }
        for (int idx = tid; idx < KC * T; idx += 256) {
            const int k = idx / T, c = idx - k * T;
            const int gk = k0 + k, gc = c0 + c;
            if (gk < d && gc < d) cp_async_elem(&Bbuf[buf][k][c], &Bi[(size_t)gk * d + gc]);
            else Bbuf[buf][k][c] = ezero<E>();
        }
    };
    const int nch = (d + KC - 1) / KC;
    issue(0, 0);
    cp_async_commit();
    for (int ch = 0; ch < nch; ++ch) {
        if (ch + 1 < nch) issue((ch + 1) & 1, (ch + 1) * KC);
        cp_async_commit();
        cp_async_wait<1>();   // chunk ch has landed
        __syncthreads();
        const ATile& As = Abuf[ch & 1];
        const BTile& Bs = Bbuf[ch & 1];
        const int kmax = min(KC, d - ch * KC);   // the last chunk may be partial (zero-padded)
#pragma unroll 4
        for (int k = 0; k < kmax; ++k) {
            E a[MT], b[MT];
#pragma unroll
            for (int x = 0; x < MT; ++x) a[x] = As[ty + 16 * x][k];
#pragma unroll
            for (int y = 0; y < MT; ++y) b[y] = Bs[k][tx + 16 * y];
            float2 bf[MT], af[MT];   // full values: of B (MODE 1), of A (MODE 2)
#pragma unroll
            for (int y = 0; y < MT; ++y) {
                if constexpr (MODE == 1) {
                    const float4 bv = *reinterpret_cast<const float4*>(&b[y]);
                    bf[y] = make_float2(bv.x + bv.z, bv.y + bv.w);
                }
                if constexpr (MODE == 2) {
                    const float4 av = *reinterpret_cast<const float4*>(&a[y]);
                    af[y] = make_float2(av.x + av.z, av.y + av.w);
                }
            }
#pragma unroll
            for (int x = 0; x < MT; ++x) {
                if (x >= xw) break;   // rows past d in every lane of this warp
#pragma unroll
                for (int y = 0; y < MT; ++y) {
                    if constexpr (MODE == 1) {
                        const float4 av = *reinterpret_cast<const float4*>(&a[x]);
                        const float4 bv = *reinterpret_cast<const float4*>(&b[y]);
                        float* c = sa[x][y];
                        c[0] = fmaf(av.x, bv.x, c[0]);
                        c[0] = fmaf(-av.y, bv.y, c[0]);
                        c[1] = fmaf(av.x, bv.y, c[1]);
                        c[1] = fmaf(av.y, bv.x, c[1]);
                        c[2] = fmaf(av.x, bv.z, c[2]);
                        c[2] = fmaf(-av.y, bv.w, c[2]);
                        c[2] = fmaf(av.z, bf[y].x, c[2]);
                        c[2] = fmaf(-av.w, bf[y].y, c[2]);
                        c[3] = fmaf(av.x, bv.w, c[3]);
                        c[3] = fmaf(av.y, bv.z, c[3]);
                        c[3] = fmaf(av.z, bf[y].y, c[3]);
                        c[3] = fmaf(av.w, bf[y].x, c[3]);
                    } else if constexpr (MODE == 2) {
                        const float4 bv = *reinterpret_cast<const float4*>(&b[y]);
                        float* c = sa[x][y];
                        c[0] = fmaf(af[x].x, bv.x, c[0]);
                        c[0] = fmaf(-af[x].y, bv.y, c[0]);
                        c[1] = fmaf(af[x].x, bv.y, c[1]);
                        c[1] = fmaf(af[x].y, bv.x, c[1]);
                    } else {
                        cfma(acc[x][y], a[x], b[y]);
                    }
                }
            }
        }
        __syncthreads();   // before this buffer is refilled
    }
    E* Ci = Cm + (size_t)item * mstride;
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y) {
            const int r = r0 + ty + 16 * x, c = c0 + tx + 16 * y;
            if (r >= d || c >= d) continue;
            const bool diag = (kind == 0) && (r == c);
            E out;
            if constexpr (MODE == 1) {
                float rh, rl, ih, il;
                two_sum(sa[x][y][0], sa[x][y][2], rh, rl);
                two_sum(sa[x][y][1], sa[x][y][3], ih, il);
                if (kind == 2) {
                    const size_t o = (size_t)item * mstride + (size_t)r * d + c;
                    const float4 xv = ps.X[o], yv = ps.X2[o];
                    pair_fma(rh, rl, ps.c1, xv.x, xv.z);
                    pair_fma(ih, il, ps.c1, xv.y, xv.w);
                    pair_fma(rh, rl, ps.c2, yv.x, yv.z);
                    pair_fma(ih, il, ps.c2, yv.y, yv.w);
                    if (r == c) df_addc(rh, rl, ps.c0);
                }
                if (kind == 0 && i > 1) {
                    big_div(rh, rl, (float)i);
                    big_div(ih, il, (float)i);
                }
                if (diag) big_add1(rh, rl);
                float4 o;
                grid_split(rh, rl, magic, o.x, o.z);
                grid_split(ih, il, magic, o.y, o.w);
                out = *reinterpret_cast<E*>(&o);
            } else if constexpr (MODE == 2) {
                float4 o;
                if (kind == 2) {
                    const size_t oi = (size_t)item * mstride + (size_t)r * d + c;
                    const float4 xv = ps.X[oi], yv = ps.X2[oi];
                    float re = fmaf(ps.c1.x, xv.x + xv.z, sa[x][y][0]);
                    float im = fmaf(ps.c1.x, xv.y + xv.w, sa[x][y][1]);
                    re = fmaf(ps.c2.x, yv.x + yv.z, re);
                    im = fmaf(ps.c2.x, yv.y + yv.w, im);
                    if (r == c) re += ps.c0.x;
                    o = make_float4(re, im, 0.f, 0.f);
                } else {
                    const float ri = 1.0f / (float)i;
                    o = make_float4(fmaf(sa[x][y][0], ri, diag ? 1.0f : 0.0f), sa[x][y][1] * ri, 0.f, 0.f);
                }
                if (magic != 0.f) {   // read by a split product
                    grid_split(o.x, 0.f, magic, o.x, o.z);
                    grid_split(o.y, 0.f, magic, o.y, o.w);
                }
                out = *reinterpret_cast<E*>(&o);
            } else {
                out = acc[x][y];
                if (kind == 0) {
                    using S = decltype(out.x);
                    const S ri = S(1) / S(i);
                    out.x = out.x * ri + (diag ? S(1) : S(0));
                    out.y = out.y * ri;
                }
            }
            Ci[(size_t)r * d + c] = out;
        }
}

// U_j (rounded) and U_j^dag into the propagator buffer (U at 0, U^dag at ustride / 2)
template <typename E, typename C>
__device__ __forceinline__ C to_c(const E v);
template <> __device__ __forceinline__ float2 to_c<float4, float2>(const float4 v) { return make_float2(v.x + v.z, v.y + v.w); }
template <> __device__ __forceinline__ float2 to_c<float2, float2>(const float2 v) { return v; }
template <> __device__ __forceinline__ double2 to_c<double2, double2>(const double2 v) { return v; }

template <typename E, typename C>
__global__ void k_big_store_u(int d, const E* __restrict__ Z, size_t mstride, C* __restrict__ Ubuf, long long ustride,
                              int wlen, int wmax) {
    const int item = blockIdx.y, jl = item % wlen, e = item / wlen;
    const size_t dd = (size_t)d * d;
    C* U = Ubuf + ((size_t)e * wmax + jl) * ustride;
    C* UH = U + ustride / 2;
    const E* Zi = Z + (size_t)item * mstride;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx / d), b = (int)(idx - (size_t)a * d);
        U[idx] = to_c<E, C>(Zi[idx]);
        C h = to_c<E, C>(Zi[(size_t)b * d + a]);
        h.y = -h.y;
        UH[idx] = h;
    }
}

// ------------------------------------------------------------------------------------------
// adjoint
// ------------------------------------------------------------------------------------------
// XH = X^dag with X = -i s H_j assembled in the compute precision R (as the per-slice adjoint
// kernel does) and, for the block recursion (Z11 set), Z11 = I + XH / p.
template <typename R>
__global__ void k_big_adj_init(const DevParams* __restrict__ prm, SysView<R> sys, int j0, int wlen,
                               C_t<R>* __restrict__ XH, C_t<R>* __restrict__ Z11, size_t mstride) {
    using C = C_t<R>;
    const int item = blockIdx.y, jl = item % wlen, e = item / wlen, j = j0 + jl;
    const int d = sys.d, M = sys.M;
    const size_t dd = (size_t)d * d;
    const R s = (R)prm->s;
    const R ip = R(1) / R(prm->p);
    const R de = sys.delta ? (R)sys.delta[e] : R(0);
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx / d), b = (int)(idx - (size_t)a * d);
        // X[b][a] = -i s H[b][a]  ->  XH[a][b] = conj(X[b][a])
        const size_t o = (size_t)b * d + a;
        C h = sys.H0[o];
        for (int k = 0; k < M; ++k) {
            const R uk = (R)sys.u[(size_t)k * sys.N + j];
            const C hk = sys.Hk[(size_t)k * dd + o];
            h.x = fma(uk, hk.x, h.x);
            h.y = fma(uk, hk.y, h.y);
        }
        if (sys.Hdet) {
            const C hd = sys.Hdet[o];
            h.x = fma(de, hd.x, h.x);
            h.y = fma(de, hd.y, h.y);
        }
        C xh;
        xh.x = s * h.y;      // X = (s hi, -s hr); conj -> (s hi, s hr)
        xh.y = s * h.x;
        const size_t base = (size_t)item * mstride + idx;
        XH[base] = xh;
        if (Z11) {
            C z1;
            z1.x = xh.x * ip + (a == b ? R(1) : R(0));
            z1.y = xh.y * ip;
            Z11[base] = z1;
        }
    }
}

// The factors of Ubar = G_j Psi_{j-1}^dag as d x d row-major matrices for the tiled product:
// Gm[a][c] = G_j[a][c] and Ph[c][b] = conj(Psi_{j-1}[b][c]) for the S propagated columns c,
// zero for c >= S (panel layout in: column c of panel c / cb).
template <typename C>
__global__ void k_big_ubar_factors(int d, StateView<typename std::conditional<sizeof(C) == 8, float, double>::type> sv,
                                   int wlen, const C* __restrict__ states, const C* __restrict__ Gbuf, int wmax,
                                   C* __restrict__ Gm, C* __restrict__ Ph, size_t mstride) {
    const int item = blockIdx.y, jl = item % wlen, e = item / wlen;
    const size_t dd = (size_t)d * d, slice = sv.slice();
    const C* Gj = Gbuf + ((size_t)e * wmax + jl) * slice;
    const C* Pj = states + ((size_t)e * (wmax + 1) + jl) * slice;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx / d), c = (int)(idx - (size_t)a * d);   // Gm row a col c; Ph row c col a
        C g = czero<C>(), q = czero<C>();
        if (c < sv.S) {
            const size_t pa = (size_t)(c / sv.cb) * sv.pstride + (size_t)a * sv.cb + (c % sv.cb);
            g = Gj[pa];
            q = Pj[pa];
            q.y = -q.y;
        }
        Gm[(size_t)item * mstride + idx] = g;
        Ph[(size_t)item * mstride + (size_t)c * d + a] = q;
    }
}

// Z12 = Ubar / p (block recursion start)
template <typename C>
__global__ void k_big_scale_p(const DevParams* __restrict__ prm, int d, const C* __restrict__ Ub, C* __restrict__ Z12,
                              size_t mstride) {
    using S = decltype(C{}.x);
    const int item = blockIdx.y;
    const size_t dd = (size_t)d * d;
    const S ip = S(1) / S(prm->p);
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        C v = Ub[(size_t)item * mstride + idx];
        v.x *= ip;
        v.y *= ip;
        Z12[(size_t)item * mstride + idx] = v;
    }
}

// P11 = A11 B11 ; P12 = A11 B12 + A12 B11 ; kind 0: Horner (I + P11 / i, P12 / i), 1: plain
template <typename C, int T>
__global__ void __launch_bounds__(256)
k_big_mm_blk(int d, const C* __restrict__ A11, const C* __restrict__ A12, const C* __restrict__ B11,
             const C* __restrict__ B12, C* __restrict__ O11, C* __restrict__ O12, size_t mstride, int kind, int i) {
    constexpr int MT = T / 16;
    // two buffers of (A1s, A2s [T][KC + 1], B1s, B2s [KC][T + 1]), filled by cp.async one K-chunk ahead
    extern __shared__ __align__(16) unsigned char smraw[];
    typedef C ATile[T][KC + 1];
    typedef C BTile[KC][T + 1];
    ATile* A1b = reinterpret_cast<ATile*>(smraw);
    ATile* A2b = A1b + 2;
    BTile* B1b = reinterpret_cast<BTile*>(smraw + 4 * sizeof(ATile));
    BTile* B2b = B1b + 2;
    const int item = blockIdx.y;
    const int ntn = (d + T - 1) / T;
    const int tm = blockIdx.x / ntn, tn = blockIdx.x - tm * ntn;
    const int r0 = tm * T, c0 = tn * T;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const size_t off = (size_t)item * mstride;
    C acc1[MT][MT], acc2[MT][MT];
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y) acc1[x][y] = acc2[x][y] = czero<C>();
    auto issue = [&](int buf, int k0) {
        for (int idx = tid; idx < T * KC; idx += 256) {
            const int r = idx / KC, k = idx - r * KC;
            const int gr = r0 + r, gk = k0 + k;
            if (gr < d && gk < d) {
                cp_async_elem(&A1b[buf][r][k], &A11[off + (size_t)gr * d + gk]);
                cp_async_elem(&A2b[buf][r][k], &A12[off + (size_t)gr * d + gk]);
            } else {
                A1b[buf][r][k] = czero<C>();
                A2b[buf][r][k] = czero<C>();
            }
        }
        for (int idx = tid; idx < KC * T; idx += 256) {
            const int k = idx / T, c = idx - k * T;
            const int gk = k0 + k, gc = c0 + c;
            if (gk < d && gc < d) {
                cp_async_elem(&B1b[buf][k][c], &B11[off + (size_t)gk * d + gc]);
                cp_async_elem(&B2b[buf][k][c], &B12[off + (size_t)gk * d + gc]);
            } else {
                B1b[buf][k][c] = czero<C>();
                B2b[buf][k][c] = czero<C>();
            }
        }
    };
    const int nch = (d + KC - 1) / KC;
    issue(0, 0);
    cp_async_commit();
    for (int ch = 0; ch < nch; ++ch) {
        if (ch + 1 < nch) issue((ch + 1) & 1, (ch + 1) * KC);
        cp_async_commit();
        cp_async_wait<1>();   // chunk ch has landed
        __syncthreads();
        const ATile& A1s = A1b[ch & 1];
        const ATile& A2s = A2b[ch & 1];
        const BTile& B1s = B1b[ch & 1];
        const BTile& B2s = B2b[ch & 1];
        const int kmax = min(KC, d - ch * KC);   // the last chunk may be partial (zero-padded)
#pragma unroll 4
        for (int k = 0; k < kmax; ++k) {
            C a1[MT], a2[MT], b1[MT], b2[MT];
#pragma unroll
            for (int x = 0; x < MT; ++x) {
                a1[x] = A1s[ty + 16 * x][k];
                a2[x] = A2s[ty + 16 * x][k];
            }
#pragma unroll
            for (int y = 0; y < MT; ++y) {
                b1[y] = B1s[k][tx + 16 * y];
                b2[y] = B2s[k][tx + 16 * y];
            }
#pragma unroll
            for (int x = 0; x < MT; ++x)
#pragma unroll
                for (int y = 0; y < MT; ++y) {
                    cfma(acc1[x][y], a1[x], b1[y]);
                    cfma(acc2[x][y], a1[x], b2[y]);
                    cfma(acc2[x][y], a2[x], b1[y]);
                }
        }
        __syncthreads();   // before this buffer is refilled
    }
    using S = decltype(acc1[0][0].x);
    const S ri = (kind == 0) ? S(1) / S(i) : S(1);
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y) {
            const int r = r0 + ty + 16 * x, c = c0 + tx + 16 * y;
            if (r >= d || c >= d) continue;
            C v1 = acc1[x][y], v2 = acc2[x][y];
            v1.x = v1.x * ri + ((kind == 0 && r == c) ? S(1) : S(0));
            v1.y *= ri;
            v2.x *= ri;
            v2.y *= ri;
            O11[off + (size_t)r * d + c] = v1;
            O12[off + (size_t)r * d + c] = v2;
        }
}

// dC/du_{k,j} = s sum_ab (Xbar_re Hk_im - Xbar_im Hk_re), one CTA per (item, k)
template <typename R>
__global__ void __launch_bounds__(256)
k_big_grad(const DevParams* __restrict__ prm, SysView<R> sys, int j0, int wlen, const C_t<R>* __restrict__ Xbar,
           size_t mstride, double* __restrict__ gpart) {
    __shared__ double red[32];
    const int item = blockIdx.x, k = blockIdx.y, jl = item % wlen, e = item / wlen, j = j0 + jl;
    const int d = sys.d;
    const size_t dd = (size_t)d * d;
    const C_t<R>* xb = Xbar + (size_t)item * mstride;
    const C_t<R>* hk = sys.Hk + (size_t)k * dd;
    // per-thread partials: FP32 form as (hi, lo) pairs of exact products, FP64 form in FP64; the
    // block sum in FP64
    double v = 0.0;
    if constexpr (sizeof(R) == 4) {
        float hi = 0.f, lo = 0.f;
        for (size_t idx = threadIdx.x; idx < dd; idx += blockDim.x) {
            pair_acc(hi, lo, xb[idx].x, hk[idx].y);
            pair_acc(hi, lo, -xb[idx].y, hk[idx].x);
        }
        v = (double)hi + (double)lo;
    } else {
        for (size_t idx = threadIdx.x; idx < dd; idx += blockDim.x)
            v += (double)xb[idx].x * (double)hk[idx].y - (double)xb[idx].y * (double)hk[idx].x;
    }
    v = block_sum(v, red);
    if (threadIdx.x == 0) gpart[((size_t)e * sys.M + k) * sys.N + j] = prm->s * v;
}

// the conjugate transpose of Z (the right operand of forward product r), rounded to the compute
// precision, into the operand store: zst + (item * cap + r) * mstride
template <typename E, typename C>
__global__ void k_big_store_ct(int d, const E* __restrict__ Z, size_t mstride, C* __restrict__ zst, int cap, int r) {
    const int item = blockIdx.y;
    const size_t dd = (size_t)d * d;
    const E* Zi = Z + (size_t)item * mstride;
    C* dst = zst + ((size_t)item * cap + r) * mstride;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx / d), b = (int)(idx - (size_t)a * d);
        C v = to_c<E, C>(Zi[(size_t)b * d + a]);
        v.y = -v.y;
        dst[idx] = v;
    }
}

// Paterson-Stockmeyer top block W_qt = c0 I + c1 X + c2 X^2 + c3 X^3 (pairs; X^2 read when p >= 2,
// X^3 when p >= 3), in the form its reader takes (grid exponent e, or kFullForm)
__global__ void k_big_ps_top(int d, const float4* __restrict__ X, const float4* __restrict__ X2,
                             const float4* __restrict__ X3, float4* __restrict__ W, size_t mstride, float2 c0, float2 c1,
                             float2 c2, float2 c3, int p, int e) {
    const size_t dd = (size_t)d * d, off = (size_t)blockIdx.y * mstride;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        const float4 xv = X[off + idx];
        pair_fma(rh, rl, c1, xv.x, xv.z);
        pair_fma(ih, il, c1, xv.y, xv.w);
        if (p >= 2) {
            const float4 yv = X2[off + idx];
            pair_fma(rh, rl, c2, yv.x, yv.z);
            pair_fma(ih, il, c2, yv.y, yv.w);
        }
        if (p >= 3) {
            const float4 zv = X3[off + idx];
            pair_fma(rh, rl, c3, zv.x, zv.z);
            pair_fma(ih, il, c3, zv.y, zv.w);
        }
        const int a = (int)(idx / d), b = (int)(idx - (size_t)a * d);
        if (a == b) df_addc(rh, rl, c0);
        W[off + idx] = big_gsplit(rh, rl, ih, il, e);
    }
}

// Cotangent accumulation of the Paterson-Stockmeyer reverse mode: Xbar += a Z, X2bar += b Z,
// Ybar += c Z (a zero coefficient leaves its target untouched)
__global__ void k_big_ps_acc(int d, const float2* __restrict__ Z, float2* __restrict__ Xb, float2* __restrict__ X2b,
                             float2* __restrict__ Yb, size_t mstride, float a, float b, float c) {
    const size_t dd = (size_t)d * d, off = (size_t)blockIdx.y * mstride;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        const float2 z = Z[off + idx];
        if (a != 0.f) {
            float2 v = Xb[off + idx];
            v.x = fmaf(a, z.x, v.x);
            v.y = fmaf(a, z.y, v.y);
            Xb[off + idx] = v;
        }
        if (b != 0.f) {
            float2 v = X2b[off + idx];
            v.x = fmaf(b, z.x, v.x);
            v.y = fmaf(b, z.y, v.y);
            X2b[off + idx] = v;
        }
        if (c != 0.f) {
            float2 v = Yb[off + idx];
            v.x = fmaf(c, z.x, v.x);
            v.y = fmaf(c, z.y, v.y);
            Yb[off + idx] = v;
        }
    }
}

// Reverse mode over the stored products (two products per tile, operands at their own item strides):
//   mode 0 (Horner step i): O1 = A1 B1 / i,  O2 += A2 B2 / i   (Zbar' = X^dag Zbar / i, Xbar += Zbar Z^dag / i)
//   mode 1 (squaring):      O1 = A1 B1 + A2 B2                (Sbar' = Sbar S^dag + S^dag Sbar)
template <typename C>
struct RevOps {
    const C* p[4];          // A1, B1, A2, B2
    size_t s[4];            // item strides
};
template <typename C, int T>
__global__ void __launch_bounds__(256)
k_big_rev(int d, RevOps<C> ops, C* __restrict__ O1, C* __restrict__ O2, size_t mstride, int mode, int i) {
    constexpr int MT = T / 16;
    extern __shared__ __align__(16) unsigned char smraw[];
    typedef C ATile[T][KC + 1];
    typedef C BTile[KC][T + 1];
    ATile* A1b = reinterpret_cast<ATile*>(smraw);
    ATile* A2b = A1b + 2;
    BTile* B1b = reinterpret_cast<BTile*>(smraw + 4 * sizeof(ATile));
    BTile* B2b = B1b + 2;
    const int item = blockIdx.y;
    const int ntn = (d + T - 1) / T;
    const int tm = blockIdx.x / ntn, tn = blockIdx.x - tm * ntn;
    const int r0 = tm * T, c0 = tn * T;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int xw = warp_rows(d - r0, ty, MT);
    const C* A1 = ops.p[0] + (size_t)item * ops.s[0];
    const C* B1 = ops.p[1] + (size_t)item * ops.s[1];
    const C* A2 = ops.p[2] + (size_t)item * ops.s[2];
    const C* B2 = ops.p[3] + (size_t)item * ops.s[3];
    C acc1[MT][MT], acc2[MT][MT];
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y) acc1[x][y] = acc2[x][y] = czero<C>();
    auto issue = [&](int buf, int k0) {
        for (int idx = tid; idx < T * KC; idx += 256) {
            const int r = idx / KC, k = idx - r * KC;
            const int gr = r0 + r, gk = k0 + k;
            if (gr < d && gk < d) {
                cp_async_elem(&A1b[buf][r][k], &A1[(size_t)gr * d + gk]);
                cp_async_elem(&A2b[buf][r][k], &A2[(size_t)gr * d + gk]);
            } else {
                A1b[buf][r][k] = czero<C>();
                A2b[buf][r][k] = czero<C>();
            }
        }
        for (int idx = tid; idx < KC * T; idx += 256) {
            const int k = idx / T, c = idx - k * T;
            const int gk = k0 + k, gc = c0 + c;
            if (gk < d && gc < d) {
                cp_async_elem(&B1b[buf][k][c], &B1[(size_t)gk * d + gc]);
                cp_async_elem(&B2b[buf][k][c], &B2[(size_t)gk * d + gc]);
            } else {
                B1b[buf][k][c] = czero<C>();
                B2b[buf][k][c] = czero<C>();
            }
        }
    };
    const int nch = (d + KC - 1) / KC;
    issue(0, 0);
    cp_async_commit();
    for (int ch = 0; ch < nch; ++ch) {
        if (ch + 1 < nch) issue((ch + 1) & 1, (ch + 1) * KC);
        cp_async_commit();
        cp_async_wait<1>();   // chunk ch has landed
        __syncthreads();
        const ATile& A1s = A1b[ch & 1];
        const ATile& A2s = A2b[ch & 1];
        const BTile& B1s = B1b[ch & 1];
        const BTile& B2s = B2b[ch & 1];
        const int kmax = min(KC, d - ch * KC);   // the last chunk may be partial (zero-padded)
#pragma unroll 4
        for (int k = 0; k < kmax; ++k) {
            C a1[MT], a2[MT], b1[MT], b2[MT];
#pragma unroll
            for (int x = 0; x < MT; ++x) {
                a1[x] = A1s[ty + 16 * x][k];
                a2[x] = A2s[ty + 16 * x][k];
            }
#pragma unroll
            for (int y = 0; y < MT; ++y) {
                b1[y] = B1s[k][tx + 16 * y];
                b2[y] = B2s[k][tx + 16 * y];
            }
#pragma unroll
            for (int x = 0; x < MT; ++x) {
                if (x >= xw) break;   // rows past d in every lane of this warp
#pragma unroll
                for (int y = 0; y < MT; ++y) {
                    cfma(acc1[x][y], a1[x], b1[y]);
                    if (mode == 0) cfma(acc2[x][y], a2[x], b2[y]);
                    else cfma(acc1[x][y], a2[x], b2[y]);
                }
            }
        }
        __syncthreads();   // before this buffer is refilled
    }
    using S = decltype(acc1[0][0].x);
    const S ri = (mode == 0) ? S(1) / S(i) : S(1);
    const size_t off = (size_t)item * mstride;
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y) {
            const int r = r0 + ty + 16 * x, c = c0 + tx + 16 * y;
            if (r >= d || c >= d) continue;
            C v1 = acc1[x][y];
            v1.x *= ri;
            v1.y *= ri;
            O1[off + (size_t)r * d + c] = v1;
            if (mode == 0) {
                C v2 = O2[off + (size_t)r * d + c];
                v2.x += acc2[x][y].x * ri;
                v2.y += acc2[x][y].y * ri;
                O2[off + (size_t)r * d + c] = v2;
            }
        }
}

// Xbar += Zbar / p (the last Horner factor Z_p = I + X / p)
template <typename C>
__global__ void k_big_axpy(int d, const C* __restrict__ Z, C* __restrict__ X, size_t mstride, int p) {
    const int item = blockIdx.y;
    const size_t dd = (size_t)d * d, off = (size_t)item * mstride;
    using S = decltype(Z[0].x);
    const S rp = S(1) / S(p);
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        const C z = Z[off + idx];
        C x = X[off + idx];
        x.x += z.x * rp;
        x.y += z.y * rp;
        X[off + idx] = x;
    }
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
static int big_tile(int d) { return d <= 96 ? 32 : 64; }

template <typename E, int T> constexpr size_t mm_smem() { return 2 * sizeof(E) * ((size_t)T * (KC + 1) + (size_t)KC * (T + 1)); }
template <typename E, int T> constexpr size_t blk_smem() { return 2 * mm_smem<E, T>(); }

template <typename E, int T, int MODE>
static cudaError_t mm_launch_t(int d, int items, const E* A, const E* B, E* Cm, size_t mstride, int kind, int i,
                               float magic, cudaStream_t st, const PsAdd& ps) {
    constexpr size_t smem = mm_smem<E, T>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_big_mm<E, T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nt = ((d + T - 1) / T) * ((d + T - 1) / T);
    k_big_mm<E, T, MODE><<<dim3(nt, items), 256, smem, st>>>(d, A, B, Cm, mstride, kind, i, magic, ps);
    return cudaGetLastError();
}

template <typename E, int MODE>
static cudaError_t mm_launch(int d, int items, const E* A, const E* B, E* Cm, size_t mstride, int kind, int i,
                             cudaStream_t st, float magic = 0.f, const PsAdd& ps = PsAdd{}) {
    if (big_tile(d) == 32) return mm_launch_t<E, 32, MODE>(d, items, A, B, Cm, mstride, kind, i, magic, st, ps);
    return mm_launch_t<E, 64, MODE>(d, items, A, B, Cm, mstride, kind, i, magic, st, ps);
}

template <typename C, int T>
static cudaError_t blk_launch_t(int d, int items, const C* A11, const C* A12, const C* B11, const C* B12, C* O11,
                                C* O12, size_t ms, int kind, int i, cudaStream_t st) {
    constexpr size_t smem = blk_smem<C, T>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_big_mm_blk<C, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nt = ((d + T - 1) / T) * ((d + T - 1) / T);
    k_big_mm_blk<C, T><<<dim3(nt, items), 256, smem, st>>>(d, A11, A12, B11, B12, O11, O12, ms, kind, i);
    return cudaGetLastError();
}

static int ew_blocks(size_t dd) {
    const size_t b = (dd + 255) / 256;
    return (int)(b < 64 ? b : 64);
}

// Paterson-Stockmeyer form of the split exponential (the per-slice k_expm_fwd_ps as batched
// products): X^2 and X^3, the top block element-wise, the chain W_q = B_q + X^3 W_{q+1} with B_q
// added in the product's epilogue (split products for q <= (m_split - 1) / 3, plain FP32 above),
// then the squarings.  Scratch per item: X, X^2, X^3 and the W ping-pong (five float4 matrices).
// Stored operands (conjugate transposes) in the slot layout of ps_slots.
static cudaError_t big_expm_ps(const BigArgs<float>& a, const DevParams& hp, cudaStream_t st, int* launches,
                               float2* zst, const OzFwd* ozf) {
    const int p = hp.p, n = hp.n, d = a.d, items = a.wlen * a.E;
    const size_t ms = a.mstride;
    const int eb = ew_blocks((size_t)d * d);
    const int qt = ps_top(p), qs = (hp.m_split - 1) / 3, cap = ps_big_slots(p, n);
    if (!a.sH || qt >= kPsMaxBlocks) return cudaErrorInvalidValue;
    auto count = [&]() { if (launches) ++*launches; };
    float4* X = reinterpret_cast<float4*>(a.scratch);
    float4* X2 = X + (size_t)items * ms;
    float4* X3 = X2 + (size_t)items * ms;
    float4* win = X3 + (size_t)items * ms;
    float4* wout = win + (size_t)items * ms;
    auto magic = [](int e) { return std::ldexp(1.5f, e + 11); };
    // the form W_q is written in: its reader is chain product q - 1 (split iff q - 1 <= qs), or the
    // squarings for W_0 = T
    auto form_w = [&](int q) { return q == 0 ? hp.eu : (q - 1 <= qs ? hp.ew[q] : kFullForm); };
    auto coef = [&](int k) { return make_float2(hp.ch[k], hp.cl[k]); };
    cudaError_t err;
    auto store = [&](const float4* Z, int slot) -> cudaError_t {
        if (!zst) return cudaSuccess;
        k_big_store_ct<float4, float2><<<dim3(eb, items), 256, 0, st>>>(d, Z, ms, zst, cap, slot);
        count();
        return cudaGetLastError();
    };
    k_big_assemble_split<<<dim3(eb, items), 256, 0, st>>>(a.prm, a.bsys, a.sH, a.j0, a.wlen, X, nullptr, ms, hp.ex,
                                                          hp.eu);
    count();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = store(X, cap - 1)) != cudaSuccess) return err;   // X^dag for the reverse mode
    // With tensor-core products (ozf) every product is split-grade, so every chain matrix is written
    // grid-split on its own bound.  Sliced matrices: 0 / 1 the A / B operand of X^2 and of the
    // squarings (1 keeps X for X^3), 2 X^2, 3 X^3 (once for the whole chain), 4 the chain operand.
    const PsAdd none{};
    auto tc = [&](const float4* A, int am, const float4* B, int bm, float4* O, int kind, float mg,
                  const PsAdd& ps) -> cudaError_t {
        int n_l = 0;
        const cudaError_t e2 = oz_fwd_product(*ozf, A, am, B, bm, O, ms, kind, mg, ps.X, ps.X2, ps.c0, ps.c1, ps.c2,
                                              st, &n_l);
        if (launches) *launches += n_l;
        return e2;
    };
    if (p >= 2) {
        err = ozf ? tc(X, 0, X, 1, X2, 1, magic(hp.e2), none)
                  : mm_launch<float4, 1>(d, items, X, X, X2, ms, 1, 0, st, magic(hp.e2));
        if (!ozf) count();
        if (err != cudaSuccess) return err;
        if ((err = store(X2, 0)) != cudaSuccess) return err;
    }
    if (p >= 3) {
        err = ozf ? tc(X2, 2, nullptr, 1, X3, 1, magic(hp.e3), none)
                  : mm_launch<float4, 1>(d, items, X2, X, X3, ms, 1, 0, st, magic(hp.e3));
        if (!ozf) count();
        if (err != cudaSuccess) return err;
        if ((err = store(X3, 1)) != cudaSuccess) return err;
    }
    auto form_of = [&](int q) { return ozf ? (q == 0 ? hp.eu : hp.ew[q]) : form_w(q); };
    k_big_ps_top<<<dim3(eb, items), 256, 0, st>>>(d, X, X2, X3, win, ms, coef(3 * qt), coef(3 * qt + 1),
                                                  coef(3 * qt + 2), coef(3 * qt + 3), p, form_of(qt));
    count();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    for (int q = qt - 1; q >= 0; --q) {
        if ((err = store(win, 2 + (qt - 1 - q))) != cudaSuccess) return err;
        PsAdd ps;
        ps.X = X;
        ps.X2 = X2;
        ps.c0 = coef(3 * q);
        ps.c1 = coef(3 * q + 1);
        ps.c2 = coef(3 * q + 2);
        const int f = form_of(q);
        const float mg = f == kFullForm ? 0.f : magic(f);
        if (ozf) {
            err = tc(q == qt - 1 ? X3 : nullptr, 3, win, 4, wout, 2, mg, ps);
        } else {
            err = (q <= qs) ? mm_launch<float4, 1>(d, items, X3, win, wout, ms, 2, 0, st, mg, ps)
                            : mm_launch<float4, 2>(d, items, X3, win, wout, ms, 2, 0, st, mg, ps);
            count();
        }
        if (err != cudaSuccess) return err;
        std::swap(win, wout);
    }
    for (int m = 0; m < n; ++m) {
        if ((err = store(win, qt + 2 + m)) != cudaSuccess) return err;
        if (ozf) {
            err = tc(win, 0, win, 1, wout, 1, magic(hp.eu), none);
        } else {
            err = mm_launch<float4, 1>(d, items, win, win, wout, ms, 1, 0, st, magic(hp.eu));
            count();
        }
        if (err != cudaSuccess) return err;
        std::swap(win, wout);
    }
    k_big_store_u<float4, float2><<<dim3(eb, items), 256, 0, st>>>(d, win, ms, reinterpret_cast<float2*>(a.Ubuf),
                                                                     a.ustride, a.wlen, a.wmax);
    count();
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_big_expm(const BigArgs<R>& a, const DevParams& hp, bool split, cudaStream_t st, int* launches,
                            C_t<R>* zst, const OzFwd* ozf) {
    const int p = hp.p, n = hp.n, m_split = hp.m_split;
    const int d = a.d, items = a.wlen * a.E;
    const size_t dd = (size_t)d * d;
    const int eb = ew_blocks(dd);
    cudaError_t err;
    auto count = [&]() { if (launches) ++*launches; };
    const int cap = p - 1 + n;
    auto store = [&](const auto* Z, int r) -> cudaError_t {   // right operand of product r, for the adjoint
        if (!zst) return cudaSuccess;
        using E = std::remove_cv_t<std::remove_pointer_t<decltype(Z)>>;
        k_big_store_ct<E, C_t<R>><<<dim3(eb, items), 256, 0, st>>>(d, Z, a.mstride, zst, cap, r);
        count();
        return cudaGetLastError();
    };
    if constexpr (sizeof(R) == 4) if (split && a.ps) return big_expm_ps(a, hp, st, launches, zst, ozf);
    if constexpr (sizeof(R) == 4) if (split) {
        float4* X = reinterpret_cast<float4*>(a.scratch);
        float4* Za = X + (size_t)items * a.mstride;
        float4* Zb = Za + (size_t)items * a.mstride;
        // the operand of a split product is grid-split (X: ex; Z_i, i >= 2: ez; T and its
        // squarings: eu), the operand of a plain FP32 Horner step is in full form
        const float mz = std::ldexp(1.5f, hp.ez + 11), mu = std::ldexp(1.5f, hp.eu + 11);
        const int ezp = (p == 1) ? hp.eu : ((p - 1 <= m_split) ? hp.ez : kFullForm);
        if (a.sH)
            k_big_assemble_split<<<dim3(eb, items), 256, 0, st>>>(a.prm, a.bsys, a.sH, a.j0, a.wlen, X, Za, a.mstride,
                                                                  hp.ex, ezp);
        else
            k_big_assemble<float4><<<dim3(eb, items), 256, 0, st>>>(a.prm, a.bsys, a.j0, a.wlen, X, Za, a.mstride,
                                                                    hp.ex, ezp);
        count();
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        float4 *zin = Za, *zout = Zb;
        for (int i = p - 1; i >= 1; --i) {
            if ((err = store(zin, p - 1 - i)) != cudaSuccess) return err;
            err = (i > m_split) ? mm_launch<float4, 2>(d, items, X, zin, zout, a.mstride, 0, i, st,
                                                       i == m_split + 1 ? mz : 0.f)
                                : mm_launch<float4, 1>(d, items, X, zin, zout, a.mstride, 0, i, st, i >= 2 ? mz : mu);
            count();
            if (err != cudaSuccess) return err;
            std::swap(zin, zout);
        }
        for (int m = 0; m < n; ++m) {
            if ((err = store(zin, p - 1 + m)) != cudaSuccess) return err;
            if ((err = mm_launch<float4, 1>(d, items, zin, zin, zout, a.mstride, 1, 0, st, mu)) != cudaSuccess) return err;
            count();
            std::swap(zin, zout);
        }
        k_big_store_u<float4, float2><<<dim3(eb, items), 256, 0, st>>>(d, zin, a.mstride,
                                                                         reinterpret_cast<float2*>(a.Ubuf), a.ustride,
                                                                         a.wlen, a.wmax);
        count();
        return cudaGetLastError();
    }
    using C = C_t<R>;
    C* X = reinterpret_cast<C*>(a.scratch);
    C* Za = X + (size_t)items * a.mstride;
    C* Zb = Za + (size_t)items * a.mstride;
    k_big_assemble<C><<<dim3(eb, items), 256, 0, st>>>(a.prm, a.bsys, a.j0, a.wlen, X, Za, a.mstride, 0, 0);
    count();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    C *zin = Za, *zout = Zb;
    for (int i = p - 1; i >= 1; --i) {
        if ((err = store(zin, p - 1 - i)) != cudaSuccess) return err;
        if ((err = mm_launch<C, 0>(d, items, X, zin, zout, a.mstride, 0, i, st)) != cudaSuccess) return err;
        count();
        std::swap(zin, zout);
    }
    for (int m = 0; m < n; ++m) {
        if ((err = store(zin, p - 1 + m)) != cudaSuccess) return err;
        if ((err = mm_launch<C, 0>(d, items, zin, zin, zout, a.mstride, 1, 0, st)) != cudaSuccess) return err;
        count();
        std::swap(zin, zout);
    }
    k_big_store_u<C, C><<<dim3(eb, items), 256, 0, st>>>(d, zin, a.mstride, reinterpret_cast<C*>(a.Ubuf), a.ustride,
                                                          a.wlen, a.wmax);
    count();
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_big_adj(const BigArgs<R>& a, const SysView<R>& sys, const StateView<R>& sv, const C_t<R>* states,
                           const C_t<R>* Gbuf, double* gpart, int p, int n, cudaStream_t st, int* launches) {
    using C = C_t<R>;
    const int d = a.d, items = a.wlen * a.E;
    const size_t dd = (size_t)d * d, ms = a.mstride;
    const int eb = ew_blocks(dd);
    auto count = [&]() { if (launches) ++*launches; };
    C* XH = reinterpret_cast<C*>(a.scratch);
    C* Ub = XH + (size_t)items * ms;
    C* Z11a = Ub + (size_t)items * ms;
    C* Z12a = Z11a + (size_t)items * ms;
    C* Z11b = Z12a + (size_t)items * ms;
    C* Z12b = Z11b + (size_t)items * ms;
    k_big_adj_init<R><<<dim3(eb, items), 256, 0, st>>>(a.prm, sys, a.j0, a.wlen, XH, Z11a, ms);
    count();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    // Ubar = G Psi^dag as a tiled product (factors staged in Z11b / Z12b, free until the first step)
    k_big_ubar_factors<C><<<dim3(eb, items), 256, 0, st>>>(d, sv, a.wlen, states, Gbuf, a.wmax, Z11b, Z12b, ms);
    count();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = mm_launch<C, 0>(d, items, Z11b, Z12b, Ub, ms, 1, 0, st)) != cudaSuccess) return err;
    count();
    k_big_scale_p<C><<<dim3(eb, items), 256, 0, st>>>(a.prm, d, Ub, Z12a, ms);
    count();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const int T = (sizeof(C) == 16) ? 32 : big_tile(d);   // 16-byte elements: 32 x 32 tiles (SMEM, registers)
    C *z11 = Z11a, *z12 = Z12a, *o11 = Z11b, *o12 = Z12b;
    auto blk = [&](const C* A11, const C* A12, const C* B11, const C* B12, int kind, int i) {
        cudaError_t e2;
        if (T == 32) e2 = blk_launch_t<C, 32>(d, items, A11, A12, B11, B12, o11, o12, ms, kind, i, st);
        else e2 = blk_launch_t<C, 64>(d, items, A11, A12, B11, B12, o11, o12, ms, kind, i, st);
        count();
        std::swap(z11, o11);
        std::swap(z12, o12);
        return e2;
    };
    for (int i = p - 1; i >= 1; --i)
        if ((err = blk(XH, Ub, z11, z12, 0, i)) != cudaSuccess) return err;
    for (int m = 0; m < n; ++m)
        if ((err = blk(z11, z12, z11, z12, 1, 0)) != cudaSuccess) return err;
    if (sys.M > 0) {
        k_big_grad<R><<<dim3(items, sys.M), 256, 0, st>>>(a.prm, sys, a.j0, a.wlen, z12, ms, gpart);
        count();
    }
    return cudaGetLastError();
}

template <typename C, int T>
static cudaError_t rev_launch_t(int d, int items, const RevOps<C>& ops, C* O1, C* O2, size_t ms, int mode, int i,
                                cudaStream_t st) {
    constexpr size_t smem = blk_smem<C, T>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_big_rev<C, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nt = ((d + T - 1) / T) * ((d + T - 1) / T);
    k_big_rev<C, T><<<dim3(nt, items), 256, smem, st>>>(d, ops, O1, O2, ms, mode, i);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_big_adj_rev(const BigArgs<R>& a, const SysView<R>& sys, const StateView<R>& sv, const C_t<R>* states,
                               const C_t<R>* Gbuf, double* gpart, int p, int n, const C_t<R>* zst, cudaStream_t st,
                               int* launches, const OzRev* oz) {
    using C = C_t<R>;
    const int d = a.d, items = a.wlen * a.E, cap = p - 1 + n;
    const size_t dd = (size_t)d * d, ms = a.mstride, zs = (size_t)cap * ms;
    const int eb = ew_blocks(dd);
    auto count = [&]() { if (launches) ++*launches; };
    C* XH = reinterpret_cast<C*>(a.scratch);
    C* Za = XH + (size_t)items * ms;
    C* Zb = Za + (size_t)items * ms;
    C* Xb = Zb + (size_t)items * ms;
    // XH; Ubar = G Psi^dag into Za by a tiled product (factors staged in Zb / Xb)
    k_big_adj_init<R><<<dim3(eb, items), 256, 0, st>>>(a.prm, sys, a.j0, a.wlen, XH, static_cast<C*>(nullptr), ms);
    count();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_big_ubar_factors<C><<<dim3(eb, items), 256, 0, st>>>(d, sv, a.wlen, states, Gbuf, a.wmax, Zb, Xb, ms);
    count();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = mm_launch<C, 0>(d, items, Zb, Xb, Za, ms, 1, 0, st)) != cudaSuccess) return err;
    count();
    if ((err = cudaMemsetAsync(Xb, 0, (size_t)items * ms * sizeof(C), st)) != cudaSuccess) return err;
    const int T = (sizeof(C) == 16) ? 32 : big_tile(d);
    C *zb = Za, *zo = Zb;
    // tensor-core products (BF16_SPLIT): X^dag is sliced once for the wave
    int xh_sliced = 0;
    OzRev tc{};
    if (oz) {
        tc = *oz;
        tc.xh = reinterpret_cast<const float2*>(XH);
        tc.xh_sliced = &xh_sliced;
    }
    auto rev = [&](const RevOps<C>& ops, C* O2, int mode, int i) {
        cudaError_t e2;
        if constexpr (sizeof(C) == 8) {
            if (oz) {
                const float2* o4[4] = {ops.p[0], ops.p[1], ops.p[2], ops.p[3]};
                e2 = oz_rev_step(tc, o4, ops.s, zo, O2, ms, mode, i, st, launches);
                std::swap(zb, zo);
                return e2;
            }
        }
        e2 = (T == 32) ? rev_launch_t<C, 32>(d, items, ops, zo, O2, ms, mode, i, st)
                       : rev_launch_t<C, 64>(d, items, ops, zo, O2, ms, mode, i, st);
        count();
        std::swap(zb, zo);
        return e2;
    };
    for (int m = n - 1; m >= 0; --m) {          // Sbar_m = Sbar_{m+1} S_m^dag + S_m^dag Sbar_{m+1}
        const C* S = zst + (size_t)(p - 1 + m) * ms;
        if ((err = rev(RevOps<C>{{zb, S, S, zb}, {ms, zs, zs, ms}}, nullptr, 1, 0)) != cudaSuccess) return err;
    }
    for (int i = 1; i <= p - 1; ++i) {          // Zbar_{i+1} = X^dag Zbar_i / i, Xbar += Zbar_i Z_{i+1}^dag / i
        const C* S = zst + (size_t)(p - 1 - i) * ms;
        if ((err = rev(RevOps<C>{{XH, zb, zb, S}, {ms, ms, ms, zs}}, Xb, 0, i)) != cudaSuccess) return err;
    }
    k_big_axpy<C><<<dim3(eb, items), 256, 0, st>>>(d, zb, Xb, ms, p);
    count();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (sys.M > 0) {
        k_big_grad<R><<<dim3(items, sys.M), 256, 0, st>>>(a.prm, sys, a.j0, a.wlen, Xb, ms, gpart);
        count();
    }
    return cudaGetLastError();
}

// Reverse mode of the Paterson-Stockmeyer form over its stored operands (the per-slice
// k_expm_adj_ps as batched products; FP32 forms): the squarings in reverse, per chain product
// Wbar_{q+1} = Y^dag Wbar_q with Ybar += Wbar_q W_{q+1}^dag in the same launch, the block
// cotangents Xbar += c_3q+1 Wbar_q, X2bar += c_3q+2 Wbar_q element-wise, then the power products
// X2bar += Ybar X^dag with Xbar += X2^dag Ybar, and Xbar += X2bar X^dag + X^dag X2bar.
// Scratch per item: X^dag, the cotangent ping-pong, Xbar, X2bar, Ybar (six float2 matrices).
template <typename R>
cudaError_t launch_big_adj_rev_ps(const BigArgs<R>& a, const SysView<R>& sys, const StateView<R>& sv,
                                  const C_t<R>* states, const C_t<R>* Gbuf, double* gpart, const DevParams& hp,
                                  const C_t<R>* zst, cudaStream_t st, int* launches, const OzRev* oz) {
    if constexpr (sizeof(R) != 4) {
        return cudaErrorInvalidValue;
    } else {
        using C = float2;
        const int p = hp.p, n = hp.n, d = a.d, items = a.wlen * a.E, cap = ps_big_slots(p, n), qt = ps_top(p);
        const size_t dd = (size_t)d * d, ms = a.mstride, zs = (size_t)cap * ms;
        const int eb = ew_blocks(dd);
        auto count = [&]() { if (launches) ++*launches; };
        // X^dag of every item: the forward stored it (the last slot, item stride zs)
        const C* XH = zst + (size_t)(cap - 1) * ms;
        C* Za = reinterpret_cast<C*>(a.scratch) + (size_t)items * ms;
        C* Zb = Za + (size_t)items * ms;
        C* Xb = Zb + (size_t)items * ms;
        C* X2b = Xb + (size_t)items * ms;
        C* Yb = X2b + (size_t)items * ms;
        cudaError_t err;
        k_big_ubar_factors<C><<<dim3(eb, items), 256, 0, st>>>(d, sv, a.wlen, states, Gbuf, a.wmax, Zb, Xb, ms);
        count();
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if ((err = mm_launch<C, 0>(d, items, Zb, Xb, Za, ms, 1, 0, st)) != cudaSuccess) return err;
        count();
        if ((err = cudaMemsetAsync(Xb, 0, 3 * (size_t)items * ms * sizeof(C), st)) != cudaSuccess) return err;
        const int T = big_tile(d);
        C *zb = Za, *zo = Zb;
        int xh_sliced = 0;
        OzRev tc{};
        if (oz) {   // the chain's A1 operand, Y^dag (slot 1), is sliced once for the wave
            tc = *oz;
            tc.xh = zst + (size_t)1 * ms;
            tc.xh_sliced = &xh_sliced;
        }
        auto rev = [&](const RevOps<C>& ops, C* O2, int mode) {
            cudaError_t e2;
            if (oz) {
                const float2* o4[4] = {ops.p[0], ops.p[1], ops.p[2], ops.p[3]};
                e2 = oz_rev_step(tc, o4, ops.s, zo, O2, ms, mode, 1, st, launches);
            } else {
                e2 = (T == 32) ? rev_launch_t<C, 32>(d, items, ops, zo, O2, ms, mode, 1, st)
                               : rev_launch_t<C, 64>(d, items, ops, zo, O2, ms, mode, 1, st);
                count();
            }
            std::swap(zb, zo);
            return e2;
        };
        auto acc = [&](const C* Z, float ca, float cb, float cc) {
            k_big_ps_acc<<<dim3(eb, items), 256, 0, st>>>(d, Z, Xb, X2b, Yb, ms, ca, cb, cc);
            count();
            return cudaGetLastError();
        };
        auto slot = [&](int r) { return zst + (size_t)r * ms; };   // item stride zs
        for (int m = n - 1; m >= 0; --m) {      // Sbar_m = Sbar_{m+1} S_m^dag + S_m^dag Sbar_{m+1}
            const C* S = slot(qt + 2 + m);
            if ((err = rev(RevOps<C>{{zb, S, S, zb}, {ms, zs, zs, ms}}, nullptr, 1)) != cudaSuccess) return err;
        }
        for (int q = 0; q < qt; ++q) {          // chain products in reverse
            if ((err = acc(zb, hp.ch[3 * q + 1], hp.ch[3 * q + 2], 0.f)) != cudaSuccess) return err;
            const C* Wn = slot(2 + (qt - 1 - q));
            if ((err = rev(RevOps<C>{{slot(1), zb, zb, Wn}, {zs, ms, ms, zs}}, Yb, 0)) != cudaSuccess) return err;
        }
        if ((err = acc(zb, hp.ch[3 * qt + 1], hp.ch[3 * qt + 2], hp.ch[3 * qt + 3])) != cudaSuccess) return err;
        if (p >= 3) {   // X2bar += Ybar X^dag, Xbar += X2^dag Ybar
            if ((err = rev(RevOps<C>{{Yb, XH, slot(0), Yb}, {ms, zs, zs, ms}}, Xb, 0)) != cudaSuccess) return err;
            if ((err = acc(zb, 0.f, 1.f, 0.f)) != cudaSuccess) return err;
        }
        if (p >= 2) {   // Xbar += X2bar X^dag + X^dag X2bar
            if ((err = rev(RevOps<C>{{X2b, XH, XH, X2b}, {ms, zs, zs, ms}}, nullptr, 1)) != cudaSuccess) return err;
            if ((err = acc(zb, 1.f, 0.f, 0.f)) != cudaSuccess) return err;
        }
        if (sys.M > 0) {
            k_big_grad<R><<<dim3(items, sys.M), 256, 0, st>>>(a.prm, sys, a.j0, a.wlen, Xb, ms, gpart);
            count();
        }
        return cudaGetLastError();
    }
}

template cudaError_t launch_big_expm<float>(const BigArgs<float>&, const DevParams&, bool, cudaStream_t, int*, float2*,
                                            const OzFwd*);
template cudaError_t launch_big_expm<double>(const BigArgs<double>&, const DevParams&, bool, cudaStream_t, int*, double2*,
                                             const OzFwd*);
template cudaError_t launch_big_adj_rev<float>(const BigArgs<float>&, const SysView<float>&, const StateView<float>&,
                                               const float2*, const float2*, double*, int, int, const float2*,
                                               cudaStream_t, int*, const OzRev*);
template cudaError_t launch_big_adj_rev<double>(const BigArgs<double>&, const SysView<double>&,
                                                const StateView<double>&, const double2*, const double2*, double*, int,
                                                int, const double2*, cudaStream_t, int*, const OzRev*);
template cudaError_t launch_big_adj<float>(const BigArgs<float>&, const SysView<float>&, const StateView<float>&,
                                           const float2*, const float2*, double*, int, int, cudaStream_t, int*);
template cudaError_t launch_big_adj<double>(const BigArgs<double>&, const SysView<double>&, const StateView<double>&,
                                            const double2*, const double2*, double*, int, int, cudaStream_t, int*);

template cudaError_t launch_big_adj_rev_ps<float>(const BigArgs<float>&, const SysView<float>&,
                                                  const StateView<float>&, const float2*, const float2*, double*,
                                                  const DevParams&, const float2*, cudaStream_t, int*, const OzRev*);

}  // namespace qoc
