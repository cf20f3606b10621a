// Slice exponential in split FP32 arithmetic for the FP32 form.
//
// Over long evolutions the FP32 rounding of H_j dt and of the Taylor / squaring products is
// nearly the same at every slice (the drift H_0 does not change), so it accumulates coherently
// along the N-slice chain.  The FP32 form therefore evaluates U_j = [T_p(X_j)]^(2^n) (Eqs. 9,
// 10) with every matrix held as an unevaluated sum of two FP32 numbers:
//   * X_j = -i s H_j is assembled in FP32 pair arithmetic from s H_0, s H_k, s H_det held as
//     FP32 pairs (written once per evaluation by k_split_scale after the (p, n) pick), with
//     no FP64 arithmetic per slice,
//   * matrices are stored grid-split (qoc_device.cuh): v = v1 + v2, v1 on the power-of-two grid
//     2^(e - 12) set by a norm bound of the matrix, so that the sums of the grid-part products
//     are exact FP32 FMAs and only the cross terms a1 b2 + a2 b are rounded (about 2^-36 of
//     the product's scale), 12 FMAs per complex multiply-add,
//   * the Horner division by i and the identity shift are done in pair (double-float)
//     arithmetic on the error-free sum of the two accumulators,
//   * Horner steps i > m_split use plain FP32: an error made there reaches T scaled by
//     ts^m / m! < 2^-6 (m_split is picked with (p, n) from the FP64 norm bound).
// Only the rounded U_j is kept for the propagation (costates and the adjoint stay FP32), plus,
// for the reverse-mode adjoint, the rounded right operand of every product (ZStore).
// The same kernel is used for the recomputation in the backward sweep, so the forward and
// backward propagators are bitwise identical.
#include "qoc_device.cuh"
#include "qoc_internal.h"

namespace qoc {

__device__ __forceinline__ void df_norm(float& hi, float& lo) {   // Fast2Sum(hi, lo)
    const float s = hi + lo;
    lo = lo - (s - hi);
    hi = s;
}

// (hi, lo) / i for a positive integer i
__device__ __forceinline__ void df_div(float& hi, float& lo, float fi) {
    const float q = hi / fi;
    const float r = fmaf(-q, fi, hi);
    const float ql = (r + lo) / fi;
    hi = q;
    lo = ql;
    df_norm(hi, lo);
}

// (hi, lo) + 1
__device__ __forceinline__ void df_add1(float& hi, float& lo) {
    const float t = hi + 1.0f;
    const float bv = t - hi;
    const float err = (hi - (t - bv)) + (1.0f - bv);
    hi = t;
    lo += err;
    df_norm(hi, lo);
}

// plain FP32 product for the early Horner steps: A grid-split (X), B in full form (.x, .y)
template <int MT>
__device__ __forceinline__ void mm_hi(float2 (&acc)[MT][MT], const float4* __restrict__ A, const float4* __restrict__ B,
                                      int kd, int LD, int ty, int tx, int G) {
    const float4* pa[MT];
    const float4* pb[MT];
#pragma unroll
    for (int i = 0; i < MT; ++i) {
        pa[i] = A + (ty + G * i) * LD;
        pb[i] = B + tx + G * i;
    }
#pragma unroll 2
    for (int k = 0; k < kd; ++k) {
        float2 a[MT], b[MT];
#pragma unroll
        for (int i = 0; i < MT; ++i) {
            const float4 v = pa[i][k];
            a[i] = make_float2(v.x + v.z, v.y + v.w);
        }
#pragma unroll
        for (int i = 0; i < MT; ++i) {
            const float4 v = *pb[i];
            pb[i] += LD;
            b[i] = make_float2(v.x, v.y);
        }
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
            for (int j = 0; j < MT; ++j) cfma(acc[i][j], a[i], b[j]);
    }
}

// X_ab = -i s H_ab (element o = a d + b) in pair arithmetic from the pairs s H_0, s H_k (times the
// control pairs us[k]) and s H_det (times us[M]; Hd = nullptr: no ensemble term)
__device__ __forceinline__ void x_pair(const float4* __restrict__ H0, const float4* __restrict__ Hk,
                                       const float4* __restrict__ Hd, size_t dd, int M, const float2* us, int o,
                                       float& xrh, float& xrl, float& xih, float& xil) {
    const float4 h0 = H0[o];
    float rh = h0.x, rl = h0.z, ih = h0.y, il = h0.w;
    for (int k = 0; k < M; ++k) {
        const float4 hk = Hk[k * dd + o];
        pair_fma(rh, rl, us[k], hk.x, hk.z);
        pair_fma(ih, il, us[k], hk.y, hk.w);
    }
    if (Hd) {
        const float4 hd = Hd[o];
        pair_fma(rh, rl, us[M], hd.x, hd.z);
        pair_fma(ih, il, us[M], hd.y, hd.w);
    }
    df_norm(rh, rl);
    df_norm(ih, il);
    // X = -i (s H): re X = im(s H), im X = -re(s H)
    xrh = ih;
    xrl = il;
    xih = -rh;
    xil = -rl;
}

// s H_0, s H_1 .. s H_M, s H_det (s = dt / 2^n) as FP32 pairs (re_hi, im_hi, re_lo, im_lo), once
// per evaluation: the slice assembly above then needs no FP64 arithmetic
__global__ void k_split_scale(const DevParams* __restrict__ prm, const double2* __restrict__ H64, size_t count,
                              float4* __restrict__ sH) {
    const double s = prm->s;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const double2 h = H64[i];
        const double xr = s * h.x, xi = s * h.y;
        const float rh = (float)xr, ih = (float)xi;
        sH[i] = make_float4(rh, ih, (float)(xr - (double)rh), (float)(xi - (double)ih));
    }
}

cudaError_t launch_split_scale(const DevParams* prm, const double2* H64, size_t count, float4* sH, cudaStream_t st) {
    const size_t b = (count + 255) / 256;
    k_split_scale<<<(int)(b < 1024 ? b : 1024), 256, 0, st>>>(prm, H64, count, sH);
    return cudaGetLastError();
}

// out = [diag I] + (grid sums + cross terms) / div  (div = 0: no division), grid-split with
// the given magic constant; zero in the padding
template <int MT>
__device__ __forceinline__ void sl_store(float4* __restrict__ out, float (&acc)[MT][MT][4], int div,
                                         bool add_identity, float magic, int d, int LD, int ty, int tx, int G) {
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j) {
            const int r = ty + G * i, c = tx + G * j;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < d && c < d) {
                float rh, rl, ih, il;
                two_sum(acc[i][j][0], acc[i][j][2], rh, rl);
                two_sum(acc[i][j][1], acc[i][j][3], ih, il);
                if (div > 1) {
                    df_div(rh, rl, (float)div);
                    df_div(ih, il, (float)div);
                }
                if (add_identity && r == c) df_add1(rh, rl);
                grid_split(rh, rl, magic, v.x, v.z);
                grid_split(ih, il, magic, v.y, v.w);
            }
            out[r * LD + c] = v;
        }
}

template <int MT>
__global__ void __launch_bounds__(512)
k_expm_fwd_split(const DevParams* __restrict__ prm, SysView<float> sys, const float4* __restrict__ sH, int j0,
                 float2* __restrict__ Ubuf, long long ustride, int wmax, ZStore<float> zs, int G) {
    const int D = G * MT, LD = D + 1, SZ = D * LD;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ float2 us[kMaxControls + 1];   // u_kj and delta_e as (hi, lo) pairs
    float4* X = reinterpret_cast<float4*>(smraw);
    float4* Za = X + SZ;
    float4* Zb = Za + SZ;
    const int jl = blockIdx.x, e = blockIdx.y, j = j0 + jl;
    const int tid = threadIdx.x, tx = tid % G, ty = tid / G;
    const bool act = tid < G * G;   // the block is rounded up to whole warps
    const int d = sys.d, M = sys.M, p = prm->p, n = prm->n;
    for (int k = tid; k <= M; k += blockDim.x) {
        const double v = (k < M) ? sys.u[(size_t)k * sys.N + j] : (sys.delta ? sys.delta[e] : 0.0);
        const float h = (float)v;
        us[k] = make_float2(h, (float)(v - (double)h));
    }
    __syncthreads();
    const size_t dd = (size_t)d * d;
    const float4* H0 = sH;
    const float4* Hk = sH + dd;
    const float4* Hd = sH + (size_t)(M + 1) * dd;
    // Grid exponents and the form each Z is kept in: the operand of a split product is
    // grid-split (X with ex; Z_i, i >= 2, with ez; T = Z_1 and its squarings with eu), the
    // operand of a plain Horner step is the full FP32 value in (.x, .y) with zero (.z, .w).
    const int m_split = prm->m_split;
    const int ex = prm->ex, ez = prm->ez, eu = prm->eu;
    const float mz = grid_magic(ez), mu = grid_magic(eu);
    // X = -i s H_j in pair arithmetic from the pairs s H_0, s H_k, s H_det, grid-split;
    // Z_p = I + X / p in the form step p - 1 reads
    const int ezp = (p == 1) ? eu : ((p - 1 <= m_split) ? ez : 1000);   // 1000: full form
    const float mx = grid_magic(ex), mzp = grid_magic(ezp == 1000 ? 0 : ezp);
    for (int idx = tid; idx < D * D; idx += blockDim.x) {
        const int a = idx / D, b = idx - a * D;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f), z = x;
        if (a < d && b < d) {
            float xrh, xrl, xih, xil;
            x_pair(H0, Hk, sys.Hdet ? Hd : nullptr, dd, M, us, a * d + b, xrh, xrl, xih, xil);
            grid_split(xrh, xrl, mx, x.x, x.z);
            grid_split(xih, xil, mx, x.y, x.w);
            if (p > 1) {
                df_div(xrh, xrl, (float)p);
                df_div(xih, xil, (float)p);
            }
            if (a == b) df_add1(xrh, xrl);
            if (ezp == 1000) {
                z.x = xrh + xrl;
                z.y = xih + xil;
            } else {
                grid_split(xrh, xrl, mzp, z.x, z.z);
                grid_split(xih, xil, mzp, z.y, z.w);
            }
        }
        X[a * LD + b] = x;
        Za[a * LD + b] = z;
    }
    __syncthreads();
    float4* zin = Za;
    float4* zout = Zb;
    float2* zst = (zs.Z && p - 1 + n <= zs.cap) ? zs.Z + ((size_t)e * zs.wmax + jl) * zs.cap * zs.mstride : nullptr;
    // the right operand of product r, rounded to FP32 and conjugate-transposed, for the adjoint
    auto store = [&](int r) {
        float2* dst = zst + (size_t)r * zs.mstride;
        for_rc(d, d, [&](int idx, int a, int b) {
            const float4 v = zin[b * LD + a];
            dst[idx] = make_float2(v.x + v.z, -(v.y + v.w));
        });
    };
    for (int i = p - 1; i >= 1; --i) {        // Horner: Z <- I + X Z / i
        if (zst) store(p - 1 - i);
        if (!act) {
        } else if (i > m_split) {
            float2 acc[MT][MT];
#pragma unroll
            for (int a = 0; a < MT; ++a)
#pragma unroll
                for (int b = 0; b < MT; ++b) acc[a][b] = make_float2(0.f, 0.f);
            mm_hi<MT>(acc, X, zin, d, LD, ty, tx, G);
            const float ri = 1.0f / (float)i;
#pragma unroll
            for (int a = 0; a < MT; ++a)
#pragma unroll
                for (int b = 0; b < MT; ++b) {
                    const int r = ty + G * a, c = tx + G * b;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (r < d && c < d) {
                        v.x = fmaf(acc[a][b].x, ri, (r == c) ? 1.0f : 0.0f);
                        v.y = acc[a][b].y * ri;
                        if (i == m_split + 1) {   // read by the first split step: grid-split
                            grid_split(v.x, 0.f, mz, v.x, v.z);
                            grid_split(v.y, 0.f, mz, v.y, v.w);
                        }
                    }
                    zout[r * LD + c] = v;
                }
        } else {
            float acc[MT][MT][4] = {};
            mm_sl<MT>(acc, X, zin, d, LD, ty, tx, G);
            sl_store<MT>(zout, acc, i, true, i >= 2 ? mz : mu, d, LD, ty, tx, G);
        }
        __syncthreads();
        float4* t = zin; zin = zout; zout = t;
    }
    for (int m = 0; m < n; ++m) {             // squaring: Z <- Z Z
        if (zst) store(p - 1 + m);
        if (act) {
            float acc[MT][MT][4] = {};
            mm_sl<MT>(acc, zin, zin, d, LD, ty, tx, G);
            sl_store<MT>(zout, acc, 0, false, mu, d, LD, ty, tx, G);
        }
        __syncthreads();
        float4* t = zin; zin = zout; zout = t;
    }
    // U_j at offset 0, U_j^dag at offset ustride / 2; the pair is rounded to FP32
    float2* U = Ubuf + ((size_t)e * wmax + jl) * ustride;
    float2* UH = U + ustride / 2;
    for (int idx = tid; idx < d * d; idx += blockDim.x) {
        const int a = idx / d, b = idx - a * d;
        const float4 z = zin[a * LD + b];
        U[idx] = make_float2(z.x + z.z, z.y + z.w);
        const float4 h = zin[b * LD + a];
        UH[idx] = make_float2(h.x + h.z, -(h.y + h.w));
    }
}

static size_t split_smem(int d) {
    const int D = slice_tile(d).D;
    return (size_t)3 * D * (D + 1) * sizeof(float4);
}

template <int MT>
static cudaError_t launch_split_mt(const DevParams* prm, const SysView<float>& sys, const float4* sH, int j0,
                                   int wlen, int E, float2* Ubuf, long long ustride, int wmax, const ZStore<float>& zs,
                                   int G, cudaStream_t st) {
    const size_t smem = split_smem(sys.d);
    cudaError_t err = cudaFuncSetAttribute(k_expm_fwd_split<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_expm_fwd_split<MT><<<dim3(wlen, E), slice_threads(G), smem, st>>>(prm, sys, sH, j0, Ubuf, ustride, wmax, zs, G);
    return cudaGetLastError();
}

int split_ctas_per_sm(int d) {
    const SliceTile tl = slice_tile(d);
    if (tl.MT <= 0) return 1;
    const size_t smem = split_smem(d);
    const int thr = slice_threads(tl.G);
    int n = 0;
    cudaError_t e;
    switch (tl.MT) {
        case 1: cudaFuncSetAttribute(k_expm_fwd_split<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd_split<1>, thr, smem); break;
        case 2: cudaFuncSetAttribute(k_expm_fwd_split<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd_split<2>, thr, smem); break;
        case 3: cudaFuncSetAttribute(k_expm_fwd_split<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd_split<3>, thr, smem); break;
        default: cudaFuncSetAttribute(k_expm_fwd_split<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd_split<4>, thr, smem); break;
    }
    return (e == cudaSuccess && n > 0) ? n : 1;
}

int split_max_d() {
    for (int d = kMaxD; d >= 1; --d)
        if (slice_tile(d).MT > 0 && split_smem(d) <= kMaxDynSmem) return d;
    return 0;
}

cudaError_t launch_expm_fwd_split(const DevParams* prm, const SysView<float>& sys, const float4* sH, int j0, int wlen,
                                  int E, float2* Ubuf, long long ustride, int wmax, const ZStore<float>& zs,
                                  cudaStream_t st) {
    const SliceTile tl = slice_tile(sys.d);
    if (sys.d > split_max_d()) return cudaErrorInvalidValue;
    switch (tl.MT) {
        case 1: return launch_split_mt<1>(prm, sys, sH, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 2: return launch_split_mt<2>(prm, sys, sH, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 3: return launch_split_mt<3>(prm, sys, sH, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 4: return launch_split_mt<4>(prm, sys, sH, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        default: return cudaErrorInvalidValue;
    }
}


// ------------------------------------------------------------------------------------------
// Paterson-Stockmeyer form (block size 3) of the same split exponential.  The order-p Taylor
// polynomial of Eq. 10 is regrouped as T = sum_q Y^q B_q with Y = X^3 and
// B_q = c_3q I + c_3q+1 X + c_3q+2 X^2 (c_k = 1/k!, zero for k > p), and evaluated from the top
// block down, W_q = B_q + Y W_{q+1}: two products for X^2 and X^3 and about p / 3 chain products
// instead of p - 1 Horner steps.  The series and its truncation are unchanged; only the order of
// the products differs, so a larger theta_max (fewer squarings) pays.
// Precision follows the Horner form's rule: a rounding error in W_q reaches T multiplied by at
// most ts^3q / (3q)! (the same factor as an error in Horner's Z_{3q+1}), so chain products with
// 3q + 1 <= m_split are split products and the others plain FP32.  X^2, X^3, T and the squarings
// are always split; the B_q terms are added in pair arithmetic with the coefficients as FP32
// pairs.  Every operand is grid-split on its own norm bound (e2, e3, ew[q] from the order pick).
// Shared memory holds X, X^2, X^3 and W (written in place after a second barrier): four split
// matrices, so d <= ps_max_d().
// ------------------------------------------------------------------------------------------

// a value given as pairs (re, im) in the form its reader takes: grid-split on magic, or the full
// FP32 value in (.x, .y) with zero (.z, .w) when magic == 0 (the operand of a plain product)
__device__ __forceinline__ float4 ps_form(float rh, float rl, float ih, float il, float magic) {
    float4 v;
    if (magic == 0.f) {
        v = make_float4(rh + rl, ih + il, 0.f, 0.f);
    } else {
        grid_split(rh, rl, magic, v.x, v.z);
        grid_split(ih, il, magic, v.y, v.w);
    }
    return v;
}

// (rh, rl, ih, il) += c_k0+1 X + c_k0+2 X^2 (+ c_k0 on the diagonal); x2 is read only when
// p >= 2 (have2)
__device__ __forceinline__ void ps_add_block(float& rh, float& rl, float& ih, float& il, const float2* cs, int k0,
                                             bool diag, float4 x, bool have2, float4 x2) {
    pair_fma(rh, rl, cs[k0 + 1], x.x, x.z);
    pair_fma(ih, il, cs[k0 + 1], x.y, x.w);
    if (have2) {
        pair_fma(rh, rl, cs[k0 + 2], x2.x, x2.z);
        pair_fma(ih, il, cs[k0 + 2], x2.y, x2.w);
    }
    if (diag) df_addc(rh, rl, cs[k0]);
}

template <int MT>
__global__ void __launch_bounds__(512)
k_expm_fwd_ps(const DevParams* __restrict__ prm, SysView<float> sys, const float4* __restrict__ sH, int j0,
              float2* __restrict__ Ubuf, long long ustride, int wmax, ZStore<float> zs, int G) {
    const int D = G * MT, LD = D + 1, SZ = D * LD;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ float2 us[kMaxControls + 1];   // u_kj and delta_e as (hi, lo) pairs
    __shared__ float2 cs[kPsCoefs];           // 1/k! as (hi, lo) pairs
    float4* X = reinterpret_cast<float4*>(smraw);
    float4* P2 = X + SZ;
    float4* P3 = P2 + SZ;
    float4* W = P3 + SZ;
    const int jl = blockIdx.x, e = blockIdx.y, j = j0 + jl;
    const int tid = threadIdx.x, tx = tid % G, ty = tid / G;
    const bool act = tid < G * G;   // the block is rounded up to whole warps
    const int d = sys.d, M = sys.M, p = prm->p, n = prm->n;
    for (int k = tid; k <= M; k += blockDim.x) {
        const double v = (k < M) ? sys.u[(size_t)k * sys.N + j] : (sys.delta ? sys.delta[e] : 0.0);
        const float h = (float)v;
        us[k] = make_float2(h, (float)(v - (double)h));
    }
    for (int k = tid; k < kPsCoefs; k += blockDim.x) cs[k] = make_float2(prm->ch[k], prm->cl[k]);
    __syncthreads();
    const size_t dd = (size_t)d * d;
    const int qt = ps_top(p), qs = (prm->m_split - 1) / 3;   // chain products q <= qs are split
    const float mx = grid_magic(prm->ex), m2 = grid_magic(prm->e2), m3 = grid_magic(prm->e3);
    const float mu = grid_magic(prm->eu);
    // the form W_q is written in: its reader is chain product q - 1 (split iff q - 1 <= qs), or the
    // squarings for W_0 = T
    auto magic_w = [&](int q) { return q == 0 ? mu : (q - 1 <= qs ? grid_magic(prm->ew[q]) : 0.f); };
    for (int idx = tid; idx < D * D; idx += blockDim.x) {   // X = -i s H_j, grid-split
        const int a = idx / D, b = idx - a * D;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a < d && b < d) {
            float xrh, xrl, xih, xil;
            x_pair(sH, sH + dd, sys.Hdet ? sH + (size_t)(M + 1) * dd : nullptr, dd, M, us, a * d + b, xrh, xrl, xih,
                   xil);
            grid_split(xrh, xrl, mx, x.x, x.z);
            grid_split(xih, xil, mx, x.y, x.w);
        }
        X[a * LD + b] = x;
    }
    __syncthreads();
    float2* zst = zs_fits(zs, p, n) ? zs.Z + ((size_t)e * zs.wmax + jl) * zs.cap * zs.mstride : nullptr;
    // the operand in a slot, rounded to FP32 and conjugate-transposed, for the adjoint
    auto store = [&](int slot, const float4* src) {
        float2* dst = zst + (size_t)slot * zs.mstride;
        for_rc(d, d, [&](int idx, int a, int b) {
            const float4 v = src[b * LD + a];
            dst[idx] = make_float2(v.x + v.z, -(v.y + v.w));
        });
    };
    if (p >= 2) {                               // X^2 = X X
        if (act) {
            float acc[MT][MT][4] = {};
            mm_sl<MT>(acc, X, X, d, LD, ty, tx, G);
            sl_store<MT>(P2, acc, 0, false, m2, d, LD, ty, tx, G);
        }
        __syncthreads();
    }
    if (p >= 3) {                               // X^3 = X^2 X
        if (act) {
            float acc[MT][MT][4] = {};
            mm_sl<MT>(acc, P2, X, d, LD, ty, tx, G);
            sl_store<MT>(P3, acc, 0, false, m3, d, LD, ty, tx, G);
        }
        __syncthreads();
    }
    {   // the top block W_qt = c_3qt I + c_3qt+1 X + c_3qt+2 X^2 + c_3qt+3 X^3, element-wise
        const float mt = magic_w(qt);
        for (int idx = tid; idx < D * D; idx += blockDim.x) {
            const int a = idx / D, b = idx - a * D;
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (a < d && b < d) {
                const int o = a * LD + b;
                float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
                ps_add_block(rh, rl, ih, il, cs, 3 * qt, a == b, X[o], p >= 2, p >= 2 ? P2[o] : w);
                if (p >= 3) {
                    const float4 y = P3[o];
                    pair_fma(rh, rl, cs[3 * qt + 3], y.x, y.z);
                    pair_fma(ih, il, cs[3 * qt + 3], y.y, y.w);
                }
                w = ps_form(rh, rl, ih, il, mt);
            }
            W[a * LD + b] = w;
        }
    }
    if (zst) {
        if (p >= 2) store(0, P2);
        if (p >= 3) store(1, P3);
    }
    __syncthreads();
    for (int q = qt - 1; q >= 0; --q) {         // W_q = B_q + X^3 W_{q+1}, in place
        if (zst) store(2 + (qt - 1 - q), W);
        float4 out[MT][MT];
        if (act) {
            const float mq = magic_w(q);
            if (q <= qs) {
                float acc[MT][MT][4] = {};
                mm_sl<MT>(acc, P3, W, d, LD, ty, tx, G);
#pragma unroll
                for (int a = 0; a < MT; ++a)
#pragma unroll
                    for (int b = 0; b < MT; ++b) {
                        const int r = ty + G * a, c = tx + G * b;
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (r < d && c < d) {
                            float rh, rl, ih, il;
                            two_sum(acc[a][b][0], acc[a][b][2], rh, rl);
                            two_sum(acc[a][b][1], acc[a][b][3], ih, il);
                            ps_add_block(rh, rl, ih, il, cs, 3 * q, r == c, X[r * LD + c], true, P2[r * LD + c]);
                            v = ps_form(rh, rl, ih, il, mq);
                        }
                        out[a][b] = v;
                    }
            } else {
                float2 acc[MT][MT];
#pragma unroll
                for (int a = 0; a < MT; ++a)
#pragma unroll
                    for (int b = 0; b < MT; ++b) acc[a][b] = make_float2(0.f, 0.f);
                mm_hi<MT>(acc, P3, W, d, LD, ty, tx, G);
                const float c0 = cs[3 * q].x, c1 = cs[3 * q + 1].x, c2 = cs[3 * q + 2].x;
#pragma unroll
                for (int a = 0; a < MT; ++a)
#pragma unroll
                    for (int b = 0; b < MT; ++b) {
                        const int r = ty + G * a, c = tx + G * b;
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (r < d && c < d) {
                            const float4 x = X[r * LD + c], y = P2[r * LD + c];
                            float re = fmaf(c1, x.x + x.z, acc[a][b].x);
                            float im = fmaf(c1, x.y + x.w, acc[a][b].y);
                            re = fmaf(c2, y.x + y.z, re);
                            im = fmaf(c2, y.y + y.w, im);
                            if (r == c) re += c0;
                            v = ps_form(re, 0.f, im, 0.f, mq);
                        }
                        out[a][b] = v;
                    }
            }
        }
        __syncthreads();   // every thread has read W
        if (act) {
#pragma unroll
            for (int a = 0; a < MT; ++a)
#pragma unroll
                for (int b = 0; b < MT; ++b) W[(ty + G * a) * LD + tx + G * b] = out[a][b];
        }
        __syncthreads();
    }
    float4* zin = W;                            // squarings, ping-pong with the X^2 buffer
    float4* zout = P2;
    for (int m = 0; m < n; ++m) {
        if (zst) store(qt + 2 + m, zin);
        if (act) {
            float acc[MT][MT][4] = {};
            mm_sl<MT>(acc, zin, zin, d, LD, ty, tx, G);
            sl_store<MT>(zout, acc, 0, false, mu, d, LD, ty, tx, G);
        }
        __syncthreads();
        float4* t = zin; zin = zout; zout = t;
    }
    // U_j at offset 0, U_j^dag at offset ustride / 2; the pair is rounded to FP32
    float2* U = Ubuf + ((size_t)e * wmax + jl) * ustride;
    float2* UH = U + ustride / 2;
    for (int idx = tid; idx < d * d; idx += blockDim.x) {
        const int a = idx / d, b = idx - a * d;
        const float4 z = zin[a * LD + b];
        U[idx] = make_float2(z.x + z.z, z.y + z.w);
        const float4 h = zin[b * LD + a];
        UH[idx] = make_float2(h.x + h.z, -(h.y + h.w));
    }
}

static size_t ps_smem(int d) {
    const int D = slice_tile(d).D;
    return (size_t)4 * D * (D + 1) * sizeof(float4);
}

int ps_max_d() {
    for (int d = kMaxD; d >= 1; --d)
        if (slice_tile(d).MT > 0 && ps_smem(d) <= kMaxDynSmem) return d;
    return 0;
}

template <int MT>
static cudaError_t launch_ps_mt(const DevParams* prm, const SysView<float>& sys, const float4* sH, int j0, int wlen,
                                int E, float2* Ubuf, long long ustride, int wmax, const ZStore<float>& zs, int G,
                                cudaStream_t st) {
    const size_t smem = ps_smem(sys.d);
    cudaError_t err = cudaFuncSetAttribute(k_expm_fwd_ps<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_expm_fwd_ps<MT><<<dim3(wlen, E), slice_threads(G), smem, st>>>(prm, sys, sH, j0, Ubuf, ustride, wmax, zs, G);
    return cudaGetLastError();
}

cudaError_t launch_expm_fwd_ps(const DevParams* prm, const SysView<float>& sys, const float4* sH, int j0, int wlen,
                               int E, float2* Ubuf, long long ustride, int wmax, const ZStore<float>& zs,
                               cudaStream_t st) {
    const SliceTile tl = slice_tile(sys.d);
    if (sys.d > ps_max_d() || !zs.ps) return cudaErrorInvalidValue;
    switch (tl.MT) {
        case 1: return launch_ps_mt<1>(prm, sys, sH, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 2: return launch_ps_mt<2>(prm, sys, sH, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 3: return launch_ps_mt<3>(prm, sys, sH, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 4: return launch_ps_mt<4>(prm, sys, sH, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        default: return cudaErrorInvalidValue;
    }
}

int ps_fwd_ctas_per_sm(int d) {
    const SliceTile tl = slice_tile(d);
    if (tl.MT <= 0 || d > ps_max_d()) return 1;
    const size_t smem = ps_smem(d);
    const int thr = slice_threads(tl.G);
    int n = 0;
    cudaError_t e;
    switch (tl.MT) {
        case 1: cudaFuncSetAttribute(k_expm_fwd_ps<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd_ps<1>, thr, smem); break;
        case 2: cudaFuncSetAttribute(k_expm_fwd_ps<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd_ps<2>, thr, smem); break;
        case 3: cudaFuncSetAttribute(k_expm_fwd_ps<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd_ps<3>, thr, smem); break;
        default: cudaFuncSetAttribute(k_expm_fwd_ps<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_fwd_ps<4>, thr, smem); break;
    }
    return (e == cudaSuccess && n > 0) ? n : 1;
}

}  // namespace qoc
