// Slice exponential in split (hi + lo) FP32 arithmetic for the FP32 form.
//
// Over long evolutions the FP32 rounding of H_j dt and of the Taylor / squaring products is
// nearly the same at every slice (the drift H_0 does not change), so it accumulates coherently
// along the N-slice chain.  The FP32 form therefore evaluates U_j = [T_p(X_j)]^(2^n) (Eqs. 9,
// 10) with every matrix held as an unevaluated sum hi + lo of two FP32 numbers ("double-float"):
//   * X_j = -i s H_j is assembled in FP64 from FP64 copies of H_0, H_k, H_det and split,
//   * each product uses an exact FP32 product (hi*hi and its FMA residual), the two cross
//     terms hi*lo + lo*hi, and an error-free TwoSum accumulation of the high parts,
//   * the Horner division by i and the identity shift are done in the same pair arithmetic,
//   * Horner steps i > m_split use plain FP32 on the hi parts: an error made there reaches T
//     scaled by ts^m / m! < 2^-6 (m_split is picked with (p, n) from the FP64 norm bound).
// Only the rounded U_j is kept for the propagation (costates and the adjoint stay FP32), plus,
// for the reverse-mode adjoint, the rounded right operand of every product (ZStore).
// The same kernel is used for the recomputation in the backward sweep, so the forward and
// backward propagators are bitwise identical.
#include "qoc_device.cuh"
#include "qoc_internal.h"

namespace qoc {

struct DF {        // one real double-float: value = h + l, |l| <= ulp(h) / 2 after renormalisation
    float h, l;
};

// hi/lo accumulation of a * b for pair operands; the low-order terms are gathered in lo
__device__ __forceinline__ void df_mac(float& hi, float& lo, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float t = hi + p;
    const float bv = t - hi;
    const float err = (hi - (t - bv)) + (p - bv);
    hi = t;
    lo += err + e;
}

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

// split-complex matrices in shared memory: four planes re_h, re_l, im_h, im_l would halve the
// loads per product; here each element is a float4 (re_h, im_h, re_l, im_l).
template <int MT>
__device__ __forceinline__ void mm_df(float (&ar)[MT][MT][2], float (&ai)[MT][MT][2], const float4* __restrict__ A,
                                      const float4* __restrict__ B, int kd, int LD, int ty, int tx, int G) {
#pragma unroll 1
    for (int k = 0; k < kd; ++k) {
        float4 a[MT], b[MT];
#pragma unroll
        for (int i = 0; i < MT; ++i) a[i] = A[(ty + G * i) * LD + k];
#pragma unroll
        for (int i = 0; i < MT; ++i) b[i] = B[k * LD + tx + G * i];
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                // (a.x + a.z) + i (a.y + a.w)   times   (b.x + b.z) + i (b.y + b.w)
                df_mac(ar[i][j][0], ar[i][j][1], a[i].x, a[i].z, b[j].x, b[j].z);
                df_mac(ar[i][j][0], ar[i][j][1], -a[i].y, -a[i].w, b[j].y, b[j].w);
                df_mac(ai[i][j][0], ai[i][j][1], a[i].x, a[i].z, b[j].y, b[j].w);
                df_mac(ai[i][j][0], ai[i][j][1], a[i].y, a[i].w, b[j].x, b[j].z);
            }
    }
}

// plain FP32 product of the hi parts (the early Horner steps)
template <int MT>
__device__ __forceinline__ void mm_hi(float2 (&acc)[MT][MT], const float4* __restrict__ A, const float4* __restrict__ B,
                                      int kd, int LD, int ty, int tx, int G) {
#pragma unroll 2
    for (int k = 0; k < kd; ++k) {
        float2 a[MT], b[MT];
#pragma unroll
        for (int i = 0; i < MT; ++i) {
            const float4 v = A[(ty + G * i) * LD + k];
            a[i] = make_float2(v.x, v.y);
        }
#pragma unroll
        for (int i = 0; i < MT; ++i) {
            const float4 v = B[k * LD + tx + G * i];
            b[i] = make_float2(v.x, v.y);
        }
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
            for (int j = 0; j < MT; ++j) cfma(acc[i][j], a[i], b[j]);
    }
}

template <int MT>
__device__ __forceinline__ void df_zero(float (&ar)[MT][MT][2], float (&ai)[MT][MT][2]) {
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j) ar[i][j][0] = ar[i][j][1] = ai[i][j][0] = ai[i][j][1] = 0.f;
}

// out = [diag I] + acc / div  (div = 0: no division), zero in the padding
template <int MT>
__device__ __forceinline__ void df_store(float4* __restrict__ out, float (&ar)[MT][MT][2], float (&ai)[MT][MT][2],
                                         int div, bool add_identity, int d, int LD, int ty, int tx, int G) {
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j) {
            const int r = ty + G * i, c = tx + G * j;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < d && c < d) {
                float rh = ar[i][j][0], rl = ar[i][j][1], ih = ai[i][j][0], il = ai[i][j][1];
                df_norm(rh, rl);
                df_norm(ih, il);
                if (div > 1) {
                    df_div(rh, rl, (float)div);
                    df_div(ih, il, (float)div);
                }
                if (add_identity && r == c) df_add1(rh, rl);
                v = make_float4(rh, ih, rl, il);
            }
            out[r * LD + c] = v;
        }
}

template <int MT>
__global__ void __launch_bounds__(512)
k_expm_fwd_split(const DevParams* __restrict__ prm, SysView<float> sys, const double2* __restrict__ H64, int j0,
                 float2* __restrict__ Ubuf, long long ustride, int wmax, ZStore<float> zs, int G) {
    const int D = G * MT, LD = D + 1, SZ = D * LD;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double us[kMaxControls];
    float4* X = reinterpret_cast<float4*>(smraw);
    float4* Za = X + SZ;
    float4* Zb = Za + SZ;
    const int jl = blockIdx.x, e = blockIdx.y, j = j0 + jl;
    const int tid = threadIdx.x, tx = tid % G, ty = tid / G;
    const bool act = tid < G * G;   // the block is rounded up to whole warps
    const int d = sys.d, M = sys.M, p = prm->p, n = prm->n;
    const double s = prm->s;
    for (int k = tid; k < M; k += blockDim.x) us[k] = sys.u[(size_t)k * sys.N + j];
    __syncthreads();
    const double de = sys.delta ? sys.delta[e] : 0.0;
    const size_t dd = (size_t)d * d;
    const double2* H0 = H64;
    const double2* Hk = H64 + dd;
    const double2* Hd = H64 + (size_t)(M + 1) * dd;
    // X = -i s H_j in FP64, split into hi + lo; Z = I + X / p in pair arithmetic
    for (int idx = tid; idx < D * D; idx += blockDim.x) {
        const int a = idx / D, b = idx - a * D;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f), z = x;
        if (a < d && b < d) {
            const int o = a * d + b;
            double2 h = H0[o];
            for (int k = 0; k < M; ++k) {
                const double2 hk = Hk[k * dd + o];
                h.x = fma(us[k], hk.x, h.x);
                h.y = fma(us[k], hk.y, h.y);
            }
            if (sys.Hdet) {
                const double2 hd = Hd[o];
                h.x = fma(de, hd.x, h.x);
                h.y = fma(de, hd.y, h.y);
            }
            const double xr = s * h.y, xi = -s * h.x;
            x.x = (float)xr;
            x.z = (float)(xr - (double)x.x);
            x.y = (float)xi;
            x.w = (float)(xi - (double)x.y);
            const double zr = xr / p + (a == b ? 1.0 : 0.0), zi = xi / p;
            z.x = (float)zr;
            z.z = (float)(zr - (double)z.x);
            z.y = (float)zi;
            z.w = (float)(zi - (double)z.y);
        }
        X[a * LD + b] = x;
        Za[a * LD + b] = z;
    }
    __syncthreads();
    float4* zin = Za;
    float4* zout = Zb;
    const int m_split = prm->m_split;
    float2* zst = (zs.Z && p - 1 + n <= zs.cap) ? zs.Z + ((size_t)e * zs.wmax + jl) * zs.cap * zs.mstride : nullptr;
    // the right operand of product r, rounded to FP32 and conjugate-transposed, for the adjoint
    auto store = [&](int r) {
        float2* dst = zst + (size_t)r * zs.mstride;
        for (int idx = tid; idx < d * d; idx += blockDim.x) {
            const int a = idx / d, b = idx - a * d;
            const float4 v = zin[b * LD + a];
            dst[idx] = make_float2(v.x + v.z, -(v.y + v.w));
        }
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
                    }
                    zout[r * LD + c] = v;
                }
        } else {
            float ar[MT][MT][2], ai[MT][MT][2];
            df_zero<MT>(ar, ai);
            mm_df<MT>(ar, ai, X, zin, d, LD, ty, tx, G);
            df_store<MT>(zout, ar, ai, i, true, d, LD, ty, tx, G);
        }
        __syncthreads();
        float4* t = zin; zin = zout; zout = t;
    }
    for (int m = 0; m < n; ++m) {             // squaring: Z <- Z Z
        if (zst) store(p - 1 + m);
        if (act) {
            float ar[MT][MT][2], ai[MT][MT][2];
            df_zero<MT>(ar, ai);
            mm_df<MT>(ar, ai, zin, zin, d, LD, ty, tx, G);
            df_store<MT>(zout, ar, ai, 0, false, d, LD, ty, tx, G);
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
static cudaError_t launch_split_mt(const DevParams* prm, const SysView<float>& sys, const double2* H64, int j0,
                                   int wlen, int E, float2* Ubuf, long long ustride, int wmax, const ZStore<float>& zs,
                                   int G, cudaStream_t st) {
    const size_t smem = split_smem(sys.d);
    cudaError_t err = cudaFuncSetAttribute(k_expm_fwd_split<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_expm_fwd_split<MT><<<dim3(wlen, E), slice_threads(G), smem, st>>>(prm, sys, H64, j0, Ubuf, ustride, wmax, zs, G);
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

cudaError_t launch_expm_fwd_split(const DevParams* prm, const SysView<float>& sys, const double2* H64, int j0, int wlen,
                                  int E, float2* Ubuf, long long ustride, int wmax, const ZStore<float>& zs,
                                  cudaStream_t st) {
    const SliceTile tl = slice_tile(sys.d);
    if (sys.d > split_max_d()) return cudaErrorInvalidValue;
    switch (tl.MT) {
        case 1: return launch_split_mt<1>(prm, sys, H64, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 2: return launch_split_mt<2>(prm, sys, H64, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 3: return launch_split_mt<3>(prm, sys, H64, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        case 4: return launch_split_mt<4>(prm, sys, H64, j0, wlen, E, Ubuf, ustride, wmax, zs, tl.G, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qoc
