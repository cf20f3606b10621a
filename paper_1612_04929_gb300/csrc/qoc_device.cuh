// Device-side helpers shared by the CUDA kernels of the quantum-control evaluation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qoc {

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

template <typename C> __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }
template <typename C, typename R> __device__ __forceinline__ C cmk(R re, R im) { C z; z.x = re; z.y = im; return z; }

// acc += a * b
template <typename C> __device__ __forceinline__ void cfma(C& acc, const C a, const C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C> __device__ __forceinline__ void cfma_cj(C& acc, const C a, const C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
// acc += a * conj(b)
template <typename C> __device__ __forceinline__ void cfma_bcj(C& acc, const C a, const C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.y, b.x, acc.y);
    acc.y = fma(-a.x, b.y, acc.y);
}

constexpr int kPsCoefs = 44;       // Taylor coefficients 1/k!, k = 0 .. kPMax + 3
constexpr int kPsMaxBlocks = 15;   // blocks of three terms, q = 0 .. kPMax / 3 + 1

// Per-evaluation scalars produced on the device by the norm kernel and read by every kernel.
struct DevParams {
    double theta;   // dt * max_j ||H_j||_1 bound (FP64)
    double s;       // dt / 2^n
    int p;          // Taylor order
    int n;          // squaring count
    int err;        // error bits (kErr*)
    int m_split;    // Horner steps i <= m_split need hi+lo arithmetic in the split exponential
    // grid exponents of the split FP32 exponential: 2^e bounds the row and column 2-norms of
    // X (ex), of the Horner matrices Z_i, i >= 2 (ez), and of T and its squarings (eu)
    int ex, ez, eu;
    // Paterson-Stockmeyer form of the split exponential (block size 3): 2^e2, 2^e3 bound the 2-norms
    // of X^2 and X^3, 2^ew[q] that of the chain matrix W_q (ew[0] = eu: W_0 = T); the Taylor
    // coefficients 1/k! as FP32 pairs (ch + cl), zero for k > p
    int e2, e3;
    int ew[kPsMaxBlocks];
    float ch[kPsCoefs], cl[kPsCoefs];
    // cross-block reduction of the final cost terms (k_finalize): per-block partials and the
    // count of blocks that have written theirs (the last block sums them in block order and
    // resets the count)
    unsigned fin_count;
    double fin_part[4 * 32];
};
constexpr int kFinBlocks = 32;

enum : int { kErrRange = 1, kErrTimeout = 2, kErrNonfinite = 4, kErrStale = 8 };

// ------------------------------------------------------------------------------------------
// Block-strided loop over a rows x cols array, f(idx, r, c) with r = idx / cols, c = idx % cols:
// the row and column are stepped, not divided out per element.
// ------------------------------------------------------------------------------------------
template <typename F>
__device__ __forceinline__ void for_rc(int rows, int cols, F f) {
    const int n = rows * cols, step = blockDim.x;
    const int sr = step / cols, sc = step - sr * cols;
    int r = threadIdx.x / cols, c = threadIdx.x - r * cols;
    for (int idx = threadIdx.x; idx < n; idx += step) {
        f(idx, r, c);
        r += sr;
        c += sc;
        if (c >= cols) {
            c -= cols;
            ++r;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Grid split of FP32 operands (split exponentials of the FP32 form).  A value v = h + l held as
// two FP32 numbers is stored as v1 + v2: v1 = h rounded to a multiple of g = 2^(e - 12), where
// 2^e bounds the row / column 2-norms of the matrix, and v2 = (h - v1) + l.  Then v1 has at
// most 13 significant bits, every product a1 b1 of two grid parts is exact in FP32, and by
// Cauchy-Schwarz every partial sum of a row-times-column contraction of grid parts stays below
// 2^24 units of g_a g_b, so it is exact as well: the FMAs sum a1 b1 without rounding, and only
// the cross terms a1 b2 + a2 b (of relative size 2^-12) are rounded.  If a bound is ever
// exceeded the grid sums round like plain FP32; nothing else changes.
// ------------------------------------------------------------------------------------------
// 1.5 * 2^(e + 11): adding and subtracting it rounds |h| <= 2^e to a multiple of 2^(e - 12)
__device__ __forceinline__ float grid_magic(int e) { return ldexpf(1.5f, e + 11); }

__device__ __forceinline__ void grid_split(float h, float l, float magic, float& v1, float& v2) {
    v1 = __fsub_rn(__fadd_rn(h, magic), magic);
    v2 = __fadd_rn(__fsub_rn(h, v1), l);
}

// error-free sum: s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// (hi, lo) += (u.x + u.y) (bh + bl), the exact product residual and the rounding of the sum in lo
__device__ __forceinline__ void pair_fma(float& hi, float& lo, float2 u, float bh, float bl) {
    const float p = u.x * bh;
    float e = fmaf(u.x, bh, -p);
    e = fmaf(u.x, bl, e);
    e = fmaf(u.y, bh, e);
    float s, r;
    two_sum(hi, p, s, r);
    hi = s;
    lo += r + e;
}

// (hi, lo) + (ch + cl), pair arithmetic
__device__ __forceinline__ void df_addc(float& hi, float& lo, float2 c) {
    float s, r;
    two_sum(hi, c.x, s, r);
    hi = s;
    lo += r + c.y;
}

// Split product of two grid-split matrices (float4 = re1, im1, re2, im2 per element):
// acc[0], acc[1] = exact sums of the grid parts (re, im), acc[2], acc[3] = the cross terms.
template <int MT>
__device__ __forceinline__ void mm_sl(float (&acc)[MT][MT][4], const float4* __restrict__ A,
                                     const float4* __restrict__ B, int kd, int LD, int ty, int tx, int G) {
    const float4* pa[MT];
    const float4* pb[MT];
#pragma unroll
    for (int i = 0; i < MT; ++i) {
        pa[i] = A + (ty + G * i) * LD;
        pb[i] = B + tx + G * i;
    }
#pragma unroll(MT >= 4 ? 1 : 2)
    for (int k = 0; k < kd; ++k) {
        float4 a[MT], b[MT];
        float2 bf[MT];
#pragma unroll
        for (int i = 0; i < MT; ++i) a[i] = pa[i][k];
#pragma unroll
        for (int j = 0; j < MT; ++j) {
            b[j] = *pb[j];
            pb[j] += LD;
            bf[j] = make_float2(b[j].x + b[j].z, b[j].y + b[j].w);
        }
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                float* c = acc[i][j];
                c[0] = fmaf(a[i].x, b[j].x, c[0]);
                c[0] = fmaf(-a[i].y, b[j].y, c[0]);
                c[1] = fmaf(a[i].x, b[j].y, c[1]);
                c[1] = fmaf(a[i].y, b[j].x, c[1]);
                c[2] = fmaf(a[i].x, b[j].z, c[2]);
                c[2] = fmaf(-a[i].y, b[j].w, c[2]);
                c[2] = fmaf(a[i].z, bf[j].x, c[2]);
                c[2] = fmaf(-a[i].w, bf[j].y, c[2]);
                c[3] = fmaf(a[i].x, b[j].w, c[3]);
                c[3] = fmaf(a[i].y, b[j].z, c[3]);
                c[3] = fmaf(a[i].z, bf[j].y, c[3]);
                c[3] = fmaf(a[i].w, bf[j].x, c[3]);
            }
    }
}

// ------------------------------------------------------------------------------------------
// cp.async (16-byte) helpers for the prefetch rings of the serial propagation kernels.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
// one 8- or 16-byte element
template <typename T> __device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
    static_assert(sizeof(T) == 8 || sizeof(T) == 16, "8- or 16-byte elements");
    if constexpr (sizeof(T) == 16) cp_async16(smem, gmem);
    else cp_async8(smem, gmem);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// FP64 block reduction (blockDim.x multiple of 32, <= 1024); result valid in thread 0.
// (hi, lo) += a b with the exact FP32 product (FMA residual) and an error-free sum: per-thread
// partial sums of products at pair precision without the FP64 pipe
__device__ __forceinline__ void pair_acc(float& hi, float& lo, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    float s, r;
    two_sum(hi, p, s, r);
    hi = s;
    lo += r + e;
}

__device__ __forceinline__ double block_sum(double v, double* scratch /* >= 32 doubles */) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace qoc
