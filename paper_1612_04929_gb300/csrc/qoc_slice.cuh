// Per-slice matrix helpers shared by the fused per-slice kernels (k_expm_fused.cu) and the
// Paterson-Stockmeyer adjoints (k_expm_ps.cu).
//
// Thread layout: a G x G grid of threads (slice_tile); thread (ty, tx) owns the MT x MT outputs
// (ty + G a, tx + G b).  Matrices sit in shared memory padded to D = G MT rows with a leading
// dimension of D + 1 complex elements; padding rows and columns are kept at zero.
#pragma once
#include "qoc_device.cuh"

namespace qoc {

template <typename C, int MT>
__device__ __forceinline__ void mm_acc(C (&acc)[MT][MT], const C* __restrict__ A,
                                       const C* __restrict__ B, int kd, int LD, int ty, int tx, int G) {
    // one pointer per operand row / column: A rows advance by k, B columns step down one row
    const C* pa[MT];
    const C* pb[MT];
#pragma unroll
    for (int i = 0; i < MT; ++i) {
        pa[i] = A + (ty + G * i) * LD;
        pb[i] = B + tx + G * i;
    }
#pragma unroll 2
    for (int k = 0; k < kd; ++k) {
        C a[MT], b[MT];
#pragma unroll
        for (int i = 0; i < MT; ++i) a[i] = pa[i][k];
#pragma unroll
        for (int i = 0; i < MT; ++i) {
            b[i] = *pb[i];
            pb[i] += LD;
        }
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
            for (int jj = 0; jj < MT; ++jj) cfma(acc[i][jj], a[i], b[jj]);
    }
}

template <typename C, int MT>
__device__ __forceinline__ void zero_acc(C (&acc)[MT][MT]) {
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int jj = 0; jj < MT; ++jj) acc[i][jj] = czero<C>();
}

// out = diag * I + scale * acc on the d x d block, zero in the padding.
template <typename C, typename R, int MT>
__device__ __forceinline__ void store_acc(C* __restrict__ out, const C (&acc)[MT][MT], R scale,
                                          R diag, int d, int LD, int ty, int tx, int G) {
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int jj = 0; jj < MT; ++jj) {
            const int r = ty + G * i, c = tx + G * jj;
            C v = czero<C>();
            if (r < d && c < d) {
                v.x = acc[i][jj].x * scale + (r == c ? diag : R(0));
                v.y = acc[i][jj].y * scale;
            }
            out[r * LD + c] = v;
        }
}

// dst (d x d, global) = conjugate transpose of the d x d block of src (shared, leading dim LD)
template <typename C>
__device__ __forceinline__ void store_ct(C* __restrict__ dst, const C* __restrict__ src, int d, int LD) {
    for_rc(d, d, [&](int idx, int a, int b) {
        C v = src[b * LD + a];
        v.y = -v.y;
        dst[idx] = v;
    });
}

// Assemble H_j (+ delta_e Hdet) and write X = -i s H into padded shared memory (rows/cols >= d
// zero).  us: the M control values of this slice (shared).
template <typename C, typename R>
__device__ __forceinline__ void assemble_X(C* __restrict__ X, int d, int D, int LD, int M,
                                           const C* __restrict__ H0, const C* __restrict__ Hk,
                                           const C* __restrict__ Hdet, R de, const R* us, R s) {
    const size_t dd = (size_t)d * d;
    for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
        const int a = idx / D, b = idx - a * D;
        C x = czero<C>();
        if (a < d && b < d) {
            const int o = a * d + b;
            C h = H0[o];
            for (int k = 0; k < M; ++k) {
                const C hk = Hk[k * dd + o];
                h.x = fma(us[k], hk.x, h.x);
                h.y = fma(us[k], hk.y, h.y);
            }
            if (Hdet) {
                const C hd = Hdet[o];
                h.x = fma(de, hd.x, h.x);
                h.y = fma(de, hd.y, h.y);
            }
            x.x = s * h.y;      // -i s (hr + i hi) = s hi - i s hr
            x.y = -s * h.x;
        }
        X[a * LD + b] = x;
    }
}

}  // namespace qoc
