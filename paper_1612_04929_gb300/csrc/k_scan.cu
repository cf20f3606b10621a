// Segment products for the parallel-in-time form of the serial recursions.
//
// Both recursions of one evaluation are linear in the carried block:
//   forward   Psi_b = P_z Psi_{a-1},            P_z = U_b ... U_a                (Eqs. 2, 4)
//   costate   Y_{z-1} = P_z^dag Y_z + h_z                                       (Appendix A)
// for a segment z of slices a..b, where h_z is the segment's own costate from a zero in-carry.
// With every P_z in hand, a scan over the segments (one step per segment, not per slice) gives
// the checkpoints and the costate carries, and the slices inside every segment then run in
// parallel from them.  The products are associative, so each P_z is formed by a pairwise tree:
// level l multiplies neighbouring partial products of level l - 1 (the later one on the left),
// ceil(log2(seg)) batched launches in all, each over every (member, segment, pair) of the wave.
// The partial products and P_z are carried in extended precision (the hi + lo FP32 pair of the
// FP32 form, FP64 in the FP64 form), like the block that the recursions carry.  In the FP32 form
// the per-CTA products (d <= 68) multiply grid-split factors (qoc_device.cuh; the factors are
// products of U_j, whose norms the exponent eu bounds), so the grid parts sum exactly and only
// the cross terms are rounded, about 2^-36 of the product's scale.
#include <algorithm>
#include <type_traits>

#include "qoc_device.cuh"
#include "qoc_internal.h"

namespace qoc {

namespace {

constexpr int KC = 16;   // K-chunk staged in shared memory

// operands widened to the carried type on load
__device__ __forceinline__ float4 widen(const float2 v) { return make_float4(v.x, v.y, 0.f, 0.f); }
__device__ __forceinline__ float4 widen(const float4 v) { return v; }
__device__ __forceinline__ double2 widen(const double2 v) { return v; }
template <typename K> __device__ __forceinline__ K kz();
template <> __device__ __forceinline__ float4 kz<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double2 kz<double2>() { return make_double2(0.0, 0.0); }

// acc += a b (FP64 form; the FP32 form multiplies grid-split factors)
__device__ __forceinline__ void kmac2(double2& acc, const double2 a, const double2 b) { cfma(acc, a, b); }
__device__ __forceinline__ double2 knorm2(double2 v) { return v; }
__device__ __forceinline__ void kconj(float4& v) {
    v.y = -v.y;
    v.w = -v.w;
}
__device__ __forceinline__ void kconj(double2& v) { v.y = -v.y; }

// a factor element as grid-split float4 (re1, im1, re2, im2): from a plain FP32 value (exact
// split) or from a carried (hi, lo) pair
__device__ __forceinline__ float4 to_grid(const float2 v, float magic) {
    float4 o;
    grid_split(v.x, 0.f, magic, o.x, o.z);
    grid_split(v.y, 0.f, magic, o.y, o.w);
    return o;
}
__device__ __forceinline__ float4 to_grid(const float4 v, float magic) {
    float4 o;
    grid_split(v.x, v.z, magic, o.x, o.z);
    grid_split(v.y, v.w, magic, o.y, o.w);
    return o;
}

// Level l of the tree.  Item i of segment z at level l covers slices a + i 2^l .. ; it is the
// product of items 2i + 1 (left) and 2i of level l - 1, or item 2i itself when that one has no
// right neighbour.  CTA (tile, member * nzmax * cap + z * cap + i) computes a T x T tile.
// Level 1 reads U_j (type EI = C) from the propagator buffer, later levels the carried partial
// products (EI = K).
template <typename R, typename EI, int T>
__global__ void __launch_bounds__(256)
k_seg_mm(SegProdArgs<R> a, int level, const EI* __restrict__ src, size_t src_item, size_t src_seg, size_t src_e,
         K_t<R>* __restrict__ dst, int cap) {
    using K = K_t<R>;
    constexpr int MT = T / 16;
    constexpr bool kGrid = std::is_same<K, float4>::value;   // FP32 form: grid-split factors
    __shared__ __align__(16) K As[T][KC + 1];                 // (grid-split float4 in the FP32 form)
    __shared__ __align__(16) K Bs[KC][T + 1];
    const int d = a.d;
    const int q = blockIdx.y;
    const int e = q / (a.nzmax * cap);
    const int z = (q / cap) % a.nzmax;
    const int i = q % cap;
    const int a0 = z * a.seg;
    if (a0 >= a.wlen) return;
    const int len = min(a.wlen, a0 + a.seg) - a0;
    const int n_prev = (len + (1 << (level - 1)) - 1) >> (level - 1);
    const int n_cur = (len + (1 << level) - 1) >> level;
    if (i >= n_cur) return;
    const EI* base = src + e * src_e + z * src_seg;
    const EI* Bm = base + (size_t)(2 * i) * src_item;          // earlier factor (right)
    const bool pair = 2 * i + 1 < n_prev;
    const EI* Am = base + (size_t)(2 * i + 1) * src_item;      // later factor (left)
    K* out = dst + ((size_t)(e * a.nzmax + z) * cap + i) * a.mstride;
    const int ntn = (d + T - 1) / T;
    const int tm = blockIdx.x / ntn, tn = blockIdx.x - tm * ntn;
    const int r0 = tm * T, c0 = tn * T;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (!pair) {   // odd tail: carried up unchanged
        for (int x = 0; x < MT; ++x)
            for (int y = 0; y < MT; ++y) {
                const int r = r0 + ty + 16 * x, c = c0 + tx + 16 * y;
                if (r < d && c < d) out[(size_t)r * d + c] = widen(Bm[(size_t)r * d + c]);
            }
        return;
    }
    float mg = 0.f;
    if constexpr (kGrid) mg = grid_magic(a.prm ? a.prm->eu : 1);
    auto stage = [&](const EI& v) -> K {
        if constexpr (kGrid) return to_grid(v, mg);
        else return widen(v);
    };
    // FP32: grid sums (re, im) and cross terms (re, im) per output; FP64: plain accumulators
    float sa[kGrid ? MT : 1][kGrid ? MT : 1][4] = {};
    K acc[MT][MT];
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y) acc[x][y] = kz<K>();
    for (int k0 = 0; k0 < d; k0 += KC) {
        for (int idx = tid; idx < T * KC; idx += 256) {
            const int r = idx / KC, k = idx - r * KC;
            const int gr = r0 + r, gk = k0 + k;
            As[r][k] = (gr < d && gk < d) ? stage(Am[(size_t)gr * d + gk]) : kz<K>();
        }
        for (int idx = tid; idx < KC * T; idx += 256) {
            const int k = idx / T, c = idx - k * T;
            const int gk = k0 + k, gc = c0 + c;
            Bs[k][c] = (gk < d && gc < d) ? stage(Bm[(size_t)gk * d + gc]) : kz<K>();
        }
        __syncthreads();
        const int kmax = min(KC, d - k0);   // the last chunk may be partial (zero-padded)
#pragma unroll 4
        for (int k = 0; k < kmax; ++k) {
            K av[MT], bv[MT];
#pragma unroll
            for (int x = 0; x < MT; ++x) av[x] = As[ty + 16 * x][k];
#pragma unroll
            for (int y = 0; y < MT; ++y) bv[y] = Bs[k][tx + 16 * y];
            if constexpr (kGrid) {
                float2 bf[MT];
#pragma unroll
                for (int y = 0; y < MT; ++y) bf[y] = make_float2(bv[y].x + bv[y].z, bv[y].y + bv[y].w);
#pragma unroll
                for (int x = 0; x < MT; ++x)
#pragma unroll
                    for (int y = 0; y < MT; ++y) {
                        float* c = sa[x][y];
                        c[0] = fmaf(av[x].x, bv[y].x, c[0]);
                        c[0] = fmaf(-av[x].y, bv[y].y, c[0]);
                        c[1] = fmaf(av[x].x, bv[y].y, c[1]);
                        c[1] = fmaf(av[x].y, bv[y].x, c[1]);
                        c[2] = fmaf(av[x].x, bv[y].z, c[2]);
                        c[2] = fmaf(-av[x].y, bv[y].w, c[2]);
                        c[2] = fmaf(av[x].z, bf[y].x, c[2]);
                        c[2] = fmaf(-av[x].w, bf[y].y, c[2]);
                        c[3] = fmaf(av[x].x, bv[y].w, c[3]);
                        c[3] = fmaf(av[x].y, bv[y].z, c[3]);
                        c[3] = fmaf(av[x].z, bf[y].y, c[3]);
                        c[3] = fmaf(av[x].w, bf[y].x, c[3]);
                    }
            } else {
#pragma unroll
                for (int x = 0; x < MT; ++x)
#pragma unroll
                    for (int y = 0; y < MT; ++y) kmac2(acc[x][y], av[x], bv[y]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y) {
            const int r = r0 + ty + 16 * x, c = c0 + tx + 16 * y;
            if (r < d && c < d) {
                if constexpr (kGrid) {
                    float4 o;
                    two_sum(sa[x][y][0], sa[x][y][2], o.x, o.z);
                    two_sum(sa[x][y][1], sa[x][y][3], o.y, o.w);
                    out[(size_t)r * d + c] = o;
                } else {
                    out[(size_t)r * d + c] = knorm2(acc[x][y]);
                }
            }
        }
}

// The same level for d <= 68: one CTA per product, both factors in shared memory (padded to
// D = G MT with leading dimension D + 1), thread (ty, tx) of a G x G grid owning the MT x MT
// outputs (ty + G a, tx + G b) as in the per-slice kernels.  FP32 form: both factors grid-split
// on staging (level 1 from the plain U_j, later levels from the carried pairs), the result the
// error-free sum of the grid sums and the cross terms; FP64 form: plain FP64 products.

__device__ __forceinline__ void kmac_any(double2& acc, const double2 a, const double2 b) { cfma(acc, a, b); }

template <typename R, typename EI, int MT>
__global__ void __launch_bounds__(512)
k_seg_mm_small(SegProdArgs<R> a, int level, const EI* __restrict__ src, size_t src_item, size_t src_seg, size_t src_e,
               K_t<R>* __restrict__ dst, int cap, int G) {
    using K = K_t<R>;
    constexpr bool kGrid = std::is_same<K, float4>::value;   // FP32 form: grid-split factors
    using SE = std::conditional_t<kGrid, float4, EI>;         // staged element
    extern __shared__ __align__(16) unsigned char smraw[];
    const int d = a.d, D = G * MT, LD = D + 1;
    SE* As = reinterpret_cast<SE*>(smraw);
    SE* Bs = As + (size_t)D * LD;
    const int q = blockIdx.x;
    const int e = q / (a.nzmax * cap);
    const int z = (q / cap) % a.nzmax;
    const int i = q % cap;
    const int a0 = z * a.seg;
    if (a0 >= a.wlen) return;
    const int len = min(a.wlen, a0 + a.seg) - a0;
    const int n_prev = (len + (1 << (level - 1)) - 1) >> (level - 1);
    const int n_cur = (len + (1 << level) - 1) >> level;
    if (i >= n_cur) return;
    const EI* base = src + e * src_e + z * src_seg;
    const EI* Bm = base + (size_t)(2 * i) * src_item;          // earlier factor (right)
    const EI* Am = base + (size_t)(2 * i + 1) * src_item;      // later factor (left)
    K* out = dst + ((size_t)(e * a.nzmax + z) * cap + i) * a.mstride;
    const int tid = threadIdx.x;
    if (2 * i + 1 >= n_prev) {   // odd tail: carried up unchanged
        for (int idx = tid; idx < d * d; idx += blockDim.x) out[idx] = widen(Bm[idx]);
        return;
    }
    if constexpr (kGrid) {
        const float mg = grid_magic(a.prm ? a.prm->eu : 1);
        for_rc(d, d, [&](int idx, int r, int c) {
            As[r * LD + c] = to_grid(Am[idx], mg);
            Bs[r * LD + c] = to_grid(Bm[idx], mg);
        });
    } else {
        for_rc(d, d, [&](int idx, int r, int c) {
            As[r * LD + c] = Am[idx];
            Bs[r * LD + c] = Bm[idx];
        });
    }
    __syncthreads();
    if (tid >= G * G) return;   // the block is rounded up to whole warps; no barrier follows
    const int tx = tid % G, ty = tid / G;
    if constexpr (kGrid) {
        float acc[MT][MT][4] = {};
        mm_sl<MT>(acc, As, Bs, d, LD, ty, tx, G);
#pragma unroll
        for (int x = 0; x < MT; ++x)
#pragma unroll
            for (int y = 0; y < MT; ++y) {
                const int r = ty + G * x, c = tx + G * y;
                if (r < d && c < d) {
                    float4 o;
                    two_sum(acc[x][y][0], acc[x][y][2], o.x, o.z);
                    two_sum(acc[x][y][1], acc[x][y][3], o.y, o.w);
                    out[(size_t)r * d + c] = o;
                }
            }
    } else {
        K acc[MT][MT];
#pragma unroll
        for (int x = 0; x < MT; ++x)
#pragma unroll
            for (int y = 0; y < MT; ++y) acc[x][y] = kz<K>();
#pragma unroll 2
        for (int k = 0; k < d; ++k) {
            EI av[MT], bv[MT];
#pragma unroll
            for (int x = 0; x < MT; ++x) av[x] = As[(ty + G * x) * LD + k];
#pragma unroll
            for (int y = 0; y < MT; ++y) bv[y] = Bs[k * LD + tx + G * y];
#pragma unroll
            for (int x = 0; x < MT; ++x)
#pragma unroll
                for (int y = 0; y < MT; ++y) kmac_any(acc[x][y], av[x], bv[y]);
        }
#pragma unroll
        for (int x = 0; x < MT; ++x)
#pragma unroll
            for (int y = 0; y < MT; ++y) {
                const int r = ty + G * x, c = tx + G * y;
                if (r < d && c < d) out[(size_t)r * d + c] = knorm2(acc[x][y]);
            }
    }
}

// P_z and P_z^dag (carried) from item 0 of the last level (or from U_a when seg = 1)
template <typename R, typename EI>
__global__ void k_seg_store(SegProdArgs<R> a, const EI* __restrict__ src, size_t src_seg, size_t src_e) {
    using C = K_t<R>;
    const int q = blockIdx.y, e = q / a.nzmax, z = q % a.nzmax;
    if (z * a.seg >= a.wlen) return;
    const int d = a.d;
    const size_t dd = (size_t)d * d;
    const EI* m = src + e * src_e + z * src_seg;
    C* P = a.P + (size_t)(e * a.nzmax + z) * a.ustride;
    C* PH = P + a.ustride / 2;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / d), c = (int)(idx - (size_t)r * d);
        P[idx] = widen(m[idx]);
        C h = widen(m[(size_t)c * d + r]);
        kconj(h);
        PH[idx] = h;
    }
}

template <typename R, typename EI, int MT>
cudaError_t small_level(const SegProdArgs<R>& a, int level, const EI* src, size_t s_item, size_t s_seg, size_t s_e,
                        K_t<R>* dst, int cap, int G, cudaStream_t st) {
    const int D = G * MT;
    const size_t esz = sizeof(K_t<R>) == sizeof(float4) && sizeof(R) == 4 ? sizeof(float4) : sizeof(EI);
    const size_t smem = 2 * (size_t)D * (D + 1) * esz;
    cudaError_t err =
        cudaFuncSetAttribute(k_seg_mm_small<R, EI, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_seg_mm_small<R, EI, MT><<<a.E * a.nzmax * cap, slice_threads(G), smem, st>>>(a, level, src, s_item, s_seg, s_e,
                                                                                  dst, cap, G);
    return cudaGetLastError();
}

template <typename R, typename EI>
cudaError_t small_level_mt(const SegProdArgs<R>& a, int level, const EI* src, size_t s_item, size_t s_seg, size_t s_e,
                           K_t<R>* dst, int cap, cudaStream_t st) {
    const SliceTile tl = slice_tile(a.d);
    switch (tl.MT) {
        case 1: return small_level<R, EI, 1>(a, level, src, s_item, s_seg, s_e, dst, cap, tl.G, st);
        case 2: return small_level<R, EI, 2>(a, level, src, s_item, s_seg, s_e, dst, cap, tl.G, st);
        case 3: return small_level<R, EI, 3>(a, level, src, s_item, s_seg, s_e, dst, cap, tl.G, st);
        default: return small_level<R, EI, 4>(a, level, src, s_item, s_seg, s_e, dst, cap, tl.G, st);
    }
}

template <typename R, int T>
cudaError_t seg_levels(const SegProdArgs<R>& a, cudaStream_t st, int* launches) {
    using C = C_t<R>;
    using K = K_t<R>;
    const int ntile = T > 0 ? (a.d + T - 1) / T : 1;
    const int nz = (a.wlen + a.seg - 1) / a.seg;
    int levels = 0;
    while ((1 << levels) < a.seg) ++levels;
    const K* last = nullptr;
    size_t last_seg = 0, last_e = 0;
    for (int l = 1; l <= levels; ++l) {
        const int cap = (a.seg + (1 << l) - 1) >> l;
        K* dst = (l & 1) ? a.lv0 : a.lv1;
        const dim3 grid(ntile * ntile, a.E * a.nzmax * cap);
        const bool small = T == 0;   // whole products per CTA (d <= 68)
        if (small) {
            cudaError_t e2;
            if (l == 1)
                e2 = small_level_mt<R, C>(a, 1, a.U, (size_t)a.ustride, (size_t)a.seg * a.ustride,
                                          (size_t)a.wmax * a.ustride, dst, cap, st);
            else {
                const int pcap = (a.seg + (1 << (l - 1)) - 1) >> (l - 1);
                e2 = small_level_mt<R, K>(a, l, last, a.mstride, (size_t)pcap * a.mstride,
                                          (size_t)a.nzmax * pcap * a.mstride, dst, cap, st);
            }
            if (e2 != cudaSuccess) return e2;
        } else if (l == 1) {
            k_seg_mm<R, C, (T > 0 ? T : 16)><<<grid, 256, 0, st>>>(a, 1, a.U, (size_t)a.ustride, (size_t)a.seg * a.ustride,
                                                  (size_t)a.wmax * a.ustride, dst, cap);
        } else {
            const int pcap = (a.seg + (1 << (l - 1)) - 1) >> (l - 1);
            k_seg_mm<R, K, (T > 0 ? T : 16)><<<grid, 256, 0, st>>>(a, l, last, a.mstride, (size_t)pcap * a.mstride,
                                                  (size_t)a.nzmax * pcap * a.mstride, dst, cap);
        }
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        ++*launches;
        last = dst;
        last_seg = (size_t)cap * a.mstride;
        last_e = (size_t)a.nzmax * cap * a.mstride;
    }
    const size_t dd = (size_t)a.d * a.d;
    const int bx = (int)std::min<size_t>((dd + 255) / 256, 64);
    (void)nz;
    if (levels == 0)
        k_seg_store<R, C><<<dim3(bx, a.E * a.nzmax), 256, 0, st>>>(a, a.U, (size_t)a.seg * a.ustride,
                                                                  (size_t)a.wmax * a.ustride);
    else
        k_seg_store<R, K><<<dim3(bx, a.E * a.nzmax), 256, 0, st>>>(a, last, last_seg, last_e);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_seg_products(const SegProdArgs<R>& a, cudaStream_t st, int* launches) {
    *launches = 0;
    if (a.wlen <= 0 || a.seg <= 0 || a.E <= 0 || (a.wlen + a.seg - 1) / a.seg > a.nzmax) return cudaErrorInvalidValue;
    if (a.d <= 68 && slice_tile(a.d).MT > 0) return seg_levels<R, 0>(a, st, launches);
    if (a.d <= 48) return seg_levels<R, 16>(a, st, launches);
    if (a.d <= 128) return seg_levels<R, 32>(a, st, launches);
    return seg_levels<R, 64>(a, st, launches);
}

template cudaError_t launch_seg_products<float>(const SegProdArgs<float>&, cudaStream_t, int*);
template cudaError_t launch_seg_products<double>(const SegProdArgs<double>&, cudaStream_t, int*);

}  // namespace qoc
