// Tensor-core products of the large-d adjoint with exact leading-level accumulation (BF16_SPLIT).
//
// The reverse-mode adjoint of the truncated series (the exact derivative of Eqs. 9-10 applied to
// Ubar, Appendix A) needs FP32-accurate complex products.  The tensor core's FP32 accumulator
// truncates, and a truncation bias in the leading part of a product adds up over the Horner and
// squaring recursion, so the leading part is made exact instead (an integer-slice splitting in
// the manner of Ozaki's error-free matrix product):
//   * every row of an A operand (every column of a B operand) is scaled by a power of two 2^e
//     with max |entry| < 2^e; the scaled value y = x 2^-e (|y| < 1) is cut into four slices of
//     seven bits, y = sum_s a_s 2^(-7 (s + 1)) + r, |r| <= 2^-29, with integers |a_0| <= 128 and
//     |a_s| <= 64 after it;
//   * the A planes hold a_s 2^(7 - 7 s) and the B planes b_t 2^(-7 t) (BF16, exact), so the MMA
//     of slices s and t contributes a_s b_t 2^(7 - 7 (s + t)): the pair (0, 0) is 2^7 times an
//     integer product of at most 2^14, and over k < 512 (two products per k for each complex
//     part) its accumulator stays an exact multiple of 2^7 below 2^31, whatever the rounding of
//     the FP32 accumulation;
//   * the nine pairs with 1 <= s + t <= 3 accumulate, already weighted, into a second FP32
//     accumulator whose size is about 2^-7 of the leading one, so its truncation errors stay far
//     below the FP32 rounding of the result; the pairs with s + t >= 4 (below 2^-28) are dropped;
//   * the epilogue scales the sum of the two accumulators by 2^(eA + eB - 21) (exact).
// Measured in emulation on identity-dominant Horner matrices this is as accurate as an FP32 SIMT
// product (and several times more accurate on dense ones); four six-bit slices scaled the same
// way lose the small off-diagonal entries of I + X / i.
//
// k_oz_mm computes one 128 x 128 tile of C = alpha A B (+ C) (+ I) for one job and one wave item:
// warp 0 issues the TMA loads of a three-stage ring (one stage: the eight slice planes of A and
// of B for a 16-wide K chunk, SWIZZLE_32B, 64 KB), warp 1 issues the tcgen05.mma (kind::f16,
// BF16 in, FP32 accumulators in tensor memory: leading re, leading im, rest re, rest im, 128
// columns each) and commits each stage back to the producer, warps 2-5 read tensor memory with
// tcgen05.ld, stage the scaled tile in the idle ring and write it with coalesced stores.  Every mbarrier wait is bounded; a wait that runs out sets
// kErrTimeout in DevParams.err and the CTA stops issuing, waits (bounded) for its copies in
// flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "qoc_device.cuh"
#include "qoc_internal.h"

namespace qoc {

namespace {

constexpr int BM = 128, BN = 128, BK = 16;         // BK in BF16 elements: 32-byte rows
constexpr int NSL = kOzSlices;                     // seven-bit slices per value
constexpr int NPART = 2 * NSL;                     // re slices, then im slices
constexpr int SBITS = 7;
constexpr int TILE_BYTES = BM * BK * 2;            // one plane tile, 4 KB (A and B alike)
constexpr int STAGE = 2 * NPART * TILE_BYTES;      // 64 KB
constexpr int NST = 3;
constexpr int OZ_SMEM = NST * STAGE + 1024;        // + alignment slack
constexpr uint32_t TMEM_COLS = 512;
constexpr int NTHREADS = 192;                      // producer warp, MMA warp, four epilogue warps
constexpr uint32_t WAIT_LIMIT = 1u << 24;
constexpr uint32_t WAIT_LIMIT_TEST = 1u << 12;     // fault-injection runs

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(su32(b)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_3d(void* smem, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            su32(smem)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
        : "memory");
}
// UMMA shared-memory descriptor: K-major, SWIZZLE_32B (one 32-byte row per M / N index, 8-row
// groups 256 bytes apart), descriptor version 1
__device__ __forceinline__ uint64_t sdesc(const void* smem) {
    const uint64_t a = su32(smem);
    return ((a >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(256 >> 4) << 32) | (1ull << 46) | (6ull << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// exponent e with |x| < 2^e for the largest |x| of a row or column (0 for an all-zero one)
__device__ __forceinline__ int scale_exp(float m) {
    int e = 0;
    if (m > 0.f) frexpf(m, &e);
    return e;
}
// four seven-bit slices of y = x 2^-e (|y| < 1), weighted for their operand role: A planes hold
// a_s 2^(7 - 7 s), B planes b_s 2^(-7 s); every step is exact
__device__ __forceinline__ void slices(float x, int e, bool role_a, float (&q)[NSL]) {
    float r = ldexpf(x, SBITS - e);
    float w = role_a ? (float)(1 << SBITS) : 1.0f;
#pragma unroll
    for (int s = 0; s < NSL; ++s) {
        const float a = rintf(r);
        q[s] = a * w;
        r = (r - a) * (float)(1 << SBITS);
        w *= 1.0f / (float)(1 << SBITS);
    }
}

}  // namespace

// plane (item, matrix, part) in the plane array
__host__ __device__ inline size_t oz_plane(int item, int mat, int part) {
    return ((size_t)item * kOzMats + mat) * NPART + part;
}

// ------------------------------------------------------------------------------------------
// slicing: FP32 complex d x d matrices (row-major, item-strided) -> exponents and BF16 planes
// ------------------------------------------------------------------------------------------
// Row layout (A operand): plane row r = row r of M, exponent per row.  Column layout (B operand,
// K-major): plane row c = column c of M, exponent per column (no conjugation is applied).
__global__ void __launch_bounds__(256)
k_oz_slice(OzSliceJobs jobs, __nv_bfloat16* __restrict__ planes, int* __restrict__ exps, int d, int ldp) {
    __shared__ float2 tile[32][33];
    __shared__ float cmax[8][32];
    __shared__ int cexp[32];
    const OzSliceJob jb = jobs.job[blockIdx.z];
    const int item = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float2* M = jb.src + (size_t)item * jb.stride;
    const size_t psz = (size_t)d * ldp;
    if (!jb.col) {
        const int r = blockIdx.x * 8 + warp;
        if (r >= d) return;
        float m = 0.f;
        for (int b = lane; b < d; b += 32) {
            const float2 v = M[(size_t)r * d + b];
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const int e = scale_exp(m);
        if (lane == 0) exps[((size_t)item * kOzMats + jb.mat) * d + r] = e;
        for (int b = lane; b < d; b += 32) {
            const float2 v = M[(size_t)r * d + b];
            float qr[NSL], qi[NSL];
            slices(v.x, e, true, qr);
            slices(v.y, e, true, qi);
#pragma unroll
            for (int s = 0; s < NSL; ++s) {
                planes[oz_plane(item, jb.mat, s) * psz + (size_t)r * ldp + b] = __float2bfloat16_rn(qr[s]);
                planes[oz_plane(item, jb.mat, NSL + s) * psz + (size_t)r * ldp + b] = __float2bfloat16_rn(qi[s]);
            }
        }
        return;
    }
    // column layout: 32 columns c0 .. c0 + 31 per CTA
    const int c0 = blockIdx.x * 32;
    if (c0 >= d) return;
    const int c = c0 + lane;
    float m = 0.f;
    if (c < d)
        for (int k = warp; k < d; k += 8) {
            const float2 v = M[(size_t)k * d + c];
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
    cmax[warp][lane] = m;
    __syncthreads();
    if (warp == 0) {
        float mm = cmax[0][lane];
        for (int w = 1; w < 8; ++w) mm = fmaxf(mm, cmax[w][lane]);
        const int e = scale_exp(mm);
        cexp[lane] = e;
        if (c < d) exps[((size_t)item * kOzMats + jb.mat) * d + c] = e;
    }
    __syncthreads();
    for (int k0 = 0; k0 < d; k0 += 32) {
        for (int q = warp; q < 32; q += 8) {   // tile[k][c]: row k0 + q of M, columns c0 ..
            const int k = k0 + q;
            tile[q][lane] = (k < d && c < d) ? M[(size_t)k * d + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int q = warp; q < 32; q += 8) {   // plane row c0 + q (a column of M), k along lanes
            const int cc = c0 + q, k = k0 + lane;
            if (cc < d && k < d) {
                const float2 v = tile[lane][q];
                float qr[NSL], qi[NSL];
                slices(v.x, cexp[q], false, qr);
                slices(v.y, cexp[q], false, qi);
#pragma unroll
                for (int s = 0; s < NSL; ++s) {
                    planes[oz_plane(item, jb.mat, s) * psz + (size_t)cc * ldp + k] = __float2bfloat16_rn(qr[s]);
                    planes[oz_plane(item, jb.mat, NSL + s) * psz + (size_t)cc * ldp + k] = __float2bfloat16_rn(qi[s]);
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// one 128 x 128 output tile of C = alpha A B (+ beta C) (+ I) for job blockIdx.z, item blockIdx.y
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(NTHREADS, 1)
k_oz_mm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzJobs jobs,
        const int* __restrict__ exps, int d, DevParams* __restrict__ prm) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[NST], empty[NST], done;
    __shared__ uint32_t tmem_holder;
    __shared__ int skip, s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // once a wait has run out in this evaluation, later launches skip their work (the result is
    // reported as QOC_ERR_TIMEOUT); thread 0 decides for the whole CTA
    if (tid == 0) {
        skip = (*(volatile int*)&prm->err & kErrTimeout) != 0;
        s_ok = 1;
    }
    __syncthreads();
    if (skip) return;
    const uint32_t limit = jobs.fault ? WAIT_LIMIT_TEST : WAIT_LIMIT;
    const int item = blockIdx.y;
    const OzJob jb = jobs.j[blockIdx.z];
    const int ntn = (d + BN - 1) / BN;
    const int r0 = (blockIdx.x / ntn) * BM, c0 = (blockIdx.x % ntn) * BN;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < NST; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;
    const int nk = (d + BK - 1) / BK;

    if (warp == 0 && lane == 0) {
        // ---- producer: the eight A planes and eight B planes of one K chunk per stage ----
        bool ok = true;
        int last_issued[NST];
#pragma unroll
        for (int b = 0; b < NST; ++b) last_issued[b] = -1;
        for (int s = 0; s < nk; ++s) {
            const int b = s % NST;
            if (s >= NST && !mbar_wait(&empty[b], (uint32_t)((s / NST - 1) & 1), limit)) {
                ok = false;
                break;
            }
            if (jobs.fault && s == 0) continue;   // fault injection: the first copy is withheld
            unsigned char* st = base + b * STAGE;
            mbar_expect_tx(&full[b], STAGE);
            for (int part = 0; part < NPART; ++part) {
                tma_3d(st + part * TILE_BYTES, &mapA, s * BK, r0, (int)oz_plane(item, jb.a_mat, part), &full[b]);
                tma_3d(st + (NPART + part) * TILE_BYTES, &mapB, s * BK, c0, (int)oz_plane(item, jb.b_mat, part),
                       &full[b]);
            }
            last_issued[b] = s;
        }
        if (!ok) {
            atomicOr(&prm->err, kErrTimeout);
            s_ok = 0;
        }
        // every copy issued into this CTA's shared memory lands before the CTA can leave (bounded)
        for (int b = 0; b < NST; ++b)
            if (last_issued[b] >= 0) mbar_wait(&full[b], (uint32_t)((last_issued[b] / NST) & 1), limit);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        // instruction descriptor: D f32, A/B bf16, both K-major, N = 128, M = 128
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
        const uint32_t idesc_nA = idesc | (1u << 13);   // negate A
        const uint32_t lead_re = tmem, lead_im = tmem + BN, rest_re = tmem + 2 * BN, rest_im = tmem + 3 * BN;
        bool ok = true;
        for (int s = 0; s < nk; ++s) {
            const int b = s % NST;
            if (!mbar_wait(&full[b], (uint32_t)((s / NST) & 1), limit)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned char* st = base + b * STAGE;
            uint64_t Ar[NSL], Ai[NSL], Br[NSL], Bi[NSL];
#pragma unroll
            for (int q = 0; q < NSL; ++q) {
                Ar[q] = sdesc(st + q * TILE_BYTES);
                Ai[q] = sdesc(st + (NSL + q) * TILE_BYTES);
                Br[q] = sdesc(st + (NPART + q) * TILE_BYTES);
                Bi[q] = sdesc(st + (NPART + NSL + q) * TILE_BYTES);
            }
#pragma unroll
            for (int sa = 0; sa < NSL; ++sa)
#pragma unroll
                for (int sb = 0; sb + sa < NSL; ++sb) {
                    const bool lead = sa + sb == 0;
                    // the first MMA into each accumulator overwrites it: (0, 0) and (0, 1) of chunk 0
                    const uint32_t en = (s > 0 || !(lead || (sa == 0 && sb == 1))) ? 1u : 0u;
                    const uint32_t acc_re = lead ? lead_re : rest_re, acc_im = lead ? lead_im : rest_im;
                    // re += Ar Br - Ai Bi ;  im += Ar Bi + Ai Br
                    mma_bf16(acc_re, Ar[sa], Br[sb], idesc, en);
                    mma_bf16(acc_re, Ai[sa], Bi[sb], idesc_nA, 1);
                    mma_bf16(acc_im, Ar[sa], Bi[sb], idesc, en);
                    mma_bf16(acc_im, Ai[sa], Br[sb], idesc, 1);
                }
            mma_commit(&empty[b]);   // the stage is free once these MMAs have read it
        }
        mma_commit(&done);
        if (!ok) {
            atomicOr(&prm->err, kErrTimeout);
            s_ok = 0;
        }
    }
    __syncthreads();
    const bool fin = mbar_wait(&done, 0, limit);
    if (!fin && tid == 0) atomicOr(&prm->err, kErrTimeout);
    // the epilogue's TMEM loads are warp-collective: the decision is the same for every thread
    const bool go = __syncthreads_and(fin && s_ok != 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (go && warp >= 2) {
        // Each epilogue warp owns 32 tile rows (the TMEM lane quarter it may read).  It scales
        // its rows into a staging area of the idle stage ring (every copy has landed and every
        // MMA has read its operands once `done` completed), then writes them row by row with
        // the lanes along the columns, so the global stores (and the reads of beta) coalesce.
        constexpr int SROW = BN + 1;                   // padded row: fewer bank conflicts
        const int q4 = warp & 3;
        const int r = r0 + q4 * 32 + lane;
        const int ncols = min(BN, d - c0);
        const int eA = r < d ? exps[((size_t)item * kOzMats + jb.a_mat) * d + r] : 0;
        const int* eBp = exps + ((size_t)item * kOzMats + jb.b_mat) * d;
        float2* stg = reinterpret_cast<float2*>(base) + (size_t)(warp - 2) * 32 * SROW;
        const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16);
        for (int cc = 0; cc < ncols; cc += 16) {
            float lr[16], li[16], rr[16], ri[16];
            tmem_ld16(lane_base + (uint32_t)cc, lr);
            tmem_ld16(lane_base + (uint32_t)(BN + cc), li);
            tmem_ld16(lane_base + (uint32_t)(2 * BN + cc), rr);
            tmem_ld16(lane_base + (uint32_t)(3 * BN + cc), ri);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int c = c0 + cc + q;
                const float sc = ldexpf(jb.alpha, eA + (c < d ? eBp[c] : 0) - 3 * SBITS);
                stg[lane * SROW + cc + q] = make_float2((lr[q] + rr[q]) * sc, (li[q] + ri[q]) * sc);
            }
        }
        __syncwarp();
        // eight rows at a time, each lane four columns (c = lane + 32 j): the 32 reads of the
        // accumulated output (beta) are in flight together
        float2* out = jb.out + (size_t)item * jb.ostride;
        const int nrows = min(32, d - (r0 + q4 * 32));
        for (int rw0 = 0; rw0 < nrows; rw0 += 8) {
            float2 old[8][BN / 32];
            if (jb.beta) {
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int j = 0; j < BN / 32; ++j) {
                        const int rw = rw0 + u, c = lane + 32 * j;
                        old[u][j] = (rw < nrows && c < ncols) ? out[(size_t)(r0 + q4 * 32 + rw) * d + c0 + c]
                                                              : make_float2(0.f, 0.f);
                    }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int j = 0; j < BN / 32; ++j) {
                    const int rw = rw0 + u, c = lane + 32 * j;
                    if (rw >= nrows || c >= ncols) continue;
                    const int row = r0 + q4 * 32 + rw;
                    float2 v = stg[rw * SROW + c];
                    if (jb.beta) {
                        v.x += old[u][j].x;
                        v.y += old[u][j].y;
                    }
                    if (jb.ident && row == c0 + c) v.x += 1.0f;
                    out[(size_t)row * d + c0 + c] = v;
                }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn oz_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

size_t oz_plane_bytes(int d, int items) { return (size_t)items * kOzMats * NPART * (size_t)d * oz_ld(d) * 2; }

size_t oz_scratch_bytes(int d, int items) {
    return (oz_plane_bytes(d, items) + 255) / 256 * 256 + (size_t)items * kOzMats * d * 4;
}

cudaError_t oz_make_maps(void* planes, int d, int items, TcMaps* maps) {
    EncodeTiledFn enc = oz_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int ld = oz_ld(d);
    // x: K (d columns of a plane row), y: plane rows (d), z: planes; reads beyond d fill zeros
    cuuint64_t dims[3] = {(cuuint64_t)d, (cuuint64_t)d, (cuuint64_t)items * kOzMats * NPART};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * d * 2};
    cuuint32_t estr[3] = {1, 1, 1};
    cuuint32_t boxA[3] = {BK, BM, 1}, boxB[3] = {BK, BN, 1};
    CUresult r1 = enc(reinterpret_cast<CUtensorMap*>(maps->a), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, planes, dims,
                      strides, boxA, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = enc(reinterpret_cast<CUtensorMap*>(maps->b), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, planes, dims,
                      strides, boxB, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return (r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS) ? cudaSuccess : cudaErrorInvalidValue;
}

// items: the wave's items; cap: the items the plane array was sized for (oz_scratch_bytes)
cudaError_t launch_oz_slice(const OzSliceJobs& jobs, int njobs, int d, int items, int cap, unsigned char* scratch,
                            cudaStream_t st) {
    if (njobs < 1 || njobs > 4 || items > cap) return cudaErrorInvalidValue;
    __nv_bfloat16* planes = reinterpret_cast<__nv_bfloat16*>(scratch);
    int* exps = reinterpret_cast<int*>(scratch + (oz_plane_bytes(d, cap) + 255) / 256 * 256);
    const int gx = std::max((d + 7) / 8, (d + 31) / 32);
    k_oz_slice<<<dim3(gx, items, njobs), 256, 0, st>>>(jobs, planes, exps, d, oz_ld(d));
    return cudaGetLastError();
}

cudaError_t launch_oz_mm(const OzJobs& jobs, int njobs, int d, int items, int cap, unsigned char* scratch,
                         const TcMaps& maps, DevParams* prm, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_oz_mm, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (njobs < 1 || njobs > 2 || d > kMaxD || items > cap) return cudaErrorInvalidValue;
    const int* exps = reinterpret_cast<const int*>(scratch + (oz_plane_bytes(d, cap) + 255) / 256 * 256);
    const int ntiles = ((d + BM - 1) / BM) * ((d + BN - 1) / BN);
    k_oz_mm<<<dim3(ntiles, items, njobs), NTHREADS, OZ_SMEM, st>>>(*reinterpret_cast<const CUtensorMap*>(maps.a),
                                                                   *reinterpret_cast<const CUtensorMap*>(maps.b), jobs,
                                                                   exps, d, prm);
    return cudaGetLastError();
}

cudaError_t oz_rev_step(const OzRev& z, const float2* const ops[4], const size_t strides[4], float2* O1, float2* O2,
                        size_t ms, int mode, int i, cudaStream_t st, int* launches) {
    auto count = [&]() { if (launches) ++*launches; };
    // slices: A1 row (mat 0), B1 column (mat 1), A2 row (mat 2), B2 column (mat 3); in Horner
    // steps A1 is X^dag, sliced once per wave into mat 4
    const bool horner = mode == 0;
    OzSliceJobs sj{};
    int n = 0;
    if (!horner || ops[0] != z.xh || !*z.xh_sliced) {
        const int mat = (horner && ops[0] == z.xh) ? 4 : 0;
        sj.job[n++] = {ops[0], strides[0], mat, 0};
        if (mat == 4) *z.xh_sliced = 1;
    }
    sj.job[n++] = {ops[1], strides[1], 1, 1};
    sj.job[n++] = {ops[2], strides[2], 2, 0};
    sj.job[n++] = {ops[3], strides[3], 3, 1};
    cudaError_t e = launch_oz_slice(sj, n, z.d, z.items, z.cap, z.scratch, st);
    count();
    if (e != cudaSuccess) return e;
    const int a1 = (horner && ops[0] == z.xh) ? 4 : 0;
    if (horner) {   // O1 = A1 B1 / i, O2 += A2 B2 / i
        const float ri = 1.0f / (float)i;
        OzJobs jobs{};
        jobs.fault = z.fault;
        jobs.j[0] = {a1, 1, O1, (long long)ms, ri, 0, 0};
        jobs.j[1] = {2, 3, O2, (long long)ms, ri, 1, 0};
        e = launch_oz_mm(jobs, 2, z.d, z.items, z.cap, z.scratch, z.maps, z.prm, st);
        count();
        return e;
    }
    // squaring: O1 = A1 B1, then O1 += A2 B2
    OzJobs jobs{};
    jobs.fault = z.fault;
    jobs.j[0] = {0, 1, O1, (long long)ms, 1.0f, 0, 0};
    if ((e = launch_oz_mm(jobs, 1, z.d, z.items, z.cap, z.scratch, z.maps, z.prm, st)) != cudaSuccess) return e;
    count();
    jobs.j[0] = {2, 3, O1, (long long)ms, 1.0f, 1, 0};
    e = launch_oz_mm(jobs, 1, z.d, z.items, z.cap, z.scratch, z.maps, z.prm, st);
    count();
    return e;
}

}  // namespace qoc
