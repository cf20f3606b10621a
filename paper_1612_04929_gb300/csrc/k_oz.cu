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
// The forward products of the Paterson-Stockmeyer form (X^2, X^3, the chain products, the
// squarings; Eqs. 9-10) need the accuracy of the split SIMT products (about 2^-36 of the scale),
// so there the operands are value pairs cut into six seven-bit slices (42 bits), and the slice
// levels s + t = 0, 1 and 2 accumulate exactly in accumulators of their own (pre-weighted by
// 2^(7 - 7 (s + t)), level L is a multiple of 2^(7 - 7L); per k and complex part at most two
// products of 2^21, 2^14 and 2^14.3 for L = 0, 1, 2, so the sums stay below 2^24 units of their
// granularity for d <= 384), the levels 3 to 5 into a fourth.  That last accumulator is the only
// inexact one: the tensor core's accumulation truncates, and in emulation of a truncating FP32
// accumulator per MMA the product of two identity-dominant matrices keeps a relative error of
// 1.5e-11 (with levels 2 to 5 in one accumulator: 7.9e-9).  128 x 64 tiles keep the eight FP32
// accumulators within the tensor memory, and the epilogue adds the Paterson-Stockmeyer block in
// pair arithmetic and writes grid-split value pairs.
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

constexpr int BM = 128, BK = 16;                   // BK in BF16 elements: 32-byte rows
constexpr int SBITS = 7;
constexpr int NTHREADS = 192;                      // producer warp, MMA warp, four epilogue warps

// One product configuration: NS slices per value, BN-wide tiles, NLEV accumulator levels (every
// level below NLEV - 1 exact, the last one taking the remaining slice pairs), NST stages.
template <int NS_, int BN_, int NLEV_, int NST_>
struct OzCfg {
    static constexpr int NS = NS_, BN = BN_, NLEV = NLEV_, NST = NST_;
    static constexpr int NPART = 2 * NS;                      // re slices, then im slices
    static constexpr int TILE_A = BM * BK * 2;                // one A plane tile, 4 KB
    static constexpr int TILE_B = BN * BK * 2;                // one B plane tile
    static constexpr int STAGE = NPART * (TILE_A + TILE_B);
    static constexpr int SMEM = NST * STAGE + 1024;           // + alignment slack
    static constexpr uint32_t TMEM_COLS = 512;
};
using AdjCfg = OzCfg<kOzSlices, 128, 2, 3>;     // 64 KB stages, four 128-column accumulators
using FwdCfg = OzCfg<kOzFwdSlices, 64, 4, 3>;   // 72 KB stages, eight 64-column accumulators
static_assert(2 * AdjCfg::NLEV * AdjCfg::BN <= 512 && 2 * FwdCfg::NLEV * FwdCfg::BN <= 512, "tensor memory");
static_assert(AdjCfg::SMEM <= (int)kMaxDynSmem && FwdCfg::SMEM <= (int)kMaxDynSmem, "shared memory");
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
// NS seven-bit slices of y = (hi + lo) 2^-e (|y| < 1), weighted for their operand role: A planes
// hold a_s 2^(7 - 7 s), B planes b_s 2^(-7 s).  The pair is normalised first (a grid-split pair
// on a grid much coarser than the row's largest value has a low part far above the high part's
// last bit, which would push the slices past the eight bits BF16 holds exactly); the residual is
// then carried as an error-free pair: a_s = rint(H), (H, L) <- TwoSum(H - a_s, L) 2^7, exact at
// every step (lo = 0 for FP32 values).
template <int NS>
__device__ __forceinline__ void slices(float hi, float lo, int e, bool role_a, float (&q)[NS]) {
    float h0, l0;
    two_sum(hi, lo, h0, l0);
    float h = ldexpf(h0, SBITS - e), l = ldexpf(l0, SBITS - e);
    float w = role_a ? (float)(1 << SBITS) : 1.0f;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const float a = rintf(h);
        q[s] = a * w;
        float t, u;
        two_sum(h - a, l, t, u);
        h = t * (float)(1 << SBITS);
        l = u * (float)(1 << SBITS);
        w *= 1.0f / (float)(1 << SBITS);
    }
}
// a complex element as value pairs (re_hi, re_lo, im_hi, im_lo)
__device__ __forceinline__ float4 as_pairs(float2 v) { return make_float4(v.x, 0.f, v.y, 0.f); }
__device__ __forceinline__ float4 as_pairs(float4 v) { return make_float4(v.x, v.z, v.y, v.w); }

}  // namespace

// plane (item, matrix, part) in a plane array of NPART planes per matrix
template <int NPART>
__host__ __device__ inline size_t oz_plane(int item, int mat, int part) {
    return ((size_t)item * kOzMats + mat) * NPART + part;
}

// ------------------------------------------------------------------------------------------
// slicing: FP32 complex d x d matrices (row-major, item-strided) -> exponents and BF16 planes
// ------------------------------------------------------------------------------------------
// Row layout (A operand): plane row r = row r of M, exponent per row.  Column layout (B operand,
// K-major): plane row c = column c of M, exponent per column (no conjugation is applied).
// Eight consecutive elements of one plane row, as one 16-byte store (the plane rows are padded to
// a multiple of eight elements and start on 16-byte boundaries)
__device__ __forceinline__ void store8(__nv_bfloat16* dst, const float (&v)[8]) {
    uint4 w;
    __nv_bfloat162 h;
    h = __floats2bfloat162_rn(v[0], v[1]);
    w.x = *reinterpret_cast<uint32_t*>(&h);
    h = __floats2bfloat162_rn(v[2], v[3]);
    w.y = *reinterpret_cast<uint32_t*>(&h);
    h = __floats2bfloat162_rn(v[4], v[5]);
    w.z = *reinterpret_cast<uint32_t*>(&h);
    h = __floats2bfloat162_rn(v[6], v[7]);
    w.w = *reinterpret_cast<uint32_t*>(&h);
    *reinterpret_cast<uint4*>(dst) = w;
}

// the slices of eight consecutive elements of one plane row (k0 .. k0 + 7; zero past d), written
// as 16-byte stores into the row's 2 NS planes
template <int NS>
__device__ __forceinline__ void put8(__nv_bfloat16* __restrict__ planes, size_t pbase, size_t psz, size_t rowoff,
                                     const float4 (&q)[8], int e, bool role_a) {
    float sr[8][NS], si[8][NS];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        slices<NS>(q[i].x, q[i].y, e, role_a, sr[i]);
        slices<NS>(q[i].z, q[i].w, e, role_a, si[i]);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        float vr[8], vi[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            vr[i] = sr[i][s];
            vi[i] = si[i][s];
        }
        store8(planes + (pbase + s) * psz + rowoff, vr);
        store8(planes + (pbase + NS + s) * psz + rowoff, vi);
    }
}

template <int NS, typename In>
__global__ void __launch_bounds__(256)
k_oz_slice(OzSliceJobs jobs, __nv_bfloat16* __restrict__ planes, int* __restrict__ exps, int d, int ldp) {
    constexpr int NPART = 2 * NS;
    constexpr int KT = 64;                       // rows of M per staged tile (column layout)
    __shared__ float4 tile[KT][33];
    __shared__ float cmax[8][32];
    __shared__ int cexp[32];
    const OzSliceJob jb = jobs.job[blockIdx.z];
    const int item = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const In* M = static_cast<const In*>(jb.src) + (size_t)item * jb.stride;
    const size_t psz = (size_t)d * ldp;
    const size_t pbase = oz_plane<NPART>(item, jb.mat, 0);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // the exponent comes from the rounded values |re|, |im| (a pair's sum rounded up to 2^e only
    // raises e: conservative)
    auto mag = [](float4 q) { return fmaxf(fabsf(q.x + q.y), fabsf(q.z + q.w)); };
    if (!jb.col) {
        // row layout: one warp per row, each lane eight consecutive columns per 256-column chunk
        // (d <= 512: at most two chunks, held in registers between the maximum and the slicing)
        const int r = blockIdx.x * 8 + warp;
        if (r >= d) return;
        float4 v[2][8];
        float m = 0.f;
#pragma unroll
        for (int ch = 0; ch < 2; ++ch)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int b = ch * 256 + lane * 8 + i;
                v[ch][i] = b < d ? as_pairs(M[(size_t)r * d + b]) : zero4;
                m = fmaxf(m, mag(v[ch][i]));
            }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const int e = scale_exp(m);
        if (lane == 0) exps[((size_t)item * kOzMats + jb.mat) * d + r] = e;
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
            const int b0 = ch * 256 + lane * 8;
            if (b0 < d) put8<NS>(planes, pbase, psz, (size_t)r * ldp + b0, v[ch], e, true);
        }
        return;
    }
    // column layout: 32 columns c0 .. c0 + 31 per CTA; plane row c (a column of M) with k along it
    const int c0 = blockIdx.x * 32;
    if (c0 >= d) return;
    const int c = c0 + lane;
    float m = 0.f;
    if (c < d)
        for (int k = warp; k < d; k += 8) m = fmaxf(m, mag(as_pairs(M[(size_t)k * d + c])));
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
    // tiles of KT rows: staged with the lanes along the columns (coalesced reads), then thread t
    // slices column t % 32 over the eight rows 8 (t / 32) .. + 7 of the tile
    const int tc = tid & 31, tk = (tid >> 5) * 8;
    for (int k0 = 0; k0 < d; k0 += KT) {
        for (int q = warp; q < KT; q += 8) {
            const int k = k0 + q;
            tile[q][lane] = (k < d && c < d) ? as_pairs(M[(size_t)k * d + c]) : zero4;
        }
        __syncthreads();
        const int cc = c0 + tc, kk = k0 + tk;
        if (cc < d && kk < d) {
            float4 q8[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) q8[i] = tile[tk + i][tc];
            put8<NS>(planes, pbase, psz, (size_t)cc * ldp + kk, q8, cexp[tc], false);
        }
        __syncthreads();
    }
}

// The forward epilogue's job: out = A B (kind 1) or A B + c0 I + c1 X + c2 X^2 (kind 2), written as
// value pairs grid-split with `magic` (item stride ostride)
struct OzFwdEpi {
    float4* out;
    long long ostride;
    int kind;
    float magic;
    const float4* X;
    const float4* X2;
    float2 c0, c1, c2;
};

// ------------------------------------------------------------------------------------------
// one 128 x BN output tile for job blockIdx.z, item blockIdx.y: adjoint products (FWD false)
// C = alpha A B (+ beta C) (+ I) in FP32; forward products (FWD true) as value pairs (OzFwdEpi)
// ------------------------------------------------------------------------------------------
template <class Cfg, bool FWD>
__global__ void __launch_bounds__(NTHREADS, 1)
k_oz_mm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzJobs jobs,
        OzFwdEpi fe, const int* __restrict__ exps, int d, DevParams* __restrict__ prm) {
    constexpr int NS = Cfg::NS, BN = Cfg::BN, NLEV = Cfg::NLEV, NST = Cfg::NST, NPART = Cfg::NPART;
    constexpr int TILE_A = Cfg::TILE_A, TILE_B = Cfg::TILE_B, STAGE = Cfg::STAGE;
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
                     "r"(Cfg::TMEM_COLS)
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
        // ---- producer: the NPART A planes and NPART B planes of one K chunk per stage ----
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
                tma_3d(st + part * TILE_A, &mapA, s * BK, r0, (int)oz_plane<NPART>(item, jb.a_mat, part), &full[b]);
                tma_3d(st + NPART * TILE_A + part * TILE_B, &mapB, s * BK, c0,
                       (int)oz_plane<NPART>(item, jb.b_mat, part), &full[b]);
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
        // instruction descriptor: D f32, A/B bf16, both K-major, N = BN, M = 128
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
        const uint32_t idesc_nA = idesc | (1u << 13);   // negate A
        bool ok = true;
        for (int s = 0; s < nk; ++s) {
            const int b = s % NST;
            if (!mbar_wait(&full[b], (uint32_t)((s / NST) & 1), limit)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned char* st = base + b * STAGE;
            uint64_t Ar[NS], Ai[NS], Br[NS], Bi[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                Ar[q] = sdesc(st + q * TILE_A);
                Ai[q] = sdesc(st + (NS + q) * TILE_A);
                Br[q] = sdesc(st + NPART * TILE_A + q * TILE_B);
                Bi[q] = sdesc(st + NPART * TILE_A + (NS + q) * TILE_B);
            }
#pragma unroll
            for (int sa = 0; sa < NS; ++sa)
#pragma unroll
                for (int sb = 0; sb + sa < NS; ++sb) {
                    // slice level sa + sb goes to its own accumulator below NLEV - 1, the rest to the
                    // last; the first MMA into each accumulator (sa = 0, sb = its level) overwrites it
                    const int lev = sa + sb < NLEV ? sa + sb : NLEV - 1;
                    const bool first = sa == 0 && sb == lev;
                    const uint32_t en = (s > 0 || !first) ? 1u : 0u;
                    const uint32_t acc_re = tmem + (uint32_t)(2 * lev * BN), acc_im = acc_re + BN;
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
        const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16);
        const int nrows = min(32, d - (r0 + q4 * 32));
        if constexpr (!FWD) {
            float2* stg = reinterpret_cast<float2*>(base) + (size_t)(warp - 2) * 32 * SROW;
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
        } else {
            // value pairs (re_hi, im_hi, re_lo, im_lo): the three exact levels summed without
            // error, the remainder level added to the low part; every scaling is by a power of two
            static_assert(NLEV == 4, "three exact levels and a remainder");
            float4* stg = reinterpret_cast<float4*>(base) + (size_t)(warp - 2) * 32 * SROW;
            for (int cc = 0; cc < ncols; cc += 16) {
#pragma unroll
                for (int part = 0; part < 2; ++part) {   // re, then im
                    float a0[16], a1[16], a2[16], a3[16];
                    tmem_ld16(lane_base + (uint32_t)(part * BN + cc), a0);
                    tmem_ld16(lane_base + (uint32_t)((2 + part) * BN + cc), a1);
                    tmem_ld16(lane_base + (uint32_t)((4 + part) * BN + cc), a2);
                    tmem_ld16(lane_base + (uint32_t)((6 + part) * BN + cc), a3);
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int c = c0 + cc + q;
                        const float sc = ldexpf(1.0f, eA + (c < d ? eBp[c] : 0) - 3 * SBITS);
                        float h, l, h2, l2;
                        two_sum(a0[q] * sc, a1[q] * sc, h, l);
                        two_sum(h, a2[q] * sc, h2, l2);
                        h = h2;
                        l = fmaf(a3[q], sc, l + l2);
                        float4& o = stg[lane * SROW + cc + q];
                        if (part == 0) {
                            o.x = h;
                            o.z = l;
                        } else {
                            o.y = h;
                            o.w = l;
                        }
                    }
                }
            }
            __syncwarp();
            // four rows at a time, each lane BN / 32 columns; the block terms' reads in flight together
            float4* out = fe.out + (size_t)item * fe.ostride;
            const size_t ioff = (size_t)item * fe.ostride;
            for (int rw0 = 0; rw0 < nrows; rw0 += 4) {
                float4 xv[4][BN / 32], yv[4][BN / 32];
                if (fe.kind == 2) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int j = 0; j < BN / 32; ++j) {
                            const int rw = rw0 + u, c = lane + 32 * j;
                            const bool in = rw < nrows && c < ncols;
                            const size_t o = ioff + (size_t)(r0 + q4 * 32 + rw) * d + c0 + c;
                            xv[u][j] = in ? fe.X[o] : make_float4(0.f, 0.f, 0.f, 0.f);
                            yv[u][j] = in ? fe.X2[o] : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int j = 0; j < BN / 32; ++j) {
                        const int rw = rw0 + u, c = lane + 32 * j;
                        if (rw >= nrows || c >= ncols) continue;
                        const int row = r0 + q4 * 32 + rw;
                        const float4 v = stg[rw * SROW + c];
                        float rh = v.x, rl = v.z, ih = v.y, il = v.w;
                        if (fe.kind == 2) {
                            pair_fma(rh, rl, fe.c1, xv[u][j].x, xv[u][j].z);
                            pair_fma(ih, il, fe.c1, xv[u][j].y, xv[u][j].w);
                            pair_fma(rh, rl, fe.c2, yv[u][j].x, yv[u][j].z);
                            pair_fma(ih, il, fe.c2, yv[u][j].y, yv[u][j].w);
                            if (row == c0 + c) df_addc(rh, rl, fe.c0);
                        }
                        float4 o;
                        grid_split(rh, rl, fe.magic, o.x, o.z);
                        grid_split(ih, il, fe.magic, o.y, o.w);
                        out[(size_t)row * d + c0 + c] = o;
                    }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS) : "memory");
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

template <class Cfg>
static size_t plane_bytes(int d, int items) {
    return (size_t)items * kOzMats * Cfg::NPART * (size_t)d * oz_ld(d) * 2;
}
template <class Cfg>
static size_t scratch_bytes(int d, int items) {
    return (plane_bytes<Cfg>(d, items) + 255) / 256 * 256 + (size_t)items * kOzMats * d * 4;
}
template <class Cfg>
static int* exps_of(unsigned char* scratch, int d, int cap) {
    return reinterpret_cast<int*>(scratch + (plane_bytes<Cfg>(d, cap) + 255) / 256 * 256);
}

template <class Cfg>
static cudaError_t make_maps(void* planes, int d, int items, TcMaps* maps) {
    EncodeTiledFn enc = oz_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int ld = oz_ld(d);
    // x: K (d columns of a plane row), y: plane rows (d), z: planes; reads beyond d fill zeros
    cuuint64_t dims[3] = {(cuuint64_t)d, (cuuint64_t)d, (cuuint64_t)items * kOzMats * Cfg::NPART};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * d * 2};
    cuuint32_t estr[3] = {1, 1, 1};
    cuuint32_t boxA[3] = {BK, BM, 1}, boxB[3] = {BK, (cuuint32_t)Cfg::BN, 1};
    CUresult r1 = enc(reinterpret_cast<CUtensorMap*>(maps->a), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, planes, dims,
                      strides, boxA, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = enc(reinterpret_cast<CUtensorMap*>(maps->b), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, planes, dims,
                      strides, boxB, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return (r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS) ? cudaSuccess : cudaErrorInvalidValue;
}

template <class Cfg, typename In>
static cudaError_t slice_launch(const OzSliceJobs& jobs, int njobs, int d, int items, int cap, unsigned char* scratch,
                                cudaStream_t st) {
    if (njobs < 1 || njobs > 4 || items > cap) return cudaErrorInvalidValue;
    __nv_bfloat16* planes = reinterpret_cast<__nv_bfloat16*>(scratch);
    const int gx = std::max((d + 7) / 8, (d + 31) / 32);
    k_oz_slice<Cfg::NS, In><<<dim3(gx, items, njobs), 256, 0, st>>>(jobs, planes, exps_of<Cfg>(scratch, d, cap), d,
                                                                    oz_ld(d));
    return cudaGetLastError();
}

template <class Cfg, bool FWD>
static cudaError_t mm_launch(const OzJobs& jobs, int njobs, const OzFwdEpi& fe, int d, int items, int cap,
                             unsigned char* scratch, const TcMaps& maps, DevParams* prm, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_oz_mm<Cfg, FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (njobs < 1 || njobs > 2 || d > kMaxD || items > cap) return cudaErrorInvalidValue;
    const int ntiles = ((d + BM - 1) / BM) * ((d + Cfg::BN - 1) / Cfg::BN);
    k_oz_mm<Cfg, FWD><<<dim3(ntiles, items, njobs), NTHREADS, Cfg::SMEM, st>>>(
        *reinterpret_cast<const CUtensorMap*>(maps.a), *reinterpret_cast<const CUtensorMap*>(maps.b), jobs, fe,
        exps_of<Cfg>(scratch, d, cap), d, prm);
    return cudaGetLastError();
}

size_t oz_plane_bytes(int d, int items) { return plane_bytes<AdjCfg>(d, items); }
size_t oz_scratch_bytes(int d, int items) { return scratch_bytes<AdjCfg>(d, items); }
cudaError_t oz_make_maps(void* planes, int d, int items, TcMaps* maps) { return make_maps<AdjCfg>(planes, d, items, maps); }

// items: the wave's items; cap: the items the plane array was sized for (oz_scratch_bytes)
cudaError_t launch_oz_slice(const OzSliceJobs& jobs, int njobs, int d, int items, int cap, unsigned char* scratch,
                            cudaStream_t st) {
    return slice_launch<AdjCfg, float2>(jobs, njobs, d, items, cap, scratch, st);
}

cudaError_t launch_oz_mm(const OzJobs& jobs, int njobs, int d, int items, int cap, unsigned char* scratch,
                         const TcMaps& maps, DevParams* prm, cudaStream_t st) {
    return mm_launch<AdjCfg, false>(jobs, njobs, OzFwdEpi{}, d, items, cap, scratch, maps, prm, st);
}

size_t oz_fwd_scratch_bytes(int d, int items) { return scratch_bytes<FwdCfg>(d, items); }
cudaError_t oz_fwd_make_maps(void* planes, int d, int items, TcMaps* maps) {
    return make_maps<FwdCfg>(planes, d, items, maps);
}

cudaError_t oz_fwd_product(const OzFwd& z, const float4* a_src, int a_mat, const float4* b_src, int b_mat,
                           float4* out, size_t ms, int kind, float magic, const float4* X, const float4* X2, float2 c0,
                           float2 c1, float2 c2, cudaStream_t st, int* launches) {
    auto count = [&]() { if (launches) ++*launches; };
    if (magic == 0.f || (kind == 2 && (!X || !X2))) return cudaErrorInvalidValue;
    OzSliceJobs sj{};
    int n = 0;
    if (a_src) sj.job[n++] = {a_src, ms, a_mat, 0};
    if (b_src) sj.job[n++] = {b_src, ms, b_mat, 1};
    cudaError_t e;
    if (n) {
        if ((e = slice_launch<FwdCfg, float4>(sj, n, z.d, z.items, z.cap, z.scratch, st)) != cudaSuccess) return e;
        count();
    }
    OzJobs jobs{};
    jobs.fault = z.fault;
    jobs.j[0] = {a_mat, b_mat, nullptr, 0, 1.0f, 0, 0};
    OzFwdEpi fe{out, (long long)ms, kind, magic, X, X2, c0, c1, c2};
    e = mm_launch<FwdCfg, true>(jobs, 1, fe, z.d, z.items, z.cap, z.scratch, z.maps, z.prm, st);
    count();
    return e;
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
