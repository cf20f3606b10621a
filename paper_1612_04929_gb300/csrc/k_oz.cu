// Tensor-core products of the large-d adjoint with exact accumulation (BF16_SPLIT form).
//
// The adjoint's block recursion on [[X^dag, Ubar], [0, X^dag]] (the exact derivative of the
// truncated series) needs FP32-level products.  The tensor core's FP32 accumulator truncates,
// and over the Horner and squaring recursion that bias adds up, so the products are made exact
// instead (an integer-slice splitting in the manner of Ozaki's error-free matrix product):
//   * every row of an A operand (every column of a B operand) is scaled by a power of two 2^e
//     with max |entry| < 2^e, and the scaled entry y (|y| < 1) is cut into four slices of six
//     bits, y = sum_s a_s 64^-(s+1) + O(2^-25), with integer a_s in [-64, 64] (stored as BF16,
//     exact);
//   * a product of slices is an integer of at most 2^12 in magnitude; the products of one level
//     l = s + t (s + t <= 3, ten slice pairs) and one complex part (re: Ar Br - Ai Bi,
//     im: Ar Bi + Ai Br) add at most 8 of them per k, so over k < 512 every accumulator holds
//     an integer below 2^24 and the FP32 accumulation is exact whatever its rounding;
//   * the epilogue scales each level by 2^(eA + eB - 6 (l + 2)) (exact) and adds the four levels
//     in FP32.
// The result carries one FP32 rounding per product, unbiased, like an FP32 SIMT product.
//
// One CTA computes a 128 x 32 tile of one output (Z11' or Z12') of one wave item; its one or two
// terms (A, B) each own eight TMEM accumulators of 32 columns (4 levels x re/im).  Operand tiles
// arrive by TMA (SWIZZLE_128B, 64-wide K chunks of all eight slice planes of A and of B); one
// thread issues the loads and the tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulation,
// M = 128, N = 32, K = 16) and commits; the four warps read TMEM back with tcgen05.ld.  Every
// mbarrier wait is bounded; a wait that runs out sets kErrTimeout in DevParams.err.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <utility>

#include "qoc_device.cuh"
#include "qoc_internal.h"

namespace qoc {

namespace {

constexpr int BM = 128, BN = 32, BK = 64;          // BK in BF16 elements (128-byte rows)
constexpr int NSL = 4;                             // six-bit slices per value
constexpr int NPART = 2 * NSL;                     // re slices, then im slices
constexpr int ATILE = BM * BK * 2;                 // 16 KB per plane
constexpr int BTILE = BN * BK * 2;                 // 4 KB per plane
constexpr int STAGE = NPART * (ATILE + BTILE);     // 160 KB
constexpr int OZ_SMEM = STAGE + 1024;              // + alignment slack
constexpr uint32_t TMEM_COLS = 512;                // two terms x 4 levels x (re, im) x 32 columns
constexpr uint32_t WAIT_LIMIT = 1u << 24;
constexpr uint32_t WAIT_LIMIT_TEST = 1u << 12;   // fault-injection runs

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint32_t limit = WAIT_LIMIT) {
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
// UMMA shared-memory descriptor: K-major, SWIZZLE_128B, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(const void* smem) {
    const uint64_t a = su32(smem);
    return ((a >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
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
// four six-bit slices of y = x 2^-e (|y| < 1): y ~ sum_s q[s] 64^-(s+1); every step is exact
__device__ __forceinline__ void slices(float x, int e, float (&q)[NSL]) {
    float r = ldexpf(x, 6 - e);
#pragma unroll
    for (int s = 0; s < NSL; ++s) {
        const float a = rintf(r);
        q[s] = a;
        r = (r - a) * 64.0f;
    }
}

}  // namespace

// plane (item, matrix, part) in the plane array
__host__ __device__ inline size_t oz_plane(int item, int mat, int part) {
    return ((size_t)item * kOzMats + mat) * NPART + part;
}

// ------------------------------------------------------------------------------------------
// slicing: values (FP32 complex, d x d row-major) -> exponents and BF16 slice planes
// ------------------------------------------------------------------------------------------
// Row layout (A operand): plane row r = row r of M, exponent per row.  Column layout (B operand,
// K-major): plane row c = column c of M (conjugation is not applied), exponent per column.
__global__ void __launch_bounds__(256)
k_oz_slice(OzSliceJobs jobs, const float2* __restrict__ vals, __nv_bfloat16* __restrict__ planes, int* __restrict__ exps,
           int d, int ldp) {
    __shared__ float2 tile[32][33];
    __shared__ float cmax[8][32];
    __shared__ int cexp[32];
    const OzSliceJob jb = jobs.job[blockIdx.z];
    const int item = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float2* M = vals + ((size_t)item * kOzVals + jb.val) * d * d;
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
            slices(v.x, e, qr);
            slices(v.y, e, qi);
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
                slices(v.x, cexp[q], qr);
                slices(v.y, cexp[q], qi);
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
// one Horner or squaring step of the block recursion
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 1)
k_oz_step(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzStep step,
          float2* __restrict__ vals, const int* __restrict__ exps, int d, DevParams* __restrict__ prm) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full, empty, done;
    __shared__ uint32_t tmem_holder;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ int skip, s_ok;
    // once a wait has run out in this evaluation, later steps skip their work (the result is
    // reported as QOC_ERR_TIMEOUT); thread 0 decides for the whole CTA
    if (tid == 0) skip = (*(volatile int*)&prm->err & kErrTimeout) != 0;
    __syncthreads();
    if (skip) return;
    const uint32_t limit = step.fault ? WAIT_LIMIT_TEST : WAIT_LIMIT;
    const int item = blockIdx.y, out = blockIdx.z;
    const OzOut oo = step.o[out];
    const int ntn = (d + BN - 1) / BN;
    const int r0 = (blockIdx.x / ntn) * BM, c0 = (blockIdx.x % ntn) * BN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&full, 1);
        mbar_init(&empty, 1);
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;
    const int nk = (d + BK - 1) / BK;
    const int nsteps = oo.nterms * nk;
    bool ok = true;
    if (tid == 0) {
        // instruction descriptor: D f32, A/B bf16, both K-major, N = 32, M = 128
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
        const uint32_t idesc_nA = idesc | (1u << 13);   // negate A
        int loaded = 0;
        auto load = [&](int s) {
            ++loaded;
            const int t = s / nk, kc = s % nk;
            mbar_expect_tx(&full, STAGE);
            for (int part = 0; part < NPART; ++part) {
                tma_3d(base + part * ATILE, &mapA, kc * BK, r0, (int)oz_plane(item, oo.t[t].a_mat, part), &full);
                tma_3d(base + NPART * ATILE + part * BTILE, &mapB, kc * BK, c0, (int)oz_plane(item, oo.t[t].b_mat, part),
                       &full);
            }
        };
        uint32_t started = 0;   // bit (term * 8 + level * 2 + part): accumulator written once
        if (!step.fault) load(0);   // fault injection: the first copy is withheld, its wait runs out
        for (int s = 0; s < nsteps && ok; ++s) {
            ok = mbar_wait(&full, (uint32_t)(s & 1), limit);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int t = s / nk;
            uint64_t Ar[NSL], Ai[NSL], Br[NSL], Bi[NSL];
#pragma unroll
            for (int q = 0; q < NSL; ++q) {
                Ar[q] = sdesc(base + q * ATILE);
                Ai[q] = sdesc(base + (NSL + q) * ATILE);
                Br[q] = sdesc(base + NPART * ATILE + q * BTILE);
                Bi[q] = sdesc(base + NPART * ATILE + (NSL + q) * BTILE);
            }
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 2);   // 32 bytes per K = 16 step, in 16-byte units
#pragma unroll
                for (int sa = 0; sa < NSL; ++sa)
#pragma unroll
                    for (int sb = 0; sb + sa < NSL; ++sb) {
                        const int lvl = sa + sb;
                        const int bit = t * 8 + lvl * 2;
                        const uint32_t acc_re = tmem + (uint32_t)(bit * BN), acc_im = acc_re + BN;
                        const uint32_t fre = (started >> bit) & 1u, fim = (started >> (bit + 1)) & 1u;
                        started |= 3u << bit;
                        // re += Ar Br - Ai Bi ;  im += Ar Bi + Ai Br
                        mma_bf16(acc_re, Ar[sa] + adv, Br[sb] + adv, idesc, fre);
                        mma_bf16(acc_re, Ai[sa] + adv, Bi[sb] + adv, idesc_nA, 1);
                        mma_bf16(acc_im, Ar[sa] + adv, Bi[sb] + adv, idesc, fim);
                        mma_bf16(acc_im, Ai[sa] + adv, Br[sb] + adv, idesc, 1);
                    }
            }
            mma_commit(&empty);
            if (s + 1 < nsteps) {   // refill the stage once its products have completed
                ok = mbar_wait(&empty, (uint32_t)(s & 1), limit);
                if (!ok) break;
                load(s + 1);
            }
        }
        mma_commit(&done);
        if (!ok) {
            atomicOr(&prm->err, kErrTimeout);
            if (loaded > 0) mbar_wait(&full, (uint32_t)((loaded - 1) & 1), limit);   // let the last copy land (bounded)
        }
    }
    if (tid == 0) s_ok = ok ? 1 : 0;   // only the issuing thread knows whether its waits ran out
    __syncthreads();
    const bool fin = mbar_wait(&done, 0, limit);
    if (!fin && tid == 0) atomicOr(&prm->err, kErrTimeout);
    // the epilogue's TMEM loads are warp-collective: the decision is the same for every thread
    const bool go = __syncthreads_and(fin && s_ok != 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (go) {
        const int r = r0 + warp * 32 + lane;
        const bool horner = step.kind == 0;
        const float ri = horner ? 1.0f / (float)step.i : 1.0f;
        int eA[2] = {0, 0};
        if (r < d)
            for (int t = 0; t < oo.nterms; ++t) eA[t] = exps[((size_t)item * kOzMats + oo.t[t].a_mat) * d + r];
        float2* dst = vals + ((size_t)item * kOzVals + oo.val) * d * d;
        for (int cc = 0; cc < BN; cc += 16) {
            float sr[16], si[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) sr[q] = si[q] = 0.f;
            for (int t = 0; t < oo.nterms; ++t) {
                const int* eBp = exps + ((size_t)item * kOzMats + oo.t[t].b_mat) * d;
                for (int lvl = NSL - 1; lvl >= 0; --lvl) {   // smallest level first
                    float vr[16], vi[16];
                    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((t * 8 + lvl * 2) * BN + cc);
                    tmem_ld16(ta, vr);
                    tmem_ld16(ta + BN, vi);
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int c = c0 + cc + q;
                        const int sh = eA[t] + (c < d ? eBp[c] : 0) - 6 * (lvl + 2);
                        sr[q] += ldexpf(vr[q], sh);
                        si[q] += ldexpf(vi[q], sh);
                    }
                }
            }
            if (r < d) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = c0 + cc + q;
                    if (c >= d) break;
                    float re = sr[q] * ri, im = si[q] * ri;
                    if (horner && oo.identity && r == c) re += 1.0f;
                    dst[(size_t)r * d + c] = make_float2(re, im);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// XH = X^dag (X assembled in FP32 from the compute-precision H), Ubar = G Psi^dag,
// Z11 = I + XH / p, Z12 = Ubar / p, as values
__global__ void k_oz_init(const DevParams* __restrict__ prm, SysView<float> sys, StateView<float> sv, int j0, int wlen,
                          const float2* __restrict__ states, const float2* __restrict__ Gbuf, int wmax,
                          float2* __restrict__ vals) {
    const int item = blockIdx.y, jl = item % wlen, e = item / wlen, j = j0 + jl;
    const int d = sys.d, M = sys.M;
    const size_t dd = (size_t)d * d, slice = sv.slice();
    const float s = (float)prm->s, ip = 1.0f / (float)prm->p;
    const float de = sys.delta ? (float)sys.delta[e] : 0.f;
    const float2* Gj = Gbuf + ((size_t)e * wmax + jl) * slice;
    const float2* Pj = states + ((size_t)e * (wmax + 1) + jl) * slice;
    float2* V = vals + (size_t)item * kOzVals * dd;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx / d), b = (int)(idx - (size_t)a * d);
        const size_t o = (size_t)b * d + a;
        float2 h = sys.H0[o];
        for (int k = 0; k < M; ++k) {
            const float uk = (float)sys.u[(size_t)k * sys.N + j];
            const float2 hk = sys.Hk[(size_t)k * dd + o];
            h.x = fmaf(uk, hk.x, h.x);
            h.y = fmaf(uk, hk.y, h.y);
        }
        if (sys.Hdet) {
            const float2 hd = sys.Hdet[o];
            h.x = fmaf(de, hd.x, h.x);
            h.y = fmaf(de, hd.y, h.y);
        }
        const float xr = s * h.y, xi = s * h.x;   // XH[a][b] = conj(-i s H[b][a])
        float ur = 0.f, ui = 0.f;
        for (int sc = 0; sc < sv.S; ++sc) {
            const size_t pa = (size_t)(sc / sv.cb) * sv.pstride + (size_t)a * sv.cb + (sc % sv.cb);
            const size_t pb = (size_t)(sc / sv.cb) * sv.pstride + (size_t)b * sv.cb + (sc % sv.cb);
            const float2 g = Gj[pa], q = Pj[pb];
            ur = fmaf(g.x, q.x, ur);     // g conj(q)
            ur = fmaf(g.y, q.y, ur);
            ui = fmaf(g.y, q.x, ui);
            ui = fmaf(-g.x, q.y, ui);
        }
        V[0 * dd + idx] = make_float2(xr, xi);
        V[1 * dd + idx] = make_float2(ur, ui);
        V[2 * dd + idx] = make_float2(xr * ip + (a == b ? 1.f : 0.f), xi * ip);
        V[4 * dd + idx] = make_float2(ur * ip, ui * ip);
    }
}

// dC/du_{k,j} = s sum_ab (Xbar_re Hk_im - Xbar_im Hk_re), Xbar the final Z12 value
__global__ void __launch_bounds__(256)
k_oz_grad(const DevParams* __restrict__ prm, SysView<float> sys, int j0, int wlen, const float2* __restrict__ vals,
          int xval, double* __restrict__ gpart) {
    __shared__ double red[32];
    const int item = blockIdx.x, k = blockIdx.y, jl = item % wlen, e = item / wlen, j = j0 + jl;
    const int d = sys.d;
    const size_t dd = (size_t)d * d;
    const float2* hk = sys.Hk + (size_t)k * dd;
    const float2* X = vals + ((size_t)item * kOzVals + xval) * dd;
    double v = 0.0;
    for (size_t idx = threadIdx.x; idx < dd; idx += blockDim.x)
        v += (double)X[idx].x * (double)hk[idx].y - (double)X[idx].y * (double)hk[idx].x;
    v = block_sum(v, red);
    if (threadIdx.x == 0) gpart[((size_t)e * sys.M + k) * sys.N + j] = prm->s * v;
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

size_t oz_scratch_bytes(int d, int items) {
    const size_t dd = (size_t)d * d;
    return (size_t)items * (kOzMats * NPART * (size_t)d * oz_ld(d) * 2   // slice planes
                            + kOzMats * (size_t)d * 4                     // exponents
                            + kOzVals * dd * 8);                          // values
}

cudaError_t oz_make_maps(void* planes, int d, int items, TcMaps* maps) {
    EncodeTiledFn enc = oz_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int ld = oz_ld(d);
    cuuint64_t dims[3] = {(cuuint64_t)d, (cuuint64_t)d, (cuuint64_t)items * kOzMats * NPART};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * d * 2};
    cuuint32_t estr[3] = {1, 1, 1};
    cuuint32_t boxA[3] = {BK, BM, 1}, boxB[3] = {BK, BN, 1};
    CUresult r1 = enc(reinterpret_cast<CUtensorMap*>(maps->a), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, planes, dims,
                      strides, boxA, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = enc(reinterpret_cast<CUtensorMap*>(maps->b), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, planes, dims,
                      strides, boxB, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return (r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS) ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_oz_adj(const OzAdjArgs& a, cudaStream_t st, int* launches) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_oz_step, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    auto count = [&]() { if (launches) ++*launches; };
    const int d = a.d, items = a.wlen * a.E, ld = oz_ld(d);
    if (d > kMaxD) return cudaErrorInvalidValue;
    const size_t dd = (size_t)d * d;
    const size_t pbytes = (size_t)items * kOzMats * NPART * (size_t)d * ld * 2;
    __nv_bfloat16* planes = reinterpret_cast<__nv_bfloat16*>(a.scratch);
    int* exps = reinterpret_cast<int*>(a.scratch + pbytes);
    float2* vals = reinterpret_cast<float2*>(a.scratch + pbytes + (((size_t)items * kOzMats * d * 4 + 255) / 256) * 256);
    // plane matrices: 0 XH (row), 1 Ubar (row), then per set q: Z11 row/col, Z12 row/col
    auto z11r = [](int q) { return 2 + 4 * q; };
    auto z11c = [](int q) { return 3 + 4 * q; };
    auto z12r = [](int q) { return 4 + 4 * q; };
    auto z12c = [](int q) { return 5 + 4 * q; };
    // values: 0 XH, 1 Ubar, 2 / 3 Z11 of set 0 / 1, 4 / 5 Z12 of set 0 / 1
    const int eb = (int)std::min<size_t>(64, (dd + 255) / 256);
    k_oz_init<<<dim3(eb, items), 256, 0, st>>>(a.prm, a.sys, a.sv, a.j0, a.wlen, a.states, a.Gbuf, a.wmax, vals);
    count();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    auto slice = [&](std::initializer_list<OzSliceJob> js) {
        OzSliceJobs J{};
        int n = 0;
        for (const OzSliceJob& j : js) J.job[n++] = j;
        const int gx = std::max((d + 7) / 8, (d + 31) / 32);
        k_oz_slice<<<dim3(gx, items, n), 256, 0, st>>>(J, vals, planes, exps, d, ld);
        count();
        return cudaGetLastError();
    };
    if ((err = slice({{0, 0, 0}, {1, 1, 0}, {2, z11r(0), 0}, {2, z11c(0), 1}, {4, z12r(0), 0}, {4, z12c(0), 1}})) !=
        cudaSuccess)
        return err;
    const CUtensorMap* mapA = reinterpret_cast<const CUtensorMap*>(a.maps.a);
    const CUtensorMap* mapB = reinterpret_cast<const CUtensorMap*>(a.maps.b);
    const int ntiles = ((d + BM - 1) / BM) * ((d + BN - 1) / BN);
    int q = 0;   // current set
    auto run = [&](int kind, int i, bool last) {
        OzStep s{};
        s.kind = kind;
        s.i = i;
        const int n = 1 - q;
        s.o[0].val = 2 + n;
        s.o[0].identity = 1;
        s.o[1].val = 4 + n;
        s.o[1].identity = 0;
        if (kind == 0) {   // Horner: Z11' = I + XH Z11 / i, Z12' = (XH Z12 + Ubar Z11) / i
            s.o[0].nterms = 1;
            s.o[0].t[0] = {0, z11c(q)};
            s.o[1].nterms = 2;
            s.o[1].t[0] = {0, z12c(q)};
            s.o[1].t[1] = {1, z11c(q)};
        } else {           // squaring: Z11' = Z11 Z11, Z12' = Z11 Z12 + Z12 Z11
            s.o[0].nterms = 1;
            s.o[0].t[0] = {z11r(q), z11c(q)};
            s.o[1].nterms = 2;
            s.o[1].t[0] = {z11r(q), z12c(q)};
            s.o[1].t[1] = {z12r(q), z11c(q)};
        }
        s.fault = a.fault;
        k_oz_step<<<dim3(ntiles, items, 2), 128, OZ_SMEM, st>>>(*mapA, *mapB, s, vals, exps, d, a.prm);
        count();
        cudaError_t e2 = cudaGetLastError();
        if (e2 != cudaSuccess) return e2;
        q = n;
        if (last) return cudaSuccess;   // the final Z12 is Xbar; nothing multiplies it again
        return slice({{2 + q, z11r(q), 0}, {2 + q, z11c(q), 1}, {4 + q, z12r(q), 0}, {4 + q, z12c(q), 1}});
    };
    const int nsteps = (a.p - 1) + a.n;
    int done = 0;
    for (int i = a.p - 1; i >= 1; --i)
        if ((err = run(0, i, ++done == nsteps)) != cudaSuccess) return err;
    for (int m = 0; m < a.n; ++m)
        if ((err = run(1, 0, ++done == nsteps)) != cudaSuccess) return err;
    if (a.sys.M > 0) {
        k_oz_grad<<<dim3(items, a.sys.M), 256, 0, st>>>(a.prm, a.sys, a.j0, a.wlen, vals, 4 + q, a.gpart);
        count();
    }
    return cudaGetLastError();
}

}  // namespace qoc
