// Tensor-core (tcgen05) products of the large-d adjoint in the TF32_SPLIT form.
//
// The exact adjoint of the truncated series (block recursion on [[X^dag, Ubar], [0, X^dag]])
// tolerates FP32-level rounding, so its complex d x d products run on the 5th-generation tensor
// cores.  Each complex matrix is kept as six planes, real and imaginary parts each split as
// x = hi + mid + lo with every term rounded to nearest TF32 (so the tensor core's truncation of
// its inputs never applies), in two layouts: row-major ("row", the A
// operand, K contiguous) and transposed ("col", the B operand, also K contiguous).  One CTA
// computes a 128 x 64 tile of up to two complex accumulators for one wave item:
//   C_re += Ar Br - Ai Bi,  C_im += Ar Bi + Ai Br,  each real product from the six largest
//   split terms (hh, hm, mh, hl, lh, mm: six TF32 MMAs, FP32 accumulation in TMEM), over the
//   K-chunks of one to three terms.  The tensor core's FP32 accumulation does not round to
//   nearest, and over the Horner and squaring recursion its error adds up coherently; the hh
//   products therefore accumulate in their own TMEM columns, apart from the small correction
//   products, and the epilogue adds the two in FP32.
// Operand tiles arrive by TMA (SWIZZLE_128B, K-chunks of 32) into a shared-memory stage; one thread
// issues the TMA loads and the tcgen05.mma instructions; tcgen05.commit releases ring stages
// and signals the epilogue, which reads TMEM with tcgen05.ld, applies the Horner or squaring
// update and writes the split planes of the result in both layouts.
// Every mbarrier wait is bounded; a wait that runs out sets kErrTimeout in DevParams.err.
#include <cuda.h>

#include <algorithm>
#include <utility>

#include "qoc_device.cuh"
#include "qoc_internal.h"

namespace qoc {

namespace {

constexpr int BM = 128, BN = 64, BK = 32;
constexpr int NPL = kTcSplit;                      // TF32 terms per real value (hi, mid, lo)
constexpr int ATILE = BM * BK * 4;                 // 16 KB
constexpr int BTILE = BN * BK * 4;                 // 8 KB
constexpr int STAGE = 2 * NPL * (ATILE + BTILE);   // re and im planes of A and B: 144 KB
constexpr int NST = 1;                             // ring stages that fit in shared memory
constexpr int TC_SMEM = NST * STAGE + 1024;        // + alignment slack
constexpr uint32_t TMEM_COLS = 512;                // two complex accumulators of 64 columns, each twice
constexpr uint32_t CORR = 256;                     // column offset of the correction accumulators
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
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
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
__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// x = p[0] + p[1] + p[2] (+ a remainder below 2^-33 |x|), each part rounded to nearest TF32
__device__ __forceinline__ void split_tf32(float x, float* p) {
    const float h = tf32_hi(x);
    const float m = tf32_hi(x - h);
    p[0] = h;
    p[1] = m;
    p[2] = tf32_hi((x - h) - m);
}

}  // namespace

// plane of (item, matrix, part) in the plane array
__host__ __device__ inline size_t tc_plane(int item, int mat, int part, int nmat) {
    return ((size_t)item * nmat + mat) * (2 * kTcSplit) + part;
}

__global__ void __launch_bounds__(128, 1)
k_tc_step(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, float* __restrict__ planes,
          TcStep step, int d, int ld, int nmat, DevParams* __restrict__ prm) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[NST], empty[NST], done;
    __shared__ uint32_t tmem_holder;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ int skip, s_ok;
    // once a wait has run out in this evaluation, later steps skip their work (the result is
    // reported as QOC_ERR_TIMEOUT); thread 0 decides for the whole CTA
    if (tid == 0) skip = (*(volatile int*)&prm->err & kErrTimeout) != 0;
    __syncthreads();
    if (skip) return;
    const uint32_t limit = step.fault ? WAIT_LIMIT_TEST : WAIT_LIMIT;
    const int item = blockIdx.y;
    const int ntn = (d + BN - 1) / BN;
    const int r0 = (blockIdx.x / ntn) * BM, c0 = (blockIdx.x % ntn) * BN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < NST; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;
    const int nk = (d + BK - 1) / BK;
    const int nsteps = step.nterms * nk;
    bool ok = true;
    if (tid == 0) {
        // instruction descriptor: D f32, A/B tf32, both K-major, N = 64, M = 128
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
        const uint32_t idesc_nA = idesc | (1u << 13);   // negate A
        int last_issued[NST];   // per ring stage: the last step whose copy was issued (-1: none)
#pragma unroll
        for (int b2 = 0; b2 < NST; ++b2) last_issued[b2] = -1;
        auto load = [&](int s) {   // planes: A re (NPL), A im (NPL), B re (NPL), B im (NPL)
            const int t = s / nk, kc = s % nk, b = s % NST;
            last_issued[b] = s;
            unsigned char* st = base + b * STAGE;
            mbar_expect_tx(&full[b], STAGE);
            for (int part = 0; part < 2 * NPL; ++part) {
                tma_3d(st + part * ATILE, &mapA, kc * BK, r0, (int)tc_plane(item, step.t[t].a_mat, part, nmat), &full[b]);
                tma_3d(st + 2 * NPL * ATILE + part * BTILE, &mapB, kc * BK, c0,
                       (int)tc_plane(item, step.t[t].b_mat, part, nmat), &full[b]);
            }
        };
        bool started[2] = {false, false};
        for (int q = 0; q < NST && q < nsteps; ++q)
            if (!(step.fault && q == 0)) load(q);   // fault injection: the first copy is withheld
        // products kept of (x_h + x_m + x_l)(y_h + y_m + y_l): hh, hm, mh, hl, lh, mm
        const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
        for (int s = 0; s < nsteps && ok; ++s) {
            const int b = s % NST;
            ok = mbar_wait(&full[b], (uint32_t)((s / NST) & 1), limit);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int t = s / nk, acc = step.t[t].acc;
            const unsigned char* st = base + b * STAGE;
            // hh products accumulate apart from the five small correction products, so that the
            // large accumulator sees few of the tensor core's FP32 accumulation roundings
            const uint32_t d_re = tmem + (uint32_t)(acc * 2 * BN), d_im = d_re + BN;
            const uint32_t c_re = d_re + CORR, c_im = d_im + CORR;
            uint64_t Ar[NPL], Ai[NPL], Br[NPL], Bi[NPL];
#pragma unroll
            for (int q = 0; q < NPL; ++q) {
                Ar[q] = sdesc(st + q * ATILE);
                Ai[q] = sdesc(st + (NPL + q) * ATILE);
                Br[q] = sdesc(st + 2 * NPL * ATILE + q * BTILE);
                Bi[q] = sdesc(st + 2 * NPL * ATILE + (NPL + q) * BTILE);
            }
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 2);   // 32 bytes per K = 8 step, in 16-byte units
                const uint32_t first = started[acc] ? 1u : 0u;
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const uint32_t acc_flag = (q <= 1) ? first : 1u;
                    const uint32_t o_re = q == 0 ? d_re : c_re, o_im = q == 0 ? d_im : c_im;
                    // C_re += Ar Br - Ai Bi ;  C_im += Ar Bi + Ai Br
                    mma_tf32(o_re, Ar[pa[q]] + adv, Br[pb[q]] + adv, idesc, acc_flag);
                    mma_tf32(o_re, Ai[pa[q]] + adv, Bi[pb[q]] + adv, idesc_nA, 1);
                    mma_tf32(o_im, Ar[pa[q]] + adv, Bi[pb[q]] + adv, idesc, acc_flag);
                    mma_tf32(o_im, Ai[pa[q]] + adv, Br[pb[q]] + adv, idesc, 1);
                }
                started[acc] = true;
            }
            mma_commit(&empty[b]);
            if (s + NST < nsteps) {   // refill this stage once its products have completed
                ok = mbar_wait(&empty[b], (uint32_t)((s / NST) & 1), limit);
                if (!ok) break;
                load(s + NST);
            }
        }
        mma_commit(&done);
        if (!ok) {
            atomicOr(&prm->err, kErrTimeout);
            // let the last copy issued into each ring stage land before the CTA leaves (bounded);
            // the issued steps need not be a prefix (fault injection withholds step 0)
            for (int b2 = 0; b2 < NST; ++b2)
                if (last_issued[b2] >= 0) mbar_wait(&full[b2], (uint32_t)((last_issued[b2] / NST) & 1), limit);
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
        const size_t psz = (size_t)d * ld;
        const bool horner = step.kind == 0;
        const float ri = horner ? 1.0f / (float)step.i : 1.0f;
        for (int cc = 0; cc < BN; cc += 16) {
            float v[2][2][16];   // [acc][re/im][col]
            for (int a = 0; a < step.nacc; ++a) {
                const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * 2 * BN + cc);
                float w[2][16];
                tmem_ld16(ta, v[a][0]);
                tmem_ld16(ta + BN, v[a][1]);
                tmem_ld16(ta + CORR, w[0]);
                tmem_ld16(ta + CORR + BN, w[1]);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    v[a][0][q] += w[0][q];
                    v[a][1][q] += w[1][q];
                }
            }
            if (r >= d) continue;
#pragma unroll 4
            for (int q = 0; q < 16; ++q) {
                const int c = c0 + cc + q;
                if (c >= d) break;
                for (int a = 0; a < step.nacc; ++a) {
                    float re = v[a][0][q] * ri, im = v[a][1][q] * ri;
                    if (horner && a == 0 && r == c) re += 1.0f;
                    float part[2 * NPL];
                    split_tf32(re, part);
                    split_tf32(im, part + NPL);
                    const int mrow = a == 0 ? step.out0_row : step.out1_row;
                    const int mcol = a == 0 ? step.out0_col : step.out1_col;
#pragma unroll
                    for (int pp = 0; pp < 2 * NPL; ++pp) {
                        if (mrow >= 0) planes[tc_plane(item, mrow, pp, nmat) * psz + (size_t)r * ld + c] = part[pp];
                        if (mcol >= 0) planes[tc_plane(item, mcol, pp, nmat) * psz + (size_t)c * ld + r] = part[pp];
                    }
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
// Z11 = I + XH / p, Z12 = Ubar / p; all written as split planes (Z11, Z12 in both layouts).
__global__ void k_tc_adj_init(const DevParams* __restrict__ prm, SysView<float> sys, StateView<float> sv, int j0,
                              int wlen, const float2* __restrict__ states, const float2* __restrict__ Gbuf, int wmax,
                              float* __restrict__ planes, int ld, int nmat, TcMats m) {
    const int item = blockIdx.y, jl = item % wlen, e = item / wlen, j = j0 + jl;
    const int d = sys.d, M = sys.M;
    const size_t dd = (size_t)d * d, slice = sv.slice(), psz = (size_t)d * ld;
    const float s = (float)prm->s, ip = 1.0f / (float)prm->p;
    const float de = sys.delta ? (float)sys.delta[e] : 0.f;
    const float2* Gj = Gbuf + ((size_t)e * wmax + jl) * slice;
    const float2* Pj = states + ((size_t)e * (wmax + 1) + jl) * slice;
    auto put = [&](int mat, int r, int c, float re, float im, bool col) {
        float part[2 * NPL];
        split_tf32(re, part);
        split_tf32(im, part + NPL);
        for (int pp = 0; pp < 2 * NPL; ++pp) {
            const size_t pl = tc_plane(item, mat, pp, nmat) * psz;
            planes[pl + (col ? (size_t)c * ld + r : (size_t)r * ld + c)] = part[pp];
        }
    };
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
        for (int sc = 0; sc < sv.Spad; ++sc) {
            const size_t pa = (size_t)(sc / sv.cb) * sv.pstride + (size_t)a * sv.cb + (sc % sv.cb);
            const size_t pb = (size_t)(sc / sv.cb) * sv.pstride + (size_t)b * sv.cb + (sc % sv.cb);
            const float2 g = Gj[pa], q = Pj[pb];
            ur = fmaf(g.x, q.x, ur);     // g conj(q)
            ur = fmaf(g.y, q.y, ur);
            ui = fmaf(g.y, q.x, ui);
            ui = fmaf(-g.x, q.y, ui);
        }
        put(m.xh, a, b, xr, xi, false);
        put(m.ub, a, b, ur, ui, false);
        const float z1r = xr * ip + (a == b ? 1.f : 0.f), z1i = xi * ip;
        put(m.z11_row, a, b, z1r, z1i, false);
        put(m.z11_col, a, b, z1r, z1i, true);
        put(m.z12_row, a, b, ur * ip, ui * ip, false);
        put(m.z12_col, a, b, ur * ip, ui * ip, true);
    }
}

// dC/du_{k,j} = s sum_ab (Xbar_re Hk_im - Xbar_im Hk_re) with Xbar = hi + lo planes
__global__ void __launch_bounds__(256)
k_tc_grad(const DevParams* __restrict__ prm, SysView<float> sys, int j0, int wlen, const float* __restrict__ planes,
          int ld, int nmat, int xbar, double* __restrict__ gpart) {
    __shared__ double red[32];
    const int item = blockIdx.x, k = blockIdx.y, jl = item % wlen, e = item / wlen, j = j0 + jl;
    const int d = sys.d;
    const size_t dd = (size_t)d * d, psz = (size_t)d * ld;
    const float2* hk = sys.Hk + (size_t)k * dd;
    double v = 0.0;
    for (size_t idx = threadIdx.x; idx < dd; idx += blockDim.x) {
        const int a = (int)(idx / d), b = (int)(idx - (size_t)a * d);
        const size_t o = (size_t)a * ld + b;
        double xr = 0.0, xi = 0.0;
        for (int q = 0; q < NPL; ++q) {
            xr += (double)planes[tc_plane(item, xbar, q, nmat) * psz + o];
            xi += (double)planes[tc_plane(item, xbar, NPL + q, nmat) * psz + o];
        }
        v += xr * (double)hk[idx].y - xi * (double)hk[idx].x;
    }
    v = block_sum(v, red);
    if (threadIdx.x == 0) gpart[((size_t)e * sys.M + k) * sys.N + j] = prm->s * v;
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
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

size_t tc_scratch_floats(int d, int items) { return (size_t)items * kTcMats * 2 * kTcSplit * d * tc_ld(d); }

cudaError_t tc_make_maps(float* planes, int d, int items, TcMaps* maps) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int ld = tc_ld(d);
    cuuint64_t dims[3] = {(cuuint64_t)d, (cuuint64_t)d, (cuuint64_t)items * kTcMats * 2 * kTcSplit};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)ld * d * 4};
    cuuint32_t estr[3] = {1, 1, 1};
    cuuint32_t boxA[3] = {BK, BM, 1}, boxB[3] = {BK, BN, 1};
    CUresult r1 = enc(reinterpret_cast<CUtensorMap*>(maps->a), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, planes, dims, strides,
                      boxA, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = enc(reinterpret_cast<CUtensorMap*>(maps->b), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, planes, dims, strides,
                      boxB, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return (r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS) ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_tc_adj(const TcAdjArgs& a, cudaStream_t st, int* launches) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_step, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    auto count = [&]() { if (launches) ++*launches; };
    const int d = a.d, items = a.wlen * a.E, ld = tc_ld(d);
    TcMats m{0, 1, 2, 3, 4, 5};        // XH, Ubar, Z11 (row, col), Z12 (row, col) of set 0
    TcMats o{0, 1, 6, 7, 8, 9};        // the same matrices of set 1
    const size_t dd = (size_t)d * d;
    const int eb = (int)std::min<size_t>(64, (dd + 255) / 256);
    k_tc_adj_init<<<dim3(eb, items), 256, 0, st>>>(a.prm, a.sys, a.sv, a.j0, a.wlen, a.states, a.Gbuf, a.wmax, a.planes,
                                                    ld, kTcMats, m);
    count();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const CUtensorMap* mapA = reinterpret_cast<const CUtensorMap*>(a.maps.a);
    const CUtensorMap* mapB = reinterpret_cast<const CUtensorMap*>(a.maps.b);
    const int ntiles = ((d + BM - 1) / BM) * ((d + BN - 1) / BN);
    auto run = [&](const TcMats& in, const TcMats& out, int kind, int i) {
        TcStep s{};
        s.nacc = 2;
        s.kind = kind;
        s.i = i;
        if (kind == 0) {   // Horner: P11 = XH Z11, P12 = XH Z12 + Ubar Z11
            s.nterms = 3;
            s.t[0] = {in.xh, in.z11_col, 0};
            s.t[1] = {in.xh, in.z12_col, 1};
            s.t[2] = {in.ub, in.z11_col, 1};
        } else {           // squaring: P11 = Z11 Z11, P12 = Z11 Z12 + Z12 Z11
            s.nterms = 3;
            s.t[0] = {in.z11_row, in.z11_col, 0};
            s.t[1] = {in.z11_row, in.z12_col, 1};
            s.t[2] = {in.z12_row, in.z11_col, 1};
        }
        s.out0_row = out.z11_row;
        s.out0_col = out.z11_col;
        s.out1_row = out.z12_row;
        s.out1_col = out.z12_col;
        s.fault = a.fault;
        k_tc_step<<<dim3(ntiles, items), 128, TC_SMEM, st>>>(*mapA, *mapB, a.planes, s, d, ld, kTcMats, a.prm);
        count();
        return cudaGetLastError();
    };
    const TcMats* cur = &m;
    const TcMats* nxt = &o;
    for (int i = a.p - 1; i >= 1; --i) {
        if ((err = run(*cur, *nxt, 0, i)) != cudaSuccess) return err;
        std::swap(cur, nxt);
    }
    for (int q = 0; q < a.n; ++q) {
        if ((err = run(*cur, *nxt, 1, 0)) != cudaSuccess) return err;
        std::swap(cur, nxt);
    }
    if (a.sys.M > 0) {
        k_tc_grad<<<dim3(items, a.sys.M), 256, 0, st>>>(a.prm, a.sys, a.j0, a.wlen, a.planes, ld, kTcMats, cur->z12_row,
                                                         a.gpart);
        count();
    }
    return cudaGetLastError();
}

}  // namespace qoc
