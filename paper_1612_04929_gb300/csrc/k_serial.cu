// Serial recursions of one evaluation (the only sequential dependency of the method):
//   forward      Psi_j = U_j Psi_{j-1}                                     (Eqs. 2, 4)
//   costate      G_{j-1} = U_j^dag G_j + src_{j-1}                          (Appendix A, Alg. 1-3)
// Both run one CTA per (column panel, ensemble member) and stream the next slice propagators
// (and sources) into a shared-memory ring with cp.async while the current step computes.
//
// The running block is carried in extended precision: FP64 in the FP64 form, and an unevaluated
// hi + lo pair of FP32 numbers in the FP32 form.  Over thousands of slices the FP32 rounding of a
// plainly carried state adds up to gradient errors near 1e-5; the carried pair keeps each step's
// rounding near 2^-36 of the block's scale while U_j, the stored states and costates (inputs of
// the parallel kernels) stay FP32.  (The FP64 form's steps and the pair helpers below with
// TwoSum accumulation serve the FP64 form and the sources' additions.)
//
// FP32 form: every step multiplies grid-split operands (qoc_device.cuh).  The carried pair block
// is re-split at the start of each step on a power-of-two grid set by a bound on its column
// norms, sqrt(2d) max |component| (the maximum is gathered while the previous step writes the
// block), and the elements of U_j^(dag) (or of P_z) are split as they are read.  The grid sums
// are exact; only the cross terms round (about 2^-36 of the scale), so a step costs 12 FMAs and
// the operand splits per complex multiply-add instead of the pair arithmetic's ~44 operations.
//
// Checkpointing: the forward sweep stores the carried block every `seg` slices (seg = ceil(sqrt
// N) by default).  In the backward sweep the states of a wave are regenerated from those
// checkpoints, one CTA per checkpoint segment in parallel (mode 1 below), so regeneration
// costs seg serial steps whatever the wave length.  Reversal (mode 2, the paper's Algorithms
// 1-3): the states of a wave are regenerated backwards from its last state,
// Psi_{j-1} = U_j^dag Psi_j, with no checkpoint inside the evolution.
#include "qoc_device.cuh"
#include "qoc_internal.h"

namespace qoc {

// ------------------------------------------------------------------------------------------
// carried-precision complex arithmetic
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float p) {
    const float t = hi + p;
    const float bv = t - hi;
    lo += (hi - (t - bv)) + (p - bv);
    hi = t;
}
// acc += u x (FP64 form; the FP32 form takes the grid step)
__device__ __forceinline__ void kmac(double2& acc, const double2 u, const double2 x) { cfma(acc, u, x); }
__device__ __forceinline__ void kadd(float4& a, const float4 b) {
    two_sum_acc(a.x, a.z, b.x);
    a.z += b.z;
    two_sum_acc(a.y, a.w, b.y);
    a.w += b.w;
}
__device__ __forceinline__ void kadd(double2& a, const double2 b) {
    a.x += b.x;
    a.y += b.y;
}
__device__ __forceinline__ void knorm(float4& a) {
    float s = a.x + a.z;
    a.z = a.z - (s - a.x);
    a.x = s;
    s = a.y + a.w;
    a.w = a.w - (s - a.y);
    a.y = s;
}
__device__ __forceinline__ void knorm(double2&) {}
__device__ __forceinline__ float2 kround(const float4 a) { return make_float2(a.x + a.z, a.y + a.w); }
__device__ __forceinline__ double2 kround(const double2 a) { return a; }
__device__ __forceinline__ float4 kfrom(const float2 a) { return make_float4(a.x, a.y, 0.f, 0.f); }
__device__ __forceinline__ float4 kfrom(const float4 a) { return a; }
__device__ __forceinline__ double2 kfrom(const double2 a) { return a; }
template <typename K> __device__ __forceinline__ K kzero();
template <> __device__ __forceinline__ float4 kzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double2 kzero<double2>() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float4 kshfl_xor(const float4 a, int o) {
    return make_float4(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o),
                       __shfl_xor_sync(0xffffffffu, a.z, o), __shfl_xor_sync(0xffffffffu, a.w, o));
}
__device__ __forceinline__ double2 kshfl_xor(const double2 a, int o) {
    return make_double2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
}

// ------------------------------------------------------------------------------------------
// ring of slice propagators (and sources) in shared memory
// ------------------------------------------------------------------------------------------
__host__ __device__ inline size_t ring_bytes(size_t elems, size_t esize) { return (elems * esize + 15) & ~(size_t)15; }

__device__ __forceinline__ void ring_issue(unsigned char* slot, const void* gsrc, size_t bytes) {
    const unsigned char* g = reinterpret_cast<const unsigned char*>(gsrc);
    for (size_t off = threadIdx.x * 16; off < bytes; off += blockDim.x * 16) cp_async16(slot + off, g + off);
}

// One step y = Mx x (+ add) on a d x cb panel.  g lanes per output (contiguous in a warp) sum
// b = q, q + g, ... of row a of Mx (contiguous reads: the forward sweep streams U_j, the backward
// sweep U_j^dag), then a shuffle reduction combines them.  Lane q = 0 owns the output: it adds
// the source, normalises the pair, keeps it for the next step and hands it to `emit`.
template <typename C, typename K, typename S = C, typename Emit>
__device__ __forceinline__ void sweep_step(const C* __restrict__ Mx, const K* __restrict__ x, K* __restrict__ y,
                                           const S* __restrict__ add, int d, int cb, int g, Emit emit) {
    const int O = d * cb;
    const int ngroups = blockDim.x / g;
    const int gi = threadIdx.x / g, q = threadIdx.x - gi * g;
    for (int base = 0; base < O; base += ngroups) {
        const int o = base + gi;
        K acc = kzero<K>();
        if (o < O) {
            const int a = o / cb, sl = o - a * cb;
            const C* Mr = Mx + (size_t)a * d;
            for (int b = q; b < d; b += g) kmac(acc, Mr[b], x[b * cb + sl]);
        }
        for (int off = g >> 1; off > 0; off >>= 1) kadd(acc, kshfl_xor(acc, off));
        if (o < O && q == 0) {
            if (add) kadd(acc, kfrom(add[o]));
            knorm(acc);
            y[o] = acc;
            emit(o, acc);
        }
    }
}

// FP32 grid step.  Element of the matrix operand, split with the magic constant mu: (u1, u2) in
// s and the full value in uf (a plain FP32 value is its own full value; a carried pair rounds).
__device__ __forceinline__ void gsplit_elem(const float2 u, float mu, float4& s, float2& uf) {
    grid_split(u.x, 0.f, mu, s.x, s.z);
    grid_split(u.y, 0.f, mu, s.y, s.w);
    uf = u;
}
__device__ __forceinline__ void gsplit_elem(const float4 u, float mu, float4& s, float2& uf) {
    grid_split(u.x, u.z, mu, s.x, s.z);
    grid_split(u.y, u.w, mu, s.y, s.w);
    uf = make_float2(s.x + s.z, s.y + s.w);
}
// magic constant of the block's grid from the largest |component| m (float bits): the column
// 2-norms are at most sqrt(2d) m
__device__ __forceinline__ float block_magic(unsigned mbits, int d) {
    const float b = sqrtf(2.0f * d) * __uint_as_float(mbits) * 1.0625f;
    int e = -100;
    if (b > 0.f) e = (b < 1e30f) ? ilogbf(b) + 1 : 100;
    return grid_magic(e < -100 ? -100 : e);
}
__device__ __forceinline__ float4 pair_to_grid(const float4 v, float mx) {
    float4 o;
    grid_split(v.x, v.z, mx, o.x, o.z);
    grid_split(v.y, v.w, mx, o.y, o.w);
    return o;
}
__device__ __forceinline__ unsigned pair_maxbits(const float4 v) {
    return __float_as_uint(fmaxf(fabsf(v.x), fabsf(v.y)));
}

// s += u x for one grid-split element u = (u1, u2) (full value uf) and one grid-split pair x:
// s[0], s[1] the grid parts (exact), s[2], s[3] the cross terms
__device__ __forceinline__ void mac_grid(float* s, const float4 u, const float2 uf, const float4 x) {
    s[0] = fmaf(u.x, x.x, s[0]);
    s[0] = fmaf(-u.y, x.y, s[0]);
    s[1] = fmaf(u.x, x.y, s[1]);
    s[1] = fmaf(u.y, x.x, s[1]);
    s[2] = fmaf(u.z, x.x, s[2]);
    s[2] = fmaf(-u.w, x.y, s[2]);
    s[2] = fmaf(uf.x, x.z, s[2]);
    s[2] = fmaf(-uf.y, x.w, s[2]);
    s[3] = fmaf(u.z, x.y, s[3]);
    s[3] = fmaf(u.w, x.x, s[3]);
    s[3] = fmaf(uf.x, x.w, s[3]);
    s[3] = fmaf(uf.y, x.z, s[3]);
}
// the output pair S + L of one grid step: S exact, so the pair is formed without error
__device__ __forceinline__ float4 grid_out(const float* s) {
    float4 v;
    two_sum(s[0], s[2], v.x, v.z);
    two_sum(s[1], s[3], v.y, v.w);
    return v;
}

// One FP32 step y = Mx x (+ add) from the grid-split block xg (panels narrower than 8 columns).
// A group of g lanes owns output (a, c); the lanes sum the grid parts (S, exact) and the cross
// terms (L) of b = q, q + g, ...; the shuffle reduction adds S and L with plain adds (S stays
// exact); lane q = 0 forms the pair S + L without error, adds the source, normalises, keeps it in
// y, hands it to `emit` and raises *ymax to the largest component.
template <typename Mt, typename S, typename Emit>
__device__ __forceinline__ void sweep_step_grid(const Mt* __restrict__ Mx, const float4* __restrict__ xg,
                                                float4* __restrict__ y, const S* __restrict__ add, int d, int cb,
                                                int g, float mu, unsigned* ymax, Emit emit) {
    const int O = d * cb;
    const int ngroups = blockDim.x / g;
    const int gi = threadIdx.x / g, q = threadIdx.x - gi * g;
    for (int base = 0; base < O; base += ngroups) {
        const int o = base + gi;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (o < O) {
            const int a = o / cb, c = o - a * cb;
            const Mt* Mr = Mx + (size_t)a * d;
            auto step = [&](const Mt m, int b) {
                float4 u;
                float2 uf;
                gsplit_elem(m, mu, u, uf);
                mac_grid(acc, u, uf, xg[b * cb + c]);
            };
            // the matrix elements come from L2 (the propagators do not fit shared memory at large
            // d): four loads in flight before their products
            int b = q;
            for (; b + 3 * g < d; b += 4 * g) {
                const Mt m0 = Mr[b], m1 = Mr[b + g], m2 = Mr[b + 2 * g], m3 = Mr[b + 3 * g];
                step(m0, b);
                step(m1, b + g);
                step(m2, b + 2 * g);
                step(m3, b + 3 * g);
            }
            for (; b < d; b += g) step(Mr[b], b);
        }
        for (int off = g >> 1; off > 0; off >>= 1)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
        if (o < O && q == 0) {
            float4 v = grid_out(acc);
            if (add) kadd(v, kfrom(add[o]));
            knorm(v);
            y[o] = v;
            emit(o, v);
            atomicMax(ymax, pair_maxbits(v));
        }
    }
}

// The FP32 step on an 8-column panel.  A group of 8 lanes owns the row pair a, a + 1 and all 8
// columns; lane q sums b = q, q + 8, ..., so each grid-split element of x read from shared memory
// serves two rows (16 complex multiply-adds per 8 loads).  xg rows are padded to kGridRow float4,
// which puts the rows b .. b + 7 that a group reads at once in distinct banks.  The elements of Mx
// are software-pipelined: those of the next PF b's are in flight while the current ones compute.
// A reduce-scatter over the group (three shuffle rounds on halves of the sums) leaves lane q with
// row a + (q >> 2 & 1), columns 4 (q >> 1 & 1) + 2 (q & 1) + {0, 1}; the sums of grid parts stay
// exact in any order, so each lane completes its two outputs like the one-row step.
constexpr int kGridRow = 9;
template <typename Mt, typename S, typename Emit>
__device__ __forceinline__ void sweep_step_rows2(const Mt* __restrict__ Mx, const float4* __restrict__ xg,
                                                 float4* __restrict__ y, const S* __restrict__ add, int d, float mu,
                                                 unsigned* ymax, Emit emit) {
    constexpr int G = 8, CB = 8;
    constexpr int PF = sizeof(Mt) == 8 ? 2 : 1;   // b's per pipeline stage (registers: carried pairs are wider)
    const int pairs = (d + 1) >> 1;
    const int ngroups = blockDim.x / G;
    const int gi = threadIdx.x / G, q = threadIdx.x & (G - 1);
    // the loop bound is the same for every thread, so all lanes reach the shuffles
    for (int base = 0; base < pairs; base += ngroups) {
        const int a = 2 * (base + gi);
        const bool on = a < d;
        float acc[2][CB][4];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < CB; ++c) acc[r][c][0] = acc[r][c][1] = acc[r][c][2] = acc[r][c][3] = 0.f;
        if (on) {
            const Mt* M0 = Mx + (size_t)a * d;
            const Mt* M1 = (a + 1 < d) ? M0 + d : M0;   // odd d: the last pair repeats its row, unused
            auto step = [&](const Mt m0, const Mt m1, int b) {
                float4 u0, u1;
                float2 f0, f1;
                gsplit_elem(m0, mu, u0, f0);
                gsplit_elem(m1, mu, u1, f1);
                const float4* xr = xg + b * kGridRow;
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    const float4 x = xr[c];
                    mac_grid(acc[0][c], u0, f0, x);
                    mac_grid(acc[1][c], u1, f1, x);
                }
            };
            Mt cur[2][PF], nxt[2][PF];
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int bb = q + u * G;
                cur[0][u] = bb < d ? M0[bb] : Mt{};
                cur[1][u] = bb < d ? M1[bb] : Mt{};
            }
            for (int b = q; b < d; b += PF * G) {
#pragma unroll
                for (int u = 0; u < PF; ++u) {
                    const int bb = b + (PF + u) * G;
                    nxt[0][u] = bb < d ? M0[bb] : Mt{};
                    nxt[1][u] = bb < d ? M1[bb] : Mt{};
                }
#pragma unroll
                for (int u = 0; u < PF; ++u)
                    if (b + u * G < d) step(cur[0][u], cur[1][u], b + u * G);
#pragma unroll
                for (int u = 0; u < PF; ++u) {
                    cur[0][u] = nxt[0][u];
                    cur[1][u] = nxt[1][u];
                }
            }
        }
        // reduce-scatter: keep the half named by the lane's bit, send the other half to the partner
        const bool h2 = q & 4, h1 = q & 2, h0 = q & 1;
        float w1[CB][4];
#pragma unroll
        for (int c = 0; c < CB; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float keep = h2 ? acc[1][c][k] : acc[0][c][k];
                const float send = h2 ? acc[0][c][k] : acc[1][c][k];
                w1[c][k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
        float w2[4][4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float keep = h1 ? w1[4 + c][k] : w1[c][k];
                const float send = h1 ? w1[c][k] : w1[4 + c][k];
                w2[c][k] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
            }
        float w3[2][4];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float keep = h0 ? w2[2 + c][k] : w2[c][k];
                const float send = h0 ? w2[c][k] : w2[2 + c][k];
                w3[c][k] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
            }
        const int row = a + (h2 ? 1 : 0);
        unsigned mb = 0u;
        if (on && row < d) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int o = row * CB + (h1 ? 4 : 0) + (h0 ? 2 : 0) + c;
                float4 v = grid_out(w3[c]);
                if (add) kadd(v, kfrom(add[o]));
                knorm(v);
                y[o] = v;
                mb = max(mb, pair_maxbits(v));
                emit(o, v);
            }
        }
        mb = __reduce_max_sync(0xffffffffu, mb);
        if ((threadIdx.x & 31) == 0) atomicMax(ymax, mb);
    }
}

// shared memory of the FP32 step's grid-split block (none in the FP64 form)
template <typename R>
static size_t grid_block_bytes(int d, int cb) {
    return sizeof(R) == 4 ? sizeof(float4) * (size_t)d * (cb == 8 ? kGridRow : cb) : 0;
}

// lanes per output group and block size.  FP32 8-column panels (two-row step): groups of 8 lanes,
// at most 8 warps (two CTAs per SM at 128 registers).  Otherwise a group is one output; minimise
// the issue time of one step on one SM (passes x warps per scheduler x instructions per lane).
static void pick_sweep_shape(int d, int cb, bool fp32, int& g, int& threads) {
    if (fp32 && cb == 8) {
        g = 8;
        const int t = ((((d + 1) / 2) * 8 + 31) / 32) * 32;
        threads = t < 256 ? t : 256;
        return;
    }
    const int O = d * cb;
    long best = -1;
    for (int gg = 1, lg = 0; gg <= 32; gg <<= 1, ++lg) {
        const int tmax = fp32 ? 512 : 1024;   // the kernels' launch bounds
        int thr = ((O * gg + 31) / 32) * 32;
        thr = thr > tmax ? tmax : thr;
        const int groups = thr / gg;
        const int passes = (O + groups - 1) / groups;
        const int wps = (thr / 32 + 3) / 4;
        // instructions per lane: per b of the row and the reduction
        const long per_b = fp32 ? 20 : 10;
        const long red = (fp32 ? 8L : 12L) * lg;
        const long cost = (long)passes * wps * (((d + gg - 1) / gg) * per_b + red);
        if (best < 0 || cost < best) {
            best = cost;
            g = gg;
            threads = thr;
        }
    }
}

// ------------------------------------------------------------------------------------------
// forward propagation (mode 0) and checkpoint replay (mode 1)
// ------------------------------------------------------------------------------------------
template <typename R, int RING, typename Mt, int NCB>
__global__ void __launch_bounds__(sizeof(R) == 4 ? 512 : 1024)
k_chain(int d, StateView<R> sv, int wlen, int seg, int mode, K_t<R>* __restrict__ ckpt, size_t ck_estride, int seg0,
        int nseg_total, const Mt* __restrict__ Ubuf, long long ustride, int wmax, C_t<R>* __restrict__ states,
        int g, const DevParams* __restrict__ prm, const C_t<R>* __restrict__ rev_src, size_t rev_estride) {
    using C = C_t<R>;
    using K = K_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int kb = blockIdx.x, e = blockIdx.y, z = blockIdx.z, tid = threadIdx.x, cb = sv.cb;
    const size_t slice = sv.slice(), panel = (size_t)d * cb;
    const size_t ub = ring_bytes((size_t)d * d, sizeof(Mt));
    unsigned char* ring = smraw;
    K* xa = reinterpret_cast<K*>(smraw + RING * ub);   // RING 0: no ring, rows read from global
    K* xb = xa + panel;
    float4* xg = reinterpret_cast<float4*>(xb + panel);   // FP32: grid-split block of the step
    __shared__ unsigned smax[2];                           // FP32: largest component, by step parity
    // mode 2 (reversal): the whole wave backwards from its last state, step k applying
    // U_{t}^dag with t = wlen - 1 - k and writing state t
    const bool rev = mode == 2;
    const int t0 = (mode == 1) ? z * seg : 0;
    const int t1 = (mode == 1) ? min(wlen, t0 + seg) : wlen;
    if (t0 >= t1) return;
    if (tid == 0) smax[0] = smax[1] = 0u;
    __syncthreads();
    K* ck_e = ckpt + e * ck_estride;
    const K* s0 = ck_e + (size_t)(seg0 + t0 / seg) * slice + (size_t)kb * sv.pstride;
    C* sdst = states + (size_t)e * (wmax + 1) * slice + (size_t)kb * sv.pstride;
    // the first state of a replayed segment z > 0 is the last state of segment z - 1, which that
    // segment's CTA writes: one writer per state (the checkpoint and the stepped value differ in
    // their last bits)
    const bool own_first = (mode != 1 || z == 0);
    const C* rsrc = rev ? rev_src + (size_t)e * rev_estride + (size_t)kb * sv.pstride : nullptr;
    for (int i = tid; i < (int)panel; i += blockDim.x) {
        const K v = rev ? kfrom(rsrc[i]) : s0[i];
        xa[i] = v;
        if (own_first) sdst[(size_t)(rev ? wlen : t0) * slice + i] = kround(v);
        if constexpr (sizeof(R) == 4) atomicMax(&smax[0], pair_maxbits(v));
    }
    float mu = 0.f;
    if constexpr (sizeof(R) == 4) mu = grid_magic(prm ? prm->eu : 1);
    // one step from the block in xa into xb (the caller has passed a barrier since xa was written)
    auto step = [&](const Mt* M, int k, auto emit) {
        if constexpr (sizeof(R) == 4) {
            const float mx = block_magic(smax[k & 1], d);
            if (tid == 0) smax[(k + 1) & 1] = 0u;
            for (int i = tid; i < (int)panel; i += blockDim.x)
                xg[NCB == 8 ? i + (i >> 3) : i] = pair_to_grid(xa[i], mx);   // 8 columns: rows of kGridRow
            __syncthreads();
            if constexpr (NCB == 8)
                sweep_step_rows2<Mt, C>(M, xg, xb, static_cast<const C*>(nullptr), d, mu, &smax[(k + 1) & 1], emit);
            else
                sweep_step_grid<Mt, C>(M, xg, xb, static_cast<const C*>(nullptr), d, cb, g, mu, &smax[(k + 1) & 1],
                                       emit);
        } else {
            sweep_step<Mt, K, C>(M, xa, xb, nullptr, d, cb, g, emit);
        }
        K* tmp = xa; xa = xb; xb = tmp;
    };
    // propagator of step t (forward: U_t; reversal: U_{wlen-1-t}^dag) and the state it writes
    const Mt* Ue = Ubuf + (size_t)e * wmax * ustride;
    auto mat = [&](int t) {
        return rev ? Ue + (size_t)(wlen - 1 - t) * ustride + ustride / 2 : Ue + (size_t)t * ustride;
    };
    auto emit_for = [&](int t) {
        C* dst = sdst + (size_t)(rev ? wlen - 1 - t : t + 1) * slice;
        K* ckd = nullptr;
        if (mode == 0 && (t + 1) % seg == 0 && seg0 + (t + 1) / seg < nseg_total)
            ckd = ck_e + (size_t)(seg0 + (t + 1) / seg) * slice + (size_t)kb * sv.pstride;
        return [=](int o, const K& v) {
            dst[o] = kround(v);
            if (ckd) ckd[o] = v;
        };
    };
    if constexpr (RING == 0) {          // slice too large for SMEM: rows streamed from global/L2
#pragma unroll 1
        for (int t = t0; t < t1; ++t) {
            __syncthreads();
            step(mat(t), t - t0, emit_for(t));
        }
    } else if constexpr (RING == 1) {   // one slot: synchronous copy
#pragma unroll 1
        for (int t = t0; t < t1; ++t) {
            __syncthreads();            // previous step done with the slot
            ring_issue(ring, mat(t), ub);
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            step(reinterpret_cast<const Mt*>(ring), t - t0, emit_for(t));
        }
    } else {
#pragma unroll 1
        for (int t = 0; t < RING - 1; ++t) {
            if (t0 + t < t1) ring_issue(ring + t * ub, mat(t0 + t), ub);
            cp_async_commit();
        }
#pragma unroll 1
        for (int t = t0; t < t1; ++t) {
            const int k = t - t0;
            cp_async_wait<(RING >= 2 ? RING - 2 : 0)>();   // the copy of step k has landed ...
            __syncthreads();                                // ... for every thread; step k - 1 is finished
            const int tn = t + RING - 1;
            if (tn < t1) ring_issue(ring + ((k + RING - 1) % RING) * ub, mat(tn), ub);
            cp_async_commit();
            step(reinterpret_cast<const Mt*>(ring + (k % RING) * ub), k, emit_for(t));
        }
    }
}

template <typename R, int RING, typename Mt, int NCB>
static cudaError_t chain_ring_n(const ChainArgs<R>& a, const Mt* U, size_t smem, cudaStream_t st) {
    cudaError_t err =
        cudaFuncSetAttribute(k_chain<R, RING, Mt, NCB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int g = 1, threads = 256;
    pick_sweep_shape(a.d, a.sv.cb, sizeof(R) == 4, g, threads);
    const int nz = a.mode == 0 ? 1 : (a.wlen + a.seg - 1) / a.seg;
    k_chain<R, RING, Mt, NCB><<<dim3(a.sv.ncb, a.E, nz), threads, smem, st>>>(
        a.d, a.sv, a.wlen, a.seg, a.mode, a.ckpt, a.ck_estride, a.seg0, a.nseg_total, U, a.ustride, a.wmax, a.states,
        g, a.prm, a.rev_src, a.rev_estride);
    return cudaGetLastError();
}

// FP32: 8-column panels take the two-row step (NCB = 8)
template <typename R, int RING, typename Mt>
static cudaError_t chain_ring(const ChainArgs<R>& a, const Mt* U, size_t smem, cudaStream_t st) {
    if (sizeof(R) == 4 && a.sv.cb == 8) return chain_ring_n<R, RING, Mt, (sizeof(R) == 4 ? 8 : 1)>(a, U, smem, st);
    return chain_ring_n<R, RING, Mt, 1>(a, U, smem, st);
}

template <typename R, typename Mt>
static cudaError_t chain_dispatch(const ChainArgs<R>& a, const Mt* U, cudaStream_t st) {
    const size_t ub = ring_bytes((size_t)a.d * a.d, sizeof(Mt));
    const size_t xs = 2 * sizeof(K_t<R>) * (size_t)a.d * a.sv.cb + grid_block_bytes<R>(a.d, a.sv.cb);
    if (xs > kMaxDynSmem) return cudaErrorInvalidValue;
    for (int ring : {8, 4, 2, 1}) {
        const size_t smem = ring * ub + xs;
        if (smem > kMaxDynSmem) continue;
        if (ring == 8) return chain_ring<R, 8, Mt>(a, U, smem, st);
        if (ring == 4) return chain_ring<R, 4, Mt>(a, U, smem, st);
        if (ring == 2) return chain_ring<R, 2, Mt>(a, U, smem, st);
        return chain_ring<R, 1, Mt>(a, U, smem, st);
    }
    return chain_ring<R, 0, Mt>(a, U, xs, st);   // slice larger than SMEM: stream its rows
}

template <typename R>
cudaError_t launch_chain(const ChainArgs<R>& a, cudaStream_t st) {
    if ((a.Ubuf != nullptr) == (a.Uk != nullptr)) return cudaErrorInvalidValue;
    if (a.mode == 2 && (!a.rev_src || !a.Ubuf)) return cudaErrorInvalidValue;
    if (a.Uk) return chain_dispatch<R, K_t<R>>(a, a.Uk, st);
    return chain_dispatch<R, C_t<R>>(a, a.Ubuf, st);
}

// ------------------------------------------------------------------------------------------
// backward costate sweep: G_{j-1} = U_j^dag G_j + src_{j-1}, one CTA per (panel, member, segment)
// ------------------------------------------------------------------------------------------
// Segment z covers local slices a = z * seg .. b = min(wlen, a + seg) - 1.  With in-carry Y
// (zero when a.cin is null) the CTA sets G_b = Y + src_b, runs G_{jl-1} = U_jl^dag G_jl + src_{jl-1}
// down to jl = a + 1, and leaves out = U_a^dag G_a, the in-carry of the segment below; `out`
// goes to a.cout.  A whole wave is one segment (seg = wlen) with the carry as in- and out-carry.
template <typename R, int RING, typename S, typename Mt, int NCB>
__global__ void __launch_bounds__(sizeof(R) == 4 ? 512 : 1024) k_costate(CostateArgs<R> A, int g) {
    using C = C_t<R>;
    using K = K_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int kb = blockIdx.x, e = blockIdx.y, z = blockIdx.z, tid = threadIdx.x;
    const int d = A.d, cb = A.sv.cb;
    const int a0 = z * A.seg;
    if (a0 >= A.wlen) return;
    const int b0 = min(A.wlen, a0 + A.seg) - 1;
    const int n = b0 - a0 + 1;
    const size_t slice = A.sv.slice(), panel = (size_t)d * cb, poff = (size_t)kb * A.sv.pstride;
    const size_t ub = ring_bytes((size_t)d * d, sizeof(Mt));
    const size_t pb = (size_t)A.sv.pstride * sizeof(S);
    const size_t slot = ub + pb;
    unsigned char* ring = smraw;
    K* xa = reinterpret_cast<K*>(smraw + RING * slot);   // RING 0: no ring
    K* xb = xa + panel;
    float4* xg = reinterpret_cast<float4*>(xb + panel);   // FP32: grid-split block of the step
    __shared__ unsigned smax[2];
    if (tid == 0) smax[0] = smax[1] = 0u;
    __syncthreads();
    const Mt* UHe = reinterpret_cast<const Mt*>(A.Uk ? (const void*)A.Uk : (const void*)A.U) + e * A.u_es +
                    A.ustride / 2;                        // U_j^dag of every slice
    const S* Se = reinterpret_cast<const S*>(A.srck ? (const void*)A.srck : (const void*)A.src) + e * A.src_es + poff;
    C* Ge = A.G ? A.G + e * A.g_es + poff : nullptr;
    K* Gk = A.Gk ? A.Gk + e * A.g_es + poff : nullptr;
    {   // G_b = Y + src_b
        const K* ci = A.cin ? A.cin + e * A.cin_es + (size_t)z * slice + poff : nullptr;
        const S* s_last = Se + (size_t)b0 * slice;
        for (int i = tid; i < (int)panel; i += blockDim.x) {
            K v = ci ? ci[i] : kzero<K>();
            kadd(v, kfrom(s_last[i]));
            knorm(v);
            xa[i] = v;
            if constexpr (sizeof(R) == 4) atomicMax(&smax[0], pair_maxbits(v));
            if (Ge) Ge[(size_t)b0 * slice + i] = kround(v);
            if (Gk) Gk[(size_t)b0 * slice + i] = v;
        }
    }
    auto emit_for = [&](int jl) {
        C* gd = (Ge && jl > a0) ? Ge + (size_t)(jl - 1) * slice : nullptr;
        K* gk = (Gk && jl > a0) ? Gk + (size_t)(jl - 1) * slice : nullptr;
        return [=](int o, const K& v) {
            if (gd) gd[o] = kround(v);
            if (gk) gk[o] = v;
        };
    };
    float mu = 0.f;
    if constexpr (sizeof(R) == 4) mu = grid_magic(A.prm ? A.prm->eu : 1);
    // one step from the block in xa into xb (the caller has passed a barrier since xa was written)
    auto step = [&](const Mt* M, const S* add, int k, auto emit) {
        if constexpr (sizeof(R) == 4) {
            const float mx = block_magic(smax[k & 1], d);
            if (tid == 0) smax[(k + 1) & 1] = 0u;
            for (int i = tid; i < (int)panel; i += blockDim.x)
                xg[NCB == 8 ? i + (i >> 3) : i] = pair_to_grid(xa[i], mx);   // 8 columns: rows of kGridRow
            __syncthreads();
            if constexpr (NCB == 8)
                sweep_step_rows2<Mt, S>(M, xg, xb, add, d, mu, &smax[(k + 1) & 1], emit);
            else
                sweep_step_grid<Mt, S>(M, xg, xb, add, d, cb, g, mu, &smax[(k + 1) & 1], emit);
        } else {
            sweep_step<Mt, K, S>(M, xa, xb, add, d, cb, g, emit);
        }
        K* tmp = xa; xa = xb; xb = tmp;
    };
    // step t handles slice jl = b0 - t: U_jl^dag and src_{jl-1} (none at the segment's first slice)
    if constexpr (RING == 0) {          // rows of U^dag and the sources read from global/L2
#pragma unroll 1
        for (int t = 0; t < n; ++t) {
            const int jl = b0 - t;
            __syncthreads();
            step(UHe + (size_t)jl * A.ustride, (jl > a0) ? Se + (size_t)(jl - 1) * slice : nullptr, t, emit_for(jl));
        }
    } else if constexpr (RING == 1) {
#pragma unroll 1
        for (int t = 0; t < n; ++t) {
            const int jl = b0 - t;
            __syncthreads();
            ring_issue(ring, UHe + (size_t)jl * A.ustride, ub);
            if (jl > a0) ring_issue(ring + ub, Se + (size_t)(jl - 1) * slice, pb);
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            step(reinterpret_cast<const Mt*>(ring), (jl > a0) ? reinterpret_cast<const S*>(ring + ub) : nullptr, t,
                 emit_for(jl));
        }
    } else {
        auto issue = [&](int t) {
            const int jl = b0 - t;
            unsigned char* sl = ring + (t % RING) * slot;
            ring_issue(sl, UHe + (size_t)jl * A.ustride, ub);
            if (jl > a0) ring_issue(sl + ub, Se + (size_t)(jl - 1) * slice, pb);
        };
#pragma unroll 1
        for (int t = 0; t < RING - 1; ++t) {
            if (t < n) issue(t);
            cp_async_commit();
        }
#pragma unroll 1
        for (int t = 0; t < n; ++t) {
            const int jl = b0 - t;
            cp_async_wait<(RING >= 2 ? RING - 2 : 0)>();
            __syncthreads();
            const int tn = t + RING - 1;
            if (tn < n) issue(tn);
            cp_async_commit();
            const unsigned char* sl = ring + (t % RING) * slot;
            step(reinterpret_cast<const Mt*>(sl), (jl > a0) ? reinterpret_cast<const S*>(sl + ub) : nullptr, t,
                 emit_for(jl));
        }
    }
    __syncthreads();
    if (A.cout) {
        K* co = A.cout + e * A.cout_es + (size_t)z * slice + poff;
        for (int i = tid; i < (int)panel; i += blockDim.x) co[i] = xa[i];
    }
    if (A.zero_next && z == gridDim.z - 1) {   // clear the slot after the last out-carry
        K* co = A.cout + e * A.cout_es + (size_t)(z + 1) * slice + poff;
        for (int i = tid; i < (int)panel; i += blockDim.x) co[i] = kzero<K>();
    }
}

template <typename R, int RING, typename S, typename Mt, int NCB>
static cudaError_t costate_ring_n(const CostateArgs<R>& a, size_t smem, cudaStream_t st) {
    cudaError_t err =
        cudaFuncSetAttribute(k_costate<R, RING, S, Mt, NCB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int g = 1, threads = 256;
    pick_sweep_shape(a.d, a.sv.cb, sizeof(R) == 4, g, threads);
    const int nz = (a.wlen + a.seg - 1) / a.seg;
    k_costate<R, RING, S, Mt, NCB><<<dim3(a.sv.ncb, a.E, nz), threads, smem, st>>>(a, g);
    return cudaGetLastError();
}

template <typename R, int RING, typename S, typename Mt>
static cudaError_t costate_ring(const CostateArgs<R>& a, size_t smem, cudaStream_t st) {
    if (sizeof(R) == 4 && a.sv.cb == 8) return costate_ring_n<R, RING, S, Mt, (sizeof(R) == 4 ? 8 : 1)>(a, smem, st);
    return costate_ring_n<R, RING, S, Mt, 1>(a, smem, st);
}

template <typename R, typename S, typename Mt>
static cudaError_t costate_dispatch(const CostateArgs<R>& a, cudaStream_t st) {
    const size_t panel = (size_t)a.d * a.sv.cb;
    const size_t ub = ring_bytes((size_t)a.d * a.d, sizeof(Mt));
    const size_t pb = (size_t)a.sv.pstride * sizeof(S);
    const size_t fixed = 2 * sizeof(K_t<R>) * panel + grid_block_bytes<R>(a.d, a.sv.cb);
    if (fixed > kMaxDynSmem) return cudaErrorInvalidValue;
    for (int ring : {8, 4, 2, 1}) {
        const size_t smem = ring * (ub + pb) + fixed;
        if (smem > kMaxDynSmem) continue;
        if (ring == 8) return costate_ring<R, 8, S, Mt>(a, smem, st);
        if (ring == 4) return costate_ring<R, 4, S, Mt>(a, smem, st);
        if (ring == 2) return costate_ring<R, 2, S, Mt>(a, smem, st);
        return costate_ring<R, 1, S, Mt>(a, smem, st);
    }
    return costate_ring<R, 0, S, Mt>(a, fixed, st);
}

template <typename R>
cudaError_t launch_costate(const CostateArgs<R>& a, cudaStream_t st) {
    if (a.wlen <= 0 || a.seg <= 0 || (a.zero_next && !a.cout) || (a.src != nullptr) == (a.srck != nullptr))
        return cudaErrorInvalidValue;
    if ((a.U != nullptr) == (a.Uk != nullptr)) return cudaErrorInvalidValue;
    // carried sources go with carried matrices (the scan over segments), plain with plain
    if (a.srck && a.Uk) return costate_dispatch<R, K_t<R>, K_t<R>>(a, st);
    if (a.src && a.U) return costate_dispatch<R, C_t<R>, C_t<R>>(a, st);
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------------------------
// row-major FP64 d x S -> carried panel blocks (checkpoint 0 of every member)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void kset(float4& o, double x, double y) {
    o.x = (float)x;
    o.y = (float)y;
    o.z = (float)(x - (double)o.x);
    o.w = (float)(y - (double)o.y);
}
__device__ __forceinline__ void kset(double2& o, double x, double y) {
    o.x = x;
    o.y = y;
}

template <typename R>
__global__ void k_to_carry(const double2* __restrict__ src, K_t<R>* __restrict__ dst, int d, int S, StateView<R> sv,
                           size_t dst_stride) {
    const size_t per = sv.slice();
    K_t<R>* out = dst + blockIdx.y * dst_stride;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
        const int kb = (int)(i / sv.pstride);
        const int rem = (int)(i - (size_t)kb * sv.pstride);
        const int a = rem / sv.cb, s = kb * sv.cb + rem % sv.cb;
        K_t<R> o;
        kset(o, 0.0, 0.0);
        if (rem < d * sv.cb && s < S) {
            const double2 z = src[(size_t)a * S + s];
            kset(o, z.x, z.y);
        }
        out[i] = o;
    }
}

template <typename R>
cudaError_t launch_to_carry(const double2* src, K_t<R>* dst, int d, int S, StateView<R> sv, int copies,
                            size_t dst_stride, cudaStream_t st) {
    const size_t per = sv.slice();
    const int blocks = (int)((per + 255) / 256 < 1024 ? (per + 255) / 256 : 1024);
    k_to_carry<R><<<dim3(blocks, copies), 256, 0, st>>>(src, dst, d, S, sv, dst_stride);
    return cudaGetLastError();
}

#define QOC_SERIAL_INST(R)                                                                                        \
    template cudaError_t launch_chain<R>(const ChainArgs<R>&, cudaStream_t);                                      \
    template cudaError_t launch_costate<R>(const CostateArgs<R>&, cudaStream_t);                                \
    template cudaError_t launch_to_carry<R>(const double2*, K_t<R>*, int, int, StateView<R>, int, size_t,        \
                                            cudaStream_t);
QOC_SERIAL_INST(float)
QOC_SERIAL_INST(double)

}  // namespace qoc
