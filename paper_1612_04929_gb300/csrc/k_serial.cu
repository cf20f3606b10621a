// Serial recursions of one evaluation (the only sequential dependency of the method):
//   forward      Psi_j = U_j Psi_{j-1}                                     (Eqs. 2, 4)
//   costate      G_{j-1} = U_j^dag G_j + src_{j-1}                          (Appendix A, Alg. 1-3)
// Both run one CTA per (column panel, ensemble member) and stream the next slice propagators
// (and sources) into a shared-memory ring with cp.async while the current step computes.
//
// The running block is carried in extended precision: FP64 in the FP64 form, and an unevaluated
// hi + lo pair of FP32 numbers in the FP32 form (exact products via FMA, error-free TwoSum
// accumulation).  Over thousands of slices the FP32 rounding of a plainly carried state adds
// up to gradient errors near 1e-5; the pair keeps the recursion at ~1e-12 while U_j, the stored
// states and costates (inputs of the parallel kernels) stay FP32.
//
// Checkpointing: the forward sweep stores the carried block every `seg` slices (seg = ceil(sqrt
// N) by default).  In the backward sweep the states of a wave are regenerated from those
// checkpoints, one CTA per checkpoint segment in parallel (mode 1 below), so regeneration
// costs seg serial steps whatever the wave length.
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
// (hi, lo) += a * (bh + bl) with the exact product residual
__device__ __forceinline__ void pair_mac(float& hi, float& lo, float a, float bh, float bl) {
    const float p = a * bh;
    lo += fmaf(a, bh, -p) + a * bl;
    two_sum_acc(hi, lo, p);
}

// acc += u x    (u plain, x carried)
__device__ __forceinline__ void kmac(float4& acc, const float2 u, const float4 x) {
    pair_mac(acc.x, acc.z, u.x, x.x, x.z);
    pair_mac(acc.x, acc.z, -u.y, x.y, x.w);
    pair_mac(acc.y, acc.w, u.x, x.y, x.w);
    pair_mac(acc.y, acc.w, u.y, x.x, x.z);
}
__device__ __forceinline__ void kmac(double2& acc, const double2 u, const double2 x) { cfma(acc, u, x); }
// acc += conj(u) x
__device__ __forceinline__ void kmac_cj(float4& acc, const float2 u, const float4 x) {
    pair_mac(acc.x, acc.z, u.x, x.x, x.z);
    pair_mac(acc.x, acc.z, u.y, x.y, x.w);
    pair_mac(acc.y, acc.w, u.x, x.y, x.w);
    pair_mac(acc.y, acc.w, -u.y, x.x, x.z);
}
__device__ __forceinline__ void kmac_cj(double2& acc, const double2 u, const double2 x) { cfma_cj(acc, u, x); }

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

// y = U x on one d x cb panel: g lanes per output sum b = q, q + g, ... then a shuffle reduction
template <typename C, typename K>
__device__ __forceinline__ void mv_U(const C* __restrict__ U, const K* __restrict__ x, K* __restrict__ y, int d,
                                     int cb, int g) {
    const int O = d * cb;
    const int ngroups = blockDim.x / g;
    const int gi = threadIdx.x / g, q = threadIdx.x - gi * g;
    for (int base = 0; base < O; base += ngroups) {
        const int o = base + gi;
        K acc = kzero<K>();
        int a = 0, sl = 0;
        if (o < O) {
            a = o / cb;
            sl = o - a * cb;
            const C* Ur = U + (size_t)a * d;
            for (int b = q; b < d; b += g) kmac(acc, Ur[b], x[b * cb + sl]);
        }
        for (int off = g >> 1; off > 0; off >>= 1) kadd(acc, kshfl_xor(acc, off));
        if (o < O && q == 0) {
            knorm(acc);
            y[a * cb + sl] = acc;
        }
    }
}

// y = U^dag x + add: lanes over outputs (contiguous reads of U[b][a]); for small panels the b
// range is split over the warps and the partials summed through `red`
template <typename C, typename K>
__device__ __forceinline__ void mv_UH(const C* __restrict__ U, const K* __restrict__ x, K* __restrict__ y,
                                      const C* __restrict__ add, int d, int cb, K* __restrict__ red) {
    const int O = d * cb;
    if (O >= (int)blockDim.x) {
        for (int o = threadIdx.x; o < O; o += blockDim.x) {
            const int a = o / cb, sl = o - a * cb;
            K acc = kzero<K>();
            for (int b = 0; b < d; ++b) kmac_cj(acc, U[(size_t)b * d + a], x[b * cb + sl]);
            if (add) kadd(acc, kfrom(add[o]));
            knorm(acc);
            y[o] = acc;
        }
        __syncthreads();
        return;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int chunk = (d + nw - 1) / nw;
    const int b0 = w * chunk, b1 = min(d, b0 + chunk);
    for (int o = l; o < O; o += 32) {
        const int a = o / cb, sl = o - a * cb;
        K acc = kzero<K>();
        for (int b = b0; b < b1; ++b) kmac_cj(acc, U[(size_t)b * d + a], x[b * cb + sl]);
        red[w * O + o] = acc;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < O; o += blockDim.x) {
        K acc = add ? kfrom(add[o]) : kzero<K>();
        for (int ww = 0; ww < nw; ++ww) kadd(acc, red[ww * O + o]);
        knorm(acc);
        y[o] = acc;
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// forward propagation (mode 0) and checkpoint replay (mode 1)
// ------------------------------------------------------------------------------------------
template <typename R, int RING>
__global__ void __launch_bounds__(256)
k_chain(int d, StateView<R> sv, int wlen, int seg, int mode, K_t<R>* __restrict__ ckpt, size_t ck_estride, int seg0,
        int nseg_total, const C_t<R>* __restrict__ Ubuf, long long ustride, int wmax, C_t<R>* __restrict__ states,
        int g) {
    using C = C_t<R>;
    using K = K_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int kb = blockIdx.x, e = blockIdx.y, z = blockIdx.z, tid = threadIdx.x, cb = sv.cb;
    const size_t slice = sv.slice(), panel = (size_t)d * cb;
    const size_t ub = ring_bytes((size_t)d * d, sizeof(C));
    unsigned char* ring = smraw;
    K* xa = reinterpret_cast<K*>(smraw + RING * ub);
    K* xb = xa + panel;
    const int t0 = (mode == 0) ? 0 : z * seg;
    const int t1 = (mode == 0) ? wlen : min(wlen, t0 + seg);
    if (t0 >= t1) return;
    K* ck_e = ckpt + e * ck_estride;
    const K* s0 = ck_e + (size_t)(seg0 + t0 / seg) * slice + (size_t)kb * sv.pstride;
    C* sdst = states + (size_t)e * (wmax + 1) * slice + (size_t)kb * sv.pstride;
    for (int i = tid; i < (int)panel; i += blockDim.x) {
        const K v = s0[i];
        xa[i] = v;
        sdst[(size_t)t0 * slice + i] = kround(v);
    }
    const C* Ue = Ubuf + (size_t)e * wmax * ustride;
#pragma unroll 1
    for (int t = 0; t < RING - 1; ++t) {
        if (t0 + t < t1) ring_issue(ring + t * ub, Ue + (size_t)(t0 + t) * ustride, ub);
        cp_async_commit();
    }
#pragma unroll 1
    for (int t = t0; t < t1; ++t) {
        const int k = t - t0;
        const int tn = t + RING - 1;
        if (tn < t1) ring_issue(ring + ((k + RING - 1) % RING) * ub, Ue + (size_t)tn * ustride, ub);
        cp_async_commit();
        cp_async_wait<RING - 1>();
        __syncthreads();
        const C* U = reinterpret_cast<const C*>(ring + (k % RING) * ub);
        mv_U<C, K>(U, xa, xb, d, cb, g);
        __syncthreads();
        C* dst = sdst + (size_t)(t + 1) * slice;
        for (int i = tid; i < (int)panel; i += blockDim.x) dst[i] = kround(xb[i]);
        if (mode == 0 && (t + 1) % seg == 0) {
            const int slot = seg0 + (t + 1) / seg;
            if (slot < nseg_total) {
                K* c = ck_e + (size_t)slot * slice + (size_t)kb * sv.pstride;
                for (int i = tid; i < (int)panel; i += blockDim.x) c[i] = xb[i];
            }
        }
        K* tmp = xa; xa = xb; xb = tmp;
    }
}

static int pick_group(int d, int cb, int threads, int term_cost) {
    // minimise ceil(O / (threads / g)) * (term_cost ceil(d / g) + 8 log2 g) over g in {1, ..., 32}
    const int O = d * cb;
    int best = 1;
    long best_cost = -1;
    for (int g = 1, lg = 0; g <= 32; g <<= 1, ++lg) {
        const long iters = (O + threads / g - 1) / (threads / g);
        const long cost = iters * ((long)term_cost * ((d + g - 1) / g) + 8 * lg);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = g; }
    }
    return best;
}

template <typename R, int RING>
static cudaError_t chain_ring(const ChainArgs<R>& a, size_t smem, cudaStream_t st) {
    cudaError_t err = cudaFuncSetAttribute(k_chain<R, RING>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int g = pick_group(a.d, a.sv.cb, 256, sizeof(R) == 4 ? 10 : 4);
    const int nz = a.mode == 0 ? 1 : (a.wlen + a.seg - 1) / a.seg;
    k_chain<R, RING><<<dim3(a.sv.ncb, a.E, nz), 256, smem, st>>>(a.d, a.sv, a.wlen, a.seg, a.mode, a.ckpt, a.ck_estride,
                                                                  a.seg0, a.nseg_total, a.Ubuf, a.ustride, a.wmax,
                                                                  a.states, g);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_chain(const ChainArgs<R>& a, cudaStream_t st) {
    const size_t ub = ring_bytes((size_t)a.d * a.d, sizeof(C_t<R>));
    const size_t xs = 2 * (size_t)a.d * a.sv.cb * sizeof(K_t<R>);
    for (int ring : {4, 2, 1}) {
        const size_t smem = ring * ub + xs;
        if (smem > kMaxDynSmem) continue;
        if (ring == 4) return chain_ring<R, 4>(a, smem, st);
        if (ring == 2) return chain_ring<R, 2>(a, smem, st);
        return chain_ring<R, 1>(a, smem, st);
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------------------------
// backward costate sweep over one wave
// ------------------------------------------------------------------------------------------
template <typename R, int RING>
__global__ void __launch_bounds__(256)
k_costate(int d, StateView<R> sv, int wlen, const C_t<R>* __restrict__ Ubuf, long long ustride, int wmax,
          const C_t<R>* __restrict__ src, K_t<R>* __restrict__ carry, C_t<R>* __restrict__ Gbuf) {
    using C = C_t<R>;
    using K = K_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int kb = blockIdx.x, e = blockIdx.y, tid = threadIdx.x, cb = sv.cb;
    const size_t slice = sv.slice(), panel = (size_t)d * cb;
    const size_t ub = ring_bytes((size_t)d * d, sizeof(C));
    const size_t pb = (size_t)sv.pstride * sizeof(C);
    const size_t slot = ub + pb;
    unsigned char* ring = smraw;
    K* xa = reinterpret_cast<K*>(smraw + RING * slot);
    K* xb = xa + panel;
    K* red = xb + panel;      // 8 * panel partials
    const C* Ue = Ubuf + (size_t)e * wmax * ustride;
    const C* Se = src + (size_t)e * wmax * slice + (size_t)kb * sv.pstride;
    C* Ge = Gbuf + (size_t)e * wmax * slice + (size_t)kb * sv.pstride;
    K* ce = carry + (size_t)e * slice + (size_t)kb * sv.pstride;
    {   // G at the last slice of the wave = carry + src
        const C* s_last = Se + (size_t)(wlen - 1) * slice;
        for (int i = tid; i < (int)panel; i += blockDim.x) {
            K v = ce[i];
            kadd(v, kfrom(s_last[i]));
            knorm(v);
            xa[i] = v;
        }
    }
    auto issue = [&](int t) {     // step t handles slice jl = wlen - 1 - t: U_jl and src_{jl-1}
        const int jl = wlen - 1 - t;
        unsigned char* sl = ring + (t % RING) * slot;
        ring_issue(sl, Ue + (size_t)jl * ustride, ub);
        if (jl > 0) ring_issue(sl + ub, Se + (size_t)(jl - 1) * slice, pb);
    };
#pragma unroll 1
    for (int t = 0; t < RING - 1; ++t) {
        if (t < wlen) issue(t);
        cp_async_commit();
    }
    __syncthreads();
#pragma unroll 1
    for (int t = 0; t < wlen; ++t) {
        const int jl = wlen - 1 - t;
        const int tn = t + RING - 1;
        if (tn < wlen) issue(tn);
        cp_async_commit();
        C* gd = Ge + (size_t)jl * slice;
        for (int i = tid; i < (int)panel; i += blockDim.x) gd[i] = kround(xa[i]);
        cp_async_wait<RING - 1>();
        __syncthreads();
        const unsigned char* sl = ring + (t % RING) * slot;
        const C* U = reinterpret_cast<const C*>(sl);
        const C* add = (jl > 0) ? reinterpret_cast<const C*>(sl + ub) : nullptr;
        mv_UH<C, K>(U, xa, xb, add, d, cb, red);
        K* tmp = xa; xa = xb; xb = tmp;
    }
    for (int i = tid; i < (int)panel; i += blockDim.x) ce[i] = xa[i];
}

template <typename R, int RING>
static cudaError_t costate_ring(int d, StateView<R> sv, int wlen, int E, const C_t<R>* Ubuf, long long ustride,
                                int wmax, const C_t<R>* src, K_t<R>* carry, C_t<R>* Gbuf, size_t smem, cudaStream_t st) {
    cudaError_t err = cudaFuncSetAttribute(k_costate<R, RING>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_costate<R, RING><<<dim3(sv.ncb, E), 256, smem, st>>>(d, sv, wlen, Ubuf, ustride, wmax, src, carry, Gbuf);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_costate(int d, StateView<R> sv, int wlen, int E, const C_t<R>* Ubuf, long long ustride, int wmax,
                           const C_t<R>* src, K_t<R>* carry, C_t<R>* Gbuf, cudaStream_t st) {
    const size_t panel = (size_t)d * sv.cb;
    const size_t ub = ring_bytes((size_t)d * d, sizeof(C_t<R>));
    const size_t pb = (size_t)sv.pstride * sizeof(C_t<R>);
    const size_t fixed = (2 + 8) * panel * sizeof(K_t<R>);
    for (int ring : {4, 2, 1}) {
        const size_t smem = ring * (ub + pb) + fixed;
        if (smem > kMaxDynSmem) continue;
        if (ring == 4) return costate_ring<R, 4>(d, sv, wlen, E, Ubuf, ustride, wmax, src, carry, Gbuf, smem, st);
        if (ring == 2) return costate_ring<R, 2>(d, sv, wlen, E, Ubuf, ustride, wmax, src, carry, Gbuf, smem, st);
        return costate_ring<R, 1>(d, sv, wlen, E, Ubuf, ustride, wmax, src, carry, Gbuf, smem, st);
    }
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
    template cudaError_t launch_costate<R>(int, StateView<R>, int, int, const C_t<R>*, long long, int,           \
                                           const C_t<R>*, K_t<R>*, C_t<R>*, cudaStream_t);                        \
    template cudaError_t launch_to_carry<R>(const double2*, K_t<R>*, int, int, StateView<R>, int, size_t,        \
                                            cudaStream_t);
QOC_SERIAL_INST(float)
QOC_SERIAL_INST(double)

}  // namespace qoc
