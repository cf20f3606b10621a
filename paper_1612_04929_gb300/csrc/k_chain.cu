// Kernels around the slice exponentials and the serial sweeps (k_serial.cu):
//  * k_norms / k_theta  : FP64 induced 1-norms of H_0, H_k, H_det and the global bound
//                         theta = dt max_j (||H_0||_1 + |delta|max ||H_det||_1 + sum_k |u_kj| ||H_k||_1)
//                         that picks one (p, n) for all slices (Sec. III).
//  * k_slice_costs      : per-slice overlaps O_j and forbidden occupations (Table I C5, C6/C7).
//  * k_sources          : dC/dPsi_j of every state-dependent cost term (Appendix A, the source
//                         terms that Algorithm 3 adds at every slice; the fidelity term at j = N).
//  * k_finalize         : FP64 cost reduction (Table I weighted sum), the C3/C4 gradient terms
//                         and the ensemble sum of the per-slice gradients.
//  * k_grad_first_order : the paper's approximate gradient (Eq. 11, dU_j ~ -i dt H_k U_j), an
//                         option in place of the exact adjoint of the truncated exponential.
#include <math.h>

#include <algorithm>

#include "qoc_device.cuh"
#include "qoc_internal.h"

namespace qoc {

// ------------------------------------------------------------------------------------------
// norms and (p, n)
// ------------------------------------------------------------------------------------------
__global__ void k_norms(const double2* __restrict__ mats, int d, double* __restrict__ norms) {
    __shared__ double red[32];
    const double2* A = mats + (size_t)blockIdx.x * d * d;
    double best = 0.0;
    for (int b = threadIdx.x; b < d; b += blockDim.x) {
        double s = 0.0;
        for (int a = 0; a < d; ++a) {
            const double2 z = A[(size_t)a * d + b];
            s += hypot(z.x, z.y);
        }
        best = fmax(best, s);
    }
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        norms[blockIdx.x] = m;
    }
}

cudaError_t launch_norms(const double2* mats, int count, int d, double* norms, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_norms<<<count, 256, 0, st>>>(mats, d, norms);
    return cudaGetLastError();
}

// 1/k!, k = 0 .. kPsCoefs - 1, evaluated at compile time (no FP64 division on the device: the
// FP64 pipe of this part issues a warp instruction in tens of cycles, and the order pick is on the
// critical path of every evaluation)
struct InvFactorials {
    double v[kPsCoefs];
};
constexpr InvFactorials make_inv_factorials() {
    InvFactorials t{};
    double f = 1.0;
    for (int k = 0; k < kPsCoefs; ++k) {
        if (k > 1) f *= k;
        t.v[k] = 1.0 / f;
    }
    return t;
}
__constant__ InvFactorials kInvFact = make_inv_factorials();

// smallest e with 2^e >= b (clamped to [-100, 100]; -100 for b <= 0)
__device__ __forceinline__ int grid_exp(double b) {
    if (!(b > 0.0)) return -100;
    if (!(b < 1e30)) return 100;
    int e = 0;
    const double f = frexp(b, &e);   // b = f 2^e, f in [0.5, 1)
    if (f == 0.5) --e;
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// (p, n) and the split exponential's parameters from the norm bound; thread 0 sets the scalars
// and returns ts = theta / 2^n (negative for a non-finite theta)
__device__ double pick_orders(double theta, double theta_max, double tol, int p_override, int n_override,
                              DevParams* __restrict__ prm, double dt) {
    if (!isfinite(theta)) {   // a NaN or Inf control (device input): flag it, keep the work small
        prm->m_split = 1;
        prm->theta = theta;
        prm->p = 1;
        prm->n = 0;
        prm->s = dt;
        prm->err = kErrNonfinite;
        prm->ex = prm->ez = prm->eu = prm->e2 = prm->e3 = 0;
        return -1.0;
    }
    int n = 0;
    while (ldexp(theta, -n) > theta_max && n < 1000) ++n;
    if (n_override >= 0) n = n_override;
    const double ts = ldexp(theta, -n);
    // 2^n ts^(p+1) / (p+1)! / (1 - ts / (p+2)) <= tol, compared without divisions (FP64 division
    // on one thread is slow here): 2^n ts^(p+1) (p+2) <= tol (p+1)! (p+2 - ts)
    int p = 1;
    double fact = 2.0;     // (p + 1)!
    double pw = ts * ts;   // ts^(p + 1)
    int err = 0;
    for (;;) {
        const double q = p + 2.0;
        if (q > ts && ldexp(pw, n) * q <= tol * fact * (q - ts)) break;
        if (p >= kPMax) { err |= kErrRange; break; }
        ++p;
        fact *= (double)(p + 1);
        pw *= ts;
    }
    if (p_override >= 1) { p = p_override < kPMax ? p_override : kPMax; err &= ~kErrRange; }
    // A rounding error e made in Horner step i + 1 reaches T = Z_1 multiplied by at most
    // ts^i / i! (the X / i' factors of steps i..1).  Steps i <= m need the hi+lo pair; beyond m
    // the factor is below 2^-6 and plain FP32 is exact enough.
    int m = 1;
    double fnum = ts, fden = 1.0;   // ts^m and m!
    while (m < p && fnum > 0.015625 * fden) {
        ++m;
        fnum *= ts;
        fden *= m;
    }
    // Grid exponents of the split FP32 exponential (smallest e with 2^e >= bound, 1/16 margin on
    // the Z bounds).  ||X||_2 <= ||X||_1 <= ts; ||Z_i||_2 <= sum_k ts^k / k! = e^ts; H_j is
    // Hermitian, so X is normal and ||T^(2^m)||_2 <= (1 + R)^(2^n) with R the truncation
    // remainder sum_{k > p} ts^k / k! <= ts^(p+1) / (p+1)! / (1 - ts / (p+2)).
    double rem_t = 1e300;
    if (ts < p + 2.0) {
        double pt = ts;
        for (int k = 2; k <= p + 1; ++k) pt *= ts;
        rem_t = pt * kInvFact.v[p + 1] * (p + 2.0) / (p + 2.0 - ts);
    }
    prm->ex = grid_exp(ts);
    prm->ez = grid_exp(1.0625 * exp(ts));
    const double rn = ldexp(rem_t, n);   // (1 + R)^(2^n) <= 1 + 2^(n+1) R while 2^n R <= 1/2
    prm->eu = grid_exp(1.0625 * (rn <= 0.5 ? 1.0 + 2.0 * rn : exp(ldexp(log1p(rem_t), n))));
    prm->e2 = grid_exp(1.0625 * ts * ts);        // ||X^2||_2 <= ts^2, ||X^3||_2 <= ts^3
    prm->e3 = grid_exp(1.0625 * ts * ts * ts);
    prm->m_split = m;
    prm->theta = theta;
    prm->p = p;
    prm->n = n;
    prm->s = ldexp(dt, -n);
    prm->err = err;
    return ts;
}

// Frozen orders (an evaluation replayed from a captured graph, whose launches were sized for one
// (p, n)): the orders and grid exponents of the capture, `frozen`, stay in force.  The series at
// (p_f, n_f) still meets the tolerance when the minimal p at n_f squarings is at most p_f; the grid
// exponents of the current controls at (p_f, n_f) must not exceed the captured ones (a larger grid
// exponent keeps the grid sums exact and only coarsens the split), nor m_split the captured one.
// Otherwise the evaluation is flagged kErrStale; the frozen values are written either way, so that
// the kernels that read them from device memory agree with the captured launches.
__device__ bool frozen_covers(const DevParams& cur, const DevParams& f) {
    return cur.ex <= f.ex && cur.ez <= f.ez && cur.eu <= f.eu && cur.e2 <= f.e2 && cur.e3 <= f.e3 &&
           cur.m_split <= f.m_split;
}

__global__ void k_theta(const double* __restrict__ u, int M, int N, const double* __restrict__ norms,
                        const double* __restrict__ delta, int E, double dt, double theta_max, double tol,
                        int p_override, int n_override, DevParams* __restrict__ prm,
                        const DevParams* __restrict__ frozen) {
    __shared__ double red[32];
    __shared__ double sh_ts;
    __shared__ int sh_stale;
    double best = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < M; ++k) s += fabs(u[(size_t)k * N + j]) * norms[1 + k];
        best = fmax(best, s);
    }
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        prm->fin_count = 0;   // the final reduction of this evaluation counts its blocks from zero
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) best = fmax(best, red[w]);
        double dmax = 0.0;
        if (delta)
            for (int e = 0; e < E; ++e) dmax = fmax(dmax, fabs(delta[e]));
        const double theta = dt * (norms[0] + dmax * norms[M + 1] + best);
        if (frozen) {
            const int pf = frozen->p, nf = frozen->n;
            double ts = pick_orders(theta, theta_max, tol, -1, nf, prm, dt);   // minimal p at n_f
            int stale = ts >= 0.0 && (prm->p > pf || (prm->err & kErrRange));
            if (ts >= 0.0) {
                ts = pick_orders(theta, theta_max, tol, pf, nf, prm, dt);      // the fields at (p_f, n_f)
                stale |= !frozen_covers(*prm, *frozen);
            }
            prm->p = pf;
            prm->n = nf;
            prm->s = ldexp(dt, -nf);
            prm->ex = frozen->ex;
            prm->ez = frozen->ez;
            prm->eu = frozen->eu;
            prm->e2 = frozen->e2;
            prm->e3 = frozen->e3;
            prm->m_split = frozen->m_split;
            if (stale) prm->err |= kErrStale;
            sh_stale = stale;
            sh_ts = ts;
        } else {
            sh_ts = pick_orders(theta, theta_max, tol, p_override, n_override, prm, dt);
        }
    }
    __syncthreads();
    // Paterson-Stockmeyer tables, one entry per thread: the coefficients 1/k! (k <= p, zero beyond)
    // as FP32 pairs, and the grid exponent of each chain matrix W_q = sum_{k >= 3q} X^(k - 3q) / k!,
    // ||W_q||_2 <= sum_{k = 3q}^{p} ts^(k - 3q) / k! (1/16 margin); W_0 = T takes eu
    const int t = threadIdx.x;
    const double ts = sh_ts;
    const bool ok = ts >= 0.0;
    const int p = ok ? prm->p : 0;
    if (t < kPsCoefs) {
        const double c = (ok && t <= p) ? kInvFact.v[t] : 0.0;
        const float h = (float)c;
        prm->ch[t] = h;
        prm->cl[t] = (float)(c - (double)h);
    }
    if (t < kPsMaxBlocks) {
        int e = ok ? prm->eu : 0;
        if (ok && t > 0) {
            double b = 0.0;   // sum_{k = 3t}^{p} ts^(k - 3t) / k!, by Horner from the top
            for (int k = p; k >= 3 * t; --k) b = fma(b, ts, kInvFact.v[k]);
            e = grid_exp(1.0625 * b);
        }
        if (frozen) {
            if (ok && e > frozen->ew[t] && !sh_stale) atomicOr(&prm->err, kErrStale);
            e = frozen->ew[t];
        }
        prm->ew[t] = e;
    }
}

cudaError_t launch_theta(const double* u, int M, int N, const double* norms, const double* delta, int E,
                         double dt, double theta_max, double tol, int p_override, int n_override,
                         DevParams* prm, cudaStream_t st, const DevParams* frozen) {
    k_theta<<<1, 1024, 0, st>>>(u, M, N, norms, delta, E, dt, theta_max, tol, p_override, n_override, prm, frozen);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// conversions
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void k_convert(const double2* __restrict__ src, C_t<R>* __restrict__ dst, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const double2 z = src[i];
        C_t<R> o;
        o.x = (R)z.x;
        o.y = (R)z.y;
        dst[i] = o;
    }
}

template <typename R>
cudaError_t launch_convert(const double2* src, C_t<R>* dst, size_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const int blocks = (int)((count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096);
    k_convert<R><<<blocks, 256, 0, st>>>(src, dst, count);
    return cudaGetLastError();
}

// row-major d x S (FP64) -> `copies` panel-layout blocks d x Spad (R), zero padding
template <typename R>
__global__ void k_to_panels(const double2* __restrict__ src, C_t<R>* __restrict__ dst, int d, int S, int ncb,
                            int cb, int pstride, size_t dst_stride, size_t src_stride) {
    const size_t per = (size_t)ncb * pstride;
    C_t<R>* out = dst + blockIdx.y * dst_stride;
    src += blockIdx.y * src_stride;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
        const int kb = (int)(i / pstride);
        const int rem = (int)(i - (size_t)kb * pstride);
        const int a = rem / cb, s = kb * cb + rem % cb;
        C_t<R> o;
        o.x = 0;
        o.y = 0;
        if (rem < d * cb && s < S) {
            const double2 z = src[(size_t)a * S + s];
            o.x = (R)z.x;
            o.y = (R)z.y;
        }
        out[i] = o;
    }
}

template <typename R>
cudaError_t launch_to_panels(const double2* src, C_t<R>* dst, int d, int S, StateView<R> sv, int copies,
                             size_t dst_stride, size_t src_stride, cudaStream_t st) {
    const size_t per = sv.slice();
    const int blocks = (int)((per + 255) / 256 < 1024 ? (per + 255) / 256 : 1024);
    k_to_panels<R><<<dim3(blocks, copies), 256, 0, st>>>(src, dst, d, S, sv.ncb, sv.cb, sv.pstride, dst_stride,
                                                         src_stride);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// per-slice costs and sources
// ------------------------------------------------------------------------------------------
// WARP: one warp per slice (8 slices per block) for panels of at most 256 elements, with warp
// shuffles for the sums; else one block per slice
template <typename R, bool WARP>
__global__ void __launch_bounds__(256)
k_slice_costs(int d, StateView<R> sv, int j0, int wlen, int N, const C_t<R>* __restrict__ states, int wmax,
              CostView<R> cv, double2* __restrict__ Oj, double* __restrict__ C5j, double2* __restrict__ Ofin) {
    using C = C_t<R>;
    __shared__ double red[32];
    const int jl = WARP ? blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) : blockIdx.x;
    if (WARP && jl >= wlen) return;   // whole warps leave; no block barrier in this mode
    const int e = blockIdx.y, j = j0 + jl, cb = sv.cb, ps = sv.pstride;
    const int t0 = WARP ? (threadIdx.x & 31) : threadIdx.x, ts = WARP ? 32 : blockDim.x;
    const size_t slice = sv.slice();
    const C* psi = states + ((size_t)e * (wmax + 1) + jl + 1) * slice;
    const C* T = cv.path ? cv.path + (size_t)j * slice : cv.psiT;
    const bool last = (j == N - 1);
    double ore = 0, oim = 0, c5 = 0, fre = 0, fim = 0;
    for (size_t i = t0; i < slice; i += ts) {
        const int kb = (int)(i / ps);
        const int rem = (int)(i - (size_t)kb * ps);
        if (rem >= d * cb) continue;
        const int a = rem / cb, s = kb * cb + rem % cb;
        const double w = cv.w[s];
        if (w == 0.0) continue;
        const C z = psi[i], t = T[i];
        ore += w * ((double)t.x * z.x + (double)t.y * z.y);
        oim += w * ((double)t.x * z.y - (double)t.y * z.x);
        if (cv.fmask[a]) c5 += w * ((double)z.x * z.x + (double)z.y * z.y);
        if (last) {
            const C f = cv.psiT[i];
            fre += w * ((double)f.x * z.x + (double)f.y * z.y);
            fim += w * ((double)f.x * z.y - (double)f.y * z.x);
        }
    }
    auto sum = [&](double v) {
        if (WARP) {
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            return v;
        }
        return block_sum(v, red);
    };
    ore = sum(ore);
    oim = sum(oim);
    c5 = sum(c5);
    if (last) {   // uniform over the warp (WARP) or the block
        fre = sum(fre);
        fim = sum(fim);
    }
    if (t0 == 0) {
        Oj[(size_t)e * N + j] = make_double2(ore / cv.Wsum, oim / cv.Wsum);
        C5j[(size_t)e * N + j] = c5;
        if (last) Ofin[e] = make_double2(fre / cv.Wsum, fim / cv.Wsum);
    }
}

template <typename R>
cudaError_t launch_slice_costs(int d, StateView<R> sv, int j0, int wlen, int N, int E, const C_t<R>* states, int wmax,
                               const CostView<R>& cv, double2* Oj, double* C5j, double2* Ofin, cudaStream_t st) {
    if (sv.slice() <= 256)
        k_slice_costs<R, true><<<dim3((wlen + 7) / 8, E), 256, 0, st>>>(d, sv, j0, wlen, N, states, wmax, cv, Oj,
                                                                         C5j, Ofin);
    else
        k_slice_costs<R, false><<<dim3(wlen, E), 256, 0, st>>>(d, sv, j0, wlen, N, states, wmax, cv, Oj, C5j, Ofin);
    return cudaGetLastError();
}

template <typename R, bool WARP>
__global__ void __launch_bounds__(256)
k_sources(int d, StateView<R> sv, int j0, int wlen, int N, int E, const C_t<R>* __restrict__ states, int wmax,
          CostView<R> cv, const double2* __restrict__ Oj, const double2* __restrict__ Ofin, C_t<R>* __restrict__ src) {
    using C = C_t<R>;
    const int jl = WARP ? blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) : blockIdx.x;
    if (WARP && jl >= wlen) return;
    const int t0 = WARP ? (threadIdx.x & 31) : threadIdx.x, ts = WARP ? 32 : blockDim.x;
    const int e = blockIdx.y, j = j0 + jl, cb = sv.cb, ps = sv.pstride;
    const size_t slice = sv.slice();
    const C* psi = states + ((size_t)e * (wmax + 1) + jl + 1) * slice;
    const C* T = cv.path ? cv.path + (size_t)j * slice : cv.psiT;
    C* out = src + ((size_t)e * wmax + jl) * slice;
    const double invE = 1.0 / E;
    const double2 o = Oj[(size_t)e * N + j];
    const bool last = (j == N - 1);
    const double2 of = last ? Ofin[e] : make_double2(0.0, 0.0);
    // coefficient of T:  -(2 a67 / N) O_j w / W ;  of psiT at j = N: -2 a_fid O_N w / W
    const double ct = -2.0 * cv.alpha[4] / N * invE / cv.Wsum;
    const double cf = -2.0 * cv.alpha[0] * invE / cv.Wsum;
    const double c5 = 2.0 * cv.alpha[3] * invE;
    for (size_t i = t0; i < slice; i += ts) {
        const int kb = (int)(i / ps);
        const int rem = (int)(i - (size_t)kb * ps);
        const bool valid = rem < d * cb;
        const int a = rem / cb, s = kb * cb + rem % cb;
        const double w = valid ? cv.w[s] : 0.0;
        double vx = 0.0, vy = 0.0;
        if (w != 0.0) {
            const C t = T[i];
            vx = ct * w * (o.x * t.x - o.y * t.y);
            vy = ct * w * (o.x * t.y + o.y * t.x);
            if (cv.fmask[a]) {
                const C z = psi[i];
                vx += c5 * w * z.x;
                vy += c5 * w * z.y;
            }
            if (last) {
                const C f = cv.psiT[i];
                vx += cf * w * (of.x * f.x - of.y * f.y);
                vy += cf * w * (of.x * f.y + of.y * f.x);
            }
        }
        C r;
        r.x = (R)vx;
        r.y = (R)vy;
        out[i] = r;
    }
}

template <typename R>
cudaError_t launch_sources(int d, StateView<R> sv, int j0, int wlen, int N, int E, const C_t<R>* states, int wmax,
                           const CostView<R>& cv, const double2* Oj, const double2* Ofin, C_t<R>* src,
                           cudaStream_t st) {
    if (sv.slice() <= 256)
        k_sources<R, true><<<dim3((wlen + 7) / 8, E), 256, 0, st>>>(d, sv, j0, wlen, N, E, states, wmax, cv, Oj, Ofin,
                                                                     src);
    else
        k_sources<R, false><<<dim3(wlen, E), 256, 0, st>>>(d, sv, j0, wlen, N, E, states, wmax, cv, Oj, Ofin, src);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// final FP64 reduction
// ------------------------------------------------------------------------------------------
struct Alpha5 { double a[5]; };

__global__ void __launch_bounds__(256)
k_finalize(int E, int M, int N, const double* __restrict__ u, Alpha5 al, const double2* __restrict__ Oj,
           const double* __restrict__ C5j, const double2* __restrict__ Ofin, const double* __restrict__ gpart,
           double* __restrict__ grad, double* __restrict__ out, DevParams* __restrict__ prm) {
    __shared__ double red[32];
    __shared__ bool last;
    const int tid = threadIdx.x, nb = gridDim.x;
    const int gt = blockIdx.x * blockDim.x + tid, gs = nb * blockDim.x;
    double c3 = 0, c4 = 0, c5 = 0, t67 = 0;
    bool finite = true;   // outputs scanned for NaN / Inf (a flag, read by the host)
    for (int i = gt; i < M * N; i += gs) {
        const int k = i / N, j = i - k * N;
        const double x = u[i];
        c3 += x * x;
        if (j > 0) {
            const double dx = x - u[i - 1];
            c4 += dx * dx;
        }
        double g = 0.0;
        for (int e = 0; e < E; ++e) g += gpart[((size_t)e * M + k) * N + j];
        g += al.a[1] * 2.0 * x;
        double gv = 0.0;
        if (j > 0) gv += 2.0 * (x - u[i - 1]);
        if (j < N - 1) gv -= 2.0 * (u[i + 1] - x);
        g += al.a[2] * gv;
        grad[i] = g;
        finite = finite && isfinite(g);
    }
    if (!finite) atomicOr(&prm->err, kErrNonfinite);
    for (int i = gt; i < E * N; i += gs) {
        c5 += C5j[i];
        const double2 o = Oj[i];
        t67 += o.x * o.x + o.y * o.y;
    }
    c3 = block_sum(c3, red);
    c4 = block_sum(c4, red);
    c5 = block_sum(c5, red);
    t67 = block_sum(t67, red);
    // the partial sums of every block, then the last block to finish adds them in block order
    // (the same order every time: the result does not depend on which block finishes last)
    if (tid == 0) {
        double* pp = prm->fin_part + 4 * blockIdx.x;
        pp[0] = c3;
        pp[1] = c4;
        pp[2] = c5;
        pp[3] = t67;
        __threadfence();
        last = atomicAdd(&prm->fin_count, 1u) == (unsigned)(nb - 1);
    }
    __syncthreads();
    if (!last || tid != 0) return;
    __threadfence();
    c3 = c4 = c5 = t67 = 0.0;
    const volatile double* vp = prm->fin_part;
    for (int b = 0; b < nb; ++b) {
        c3 += vp[4 * b];
        c4 += vp[4 * b + 1];
        c5 += vp[4 * b + 2];
        t67 += vp[4 * b + 3];
    }
    prm->fin_count = 0;
    double fid = 0.0;
    for (int e = 0; e < E; ++e) fid += 1.0 - (Ofin[e].x * Ofin[e].x + Ofin[e].y * Ofin[e].y);
    fid /= E;
    c5 /= E;
    const double c67 = 1.0 - t67 / ((double)N * E);
    out[1] = fid;
    out[2] = c3;
    out[3] = c4;
    out[4] = c5;
    out[5] = c67;
    out[0] = al.a[0] * fid + al.a[1] * c3 + al.a[2] * c4 + al.a[3] * c5 + al.a[4] * c67;
    if (!isfinite(out[0])) atomicOr(&prm->err, kErrNonfinite);
    // every failure flagged on the device in this evaluation (non-finite input or result, a
    // Taylor order at its cap, a bounded wait that ran out) also leaves C = NaN, so a caller
    // that cannot read the flag still cannot mistake the result for a valid one
    if (*(volatile int*)&prm->err != 0) out[0] = __longlong_as_double(0x7ff8000000000000ll);
}

cudaError_t launch_finalize(int E, int M, int N, const double* u, const double* alpha, const double2* Oj,
                            const double* C5j, const double2* Ofin, const double* gpart, double* grad, double* out,
                            DevParams* prm, cudaStream_t st) {
    Alpha5 al;
    for (int i = 0; i < 5; ++i) al.a[i] = alpha[i];
    const int work = std::max(M * N, E * N);
    const int nb = std::max(1, std::min(kFinBlocks, (work + 255) / 256));
    k_finalize<<<nb, 256, 0, st>>>(E, M, N, u, al, Oj, C5j, Ofin, gpart, grad, out, prm);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// first-order gradient (Eq. 11): dC/du_{k,j} = Re tr(Ubar_j^dag (-i dt H_k U_j)) with
// Ubar_j = G_j Psi_{j-1}^dag; since U_j Ubar_j^dag = Psi_j G_j^dag this is
//   dt Im sum_s G_j[:, s]^dag H_k Psi_j[:, s],
// O(M d^2 S) per slice and no exponential.  One CTA per (slice, member).
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
k_grad_first_order(SysView<R> sys, StateView<R> sv, int j0, const C_t<R>* __restrict__ states,
                   const C_t<R>* __restrict__ Gbuf, int wmax, double dt, double* __restrict__ gpart) {
    using C = C_t<R>;
    __shared__ double red[32];
    const int jl = blockIdx.x, e = blockIdx.y, j = j0 + jl;
    const int d = sys.d, S = sv.S;
    const size_t slice = sv.slice(), dd = (size_t)d * d;
    const C* Gj = Gbuf + ((size_t)e * wmax + jl) * slice;
    const C* Pj = states + ((size_t)e * (wmax + 1) + jl + 1) * slice;   // Psi_j, after slice j
    auto at = [&](int a, int s) { return (size_t)(s / sv.cb) * sv.pstride + (size_t)a * sv.cb + (s % sv.cb); };
    for (int k = 0; k < sys.M; ++k) {
        const C* hk = sys.Hk + (size_t)k * dd;
        double v = 0.0;
        for (int idx = threadIdx.x; idx < d * S; idx += blockDim.x) {   // (a, s): conj(G[a][s]) (H_k Psi)[a][s]
            const int a = idx / S, s = idx - a * S;
            double hr = 0.0, hi = 0.0;
            for (int b = 0; b < d; ++b) {
                const C h = hk[(size_t)a * d + b], q = Pj[at(b, s)];
                hr += (double)h.x * (double)q.x - (double)h.y * (double)q.y;
                hi += (double)h.x * (double)q.y + (double)h.y * (double)q.x;
            }
            const C g = Gj[at(a, s)];
            v += (double)g.x * hi - (double)g.y * hr;   // Im(conj(g) (hr + i hi))
        }
        v = block_sum(v, red);
        if (threadIdx.x == 0) gpart[((size_t)e * sys.M + k) * sys.N + j] = dt * v;
    }
}

template <typename R>
cudaError_t launch_grad_first_order(const SysView<R>& sys, const StateView<R>& sv, int j0, int wlen, int E,
                                    const C_t<R>* states, const C_t<R>* Gbuf, int wmax, double dt, double* gpart,
                                    cudaStream_t st) {
    if (sys.M == 0) return cudaSuccess;
    k_grad_first_order<R><<<dim3(wlen, E), 256, 0, st>>>(sys, sv, j0, states, Gbuf, wmax, dt, gpart);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// instantiations
// ------------------------------------------------------------------------------------------
#define QOC_INST(R)                                                                                              \
    template cudaError_t launch_convert<R>(const double2*, C_t<R>*, size_t, cudaStream_t);                       \
    template cudaError_t launch_to_panels<R>(const double2*, C_t<R>*, int, int, StateView<R>, int, size_t,       \
                                             size_t, cudaStream_t);                                              \
    template cudaError_t launch_slice_costs<R>(int, StateView<R>, int, int, int, int, const C_t<R>*, int,        \
                                               const CostView<R>&, double2*, double*, double2*, cudaStream_t);   \
    template cudaError_t launch_sources<R>(int, StateView<R>, int, int, int, int, const C_t<R>*, int,            \
                                           const CostView<R>&, const double2*, const double2*, C_t<R>*,          \
                                           cudaStream_t);                                                        \
    template cudaError_t launch_grad_first_order<R>(const SysView<R>&, const StateView<R>&, int, int, int,       \
                                                    const C_t<R>*, const C_t<R>*, int, double, double*,          \
                                                    cudaStream_t);                                               \

QOC_INST(float)
QOC_INST(double)

}  // namespace qoc
