// qoc_evaluate_static: one cost + gradient evaluation that allocates no memory.
//
// Who needs it: callers that may not allocate device memory at the moment they evaluate, for
// example code running while a CUDA stream is being captured into a graph (cudaMalloc is not
// allowed there), real-time control loops that forbid allocator calls (they can block and take
// locks), or hosts whose memory is managed by a pool that must not be bypassed.  The regular
// entry points allocate their working buffers inside a context; this one instead uses a fixed
// device array compiled into the library, so it needs no context and no allocation at all.
//
// The array is a file-scope __device__ variable of QOC_STATIC_ARENA_BYTES bytes.  Every GPU
// that loads the library holds it until the process exits.  On the host its name only stands
// for the variable, so its device address is looked up once per device, with that device
// current, by cudaGetSymbolAddress on the first call made on that device.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/qoc.h"
#include "qoc_internal.h"

using namespace qoc;

namespace {

static __device__ __align__(256) unsigned char g_arena[QOC_STATIC_ARENA_BYTES];

constexpr int kMaxDevices = 64;
void* g_arena_addr[kMaxDevices] = {nullptr};

// carve 256-byte-aligned pieces out of the arena: offsets first (no base), pointers once the
// device address is known
struct Carver {
    uintptr_t base = 0;
    size_t used = 0;
    template <typename T>
    T* take(size_t count) {
        used = (used + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base + used);
        used += count * sizeof(T);
        return p;
    }
};

// The arena's layout for one problem; with base = 0 only the size (used) is meaningful.
template <typename R>
struct StaticLayout {
    using C = C_t<R>;
    using K = K_t<R>;
    DevParams* prm;
    double* norms;
    C *psiT, *Ubuf, *states, *Gbuf, *src;
    K *ckpt, *carry;
    double2 *Oj, *Ofin;
    double *C5j, *gpart, *colw;
    int* fmask_zero;
    size_t used;
    StaticLayout(uintptr_t base, int d, int M, int N, size_t slice, int Spad, long long ustride) {
        Carver cv;
        cv.base = base;
        prm = cv.take<DevParams>(1);
        norms = cv.take<double>(M + 2);
        psiT = cv.take<C>(slice);
        ckpt = cv.take<K>(slice);
        Ubuf = cv.take<C>((size_t)N * ustride);
        states = cv.take<C>((size_t)(N + 1) * slice);
        Gbuf = cv.take<C>((size_t)N * slice);
        src = cv.take<C>((size_t)N * slice);
        carry = cv.take<K>(slice);
        Oj = cv.take<double2>(N);
        C5j = cv.take<double>(N);
        Ofin = cv.take<double2>(1);
        gpart = cv.take<double>((size_t)M * N + 1);
        colw = cv.take<double>(Spad);
        fmask_zero = cv.take<int>(d);
        used = cv.used;
    }
};

__global__ void k_static_weights(double* w, int S, int Spad) {
    for (int s = threadIdx.x; s < Spad; s += blockDim.x) w[s] = (s < S) ? 1.0 : 0.0;
}

}  // namespace

extern "C" qoc_status qoc_evaluate_static(int d, int M, int N, int S, double dt, const double* H0_dev,
                                          const double* Hk_dev, const double* u_dev, const double* psi0_dev,
                                          const double* psiT_dev, const int* fmask_dev, const double* alpha,
                                          double* grad_dev, double* out_dev, void* stream) {
    if (!H0_dev || (M > 0 && (!Hk_dev || !u_dev)) || !psi0_dev || !psiT_dev || !alpha || !out_dev ||
        (M > 0 && !grad_dev))
        return QOC_ERR_ARG;
    if (d < 1 || d > fused_max_d<double>() || M < 0 || M > kMaxControls || N < 1 || S < 1 || S > d)
        return QOC_ERR_SHAPE;
    if (!(dt > 0.0)) return QOC_ERR_ARG;
    using R = double;
    using C = C_t<R>;
    using K = K_t<R>;
    StateView<R> sv;
    sv.cb = S < 8 ? S : 8;
    sv.ncb = (S + sv.cb - 1) / sv.cb;
    sv.Spad = sv.ncb * sv.cb;
    sv.pstride = d * sv.cb;                       // 16-byte elements: always aligned
    sv.S = S;
    const size_t slice = sv.slice();
    const long long ustride = 2 * (((long long)d * d + 15) / 16 * 16);   // U_j and U_j^dag
    // the size check comes before any CUDA call
    if (StaticLayout<R>(0, d, M, N, slice, sv.Spad, ustride).used > QOC_STATIC_ARENA_BYTES)
        return QOC_ERR_SHAPE;   // the problem does not fit
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QOC_ERR_CUDA;
    if (!g_arena_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_arena) != cudaSuccess || !p) return QOC_ERR_CUDA;
        g_arena_addr[dev] = p;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const StaticLayout<R> L(reinterpret_cast<uintptr_t>(g_arena_addr[dev]), d, M, N, slice, sv.Spad, ustride);
    DevParams* prm = L.prm;
    double* norms = L.norms;
    C* psiT = L.psiT;
    K* ckpt = L.ckpt;
    C* Ubuf = L.Ubuf;
    C* states = L.states;
    C* Gbuf = L.Gbuf;
    C* src = L.src;
    K* carry = L.carry;
    double2* Oj = L.Oj;
    double* C5j = L.C5j;
    double2* Ofin = L.Ofin;
    double* gpart = L.gpart;
    double* colw = L.colw;
    int* fmask_zero = L.fmask_zero;

    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    const double2* H0 = reinterpret_cast<const double2*>(H0_dev);
    const double2* Hk = reinterpret_cast<const double2*>(Hk_dev);
    // state a previous call left behind that must start at zero: the unused norm slot of the
    // detuning operator, the costate carry and (without forbidden states) the mask
    if (!ok(cudaMemsetAsync(norms + M + 1, 0, sizeof(double), st))) return QOC_ERR_CUDA;
    if (!ok(cudaMemsetAsync(carry, 0, slice * sizeof(K), st))) return QOC_ERR_CUDA;
    if (!fmask_dev && !ok(cudaMemsetAsync(fmask_zero, 0, d * sizeof(int), st))) return QOC_ERR_CUDA;
    if (!ok(launch_norms(H0, 1, d, norms, st))) return QOC_ERR_CUDA;
    if (M > 0 && !ok(launch_norms(Hk, M, d, norms + 1, st))) return QOC_ERR_CUDA;
    k_static_weights<<<1, 64, 0, st>>>(colw, S, sv.Spad);
    if (!ok(cudaGetLastError())) return QOC_ERR_CUDA;
    if (!ok(launch_to_panels<R>(reinterpret_cast<const double2*>(psiT_dev), psiT, d, S, sv, 1, 0, 0, st)))
        return QOC_ERR_CUDA;
    if (!ok(launch_to_carry<R>(reinterpret_cast<const double2*>(psi0_dev), ckpt, d, S, sv, 1, slice, st)))
        return QOC_ERR_CUDA;

    SysView<R> sys{d, M, N, H0, Hk, nullptr, nullptr, u_dev};
    CostView<R> cost{0, fmask_dev ? fmask_dev : fmask_zero, colw, (double)S, psiT, nullptr,
                     {alpha[0], alpha[1], alpha[2], alpha[3], alpha[4]}};
    ChainArgs<R> ch{d, sv, N, N, 0, 1, ckpt, slice, 0, 1, Ubuf, ustride, N, states, nullptr, prm};
    if (!ok(launch_theta(u_dev, M, N, norms, nullptr, 1, dt, 0.25, 1e-15, 0, -1, prm, st))) return QOC_ERR_CUDA;
    const ZStore<R> nostore{nullptr, 0, 0, 0};   // the arena holds no product operands: block recursion
    if (!ok(launch_expm_fwd_fused<R>(prm, sys, 0, N, 1, Ubuf, ustride, N, nostore, st))) return QOC_ERR_CUDA;
    if (!ok(launch_chain<R>(ch, st))) return QOC_ERR_CUDA;
    if (!ok(launch_slice_costs<R>(d, sv, 0, N, N, 1, states, N, cost, Oj, C5j, Ofin, st))) return QOC_ERR_CUDA;
    if (!ok(launch_sources<R>(d, sv, 0, N, N, 1, states, N, cost, Oj, Ofin, src, st))) return QOC_ERR_CUDA;
    CostateArgs<R> co{};
    co.d = d;
    co.sv = sv;
    co.wlen = co.seg = N;
    co.E = 1;
    co.U = Ubuf;
    co.ustride = ustride;
    co.src = src;
    co.G = Gbuf;
    co.cin = co.cout = carry;
    co.prm = prm;
    if (!ok(launch_costate<R>(co, st))) return QOC_ERR_CUDA;
    int n_adj = 0;
    if (!ok(launch_expm_adj_fused<R>(prm, sys, sv, 0, N, 1, states, Gbuf, N, gpart, nostore, st, &n_adj)))
        return QOC_ERR_CUDA;
    if (!ok(launch_finalize(1, M, N, u_dev, alpha, Oj, C5j, Ofin, gpart, grad_dev, out_dev, prm, st)))
        return QOC_ERR_CUDA;
    return QOC_OK;
}
