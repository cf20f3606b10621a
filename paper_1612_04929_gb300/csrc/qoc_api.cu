// C ABI of the quantum-control cost + gradient evaluation (declared in include/qoc.h).
//
// One evaluation runs, on the context stream:
//   k_theta                      FP64 norm bound -> one global (p, n)               (Sec. III)
//   per wave w = 0 .. nw-1 (forward; a wave is a multiple of the checkpoint stride):
//     expm_fwd (all slices of w) U_j = [Taylor_p(-i s H_j)]^(2^n)                 (Eqs. 1, 9, 10)
//     chain_fwd                  Psi_j = U_j Psi_{j-1}; checkpoint every stride     (Eqs. 2, 4)
//     slice_costs                O_j, forbidden occupation per slice                (Table I)
//   per wave w = nw-1 .. 0 (backward):
//     [expm_fwd + chain replay]  recompute U_j, regenerate Psi_j from the checkpoints, one
//                                segment per CTA (skipped for the wave still resident from the
//                                forward sweep)
//     sources                    dC/dPsi_j of every cost term                       (App. A)
//     costate                    G_{j-1} = U_j^dag G_j + src_{j-1}                  (Alg. 1-3)
//     expm_adj                   exact adjoint of the truncated series, dC/du_{k,j}  (Eq. A3)
//   finalize                     FP64 costs, C3/C4 gradients, ensemble sum          (Table I)
// Only the checkpoints (one d x S block per stride c) and one wave (W slices) of propagators,
// states and costates live at a time: device memory is O(N/c d S + W d^2), independent of N
// apart from the checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/qoc.h"
#include "qoc_internal.h"

using namespace qoc;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t alloc(size_t n) {
        release();
        if (n == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = n;
        return cudaSuccess;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct Fail {
    qoc_status st;
};

// CUDA-event brackets around kernel launches, harvested when the stream is synchronised.
struct Profiler {
    struct Pending { int cls; cudaEvent_t a, b; };
    std::vector<std::string> names;
    std::vector<long long> launches;
    std::vector<double> ms;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    int cls(const char* name) {
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == name) return (int)i;
        names.push_back(name);
        launches.push_back(0);
        ms.push_back(0.0);
        return (int)names.size() - 1;
    }
    void harvest() {   // stream already synchronised
        for (auto& p : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
                launches[p.cls] += 1;
                ms[p.cls] += t;
            }
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
    void reset() {
        for (auto& v : launches) v = 0;
        for (auto& v : ms) v = 0.0;
    }
    ~Profiler() {
        for (auto& p : pending) { pool.push_back(p.a); pool.push_back(p.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

}  // namespace

struct qoc_ctx {
    qoc_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t aux = nullptr;          // second stream of the evaluation (serial sweeps)
    std::vector<cudaEvent_t> events;     // dependencies between the two streams
    std::string err;

    // problem (host FP64 copies; the device copies are made by the planner)
    bool has_sys = false, has_tgt = false;
    int d = 0, M = 0, N = 0, S = 0, nF = 0, E = 1;
    double dt = 0.0;
    std::vector<double> H0, Hk, Hdet, delta, psi0, psiT, path, w;
    std::vector<int> forb;
    double alpha[5] = {0, 0, 0, 0, 0};
    double Wsum = 0.0;

    // plan
    bool planned = false;
    bool tuned = false;                  // the autotuner has run (or found a cached choice)
    int tune_candidates = 0;             // configurations it timed
    bool theta_user = false;             // theta_max was set by the caller (not tuned)
    int W = 0, nw = 0, seg = 0, nseg_total = 0, path_kind = 0;
    int Spad = 0, cb = 0, ncb = 0, pstride = 0, S_eff = 0;
    bool scan = false;                   // segmented-scan form of the two recursions
    double theta_max = 0.0;              // in effect (the option, or the path's default)
    bool ps = false;                     // Paterson-Stockmeyer form of the per-slice FP32 exponential
    int nzmax = 0;                       // checkpoint segments per wave
    std::vector<int> cols;               // propagated columns (positive weight)
    size_t mstride = 0;                  // elements per matrix slot of the batched path
    long long ustride = 0;
    int launches = 0;

    Profiler prof;

    DevBuf H64, HR, dDelta, norms, psiTR, pathR, fmask, colw, ckpt, Ubuf, states, Gbuf, src, carry, Oj, C5j, Ofin,
        gpart, prm, u_h, grad_h, out_h, scratch, tc_planes;
    DevBuf sH;                           // s H_0 .. s H_det as FP32 pairs (per-slice split exponential)
    DevBuf chebd;                        // Chebyshev coefficients of the evaluation (state mode)
    DevBuf stscr;                        // state mode: the gradient kernel's per-item scratch
    ChebCoef cheb_host{};                // their host copy (kept alive for the asynchronous copy)
    // segmented scan: segment products (two wave sets), tree levels, scan states, costate carries
    DevBuf Pbuf, lv0, lv1, scanst, hbuf, Ybuf;
    DevBuf Zbuf;                         // product operands for the reverse-mode adjoint (per-slice path)
    size_t zmstride = 0;
    DevBuf Zbig;                         // the same for the batched path, sized at evaluation for p - 1 + n
    bool last_big_rev = false;           // the last batched-path evaluation used the reverse mode
    cudaGraphExec_t gexec = nullptr;     // captured evaluation (qoc_options.graph) and its pointers
    const void* gkey[3] = {nullptr, nullptr, nullptr};
    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        gkey[0] = gkey[1] = gkey[2] = nullptr;
    }
    TcMaps tc_maps{};
    TcMaps tc_fwd_maps{};                // the tensor-core forward products' maps over the same planes
    // orders of a captured batch (qoc_batch_create): the batched path launches for the frozen
    // (p, n) and grid exponents without reading them back, and k_theta checks that they still
    // cover the controls
    int batches = 0;                     // captured batches that hold this context
    bool destroy_pending = false;        // qoc_destroy called while a batch held it
    bool frozen = false;
    DevParams hp_frozen{};
    DevBuf frozen_d;

    size_t device_bytes() const {
        const DevBuf* all[] = {&H64, &HR, &dDelta, &norms, &psiTR, &pathR, &fmask, &colw, &ckpt, &Ubuf, &states,
                               &Gbuf, &src, &carry, &Oj, &C5j, &Ofin, &gpart, &prm, &u_h, &grad_h, &out_h, &scratch,
                               &tc_planes, &Pbuf, &lv0, &lv1, &scanst, &hbuf, &Ybuf, &Zbuf, &Zbig, &sH, &chebd, &stscr,
                               &frozen_d};
        size_t s = 0;
        for (auto* b : all) s += b->bytes;
        return s;
    }
};

namespace {

thread_local std::string g_create_error;

qoc_status set_err(qoc_ctx* c, qoc_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

void check_cuda(qoc_ctx* c, cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        c->err = std::string(what) + ": " + cudaGetErrorString(e);
        throw Fail{e == cudaErrorMemoryAllocation ? QOC_ERR_OOM : QOC_ERR_CUDA};
    }
}

bool all_finite(const double* x, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

// max |H_ab - conj(H_ba)| <= 1e-12 * max(1, max |H|)
bool hermitian(const double* H, int d) {
    double mx = 0.0, dev = 0.0;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            const double* x = H + 2 * ((size_t)a * d + b);
            const double* y = H + 2 * ((size_t)b * d + a);
            mx = std::max(mx, std::hypot(x[0], x[1]));
            dev = std::max(dev, std::hypot(x[0] - y[0], x[1] + y[1]));
        }
    return dev <= 1e-12 * std::max(1.0, mx);
}

bool is_fp64(const qoc_ctx* c) { return c->opt.precision == QOC_PREC_FP64; }

// TF32_SPLIT: the FP32 form with the large-d adjoint products on tcgen05 (TF32 x3 split)
bool use_tc(const qoc_ctx* c) { return c->opt.precision == QOC_PREC_TF32_SPLIT && c->path_kind == 1; }
// BF16_SPLIT: the FP32 form with the large-d adjoint products on tcgen05 with exact accumulation
bool use_oz(const qoc_ctx* c) { return c->opt.precision == QOC_PREC_BF16_SPLIT && c->path_kind == 1; }
// ... and its Paterson-Stockmeyer forward products too, for kOzFwdMinD <= d <= kOzFwdMaxD (below,
// the 128 x 64 tiles are mostly padding and the SIMT split products are faster; above, the exact
// slice levels could overflow their accumulators)
bool oz_fwd_on(const qoc_ctx* c) {
    return use_oz(c) && c->ps && c->d >= kOzFwdMinD && c->d <= kOzFwdMaxD;
}

template <typename R>
bool split_exp(const qoc_ctx* c) {
    return sizeof(R) == 4 && c->opt.plain_fp32_exp == 0;
}

template <typename R>
void plan_impl(qoc_ctx* c) {
    using C = C_t<R>;
    const int d = c->d, N = c->N, E = c->E, M = c->M;
    const size_t cs = sizeof(C);
    const int dmax = split_exp<R>(c) ? std::min(fused_max_d<R>(), split_max_d()) : fused_max_d<R>();
    c->path_kind = (d <= dmax) ? 0 : 1;   // 0: per-slice fused kernels, 1: batched tiled GEMMs
    const bool state_mode = c->opt.propagation == QOC_PROP_STATE;
    if (state_mode) c->path_kind = 2;     // 2: state mode (Taylor on the propagated columns)
    // default theta_max of the FP32 forms: 0.5 with the per-slice kernels (split squarings: one
    // split product fewer than 1.0 on long evolutions); 1.0 on the batched path, whose plain
    // FP32 adjoint loses accuracy with every extra squaring
    // The Paterson-Stockmeyer form costs about p / 3 + 2 products instead of p - 1, so a larger
    // theta_max (fewer squarings, each a split product plus two adjoint products) pays: on the
    // d = 40 workload theta_max = 2 (p = 14, n = 2) against Horner's 0.5 (p = 9, n = 4).
    c->ps = split_exp<R>(c) && c->opt.taylor_scheme == QOC_TAYLOR_AUTO &&
            ((c->path_kind == 0 && d <= ps_max_d()) || (c->path_kind == 1 && !use_tc(c)));
    c->theta_max = c->opt.theta_max > 0.0 ? c->opt.theta_max : (c->ps ? 2.0 : (c->path_kind == 0 ? 0.5 : 1.0));
    // Columns whose weight is zero enter no cost term (every term is weighted by w_s), so they
    // are not propagated at all.
    c->cols.clear();
    for (int s = 0; s < c->S; ++s)
        if (c->w[s] > 0.0) c->cols.push_back(s);
    const int S = (int)c->cols.size();
    c->S_eff = S;
    if (state_mode && S > kStateMaxColumns)
        throw Fail{set_err(c, QOC_ERR_UNSUPPORTED, "state mode propagates at most 8 weighted columns")};
    // checkpoint stride (sqrt N by default) and the form of the recursions
    // Reversal (the paper's Algorithms 1-3): no checkpoint inside a wave; the wave size is chosen
    // freely (stride 1 below), then the stride becomes the wave, so the forward pass hands its
    // carried block from wave to wave and the backward pass regenerates each wave's states from
    // the next wave's first state by Psi_{j-1} = U_j^dag Psi_j.
    const bool rev = c->opt.reversal != 0 || state_mode;
    int seg = rev ? 1 : (c->opt.ckpt_stride > 0 ? c->opt.ckpt_stride : (int)std::ceil(std::sqrt((double)N)));
    seg = std::max(1, std::min(seg, N));
    c->scan = !rev && (c->opt.sweep == QOC_SWEEP_SCAN || (c->opt.sweep == QOC_SWEEP_AUTO && seg >= 4));
    int sms0 = 0;
    cudaDeviceGetAttribute(&sms0, cudaDevAttrMultiProcessorCount, c->opt.device);
    const long want_ctas = 2L * std::max(sms0, 1);
    // column panel width: a sweep CTA owns one panel of one member (and, in the segmented form,
    // one segment); wide panels read each U_j once for more columns, narrow ones spread the work
    // over more SMs: about two sweep CTAs per SM, up to 8 columns per panel.  The segments of a
    // (default, half-evolution) wave count towards the parallelism of the segmented form.
    auto panel_width = [&](long par) {
        return (int)std::min<long>(S, std::max(1L, std::min<long>(8, ((long)S * E * par + want_ctas - 1) / want_ctas)));
    };
    // The FP32 sweeps' 8-column step (two rows per lane group) costs about 0.62 of the narrower
    // panels' one-output step per column (instructions per FMA, 1.14 against 1.83).
    const bool wide8 = sizeof(R) == 4 && S >= 8;
    auto col_cost = [&](int w) { return (wide8 && w == 8) ? 0.62 * w : (double)w; };
    const long par = c->scan ? std::max(1L, ((long)(N + 1) / 2 + seg - 1) / seg) : 1L;
    int cbw = panel_width(par);
    if (wide8 && cbw >= 5) cbw = 8;
    if (c->scan && c->opt.ckpt_stride <= 0 && N >= 16) {
        // Checkpoint stride and panel width of the segmented form from a cost model of one wave's
        // sweeps: three passes of `seg` dependent steps over all segments at once (replay, the
        // costate's two segment passes), each running in whole rounds of resident CTAs, and two
        // scans of `nseg` steps (one CTA per panel); a CTA step costs col_cost(panel width).
        const long wave = ((long)N + 1) / 2;
        double best = -1.0;
        int best_seg = seg;
        const int lo = std::max(4, (int)std::sqrt((double)N) / 2), hi = std::min(N, 2 * (int)std::ceil(std::sqrt((double)N)));
        for (int sg = lo; sg <= hi; ++sg) {
            const long nseg = (wave + sg - 1) / sg;
            for (int w : {panel_width(nseg), wide8 ? 8 : 0}) {
                if (w < 1) continue;
                const long ctas = (long)((S + w - 1) / w) * E * nseg;
                const long rounds = (ctas + want_ctas - 1) / want_ctas;
                const double cost = col_cost(w) * (3.0 * sg * rounds + 2.0 * nseg);
                if (best < 0.0 || cost < best) {
                    best = cost;
                    best_seg = sg;
                    cbw = w;
                }
            }
        }
        seg = best_seg;
    }
    c->cb = std::min(cbw, S);
    c->ncb = (S + c->cb - 1) / c->cb;
    c->Spad = c->ncb * c->cb;
    const int align_elems = (int)(16 / cs) > 0 ? (int)(16 / cs) : 1;
    c->pstride = ((d * c->cb + align_elems - 1) / align_elems) * align_elems;
    const size_t slice = (size_t)c->ncb * c->pstride;
    // one slice of the propagator buffer holds U_j and U_j^dag, each padded to 256 bytes
    const long long ue = 256 / (long long)cs;
    c->ustride = 2 * ((((long long)d * d + ue - 1) / ue) * ue);
    // Wave: the slices whose propagators are held at once (a multiple of the stride).  Two wave
    // sets alternate, and after the forward pass they still hold the last two waves, so with at
    // most two waves nothing is recomputed in the backward pass.  By default the wave is half the
    // evolution when both sets fit a memory budget (1/8 of the free device memory, between 1 and
    // 32 GiB), else the largest wave that fits.
    int W = 0;
    if (c->opt.wave_slices > 0) {
        W = ((c->opt.wave_slices + seg - 1) / seg) * seg;
    } else {
        const size_t dd0 = (size_t)d * d, ks = sizeof(K_t<R>);
        size_t per = 2 * ((size_t)c->ustride * cs + 3 * slice * cs);          // U, states, G, sources
        if (c->path_kind == 1) per += big_scratch_per_item(d, sizeof(R) == 8, c->ps);
        if (use_tc(c)) per += tc_scratch_floats(d, 1) * sizeof(float);
        if (use_oz(c)) per += std::max(oz_scratch_bytes(d, 1), oz_fwd_on(c) ? oz_fwd_scratch_bytes(d, 1) : 0);
        if (c->scan) per += dd0 * ks + (2 * (size_t)c->ustride * ks + seg - 1) / seg;
        if (c->path_kind == 0 && c->opt.gradient == QOC_GRAD_EXACT && c->opt.adjoint == QOC_ADJ_AUTO)
            per += 2 * (size_t)kZCap * ((dd0 + 31) / 32 * 32) * cs;
        per *= (size_t)E;
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = (size_t)8 << 30;
        const size_t budget = std::min<size_t>((size_t)32 << 30, std::max<size_t>((size_t)1 << 30, free_b / 8));
        const long long w_mem = std::max<long long>(seg, (long long)(budget / std::max<size_t>(per, 1)) / seg * seg);
        const long long w_half = (((long long)N + 1) / 2 + seg - 1) / seg * seg;
        W = (int)std::min<long long>(w_half, w_mem);
        if (c->path_kind == 0 && W == w_half && 2 * (long long)seg < N) {
            // Per-slice kernels run in whole rounds of resident CTAs: among the two-wave sizes
            // that fit, take the one with the fewest rounds of the forward exponential (weight 2)
            // and of the adjoint (weight 1) over both waves.
            int sms1 = 0;
            cudaDeviceGetAttribute(&sms1, cudaDevAttrMultiProcessorCount, c->opt.device);
            const long slots_f = (long)std::max(sms1, 1) *
                                 (c->ps ? ps_fwd_ctas_per_sm(d)
                                        : (split_exp<R>(c) ? split_ctas_per_sm(d) : fused_ctas_per_sm<R>(d, false)));
            const long slots_a = (long)std::max(sms1, 1) * (c->ps ? ps_adj_ctas_per_sm(d) : fused_ctas_per_sm<R>(d, true));
            const bool adj = c->opt.gradient == QOC_GRAD_EXACT;
            auto rounds = [](long units, long slots) { return (units + slots - 1) / slots; };
            long best = -1;
            for (long long w = w_half; w < N && w <= w_mem; w += seg) {
                const long len0 = (long)w * E, len1 = (long)(N - w) * E;
                const long cost = 2 * (rounds(len0, slots_f) + rounds(len1, slots_f)) +
                                  (adj ? rounds(len0, slots_a) + rounds(len1, slots_a) : 0);
                if (best < 0 || cost < best) {
                    best = cost;
                    W = (int)w;
                }
            }
        }
    }
    W = std::max(seg, std::min(W, ((N + seg - 1) / seg) * seg));
    if (state_mode && c->opt.wave_slices <= 0) {
        // state mode holds X_j (one d x d matrix of pairs per slice and member) for a wave: the
        // whole evolution when it fits 1/8 of the free memory (1..32 GiB), else the largest wave
        const size_t per = (size_t)E * (2 * (size_t)c->ustride * cs + 3 * slice * cs);
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = (size_t)8 << 30;
        const size_t budget = std::min<size_t>((size_t)32 << 30, std::max<size_t>((size_t)1 << 30, free_b / 8));
        W = (int)std::max<size_t>(1, std::min<size_t>((size_t)N, budget / std::max<size_t>(per, 1)));
    }
    if (rev) seg = W;
    c->seg = seg;
    c->W = W;
    c->nw = (N + W - 1) / W;
    c->nseg_total = (N + seg - 1) / seg;
    c->nzmax = W / seg;
    const int nseg_total = c->nseg_total;

    StateView<R> sv{c->Spad, c->cb, c->ncb, c->pstride, c->S_eff};
    cudaStream_t st = c->stream;
    auto A = [&](DevBuf& b, size_t bytes, const char* what) { check_cuda(c, b.alloc(bytes), what); };

    // system in the compute precision (H0, Hk, Hdet consecutive)
    const size_t dd = (size_t)d * d;
    A(c->HR, (M + 2) * dd * cs, "alloc H");
    check_cuda(c, launch_convert<R>(c->H64.as<double2>(), c->HR.as<C>(), (M + 2) * dd, st), "convert H");
    if (split_exp<R>(c) || (c->path_kind == 2 && sizeof(R) == 4)) A(c->sH, (M + 2) * dd * sizeof(float4), "alloc sH");
    else c->sH.release();
    // costs
    std::vector<int> mask(d, 0);
    for (int f : c->forb) mask[f] = 1;
    A(c->fmask, d * sizeof(int), "alloc mask");
    check_cuda(c, cudaMemcpyAsync(c->fmask.p, mask.data(), d * sizeof(int), cudaMemcpyHostToDevice, st), "copy mask");
    std::vector<double> wpad(c->Spad, 0.0);
    for (int s = 0; s < S; ++s) wpad[s] = c->w[c->cols[s]];
    // d x S blocks restricted to the propagated columns
    auto prune = [&](const std::vector<double>& full, int blocks) {
        std::vector<double> out((size_t)blocks * d * S * 2);
        for (int b = 0; b < blocks; ++b)
            for (int a = 0; a < d; ++a)
                for (int s = 0; s < S; ++s) {
                    const size_t src = (((size_t)b * d + a) * c->S + c->cols[s]) * 2;
                    const size_t dst = (((size_t)b * d + a) * S + s) * 2;
                    out[dst] = full[src];
                    out[dst + 1] = full[src + 1];
                }
        return out;
    };
    const std::vector<double> psi0p = prune(c->psi0, 1), psiTp = prune(c->psiT, 1);
    const std::vector<double> pathp = c->path.empty() ? std::vector<double>() : prune(c->path, N);
    A(c->colw, c->Spad * sizeof(double), "alloc weights");
    check_cuda(c, cudaMemcpyAsync(c->colw.p, wpad.data(), c->Spad * sizeof(double), cudaMemcpyHostToDevice, st),
               "copy weights");
    // targets and the initial block (checkpoint 0 of every member) through an FP64 staging buffer
    DevBuf stage;
    const size_t blk = (size_t)d * S * 2 * sizeof(double);
    A(stage, std::max(blk, c->path.empty() ? blk : (size_t)N * blk), "alloc staging");
    A(c->psiTR, slice * cs, "alloc target");
    check_cuda(c, cudaMemcpyAsync(stage.p, psiTp.data(), blk, cudaMemcpyHostToDevice, st), "copy target");
    check_cuda(c, launch_to_panels<R>(stage.as<double2>(), c->psiTR.as<C>(), d, S, sv, 1, 0, 0, st), "target panels");
    A(c->ckpt, (size_t)E * nseg_total * slice * sizeof(K_t<R>), "alloc checkpoints");
    check_cuda(c, cudaStreamSynchronize(st), "sync");
    check_cuda(c, cudaMemcpyAsync(stage.p, psi0p.data(), blk, cudaMemcpyHostToDevice, st), "copy psi0");
    check_cuda(c, launch_to_carry<R>(stage.as<double2>(), c->ckpt.as<K_t<R>>(), d, S, sv, E,
                                     (size_t)nseg_total * slice, st),
               "psi0 panels");
    if (!c->path.empty()) {
        check_cuda(c, cudaStreamSynchronize(st), "sync");
        A(c->pathR, (size_t)N * slice * cs, "alloc path");
        check_cuda(c, cudaMemcpyAsync(stage.p, pathp.data(), (size_t)N * blk, cudaMemcpyHostToDevice, st),
                   "copy path");
        check_cuda(c, launch_to_panels<R>(stage.as<double2>(), c->pathR.as<C>(), d, S, sv, N, slice, (size_t)d * S, st),
                   "path panels");
    } else {
        c->pathR.release();
    }
    // per-segment work buffers
    // two sets of wave buffers (waves alternate between them)
    A(c->Ubuf, 2 * (size_t)E * W * c->ustride * cs, "alloc U");
    A(c->states, 2 * (size_t)E * (W + 1) * slice * cs, "alloc states");
    A(c->Gbuf, 2 * (size_t)E * W * slice * cs, "alloc costates");
    A(c->src, 2 * (size_t)E * W * slice * cs, "alloc sources");
    if (c->path_kind == 1) {
        c->mstride = (((size_t)d * d + 15) / 16) * 16;
        const size_t per = big_scratch_per_item(d, sizeof(R) == 8, c->ps) / ((size_t)d * d) * c->mstride;
        A(c->scratch, per * (size_t)E * W, "alloc batched scratch");
    } else {
        c->scratch.release();
    }
    if (use_oz(c)) {
        // the tensor maps cover exactly d x d of every plane (reads past d fill zeros), so the
        // padding columns of the planes are never read and need no clearing
        // the forward's and the adjoint's products run on one stream and share the plane array
        A(c->tc_planes, std::max(oz_scratch_bytes(d, E * W), oz_fwd_on(c) ? oz_fwd_scratch_bytes(d, E * W) : 0),
          "alloc tensor-core slices");
        check_cuda(c, oz_make_maps(c->tc_planes.p, d, E * W, &c->tc_maps), "tensor maps");
        if (oz_fwd_on(c)) check_cuda(c, oz_fwd_make_maps(c->tc_planes.p, d, E * W, &c->tc_fwd_maps), "tensor maps");
    } else if (use_tc(c)) {
        A(c->tc_planes, tc_scratch_floats(d, E * W) * sizeof(float), "alloc tensor-core planes");
        check_cuda(c, cudaMemsetAsync(c->tc_planes.p, 0, c->tc_planes.bytes, st), "clear planes");
        check_cuda(c, tc_make_maps(c->tc_planes.as<float>(), d, E * W, &c->tc_maps), "tensor maps");
    } else {
        c->tc_planes.release();
    }
    if (c->path_kind == 0 && c->opt.gradient == QOC_GRAD_EXACT && c->opt.adjoint == QOC_ADJ_AUTO) {
        c->zmstride = (dd + 31) / 32 * 32;
        A(c->Zbuf, 2 * (size_t)E * W * kZCap * c->zmstride * cs, "alloc product operands");
    } else {
        c->Zbuf.release();
    }
    if (c->scan) {
        const size_t nz = (size_t)c->nzmax, ks = sizeof(K_t<R>);
        const size_t half = (size_t)((seg + 1) / 2);
        A(c->Pbuf, 2 * (size_t)E * nz * c->ustride * ks, "alloc segment products");
        A(c->lv0, (size_t)E * nz * half * dd * ks, "alloc tree level");
        A(c->lv1, (size_t)E * nz * half * dd * ks, "alloc tree level");
        A(c->scanst, (size_t)E * (nz + 1) * slice * cs, "alloc scan states");
        A(c->hbuf, (size_t)E * (nz + 1) * slice * ks, "alloc segment costates");
        A(c->Ybuf, 2 * (size_t)E * nz * slice * ks, "alloc segment carries");
    } else {
        for (DevBuf* b : {&c->Pbuf, &c->lv0, &c->lv1, &c->scanst, &c->hbuf, &c->Ybuf}) b->release();
    }
    // second stream and the dependency events between the two streams
    if (!c->aux) {   // the serial sweeps' stream takes the highest priority: its few dependent CTAs are
                     // the critical path, and the parallel kernels on the other stream fill the rest
        int least = 0, greatest = 0;
        check_cuda(c, cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
        check_cuda(c, cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, greatest), "create stream");
    }
    for (auto e : c->events) cudaEventDestroy(e);
    c->events.assign(4 * c->nw + 3, nullptr);
    for (auto& e : c->events) check_cuda(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "create event");
    A(c->carry, (size_t)E * slice * sizeof(K_t<R>), "alloc carry");
    A(c->Oj, (size_t)E * N * sizeof(double2), "alloc O");
    A(c->C5j, (size_t)E * N * sizeof(double), "alloc C5");
    A(c->Ofin, (size_t)E * sizeof(double2), "alloc Ofin");
    A(c->gpart, (size_t)E * M * N * sizeof(double) + 8, "alloc gpart");
    A(c->prm, sizeof(DevParams), "alloc params");
    check_cuda(c, cudaMemsetAsync(c->prm.p, 0, sizeof(DevParams), st), "memset params");
    // the host API's staging buffers survive a re-plan of the same shape (the autotuner re-plans
    // while the caller's controls already sit in u_h)
    auto keep = [&](DevBuf& b, size_t bytes, const char* what) {
        if (!(b.p && b.bytes == bytes)) A(b, bytes, what);
    };
    keep(c->u_h, (size_t)M * N * sizeof(double) + 8, "alloc u");
    keep(c->grad_h, (size_t)M * N * sizeof(double) + 8, "alloc grad");
    keep(c->out_h, 8 * sizeof(double), "alloc out");
    check_cuda(c, cudaStreamSynchronize(st), "plan sync");
    c->planned = true;
}

// known: (p, n) already picked on the device by an earlier launch_theta on c->stream and read
// back (batched evaluation); nullptr: pick them here.
template <typename R>
void evaluate_impl(qoc_ctx* c, const double* u, double* grad, double* out, const DevParams* known = nullptr) {
    using C = C_t<R>;
    using K = K_t<R>;
    const int d = c->d, N = c->N, E = c->E, M = c->M, W = c->W, nw = c->nw;
    cudaStream_t st = c->stream;   // parallel kernels (the caller's stream)
    cudaStream_t sx = c->aux;      // serial sweeps and the small per-slice kernels
    StateView<R> sv{c->Spad, c->cb, c->ncb, c->pstride, c->S_eff};
    const size_t slice = sv.slice();
    const size_t dd = (size_t)d * d;
    C* HR = c->HR.as<C>();
    SysView<R> sys{d, M, N, HR, HR + dd, c->Hdet.empty() ? nullptr : HR + (size_t)(M + 1) * dd,
                   c->delta.empty() ? nullptr : c->dDelta.as<double>(), u};
    CostView<R> cv{c->nF, c->fmask.as<int>(), c->colw.as<double>(), c->Wsum, c->psiTR.as<C>(),
                   c->path.empty() ? nullptr : c->pathR.as<C>(), {c->alpha[0], c->alpha[1], c->alpha[2], c->alpha[3], c->alpha[4]}};
    DevParams* prm = c->prm.as<DevParams>();
    const int seg = c->seg;
    // two sets of wave buffers: wave w uses set w % 2, so the serial sweep of one wave overlaps
    // the parallel kernels of its neighbour
    const size_t u_set = (size_t)E * W * c->ustride, s_set = (size_t)E * (W + 1) * slice, g_set = (size_t)E * W * slice;
    auto Ub = [&](int w) { return c->Ubuf.as<C>() + (w & 1) * u_set; };
    auto Sb = [&](int w) { return c->states.as<C>() + (w & 1) * s_set; };
    auto Gb = [&](int w) { return c->Gbuf.as<C>() + (w & 1) * g_set; };
    auto Rb = [&](int w) { return c->src.as<C>() + (w & 1) * g_set; };
    auto chain_args = [&](int w, int mode) {
        const int j0 = w * W;
        return ChainArgs<R>{d, sv, std::min(W, N - j0), seg, mode, E, c->ckpt.as<K>(), (size_t)c->nseg_total * slice,
                            j0 / seg, c->nseg_total, Ub(w), c->ustride, W, Sb(w), nullptr, prm};
    };
    int launches = 0;
    const bool prof = c->opt.profile != 0;
    cudaEvent_t ev0 = nullptr;
    // B(stream) opens an event bracket before a launch, L(..., stream) closes it after the launch
    auto B = [&](cudaStream_t s) {
        if (prof) {
            ev0 = c->prof.get();
            cudaEventRecord(ev0, s);
        }
    };
    auto L = [&](cudaError_t e, const char* what, cudaStream_t s) {
        ++launches;
        check_cuda(c, e, what);
        if (prof) {
            cudaEvent_t ev1 = c->prof.get();
            cudaEventRecord(ev1, s);
            c->prof.pending.push_back({c->prof.cls(what), ev0, ev1});
        }
    };
    auto rec = [&](cudaEvent_t e, cudaStream_t s) { check_cuda(c, cudaEventRecord(e, s), "event record"); };
    auto wait = [&](cudaStream_t s, cudaEvent_t e) { check_cuda(c, cudaStreamWaitEvent(s, e, 0), "event wait"); };
    cudaEvent_t* ev_exp = &c->events[0];
    cudaEvent_t* ev_fwd = &c->events[nw];
    cudaEvent_t* ev_rep = &c->events[2 * nw];
    cudaEvent_t* ev_cost = &c->events[3 * nw];
    cudaEvent_t ev_fork = c->events[4 * nw], ev_fwd_done = c->events[4 * nw + 1], ev_join = c->events[4 * nw + 2];

    if (!known) {
        B(st);
        L(launch_theta(u, M, N, c->norms.as<double>(), c->delta.empty() ? nullptr : c->dDelta.as<double>(), E, c->dt,
                       c->theta_max, c->opt.tol, c->opt.p_override, c->opt.n_override, prm, st,
                       c->frozen ? c->frozen_d.as<DevParams>() : nullptr),
          "theta", st);
    } else {
        ++launches;
    }
    if constexpr (sizeof(R) == 4) {
        if (split_exp<R>(c)) {   // s H_k pairs for this evaluation's (p, n)
            B(st);
            L(launch_split_scale(prm, c->H64.as<double2>(), (M + 2) * dd, c->sH.as<float4>(), st), "theta", st);
        }
    }
    rec(ev_fork, st);
    wait(sx, ev_fork);
    // slice exponentials: split hi+lo FP32 for the FP32 form (unless disabled), else plain
    const bool split = split_exp<R>(c);
    const bool big = c->path_kind == 1;
    DevParams hp{};
    if (big) {   // the batched path launches one kernel per product: read (p, n) back once
        if (known) {
            hp = *known;
        } else if (c->frozen) {   // a captured batch's orders: no read-back (capture-safe)
            hp = c->hp_frozen;
        } else {
            check_cuda(c, cudaMemcpyAsync(&hp, prm, sizeof(DevParams), cudaMemcpyDeviceToHost, st), "read (p, n)");
            check_cuda(c, cudaStreamSynchronize(st), "sync (p, n)");
        }
        hp.p = std::max(1, std::min(hp.p, kPMax));
        hp.n = std::max(0, std::min(hp.n, 1000));
    }
    BigSys bsys{d, M, N, c->H64.as<double2>(), u, c->delta.empty() ? nullptr : c->dDelta.as<double>(),
                c->Hdet.empty() ? 0 : 1};
    // batched path: reverse-mode adjoint over stored product operands when the store fits (1/4 of
    // the free device memory); else the block recursion, which stores nothing
    bool big_rev = false;
    size_t zbig_set = 0;
    if (big && c->opt.gradient == QOC_GRAD_EXACT && c->opt.adjoint == QOC_ADJ_AUTO && !use_tc(c)) {
        zbig_set = (size_t)E * W * (size_t)(c->ps ? ps_big_slots(hp.p, hp.n) : hp.p - 1 + hp.n) * c->mstride;
        const size_t need = 2 * zbig_set * sizeof(C);
        if (c->Zbig.bytes >= need) {
            big_rev = true;
        } else if (!c->frozen) {   // frozen orders: the store of the first evaluation, no allocation
            c->Zbig.release();
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && need <= free_b / 4 &&
                c->Zbig.alloc(need) == cudaSuccess)
                big_rev = true;
            else
                cudaGetLastError();   // a failed allocation only means: block recursion
        }
    }
    if (big) c->last_big_rev = big_rev;
    auto zbig = [&](int w) { return big_rev ? c->Zbig.as<C>() + (size_t)(w & 1) * zbig_set : nullptr; };
    auto big_args = [&](int w) {
        const int j0 = w * W;
        return BigArgs<R>{prm,      bsys,          d,     E,          j0, std::min(W, N - j0), W, c->scratch.p,
                          c->mstride, Ub(w), c->ustride, c->sH.p ? c->sH.as<float4>() : nullptr, c->ps ? 1 : 0};
    };
    int extra = 0;   // kernels of the batched calls beyond the one counted by L
    // stored product operands of the per-slice path (two wave sets)
    auto zstore = [&](int w) {
        ZStore<R> z{nullptr, kZCap, c->zmstride, W, c->ps ? 1 : 0};
        if (c->Zbuf.p) z.Z = c->Zbuf.as<C>() + (size_t)(w & 1) * E * W * kZCap * c->zmstride;
        return z;
    };
    auto expm_fwd = [&](int w) -> cudaError_t {
        const int j0 = w * W, wlen = std::min(W, N - j0);
        if (big) {
            int n_l = 0;
            OzFwd ozf{c->opt.fault_inject, prm, d, E * wlen, E * W, c->tc_planes.as<unsigned char>(), c->tc_fwd_maps};
            cudaError_t e = launch_big_expm<R>(big_args(w), hp, split, st, &n_l, zbig(w), oz_fwd_on(c) ? &ozf : nullptr);
            extra += n_l - 1;
            return e;
        }
        if constexpr (sizeof(R) == 4) {
            if (c->ps)
                return launch_expm_fwd_ps(prm, sys, c->sH.as<float4>(), j0, wlen, E, Ub(w), c->ustride, W, zstore(w),
                                          st);
            if (split)
                return launch_expm_fwd_split(prm, sys, c->sH.as<float4>(), j0, wlen, E, Ub(w), c->ustride, W,
                                             zstore(w), st);
        }
        return launch_expm_fwd_fused<R>(prm, sys, j0, wlen, E, Ub(w), c->ustride, W, zstore(w), st);
    };
    auto expm_adj = [&](int w) -> cudaError_t {
        const int j0 = w * W, wlen = std::min(W, N - j0);
        if (c->opt.gradient == QOC_GRAD_FIRST_ORDER)
            return launch_grad_first_order<R>(sys, sv, j0, wlen, E, Sb(w), Gb(w), W, c->dt, c->gpart.as<double>(), st);
        if constexpr (sizeof(R) == 4) {
            if (big && big_rev && c->ps) {       // Paterson-Stockmeyer reverse mode (tensor cores: BF16_SPLIT)
                int n_l = 0;
                OzRev oz{c->opt.fault_inject, prm, d, E * wlen, E * W, c->tc_planes.as<unsigned char>(), c->tc_maps,
                         nullptr, nullptr};
                cudaError_t e = launch_big_adj_rev_ps<R>(big_args(w), sys, sv, Sb(w), Gb(w), c->gpart.as<double>(), hp,
                                                         zbig(w), st, &n_l, use_oz(c) ? &oz : nullptr);
                extra += n_l - 1;
                return e;
            }
            if (big && use_oz(c) && big_rev) {   // reverse mode, products on the tensor cores
                int n_l = 0;
                OzRev oz{c->opt.fault_inject, prm, d, E * wlen, E * W, c->tc_planes.as<unsigned char>(), c->tc_maps,
                         nullptr, nullptr};
                cudaError_t e = launch_big_adj_rev<R>(big_args(w), sys, sv, Sb(w), Gb(w), c->gpart.as<double>(), hp.p,
                                                      hp.n, zbig(w), st, &n_l, &oz);
                extra += n_l - 1;
                return e;
            }
            if (big && use_tc(c)) {
                int n_l = 0;
                TcAdjArgs ta{c->opt.fault_inject, prm, sys, sv, d, E, j0, wlen, W, hp.p, hp.n, Sb(w), Gb(w),
                             c->tc_planes.as<float>(),
                             c->tc_maps, c->gpart.as<double>()};
                cudaError_t e = launch_tc_adj(ta, st, &n_l);
                extra += n_l - 1;
                return e;
            }
        }
        if (big) {
            int n_l = 0;
            cudaError_t e = big_rev ? launch_big_adj_rev<R>(big_args(w), sys, sv, Sb(w), Gb(w), c->gpart.as<double>(),
                                                            hp.p, hp.n, zbig(w), st, &n_l)
                                    : launch_big_adj<R>(big_args(w), sys, sv, Sb(w), Gb(w), c->gpart.as<double>(), hp.p,
                                                        hp.n, st, &n_l);
            extra += n_l - 1;
            return e;
        }
        int n_l = 0;
        cudaError_t e = launch_expm_adj_fused<R>(prm, sys, sv, j0, wlen, E, Sb(w), Gb(w), W, c->gpart.as<double>(),
                                                 zstore(w), st, &n_l);
        extra += n_l - 1;
        return e;
    };
    const int nzmax = c->nzmax;
    const size_t p_set = (size_t)E * nzmax * c->ustride;
    auto Pb = [&](int w) { return c->Pbuf.as<K>() + (w & 1) * p_set; };
    auto Yb = [&](int w) { return c->Ybuf.as<K>() + (w & 1) * (size_t)E * nzmax * slice; };
    auto seg_products = [&](int w, cudaStream_t s) -> cudaError_t {
        const int j0 = w * W;
        SegProdArgs<R> a{d, E, std::min(W, N - j0), seg, nzmax, Ub(w), c->ustride, W,
                         c->lv0.as<K>(), c->lv1.as<K>(), dd, Pb(w), prm};
        int n_l = 0;
        cudaError_t e = launch_seg_products<R>(a, s, &n_l);
        extra += n_l - 1;
        return e;
    };
    auto costate_args = [&](int w) {
        const int j0 = w * W;
        CostateArgs<R> a{};
        a.d = d;
        a.sv = sv;
        a.wlen = std::min(W, N - j0);
        a.seg = seg;
        a.E = E;
        a.U = Ub(w);
        a.ustride = c->ustride;
        a.u_es = (size_t)W * c->ustride;
        a.src = Rb(w);
        a.src_es = (size_t)W * slice;
        a.g_es = (size_t)W * slice;
        a.prm = prm;
        return a;
    };
    if (!c->scan) {
        // ---- forward: exponentials on st, propagation and per-slice costs on sx ----
        for (int w = 0; w < nw; ++w) {
            const int j0 = w * W, wlen = std::min(W, N - j0);
            if (w >= 2) wait(st, ev_fwd[w - 2]);           // set w % 2 released by wave w - 2
            B(st);
            L(expm_fwd(w), "expm_fwd", st);
            rec(ev_exp[w], st);
            wait(sx, ev_exp[w]);
            B(sx);
            L(launch_chain<R>(chain_args(w, 0), sx), "chain_fwd", sx);
            B(sx);
            L(launch_slice_costs<R>(d, sv, j0, wlen, N, E, Sb(w), W, cv, c->Oj.as<double2>(), c->C5j.as<double>(),
                                    c->Ofin.as<double2>(), sx),
              "slice_costs", sx);
            rec(ev_fwd[w], sx);
        }
        check_cuda(c, cudaMemsetAsync(c->carry.p, 0, c->carry.bytes, sx), "memset carry");
        rec(ev_fwd_done, sx);
        wait(st, ev_fwd_done);
        // ---- backward: recompute + replay of wave w - 1 on st overlap the costate of wave w on sx ----
        for (int w = nw - 1; w >= 0; --w) {
            const int j0 = w * W, wlen = std::min(W, N - j0);
            if (w != nw - 1) wait(sx, ev_rep[w]);           // the last wave is resident from the forward sweep
            B(sx);
            L(launch_sources<R>(d, sv, j0, wlen, N, E, Sb(w), W, cv, c->Oj.as<double2>(), c->Ofin.as<double2>(), Rb(w),
                                sx),
              "sources", sx);
            B(sx);
            CostateArgs<R> ca = costate_args(w);
            ca.seg = ca.wlen;                                // the whole wave as one segment
            ca.G = Gb(w);
            ca.cin = c->carry.as<K>();
            ca.cin_es = slice;
            ca.cout = c->carry.as<K>();
            ca.cout_es = slice;
            L(launch_costate<R>(ca, sx), "costate", sx);
            rec(ev_cost[w], sx);
            if (w >= 1) {                                    // set (w - 1) % 2 was released by wave w + 1
                if (w - 1 != nw - 2) {                       // wave nw - 2 is still resident
                    B(st);
                    L(expm_fwd(w - 1), "expm_fwd (recompute)", st);
                    if (c->opt.reversal) {                   // backwards from wave w's first state
                        ChainArgs<R> ra = chain_args(w - 1, 2);
                        ra.rev_src = Sb(w);
                        ra.rev_estride = (size_t)(W + 1) * slice;
                        B(st);
                        L(launch_chain<R>(ra, st), "chain (reversal)", st);
                    } else {
                        B(st);
                        L(launch_chain<R>(chain_args(w - 1, 1), st), "chain (replay)", st);
                    }
                }
                rec(ev_rep[w - 1], st);
            }
            wait(st, ev_cost[w]);
            B(st);
            L(expm_adj(w), "expm_adj", st);
        }
    } else {
        // ---- forward: exponentials on st; the segment products and the scan over segments
        //      (checkpoints) on sx, overlapping the next wave's exponentials; replay of every
        //      segment and the per-slice costs on st.  The tree buffers are used on sx only
        //      until the last scan, which st waits for before any backward recomputation. ----
        cudaEvent_t* ev_scan = ev_fwd;
        auto replay_costs = [&](int w) {
            const int j0 = w * W, wlen = std::min(W, N - j0);
            wait(st, ev_scan[w]);
            B(st);
            L(launch_chain<R>(chain_args(w, 1), st), "chain (replay)", st);
            B(st);
            L(launch_slice_costs<R>(d, sv, j0, wlen, N, E, Sb(w), W, cv, c->Oj.as<double2>(), c->C5j.as<double>(),
                                    c->Ofin.as<double2>(), st),
              "slice_costs", st);
        };
        for (int w = 0; w < nw; ++w) {
            const int j0 = w * W, wlen = std::min(W, N - j0);
            const int nz = (wlen + seg - 1) / seg;
            B(st);
            L(expm_fwd(w), "expm_fwd", st);
            rec(ev_exp[w], st);
            wait(sx, ev_exp[w]);
            B(sx);
            L(seg_products(w, sx), "seg_products", sx);
            B(sx);
            L(launch_chain<R>(ChainArgs<R>{d, sv, nz, 1, 0, E, c->ckpt.as<K>(), (size_t)c->nseg_total * slice, j0 / seg,
                                           c->nseg_total, nullptr, c->ustride, nzmax, c->scanst.as<C>(), Pb(w), prm},
                              sx),
              "scan", sx);
            rec(ev_scan[w], sx);
            if (w >= 1) replay_costs(w - 1);
        }
        replay_costs(nw - 1);
        rec(ev_fwd_done, st);
        wait(sx, ev_fwd_done);
        // ---- backward: per wave, the costate of every segment from a zero in-carry, the scan
        //      Y_{z-1} = P_z^dag Y_z + h_z over segments, then every segment from its carry (sx);
        //      recompute + replay of wave w - 1 and the adjoint of wave w on st ----
        for (int w = nw - 1; w >= 0; --w) {
            const int j0 = w * W, wlen = std::min(W, N - j0);
            const int nz = (wlen + seg - 1) / seg;
            if (w != nw - 1) wait(sx, ev_rep[w]);
            B(sx);
            L(launch_sources<R>(d, sv, j0, wlen, N, E, Sb(w), W, cv, c->Oj.as<double2>(), c->Ofin.as<double2>(), Rb(w),
                                sx),
              "sources", sx);
            CostateArgs<R> loc = costate_args(w);
            loc.cout = c->hbuf.as<K>();
            loc.cout_es = (size_t)(nzmax + 1) * slice;
            loc.zero_next = 1;
            B(sx);
            L(launch_costate<R>(loc, sx), "costate (segments)", sx);
            CostateArgs<R> sc{};
            sc.prm = prm;
            sc.d = d;
            sc.sv = sv;
            sc.wlen = nz;
            sc.seg = nz;
            sc.E = E;
            sc.Uk = Pb(w);
            sc.ustride = c->ustride;
            sc.u_es = (size_t)nzmax * c->ustride;
            sc.srck = c->hbuf.as<K>() + slice;   // h_{z} is the source added after step z (slot nz is zero)
            sc.src_es = (size_t)(nzmax + 1) * slice;
            sc.Gk = Yb(w);
            sc.g_es = (size_t)nzmax * slice;
            sc.cin = (w == nw - 1) ? nullptr : Yb(w + 1);
            sc.cin_es = (size_t)nzmax * slice;
            B(sx);
            L(launch_costate<R>(sc, sx), "costate (scan)", sx);
            CostateArgs<R> fin = costate_args(w);
            fin.G = Gb(w);
            fin.cin = Yb(w);
            fin.cin_es = (size_t)nzmax * slice;
            fin.cout = Yb(w);   // out of segment z replaces its own in-carry; slot 0 feeds wave w - 1
            fin.cout_es = (size_t)nzmax * slice;
            B(sx);
            L(launch_costate<R>(fin, sx), "costate (final)", sx);
            rec(ev_cost[w], sx);
            if (w >= 1) {
                if (w - 1 != nw - 2) {   // the last two waves are still resident from the forward pass
                    B(st);
                    L(expm_fwd(w - 1), "expm_fwd (recompute)", st);
                    B(st);
                    L(seg_products(w - 1, st), "seg_products", st);
                    B(st);
                    L(launch_chain<R>(chain_args(w - 1, 1), st), "chain (replay)", st);
                }
                rec(ev_rep[w - 1], st);
            }
            wait(st, ev_cost[w]);
            B(st);
            L(expm_adj(w), "expm_adj", st);
        }
    }
    rec(ev_join, sx);
    wait(st, ev_join);
    B(st);
    L(launch_finalize(E, M, N, u, c->alpha, c->Oj.as<double2>(), c->C5j.as<double>(), c->Ofin.as<double2>(),
                      c->gpart.as<double>(), grad, out, prm, st),
      "finalize", st);
    c->launches = launches + extra;
}

void plan(qoc_ctx* c) {
    c->drop_graph();   // a captured evaluation refers to the buffers of the previous plan
    if (is_fp64(c)) plan_impl<double>(c);
    else plan_impl<float>(c);
}

// Chebyshev expansion of exp(-i theta x) on [-1, 1] (the Jacobi-Anger expansion): coefficients
// a_0 = J_0(theta), a_k = 2 J_k(theta) of (-i)^k T_k(x), the degree K the least with the tail
// bound 2 sum_{k > K} |J_k(theta)| <= 2 (theta/2)^(K+1) / (K+1)! / (1 - theta / (2 (K+2))) <= tol
// (|J_k(t)| <= (t/2)^k / k!).  The Bessel values by the downward (Miller) recurrence
// J_{k-1} = (2k / theta) J_k - J_{k+1} from a start far above K, normalised by
// J_0 + 2 sum_{k >= 1} J_{2k} = 1.  Returns false when K would exceed kChebMax.
bool chebyshev_coefficients(double theta, double tol, ChebCoef& cc) {
    cc = ChebCoef{};
    if (!(theta > 1e-300)) {                 // zero Hamiltonian: exp = I
        cc.K = 0;
        cc.a[0] = 1.0;
        cc.inv_theta = 0.0;
        return true;
    }
    int K = 1;
    for (;;) {
        const double h = 0.5 * theta;
        double t = 2.0;
        for (int k = 1; k <= K + 1; ++k) t *= h / k;       // 2 (theta/2)^(K+1) / (K+1)!
        if (h < K + 2 && t / (1.0 - h / (K + 2)) <= tol) break;
        if (++K > kChebMax) return false;
    }
    const int m = K + 40 + 2 * (int)theta;
    std::vector<double> J(m + 2, 0.0);
    J[m + 1] = 0.0;
    J[m] = 1e-30;
    for (int k = m; k >= 1; --k) {
        J[k - 1] = (2.0 * k / theta) * J[k] - J[k + 1];
        if (std::fabs(J[k - 1]) > 1e250)
            for (int q = k - 1; q <= m; ++q) J[q] *= 1e-250;
    }
    double norm = J[0];
    for (int k = 2; k <= m; k += 2) norm += 2.0 * J[k];
    cc.K = K;
    cc.inv_theta = 1.0 / theta;
    cc.a[0] = J[0] / norm;
    for (int k = 1; k <= K; ++k) cc.a[k] = 2.0 * J[k] / norm;
    return true;
}

// State mode (the paper's Eq. 12): per wave, X_j for the wave's slices, the forward recursion of
// the propagated columns by Horner matrix-vector products, the per-slice costs; backwards, per
// wave, X_j and the states again (from the wave's checkpoint) unless resident, the sources, the
// costate recursion (the adjoint of the same map), and the exact gradient of every slice's map
// in parallel.  One stream; (p, n) is read back once to size the gradient kernel.
template <typename R>
void evaluate_state_impl(qoc_ctx* c, const double* u, double* grad, double* out) {
    using C = C_t<R>;
    using K = K_t<R>;
    const int d = c->d, N = c->N, E = c->E, M = c->M, W = c->W, nw = c->nw;
    cudaStream_t st = c->stream;
    StateView<R> sv{c->Spad, c->cb, c->ncb, c->pstride, c->S_eff};
    const size_t slice = sv.slice(), dd = (size_t)d * d;
    C* HR = c->HR.as<C>();
    SysView<R> sys{d, M, N, HR, HR + dd, c->Hdet.empty() ? nullptr : HR + (size_t)(M + 1) * dd,
                   c->delta.empty() ? nullptr : c->dDelta.as<double>(), u};
    CostView<R> cv{c->nF, c->fmask.as<int>(), c->colw.as<double>(), c->Wsum, c->psiTR.as<C>(),
                   c->path.empty() ? nullptr : c->pathR.as<C>(), {c->alpha[0], c->alpha[1], c->alpha[2], c->alpha[3], c->alpha[4]}};
    DevParams* prm = c->prm.as<DevParams>();
    int launches = 0;
    const bool prof = c->opt.profile != 0;
    cudaEvent_t ev0 = nullptr;
    auto B = [&]() {
        if (prof) {
            ev0 = c->prof.get();
            cudaEventRecord(ev0, st);
        }
    };
    auto L = [&](cudaError_t e, const char* what) {
        ++launches;
        check_cuda(c, e, what);
        if (prof) {
            cudaEvent_t ev1 = c->prof.get();
            cudaEventRecord(ev1, st);
            c->prof.pending.push_back({c->prof.cls(what), ev0, ev1});
        }
    };
    const double* delta = c->delta.empty() ? nullptr : c->dDelta.as<double>();
    const bool cheb = c->opt.exponential == QOC_EXP_CHEBYSHEV;
    B();
    // Chebyshev: n = 0 (s = dt) and no Taylor order (p forced to 1 so that no range error is flagged);
    // the degree comes from theta below
    L(launch_theta(u, M, N, c->norms.as<double>(), delta, E, c->dt, c->theta_max, c->opt.tol,
                   cheb ? 1 : c->opt.p_override, cheb ? 0 : c->opt.n_override, prm, st),
      "theta");
    const void* Hsrc = c->H64.p;
    if constexpr (sizeof(R) == 4) {
        B();
        L(launch_split_scale(prm, c->H64.as<double2>(), (M + 2) * dd, c->sH.as<float4>(), st), "theta");
        Hsrc = c->sH.p;
    }
    DevParams hp{};
    check_cuda(c, cudaMemcpyAsync(&hp, prm, sizeof(DevParams), cudaMemcpyDeviceToHost, st), "read (p, n)");
    check_cuda(c, cudaStreamSynchronize(st), "sync (p, n)");
    const int p = std::max(1, std::min(hp.p, kPMax)), n = std::max(0, std::min(hp.n, 30));
    const ChebCoef* chebd = nullptr;
    if (cheb) {   // dt * spectral radius <= theta (the FP64 1-norm bound of k_theta, n = 0)
        if (!chebyshev_coefficients(hp.theta, c->opt.tol, c->cheb_host))
            throw Fail{set_err(c, QOC_ERR_RANGE, "Chebyshev degree above its maximum for theta = " + std::to_string(hp.theta))};
        if (!c->chebd.p) check_cuda(c, c->chebd.alloc(sizeof(ChebCoef)), "alloc Chebyshev coefficients");
        check_cuda(c, cudaMemcpyAsync(c->chebd.p, &c->cheb_host, sizeof(ChebCoef), cudaMemcpyHostToDevice, st),
                   "copy Chebyshev coefficients");
        chebd = c->chebd.as<ChebCoef>();
    }
    if (state_grad_smem<R>(d, c->S_eff, p, n, cheb ? c->cheb_host.K : 0) > kMaxDynSmem)
        throw Fail{set_err(c, QOC_ERR_UNSUPPORTED, "state mode: d x d and five d x S blocks exceed a CTA's shared memory")};
    if (c->opt.gradient == QOC_GRAD_EXACT && n > 16)
        throw Fail{set_err(c, QOC_ERR_UNSUPPORTED, "state mode: more than 2^16 applications per slice")};
    // the gradient kernel's per-item scratch: application inputs and intermediates (or terms)
    const size_t scr_stride = state_grad_scratch(d, c->S_eff, p, n, cheb ? c->cheb_host.K : 0);
    const size_t scr_bytes = scr_stride * (size_t)E * W * sizeof(C);
    if (c->opt.gradient == QOC_GRAD_EXACT && c->stscr.bytes < scr_bytes) {
        c->stscr.release();
        check_cuda(c, c->stscr.alloc(scr_bytes), "alloc state-mode scratch");
    }
    const size_t xs = (size_t)c->ustride * sizeof(C) / (sizeof(R) == 4 ? sizeof(float4) : sizeof(double2));
    void* X = c->Ubuf.p;
    C* states = c->states.as<C>();
    C* G = c->Gbuf.as<C>();
    C* src = c->src.as<C>();
    K* ck = c->ckpt.as<K>();
    const size_t ck_es = (size_t)c->nseg_total * slice;
    const int has_det = c->Hdet.empty() ? 0 : 1;
    auto xw = [&](int w) {
        const int j0 = w * W, wlen = std::min(W, N - j0);
        B();
        L(launch_state_x<R>(prm, d, M, N, u, delta, has_det, Hsrc, j0, wlen, E, X, xs, st), "state_x");
    };
    auto fwd = [&](int w, bool store_next) {
        const int j0 = w * W, wlen = std::min(W, N - j0);
        StateChainArgs<R> a{d, E, wlen, 0, sv, X, xs, ck + (size_t)w * slice, ck_es,
                            (store_next && w + 1 < nw) ? ck + (size_t)(w + 1) * slice : nullptr, ck_es,
                            states, (size_t)(W + 1) * slice, nullptr, 0, prm, chebd};
        B();
        L(launch_state_chain<R>(a, st), "state_chain (forward)");
    };
    for (int w = 0; w < nw; ++w) {
        const int j0 = w * W, wlen = std::min(W, N - j0);
        xw(w);
        fwd(w, true);
        B();
        L(launch_slice_costs<R>(d, sv, j0, wlen, N, E, states, W, cv, c->Oj.as<double2>(), c->C5j.as<double>(),
                                c->Ofin.as<double2>(), st),
          "slice_costs");
    }
    check_cuda(c, cudaMemsetAsync(c->carry.p, 0, c->carry.bytes, st), "memset carry");
    for (int w = nw - 1; w >= 0; --w) {
        const int j0 = w * W, wlen = std::min(W, N - j0);
        if (w != nw - 1) {   // the last wave is resident from the forward pass
            xw(w);
            fwd(w, false);
        }
        B();
        L(launch_sources<R>(d, sv, j0, wlen, N, E, states, W, cv, c->Oj.as<double2>(), c->Ofin.as<double2>(), src, st),
          "sources");
        StateChainArgs<R> b{d, E, wlen, 1, sv, X, xs, c->carry.as<K>(), slice, c->carry.as<K>(), slice,
                            G, (size_t)W * slice, src, (size_t)W * slice, prm, chebd};
        B();
        L(launch_state_chain<R>(b, st), "state_chain (costate)");
        if (c->opt.gradient == QOC_GRAD_FIRST_ORDER) {
            B();
            L(launch_grad_first_order<R>(sys, sv, j0, wlen, E, states, G, W, c->dt, c->gpart.as<double>(), st),
              "expm_adj");
        } else {
            StateGradArgs<R> g{d, E, M, N, j0, wlen, W, sv, X, xs, states, G, sys.Hk, c->gpart.as<double>(), prm,
                               chebd, cheb ? c->cheb_host.K : 0, c->stscr.as<C>(), scr_stride};
            B();
            L(launch_state_grad<R>(g, p, n, st), "expm_adj");
        }
    }
    B();
    L(launch_finalize(E, M, N, u, c->alpha, c->Oj.as<double2>(), c->C5j.as<double>(), c->Ofin.as<double2>(),
                      c->gpart.as<double>(), grad, out, prm, st),
      "finalize");
    c->launches = launches;
}

void autotune(qoc_ctx* c, const double* u, double* grad, double* out);

void evaluate(qoc_ctx* c, const double* u, double* grad, double* out, const DevParams* known = nullptr) {
    if (!c->planned) plan(c);
    if (c->opt.autotune && !c->tuned) autotune(c, u, grad, out);
    if (c->path_kind == 2) {
        if (is_fp64(c)) evaluate_state_impl<double>(c, u, grad, out);
        else evaluate_state_impl<float>(c, u, grad, out);
        return;
    }
    if (is_fp64(c)) evaluate_impl<double>(c, u, grad, out, known);
    else evaluate_impl<float>(c, u, grad, out, known);
}

// ------------------------------------------------------------------------------------------
// autotuner (qoc_options.autotune): coordinate descent over the Taylor scheme, theta_max and the
// sweep form, each candidate timed by CUDA events on the context stream over two evaluations of
// the caller's inputs after one warm-up; the choice is cached per process and shape
// ------------------------------------------------------------------------------------------
struct TuneChoice {
    int taylor_scheme;
    int sweep;
    double theta_max;
    int wave_slices;   // 0: the planner's
};
std::mutex g_tune_mu;
std::map<std::vector<long long>, TuneChoice> g_tune_cache;

// One evaluation, replayed from the context's captured graph when qoc_options.graph applies (the
// per-slice path, where every decision is taken on the device; one graph per (u, grad, out)
// pointer triple, captured on first use and dropped by a new plan), else launched directly.
void run_eval(qoc_ctx* ctx, const double* u, double* grad, double* out) {
    if (ctx->opt.graph && !ctx->opt.profile && ctx->path_kind == 0) {
        const void* key[3] = {u, grad, out};
        if (!(ctx->gexec && key[0] == ctx->gkey[0] && key[1] == ctx->gkey[1] && key[2] == ctx->gkey[2])) {
            ctx->drop_graph();
            cudaGraph_t g = nullptr;
            check_cuda(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            try {
                evaluate(ctx, u, grad, out);
            } catch (...) {
                cudaStreamEndCapture(ctx->stream, &g);   // leave the stream usable
                if (g) cudaGraphDestroy(g);
                throw;
            }
            check_cuda(ctx, cudaStreamEndCapture(ctx->stream, &g), "end capture");
            // the serial sweeps' stream priority is recorded in its nodes; the graph keeps it
            cudaError_t e = cudaGraphInstantiate(&ctx->gexec, g, cudaGraphInstantiateFlagUseNodePriority);
            cudaGraphDestroy(g);
            check_cuda(ctx, e, "instantiate graph");
            for (int i = 0; i < 3; ++i) ctx->gkey[i] = key[i];
        }
        check_cuda(ctx, cudaGraphLaunch(ctx->gexec, ctx->stream), "graph launch");
        return;
    }
    evaluate(ctx, u, grad, out);
}

// mean device time of one evaluation as the context will run it (graph replay included)
double time_evals(qoc_ctx* c, const double* u, double* grad, double* out) {
    run_eval(c, u, grad, out);   // warm-up: first touches, the launch attributes, the capture
    cudaEvent_t a = nullptr, b = nullptr;
    check_cuda(c, cudaEventCreate(&a), "autotune event");
    check_cuda(c, cudaEventCreate(&b), "autotune event");
    const int reps = c->path_kind == 0 ? 4 : 2;   // short per-slice evaluations: more of them
    cudaEventRecord(a, c->stream);
    for (int k = 0; k < reps; ++k) run_eval(c, u, grad, out);
    cudaEventRecord(b, c->stream);
    const cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    check_cuda(c, e, "autotune timing");
    return ms / reps;
}

void apply_choice(qoc_ctx* c, const TuneChoice& t) {
    c->opt.taylor_scheme = t.taylor_scheme;
    c->opt.sweep = t.sweep;
    c->opt.theta_max = t.theta_max;
    c->opt.wave_slices = t.wave_slices;
    c->planned = false;
    plan(c);
}

void autotune(qoc_ctx* c, const double* u, double* grad, double* out) {
    c->tuned = true;   // set first: the timed evaluations below run the normal path
    c->tune_candidates = 0;
    if (c->path_kind == 2) return;   // state mode: nothing here to choose
    const qoc_options& o = c->opt;
    const int wave_user = o.wave_slices;
    const std::vector<long long> key = {o.precision, c->d, c->N, c->M, c->S_eff, c->E, o.gradient, o.adjoint,
                                        o.taylor_scheme, o.sweep, c->theta_user ? (long long)(o.theta_max * 1e9) : -1,
                                        o.plain_fp32_exp, o.reversal, wave_user, o.ckpt_stride};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            apply_choice(c, it->second);
            return;
        }
    }
    TuneChoice best{o.taylor_scheme, o.sweep, o.theta_max, wave_user};
    double best_ms = time_evals(c, u, grad, out);
    c->tune_candidates = 1;
    auto trial = [&](const TuneChoice& t) {
        apply_choice(c, t);
        const double ms = time_evals(c, u, grad, out);
        ++c->tune_candidates;
        if (ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    };
    if (best.taylor_scheme == QOC_TAYLOR_AUTO && c->ps) trial({QOC_TAYLOR_HORNER, best.sweep, best.theta_max, wave_user});
    if (!c->theta_user) {
        apply_choice(c, best);
        const double t0 = c->theta_max;   // the planner's default for the scheme chosen so far
        const TuneChoice base = best;
        trial({base.taylor_scheme, base.sweep, 0.5 * t0, wave_user});
        trial({base.taylor_scheme, base.sweep, 2.0 * t0, wave_user});
    }
    if (best.sweep == QOC_SWEEP_AUTO) {
        const TuneChoice base = best;
        trial({base.taylor_scheme, QOC_SWEEP_SERIAL, base.theta_max, wave_user});
        trial({base.taylor_scheme, QOC_SWEEP_SCAN, base.theta_max, wave_user});
    }
    if (wave_user == 0 && c->path_kind == 0) {
        // the split of the evolution into its two waves (per-slice path: the planner counts whole
        // rounds of resident CTAs, which the other stream's kernels partly fill): up to three
        // strides either way, keeping two waves
        apply_choice(c, best);
        const TuneChoice base = best;
        const int W0 = c->W, sg = c->seg, N = c->N;
        if (c->nw == 2)
            for (int k : {-3, -2, -1, 1, 2, 3}) {
                const int w = W0 + k * sg;
                if (2 * w < N || w >= N) continue;
                TuneChoice t = base;
                t.wave_slices = w;
                trial(t);
            }
    }
    apply_choice(c, best);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
}

qoc_status device_error(qoc_ctx* c) {
    DevParams h{};
    check_cuda(c, cudaMemcpyAsync(&h, c->prm.p, sizeof(DevParams), cudaMemcpyDeviceToHost, c->stream), "read params");
    check_cuda(c, cudaStreamSynchronize(c->stream), "sync");
    c->prof.harvest();
    if (h.err & kErrTimeout) return set_err(c, QOC_ERR_TIMEOUT, "a bounded device wait ran out");
    if (h.err & kErrStale)   // first: results computed with too small orders may overflow
        return set_err(c, QOC_ERR_STALE, "the controls need Taylor orders or grid exponents above those of the "
                                         "captured batch (theta = " + std::to_string(h.theta) + "); re-create the batch");
    if (h.err & kErrNonfinite) return set_err(c, QOC_ERR_NONFINITE, "NaN or Inf in the controls or the results");
    if (h.err & kErrRange)
        return set_err(c, QOC_ERR_RANGE, "Taylor order above its maximum for theta = " + std::to_string(h.theta));
    return QOC_OK;
}

#define QOC_GUARD_BEGIN try {
#define QOC_GUARD_END                                               \
    }                                                               \
    catch (const Fail& f) { return f.st; }                          \
    catch (const std::bad_alloc&) { return set_err(ctx, QOC_ERR_OOM, "host allocation failed"); } \
    catch (...) { return set_err(ctx, QOC_ERR_CUDA, "unexpected exception"); }

// One evaluation from an entry point: tuned first when qoc_options.autotune asks (never inside a
// capture), then run as run_eval runs it.
void evaluate_entry(qoc_ctx* ctx, const double* u, double* grad, double* out) {
    if (ctx->opt.autotune && !ctx->tuned) autotune(ctx, u, grad, out);
    run_eval(ctx, u, grad, out);
}

// argument checks of a batch call (errors through the offending context's qoc_last_error)
qoc_status check_batch(int count, qoc_ctx* const* ctxs, const double* const* u_dev, double* const* grad_dev,
                       double* const* out_dev) {
    if (count < 0 || (count > 0 && (!ctxs || !u_dev || !grad_dev || !out_dev))) return QOC_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        qoc_ctx* c = ctxs[i];
        if (!c) return QOC_ERR_ARG;
        c->err.clear();
        if (!c->has_sys || !c->has_tgt) return set_err(c, QOC_ERR_STATE, "set_system and set_targets must come first");
        if (!u_dev[i] || !grad_dev[i] || !out_dev[i]) return set_err(c, QOC_ERR_ARG, "NULL device pointer");
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == c) return set_err(c, QOC_ERR_ARG, "a context appears twice in the batch");
    }
    return QOC_OK;
}

// fork and join events of a batch, one pair per context (on the context's device)
struct BatchEvents {
    std::vector<cudaEvent_t> fork, join;
    qoc_status create(int count, qoc_ctx* const* ctxs) {
        fork.assign(count, nullptr);
        join.assign(count, nullptr);
        for (int i = 0; i < count; ++i) {
            cudaSetDevice(ctxs[i]->opt.device);
            if (cudaEventCreateWithFlags(&fork[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) != cudaSuccess)
                return set_err(ctxs[i], QOC_ERR_CUDA, "create event");
        }
        return QOC_OK;
    }
    ~BatchEvents() {
        for (auto e : fork)
            if (e) cudaEventDestroy(e);
        for (auto e : join)
            if (e) cudaEventDestroy(e);
    }
};

// Enqueues one evaluation of every context: the (p, n) of every batched-path context without
// frozen orders are picked first and read back with one wait; then every evaluation runs on its
// own context's streams, forked from `caller` (fork[i]) and joined into it (join[i]).  With frozen
// orders and tuning done nothing here waits on the host, so the caller's stream may be capturing.
qoc_status batch_body(int count, qoc_ctx* const* ctxs, const double* const* u_dev, double* const* grad_dev,
                      double* const* out_dev, cudaStream_t caller, const cudaEvent_t* fork, const cudaEvent_t* join) {
    qoc_ctx* cur = nullptr;
    try {
        std::vector<DevParams> hp(count);
        std::vector<char> known(count, 0);
        bool any = false;
        for (int i = 0; i < count; ++i) {
            qoc_ctx* c = cur = ctxs[i];
            check_cuda(c, cudaSetDevice(c->opt.device), "set device");
            if (!c->planned) plan(c);
            check_cuda(c, cudaEventRecord(fork[i], caller), "fork");
            check_cuda(c, cudaStreamWaitEvent(c->stream, fork[i], 0), "fork wait");
            if (c->opt.autotune && !c->tuned) autotune(c, u_dev[i], grad_dev[i], out_dev[i]);
            if (c->path_kind == 1 && !c->frozen) {
                check_cuda(c, launch_theta(u_dev[i], c->M, c->N, c->norms.as<double>(),
                                           c->delta.empty() ? nullptr : c->dDelta.as<double>(), c->E, c->dt,
                                           c->theta_max, c->opt.tol, c->opt.p_override, c->opt.n_override,
                                           c->prm.as<DevParams>(), c->stream),
                           "theta");
                check_cuda(c, cudaMemcpyAsync(&hp[i], c->prm.p, sizeof(DevParams), cudaMemcpyDeviceToHost, c->stream),
                           "read (p, n)");
                known[i] = 1;
                any = true;
            }
        }
        if (any)   // one wait for the (p, n) of the batched-path problems
            for (int i = 0; i < count; ++i)
                if (known[i]) check_cuda(cur = ctxs[i], cudaStreamSynchronize(ctxs[i]->stream), "sync (p, n)");
        for (int i = 0; i < count; ++i) {   // every evaluation on its own streams
            qoc_ctx* c = cur = ctxs[i];
            evaluate(c, u_dev[i], grad_dev[i], out_dev[i], known[i] ? &hp[i] : nullptr);
        }
        for (int i = 0; i < count; ++i) {   // join into the caller's stream
            qoc_ctx* c = cur = ctxs[i];
            check_cuda(c, cudaEventRecord(join[i], c->stream), "join");
            check_cuda(c, cudaStreamWaitEvent(caller, join[i], 0), "join wait");
        }
        return QOC_OK;
    } catch (const Fail& f) {
        return f.st;
    } catch (...) {
        return set_err(cur, QOC_ERR_CUDA, "unexpected exception");
    }
}

}  // namespace

// a captured batch (qoc_batch_create): the graph of one evaluation of every context
struct qoc_batch {
    std::vector<qoc_ctx*> ctxs;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
    cudaStream_t last = nullptr;   // stream of the last launch
    bool launched = false;
};

extern "C" {

void qoc_default_options(qoc_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = QOC_PREC_FP64;
    opt->tol = 0.0;
    opt->theta_max = 0.0;
    opt->ckpt_stride = 0;
    opt->device = 0;
    opt->stream = nullptr;
    opt->p_override = 0;
    opt->n_override = -1;
    opt->wave_slices = 0;
}

const char* qoc_status_string(qoc_status s) {
    switch (s) {
        case QOC_OK: return "QOC_OK";
        case QOC_ERR_ARG: return "QOC_ERR_ARG";
        case QOC_ERR_SHAPE: return "QOC_ERR_SHAPE";
        case QOC_ERR_NOT_HERMITIAN: return "QOC_ERR_NOT_HERMITIAN";
        case QOC_ERR_NONFINITE: return "QOC_ERR_NONFINITE";
        case QOC_ERR_STATE: return "QOC_ERR_STATE";
        case QOC_ERR_OOM: return "QOC_ERR_OOM";
        case QOC_ERR_CUDA: return "QOC_ERR_CUDA";
        case QOC_ERR_TIMEOUT: return "QOC_ERR_TIMEOUT";
        case QOC_ERR_UNSUPPORTED: return "QOC_ERR_UNSUPPORTED";
        case QOC_ERR_RANGE: return "QOC_ERR_RANGE";
        case QOC_ERR_STALE: return "QOC_ERR_STALE";
    }
    return "QOC_ERR_UNKNOWN";
}

qoc_status qoc_create(qoc_ctx** out, const qoc_options* opt) {
    if (!out) return QOC_ERR_ARG;
    *out = nullptr;
    qoc_options o;
    qoc_default_options(&o);
    if (opt) o = *opt;
    if (o.precision < QOC_PREC_FP64 || o.precision > QOC_PREC_BF16_SPLIT) return QOC_ERR_ARG;
    if (!(o.tol >= 0.0) || !(o.theta_max >= 0.0) || o.ckpt_stride < 0 || o.wave_slices < 0 || o.sweep < 0 ||
        o.sweep > QOC_SWEEP_SCAN || o.gradient < QOC_GRAD_EXACT || o.gradient > QOC_GRAD_FIRST_ORDER ||
        o.fault_inject < 0 || o.fault_inject > 1 || o.adjoint < QOC_ADJ_AUTO || o.adjoint > QOC_ADJ_RECOMPUTE ||
        o.reversal < 0 || o.reversal > 1 || o.propagation < QOC_PROP_UNITARY || o.propagation > QOC_PROP_STATE ||
        o.exponential < QOC_EXP_TAYLOR || o.exponential > QOC_EXP_CHEBYSHEV || o.taylor_scheme < QOC_TAYLOR_AUTO ||
        o.taylor_scheme > QOC_TAYLOR_HORNER || o.autotune < 0 || o.autotune > 1)
        return QOC_ERR_ARG;
    if (o.exponential == QOC_EXP_CHEBYSHEV && o.propagation != QOC_PROP_STATE) return QOC_ERR_UNSUPPORTED;
    // reversal regenerates states through the stored propagators, whose FP32 rounding would
    // accumulate over the backward pass: FP64 form only
    if (o.reversal && o.precision != QOC_PREC_FP64) return QOC_ERR_UNSUPPORTED;
    const bool f64 = o.precision == QOC_PREC_FP64;
    if (o.tol == 0.0) o.tol = f64 ? 1e-15 : 1e-8;
    const bool theta_user = o.theta_max > 0.0;
    if (o.theta_max == 0.0 && f64) o.theta_max = 0.25;   // FP32 forms: resolved by the planner
    qoc_ctx* ctx = new (std::nothrow) qoc_ctx;
    if (!ctx) return QOC_ERR_OOM;
    ctx->opt = o;
    ctx->theta_user = theta_user || f64;
    cudaError_t e = cudaSetDevice(o.device);
    if (e == cudaSuccess) {
        if (o.stream) {
            ctx->stream = reinterpret_cast<cudaStream_t>(o.stream);
        } else {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            ctx->own_stream = (e == cudaSuccess);
        }
    }
    if (e != cudaSuccess) {
        delete ctx;
        return QOC_ERR_CUDA;
    }
    *out = ctx;
    return QOC_OK;
}

void qoc_destroy(qoc_ctx* ctx) {
    if (!ctx) return;
    if (ctx->batches > 0) {   // a captured batch still refers to its buffers: the last batch frees it
        ctx->destroy_pending = true;
        return;
    }
    cudaSetDevice(ctx->opt.device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    ctx->drop_graph();
    if (ctx->aux) {
        cudaStreamSynchronize(ctx->aux);
        cudaStreamDestroy(ctx->aux);
    }
    for (auto e : ctx->events) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* qoc_last_error(const qoc_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

qoc_status qoc_set_system(qoc_ctx* ctx, int d, int M, const double* H0, const double* Hk, double dt, int N) {
    if (!ctx) return QOC_ERR_ARG;
    ctx->err.clear();
    if (ctx->batches > 0) return set_err(ctx, QOC_ERR_STATE, "the context belongs to a captured batch (qoc_batch_destroy first)");
    if (!H0 || (M > 0 && !Hk)) return set_err(ctx, QOC_ERR_ARG, "H0 or Hk is NULL");
    if (d < 1 || d > kMaxD) return set_err(ctx, QOC_ERR_SHAPE, "d must be in [1, 512]");
    if (M < 0 || M > kMaxControls) return set_err(ctx, QOC_ERR_SHAPE, "M must be in [0, 64]");
    if (N < 1) return set_err(ctx, QOC_ERR_SHAPE, "N must be >= 1");
    if (!std::isfinite(dt) || dt <= 0.0) return set_err(ctx, QOC_ERR_ARG, "dt must be finite and > 0");
    const size_t dd2 = (size_t)d * d * 2;
    if (!all_finite(H0, dd2) || (M > 0 && !all_finite(Hk, M * dd2)))
        return set_err(ctx, QOC_ERR_NONFINITE, "non-finite entry in H0 or Hk");
    if (!hermitian(H0, d)) return set_err(ctx, QOC_ERR_NOT_HERMITIAN, "H0 is not Hermitian");
    for (int k = 0; k < M; ++k)
        if (!hermitian(Hk + k * dd2, d))
            return set_err(ctx, QOC_ERR_NOT_HERMITIAN, "H_" + std::to_string(k + 1) + " is not Hermitian");
    QOC_GUARD_BEGIN
    check_cuda(ctx, cudaSetDevice(ctx->opt.device), "set device");
    ctx->planned = false;
    ctx->tuned = false;
    ctx->has_sys = ctx->has_tgt = false;
    ctx->d = d;
    ctx->M = M;
    ctx->N = N;
    ctx->dt = dt;
    ctx->H0.assign(H0, H0 + dd2);
    ctx->Hk.assign(Hk ? Hk : H0, Hk ? Hk + M * dd2 : H0);
    ctx->Hdet.clear();
    ctx->delta.clear();
    ctx->E = 1;
    // FP64 device copy [H0, H1..HM, Hdet] and the FP64 1-norms used by the (p, n) pick
    check_cuda(ctx, ctx->H64.alloc((M + 2) * dd2 * sizeof(double)), "alloc H64");
    check_cuda(ctx, cudaMemsetAsync(ctx->H64.p, 0, ctx->H64.bytes, ctx->stream), "memset H64");
    check_cuda(ctx, cudaMemcpyAsync(ctx->H64.p, H0, dd2 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream),
               "copy H0");
    if (M > 0)
        check_cuda(ctx, cudaMemcpyAsync(ctx->H64.as<double>() + dd2, Hk, M * dd2 * sizeof(double),
                                        cudaMemcpyHostToDevice, ctx->stream),
                   "copy Hk");
    check_cuda(ctx, ctx->norms.alloc((M + 2) * sizeof(double)), "alloc norms");
    check_cuda(ctx, launch_norms(ctx->H64.as<double2>(), M + 2, d, ctx->norms.as<double>(), ctx->stream), "norms");
    check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
    ctx->has_sys = true;
    return QOC_OK;
    QOC_GUARD_END
}

qoc_status qoc_set_targets(qoc_ctx* ctx, int S, const double* psi0, const double* psiT, int nF, const int* forbidden,
                           const double* col_weight, const double* psiT_path, const double* alpha) {
    if (!ctx) return QOC_ERR_ARG;
    ctx->err.clear();
    if (ctx->batches > 0) return set_err(ctx, QOC_ERR_STATE, "the context belongs to a captured batch (qoc_batch_destroy first)");
    if (!ctx->has_sys) return set_err(ctx, QOC_ERR_STATE, "qoc_set_system must come first");
    const int d = ctx->d, N = ctx->N;
    if (!psi0 || !psiT || !alpha || (nF > 0 && !forbidden)) return set_err(ctx, QOC_ERR_ARG, "NULL argument");
    if (S < 1 || S > d) return set_err(ctx, QOC_ERR_SHAPE, "S must be in [1, d]");
    if (nF < 0 || nF > d) return set_err(ctx, QOC_ERR_SHAPE, "nF must be in [0, d]");
    for (int i = 0; i < nF; ++i)
        if (forbidden[i] < 0 || forbidden[i] >= d) return set_err(ctx, QOC_ERR_SHAPE, "forbidden index out of range");
    const size_t blk = (size_t)d * S * 2;
    if (!all_finite(psi0, blk) || !all_finite(psiT, blk) || !all_finite(alpha, 5) ||
        (psiT_path && !all_finite(psiT_path, (size_t)N * blk)))
        return set_err(ctx, QOC_ERR_NONFINITE, "non-finite target, initial state or weight");
    double wsum = 0.0;
    std::vector<double> w(S, 1.0);
    if (col_weight) {
        for (int s = 0; s < S; ++s) {
            if (!std::isfinite(col_weight[s]) || col_weight[s] < 0.0)
                return set_err(ctx, QOC_ERR_ARG, "column weights must be finite and >= 0");
            w[s] = col_weight[s];
        }
    }
    for (double x : w) wsum += x;
    if (!(wsum > 0.0)) return set_err(ctx, QOC_ERR_ARG, "column weights must have a positive sum");
    ctx->planned = false;
    ctx->tuned = false;
    ctx->S = S;
    ctx->nF = nF;
    ctx->psi0.assign(psi0, psi0 + blk);
    ctx->psiT.assign(psiT, psiT + blk);
    if (psiT_path) ctx->path.assign(psiT_path, psiT_path + (size_t)N * blk);
    else ctx->path.clear();
    ctx->forb.assign(forbidden ? forbidden : nullptr, forbidden ? forbidden + nF : nullptr);
    ctx->w = w;
    ctx->Wsum = wsum;
    for (int i = 0; i < 5; ++i) ctx->alpha[i] = alpha[i];
    ctx->has_tgt = true;
    return QOC_OK;
}

qoc_status qoc_set_ensemble(qoc_ctx* ctx, int E, const double* delta, const double* Hdet) {
    if (!ctx) return QOC_ERR_ARG;
    ctx->err.clear();
    if (ctx->batches > 0) return set_err(ctx, QOC_ERR_STATE, "the context belongs to a captured batch (qoc_batch_destroy first)");
    if (!ctx->has_sys) return set_err(ctx, QOC_ERR_STATE, "qoc_set_system must come first");
    if (E < 1 || E > 65535) return set_err(ctx, QOC_ERR_SHAPE, "E must be in [1, 65535]");
    if (!delta) return set_err(ctx, QOC_ERR_ARG, "delta is NULL");
    if (!all_finite(delta, E)) return set_err(ctx, QOC_ERR_NONFINITE, "non-finite detuning");
    bool nonzero = false;
    for (int e = 0; e < E; ++e) nonzero |= (delta[e] != 0.0);
    const int d = ctx->d, M = ctx->M;
    const size_t dd2 = (size_t)d * d * 2;
    if (nonzero && !Hdet) return set_err(ctx, QOC_ERR_ARG, "Hdet is NULL while a detuning is non-zero");
    if (Hdet) {
        if (!all_finite(Hdet, dd2)) return set_err(ctx, QOC_ERR_NONFINITE, "non-finite entry in Hdet");
        if (!hermitian(Hdet, d)) return set_err(ctx, QOC_ERR_NOT_HERMITIAN, "Hdet is not Hermitian");
    }
    QOC_GUARD_BEGIN
    ctx->planned = false;
    ctx->tuned = false;
    ctx->E = E;
    ctx->delta.assign(delta, delta + E);
    if (Hdet) ctx->Hdet.assign(Hdet, Hdet + dd2);
    else ctx->Hdet.clear();
    check_cuda(ctx, ctx->dDelta.alloc(E * sizeof(double)), "alloc delta");
    check_cuda(ctx, cudaMemcpyAsync(ctx->dDelta.p, delta, E * sizeof(double), cudaMemcpyHostToDevice, ctx->stream),
               "copy delta");
    double* slot = ctx->H64.as<double>() + (size_t)(M + 1) * dd2;
    if (Hdet) {
        check_cuda(ctx, cudaMemcpyAsync(slot, Hdet, dd2 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream),
                   "copy Hdet");
    } else {
        check_cuda(ctx, cudaMemsetAsync(slot, 0, dd2 * sizeof(double), ctx->stream), "clear Hdet");
    }
    check_cuda(ctx, launch_norms(ctx->H64.as<double2>() + (size_t)(M + 1) * d * d, 1, d,
                                 ctx->norms.as<double>() + M + 1, ctx->stream),
               "Hdet norm");
    check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
    return QOC_OK;
    QOC_GUARD_END
}

qoc_status qoc_evaluate_device(qoc_ctx* ctx, const double* u_dev, double* grad_dev, double* out_dev) {
    if (!ctx) return QOC_ERR_ARG;
    ctx->err.clear();
    if (!ctx->has_sys || !ctx->has_tgt) return set_err(ctx, QOC_ERR_STATE, "set_system and set_targets must come first");
    if (!u_dev || !grad_dev || !out_dev) return set_err(ctx, QOC_ERR_ARG, "NULL device pointer");
    QOC_GUARD_BEGIN
    check_cuda(ctx, cudaSetDevice(ctx->opt.device), "set device");
    if (!ctx->planned) plan(ctx);
    evaluate_entry(ctx, u_dev, grad_dev, out_dev);
    return QOC_OK;
    QOC_GUARD_END
}

qoc_status qoc_evaluate_cost_and_grad(qoc_ctx* ctx, const double* u, double* cost, double* grad, double* terms) {
    if (!ctx) return QOC_ERR_ARG;
    ctx->err.clear();
    if (!ctx->has_sys || !ctx->has_tgt) return set_err(ctx, QOC_ERR_STATE, "set_system and set_targets must come first");
    if (!u || !cost || (!grad && ctx->M > 0)) return set_err(ctx, QOC_ERR_ARG, "NULL argument");
    const size_t mn = (size_t)ctx->M * ctx->N;
    if (!all_finite(u, mn)) return set_err(ctx, QOC_ERR_NONFINITE, "non-finite control");
    QOC_GUARD_BEGIN
    check_cuda(ctx, cudaSetDevice(ctx->opt.device), "set device");
    if (!ctx->planned) plan(ctx);
    cudaStream_t st = ctx->stream;
    if (mn) check_cuda(ctx, cudaMemcpyAsync(ctx->u_h.p, u, mn * sizeof(double), cudaMemcpyHostToDevice, st), "copy u");
    evaluate_entry(ctx, ctx->u_h.as<double>(), ctx->grad_h.as<double>(), ctx->out_h.as<double>());
    double out[6];
    if (mn)
        check_cuda(ctx, cudaMemcpyAsync(grad, ctx->grad_h.p, mn * sizeof(double), cudaMemcpyDeviceToHost, st),
                   "copy grad");
    check_cuda(ctx, cudaMemcpyAsync(out, ctx->out_h.p, 6 * sizeof(double), cudaMemcpyDeviceToHost, st), "copy cost");
    qoc_status s = device_error(ctx);   // synchronises
    if (s != QOC_OK) return s;
    *cost = out[0];
    if (terms)
        for (int i = 0; i < 5; ++i) terms[i] = out[1 + i];
    return QOC_OK;
    QOC_GUARD_END
}

qoc_status qoc_sync(qoc_ctx* ctx) {
    if (!ctx) return QOC_ERR_ARG;
    ctx->err.clear();
    QOC_GUARD_BEGIN
    if (!ctx->planned) {
        check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
        return QOC_OK;
    }
    return device_error(ctx);
    QOC_GUARD_END
}

qoc_status qoc_get_info(qoc_ctx* ctx, qoc_info* info) {
    if (!ctx || !info) return QOC_ERR_ARG;
    ctx->err.clear();
    std::memset(info, 0, sizeof(*info));
    QOC_GUARD_BEGIN
    if (ctx->planned) {
        DevParams h{};
        check_cuda(ctx, cudaMemcpyAsync(&h, ctx->prm.p, sizeof(DevParams), cudaMemcpyDeviceToHost, ctx->stream),
                   "read params");
        check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
        info->p = h.p;
        info->n = h.n;
        info->theta = h.theta;
        ctx->prof.harvest();
    }
    info->ckpt_stride = ctx->seg;
    info->wave_slices = ctx->W;
    info->n_waves = ctx->nw;
    info->launches_per_eval = ctx->launches;
    info->kernel_path = ctx->path_kind;
    info->device_bytes = (long long)ctx->device_bytes();
    if (ctx->opt.gradient == QOC_GRAD_FIRST_ORDER) info->adjoint_form = 2;
    else if (ctx->path_kind == 2) info->adjoint_form = 4;
    else if (ctx->path_kind == 1) info->adjoint_form = ctx->last_big_rev ? 0 : 1;
    else if (ctx->Zbuf.p && (ctx->ps ? ps_slots(info->p, info->n) : info->p - 1 + info->n) <= kZCap)
        info->adjoint_form = adj_lowrank_applies(ctx->S_eff, info->n, ctx->d) ? 3 : 0;
    else info->adjoint_form = 1;
    info->taylor_scheme = ctx->planned && ctx->ps ? 1 : 0;
    info->autotune_candidates = ctx->tune_candidates;
    if (ctx->planned && ctx->path_kind == 2 && ctx->opt.exponential == QOC_EXP_CHEBYSHEV) {
        info->p = ctx->cheb_host.K;       // the Chebyshev degree, no squaring
        info->n = 0;
    }
    return QOC_OK;
    QOC_GUARD_END
}

qoc_status qoc_evaluate_batch(int count, qoc_ctx* const* ctxs, const double* const* u_dev, double* const* grad_dev,
                              double* const* out_dev, void* stream) {
    qoc_status st = check_batch(count, ctxs, u_dev, grad_dev, out_dev);
    if (st != QOC_OK || count == 0) return st;
    BatchEvents ev;
    if ((st = ev.create(count, ctxs)) != QOC_OK) return st;
    return batch_body(count, ctxs, u_dev, grad_dev, out_dev, reinterpret_cast<cudaStream_t>(stream), ev.fork.data(),
                      ev.join.data());
}

qoc_status qoc_batch_create(int count, qoc_ctx* const* ctxs, const double* const* u_dev, double* const* grad_dev,
                            double* const* out_dev, void* stream, qoc_batch** out) {
    if (!out) return QOC_ERR_ARG;
    *out = nullptr;
    if (count < 1) return QOC_ERR_ARG;
    qoc_status st = check_batch(count, ctxs, u_dev, grad_dev, out_dev);
    if (st != QOC_OK) return st;
    const int dev = ctxs[0]->opt.device;
    for (int i = 0; i < count; ++i) {
        qoc_ctx* c = ctxs[i];
        if (c->opt.device != dev) return set_err(c, QOC_ERR_UNSUPPORTED, "a captured batch runs on one device");
        if (c->opt.profile) return set_err(c, QOC_ERR_UNSUPPORTED, "a captured batch takes no profiled context");
        try {
            check_cuda(c, cudaSetDevice(dev), "set device");
            if (!c->planned) plan(c);
        } catch (const Fail& f) {
            return f.st;
        } catch (...) {
            return set_err(c, QOC_ERR_CUDA, "unexpected exception");
        }
        if (c->path_kind == 2)
            return set_err(c, QOC_ERR_UNSUPPORTED, "state mode picks its orders on the host: not in a captured batch");
    }
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    BatchEvents ev;
    if ((st = ev.create(count, ctxs)) != QOC_OK) return st;
    // 1) one evaluation as qoc_evaluate_batch runs it: plans, allocations, tuning, and the orders
    if ((st = batch_body(count, ctxs, u_dev, grad_dev, out_dev, caller, ev.fork.data(), ev.join.data())) != QOC_OK)
        return st;
    if (cudaStreamSynchronize(caller) != cudaSuccess) return set_err(ctxs[0], QOC_ERR_CUDA, "sync the caller stream");
    for (int i = 0; i < count; ++i)
        if ((st = device_error(ctxs[i])) != QOC_OK) return st;
    // 2) freeze the batched-path contexts' orders at those of this evaluation
    std::vector<qoc_ctx*> froze;
    auto thaw = [&]() {
        for (qoc_ctx* c : froze) c->frozen = false;
    };
    for (int i = 0; i < count; ++i) {
        qoc_ctx* c = ctxs[i];
        if (c->path_kind != 1 || c->frozen) continue;
        DevParams h{};
        cudaError_t e = cudaMemcpy(&h, c->prm.p, sizeof(DevParams), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && !c->frozen_d.p) e = c->frozen_d.alloc(sizeof(DevParams));
        if (e == cudaSuccess) e = cudaMemcpy(c->frozen_d.p, &h, sizeof(DevParams), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            thaw();
            return set_err(c, QOC_ERR_CUDA, std::string("freeze orders: ") + cudaGetErrorString(e));
        }
        c->hp_frozen = h;
        c->frozen = true;
        froze.push_back(c);
    }
    // 3) capture a second evaluation on a private stream (the caller's may be the legacy stream)
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        thaw();
        return set_err(ctxs[0], QOC_ERR_CUDA, "create the capture stream");
    }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = batch_body(count, ctxs, u_dev, grad_dev, out_dev, cs, ev.fork.data(), ev.join.data());
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (st == QOC_OK && e2 != cudaSuccess) e = e2;
    }
    if (st == QOC_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, cudaGraphInstantiateFlagUseNodePriority);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (st == QOC_OK && e != cudaSuccess) st = set_err(ctxs[0], QOC_ERR_CUDA, std::string("capture the batch: ") + cudaGetErrorString(e));
    if (st != QOC_OK) {
        if (exec) cudaGraphExecDestroy(exec);
        cudaGetLastError();
        thaw();
        return st;
    }
    qoc_batch* b = new (std::nothrow) qoc_batch;
    if (!b) {
        cudaGraphExecDestroy(exec);
        thaw();
        return set_err(ctxs[0], QOC_ERR_OOM, "host allocation failed");
    }
    b->ctxs.assign(ctxs, ctxs + count);
    b->exec = exec;
    b->device = dev;
    for (qoc_ctx* c : b->ctxs) ++c->batches;
    *out = b;
    return QOC_OK;
}

qoc_status qoc_batch_launch(qoc_batch* b, void* stream) {
    if (!b) return QOC_ERR_ARG;
    qoc_ctx* c0 = b->ctxs[0];
    c0->err.clear();
    if (cudaSetDevice(b->device) != cudaSuccess) return set_err(c0, QOC_ERR_CUDA, "set device");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const cudaError_t e = cudaGraphLaunch(b->exec, st);
    if (e != cudaSuccess) return set_err(c0, QOC_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    b->last = st;
    b->launched = true;
    return QOC_OK;
}

qoc_status qoc_batch_sync(qoc_batch* b) {
    if (!b) return QOC_ERR_ARG;
    qoc_ctx* c0 = b->ctxs[0];
    c0->err.clear();
    if (cudaSetDevice(b->device) != cudaSuccess) return set_err(c0, QOC_ERR_CUDA, "set device");
    if (b->launched && cudaStreamSynchronize(b->last) != cudaSuccess)
        return set_err(c0, QOC_ERR_CUDA, "sync the launch stream");
    qoc_status first = QOC_OK;
    for (qoc_ctx* c : b->ctxs) {
        c->err.clear();
        qoc_status st = QOC_OK;
        try {
            st = device_error(c);
        } catch (const Fail& f) {
            st = f.st;
        }
        if (first == QOC_OK) first = st;
    }
    return first;
}

void qoc_batch_destroy(qoc_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->launched) cudaStreamSynchronize(b->last);
    cudaGraphExecDestroy(b->exec);
    for (qoc_ctx* c : b->ctxs)
        if (--c->batches == 0) {
            c->frozen = false;
            if (c->destroy_pending) qoc_destroy(c);
        }
    delete b;
}

qoc_status qoc_get_profile(qoc_ctx* ctx, qoc_profile* out) {
    if (!ctx || !out) return QOC_ERR_ARG;
    ctx->err.clear();
    std::memset(out, 0, sizeof(*out));
    QOC_GUARD_BEGIN
    check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
    ctx->prof.harvest();
    const int n = std::min((int)ctx->prof.names.size(), QOC_PROFILE_SLOTS);
    out->count = n;
    for (int i = 0; i < n; ++i) {
        std::snprintf(out->name[i], sizeof(out->name[i]), "%s", ctx->prof.names[i].c_str());
        out->launches[i] = ctx->prof.launches[i];
        out->total_ms[i] = ctx->prof.ms[i];
    }
    return QOC_OK;
    QOC_GUARD_END
}

qoc_status qoc_reset_profile(qoc_ctx* ctx) {
    if (!ctx) return QOC_ERR_ARG;
    ctx->err.clear();
    QOC_GUARD_BEGIN
    check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
    ctx->prof.harvest();
    ctx->prof.reset();
    return QOC_OK;
    QOC_GUARD_END
}

}  // extern "C"
