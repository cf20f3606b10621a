// Host/device interface between the C ABI layer and the CUDA kernels (internal, not installed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "qoc_device.cuh"

namespace qoc {

template <typename R> using C_t = typename Cplx<R>::T;

// Element of the block carried by the serial sweeps: FP64 complex in the FP64 form, an
// unevaluated pair hi + lo of FP32 complex numbers (x, y = hi; z, w = lo) in the FP32 form.
template <typename R> struct Carry;
template <> struct Carry<float> { using T = float4; };
template <> struct Carry<double> { using T = double2; };
template <typename R> using K_t = typename Carry<R>::T;

constexpr int kMaxControls = 64;
constexpr int kMaxD = 512;
constexpr int kPMax = 40;                 // largest Taylor order the heuristic may pick
constexpr size_t kMaxDynSmem = 232448 - 2048;   // opt-in dynamic shared memory per CTA

// The system (Eq. 1) in the compute precision R; u and delta stay FP64.
template <typename R>
struct SysView {
    int d, M, N;
    const C_t<R>* H0;     // d x d
    const C_t<R>* Hk;     // M x d x d
    const C_t<R>* Hdet;   // d x d or nullptr
    const double* delta;  // E or nullptr
    const double* u;      // M x N
};

// Column-panel layout of every d x S block on the device: the S columns are padded to
// Spad = ncb * cb and stored as ncb contiguous d x cb panels, so a CTA that owns one panel
// reads and writes contiguous memory.  Element (a, s) sits at (s / cb) * pstride + a * cb + s % cb;
// pstride >= d * cb is rounded up to 16 bytes so that every panel can be copied by cp.async.
// A block (one state, costate or source) occupies slice() = ncb * pstride elements.
template <typename R>
struct StateView {
    int Spad, cb, ncb, pstride;
    int S;                  // propagated columns (<= Spad; the padding columns are zero)
    __host__ __device__ size_t slice() const { return (size_t)ncb * pstride; }
};

// Cost inputs (Table I).
template <typename R>
struct CostView {
    int nF;
    const int* fmask;       // d: 1 for forbidden basis states
    const double* w;        // Spad column weights (0 on padding)
    double Wsum;            // sum of weights
    const C_t<R>* psiT;     // final target, panel layout d x Spad
    const C_t<R>* path;     // N targets (panel layout) or nullptr
    double alpha[5];        // [fid, C3, C4, C5, C67]
};

// ---- norms / (p, n) ----
cudaError_t launch_norms(const double2* mats, int count, int d, double* norms, cudaStream_t st);
cudaError_t launch_theta(const double* u, int M, int N, const double* norms, const double* delta, int E,
                         double dt, double theta_max, double tol, int p_override, int n_override,
                         DevParams* prm, cudaStream_t st, const DevParams* frozen = nullptr);

// ---- conversions ----
template <typename R>
cudaError_t launch_convert(const double2* src, C_t<R>* dst, size_t count, cudaStream_t st);
template <typename R>
cudaError_t launch_to_panels(const double2* src, C_t<R>* dst, int d, int S, StateView<R> sv,
                             int copies, size_t dst_stride, size_t src_stride, cudaStream_t st);

// ---- fused per-slice exponential kernels ----
// Thread layout of the per-slice kernels: a G x G grid of threads, thread (ty, tx) owning the
// MT x MT outputs (ty + G a, tx + G b), so the padded dimension is D = MT G.  MT in 1..4 is the
// one with the least padding for G <= 22 (at most 484 threads); on ties the smaller MT (more
// threads).
struct SliceTile { int MT, G, D; };
// wide: among tiles of equal padding prefer more outputs per thread when the grid keeps at least
// 10 threads a side (the FP32 adjoint kernels: at d = 40, 4 x 4 outputs on a 10 x 10 grid ran the
// adjoint in 0.82 ms against 0.89 ms with 2 x 2 on 20 x 20, while the forward was slower with 4 x 4)
inline SliceTile slice_tile(int d, bool wide = false) {
    SliceTile best{0, 0, 1 << 30};
    for (int mt = 1; mt <= 4; ++mt) {
        const int g = (d + mt - 1) / mt;
        if (g > 22) continue;
        if (mt * g < best.D || (wide && mt * g == best.D && g >= 10)) best = {mt, g, mt * g};
    }
    return best;
}
// threads of a per-slice CTA: G x G rounded up to whole warps (the extra threads take part in
// the element-wise loops and reductions only)
inline int slice_threads(int G) { return (G * G + 31) / 32 * 32; }
// Inputs of the forward products of every slice exponential, kept for the reverse-mode adjoint:
// product r (r = 0 .. p-2: Horner step i = p-1-r, right operand Z_{i+1}; r = p-1+m: squaring m,
// operand S_m = T^(2^m)) stores the conjugate transpose of its right operand, rounded to the
// compute precision, at Z + ((e * wmax + j) * cap + r) * mstride.  Used when p - 1 + n <= cap.
template <typename R>
struct ZStore {
    C_t<R>* Z;              // nullptr: no stores (the adjoint recomputes, block recursion)
    int cap;
    size_t mstride;
    int wmax;
    int ps;                 // 1: the forward evaluates T by Paterson-Stockmeyer (slot layout below)
};
constexpr int kZCap = 24;

// Paterson-Stockmeyer form of the FP32 per-slice exponential (block size 3):
//   T_p(X) = sum_q (X^3)^q B_q,  B_q = c_3q I + c_3q+1 X + c_3q+2 X^2  (c_k = 1/k!, 0 for k > p),
// evaluated as W_qt (formed element-wise) and W_q = B_q + X^3 W_{q+1}, q = qt-1 .. 0, T = W_0.
// The top block qt is p / 3, or p / 3 - 1 when 3 divides p (the last block c_p I is then folded
// into the one below it as c_p X^3).  The stored operands (conjugate transposes, as in ZStore):
// slot 0 X^2, slot 1 X^3, slot 2 + (qt - 1 - q) W_{q+1} (chain product q), slot qt + 2 + m the
// squaring operand S_m.
__host__ __device__ inline int ps_top(int p) { return (p % 3 == 0 && p >= 3) ? p / 3 - 1 : p / 3; }
__host__ __device__ inline int ps_slots(int p, int n) { return ps_top(p) + 2 + n; }
// the batched path also keeps X^dag of every item (the last slot) for its reverse mode
inline int ps_big_slots(int p, int n) { return ps_slots(p, n) + 1; }
// the forward stored the operands of this evaluation's (p, n) (the reverse mode applies)
template <typename R>
__host__ __device__ inline bool zs_fits(const ZStore<R>& zs, int p, int n) {
    return zs.Z && (zs.ps ? ps_slots(p, n) : p - 1 + n) <= zs.cap;
}
static_assert(kPsCoefs >= kPMax + 4, "coefficients up to index 3 qt + 3 <= p + 3");
static_assert(kPsMaxBlocks > kPMax / 3, "one grid exponent per block");

template <typename R> int fused_max_d();
// resident CTAs per SM of the per-slice forward (adjoint = false) or reverse-mode adjoint kernel
template <typename R> int fused_ctas_per_sm(int d, bool adjoint);
int split_ctas_per_sm(int d);
template <typename R> size_t fused_adj_smem(int d);   // dynamic SMEM of the per-slice adjoint kernel
template <typename R>
cudaError_t launch_expm_fwd_fused(const DevParams* prm, const SysView<R>& sys, int j0, int wlen, int E,
                                  C_t<R>* Ubuf, long long ustride, int wmax, const ZStore<R>& zs, cudaStream_t st);
// the adjoint: reverse mode over the stored products when they are there (two products per step),
// else the block recursion (three); the kernel of the other mode exits at once
template <typename R>
cudaError_t launch_expm_adj_fused(const DevParams* prm, const SysView<R>& sys, const StateView<R>& sv, int j0,
                                  int wlen, int E, const C_t<R>* states, const C_t<R>* Gbuf, int wmax,
                                  double* gpart, const ZStore<R>& zs, cudaStream_t st, int* launches);

// The per-slice low-rank reverse-mode adjoint (k_expm_adj_lr) applies when the cotangent's rank
// after the squarings, r = 2^n S, is at most kLrMax and at most d / 8.  Measured on GB300 (FP32,
// N = 2000): r = 2 at d = 64 takes the adjoint from 1.81 to 0.73 ms, r = 2 at d = 40 from 0.54 to
// 0.33 ms, r = 4 at d = 48 from 0.75 to 0.52 ms; r = 16 at d = 40 is slower (1.27 against 0.88 ms):
// its d x r products reuse operands less than the dense d x d ones.
constexpr int kLrMax = 16;
__host__ __device__ inline bool adj_lowrank_applies(int S, int n, int d) {
    if (n > 10) return false;
    const int r = S << n;
    return r <= kLrMax && 8 * r <= d;
}

// ---- split hi+lo FP32 slice exponential (FP32 form) ----
int split_max_d();
// sH: s H_0, s H_1 .. s H_M, s H_det as FP32 pairs, written by launch_split_scale after the
// (p, n) pick of the evaluation
cudaError_t launch_split_scale(const DevParams* prm, const double2* H64, size_t count, float4* sH, cudaStream_t st);
cudaError_t launch_expm_fwd_split(const DevParams* prm, const SysView<float>& sys, const float4* sH, int j0, int wlen,
                                  int E, float2* Ubuf, long long ustride, int wmax, const ZStore<float>& zs,
                                  cudaStream_t st);
// Paterson-Stockmeyer form of the same exponential (zs.ps = 1), d <= ps_max_d(): the forward
// (k_expm_split.cu) and its reverse-mode adjoints, dense and low-rank (k_expm_ps.cu); without
// stored operands the block recursion (k_expm_adj) differentiates the same polynomial
int ps_max_d();
int ps_fwd_ctas_per_sm(int d);
int ps_adj_ctas_per_sm(int d);
cudaError_t launch_expm_fwd_ps(const DevParams* prm, const SysView<float>& sys, const float4* sH, int j0, int wlen,
                               int E, float2* Ubuf, long long ustride, int wmax, const ZStore<float>& zs,
                               cudaStream_t st);
cudaError_t launch_expm_adj_ps(const DevParams* prm, const SysView<float>& sys, const StateView<float>& sv, int j0,
                               int wlen, int E, const float2* states, const float2* Gbuf, int wmax, double* gpart,
                               const ZStore<float>& zs, cudaStream_t st, int* launches);

// ---- large-d batched slice exponentials and adjoint (k_big.cu) ----
struct BigSys {
    int d, M, N;
    const double2* H64;   // FP64 [H0, H1..HM, Hdet]
    const double* u;      // M x N
    const double* delta;  // E or nullptr
    int has_det;
};
template <typename R>
struct BigArgs {
    const DevParams* prm;
    BigSys bsys;
    int d, E, j0, wlen, wmax;
    void* scratch;        // per-item matrices of the wave (mstride elements apart)
    size_t mstride;       // elements per matrix slot (>= d * d)
    void* Ubuf;           // propagator buffer of the wave (C_t<R>, U at 0 and U^dag at ustride / 2)
    long long ustride;
    const float4* sH;     // FP32 split form: s H_0 .. s H_det as pairs (launch_split_scale), or nullptr
    int ps;               // 1: Paterson-Stockmeyer form of the split exponential (FP32 forms)
};
// bytes of scratch per wave item: FP64 six double2 matrices; FP32 the larger of the adjoint's six
// float2 matrices and the forward's float4 matrices (three for Horner, five for Paterson-Stockmeyer)
inline size_t big_scratch_per_item(int d, bool fp64, bool ps = false) {
    const size_t dd = (size_t)d * d, fwd = (ps ? 5 : 3) * dd * 16;
    return fp64 ? 6 * dd * 16 : (6 * dd * 8 > fwd ? 6 * dd * 8 : fwd);
}
// zst (or nullptr): store of the p - 1 + n product operands for the reverse-mode adjoint
// (conjugate transposes, rounded, at zst + (item * (p - 1 + n) + r) * mstride)
struct OzFwd;
// ozf (FP32 forms with the Paterson-Stockmeyer form only): its products on the tensor cores
template <typename R>
cudaError_t launch_big_expm(const BigArgs<R>& a, const DevParams& hp, bool split, cudaStream_t st, int* launches,
                            C_t<R>* zst = nullptr, const OzFwd* ozf = nullptr);
struct OzRev;
// oz (FP32 form only, or nullptr): run the reverse-mode products on the tensor cores (BF16_SPLIT)
template <typename R>
cudaError_t launch_big_adj_rev(const BigArgs<R>& a, const SysView<R>& sys, const StateView<R>& sv, const C_t<R>* states,
                               const C_t<R>* Gbuf, double* gpart, int p, int n, const C_t<R>* zst, cudaStream_t st,
                               int* launches, const OzRev* oz = nullptr);
// the reverse mode of the Paterson-Stockmeyer form (FP32 forms; hp: the evaluation's parameters,
// zst: the ps_slots(p, n) operands of each item)
template <typename R>
cudaError_t launch_big_adj_rev_ps(const BigArgs<R>& a, const SysView<R>& sys, const StateView<R>& sv,
                                  const C_t<R>* states, const C_t<R>* Gbuf, double* gpart, const DevParams& hp,
                                  const C_t<R>* zst, cudaStream_t st, int* launches, const OzRev* oz = nullptr);
template <typename R>
cudaError_t launch_big_adj(const BigArgs<R>& a, const SysView<R>& sys, const StateView<R>& sv, const C_t<R>* states,
                           const C_t<R>* Gbuf, double* gpart, int p, int n, cudaStream_t st, int* launches);

// ---- tensor-core (tcgen05) adjoint products of the large-d path, TF32_SPLIT form (k_tc.cu) ----
constexpr int kTcMats = 10;   // XH, Ubar, and two sets of Z11 / Z12 in row and column layouts
constexpr int kTcSplit = 3;   // TF32 terms per real value (hi, mid, lo)
inline int tc_ld(int d) { return (d + 3) / 4 * 4; }   // row stride (elements): 16-byte rows for TMA
struct TcTerm { int a_mat, b_mat, acc; };
struct TcStep {
    int nterms;
    TcTerm t[3];
    int kind, i, nacc;            // kind 0: Horner step i, 1: squaring
    int out0_row, out0_col, out1_row, out1_col;
    int fault;              // withhold the first operand copy (test of the bounded wait)
};
struct TcMats { int xh, ub, z11_row, z11_col, z12_row, z12_col; };
struct TcMaps {                   // two CUtensorMap (128 bytes, 64-byte aligned) over the planes
    alignas(64) unsigned char a[128];
    alignas(64) unsigned char b[128];
};
struct TcAdjArgs {
    int fault;              // qoc_options.fault_inject
    DevParams* prm;
    SysView<float> sys;
    StateView<float> sv;
    int d, E, j0, wlen, wmax, p, n;
    const float2* states;
    const float2* Gbuf;
    float* planes;
    TcMaps maps;
    double* gpart;
};
size_t tc_scratch_floats(int d, int items);
cudaError_t tc_make_maps(float* planes, int d, int items, TcMaps* maps);
cudaError_t launch_tc_adj(const TcAdjArgs& a, cudaStream_t st, int* launches);

// ---- tensor-core adjoint products with exact leading-level accumulation, BF16_SPLIT (k_oz.cu) ----
constexpr int kOzSlices = 4;     // seven-bit slices per value (adjoint products: FP32-grade)
constexpr int kOzFwdSlices = 6;  // seven-bit slices per value (forward products: split-grade)
constexpr int kOzFwdMinD = 128;  // d range whose forward products BF16_SPLIT runs on the tensor cores
constexpr int kOzFwdMaxD = 384;  // (the three exact slice levels stay exact up to here)
constexpr int kOzMats = 5;       // sliced matrices per item: A1, B1, A2, B2 of a reverse step, X^dag
inline int oz_ld(int d) { return (d + 7) / 8 * 8; }   // plane row stride (BF16): 16-byte rows for TMA
struct OzSliceJob {
    const void* src;        // d x d row-major complex matrices, item i at src + i * stride elements:
                            // float2 (adjoint) or float4 value pairs (forward)
    size_t stride;
    int mat;                // plane matrix to write
    int col;                // 0: row layout (A operand), 1: column layout (B operand)
};
struct OzSliceJobs { OzSliceJob job[4]; };
struct OzJob {              // out = alpha A B (+ out if beta) (+ I if ident), per item
    int a_mat, b_mat;
    float2* out;
    long long ostride;
    float alpha;
    int beta, ident;
};
struct OzJobs {
    OzJob j[2];
    int fault;              // withhold the first operand copy (test of the bounded wait)
};
// the reverse-mode adjoint's products on the tensor cores: state of one wave
struct OzRev {
    int fault;              // qoc_options.fault_inject
    DevParams* prm;
    int d, items, cap;      // items of this wave; items the plane array holds
    unsigned char* scratch; // oz_scratch_bytes(d, cap): planes, then exponents
    TcMaps maps;            // oz_make_maps over the planes
    const float2* xh;       // X^dag of the wave (sliced once, into matrix 4)
    int* xh_sliced;         // host flag: X^dag already sliced for this wave
};
size_t oz_plane_bytes(int d, int items);
size_t oz_scratch_bytes(int d, int items);
cudaError_t oz_make_maps(void* planes, int d, int items, TcMaps* maps);
cudaError_t launch_oz_slice(const OzSliceJobs& jobs, int njobs, int d, int items, int cap, unsigned char* scratch,
                            cudaStream_t st);
cudaError_t launch_oz_mm(const OzJobs& jobs, int njobs, int d, int items, int cap, unsigned char* scratch,
                         const TcMaps& maps, DevParams* prm, cudaStream_t st);
// one reverse-mode step (the products of k_big_rev): mode 0 (Horner step i) O1 = A1 B1 / i and
// O2 += A2 B2 / i; mode 1 (squaring) O1 = A1 B1 + A2 B2; ops = {A1, B1, A2, B2} with item strides
cudaError_t oz_rev_step(const OzRev& z, const float2* const ops[4], const size_t strides[4], float2* O1, float2* O2,
                        size_t ms, int mode, int i, cudaStream_t st, int* launches);

// The forward products of the Paterson-Stockmeyer form on the tensor cores (BF16_SPLIT, batched
// path): six seven-bit slices of the value pairs, the leading two slice levels accumulated exactly
// and the rest pre-weighted, so a product is as accurate as the split SIMT product it replaces.
struct OzFwd {
    int fault;              // qoc_options.fault_inject
    DevParams* prm;
    int d, items, cap;
    unsigned char* scratch; // oz_fwd_scratch_bytes(d, cap): planes, then exponents
    TcMaps maps;            // oz_fwd_make_maps over the planes
};
size_t oz_fwd_scratch_bytes(int d, int items);
cudaError_t oz_fwd_make_maps(void* planes, int d, int items, TcMaps* maps);
// out = A B (kind 1) or A B + c0 I + c1 X + c2 X^2 (kind 2, the chain product), written as value
// pairs grid-split with `magic`; a_src / b_src (item stride ms) are sliced into matrices a_mat /
// b_mat first, or null when that matrix already holds the operand's slices
cudaError_t oz_fwd_product(const OzFwd& z, const float4* a_src, int a_mat, const float4* b_src, int b_mat,
                           float4* out, size_t ms, int kind, float magic, const float4* X, const float4* X2, float2 c0,
                           float2 c1, float2 c2, cudaStream_t st, int* launches);

// ---- serial sweeps (k_serial.cu) ----
// mode 0: forward propagation of one wave (grid z = 1) from checkpoint `seg0`, storing the
//         states of the wave and the carried block every `seg` slices (checkpoints seg0 + 1, ..)
// mode 1: regeneration of the wave's states, one CTA per checkpoint segment in parallel
// mode 2: reversal: the wave's states regenerated backwards from its last state (rev_src, the
//         first state of the next wave), Psi_{j-1} = U_j^dag Psi_j (grid z = 1)
template <typename R>
struct ChainArgs {
    int d;
    StateView<R> sv;
    int wlen, seg, mode, E;
    K_t<R>* ckpt;           // [E][nseg_total] carried blocks
    size_t ck_estride;      // elements per member
    int seg0, nseg_total;
    const C_t<R>* Ubuf;     // slice propagators, or ...
    long long ustride;
    int wmax;
    C_t<R>* states;         // [E][wmax + 1] FP32/FP64 blocks of the wave
    const K_t<R>* Uk;       // ... carried segment products (exactly one of the two is set)
    const DevParams* prm;   // grid exponent eu of the FP32 form (nullptr: 1)
    const C_t<R>* rev_src = nullptr;   // mode 2: last state of the wave, member e at + e * rev_estride
    size_t rev_estride = 0;
};
template <typename R> cudaError_t launch_chain(const ChainArgs<R>& a, cudaStream_t st);
// Costate sweep G_{j-1} = U_j^dag G_j + src_{j-1}, split into segments of `seg` slices that run in
// parallel (grid z): segment z (slices a..b) starts from G_b = Y_z + src_b with in-carry Y_z
// (cin, or zero), writes G_b..G_a (rounded to G and/or carried to Gk) and leaves
// U_a^dag G_a in cout.  Block (e, z) of cin / cout sits at base + e * es + z * slice.
template <typename R>
struct CostateArgs {
    int d;
    StateView<R> sv;
    int wlen, seg, E;
    const C_t<R>* U;        // U_j at U + e * u_es + j * ustride, U_j^dag at + ustride / 2, or ...
    const K_t<R>* Uk;       // ... carried segment products, same layout (exactly one is set)
    long long ustride;
    size_t u_es;
    const C_t<R>* src;      // src_j at src + e * src_es + j * slice ...
    const K_t<R>* srck;     // ... or carried sources (exactly one of the two is set)
    size_t src_es;
    C_t<R>* G;              // G_j (rounded) at G + e * g_es + j * slice, or nullptr
    K_t<R>* Gk;             // G_j (carried), same layout, or nullptr
    size_t g_es;
    const K_t<R>* cin;      // in-carries or nullptr (zero)
    size_t cin_es;
    K_t<R>* cout;           // out-carries or nullptr
    size_t cout_es;
    int zero_next;          // also clear block (e, nz) of cout
    const DevParams* prm;   // grid exponent eu of the FP32 form (nullptr: 1)
};
template <typename R> cudaError_t launch_costate(const CostateArgs<R>& a, cudaStream_t st);

// ---- segment products (k_scan.cu) ----
// P_z = U_b ... U_a for every checkpoint segment z of a wave (a = z * seg, b = min(wlen, a + seg)
// - 1) by a pairwise product tree in carried precision (log2(seg) batched launches), stored
// carried with its adjoint: P_z at P + (e * nzmax + z) * ustride, P_z^dag at + ustride / 2.
template <typename R>
struct SegProdArgs {
    int d, E, wlen, seg, nzmax;
    const C_t<R>* U;        // U_j at U + (e * wmax + j) * ustride
    long long ustride;
    int wmax;
    K_t<R>* lv0;            // two level buffers of E * nzmax * ceil(seg / 2) matrices of mstride
    K_t<R>* lv1;
    size_t mstride;
    K_t<R>* P;
    const DevParams* prm;   // grid exponent eu of the FP32 form (bound on the norms of U_j)
};
template <typename R> cudaError_t launch_seg_products(const SegProdArgs<R>& a, cudaStream_t st, int* launches);
template <typename R>
cudaError_t launch_to_carry(const double2* src, K_t<R>* dst, int d, int S, StateView<R> sv, int copies,
                            size_t dst_stride, cudaStream_t st);

// ---- state-mode propagation (k_state.cu): Taylor-on-vector without forming U_j ----
// Chebyshev expansion of the slice map (state mode): exp(-i dt H) = sum_k (-i)^k a_k T_k(dt H /
// theta), a_0 = J_0(theta), a_k = 2 J_k(theta), theta >= dt * spectral radius; device copy
constexpr int kChebMax = 96;
struct ChebCoef {
    int K;                  // degree
    double inv_theta;       // 1 / theta
    double a[kChebMax + 1];
};
template <typename R>
struct StateChainArgs {
    int d, E, wlen, dir;    // dir 0: forward Psi_j = T(X_j)^(2^n) Psi_{j-1}; 1: costate
    StateView<R> sv;
    const void* X;          // X_j of item e * wlen + jl at X + item * xs (FP32: float4 pairs; FP64: double2)
    size_t xs;
    const K_t<R>* cin;      // starting block of member e at + e * cin_es (costate: in-carry, may be null)
    size_t cin_es;
    K_t<R>* cout;           // carried block after the wave (forward: next checkpoint; costate: out-carry)
    size_t cout_es;
    C_t<R>* out;            // forward: states (wlen + 1 blocks); costate: G (wlen blocks), + e * out_es
    size_t out_es;
    const C_t<R>* src;      // costate: sources, + e * src_es
    size_t src_es;
    const DevParams* prm;
    const ChebCoef* cheb = nullptr;   // device coefficients: Chebyshev in place of Taylor
};
template <typename R>
struct StateGradArgs {
    int d, E, M, N, j0, wlen, wmax;
    StateView<R> sv;
    const void* X;
    size_t xs;
    const C_t<R>* states;   // Psi of the wave, (wmax + 1) blocks per member
    const C_t<R>* G;        // costates, wmax blocks per member
    const C_t<R>* Hk;       // M x d x d in the compute precision
    double* gpart;          // E x M x N
    const DevParams* prm;
    const ChebCoef* cheb = nullptr;   // device coefficients: Chebyshev in place of Taylor
    int K = 0;              // Chebyshev degree (host copy, for the shared-memory size)
    C_t<R>* scr = nullptr;  // per-item global scratch (state_grad_scratch elements each)
    size_t scr_stride = 0;
};
constexpr int kStateMaxColumns = 8;
template <typename R> size_t state_grad_smem(int d, int S, int p, int n, int K);
size_t state_grad_scratch(int d, int S, int p, int n, int K);
template <typename R>
cudaError_t launch_state_x(const DevParams* prm, int d, int M, int N, const double* u, const double* delta, int has_det,
                           const void* Hsrc, int j0, int wlen, int E, void* X, size_t xs, cudaStream_t st);
template <typename R> cudaError_t launch_state_chain(const StateChainArgs<R>& a, cudaStream_t st);
template <typename R> cudaError_t launch_state_grad(const StateGradArgs<R>& a, int p, int n, cudaStream_t st);

// ---- per-slice costs, sources, final reduction (k_chain.cu) ----
template <typename R>
cudaError_t launch_slice_costs(int d, StateView<R> sv, int j0, int wlen, int N, int E, const C_t<R>* states,
                               int wmax, const CostView<R>& cv, double2* Oj, double* C5j, double2* Ofin,
                               cudaStream_t st);
template <typename R>
cudaError_t launch_sources(int d, StateView<R> sv, int j0, int wlen, int N, int E, const C_t<R>* states,
                           int wmax, const CostView<R>& cv, const double2* Oj, const double2* Ofin,
                           C_t<R>* src, cudaStream_t st);
// the paper's first-order gradient (Eq. 11) from Psi_j and G_j, in place of the exact adjoint
template <typename R>
cudaError_t launch_grad_first_order(const SysView<R>& sys, const StateView<R>& sv, int j0, int wlen, int E,
                                    const C_t<R>* states, const C_t<R>* Gbuf, int wmax, double dt, double* gpart,
                                    cudaStream_t st);
cudaError_t launch_finalize(int E, int M, int N, const double* u, const double* alpha, const double2* Oj,
                            const double* C5j, const double2* Ofin, const double* gpart, double* grad,
                            double* out, DevParams* prm, cudaStream_t st);

}  // namespace qoc
