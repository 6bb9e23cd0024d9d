// Shared definitions of the LO-AFQMC CUDA library: the context, status
// plumbing and small device helpers.  Every kernel and host routine of the
// library includes this file; nothing here is visible through the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <cusolverDn.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include <cuda.h>

#include "../../include/lo_afqmc.h"

namespace loaf {

// ---------------------------------------------------------------------------
// status plumbing
// ---------------------------------------------------------------------------

struct Error {
    loaf_status code;
    std::string msg;
};

#define LOAF_CUDA(call)                                                              \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            throw ::loaf::Error{e_ == cudaErrorMemoryAllocation ? LOAF_ERR_OOM       \
                                                                : LOAF_ERR_CUDA,     \
                                std::string(#call) + ": " + cudaGetErrorString(e_)}; \
        }                                                                            \
    } while (0)

#define LOAF_CUBLAS(call)                                                            \
    do {                                                                             \
        cublasStatus_t s_ = (call);                                                  \
        if (s_ != CUBLAS_STATUS_SUCCESS)                                             \
            throw ::loaf::Error{LOAF_ERR_CUDA,                                       \
                                std::string(#call) + ": cublas status " +            \
                                    std::to_string((int)s_)};                        \
    } while (0)

#define LOAF_CUSOLVER(call)                                                          \
    do {                                                                             \
        cusolverStatus_t s_ = (call);                                                \
        if (s_ != CUSOLVER_STATUS_SUCCESS)                                           \
            throw ::loaf::Error{LOAF_ERR_CUDA,                                       \
                                std::string(#call) + ": cusolver status " +          \
                                    std::to_string((int)s_)};                        \
    } while (0)

#define LOAF_REQUIRE(cond, code, text)                       \
    do {                                                     \
        if (!(cond)) throw ::loaf::Error{(code), (text)};    \
    } while (0)

#define LOAF_LAUNCH_CHECK() LOAF_CUDA(cudaGetLastError())

// ---------------------------------------------------------------------------
// device buffers owned by the context
// ---------------------------------------------------------------------------

// Number of device allocations and frees made through DevBuf in this process.
// A recorded CUDA graph holds buffer addresses, so a graph is replayed only
// while this count is the one it was recorded at.
inline std::atomic<unsigned long long>& devbuf_generation() {
    static std::atomic<unsigned long long> g{0};
    return g;
}

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    void release() {
        if (ptr) {
            cudaFree(ptr);
            devbuf_generation().fetch_add(1);
        }
        ptr = nullptr;
        bytes = 0;
    }
    // grow (never shrink); contents are not preserved
    void ensure(size_t nbytes) {
        if (nbytes <= bytes) return;
        release();
        LOAF_CUDA(cudaMalloc(&ptr, nbytes));
        devbuf_generation().fetch_add(1);
        bytes = nbytes;
    }
    // as ensure, and zero-filled whenever it had to (re)allocate
    void ensure_zeroed(size_t nbytes, cudaStream_t stream) {
        if (nbytes <= bytes) return;
        ensure(nbytes);
        LOAF_CUDA(cudaMemsetAsync(ptr, 0, nbytes, stream));
    }
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// ---------------------------------------------------------------------------
// 16-bit operand tiles for the tensor cores
// ---------------------------------------------------------------------------
// A tile is 128 rows x 64 k of 16-bit values (16 KB) stored as the shared-
// memory image the MMA reads with the 128-byte swizzle: row r occupies bytes
// [128 r, 128 r + 128) and its 16-byte chunk j (k = 8 j .. 8 j + 7) sits at
// chunk position j ^ (r mod 8).  A whole tile moves with one bulk copy.
constexpr int kTileRows = 128;
constexpr int kTileK = 64;
constexpr int kTileElems = kTileRows * kTileK;
constexpr uint32_t kTileBytes = kTileElems * 2;

__host__ __device__ inline int sw128_elem(int row, int k) {
    return row * kTileK + ((((k >> 3) ^ (row & 7)) << 3) | (k & 7));
}

// Delta planes (hi and lo, one each): tile (c, rb, kb) holds walker rows
// z = 2w + re/im in [128 rb, 128 rb + 128) of orbital column c and basis
// functions r in [64 kb, 64 kb + 64); r >= M stays zero (the planes are zero-
// filled on allocation and never written there).
struct DeltaGeom {
    int nkb = 0, nrb = 0;
    size_t plane = 0;  // 16-bit elements per plane
};
inline DeltaGeom delta_geom(int M, int ntot, int W) {
    DeltaGeom g;
    g.nkb = (M + kTileK - 1) / kTileK;
    g.nrb = 2 * ((W + kTileRows - 1) / kTileRows);  // even: whole 128-walker tiles
    g.plane = (size_t)ntot * g.nrb * g.nkb * kTileElems;
    return g;
}
// FP32 copy of the scaled Delta for the dense LO epilogue: element (walker row
// z, basis function s) of orbital c at [c][z / 128][s / 4][z % 128][s % 4], so that
// the 32 rows of a warp read four consecutive s as 512 contiguous bytes
__host__ __device__ inline size_t dfull_elem(int c, int nrb, int Sd, int z, int s) {
    return ((((size_t)c * nrb + (z >> 7)) * (size_t)(Sd >> 2) + (s >> 2)) * 128 + (z & 127)) * 4 + (s & 3);
}
__device__ inline size_t delta_elem(int z, int c, int r, int nrb, int nkb) {
    return ((size_t)((size_t)c * nrb + (z >> 7)) * nkb + (r >> 6)) * kTileElems +
           sw128_elem(z & 127, r & 63);
}

// ---------------------------------------------------------------------------
// per-spin data
// ---------------------------------------------------------------------------

// Split-precision copy of a row-major FP64 matrix: rows x cols values in four
// planes hi/lo (16-bit floats, FP16 or BF16 by `bf16`), each row scaled by a
// power of two (value = (hi + lo) / scale[row]).  Rows are padded to `ld`
// columns with zeros so every row starts on a 16-byte boundary.
struct SplitMatrix {
    int rows = 0, cols = 0, ld = 0;
    bool bf16 = false;
    DevBuf hi, lo, scale;  // hi/lo: rows x ld 16-bit; scale: rows doubles
    void release() { hi.release(); lo.release(); scale.release(); rows = cols = ld = 0; }
};

struct PairTable {
    int npairs = 0;
    long rows = 0;                     // sum of K over pairs
    std::vector<int> i, j, K;          // host copies
    std::vector<long> off;             // first packed row of each pair
    std::vector<double> sig;           // per pair: s_1, s_2, sum s^2 of Y^[ij]
    DevBuf d_i, d_j, d_K, d_off;       // device copies (int, int, int, long)
    DevBuf d_U, d_V;                   // FP64: rows x M (row k of Ubar^T, row k of Vbar)
    // mixed-precision operands (built lazily for FP16X3 / BF16X3)
    SplitMatrix sU[2], sV[2];          // index 0: FP16, 1: BF16
    DevBuf d_p, d_q;                   // FP64 rows: p = Ubar^T Phi_j, q = Vbar Phi_i
    DevBuf d_e0;                       // FP64 per pair: p . q
    void release() {
        d_i.release(); d_j.release(); d_K.release(); d_off.release();
        d_U.release(); d_V.release();
        for (auto& s : sU) s.release();
        for (auto& s : sV) s.release();
        d_p.release(); d_q.release(); d_e0.release();
        npairs = 0; rows = 0; i.clear(); j.clear(); K.clear(); off.clear(); sig.clear();
    }
};

struct SpinData {
    int N = 0;             // occupied orbitals of this spin
    int col0 = 0;          // first column of this spin inside a packed walker
    double mult = 1.0;     // 2 for a restricted closed shell, else 1
    std::vector<double> h_trial;  // M x N current trial (canonical or localized)
    DevBuf d_trial;        // M x N FP64
    DevBuf d_Lbar;         // X x N x M FP64
    DevBuf d_hbar;         // N x M FP64
    SplitMatrix sLbar[2];  // (X+1) x (N*M) rows gamma (last row hbar); FP16 / BF16
    DevBuf d_J0;           // X doubles: tr(Lbar_g Phi) (trial Coulomb vector)
    double E1_0 = 0.0;     // sum_ir hbar_ir Phi_ri
    PairTable pairs;
    DevBuf oz_trialT, oz_rowexp;   // digit slices of Phi_T^T (tensor-core Theta)
    DevBuf oz_trial_cm;            // Phi_T column-major (N x M, int64 units of 2^-56): coalesced epilogue reads
    int oz_trial_version = -1;
    void release() {
        oz_trialT.release(); oz_rowexp.release(); oz_trial_version = -1;
        d_trial.release(); d_Lbar.release(); d_hbar.release();
        for (auto& s : sLbar) s.release();
        d_J0.release();
        pairs.release();
    }
};

// Walker-independent operands of the split-precision path for one 16-bit
// format.  Orbital index c runs over both spins (alpha first); rows of 16-bit
// planes are padded to r_pad (a multiple of 8) basis functions with zeros.
struct MixedOps {
    bool coul_ready = false, lo_ready = false, bf16 = false;
    bool tf32 = false;         // one plane of TF32-rounded FP32 values (tiles of 32-wide basis blocks)
    int r_pad = 0;
    long kflat = 0;            // ntot * r_pad
    // Coulomb operand: rows g < X are mult_sigma * Lbar^sigma_g, row X is
    // mult_sigma * hbar^sigma, flattened over (c, r)
    DevBuf L_hi, L_lo, L_inv;  // (X+1) x kflat 16-bit; inverse row scale (float)
    DevBuf J0;                 // X doubles: trial Coulomb vector
    double E1_0 = 0.0;         // trial one-body energy
    int nkb = 0;               // 64-wide basis blocks per orbital
    int n_mt = 0;              // 128-row blocks of the Coulomb operand
    DevBuf Lb_hi, Lb_lo;       // Coulomb operand tiles [mt][c][kb]
    // LO operand: rows of Ubar^T and Vbar of both spins, concatenated
    long R = 0;
    DevBuf U_hi, U_lo, V_hi, V_lo;  // R x r_pad 16-bit
    DevBuf row_c;              // R float4 {inv_su, inv_sv, p, q}
    DevBuf pt;                 // weight half-tiles, two per rank chunk: int4 {row0, nvalid | H << 16, ci << 16 | cj, element offset}
    int n_pt = 0;
    int n_pairs = 0;           // pairs over both spins
    DevBuf pair_pt0, pair_npt; // first half-tile and half-tile count per pair (int, both even)
    DevBuf pair_w;             // per pair: 0.5 * mult * (1 or 2) (double)
    DevBuf e0;                 // per pair: trial value p . q (double)
    double EK0 = 0.0;          // 1/2 sum_sigma mult sum_n wgt_n e0_n
    DevBuf Ub_hi, Ub_lo, Vb_hi, Vb_lo;  // LO weight half-tiles (H rows x 64 per basis block)
    // host copies of the unscreened tile list, and the screened list
    std::vector<int4> h_tiles;
    std::vector<int> h_pt0, h_npt, h_order;
    std::vector<double> h_pw, h_e0;
    DevBuf s_pt, s_pt0, s_npt, s_pw;
    int s_n_pt = 0, screen_built = -1;
    double s_EK0 = 0.0;
    // rank-adaptive plan (mode LO): pairs whose dense truncated block Ytil =
    // Ubar Vbar costs fewer MMA columns than the two factor sides are contracted
    // densely; their half-tiles (B rows: Ytil rows s, then g = Vbar^T p) come
    // first in pair_pt0.  lo_dense_ok records which plan the LO operands hold.
    bool lo_dense_ok = false;
    int chunk_cap = 0;         // largest chunk (MMA N) the LO operands were cut with
    int n_dpt = 0;             // dense half-tiles
    int Sd = 0;                // s-extent of the FP32 Delta copy the dense kernel reads
    DevBuf dpt, Yb_hi, Yb_lo;  // dense half-tile list {row0, nvalid | H << 16, ci << 24 | cj << 16 | s0, offset}, B tiles
    DevBuf rowc_d;             // per dense row {1 / row scale, h = (Ubar q)[s]} (float2)
    std::vector<int4> h_dtiles;
    std::vector<unsigned char> h_dense;  // per pair: contracted densely
    DevBuf s_dpt;
    int s_n_dpt = 0;
    // compressed Coulomb (closed shell): the same tiles with the pair's
    // orbitals swapped, row constants {inv_su, inv_sv, U.Phi_i, V.Phi_j},
    // per-pair trial parts, weights 2 (1 or 2) and their trial sum
    DevBuf pt_J, row_cJ, e0_J, pw_J;
    double EJ0 = 0.0;
    // propagator operator: L^T tiles [mt][kb] (rows pq, per-row scale)
    bool prop_ready = false;
    int prop_nkb = 0, prop_nmt = 0;
    DevBuf Lt_hi, Lt_lo, Lt_inv;
    void release() {
        for (DevBuf* b : {&L_hi, &L_lo, &L_inv, &J0, &U_hi, &U_lo, &V_hi, &V_lo, &row_c, &pt,
                          &pair_pt0, &pair_npt, &pair_w, &e0, &s_pt, &s_pt0, &s_npt, &s_pw,
                          &Lb_hi, &Lb_lo, &Ub_hi, &Ub_lo, &Vb_hi, &Vb_lo, &pt_J, &row_cJ, &e0_J, &pw_J,
                          &Lt_hi, &Lt_lo, &Lt_inv, &dpt, &Yb_hi, &Yb_lo, &rowc_d, &s_dpt})
            b->release();
        coul_ready = lo_ready = prop_ready = false;
        screen_built = -1;
        h_tiles.clear(); h_pt0.clear(); h_npt.clear(); h_order.clear(); h_pw.clear(); h_e0.clear();
        h_dtiles.clear(); h_dense.clear();
        n_pt = n_dpt = n_pairs = s_n_pt = s_n_dpt = 0;
        Sd = 0;
        R = 0;
    }
};

}  // namespace loaf

// ---------------------------------------------------------------------------
// the context
// ---------------------------------------------------------------------------

struct loaf_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // host walker arrays are uploaded in chunks while the previous chunk
    // computes, each chunk as two copies on two streams (two copy engines move
    // about 55 GB/s over the host link where one moves 51; created on first use)
    cudaStream_t copy_stream[2] = {nullptr, nullptr};
    cudaEvent_t ev_start = nullptr, ev_copied[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}},
                ev_free[2] = {nullptr, nullptr};
    cublasHandle_t cublas = nullptr;
    cusolverDnHandle_t cusolver = nullptr;
    int sm_count = 0;
    // SMs the persistent tensor-core kernels of this context may fill (0: all);
    // set by the multi-system launch so that several systems share the GPU
    int grid_cap = 0;
    // tile shapes of the tensor-core kernels (loaf_set_tiles; the multi-system
    // autotuner sets them per context): the largest LO chunk, i.e. the MMA's N
    // (a multiple of 32 in [64, 256]), and the Coulomb k-split (0: the rule that
    // fills the last round of the persistent grid)
    int tile_lo_cap = 256;
    int tile_coul_split = 0;
    int tile_version = 0;  // bumped whenever the tile shapes change
    int persistent_grid() const { return grid_cap > 0 ? std::min(grid_cap, sm_count) : sm_count; }
    // walkers_energy_submit: two call slots used in turn, each with its own
    // device copy of the walkers, device results and pinned flags, so that one
    // call's upload runs on the copy streams while the previous call computes
    struct AsyncSlot {
        loaf::DevBuf phi, out;
        int* h_flags = nullptr;  // [worst walker status, timeout], pinned host memory
        cudaEvent_t done = nullptr;
        bool pending = false;    // submitted and not yet harvested
    };
    AsyncSlot aslot[2];
    int aslot_next = 0;
    long long async_key = -1;         // (W, mode, precision) of the calls the workspace is sized for
    int async_flags[2] = {0, 0};      // harvested flags of the calls not yet waited for
    // multi-system launches: a private branch stream, fork/join events, pinned flags
    cudaStream_t branch_stream = nullptr;
    cudaEvent_t ev_join = nullptr;
    int* h_flags = nullptr;

    bool loaded = false;
    bool compressed = false;
    bool localized = false;
    double t_svd = 0.0;
    int M = 0, X = 0, na = 0, nb = 0, nspin = 0, ntot = 0;
    bool closed = false;
    double e0 = 0.0;
    double trial_E_J = 0.0;  // walker-independent parts (mixed mode)
    loaf::DevBuf d_h, d_L;
    loaf::SpinData sp[2];
    std::vector<double> canonical[2];  // trial orbitals as loaded (host)
    loaf::MixedOps mix[3];             // tensor-core operands: [0] FP16, [1] BF16, [2] TF32

    // learned pair screen
    std::vector<double> features;      // 8 descriptors per pair (spins concatenated)
    std::vector<unsigned char> keep;   // 1 = evaluate the pair; empty = no screen
    int screen_version = 0;            // bumped whenever keep changes
    std::vector<float> mlp_params;     // trained network (FP32 master copy)
    std::vector<double> mlp_target;    // training targets (log10 max |e_ij|)
    std::vector<double> mlp_pred;      // predicted log10 |e_ij| of every pair
    loaf::DevBuf d_keep;               // device copy of keep
    int d_keep_version = -1;
    double feat_mu[8] = {0}, feat_sd[8] = {1, 1, 1, 1, 1, 1, 1, 1}, tgt_mu = 0.0, tgt_sd = 1.0;

    loaf::DevBuf w_cas;                // multi-determinant (CAS) energy workspace
    // workspace for walkers_energy (grown to the largest W seen)
    int ws_W = 0;
    loaf::DevBuf w_phi, w_theta, w_z, w_lu, w_perm, w_logdet, w_status, w_out, w_part,
        w_part2, w_dhi, w_dlo, w_dscale, w_host_stage, w_cpart, w_lopart, w_red, w_flag, w_oz_at,
        w_oz_bt, w_oz_S, w_oz_int, w_oz_key, w_prop_x, w_prop_part;
    // FP32 copy of the scaled Delta for the dense LO epilogue (dfull_elem layout);
    // zeroed whenever its geometry changes (the columns past M stay zero)
    loaf::DevBuf w_dfull;
    long dfull_key = -1;
    loaf::DevBuf w_dtf;  // TF32 precision: Delta tiles [c][rb][32-wide block] of FP32 (from w_dfull)
    int trial_version = 0;  // bumped whenever a trial (canonical or localized) is loaded
    int test_withhold = 0;  // LO kernel launches left that withhold a stage (failure-path tests)

    // per-stage CUDA-event timers (loaf_profile); stage kernels are bracketed
    // by events on the context stream while enabled
    struct ProfStage { std::string name; double total_ms = 0.0; long calls = 0; long launches = 0; };
    struct ProfMark { int stage; cudaEvent_t a, b; int launches; };
    bool prof_on = false;
    std::vector<ProfStage> prof;
    std::vector<ProfMark> prof_open;
    std::vector<cudaEvent_t> prof_pool;

    std::string err;
};

namespace loaf {
// Brackets the kernels of one named stage with events on the context stream
// (no-op while profiling is off).  Elapsed times are collected by
// prof_collect() once the stream has been synchronized.
struct StageScope {
    loaf_ctx* c;
    int idx = -1;
    cudaEvent_t a = nullptr, b = nullptr;
    int launches;
    StageScope(loaf_ctx* ctx, const char* name, int nlaunch = 1);
    void end();  // record the closing event now (idempotent)
    ~StageScope() { end(); }
};
void prof_collect(loaf_ctx* c);
// Waits for the calls queued by walkers_energy_submit, keeping their walker
// and timeout flags for walkers_energy_wait; entry points that change the
// context's operands, tile shapes or screen call it first, so that no queued
// call computes with operands rewritten under it.
void drain_submitted(loaf_ctx* c);
}  // namespace loaf

namespace loaf {

// complex helpers on double2
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ inline double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm keeps the intermediate in range
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.x * r + b.y;
        return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// operand set of a tensor-core precision: 0 FP16 hi/lo, 1 BF16 hi/lo, 2 TF32
inline int mix_slot(int precision) {
    return precision == LOAF_PREC_BF16X3 ? 1 : (precision == LOAF_PREC_TF32 ? 2 : 0);
}

// kernels and host stages (defined in the .cu files)
void run_theta_fp64(loaf_ctx* c, int W, const double2* phi, double2* theta, double2* logdet,
                    int* status);
void run_energy_fp64_full(loaf_ctx* c, int W, const double2* theta, double2* e_out);
void run_energy_fp64_lo(loaf_ctx* c, int W, const double2* theta, double2* e_out,
                        double2* e_pairs);
void run_coulomb_fp64(loaf_ctx* c, int W, const double2* theta, double2* e_part);
// E_J from the compressed pair factors (closed shell): 2 sum_ij (Ubar^T Theta_i).(Vbar Theta_j)
void run_coulomb_lo_fp64(loaf_ctx* c, int W, const double2* theta, double2* ej_out, double2* scratch);
// part[row][col] = sum_k A[row][k] B[col][k] over 16-bit hi/lo tiles (A tiles
// [mt][kb], B tiles [rb][kb], 128 x 64 each, three products, 128-term chains
// folded in double-float), FP64 out, rows x (n_wt * 128) with leading dim ldp;
// with out set, columns (2w, 2w + 1) go to out[w][row] as one complex value,
// scaled by inv_row[row] * inv_col[col] (w < out_W, leading dim out_ld)
void tc_split_gemm(loaf_ctx* c, const uint16_t* a_hi, const uint16_t* a_lo, int rows, int n_mt,
                   const uint16_t* b_hi, const uint16_t* b_lo, int nrb, int n_wt, int nkb, bool bf16,
                   double* part, int ldp, int* err, double2* out, const float* inv_row,
                   const float* inv_col, long out_ld, int out_W);
// V_w = sum_g x_wg L_g for W walkers (x: W x X, V: W x M x M, device)
void run_propagator(loaf_ctx* c, int W, const double2* x, int precision, double2* V);
// multi-determinant (CAS) trial: argument checks (host) and the FP64 energy
void cas_check_dets(int N, int Nc, int n_det, const int* dets);
void run_energy_cas(loaf_ctx* c, int W, int N, const double2* phi, int n_det, const int* h_dets,
                    const double* h_coeffs, double2* e_dev, double2* logov_dev, int* status_dev);
// <L_g>_w of the batch whose Delta tiles the tensor-core Theta stage wrote
void run_force_bias_mixed(loaf_ctx* c, int W, int precision, double2* e_scratch, double2* j_out);
void run_energy_mixed(loaf_ctx* c, int W, int mode, int precision, const double2* theta,
                      double2* e_out, double2* e_pairs);
// Sd > 0: also write the FP32 copy of the scaled Delta (s-extent Sd) for the
// dense LO kernel
void run_theta_tc(loaf_ctx* c, int W, const double2* phi, int precision, int Sd = 0);
// LO operands of the mode (LO: rank-adaptive, LO_JK: factored); returns the
// s-extent of the FP32 Delta copy the dense kernel reads (0: no dense pair)
int prepare_lo_operands(loaf_ctx* c, int mode, int precision);
int coulomb_split_rule(loaf_ctx* c, int W, int precision);
void setup_load(loaf_ctx* c, int M, int X, const double* h, const double* L, int na, int nb,
                const double* ta, const double* tb, double e0, int on_device);
void setup_compress(loaf_ctx* c, double t_svd, const double* r_ops, int n_ops, int localize,
                    double* pct, int* m_svd);
void setup_mixed_operands(loaf_ctx* c, int mode, bool bf16);
void half_rotate(loaf_ctx* c, SpinData& s);

}  // namespace loaf
