// Split-precision tensor-core path (LOAF_PREC_FP16X3 / LOAF_PREC_BF16X3).
//
// Trial-delta form.  Theta = Phi_T + Delta with Phi_T^T Delta = 0 (eq. Q with
// Phi_T^T Phi_T = 1).  Every walker-independent product with Phi_T is taken
// once in FP64 (J0, E1_0, the pair vectors p = Ubar^T Phi_j, q = Vbar Phi_i and
// their dot products e0); only the products with Delta, which is an order of
// magnitude smaller than Theta, go through the 16-bit tensor cores:
//   x = (x_hi + x_lo) / scale,  x_hi = rn16(x * scale), x_lo = rn16(x * scale - x_hi)
//   A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi   (tcgen05.mma kind::f16, FP32 accumulate)
// with power-of-two scales per operand row (weights) and per walker (Delta).
//
// Kernels (sm_103a, persistent, warp-specialised: one thread of warp 0 issues
// the bulk copies, one of warp 1 the tcgen05.mma, 16 epilogue warps drain TMEM):
//   coulomb_tc_pair_kernel  dJ[g][w] = sum_(c,r) Lbar'[g][c][r] Delta[w][c][r]
//                      (rows g < X: Cholesky vectors, row X: hbar -> dE1) on CTA
//                      pairs (cta_group::2, M = 256 rows g, N = 64 walkers x
//                      re/im): 128-term TMEM chains folded into double-float,
//                      FP64 partials per split of the contraction.
//   coulomb_tc_kernel  the same contraction on single CTAs with a direct
//                      walker-major output (the propagator operator).
//   lo_exchange_tc_kernel  per rank chunk of a pair [ij] (at most 256 ranks) and
//                      128 walkers, on CTA pairs (M = 256 Delta rows, N = the
//                      chunk's ranks): a = Delta_j^T Ubar, b = Delta_i^T Vbar in
//                      two TMEM accumulators, then the epilogue forms
//                      p.db + q.da + da.db and sums over the ranks.
// All mbarrier waits are bounded (tc_ptx.cuh); a timeout raises an error flag
// the host turns into LOAF_ERR_TIMEOUT.
#include "common.cuh"
#include "split16.cuh"
#include "tc_ptx.cuh"


#include <algorithm>
#include <cmath>

namespace loaf {

namespace {

constexpr int kBM = 128;             // MMA rows per CTA
constexpr int kBNW = 128;            // walkers per LO unit (64 per CTA of the pair)
constexpr int kBN = 2 * kBNW;        // LO: Delta rows per unit (walker, re/im) = the largest
                                     // rank chunk = TMEM columns per accumulator


__device__ inline double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

struct SpinRef {
    const double* Lbar;   // X x N x M
    const double* hbar;   // N x M
    const double* trial;  // M x N
    int N, col0;
    double mult;
};

// ---------------------------------------------------------------------------
// setup kernels of the split operands (FP64 in, 16-bit planes out)
// ---------------------------------------------------------------------------

// row g <= X of the Coulomb operand: mult * Lbar_g (g < X) or mult * hbar (g = X)
template <bool BF16>
__global__ void coul_split_kernel(int M, int X, int r_pad, int nspin, SpinRef s0, SpinRef s1,
                                  uint16_t* __restrict__ hi, uint16_t* __restrict__ lo,
                                  float* __restrict__ inv) {
    __shared__ double red[32];
    const int g = blockIdx.x;
    const long kflat = (long)(s0.N + (nspin > 1 ? s1.N : 0)) * r_pad;
    double m = 0.0;
    for (int s = 0; s < nspin; ++s) {
        const SpinRef sp = s == 0 ? s0 : s1;
        const double* src = g < X ? sp.Lbar + (size_t)g * sp.N * M : sp.hbar;
        for (long e = threadIdx.x; e < (long)sp.N * M; e += blockDim.x)
            m = fmax(m, fabs(sp.mult * src[e]));
    }
    const double sc = pow2_scale(block_max(m, red));
    for (int s = 0; s < nspin; ++s) {
        const SpinRef sp = s == 0 ? s0 : s1;
        const double* src = g < X ? sp.Lbar + (size_t)g * sp.N * M : sp.hbar;
        for (long e = threadIdx.x; e < (long)sp.N * r_pad; e += blockDim.x) {
            const int i = (int)(e / r_pad), r = (int)(e % r_pad);
            const double v = r < M ? sp.mult * src[(size_t)i * M + r] * sc : 0.0;
            uint16_t h, l;
            split16<BF16>(v, h, l);
            const size_t o = (size_t)g * kflat + (size_t)(sp.col0 + i) * r_pad + r;
            hi[o] = h;
            lo[o] = l;
        }
    }
    if (threadIdx.x == 0) inv[g] = (float)(1.0 / sc);
}

// FP32 rounded to the nearest TF32 value (10 stored significand bits; ties away
// from zero): the tensor cores read the upper 19 bits of each operand
__device__ inline float tf32_round(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    return __uint_as_float(u);
}

// row g <= X of the Coulomb operand as TF32-rounded FP32 (same rows and scale as
// coul_split_kernel), rows of r_pad32 values per orbital
__global__ void coul_tf32_kernel(int M, int X, int r_pad32, int nspin, SpinRef s0, SpinRef s1,
                                 float* __restrict__ out, float* __restrict__ inv) {
    __shared__ double red[32];
    const int g = blockIdx.x;
    const long kflat = (long)(s0.N + (nspin > 1 ? s1.N : 0)) * r_pad32;
    double m = 0.0;
    for (int s = 0; s < nspin; ++s) {
        const SpinRef sp = s == 0 ? s0 : s1;
        const double* src = g < X ? sp.Lbar + (size_t)g * sp.N * M : sp.hbar;
        for (long e = threadIdx.x; e < (long)sp.N * M; e += blockDim.x)
            m = fmax(m, fabs(sp.mult * src[e]));
    }
    const double sc = pow2_scale(block_max(m, red));
    for (int s = 0; s < nspin; ++s) {
        const SpinRef sp = s == 0 ? s0 : s1;
        const double* src = g < X ? sp.Lbar + (size_t)g * sp.N * M : sp.hbar;
        for (long e = threadIdx.x; e < (long)sp.N * r_pad32; e += blockDim.x) {
            const int i = (int)(e / r_pad32), r = (int)(e % r_pad32);
            const double v = r < M ? sp.mult * src[(size_t)i * M + r] * sc : 0.0;
            out[(size_t)g * kflat + (size_t)(sp.col0 + i) * r_pad32 + r] = tf32_round((float)v);
        }
    }
    if (threadIdx.x == 0) inv[g] = (float)(1.0 / sc);
}

// J0[g] = sum_sigma mult sum_ir Lbar_gir Phi_ri (g < X); E1_0 at g = X (FP64)
__global__ void trial_coulomb_kernel(int M, int X, int nspin, SpinRef s0, SpinRef s1,
                                     double* __restrict__ J0) {
    __shared__ double red[32];
    const int g = blockIdx.x;
    double acc = 0.0;
    for (int s = 0; s < nspin; ++s) {
        const SpinRef sp = s == 0 ? s0 : s1;
        const double* src = g < X ? sp.Lbar + (size_t)g * sp.N * M : sp.hbar;
        double a = 0.0;
        for (long e = threadIdx.x; e < (long)sp.N * M; e += blockDim.x) {
            const int i = (int)(e / M), r = (int)(e % M);
            a += src[e] * sp.trial[(size_t)r * sp.N + i];
        }
        acc += sp.mult * a;
    }
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) J0[g] = t;
}

// one packed factor row (Ubar^T or Vbar) -> 16-bit planes, inverse scale
template <bool BF16>
__global__ void row_split_kernel(int M, int r_pad, const double* __restrict__ src,
                                 uint16_t* __restrict__ hi, uint16_t* __restrict__ lo,
                                 float* __restrict__ inv) {
    __shared__ double red[32];
    const long row = blockIdx.x;
    const double* s = src + row * M;
    double m = 0.0;
    for (int r = threadIdx.x; r < M; r += blockDim.x) m = fmax(m, fabs(s[r]));
    const double sc = pow2_scale(block_max(m, red));
    for (int r = threadIdx.x; r < r_pad; r += blockDim.x) {
        uint16_t h, l;
        split16<BF16>(r < M ? s[r] * sc : 0.0, h, l);
        hi[row * r_pad + r] = h;
        lo[row * r_pad + r] = l;
    }
    if (threadIdx.x == 0) inv[row] = (float)(1.0 / sc);
}

// One 128 x 64 operand tile from a row-major 16-bit plane (rows `ld` apart):
// rows [row0, row0 + nvalid), columns [col0, col0 + kvalid) (kvalid a multiple
// of 8), zero elsewhere, written as the swizzled shared-memory image.
__device__ void write_tile(const uint16_t* __restrict__ src, long ld, long row0, int nvalid,
                           long col0, int kvalid, uint16_t* __restrict__ dst) {
    for (int q = threadIdx.x; q < kTileRows * 8; q += blockDim.x) {
        const int row = q >> 3, j = q & 7;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row < nvalid && j * 8 < kvalid)
            v = *reinterpret_cast<const uint4*>(src + (row0 + row) * ld + col0 + j * 8);
        *reinterpret_cast<uint4*>(dst + sw128_elem(row, j * 8)) = v;
    }
}

// LO weight half-tiles: list entry t = {row0, nvalid | H << 16, -, element offset};
// its basis block kb holds H rows x 64 (swizzled image of H rows) at
// offset + kb H 64, rows [row0, row0 + nvalid) of the plane, zero elsewhere
__global__ void lo_tiles_kernel(const uint16_t* __restrict__ plane, int r_pad, int nkb,
                                const int4* __restrict__ tiles, uint16_t* __restrict__ out) {
    const int4 t = tiles[blockIdx.x];
    const int kb = blockIdx.y;
    const int nvalid = t.y & 0xffff, H = t.y >> 16;
    const long col0 = (long)kb * kTileK;
    const int kvalid = r_pad - kb * kTileK;
    uint16_t* dst = out + (size_t)(unsigned)t.w + (size_t)kb * H * kTileK;
    for (int q = threadIdx.x; q < H * 8; q += blockDim.x) {
        const int row = q >> 3, j = q & 7;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row < nvalid && j * 8 < kvalid)
            v = *reinterpret_cast<const uint4*>(plane + ((long)t.x + row) * r_pad + col0 + j * 8);
        *reinterpret_cast<uint4*>(dst + sw128_elem(row, j * 8)) = v;
    }
}

// Coulomb operand tiles [mt][c][kb] from the (X+1) x (ntot r_pad) plane
__global__ void coul_tiles_kernel(const uint16_t* __restrict__ plane, int rows, int ntot, int r_pad,
                                  int nkb, uint16_t* __restrict__ out) {
    const int mt = blockIdx.x / ntot, c = blockIdx.x % ntot, kb = blockIdx.y;
    const long ld = (long)ntot * r_pad;
    write_tile(plane, ld, (long)mt * kTileRows, min(kTileRows, rows - mt * kTileRows),
               (long)c * r_pad + (long)kb * kTileK, r_pad - kb * kTileK,
               out + (((size_t)mt * ntot + c) * nkb + kb) * kTileElems);
}

// p = Ubar^T row . Phi_j, q = Vbar row . Phi_i (FP64), one warp per row
__global__ void pq_kernel(int M, long rows, const double* __restrict__ U,
                          const double* __restrict__ V, const int* __restrict__ row_pair,
                          const int* __restrict__ pi, const int* __restrict__ pj,
                          const double* __restrict__ trial, int N, double* __restrict__ p_out,
                          double* __restrict__ q_out) {
    const long row = (long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const int n = row_pair[row];
    const int i = pi[n], j = pj[n];
    double p = 0.0, q = 0.0;
    for (int r = lane; r < M; r += 32) {
        p += U[row * M + r] * trial[(size_t)r * N + j];
        q += V[row * M + r] * trial[(size_t)r * N + i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        p += __shfl_xor_sync(0xffffffffu, p, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if (lane == 0) { p_out[row] = p; q_out[row] = q; }
}

__global__ void row_consts_kernel(long rows, const float* __restrict__ inv_u,
                                  const float* __restrict__ inv_v, const double* __restrict__ p,
                                  const double* __restrict__ q, float4* __restrict__ out) {
    const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows) out[r] = make_float4(inv_u[r], inv_v[r], (float)p[r], (float)q[r]);
}

// e0[n] = sum_k p_k q_k over the pair's rows (FP64)
__global__ void pair_e0_kernel(int npairs, const long* __restrict__ off, const int* __restrict__ K,
                               const double* __restrict__ p, const double* __restrict__ q,
                               double* __restrict__ e0) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= npairs) return;
    double s = 0.0;
    for (int k = 0; k < K[n]; ++k) s += p[off[n] + k] * q[off[n] + k];
    e0[n] = s;
}

// ---------------------------------------------------------------------------
// per-call: Delta = Theta - Phi_T -> scaled 16-bit planes
// ---------------------------------------------------------------------------
__global__ void delta_max_kernel(int M, int ntot, int nspin, SpinRef s0, SpinRef s1,
                                 const double2* __restrict__ theta, float* __restrict__ inv_t,
                                 double* __restrict__ scale) {
    __shared__ double red[32];
    const int w = blockIdx.x;
    double m = 0.0;
    for (int s = 0; s < nspin; ++s) {
        const SpinRef sp = s == 0 ? s0 : s1;
        const double2* th = theta + ((size_t)w * ntot + sp.col0) * M;
        for (long e = threadIdx.x; e < (long)sp.N * M; e += blockDim.x) {
            const int i = (int)(e / M), r = (int)(e % M);
            const double2 t = th[e];
            m = fmax(m, fmax(fabs(t.x - sp.trial[(size_t)r * sp.N + i]), fabs(t.y)));
        }
    }
    const double sc = pow2_scale(block_max(m, red));
    if (threadIdx.x == 0) { inv_t[w] = (float)(1.0 / sc); scale[w] = sc; }
}

template <bool BF16>
__global__ void delta_split_kernel(int M, int ntot, int nrb, int nkb, int nspin, SpinRef s0,
                                   SpinRef s1, const double2* __restrict__ theta,
                                   const double* __restrict__ scale, uint16_t* __restrict__ hi,
                                   uint16_t* __restrict__ lo) {
    const int w = blockIdx.x / ntot, c = blockIdx.x % ntot;
    const SpinRef sp = (nspin > 1 && c >= s1.col0) ? s1 : s0;
    const int i = c - sp.col0;
    const double sc = scale[w];
    const double2* th = theta + ((size_t)w * ntot + c) * M;
    for (int r = threadIdx.x; r < M; r += blockDim.x) {
        const double2 t = th[r];
        const double vr = (t.x - sp.trial[(size_t)r * sp.N + i]) * sc;
        const double vi = t.y * sc;
        const size_t o_re = delta_elem(2 * w, c, r, nrb, nkb);
        const size_t o_im = delta_elem(2 * w + 1, c, r, nrb, nkb);
        uint16_t h, l;
        split16<BF16>(vr, h, l);
        hi[o_re] = h;
        lo[o_re] = l;
        split16<BF16>(vi, h, l);
        hi[o_im] = h;
        lo[o_im] = l;
    }
}

// ---------------------------------------------------------------------------
// tensor-core kernels
// ---------------------------------------------------------------------------
__device__ inline uint8_t* align1024(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// ---- Coulomb kernel geometry ----
// The tensor cores accumulate in FP32 with an error that grows with the
// length of the accumulation chain (measured on B300: 0.235 / 0.151 / 0.038 /
// 0.022 mHa in E_J at pentacene scale for 803 / 446 / 111 / 32-term chains).
// Chains are therefore cut at kCGroup k-chunks (128 terms): each group
// accumulates into one of four rotating TMEM buffers, and the epilogue folds
// the finished buffer into a double-float (hi, lo) register accumulator with
// an error-free TwoSum, so the long (c, r) contraction is summed to ~2^-44.
constexpr int kCBN = 128;            // columns: 64 walkers, re/im interleaved
constexpr int kCStages = 2;
constexpr int kCGroup = 2;           // 64-wide k-chunks per TMEM accumulation chain
constexpr int kCBufs = 4;            // TMEM buffers of kCBN columns
constexpr int kCEpiWarps = 16;       // 4 per TMEM lane quarter, 32 columns each
constexpr int kCThreads = 64 + 32 * kCEpiWarps;

struct CoulShared {
    uint64_t full[kCStages];
    uint64_t empty[kCStages];
    uint64_t acc_full[kCBufs];
    uint64_t acc_empty[kCBufs];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

struct CoulParams {
    const uint16_t* a_hi;  // operand tiles [mt][c][kb]
    const uint16_t* a_lo;
    const uint16_t* b_hi;  // Delta tiles [c][rb][kb]
    const uint16_t* b_lo;
    double* part;      // [split][rows][ldp] FP64 partial sums
    // optional direct output instead of part (one split): out[w][row] =
    // (col 2w, col 2w + 1) * inv_row[row] * (inv_col[2w], inv_col[2w + 1])
    double2* out;
    const float* inv_row;
    const float* inv_col;
    long out_ld;
    int out_W;
    // unit order: row tiles fastest (the column operand is the large one, as
    // for the Coulomb energy) or column tiles fastest (the row operand is)
    int wt_fast;
    int rows;          // X + 1
    int n_mt, n_wt, n_split, nk, ldp;
    int nkb, nrb;      // basis blocks per orbital, Delta row blocks
    uint32_t idesc;
    int* err;
};

// the FP64 value of a float from its bit pattern with integer operations only
// (the conversion instruction runs on the FP64 pipe, 1/64 of the FP32 rate);
// exact for normal floats and infinities, 0 for zero and subnormal floats
__device__ __forceinline__ double f2d_bits(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long ex = e == 0xffu ? 0x7ffull : (unsigned long long)(e + (1023u - 127u));
    const unsigned long long bits = ((unsigned long long)(b >> 31) << 63) | (ex << 52) |
                                    ((unsigned long long)(b & 0x7fffffu) << 29);
    return e == 0 ? 0.0 : __longlong_as_double((long long)bits);
}

// two columns at once: the same operations on the two lanes of sm_100 FP32x2
// instructions (the _rn forms are never contracted)
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void two_sum_acc2(float2& hi, float2& lo, float2 x) {
    const float2 s = __fadd2_rn(hi, x);
    const float2 bp = __fadd2_rn(s, neg2(hi));
    const float2 e = __fadd2_rn(__fadd2_rn(hi, neg2(__fadd2_rn(s, neg2(bp)))), __fadd2_rn(x, neg2(bp)));
    hi = s;
    lo = __fadd2_rn(lo, e);
}
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += e;
}

// dJ partial tile: rows g (128) x 128 columns (64 walkers, re/im) over the
// k-chunks [split * nk / n_split, (split+1) * nk / n_split)
__global__ void __launch_bounds__(kCThreads, 1)
coulomb_tc_kernel(CoulParams P) {
    extern __shared__ uint8_t dyn_smem[];
    __shared__ CoulShared sh;
    uint8_t* base = align1024(dyn_smem);
    constexpr uint32_t kStageBytes = 4 * kTileBytes;  // A hi, A lo, B hi, B lo: 64 KB
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_units = P.n_mt * P.n_wt * P.n_split;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kCStages; ++s) { tc::mbar_init(&sh.full[s], 1); tc::mbar_init(&sh.empty[s], 1); }
        for (int b = 0; b < kCBufs; ++b) { tc::mbar_init(&sh.acc_full[b], 1); tc::mbar_init(&sh.acc_empty[b], kCEpiWarps); }
        tc::mbar_init(&sh.drain, 1);
        sh.abort = 0;
        tc::fence_barrier_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&sh.tmem_base, kCBufs * kCBN);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = sh.tmem_base;
    volatile int* abort = &sh.abort;

    if (warp == 0 && lane == 0) {
        // ---------------- bulk-copy producer ----------------
        int s = 0;
        uint32_t ph = 0, filled = 0, last_par = 0;
        for (int u = blockIdx.x; u < n_units && !*abort; u += gridDim.x) {
            const int mt = P.wt_fast ? (u / P.n_wt) % P.n_mt : u % P.n_mt,
                      wt = P.wt_fast ? u % P.n_wt : (u / P.n_mt) % P.n_wt, sp = u / (P.n_mt * P.n_wt);
            const int k0 = (int)((long)sp * P.nk / P.n_split), k1 = (int)((long)(sp + 1) * P.nk / P.n_split);
            for (int kc = k0; kc < k1; ++kc) {
                if (!tc::mbar_wait(&sh.empty[s], ph ^ 1, abort)) break;
                uint8_t* st = base + s * kStageBytes;
                tc::mbar_arrive_expect_tx(&sh.full[s], kStageBytes);
                const int cc = kc / P.nkb, kb = kc - cc * P.nkb;
                const size_t ao = ((size_t)mt * P.nk + kc) * kTileElems;
                const size_t bo = (((size_t)cc * P.nrb + wt) * P.nkb + kb) * kTileElems;
                tc::bulk_load(st, P.a_hi + ao, kTileBytes, &sh.full[s]);
                tc::bulk_load(st + kTileBytes, P.a_lo + ao, kTileBytes, &sh.full[s]);
                tc::bulk_load(st + 2 * kTileBytes, P.b_hi + bo, kTileBytes, &sh.full[s]);
                tc::bulk_load(st + 3 * kTileBytes, P.b_lo + bo, kTileBytes, &sh.full[s]);
                filled |= 1u << s;
                last_par = (last_par & ~(1u << s)) | (ph << s);
                if (++s == kCStages) { s = 0; ph ^= 1; }
            }
        }
        // drain: every stage ever filled must have landed before the CTA exits
        if (*abort) {
            for (int q = 0; q < kCStages; ++q)
                if (filled & (1u << q)) {
                    volatile int never = 0;
                    tc::mbar_wait(&sh.full[q], (last_par >> q) & 1, &never);
                }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        int s = 0;
        uint32_t ph = 0, gcount = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < n_units && ok && !*abort; u += gridDim.x) {
            const int sp = u / (P.n_mt * P.n_wt);
            const int k0 = (int)((long)sp * P.nk / P.n_split), k1 = (int)((long)(sp + 1) * P.nk / P.n_split);
            for (int g0 = k0; g0 < k1 && ok; g0 += kCGroup, ++gcount) {
                const uint32_t b = gcount % kCBufs, use = gcount / kCBufs;
                if (!tc::mbar_wait(&sh.acc_empty[b], (use & 1) ^ 1, abort)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t d = tmem + b * kCBN;
                const int g1 = min(g0 + kCGroup, k1);
                for (int kc = g0; kc < g1; ++kc) {
                    if (!tc::mbar_wait(&sh.full[s], ph, abort)) { ok = false; break; }
                    tc::tc_fence_after();
                    const uint32_t st = tc::smem_u32(base + s * kStageBytes);
#pragma unroll
                    for (int kk = 0; kk < kTileK / 16; ++kk) {
                        const uint32_t off = kk * 32;
                        const uint64_t ahi = tc::smem_desc(st + off, 128);
                        const uint64_t alo = tc::smem_desc(st + kTileBytes + off, 128);
                        const uint64_t bhi = tc::smem_desc(st + 2 * kTileBytes + off, 128);
                        const uint64_t blo = tc::smem_desc(st + 3 * kTileBytes + off, 128);
                        const uint32_t acc = (kc > g0 || kk > 0) ? 1u : 0u;
                        tc::mma_f16(d, ahi, bhi, P.idesc, acc);
                        tc::mma_f16(d, ahi, blo, P.idesc, 1u);
                        tc::mma_f16(d, alo, bhi, P.idesc, 1u);
                    }
                    tc::mma_commit(&sh.empty[s]);
                    if (++s == kCStages) { s = 0; ph ^= 1; }
                }
                if (!ok) break;
                tc::mma_commit(&sh.acc_full[b]);
            }
        }
        tc::mma_commit(&sh.drain);
        volatile int never = 0;
        tc::mbar_wait(&sh.drain, 0, &never);
    } else if (warp >= 2) {
        // ---------------- epilogue: TMEM groups -> double-float -> FP64 ----------------
        const int q = warp & 3;          // TMEM lane quarter this warp may access
        const int h = (warp - 2) >> 2;   // column block: 32 columns per warp
        uint32_t gcount = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < n_units && ok && !*abort; u += gridDim.x) {
            const int mt = P.wt_fast ? (u / P.n_wt) % P.n_mt : u % P.n_mt,
                      wt = P.wt_fast ? u % P.n_wt : (u / P.n_mt) % P.n_wt, sp = u / (P.n_mt * P.n_wt);
            const int k0 = (int)((long)sp * P.nk / P.n_split), k1 = (int)((long)(sp + 1) * P.nk / P.n_split);
            // hi in registers, lo in shared memory ([column][epilogue thread])
            float hi[32];
            float* lo = reinterpret_cast<float*>(base + kCStages * kStageBytes) + (threadIdx.x - 64);
#pragma unroll
            for (int k = 0; k < 32; ++k) { hi[k] = 0.f; lo[k * kCEpiWarps * 32] = 0.f; }
            for (int g0 = k0; g0 < k1; g0 += kCGroup, ++gcount) {
                const uint32_t b = gcount % kCBufs, use = gcount / kCBufs;
                if (!tc::mbar_wait(&sh.acc_full[b], use & 1, abort)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + b * kCBN + h * 32;
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    float v[16];
                    tc::tmem_ld16(taddr + part * 16, v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        two_sum_acc(hi[part * 16 + k], lo[(part * 16 + k) * kCEpiWarps * 32], v[k]);
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&sh.acc_empty[b]);
            }
            if (!ok) break;
            const int g = mt * kBM + q * 32 + lane;
            if (P.out) {
                // columns (2w, 2w + 1) are walker w's real and imaginary part: a warp
                // writes 32 consecutive rows of one walker (512 contiguous bytes)
                if (g < P.rows) {
                    const double ir = (double)P.inv_row[g];
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int w = wt * (kCBN / 2) + h * 16 + k;
                        if (w < P.out_W)
                            P.out[(size_t)w * P.out_ld + g] = make_double2(
                                ((double)hi[2 * k] + (double)lo[(2 * k) * kCEpiWarps * 32]) * ir *
                                    (double)P.inv_col[2 * w],
                                ((double)hi[2 * k + 1] + (double)lo[(2 * k + 1) * kCEpiWarps * 32]) * ir *
                                    (double)P.inv_col[2 * w + 1]);
                    }
                }
            } else if (g < P.rows) {
                double2* dst = reinterpret_cast<double2*>(
                    P.part + ((size_t)sp * P.rows + g) * P.ldp + (size_t)wt * kCBN + h * 32);
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    dst[k] = make_double2(f2d_bits(hi[2 * k]) + f2d_bits(lo[(2 * k) * kCEpiWarps * 32]),
                                          f2d_bits(hi[2 * k + 1]) +
                                              f2d_bits(lo[(2 * k + 1) * kCEpiWarps * 32]));
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, kCBufs * kCBN);
    if (threadIdx.x == 0 && sh.abort) atomicExch(P.err, 1);
}

// ---- Coulomb on CTA pairs ----
// The same contraction with a cta_group::2 MMA of M = 256 (row tiles 2m and
// 2m + 1: one per CTA) and N = 128: each CTA stages its own 128 operand rows
// and half of the 128 Delta rows (the first or second 8 KB of a Delta tile,
// itself a 64-row swizzled image), 48 KB per k-chunk instead of 64 KB, so
// three k-chunks are in flight per SM.  TMEM per CTA and the epilogue are
// those of coulomb_tc_kernel.  The row tiles are padded to an even count
// (a zero tile).
constexpr int kCPStages = 3;
constexpr uint32_t kCPStageBytes = 2 * kTileBytes + kTileBytes;  // A hi, A lo, B hi half, B lo half

struct CoulPairShared {
    uint64_t full[kCPStages];       // even CTA: own bytes + the odd CTA's forward
    uint64_t empty[kCPStages];      // both: the pair MMA's commit (multicast)
    uint64_t acc_full[kCBufs];      // both: the pair MMA's commit (multicast)
    uint64_t acc_empty[kCBufs];     // even CTA: 16 local + 16 remote epilogue warps
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

// units (row-tile pair, walker tile, split), row-tile pairs fastest; P.n_mt is
// the padded (even) row-tile count
// TF32: operands are one plane of FP32 values read as TF32 (tiles of 128 rows x
// 32 values, the same 16 KB swizzled image), one product per k-step, and a
// chain of four 32-wide k-chunks keeps 128 terms.
template <bool TF32>
__global__ void __launch_bounds__(kCThreads, 1)
coulomb_tc_pair_kernel(CoulParams P) {
    constexpr int kGroup = TF32 ? 2 * kCGroup : kCGroup;
    constexpr uint32_t kStageTx = TF32 ? kTileBytes + kTileBytes / 2 : kCPStageBytes;
    extern __shared__ uint8_t dyn_smem[];
    __shared__ CoulPairShared sh;
    uint8_t* base = align1024(dyn_smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = tc::cluster_ctarank();
    const bool even = rank == 0;
    const int cid = blockIdx.x >> 1, n_cl = gridDim.x >> 1;
    const int n_mp = P.n_mt >> 1;
    const int n_units = n_mp * P.n_wt * P.n_split;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kCPStages; ++s) {
            tc::mbar_init(&sh.full[s], even ? 2 : 1);
            tc::mbar_init(&sh.empty[s], 1);
        }
        for (int b = 0; b < kCBufs; ++b) {
            tc::mbar_init(&sh.acc_full[b], 1);
            tc::mbar_init(&sh.acc_empty[b], 2 * kCEpiWarps);
        }
        tc::mbar_init(&sh.drain, 1);
        sh.abort = 0;
        tc::fence_barrier_init();
    }
    if (warp == 0) {
        tc::tmem_alloc_pair(&sh.tmem_base, kCBufs * kCBN);
        tc::tmem_relinquish_pair();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::cluster_sync();  // both CTAs' barriers initialised before any remote arrive
    tc::tc_fence_after();
    const uint32_t tmem = sh.tmem_base;
    volatile int* abort = &sh.abort;

    if (warp == 0 && lane == 0) {
        // ---------------- bulk-copy producer (both CTAs) ----------------
        int s = 0;
        uint32_t ph = 0, filled = 0, last_par = 0;
        for (int u = cid; u < n_units && !*abort; u += n_cl) {
            const int mp = u % n_mp, wt = (u / n_mp) % P.n_wt, sp = u / (n_mp * P.n_wt);
            const int mt = 2 * mp + (int)rank;
            const int k0 = (int)((long)sp * P.nk / P.n_split), k1 = (int)((long)(sp + 1) * P.nk / P.n_split);
            for (int kc = k0; kc < k1; ++kc) {
                if (!tc::mbar_wait_cluster(&sh.empty[s], ph ^ 1, abort)) break;
                uint8_t* st = base + s * kCPStageBytes;
                tc::mbar_arrive_expect_tx(&sh.full[s], kStageTx);
                const int cc = kc / P.nkb, kb = kc - cc * P.nkb;
                const size_t ao = ((size_t)mt * P.nk + kc) * kTileElems;
                const size_t bo = (((size_t)cc * P.nrb + wt) * P.nkb + kb) * kTileElems + rank * (kTileElems / 2);
                tc::bulk_load(st, P.a_hi + ao, kTileBytes, &sh.full[s]);
                if (!TF32) tc::bulk_load(st + kTileBytes, P.a_lo + ao, kTileBytes, &sh.full[s]);
                tc::bulk_load(st + 2 * kTileBytes, P.b_hi + bo, kTileBytes / 2, &sh.full[s]);
                if (!TF32)
                    tc::bulk_load(st + 2 * kTileBytes + kTileBytes / 2, P.b_lo + bo, kTileBytes / 2, &sh.full[s]);
                filled |= 1u << s;
                last_par = (last_par & ~(1u << s)) | (ph << s);
                if (++s == kCPStages) { s = 0; ph ^= 1; }
            }
        }
        if (*abort) {
            // every copy issued has landed once its phase completes; bounded waits
            for (int q = 0; q < kCPStages; ++q)
                if (filled & (1u << q)) {
                    volatile int never = 0;
                    if (even)
                        tc::mbar_wait_cluster(&sh.full[q], (last_par >> q) & 1, &never);
                    else
                        tc::mbar_wait(&sh.full[q], (last_par >> q) & 1, &never);
                }
        }
    } else if (warp == 1 && lane == 0 && !even) {
        // ---------------- forwarder (odd CTA) ----------------
        const uint32_t peer_full0 = tc::mapa_shared(&sh.full[0], 0);
        int s = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int u = cid; u < n_units && ok && !*abort; u += n_cl) {
            const int sp = u / (n_mp * P.n_wt);
            const int k0 = (int)((long)sp * P.nk / P.n_split), k1 = (int)((long)(sp + 1) * P.nk / P.n_split);
            for (int kc = k0; kc < k1; ++kc) {
                if (!tc::mbar_wait(&sh.full[s], ph, abort)) { ok = false; break; }
                tc::mbar_arrive_remote(peer_full0 + s * (uint32_t)sizeof(uint64_t));
                if (++s == kCPStages) { s = 0; ph ^= 1; }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- pair MMA issuer (even CTA) ----------------
        int s = 0;
        uint32_t ph = 0, gcount = 0;
        bool ok = true;
        for (int u = cid; u < n_units && ok && !*abort; u += n_cl) {
            const int sp = u / (n_mp * P.n_wt);
            const int k0 = (int)((long)sp * P.nk / P.n_split), k1 = (int)((long)(sp + 1) * P.nk / P.n_split);
            for (int g0 = k0; g0 < k1 && ok; g0 += kGroup, ++gcount) {
                const uint32_t b = gcount % kCBufs, use = gcount / kCBufs;
                if (!tc::mbar_wait_cluster(&sh.acc_empty[b], (use & 1) ^ 1, abort)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t d = tmem + b * kCBN;
                const int g1 = min(g0 + kGroup, k1);
                for (int kc = g0; kc < g1; ++kc) {
                    if (!tc::mbar_wait_cluster(&sh.full[s], ph, abort)) { ok = false; break; }
                    tc::tc_fence_after();
                    const uint32_t st = tc::smem_u32(base + s * kCPStageBytes);
#pragma unroll
                    for (int kk = 0; kk < kTileK / 16; ++kk) {
                        const uint32_t off = kk * 32;
                        const uint64_t ahi = tc::smem_desc(st + off, 128);
                        const uint64_t alo = tc::smem_desc(st + kTileBytes + off, 128);
                        const uint64_t bhi = tc::smem_desc(st + 2 * kTileBytes + off, 128);
                        const uint64_t blo = tc::smem_desc(st + 2 * kTileBytes + kTileBytes / 2 + off, 128);
                        const uint32_t acc = (kc > g0 || kk > 0) ? 1u : 0u;
                        if (TF32) {
                            tc::mma_tf32_pair(d, ahi, bhi, P.idesc, acc);
                        } else {
                            tc::mma_f16_pair(d, ahi, bhi, P.idesc, acc);
                            tc::mma_f16_pair(d, ahi, blo, P.idesc, 1u);
                            tc::mma_f16_pair(d, alo, bhi, P.idesc, 1u);
                        }
                    }
                    tc::mma_commit_pair(&sh.empty[s], 0x3);
                    if (++s == kCPStages) { s = 0; ph ^= 1; }
                }
                if (!ok) break;
                tc::mma_commit_pair(&sh.acc_full[b], 0x3);
            }
        }
        tc::mma_commit_pair(&sh.drain, 0x1);
        volatile int never = 0;
        tc::mbar_wait(&sh.drain, 0, &never);
    } else if (warp >= 2) {
        // ---------------- epilogue (both CTAs) ----------------
        const int q = warp & 3;          // TMEM lane quarter
        const int h = (warp - 2) >> 2;   // column block: 32 columns per warp
        const uint32_t even_acc_empty0 = tc::mapa_shared(&sh.acc_empty[0], 0);
        uint32_t gcount = 0;
        bool ok = true;
        for (int u = cid; u < n_units && ok && !*abort; u += n_cl) {
            const int mp = u % n_mp, wt = (u / n_mp) % P.n_wt, sp = u / (n_mp * P.n_wt);
            const int mt = 2 * mp + (int)rank;
            const int k0 = (int)((long)sp * P.nk / P.n_split), k1 = (int)((long)(sp + 1) * P.nk / P.n_split);
            // the double-float sums of this thread's 32 columns as 16 column pairs
            // (column 2k in .x, 2k + 1 in .y): hi in registers, lo in shared memory
            // ([pair][epilogue thread], 8-byte accesses)
            float2 hi[16];
            float2* lo = reinterpret_cast<float2*>(base + kCPStages * kCPStageBytes) + (threadIdx.x - 64);
#pragma unroll
            for (int k = 0; k < 16; ++k) { hi[k] = make_float2(0.f, 0.f); lo[k * kCEpiWarps * 32] = make_float2(0.f, 0.f); }
            for (int g0 = k0; g0 < k1; g0 += kGroup, ++gcount) {
                const uint32_t b = gcount % kCBufs, use = gcount / kCBufs;
                if (!tc::mbar_wait_cluster(&sh.acc_full[b], use & 1, abort)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + b * kCBN + h * 32;
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    float v[16];
                    tc::tmem_ld16(taddr + part * 16, v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        float2 l = lo[(part * 8 + k) * kCEpiWarps * 32];
                        two_sum_acc2(hi[part * 8 + k], l, make_float2(v[2 * k], v[2 * k + 1]));
                        lo[(part * 8 + k) * kCEpiWarps * 32] = l;
                    }
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive_remote(even_acc_empty0 + b * (uint32_t)sizeof(uint64_t));
            }
            if (!ok) break;
            const int g = mt * kBM + q * 32 + lane;
            if (g < P.rows) {
                double2* dst = reinterpret_cast<double2*>(
                    P.part + ((size_t)sp * P.rows + g) * P.ldp + (size_t)wt * kCBN + h * 32);
#pragma unroll
                for (int k = 0; k < 16; ++k)
                {
                    const float2 l = lo[k * kCEpiWarps * 32];
                    dst[k] = make_double2(f2d_bits(hi[k].x) + f2d_bits(l.x), f2d_bits(hi[k].y) + f2d_bits(l.y));
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    // the even CTA's MMAs read the odd CTA's shared memory and write its TMEM,
    // and both CTAs arrive on each other's barriers: neither leaves early
    tc::cluster_sync();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc_pair(tmem, kCBufs * kCBN);
    if (threadIdx.x == 0 && sh.abort) atomicExch(P.err, 1);
}

struct LoParams {
    const uint16_t* u_hi;  // operand tiles [tile][kb]
    const uint16_t* u_lo;
    const uint16_t* v_hi;
    const uint16_t* v_lo;
    const uint16_t* d_hi;  // Delta tiles [c][rb][kb]
    const uint16_t* d_lo;
    int nrb;
    const int4* pt;       // half-tiles {row0, nvalid | H << 16, ci << 16 | cj, element offset}
    const float4* rowc;   // per packed row {inv_su, inv_sv, p, q}
    const float* inv_t;   // per walker inverse Delta scale
    double2* part;        // [n_pt / 2][ldp] per rank chunk and walker
    int n_pt, n_wt, W, ldp, nk;
    uint32_t idesc;
    int* err;
    // failure-path test hook: the even CTA of the first CTA pair leaves the
    // first stage of its first unit unfilled, so that its waits run out
    int withhold;
};

// ---- LO exchange kernel: one CTA pair per (rank chunk of a pair, 128 walkers) ----
// A cta_group::2 MMA of M = 256 Delta rows (128 walkers x re/im; the even CTA
// holds walkers 0-63 of the block, the odd CTA walkers 64-127) by N = the
// chunk's ranks (at most 256, a multiple of 16; each CTA holds one half-tile of
// N / 2 weight rows).  A pair's ranks are cut into balanced chunks, so rank
// padding stays at a few percent.  The a (Delta_j, U) and b (Delta_i, V)
// products are independent GEMMs: the ring holds half-stages of one side each,
// 64 basis functions deep (2 x 16 KB Delta tile + 2 weight half-tiles), three
// of them, consumed a, b, a, b, ...  TMEM lane = walker row, column = rank: the
// epilogue sums over ranks along its own columns, with one lane-pair shuffle
// for the complex product.
constexpr int kLBK = kTileK;                                 // basis functions per k-step
constexpr uint32_t kLTileA = kTileBytes;                     // 16 KB: up to 128 weight rows
constexpr uint32_t kLTileBh = kTileBytes;                    // 16 KB: 128 Delta rows
constexpr uint32_t kLSlotBytes = 2 * kLTileA + 2 * kLTileBh;  // 64 KB
constexpr int kLSlots = 3;
constexpr int kLEpiWarps = 16;
constexpr int kLThreads = 64 + 32 * kLEpiWarps;

struct LoShared {
    uint64_t full[kLSlots];    // even CTA: own TMA bytes + the odd CTA's forward
    uint64_t empty[kLSlots];   // both: the pair MMA's commit (multicast)
    uint64_t tmem_full;        // both: the pair MMA's commit (multicast)
    uint64_t tmem_empty;       // even CTA: 16 local + 16 remote epilogue warps
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
    float red[4][kBM];         // per column group: sum over its ranks, per walker row
    float4 cst[kBN];           // per rank of the chunk: {p inv_sv, q inv_su, inv_su inv_sv, 0}
};

// Roles per CTA: warp 0 lane 0 TMA producer; warp 1 lane 0 the MMA issuer on
// the even CTA, on the odd CTA the forwarder that passes each landed stage on
// to the even CTA's full barrier; warps 2-17 the epilogue (four per TMEM lane
// quarter, each draining 2 of the 8 32-column chunks).
__global__ void __launch_bounds__(kLThreads, 1)
lo_exchange_tc_kernel(LoParams P) {
    extern __shared__ uint8_t dyn_smem[];
    __shared__ LoShared sh;
    uint8_t* base = align1024(dyn_smem);
    // slot: W hi, W lo (the chunk's H weight rows, up to 16 KB each), D hi, D lo
    // (16 KB each); W = U, D = Delta_j on the a side, W = V, D = Delta_i on the b side
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = tc::cluster_ctarank();
    const bool even = rank == 0;
    const int cid = blockIdx.x >> 1, n_cl = gridDim.x >> 1;
    const int n_units = (P.n_pt >> 1) * P.n_wt;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kLSlots; ++s) {
            tc::mbar_init(&sh.full[s], even ? 2 : 1);
            tc::mbar_init(&sh.empty[s], 1);
        }
        tc::mbar_init(&sh.tmem_full, 1);
        tc::mbar_init(&sh.tmem_empty, 2 * kLEpiWarps);
        tc::mbar_init(&sh.drain, 1);
        sh.abort = 0;
        tc::fence_barrier_init();
    }
    if (warp == 0) {
        tc::tmem_alloc_pair(&sh.tmem_base, 2 * kBN);
        tc::tmem_relinquish_pair();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::cluster_sync();  // both CTAs' barriers initialised before any remote arrive
    tc::tc_fence_after();
    const uint32_t tmem = sh.tmem_base;
    volatile int* abort = &sh.abort;

    if (warp == 0 && lane == 0) {
        // ---------------- bulk-copy producer (both CTAs) ----------------
        int s = 0;
        uint32_t ph = 0, filled = 0, last_par = 0;
        for (int u = cid; u < n_units && !*abort; u += n_cl) {
            const int4 t = P.pt[2 * (u / P.n_wt) + rank];
            const int rb = 2 * (u % P.n_wt) + (int)rank;  // this CTA's 128 Delta rows
            const uint32_t wbytes = (uint32_t)(t.y >> 16) * 128u;  // H weight rows of 128 bytes
            for (int h = 0; h < 2 * P.nk; ++h) {
                if (!tc::mbar_wait_cluster(&sh.empty[s], ph ^ 1, abort)) break;
                if (P.withhold && cid == 0 && even && u == cid && h == 0) {
                    // no arrival and no copy: the MMA issuer's wait on this stage
                    // (and every wait behind it) runs out after the wait limit
                    if (++s == kLSlots) { s = 0; ph ^= 1; }
                    continue;
                }
                uint8_t* st = base + s * kLSlotBytes;
                tc::mbar_arrive_expect_tx(&sh.full[s], 2 * wbytes + 2 * kLTileBh);
                const int kb = h >> 1;
                const bool side_b = h & 1;
                const size_t ao = (size_t)(unsigned)t.w + (size_t)kb * (t.y >> 16) * kTileK;
                const int orb = side_b ? (t.z >> 16) : (t.z & 0xffff);
                const size_t bo = (((size_t)orb * P.nrb + rb) * P.nk + kb) * kTileElems;
                tc::bulk_load(st, (side_b ? P.v_hi : P.u_hi) + ao, wbytes, &sh.full[s]);
                tc::bulk_load(st + kLTileA, (side_b ? P.v_lo : P.u_lo) + ao, wbytes, &sh.full[s]);
                tc::bulk_load(st + 2 * kLTileA, P.d_hi + bo, kLTileBh, &sh.full[s]);
                tc::bulk_load(st + 2 * kLTileA + kLTileBh, P.d_lo + bo, kLTileBh, &sh.full[s]);
                filled |= 1u << s;
                last_par = (last_par & ~(1u << s)) | (ph << s);
                if (++s == kLSlots) { s = 0; ph ^= 1; }
            }
        }
        if (*abort) {
            // the even CTA's full barriers also count the forward, so wait for
            // the transaction bytes only: every load issued has landed once the
            // phase's tx count is back to zero; bounded by the wait limit
            for (int q = 0; q < kLSlots; ++q)
                if (filled & (1u << q)) {
                    volatile int never = 0;
                    if (even) {
                        // one arrive of ours is outstanding only if the odd
                        // CTA's forward is missing; give it up to the limit
                        tc::mbar_wait_cluster(&sh.full[q], (last_par >> q) & 1, &never);
                    } else {
                        tc::mbar_wait(&sh.full[q], (last_par >> q) & 1, &never);
                    }
                }
        }
    } else if (warp == 1 && lane == 0 && !even) {
        // ---------------- forwarder (odd CTA) ----------------
        const uint32_t peer_full0 = tc::mapa_shared(&sh.full[0], 0);
        int s = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int u = cid; u < n_units && ok && !*abort; u += n_cl) {
            for (int h = 0; h < 2 * P.nk; ++h) {
                if (!tc::mbar_wait(&sh.full[s], ph, abort)) { ok = false; break; }
                tc::mbar_arrive_remote(peer_full0 + s * (uint32_t)sizeof(uint64_t));
                if (++s == kLSlots) { s = 0; ph ^= 1; }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- pair MMA issuer (even CTA) ----------------
        int s = 0;
        uint32_t ph = 0, tph = 0;
        const uint32_t tA = tmem, tB = tmem + kBN;  // accumulators a (U side), b (V side)
        for (int u = cid; u < n_units && !*abort; u += n_cl) {
            // N = the chunk's ranks = twice the half-tile height
            const int Nc = 2 * (P.pt[2 * (u / P.n_wt)].y >> 16);
            const uint32_t idesc = (P.idesc & ~(0x3fu << 17)) | ((uint32_t)(Nc >> 3) << 17);
            if (!tc::mbar_wait_cluster(&sh.tmem_empty, tph ^ 1, abort)) break;
            tc::tc_fence_after();
            bool ok = true;
            for (int h = 0; h < 2 * P.nk; ++h) {
                if (!tc::mbar_wait_cluster(&sh.full[s], ph, abort)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t st = tc::smem_u32(base + s * kLSlotBytes);
                const uint32_t d = (h & 1) ? tB : tA;
#pragma unroll
                for (int kk = 0; kk < kLBK / 16; ++kk) {
                    const uint32_t off = kk * 32;
                    const uint64_t whi = tc::smem_desc(st + off, 128);
                    const uint64_t wlo = tc::smem_desc(st + kLTileA + off, 128);
                    const uint64_t dhi = tc::smem_desc(st + 2 * kLTileA + off, 128);
                    const uint64_t dlo = tc::smem_desc(st + 2 * kLTileA + kLTileBh + off, 128);
                    const uint32_t acc = (h > 1 || kk > 0) ? 1u : 0u;
                    // A = Delta rows (walkers), B = weight rows (ranks)
                    tc::mma_f16_pair(d, dhi, whi, idesc, acc);
                    tc::mma_f16_pair(d, dlo, whi, idesc, 1u);
                    tc::mma_f16_pair(d, dhi, wlo, idesc, 1u);
                }
                tc::mma_commit_pair(&sh.empty[s], 0x3);
                if (++s == kLSlots) { s = 0; ph ^= 1; }
            }
            if (!ok) break;
            tc::mma_commit_pair(&sh.tmem_full, 0x3);
            tph ^= 1;
        }
        tc::mma_commit_pair(&sh.drain, 0x1);
        volatile int never = 0;
        tc::mbar_wait(&sh.drain, 0, &never);
    } else if (warp >= 2) {
        // ---------------- epilogue (both CTAs) ----------------
        // lane = walker row z = 2 w + re/im of this CTA, column = rank n of the
        // chunk.  Per rank and walker (complex; the other component sits in the
        // partner lane z ^ 1):
        //   da = inv_su it a, db = inv_sv it b,   val = p db + q da + da db
        // summed over this warp's column group (64 ranks, in 32-column loads);
        // the four groups add in shared memory; one FP64 value per (chunk, walker).
        const int q = warp & 3;                       // TMEM lane quarter
        const int grp = (warp - 2) >> 2;              // column group
        const int ep_tid = threadIdx.x - 64;          // 0..511
        const int z = q * 32 + lane;                  // walker row of this CTA
        const bool odd = (lane & 1) != 0;             // imaginary component
        const uint32_t even_tmem_empty = tc::mapa_shared(&sh.tmem_empty, 0);
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        uint32_t tph = 0;
        for (int u = cid; u < n_units; u += n_cl) {
            const int ch = u / P.n_wt, wt = u % P.n_wt;
            const int4 t0 = P.pt[2 * ch], t1 = P.pt[2 * ch + 1];
            const int Nc = 2 * (t0.y >> 16);
            const int nvalid = (t0.y & 0xffff) + (t1.y & 0xffff);
            const int w = wt * kBNW + (int)rank * (kBNW / 2) + (z >> 1);
            const float it = w < P.W ? __ldg(P.inv_t + w) : 0.f;
            // the chunk's per-rank constants (zero beyond its valid ranks); the
            // previous unit's readers are past its closing barrier
            if (ep_tid < kBN) {
                float4 k4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (ep_tid < nvalid) {
                    const float4 rc = __ldg(P.rowc + t0.x + ep_tid);
                    k4 = make_float4(rc.z * rc.y, rc.w * rc.x, rc.x * rc.y, 0.f);
                }
                sh.cst[ep_tid] = k4;
            }
            asm volatile("bar.sync 1, %0;" :: "n"(32 * kLEpiWarps) : "memory");
            const bool got = tc::mbar_wait_cluster(&sh.tmem_full, tph, abort);
            // leave together: the named barriers below expect every epilogue warp
            if (tc::bar_or(!got, 1, 32 * kLEpiWarps)) break;
            tc::tc_fence_after();
            const int c_begin = grp * 64;
            const int nld = c_begin >= Nc ? 0 : (min(Nc - c_begin, 64) + 31) / 32;
            if (nld == 0) {
                // no columns for this warp: release at once
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive_remote(even_tmem_empty);
            }
            float acc = 0.f;
#pragma unroll 1
            for (int c2 = 0; c2 < nld; ++c2) {
                const int col0 = c_begin + 32 * c2;
                float va[32], vb[32];
                tc::tmem_ld32(tmem + lane_off + col0, va);
                tc::tmem_ld32(tmem + lane_off + kBN + col0, vb);
                tc::tmem_wait_ld();
                if (c2 == nld - 1) {
                    // the last TMEM read of this warp is complete: release
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive_remote(even_tmem_empty);
                }
#pragma unroll
                for (int m = 0; m < 32; ++m) {
                    const float a = va[m], b = vb[m];
                    const float pa = __shfl_xor_sync(0xffffffffu, a, 1);
                    const float pb = __shfl_xor_sync(0xffffffffu, b, 1);
                    const float4 k4 = sh.cst[col0 + m];        // broadcast
                    const float lin = fmaf(k4.x, b, k4.y * a);  // p inv_sv db' + q inv_su da'
                    const float quad = odd ? fmaf(pa, b, a * pb) : fmaf(a, b, -pa * pb);
                    const float v = fmaf(k4.z * it, quad, lin);
                    // columns past the chunk were not written by this unit's MMAs
                    acc += col0 + m < Nc ? v : 0.f;
                }
            }
            tph ^= 1;
            sh.red[grp][z] = acc * it;
            asm volatile("bar.sync 1, %0;" :: "n"(32 * kLEpiWarps) : "memory");
            if (ep_tid < kBNW / 2) {
                const int wl = wt * kBNW + (int)rank * (kBNW / 2) + ep_tid;
                const double re = f2d_bits(sh.red[0][2 * ep_tid]) + f2d_bits(sh.red[1][2 * ep_tid]) +
                                  f2d_bits(sh.red[2][2 * ep_tid]) + f2d_bits(sh.red[3][2 * ep_tid]);
                const double im = f2d_bits(sh.red[0][2 * ep_tid + 1]) + f2d_bits(sh.red[1][2 * ep_tid + 1]) +
                                  f2d_bits(sh.red[2][2 * ep_tid + 1]) + f2d_bits(sh.red[3][2 * ep_tid + 1]);
                if (wl < P.W) P.part[(size_t)ch * P.ldp + wl] = make_double2(re, im);
            }
            asm volatile("bar.sync 1, %0;" :: "n"(32 * kLEpiWarps) : "memory");
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    // the even CTA's MMAs read the odd CTA's shared memory and write its TMEM,
    // and both CTAs arrive on each other's barriers: neither leaves early
    tc::cluster_sync();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc_pair(tmem, 2 * kBN);
    if (threadIdx.x == 0 && sh.abort) atomicExch(P.err, 1);
}

// ---- LO exchange through dense truncated blocks ----
// For a pair [ij] whose kept rank K is above about M / 2, the truncated block
// Ytil = Ubar Vbar (M x M) costs M^2 multiply-adds per walker against 2 M K
// through its factors, and gives the same pair value (eq. 2e_HR_RCAS_LO read
// right to left):  e_ij = Theta_j^T Ytil Theta_i.  With Theta = Phi_T + Delta,
//   e_ij = e0 + g . Delta_i + Delta_j . (Ytil Delta_i + h),
//   g = Ytil^T Phi_j = Vbar^T p,  h = Ytil Phi_i = Ubar q,  e0 = p . q,
// all walker-independent parts in FP64 at setup.  B operand: the rows s of
// Ytil followed by g (M + 1 rows, in balanced chunks of at most 256, two
// half-tiles per chunk as in the factored kernel); A operand: the Delta_i rows
// of 128 walkers (M = 256 over the CTA pair); K = the basis.  The accumulator
// Z[z][s] = (Ytil Delta_i)[s] (row g: g . Delta_i) sits in one of two TMEM
// buffers of 256 columns, so the epilogue of one unit runs under the MMAs of
// the next.  The epilogue reads Delta_j[w][s] in FP32 from the walker-row-major
// copy the Theta stage writes and sums the complex products along its columns.
struct LoDenseParams {
    const uint16_t* y_hi;  // B half-tiles [tile][kb]
    const uint16_t* y_lo;
    const uint16_t* d_hi;  // Delta tiles [c][rb][kb]
    const uint16_t* d_lo;
    const float* dfull;    // Delta t, FP32, dfull_elem layout
    int nrb, Sd;
    const int4* pt;        // half-tiles {row0, nvalid | H << 16, ci << 24 | cj << 16 | s0, element offset}
    const float2* rowc;    // per dense row {1 / row scale, h}
    const float* inv_t;    // per walker 1 / t
    double2* part;         // [chunk][ldp]
    int n_pt, n_wt, W, ldp, nk, M;
    uint32_t idesc;
    int* err;
    int withhold;          // failure-path test hook, as in the factored kernel
};

struct LoDenseShared {
    uint64_t full[kLSlots];     // even CTA: own bytes + the odd CTA's forward
    uint64_t empty[kLSlots];    // both: the pair MMA's commit (multicast)
    uint64_t tmem_full[2];      // both: the pair MMA's commit (multicast)
    uint64_t tmem_empty[2];     // even CTA: 16 local + 16 remote epilogue warps
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
    float red[4][kBM];          // per column group: sum over its columns, per walker row
    __align__(16) float2 cst[2][kBN];  // per column of a chunk: {1 / row scale, h}; two units
};

// TF32: one plane of FP32 values read as TF32 (same tile images, 32-wide basis
// blocks), one product per k-step.
template <bool TF32>
__global__ void __launch_bounds__(kLThreads, 1)
lo_dense_tc_kernel(LoDenseParams P) {
    constexpr uint32_t kPlanes = TF32 ? 1u : 2u;
    extern __shared__ uint8_t dyn_smem[];
    __shared__ LoDenseShared sh;
    uint8_t* base = align1024(dyn_smem);
    // slot: Y hi, Y lo (the chunk's H rows, up to 16 KB each), D hi, D lo (16 KB each)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = tc::cluster_ctarank();
    const bool even = rank == 0;
    const int cid = blockIdx.x >> 1, n_cl = gridDim.x >> 1;
    const int n_units = (P.n_pt >> 1) * P.n_wt;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kLSlots; ++s) {
            tc::mbar_init(&sh.full[s], even ? 2 : 1);
            tc::mbar_init(&sh.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&sh.tmem_full[b], 1);
            tc::mbar_init(&sh.tmem_empty[b], 2 * kLEpiWarps);
        }
        tc::mbar_init(&sh.drain, 1);
        sh.abort = 0;
        tc::fence_barrier_init();
    }
    if (warp == 0) {
        tc::tmem_alloc_pair(&sh.tmem_base, 2 * kBN);
        tc::tmem_relinquish_pair();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::cluster_sync();  // both CTAs' barriers initialised before any remote arrive
    tc::tc_fence_after();
    const uint32_t tmem = sh.tmem_base;
    volatile int* abort = &sh.abort;

    if (warp == 0 && lane == 0) {
        // ---------------- bulk-copy producer (both CTAs) ----------------
        int s = 0;
        uint32_t ph = 0, filled = 0, last_par = 0;
        for (int u = cid; u < n_units && !*abort; u += n_cl) {
            const int4 t = P.pt[2 * (u / P.n_wt) + rank];
            const int rb = 2 * (u % P.n_wt) + (int)rank;  // this CTA's 128 Delta rows
            const uint32_t H = (uint32_t)(t.y >> 16);
            const uint32_t wbytes = H * 128u;  // H rows of 128 bytes
            const int orb = (int)((unsigned)t.z >> 24);
            for (int kb = 0; kb < P.nk; ++kb) {
                if (!tc::mbar_wait_cluster(&sh.empty[s], ph ^ 1, abort)) break;
                if (P.withhold && cid == 0 && even && u == cid && kb == 0) {
                    // no arrival and no copy: the waits behind this stage run out
                    if (++s == kLSlots) { s = 0; ph ^= 1; }
                    continue;
                }
                uint8_t* st = base + s * kLSlotBytes;
                tc::mbar_arrive_expect_tx(&sh.full[s], kPlanes * (wbytes + kLTileBh));
                const size_t ao = (size_t)(unsigned)t.w + (size_t)kb * H * kTileK;
                const size_t bo = (((size_t)orb * P.nrb + rb) * P.nk + kb) * kTileElems;
                tc::bulk_load(st, P.y_hi + ao, wbytes, &sh.full[s]);
                if (!TF32) tc::bulk_load(st + kLTileA, P.y_lo + ao, wbytes, &sh.full[s]);
                tc::bulk_load(st + 2 * kLTileA, P.d_hi + bo, kLTileBh, &sh.full[s]);
                if (!TF32) tc::bulk_load(st + 2 * kLTileA + kLTileBh, P.d_lo + bo, kLTileBh, &sh.full[s]);
                filled |= 1u << s;
                last_par = (last_par & ~(1u << s)) | (ph << s);
                if (++s == kLSlots) { s = 0; ph ^= 1; }
            }
        }
        if (*abort) {
            // every load issued has landed once its phase completes; bounded waits
            for (int q = 0; q < kLSlots; ++q)
                if (filled & (1u << q)) {
                    volatile int never = 0;
                    if (even)
                        tc::mbar_wait_cluster(&sh.full[q], (last_par >> q) & 1, &never);
                    else
                        tc::mbar_wait(&sh.full[q], (last_par >> q) & 1, &never);
                }
        }
    } else if (warp == 1 && lane == 0 && !even) {
        // ---------------- forwarder (odd CTA) ----------------
        const uint32_t peer_full0 = tc::mapa_shared(&sh.full[0], 0);
        int s = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int u = cid; u < n_units && ok && !*abort; u += n_cl) {
            for (int kb = 0; kb < P.nk; ++kb) {
                if (!tc::mbar_wait(&sh.full[s], ph, abort)) { ok = false; break; }
                tc::mbar_arrive_remote(peer_full0 + s * (uint32_t)sizeof(uint64_t));
                if (++s == kLSlots) { s = 0; ph ^= 1; }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- pair MMA issuer (even CTA) ----------------
        int s = 0, k = 0;
        uint32_t ph = 0;
        for (int u = cid; u < n_units && !*abort; u += n_cl, ++k) {
            const int Nc = 2 * (P.pt[2 * (u / P.n_wt)].y >> 16);
            const uint32_t idesc = (P.idesc & ~(0x3fu << 17)) | ((uint32_t)(Nc >> 3) << 17);
            const uint32_t buf = (uint32_t)k & 1u, use = (uint32_t)k >> 1;
            if (!tc::mbar_wait_cluster(&sh.tmem_empty[buf], (use & 1u) ^ 1u, abort)) break;
            tc::tc_fence_after();
            const uint32_t d = tmem + buf * kBN;
            bool ok = true;
            for (int kb = 0; kb < P.nk; ++kb) {
                if (!tc::mbar_wait_cluster(&sh.full[s], ph, abort)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t st = tc::smem_u32(base + s * kLSlotBytes);
#pragma unroll
                for (int kk = 0; kk < kLBK / 16; ++kk) {
                    const uint32_t off = kk * 32;
                    const uint64_t whi = tc::smem_desc(st + off, 128);
                    const uint64_t wlo = tc::smem_desc(st + kLTileA + off, 128);
                    const uint64_t dhi = tc::smem_desc(st + 2 * kLTileA + off, 128);
                    const uint64_t dlo = tc::smem_desc(st + 2 * kLTileA + kLTileBh + off, 128);
                    const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                    // A = Delta_i rows (walkers), B = rows of Ytil and g
                    if (TF32) {
                        tc::mma_tf32_pair(d, dhi, whi, idesc, acc);
                    } else {
                        tc::mma_f16_pair(d, dhi, whi, idesc, acc);
                        tc::mma_f16_pair(d, dlo, whi, idesc, 1u);
                        tc::mma_f16_pair(d, dhi, wlo, idesc, 1u);
                    }
                }
                tc::mma_commit_pair(&sh.empty[s], 0x3);
                if (++s == kLSlots) { s = 0; ph ^= 1; }
            }
            if (!ok) break;
            tc::mma_commit_pair(&sh.tmem_full[buf], 0x3);
        }
        tc::mma_commit_pair(&sh.drain, 0x1);
        volatile int never = 0;
        tc::mbar_wait(&sh.drain, 0, &never);
    } else if (warp >= 2) {
        // ---------------- epilogue (both CTAs) ----------------
        // lane = walker row z = 2 w + re/im of this CTA, column = row s of the
        // chunk.  Y = Z / (row scale) / t + h is this lane's component of
        // Ytil Theta_i (h on the real row only); D = t Delta_j from the FP32
        // copy (the partner row's value by a shuffle).  Each lane sums
        //   a1 = sum_s D_own Y,  a2 = sum_s D_other Y
        // and the walker's part is (a1(re) - a1(im), a2(re) + a2(im)) / t.  The g
        // row (g . Delta_i) needs no case of its own: the copy holds t in the
        // real row and 0 in the imaginary row at s = M.
        const int q = warp & 3;                       // TMEM lane quarter
        const int grp = (warp - 2) >> 2;              // column group of 64
        const int ep_tid = threadIdx.x - 64;          // 0..511
        const int z = q * 32 + lane;                  // walker row of this CTA
        const float hsel = (lane & 1) ? 0.f : 1.f;    // h enters the real row
        const uint32_t even_tmem_empty0 = tc::mapa_shared(&sh.tmem_empty[0], 0);
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        // per-row constants of a unit's chunk into cst[b] (zero past its rows)
        auto fetch_cst = [&](int u) {
            float2 k2 = make_float2(0.f, 0.f);
            if (u < n_units && ep_tid < kBN) {
                const int ch = u / P.n_wt;
                const int4 t0 = P.pt[2 * ch], t1 = P.pt[2 * ch + 1];
                if (ep_tid < (t0.y & 0xffff) + (t1.y & 0xffff)) k2 = __ldg(P.rowc + t0.x + ep_tid);
            }
            return k2;
        };
        {
            const float2 k2 = fetch_cst(cid);
            if (ep_tid < kBN) sh.cst[0][ep_tid] = k2;
        }
        asm volatile("bar.sync 1, %0;" :: "n"(32 * kLEpiWarps) : "memory");
        int k = 0;
        for (int u = cid; u < n_units; u += n_cl, ++k) {
            const uint32_t buf = (uint32_t)k & 1u, use = (uint32_t)k >> 1;
            const int ch = u / P.n_wt, wt = u % P.n_wt;
            const int4 t0 = P.pt[2 * ch];
            const int Nc = 2 * (t0.y >> 16);
            const int cj = (int)(((unsigned)t0.z >> 16) & 0xffu);
            const int s0 = t0.z & 0xffff;
            const int rb = 2 * wt + (int)rank;
            const int w = wt * kBNW + (int)rank * (kBNW / 2) + (z >> 1);
            const float it = w < P.W ? __ldg(P.inv_t + w) : 0.f;
            const float2* cst = sh.cst[k & 1];
            // the next unit's constants, stored after this unit's columns
            const float2 next_cst = fetch_cst(u + n_cl);
            const int c_begin = grp * 64;
            const int nb = c_begin >= Nc ? 0 : min(Nc - c_begin, 64) / 16;  // 16-column batches
            // this lane's row in the dfull_elem layout: float4 q of the chunk's
            // columns (s = s0 + c_begin + 4 q ..) at d_own[128 q]
            const float4* d_own = reinterpret_cast<const float4*>(P.dfull) +
                                  ((size_t)cj * P.nrb + rb) * (size_t)(P.Sd >> 2) * 128 +
                                  (size_t)((s0 + c_begin) >> 2) * 128 + z;
            // the first three batches of Delta_j are requested before the wait for
            // the MMAs, the fourth once the first is summed: the loads' latency
            // (microseconds from L2 under the operand copies) runs under the MMAs
            // instead of between batches (registers allow three in flight)
            float4 da[3][4];
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int m4 = 0; m4 < 4; ++m4)
                    da[b][m4] = b < nb ? __ldg(d_own + 128 * (4 * b + m4)) : make_float4(0.f, 0.f, 0.f, 0.f);
            const bool got = tc::mbar_wait_cluster(&sh.tmem_full[buf], use & 1u, abort);
            // leave together: the named barriers below expect every epilogue warp
            if (tc::bar_or(!got, 1, 32 * kLEpiWarps)) break;
            tc::tc_fence_after();
            if (nb == 0) {
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive_remote(even_tmem_empty0 + buf * (uint32_t)sizeof(uint64_t));
            }
            float a1 = 0.f, a2 = 0.f;
#pragma unroll
            for (int bi = 0; bi < 4; ++bi) {
                if (bi >= nb) break;
                const int col0 = c_begin + 16 * bi;
                float zv[16];
                tc::tmem_ld16(tmem + lane_off + buf * kBN + col0, zv);
                tc::tmem_wait_ld();
                if (bi == nb - 1) {
                    // the last TMEM read of this warp is complete: release the buffer
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive_remote(even_tmem_empty0 + buf * (uint32_t)sizeof(uint64_t));
                }
                const float* dov = reinterpret_cast<const float*>(da[bi == 3 ? 0 : bi]);
                const float4* c4 = reinterpret_cast<const float4*>(cst + col0);
#pragma unroll
                for (int m2 = 0; m2 < 8; ++m2) {
                    const float4 kk = c4[m2];  // two columns: {1/scale, h, 1/scale, h}
                    const float y0 = fmaf(zv[2 * m2], kk.x * it, kk.y * hsel);
                    const float y1 = fmaf(zv[2 * m2 + 1], kk.z * it, kk.w * hsel);
                    // the partner row's Delta_j (the other component of the walker)
                    const float o0 = __shfl_xor_sync(0xffffffffu, dov[2 * m2], 1);
                    const float o1 = __shfl_xor_sync(0xffffffffu, dov[2 * m2 + 1], 1);
                    a1 = fmaf(dov[2 * m2], y0, a1);
                    a2 = fmaf(o0, y0, a2);
                    a1 = fmaf(dov[2 * m2 + 1], y1, a1);
                    a2 = fmaf(o1, y1, a2);
                }
                if (bi == 0 && nb == 4) {
#pragma unroll
                    for (int m4 = 0; m4 < 4; ++m4) da[0][m4] = __ldg(d_own + 128 * (12 + m4));
                }
            }
            // this walker's real part from the real row's a1 and the imaginary row's
            // a1; its imaginary part from both rows' a2
            const float p1 = __shfl_xor_sync(0xffffffffu, a1, 1);
            const float p2 = __shfl_xor_sync(0xffffffffu, a2, 1);
            sh.red[grp][z] = ((lane & 1) ? a2 + p2 : a1 - p1) * it;
            asm volatile("bar.sync 1, %0;" :: "n"(32 * kLEpiWarps) : "memory");
            if (ep_tid < kBNW / 2) {
                const int wl = wt * kBNW + (int)rank * (kBNW / 2) + ep_tid;
                const double re = f2d_bits(sh.red[0][2 * ep_tid]) + f2d_bits(sh.red[1][2 * ep_tid]) +
                                  f2d_bits(sh.red[2][2 * ep_tid]) + f2d_bits(sh.red[3][2 * ep_tid]);
                const double im = f2d_bits(sh.red[0][2 * ep_tid + 1]) + f2d_bits(sh.red[1][2 * ep_tid + 1]) +
                                  f2d_bits(sh.red[2][2 * ep_tid + 1]) + f2d_bits(sh.red[3][2 * ep_tid + 1]);
                if (wl < P.W) P.part[(size_t)ch * P.ldp + wl] = make_double2(re, im);
            }
            if (ep_tid < kBN) sh.cst[(k + 1) & 1][ep_tid] = next_cst;
            asm volatile("bar.sync 1, %0;" :: "n"(32 * kLEpiWarps) : "memory");
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    // the even CTA's MMAs read the odd CTA's shared memory and write its TMEM,
    // and both CTAs arrive on each other's barriers: neither leaves early
    tc::cluster_sync();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc_pair(tmem, 2 * kBN);
    if (threadIdx.x == 0 && sh.abort) atomicExch(P.err, 1);
}

// ---------------------------------------------------------------------------
// FP64 reductions of the tensor-core partials
// ---------------------------------------------------------------------------

// E1 = E1_0 + dE1,  E_J = 1/2 sum_g (J0_g + dJ_g)^2,  dJ from the split partials
// The reductions run on a (walker block, slice) grid: slice sl of the rows g
// (Coulomb) or pairs n (exchange) sums into red[sl][w]; a final pass adds the
// slices in order, so the result does not depend on the launch.
constexpr int kRedSlices = 16;

// sum_g (J0_g + dJ_g)^2 over the rows of this slice, dJ from the split partials
__global__ void coulomb_tc_reduce_kernel(int X, int W, int n_split, int ldp,
                                         const double* __restrict__ part,
                                         const float* __restrict__ inv_s,
                                         const float* __restrict__ inv_t,
                                         const double* __restrict__ J0,
                                         double2* __restrict__ red_out, double2* __restrict__ j_out) {
    // 32 walkers x 8 row groups
    __shared__ double2 red[8][32];
    const int wl = threadIdx.x & 31, gg = threadIdx.x >> 5;
    const int w = blockIdx.x * 32 + wl, sl = blockIdx.y, nsl = gridDim.y;
    const int g0 = (int)((long)sl * X / nsl), g1 = (int)((long)(sl + 1) * X / nsl);
    double2 acc = make_double2(0.0, 0.0);
    const size_t plane = (size_t)(X + 1) * ldp;
    if (w < W) {
        const double it = inv_t[w];
        for (int g = g0 + gg; g < g1; g += 8) {
            double re = 0.0, im = 0.0;
            for (int s = 0; s < n_split; ++s) {
                const double2 v = *reinterpret_cast<const double2*>(part + s * plane + (size_t)g * ldp + 2 * w);
                re += v.x;
                im += v.y;
            }
            const double f = (double)inv_s[g] * it;
            const double2 J = make_double2(J0[g] + re * f, im * f);
            if (j_out) j_out[(size_t)w * X + g] = J;
            acc = cadd(acc, cmul(J, J));
        }
    }
    red[gg][wl] = acc;
    __syncthreads();
    if (gg == 0 && w < W) {
        double2 t = make_double2(0.0, 0.0);
        for (int k = 0; k < 8; ++k) t = cadd(t, red[k][wl]);
        red_out[(size_t)sl * W + w] = t;
    }
}

// E_J = 1/2 sum over slices; E1 = E1_0 + the one-body row X
__global__ void coulomb_tc_final_kernel(int X, int W, int n_split, int ldp, int nsl,
                                        const double* __restrict__ part,
                                        const float* __restrict__ inv_s,
                                        const float* __restrict__ inv_t, double E1_0,
                                        const double2* __restrict__ red, double2* __restrict__ e1,
                                        double2* __restrict__ ej) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    double2 t = make_double2(0.0, 0.0);
    for (int sl = 0; sl < nsl; ++sl) t = cadd(t, red[(size_t)sl * W + w]);
    ej[w] = cscale(t, 0.5);
    const size_t plane = (size_t)(X + 1) * ldp;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < n_split; ++s) {
        const double2 v = *reinterpret_cast<const double2*>(part + s * plane + (size_t)X * ldp + 2 * w);
        re += v.x;
        im += v.y;
    }
    const double f = (double)inv_s[X] * inv_t[w];
    e1[w] = make_double2(E1_0 + re * f, im * f);
}

// per pair of this slice: e_n(w) = e0_n + sum over its tiles; the slice's
// share of E_K - EK0 = sum_n pw_n de_n(w)
__global__ void lo_tc_reduce_kernel(int n_pairs, int W, int ldp, const int* __restrict__ pt0,
                                    const int* __restrict__ npt, const double* __restrict__ pw,
                                    const double* __restrict__ e0,
                                    const double2* __restrict__ part, double2* __restrict__ red_out,
                                    double2* __restrict__ e_pairs) {
    __shared__ double2 red[8][32];
    const int wl = threadIdx.x & 31, gg = threadIdx.x >> 5;
    const int w = blockIdx.x * 32 + wl, sl = blockIdx.y, nsl = gridDim.y;
    const int n0 = (int)((long)sl * n_pairs / nsl), n1 = (int)((long)(sl + 1) * n_pairs / nsl);
    double2 acc = make_double2(0.0, 0.0);
    if (w < W) {
        for (int n = n0 + gg; n < n1; n += 8) {
            double2 d = make_double2(0.0, 0.0);
            // a pair's half-tiles come in pairs, one partial row per pair of them
            for (int k = 0; k < (npt[n] >> 1); ++k) d = cadd(d, part[(size_t)((pt0[n] >> 1) + k) * ldp + w]);
            if (e_pairs) e_pairs[(size_t)n * W + w] = make_double2(e0[n] + d.x, d.y);
            acc = cadd(acc, cscale(d, pw[n]));
        }
    }
    red[gg][wl] = acc;
    __syncthreads();
    if (gg == 0 && w < W) {
        double2 t = make_double2(0.0, 0.0);
        for (int k = 0; k < 8; ++k) t = cadd(t, red[k][wl]);
        red_out[(size_t)sl * W + w] = t;
    }
}

// E_K(w) = EK0 + the slices in order
__global__ void lo_tc_final_kernel(int W, int nsl, double EK0, const double2* __restrict__ red,
                                   double2* __restrict__ ek) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    double2 t = make_double2(EK0, 0.0);
    for (int sl = 0; sl < nsl; ++sl) t = cadd(t, red[(size_t)sl * W + w]);
    ek[w] = t;
}

SpinRef spin_ref(const SpinData& s) {
    return SpinRef{s.d_Lbar.as<double>(), s.d_hbar.as<double>(), s.d_trial.as<double>(), s.N,
                   s.col0, s.mult};
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
// Row padding of the operand planes in 16-bit units: 16-bit values padded to a
// multiple of 8, TF32 values (two units each) to a multiple of 4
inline int plane_pad(int M, bool tf32) { return tf32 ? 2 * ((M + 3) / 4 * 4) : (M + 7) / 8 * 8; }

void ensure_coulomb_ops(loaf_ctx* c, MixedOps& mx, bool bf16, bool tf32) {
    if (mx.coul_ready) return;
    mx.bf16 = bf16;
    mx.tf32 = tf32;
    mx.r_pad = plane_pad(c->M, tf32);
    mx.kflat = (long)c->ntot * mx.r_pad;
    const int rows = c->X + 1;
    mx.L_hi.ensure((size_t)rows * mx.kflat * 2);
    if (!tf32) mx.L_lo.ensure((size_t)rows * mx.kflat * 2);
    mx.L_inv.ensure((size_t)rows * sizeof(float));
    mx.J0.ensure((size_t)rows * sizeof(double));
    SpinRef s0 = spin_ref(c->sp[0]), s1 = c->nspin > 1 ? spin_ref(c->sp[1]) : s0;
    if (tf32)
        coul_tf32_kernel<<<rows, 256, 0, c->stream>>>(c->M, c->X, mx.r_pad / 2, c->nspin, s0, s1,
                                                     mx.L_hi.as<float>(), mx.L_inv.as<float>());
    else if (bf16)
        coul_split_kernel<true><<<rows, 256, 0, c->stream>>>(c->M, c->X, mx.r_pad, c->nspin, s0, s1,
                                                            mx.L_hi.as<uint16_t>(), mx.L_lo.as<uint16_t>(),
                                                            mx.L_inv.as<float>());
    else
        coul_split_kernel<false><<<rows, 256, 0, c->stream>>>(c->M, c->X, mx.r_pad, c->nspin, s0, s1,
                                                             mx.L_hi.as<uint16_t>(), mx.L_lo.as<uint16_t>(),
                                                             mx.L_inv.as<float>());
    LOAF_LAUNCH_CHECK();
    trial_coulomb_kernel<<<rows, 256, 0, c->stream>>>(c->M, c->X, c->nspin, s0, s1, mx.J0.as<double>());
    LOAF_LAUNCH_CHECK();
    // operand tiles [mt][c][kb] (a TF32 tile holds 32 basis functions in the same
    // 16 KB image); the row-major staging planes are then dropped
    mx.nkb = ceil_div(c->M, tf32 ? kTileK / 2 : kTileK);
    mx.n_mt = ceil_div(rows, kTileRows);
    // an even number of row tiles for the CTA-pair kernel: the last one may be zeros
    const size_t tile_set = (size_t)c->ntot * mx.nkb * kTileBytes;  // one row tile
    const size_t tiles_bytes = (size_t)((mx.n_mt + 1) & ~1) * tile_set;
    mx.Lb_hi.ensure(tiles_bytes);
    if (!tf32) mx.Lb_lo.ensure(tiles_bytes);
    if (mx.n_mt & 1) {
        LOAF_CUDA(cudaMemsetAsync(mx.Lb_hi.as<uint8_t>() + mx.n_mt * tile_set, 0, tile_set, c->stream));
        if (!tf32)
            LOAF_CUDA(cudaMemsetAsync(mx.Lb_lo.as<uint8_t>() + mx.n_mt * tile_set, 0, tile_set, c->stream));
    }
    const dim3 tg(mx.n_mt * c->ntot, mx.nkb);
    coul_tiles_kernel<<<tg, 256, 0, c->stream>>>(mx.L_hi.as<uint16_t>(), rows, c->ntot, mx.r_pad, mx.nkb,
                                                mx.Lb_hi.as<uint16_t>());
    if (!tf32)
        coul_tiles_kernel<<<tg, 256, 0, c->stream>>>(mx.L_lo.as<uint16_t>(), rows, c->ntot, mx.r_pad, mx.nkb,
                                                    mx.Lb_lo.as<uint16_t>());
    LOAF_LAUNCH_CHECK();
    LOAF_CUDA(cudaMemcpyAsync(&mx.E1_0, mx.J0.as<double>() + c->X, sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
    LOAF_CUDA(cudaStreamSynchronize(c->stream));
    mx.L_hi.release();
    mx.L_lo.release();
    mx.coul_ready = true;
}

// rank chunks of a list of K rows: ceil(K / cap) balanced chunks of Nc rows
// (a multiple of 16, the MMA's N, at most cap <= 256), two half-tiles of Nc / 2
// rows each
struct ChunkGeom {
    int nch = 0, Nc = 0;
    int cols() const { return nch * Nc; }
};
inline ChunkGeom chunk_geom(int K, int cap) {
    ChunkGeom g;
    if (K <= 0) return g;
    g.nch = (K + cap - 1) / cap;
    g.Nc = ((K + g.nch - 1) / g.nch + 15) / 16 * 16;
    return g;
}

// FP64 rows of the dense blocks -> 16-bit planes, per-row inverse scale and h
template <bool BF16>
__global__ void dense_rows_kernel(int M, int r_pad, const double* __restrict__ rows,
                                  const double* __restrict__ hrow, uint16_t* __restrict__ hi,
                                  uint16_t* __restrict__ lo, float2* __restrict__ rowc) {
    __shared__ double red[32];
    const long row = blockIdx.x;
    const double* s = rows + row * M;
    double m = 0.0;
    for (int r = threadIdx.x; r < M; r += blockDim.x) m = fmax(m, fabs(s[r]));
    const double sc = pow2_scale(block_max(m, red));
    for (int r = threadIdx.x; r < r_pad; r += blockDim.x) {
        uint16_t h, l;
        split16<BF16>(r < M ? s[r] * sc : 0.0, h, l);
        hi[row * r_pad + r] = h;
        lo[row * r_pad + r] = l;
    }
    if (threadIdx.x == 0) rowc[row] = make_float2((float)(1.0 / sc), (float)hrow[row]);
}

// the same rows as TF32-rounded FP32 (one plane, rows of r_pad32 values)
__global__ void dense_rows_tf32_kernel(int M, int r_pad32, const double* __restrict__ rows,
                                       const double* __restrict__ hrow, float* __restrict__ out,
                                       float2* __restrict__ rowc) {
    __shared__ double red[32];
    const long row = blockIdx.x;
    const double* s = rows + row * M;
    double m = 0.0;
    for (int r = threadIdx.x; r < M; r += blockDim.x) m = fmax(m, fabs(s[r]));
    const double sc = pow2_scale(block_max(m, red));
    for (int r = threadIdx.x; r < r_pad32; r += blockDim.x)
        out[row * r_pad32 + r] = tf32_round(r < M ? (float)(s[r] * sc) : 0.f);
    if (threadIdx.x == 0) rowc[row] = make_float2((float)(1.0 / sc), (float)hrow[row]);
}

// TF32 Delta tiles [c][rb][kb] (128 walker rows x 32 basis functions, the
// 128-byte swizzled image) from the FP32 Delta copy: the copy's float4 of four
// consecutive s of row z is exactly the tile's 16-byte chunk of that row
__global__ void delta_tf32_tiles_kernel(int nrb, int Sd, int nkb32, const float4* __restrict__ dfull,
                                        float4* __restrict__ out) {
    const int tile = blockIdx.x;  // (c * nrb + rb) * nkb32 + kb
    const int kb = tile % nkb32, crb = tile / nkb32;
    const float4* src = dfull + ((size_t)crb * (Sd >> 2) + (size_t)kb * 8) * 128;
    float4* dst = out + (size_t)tile * 1024;
    for (int q = threadIdx.x; q < 1024; q += blockDim.x) {
        const int k4 = q >> 7, z = q & 127;
        float4 v = src[(size_t)k4 * 128 + z];
        v = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
        dst[z * 8 + (k4 ^ (z & 7))] = v;
    }
}

void release_lo(MixedOps& mx) {
    for (DevBuf* b : {&mx.U_hi, &mx.U_lo, &mx.V_hi, &mx.V_lo, &mx.row_c, &mx.pt, &mx.pair_pt0,
                      &mx.pair_npt, &mx.pair_w, &mx.e0, &mx.s_pt, &mx.s_pt0, &mx.s_npt, &mx.s_pw,
                      &mx.Ub_hi, &mx.Ub_lo, &mx.Vb_hi, &mx.Vb_lo, &mx.pt_J, &mx.row_cJ, &mx.e0_J,
                      &mx.pw_J, &mx.dpt, &mx.Yb_hi, &mx.Yb_lo, &mx.rowc_d, &mx.s_dpt})
        b->release();
    mx.lo_ready = false;
    mx.screen_built = -1;
    mx.h_tiles.clear(); mx.h_dtiles.clear(); mx.h_pt0.clear(); mx.h_npt.clear(); mx.h_order.clear();
    mx.h_pw.clear(); mx.h_e0.clear(); mx.h_dense.clear();
    mx.n_pt = mx.n_dpt = mx.n_pairs = mx.s_n_pt = mx.s_n_dpt = 0;
    mx.Sd = 0;
    mx.R = 0;
}

// LO operands.  dense_ok (mode LO): every pair whose dense truncated block
// (M + 1 rows in chunks) costs fewer MMA columns than its two factor sides is
// contracted densely (lo_dense_tc_kernel), the rest through its factors
// (lo_exchange_tc_kernel); the dense half-tiles come first in the pair lists.
// Without dense_ok (mode LO_JK) every pair goes through its factors, and the
// swapped lists of the compressed Coulomb are built too (closed shells).
void ensure_lo_ops(loaf_ctx* c, MixedOps& mx, bool bf16, bool tf32, bool dense_ok) {
    if (mx.lo_ready && mx.lo_dense_ok == dense_ok && mx.chunk_cap == c->tile_lo_cap) return;
    if (mx.lo_ready) release_lo(mx);
    mx.bf16 = bf16;
    mx.tf32 = tf32;
    mx.lo_dense_ok = dense_ok;
    const int cap = c->tile_lo_cap;
    mx.chunk_cap = cap;
    mx.r_pad = plane_pad(c->M, tf32);
    const int M = c->M;
    long R = 0;
    int npairs = 0;
    for (int s = 0; s < c->nspin; ++s) { R += c->sp[s].pairs.rows; npairs += c->sp[s].pairs.npairs; }
    mx.R = R;
    mx.n_pairs = npairs;
    const long Rb = std::max<long>(R, 1);
    if (!tf32) {  // the factor planes (TF32 contracts every pair densely)
        mx.U_hi.ensure((size_t)Rb * mx.r_pad * 2);
        mx.U_lo.ensure((size_t)Rb * mx.r_pad * 2);
        mx.V_hi.ensure((size_t)Rb * mx.r_pad * 2);
        mx.V_lo.ensure((size_t)Rb * mx.r_pad * 2);
        mx.row_c.ensure((size_t)Rb * sizeof(float4));
    }
    DevBuf inv_u, inv_v, pbuf, qbuf, pJ, qJ;
    inv_u.ensure(Rb * sizeof(float));
    inv_v.ensure(Rb * sizeof(float));
    pbuf.ensure(Rb * sizeof(double));
    qbuf.ensure(Rb * sizeof(double));
    // the compressed Coulomb is built for closed shells, with the factored plan
    const bool jk = c->nspin == 1 && !dense_ok;
    if (jk) {
        pJ.ensure(Rb * sizeof(double));
        qJ.ensure(Rb * sizeof(double));
        mx.e0_J.ensure(std::max(npairs, 1) * sizeof(double));
    }
    mx.e0.ensure(std::max(npairs, 1) * sizeof(double));
    mx.pair_w.ensure(std::max(npairs, 1) * sizeof(double));

    const int nkb = ceil_div(M, tf32 ? kTileK / 2 : kTileK);
    const ChunkGeom dg = chunk_geom(M + 1, cap);  // dense: the rows s of Ytil and g
    std::vector<double> pw;
    std::vector<int4> tiles, dtiles;
    std::vector<int> pt0(npairs), npt(npairs);
    std::vector<unsigned char> is_dense(npairs, 0);
    std::vector<long> prow(npairs);  // first packed factor row of each pair (both spins)
    std::vector<int> pspin(npairs), plocal(npairs);
    long row_base = 0;
    int pair_base = 0;
    for (int s = 0; s < c->nspin; ++s) {
        SpinData& sd = c->sp[s];
        PairTable& pt = sd.pairs;
        if (pt.rows > 0) {
            const size_t o = (size_t)row_base * mx.r_pad;
            if (tf32) {
                // no factor planes: every pair is contracted through its dense block
            } else if (bf16) {
                row_split_kernel<true><<<pt.rows, 128, 0, c->stream>>>(M, mx.r_pad, pt.d_U.as<double>(),
                    mx.U_hi.as<uint16_t>() + o, mx.U_lo.as<uint16_t>() + o, inv_u.as<float>() + row_base);
                row_split_kernel<true><<<pt.rows, 128, 0, c->stream>>>(M, mx.r_pad, pt.d_V.as<double>(),
                    mx.V_hi.as<uint16_t>() + o, mx.V_lo.as<uint16_t>() + o, inv_v.as<float>() + row_base);
            } else {
                row_split_kernel<false><<<pt.rows, 128, 0, c->stream>>>(M, mx.r_pad, pt.d_U.as<double>(),
                    mx.U_hi.as<uint16_t>() + o, mx.U_lo.as<uint16_t>() + o, inv_u.as<float>() + row_base);
                row_split_kernel<false><<<pt.rows, 128, 0, c->stream>>>(M, mx.r_pad, pt.d_V.as<double>(),
                    mx.V_hi.as<uint16_t>() + o, mx.V_lo.as<uint16_t>() + o, inv_v.as<float>() + row_base);
            }
            LOAF_LAUNCH_CHECK();
            // row -> pair map of this spin
            std::vector<int> row_pair(pt.rows);
            for (int n = 0; n < pt.npairs; ++n)
                for (int k = 0; k < pt.K[n]; ++k) row_pair[pt.off[n] + k] = n;
            DevBuf d_rp;
            d_rp.ensure(row_pair.size() * sizeof(int));
            LOAF_CUDA(cudaMemcpyAsync(d_rp.ptr, row_pair.data(), row_pair.size() * sizeof(int),
                                      cudaMemcpyHostToDevice, c->stream));
            pq_kernel<<<ceil_div(pt.rows, 8), 256, 0, c->stream>>>(
                M, pt.rows, pt.d_U.as<double>(), pt.d_V.as<double>(), d_rp.as<int>(),
                pt.d_i.as<int>(), pt.d_j.as<int>(), sd.d_trial.as<double>(), sd.N,
                pbuf.as<double>() + row_base, qbuf.as<double>() + row_base);
            LOAF_LAUNCH_CHECK();
            if (jk) {  // i and j exchanged: U row . Phi_i, V row . Phi_j
                pq_kernel<<<ceil_div(pt.rows, 8), 256, 0, c->stream>>>(
                    M, pt.rows, pt.d_U.as<double>(), pt.d_V.as<double>(), d_rp.as<int>(),
                    pt.d_j.as<int>(), pt.d_i.as<int>(), sd.d_trial.as<double>(), sd.N,
                    pJ.as<double>() + row_base, qJ.as<double>() + row_base);
                LOAF_LAUNCH_CHECK();
            }
            LOAF_CUDA(cudaStreamSynchronize(c->stream));  // d_rp goes out of scope
        }
        // e0 per pair (pair offsets are spin-local rows)
        {
            DevBuf d_off;
            d_off.ensure(std::max(pt.npairs, 1) * sizeof(long));
            std::vector<long> goff(pt.npairs);
            for (int n = 0; n < pt.npairs; ++n) goff[n] = pt.off[n] + row_base;
            LOAF_CUDA(cudaMemcpyAsync(d_off.ptr, goff.data(), goff.size() * sizeof(long),
                                      cudaMemcpyHostToDevice, c->stream));
            pair_e0_kernel<<<ceil_div(std::max(pt.npairs, 1), 128), 128, 0, c->stream>>>(
                pt.npairs, d_off.as<long>(), pt.d_K.as<int>(), pbuf.as<double>(),
                qbuf.as<double>(), mx.e0.as<double>() + pair_base);
            LOAF_LAUNCH_CHECK();
            if (jk) {
                pair_e0_kernel<<<ceil_div(std::max(pt.npairs, 1), 128), 128, 0, c->stream>>>(
                    pt.npairs, d_off.as<long>(), pt.d_K.as<int>(), pJ.as<double>(), qJ.as<double>(),
                    mx.e0_J.as<double>() + pair_base);
                LOAF_LAUNCH_CHECK();
            }
            LOAF_CUDA(cudaStreamSynchronize(c->stream));
        }
        for (int n = 0; n < pt.npairs; ++n) {
            const int g = pair_base + n;
            prow[g] = row_base + pt.off[n];
            pspin[g] = s;
            plocal[g] = n;
            const ChunkGeom fg = chunk_geom(pt.K[n], cap);
            is_dense[g] = fg.nch > 0 && (tf32 || (dense_ok && dg.cols() < 2 * fg.cols()));
            pw.push_back(0.5 * sd.mult * (pt.i[n] == pt.j[n] ? 1.0 : 2.0));
        }
        // pair order: 8 x 8 orbital blocks (pairs sharing orbitals run together)
        std::vector<int> order(pt.npairs);
        for (int n = 0; n < pt.npairs; ++n) order[n] = n;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const int ba = (pt.i[a] / 8) * 1024 + pt.j[a] / 8, bb = (pt.i[b] / 8) * 1024 + pt.j[b] / 8;
            return ba < bb;
        });
        for (int n : order) mx.h_order.push_back(pair_base + n);
        row_base += pt.rows;
        pair_base += pt.npairs;
    }
    // half-tile lists in pair order: dense chunks of the dense pairs, then the
    // factor chunks of the others; pair_pt0 indexes the two lists as one
    long woff = 0, doff = 0;  // tile elements so far (factored, dense)
    std::vector<int> dense_rank(npairs, -1);  // index among the dense pairs
    int n_dense_pairs = 0;
    for (int g : mx.h_order) {
        if (!is_dense[g]) continue;
        dense_rank[g] = n_dense_pairs++;
        const SpinData& sd = c->sp[pspin[g]];
        const PairTable& pt = sd.pairs;
        const int n = plocal[g];
        const unsigned ci = (unsigned)(sd.col0 + pt.i[n]), cj = (unsigned)(sd.col0 + pt.j[n]);
        pt0[g] = (int)dtiles.size();
        const int H = dg.Nc / 2, Kd = M + 1;
        for (int ch = 0; ch < dg.nch; ++ch)
            for (int hf = 0; hf < 2; ++hf) {
                const int r0 = ch * dg.Nc + hf * H;
                const int nv = std::max(0, std::min(H, Kd - r0));
                const long row0 = (long)dense_rank[g] * Kd + (nv > 0 ? r0 : 0);
                dtiles.push_back(make_int4((int)row0, nv | (H << 16),
                                           (int)((ci << 24) | (cj << 16) | (unsigned)(ch * dg.Nc)), (int)doff));
                doff += (long)H * kTileK * nkb;
            }
        npt[g] = 2 * dg.nch;
    }
    const int n_dpt = (int)dtiles.size();
    for (int g : mx.h_order) {
        if (is_dense[g]) continue;
        const SpinData& sd = c->sp[pspin[g]];
        const PairTable& pt = sd.pairs;
        const int n = plocal[g];
        pt0[g] = n_dpt + (int)tiles.size();
        int cnt = 0;
        const int cij = ((sd.col0 + pt.i[n]) << 16) | (sd.col0 + pt.j[n]);
        // the pair's ranks in balanced chunks of at most cap (the MMA's N, a
        // multiple of 16); each chunk is two half-tiles of H = N / 2 rows, one
        // per CTA of the pair, stored at element offset woff
        const int K = pt.K[n];
        const ChunkGeom fg = chunk_geom(K, cap);
        const int H = fg.Nc / 2;
        for (int ch = 0; ch < fg.nch; ++ch)
            for (int hf = 0; hf < 2; ++hf) {
                const int r0 = ch * fg.Nc + hf * H;
                const int nv = std::max(0, std::min(H, K - r0));
                tiles.push_back(make_int4((int)(prow[g] + (nv > 0 ? r0 : 0)), nv | (H << 16), cij, (int)woff));
                woff += (long)H * kTileK * nkb;
                ++cnt;
            }
        npt[g] = cnt;
    }
    if (R > 0 && !tf32) {
        row_consts_kernel<<<ceil_div(R, 256), 256, 0, c->stream>>>(R, inv_u.as<float>(), inv_v.as<float>(),
                                                                 pbuf.as<double>(), qbuf.as<double>(),
                                                                 mx.row_c.as<float4>());
        LOAF_LAUNCH_CHECK();
    }
    if (jk && R > 0) {
        mx.row_cJ.ensure((size_t)Rb * sizeof(float4));
        row_consts_kernel<<<ceil_div(R, 256), 256, 0, c->stream>>>(R, inv_u.as<float>(), inv_v.as<float>(),
                                                                 pJ.as<double>(), qJ.as<double>(),
                                                                 mx.row_cJ.as<float4>());
        LOAF_LAUNCH_CHECK();
    }
    mx.n_pt = (int)tiles.size();
    mx.n_dpt = n_dpt;
    mx.pt.ensure(std::max<size_t>(tiles.size(), 1) * sizeof(int4));
    mx.dpt.ensure(std::max<size_t>(dtiles.size(), 1) * sizeof(int4));
    mx.pair_pt0.ensure(std::max(npairs, 1) * sizeof(int));
    mx.pair_npt.ensure(std::max(npairs, 1) * sizeof(int));
    if (!tiles.empty())
        LOAF_CUDA(cudaMemcpyAsync(mx.pt.ptr, tiles.data(), tiles.size() * sizeof(int4),
                                  cudaMemcpyHostToDevice, c->stream));
    if (!dtiles.empty())
        LOAF_CUDA(cudaMemcpyAsync(mx.dpt.ptr, dtiles.data(), dtiles.size() * sizeof(int4),
                                  cudaMemcpyHostToDevice, c->stream));
    LOAF_CUDA(cudaMemcpyAsync(mx.pair_pt0.ptr, pt0.data(), npairs * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    LOAF_CUDA(cudaMemcpyAsync(mx.pair_npt.ptr, npt.data(), npairs * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    LOAF_CUDA(cudaMemcpyAsync(mx.pair_w.ptr, pw.data(), npairs * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    std::vector<double> e0(npairs);
    LOAF_CUDA(cudaMemcpyAsync(e0.data(), mx.e0.ptr, npairs * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LOAF_CUDA(cudaStreamSynchronize(c->stream));
    double ek0 = 0.0;
    for (int n = 0; n < npairs; ++n) ek0 += pw[n] * e0[n];
    mx.EK0 = ek0;
    if (jk) {
        // E_J = 2 sum_ij d_ij: weight 2 (diagonal) or 4; tiles with the orbitals exchanged
        std::vector<double> e0J(npairs), pwJ(npairs);
        if (npairs > 0)
            LOAF_CUDA(cudaMemcpyAsync(e0J.data(), mx.e0_J.ptr, npairs * sizeof(double), cudaMemcpyDeviceToHost,
                                      c->stream));
        std::vector<int4> tJ(tiles);
        for (int4& t : tJ) t.z = ((t.z & 0xffff) << 16) | (t.z >> 16);
        mx.pt_J.ensure(std::max<size_t>(tJ.size(), 1) * sizeof(int4));
        if (!tJ.empty())
            LOAF_CUDA(cudaMemcpyAsync(mx.pt_J.ptr, tJ.data(), tJ.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                      c->stream));
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
        const PairTable& pt0t = c->sp[0].pairs;
        double ej0 = 0.0;
        for (int n = 0; n < npairs; ++n) {
            pwJ[n] = pt0t.i[n] == pt0t.j[n] ? 2.0 : 4.0;
            ej0 += pwJ[n] * e0J[n];
        }
        mx.pw_J.ensure(std::max(npairs, 1) * sizeof(double));
        if (npairs > 0)
            LOAF_CUDA(cudaMemcpyAsync(mx.pw_J.ptr, pwJ.data(), npairs * sizeof(double), cudaMemcpyHostToDevice,
                                      c->stream));
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
        mx.EJ0 = ej0;
    }
    mx.h_tiles = tiles;
    mx.h_dtiles = dtiles;
    mx.h_pt0 = pt0;
    mx.h_npt = npt;
    mx.h_pw = pw;
    mx.h_e0 = e0;
    mx.h_dense = is_dense;
    mx.screen_built = -1;
    mx.nkb = nkb;
    LOAF_REQUIRE(woff < (1L << 31) && doff < (1L << 31), LOAF_ERR_SHAPE, "LO weight tiles beyond 2^31 elements");
    // factor tiles [tile][kb]
    if (mx.n_pt > 0) {
        const size_t tb = (size_t)woff * sizeof(uint16_t);
        const dim3 tg(mx.n_pt, mx.nkb);
        DevBuf* dst[4] = {&mx.Ub_hi, &mx.Ub_lo, &mx.Vb_hi, &mx.Vb_lo};
        DevBuf* src[4] = {&mx.U_hi, &mx.U_lo, &mx.V_hi, &mx.V_lo};
        for (int q = 0; q < 4; ++q) {
            dst[q]->ensure(tb);
            lo_tiles_kernel<<<tg, 256, 0, c->stream>>>(src[q]->as<uint16_t>(), mx.r_pad, mx.nkb,
                                                      mx.pt.as<int4>(), dst[q]->as<uint16_t>());
            LOAF_LAUNCH_CHECK();
        }
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
    }
    for (DevBuf* b : {&mx.U_hi, &mx.U_lo, &mx.V_hi, &mx.V_lo}) b->release();
    // dense blocks: Ytil = Ubar Vbar (rows s), g = Vbar^T p, h = Ubar q in FP64
    // (cuBLAS), split into 16-bit rows with per-row scales, then tiled
    // columns a chunk's epilogue may read, padded (TF32: the Delta tiles of
    // every call are cut from the FP32 copy as well, even without a dense pair)
    mx.Sd = dg.cols() + 32;
    if (n_dense_pairs > 0) {
        const int Kd = M + 1;
        mx.Yb_hi.ensure((size_t)doff * sizeof(uint16_t));
        if (!tf32) mx.Yb_lo.ensure((size_t)doff * sizeof(uint16_t));
        mx.rowc_d.ensure((size_t)n_dense_pairs * Kd * sizeof(float2));
        const int batch = std::max(1, std::min(n_dense_pairs, (int)((256L << 20) / ((long)Kd * M * 8))));
        DevBuf ytmp, htmp, plane_hi, plane_lo, btiles;
        ytmp.ensure((size_t)batch * Kd * M * sizeof(double));
        htmp.ensure((size_t)batch * Kd * sizeof(double));
        plane_hi.ensure((size_t)batch * Kd * mx.r_pad * 2);
        plane_lo.ensure((size_t)batch * Kd * mx.r_pad * 2);
        btiles.ensure((size_t)batch * 2 * dg.nch * sizeof(int4));
        std::vector<int> dense_pairs(n_dense_pairs);
        for (int g = 0; g < npairs; ++g)
            if (dense_rank[g] >= 0) dense_pairs[dense_rank[g]] = g;
        const double one = 1.0, zero = 0.0;
        LOAF_CUBLAS(cublasSetStream(c->cublas, c->stream));
        for (int b0 = 0; b0 < n_dense_pairs; b0 += batch) {
            const int nb = std::min(batch, n_dense_pairs - b0);
            LOAF_CUDA(cudaMemsetAsync(htmp.ptr, 0, (size_t)nb * Kd * sizeof(double), c->stream));
            std::vector<int4> bt;
            for (int b = 0; b < nb; ++b) {
                const int g = dense_pairs[b0 + b];
                const PairTable& pt = c->sp[pspin[g]].pairs;
                const int n = plocal[g], K = pt.K[n];
                const double* U = pt.d_U.as<double>() + (size_t)pt.off[n] * M;  // K rows of Ubar^T
                const double* V = pt.d_V.as<double>() + (size_t)pt.off[n] * M;  // K rows of Vbar
                double* Y = ytmp.as<double>() + (size_t)b * Kd * M;
                // Ytil[s][r] = sum_k U[k][s] V[k][r]: column-major V U^T
                LOAF_CUBLAS(cublasDgemm(c->cublas, CUBLAS_OP_N, CUBLAS_OP_T, M, M, K, &one, V, M, U, M,
                                        &zero, Y, M));
                // row M: g[r] = sum_k V[k][r] p[k];  h[s] = sum_k U[k][s] q[k]
                LOAF_CUBLAS(cublasDgemv(c->cublas, CUBLAS_OP_N, M, K, &one, V, M,
                                        pbuf.as<double>() + prow[g], 1, &zero, Y + (size_t)M * M, 1));
                LOAF_CUBLAS(cublasDgemv(c->cublas, CUBLAS_OP_N, M, K, &one, U, M,
                                        qbuf.as<double>() + prow[g], 1, &zero,
                                        htmp.as<double>() + (size_t)b * Kd, 1));
                for (int q = 0; q < 2 * dg.nch; ++q) {
                    int4 t = dtiles[mx.h_pt0[g] + q];
                    t.x -= b0 * Kd;  // row of the batch's plane
                    bt.push_back(t);
                }
            }
            const long rows = (long)nb * Kd;
            const size_t roff = (size_t)b0 * Kd;
            if (tf32)
                dense_rows_tf32_kernel<<<rows, 128, 0, c->stream>>>(M, mx.r_pad / 2, ytmp.as<double>(),
                    htmp.as<double>(), plane_hi.as<float>(), mx.rowc_d.as<float2>() + roff);
            else if (bf16)
                dense_rows_kernel<true><<<rows, 128, 0, c->stream>>>(M, mx.r_pad, ytmp.as<double>(), htmp.as<double>(),
                    plane_hi.as<uint16_t>(), plane_lo.as<uint16_t>(), mx.rowc_d.as<float2>() + roff);
            else
                dense_rows_kernel<false><<<rows, 128, 0, c->stream>>>(M, mx.r_pad, ytmp.as<double>(), htmp.as<double>(),
                    plane_hi.as<uint16_t>(), plane_lo.as<uint16_t>(), mx.rowc_d.as<float2>() + roff);
            LOAF_LAUNCH_CHECK();
            LOAF_CUDA(cudaMemcpyAsync(btiles.ptr, bt.data(), bt.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                      c->stream));
            const dim3 tg((unsigned)bt.size(), mx.nkb);
            lo_tiles_kernel<<<tg, 256, 0, c->stream>>>(plane_hi.as<uint16_t>(), mx.r_pad, mx.nkb,
                                                      btiles.as<int4>(), mx.Yb_hi.as<uint16_t>());
            if (!tf32)
                lo_tiles_kernel<<<tg, 256, 0, c->stream>>>(plane_lo.as<uint16_t>(), mx.r_pad, mx.nkb,
                                                          btiles.as<int4>(), mx.Yb_lo.as<uint16_t>());
            LOAF_LAUNCH_CHECK();
            LOAF_CUDA(cudaStreamSynchronize(c->stream));  // bt and the batch buffers are reused
        }
    }
    mx.lo_ready = true;
}

// Tile lists restricted to the pairs the screen keeps (same order as the full
// lists, dense half-tiles first); a dropped pair loses both its walker part
// and its trial part e0.
void ensure_screened_tiles(loaf_ctx* c, MixedOps& mx) {
    if (mx.screen_built == c->screen_version) return;
    const int npairs = mx.n_pairs;
    std::vector<int4> tiles, dtiles;
    std::vector<int> pt0(npairs, 0), npt(npairs, 0);
    std::vector<double> pw(npairs, 0.0);
    double ek0 = 0.0;
    auto kept = [&](int g) { return c->keep.empty() || c->keep[g]; };
    for (int g : mx.h_order) {
        if (!mx.h_dense[g] || !kept(g)) continue;
        pt0[g] = (int)dtiles.size();
        for (int t = 0; t < mx.h_npt[g]; ++t) dtiles.push_back(mx.h_dtiles[mx.h_pt0[g] + t]);
        npt[g] = mx.h_npt[g];
        pw[g] = mx.h_pw[g];
    }
    const int nd = (int)dtiles.size();
    for (int g : mx.h_order) {
        if (mx.h_dense[g] || !kept(g)) continue;
        pt0[g] = nd + (int)tiles.size();
        for (int t = 0; t < mx.h_npt[g]; ++t) tiles.push_back(mx.h_tiles[mx.h_pt0[g] - mx.n_dpt + t]);
        npt[g] = mx.h_npt[g];
        pw[g] = mx.h_pw[g];
    }
    for (int g = 0; g < npairs; ++g) ek0 += pw[g] * mx.h_e0[g];  // same order as the full list
    mx.s_n_pt = (int)tiles.size();
    mx.s_n_dpt = nd;
    mx.s_pt.ensure(std::max<size_t>(tiles.size(), 1) * sizeof(int4));
    mx.s_dpt.ensure(std::max<size_t>(dtiles.size(), 1) * sizeof(int4));
    mx.s_pt0.ensure(std::max(npairs, 1) * sizeof(int));
    mx.s_npt.ensure(std::max(npairs, 1) * sizeof(int));
    mx.s_pw.ensure(std::max(npairs, 1) * sizeof(double));
    if (!tiles.empty())
        LOAF_CUDA(cudaMemcpyAsync(mx.s_pt.ptr, tiles.data(), tiles.size() * sizeof(int4),
                                  cudaMemcpyHostToDevice, c->stream));
    if (!dtiles.empty())
        LOAF_CUDA(cudaMemcpyAsync(mx.s_dpt.ptr, dtiles.data(), dtiles.size() * sizeof(int4),
                                  cudaMemcpyHostToDevice, c->stream));
    LOAF_CUDA(cudaMemcpyAsync(mx.s_pt0.ptr, pt0.data(), npairs * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    LOAF_CUDA(cudaMemcpyAsync(mx.s_npt.ptr, npt.data(), npairs * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    LOAF_CUDA(cudaMemcpyAsync(mx.s_pw.ptr, pw.data(), npairs * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    LOAF_CUDA(cudaStreamSynchronize(c->stream));
    mx.s_EK0 = ek0;
    mx.screen_built = c->screen_version;
}

constexpr size_t kCoulSmem =
    kCStages * 4 * kTileBytes + 32 * kCEpiWarps * 32 * sizeof(float) + 1024;
constexpr size_t kLoSmem = kLSlots * kLSlotBytes + 1024;
constexpr size_t kCoulPairSmem =
    kCPStages * kCPStageBytes + 32 * kCEpiWarps * 32 * sizeof(float) + 1024;

// CTA pairs of a cluster kernel that fit on the GPU at once
int max_pair_clusters(const void* kernel, int threads, size_t smem, int sm_count) {
    LOAF_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * (sm_count / 2));
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    LOAF_CUDA(cudaOccupancyMaxActiveClusters(&n, kernel, &cfg));
    return n;
}

int coul_max_clusters(loaf_ctx* c) {
    static int cached[64] = {0};
    int dev = 0;
    LOAF_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && cached[dev] > 0) return cached[dev];
    const int n = max_pair_clusters((const void*)coulomb_tc_pair_kernel<false>, kCThreads, kCoulPairSmem, c->sm_count);
    LOAF_REQUIRE(n > 0, LOAF_ERR_CUDA, "the Coulomb kernel's CTA pair does not fit on an SM pair");
    if (dev < 64) cached[dev] = n;
    return n;
}

// k-splits of a contraction with `tiles` output tiles dealt round-robin to
// `slots` persistent workers: the fewest that fill the last round to >= 90 %
// (the split fixes the FP32 chain boundaries, so slots must not depend on an
// SM budget)
int wave_splits(int tiles, int max_split, int slots) {
    int best = 1;
    double best_eff = 0.0;
    for (int sp = 1; sp <= max_split; ++sp) {
        const long units = (long)tiles * sp;
        const long rounds = (units + slots - 1) / slots;
        const double eff = (double)units / (double)(rounds * slots);
        if (units >= slots && eff >= 0.9) return sp;
        if (eff > best_eff + 1e-12) { best_eff = eff; best = sp; }
    }
    return best;
}

// the largest Coulomb k-split: at least 64 k-chunks (32 chains) per unit, since
// every unit ends in an FP64 write of its partial sums, whose cost does not
// shrink with the unit
int coul_max_split(int nk, bool tf32) { return std::max(1, std::min(16, nk / (tf32 ? 128 : 64))); }

// CTA pairs of the LO kernel that fit on the GPU at once (the persistent grid):
// clusters sit inside a GPC, so this can be below half the SM count
int lo_max_clusters(loaf_ctx* c) {
    static int cached[64] = {0};
    int dev = 0;
    LOAF_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && cached[dev] > 0) return cached[dev];
    LOAF_CUDA(cudaFuncSetAttribute(lo_exchange_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kLoSmem));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * (c->sm_count / 2));
    cfg.blockDim = dim3(kLThreads);
    cfg.dynamicSmemBytes = kLoSmem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    LOAF_CUDA(cudaOccupancyMaxActiveClusters(&n, lo_exchange_tc_kernel, &cfg));
    LOAF_REQUIRE(n > 0, LOAF_ERR_CUDA, "the LO exchange kernel's CTA pair does not fit on an SM pair");
    if (dev < 64) cached[dev] = n;
    return n;
}

int lo_dense_max_clusters(loaf_ctx* c) {
    static int cached[64] = {0};
    int dev = 0;
    LOAF_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && cached[dev] > 0) return cached[dev];
    const int n = max_pair_clusters((const void*)lo_dense_tc_kernel<false>, kLThreads, kLoSmem, c->sm_count);
    LOAF_REQUIRE(n > 0, LOAF_ERR_CUDA, "the dense LO kernel's CTA pair does not fit on an SM pair");
    if (dev < 64) cached[dev] = n;
    return n;
}

// One-body energy and Coulomb on the tensor cores from the Delta tiles of
// this batch: e_out[0..W) = E1, e_out[W..2W) = E_J; j_out (optional, W x X)
// receives <L_g>_w = sum_sigma tr(Lbar^sigma_g Theta^sigma).
void coulomb_mixed(loaf_ctx* c, MixedOps& mx, int W, bool bf16, const float* inv_t, int* err,
                   double2* e_out, double2* j_out) {
    const DeltaGeom dg = delta_geom(c->M, c->ntot, W);
    // ---- Coulomb + one-body on the tensor cores ----
    CoulParams P;
    P.out = nullptr;
    P.wt_fast = 0;
    // TF32: one plane of operand tiles and the TF32 Delta tiles, 32-wide blocks
    P.a_hi = mx.Lb_hi.as<uint16_t>();
    P.a_lo = mx.tf32 ? nullptr : mx.Lb_lo.as<uint16_t>();
    P.b_hi = mx.tf32 ? c->w_dtf.as<uint16_t>() : c->w_dhi.as<uint16_t>();
    P.b_lo = mx.tf32 ? nullptr : c->w_dlo.as<uint16_t>();
    P.nkb = mx.tf32 ? mx.nkb : dg.nkb;
    P.nrb = dg.nrb;
    P.rows = c->X + 1;
    P.n_mt = (mx.n_mt + 1) & ~1;  // row-tile pairs (the padding tile is zeros)
    P.n_wt = ceil_div(2L * W, kCBN);
    P.nk = c->ntot * P.nkb;
    const int tiles = (P.n_mt / 2) * P.n_wt;
    // the split fixes the chain boundaries of the FP32 accumulation, so it depends
    // on the device and the context's tile shapes only (not on an SM budget):
    // results do not depend on scheduling
    P.n_split = c->tile_coul_split > 0 ? std::min(c->tile_coul_split, P.nk)
                                        : wave_splits(tiles, coul_max_split(P.nk, mx.tf32), c->sm_count / 2);
    P.ldp = P.n_wt * kCBN;
    // pair MMA: M = 256, N = 128
    P.idesc = mx.tf32 ? tc::idesc_tf32(2 * kBM, kCBN) : tc::idesc_f16(2 * kBM, kCBN, bf16);
    P.err = err;
    c->w_cpart.ensure((size_t)P.n_split * P.rows * P.ldp * sizeof(double));
    P.part = c->w_cpart.as<double>();
    const int units = tiles * P.n_split;
    const int n_cl = std::max(1, std::min({units, coul_max_clusters(c), c->persistent_grid() / 2}));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * n_cl);
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = kCoulPairSmem;
    cfg.stream = c->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    StageScope csc(c, "coulomb_tc", 1);
    if (mx.tf32) {
        LOAF_CUDA(cudaFuncSetAttribute(coulomb_tc_pair_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kCoulPairSmem));
        LOAF_CUDA(cudaLaunchKernelEx(&cfg, coulomb_tc_pair_kernel<true>, P));
    } else {
        LOAF_CUDA(cudaLaunchKernelEx(&cfg, coulomb_tc_pair_kernel<false>, P));
    }
    LOAF_LAUNCH_CHECK();
    csc.end();
    StageScope rsc(c, "coulomb_reduce", 2);
    c->w_red.ensure((size_t)kRedSlices * W * sizeof(double2));
    coulomb_tc_reduce_kernel<<<dim3(ceil_div(W, 32), kRedSlices), 256, 0, c->stream>>>(
        c->X, W, P.n_split, P.ldp, P.part, mx.L_inv.as<float>(), inv_t, mx.J0.as<double>(),
        c->w_red.as<double2>(), j_out);
    LOAF_LAUNCH_CHECK();
    coulomb_tc_final_kernel<<<ceil_div(W, 128), 128, 0, c->stream>>>(
        c->X, W, P.n_split, P.ldp, kRedSlices, P.part, mx.L_inv.as<float>(), inv_t, mx.E1_0,
        c->w_red.as<double2>(), e_out, e_out + W);
    LOAF_LAUNCH_CHECK();
}

}  // namespace

void tc_split_gemm(loaf_ctx* c, const uint16_t* a_hi, const uint16_t* a_lo, int rows, int n_mt,
                   const uint16_t* b_hi, const uint16_t* b_lo, int nrb, int n_wt, int nkb, bool bf16,
                   double* part, int ldp, int* err, double2* out, const float* inv_row,
                   const float* inv_col, long out_ld, int out_W) {
    CoulParams P;
    P.out = out;
    P.inv_row = inv_row;
    P.inv_col = inv_col;
    P.out_ld = out_ld;
    P.out_W = out_W;
    P.wt_fast = 1;  // the row operand (rows x K) is the large one
    P.a_hi = a_hi;
    P.a_lo = a_lo;
    P.b_hi = b_hi;
    P.b_lo = b_lo;
    P.nkb = nkb;
    P.nrb = nrb;
    P.rows = rows;
    P.n_mt = n_mt;
    P.n_wt = n_wt;
    P.nk = nkb;  // one orbital block: K = nkb tiles of 64
    P.n_split = 1;
    P.ldp = ldp;
    P.idesc = tc::idesc_f16(kBM, kCBN, bf16);
    P.err = err;
    P.part = part;
    LOAF_CUDA(cudaFuncSetAttribute(coulomb_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kCoulSmem));
    coulomb_tc_kernel<<<std::min(n_mt * n_wt, c->persistent_grid()), kCThreads, kCoulSmem, c->stream>>>(P);
    LOAF_LAUNCH_CHECK();
}

void run_force_bias_mixed(loaf_ctx* c, int W, int precision, double2* e_scratch, double2* j_out) {
    const bool bf16 = precision == LOAF_PREC_BF16X3;
    MixedOps& mx = c->mix[mix_slot(precision)];
    ensure_coulomb_ops(c, mx, bf16, false);
    float* inv_t = c->w_dscale.as<float>();
    c->w_flag.ensure(16);
    coulomb_mixed(c, mx, W, bf16, inv_t, c->w_flag.as<int>(), e_scratch, j_out);
}

void setup_mixed_operands(loaf_ctx* c, int mode, bool bf16) {
    MixedOps& mx = c->mix[bf16 ? 1 : 0];
    ensure_coulomb_ops(c, mx, bf16, false);
    if (mode != LOAF_MODE_FULL) ensure_lo_ops(c, mx, bf16, false, mode == LOAF_MODE_LO);
}

// the k-split rule for W walkers once the Coulomb operands exist (0 before)
int coulomb_split_rule(loaf_ctx* c, int W, int precision) {
    const MixedOps& mx = c->mix[mix_slot(precision)];
    if (!mx.coul_ready) return 0;
    const DeltaGeom dg = delta_geom(c->M, c->ntot, W);
    const int nk = c->ntot * (mx.tf32 ? mx.nkb : dg.nkb);
    const int tiles = (((mx.n_mt + 1) & ~1) / 2) * ceil_div(2L * W, kCBN);
    return wave_splits(tiles, coul_max_split(nk, mx.tf32), c->sm_count / 2);
}

int prepare_lo_operands(loaf_ctx* c, int mode, int precision) {
    if (mode == LOAF_MODE_FULL || precision == LOAF_PREC_FP64) return 0;
    const bool bf16 = precision == LOAF_PREC_BF16X3, tf32 = precision == LOAF_PREC_TF32;
    MixedOps& mx = c->mix[mix_slot(precision)];
    ensure_lo_ops(c, mx, bf16, tf32, mode == LOAF_MODE_LO);
    // TF32 cuts its Delta tiles from the FP32 copy, dense pairs or not
    return (mx.n_dpt > 0 || tf32) ? mx.Sd : 0;
}

void run_energy_mixed(loaf_ctx* c, int W, int mode, int precision, const double2* theta,
                      double2* e_out, double2* e_pairs) {
    const bool bf16 = precision == LOAF_PREC_BF16X3, tf32 = precision == LOAF_PREC_TF32;
    MixedOps& mx = c->mix[mix_slot(precision)];
    if (e_out) ensure_coulomb_ops(c, mx, bf16, tf32);
    if (mode != LOAF_MODE_FULL) ensure_lo_ops(c, mx, bf16, tf32, mode == LOAF_MODE_LO);

    // Delta planes for this batch: formed here from an FP64 Theta, or already
    // written by the tensor-core Theta stage when theta is NULL
    const int n_wt = ceil_div(W, kBNW);
    const int Wpad = n_wt * kBNW;
    const DeltaGeom dg = delta_geom(c->M, c->ntot, W);
    c->w_dscale.ensure((size_t)W * (sizeof(float) + sizeof(double)) + 64);
    float* inv_t = c->w_dscale.as<float>();
    double* scale = reinterpret_cast<double*>(c->w_dscale.as<uint8_t>() + ((W * sizeof(float) + 15) / 16) * 16);
    c->w_flag.ensure(16);
    int* err = c->w_flag.as<int>();
    if (theta) {
        c->w_dhi.ensure_zeroed(dg.plane * 2, c->stream);
        c->w_dlo.ensure_zeroed(dg.plane * 2, c->stream);
        LOAF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
        SpinRef s0 = spin_ref(c->sp[0]), s1 = c->nspin > 1 ? spin_ref(c->sp[1]) : s0;
        StageScope dsc(c, "delta_split", 2);
        delta_max_kernel<<<W, 256, 0, c->stream>>>(c->M, c->ntot, c->nspin, s0, s1, theta, inv_t, scale);
        LOAF_LAUNCH_CHECK();
        if (bf16)
            delta_split_kernel<true><<<W * c->ntot, 128, 0, c->stream>>>(c->M, c->ntot, dg.nrb, dg.nkb,
                c->nspin, s0, s1, theta, scale, c->w_dhi.as<uint16_t>(), c->w_dlo.as<uint16_t>());
        else
            delta_split_kernel<false><<<W * c->ntot, 128, 0, c->stream>>>(c->M, c->ntot, dg.nrb, dg.nkb,
                c->nspin, s0, s1, theta, scale, c->w_dhi.as<uint16_t>(), c->w_dlo.as<uint16_t>());
        LOAF_LAUNCH_CHECK();
    }
    // pair MMA: M = 256; N is set per unit from the chunk's rank count
    const uint32_t idesc = tf32 ? tc::idesc_tf32(2 * kBM, kBN) : tc::idesc_f16(2 * kBM, kBN, bf16);
    if (tf32) {
        // TF32 Delta tiles of 32-wide basis blocks, cut from the FP32 copy the
        // Theta stage wrote
        LOAF_REQUIRE(theta == nullptr, LOAF_ERR_UNSUPPORTED, "the TF32 precision needs the tensor-core Theta stage");
        const size_t n_tiles = (size_t)c->ntot * dg.nrb * mx.nkb;
        c->w_dtf.ensure(n_tiles * kTileBytes);
        StageScope tsc(c, "delta_tf32", 1);
        delta_tf32_tiles_kernel<<<(unsigned)n_tiles, 256, 0, c->stream>>>(
            dg.nrb, mx.Sd, mx.nkb, c->w_dfull.as<float4>(), c->w_dtf.as<float4>());
        LOAF_LAUNCH_CHECK();
    }

    if (e_out) coulomb_mixed(c, mx, W, bf16, inv_t, err, e_out, nullptr);
    if (mode != LOAF_MODE_FULL) {
        // ---- LO pair exchange on the tensor cores ----
        double2* ek = e_out ? e_out + 2 * W : nullptr;
        // energies honour the pair screen; pair values are always for every pair
        const bool screened = !c->keep.empty() && e_pairs == nullptr;
        if (screened) ensure_screened_tiles(c, mx);
        const int n_pt = screened ? mx.s_n_pt : mx.n_pt;
        const int n_dpt = screened ? mx.s_n_dpt : mx.n_dpt;
        const int4* tile_list = screened ? mx.s_pt.as<int4>() : mx.pt.as<int4>();
        const int4* dense_list = screened ? mx.s_dpt.as<int4>() : mx.dpt.as<int4>();
        const int* list_pt0 = screened ? mx.s_pt0.as<int>() : mx.pair_pt0.as<int>();
        const int* list_npt = screened ? mx.s_npt.as<int>() : mx.pair_npt.as<int>();
        const double* list_pw = screened ? mx.s_pw.as<double>() : mx.pair_w.as<double>();
        const double list_ek0 = screened ? mx.s_EK0 : mx.EK0;
        // partial sums per chunk and walker: the dense chunks first, then the factored
        c->w_lopart.ensure((size_t)std::max(n_pt + n_dpt, 2) / 2 * Wpad * sizeof(double2));
        auto take_withhold = [&] {
            if (c->test_withhold <= 0) return 0;
            --c->test_withhold;
            return 1;
        };
        auto cluster_cfg = [&](int n_cl) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(2 * n_cl);
            cfg.blockDim = dim3(kLThreads);
            cfg.dynamicSmemBytes = kLoSmem;
            cfg.stream = c->stream;
            return cfg;
        };
        cudaLaunchAttribute cl_attr[1];
        cl_attr[0].id = cudaLaunchAttributeClusterDimension;
        cl_attr[0].val.clusterDim.x = 2;
        cl_attr[0].val.clusterDim.y = 1;
        cl_attr[0].val.clusterDim.z = 1;
        // the dense kernel over its half-tile list (partial rows 0 .. n_dpt / 2)
        if (n_dpt > 0) {
            LoDenseParams P;
            P.y_hi = mx.Yb_hi.as<uint16_t>();
            P.y_lo = tf32 ? nullptr : mx.Yb_lo.as<uint16_t>();
            P.d_hi = tf32 ? c->w_dtf.as<uint16_t>() : c->w_dhi.as<uint16_t>();
            P.d_lo = tf32 ? nullptr : c->w_dlo.as<uint16_t>();
            P.dfull = c->w_dfull.as<float>();
            P.nrb = dg.nrb;
            P.Sd = mx.Sd;
            P.pt = dense_list;
            P.rowc = mx.rowc_d.as<float2>();
            P.inv_t = inv_t;
            P.part = c->w_lopart.as<double2>();
            P.n_pt = n_dpt;
            P.n_wt = n_wt;
            P.W = W;
            P.ldp = Wpad;
            P.nk = tf32 ? mx.nkb : dg.nkb;
            P.M = c->M;
            P.idesc = idesc;
            P.err = err;
            P.withhold = take_withhold();
            const int units = (n_dpt / 2) * n_wt;
            const int n_cl = std::max(1, std::min({units, lo_dense_max_clusters(c), c->persistent_grid() / 2}));
            cudaLaunchConfig_t cfg = cluster_cfg(n_cl);
            cfg.attrs = cl_attr;
            cfg.numAttrs = 1;
            StageScope dsc(c, "lo_dense_tc", 1);
            if (tf32) {
                LOAF_CUDA(cudaFuncSetAttribute(lo_dense_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kLoSmem));
                LOAF_CUDA(cudaLaunchKernelEx(&cfg, lo_dense_tc_kernel<true>, P));
            } else {
                LOAF_CUDA(cudaLaunchKernelEx(&cfg, lo_dense_tc_kernel<false>, P));
            }
            LOAF_LAUNCH_CHECK();
        }
        // one launch of the factored CTA-pair kernel over a tile list with its
        // row constants, writing partial rows from part_row0
        auto launch_lo = [&](const int4* tiles, int ntiles, const float4* rowc, const char* stage,
                             int part_row0) {
            if (ntiles <= 0) return;
            LoParams P;
            P.u_hi = mx.Ub_hi.as<uint16_t>();
            P.u_lo = mx.Ub_lo.as<uint16_t>();
            P.v_hi = mx.Vb_hi.as<uint16_t>();
            P.v_lo = mx.Vb_lo.as<uint16_t>();
            P.d_hi = c->w_dhi.as<uint16_t>();
            P.d_lo = c->w_dlo.as<uint16_t>();
            P.nrb = dg.nrb;
            P.pt = tiles;
            P.rowc = rowc;
            P.inv_t = inv_t;
            P.n_pt = ntiles;
            P.n_wt = n_wt;
            P.W = W;
            P.ldp = Wpad;
            P.nk = dg.nkb;
            P.idesc = idesc;
            P.err = err;
            P.withhold = take_withhold();
            P.part = c->w_lopart.as<double2>() + (size_t)part_row0 * Wpad;
            const int units = (ntiles / 2) * n_wt;
            const int n_cl = std::max(1, std::min({units, lo_max_clusters(c), c->persistent_grid() / 2}));
            cudaLaunchConfig_t cfg = cluster_cfg(n_cl);
            cfg.attrs = cl_attr;
            cfg.numAttrs = 1;
            StageScope lsc(c, stage, 1);
            LOAF_CUDA(cudaLaunchKernelEx(&cfg, lo_exchange_tc_kernel, P));
            LOAF_LAUNCH_CHECK();
        };
        launch_lo(tile_list, n_pt, mx.row_c.as<float4>(), "lo_exchange_tc", n_dpt / 2);
        StageScope lrs(c, "lo_reduce", ek ? 2 : 1);
        const int nsl = std::max(1, std::min(kRedSlices, mx.n_pairs));
        c->w_red.ensure((size_t)kRedSlices * W * sizeof(double2));
        lo_tc_reduce_kernel<<<dim3(ceil_div(W, 32), nsl), 256, 0, c->stream>>>(
            mx.n_pairs, W, Wpad, list_pt0, list_npt, list_pw, mx.e0.as<double>(),
            c->w_lopart.as<double2>(), c->w_red.as<double2>(), e_pairs);
        LOAF_LAUNCH_CHECK();
        if (ek) {
            lo_tc_final_kernel<<<ceil_div(W, 128), 128, 0, c->stream>>>(W, nsl, list_ek0,
                                                                      c->w_red.as<double2>(), ek);
            LOAF_LAUNCH_CHECK();
        }
        lrs.end();
        if (mode == LOAF_MODE_LO_JK && e_out) {
            // E_J from the compressed factors replaces the exact Coulomb term:
            // the pair's orbitals exchanged, every pair (the screen is for exchange)
            launch_lo(mx.pt_J.as<int4>(), mx.n_pt, mx.row_cJ.as<float4>(), "lo_coulomb_tc", 0);
            StageScope jrs(c, "lo_coulomb_reduce", 2);
            lo_tc_reduce_kernel<<<dim3(ceil_div(W, 32), nsl), 256, 0, c->stream>>>(
                mx.n_pairs, W, Wpad, mx.pair_pt0.as<int>(), mx.pair_npt.as<int>(), mx.pw_J.as<double>(),
                mx.e0_J.as<double>(), c->w_lopart.as<double2>(), c->w_red.as<double2>(), nullptr);
            LOAF_LAUNCH_CHECK();
            lo_tc_final_kernel<<<ceil_div(W, 128), 128, 0, c->stream>>>(W, nsl, mx.EJ0, c->w_red.as<double2>(),
                                                                      e_out + W);
            LOAF_LAUNCH_CHECK();
        }
    } else if (e_out) {
        // full mode: Coulomb on the tensor cores, exchange in FP64
        StageScope fsc(c, "exchange_full_fp64", c->nspin + 1);
        run_energy_fp64_full(c, W, theta, e_out + 2 * W);
    }
}

}  // namespace loaf
