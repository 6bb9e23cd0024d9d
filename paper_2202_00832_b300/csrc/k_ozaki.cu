// Theta on the tensor cores with exact integer slices (split-precision path).
//
// The overlap S = Phi_T^T phi and Theta = phi S^-1 (eq. Q) need close to FP64
// accuracy: Delta = Theta - Phi_T is a small difference of O(1) numbers.  B300
// runs FP64 at ~1 TFLOP/s, so the two M N^2-sized products run on the FP16
// tensor cores instead, error-free:
//   every operand row (or column) is scaled by a power of two into [-1/4, 1/4]
//   and written as six balanced base-128 digits d_s in [-64, 63]
//   (x = sum_s d_s 2^-7s, 42 bits); digits are exact in FP16;
//   a digit product is at most 2^12 and the sums below stay under 2^24, so the
//   FP32 tensor-core accumulation is exact;
//   products with s + t = D (D = 2..7, 21 products per k-step) accumulate into
//   one of six TMEM accumulators and are combined exactly in int64:
//   value = 2^(e_row + e_col - 49) * sum_D acc_D * 2^(7 (7 - D)).
// Omitting s + t >= 8 leaves an error near 2^-49 of the operands' scale.
// Only the O(N^3) part -- Gauss-Jordan inversion of S with partial pivoting
// and the log-determinant -- runs on the CUDA cores, in double-float (pairs of
// FP32 numbers) with the log-determinant summed in FP64 (one CTA per walker
// and spin).
//
// Stages per spin: slice phi (two layouts) -> S GEMM (A = phi slices,
// B = Phi_T^T slices: S^T) -> Gauss-Jordan (Z = S^-1, log det, Z slices) -> Delta scale
// -> Theta GEMM (A = phi slices, B = Z slices) whose epilogue writes
// Delta = Theta - Phi_T as the 16-bit hi/lo planes the Coulomb and LO kernels read.
#include "common.cuh"
#include "tc_ptx.cuh"
#include "dfloat.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

namespace loaf {

namespace {

constexpr int kNS = 6;          // digit slices
constexpr int kND = 6;          // accumulated diagonals D = s + t = 2..7
constexpr int kOBK = 32;        // K per stage (64-byte rows, SWIZZLE_64B)
constexpr int kOBM = 128;
constexpr int kOBN = 80;
constexpr int kOStages = 2;
constexpr uint32_t kOTileA = kOBM * 64;              // 8 KB
constexpr uint32_t kOTileB = kOBN * 64;              // 5 KB
constexpr uint32_t kOStage = kNS * (kOTileA + kOTileB);  // 78 KB
// S GEMM, MN-major A tile (two 64-row boxes of 32 k-rows of 128 bytes): bytes
// between the 64-row blocks and between groups of 8 k-rows
constexpr uint32_t kMnLbo = kOTileA / 2, kMnSbo = 8 * 128;
constexpr size_t kOSmem = kOStages * kOStage + 1024;

PFN_cuTensorMapEncodeTiled_v12000 encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        LOAF_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                   cudaEnableDefault, &q));
        LOAF_REQUIRE(p && q == cudaDriverEntryPointSuccess, LOAF_ERR_CUDA,
                     "cuTensorMapEncodeTiled is unavailable");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// walker slices At[slice][p][w][kpad] as the MN-major A operand of the S GEMM:
// x = row (w, 2j + ri) (extent W kpad), y = k = p (extent M), z = 1, w = slice;
// boxes of 64 rows x 32 k with the 128-byte swizzle
void map_slices_mn(CUtensorMap* m, const void* base, uint64_t rows, uint64_t k) {
    cuuint64_t dims[4] = {rows, k, 1, (cuuint64_t)kNS};
    cuuint64_t strides[3] = {rows * 2, rows * k * 2, rows * k * 2};
    cuuint32_t box[4] = {64, (cuuint32_t)kOBK, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = encode()(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void*>(base), dims,
                          strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    LOAF_REQUIRE(r == CUDA_SUCCESS, LOAF_ERR_CUDA, "cuTensorMapEncodeTiled (MN-major slices) failed");
}

// walker slices At[slice][p][w][kpad] as the K-major A operand of the Theta GEMM:
// x = K = 2j + ri (extent 2N), y = walker, z = row p (extent M), w = slice;
// boxes of 32 k x 1 walker x 128 rows with the 64-byte swizzle
void map_slices_rows(CUtensorMap* m, const void* base, uint64_t k, uint64_t kpad, uint64_t W, uint64_t M) {
    cuuint64_t dims[4] = {k, W, M, (cuuint64_t)kNS};
    cuuint64_t strides[3] = {kpad * 2, kpad * W * 2, kpad * W * M * 2};
    cuuint32_t box[4] = {(cuuint32_t)kOBK, 1, (cuuint32_t)kOBM, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = encode()(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void*>(base), dims,
                          strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    LOAF_REQUIRE(r == CUDA_SUCCESS, LOAF_ERR_CUDA, "cuTensorMapEncodeTiled (row slices) failed");
}

// 16-bit slices [slice][batch][rows][ld]: x = K (extent k), y = row, z = batch, w = slice
void map_slices(CUtensorMap* m, const void* base, uint64_t k, uint64_t ld, uint64_t rows,
                uint64_t batch, uint32_t box_rows) {
    cuuint64_t dims[4] = {k, rows, batch, (cuuint64_t)kNS};
    cuuint64_t strides[3] = {ld * 2, ld * rows * 2, ld * rows * batch * 2};
    cuuint32_t box[4] = {(cuuint32_t)kOBK, box_rows, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = encode()(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void*>(base), dims,
                          strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    LOAF_REQUIRE(r == CUDA_SUCCESS, LOAF_ERR_CUDA, "cuTensorMapEncodeTiled (slices) failed");
}

// smallest E with max|v| <= 2^(E-2)  (0 for an all-zero set)
__device__ inline int slice_exponent(double maxabs) {
    if (!(maxabs > 0.0)) return 0;
    int e;
    frexp(maxabs, &e);  // maxabs < 2^e
    return e + 2;
}

// 2^e as a double from its bit pattern (|e| < 1000)
__device__ inline double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// 2^e as a float (e clamped to the normal range)
__device__ inline float pow2f(int e) { return __int_as_float((min(max(e, -126), 127) + 127) << 23); }

// round(v 2^s) for a double v, from its bit pattern with integer arithmetic
// only (B300 issues FP64 at 1/64 of the FP32 rate); the caller keeps
// |v| 2^s < 2^62.  Ties round away from zero.
__device__ inline long long round_scaled(double v, int s) {
    const long long b = __double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;  // zero or subnormal
    const long long m = (b & 0xfffffffffffffLL) | 0x10000000000000LL;  // 53-bit significand
    const int sh = 1075 - ex - s;                                        // v 2^s = m 2^-sh
    long long r;
    if (sh <= 0) r = m << (-sh);
    else if (sh > 54) r = 0;
    else r = (m + (1LL << (sh - 1))) >> sh;
    return b < 0 ? -r : r;
}

// |v| as an ordered integer key (non-negative doubles order like their bits)
__device__ inline unsigned long long abs_key(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

// low 7 bits of x as a signed value in [-64, 63]
__device__ inline int sext7(int x) { return (int)((unsigned)x << 25) >> 25; }

// six balanced base-128 digits of x = v 2^-E (|x| <= 1/4), most significant first.
// X = hi 2^21 + lo with lo in [0, 2^21); the three low digits come from lo in
// 32-bit arithmetic and leave a carry of 0 or 1 for hi -- the same digits as
// taking all six from X one after another (digit = low 7 bits read as signed,
// then X <- (X + 64) >> 7).
__device__ inline void digits_of(long long X, int (&d)[kNS]) {
    int lo = (int)(X & 0x1fffff);
    int hi = (int)(X >> 21);
#pragma unroll
    for (int s = kNS - 1; s >= kNS / 2; --s) {
        d[s] = sext7(lo);
        lo = (lo + 64) >> 7;
    }
    hi += lo;
#pragma unroll
    for (int s = kNS / 2 - 1; s >= 0; --s) {
        d[s] = sext7(hi);
        hi = (hi + 64) >> 7;
    }
}
__device__ inline void digits6(double v, int E, int (&d)[kNS]) { digits_of(round_scaled(v, 42 - E), d); }

// round(v 2^s) for a float v, from its bit pattern (|v| 2^s < 2^62)
__device__ inline long long round_scaled_f(float v, int s) {
    const int b = __float_as_int(v);
    const int ex = (b >> 23) & 0xff;
    if (ex == 0) return 0;  // zero or subnormal
    const long long m = (b & 0x7fffff) | 0x800000;  // 24-bit significand
    const int sh = 150 - ex - s;                     // v 2^s = m 2^-sh
    long long r;
    if (sh <= 0) r = m << (-sh);
    else if (sh > 25) r = 0;
    else r = (m + (1LL << (sh - 1))) >> sh;
    return b < 0 ? -r : r;
}

__device__ inline uint16_t h16(int d) { return __half_as_ushort(__int2half_rn(d)); }

// FP16 bit patterns of two digits a, b in [-64, 63], a in the low half: 1536 + d
// is exact in FP16 (spacing 1 on [1024, 2048), pattern 0x6600 + d), and one
// packed FP16 subtraction of 1536 leaves d exactly -- no conversion instructions.
__device__ inline uint32_t h16x2(int a, int b) {
    const uint32_t u = (uint32_t)(a + 0x6600) | ((uint32_t)(b + 0x6600) << 16);
    __half2 v;
    memcpy(&v, &u, 4);
    v = __hsub2(v, __half2half2(__ushort_as_half((unsigned short)0x6600)));
    uint32_t r;
    memcpy(&r, &v, 4);
    return r;
}

__device__ inline unsigned long long block_max_key(unsigned long long v, unsigned long long* red) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long m = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = max(m, red[k]);
    return m;
}

__device__ inline double block_max_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double m = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, red[k]);
    return m;
}

// ---------------------------------------------------------------------------
// slicing
// ---------------------------------------------------------------------------

// Phi_T (M x N, row-major) -> column-major copy (N x M) in fixed point,
// round(t 2^56) (the trial's columns are orthonormal: |t| <= 1)
constexpr int kTrialFx = 56;
__global__ void transpose_trial_kernel(int M, int N, const double* __restrict__ trial,
                                       long long* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < M * N) {
        const int k = e / M, r = e - k * M;
        out[e] = __double2ll_rn(ldexp(trial[(size_t)r * N + k], kTrialFx));
    }
}

// round(T 2^-sh) of a fixed-point integer, ties upward
__device__ inline long long fx_round(long long T, int sh) {
    if (sh >= 63) return 0;
    if (sh <= 0) return T << (-sh);
    return (T + (1LL << (sh - 1))) >> sh;
}

// a 64-bit integer as a float from two 32-bit conversions of its magnitude
// (|D| < 2^32: correctly rounded; above, within one unit in the last place;
// avoids the 64-bit conversion, which runs on the FP64 pipe)
__device__ inline float ll_to_float(long long D) {
    const unsigned long long a = D < 0 ? 0ull - (unsigned long long)D : (unsigned long long)D;
    const float f = fmaf(__uint2float_rn((unsigned)(a >> 32)), 4294967296.f, __uint2float_rn((unsigned)(a & 0xffffffffull)));
    return D < 0 ? -f : f;
}

// Phi_T^T rows i (per-row exponent), K = basis p: A_S[s][i][p_pad]
__global__ void slice_trial_kernel(int M, int N, int p_pad, const double* __restrict__ trial,
                                   uint16_t* __restrict__ out, int* __restrict__ row_exp) {
    __shared__ double red[32];
    const int i = blockIdx.x;
    double m = 0.0;
    for (int p = threadIdx.x; p < M; p += blockDim.x) m = fmax(m, fabs(trial[(size_t)p * N + i]));
    const int E = slice_exponent(block_max_d(m, red));
    for (int p = threadIdx.x; p < p_pad; p += blockDim.x) {
        int d[kNS];
        digits6(p < M ? trial[(size_t)p * N + i] : 0.0, E, d);
#pragma unroll
        for (int s = 0; s < kNS; ++s) out[((size_t)s * N + i) * p_pad + p] = h16(d[s]);
    }
    if (threadIdx.x == 0) row_exp[i] = E;
}

// One walker's spin block of phi (M x N complex) -> digits, one exponent per
// walker and spin, in the layout
//   At[s][p][w][kpad]        K = 2j + ri, zero for 2j + ri >= 2N
// which is the K-major A operand of the Theta GEMM (rows p of one walker) and,
// read with k = p, the MN-major A operand of the S GEMM (rows (w, 2j + ri) of
// all walkers contiguous for each p).  64 basis rows per CTA.
constexpr int kSliceRows = 64;
// Largest |phi| of each walker's spin block: kMaxSplit CTAs per walker over
// row ranges, integer maxima of the absolute bit patterns (key[w] starts at 0).
constexpr int kMaxSplit = 4;
__global__ void __launch_bounds__(256)
phi_max_kernel(int M, int N, int ntot, int col0, const double2* __restrict__ phi,
               unsigned long long* __restrict__ key) {
    __shared__ unsigned long long red[32];
    const int w = blockIdx.x / kMaxSplit, part = blockIdx.x % kMaxSplit;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const double2* pw = phi + (size_t)w * M * ntot + col0;
    const int p0 = (int)((long)part * M / kMaxSplit), p1 = (int)((long)(part + 1) * M / kMaxSplit);
    unsigned long long m = 0;
    for (int p = p0 + warp; p < p1; p += nwarp)
        for (int j = lane; j < N; j += 32) {
            const double2 v = pw[(size_t)p * ntot + j];
            m = max(m, max(abs_key(v.x), abs_key(v.y)));
        }
    m = block_max_key(m, red);
    if (threadIdx.x == 0) atomicMax(key + w, m);
}

// One (walker, 64-row chunk) per CTA: the chunk's digits, with the walker's
// exponent from its maximum key.  The (row, orbital pair) elements of the chunk
// are spread over all threads, row-major, so that the reads of phi and the
// writes of At stay coalesced.
__global__ void __launch_bounds__(256)
slice_phi_kernel(int M, int N, int ntot, int col0, int kpad, int W,
                 const double2* __restrict__ phi, const unsigned long long* __restrict__ key,
                 uint16_t* __restrict__ At, int* __restrict__ wexp) {
    const int w = blockIdx.x;
    const double2* pw = phi + (size_t)w * M * ntot + col0;
    const int E = slice_exponent(__longlong_as_double((long long)key[w]));
    if (blockIdx.y == 0 && threadIdx.x == 0) wexp[w] = E;
    const int half = kpad >> 1;  // (re, im) pairs per row, those past N zero
    const int p0 = blockIdx.y * kSliceRows;
    const int np = min(kSliceRows, M - p0);
    const size_t at_s = (size_t)M * W * kpad;  // At slice stride
    const int dpp = blockDim.x / half, dj = blockDim.x - dpp * half;
    int pp = threadIdx.x / half, j = threadIdx.x - pp * half;
    while (pp < np) {
        const int p = p0 + pp;
        double2 z = make_double2(0.0, 0.0);
        if (j < N) z = pw[(size_t)p * ntot + j];
        int dr[kNS], di[kNS];
        digits6(z.x, E, dr);
        digits6(z.y, E, di);
        uint32_t* at = reinterpret_cast<uint32_t*>(At + ((size_t)p * W + w) * kpad + 2 * j);
#pragma unroll
        for (int s = 0; s < kNS; ++s) at[s * at_s / 2] = h16x2(dr[s], di[s]);
        pp += dpp;
        j += dj;
        if (j >= half) {
            j -= half;
            ++pp;
        }
    }
}

// ---------------------------------------------------------------------------
// the slice GEMM (tcgen05, 21 products into six diagonal accumulators)
// ---------------------------------------------------------------------------
struct OzParams {
    int n_rt, n_ct, n_b, nk;
    uint32_t idesc;
    int* err;
    int mode;  // 0: overlap S, 1: Theta -> Delta planes
    int M, N, ntot, col0, r_pad, W, rows_valid, cols_valid;
    int kpad;             // mode 0: rows (w, 2j + ri) of the walker slices per walker
    int nrb, nkb;         // mode 1: Delta tile geometry
    const int* row_exp;   // mode 0: exponent of each Phi_T^T row i (column i of the GEMM)
    const int* wexp;      // exponent of each walker's phi block
    const int* col_exp;   // mode 1: [W][N] exponent of each column of S^-1
    double* S_out;        // mode 0: [W][N][N] complex as (re, im) doubles
    const long long* trial_fx;  // mode 1: Phi_T column-major, N x M, in units of 2^-56
    const int* texp;      // mode 1: per-walker Delta scale exponent (scale = 2^texp)
    uint16_t* dhi;
    uint16_t* dlo;
    int bf16;
    float* dfull;         // mode 1, optional: FP32 Delta t in the dfull_elem layout (dense LO epilogue)
    int Sd;
};

struct OzShared {
    uint64_t full[kOStages];
    uint64_t empty[kOStages];
    uint64_t tmem_full;
    uint64_t diag_empty[kND];  // diagonal D of the accumulators read by every epilogue warp
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

__device__ inline uint8_t* align1k(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// z 2^e - Phi_T (real part only), times the walker's Delta scale 2^te, as the
// 16-bit hi/lo pair of the Delta planes; cc = 2k + ro of this spin
// Delta = z 2^e - Phi_T (the trial is real: only the real part ro = 0 moves),
// formed exactly in integer units of 2^e, then scaled by the walker's 2^te
__device__ inline void store_delta(const OzParams& P, int w, int r, int cc, long long z, int e, int te,
                                   long long tfx) {
    const int k = cc >> 1, ro = cc & 1;
    long long D = z;
    if (!ro) D -= fx_round(tfx, kTrialFx + e);
    const float f = ll_to_float(D) * pow2f(e + te);
    uint16_t h, l;
    if (P.bf16) {
        const __nv_bfloat16 a = __float2bfloat16(f);
        h = __bfloat16_as_ushort(a);
        l = __bfloat16_as_ushort(__float2bfloat16(f - __bfloat162float(a)));
    } else {
        const __half a = __float2half(f);
        h = __half_as_ushort(a);
        l = __half_as_ushort(__float2half(f - __half2float(a)));
    }
    const size_t o = delta_elem(2 * w + ro, P.col0 + k, r, P.nrb, P.nkb);
    P.dhi[o] = h;
    P.dlo[o] = l;
    if (P.dfull) P.dfull[dfull_elem(P.col0 + k, P.nrb, P.Sd, 2 * w + ro, r)] = f;
}

constexpr int kOEpiWarps = 16;  // four per TMEM lane quarter, 8-column chunks h, h + 4, h + 8
constexpr int kOThreads = 64 + 32 * kOEpiWarps;

__global__ void __launch_bounds__(kOThreads, 1)
ozaki_gemm_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                  OzParams P) {
    extern __shared__ uint8_t dyn[];
    __shared__ OzShared sh;
    uint8_t* base = align1k(dyn);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_units = P.n_b * P.n_rt * P.n_ct;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kOStages; ++s) { tc::mbar_init(&sh.full[s], 1); tc::mbar_init(&sh.empty[s], 1); }
        tc::mbar_init(&sh.tmem_full, 1);
        for (int D = 0; D < kND; ++D) tc::mbar_init(&sh.diag_empty[D], kOEpiWarps);
        tc::mbar_init(&sh.drain, 1);
        sh.abort = 0;
        tc::fence_barrier_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&sh.tmem_base, 512);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 32) { tc::tma_prefetch(&mA); tc::tma_prefetch(&mB); }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = sh.tmem_base;
    volatile int* abort = &sh.abort;

    if (warp == 0 && lane == 0) {
        int s = 0;
        uint32_t ph = 0, filled = 0, last_par = 0;
        for (int u = blockIdx.x; u < n_units && !*abort; u += gridDim.x) {
            const int ct = u % P.n_ct, rt = (u / P.n_ct) % P.n_rt, b = u / (P.n_ct * P.n_rt);
            for (int kc = 0; kc < P.nk; ++kc) {
                if (!tc::mbar_wait(&sh.empty[s], ph ^ 1, abort)) break;
                uint8_t* st = base + s * kOStage;
                tc::mbar_arrive_expect_tx(&sh.full[s], kOStage);
                for (int q = 0; q < kNS; ++q) {
                    if (P.mode == 0) {
                        // MN-major: rows (w, 2j + ri) contiguous for each k = p, two
                        // boxes of 64 rows x 32 k
                        tc::tma_load_4d(st + q * kOTileA, &mA, &sh.full[s], rt * kOBM, kc * kOBK, 0, q);
                        tc::tma_load_4d(st + q * kOTileA + kOTileA / 2, &mA, &sh.full[s], rt * kOBM + 64,
                                        kc * kOBK, 0, q);
                    } else {
                        // K-major rows p of walker b
                        tc::tma_load_4d(st + q * kOTileA, &mA, &sh.full[s], kc * kOBK, b, rt * kOBM, q);
                    }
                    tc::tma_load_4d(st + kNS * kOTileA + q * kOTileB, &mB, &sh.full[s], kc * kOBK,
                                    ct * kOBN, b, q);
                }
                filled |= 1u << s;
                last_par = (last_par & ~(1u << s)) | (ph << s);
                if (++s == kOStages) { s = 0; ph ^= 1; }
            }
        }
        if (*abort) {
            for (int q = 0; q < kOStages; ++q)
                if (filled & (1u << q)) {
                    volatile int never = 0;
                    tc::mbar_wait(&sh.full[q], (last_par >> q) & 1, &never);
                }
        }
    } else if (warp == 1 && lane == 0) {
        int s = 0;
        uint32_t ph = 0, tph = 0;
        for (int u = blockIdx.x; u < n_units && !*abort; u += gridDim.x) {
            bool ok = true;
            uint32_t started = 0;  // bit D: diagonal D already has a product this unit
            uint32_t owned = 0;    // bit D: the previous unit's epilogue has read diagonal D
            for (int kc = 0; kc < P.nk && ok; ++kc) {
                if (!tc::mbar_wait(&sh.full[s], ph, abort)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t st = tc::smem_u32(base + s * kOStage);
                // diagonal by diagonal, so that this unit's first products only
                // wait for the diagonals the last unit's epilogue has read; the
                // order of the products within a diagonal is that of k
#pragma unroll
                for (int D = 0; D < kND; ++D) {
                    if (!((owned >> D) & 1u)) {
                        if (!tc::mbar_wait(&sh.diag_empty[D], tph ^ 1, abort)) { ok = false; break; }
                        tc::tc_fence_after();
                        owned |= 1u << D;
                    }
#pragma unroll
                    for (int kk = 0; kk < kOBK / 16; ++kk) {
#pragma unroll
                        for (int a = 0; a < kNS; ++a) {
                            const int bq = D - a;  // digit pairs with a + bq = D
                            if (bq < 0 || bq >= kNS) continue;
                            const uint64_t da =
                                P.mode == 0
                                    ? tc::smem_desc_mn128(st + a * kOTileA + kk * 16 * 128, kMnLbo, kMnSbo)
                                    : tc::smem_desc(st + a * kOTileA + kk * 32, 64);
                            const uint64_t db = tc::smem_desc(st + kNS * kOTileA + bq * kOTileB + kk * 32, 64);
                            const uint32_t acc = (started >> D) & 1u;
                            tc::mma_f16(tmem + D * kOBN, da, db, P.idesc, acc);
                            started |= 1u << D;
                        }
                    }
                }
                if (!ok) break;
                tc::mma_commit(&sh.empty[s]);
                if (++s == kOStages) { s = 0; ph ^= 1; }
            }
            if (!ok) break;
            tc::mma_commit(&sh.tmem_full);
            tph ^= 1;
        }
        tc::mma_commit(&sh.drain);
        volatile int never = 0;
        tc::mbar_wait(&sh.drain, 0, &never);
    } else if (warp >= 2) {
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;  // chunks h, h + 4, h + 8 of 8 columns
        constexpr int kCh = (kOBN + 31) / 32;  // chunks per thread at most
        uint32_t tph = 0;
        for (int u = blockIdx.x; u < n_units && !*abort; u += gridDim.x) {
            const int ct = u % P.n_ct, rt = (u / P.n_ct) % P.n_rt, b = u / (P.n_ct * P.n_rt);
            if (!tc::mbar_wait(&sh.tmem_full, tph, abort)) break;
            tc::tc_fence_after();
            // z = sum_D acc_D 2^(7 (kND - 1 - D)) by Horner's rule, most
            // significant diagonal first; each diagonal is handed back to the
            // MMA issuer (the next unit) as soon as every warp has read it
            long long z[kCh][8];
#pragma unroll
            for (int D = 0; D < kND; ++D) {
#pragma unroll
                for (int i = 0; i < kCh; ++i) {
                    if (h * 8 + 32 * i >= kOBN) continue;
                    float v[8];
                    tc::tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + D * kOBN + h * 8 + 32 * i, v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < 8; ++c) {  // |v| < 2^24: exact as int32
                        const long long a = (long long)__float2int_rn(v[c]);
                        z[i][c] = D == 0 ? a : z[i][c] * 128 + a;
                    }
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&sh.diag_empty[D]);
            }
            const int row = rt * kOBM + q * 32 + lane;
            // mode 0: row = w kpad + 2j + ri of the walker slices
            int w0 = 0, ri0 = 0, j0 = 0;
            bool row_ok = row < P.rows_valid;
            if (P.mode == 0) {
                w0 = row / P.kpad;
                const int cc = row - w0 * P.kpad;
                ri0 = cc & 1;
                j0 = cc >> 1;
                row_ok = row_ok && j0 < P.N;
            }
            const int wexp_b = P.mode == 1 ? P.wexp[b] : 0, texp_b = P.mode == 1 ? P.texp[b] : 0;
#pragma unroll
            for (int i = 0; i < kCh; ++i) {
                const int c0 = h * 8 + 32 * i;
                if (c0 >= kOBN) continue;
                // mode 1: the chunk's four orbitals k: exponents and trial values
                int ek[4] = {0, 0, 0, 0};
                long long tk[4] = {0, 0, 0, 0};
                if (P.mode == 1) {
                    const int kb0 = (ct * kOBN + c0) >> 1;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int k = kb0 + m;
                        if (k < P.N) {
                            ek[m] = P.col_exp[(size_t)b * P.N + k];
                            if (row < P.M) tk[m] = P.trial_fx[(size_t)k * P.M + row];
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int col = ct * kOBN + c0 + c;
                    if (!row_ok || col >= P.cols_valid) continue;
                    if (P.mode == 0) {
                        // S_w[i][j] (part ri) for column col = i of Phi_T
                        P.S_out[(((size_t)w0 * P.N + col) * P.N + j0) * 2 + ri0] =
                            (double)z[i][c] * pow2d(P.row_exp[col] + P.wexp[w0] - 49);
                    } else {
                        store_delta(P, b, row, col, z[i][c], wexp_b + ek[c >> 1] - 49, texp_b, tk[c >> 1]);
                    }
                }
            }
            tph ^= 1;
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
    if (threadIdx.x == 0 && sh.abort) atomicExch(P.err, 1);
}

// ---------------------------------------------------------------------------
// Gauss-Jordan inversion with partial pivoting (double-float), log-det, S^-1 slices
// ---------------------------------------------------------------------------

// double-float arithmetic (dfl, df_fma, ...): dfloat.cuh
__device__ inline double2 cdf_to(float4 z) {
    return make_double2(df_to(dfl{z.x, z.y}), df_to(dfl{z.z, z.w}));
}
// v - f u (complex)
__device__ inline float4 cdf_sub_mul(float4 v, float4 f, float4 u) {
    const dfl fr{f.x, f.y}, fi{f.z, f.w}, ur{u.x, u.y}, ui{u.z, u.w};
    dfl re{v.x, v.y}, im{v.z, v.w};
    re = df_fma(df_neg(fr), ur, re);
    re = df_fma(fi, ui, re);
    im = df_fma(df_neg(fr), ui, im);
    im = df_fma(df_neg(fi), ur, im);
    return make_float4(re.hi, re.lo, im.hi, im.lo);
}
// 1 / z (complex): |z|^2 in double-float, its reciprocal from the FP32 one and
// one double-float Newton correction r0 (2 - |z|^2 r0), then conj(z) / |z|^2
__device__ inline float4 cdf_recip(float4 z) {
    const dfl re{z.x, z.y}, im{z.z, z.w};
    const dfl n2 = df_fma(im, im, df_mul(re, re));
    const dfl r0{__frcp_rn(n2.hi), 0.f};
    const dfl e = df_fma(df_neg(n2), r0, dfl{1.f, 0.f});  // 1 - |z|^2 r0
    const dfl r = df_fma(r0, e, r0);
    const dfl a = df_mul(re, r), b = df_mul(df_neg(im), r);
    return make_float4(a.hi, a.lo, b.hi, b.lo);
}

// x y (complex)
__device__ inline float4 cdf_mul(float4 x, float4 y) {
    const dfl xr{x.x, x.y}, xi{x.z, x.w}, yr{y.x, y.y}, yi{y.z, y.w};
    const dfl re = df_fma(df_neg(xi), yi, df_mul(xr, yr));
    const dfl im = df_fma(xi, yr, df_mul(xr, yi));
    return make_float4(re.hi, re.lo, im.hi, im.lo);
}

constexpr int kGJMaxCols = (LOAF_MAX_NOCC + 15) / 16;  // columns per thread of the 16 x 16 grid

// Element arithmetic of the Gauss-Jordan kernel.  Both forms hold a complex
// value in 16 bytes, so the shared-memory layout is the same.
//   DFArith:  double-float float4 {re.hi, re.lo, im.hi, im.lo} on the FP32
//             pipe (about 48 significant bits); pivot moduli from the leading parts
//   F64Arith: double2 on the FP64 pipe (B300: about 1/64 of the FP32 rate)
struct DFArith {
    using T = float4;
    using R = float;
    __device__ static T from(double2 z) {
        const dfl r = df_split_bits(z.x), i = df_split_bits(z.y);
        return make_float4(r.hi, r.lo, i.hi, i.lo);
    }
    __device__ static R mag2(T a) { return fmaf(a.x, a.x, a.z * a.z); }
    __device__ static double mag2d(T a) { return (double)a.x * a.x + (double)a.z * a.z; }
    __device__ static bool finite(T a) { return isfinite(a.x) && isfinite(a.z); }
    __device__ static T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static T sub_mul(T v, T f, T u) { return cdf_sub_mul(v, f, u); }
    __device__ static T mul(T x, T y) { return cdf_mul(x, y); }
    __device__ static T recip(T z) { return cdf_recip(z); }
    __device__ static double2 to_d(T z) { return cdf_to(z); }
    __device__ static R absmax(T z) { return fmaxf(fabsf(z.x), fabsf(z.z)); }
    // round(z 2^sh) of both parts, from hi + lo (one more unit of rounding)
    __device__ static void scaled(T z, int sh, long long& xr, long long& xi) {
        xr = round_scaled_f(z.x, sh) + round_scaled_f(z.y, sh);
        xi = round_scaled_f(z.z, sh) + round_scaled_f(z.w, sh);
    }
};
struct F64Arith {
    using T = double2;
    using R = double;
    __device__ static T from(double2 z) { return z; }
    __device__ static R mag2(T a) { return fma(a.x, a.x, a.y * a.y); }
    __device__ static double mag2d(T a) { return a.x * a.x + a.y * a.y; }
    __device__ static bool finite(T a) { return isfinite(a.x) && isfinite(a.y); }
    __device__ static T zero() { return make_double2(0.0, 0.0); }
    __device__ static T sub_mul(T v, T f, T u) {  // v - f u
        return make_double2(fma(f.y, u.y, fma(-f.x, u.x, v.x)), fma(-f.y, u.x, fma(-f.x, u.y, v.y)));
    }
    __device__ static T mul(T x, T y) { return cmul(x, y); }
    __device__ static T recip(T z) { return cdiv(make_double2(1.0, 0.0), z); }
    __device__ static double2 to_d(T z) { return z; }
    __device__ static R absmax(T z) { return fmax(fabs(z.x), fabs(z.y)); }
    __device__ static void scaled(T z, int sh, long long& xr, long long& xi) {
        xr = round_scaled(z.x, sh);
        xi = round_scaled(z.y, sh);
    }
};

// Z = S^-1 of one walker and spin by Gauss-Jordan elimination with partial
// pivoting in the arithmetic Ar (double-float: pivot search on |.|^2 of the
// leading parts; the singularity test and the log-det in FP64 either way).  Writes the log-det
// part, the status, the per-column exponents g_k and the digits of the real
// block form of Z:
//   Bt[s][w][2k + ro][2j + ri] = {Zr, -Zi, Zi, Zr}[ri][ro] (j, k) / 2^g_k,
// the B operand of the Theta GEMM (Theta = [phi_re phi_im] B, column pairs).
constexpr int kGJThreads = 256;  // update grid: 16 row groups x 16 column groups

template <int MAXC, class Ar>  // column slots per thread: ceil(N / 16); element arithmetic
__global__ void __launch_bounds__(kGJThreads)
gauss_jordan_kernel(int N, int kpad, int W, const double2* __restrict__ S,
                    const unsigned long long* __restrict__ phi_key, uint16_t* __restrict__ Bt,
                    int* __restrict__ col_exp, int* __restrict__ gmax, double2* __restrict__ ld_part,
                    int* __restrict__ st_part) {
    extern __shared__ __align__(16) unsigned char sm[];
    using T = typename Ar::T;
    using R = typename Ar::R;
    T* A = reinterpret_cast<T*>(sm);              // N x N complex
    T* colk = A + N * N;                          // N
    T* pivv = colk + N;                           // N pivots
    int* piv = reinterpret_cast<int*>(pivv + N);  // N
    int* gk = piv + N;                            // N
    __shared__ double red_v[32];
    __shared__ double2 red_c[32];
    __shared__ int s_p, s_flag, s_swaps;
    __shared__ double s_tol;
    __shared__ T s_inv;
    const int w = blockIdx.x, tid = threadIdx.x;
    const int ti = tid >> 4, tj = tid & 15;  // 16 x 16 grid over the matrix
    double m = 0.0;
    R mf = 0;
    // a NaN or infinity anywhere in the walker's spin block (its largest |phi|
    // key is that of a non-finite double) marks the walker; its digit slices,
    // and so S, would otherwise be finite and meaningless
    bool finite = phi_key[w] < 0x7ff0000000000000ull;
    for (int e = tid; e < N * N; e += blockDim.x) {
        const double2 z = S[(size_t)w * N * N + e];
        const T a = Ar::from(z);
        A[e] = a;
        mf = max(mf, Ar::mag2(a));
        finite = finite && Ar::finite(a);
    }
    m = block_max_d(finite ? (double)mf : (double)INFINITY, red_v);
    if (tid == 0) {
        // S comes from 42-bit digit slices of phi and Phi_T, and the digit
        // products left out (s + t >= 8) add up to about M 2^-44 of the operand
        // scale per entry (1.4e-11 measured on a 60-orbital case): a pivot below
        // N 2^-36 max|S| is not distinguishable from zero and marks the walker
        // singular
        const double tol = (double)N * 1.4551915228366852e-11 * sqrt(m);
        s_tol = tol * tol;
        s_flag = (m == m && !isinf(m)) ? 0 : 2;
        s_swaps = 0;
    }
    __syncthreads();
    __shared__ T s_akk;
    // s_flag is written (phase A) only before the first barrier of a step and
    // read only after it, so every thread leaves the loop at the same step
    const bool run = s_flag == 0;
    for (int k = 0; run && k < N; ++k) {
        // phase A (one warp): pivot row p of column k, 1/pivot, the old A[k][k]
        if (tid < 32) {
            R best = -1;
            int bi = k;
            for (int i = k + tid; i < N; i += 32) {
                const R v = Ar::mag2(A[i * N + k]);
                if (v > best) { best = v; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const R ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (tid == 0) {
                s_p = bi;
                piv[k] = bi;
                if (bi != k) s_swaps += 1;
                s_akk = A[k * N + k];
                const T pv = A[bi * N + k];
                // |pivot|^2 against the tolerance, in FP64 (no underflow)
                if (!(Ar::mag2d(pv) > s_tol)) {
                    s_flag = 1;
                } else {
                    pivv[k] = pv;
                    s_inv = Ar::recip(pv);
                }
            }
        }
        __syncthreads();
        if (s_flag) break;
        const int p = s_p;
        const T inv = s_inv;
        // phase B: exchange rows k and p, scale the new row k (A[k][k] = 1/pivot),
        // and take column k of the other rows (row p's entry is the old A[k][k])
        for (int j = tid; j < N; j += blockDim.x) {
            const T rk = A[k * N + j];
            const T rp = p != k ? A[p * N + j] : rk;
            if (p != k) A[p * N + j] = rk;
            A[k * N + j] = j == k ? inv : Ar::mul(rp, inv);
        }
        for (int i = tid; i < N; i += blockDim.x)
            if (i != k) colk[i] = i == p ? s_akk : A[i * N + k];
        __syncthreads();
        // phase C: other rows, A[i][j] -= A[i][k] (old) * A[k][j] (new); A[i][k]
        // starts from 0.  Each thread's columns are loaded, updated and stored
        // as a group so that their independent error-free chains interleave.
        T u[MAXC];
#pragma unroll
        for (int q = 0; q < MAXC; ++q) {
            const int j = tj + 16 * q;
            u[q] = j < N ? A[k * N + j] : Ar::zero();
        }
        for (int i = ti; i < N; i += kGJThreads / 16) {
            if (i == k) continue;
            const T f = colk[i];
            T v[MAXC];
#pragma unroll
            for (int q = 0; q < MAXC; ++q) {
                const int j = tj + 16 * q;
                v[q] = (j < N && j != k) ? A[i * N + j] : Ar::zero();
            }
#pragma unroll
            for (int q = 0; q < MAXC; ++q) v[q] = Ar::sub_mul(v[q], f, u[q]);
#pragma unroll
            for (int q = 0; q < MAXC; ++q) {
                const int j = tj + 16 * q;
                if (j < N) A[i * N + j] = v[q];
            }
        }
        __syncthreads();
    }
    __syncthreads();
    const int flag = s_flag;
    // undo the row interchanges on the columns, in reverse order
    if (flag == 0) {
        for (int k = N - 1; k >= 0; --k) {
            const int p = piv[k];
            if (p != k)
                for (int i = tid; i < N; i += blockDim.x) {
                    const T t = A[i * N + k];
                    A[i * N + k] = A[i * N + p];
                    A[i * N + p] = t;
                }
            __syncthreads();
        }
    }
    // log det = sum_k log(pivot_k) + i pi (row exchanges mod 2)
    double2 lp = make_double2(0.0, 0.0);
    if (flag == 0)
        for (int k = tid; k < N; k += blockDim.x) {
            const double2 d = Ar::to_d(pivv[k]);
            lp.x += log(hypot(d.x, d.y));
            lp.y += atan2(d.y, d.x);
        }
    for (int o = 16; o > 0; o >>= 1) {
        lp.x += __shfl_xor_sync(0xffffffffu, lp.x, o);
        lp.y += __shfl_xor_sync(0xffffffffu, lp.y, o);
    }
    if ((tid & 31) == 0) red_c[tid >> 5] = lp;
    __syncthreads();
    if (tid == 0) {
        st_part[w] = flag == 0 ? LOAF_WALKER_OK : (flag == 1 ? LOAF_WALKER_SINGULAR : LOAF_WALKER_NAN);
        double2 ld = make_double2(0.0, 0.0);
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) ld = cadd(ld, red_c[q]);
        if (flag == 0) {
            if (s_swaps & 1) ld.y += 3.141592653589793;
            ld.y = remainder(ld.y, 6.283185307179586);
        } else {
            ld = make_double2(-INFINITY, 0.0);
        }
        ld_part[w] = ld;
    }
    // per-column exponents of Z (one warp per column)
    const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int k = wid; k < N; k += nw) {
        R mm = 0;  // double-float: leading parts, |z| <= |hi| (1 + 2^-23), within the 2-bit headroom
        if (flag == 0)
            for (int j = lane; j < N; j += 32) mm = max(mm, Ar::absmax(A[j * N + k]));
        for (int o = 16; o > 0; o >>= 1) mm = max(mm, __shfl_xor_sync(0xffffffffu, mm, o));
        if (lane == 0) {
            const int g = slice_exponent((double)mm);
            gk[k] = g;
            col_exp[(size_t)w * N + k] = g;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int g = -1 << 30;
        for (int k = 0; k < N; ++k) g = max(g, gk[k]);
        gmax[w] = g;
    }
    const int twoN = 2 * N;
    // row cc = 2k + ro of Bt, columns K = 2j (ri = 0) and 2j + 1 (ri = 1): the
    // real form [[Zr, -Zi], [Zi, Zr]] of the complex column k
    for (int e = tid; e < twoN * N; e += blockDim.x) {
        const int cc = e / N, j = e - cc * N;
        const int k = cc >> 1, ro = cc & 1;
        long long X0 = 0, X1 = 0;
        if (flag == 0) {
            long long xr, xi;
            Ar::scaled(A[j * N + k], 42 - gk[k], xr, xi);
            X0 = ro ? xi : xr;   // ri = 0: Zr (ro = 0) or Zi (ro = 1)
            X1 = ro ? xr : -xi;  // ri = 1: -Zi (ro = 0) or Zr (ro = 1)
        }
        int d0[kNS], d1[kNS];
        digits_of(X0, d0);
        digits_of(X1, d1);
        uint32_t* bt = reinterpret_cast<uint32_t*>(Bt + (((size_t)w * twoN + cc) * kpad + 2 * j));
        const size_t bt_s = (size_t)W * twoN * kpad / 2;
#pragma unroll
        for (int s = 0; s < kNS; ++s) bt[s * bt_s] = h16x2(d0[s], d1[s]);
    }
}

// Delta scale per walker from the slice exponents: |Theta| <= 2N 2^(E + G - 4)
// < 2^(E + G + 4) and |Phi_T| <= 1, so t = 2^(12 - max(E + G + 4, 0)) keeps
// |Delta t| <= 2^13 for fp16.
__global__ void delta_scale_kernel(int W, int nspin, const int* __restrict__ wexp0,
                                   const int* __restrict__ gmax0, const int* __restrict__ wexp1,
                                   const int* __restrict__ gmax1, float* __restrict__ inv_t,
                                   double* __restrict__ scale, int* __restrict__ texp) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    int b = max(wexp0[w] + gmax0[w] + 4, 0);
    if (nspin > 1) b = max(b, wexp1[w] + gmax1[w] + 4);
    b = min(b, 900);
    scale[w] = ldexp(1.0, 12 - b);
    inv_t[w] = (float)ldexp(1.0, b - 12);
    texp[w] = 12 - b;
}

// The g row of the dense LO blocks reads its "Delta_j" from column s = M of the
// FP32 copy: t (the walker's Delta scale) in the real row, 0 in the imaginary
// row, so that it adds g . Delta_i to the pair value unchanged
__global__ void dfull_gcol_kernel(int W, int ntot, int nrb, int Sd, int M, const int* __restrict__ texp,
                                  float* __restrict__ dfull) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;  // (orbital, walker)
    if (e >= ntot * W) return;
    const int c = e / W, w = e - c * W;
    dfull[dfull_elem(c, nrb, Sd, 2 * w, M)] = ldexpf(1.f, texp[w]);
}

}  // namespace

void run_theta_tc(loaf_ctx* c, int W, const double2* phi, int precision, int Sd) {
    const int M = c->M;
    const int p_pad = (M + 15) / 16 * 16;  // 32-byte rows: whole L2 sectors
    const int r_pad = p_pad;
    const bool bf16 = precision == LOAF_PREC_BF16X3;
    int nmax = 0;
    for (int s = 0; s < c->nspin; ++s) nmax = std::max(nmax, c->sp[s].N);
    const int kpad_max = (2 * nmax + 15) / 16 * 16;
    const size_t at_spin = (size_t)kNS * W * M * kpad_max;        // 16-bit entries per spin
    const size_t bt_spin = (size_t)kNS * W * 2 * nmax * kpad_max;
    c->w_oz_at.ensure(at_spin * c->nspin * 2);
    c->w_oz_bt.ensure(bt_spin * c->nspin * 2);
    c->w_oz_S.ensure((size_t)W * nmax * nmax * sizeof(double2));
    c->w_oz_key.ensure((size_t)W * sizeof(unsigned long long));
    c->w_oz_int.ensure((size_t)(2 * W * (2 + nmax) + W) * sizeof(int) + 256);
    const DeltaGeom dg = delta_geom(M, c->ntot, W);
    c->w_dhi.ensure_zeroed(dg.plane * 2, c->stream);
    c->w_dlo.ensure_zeroed(dg.plane * 2, c->stream);
    if (Sd > 0) {
        // the FP32 copy for the dense LO epilogue: zero wherever the Theta stage
        // does not write (basis columns past M, walker rows past W)
        const size_t n = (size_t)c->ntot * dg.nrb * 128 * Sd;
        const long key = (((long)Sd * 2048 + c->M) * 65536 + dg.nrb) * 256 + c->ntot;
        if (c->w_dfull.bytes < n * sizeof(float) || c->dfull_key != key) {
            c->w_dfull.ensure(n * sizeof(float));
            LOAF_CUDA(cudaMemsetAsync(c->w_dfull.ptr, 0, n * sizeof(float), c->stream));
            c->dfull_key = key;
        }
    }
    c->w_dscale.ensure((size_t)W * (sizeof(float) + sizeof(double)) + 64);
    float* inv_t = c->w_dscale.as<float>();
    double* tscale =
        reinterpret_cast<double*>(c->w_dscale.as<uint8_t>() + ((W * sizeof(float) + 15) / 16) * 16);
    c->w_flag.ensure(16);
    int* err = c->w_flag.as<int>();
    LOAF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
    // int scratch per spin: [wexp W][gmax W][col_exp W * nmax]
    int* ib = c->w_oz_int.as<int>();
    auto wexp = [&](int s) { return ib + (size_t)s * W * (2 + nmax); };
    auto gmx = [&](int s) { return ib + (size_t)s * W * (2 + nmax) + W; };
    auto cexp = [&](int s) { return ib + (size_t)s * W * (2 + nmax) + 2 * W; };
    int* texp = ib + (size_t)2 * W * (2 + nmax);
    uint16_t* At = c->w_oz_at.as<uint16_t>();
    uint16_t* Bt = c->w_oz_bt.as<uint16_t>();
    LOAF_CUDA(cudaFuncSetAttribute(ozaki_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kOSmem));

    // phase 1, per spin: slices of phi, S = Phi_T^T phi, Z = S^-1 (double-float) and its slices
    for (int s = 0; s < c->nspin; ++s) {
        SpinData& sd = c->sp[s];
        const int N = sd.N, twoN = 2 * N, kpad = (twoN + 15) / 16 * 16;
        if (sd.oz_trial_version != c->trial_version) {
            sd.oz_trialT.ensure((size_t)kNS * N * p_pad * 2);
            sd.oz_rowexp.ensure((size_t)N * sizeof(int));
            slice_trial_kernel<<<N, 128, 0, c->stream>>>(M, N, p_pad, sd.d_trial.as<double>(),
                                                       sd.oz_trialT.as<uint16_t>(),
                                                       sd.oz_rowexp.as<int>());
            LOAF_LAUNCH_CHECK();
            sd.oz_trial_cm.ensure((size_t)N * M * sizeof(long long));
            transpose_trial_kernel<<<ceil_div(M * N, 256), 256, 0, c->stream>>>(
                M, N, sd.d_trial.as<double>(), sd.oz_trial_cm.as<long long>());
            LOAF_LAUNCH_CHECK();
            sd.oz_trial_version = c->trial_version;
        }
        {
            StageScope sc(c, "theta_slice", 2);
            unsigned long long* key = c->w_oz_key.as<unsigned long long>();
            LOAF_CUDA(cudaMemsetAsync(key, 0, (size_t)W * sizeof(unsigned long long), c->stream));
            phi_max_kernel<<<W * kMaxSplit, 256, 0, c->stream>>>(M, N, c->ntot, sd.col0, phi, key);
            LOAF_LAUNCH_CHECK();
            slice_phi_kernel<<<dim3(W, ceil_div(M, kSliceRows)), 256, 0, c->stream>>>(
                M, N, c->ntot, sd.col0, kpad, W, phi, key, At + at_spin * s, wexp(s));
            LOAF_LAUNCH_CHECK();
        }
        {
            // S = Phi_T^T phi computed as its transpose: rows w kpad + 2j + ri of the
            // walker slices read MN-major from the Theta GEMM's layout (128-row
            // tiles; rows 2j + ri >= 2N are zero), columns i of Phi_T (80-wide
            // tiles, little padding for N <= 80), K = basis
            StageScope sc(c, "overlap_tc", 1);
            CUtensorMap mA, mB;
            map_slices_mn(&mA, At + at_spin * s, (uint64_t)W * kpad, M);
            map_slices(&mB, sd.oz_trialT.ptr, p_pad, p_pad, N, 1, kOBN);
            OzParams P{};
            P.n_rt = ceil_div((long)kpad * W, kOBM);
            P.n_ct = ceil_div(N, kOBN);
            P.n_b = 1;
            P.nk = ceil_div(p_pad, kOBK);
            P.idesc = tc::idesc_f16(kOBM, kOBN, false) | tc::kIdescAMnMajor;
            P.kpad = kpad;
            P.err = err;
            P.mode = 0;
            P.M = M; P.N = N; P.ntot = c->ntot; P.col0 = sd.col0; P.r_pad = r_pad; P.W = W;
            P.nrb = dg.nrb; P.nkb = dg.nkb;
            P.rows_valid = kpad * W;
            P.cols_valid = N;
            P.row_exp = sd.oz_rowexp.as<int>();
            P.wexp = wexp(s);
            P.S_out = c->w_oz_S.as<double>();
            const int units = P.n_rt * P.n_ct * P.n_b;
            ozaki_gemm_kernel<<<std::min(units, c->persistent_grid()), kOThreads, kOSmem, c->stream>>>(mA, mB, P);
            LOAF_LAUNCH_CHECK();
        }
        {
            const bool f64 = precision == LOAF_PREC_FP16X3_F64INV;
            StageScope sc(c, f64 ? "inverse_f64" : "inverse_df", 1);
            const size_t smem = (size_t)N * N * sizeof(double2) + (size_t)2 * N * sizeof(double2) +
                                2 * N * sizeof(int) + 16;
            // as many column slots per thread as N needs: empty slots would still
            // be computed (on zeros) in every elimination step
            auto launch = [&](auto kern) {
                LOAF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                kern<<<W, kGJThreads, smem, c->stream>>>(
                    N, kpad, W, c->w_oz_S.as<double2>(), c->w_oz_key.as<unsigned long long>(),
                    Bt + bt_spin * s, cexp(s), gmx(s),
                    c->w_logdet.as<double2>() + (size_t)s * W, c->w_status.as<int>() + (size_t)s * W);
            };
            if (f64) {
                switch (ceil_div(N, 16)) {
                    case 1: launch(gauss_jordan_kernel<1, F64Arith>); break;
                    case 2: launch(gauss_jordan_kernel<2, F64Arith>); break;
                    case 3: launch(gauss_jordan_kernel<3, F64Arith>); break;
                    case 4: launch(gauss_jordan_kernel<4, F64Arith>); break;
                    case 5: launch(gauss_jordan_kernel<5, F64Arith>); break;
                    default: launch(gauss_jordan_kernel<kGJMaxCols, F64Arith>); break;
                }
            } else {
                switch (ceil_div(N, 16)) {
                    case 1: launch(gauss_jordan_kernel<1, DFArith>); break;
                    case 2: launch(gauss_jordan_kernel<2, DFArith>); break;
                    case 3: launch(gauss_jordan_kernel<3, DFArith>); break;
                    case 4: launch(gauss_jordan_kernel<4, DFArith>); break;
                    case 5: launch(gauss_jordan_kernel<5, DFArith>); break;
                    default: launch(gauss_jordan_kernel<kGJMaxCols, DFArith>); break;
                }
            }
            LOAF_LAUNCH_CHECK();
        }
    }
    // phase 2: one Delta scale per walker over both spins
    delta_scale_kernel<<<ceil_div(W, 128), 128, 0, c->stream>>>(
        W, c->nspin, wexp(0), gmx(0), wexp(c->nspin - 1), gmx(c->nspin - 1), inv_t, tscale, texp);
    LOAF_LAUNCH_CHECK();
    if (Sd > 0) {
        dfull_gcol_kernel<<<ceil_div((long)c->ntot * W, 256), 256, 0, c->stream>>>(
            W, c->ntot, dg.nrb, Sd, M, texp, c->w_dfull.as<float>());
        LOAF_LAUNCH_CHECK();
    }
    // phase 3, per spin: Theta = phi Z on the tensor cores -> Delta planes
    for (int s = 0; s < c->nspin; ++s) {
        SpinData& sd = c->sp[s];
        const int N = sd.N, twoN = 2 * N, kpad = (twoN + 15) / 16 * 16;
        StageScope sc(c, "theta_tc", 1);
        CUtensorMap mA, mB;
        map_slices_rows(&mA, At + at_spin * s, twoN, kpad, W, M);
        map_slices(&mB, Bt + bt_spin * s, twoN, kpad, twoN, W, kOBN);
        OzParams P{};
        P.n_rt = ceil_div(M, kOBM);
        P.n_ct = ceil_div(twoN, kOBN);
        P.n_b = W;
        P.nk = ceil_div(twoN, kOBK);
        P.idesc = tc::idesc_f16(kOBM, kOBN, false);
        P.err = err;
        P.mode = 1;
        P.M = M; P.N = N; P.ntot = c->ntot; P.col0 = sd.col0; P.r_pad = r_pad; P.W = W;
        P.nrb = dg.nrb; P.nkb = dg.nkb;
        P.rows_valid = M;
        P.cols_valid = twoN;
        P.wexp = wexp(s);
        P.col_exp = cexp(s);
        P.trial_fx = sd.oz_trial_cm.as<long long>();
        P.texp = texp;
        P.dhi = c->w_dhi.as<uint16_t>();
        P.dlo = c->w_dlo.as<uint16_t>();
        P.bf16 = bf16 ? 1 : 0;
        P.dfull = Sd > 0 ? c->w_dfull.as<float>() : nullptr;
        P.Sd = Sd;
        const int units = P.n_rt * P.n_ct * P.n_b;
        ozaki_gemm_kernel<<<std::min(units, c->persistent_grid()), kOThreads, kOSmem, c->stream>>>(mA, mB, P);
        LOAF_LAUNCH_CHECK();
    }
}

}  // namespace loaf
