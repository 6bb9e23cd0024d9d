// K1: per-walker overlap, LU with partial pivoting, log-determinant and
// Theta = phi (Phi_T^T phi)^-1 (eq. Q, Sec. 2.2), all in FP64.
//
// One CTA per (walker, spin).  The N x N overlap lives in shared memory for
// the LU; the M x N solve is done row by row (rows are independent), each
// thread owning rows of phi.  B300 runs FP64 at about 2 FMA per clock per SM,
// so this kernel is bound by the FP64 pipe: ~(2 N^2 M + 4/3 N^3 + 4 M N^2)
// FMAs per walker and spin.
#include "common.cuh"

#include <mutex>

namespace loaf {

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 16;   // 16 x 16 thread grid over the N x N overlap
constexpr int kChunk = 16;  // basis rows of phi / Phi staged per step

// modulus squared, the pivot criterion (ties: first row)
__device__ inline double mag2(double2 a) { return a.x * a.x + a.y * a.y; }

template <int NI>
__global__ void __launch_bounds__(kThreads)
theta_fp64_kernel(int M, int N, int ntot, const double* __restrict__ trial,
                  const double2* __restrict__ phi, double2* __restrict__ theta,
                  double2* __restrict__ zbuf, double2* __restrict__ ld_part,
                  int* __restrict__ st_part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // phi, theta and zbuf point at this spin's first column; the walker
    // stride is the packed width ntot
    const int w = blockIdx.x;
    const int col0 = 0;
    const int tid = threadIdx.x;

    double2* A = reinterpret_cast<double2*>(smem_raw);               // N x N
    double2* ph = A + N * N;                                         // kChunk x N
    double* tr = reinterpret_cast<double*>(ph + kChunk * N);         // kChunk x N
    int* perm = reinterpret_cast<int*>(tr + kChunk * N);             // N
    __shared__ double red_v[32];
    __shared__ int red_i[32];
    __shared__ int s_flag;
    __shared__ int s_swaps;
    __shared__ double s_tol;

    const double2* phw = phi + (size_t)w * M * ntot;

    // ---- 1. S_ij = sum_p Phi_pi phi_pj --------------------------------------
    const int ti = tid / kTile, tj = tid % kTile;
    double2 acc[NI][NI];
#pragma unroll
    for (int a = 0; a < NI; ++a)
#pragma unroll
        for (int b = 0; b < NI; ++b) acc[a][b] = make_double2(0.0, 0.0);

    for (int p0 = 0; p0 < M; p0 += kChunk) {
        const int np = min(kChunk, M - p0);
        __syncthreads();
        for (int e = tid; e < np * N; e += kThreads) {
            const int pp = e / N, c = e % N;
            ph[pp * N + c] = phw[(size_t)(p0 + pp) * ntot + col0 + c];
            tr[pp * N + c] = trial[(size_t)(p0 + pp) * N + c];
        }
        __syncthreads();
        for (int pp = 0; pp < np; ++pp) {
            double ti_v[NI];
            double2 pj_v[NI];
#pragma unroll
            for (int a = 0; a < NI; ++a) {
                const int i = ti + kTile * a;
                ti_v[a] = i < N ? tr[pp * N + i] : 0.0;
                const int j = tj + kTile * a;
                pj_v[a] = j < N ? ph[pp * N + j] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int a = 0; a < NI; ++a)
#pragma unroll
                for (int b = 0; b < NI; ++b) {
                    acc[a][b].x = fma(ti_v[a], pj_v[b].x, acc[a][b].x);
                    acc[a][b].y = fma(ti_v[a], pj_v[b].y, acc[a][b].y);
                }
        }
    }
    __syncthreads();
    double local_max = 0.0;
    bool local_finite = true;
#pragma unroll
    for (int a = 0; a < NI; ++a)
#pragma unroll
        for (int b = 0; b < NI; ++b) {
            const int i = ti + kTile * a, j = tj + kTile * b;
            if (i < N && j < N) {
                A[i * N + j] = acc[a][b];
                local_max = fmax(local_max, mag2(acc[a][b]));
                local_finite = local_finite && isfinite(acc[a][b].x) && isfinite(acc[a][b].y);
            }
        }
    // block max of |S|^2 (singularity tolerance); fmax passes over a NaN, so
    // finiteness is reduced on its own
    for (int o = 16; o > 0; o >>= 1) local_max = fmax(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if ((tid & 31) == 0) red_v[tid >> 5] = local_max;
    if (tid == 0) { s_flag = 0; s_swaps = 0; }
    const int all_finite = __syncthreads_and(local_finite);
    if (tid == 0) {
        double m = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) m = fmax(m, red_v[k]);
        // pivots below N * 2^-52 * max|S| count as zero
        const double tol = (double)N * 2.220446049250313e-16 * sqrt(m);
        s_tol = tol * tol;
        if (!all_finite || !(m == m) || isinf(m)) s_flag = 2;  // non-finite input
    }
    for (int k = tid; k < N; k += kThreads) perm[k] = k;
    __syncthreads();

    // ---- 2. LU with partial pivoting (Doolittle, row exchanges) --------------
    for (int k = 0; k < N && s_flag == 0; ++k) {
        if (tid < 32) {
            double best = -1.0;
            int bi = k;
            for (int i = k + tid; i < N; i += 32) {
                const double v = mag2(A[i * N + k]);
                if (v > best) { best = v; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (tid == 0) {
                red_i[0] = bi;
                if (!(best > s_tol)) s_flag = 1;
            }
        }
        __syncthreads();
        if (s_flag) break;
        const int p = red_i[0];
        if (p != k) {
            for (int c = tid; c < N; c += kThreads) {
                const double2 t = A[k * N + c];
                A[k * N + c] = A[p * N + c];
                A[p * N + c] = t;
            }
            if (tid == 0) {
                const int t = perm[k]; perm[k] = perm[p]; perm[p] = t;
                s_swaps += 1;
            }
        }
        __syncthreads();
        const double2 piv = A[k * N + k];
        for (int i = k + 1 + tid; i < N; i += kThreads) A[i * N + k] = cdiv(A[i * N + k], piv);
        __syncthreads();
        const int rem = N - k - 1;
        for (int e = tid; e < rem * rem; e += kThreads) {
            const int i = k + 1 + e / rem, j = k + 1 + e % rem;
            const double2 l = A[i * N + k], u = A[k * N + j];
            double2 v = A[i * N + j];
            v.x = fma(-l.x, u.x, fma(l.y, u.y, v.x));
            v.y = fma(-l.x, u.y, fma(-l.y, u.x, v.y));
            A[i * N + j] = v;
        }
        __syncthreads();
    }
    __syncthreads();
    const int flag = s_flag;
    if (tid == 0) {
        st_part[w] = flag == 0 ? LOAF_WALKER_OK
                                              : (flag == 1 ? LOAF_WALKER_SINGULAR : LOAF_WALKER_NAN);
        double2 ld = make_double2(0.0, 0.0);
        if (flag == 0) {
            for (int k = 0; k < N; ++k) {
                const double2 d = A[k * N + k];
                ld.x += log(hypot(d.x, d.y));
                ld.y += atan2(d.y, d.x);
            }
            if (s_swaps & 1) ld.y += 3.141592653589793;
            // fold the phase into (-pi, pi]
            ld.y = remainder(ld.y, 6.283185307179586);
        } else {
            ld.x = -INFINITY;
            ld.y = 0.0;
        }
        ld_part[w] = ld;
    }

    // ---- 3. Theta = phi S^-1: per row, Z U = phi_row, Y L = Z, Theta_perm = Y -
    double2* thw = theta + (size_t)w * ntot * M + (size_t)col0 * M;
    double2* zw = zbuf + (size_t)w * ntot * M + (size_t)col0 * M;
    if (flag != 0) {
        const double2 nan2 = make_double2(__longlong_as_double(0x7ff8000000000000LL),
                                          __longlong_as_double(0x7ff8000000000000LL));
        for (int e = tid; e < N * M; e += kThreads) thw[e] = nan2;
        return;
    }
    for (int r = tid; r < M; r += kThreads) {
        const double2* prow = phw + (size_t)r * ntot + col0;
        // forward: Z_k = (phi_k - sum_{m<k} Z_m U_mk) / U_kk
        for (int k = 0; k < N; ++k) {
            double2 s = prow[k];
            for (int m = 0; m < k; ++m) {
                const double2 z = zw[(size_t)m * M + r], u = A[m * N + k];
                s.x = fma(-z.x, u.x, fma(z.y, u.y, s.x));
                s.y = fma(-z.x, u.y, fma(-z.y, u.x, s.y));
            }
            zw[(size_t)k * M + r] = cdiv(s, A[k * N + k]);
        }
        // backward: Y_k = Z_k - sum_{m>k} Y_m L_mk; Theta_{perm[k]} = Y_k
        for (int k = N - 1; k >= 0; --k) {
            double2 s = zw[(size_t)k * M + r];
            for (int m = k + 1; m < N; ++m) {
                const double2 y = thw[(size_t)perm[m] * M + r], l = A[m * N + k];
                s.x = fma(-y.x, l.x, fma(y.y, l.y, s.x));
                s.y = fma(-y.x, l.y, fma(-y.y, l.x, s.y));
            }
            thw[(size_t)perm[k] * M + r] = s;
        }
    }
}

}  // namespace

void run_theta_fp64(loaf_ctx* c, int W, const double2* phi, double2* theta, double2* ld_part,
                    int* st_part) {
    // ld_part / st_part are [spin][walker]
    for (int s = 0; s < c->nspin; ++s) {
        const SpinData& sd = c->sp[s];
        const int NI = (sd.N + kTile - 1) / kTile;
        const size_t smem = (size_t)sd.N * sd.N * sizeof(double2) +
                            (size_t)kChunk * sd.N * (sizeof(double2) + sizeof(double)) +
                            (size_t)sd.N * sizeof(int) + 16;
        auto launch = [&](auto kern) {
            LOAF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
            kern<<<W, kThreads, smem, c->stream>>>(
                c->M, sd.N, c->ntot, sd.d_trial.as<double>(), phi + sd.col0,
                theta + (size_t)sd.col0 * c->M, c->w_z.as<double2>() + (size_t)sd.col0 * c->M,
                ld_part + (size_t)s * W, st_part + (size_t)s * W);
            LOAF_LAUNCH_CHECK();
        };
        switch (NI) {
            case 1: launch(theta_fp64_kernel<1>); break;
            case 2: launch(theta_fp64_kernel<2>); break;
            case 3: launch(theta_fp64_kernel<3>); break;
            case 4: launch(theta_fp64_kernel<4>); break;
            case 5: launch(theta_fp64_kernel<5>); break;
            case 6: launch(theta_fp64_kernel<6>); break;
            default: throw Error{LOAF_ERR_SHAPE, "occupied orbitals beyond LOAF_MAX_NOCC"};
        }
    }
}

// ---------------------------------------------------------------------------
// walkers_theta_noalloc: the Theta kernel above with its scratch (the forward-
// solve rows Z and the per-spin log-det / status parts) in one fixed device
// array, for callers that must not allocate device memory during a call.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = 32ull << 20;  // 32 MiB, held by every device that loads the library
constexpr int kNoAllocMaxW = 4096;
constexpr size_t kNoAllocLdBytes = 2ull * kNoAllocMaxW * sizeof(double2);
constexpr size_t kNoAllocStBytes = 2ull * kNoAllocMaxW * sizeof(int);
constexpr size_t kNoAllocZOffset = kNoAllocLdBytes + kNoAllocStBytes;  // multiple of 256
constexpr size_t kNoAllocZEntries = (kNoAllocBytes - kNoAllocZOffset) / sizeof(double2);

// layout: [2][kNoAllocMaxW] double2 log-det parts | [2][kNoAllocMaxW] int
// status parts | Z rows (W x ntot x M complex) in the rest
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};  // device address of g_noalloc_scratch per device ordinal

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in for it).
unsigned char* noalloc_scratch(int device) {
    LOAF_REQUIRE(device >= 0 && device < 256, LOAF_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        LOAF_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[device] = p;
    }
    return static_cast<unsigned char*>(g_noalloc_addr[device]);
}

__global__ void theta_noalloc_combine_kernel(int W, int nspin, double mult0,
                                             const double2* __restrict__ ld_part,
                                             const int* __restrict__ st_part,
                                             double2* __restrict__ ld_out,
                                             int* __restrict__ st_out) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    double2 ld = cscale(ld_part[w], mult0 == 2.0 ? 2.0 : 1.0);
    int st = st_part[w];
    if (nspin > 1) {
        ld = cadd(ld, ld_part[kNoAllocMaxW + w]);
        st = max(st, st_part[kNoAllocMaxW + w]);
    }
    if (ld_out) ld_out[w] = ld;
    if (st_out) st_out[w] = st;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace loaf

extern "C" loaf_status walkers_theta_noalloc(loaf_ctx* c, int W, const void* phi, void* theta_out,
                                             void* logdet_out, int* walker_status) {
    using namespace loaf;
    if (!c) return LOAF_ERR_ARG;
    try {
        LOAF_REQUIRE(c->loaded, LOAF_ERR_NOT_READY, "ao_load_cholesky has not been called");
        LOAF_REQUIRE(phi && theta_out, LOAF_ERR_ARG, "phi and theta_out are required");
        LOAF_REQUIRE(W >= 1 && W <= kNoAllocMaxW, LOAF_ERR_SHAPE,
                     "walkers_theta_noalloc: W must be between 1 and 4096");
        const size_t need = (size_t)W * c->ntot * c->M;
        LOAF_REQUIRE(need <= kNoAllocZEntries, LOAF_ERR_SHAPE,
                     "walkers_theta_noalloc: W * Ntot * M = " + std::to_string(need) +
                         " exceeds the fixed scratch (" + std::to_string(kNoAllocZEntries) +
                         " complex entries, 32 MiB); use walkers_theta or fewer walkers");
        LOAF_CUDA(cudaSetDevice(c->device));
        LOAF_REQUIRE(on_device(phi) && on_device(theta_out) &&
                         (!logdet_out || on_device(logdet_out)) &&
                         (!walker_status || on_device(walker_status)),
                     LOAF_ERR_ARG, "walkers_theta_noalloc takes device buffers only");
        unsigned char* scratch = noalloc_scratch(c->device);
        double2* ld_part = reinterpret_cast<double2*>(scratch);
        int* st_part = reinterpret_cast<int*>(scratch + kNoAllocLdBytes);
        double2* zbuf = reinterpret_cast<double2*>(scratch + kNoAllocZOffset);
        const double2* dphi = static_cast<const double2*>(phi);
        double2* theta = static_cast<double2*>(theta_out);
        for (int s = 0; s < c->nspin; ++s) {
            const SpinData& sd = c->sp[s];
            const int NI = (sd.N + kTile - 1) / kTile;
            const size_t smem = (size_t)sd.N * sd.N * sizeof(double2) +
                                (size_t)kChunk * sd.N * (sizeof(double2) + sizeof(double)) +
                                (size_t)sd.N * sizeof(int) + 16;
            auto launch = [&](auto kern) {
                LOAF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
                kern<<<W, kThreads, smem, c->stream>>>(
                    c->M, sd.N, c->ntot, sd.d_trial.as<double>(), dphi + sd.col0,
                    theta + (size_t)sd.col0 * c->M, zbuf + (size_t)sd.col0 * c->M,
                    ld_part + (size_t)s * kNoAllocMaxW, st_part + (size_t)s * kNoAllocMaxW);
                LOAF_LAUNCH_CHECK();
            };
            switch (NI) {
                case 1: launch(theta_fp64_kernel<1>); break;
                case 2: launch(theta_fp64_kernel<2>); break;
                case 3: launch(theta_fp64_kernel<3>); break;
                case 4: launch(theta_fp64_kernel<4>); break;
                case 5: launch(theta_fp64_kernel<5>); break;
                case 6: launch(theta_fp64_kernel<6>); break;
                default: throw Error{LOAF_ERR_SHAPE, "occupied orbitals beyond LOAF_MAX_NOCC"};
            }
        }
        theta_noalloc_combine_kernel<<<ceil_div(W, 128), 128, 0, c->stream>>>(
            W, c->nspin, c->sp[0].mult, ld_part, st_part, static_cast<double2*>(logdet_out),
            walker_status);
        LOAF_LAUNCH_CHECK();
        c->err.clear();
        return LOAF_OK;
    } catch (const Error& e) {
        c->err = e.msg;
        return e.code;
    }
}
