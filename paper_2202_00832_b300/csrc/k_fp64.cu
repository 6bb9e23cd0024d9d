// FP64 energy stages (precision LOAF_PREC_FP64): one-body + Coulomb, the
// full exchange and the LO pair exchange, and the deterministic per-walker
// reductions.  These are the parity path and the "plain FP64" baseline the
// mixed-precision path is measured against; on B300 they are bound by the
// FP64 pipe (~1 TFLOP/s per GPU).
//
// Layouts (all row-major):
//   theta  [W][ntot][M] complex   (orbital-major: theta[w][c][r] = Theta_rc)
//   Lbar   [X][N][M] real per spin, hbar [N][M]
//   pair factors: rows of Ubar^T and Vbar, [R][M], pair n owns rows off[n]..off[n]+K[n)
#include "common.cuh"

namespace loaf {

namespace {

constexpr int kThreads = 256;

__device__ inline double2 warp_sum2(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// ---------------------------------------------------------------------------
// one-body + Coulomb: Jt[w][g] = sum_sigma mult_sigma sum_ir Lbar^s_gir Theta^s_ri
// for g < X, and Jt[w][X] = sum_sigma mult_sigma sum_ir hbar^s_ir Theta^s_ri (= E1)
// Tile: 64 rows g x 16 walkers, K chunks of 32 along (i, r).
// ---------------------------------------------------------------------------
constexpr int kCG = 64, kCW = 16, kCK = 32;

struct CoulombSpin {
    const double* Lbar;
    const double* hbar;
    int N, col0;
    double mult;
};

__global__ void __launch_bounds__(kThreads)
coulomb_fp64_kernel(int M, int X, int W, int ntot, int nspin, CoulombSpin s0, CoulombSpin s1,
                    const double2* __restrict__ theta, double2* __restrict__ Jt) {
    __shared__ double sL[kCG][kCK + 1];
    __shared__ double2 sT[kCW][kCK + 1];
    const int g0 = blockIdx.x * kCG, w0 = blockIdx.y * kCW;
    const int tid = threadIdx.x;
    const int tw = tid % kCW, tg = tid / kCW;  // 16 walkers x 16 row groups of 4
    double2 acc[4];
    for (int a = 0; a < 4; ++a) acc[a] = make_double2(0.0, 0.0);
    for (int s = 0; s < nspin; ++s) {
        const CoulombSpin sp = s == 0 ? s0 : s1;
        const long K = (long)sp.N * M;
        double2 part[4];
        for (int a = 0; a < 4; ++a) part[a] = make_double2(0.0, 0.0);
        for (long k0 = 0; k0 < K; k0 += kCK) {
            __syncthreads();
            for (int e = tid; e < kCG * kCK; e += kThreads) {
                const int gg = e / kCK, kk = e % kCK;
                const int g = g0 + gg;
                const long k = k0 + kk;
                double v = 0.0;
                if (k < K) {
                    if (g < X) v = sp.Lbar[(size_t)g * K + k];
                    else if (g == X) v = sp.hbar[k];
                }
                sL[gg][kk] = v;
            }
            for (int e = tid; e < kCW * kCK; e += kThreads) {
                const int ww = e / kCK, kk = e % kCK;
                const int w = w0 + ww;
                const long k = k0 + kk;
                double2 v = make_double2(0.0, 0.0);
                if (w < W && k < K) v = theta[(size_t)w * ntot * M + (size_t)sp.col0 * M + k];
                sT[ww][kk] = v;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < kCK; ++kk) {
                const double2 t = sT[tw][kk];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const double l = sL[tg * 4 + a][kk];
                    part[a].x = fma(l, t.x, part[a].x);
                    part[a].y = fma(l, t.y, part[a].y);
                }
            }
        }
        for (int a = 0; a < 4; ++a) acc[a] = cadd(acc[a], cscale(part[a], sp.mult));
    }
    const int w = w0 + tw;
    if (w >= W) return;
    for (int a = 0; a < 4; ++a) {
        const int g = g0 + tg * 4 + a;
        if (g <= X) Jt[(size_t)w * (X + 1) + g] = acc[a];
    }
}

// E1 and E_J per walker from Jt (fixed summation order)
__global__ void coulomb_reduce_kernel(int X, int W, const double2* __restrict__ Jt,
                                      double2* __restrict__ e1, double2* __restrict__ ej) {
    const int w = blockIdx.x;
    double2 s = make_double2(0.0, 0.0);
    for (int g = threadIdx.x; g < X; g += blockDim.x) {
        const double2 j = Jt[(size_t)w * (X + 1) + g];
        s = cadd(s, cmul(j, j));
    }
    __shared__ double2 red[32];
    s = warp_sum2(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = cadd(t, red[k]);
        ej[w] = cscale(t, 0.5);
        e1[w] = Jt[(size_t)w * (X + 1) + X];
    }
}

// ---------------------------------------------------------------------------
// full exchange: ek[w][g] += mult * sum_ij T_ij T_ji, T = Lbar_g Theta_w (N x N)
// one CTA per (g, w); r in chunks of 16 staged in shared memory
// ---------------------------------------------------------------------------
template <int NI>
__global__ void __launch_bounds__(kThreads)
exchange_full_fp64_kernel(int M, int N, int X, int ntot, int col0, double mult,
                          const double* __restrict__ Lbar, const double2* __restrict__ theta,
                          double2* __restrict__ ek, int accumulate) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int RC = 16;
    const int g = blockIdx.x, w = blockIdx.y;
    const int tid = threadIdx.x, ti = tid / 16, tj = tid % 16;
    double* sLb = reinterpret_cast<double*>(smem_raw);            // N x RC
    double2* sTh = reinterpret_cast<double2*>(sLb + N * RC);      // N x RC
    double2 acc[NI][NI];
#pragma unroll
    for (int a = 0; a < NI; ++a)
#pragma unroll
        for (int b = 0; b < NI; ++b) acc[a][b] = make_double2(0.0, 0.0);
    const double* Lg = Lbar + (size_t)g * N * M;
    const double2* Tw = theta + (size_t)w * ntot * M + (size_t)col0 * M;
    for (int r0 = 0; r0 < M; r0 += RC) {
        const int nr = min(RC, M - r0);
        __syncthreads();
        for (int e = tid; e < N * RC; e += kThreads) {
            const int i = e / RC, rr = e % RC;
            sLb[i * RC + rr] = rr < nr ? Lg[(size_t)i * M + r0 + rr] : 0.0;
            sTh[i * RC + rr] = rr < nr ? Tw[(size_t)i * M + r0 + rr] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        for (int rr = 0; rr < nr; ++rr) {
            double lv[NI];
            double2 tv[NI];
#pragma unroll
            for (int a = 0; a < NI; ++a) {
                const int i = ti + 16 * a, j = tj + 16 * a;
                lv[a] = i < N ? sLb[i * RC + rr] : 0.0;
                tv[a] = j < N ? sTh[j * RC + rr] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int a = 0; a < NI; ++a)
#pragma unroll
                for (int b = 0; b < NI; ++b) {
                    acc[a][b].x = fma(lv[a], tv[b].x, acc[a][b].x);
                    acc[a][b].y = fma(lv[a], tv[b].y, acc[a][b].y);
                }
        }
    }
    __syncthreads();
    double2* sT = reinterpret_cast<double2*>(smem_raw);  // N x N (reuses the staging area)
#pragma unroll
    for (int a = 0; a < NI; ++a)
#pragma unroll
        for (int b = 0; b < NI; ++b) {
            const int i = ti + 16 * a, j = tj + 16 * b;
            if (i < N && j < N) sT[i * N + j] = acc[a][b];
        }
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int a = 0; a < NI; ++a)
#pragma unroll
        for (int b = 0; b < NI; ++b) {
            const int i = ti + 16 * a, j = tj + 16 * b;
            if (i < N && j < N) s = cadd(s, cmul(sT[i * N + j], sT[j * N + i]));
        }
    __shared__ double2 red[kThreads / 32];
    s = warp_sum2(s);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int k = 0; k < kThreads / 32; ++k) t = cadd(t, red[k]);
        t = cscale(t, mult);
        double2* out = ek + (size_t)w * X + g;
        *out = accumulate ? cadd(*out, t) : t;
    }
}

// E_K[w] = 1/2 sum_g ek[w][g]
__global__ void sum_rows_kernel(int X, const double2* __restrict__ part, double scale,
                                double2* __restrict__ out) {
    const int w = blockIdx.x;
    double2 s = make_double2(0.0, 0.0);
    for (int g = threadIdx.x; g < X; g += blockDim.x) s = cadd(s, part[(size_t)w * X + g]);
    __shared__ double2 red[32];
    s = warp_sum2(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = cadd(t, red[k]);
        out[w] = cscale(t, scale);
    }
}

// ---------------------------------------------------------------------------
// LO pair exchange: e[n][w] = (Ubar^T Theta_j) . (Vbar Theta_i), unweighted
// one CTA per (pair, 4 walkers); warps over the pair's ranks K
// ---------------------------------------------------------------------------
constexpr int kLW = 4;

__global__ void __launch_bounds__(kThreads)
pair_exchange_fp64_kernel(int M, int W, int ntot, int col0, const int* __restrict__ pi,
                          const int* __restrict__ pj, const int* __restrict__ pK,
                          const long* __restrict__ poff, const double* __restrict__ U,
                          const double* __restrict__ V, const double2* __restrict__ theta,
                          double2* __restrict__ e_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* sTj = reinterpret_cast<double2*>(smem_raw);  // kLW x M
    double2* sTi = sTj + kLW * M;                         // kLW x M
    const int n = blockIdx.x, w0 = blockIdx.y * kLW;
    const int i = pi[n], j = pj[n], K = pK[n];
    const long off = poff[n];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < kLW * M; e += kThreads) {
        const int ww = e / M, r = e % M;
        const int w = w0 + ww;
        double2 a = make_double2(0.0, 0.0), b = a;
        if (w < W) {
            a = theta[(size_t)w * ntot * M + (size_t)(col0 + j) * M + r];
            b = theta[(size_t)w * ntot * M + (size_t)(col0 + i) * M + r];
        }
        sTj[e] = a;
        sTi[e] = b;
    }
    __syncthreads();
    double2 tot[kLW];
    for (int ww = 0; ww < kLW; ++ww) tot[ww] = make_double2(0.0, 0.0);
    for (int k = warp; k < K; k += kThreads / 32) {
        const double* u = U + (size_t)(off + k) * M;
        const double* v = V + (size_t)(off + k) * M;
        double2 a[kLW], b[kLW];
        for (int ww = 0; ww < kLW; ++ww) a[ww] = b[ww] = make_double2(0.0, 0.0);
        for (int r = lane; r < M; r += 32) {
            const double uu = u[r], vv = v[r];
#pragma unroll
            for (int ww = 0; ww < kLW; ++ww) {
                const double2 tj = sTj[ww * M + r], tiv = sTi[ww * M + r];
                a[ww].x = fma(uu, tj.x, a[ww].x);
                a[ww].y = fma(uu, tj.y, a[ww].y);
                b[ww].x = fma(vv, tiv.x, b[ww].x);
                b[ww].y = fma(vv, tiv.y, b[ww].y);
            }
        }
#pragma unroll
        for (int ww = 0; ww < kLW; ++ww) {
            a[ww] = warp_sum2(a[ww]);
            b[ww] = warp_sum2(b[ww]);
            tot[ww] = cadd(tot[ww], cmul(a[ww], b[ww]));
        }
    }
    __shared__ double2 red[kThreads / 32][kLW];
    if (lane == 0)
        for (int ww = 0; ww < kLW; ++ww) red[warp][ww] = tot[ww];
    __syncthreads();
    if (tid < kLW) {
        const int w = w0 + tid;
        if (w < W) {
            double2 t = make_double2(0.0, 0.0);
            for (int k = 0; k < kThreads / 32; ++k) t = cadd(t, red[k][tid]);
            e_out[(size_t)n * W + w] = t;
        }
    }
}

// E_K[w] = 1/2 sum_sigma mult_sigma sum_n wgt_n e[n][w], wgt = 1 (i == j) or 2
__global__ void pair_reduce_kernel(int npairs, int W, const int* __restrict__ pi,
                                   const int* __restrict__ pj, const double2* __restrict__ e,
                                   const unsigned char* __restrict__ keep, double scale,
                                   double2* __restrict__ out, int accumulate) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    double2 s = make_double2(0.0, 0.0);
    for (int n = 0; n < npairs; ++n) {
        if (keep && !keep[n]) continue;  // pair dropped by the screen
        const double wg = pi[n] == pj[n] ? 1.0 : 2.0;
        s = cadd(s, cscale(e[(size_t)n * W + w], wg));
    }
    s = cscale(s, scale);
    out[w] = accumulate ? cadd(out[w], s) : s;
}

}  // namespace

// ---------------------------------------------------------------------------
// host stages
// ---------------------------------------------------------------------------

// part layout in c->w_part: [W][X+1] complex (Coulomb rows), then e1, ej, ek (W each)
void run_coulomb_fp64(loaf_ctx* c, int W, const double2* theta, double2* e_part) {
    CoulombSpin s[2];
    for (int k = 0; k < 2; ++k) {
        const SpinData& sd = c->sp[k < c->nspin ? k : 0];
        s[k] = CoulombSpin{sd.d_Lbar.as<double>(), sd.d_hbar.as<double>(), sd.N, sd.col0, sd.mult};
    }
    double2* Jt = c->w_part2.as<double2>();
    dim3 grid(ceil_div(c->X + 1, kCG), ceil_div(W, kCW));
    coulomb_fp64_kernel<<<grid, kThreads, 0, c->stream>>>(c->M, c->X, W, c->ntot, c->nspin, s[0],
                                                          s[1], theta, Jt);
    LOAF_LAUNCH_CHECK();
    coulomb_reduce_kernel<<<W, 256, 0, c->stream>>>(c->X, W, Jt, e_part, e_part + W);
    LOAF_LAUNCH_CHECK();
}

void run_energy_fp64_full(loaf_ctx* c, int W, const double2* theta, double2* ek_out) {
    double2* part = c->w_part2.as<double2>();  // [W][X]
    for (int s = 0; s < c->nspin; ++s) {
        const SpinData& sd = c->sp[s];
        const int NI = (sd.N + 15) / 16;
        const size_t stage = (size_t)sd.N * 16 * (sizeof(double) + sizeof(double2));
        const size_t smem = std::max(stage, (size_t)sd.N * sd.N * sizeof(double2));
        auto launch = [&](auto kern) {
            LOAF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
            kern<<<dim3(c->X, W), kThreads, smem, c->stream>>>(
                c->M, sd.N, c->X, c->ntot, sd.col0, sd.mult, sd.d_Lbar.as<double>(), theta, part,
                s > 0);
            LOAF_LAUNCH_CHECK();
        };
        switch (NI) {
            case 1: launch(exchange_full_fp64_kernel<1>); break;
            case 2: launch(exchange_full_fp64_kernel<2>); break;
            case 3: launch(exchange_full_fp64_kernel<3>); break;
            case 4: launch(exchange_full_fp64_kernel<4>); break;
            case 5: launch(exchange_full_fp64_kernel<5>); break;
            case 6: launch(exchange_full_fp64_kernel<6>); break;
            default: throw Error{LOAF_ERR_SHAPE, "occupied orbitals beyond LOAF_MAX_NOCC"};
        }
    }
    sum_rows_kernel<<<W, 256, 0, c->stream>>>(c->X, part, 0.5, ek_out);
    LOAF_LAUNCH_CHECK();
}

void run_energy_fp64_lo(loaf_ctx* c, int W, const double2* theta, double2* ek_out,
                        double2* e_pairs) {
    if (!c->keep.empty() && c->d_keep_version != c->screen_version) {
        c->d_keep.ensure(c->keep.size());
        LOAF_CUDA(cudaMemcpyAsync(c->d_keep.ptr, c->keep.data(), c->keep.size(),
                                  cudaMemcpyHostToDevice, c->stream));
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
        c->d_keep_version = c->screen_version;
    }
    // e_pairs: [total pairs][W]; spin blocks consecutive
    long base = 0;
    for (int s = 0; s < c->nspin; ++s) {
        const SpinData& sd = c->sp[s];
        const PairTable& pt = sd.pairs;
        if (pt.npairs == 0) continue;
        const size_t smem = (size_t)2 * kLW * c->M * sizeof(double2);
        LOAF_CUDA(cudaFuncSetAttribute(pair_exchange_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        pair_exchange_fp64_kernel<<<dim3(pt.npairs, ceil_div(W, kLW)), kThreads, smem,
                                    c->stream>>>(
            c->M, W, c->ntot, sd.col0, pt.d_i.as<int>(), pt.d_j.as<int>(), pt.d_K.as<int>(),
            pt.d_off.as<long>(), pt.d_U.as<double>(), pt.d_V.as<double>(), theta,
            e_pairs + base * W);
        LOAF_LAUNCH_CHECK();
        if (ek_out) {
            const unsigned char* keep =
                c->keep.empty() ? nullptr : c->d_keep.as<unsigned char>() + base;
            pair_reduce_kernel<<<ceil_div(W, 128), 128, 0, c->stream>>>(
                pt.npairs, W, pt.d_i.as<int>(), pt.d_j.as<int>(), e_pairs + base * W, keep,
                0.5 * sd.mult, ek_out, s > 0);
            LOAF_LAUNCH_CHECK();
        }
        base += pt.npairs;
    }
}

// The pair kernel with i and j exchanged gives d_ij = (Ubar^T Theta_i).(Vbar Theta_j);
// E_J = 2 sum_ij d_ij = 2 (sum_i d_ii + 2 sum_{i<j} d_ij)  (closed shell, eq. 2e_HR_RCAS)
void run_coulomb_lo_fp64(loaf_ctx* c, int W, const double2* theta, double2* ej_out, double2* scratch) {
    LOAF_REQUIRE(c->nspin == 1, LOAF_ERR_UNSUPPORTED, "the compressed Coulomb is defined for closed shells");
    const SpinData& sd = c->sp[0];
    const PairTable& pt = sd.pairs;
    if (pt.npairs == 0) {
        LOAF_CUDA(cudaMemsetAsync(ej_out, 0, (size_t)W * sizeof(double2), c->stream));
        return;
    }
    const size_t smem = (size_t)2 * kLW * c->M * sizeof(double2);
    LOAF_CUDA(cudaFuncSetAttribute(pair_exchange_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    pair_exchange_fp64_kernel<<<dim3(pt.npairs, ceil_div(W, kLW)), kThreads, smem, c->stream>>>(
        c->M, W, c->ntot, sd.col0, pt.d_j.as<int>(), pt.d_i.as<int>(), pt.d_K.as<int>(), pt.d_off.as<long>(),
        pt.d_U.as<double>(), pt.d_V.as<double>(), theta, scratch);
    LOAF_LAUNCH_CHECK();
    pair_reduce_kernel<<<ceil_div(W, 128), 128, 0, c->stream>>>(pt.npairs, W, pt.d_i.as<int>(),
                                                                pt.d_j.as<int>(), scratch, nullptr, 2.0,
                                                                ej_out, 0);
    LOAF_LAUNCH_CHECK();
}

}  // namespace loaf
