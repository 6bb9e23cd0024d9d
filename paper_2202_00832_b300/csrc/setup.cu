// Setup stages (once per molecule, outside the timed path):
//   S1 half-rotation  Lbar^g = Phi^T L^g, hbar = Phi^T h    (Sec. 2.2)
//   S2 Foster-Boys localization of the occupied orbitals    (Sec. 4)
//   S3 pair blocks Y^[ij] = A_i^T A_j (A_i[g, r] = Lbar^g_ir), their SVD and
//      truncation at T_SVD, packed contiguously              (Sec. 3.1.1, 4.4)
//
// The half-rotation and the pair Gram blocks are plain FP64 GEMMs (cuBLAS).
// The SVD of each off-diagonal block uses the symmetric Jordan-Wielandt
// matrix [[0, Y], [Y^T, 0]] whose eigenpairs are (+-s_k, [u_k; +-v_k]/sqrt 2);
// the diagonal blocks Y^[ii] are symmetric and decompose directly.  Both go
// through cuSOLVER's batched symmetric eigensolver, which keeps the absolute
// accuracy of the singular values at eps * |Y| (forming Y^T Y would square it).
#include "common.cuh"

#include <algorithm>
#include <cmath>

namespace loaf {

// ---------------------------------------------------------------------------
// S1
// ---------------------------------------------------------------------------

void half_rotate(loaf_ctx* c, SpinData& s) {
    const int M = c->M, N = s.N;
    s.d_Lbar.ensure((size_t)c->X * N * M * sizeof(double));
    s.d_hbar.ensure((size_t)N * M * sizeof(double));
    const double one = 1.0, zero = 0.0;
    LOAF_CUBLAS(cublasSetStream(c->cublas, c->stream));
    // column-major view: Lbar_g^T (M x N) = L_g (M x M, symmetric) * Phi (M x N)
    // with Phi stored row-major M x N, i.e. column-major N x M -> op T
    LOAF_CUBLAS(cublasDgemmStridedBatched(c->cublas, CUBLAS_OP_N, CUBLAS_OP_T, M, N, M, &one,
                                          c->d_L.as<double>(), M, (long long)M * M,
                                          s.d_trial.as<double>(), N, 0, &zero,
                                          s.d_Lbar.as<double>(), M, (long long)N * M, c->X));
    LOAF_CUBLAS(cublasDgemm(c->cublas, CUBLAS_OP_N, CUBLAS_OP_T, M, N, M, &one,
                            c->d_h.as<double>(), M, s.d_trial.as<double>(), N, &zero,
                            s.d_hbar.as<double>(), M));
}

void setup_load(loaf_ctx* c, int M, int X, const double* h, const double* L, int na, int nb,
                const double* ta, const double* tb, double e0, int on_device) {
    LOAF_REQUIRE(h && L && ta, LOAF_ERR_ARG, "h, L and trial_a are required");
    LOAF_REQUIRE(M >= 1 && M <= LOAF_MAX_BASIS, LOAF_ERR_SHAPE, "basis size out of range");
    LOAF_REQUIRE(X >= 1, LOAF_ERR_SHAPE, "need at least one Cholesky vector");
    const bool closed = (tb == nullptr);
    if (closed) nb = na;
    LOAF_REQUIRE(na >= 1 && na <= std::min(M, LOAF_MAX_NOCC), LOAF_ERR_SHAPE, "n_alpha out of range");
    LOAF_REQUIRE(nb >= 0 && nb <= std::min(M, LOAF_MAX_NOCC), LOAF_ERR_SHAPE, "n_beta out of range");
    LOAF_REQUIRE(closed || nb >= 1, LOAF_ERR_SHAPE, "open shell needs n_beta >= 1");

    for (auto& s : c->sp) s.release();
    for (auto& m : c->mix) m.release();
    c->loaded = c->compressed = c->localized = false;
    c->M = M; c->X = X; c->na = na; c->nb = nb; c->closed = closed; c->e0 = e0;
    c->nspin = closed ? 1 : 2;
    c->ntot = closed ? na : na + nb;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    c->d_h.ensure((size_t)M * M * sizeof(double));
    c->d_L.ensure((size_t)X * M * M * sizeof(double));
    LOAF_CUDA(cudaMemcpyAsync(c->d_h.ptr, h, (size_t)M * M * sizeof(double), kind, c->stream));
    LOAF_CUDA(cudaMemcpyAsync(c->d_L.ptr, L, (size_t)X * M * M * sizeof(double), kind, c->stream));
    for (int s = 0; s < c->nspin; ++s) {
        SpinData& sd = c->sp[s];
        sd.N = s == 0 ? na : nb;
        sd.col0 = s == 0 ? 0 : na;
        sd.mult = closed ? 2.0 : 1.0;
        const double* src = s == 0 ? ta : tb;
        sd.h_trial.resize((size_t)M * sd.N);
        if (on_device)
            LOAF_CUDA(cudaMemcpy(sd.h_trial.data(), src, sd.h_trial.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost));
        else
            std::copy(src, src + sd.h_trial.size(), sd.h_trial.begin());
        sd.d_trial.ensure(sd.h_trial.size() * sizeof(double));
        LOAF_CUDA(cudaMemcpyAsync(sd.d_trial.ptr, src, sd.h_trial.size() * sizeof(double), kind,
                                  c->stream));
    }
    LOAF_CUDA(cudaStreamSynchronize(c->stream));
    c->canonical[0] = c->sp[0].h_trial;
    c->canonical[1] = c->nspin > 1 ? c->sp[1].h_trial : std::vector<double>();
    for (int s = 0; s < c->nspin; ++s) half_rotate(c, c->sp[s]);
    LOAF_CUDA(cudaStreamSynchronize(c->stream));
    c->trial_version++;
    c->loaded = true;
}

// ---------------------------------------------------------------------------
// S2: Foster-Boys by Jacobi sweeps (host; N x N problem)
// ---------------------------------------------------------------------------

// Maximise sum_i sum_d (C^T r_d C)_ii^2 over orthogonal rotations of the
// columns of C (M x N row-major).  For pair (i, j) with a = R_ii, b = R_jj,
// m = R_ij (per operator d) the rotation i' = c i + s j, j' = -s i + c j by t
// changes the objective by P cos 4t + Q sin 4t + const with
// P = sum_d ((a - b)^2 / 4 - m^2) and Q = sum_d (a - b) m, so t = atan2(Q, P)/4.
static void boys_host(std::vector<double>& C, int M, int N, const double* r_ops, int n_ops,
                      double angle_tol = 1e-13, int max_sweeps = 1000) {
    if (N < 2 || n_ops < 1) return;
    std::vector<double> R((size_t)n_ops * N * N, 0.0), T((size_t)M * N);
    for (int d = 0; d < n_ops; ++d) {
        const double* r = r_ops + (size_t)d * M * M;
        // T = r_d C
        for (int p = 0; p < M; ++p)
            for (int i = 0; i < N; ++i) {
                double s = 0.0;
                for (int q = 0; q < M; ++q) s += r[(size_t)p * M + q] * C[(size_t)q * N + i];
                T[(size_t)p * N + i] = s;
            }
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                double s = 0.0;
                for (int p = 0; p < M; ++p) s += C[(size_t)p * N + i] * T[(size_t)p * N + j];
                R[((size_t)d * N + i) * N + j] = s;
            }
    }
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double biggest = 0.0;
        for (int i = 0; i < N - 1; ++i)
            for (int j = i + 1; j < N; ++j) {
                double P = 0.0, Q = 0.0;
                for (int d = 0; d < n_ops; ++d) {
                    const double* Rd = &R[(size_t)d * N * N];
                    const double a = Rd[i * N + i], b = Rd[j * N + j], m = Rd[i * N + j];
                    P += 0.25 * (a - b) * (a - b) - m * m;
                    Q += (a - b) * m;
                }
                const double t = 0.25 * std::atan2(Q, P);
                if (t == 0.0) continue;
                biggest = std::max(biggest, std::fabs(t));
                const double cs = std::cos(t), sn = std::sin(t);
                for (int p = 0; p < M; ++p) {
                    double& ci = C[(size_t)p * N + i];
                    double& cj = C[(size_t)p * N + j];
                    const double x = ci, y = cj;
                    ci = cs * x + sn * y;
                    cj = -sn * x + cs * y;
                }
                for (int d = 0; d < n_ops; ++d) {
                    double* Rd = &R[(size_t)d * N * N];
                    for (int k = 0; k < N; ++k) {  // columns
                        const double x = Rd[k * N + i], y = Rd[k * N + j];
                        Rd[k * N + i] = cs * x + sn * y;
                        Rd[k * N + j] = -sn * x + cs * y;
                    }
                    for (int k = 0; k < N; ++k) {  // rows
                        const double x = Rd[i * N + k], y = Rd[j * N + k];
                        Rd[i * N + k] = cs * x + sn * y;
                        Rd[j * N + k] = -sn * x + cs * y;
                    }
                }
            }
        if (biggest < angle_tol) break;
    }
}

// ---------------------------------------------------------------------------
// S3 kernels
// ---------------------------------------------------------------------------

namespace {

// Jordan-Wielandt matrix H (2M x 2M, column-major) of block Y (M x M column-
// major, leading dimension ldy): H[a, M + b] = Y[a, b], H[M + b, a] = Y[a, b]
__global__ void build_jw_kernel(int M, const double* __restrict__ Y, long ldy,
                                double* __restrict__ H) {
    const long n2 = 2L * M;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n2 * n2;
         e += (long)gridDim.x * blockDim.x) {
        const long a = e % n2, b = e / n2;  // row a, column b
        double v = 0.0;
        if (a < M && b >= M) v = Y[(b - M) * ldy + a];
        else if (a >= M && b < M) v = Y[(a - M) * ldy + b];
        H[e] = v;
    }
}

__global__ void copy_block_kernel(int M, const double* __restrict__ Y, long ldy,
                                  double* __restrict__ H) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)M * M;
         e += (long)gridDim.x * blockDim.x) {
        const long a = e % M, b = e / M;
        H[e] = Y[b * ldy + a];
    }
}

// From the eigenpairs (ascending) of a batch of problems, keep the kept
// singular triplets and write rows of Ubar^T and Vbar into per-pair slots
// of M rows each.  jw = 1: 2M x 2M Jordan-Wielandt problems; jw = 0: M x M
// symmetric blocks (eigenvalues may be tiny negative; at threshold 0 they
// are kept with their sign so the reconstruction stays exact).
__global__ void extract_factors_kernel(int M, int jw, double thr, const double* __restrict__ Z,
                                       const double* __restrict__ lam, const int* __restrict__ slot,
                                       double* __restrict__ Uslots, double* __restrict__ Vslots,
                                       int* __restrict__ Kout, double* __restrict__ sig3) {
    const int b = blockIdx.x;
    const long n = jw ? 2L * M : (long)M;
    const double* zb = Z + (size_t)b * n * n;
    const double* lb = lam + (size_t)b * n;
    // count kept values among the candidates (the top M eigenvalues)
    __shared__ int sK;
    if (threadIdx.x == 0) {
        int k = 0;
        for (int t = 0; t < M; ++t) {
            // jw: the top M eigenvalues +s_k, descending; symmetric: |lambda|
            const double sv = jw ? lb[n - 1 - t] : fabs(lb[t]);
            if (thr == 0.0 || sv >= thr) ++k;
        }
        sK = k;
        Kout[slot[b]] = k;
        // pair descriptors: the two largest singular values and sum s^2
        double s1 = 0.0, s2 = 0.0, ss = 0.0;
        for (int t = 0; t < M; ++t) {
            const double sv = jw ? fmax(lb[n - 1 - t], 0.0) : fabs(lb[t]);
            ss += sv * sv;
            if (sv > s1) { s2 = s1; s1 = sv; } else if (sv > s2) { s2 = sv; }
        }
        sig3[3 * slot[b]] = s1;
        sig3[3 * slot[b] + 1] = s2;
        sig3[3 * slot[b] + 2] = ss;
    }
    __syncthreads();
    const int K = sK;
    double* Us = Uslots + (size_t)slot[b] * M * M;
    double* Vs = Vslots + (size_t)slot[b] * M * M;
    if (jw) {
        // candidates in descending order: columns n-1, n-2, ...
        for (long e = threadIdx.x; e < (long)K * M; e += blockDim.x) {
            const int k = (int)(e / M), r = (int)(e % M);
            const long col = n - 1 - k;
            const double sv = fmax(lb[col], 0.0);
            const double f = sqrt(2.0 * sv);
            Us[(size_t)k * M + r] = f * zb[col * n + r];
            Vs[(size_t)k * M + r] = f * zb[col * n + M + r];
        }
    } else {
        // order by |lambda| descending: sort indices in shared memory (M <= 1536)
        extern __shared__ int order[];
        if (threadIdx.x == 0) {
            for (int t = 0; t < M; ++t) order[t] = t;
            // insertion sort by |lambda| descending (M is small, setup only)
            for (int t = 1; t < M; ++t) {
                const int v = order[t];
                const double key = fabs(lb[v]);
                int u = t - 1;
                while (u >= 0 && fabs(lb[order[u]]) < key) { order[u + 1] = order[u]; --u; }
                order[u + 1] = v;
            }
        }
        __syncthreads();
        for (long e = threadIdx.x; e < (long)K * M; e += blockDim.x) {
            const int k = (int)(e / M), r = (int)(e % M);
            const int col = order[k];
            const double l = lb[col];
            const double f = sqrt(fabs(l));
            const double z = zb[(size_t)col * n + r];
            Us[(size_t)k * M + r] = (l < 0.0 ? -f : f) * z;
            Vs[(size_t)k * M + r] = f * z;
        }
    }
}

__global__ void compact_rows_kernel(int M, const int* __restrict__ K, const long* __restrict__ off,
                                    const double* __restrict__ Uslots,
                                    const double* __restrict__ Vslots, double* __restrict__ U,
                                    double* __restrict__ V) {
    const int n = blockIdx.x;
    const long o = off[n];
    const int k = K[n];
    for (long e = threadIdx.x; e < (long)k * M; e += blockDim.x) {
        U[o * M + e] = Uslots[(size_t)n * M * M + e];
        V[o * M + e] = Vslots[(size_t)n * M * M + e];
    }
}

struct EigBatch {
    int n = 0, cap = 0;
    DevBuf A, lam, info, work, slots;
    std::vector<char> hwork;
    size_t dws = 0, hws = 0;
    std::vector<int> pending_slots;
};

}  // namespace

static void run_eig_batch(loaf_ctx* c, cusolverDnParams_t prm, EigBatch& eb, int M, bool jw,
                          double thr, double* Uslots, double* Vslots, int* dK, double* dSig) {
    const int cnt = (int)eb.pending_slots.size();
    if (cnt == 0) return;
    LOAF_CUDA(cudaMemcpyAsync(eb.slots.ptr, eb.pending_slots.data(), cnt * sizeof(int),
                              cudaMemcpyHostToDevice, c->stream));
    LOAF_CUSOLVER(cusolverDnXsyevBatched(c->cusolver, prm, CUSOLVER_EIG_MODE_VECTOR,
                                         CUBLAS_FILL_MODE_LOWER, eb.n, CUDA_R_64F, eb.A.ptr, eb.n,
                                         CUDA_R_64F, eb.lam.ptr, CUDA_R_64F, eb.work.ptr, eb.dws,
                                         eb.hwork.data(), eb.hws, eb.info.as<int>(), cnt));
    const size_t smem = jw ? 0 : (size_t)M * sizeof(int);
    extract_factors_kernel<<<cnt, 256, smem, c->stream>>>(M, jw ? 1 : 0, thr, eb.A.as<double>(),
                                                         eb.lam.as<double>(), eb.slots.as<int>(),
                                                         Uslots, Vslots, dK, dSig);
    LOAF_LAUNCH_CHECK();
    // the host-side slot list is reused by the next batch: wait for the copy
    LOAF_CUDA(cudaStreamSynchronize(c->stream));
    eb.pending_slots.clear();
}

static void prepare_batch(loaf_ctx* c, cusolverDnParams_t prm, EigBatch& eb, int n, int cap) {
    eb.n = n;
    eb.cap = cap;
    eb.A.ensure((size_t)cap * n * n * sizeof(double));
    eb.lam.ensure((size_t)cap * n * sizeof(double));
    eb.info.ensure((size_t)cap * sizeof(int));
    eb.slots.ensure((size_t)cap * sizeof(int));
    LOAF_CUSOLVER(cusolverDnXsyevBatched_bufferSize(
        c->cusolver, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F,
        eb.A.ptr, n, CUDA_R_64F, eb.lam.ptr, CUDA_R_64F, &eb.dws, &eb.hws, cap));
    eb.work.ensure(eb.dws + 16);
    eb.hwork.resize(eb.hws + 16);
}

// Pair Gram blocks, SVDs, truncation and packing for one spin.
static void compress_spin(loaf_ctx* c, SpinData& s, double thr) {
    const int M = c->M, N = s.N, X = c->X;
    PairTable& pt = s.pairs;
    pt.release();
    const int npairs = N * (N + 1) / 2;
    pt.npairs = npairs;
    for (int i = 0; i < N; ++i)
        for (int j = i; j < N; ++j) { pt.i.push_back(i); pt.j.push_back(j); }

    DevBuf Uslots, Vslots, dK, G, dSig;
    dSig.ensure((size_t)npairs * 3 * sizeof(double));
    Uslots.ensure((size_t)npairs * M * M * sizeof(double));
    Vslots.ensure((size_t)npairs * M * M * sizeof(double));
    dK.ensure((size_t)npairs * sizeof(int));
    G.ensure((size_t)M * N * M * sizeof(double));

    cusolverDnParams_t prm;
    LOAF_CUSOLVER(cusolverDnCreateParams(&prm));
    LOAF_CUSOLVER(cusolverDnSetStream(c->cusolver, c->stream));
    EigBatch off_b, diag_b;
    const int cap_off = std::max(1, std::min(32, npairs - N));
    prepare_batch(c, prm, off_b, 2 * M, cap_off);
    prepare_batch(c, prm, diag_b, M, std::min(N, 32));

    const double one = 1.0, zero = 0.0;
    LOAF_CUBLAS(cublasSetStream(c->cublas, c->stream));
    const long NM = (long)N * M;
    int slot = 0;
    const int threads = 256;
    try {
        for (int i = 0; i < N; ++i) {
            // G (column-major M x (N-i)M): G[r, (j-i)M + s] = sum_g Lbar[g][i][r] Lbar[g][j][s]
            const double* Ai = s.d_Lbar.as<double>() + (size_t)i * M;
            LOAF_CUBLAS(cublasDgemm(c->cublas, CUBLAS_OP_N, CUBLAS_OP_T, M, (N - i) * M, X, &one, Ai,
                                    NM, Ai, NM, &zero, G.as<double>(), M));
            for (int j = i; j < N; ++j, ++slot) {
                const double* Y = G.as<double>() + (size_t)(j - i) * M * M;
                if (i == j) {
                    double* H = diag_b.A.as<double>() + (size_t)diag_b.pending_slots.size() * M * M;
                    copy_block_kernel<<<std::min(1024, ceil_div((long)M * M, threads)), threads, 0,
                                        c->stream>>>(M, Y, M, H);
                    LOAF_LAUNCH_CHECK();
                    diag_b.pending_slots.push_back(slot);
                    if ((int)diag_b.pending_slots.size() == diag_b.cap)
                        run_eig_batch(c, prm, diag_b, M, false, thr, Uslots.as<double>(),
                                      Vslots.as<double>(), dK.as<int>(), dSig.as<double>());
                } else {
                    double* H = off_b.A.as<double>() +
                                (size_t)off_b.pending_slots.size() * 4 * M * M;
                    build_jw_kernel<<<std::min(2048, ceil_div(4L * M * M, threads)), threads, 0,
                                      c->stream>>>(M, Y, M, H);
                    LOAF_LAUNCH_CHECK();
                    off_b.pending_slots.push_back(slot);
                    if ((int)off_b.pending_slots.size() == off_b.cap)
                        run_eig_batch(c, prm, off_b, M, true, thr, Uslots.as<double>(),
                                      Vslots.as<double>(), dK.as<int>(), dSig.as<double>());
                }
            }
            // G is overwritten by the next row: flush what still points into it
            run_eig_batch(c, prm, diag_b, M, false, thr, Uslots.as<double>(), Vslots.as<double>(),
                          dK.as<int>(), dSig.as<double>());
            run_eig_batch(c, prm, off_b, M, true, thr, Uslots.as<double>(), Vslots.as<double>(),
                          dK.as<int>(), dSig.as<double>());
        }
    } catch (...) {
        cusolverDnDestroyParams(prm);
        throw;
    }
    cusolverDnDestroyParams(prm);

    pt.K.resize(npairs);
    pt.sig.resize((size_t)npairs * 3);
    LOAF_CUDA(cudaMemcpyAsync(pt.K.data(), dK.ptr, npairs * sizeof(int), cudaMemcpyDeviceToHost,
                              c->stream));
    LOAF_CUDA(cudaMemcpyAsync(pt.sig.data(), dSig.ptr, pt.sig.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
    LOAF_CUDA(cudaStreamSynchronize(c->stream));
    pt.off.resize(npairs);
    long rows = 0;
    for (int n = 0; n < npairs; ++n) { pt.off[n] = rows; rows += pt.K[n]; }
    pt.rows = rows;
    pt.d_U.ensure(std::max<long>(rows, 1) * M * sizeof(double));
    pt.d_V.ensure(std::max<long>(rows, 1) * M * sizeof(double));
    pt.d_i.ensure(npairs * sizeof(int));
    pt.d_j.ensure(npairs * sizeof(int));
    pt.d_K.ensure(npairs * sizeof(int));
    pt.d_off.ensure(npairs * sizeof(long));
    LOAF_CUDA(cudaMemcpyAsync(pt.d_i.ptr, pt.i.data(), npairs * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    LOAF_CUDA(cudaMemcpyAsync(pt.d_j.ptr, pt.j.data(), npairs * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    LOAF_CUDA(cudaMemcpyAsync(pt.d_K.ptr, pt.K.data(), npairs * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    LOAF_CUDA(cudaMemcpyAsync(pt.d_off.ptr, pt.off.data(), npairs * sizeof(long), cudaMemcpyHostToDevice, c->stream));
    compact_rows_kernel<<<npairs, 256, 0, c->stream>>>(M, pt.d_K.as<int>(), pt.d_off.as<long>(),
                                                       Uslots.as<double>(), Vslots.as<double>(),
                                                       pt.d_U.as<double>(), pt.d_V.as<double>());
    LOAF_LAUNCH_CHECK();
    LOAF_CUDA(cudaStreamSynchronize(c->stream));
}

// Eight walker-independent descriptors per pair [ij] for the pair screen:
// centroid distance d, 1/(1+d), s_i + s_j, |s_i - s_j|, log s_1, log s_2,
// M_SVD/M and log |Y^[ij]|_F, with centroid c_i = <i|r_d|i> and spread
// s_i = sqrt(sum_d |r_d i|^2 - c_id^2) of the (localized) trial orbitals.
static void pair_features_host(loaf_ctx* c, const double* r_ops, int n_ops) {
    const int M = c->M;
    c->features.clear();
    auto lg = [](double v) { return std::log(std::max(v, 1e-300)); };
    for (int s = 0; s < c->nspin; ++s) {
        const SpinData& sd = c->sp[s];
        const int N = sd.N;
        std::vector<double> cen((size_t)N * 3, 0.0), sq((size_t)N * 3, 0.0), spread(N, 0.0);
        for (int d = 0; d < std::min(n_ops, 3) && r_ops; ++d) {
            const double* r = r_ops + (size_t)d * M * M;
            for (int i = 0; i < N; ++i) {
                double cc = 0.0, nn = 0.0;
                for (int p = 0; p < M; ++p) {
                    double rc = 0.0;
                    for (int q = 0; q < M; ++q) rc += r[(size_t)p * M + q] * sd.h_trial[(size_t)q * N + i];
                    cc += sd.h_trial[(size_t)p * N + i] * rc;
                    nn += rc * rc;
                }
                cen[i * 3 + d] = cc;
                sq[i * 3 + d] = nn;
            }
        }
        for (int i = 0; i < N; ++i) {
            double v = 0.0;
            for (int d = 0; d < 3; ++d) v += sq[i * 3 + d] - cen[i * 3 + d] * cen[i * 3 + d];
            spread[i] = std::sqrt(std::max(v, 0.0));
        }
        const PairTable& pt = sd.pairs;
        for (int n = 0; n < pt.npairs; ++n) {
            const int i = pt.i[n], j = pt.j[n];
            double dd = 0.0;
            for (int d = 0; d < 3; ++d) dd += (cen[i * 3 + d] - cen[j * 3 + d]) * (cen[i * 3 + d] - cen[j * 3 + d]);
            dd = std::sqrt(dd);
            const double f[8] = {dd, 1.0 / (1.0 + dd), spread[i] + spread[j],
                                 std::fabs(spread[i] - spread[j]), lg(pt.sig[3 * n]),
                                 lg(pt.sig[3 * n + 1]), (double)pt.K[n] / M, 0.5 * lg(pt.sig[3 * n + 2])};
            c->features.insert(c->features.end(), f, f + 8);
        }
    }
}

void setup_compress(loaf_ctx* c, double t_svd, const double* r_ops, int n_ops, int localize,
                    double* pct, int* m_svd) {
    LOAF_REQUIRE(c->loaded, LOAF_ERR_NOT_READY, "ao_load_cholesky has not been called");
    LOAF_REQUIRE(t_svd >= 0.0 && std::isfinite(t_svd), LOAF_ERR_ARG, "t_svd must be finite and >= 0");
    LOAF_REQUIRE(!localize || (r_ops && n_ops >= 1), LOAF_ERR_ARG,
                 "localization needs the position operators");
    c->compressed = false;
    for (auto& m : c->mix) m.release();
    for (int s = 0; s < c->nspin; ++s) {
        SpinData& sd = c->sp[s];
        std::vector<double> C = c->canonical[s];
        if (localize) boys_host(C, c->M, sd.N, r_ops, n_ops);
        sd.h_trial = C;
        LOAF_CUDA(cudaMemcpyAsync(sd.d_trial.ptr, C.data(), C.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, c->stream));
        for (auto& m : sd.sLbar) m.release();
        c->trial_version++;
        half_rotate(c, sd);
        compress_spin(c, sd, t_svd);
    }
    c->localized = localize != 0;
    c->t_svd = t_svd;
    c->compressed = true;
    pair_features_host(c, r_ops, n_ops);
    c->keep.clear();
    c->screen_version++;
    long tot = 0, cnt = 0;
    int k = 0;
    for (int s = 0; s < c->nspin; ++s)
        for (int n = 0; n < c->sp[s].pairs.npairs; ++n) {
            tot += c->sp[s].pairs.K[n];
            ++cnt;
            if (m_svd) m_svd[k] = c->sp[s].pairs.K[n];
            ++k;
        }
    if (pct) *pct = cnt ? (c->M - (double)tot / cnt) / c->M * 100.0 : 0.0;
}

}  // namespace loaf
