// Multi-determinant (CAS) trial: mixed-estimate local energy through
// Sherman-Morrison-Woodbury updates of the reference determinant (Sec. 3.1.2:
// eqs. Q_SMW_reg, Q_SMW, BigQ, 2e_HR_RCAS and the intermediates table), FP64.
//
// The context holds the CAS orbitals as its (closed-shell) trial, so its
// half-rotated vectors Lbar (X x n_cas x M), hbar (n_cas x M) and the pair
// factors of every CAS orbital pair [ij] (packed FP64 rows) serve here as they
// are.  Per walker (N occupied orbitals per spin, both spins alike):
//   B = C^T phi (n_cas x N): the overlap of every CAS orbital with the walker;
//   A = rows of the reference's orbitals, A^-1 and log det A (Gauss-Jordan with
//   partial pivoting); Theta^0 = phi A^-1;
//   projections of the reference columns: Ubar^[ij]T Theta^0 and
//   Vbar^[ij] Theta^0 for every packed factor row, hbar Theta^0 and
//   Lbar_g Theta^0 for every g;
//   per determinant d (slots s_1..s_k holding new orbitals): V^T A^-1 from the
//   changed rows of B, M_d = I + V^T A^-1 U (k x k), S_d = M_d^-1 V^T A^-1 and
//   the overlap ratio det M_d; every column of Q^d is the reference column
//   minus the excited-slot columns times S_d, applied to the projections
//   (eq. BigQ), which gives E1, E_J and E_K of the determinant;
//   E = sum_d c_d r_d^2 E_d / sum_d c_d r_d^2 (closed shell: r_d^2).
#include "common.cuh"
#include "dfloat.cuh"

namespace loaf {

namespace {

constexpr int kCasMaxN = 64;    // occupied orbitals per determinant
constexpr int kCasMaxExc = 8;   // changed slots per determinant
constexpr int kCasThreads = 256;

__device__ inline double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ inline double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ inline double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ inline double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ inline double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ inline double2 zinv(double2 a) {
    const double d = zabs2(a);
    return make_double2(a.x / d, -a.y / d);
}
__device__ inline double2 zmad(double2 acc, double2 a, double2 b) {  // acc + a b
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}

__device__ double2 block_sum2(double2 v, double2* red) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = zadd(t, red[k]);
    return t;
}

// B[w][o][j] = sum_p C[p][o] phi[w][p][j]; grid (W, n_cas), threads over j
__global__ void cas_overlap_kernel(int M, int Nc, int N, const double* __restrict__ C,
                                   const double2* __restrict__ phi, double2* __restrict__ B) {
    const int w = blockIdx.x, o = blockIdx.y;
    const double2* pw = phi + (size_t)w * M * N;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int p = 0; p < M; ++p) {
            const double c = C[(size_t)p * Nc + o];
            const double2 v = pw[(size_t)p * N + j];
            acc.x = fma(c, v.x, acc.x);
            acc.y = fma(c, v.y, acc.y);
        }
        B[((size_t)w * Nc + o) * N + j] = acc;
    }
}

// one CTA per walker: A = rows ref[s] of B, A^-1 by Gauss-Jordan with partial
// pivoting (rows exchanged, then the columns exchanged back in reverse order),
// log det A = sum log pivot + i pi (exchanges mod 2); a pivot below
// N 2^-52 max|A| marks the walker singular
__global__ void __launch_bounds__(kCasThreads)
cas_inverse_kernel(int N, int Nc, const int* __restrict__ ref, const double2* __restrict__ B,
                   double2* __restrict__ Ainv, double2* __restrict__ logdet, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char sm[];
    double2* A = reinterpret_cast<double2*>(sm);  // N x N
    double2* colk = A + N * N;                    // N
    __shared__ double red_m[32];
    __shared__ double s_max;
    __shared__ int s_p, s_flag, s_swaps, s_perm[kCasMaxN];
    __shared__ double2 s_inv, s_piv[kCasMaxN];
    const int w = blockIdx.x, tid = threadIdx.x;
    double m = 0.0;
    for (int e = tid; e < N * N; e += blockDim.x) {
        const int s = e / N, j = e - s * N;
        const double2 v = B[((size_t)w * Nc + ref[s]) * N + j];
        A[e] = v;
        m = fmax(m, zabs2(v));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) red_m[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmax(t, red_m[k]);
        s_max = t;
        s_flag = (t == t && t < INFINITY) ? 0 : 2;
        s_swaps = 0;
    }
    __syncthreads();
    const double tol = (double)N * 2.220446049250313e-16 * sqrt(s_max);
    for (int k = 0; k < N && s_flag == 0; ++k) {
        if (tid < 32) {
            double best = -1.0;
            int bi = k;
            for (int i = k + tid; i < N; i += 32) {
                const double v = zabs2(A[i * N + k]);
                if (v > best) { best = v; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                s_p = bi;
                s_perm[k] = bi;
                if (bi != k) s_swaps += 1;
                const double2 pv = A[bi * N + k];
                if (!(sqrt(zabs2(pv)) > tol)) {
                    s_flag = 1;
                } else {
                    s_piv[k] = pv;
                    s_inv = zinv(pv);
                }
            }
        }
        __syncthreads();
        if (s_flag) break;
        const int p = s_p;
        if (p != k)
            for (int j = tid; j < N; j += blockDim.x) {
                const double2 t = A[k * N + j];
                A[k * N + j] = A[p * N + j];
                A[p * N + j] = t;
            }
        __syncthreads();
        for (int i = tid; i < N; i += blockDim.x) colk[i] = A[i * N + k];
        __syncthreads();
        const double2 inv = s_inv;
        for (int j = tid; j < N; j += blockDim.x) A[k * N + j] = j == k ? inv : zmul(A[k * N + j], inv);
        __syncthreads();
        for (int e = tid; e < N * N; e += blockDim.x) {
            const int i = e / N, j = e - i * N;
            if (i == k) continue;
            const double2 f = colk[i];
            A[e] = j == k ? zmul(make_double2(-f.x, -f.y), inv) : zsub(A[e], zmul(f, A[k * N + j]));
        }
        __syncthreads();
    }
    const int flag = s_flag;
    if (flag == 0) {
        for (int k = N - 1; k >= 0; --k) {
            const int p = s_perm[k];
            if (p != k)
                for (int i = tid; i < N; i += blockDim.x) {
                    const double2 t = A[i * N + k];
                    A[i * N + k] = A[i * N + p];
                    A[i * N + p] = t;
                }
            __syncthreads();
        }
        for (int e = tid; e < N * N; e += blockDim.x) Ainv[(size_t)w * N * N + e] = A[e];
    }
    if (tid == 0) {
        double2 ld = make_double2(0.0, 0.0);
        if (flag == 0) {
            for (int k = 0; k < N; ++k) {
                ld.x += log(sqrt(zabs2(s_piv[k])));
                ld.y += atan2(s_piv[k].y, s_piv[k].x);
            }
            if (s_swaps & 1) ld.y += 3.141592653589793;
            ld.y = remainder(ld.y, 6.283185307179586);
        } else {
            ld = make_double2(-INFINITY, 0.0);
        }
        logdet[w] = ld;
        status[w] = flag == 0 ? LOAF_WALKER_OK : (flag == 1 ? LOAF_WALKER_SINGULAR : LOAF_WALKER_NAN);
    }
}

// Theta^0[w][r][s] = sum_j phi[w][r][j] A^-1[w][j][s]
__global__ void cas_theta_kernel(int M, int N, const double2* __restrict__ phi, const double2* __restrict__ Ainv,
                                 double2* __restrict__ th0) {
    const int w = blockIdx.x;
    const long e = (long)blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= (long)M * N) return;
    const int r = (int)(e / N), s = (int)(e - (long)r * N);
    const double2* pr = phi + ((size_t)w * M + r) * N;
    const double2* ai = Ainv + (size_t)w * N * N;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < N; ++j) acc = zmad(acc, pr[j], ai[j * N + s]);
    th0[(size_t)w * M * N + e] = acc;
}

// Projections of the reference columns, only those a determinant can use
// (eq. BigQ and the intermediates table): column 0 is the fixed slot of the
// row's orbital (the slot it holds in every determinant, if any; else zeros),
// columns 1..nv the variable slots (those some determinant changes).
//   out[w * out_stride + row C + c] = sum_r F[row][r] Theta^0[w][r][slot(row, c)]
// The row's orbital: mode 0, orbital b of its pair (Ubar rows), mode 1,
// orbital a (Vbar rows), mode 2, row mod Nc (Lbar and hbar rows).
// Computed on the FP32 pipe in double-float (about 48 significant bits: the
// FP64 results to ~1e-14 relative, at B300's FP32 rate instead of its FP64
// rate, about 1/64 of it).  A CTA takes 64 rows and kProjW walkers; the
// factor rows and the walkers' Theta^0 rows are staged kProjRB at a time in
// shared memory, split into hi + lo as they are stored.  Each thread keeps the
// double-float sums of one (row, walker) for up to kProjC columns at a time.
constexpr int kProjRows = 64, kProjW = 4, kProjRB = 16, kProjC = 6;
__global__ void __launch_bounds__(kProjRows * kProjW, 3)
cas_project_df_kernel(int M, int N, int C, long rows, int W, const double* __restrict__ F,
                      const double2* __restrict__ th0, double2* __restrict__ out, size_t out_stride, int mode,
                      int Nc, const int* __restrict__ row_pair, const int* __restrict__ pa,
                      const int* __restrict__ pb, const int* __restrict__ fixed_slot,
                      const int* __restrict__ var_slot) {
    extern __shared__ __align__(16) unsigned char sm[];
    // strides padded so that the 4 walkers' and the 8 rows' values of a warp's
    // loads fall in different banks
    const int th_w = kProjRB * N + 1;                                                  // float4 per walker
    float4* th = reinterpret_cast<float4*>(sm);                                        // [kProjW][kProjRB][N]
    float2* fs = reinterpret_cast<float2*>(th + (size_t)kProjW * th_w);                // [kProjRows][kProjRB + 1]
    const int tid = threadIdx.x;
    const int wq = tid % kProjW, rl = tid / kProjW;
    const int w0 = blockIdx.y * kProjW;
    const int nw = min(kProjW, W - w0);
    const long row0 = (long)blockIdx.x * kProjRows;
    const long row = row0 + rl;
    const bool active = row < rows && wq < nw;
    int orb = 0;
    if (active) orb = mode == 0 ? pb[row_pair[row]] : mode == 1 ? pa[row_pair[row]] : (int)(row % Nc);
    for (int cb = 0; cb < C; cb += kProjC) {
        int sl[kProjC];
#pragma unroll
        for (int q = 0; q < kProjC; ++q) {
            const int c = cb + q;
            sl[q] = c >= C ? -1 : (c > 0 ? var_slot[c - 1] : fixed_slot[orb]);
        }
        // (re, im) as the two lanes of one packed double-float per column
        dfl2 acc[kProjC];
#pragma unroll
        for (int q = 0; q < kProjC; ++q) acc[q] = dfl2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        for (int r0 = 0; r0 < M; r0 += kProjRB) {
            const int nr = min(kProjRB, M - r0);
            __syncthreads();  // the previous block's reads are done
            for (int e = tid; e < kProjW * nr * N; e += blockDim.x) {
                const int ww = e / (nr * N), rem = e - ww * nr * N;
                const int r = rem / N, sidx = rem - r * N;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (ww < nw) {
                    const double2 z = th0[((size_t)(w0 + ww) * M + r0 + r) * N + sidx];
                    const dfl a = df_split_bits(z.x), b = df_split_bits(z.y);
                    v = make_float4(a.hi, b.hi, a.lo, b.lo);  // {re.hi, im.hi, re.lo, im.lo}
                }
                th[(size_t)ww * th_w + r * N + sidx] = v;
            }
            for (int e = tid; e < kProjRows * nr; e += blockDim.x) {
                const int rr = e / nr, r = e - rr * nr;
                float2 v = make_float2(0.f, 0.f);
                if (row0 + rr < rows) {
                    const dfl a = df_split_bits(F[(size_t)(row0 + rr) * M + r0 + r]);
                    v = make_float2(a.hi, a.lo);
                }
                fs[rr * (kProjRB + 1) + r] = v;
            }
            __syncthreads();
            if (active) {
                const float4* thw = th + (size_t)wq * th_w;
                for (int r = 0; r < nr; ++r) {
                    const float2 f2 = fs[rl * (kProjRB + 1) + r];
                    const dfl2 fv{make_float2(f2.x, f2.x), make_float2(f2.y, f2.y)};
#pragma unroll
                    for (int q = 0; q < kProjC; ++q) {
                        if (sl[q] < 0) continue;
                        const float4 t = thw[r * N + sl[q]];
                        acc[q] = df2_fma(fv, dfl2{make_float2(t.x, t.y), make_float2(t.z, t.w)}, acc[q]);
                    }
                }
            }
        }
        if (active) {
#pragma unroll
            for (int q = 0; q < kProjC; ++q) {
                const int c = cb + q;
                if (c < C)
                    out[(size_t)(w0 + wq) * out_stride + (size_t)row * C + c] =
                        make_double2(df_to(dfl{acc[q].hi.x, acc[q].lo.x}), df_to(dfl{acc[q].hi.y, acc[q].lo.y}));
            }
        }
    }
}

struct CasParams {
    int M, N, Nc, X, n_det;
    int C;                      // projected columns: fixed slot + variable slots
    const int* slot_col;        // N: column of each slot (0 for fixed slots)
    long R;                     // packed factor rows
    const int* dets;            // n_det x N
    const int* pair_id;         // Nc x Nc: pair index of (min, max)
    const int* K;               // per pair
    const long* off;            // per pair
    const double2* B;           // [W][Nc][N]
    const double2* Ainv;        // [W][N][N]
    const double2* PL;          // [W][R][C]
    const double2* PR;          // [W][R][C]
    const double2* PJ;          // [W][X + 1][Nc][C]; plane X: hbar Theta^0
    const double2* G;           // [walker - w0][pair][C][C]: sum over the pair's rows of PL[c1] PR[c2]
    int w0;                     // first walker of this launch
    int npairs;
    double e0;
    double2* Ed;                // [W][n_det]
    double2* rd;                // [W][n_det]
};

// The pair Gram blocks of the exchange (the determinant-independent
// intermediates of the table of Sec. 3.1.2): for every stored CAS orbital pair
// n = [ab] and walker, G_n[c1][c2] = sum over the pair's kept ranks of
// (Ubar^[ab]T Theta^0)[c1] (Vbar^[ab] Theta^0)[c2], c1, c2 over the projected
// columns.  A determinant's pair value (Ubar^T Q^d_t) . (Vbar Q^d_s) is then a
// bilinear form in G with the SMW coefficients S_d (eq. BigQ), so the ranks
// are summed once per walker instead of once per determinant.
// grid (pairs, walkers of the slice), threads over (c1, c2)
__global__ void cas_pair_gram_kernel(int C, const long* __restrict__ off, const int* __restrict__ K,
                                     const double2* __restrict__ PL, const double2* __restrict__ PR, long R,
                                     int npairs, int w0, double2* __restrict__ G) {
    const int n = blockIdx.x, ws = blockIdx.y, w = w0 + ws;
    const long o = off[n];
    const int Kn = K[n];
    const double2* pl = PL + ((size_t)w * R + o) * C;
    const double2* pr = PR + ((size_t)w * R + o) * C;
    double2* g = G + ((size_t)ws * npairs + n) * C * C;
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
        const int c1 = e / C, c2 = e - c1 * C;
        double2 acc = make_double2(0.0, 0.0);
        for (int kk = 0; kk < Kn; ++kk) acc = zmad(acc, pl[(size_t)kk * C + c1], pr[(size_t)kk * C + c2]);
        g[e] = acc;
    }
}

// one CTA per (determinant, walker): S_d, the overlap ratio and E_d
__global__ void __launch_bounds__(kCasThreads) cas_det_energy_kernel(CasParams P) {
    const int d = blockIdx.x, ws = blockIdx.y, w = P.w0 + ws, tid = threadIdx.x;
    const int N = P.N, Nc = P.Nc;
    __shared__ int occ[kCasMaxN], slot[kCasMaxExc], neworb[kCasMaxExc], oldorb[kCasMaxExc];
    __shared__ int s_k, s_sing;
    __shared__ double2 VA[kCasMaxExc][kCasMaxN];   // V^T A^-1
    __shared__ double2 LU[kCasMaxExc][kCasMaxExc];
    __shared__ int piv[kCasMaxExc];
    __shared__ double2 S[kCasMaxExc][kCasMaxN];
    __shared__ double2 s_ratio;
    __shared__ double2 red[32];
    const int* det = P.dets + (size_t)d * N;
    const int* ref = P.dets;
    for (int s = tid; s < N; s += blockDim.x) occ[s] = det[s];
    if (tid == 0) {
        int k = 0;
        for (int s = 0; s < N && k < kCasMaxExc; ++s)
            if (det[s] != ref[s]) { slot[k] = s; neworb[k] = det[s]; oldorb[k] = ref[s]; ++k; }
        s_k = k;
        s_sing = 0;
    }
    __syncthreads();
    const int k = s_k;
    const double2* Bw = P.B + (size_t)w * Nc * N;
    const double2* Ai = P.Ainv + (size_t)w * N * N;
    // V^T A^-1: row e = (B[new_e] - B[old_e]) A^-1
    for (int e = tid; e < k * N; e += blockDim.x) {
        const int r = e / N, s = e - r * N;
        double2 acc = make_double2(0.0, 0.0);
        for (int j = 0; j < N; ++j)
            acc = zmad(acc, zsub(Bw[(size_t)neworb[r] * N + j], Bw[(size_t)oldorb[r] * N + j]), Ai[j * N + s]);
        VA[r][s] = acc;
    }
    __syncthreads();
    // M_d = I + V^T A^-1 U (columns = the changed slots), LU with partial pivoting
    if (tid == 0) {
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b) {
                LU[a][b] = VA[a][slot[b]];
                if (a == b) LU[a][b].x += 1.0;
            }
        double2 det_m = make_double2(1.0, 0.0);
        for (int c = 0; c < k; ++c) {
            int p = c;
            for (int r = c + 1; r < k; ++r)
                if (zabs2(LU[r][c]) > zabs2(LU[p][c])) p = r;
            piv[c] = p;
            if (p != c) {
                for (int b = 0; b < k; ++b) { const double2 t = LU[c][b]; LU[c][b] = LU[p][b]; LU[p][b] = t; }
                det_m = make_double2(-det_m.x, -det_m.y);
            }
            if (!(zabs2(LU[c][c]) > 0.0)) { s_sing = 1; break; }
            det_m = zmul(det_m, LU[c][c]);
            const double2 ic = zinv(LU[c][c]);
            for (int r = c + 1; r < k; ++r) {
                const double2 f = zmul(LU[r][c], ic);
                LU[r][c] = f;
                for (int b = c + 1; b < k; ++b) LU[r][b] = zsub(LU[r][b], zmul(f, LU[c][b]));
            }
        }
        s_ratio = s_sing ? make_double2(0.0, 0.0) : det_m;
    }
    __syncthreads();
    const bool sing = s_sing != 0;
    // S_d = M_d^-1 V^T A^-1, one column s per thread
    for (int s = tid; s < N && !sing; s += blockDim.x) {
        double2 x[kCasMaxExc];
        for (int a = 0; a < k; ++a) x[a] = VA[a][s];
        for (int c = 0; c < k; ++c)
            if (piv[c] != c) { const double2 t = x[c]; x[c] = x[piv[c]]; x[piv[c]] = t; }
        for (int r = 1; r < k; ++r)
            for (int c = 0; c < r; ++c) x[r] = zsub(x[r], zmul(LU[r][c], x[c]));
        for (int r = k - 1; r >= 0; --r) {
            for (int c = r + 1; c < k; ++c) x[r] = zsub(x[r], zmul(LU[r][c], x[c]));
            x[r] = zmul(x[r], zinv(LU[r][r]));
        }
        for (int a = 0; a < k; ++a) S[a][s] = x[a];
    }
    __syncthreads();
    if (sing) {
        // zero overlap with this walker: weight 0
        if (tid == 0) {
            P.Ed[(size_t)w * P.n_det + d] = make_double2(0.0, 0.0);
            P.rd[(size_t)w * P.n_det + d] = make_double2(0.0, 0.0);
        }
        return;
    }
    // column s of Q^d projected by a row: ref[row][s] - sum_e ref[row][slot_e] S[e][s]
    // (projections stored by column: slot_col maps a slot to its column)
    const int* scol = P.slot_col;
    auto qcol = [&](const double2* rowp, int s) {
        double2 v = rowp[scol[s]];
        for (int e = 0; e < k; ++e) v = zsub(v, zmul(rowp[scol[slot[e]]], S[e][s]));
        return v;
    };
    const int Cc = P.C;
    const size_t plane = (size_t)Nc * Cc;
    const double2* PJw = P.PJ + (size_t)w * (P.X + 1) * plane;
    // one-body: 2 sum_s hbar[occ_s] . Q^d_s
    double2 e1 = make_double2(0.0, 0.0);
    for (int s = tid; s < N; s += blockDim.x) e1 = zadd(e1, qcol(PJw + (size_t)P.X * plane + (size_t)occ[s] * Cc, s));
    e1 = zscale(block_sum2(e1, red), 2.0);
    // Coulomb: J_g = 2 sum_s Lbar_g[occ_s] . Q^d_s, E_J = 1/2 sum_g J_g^2
    double2 ej = make_double2(0.0, 0.0);
    for (int g = tid; g < P.X; g += blockDim.x) {
        double2 J = make_double2(0.0, 0.0);
        for (int s = 0; s < N; ++s) J = zadd(J, qcol(PJw + (size_t)g * plane + (size_t)occ[s] * Cc, s));
        J = zscale(J, 2.0);
        ej = zadd(ej, zmul(J, J));
    }
    ej = zscale(block_sum2(ej, red), 0.5);
    // exchange: sum_{s,t} (Ubar^[ij]T Q_t) . (Vbar^[ij] Q_s), (i, j) = (occ_s, occ_t);
    // for i > j the [ji] factors with U and V exchanged (Y^[ij] = Y^[ji]T).  In
    // both cases the Ubar rows of the stored pair (a, b) = (min, max) meet the
    // column of b's slot and the Vbar rows that of a's slot.  With Q_t = col_t -
    // sum_e col(slot_e) S[e][t] on both sides, the sum over the pair's ranks is
    //   G(ct, cs) - sum_f S[f][s] G(ct, c_f) - sum_e S[e][t] G(c_e, cs)
    //   + sum_{e,f} S[e][t] S[f][s] G(c_e, c_f)
    // with G the pair's Gram block (transposed for i > j), ct = col of slot t,
    // c_e = col of the e-th changed slot.
    const double2* Gw = P.G + (size_t)ws * P.npairs * Cc * Cc;
    double2 ek = make_double2(0.0, 0.0);
    for (int e = tid; e < N * N; e += blockDim.x) {
        const int s = e / N, t = e - s * N;
        const int i = occ[s], j = occ[t];
        const int n = P.pair_id[(size_t)min(i, j) * Nc + max(i, j)];
        const double2* g = Gw + (size_t)n * Cc * Cc;
        const bool fwd = i <= j;
        auto gat = [&](int cl, int cr) { return fwd ? g[cl * Cc + cr] : g[cr * Cc + cl]; };
        const int ct = scol[t], cs = scol[s];
        double2 v = gat(ct, cs);
        for (int f = 0; f < k; ++f) v = zsub(v, zmul(S[f][s], gat(ct, scol[slot[f]])));
        for (int e2 = 0; e2 < k; ++e2) {
            const int ce = scol[slot[e2]];
            double2 inner = gat(ce, cs);
            for (int f = 0; f < k; ++f) inner = zsub(inner, zmul(S[f][s], gat(ce, scol[slot[f]])));
            v = zsub(v, zmul(S[e2][t], inner));
        }
        ek = zadd(ek, v);
    }
    ek = block_sum2(ek, red);
    if (tid == 0) {
        P.Ed[(size_t)w * P.n_det + d] = make_double2(P.e0 + e1.x + ej.x - ek.x, e1.y + ej.y - ek.y);
        P.rd[(size_t)w * P.n_det + d] = s_ratio;
    }
}

// E = sum_d c_d r_d^2 E_d / sum_d c_d r_d^2; log overlap = 2 log det A + log sum_d c_d r_d^2
__global__ void cas_combine_kernel(int W, int n_det, const double* __restrict__ coeffs,
                                   const double2* __restrict__ Ed, const double2* __restrict__ rd,
                                   const double2* __restrict__ logdetA, const int* __restrict__ status,
                                   double2* __restrict__ e_out, double2* __restrict__ logov_out) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    if (status[w] != LOAF_WALKER_OK) {
        e_out[w] = make_double2(NAN, NAN);
        logov_out[w] = make_double2(-INFINITY, 0.0);
        return;
    }
    double2 num = make_double2(0.0, 0.0), den = make_double2(0.0, 0.0);
    for (int d = 0; d < n_det; ++d) {
        const double2 r = rd[(size_t)w * n_det + d];
        const double2 cw = zscale(zmul(r, r), coeffs[d]);
        den = zadd(den, cw);
        num = zadd(num, zmul(cw, Ed[(size_t)w * n_det + d]));
    }
    const double dd = zabs2(den);
    e_out[w] = make_double2((num.x * den.x + num.y * den.y) / dd, (num.y * den.x - num.x * den.y) / dd);
    const double2 la = logdetA[w];
    logov_out[w] = make_double2(2.0 * la.x + 0.5 * log(dd),
                                remainder(2.0 * la.y + atan2(den.y, den.x), 6.283185307179586));
}

}  // namespace

void cas_check_dets(int N, int Nc, int n_det, const int* dets) {
    LOAF_REQUIRE(n_det >= 1, LOAF_ERR_ARG, "need at least the reference determinant");
    LOAF_REQUIRE(N >= 1 && N <= kCasMaxN && N <= Nc, LOAF_ERR_SHAPE,
                 "occupied orbitals per determinant must be 1..min(64, CAS orbitals)");
    for (int d = 0; d < n_det; ++d) {
        std::vector<char> seen(Nc, 0);
        int k = 0;
        for (int s = 0; s < N; ++s) {
            const int o = dets[(size_t)d * N + s];
            LOAF_REQUIRE(o >= 0 && o < Nc, LOAF_ERR_ARG, "orbital index outside the CAS orbitals");
            LOAF_REQUIRE(!seen[o], LOAF_ERR_ARG, "an orbital appears twice in one determinant");
            seen[o] = 1;
            if (o != dets[s]) ++k;
        }
        LOAF_REQUIRE(k <= kCasMaxExc, LOAF_ERR_SHAPE, "a determinant changes more than 8 slots of the reference");
    }
}

void run_energy_cas(loaf_ctx* c, int W, int N, const double2* phi, int n_det, const int* h_dets,
                    const double* h_coeffs, double2* e_dev, double2* logov_dev, int* status_dev) {
    SpinData& sp = c->sp[0];
    PairTable& pt = sp.pairs;
    const int M = c->M, X = c->X, Nc = sp.N;
    const long R = pt.rows;
    // pair index of (min, max); packed row -> pair
    std::vector<int> pid((size_t)Nc * Nc, 0);
    for (int n = 0; n < pt.npairs; ++n) pid[(size_t)pt.i[n] * Nc + pt.j[n]] = n;
    std::vector<int> row_pair(std::max<long>(R, 1), 0);
    for (int n = 0; n < pt.npairs; ++n)
        for (int k = 0; k < pt.K[n]; ++k) row_pair[pt.off[n] + k] = n;
    // variable slots (changed by some determinant) and the fixed slot of each orbital
    std::vector<char> var(N, 0);
    for (int d = 1; d < n_det; ++d)
        for (int s = 0; s < N; ++s)
            if (h_dets[(size_t)d * N + s] != h_dets[s]) var[s] = 1;
    std::vector<int> var_slot, slot_col(N, 0), fixed_slot(Nc, -1);
    for (int s = 0; s < N; ++s) {
        if (var[s]) {
            slot_col[s] = 1 + (int)var_slot.size();
            var_slot.push_back(s);
        } else {
            fixed_slot[h_dets[s]] = s;
        }
    }
    const int C = 1 + (int)var_slot.size();
    const size_t per_w = (size_t)Nc * N + (size_t)N * N + (size_t)M * N + 2 * (size_t)R * C +
                         (size_t)(X + 1) * Nc * C + 2 * (size_t)n_det + 1;
    const size_t n_int = (size_t)n_det * N + 1 + pid.size() + row_pair.size() + var_slot.size() + N + Nc + 8;
    // pair Gram blocks for a slice of walkers at a time (at most 512 MB of them)
    const int npairs = pt.npairs;
    const size_t g_per_w = (size_t)std::max(npairs, 1) * C * C;
    const int Ws = (int)std::max<size_t>(1, std::min<size_t>((size_t)W, ((size_t)512 << 20) / (g_per_w * sizeof(double2))));
    c->w_cas.ensure((size_t)W * per_w * sizeof(double2) + (size_t)Ws * g_per_w * sizeof(double2) +
                    (size_t)n_det * sizeof(double) + n_int * sizeof(int) + 4096);
    double2* B = c->w_cas.as<double2>();
    double2* Ainv = B + (size_t)W * Nc * N;
    double2* th0 = Ainv + (size_t)W * N * N;
    double2* PL = th0 + (size_t)W * M * N;
    double2* PR = PL + (size_t)W * R * C;
    double2* PJ = PR + (size_t)W * R * C;
    double2* Ed = PJ + (size_t)W * (X + 1) * Nc * C;
    double2* rd = Ed + (size_t)W * n_det;
    double2* ldA = rd + (size_t)W * n_det;
    double2* Gbuf = ldA + W;
    double* d_coeffs = reinterpret_cast<double*>(Gbuf + (size_t)Ws * g_per_w);
    int* d_dets = reinterpret_cast<int*>(d_coeffs + n_det);
    int* d_pid = d_dets + (size_t)n_det * N;
    int* d_row_pair = d_pid + pid.size();
    int* d_var = d_row_pair + row_pair.size();
    int* d_slot_col = d_var + std::max<size_t>(var_slot.size(), 1);
    int* d_fixed = d_slot_col + N;
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (bytes) LOAF_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    };
    up(d_coeffs, h_coeffs, (size_t)n_det * sizeof(double));
    up(d_dets, h_dets, (size_t)n_det * N * sizeof(int));
    up(d_pid, pid.data(), pid.size() * sizeof(int));
    up(d_row_pair, row_pair.data(), row_pair.size() * sizeof(int));
    up(d_var, var_slot.data(), var_slot.size() * sizeof(int));
    up(d_slot_col, slot_col.data(), (size_t)N * sizeof(int));
    up(d_fixed, fixed_slot.data(), (size_t)Nc * sizeof(int));
    StageScope sc(c, "cas_energy", (R > 0 ? 7 : 5) + 2 * ceil_div(W, Ws));
    cas_overlap_kernel<<<dim3(W, Nc), 64, 0, c->stream>>>(M, Nc, N, sp.d_trial.as<double>(), phi, B);
    LOAF_LAUNCH_CHECK();
    const size_t smem = (size_t)(N * N + N) * sizeof(double2);
    LOAF_CUDA(cudaFuncSetAttribute(cas_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cas_inverse_kernel<<<W, kCasThreads, smem, c->stream>>>(N, Nc, d_dets, B, Ainv, ldA, status_dev);
    LOAF_LAUNCH_CHECK();
    cas_theta_kernel<<<dim3(W, ceil_div((long)M * N, 256)), 256, 0, c->stream>>>(M, N, phi, Ainv, th0);
    LOAF_LAUNCH_CHECK();
    const int* pa = pt.d_i.as<int>();
    const int* pb = pt.d_j.as<int>();
    const size_t proj_smem = (size_t)kProjW * (kProjRB * N + 1) * sizeof(float4) +
                             (size_t)kProjRows * (kProjRB + 1) * sizeof(float2);
    LOAF_CUDA(cudaFuncSetAttribute(cas_project_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem));
    auto project = [&](const double* F, long rows, double2* out, size_t stride, int mode) {
        if (rows <= 0) return;
        cas_project_df_kernel<<<dim3(ceil_div(rows, kProjRows), ceil_div(W, kProjW)), kProjRows * kProjW, proj_smem,
                                c->stream>>>(M, N, C, rows, W, F, th0, out, stride, mode, Nc, d_row_pair, pa, pb,
                                             d_fixed, d_var);
        LOAF_LAUNCH_CHECK();
    };
    project(pt.d_U.as<double>(), R, PL, (size_t)R * C, 0);
    project(pt.d_V.as<double>(), R, PR, (size_t)R * C, 1);
    // planes g < X: Lbar_g Theta^0 (the X Nc Lbar rows are contiguous); plane X: hbar Theta^0
    const size_t pj_stride = (size_t)(X + 1) * Nc * C;
    project(sp.d_Lbar.as<double>(), (long)X * Nc, PJ, pj_stride, 2);
    project(sp.d_hbar.as<double>(), Nc, PJ + (size_t)X * Nc * C, pj_stride, 2);
    CasParams P;
    P.M = M; P.N = N; P.Nc = Nc; P.X = X; P.n_det = n_det; P.R = R; P.C = C; P.slot_col = d_slot_col;
    P.dets = d_dets; P.pair_id = d_pid; P.K = pt.d_K.as<int>(); P.off = pt.d_off.as<long>();
    P.B = B; P.Ainv = Ainv; P.PL = PL; P.PR = PR; P.PJ = PJ; P.e0 = c->e0; P.Ed = Ed; P.rd = rd;
    P.G = Gbuf; P.npairs = npairs;
    for (int w0 = 0; w0 < W; w0 += Ws) {
        const int wn = std::min(Ws, W - w0);
        if (npairs > 0) {
            cas_pair_gram_kernel<<<dim3(npairs, wn), 128, 0, c->stream>>>(C, pt.d_off.as<long>(), pt.d_K.as<int>(),
                                                                        PL, PR, R, npairs, w0, Gbuf);
            LOAF_LAUNCH_CHECK();
        }
        P.w0 = w0;
        cas_det_energy_kernel<<<dim3(n_det, wn), kCasThreads, 0, c->stream>>>(P);
        LOAF_LAUNCH_CHECK();
    }
    cas_combine_kernel<<<ceil_div(W, 128), 128, 0, c->stream>>>(W, n_det, d_coeffs, Ed, rd, ldA, status_dev, e_dev,
                                                                logov_dev);
    LOAF_LAUNCH_CHECK();
}

}  // namespace loaf
