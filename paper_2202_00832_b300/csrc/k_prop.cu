// Propagator one-body operator of every walker: V_w = sum_g x_wg L_g (M x M),
// the B = sum_alpha x_alpha L_alpha formation of the propagation step (the
// Hubbard-Stratonovich one-body operators of Sec. 2.1; its cost is weighed
// against the energy's in Sec. 5).  The fields x arrive already scaled by
// sqrt(dtau) and shifted by the force bias.
//
// Split precision: one tensor-core contraction over the Cholesky index g,
//   part[pq][2w + ri] = sum_g L^T[pq][g] x_ri[w][g],
// with L^T (rows pq, per-row power-of-two scale) tiled once per molecule and
// the fields (rows (w, re/im), per-row scale) tiled per call, both as 16-bit
// hi + lo pre-swizzled 128 x 64 tiles; the contraction's epilogue unscales and
// writes the walker-major output.  FP64: two cuBLAS DGEMMs (re and im of x).
#include "common.cuh"
#include "split16.cuh"

#include <algorithm>

namespace loaf {

namespace {

// per pq: power-of-two scale of row pq of L^T (largest |L_g,pq| over g)
__global__ void lt_scale_kernel(int X, long MM, const double* __restrict__ L, double* __restrict__ sc,
                                float* __restrict__ inv) {
    const long pq = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pq >= MM) return;
    double m = 0.0;
    for (int g = 0; g < X; ++g) m = fmax(m, fabs(L[(size_t)g * MM + pq]));
    const double s = pow2_scale(m);
    sc[pq] = s;
    inv[pq] = (float)(1.0 / s);
}

// tile (mt, kb) of L^T: rows pq = 128 mt + r, columns g = 64 kb + k; the threads
// of a warp take consecutive rows so that each read of L is coalesced
template <bool BF16>
__global__ void lt_tiles_kernel(int X, long MM, int nkb, const double* __restrict__ L,
                                const double* __restrict__ sc, uint16_t* __restrict__ hi,
                                uint16_t* __restrict__ lo) {
    const int mt = blockIdx.x, kb = blockIdx.y;
    uint16_t* th = hi + ((size_t)mt * nkb + kb) * kTileElems;
    uint16_t* tl = lo + ((size_t)mt * nkb + kb) * kTileElems;
    for (int q = threadIdx.x; q < kTileRows * 8; q += blockDim.x) {
        const int r = q & (kTileRows - 1), chunk = q >> 7;
        const long pq = (long)mt * kTileRows + r;
        const double s = pq < MM ? sc[pq] : 0.0;
        __align__(16) uint16_t h[8], l[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int g = kb * kTileK + chunk * 8 + j;
            const double v = (pq < MM && g < X) ? L[(size_t)g * MM + pq] * s : 0.0;
            split16<BF16>(v, h[j], l[j]);
        }
        const int e = sw128_elem(r, chunk * 8);
        *reinterpret_cast<uint4*>(th + e) = *reinterpret_cast<const uint4*>(h);
        *reinterpret_cast<uint4*>(tl + e) = *reinterpret_cast<const uint4*>(l);
    }
}

// field rows z = 2w + ri (re, im) with a power-of-two scale each, as tiles [rb][kb]
template <bool BF16>
__global__ void x_tiles_kernel(int X, int nkb, const double2* __restrict__ x, uint16_t* __restrict__ hi,
                               uint16_t* __restrict__ lo, float* __restrict__ inv) {
    __shared__ double red[32];
    const int z = blockIdx.x, w = z >> 1, ri = z & 1;
    const double2* xw = x + (size_t)w * X;
    double m = 0.0;
    for (int g = threadIdx.x; g < X; g += blockDim.x) m = fmax(m, fabs(ri ? xw[g].y : xw[g].x));
    const double s = pow2_scale(block_max(m, red));
    if (threadIdx.x == 0) inv[z] = (float)(1.0 / s);
    const int r = z & (kTileRows - 1), rb = z >> 7;
    for (int g = threadIdx.x; g < nkb * kTileK; g += blockDim.x) {
        const double v = g < X ? (ri ? xw[g].y : xw[g].x) * s : 0.0;
        uint16_t h, l;
        split16<BF16>(v, h, l);
        const size_t o = ((size_t)rb * nkb + (g >> 6)) * kTileElems + sw128_elem(r, g & 63);
        hi[o] = h;
        lo[o] = l;
    }
}

// FP64 path: the fields' real and imaginary parts as separate row-major planes
__global__ void x_deinterleave_kernel(long n, const double2* __restrict__ x, double* __restrict__ xr,
                                      double* __restrict__ xi) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) {
        xr[e] = x[e].x;
        xi[e] = x[e].y;
    }
}
__global__ void v_interleave_kernel(long n, const double* __restrict__ vr, const double* __restrict__ vi,
                                    double2* __restrict__ V) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) V[e] = make_double2(vr[e], vi[e]);
}

void ensure_prop_ops(loaf_ctx* c, MixedOps& mx, bool bf16) {
    if (mx.prop_ready) return;
    const long MM = (long)c->M * c->M;
    mx.prop_nkb = ceil_div(c->X, kTileK);
    mx.prop_nmt = (int)((MM + kTileRows - 1) / kTileRows);
    const size_t tb = (size_t)mx.prop_nmt * mx.prop_nkb * kTileBytes;
    mx.Lt_hi.ensure(tb);
    mx.Lt_lo.ensure(tb);
    mx.Lt_inv.ensure((size_t)MM * sizeof(float));
    DevBuf sc;
    sc.ensure((size_t)MM * sizeof(double));
    lt_scale_kernel<<<ceil_div(MM, 256), 256, 0, c->stream>>>(c->X, MM, c->d_L.as<double>(), sc.as<double>(),
                                                            mx.Lt_inv.as<float>());
    LOAF_LAUNCH_CHECK();
    const dim3 grid(mx.prop_nmt, mx.prop_nkb);
    if (bf16)
        lt_tiles_kernel<true><<<grid, 256, 0, c->stream>>>(c->X, MM, mx.prop_nkb, c->d_L.as<double>(),
                                                          sc.as<double>(), mx.Lt_hi.as<uint16_t>(),
                                                          mx.Lt_lo.as<uint16_t>());
    else
        lt_tiles_kernel<false><<<grid, 256, 0, c->stream>>>(c->X, MM, mx.prop_nkb, c->d_L.as<double>(),
                                                           sc.as<double>(), mx.Lt_hi.as<uint16_t>(),
                                                           mx.Lt_lo.as<uint16_t>());
    LOAF_LAUNCH_CHECK();
    LOAF_CUDA(cudaStreamSynchronize(c->stream));  // sc goes out of scope
    mx.prop_ready = true;
}

}  // namespace

void run_propagator(loaf_ctx* c, int W, const double2* x, int precision, double2* V) {
    const long MM = (long)c->M * c->M;
    if (precision == LOAF_PREC_FP64) {
        const size_t nx = (size_t)W * c->X, nv = (size_t)W * MM;
        c->w_prop_x.ensure(2 * nx * sizeof(double));
        c->w_prop_part.ensure(2 * nv * sizeof(double));
        double* xr = c->w_prop_x.as<double>();
        double* xi = xr + nx;
        double* vr = c->w_prop_part.as<double>();
        double* vi = vr + nv;
        x_deinterleave_kernel<<<ceil_div((long)nx, 256), 256, 0, c->stream>>>((long)nx, x, xr, xi);
        LOAF_LAUNCH_CHECK();
        // column-major: V_re (MM x W) = L (MM x X, ld MM) * x_re (X x W, ld X)
        const double one = 1.0, zero = 0.0;
        LOAF_CUBLAS(cublasSetStream(c->cublas, c->stream));
        LOAF_CUBLAS(cublasDgemm(c->cublas, CUBLAS_OP_N, CUBLAS_OP_N, (int)MM, W, c->X, &one, c->d_L.as<double>(),
                                (int)MM, xr, c->X, &zero, vr, (int)MM));
        LOAF_CUBLAS(cublasDgemm(c->cublas, CUBLAS_OP_N, CUBLAS_OP_N, (int)MM, W, c->X, &one, c->d_L.as<double>(),
                                (int)MM, xi, c->X, &zero, vi, (int)MM));
        v_interleave_kernel<<<ceil_div((long)nv, 256), 256, 0, c->stream>>>((long)nv, vr, vi, V);
        LOAF_LAUNCH_CHECK();
        return;
    }
    const bool bf16 = precision == LOAF_PREC_BF16X3;
    MixedOps& mx = c->mix[bf16 ? 1 : 0];
    ensure_prop_ops(c, mx, bf16);
    const int nkb = mx.prop_nkb;
    const int nrb = ceil_div(2 * W, kTileRows);
    const int n_wt = nrb;  // 128 field rows = 64 walkers per output tile
    const int ldp = n_wt * kTileRows;
    const size_t xb = (size_t)nrb * nkb * kTileBytes;
    c->w_prop_x.ensure_zeroed(2 * xb + (size_t)2 * W * sizeof(float) + 256, c->stream);
    uint16_t* x_hi = c->w_prop_x.as<uint16_t>();
    uint16_t* x_lo = x_hi + xb / 2;
    float* inv_x = reinterpret_cast<float*>(c->w_prop_x.as<uint8_t>() + 2 * xb);
    c->w_flag.ensure(16);
    LOAF_CUDA(cudaMemsetAsync(c->w_flag.ptr, 0, sizeof(int), c->stream));
    StageScope sc(c, "propagator_tc", 2);
    if (bf16)
        x_tiles_kernel<true><<<2 * W, 256, 0, c->stream>>>(c->X, nkb, x, x_hi, x_lo, inv_x);
    else
        x_tiles_kernel<false><<<2 * W, 256, 0, c->stream>>>(c->X, nkb, x, x_hi, x_lo, inv_x);
    LOAF_LAUNCH_CHECK();
    // the contraction's epilogue writes V[w][pq] directly (scaled), no FP64 table
    tc_split_gemm(c, mx.Lt_hi.as<uint16_t>(), mx.Lt_lo.as<uint16_t>(), (int)MM, mx.prop_nmt, x_hi, x_lo, nrb,
                  n_wt, nkb, bf16, nullptr, ldp, c->w_flag.as<int>(), V, mx.Lt_inv.as<float>(), inv_x, MM, W);
}

}  // namespace loaf
