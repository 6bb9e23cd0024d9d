// Learned pair screen (a refinement the paper's conclusions propose: keep only
// the electron pairs that contribute meaningfully).  A network 8 -> 64 -> 64 -> 1
// with tanh hidden layers predicts log10 of the largest |e_ij| of a pair over a
// set of training walkers from eight walker-independent descriptors; pairs
// predicted below a cutoff are left out of the LO exchange.
//
// Arithmetic: FP16 weights and activations, FP32 accumulation, FP32 master
// weights; full-batch Adam.  One CTA of 64 threads (one per hidden unit) runs
// samples one after another and keeps its gradient rows in registers; the
// per-CTA partial gradients are summed in a fixed order by the Adam kernel.
#include "common.cuh"

#include <algorithm>
#include <cmath>

namespace loaf {
namespace {

constexpr int kF = 8, kH = 64;
constexpr int oW1 = 0, ob1 = oW1 + kH * kF, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH, kNP = ob3 + 1;
constexpr int kPart = kNP + 1;  // per-CTA partial: gradient, then the summed squared error

__global__ void __launch_bounds__(kH)
mlp_fwd_bwd_kernel(int n, const __half* __restrict__ x, const float* __restrict__ t,
                   const float* __restrict__ prm, float* __restrict__ part, float* __restrict__ y_out,
                   int backward) {
    __shared__ __half sW1[kH * kF], sW2[kH * kH], sW3[kH];
    __shared__ float sb1[kH], sb2[kH], sb3;
    __shared__ __half sx[kF], sh1[kH];
    __shared__ float sda2[kH], sred[2];
    const int k = threadIdx.x, lane = k & 31, warp = k >> 5;
    for (int e = k; e < kH * kF; e += kH) sW1[e] = __float2half(prm[oW1 + e]);
    for (int e = k; e < kH * kH; e += kH) sW2[e] = __float2half(prm[oW2 + e]);
    sW3[k] = __float2half(prm[oW3 + k]);
    sb1[k] = prm[ob1 + k];
    sb2[k] = prm[ob2 + k];
    if (k == 0) sb3 = prm[ob3];
    float gW1[kF], gW2[kH];
#pragma unroll
    for (int i = 0; i < kF; ++i) gW1[i] = 0.f;
#pragma unroll
    for (int j = 0; j < kH; ++j) gW2[j] = 0.f;
    float gb1 = 0.f, gb2 = 0.f, gW3 = 0.f, gb3 = 0.f, lsum = 0.f;
    const int s0 = (int)((long)blockIdx.x * n / gridDim.x);
    const int s1 = (int)((long)(blockIdx.x + 1) * n / gridDim.x);
    __syncthreads();
    for (int s = s0; s < s1; ++s) {
        if (k < kF) sx[k] = x[(size_t)s * kF + k];
        __syncthreads();
        float a1 = sb1[k];
#pragma unroll
        for (int i = 0; i < kF; ++i) a1 = fmaf(__half2float(sW1[k * kF + i]), __half2float(sx[i]), a1);
        const __half h1 = __float2half(tanhf(a1));
        sh1[k] = h1;
        __syncthreads();
        float a2 = sb2[k];
#pragma unroll 16
        for (int j = 0; j < kH; ++j) a2 = fmaf(__half2float(sW2[k * kH + j]), __half2float(sh1[j]), a2);
        const float h2f = __half2float(__float2half(tanhf(a2)));
        float c = __half2float(sW3[k]) * h2f;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) sred[warp] = c;
        __syncthreads();
        const float y = sb3 + sred[0] + sred[1];
        if (y_out && k == 0) y_out[s] = y;
        if (backward) {
            const float r = y - t[s];
            const float dy = 2.f * r / (float)n;
            if (k == 0) { gb3 += dy; lsum = fmaf(r, r, lsum); }
            gW3 = fmaf(dy, h2f, gW3);
            const float da2 = dy * __half2float(sW3[k]) * (1.f - h2f * h2f);
            sda2[k] = da2;
            gb2 += da2;
#pragma unroll
            for (int j = 0; j < kH; ++j) gW2[j] = fmaf(da2, __half2float(sh1[j]), gW2[j]);
            __syncthreads();
            float dh1 = 0.f;
#pragma unroll 16
            for (int m = 0; m < kH; ++m) dh1 = fmaf(sda2[m], __half2float(sW2[m * kH + k]), dh1);
            const float h1f = __half2float(h1);
            const float da1 = dh1 * (1.f - h1f * h1f);
            gb1 += da1;
#pragma unroll
            for (int i = 0; i < kF; ++i) gW1[i] = fmaf(da1, __half2float(sx[i]), gW1[i]);
        }
        __syncthreads();  // sx, sh1, sda2 and sred are rewritten by the next sample
    }
    if (!backward) return;
    float* p = part + (size_t)blockIdx.x * kPart;
#pragma unroll
    for (int i = 0; i < kF; ++i) p[oW1 + k * kF + i] = gW1[i];
    p[ob1 + k] = gb1;
#pragma unroll
    for (int j = 0; j < kH; ++j) p[oW2 + k * kH + j] = gW2[j];
    p[ob2 + k] = gb2;
    p[oW3 + k] = gW3;
    if (k == 0) { p[ob3] = gb3; p[kNP] = lsum; }
}

// Fixed-order sum of the per-CTA partials; then either one Adam step on the
// FP32 master weights (step >= 1) or a plain copy of the gradient (step 0).
__global__ void mlp_reduce_adam_kernel(int nblk, int n, const float* __restrict__ part,
                                       float* __restrict__ prm, float* __restrict__ m1,
                                       float* __restrict__ m2, float lr, int step,
                                       float* __restrict__ grad_out, float* __restrict__ loss_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kNP) return;
    float g = 0.f;
    for (int b = 0; b < nblk; ++b) g += part[(size_t)b * kPart + p];
    if (p == kNP) {
        if (loss_out) loss_out[step > 0 ? step - 1 : 0] = g / (float)n;
        return;
    }
    if (step == 0) {
        grad_out[p] = g;
        return;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mm = b1 * m1[p] + (1.f - b1) * g;
    const float vv = b2 * m2[p] + (1.f - b2) * g * g;
    m1[p] = mm;
    m2[p] = vv;
    const float mh = mm / (1.f - powf(b1, (float)step));
    const float vh = vv / (1.f - powf(b2, (float)step));
    prm[p] -= lr * mh / (sqrtf(vh) + eps);
}

int mlp_grid(int n) { return std::max(1, std::min(296, (n + 7) / 8)); }

struct MlpBuffers {
    DevBuf x, t, prm, m1, m2, part, y, loss, grad;
    void size(int n, int epochs) {
        const int g = mlp_grid(n);
        x.ensure((size_t)std::max(n, 1) * kF * sizeof(__half));
        t.ensure((size_t)std::max(n, 1) * sizeof(float));
        prm.ensure(kNP * sizeof(float));
        m1.ensure(kNP * sizeof(float));
        m2.ensure(kNP * sizeof(float));
        part.ensure((size_t)g * kPart * sizeof(float));
        y.ensure((size_t)std::max(n, 1) * sizeof(float));
        loss.ensure((size_t)std::max(epochs, 1) * sizeof(float));
        grad.ensure(kNP * sizeof(float));
    }
};

void upload_x(cudaStream_t st, DevBuf& d, const std::vector<float>& xs) {
    std::vector<__half> h(xs.size());
    for (size_t e = 0; e < xs.size(); ++e) h[e] = __float2half(xs[e]);
    LOAF_CUDA(cudaMemcpyAsync(d.ptr, h.data(), h.size() * sizeof(__half), cudaMemcpyHostToDevice, st));
    LOAF_CUDA(cudaStreamSynchronize(st));
}

template <class F>
loaf_status guard(loaf_ctx* c, F&& f) {
    try {
        f();
        if (c) c->err.clear();
        return LOAF_OK;
    } catch (const Error& e) {
        if (c) c->err = e.msg;
        return e.code;
    }
}

}  // namespace
}  // namespace loaf

using namespace loaf;

extern "C" int loaf_screen_num_params(void) { return kNP; }

extern "C" loaf_status mlp_loss_grad(int device, int n, const float* x, const float* t,
                                     const float* params, float* loss_out, float* grad_out) {
    if (n < 1 || !x || !t || !params || !grad_out) return LOAF_ERR_ARG;
    return guard(nullptr, [&] {
        LOAF_CUDA(cudaSetDevice(device));
        cudaStream_t st;
        LOAF_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        MlpBuffers b;
        try {
            b.size(n, 1);
            upload_x(st, b.x, std::vector<float>(x, x + (size_t)n * kF));
            LOAF_CUDA(cudaMemcpyAsync(b.t.ptr, t, n * sizeof(float), cudaMemcpyHostToDevice, st));
            LOAF_CUDA(cudaMemcpyAsync(b.prm.ptr, params, kNP * sizeof(float), cudaMemcpyHostToDevice, st));
            const int g = mlp_grid(n);
            mlp_fwd_bwd_kernel<<<g, kH, 0, st>>>(n, b.x.as<__half>(), b.t.as<float>(), b.prm.as<float>(),
                                                b.part.as<float>(), nullptr, 1);
            LOAF_LAUNCH_CHECK();
            mlp_reduce_adam_kernel<<<ceil_div(kNP + 1, 256), 256, 0, st>>>(
                g, n, b.part.as<float>(), b.prm.as<float>(), nullptr, nullptr, 0.f, 0, b.grad.as<float>(),
                b.loss.as<float>());
            LOAF_LAUNCH_CHECK();
            float l = 0.f;
            LOAF_CUDA(cudaMemcpyAsync(grad_out, b.grad.ptr, kNP * sizeof(float), cudaMemcpyDeviceToHost, st));
            LOAF_CUDA(cudaMemcpyAsync(&l, b.loss.ptr, sizeof(float), cudaMemcpyDeviceToHost, st));
            LOAF_CUDA(cudaStreamSynchronize(st));
            if (loss_out) *loss_out = l;
        } catch (...) {
            cudaStreamDestroy(st);
            throw;
        }
        cudaStreamDestroy(st);
    });
}

extern "C" loaf_status pair_screen_train(loaf_ctx* c, int W_train, const void* phi, int epochs,
                                         float lr, const float* init_params, float* loss_history) {
    if (!c) return LOAF_ERR_ARG;
    return guard(c, [&] {
        drain_submitted(c);
        LOAF_REQUIRE(c->compressed, LOAF_ERR_NOT_READY, "pair_screen_train needs lo_localize_compress");
        LOAF_REQUIRE(W_train >= 1 && phi && epochs >= 1 && lr > 0.f && init_params, LOAF_ERR_ARG,
                     "pair_screen_train: W_train, phi, epochs, lr and init_params are required");
        LOAF_CUDA(cudaSetDevice(c->device));
        // labels: the method's own pair contributions on the training walkers
        c->keep.clear();
        c->screen_version++;
        const int np = loaf_num_pairs(c);
        std::vector<double> ep((size_t)np * W_train * 2);
        const loaf_status st = walkers_pair_exchange(c, W_train, phi, LOAF_PREC_FP16X3, ep.data());
        if (st != LOAF_OK) throw Error{st, "pair_screen_train: " + c->err};
        c->mlp_target.assign(np, -300.0);
        for (int p = 0; p < np; ++p) {
            double mx = 0.0;
            for (int w = 0; w < W_train; ++w)
                mx = std::max(mx, std::hypot(ep[((size_t)p * W_train + w) * 2], ep[((size_t)p * W_train + w) * 2 + 1]));
            c->mlp_target[p] = std::log10(std::max(mx, 1e-300));
        }
        // standardise descriptors and targets with the training set's moments
        for (int f = 0; f < kF; ++f) {
            double s = 0.0, s2 = 0.0;
            for (int p = 0; p < np; ++p) s += c->features[(size_t)p * kF + f];
            const double mu = s / np;
            for (int p = 0; p < np; ++p) {
                const double d = c->features[(size_t)p * kF + f] - mu;
                s2 += d * d;
            }
            const double sd = std::sqrt(s2 / np);
            c->feat_mu[f] = mu;
            c->feat_sd[f] = sd > 0.0 ? sd : 1.0;
        }
        {
            double s = 0.0, s2 = 0.0;
            for (double v : c->mlp_target) s += v;
            c->tgt_mu = s / np;
            for (double v : c->mlp_target) s2 += (v - c->tgt_mu) * (v - c->tgt_mu);
            const double sd = std::sqrt(s2 / np);
            c->tgt_sd = sd > 0.0 ? sd : 1.0;
        }
        std::vector<float> xs((size_t)np * kF), ts(np);
        for (int p = 0; p < np; ++p) {
            for (int f = 0; f < kF; ++f)
                xs[(size_t)p * kF + f] = (float)((c->features[(size_t)p * kF + f] - c->feat_mu[f]) / c->feat_sd[f]);
            ts[p] = (float)((c->mlp_target[p] - c->tgt_mu) / c->tgt_sd);
        }
        MlpBuffers b;
        b.size(np, epochs);
        upload_x(c->stream, b.x, xs);
        LOAF_CUDA(cudaMemcpyAsync(b.t.ptr, ts.data(), np * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        LOAF_CUDA(cudaMemcpyAsync(b.prm.ptr, init_params, kNP * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        LOAF_CUDA(cudaMemsetAsync(b.m1.ptr, 0, kNP * sizeof(float), c->stream));
        LOAF_CUDA(cudaMemsetAsync(b.m2.ptr, 0, kNP * sizeof(float), c->stream));
        const int g = mlp_grid(np);
        for (int e = 1; e <= epochs; ++e) {
            mlp_fwd_bwd_kernel<<<g, kH, 0, c->stream>>>(np, b.x.as<__half>(), b.t.as<float>(),
                                                       b.prm.as<float>(), b.part.as<float>(), nullptr, 1);
            LOAF_LAUNCH_CHECK();
            mlp_reduce_adam_kernel<<<ceil_div(kNP + 1, 256), 256, 0, c->stream>>>(
                g, np, b.part.as<float>(), b.prm.as<float>(), b.m1.as<float>(), b.m2.as<float>(), lr, e,
                nullptr, b.loss.as<float>());
            LOAF_LAUNCH_CHECK();
        }
        // predictions of every pair with the trained weights
        mlp_fwd_bwd_kernel<<<g, kH, 0, c->stream>>>(np, b.x.as<__half>(), b.t.as<float>(), b.prm.as<float>(),
                                                   b.part.as<float>(), b.y.as<float>(), 0);
        LOAF_LAUNCH_CHECK();
        std::vector<float> y(np);
        c->mlp_params.assign(kNP, 0.f);
        LOAF_CUDA(cudaMemcpyAsync(c->mlp_params.data(), b.prm.ptr, kNP * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        LOAF_CUDA(cudaMemcpyAsync(y.data(), b.y.ptr, np * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        if (loss_history)
            LOAF_CUDA(cudaMemcpyAsync(loss_history, b.loss.ptr, epochs * sizeof(float), cudaMemcpyDeviceToHost,
                                      c->stream));
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
        c->mlp_pred.resize(np);
        for (int p = 0; p < np; ++p) c->mlp_pred[p] = c->tgt_mu + c->tgt_sd * y[p];
    });
}

extern "C" loaf_status pair_screen_set(loaf_ctx* c, double cutoff_ha, int* kept_pairs) {
    if (!c) return LOAF_ERR_ARG;
    return guard(c, [&] {
        drain_submitted(c);
        LOAF_REQUIRE(c->compressed, LOAF_ERR_NOT_READY, "pair_screen_set needs lo_localize_compress");
        const int np = loaf_num_pairs(c);
        if (cutoff_ha < 0.0) {
            c->keep.clear();
        } else {
            LOAF_REQUIRE((int)c->mlp_pred.size() == np, LOAF_ERR_NOT_READY,
                         "pair_screen_set needs pair_screen_train");
            const double lc = std::log10(std::max(cutoff_ha, 1e-300));
            c->keep.assign(np, 1);
            for (int p = 0; p < np; ++p) c->keep[p] = c->mlp_pred[p] >= lc ? 1 : 0;
        }
        c->screen_version++;
        if (kept_pairs) {
            int k = np;
            if (!c->keep.empty()) k = (int)std::count(c->keep.begin(), c->keep.end(), (unsigned char)1);
            *kept_pairs = k;
        }
    });
}

extern "C" loaf_status pair_screen_query(const loaf_ctx* c, float* params_out, double* features_out,
                                         double* pred_log10_out, double* target_log10_out,
                                         unsigned char* keep_out) {
    if (!c) return LOAF_ERR_ARG;
    if (!c->compressed) return LOAF_ERR_NOT_READY;
    const int np = loaf_num_pairs(c);
    if (features_out) std::copy(c->features.begin(), c->features.end(), features_out);
    const bool trained = (int)c->mlp_pred.size() == np;
    if ((params_out || pred_log10_out || target_log10_out) && !trained) return LOAF_ERR_NOT_READY;
    if (params_out) std::copy(c->mlp_params.begin(), c->mlp_params.end(), params_out);
    if (pred_log10_out) std::copy(c->mlp_pred.begin(), c->mlp_pred.end(), pred_log10_out);
    if (target_log10_out) std::copy(c->mlp_target.begin(), c->mlp_target.end(), target_log10_out);
    if (keep_out) {
        for (int p = 0; p < np; ++p) keep_out[p] = c->keep.empty() ? 1 : c->keep[p];
    }
    return LOAF_OK;
}
