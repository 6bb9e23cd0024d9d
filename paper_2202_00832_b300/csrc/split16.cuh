// 16-bit hi + lo splitting of FP64 values for the tensor-core contractions:
// v ~= hi + lo with hi = fp16(v) (or bf16) and lo = fp16(v - hi), after a
// power-of-two scale that puts the largest |value| of a row in [2^13, 2^14).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

namespace loaf {
namespace {

template <bool BF16> struct Half16;
template <> struct Half16<false> {
    __device__ static uint16_t from(double v, double& back) {
        const __half h = __double2half(v);
        back = (double)__half2float(h);
        return __half_as_ushort(h);
    }
};
template <> struct Half16<true> {
    __device__ static uint16_t from(double v, double& back) {
        const __nv_bfloat16 h = __double2bfloat16(v);
        back = (double)__bfloat162float(h);
        return __bfloat16_as_ushort(h);
    }
};

template <bool BF16>
__device__ inline void split16(double v, uint16_t& hi, uint16_t& lo) {
    double b;
    hi = Half16<BF16>::from(v, b);
    double b2;
    lo = Half16<BF16>::from(v - b, b2);
}

// power-of-two scale putting the largest |value| in [2^13, 2^14)
__device__ inline double pow2_scale(double maxabs) {
    if (!(maxabs > 0.0) || !isfinite(maxabs)) return 1.0;
    int e;
    frexp(maxabs, &e);  // maxabs = f * 2^e, f in [0.5, 1)
    return ldexp(1.0, 14 - e);
}

__device__ inline double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double m = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, red[k]);
    return m;
}

}  // namespace
}  // namespace loaf
