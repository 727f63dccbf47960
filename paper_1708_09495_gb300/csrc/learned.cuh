// The learned-bucket model: a monotone piecewise-linear CDF over normalised
// keys, shared by the training kernels, the splitter-table kernel and the
// bucket digit function of the distribution passes.
//
// Keys are normalised as u = float(key) * 2^-key_bits (round to nearest).
// The model has K segments with knots X_0 = 0 < X_1 < ... < X_K = 1 and values
// Y_0 = 0 <= Y_1 <= ... <= Y_K = 1, each from K positive increments
// softplus(theta_i) normalised by their sum (monotone by construction):
//   F(u) = Y_j + (Y_{j+1} - Y_j) * (u - X_j) / (X_{j+1} - X_j),  X_j <= u < X_{j+1}.
// Every fp32 operation of the bucket model is written with an explicit
// round-to-nearest intrinsic in a fixed order, so that the buckets (and the
// splitter table derived from them) are a function of (X, Y) alone,
// reproducible off the GPU.
#pragma once

#include "common.cuh"

namespace isort {

constexpr int kPwlSegments = 256;
constexpr int kPwlKnots = kPwlSegments + 1;
constexpr int kTrainSteps = 64;  // Adam steps of either model's fit

template <typename K>
__device__ __forceinline__ float normalise_key(K k, float scale) {
    if constexpr (sizeof(K) == 4) return __fmul_rn(__uint2float_rn((uint32_t)k), scale);
    else return __fmul_rn(__ull2float_rn((unsigned long long)k), scale);
}

// Largest j in [0, K-1] with X[j] <= u (X[0] = 0 <= u); u >= X[K] gives K-1.
__device__ __forceinline__ int pwl_segment(const float* X, float u) {
    int lo = 0, hi = kPwlSegments;
#pragma unroll
    for (int it = 0; it < 8; ++it) {  // kPwlSegments = 2^8
        const int mid = (lo + hi) >> 1;
        if (X[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The bucket model (the definition the sort uses), every fp32 operation
// rounded to nearest in this order:
//   j = pwl_segment(X, u); slope_j = (Y_{j+1} - Y_j) / (X_{j+1} - X_j) (0 for
//   an empty segment, at most 1e30); f = Y_j + (u - X_j) slope_j clamped to
//   [Y_j, Y_{j+1}]; bucket = min(B - 1, trunc(f B)).
// Each operation is monotone and the clamp keeps segment j below segment j+1,
// so the bucket never decreases as the key grows: buckets are key ranges.
__device__ __forceinline__ float pwl_slope(const float* X, const float* Y, int j) {
    const float dx = __fsub_rn(X[j + 1], X[j]);
    if (!(dx > 0.f)) return 0.f;
    const float sl = __fdiv_rn(__fsub_rn(Y[j + 1], Y[j]), dx);
    return sl < 1e30f ? sl : 1e30f;
}

__device__ __forceinline__ uint32_t pwl_bucket_in(const float* X, const float* Y, float slope, int j, float u, int B) {
    float f = __fadd_rn(Y[j], __fmul_rn(__fsub_rn(u, X[j]), slope));
    f = f < Y[j] ? Y[j] : f;
    f = f > Y[j + 1] ? Y[j + 1] : f;
    const uint32_t b = (uint32_t)__fmul_rn(f, __int2float_rn(B));
    return b > (uint32_t)(B - 1) ? (uint32_t)(B - 1) : b;
}

__device__ __forceinline__ uint32_t pwl_bucket(const float* X, const float* Y, float u, int B) {
    const int j = u < X[kPwlSegments] ? pwl_segment(X, u) : kPwlSegments - 1;
    return pwl_bucket_in(X, Y, pwl_slope(X, Y, j), j, u, B);
}

}  // namespace isort
