// The learned-bucket model: a monotone piecewise-linear CDF over normalised
// keys, shared by the training kernels, the splitter-table kernel and the
// bucket digit function of the distribution passes.
//
// Keys are normalised as u = float(key) * 2^-key_bits (round to nearest).
// The model has K segments with knots X_0 = 0 < X_1 < ... < X_K = 1 and values
// Y_0 = 0 <= Y_1 <= ... <= Y_K = 1, each from K positive increments
// softplus(theta_i) normalised by their sum (monotone by construction):
//   F(u) = Y_j + (Y_{j+1} - Y_j) * (u - X_j) / (X_{j+1} - X_j),  X_j <= u < X_{j+1}.
// Every fp32 operation of F is written with an explicit round-to-nearest
// intrinsic in a fixed order, so that the splitter table derived from F is a
// function of (X, Y) alone, reproducible off the GPU.
#pragma once

#include "common.cuh"

namespace isort {

constexpr int kPwlSegments = 256;
constexpr int kPwlKnots = kPwlSegments + 1;

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

__device__ __forceinline__ float pwl_eval(const float* X, const float* Y, float u) {
    if (!(u < X[kPwlSegments])) return Y[kPwlSegments];
    const int j = pwl_segment(X, u);
    const float dx = __fsub_rn(X[j + 1], X[j]);
    const float w = dx > 0.f ? __fdiv_rn(__fsub_rn(u, X[j]), dx) : 0.f;
    float f = __fadd_rn(Y[j], __fmul_rn(__fsub_rn(Y[j + 1], Y[j]), w));
    f = f < 0.f ? 0.f : (f > 1.f ? 1.f : f);
    return f;
}

}  // namespace isort
