// The alternative learned model: a 1-32-1 monotone MLP CDF over normalised
// keys u = key * 2^-key_bits. With a1, b1, a2 (32 each) and b2,
//   W1_j = softplus(a1_j), W2_j = softplus(a2_j),
//   z(u) = sum_j W2_j sigma(W1_j u + b1_j) + b2,
//   F(u) = (z(u) - z(0)) / (z(1) - z(0)),
// F is increasing (positive weights, increasing sigma) with F(0) = 0 and
// F(1) = 1; b2 cancels. It is trained on the same sample loss as the
// piecewise-linear model, (1/m) sum_i (F(u_i) - (i + 1/2)/m)^2, by Adam on one
// cluster of CTAs, and then tabulated at 257 knots placed at the sample's
// quantiles (X_k, Y_k = F(X_k) made non-decreasing). The bucket machinery
// reads the table as a monotone piecewise-linear CDF, so the buckets remain
// key ranges and the sort stays exact whatever the network learned.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "isort.h"
#include "learned.cuh"
#include "runtime.h"

namespace cg = cooperative_groups;

namespace isort {

constexpr int kMlpUnits = 32;
constexpr int kMlpParams = 3 * kMlpUnits + 1;  // a1, b1, a2, b2
constexpr int kMlpTrained = 3 * kMlpUnits;     // b2 has no gradient
constexpr int kMlpCluster = 8;                 // CTAs sharing the sample points
constexpr int kMlpThreads = 512;
constexpr int kMlpWarps = kMlpThreads / 32;
constexpr int kMlpPart = 3 * kMlpUnits + 3;    // per-unit sums A, B, C; loss, c0, c1
constexpr float kMlpRate = 0.02f;
constexpr uint32_t kMlpStride = 16;  // the fit sees every 16th point of the sorted sample

namespace {

__device__ __forceinline__ float mlp_softplus(float t) { return t > 20.f ? t : log1pf(expf(t)); }
__device__ __forceinline__ float mlp_inv_softplus(float v) { return v > 20.f ? v : logf(expm1f(v)); }
__device__ __forceinline__ float mlp_sigmoid(float t) { return 1.f / (1.f + expf(-t)); }
// The fit's sigmoid on the fast exponential and division (the table keeps mlp_sigmoid).
__device__ __forceinline__ float mlp_sigmoid_fast(float t) { return __fdividef(1.f, 1.f + __expf(-t)); }

__device__ __forceinline__ float mlp_warp_total(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

// Initial parameters from the sorted sample (32 threads, one per unit): unit
// j is centred at the sample's (j + 1/2)/32 quantile c_j and rises over the
// width of its quantile interval [q_j, q_{j+1}] (W1 = 4 / width, the width
// floored at 4e-6 so that W1 <= 1e6); every W2 = 1/32; b2 = 0.
template <typename K>
__global__ void k_mlp_init(const K* __restrict__ sorted, uint32_t m, float scale, float* __restrict__ p) {
    const int j = threadIdx.x;
    if (j >= kMlpUnits) return;
    auto q = [&](uint64_t idx) -> float {
        const float v = normalise_key(sorted[idx < m ? idx : m - 1], scale);
        return v < 1.f ? v : 1.f;
    };
    const float lo = q((uint64_t)j * m / kMlpUnits), hi = q((uint64_t)(j + 1) * m / kMlpUnits);
    const float c = q((uint64_t)(2 * j + 1) * m / (2 * kMlpUnits));
    const float w1 = fminf(4.f / fmaxf(hi - lo, 4e-6f), 1e6f);
    p[j] = mlp_inv_softplus(w1);
    p[kMlpUnits + j] = -w1 * c;
    p[2 * kMlpUnits + j] = mlp_inv_softplus(1.f / kMlpUnits);
    if (j == 0) p[3 * kMlpUnits] = 0.f;
}

// u[j] = the normalised value of sorted[j * stride + stride / 2], j < m.
template <typename K>
__global__ void k_mlp_points(const K* __restrict__ sorted, uint32_t m, uint32_t stride, float scale,
                             float* __restrict__ u) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) u[j] = normalise_key(sorted[(size_t)j * stride + stride / 2], scale);
}

// Adam on the sample loss, one cluster of C CTAs: CTA r takes the points
// [m r / C, m (r + 1) / C); lane j of every warp is unit j and the warps
// stride over the points, four at a time. Per point i (F_i = F(u_i),
// e_i = F_i - (i + 1/2)/m, r_i = 2 e_i / (m D), D = z(1) - z(0), h = sigma):
//   A_j = sum r_i h_ij (1 - h_ij) u_i,  B_j = sum r_i h_ij (1 - h_ij),
//   C_j = sum r_i h_ij,  c0 = sum r_i (F_i - 1),  c1 = -sum r_i F_i,
// and then, with s = h (1 - h) at u = 0 and u = 1,
//   dL/dW1_j = W2_j (A_j + c1 s1_j),  dL/db1_j = W2_j (B_j + c0 s0_j + c1 s1_j),
//   dL/dW2_j = C_j + c0 h0_j + c1 h1_j,
// through softplus for a1 and a2 (dL/da = dL/dW sigma(a)). The per-CTA sums
// go through shared memory in a fixed order and every CTA adds the C CTAs'
// sums in rank order, so all CTAs hold the same bits and take the same steps.
// params (device, 97) is read as the start and receives the parameters with
// the lowest loss seen (b2 unchanged); losses (optional, steps + 2): the loss
// before each step, of the returned parameters, at the start; loss0 and
// grad_out (optional): the loss and gradient at the start.
template <int C>
__global__ void __launch_bounds__(kMlpThreads, 1)
    k_mlp_fit(const float* __restrict__ u, uint32_t m, float* params, float* losses, float* loss0, float* grad_out,
              int steps, float lr) {
    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t rank = C == 1 ? 0u : cluster.block_rank();
    __shared__ float th[kMlpParams], mo1[kMlpTrained], mo2[kMlpTrained], best[kMlpTrained], g[kMlpTrained];
    __shared__ float part[kMlpWarps][kMlpPart];
    __shared__ float cta[2][kMlpPart];
    __shared__ float tot[kMlpPart];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t < kMlpParams) th[t] = params[t];
    if (t < kMlpTrained) {
        best[t] = params[t];
        mo1[t] = mo2[t] = 0.f;
    }
    __syncthreads();
    const uint32_t i0 = (uint32_t)((uint64_t)m * rank / C), i1 = (uint32_t)((uint64_t)m * (rank + 1) / C);
    const float inv_m = 1.f / (float)m;
    float best_loss = INFINITY, first = 0.f;
    const float be1 = 0.9f, be2 = 0.999f;
    float pw1 = 1.f, pw2 = 1.f;  // be1^(step + 1), be2^(step + 1) after the update below
    for (int step = 0;; ++step) {
        const int buf = step & 1;
        const float w1 = mlp_softplus(th[lane]), b1 = th[kMlpUnits + lane], w2 = mlp_softplus(th[2 * kMlpUnits + lane]);
        const float h0 = mlp_sigmoid_fast(b1), h1 = mlp_sigmoid_fast(fmaf(w1, 1.f, b1));
        const float inv_D = 1.f / mlp_warp_total(w2 * (h1 - h0));
        float A = 0.f, Bs = 0.f, Cs = 0.f, loss = 0.f, c0 = 0.f, c1 = 0.f;
        for (uint32_t base = i0 + warp; base < i1; base += 4 * kMlpWarps) {
            float x[4], h[4], z[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t i = base + q * kMlpWarps;
                x[q] = i < i1 ? u[i] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                h[q] = mlp_sigmoid_fast(fmaf(w1, x[q], b1));
                z[q] = w2 * (h[q] - h0);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int q = 0; q < 4; ++q) z[q] += __shfl_xor_sync(kFullMask, z[q], o);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t i = base + q * kMlpWarps;
                if (i >= i1) break;  // uniform over the warp
                const float F = z[q] * inv_D;
                const float e = F - ((float)i + 0.5f) * inv_m;
                const float r = 2.f * e * inv_m * inv_D;
                const float s = h[q] * (1.f - h[q]);
                A += r * s * x[q];
                Bs += r * s;
                Cs += r * h[q];
                loss += e * e;
                c0 += r * (F - 1.f);
                c1 -= r * F;
            }
        }
        part[warp][lane] = A;
        part[warp][kMlpUnits + lane] = Bs;
        part[warp][2 * kMlpUnits + lane] = Cs;
        if (lane == 0) {
            part[warp][3 * kMlpUnits] = loss;
            part[warp][3 * kMlpUnits + 1] = c0;
            part[warp][3 * kMlpUnits + 2] = c1;
        }
        __syncthreads();
        if (t < kMlpPart) {
            float v = 0.f;
            for (int w = 0; w < kMlpWarps; ++w) v += part[w][t];
            cta[buf][t] = v;
        }
        if constexpr (C > 1) cluster.sync();  // every CTA's sums are visible
        else __syncthreads();
        if (t < kMlpPart) {
            float v = 0.f;
            for (int rr = 0; rr < C; ++rr) v += C == 1 ? cta[buf][t] : *cluster.map_shared_rank(&cta[buf][t], rr);
            tot[t] = v;
        }
        __syncthreads();
        const float L = tot[3 * kMlpUnits] * inv_m;  // the same value in every thread of every CTA
        if (step == 0) first = L;
        if (losses && rank == 0 && t == 0 && step < steps) losses[step] = L;
        if (L < best_loss) {
            best_loss = L;
            if (t < kMlpTrained) best[t] = th[t];
        }
        if (step == steps && !(step == 0 && grad_out)) break;
        if (warp == 0) {
            const float s0 = h0 * (1.f - h0), s1 = h1 * (1.f - h1);
            const float tc0 = tot[3 * kMlpUnits + 1], tc1 = tot[3 * kMlpUnits + 2];
            const float gw1 = w2 * (tot[lane] + tc1 * s1);
            const float gb1 = w2 * (tot[kMlpUnits + lane] + tc0 * s0 + tc1 * s1);
            const float gw2 = tot[2 * kMlpUnits + lane] + tc0 * h0 + tc1 * h1;
            g[lane] = gw1 * mlp_sigmoid(th[lane]);
            g[kMlpUnits + lane] = gb1;
            g[2 * kMlpUnits + lane] = gw2 * mlp_sigmoid(th[2 * kMlpUnits + lane]);
        }
        __syncthreads();
        if (step == 0 && grad_out && rank == 0) {
            if (t < kMlpTrained) grad_out[t] = g[t];
            if (t == kMlpTrained) grad_out[t] = 0.f;
        }
        if (step == steps) break;
        pw1 *= be1;
        pw2 *= be2;
        if (t < kMlpTrained) {
            const float d = g[t];
            const float a = mo1[t] = be1 * mo1[t] + (1.f - be1) * d;
            const float v = mo2[t] = be2 * mo2[t] + (1.f - be2) * d * d;
            th[t] -= lr * (a / (1.f - pw1)) / (sqrtf(v / (1.f - pw2)) + 1e-8f);
        }
        __syncthreads();
    }
    if (rank == 0) {
        if (t < kMlpTrained) params[t] = best[t];
        if (t == 0) {
            if (losses) {
                losses[steps] = best_loss;
                losses[steps + 1] = first;
            }
            if (loss0) *loss0 = first;
        }
    }
    if constexpr (C > 1) cluster.sync();  // no CTA leaves while others may still read its shared memory
}

// The table the bucket machinery reads: X_0 = 0, X_k = the normalised sample
// key at rank k m / 256 (at most 1), X_256 = 1; Y_k = F(X_k) clamped to
// [0, 1], Y_0 = 0, Y_256 = 1, then the running maximum over k. One CTA.
constexpr int kKnotThreads = 288;  // 9 warps cover the 257 knots

template <typename K>
__global__ void __launch_bounds__(kKnotThreads) k_mlp_knots(const K* __restrict__ sorted, uint32_t m, float scale,
                                                          const float* __restrict__ p, float* __restrict__ X,
                                                          float* __restrict__ Y) {
    __shared__ float w1s[kMlpUnits], b1s[kMlpUnits], w2s[kMlpUnits], h0s[kMlpUnits];
    __shared__ float ys[kKnotThreads];
    __shared__ float wmax[kKnotThreads / 32];
    const int k = threadIdx.x, lane = k & 31, warp = k >> 5;
    if (k < kMlpUnits) {
        w1s[k] = mlp_softplus(p[k]);
        b1s[k] = p[kMlpUnits + k];
        w2s[k] = mlp_softplus(p[2 * kMlpUnits + k]);
        h0s[k] = mlp_sigmoid(b1s[k]);
    }
    __syncthreads();
    float x = 0.f, y = 0.f;
    if (k <= kPwlSegments) {
        if (k == kPwlSegments) x = 1.f;
        else if (k > 0) x = fminf(normalise_key(sorted[(uint64_t)k * m / kPwlSegments], scale), 1.f);
        float z = 0.f, D = 0.f;
        for (int j = 0; j < kMlpUnits; ++j) {
            z += w2s[j] * (mlp_sigmoid(fmaf(w1s[j], x, b1s[j])) - h0s[j]);
            D += w2s[j] * (mlp_sigmoid(fmaf(w1s[j], 1.f, b1s[j])) - h0s[j]);
        }
        y = z / D;
        y = y > 0.f ? (y < 1.f ? y : 1.f) : 0.f;  // NaN -> 0
        if (k == 0) y = 0.f;
        if (k == kPwlSegments) y = 1.f;
        X[k] = x;
    }
    // running maximum: within each warp, then across the warps
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float v = __shfl_up_sync(kFullMask, y, o);
        if (lane >= o) y = fmaxf(y, v);
    }
    if (lane == 31) wmax[warp] = y;
    __syncthreads();
    for (int w = 0; w < warp; ++w) y = fmaxf(y, wmax[w]);
    if (k <= kPwlSegments) Y[k] = y;
}

isort_status launch_mlp_fit(const float* u, uint32_t m, float* params, float* losses, float* loss0, float* grad,
                            int steps, cudaStream_t s) {
    auto kern = k_mlp_fit<kMlpCluster>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(kMlpThreads);
    cfg.gridDim = dim3(kMlpCluster);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kMlpCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    ISORT_TRY_CUDA(cudaOccupancyMaxActiveClusters(&clusters, (void*)kern, &cfg));
    if (clusters < 1) return ISORT_ERR_UNSUPPORTED;
    LaunchScope ls("mlp_fit", s);
    ISORT_TRY_CUDA(cudaLaunchKernelEx(&cfg, kern, u, m, params, losses, loss0, grad, steps, kMlpRate));
    return ISORT_OK;
}

}  // namespace

// The MLP model of a sorted sample (device, m keys): u (device, m / 16
// floats of scratch) receives the fit's points, params (device, 97) the
// trained parameters, X and Y (device, 257 each) the table, losses (device,
// 66) the training record as k_mlp_fit writes it.
template <typename K>
isort_status mlp_model(const K* sorted, uint32_t m, float scale, float* u, float* params, float* X, float* Y,
                       float* losses, cudaStream_t s) {
    const uint32_t mf = m / kMlpStride;
    if (mf == 0) return ISORT_ERR_INVALID_ARG;
    {
        LaunchScope ls("mlp_init", s);
        k_mlp_points<K><<<(mf + 255) / 256, 256, 0, s>>>(sorted, mf, kMlpStride, scale, u);
        k_mlp_init<K><<<1, kMlpUnits, 0, s>>>(sorted, m, scale, params);
        ISORT_TRY_CUDA(cudaGetLastError());
    }
    ISORT_TRY(launch_mlp_fit(u, mf, params, losses, nullptr, nullptr, kTrainSteps, s));
    LaunchScope ls("mlp_knots", s);
    k_mlp_knots<K><<<1, kKnotThreads, 0, s>>>(sorted, m, scale, params, X, Y);
    ISORT_TRY_CUDA(cudaGetLastError());
    return ISORT_OK;
}

template isort_status mlp_model<uint32_t>(const uint32_t*, uint32_t, float, float*, float*, float*, float*, float*,
                                          cudaStream_t);
template isort_status mlp_model<uint64_t>(const uint64_t*, uint32_t, float, float*, float*, float*, float*, float*,
                                          cudaStream_t);

}  // namespace isort

using namespace isort;

extern "C" {

isort_status isort_mlp_loss_grad(const float* u, uint32_t m, const float* params, float* grad, float* loss,
                                 void* stream) {
    if (!u || !params || !grad || !loss || m == 0) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float* p = nullptr;  // the fit writes its parameters back: work on a copy
    isort_status st = scratch_alloc((void**)&p, kMlpParams * 4, s);
    if (st != ISORT_OK) return st;
    cudaError_t ce = cudaMemcpyAsync(p, params, kMlpParams * 4, cudaMemcpyDeviceToDevice, s);
    st = ce == cudaSuccess ? launch_mlp_fit(u, m, p, nullptr, loss, grad, 0, s) : from_cuda(ce);
    scratch_free(p, s);
    if (st == ISORT_OK && sync_mode()) st = from_cuda(cudaStreamSynchronize(s));
    return st;
}

isort_status isort_mlp_train(const uint32_t* sorted_sample, uint32_t m, int key_bits, float* params, float* X,
                             float* Y, float* losses, void* stream) {
    if (!sorted_sample || !params || !X || !Y || !losses || m < 2) return ISORT_ERR_INVALID_ARG;
    if (key_bits == 0) key_bits = 32;
    if (key_bits < 1 || key_bits > 32) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float* u = nullptr;
    isort_status st = scratch_alloc((void**)&u, (size_t)m * 4, s);
    if (st != ISORT_OK) return st;
    const float scale = std::ldexp(1.0f, -key_bits);
    {
        LaunchScope ls("mlp_init", s);
        k_mlp_points<uint32_t><<<(m + 255) / 256, 256, 0, s>>>(sorted_sample, m, 1, scale, u);
        k_mlp_init<uint32_t><<<1, kMlpUnits, 0, s>>>(sorted_sample, m, scale, params);
        st = from_cuda(cudaGetLastError());
    }
    if (st == ISORT_OK) st = launch_mlp_fit(u, m, params, losses, nullptr, nullptr, kTrainSteps, s);
    if (st == ISORT_OK) {
        LaunchScope ls("mlp_knots", s);
        k_mlp_knots<uint32_t><<<1, kKnotThreads, 0, s>>>(sorted_sample, m, scale, params, X, Y);
        st = from_cuda(cudaGetLastError());
    }
    scratch_free(u, s);
    if (st == ISORT_OK && sync_mode()) st = from_cuda(cudaStreamSynchronize(s));
    return st;
}

}  // extern "C"
