// Learned-bucket sort: a monotone CDF model, trained on the GPU on a sample
// that the method sorts itself, gives each key its bucket for an MSD
// distribution (the bucket function is monotone in the key, so buckets are
// key ranges), and the buckets are then finished independently on chip.
//
// There is no counterpart in Gerbessiotis (arXiv:1708.09495). The bucketing
// grows out of the splitter-based sample sorts the paper discusses (Section 2:
// random oversampling, regular sampling and oversampling), with the splitters
// read off a learned CDF instead of a sorted sample; the finishing sorts are the
// paper's count-sort rounds (Section 3) run per bucket.
//
// Steps (one call):
//   1. sample m = 2^16 keys at indices drawn from SplitMix64 (Steele, Lea &
//      Flood 2014), sort them with the library's own radix rounds;
//   2. train the 256-segment PWL CDF (learned.cuh) by Adam on the mean squared
//      error between F(u_i) and the empirical CDF (i + 1/2)/m of every 8th
//      point of the sorted sample (m = 2^13, 32 points per segment); knot
//      positions start at sample quantiles, values at i/256; all steps run in
//      one single-CTA kernel, and the parameters with the lowest loss seen
//      (the initial ones included) are kept;
//   3. bucket(key) = min(B - 1, floor(F(u) B)) with F evaluated in a fixed
//      fp32 order and clamped per segment (learned.cuh), which makes it
//      monotone in the key; the splitter table s_b = the first key of bucket
//      b gives each bucket's key range;
//   4. census: bucket sizes, fix-ups, per-chunk counts for the first pass;
//      too many keys in buckets beyond the on-chip capacity -> plain LSD;
//   5. stable distribution by bucket: two stable passes over the bucket id's
//      low and high halves (chunked count-sort rounds whose digit function is
//      the bucket lookup); a 2^12-way stable ranking inside a tile would not
//      fit on chip, two 2^6-way ones do;
//   6. finish: every bucket is a segment of the batched segmented sort, sorted
//      on the bits its key range spans (a bucket of one key value is skipped).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "learned.cuh"
#include "runtime.h"
#include "sweep.cuh"

namespace isort {

isort_status radix_sort_u32_device(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, size_t n,
                                   int key_bits, int rb, cudaStream_t s);
isort_status radix_sort_u64_device(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout, size_t n,
                                   int key_bits, int rb, cudaStream_t s);
isort_status segmented_finish_u64(uint64_t* keys, uint32_t* vals, const uint64_t* off, uint32_t nseg,
                                  const uint64_t* seg_lo, const uint8_t* seg_bits, cudaStream_t s);
isort_status segmented_finish_u32(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint32_t nseg,
                                  const uint32_t* seg_lo, const uint8_t* seg_bits, cudaStream_t s);
// The MLP model of a sorted sample, tabulated as X, Y (mlp.cu).
template <typename K>
isort_status mlp_model(const K* sorted, uint32_t m, float scale, float* u, float* params, float* X, float* Y,
                       float* losses, cudaStream_t s);
extern template isort_status mlp_model<uint32_t>(const uint32_t*, uint32_t, float, float*, float*, float*, float*,
                                                 float*, cudaStream_t);
extern template isort_status mlp_model<uint64_t>(const uint64_t*, uint32_t, float, float*, float*, float*, float*,
                                                 float*, cudaStream_t);

namespace {

// The plain count-sort rounds (Section 3), in place.
isort_status plain_sort(uint32_t* k, uint32_t* v, size_t n, int key_bits, cudaStream_t s) {
    return radix_sort_u32_device(k, v, k, v, n, key_bits, 8, s);
}
isort_status plain_sort(uint64_t* k, uint32_t* v, size_t n, int key_bits, cudaStream_t s) {
    return radix_sort_u64_device(k, v, k, v, n, key_bits, 8, s);
}
isort_status finish_buckets(uint32_t* k, uint32_t* v, const uint64_t* off, uint32_t nseg, const uint32_t* lo,
                            const uint8_t* bits, cudaStream_t s) {
    return segmented_finish_u32(k, v, off, nseg, lo, bits, s);
}
isort_status finish_buckets(uint64_t* k, uint32_t* v, const uint64_t* off, uint32_t nseg, const uint64_t* lo,
                            const uint8_t* bits, cudaStream_t s) {
    return segmented_finish_u64(k, v, off, nseg, lo, bits, s);
}

constexpr uint32_t kSampleSize = 1u << 16;

// One segment [0, m) over key_bits bits from key 0, for the segmented finish.
template <typename K>
__global__ void k_one_segment(uint64_t* off, K* lo, uint8_t* bits, uint32_t m, int key_bits) {
    off[0] = 0;
    off[1] = m;
    lo[0] = 0;
    bits[0] = (uint8_t)key_bits;
}

// Sorts the sample (m <= 65,536 keys) in place: u32 keys by the plain rounds
// (one on-chip cluster launch at this size); u64 keys as one segment of the
// segmented finish (one cluster of CTAs, on chip) instead of 6-8 launches of
// plain rounds. off, lo, bits: device scratch for the segment's description.
isort_status sort_sample(uint32_t* k, uint32_t m, int key_bits, uint64_t*, uint32_t*, uint8_t*, cudaStream_t s) {
    return plain_sort(k, nullptr, m, key_bits, s);
}
isort_status sort_sample(uint64_t* k, uint32_t m, int key_bits, uint64_t* off, uint64_t* lo, uint8_t* bits,
                         cudaStream_t s) {
    {
        LaunchScope ls("sample_segment", s);
        k_one_segment<uint64_t><<<1, 1, 0, s>>>(off, lo, bits, m, key_bits);
        const cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) return from_cuda(ce);
    }
    return finish_buckets(k, nullptr, off, 1, lo, bits, s);
}
constexpr uint64_t kSampleSeed = 0x5EED5EED5EEDull;
constexpr uint32_t kFitStride = 8;  // the fit sees every 8th point of the sorted sample
constexpr float kLearningRate = 0.002f;  // at 0.02 the first steps overshoot the quantile start (no step improved it)
constexpr uint32_t kOnChipCapacity = 65536;  // keys a cluster finishes on chip
constexpr int kMaxBuckets = 32768;           // the census counts every bucket in shared memory
static_assert(kMaxBuckets <= 65536, "bucket ids are stored in 16 bits");

// ---------------------------------------------------------------- sampling

template <typename K>
__global__ void k_sample_gather(const K* __restrict__ keys, uint64_t n, uint32_t m, K* __restrict__ out) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const uint64_t r = splitmix_mix(kSampleSeed + (uint64_t)(j + 1) * kSplitmixGamma);
    const uint64_t idx = __umul64hi(r, n);  // floor(r * n / 2^64) < n
    out[j] = keys[idx];
}

// u[j] = the normalised value of sorted[j * stride + stride / 2], j < m.
template <typename K>
__global__ void k_normalise(const K* __restrict__ sorted, uint32_t m, uint32_t stride, float scale,
                            float* __restrict__ u) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) u[j] = normalise_key(sorted[(size_t)j * stride + stride / 2], scale);
}

// ---------------------------------------------------------------- the model

__device__ __forceinline__ float softplus(float t) { return t > 20.f ? t : log1pf(expf(t)); }
__device__ __forceinline__ float inv_softplus(float v) { return v > 20.f ? v : logf(expm1f(v)); }
__device__ __forceinline__ float sigmoidf_(float t) { return 1.f / (1.f + expf(-t)); }

// Initial parameters from the sorted sample: knot positions at the sample's
// quantiles j/256 (increments floored at 1e-3 of the mean), values j/256.
template <typename K>
__global__ void __launch_bounds__(kPwlSegments) k_model_init(const K* __restrict__ sorted, uint32_t m, float scale,
                                                             float* theta) {
    const int t = threadIdx.x;
    auto q = [&](int j) -> float {
        if (j <= 0) return 0.f;
        if (j >= kPwlSegments) return 1.f;
        const float v = normalise_key(sorted[(uint64_t)j * m / kPwlSegments], scale);
        return v < 1.f ? v : 1.f;
    };
    const float dx = fmaxf(q(t + 1) - q(t), 0.f) * (float)kPwlSegments;
    theta[t] = inv_softplus(fmaxf(dx, 1e-3f));
    theta[kPwlSegments + t] = inv_softplus(1.f);
}

// One CTA fits the model: all steps in one launch, every reduction in a fixed
// order except the per-knot gradient sums (shared-memory float atomics).
constexpr int kFitThreads = 1024;

__device__ __forceinline__ float warp_incl_scan(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(kFullMask, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

__device__ __forceinline__ float warp_suffix_scan(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_down_sync(kFullMask, v, o);
        if (lane + o < 32) v += y;
    }
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

// X, Y from theta: threads 0..255 make X, 256..511 make Y (warps 0-7, 8-15):
// V_i = (sum_{k<i} softplus(theta_k)) / (sum_k softplus(theta_k)), V_256 = 1.
__device__ void fit_derive(const float* th, float* X, float* Y, float* wt) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float v = 0.f, incl = 0.f;
    if (t < 2 * kPwlSegments) {
        v = softplus(th[t]);
        incl = warp_incl_scan(v, lane);
        if (lane == 31) wt[warp] = incl;
    }
    __syncthreads();
    if (t < 2 * kPwlSegments) {
        const int g = t >> 8, i = t & (kPwlSegments - 1);
        float before = 0.f, total = 0.f;
        for (int w = g * 8; w < g * 8 + 8; ++w) {
            if (w < warp) before += wt[w];
            total += wt[w];
        }
        float excl = __shfl_up_sync(kFullMask, incl, 1);
        excl = lane == 0 ? before : before + excl;
        float* V = g ? Y : X;
        V[i] = i == 0 ? 0.f : fminf(excl / total, 1.f);
        if (i == 0) V[kPwlSegments] = 1.f;
    }
    __syncthreads();
}

// Loss L = (1/m) sum_i (F(u_i) - (i + 1/2)/m)^2 and its gradient with respect
// to the knots (gX, gY, zeroed here); u sorted. Each thread takes a contiguous
// run of points, so its segment index only grows; partial sums are flushed to
// shared memory when it changes. Returns L (the same value in every thread).
__device__ float fit_loss_grad(const float* __restrict__ u, uint32_t m, const float* X, const float* Y, float* gX,
                               float* gY, float* red) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int j = t; j < kPwlKnots; j += kFitThreads) gX[j] = gY[j] = 0.f;
    __syncthreads();
    const uint32_t P = (m + kFitThreads - 1) / kFitThreads;
    const uint32_t i0 = min(m, (uint32_t)t * P), i1 = min(m, i0 + P);
    const float inv_m = 1.f / (float)m;
    float loss = 0.f;
    if (i0 < i1) {
        int j = pwl_segment(X, u[i0]);
        float xj = X[j], xj1 = X[j + 1], yj = Y[j], dy = Y[j + 1] - yj, dx = xj1 - xj;
        float inv = dx > 0.f ? 1.f / dx : 0.f;
        float aY0 = 0.f, aY1 = 0.f, aX0 = 0.f, aX1 = 0.f;
        for (uint32_t base = i0; base < i1; base += 8) {
            float xs[8];  // loads first, so that eight are in flight
#pragma unroll
            for (int r = 0; r < 8; ++r) xs[r] = base + r < i1 ? u[base + r] : 0.f;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
            const uint32_t i = base + r;
            if (i >= i1) break;
            const float x = xs[r];
            if (j < kPwlSegments - 1 && xj1 <= x) {
                atomicAdd(&gY[j], aY0);
                atomicAdd(&gY[j + 1], aY1);
                atomicAdd(&gX[j], aX0);
                atomicAdd(&gX[j + 1], aX1);
                aY0 = aY1 = aX0 = aX1 = 0.f;
                while (j < kPwlSegments - 1 && X[j + 1] <= x) ++j;
                xj = X[j];
                xj1 = X[j + 1];
                yj = Y[j];
                dy = Y[j + 1] - yj;
                dx = xj1 - xj;
                inv = dx > 0.f ? 1.f / dx : 0.f;
            }
            const float w = fminf(fmaxf((x - xj) * inv, 0.f), 1.f);
            const float e = yj + dy * w - ((float)i + 0.5f) * inv_m;
            loss += e * e;
            const float ge = 2.f * e * inv_m;
            aY0 += ge * (1.f - w);
            aY1 += ge * w;
            if (dx > 0.f && x < xj1) {
                const float k = ge * dy * inv * inv;
                aX0 += k * (x - xj1);
                aX1 -= k * (x - xj);
            }
            }
        }
        atomicAdd(&gY[j], aY0);
        atomicAdd(&gY[j + 1], aY1);
        atomicAdd(&gX[j], aX0);
        atomicAdd(&gX[j + 1], aX1);
    }
    loss = warp_sum(loss * inv_m);
    if (lane == 0) red[warp] = loss;
    __syncthreads();
    float L = 0.f;
    for (int w = 0; w < kFitThreads / 32; ++w) L += red[w];
    __syncthreads();
    return L;
}

// d L / d theta (threads 0..511): with V the knots of one half, g their
// gradient, S = sum softplus(theta), A = sum_j g_j V_j:
//   d L / d theta_i = sigmoid(theta_i) / S * (sum_{j > i} g_j - A).
__device__ float fit_theta_grad(const float* th, const float* X, const float* Y, const float* gX, const float* gY,
                                float* wt) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float pa = 0.f, ps = 0.f, suf = 0.f, sp = 0.f;
    if (t < 2 * kPwlSegments) {
        const int g = t >> 8, i = t & (kPwlSegments - 1);
        const float* V = g ? Y : X;
        const float* G = g ? gY : gX;
        float prod = G[i] * V[i];
        if (i == kPwlSegments - 1) prod += G[kPwlSegments] * V[kPwlSegments];
        sp = softplus(th[t]);
        pa = warp_sum(prod);
        ps = warp_sum(sp);
        suf = warp_suffix_scan(G[i + 1], lane);
        if (lane == 0) {
            wt[warp] = pa;
            wt[16 + warp] = ps;
            wt[32 + warp] = suf;  // the warp's total (lane 0 holds the whole suffix)
        }
    }
    __syncthreads();
    float d = 0.f;
    if (t < 2 * kPwlSegments) {
        const int g = t >> 8;
        float A = 0.f, S = 0.f, later = 0.f;
        for (int w = g * 8; w < g * 8 + 8; ++w) {
            A += wt[w];
            S += wt[16 + w];
            if (w > warp) later += wt[32 + w];
        }
        d = sigmoidf_(th[t]) / S * ((suf + later) - A);
    }
    __syncthreads();
    return d;
}

// Fits theta (device, 512; read as the start, written with the result) on the
// normalised sorted sample u by `steps` Adam steps; keeps the parameters with
// the lowest loss seen. losses (optional): [step] the loss before each step,
// [steps] the loss of the returned parameters, [steps + 1] the initial loss.
// loss0, grad_out (optional): the loss and d L / d theta at the initial theta.
__global__ void __launch_bounds__(kFitThreads, 1)
    k_cdf_fit(const float* __restrict__ u, uint32_t m, float* theta, float* X_out, float* Y_out, float* losses,
              float* loss0, float* grad_out, int steps, float lr) {
    __shared__ float sX[kPwlKnots], sY[kPwlKnots], gX[kPwlKnots], gY[kPwlKnots];
    __shared__ float th[2 * kPwlSegments], m1[2 * kPwlSegments], m2[2 * kPwlSegments], best[2 * kPwlSegments];
    __shared__ float wt[48];
    __shared__ float red[kFitThreads / 32];
    const int t = threadIdx.x;
    if (t < 2 * kPwlSegments) {
        th[t] = theta[t];
        best[t] = th[t];
        m1[t] = m2[t] = 0.f;
    }
    __syncthreads();
    fit_derive(th, sX, sY, wt);
    float best_loss = INFINITY, first = 0.f;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int step = 0;; ++step) {
        const float L = fit_loss_grad(u, m, sX, sY, gX, gY, red);
        if (step == 0) first = L;
        if (losses && step < steps && t == 0) losses[step] = L;
        if (L < best_loss) {  // L is the same in every thread
            best_loss = L;
            if (t < 2 * kPwlSegments) best[t] = th[t];
        }
        if (step == steps && !(step == 0 && grad_out)) break;
        const float d = fit_theta_grad(th, sX, sY, gX, gY, wt);
        if (step == 0 && grad_out && t < 2 * kPwlSegments) grad_out[t] = d;
        if (step == steps) break;
        if (t < 2 * kPwlSegments) {
            const float a = m1[t] = b1 * m1[t] + (1.f - b1) * d;
            const float v = m2[t] = b2 * m2[t] + (1.f - b2) * d * d;
            const float c1 = 1.f - powf(b1, (float)(step + 1)), c2 = 1.f - powf(b2, (float)(step + 1));
            th[t] -= lr * (a / c1) / (sqrtf(v / c2) + 1e-8f);
        }
        __syncthreads();
        fit_derive(th, sX, sY, wt);
    }
    if (t < 2 * kPwlSegments) th[t] = best[t];
    __syncthreads();
    fit_derive(th, sX, sY, wt);
    if (t < 2 * kPwlSegments) theta[t] = th[t];
    for (int j = t; j < kPwlKnots; j += kFitThreads) {
        if (X_out) X_out[j] = sX[j];
        if (Y_out) Y_out[j] = sY[j];
    }
    if (t == 0) {
        if (losses) {
            losses[steps] = best_loss;
            losses[steps + 1] = first;
        }
        if (loss0) *loss0 = first;
    }
}

// ---------------------------------------------------------------- overflow buckets

// Moves nr ranges between the array (keys, vals) and a packed copy (pk, pv):
// range r is [off[r], off[r] + len_r) in the array and [pos[r], pos[r + 1])
// in the copy; chunk c (kMoveChunk elements) of the launch belongs to range r
// with cstart[r] <= c < cstart[r + 1]. gather: array -> copy; else copy -> array.
constexpr uint32_t kMoveChunk = 4096;

template <typename K>
__global__ void k_move_ranges(K* keys, uint32_t* vals, K* pk, uint32_t* pv, const uint64_t* __restrict__ off,
                              const uint64_t* __restrict__ pos, const uint32_t* __restrict__ cstart, uint32_t nr,
                              int gather) {
    const uint32_t c = blockIdx.x;
    uint32_t lo = 0, hi = nr;  // the last r with cstart[r] <= c
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (cstart[mid] <= c) lo = mid;
        else hi = mid;
    }
    const uint32_t r = lo;
    const uint64_t len = pos[r + 1] - pos[r];
    const uint64_t e0 = (uint64_t)(c - cstart[r]) * kMoveChunk;
    const uint64_t e1 = min(len, e0 + kMoveChunk);
    for (uint64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const uint64_t a = off[r] + e, p = pos[r] + e;
        if (gather) {
            pk[p] = keys[a];
            if (vals) pv[p] = vals[a];
        } else {
            keys[a] = pk[p];
            if (vals) vals[a] = pv[p];
        }
    }
}

// ---------------------------------------------------------------- splitters

// s_0 = 0; s_b = the first key whose bucket is at least b (the largest key if
// none): the buckets' lower key bounds, by bisection over the keys.
template <typename K>
__global__ void k_splitters(const float* __restrict__ X, const float* __restrict__ Y, int B, int key_bits,
                            float scale, K* __restrict__ split) {
    __shared__ float sX[kPwlKnots], sY[kPwlKnots];
    for (int i = threadIdx.x; i < kPwlKnots; i += blockDim.x) {
        sX[i] = X[i];
        sY[i] = Y[i];
    }
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < 1 || b >= B) {
        if (b == 0) split[0] = 0;
        return;
    }
    uint64_t lo = 0, hi = key_bits >= 64 ? ~0ull : ((1ull << key_bits) - 1ull);
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (pwl_bucket(sX, sY, normalise_key((K)mid, scale), B) >= (uint32_t)b) hi = mid;
        else lo = mid + 1;
    }
    split[b] = (K)lo;
}

// ---------------------------------------------------------------- bucket lookup

constexpr int kSegTable = 1024;  // segment index table over u in [0, 1)

// Shared-memory bytes of a bucket lookup: X, Y, slopes, segment table.
__host__ __device__ constexpr size_t bucket_tab_bytes() {
    return 2 * ((kPwlKnots * 4 + 15) / 16 * 16) + kPwlSegments * 4 + ((kSegTable + 1) + 15) / 16 * 16;
}

// The bucket model (learned.cuh) with the segment found through a table over
// u: s_seg[q] = pwl_segment(X, q / kSegTable), so the segment of u lies in
// [s_seg[q], s_seg[q + 1]] for q = floor(u kSegTable); a bisection there gives
// pwl_segment(X, u) itself. Slopes are computed once per CTA by pwl_slope.
template <typename K>
struct BucketDigit {
    static constexpr bool kCheap = false;
    static constexpr bool kIndexed = false;
    const float* g_X;
    const float* g_Y;
    int B;
    float scale;
    int sub_shift;
    uint32_t sub_mask;
    float* s_X;
    float* s_Y;
    float* s_slope;
    uint8_t* s_seg;
    __device__ __forceinline__ size_t table_bytes() const { return bucket_tab_bytes(); }
    __device__ __forceinline__ void setup(unsigned char* p) {
        constexpr size_t kv = (kPwlKnots * 4 + 15) / 16 * 16;
        s_X = reinterpret_cast<float*>(p);
        s_Y = reinterpret_cast<float*>(p + kv);
        s_slope = reinterpret_cast<float*>(p + 2 * kv);
        s_seg = p + 2 * kv + kPwlSegments * 4;
        for (int i = threadIdx.x; i < kPwlKnots; i += blockDim.x) {
            s_X[i] = g_X[i];
            s_Y[i] = g_Y[i];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < kPwlSegments; j += blockDim.x) s_slope[j] = pwl_slope(s_X, s_Y, j);
        for (int q = threadIdx.x; q <= kSegTable; q += blockDim.x)
            s_seg[q] = (uint8_t)pwl_segment(s_X, (float)q * (1.f / kSegTable));
        __syncthreads();
    }
    __device__ __forceinline__ uint32_t bucket(K k) const {
        const float u = normalise_key(k, scale);
        const int q = min((int)(u * (float)kSegTable), kSegTable - 1);
        int lo = s_seg[q], hi = s_seg[q + 1];  // lo <= segment(u) <= hi
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_X[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        return pwl_bucket_in(s_X, s_Y, s_slope[lo], lo, u, B);
    }
    __device__ __forceinline__ uint32_t digit(K k) const { return (bucket(k) >> sub_shift) & sub_mask; }
};

// The bucket ids the census stored (one 16-bit id per key, B <= 2^15) as the
// digit of a distribution pass: the pass reads the id at each key's input
// position, takes its digit, and writes the id to the key's output position
// for the next pass (ids_out may be null on the last pass). The model is then
// evaluated once per key, in the census, instead of once per pass.
struct IdDigit {
    static constexpr bool kCheap = false;
    static constexpr bool kIndexed = true;
    const uint16_t* ids_in;
    uint16_t* ids_out;
    int sub_shift;
    uint32_t sub_mask;
    __device__ __forceinline__ size_t table_bytes() const { return 0; }
    __device__ __forceinline__ void setup(unsigned char*) {}
    __device__ __forceinline__ uint32_t load(uint32_t i) const { return ids_in[i]; }
    __device__ __forceinline__ uint32_t digit_of(uint32_t id) const { return (id >> sub_shift) & sub_mask; }
    __device__ __forceinline__ void store(uint32_t i, uint32_t id) const {
        if (ids_out) ids_out[i] = (uint16_t)id;
    }
};

// Loads of a chunk: 16-byte vectors when the base allows, else scalars.
template <typename K>
struct KeyVec {
    static constexpr int kN = 16 / sizeof(K);
};

template <typename K, typename F>
__device__ __forceinline__ void for_chunk_keys(const K* __restrict__ keys, uint32_t lo, uint32_t hi, bool vec, F&& f) {
    constexpr int V = KeyVec<K>::kN;
    uint32_t i = lo;
    if (vec) {
        for (uint32_t b = lo + threadIdx.x * V; b + V <= hi; b += blockDim.x * V) {
            const uint4 w = *reinterpret_cast<const uint4*>(keys + b);
            if constexpr (sizeof(K) == 4) {
                f(b, (K)w.x);
                f(b + 1, (K)w.y);
                f(b + 2, (K)w.z);
                f(b + 3, (K)w.w);
            } else {
                f(b, (K)(((uint64_t)w.y << 32) | w.x));
                f(b + 1, (K)(((uint64_t)w.w << 32) | w.z));
            }
        }
        i = lo + (hi - lo) / V * V;
    }
    for (uint32_t b = i + threadIdx.x; b < hi; b += blockDim.x) f(b, keys[b]);
}

// Census: per-chunk counts of the first pass's digit, every bucket's size per
// chunk, and the key-range check (a key of key_bits or more bits sets the
// status).
constexpr int kCensusThreads = 512;

template <typename K>
__global__ void __launch_bounds__(kCensusThreads) k_bucket_census(const K* __restrict__ keys, uint32_t n,
                                                                  uint32_t chunk_keys, BucketDigit<K> df,
                                                                  uint32_t* __restrict__ hist,
                                                                  uint32_t* __restrict__ bucket_count,
                                                                  int key_bits, uint32_t* status, int vec,
                                                                  uint16_t* __restrict__ ids = nullptr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int bins = (int)df.sub_mask + 1;
    uint32_t* s_h = reinterpret_cast<uint32_t*>(smem);             // [bins]
    uint32_t* s_b = s_h + bins;                                    // [B]
    unsigned char* tab = reinterpret_cast<unsigned char*>(s_b + align_up_dev((size_t)df.B, 4));
    for (int i = threadIdx.x; i < bins; i += kCensusThreads) s_h[i] = 0;
    for (int i = threadIdx.x; i < df.B; i += kCensusThreads) s_b[i] = 0;
    df.setup(tab);
    const uint32_t lo = blockIdx.x * chunk_keys, hi = min(n, lo + chunk_keys);
    K kor = 0;
    for_chunk_keys<K>(keys, lo, hi, vec != 0, [&](uint32_t i, K k) {
        kor |= k;
        const uint32_t b = df.bucket(k);
        atomicAdd(&s_h[(b >> df.sub_shift) & df.sub_mask], 1u);
        atomicAdd(&s_b[b], 1u);
        if (ids) ids[i] = (uint16_t)b;  // the distribution passes read it back
    });
    __syncthreads();
    for (int i = threadIdx.x; i < bins; i += kCensusThreads) hist[(size_t)blockIdx.x * bins + i] = s_h[i];
    // this chunk's bucket sizes (summed over chunks by k_sum_columns)
    for (int i = threadIdx.x; i < df.B; i += kCensusThreads) bucket_count[(size_t)blockIdx.x * df.B + i] = s_b[i];
    if (key_bits < (int)sizeof(K) * 8 && (kor >> key_bits) != 0) set_status(status, kStatKeyRange);
}

// out[c] = sum over rows r of in[r * cols + c] (fixed order).
__global__ void k_sum_columns(const uint32_t* __restrict__ in, uint32_t rows, uint32_t cols, uint32_t* __restrict__ out) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    uint32_t sum = 0;
    for (uint32_t r = 0; r < rows; ++r) sum += in[(size_t)r * cols + c];
    out[c] = sum;
}

// Bucket ids of every key (the distribution passes' lookup, for checking).
template <typename K>
__global__ void k_bucket_ids(const K* __restrict__ keys, uint32_t n, BucketDigit<K> df, uint32_t* __restrict__ ids) {
    extern __shared__ __align__(16) unsigned char smem[];
    df.setup(smem);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        ids[i] = df.bucket(keys[i]);
}

// ---------------------------------------------------------------- host side

// Fits the model on u (device, m normalised sorted sample values); see k_cdf_fit.
isort_status launch_fit(const float* u, uint32_t m, float* theta, float* X, float* Y, float* losses, float* loss0,
                        float* grad, int steps, cudaStream_t s) {
    LaunchScope ls("cdf_fit", s);
    k_cdf_fit<<<1, kFitThreads, 0, s>>>(u, m, theta, X, Y, losses, loss0, grad, steps, kLearningRate);
    return from_cuda(cudaGetLastError());
}

int ceil_log2(uint32_t v) {
    int b = 0;
    while ((1u << b) < v) ++b;
    return b;
}

int bit_length(uint64_t v) {
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

// Launch shape of the distribution passes: 512 x 8 for u32 keys; 256 x 8 for
// u64 keys, whose larger buffers would otherwise leave one CTA per SM.
template <typename K>
struct BucketShape {
    static constexpr int kThreads = sizeof(K) == 4 ? 512 : 256;
    static constexpr int kItems = 8;
    static constexpr uint32_t kTile = (uint32_t)kThreads * kItems;
};

// Sets the pass kernel's shared-memory size and returns it (per_sm: resident
// CTAs per SM, optional).
template <typename K, bool VALS>
isort_status bucket_sweep_setup(int bins, size_t* smem, int* per_sm) {
    using Sh = BucketShape<K>;
    *smem = SweepCfg<K, VALS, Sh::kThreads, Sh::kItems>::smem_bytes(bins, false, 0);
    if (*smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    auto kern = k_downsweep<K, VALS, Sh::kThreads, Sh::kItems, 0, IdDigit>;
    ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem));
    if (per_sm) {
        ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, Sh::kThreads, *smem));
        if (*per_sm < 1) return ISORT_ERR_UNSUPPORTED;
    }
    return ISORT_OK;
}

template <typename K>
isort_status launch_bucket_sweep(const SweepArgs& a, const IdDigit& df, uint32_t chunks, bool vals, cudaStream_t s) {
    using Sh = BucketShape<K>;
    size_t smem = 0;
    LaunchScope ls("bucket_sweep", s);
    if (vals) {
        ISORT_TRY((bucket_sweep_setup<K, true>(a.bins, &smem, nullptr)));
        k_downsweep<K, true, Sh::kThreads, Sh::kItems, 0, IdDigit><<<chunks, Sh::kThreads, smem, s>>>(a, df);
    } else {
        ISORT_TRY((bucket_sweep_setup<K, false>(a.bins, &smem, nullptr)));
        k_downsweep<K, false, Sh::kThreads, Sh::kItems, 0, IdDigit><<<chunks, Sh::kThreads, smem, s>>>(a, df);
    }
    return from_cuda(cudaGetLastError());
}

template <typename K>
isort_status learned_device(K* keys, uint32_t* vals, size_t n, int key_bits, int B, int model,
                            isort_learned_stats* stats, cudaStream_t s) {
    std::memset(stats, 0, sizeof(*stats));
    const float scale = std::ldexp(1.0f, -key_bits);
    const uint32_t m = kSampleSize;
    const int id_bits = ceil_log2((uint32_t)B);
    const int passes = id_bits > 8 ? 2 : 1;
    const int wsub = (id_bits + passes - 1) / passes;
    const int bins = 1 << wsub;
    const bool hv = vals != nullptr;

    // launch geometry of the distribution passes
    const uint32_t tile = BucketShape<K>::kTile;
    const size_t tb = bucket_tab_bytes();
    const size_t census_smem = align_up((size_t)bins * 4 + align_up((size_t)B, 4) * 4, 16) + tb;
    if (census_smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    int per_sm = 0;
    {
        size_t sweep_smem = 0;
        const isort_status so = hv ? bucket_sweep_setup<K, true>(bins, &sweep_smem, &per_sm)
                                   : bucket_sweep_setup<K, false>(bins, &sweep_smem, &per_sm);
        if (so != ISORT_OK) return so;
    }
    {
        // the census runs one CTA per chunk too: no more chunks than it keeps
        // resident, so that it runs in one wave
        int census_per_sm = 0;
        ISORT_TRY_CUDA(cudaFuncSetAttribute(k_bucket_census<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)census_smem));
        ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&census_per_sm, k_bucket_census<K>,
                                                                     kCensusThreads, census_smem));
        if (census_per_sm >= 1) per_sm = std::min(per_sm, census_per_sm);
    }
    const uint32_t num_tiles = (uint32_t)((n + tile - 1) / tile);
    const uint32_t want = (uint32_t)per_sm * (uint32_t)sm_count();
    const uint32_t chunk_tiles = (num_tiles + want - 1) / want;
    const uint32_t chunks = (num_tiles + chunk_tiles - 1) / chunk_tiles;

    // scratch
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes, 256);
        return o;
    };
    const size_t o_status = take(64);
    const size_t o_sample = take((size_t)m * sizeof(K)), o_u = take((size_t)m * 4);
    const size_t o_theta = take(2 * kPwlSegments * 4);  // also holds the MLP's 97 parameters
    const size_t o_X = take(kPwlKnots * 4), o_Y = take(kPwlKnots * 4);
    const size_t o_loss = take((kTrainSteps + 2) * 4);
    const size_t o_split = take((size_t)B * sizeof(K)), o_bcount = take((size_t)B * 4);
    const size_t o_bpart = take((size_t)chunks * B * 4);
    const size_t o_hist = take((size_t)chunks * bins * 4), o_coff = take((size_t)chunks * bins * 4);
    const size_t o_segoff = take((size_t)(B + 1) * 8), o_seglo = take((size_t)B * sizeof(K)), o_segbits = take((size_t)B);
    const size_t o_buf = take(n * sizeof(K) + (hv ? align_up(n * 4, 256) : 0));
    const size_t o_ids = take(2 * align_up(n * 2, 256));  // bucket ids: the census's, then the first pass's output
    unsigned char* ws = nullptr;
    isort_status st = scratch_alloc((void**)&ws, off, s);
    if (st != ISORT_OK) return st;
    auto fail = [&](isort_status e) {
        scratch_free(ws, s);
        return e;
    };
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + o_status);
    K* sample = reinterpret_cast<K*>(ws + o_sample);
    float* u = reinterpret_cast<float*>(ws + o_u);
    float* theta = reinterpret_cast<float*>(ws + o_theta);
    float* X = reinterpret_cast<float*>(ws + o_X);
    float* Y = reinterpret_cast<float*>(ws + o_Y);
    float* losses = reinterpret_cast<float*>(ws + o_loss);
    K* split = reinterpret_cast<K*>(ws + o_split);
    uint32_t* bcount = reinterpret_cast<uint32_t*>(ws + o_bcount);
    uint32_t* bpart = reinterpret_cast<uint32_t*>(ws + o_bpart);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + o_hist);
    uint32_t* coff = reinterpret_cast<uint32_t*>(ws + o_coff);
    uint64_t* segoff = reinterpret_cast<uint64_t*>(ws + o_segoff);
    K* seglo = reinterpret_cast<K*>(ws + o_seglo);
    uint8_t* segbits = reinterpret_cast<uint8_t*>(ws + o_segbits);
    K* wk = reinterpret_cast<K*>(ws + o_buf);
    uint32_t* wv = hv ? reinterpret_cast<uint32_t*>(ws + o_buf + align_up(n * sizeof(K), 256)) : nullptr;
    uint16_t* ids[2] = {reinterpret_cast<uint16_t*>(ws + o_ids),
                        reinterpret_cast<uint16_t*>(ws + o_ids + align_up(n * 2, 256))};

    cudaError_t ce = cudaMemsetAsync(ws, 0, 128, s);
    if (ce != cudaSuccess) return fail(from_cuda(ce));

    // 1. sample and sort it
    {
        LaunchScope ls("sample_gather", s);
        k_sample_gather<K><<<(m + 255) / 256, 256, 0, s>>>(keys, (uint64_t)n, m, sample);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    st = sort_sample(sample, m, key_bits, segoff, seglo, segbits, s);
    if (st != ISORT_OK) return fail(st);

    // 2. train the model (both leave their CDF as the table X, Y)
    if (model == 0 || model == 2) {
        {
            LaunchScope ls("cdf_init", s);
            k_normalise<K><<<(m / kFitStride + 255) / 256, 256, 0, s>>>(sample, m / kFitStride, kFitStride, scale, u);
            k_model_init<K><<<1, kPwlSegments, 0, s>>>(sample, m, scale, theta);
            ce = cudaGetLastError();
            if (ce != cudaSuccess) return fail(from_cuda(ce));
        }
        // model 2 (regular sampling): no steps, the table of the start; its
        // loss lands where the record of a trained model keeps it
        st = model == 0 ? launch_fit(u, m / kFitStride, theta, X, Y, losses, nullptr, nullptr, kTrainSteps, s)
                        : launch_fit(u, m / kFitStride, theta, X, Y, losses + kTrainSteps, nullptr, nullptr, 0, s);
    } else {
        st = mlp_model<K>(sample, m, scale, u, theta, X, Y, losses, s);
    }
    if (st != ISORT_OK) return fail(st);

    // 3. splitters
    {
        LaunchScope ls("splitters", s);
        k_splitters<K><<<(B + 255) / 256, 256, 0, s>>>(X, Y, B, key_bits, scale, split);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    BucketDigit<K> df;
    df.g_X = X;
    df.g_Y = Y;
    df.B = B;
    df.scale = scale;
    df.sub_shift = 0;
    df.sub_mask = (uint32_t)bins - 1u;

    // 4. census
    const int vec = ((uintptr_t)keys % 16) == 0 ? 1 : 0;
    {
        const size_t smem = census_smem;
        ce = cudaFuncSetAttribute(k_bucket_census<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ce != cudaSuccess) return fail(from_cuda(ce));
        LaunchScope ls("bucket_census", s);
        k_bucket_census<K><<<chunks, kCensusThreads, smem, s>>>(keys, (uint32_t)n, chunk_tiles * tile, df, hist, bpart,
                                                              key_bits, status, vec, ids[0]);
        k_sum_columns<<<(B + 255) / 256, 256, 0, s>>>(bpart, chunks, (uint32_t)B, bcount);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    std::vector<uint32_t> h_count(B);
    std::vector<K> h_split(B);
    std::vector<float> h_loss(kTrainSteps + 2);
    uint32_t h_status = 0;
    ce = cudaMemcpyAsync(h_count.data(), bcount, (size_t)B * 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_split.data(), split, (size_t)B * sizeof(K), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_loss.data(), losses, (kTrainSteps + 2) * 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return fail(from_cuda(ce));
    if (h_status != 0) return fail(map_bits(h_status));  // keys unchanged
    uint64_t maxc = 0, over = 0, over_b = 0;
    for (int b = 0; b < B; ++b) {
        maxc = std::max<uint64_t>(maxc, h_count[b]);
        if (h_count[b] > kOnChipCapacity) {
            over += h_count[b];
            ++over_b;
        }
    }
    stats->imbalance_max_over_mean = (double)maxc / ((double)n / B);
    stats->overflow_fraction = (double)over / (double)n;
    stats->overflow_buckets = over_b;
    stats->fixups = 0;  // the bucket function is monotone: nothing to correct
    stats->train_loss = h_loss[kTrainSteps];
    stats->train_loss_initial = h_loss[kTrainSteps + 1];
    stats->train_steps = model == 2 ? 0 : kTrainSteps;
    stats->nbuckets = B;
    if (stats->overflow_fraction > 0.5) {
        stats->fell_back_to_lsd = 1;
        st = plain_sort(keys, vals, n, key_bits, s);
        scratch_free(ws, s);
        return st;
    }

    // 5. stable distribution by bucket id (LSD over its halves); the ids the
    // census stored move with their keys (IdDigit), so the model is not
    // evaluated again
    K* src_k = keys;
    uint32_t* src_v = vals;
    for (int p = 0; p < passes; ++p) {
        const bool to_buf = (p % 2) == 0;
        K* dk = to_buf ? wk : keys;
        uint32_t* dv = to_buf ? wv : vals;
        IdDigit idf;
        idf.ids_in = ids[p];
        idf.ids_out = p + 1 < passes ? ids[p + 1] : nullptr;
        idf.sub_shift = p * wsub;
        idf.sub_mask = (uint32_t)((1 << std::min(wsub, id_bits - p * wsub)) - 1);
        const int pbins = (int)idf.sub_mask + 1;
        if (p > 0) {  // per-chunk counts of this pass's digit, from the moved ids
            constexpr int kIdSub = 16;
            const size_t smem = (size_t)kIdSub * pbins * 4;
            ce = cudaFuncSetAttribute(k_chunk_hist<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (ce != cudaSuccess) return fail(from_cuda(ce));
            LaunchScope ls("bucket_hist", s);
            k_chunk_hist<uint16_t><<<chunks, kChunkHistThreads, smem, s>>>(
                ids[p], (uint32_t)n, idf.sub_shift, ceil_log2((uint32_t)pbins), chunk_tiles * tile, kIdSub, hist,
                nullptr, 1);
            ce = cudaGetLastError();
            if (ce != cudaSuccess) return fail(from_cuda(ce));
        }
        {
            const int groups = pbins >= kChunkScanThreads ? 1 : kChunkScanThreads / pbins;
            LaunchScope ls("chunk_scan", s);
            k_chunk_scan<<<1, kChunkScanThreads, (size_t)(groups + 1) * pbins * 4, s>>>(
                hist, (int)chunks, pbins, coff, nullptr, key_bits, (int)sizeof(K) * 8, status);
            ce = cudaGetLastError();
            if (ce != cudaSuccess) return fail(from_cuda(ce));
        }
        SweepArgs a;
        a.keys_in = src_k;
        a.vals_in = src_v;
        a.keys_out = dk;
        a.vals_out = dv;
        a.n = (uint32_t)n;
        a.shift = 0;
        a.width = ceil_log2((uint32_t)pbins);
        a.bins = pbins;
        a.chunk_off = coff;
        a.chunk_tiles = chunk_tiles;
        a.num_tiles = num_tiles;
        a.status = status;
        a.limit_ns = spin_limit_ns();
        a.use_bulk = (((uintptr_t)src_k % 16) == 0) && (!hv || ((uintptr_t)src_v % 16) == 0);
        st = launch_bucket_sweep<K>(a, idf, chunks, hv, s);
        if (st != ISORT_OK) return fail(st);
        src_k = dk;
        src_v = dv;
    }
    if (src_k != keys) {
        ce = cudaMemcpyAsync(keys, src_k, n * sizeof(K), cudaMemcpyDeviceToDevice, s);
        if (ce == cudaSuccess && hv) ce = cudaMemcpyAsync(vals, src_v, n * 4, cudaMemcpyDeviceToDevice, s);
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }

    // 6. finish every bucket on the bits its key range spans; buckets beyond
    // the on-chip capacity are sorted by the plain rounds, one at a time
    std::vector<uint64_t> h_off(B + 1);
    std::vector<K> h_lo(B);
    std::vector<uint8_t> h_bits(B);
    std::vector<int> big;
    h_off[0] = 0;
    const uint64_t kmax = key_bits >= 64 ? ~0ull : ((1ull << key_bits) - 1ull);
    for (int b = 0; b < B; ++b) {
        h_off[b + 1] = h_off[b] + h_count[b];
        const uint64_t lo = b == 0 ? 0 : (uint64_t)h_split[b];
        const uint64_t hi_incl = b + 1 < B ? (uint64_t)h_split[b + 1] - (h_split[b + 1] > 0 ? 1 : 0) : kmax;
        h_lo[b] = (K)lo;
        const uint64_t span = hi_incl >= lo ? hi_incl - lo : 0;
        h_bits[b] = (uint8_t)bit_length(span);
        if (h_count[b] > kOnChipCapacity && h_bits[b] > 0) {
            big.push_back(b);
            h_bits[b] = 0;  // not a segment of the on-chip finish
        }
    }
    ce = cudaMemcpyAsync(segoff, h_off.data(), (size_t)(B + 1) * 8, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(seglo, h_lo.data(), (size_t)B * sizeof(K), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(segbits, h_bits.data(), (size_t)B, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return fail(from_cuda(ce));
    st = finish_buckets(keys, vals, segoff, (uint32_t)B, seglo, segbits, s);
    if (st == ISORT_OK && big.size() == 1) {
        const int b = big[0];
        st = plain_sort(keys + h_off[b], hv ? vals + h_off[b] : nullptr, h_count[b], key_bits, s);
    } else if (st == ISORT_OK && big.size() > 1) {
        // The overflow buckets hold disjoint key ranges in increasing order, so
        // their concatenation (in bucket order) sorted stably is each of them
        // sorted: gather them into the free distribution buffer, sort that
        // once with the plain rounds, scatter back.
        const uint32_t nr = (uint32_t)big.size();
        std::vector<uint64_t> h_roff(nr), h_pos(nr + 1);
        std::vector<uint32_t> h_cst(nr + 1);
        h_pos[0] = 0;
        h_cst[0] = 0;
        for (uint32_t r = 0; r < nr; ++r) {
            h_roff[r] = h_off[big[r]];
            h_pos[r + 1] = h_pos[r] + h_count[big[r]];
            h_cst[r + 1] = h_cst[r] + (uint32_t)((h_count[big[r]] + kMoveChunk - 1) / kMoveChunk);
        }
        unsigned char* tab = nullptr;
        const size_t tb8 = align_up((size_t)(nr + 1) * 8, 256);
        st = scratch_alloc((void**)&tab, 3 * tb8, s);
        if (st == ISORT_OK) {
            uint64_t* d_roff = reinterpret_cast<uint64_t*>(tab);
            uint64_t* d_pos = reinterpret_cast<uint64_t*>(tab + tb8);
            uint32_t* d_cst = reinterpret_cast<uint32_t*>(tab + 2 * tb8);
            ce = cudaMemcpyAsync(d_roff, h_roff.data(), (size_t)nr * 8, cudaMemcpyHostToDevice, s);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_pos, h_pos.data(), (size_t)(nr + 1) * 8, cudaMemcpyHostToDevice, s);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_cst, h_cst.data(), (size_t)(nr + 1) * 4, cudaMemcpyHostToDevice, s);
            if (ce == cudaSuccess) {
                LaunchScope ls("overflow_gather", s);
                k_move_ranges<K><<<h_cst[nr], 256, 0, s>>>(keys, vals, wk, wv, d_roff, d_pos, d_cst, nr, 1);
                ce = cudaGetLastError();
            }
            st = from_cuda(ce);
            if (st == ISORT_OK) st = plain_sort(wk, wv, h_pos[nr], key_bits, s);
            if (st == ISORT_OK) {
                LaunchScope ls("overflow_scatter", s);
                k_move_ranges<K><<<h_cst[nr], 256, 0, s>>>(keys, vals, wk, wv, d_roff, d_pos, d_cst, nr, 0);
                st = from_cuda(cudaGetLastError());
            }
            scratch_free(tab, s);
        }
    }
    if (st != ISORT_OK) return fail(st);
    st = finish_status(status, s);
    scratch_free(ws, s);
    return st;
}

}  // namespace
}  // namespace isort

using namespace isort;

namespace {

template <typename K>
isort_status learned_entry(K* keys, uint32_t* vals, size_t n, int key_bits, int nbuckets, int model,
                           isort_learned_stats* stats, void* stream) {
    constexpr int kw = (int)sizeof(K) * 8;
    isort_learned_stats local;
    isort_learned_stats* st = stats ? stats : &local;
    std::memset(st, 0, sizeof(*st));
    if (key_bits == 0) key_bits = kw;
    if (key_bits < 1 || key_bits > kw) return ISORT_ERR_INVALID_ARG;
    if (nbuckets == 0) {
        if constexpr (sizeof(K) == 4) {
            // 4096 buckets, doubled (up to the table limit) while the mean
            // bucket would exceed a quarter of the on-chip capacity
            nbuckets = 4096;
            while (nbuckets < kMaxBuckets && (uint64_t)nbuckets * (kOnChipCapacity / 4) < n) nbuckets <<= 1;
        } else {
            // u64: a multiple of 4096 with a mean bucket of at most 6,656 keys,
            // so that buckets (about +-1.5 % apart at these sizes) stay within
            // one CTA's 8,192 keys, the fine finish's class
            const uint64_t want = (n + 4096ull * 6656 - 1) / (4096ull * 6656);
            nbuckets = (int)std::min<uint64_t>(std::max<uint64_t>(want, 1), kMaxBuckets / 4096) * 4096;
        }
    }
    if (nbuckets < 2 || nbuckets > kMaxBuckets) return ISORT_ERR_INVALID_ARG;
    if (model < 0 || model > 2) return ISORT_ERR_INVALID_ARG;
    if (n >= (size_t(1) << 30)) return ISORT_ERR_UNSUPPORTED;
    if (n > 1 && !keys) return ISORT_ERR_INVALID_ARG;
    if (n <= 1) return ISORT_OK;
    if (is_host_pointer(keys) || (vals && is_host_pointer(vals))) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n < (size_t)4 * kSampleSize) {
        // too few keys for a sample to pay off: the plain rounds
        st->fell_back_to_lsd = 1;
        return plain_sort(keys, vals, n, key_bits, s);
    }
    return learned_device<K>(keys, vals, n, key_bits, nbuckets, model, st, s);
}

}  // namespace


extern "C" {

isort_status isort_learned(uint32_t* keys, uint32_t* vals, size_t n, int key_bits, int nbuckets, int model,
                           isort_learned_stats* stats, void* stream) {
    return learned_entry<uint32_t>(keys, vals, n, key_bits, nbuckets, model, stats, stream);
}

isort_status isort_learned_u64(uint64_t* keys, uint32_t* vals, size_t n, int key_bits, int nbuckets, int model,
                               isort_learned_stats* stats, void* stream) {
    return learned_entry<uint64_t>(keys, vals, n, key_bits, nbuckets, model, stats, stream);
}

isort_status isort_cdf_splitters(const float* X, const float* Y, int key_width, int key_bits, int nbuckets,
                                 void* splitters, void* stream) {
    if (key_width != 32 && key_width != 64) return ISORT_ERR_INVALID_ARG;
    if (key_bits == 0) key_bits = key_width;
    if (key_bits < 1 || key_bits > key_width || nbuckets < 2 || nbuckets > 65536 || !X || !Y || !splitters)
        return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float scale = std::ldexp(1.0f, -key_bits);
    LaunchScope ls("splitters", s);
    if (key_width == 32) {
        k_splitters<uint32_t><<<(nbuckets + 255) / 256, 256, 0, s>>>(X, Y, nbuckets, key_bits, scale,
                                                                     static_cast<uint32_t*>(splitters));
    } else {
        k_splitters<uint64_t><<<(nbuckets + 255) / 256, 256, 0, s>>>(X, Y, nbuckets, key_bits, scale,
                                                                     static_cast<uint64_t*>(splitters));
    }
    ISORT_TRY_CUDA(cudaGetLastError());
    if (sync_mode()) ISORT_TRY_CUDA(cudaStreamSynchronize(s));
    return ISORT_OK;
}

isort_status isort_bucket_ids(const void* keys, int key_width, size_t n, int key_bits, const float* X, const float* Y,
                              int nbuckets, uint32_t* ids, void* stream) {
    if (key_width != 32 && key_width != 64) return ISORT_ERR_INVALID_ARG;
    if (key_bits == 0) key_bits = key_width;
    if (key_bits < 1 || key_bits > key_width || nbuckets < 2 || nbuckets > 65536) return ISORT_ERR_INVALID_ARG;
    if (n == 0) return ISORT_OK;
    if (!keys || !X || !Y || !ids || n >= (size_t(1) << 32)) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float scale = std::ldexp(1.0f, -key_bits);
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 8);
    const size_t smem = bucket_tab_bytes();
    LaunchScope ls("bucket_ids", s);
    if (key_width == 32) {
        BucketDigit<uint32_t> df{X, Y, nbuckets, scale, 0, 0xffffu, nullptr, nullptr, nullptr, nullptr};
        k_bucket_ids<uint32_t><<<grid, 256, smem, s>>>(static_cast<const uint32_t*>(keys), (uint32_t)n, df, ids);
    } else {
        BucketDigit<uint64_t> df{X, Y, nbuckets, scale, 0, 0xffffu, nullptr, nullptr, nullptr, nullptr};
        k_bucket_ids<uint64_t><<<grid, 256, smem, s>>>(static_cast<const uint64_t*>(keys), (uint32_t)n, df, ids);
    }
    ISORT_TRY_CUDA(cudaGetLastError());
    if (sync_mode()) ISORT_TRY_CUDA(cudaStreamSynchronize(s));
    return ISORT_OK;
}

isort_status isort_cdf_loss_grad(const float* u, uint32_t m, const float* theta, float* grad, float* loss,
                                 void* stream) {
    if (!u || !theta || !grad || !loss || m == 0) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float* th = nullptr;  // the fit writes its parameters back: work on a copy
    isort_status st = scratch_alloc((void**)&th, 2 * kPwlSegments * 4, s);
    if (st != ISORT_OK) return st;
    cudaError_t ce = cudaMemcpyAsync(th, theta, 2 * kPwlSegments * 4, cudaMemcpyDeviceToDevice, s);
    st = ce == cudaSuccess ? launch_fit(u, m, th, nullptr, nullptr, nullptr, loss, grad, 0, s) : from_cuda(ce);
    scratch_free(th, s);
    if (st == ISORT_OK && sync_mode()) st = from_cuda(cudaStreamSynchronize(s));
    return st;
}

isort_status isort_cdf_train(const uint32_t* sorted_sample, uint32_t m, int key_bits, float* theta, float* X,
                             float* Y, float* losses, void* stream) {
    if (!sorted_sample || !theta || !X || !Y || !losses || m < 2) return ISORT_ERR_INVALID_ARG;
    if (key_bits == 0) key_bits = 32;
    if (key_bits < 1 || key_bits > 32) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float* u = nullptr;
    isort_status st = scratch_alloc((void**)&u, (size_t)m * 4, s);
    if (st != ISORT_OK) return st;
    const float scale = std::ldexp(1.0f, -key_bits);
    {
        LaunchScope ls("cdf_init", s);
        k_normalise<uint32_t><<<(m + 255) / 256, 256, 0, s>>>(sorted_sample, m, 1, scale, u);
        k_model_init<uint32_t><<<1, kPwlSegments, 0, s>>>(sorted_sample, m, scale, theta);
        st = from_cuda(cudaGetLastError());
    }
    if (st == ISORT_OK) st = launch_fit(u, m, theta, X, Y, losses, nullptr, nullptr, kTrainSteps, s);
    scratch_free(u, s);
    if (st == ISORT_OK && sync_mode()) st = from_cuda(cudaStreamSynchronize(s));
    return st;
}

}  // extern "C"
