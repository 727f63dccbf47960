// Learned-bucket sort: a monotone CDF model, trained on the GPU on a sample
// that the method sorts itself, proposes each key's bucket for an MSD
// distribution pass; exact integer splitters fix the proposals up, and the
// buckets are then finished independently on chip.
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
//      error between F(u_i) and the sample's empirical CDF (i + 1/2)/m; knot
//      positions start at sample quantiles, values at i/256; the steps are
//      captured in a CUDA graph, and the parameters with the lowest loss seen
//      (the initial ones included) are kept;
//   3. splitter table: s_b = first key with F(key) >= b/B (fp32, fixed
//      operation order), made non-decreasing; bucket(key) = #{b in 1..B-1 :
//      s_b <= key}. The model's proposal floor(F(u) B) is accepted when the
//      splitters confirm it, else a binary search fixes it (counted);
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
isort_status segmented_finish_u32(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint32_t nseg,
                                  const uint32_t* seg_lo, const uint8_t* seg_bits, cudaStream_t s);

namespace {

constexpr uint32_t kSampleSize = 1u << 16;
constexpr uint64_t kSampleSeed = 0x5EED5EED5EEDull;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kTrainSteps = 64;
constexpr float kLearningRate = 0.02f;
constexpr int kGradCtas = 64;
constexpr int kGradThreads = 256;
constexpr int kPartial = 2 * kPwlKnots + 1;  // gX[257] gY[257] loss
constexpr uint32_t kOnChipCapacity = 65536;  // keys a cluster finishes on chip
constexpr int kMaxBuckets = 16384;           // the splitter table is held in shared memory

__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------- sampling

template <typename K>
__global__ void k_sample_gather(const K* __restrict__ keys, uint64_t n, uint32_t m, K* __restrict__ out) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const uint64_t r = splitmix_mix(kSampleSeed + (uint64_t)(j + 1) * kGamma);
    const uint64_t idx = __umul64hi(r, n);  // floor(r * n / 2^64) < n
    out[j] = keys[idx];
}

template <typename K>
__global__ void k_normalise(const K* __restrict__ sorted, uint32_t m, float scale, float* __restrict__ u) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) u[j] = normalise_key(sorted[j], scale);
}

// ---------------------------------------------------------------- the model

__device__ __forceinline__ float softplus(float t) { return t > 20.f ? t : log1pf(expf(t)); }
__device__ __forceinline__ float inv_softplus(float v) { return v > 20.f ? v : logf(expm1f(v)); }
__device__ __forceinline__ float sigmoidf_(float t) { return 1.f / (1.f + expf(-t)); }

// theta[0..255]: knot-position increments; theta[256..511]: value increments.
// X, Y: cumulative sums of softplus(theta) normalised to end at 1 (one CTA of
// 256 threads, fixed order, so the result is a function of theta alone).
__device__ void derive_knots(const float* theta, float* X, float* Y, float* s_tmp) {
    const int t = threadIdx.x;
    for (int which = 0; which < 2; ++which) {
        float* V = which == 0 ? X : Y;
        s_tmp[t] = softplus(theta[which * kPwlSegments + t]);
        __syncthreads();
        if (t == 0) {
            float run = 0.f;
            for (int i = 0; i < kPwlSegments; ++i) {
                const float v = s_tmp[i];
                s_tmp[i] = run;
                run += v;
            }
            s_tmp[kPwlSegments] = run;
        }
        __syncthreads();
        const float total = s_tmp[kPwlSegments];
        V[t] = t == 0 ? 0.f : s_tmp[t] / total;
        if (t == 0) V[kPwlSegments] = 1.f;
        __syncthreads();
    }
}

// Initial parameters from the sorted sample: knot positions at the sample's
// quantiles j/256, values j/256.
template <typename K>
__global__ void __launch_bounds__(kPwlSegments) k_model_init(const K* __restrict__ sorted, uint32_t m, float scale,
                                                             float* theta, float* X, float* Y, float* adam) {
    __shared__ float s_tmp[kPwlKnots];
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
    adam[t] = adam[kPwlSegments + t] = 0.f;
    adam[2 * kPwlSegments + t] = adam[3 * kPwlSegments + t] = 0.f;
    __syncthreads();
    derive_knots(theta, X, Y, s_tmp);
}

__global__ void __launch_bounds__(kPwlSegments) k_model_derive(const float* theta, float* X, float* Y) {
    __shared__ float s_tmp[kPwlKnots];
    derive_knots(theta, X, Y, s_tmp);
}

// Loss and gradient with respect to the knots, partial sums per CTA:
// L = (1/m) sum_i (F(u_i) - (i + 1/2)/m)^2.
__global__ void __launch_bounds__(kGradThreads) k_model_grad(const float* __restrict__ u, uint32_t m,
                                                              const float* __restrict__ X,
                                                              const float* __restrict__ Y, float* __restrict__ partial) {
    __shared__ float sX[kPwlKnots], sY[kPwlKnots], gX[kPwlKnots], gY[kPwlKnots];
    __shared__ float s_loss;
    const int t = threadIdx.x;
    for (int i = t; i < kPwlKnots; i += kGradThreads) {
        sX[i] = X[i];
        sY[i] = Y[i];
        gX[i] = 0.f;
        gY[i] = 0.f;
    }
    if (t == 0) s_loss = 0.f;
    __syncthreads();
    const uint32_t per_cta = (m + gridDim.x - 1) / gridDim.x;
    const uint32_t c0 = blockIdx.x * per_cta, c1 = min(m, c0 + per_cta);
    const uint32_t per_thread = (per_cta + kGradThreads - 1) / kGradThreads;
    const uint32_t p0 = c0 + t * per_thread, p1 = min(c1, p0 + per_thread);  // contiguous points per thread
    const float inv_m = 1.f / (float)m;
    float loss = 0.f;
    for (uint32_t i = p0; i < p1; ++i) {
        const float x = u[i];
        const int j = x < sX[kPwlSegments] ? pwl_segment(sX, x) : kPwlSegments - 1;
        const float dx = sX[j + 1] - sX[j];
        const float dy = sY[j + 1] - sY[j];
        const float w = dx > 0.f ? fminf(fmaxf((x - sX[j]) / dx, 0.f), 1.f) : 0.f;
        const float f = sY[j] + dy * w;
        const float e = f - ((float)i + 0.5f) * inv_m;
        loss += e * e;
        const float ge = 2.f * e * inv_m;
        atomicAdd(&gY[j], ge * (1.f - w));
        atomicAdd(&gY[j + 1], ge * w);
        if (dx > 0.f && x < sX[j + 1]) {
            const float k = ge * dy / (dx * dx);
            atomicAdd(&gX[j], k * (x - sX[j + 1]));
            atomicAdd(&gX[j + 1], -k * (x - sX[j]));
        }
    }
    atomicAdd(&s_loss, loss * inv_m);
    __syncthreads();
    float* out = partial + (size_t)blockIdx.x * kPartial;
    for (int i = t; i < kPwlKnots; i += kGradThreads) {
        out[i] = gX[i];
        out[kPwlKnots + i] = gY[i];
    }
    if (t == 0) out[2 * kPwlKnots] = s_loss;
}

// Reduces the partials (fixed order), maps knot gradients to theta through the
// normalised softplus sums, and applies one Adam step (lr = 0: gradient only).
// grad_out (optional): dL/dtheta; loss_out[step]: loss at the current theta.
// best[0..511], best[512]: the parameters with the lowest loss seen so far.
// mode kStepPlain: no record; kStepTrain: record (the first step resets it);
// kStepFinal: keep the current parameters if they beat the record, else
// restore the record (loss_out[step] then holds the record's loss).
enum { kStepPlain = 0, kStepTrain = 1, kStepFinal = 2 };

__global__ void __launch_bounds__(kPwlSegments) k_model_step(const float* __restrict__ partial, int parts,
                                                             float* theta, float* adam, float* X, float* Y,
                                                             int step, float lr, float* loss_out, float* grad_out,
                                                             float* best, int mode) {
    __shared__ float s_g[2][kPwlKnots];
    __shared__ float s_tmp[kPwlKnots];
    __shared__ float s_red[2];
    __shared__ int s_take;  // 1: record the current parameters; 2: restore the record
    const int t = threadIdx.x;
    for (int i = t; i < kPwlKnots; i += kPwlSegments) {
        float gx = 0.f, gy = 0.f;
        for (int c = 0; c < parts; ++c) {
            gx += partial[(size_t)c * kPartial + i];
            gy += partial[(size_t)c * kPartial + kPwlKnots + i];
        }
        s_g[0][i] = gx;
        s_g[1][i] = gy;
    }
    if (t == 0) {
        float l = 0.f;
        for (int c = 0; c < parts; ++c) l += partial[(size_t)c * kPartial + 2 * kPwlKnots];
        int take = 0;
        if (mode == kStepTrain) take = (step == 0 || l < best[2 * kPwlSegments]) ? 1 : 0;
        if (mode == kStepFinal) take = l < best[2 * kPwlSegments] ? 1 : 2;
        if (take == 1) best[2 * kPwlSegments] = l;
        if (take == 2) l = best[2 * kPwlSegments];
        if (loss_out) loss_out[step] = l;
        s_take = take;
    }
    __syncthreads();
    if (s_take == 1) {
        best[t] = theta[t];
        best[kPwlSegments + t] = theta[kPwlSegments + t];
    }
    if (mode == kStepFinal) {
        if (s_take == 2) {
            theta[t] = best[t];
            theta[kPwlSegments + t] = best[kPwlSegments + t];
        }
        __syncthreads();
        derive_knots(theta, X, Y, s_tmp);
        return;
    }
    float dtheta[2];
    for (int which = 0; which < 2; ++which) {
        const float* V = which == 0 ? X : Y;
        const float* g = s_g[which];
        // A = sum_j g_j V_j ; suffix(i) = sum_{j > i} g_j ; S = sum softplus
        if (t == 0) {
            float A = 0.f, S = 0.f;
            for (int j = 0; j < kPwlKnots; ++j) A += g[j] * V[j];
            for (int i = 0; i < kPwlSegments; ++i) S += softplus(theta[which * kPwlSegments + i]);
            s_red[0] = A;
            s_red[1] = S;
            float run = 0.f;
            for (int i = kPwlSegments - 1; i >= 0; --i) {
                run += g[i + 1];
                s_tmp[i] = run;
            }
        }
        __syncthreads();
        const float th = theta[which * kPwlSegments + t];
        dtheta[which] = sigmoidf_(th) / s_red[1] * (s_tmp[t] - s_red[0]);
        __syncthreads();
    }
    for (int which = 0; which < 2; ++which) {
        const int idx = which * kPwlSegments + t;
        const float g = dtheta[which];
        if (grad_out) grad_out[idx] = g;
        if (lr > 0.f) {
            const float b1 = 0.9f, b2 = 0.999f;
            float m1 = adam[idx] = b1 * adam[idx] + (1.f - b1) * g;
            float m2 = adam[2 * kPwlSegments + idx] = b2 * adam[2 * kPwlSegments + idx] + (1.f - b2) * g * g;
            const float c1 = 1.f - powf(b1, (float)(step + 1)), c2 = 1.f - powf(b2, (float)(step + 1));
            theta[idx] -= lr * (m1 / c1) / (sqrtf(m2 / c2) + 1e-8f);
        }
    }
    __syncthreads();
    derive_knots(theta, X, Y, s_tmp);
}

// ---------------------------------------------------------------- splitters

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
    const float target = __fdiv_rn(__int2float_rn(b), __int2float_rn(B));
    uint64_t lo = 0, hi = key_bits >= 64 ? ~0ull : ((1ull << key_bits) - 1ull);
    while (lo < hi) {  // first key with F(key) >= target (the largest key if none)
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (pwl_eval(sX, sY, normalise_key((K)mid, scale)) >= target) hi = mid;
        else lo = mid + 1;
    }
    split[b] = (K)lo;
}

template <typename K>
__global__ void k_splitters_monotone(K* split, int B) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    K run = 0;
    for (int b = 1; b < B; ++b) {
        if (split[b] < run) split[b] = run;
        run = split[b];
    }
}

// ---------------------------------------------------------------- bucket lookup

// Bucket of a key from the splitter table: #{b in 1..B-1 : s_b <= key}. The
// model's proposal floor(F(u) B) is tried first.
template <typename K>
__device__ __forceinline__ uint32_t bucket_of(K k, const K* s, const float* X, const float* Y, int B, float scale,
                                              bool* fixed) {
    const float f = pwl_eval(X, Y, normalise_key(k, scale));
    int b0 = __float2int_rz(__fmul_rn(f, __int2float_rn(B)));
    b0 = b0 < 0 ? 0 : (b0 > B - 1 ? B - 1 : b0);
    if ((b0 == 0 || s[b0] <= k) && (b0 == B - 1 || k < s[b0 + 1])) {
        *fixed = false;
        return (uint32_t)b0;
    }
    *fixed = true;
    int lo = 0, hi = B - 1;  // largest b with (b == 0 || s_b <= k)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return (uint32_t)lo;
}

template <typename K>
struct BucketDigit {
    static constexpr bool kCheap = false;
    const K* g_split;
    const float* g_X;
    const float* g_Y;
    int B;
    float scale;
    int sub_shift;
    uint32_t sub_mask;
    K* s_split;
    float* s_X;
    float* s_Y;
    __device__ __forceinline__ size_t table_bytes() const {
        return 2 * align_up_dev(kPwlKnots * 4, 16) + align_up_dev((size_t)B * sizeof(K), 16);
    }
    __device__ __forceinline__ void setup(unsigned char* p) {
        s_X = reinterpret_cast<float*>(p);
        s_Y = reinterpret_cast<float*>(p + align_up_dev(kPwlKnots * 4, 16));
        s_split = reinterpret_cast<K*>(p + 2 * align_up_dev(kPwlKnots * 4, 16));
        for (int i = threadIdx.x; i < kPwlKnots; i += blockDim.x) {
            s_X[i] = g_X[i];
            s_Y[i] = g_Y[i];
        }
        for (int i = threadIdx.x; i < B; i += blockDim.x) s_split[i] = g_split[i];
        __syncthreads();
    }
    __device__ __forceinline__ uint32_t bucket(K k) const {
        bool fixed;
        return bucket_of<K>(k, s_split, s_X, s_Y, B, scale, &fixed);
    }
    __device__ __forceinline__ uint32_t digit(K k) const { return (bucket(k) >> sub_shift) & sub_mask; }
};

// Census: per-chunk counts of the first pass's digit, every bucket's size
// (global), the number of proposals the splitters corrected, and the key-range
// check (a key of key_bits or more bits sets the status).
constexpr int kCensusThreads = 512;

template <typename K>
__global__ void __launch_bounds__(kCensusThreads) k_bucket_census(const K* __restrict__ keys, uint32_t n,
                                                                  uint32_t chunk_keys, BucketDigit<K> df,
                                                                  uint32_t* __restrict__ hist,
                                                                  uint32_t* __restrict__ bucket_count,
                                                                  unsigned long long* fixups, int key_bits,
                                                                  uint32_t* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int bins = (int)df.sub_mask + 1;
    uint32_t* s_h = reinterpret_cast<uint32_t*>(smem);             // [bins]
    uint32_t* s_b = s_h + bins;                                    // [B]
    unsigned char* tab = reinterpret_cast<unsigned char*>(s_b + align_up_dev((size_t)df.B, 4));
    for (int i = threadIdx.x; i < bins; i += kCensusThreads) s_h[i] = 0;
    for (int i = threadIdx.x; i < df.B; i += kCensusThreads) s_b[i] = 0;
    df.setup(tab);
    const uint32_t lo = blockIdx.x * chunk_keys, hi = min(n, lo + chunk_keys);
    uint32_t fix = 0;
    K kor = 0;
    for (uint32_t i = lo + threadIdx.x; i < hi; i += kCensusThreads) {
        const K k = keys[i];
        kor |= k;
        bool fixed;
        const uint32_t b = bucket_of<K>(k, df.s_split, df.s_X, df.s_Y, df.B, df.scale, &fixed);
        fix += fixed ? 1u : 0u;
        atomicAdd(&s_h[(b >> df.sub_shift) & df.sub_mask], 1u);
        atomicAdd(&s_b[b], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < bins; i += kCensusThreads) hist[(size_t)blockIdx.x * bins + i] = s_h[i];
    for (int i = threadIdx.x; i < df.B; i += kCensusThreads)
        if (s_b[i]) atomicAdd(&bucket_count[i], s_b[i]);
    fix = __reduce_add_sync(kFullMask, fix);
    if ((threadIdx.x & 31) == 0 && fix) atomicAdd(fixups, (unsigned long long)fix);
    if (key_bits < (int)sizeof(K) * 8 && (kor >> key_bits) != 0) set_status(status, kStatKeyRange);
}

// Per-chunk counts of a later pass's digit.
template <typename K>
__global__ void __launch_bounds__(kCensusThreads) k_bucket_hist(const K* __restrict__ keys, uint32_t n,
                                                                uint32_t chunk_keys, BucketDigit<K> df,
                                                                uint32_t* __restrict__ hist) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int bins = (int)df.sub_mask + 1;
    uint32_t* s_h = reinterpret_cast<uint32_t*>(smem);
    unsigned char* tab = smem + align_up_dev((size_t)bins * 4, 16);
    for (int i = threadIdx.x; i < bins; i += kCensusThreads) s_h[i] = 0;
    df.setup(tab);
    const uint32_t lo = blockIdx.x * chunk_keys, hi = min(n, lo + chunk_keys);
    for (uint32_t i = lo + threadIdx.x; i < hi; i += kCensusThreads) atomicAdd(&s_h[df.digit(keys[i])], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < bins; i += kCensusThreads) hist[(size_t)blockIdx.x * bins + i] = s_h[i];
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

struct ModelBufs {
    float* u;        // normalised sorted sample [m]
    float* theta;    // [512]
    float* adam;     // [1024]
    float* best;     // [513]: best parameters so far and their loss
    float* X;        // [257]
    float* Y;        // [257]
    float* partial;  // [kGradCtas][kPartial]
    float* losses;   // [kTrainSteps + 1]
};

isort_status launch_grad_step(const ModelBufs& mb, uint32_t m, int step, float lr, float* grad_out, int mode,
                              cudaStream_t s) {
    {
        LaunchScope ls("cdf_grad", s);
        k_model_grad<<<kGradCtas, kGradThreads, 0, s>>>(mb.u, m, mb.X, mb.Y, mb.partial);
        ISORT_TRY_CUDA(cudaGetLastError());
    }
    LaunchScope ls("cdf_step", s);
    k_model_step<<<1, kPwlSegments, 0, s>>>(mb.partial, kGradCtas, mb.theta, mb.adam, mb.X, mb.Y, step, lr,
                                           mb.losses, grad_out, mb.best, mode);
    return from_cuda(cudaGetLastError());
}

// kTrainSteps Adam steps, captured once per call into a CUDA graph.
isort_status train_model(const ModelBufs& mb, uint32_t m, int steps, cudaStream_t s) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    if (cap == cudaStreamCaptureStatusActive) {
        for (int i = 0; i < steps; ++i) {
            isort_status st = launch_grad_step(mb, m, i, kLearningRate, nullptr, kStepTrain, s);
            if (st != ISORT_OK) return st;
        }
    } else {
        cudaStream_t cs = nullptr;
        ISORT_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        isort_status st = ISORT_OK;
        if (ce == cudaSuccess) {
            CaptureScope scope;
            for (int i = 0; i < steps && st == ISORT_OK; ++i)
                st = launch_grad_step(mb, m, i, kLearningRate, nullptr, kStepTrain, cs);
            ce = cudaStreamEndCapture(cs, &g);
        }
        cudaGraphExec_t ex = nullptr;
        if (ce == cudaSuccess && st == ISORT_OK) ce = cudaGraphInstantiate(&ex, g, 0);
        if (ce == cudaSuccess && st == ISORT_OK) {
            LaunchScope ls("cdf_train_graph", s, false);
            ce = cudaGraphLaunch(ex, s);
        }
        if (ex) cudaGraphExecDestroy(ex);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (st != ISORT_OK) return st;
        if (ce != cudaSuccess) return from_cuda(ce);
    }
    // the loss of the final parameters; the best ones seen are kept
    return launch_grad_step(mb, m, steps, 0.f, nullptr, kStepFinal, s);
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

template <typename K>
isort_status launch_bucket_sweep(const SweepArgs& a, const BucketDigit<K>& df, uint32_t chunks, bool vals,
                                 cudaStream_t s) {
    using Cfg = SweepCfg<K, true, 512, 8>;
    using CfgK = SweepCfg<K, false, 512, 8>;
    const size_t tb = 2 * align_up(kPwlKnots * 4, 16) + align_up((size_t)df.B * sizeof(K), 16);
    LaunchScope ls("bucket_sweep", s);
    if (vals) {
        const size_t smem = Cfg::smem_bytes(a.bins, false, tb);
        auto kern = k_downsweep<K, true, 512, 8, 0, BucketDigit<K>>;
        ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<chunks, 512, smem, s>>>(a, df);
    } else {
        const size_t smem = CfgK::smem_bytes(a.bins, false, tb);
        auto kern = k_downsweep<K, false, 512, 8, 0, BucketDigit<K>>;
        ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<chunks, 512, smem, s>>>(a, df);
    }
    return from_cuda(cudaGetLastError());
}

template <typename K>
isort_status learned_device(K* keys, uint32_t* vals, size_t n, int key_bits, int B, isort_learned_stats* stats,
                            cudaStream_t s) {
    std::memset(stats, 0, sizeof(*stats));
    const float scale = std::ldexp(1.0f, -key_bits);
    const uint32_t m = kSampleSize;
    const int id_bits = ceil_log2((uint32_t)B);
    const int passes = id_bits > 8 ? 2 : 1;
    const int wsub = (id_bits + passes - 1) / passes;
    const int bins = 1 << wsub;
    const bool hv = vals != nullptr;

    // launch geometry of the distribution passes
    using Cfg = SweepCfg<K, true, 512, 8>;
    const uint32_t tile = 512 * 8;
    const size_t tb = 2 * align_up(kPwlKnots * 4, 16) + align_up((size_t)B * sizeof(K), 16);
    const size_t sweep_smem = Cfg::smem_bytes(bins, false, tb);
    const size_t census_smem = align_up((size_t)bins * 4 + align_up((size_t)B, 4) * 4, 16) + tb;
    if (sweep_smem > max_smem_optin() || census_smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    int per_sm = 0;
    {
        auto kern = k_downsweep<K, true, 512, 8, 0, BucketDigit<K>>;
        ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_smem));
        ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, sweep_smem));
        if (per_sm < 1) return ISORT_ERR_UNSUPPORTED;
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
    const size_t o_status = take(64), o_fix = take(64);
    const size_t o_sample = take((size_t)m * sizeof(K)), o_u = take((size_t)m * 4);
    const size_t o_theta = take(2 * kPwlSegments * 4), o_adam = take(4 * kPwlSegments * 4);
    const size_t o_best = take((2 * kPwlSegments + 1) * 4);
    const size_t o_X = take(kPwlKnots * 4), o_Y = take(kPwlKnots * 4);
    const size_t o_part = take((size_t)kGradCtas * kPartial * 4), o_loss = take((kTrainSteps + 2) * 4);
    const size_t o_split = take((size_t)B * sizeof(K)), o_bcount = take((size_t)B * 4);
    const size_t o_hist = take((size_t)chunks * bins * 4), o_coff = take((size_t)chunks * bins * 4);
    const size_t o_segoff = take((size_t)(B + 1) * 8), o_seglo = take((size_t)B * 4), o_segbits = take((size_t)B);
    const size_t o_buf = take(n * sizeof(K) + (hv ? align_up(n * 4, 256) : 0));
    unsigned char* ws = nullptr;
    isort_status st = scratch_alloc((void**)&ws, off, s);
    if (st != ISORT_OK) return st;
    auto fail = [&](isort_status e) {
        scratch_free(ws, s);
        return e;
    };
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + o_status);
    unsigned long long* fixups = reinterpret_cast<unsigned long long*>(ws + o_fix);
    K* sample = reinterpret_cast<K*>(ws + o_sample);
    ModelBufs mb;
    mb.u = reinterpret_cast<float*>(ws + o_u);
    mb.theta = reinterpret_cast<float*>(ws + o_theta);
    mb.adam = reinterpret_cast<float*>(ws + o_adam);
    mb.best = reinterpret_cast<float*>(ws + o_best);
    mb.X = reinterpret_cast<float*>(ws + o_X);
    mb.Y = reinterpret_cast<float*>(ws + o_Y);
    mb.partial = reinterpret_cast<float*>(ws + o_part);
    mb.losses = reinterpret_cast<float*>(ws + o_loss);
    K* split = reinterpret_cast<K*>(ws + o_split);
    uint32_t* bcount = reinterpret_cast<uint32_t*>(ws + o_bcount);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + o_hist);
    uint32_t* coff = reinterpret_cast<uint32_t*>(ws + o_coff);
    uint64_t* segoff = reinterpret_cast<uint64_t*>(ws + o_segoff);
    uint32_t* seglo = reinterpret_cast<uint32_t*>(ws + o_seglo);
    uint8_t* segbits = reinterpret_cast<uint8_t*>(ws + o_segbits);
    K* wk = reinterpret_cast<K*>(ws + o_buf);
    uint32_t* wv = hv ? reinterpret_cast<uint32_t*>(ws + o_buf + align_up(n * sizeof(K), 256)) : nullptr;

    cudaError_t ce = cudaMemsetAsync(ws, 0, 128, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(bcount, 0, (size_t)B * 4, s);
    if (ce != cudaSuccess) return fail(from_cuda(ce));

    // 1. sample and sort it
    {
        LaunchScope ls("sample_gather", s);
        k_sample_gather<K><<<(m + 255) / 256, 256, 0, s>>>(keys, (uint64_t)n, m, sample);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    if constexpr (sizeof(K) == 4) st = radix_sort_u32_device(sample, nullptr, sample, nullptr, m, key_bits, 8, s);
    else st = ISORT_ERR_UNSUPPORTED;
    if (st != ISORT_OK) return fail(st);

    // 2. train the model
    {
        LaunchScope ls("cdf_init", s);
        k_normalise<K><<<(m + 255) / 256, 256, 0, s>>>(sample, m, scale, mb.u);
        k_model_init<K><<<1, kPwlSegments, 0, s>>>(sample, m, scale, mb.theta, mb.X, mb.Y, mb.adam);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    // the loss before training
    st = launch_grad_step(mb, m, kTrainSteps + 1, 0.f, nullptr, kStepPlain, s);
    if (st != ISORT_OK) return fail(st);
    st = train_model(mb, m, kTrainSteps, s);
    if (st != ISORT_OK) return fail(st);

    // 3. splitters
    {
        LaunchScope ls("splitters", s);
        k_splitters<K><<<(B + 255) / 256, 256, 0, s>>>(mb.X, mb.Y, B, key_bits, scale, split);
        k_splitters_monotone<K><<<1, 32, 0, s>>>(split, B);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    BucketDigit<K> df;
    df.g_split = split;
    df.g_X = mb.X;
    df.g_Y = mb.Y;
    df.B = B;
    df.scale = scale;
    df.sub_shift = 0;
    df.sub_mask = (uint32_t)bins - 1u;

    // 4. census
    {
        const size_t smem = census_smem;
        ce = cudaFuncSetAttribute(k_bucket_census<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ce != cudaSuccess) return fail(from_cuda(ce));
        LaunchScope ls("bucket_census", s);
        k_bucket_census<K><<<chunks, kCensusThreads, smem, s>>>(keys, (uint32_t)n, chunk_tiles * tile, df, hist, bcount,
                                                              fixups, key_bits, status);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    std::vector<uint32_t> h_count(B);
    std::vector<K> h_split(B);
    std::vector<float> h_loss(kTrainSteps + 2);
    unsigned long long h_fix = 0;
    uint32_t h_status = 0;
    ce = cudaMemcpyAsync(h_count.data(), bcount, (size_t)B * 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_split.data(), split, (size_t)B * sizeof(K), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_loss.data(), mb.losses, (kTrainSteps + 2) * 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_fix, fixups, 8, cudaMemcpyDeviceToHost, s);
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
    stats->fixups = h_fix;
    stats->train_loss = h_loss[kTrainSteps];
    stats->train_loss_initial = h_loss[kTrainSteps + 1];
    stats->train_steps = kTrainSteps;
    stats->nbuckets = B;
    if (stats->overflow_fraction > 0.5) {
        stats->fell_back_to_lsd = 1;
        st = radix_sort_u32_device(reinterpret_cast<uint32_t*>(keys), vals, reinterpret_cast<uint32_t*>(keys), vals, n,
                                   key_bits, 8, s);
        scratch_free(ws, s);
        return st;
    }

    // 5. stable distribution by bucket id (LSD over its halves)
    K* src_k = keys;
    uint32_t* src_v = vals;
    for (int p = 0; p < passes; ++p) {
        const bool to_buf = (p % 2) == 0;
        K* dk = to_buf ? wk : keys;
        uint32_t* dv = to_buf ? wv : vals;
        df.sub_shift = p * wsub;
        df.sub_mask = (uint32_t)((1 << std::min(wsub, id_bits - p * wsub)) - 1);
        const int pbins = (int)df.sub_mask + 1;
        if (p > 0) {
            const size_t smem = align_up((size_t)pbins * 4, 16) + tb;
            ce = cudaFuncSetAttribute(k_bucket_hist<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (ce != cudaSuccess) return fail(from_cuda(ce));
            LaunchScope ls("bucket_hist", s);
            k_bucket_hist<K><<<chunks, kCensusThreads, smem, s>>>(src_k, (uint32_t)n, chunk_tiles * tile, df, hist);
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
        st = launch_bucket_sweep<K>(a, df, chunks, hv, s);
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
    std::vector<uint32_t> h_lo(B);
    std::vector<uint8_t> h_bits(B);
    std::vector<int> big;
    h_off[0] = 0;
    const uint64_t kmax = key_bits >= 64 ? ~0ull : ((1ull << key_bits) - 1ull);
    for (int b = 0; b < B; ++b) {
        h_off[b + 1] = h_off[b] + h_count[b];
        const uint64_t lo = b == 0 ? 0 : (uint64_t)h_split[b];
        const uint64_t hi_incl = b + 1 < B ? (uint64_t)h_split[b + 1] - (h_split[b + 1] > 0 ? 1 : 0) : kmax;
        h_lo[b] = (uint32_t)lo;
        const uint64_t span = hi_incl >= lo ? hi_incl - lo : 0;
        h_bits[b] = (uint8_t)bit_length(span);
        if (h_count[b] > kOnChipCapacity && h_bits[b] > 0) {
            big.push_back(b);
            h_bits[b] = 0;  // not a segment of the on-chip finish
        }
    }
    ce = cudaMemcpyAsync(segoff, h_off.data(), (size_t)(B + 1) * 8, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(seglo, h_lo.data(), (size_t)B * 4, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(segbits, h_bits.data(), (size_t)B, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return fail(from_cuda(ce));
    if constexpr (sizeof(K) == 4) {
        st = segmented_finish_u32(reinterpret_cast<uint32_t*>(keys), vals, segoff, (uint32_t)B, seglo, segbits, s);
        for (size_t i = 0; i < big.size() && st == ISORT_OK; ++i) {
            const int b = big[i];
            uint32_t* k = reinterpret_cast<uint32_t*>(keys) + h_off[b];
            uint32_t* v = hv ? vals + h_off[b] : nullptr;
            st = radix_sort_u32_device(k, v, k, v, h_count[b], key_bits, 8, s);
        }
    } else {
        st = ISORT_ERR_UNSUPPORTED;
    }
    if (st != ISORT_OK) return fail(st);
    st = finish_status(status, s);
    scratch_free(ws, s);
    return st;
}

}  // namespace
}  // namespace isort

using namespace isort;

extern "C" {

isort_status isort_learned(uint32_t* keys, uint32_t* vals, size_t n, int key_bits, int nbuckets, int model,
                           isort_learned_stats* stats, void* stream) {
    isort_learned_stats local;
    isort_learned_stats* st = stats ? stats : &local;
    std::memset(st, 0, sizeof(*st));
    if (key_bits == 0) key_bits = 32;
    if (key_bits < 1 || key_bits > 32) return ISORT_ERR_INVALID_ARG;
    if (nbuckets == 0) nbuckets = 4096;
    if (nbuckets < 2 || nbuckets > kMaxBuckets) return ISORT_ERR_INVALID_ARG;
    if (model != 0 && model != 1) return ISORT_ERR_INVALID_ARG;
    if (model == 1) return ISORT_ERR_UNSUPPORTED;
    if (n >= (size_t(1) << 30)) return ISORT_ERR_UNSUPPORTED;
    if (n > 1 && !keys) return ISORT_ERR_INVALID_ARG;
    if (n <= 1) return ISORT_OK;
    if (is_host_pointer(keys) || (vals && is_host_pointer(vals))) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n < (size_t)4 * kSampleSize) {
        // too few keys for a sample to pay off: the plain rounds
        st->fell_back_to_lsd = 1;
        return radix_sort_u32_device(keys, vals, keys, vals, n, key_bits, 8, s);
    }
    return learned_device<uint32_t>(keys, vals, n, key_bits, nbuckets, st, s);
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
        k_splitters_monotone<uint32_t><<<1, 32, 0, s>>>(static_cast<uint32_t*>(splitters), nbuckets);
    } else {
        k_splitters<uint64_t><<<(nbuckets + 255) / 256, 256, 0, s>>>(X, Y, nbuckets, key_bits, scale,
                                                                     static_cast<uint64_t*>(splitters));
        k_splitters_monotone<uint64_t><<<1, 32, 0, s>>>(static_cast<uint64_t*>(splitters), nbuckets);
    }
    ISORT_TRY_CUDA(cudaGetLastError());
    if (sync_mode()) ISORT_TRY_CUDA(cudaStreamSynchronize(s));
    return ISORT_OK;
}

isort_status isort_bucket_ids(const void* keys, int key_width, size_t n, int key_bits, const float* X, const float* Y,
                              const void* splitters, int nbuckets, uint32_t* ids, void* stream) {
    if (key_width != 32 && key_width != 64) return ISORT_ERR_INVALID_ARG;
    if (key_bits == 0) key_bits = key_width;
    if (key_bits < 1 || key_bits > key_width || nbuckets < 2 || nbuckets > kMaxBuckets) return ISORT_ERR_INVALID_ARG;
    if (n == 0) return ISORT_OK;
    if (!keys || !X || !Y || !splitters || !ids || n >= (size_t(1) << 32)) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float scale = std::ldexp(1.0f, -key_bits);
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 8);
    LaunchScope ls("bucket_ids", s);
    if (key_width == 32) {
        BucketDigit<uint32_t> df{static_cast<const uint32_t*>(splitters), X, Y, nbuckets, scale, 0, 0xffffu,
                                 nullptr, nullptr, nullptr};
        const size_t smem = 2 * align_up(kPwlKnots * 4, 16) + align_up((size_t)nbuckets * 4, 16);
        ISORT_TRY_CUDA(cudaFuncSetAttribute(k_bucket_ids<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
        k_bucket_ids<uint32_t><<<grid, 256, smem, s>>>(static_cast<const uint32_t*>(keys), (uint32_t)n, df, ids);
    } else {
        BucketDigit<uint64_t> df{static_cast<const uint64_t*>(splitters), X, Y, nbuckets, scale, 0, 0xffffu,
                                 nullptr, nullptr, nullptr};
        const size_t smem = 2 * align_up(kPwlKnots * 4, 16) + align_up((size_t)nbuckets * 8, 16);
        ISORT_TRY_CUDA(cudaFuncSetAttribute(k_bucket_ids<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
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
    float* buf = nullptr;
    // theta copy, adam, X, Y, partials
    const size_t floats = 2 * kPwlSegments + 4 * kPwlSegments + 2 * kPwlKnots + (size_t)kGradCtas * kPartial;
    isort_status st = scratch_alloc((void**)&buf, floats * 4, s);
    if (st != ISORT_OK) return st;
    ModelBufs mb;
    mb.u = const_cast<float*>(u);
    mb.theta = buf;
    mb.adam = buf + 2 * kPwlSegments;
    mb.X = mb.adam + 4 * kPwlSegments;
    mb.Y = mb.X + kPwlKnots;
    mb.partial = mb.Y + kPwlKnots;
    mb.best = nullptr;
    mb.losses = loss;  // loss_out[0]
    cudaError_t ce = cudaMemcpyAsync(mb.theta, theta, 2 * kPwlSegments * 4, cudaMemcpyDeviceToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(mb.adam, 0, 4 * kPwlSegments * 4, s);
    if (ce != cudaSuccess) {
        scratch_free(buf, s);
        return from_cuda(ce);
    }
    {
        LaunchScope ls("cdf_derive", s);
        k_model_derive<<<1, kPwlSegments, 0, s>>>(mb.theta, mb.X, mb.Y);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) st = launch_grad_step(mb, m, 0, 0.f, grad, kStepPlain, s);
    else st = from_cuda(ce);
    scratch_free(buf, s);
    if (st == ISORT_OK && sync_mode()) st = from_cuda(cudaStreamSynchronize(s));
    return st;
}

isort_status isort_cdf_train(const uint32_t* sorted_sample, uint32_t m, int key_bits, float* theta, float* X,
                             float* Y, float* losses, void* stream) {
    if (!sorted_sample || !theta || !X || !Y || !losses || m < 2) return ISORT_ERR_INVALID_ARG;
    if (key_bits == 0) key_bits = 32;
    if (key_bits < 1 || key_bits > 32) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float* buf = nullptr;
    const size_t floats = (size_t)m + 4 * kPwlSegments + (size_t)kGradCtas * kPartial + 2 * kPwlSegments + 1;
    isort_status st = scratch_alloc((void**)&buf, floats * 4, s);
    if (st != ISORT_OK) return st;
    ModelBufs mb;
    mb.u = buf;
    mb.adam = buf + m;
    mb.partial = mb.adam + 4 * kPwlSegments;
    mb.best = mb.partial + (size_t)kGradCtas * kPartial;
    mb.theta = theta;
    mb.X = X;
    mb.Y = Y;
    mb.losses = losses;  // [kTrainSteps + 2]: per step, then the initial loss last
    const float scale = std::ldexp(1.0f, -key_bits);
    {
        LaunchScope ls("cdf_init", s);
        k_normalise<uint32_t><<<(m + 255) / 256, 256, 0, s>>>(sorted_sample, m, scale, mb.u);
        k_model_init<uint32_t><<<1, kPwlSegments, 0, s>>>(sorted_sample, m, scale, mb.theta, mb.X, mb.Y, mb.adam);
        st = from_cuda(cudaGetLastError());
    }
    if (st == ISORT_OK) st = launch_grad_step(mb, m, kTrainSteps + 1, 0.f, nullptr, kStepPlain, s);
    if (st == ISORT_OK) st = train_model(mb, m, kTrainSteps, s);
    scratch_free(buf, s);
    if (st == ISORT_OK && sync_mode()) st = from_cuda(cudaStreamSynchronize(s));
    return st;
}

}  // extern "C"
