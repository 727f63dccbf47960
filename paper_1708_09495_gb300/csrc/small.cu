// BTN and OET: the paper's small-n block networks (Gerbessiotis,
// arXiv:1708.09495, Section 2; Section 3 "Bitonic Sort" eq. Tb and "Odd-even
// transposition sort" eq. To).
//
// p "processors" are p threads of one CTA. Thread t holds block t: B
// consecutive items of the (padded) input in registers, as 64-bit composites
// (key << 32 | original index). Comparing composites compares (key, index), so
// the networks' result is the unique stable order even though merge-split
// networks are not stable by themselves.
//
// Merge-split of two ascending blocks X (this thread) and Y (partner) without
// a serial merge: Z[i] = min(X[i], Y[B-1-i]) is exactly the B smallest items of
// X u Y and forms a bitonic sequence (the first half-cleaner of the bitonic
// sequence X ++ reverse(Y)); max() gives the B largest. A log2(B)-stage
// bitonic merge in registers then sorts Z. The partner's items are fetched one
// at a time (warp shuffle when the partner is in the same warp, shared memory
// otherwise), so a thread never holds two blocks.
#include <algorithm>

#include "common.cuh"
#include "runtime.h"

namespace isort {
namespace {

constexpr uint64_t kPadHi = 0xFFFFFFFFull << 32;

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a < b ? b : a; }

template <int B>
__device__ __forceinline__ void cswap(uint64_t (&x)[B], int i, int l, bool asc) {
    const uint64_t a = x[i], b = x[l];
    const bool sw = asc ? (a > b) : (a < b);
    x[i] = sw ? b : a;
    x[l] = sw ? a : b;
}

// Local sort of a block (a register bitonic sorting network, ascending).
template <int B>
__device__ __forceinline__ void local_sort(uint64_t (&x)[B]) {
#pragma unroll
    for (int k = 2; k <= B; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < B; ++i) {
                const int l = i ^ j;
                if (l > i) cswap<B>(x, i, l, (i & k) == 0);
            }
}

// Sorts a bitonic block ascending.
template <int B>
__device__ __forceinline__ void bitonic_merge(uint64_t (&x)[B]) {
#pragma unroll
    for (int j = B >> 1; j > 0; j >>= 1)
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int l = i ^ j;
            if (l > i) cswap<B>(x, i, l, true);
        }
}

template <int B>
__device__ __forceinline__ void load_block(uint64_t (&x)[B], const uint32_t* keys, uint32_t n, int t) {
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const uint32_t g = (uint32_t)t * B + i;
        x[i] = g < n ? (((uint64_t)keys[g] << 32) | g) : (kPadHi | g);
    }
}

// Writes the first n items of the sorted sequence; payloads are gathered by
// original index. All reads of the inputs finish before any write (in place).
template <int B>
__device__ __forceinline__ void store_block(const uint64_t (&x)[B], uint32_t* keys, uint32_t* vals, uint32_t n,
                                            int t, bool active) {
    uint32_t v[B];
    if (vals && active) {
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const uint32_t g = (uint32_t)t * B + i;
            v[i] = g < n ? vals[(uint32_t)x[i]] : 0u;
        }
    }
    __syncthreads();
    if (!active) return;
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const uint32_t g = (uint32_t)t * B + i;
        if (g < n) {
            keys[g] = (uint32_t)(x[i] >> 32);
            if (vals) vals[g] = v[i];
        }
    }
}

// Half-cleaner against the partner lane (t ^ j) of the same warp. Slots i and
// B-1-i are exchanged together so that only original values are sent.
template <int B>
__device__ __forceinline__ void merge_split_shfl(uint64_t (&x)[B], int j, bool keep_small) {
    if constexpr (B == 1) {
        const uint64_t y = __shfl_xor_sync(kFullMask, x[0], j);
        x[0] = keep_small ? umin64(x[0], y) : umax64(x[0], y);
    } else {
#pragma unroll
        for (int i = 0; i < B / 2; ++i) {
            const uint64_t a = x[i], b = x[B - 1 - i];
            const uint64_t ya = __shfl_xor_sync(kFullMask, b, j);  // partner's item B-1-i
            const uint64_t yb = __shfl_xor_sync(kFullMask, a, j);  // partner's item i
            x[i] = keep_small ? umin64(a, ya) : umax64(a, ya);
            x[B - 1 - i] = keep_small ? umin64(b, yb) : umax64(b, yb);
        }
    }
}

// Half-cleaner against block `partner` through shared memory.
template <int B>
__device__ __forceinline__ void merge_split_smem(uint64_t (&x)[B], uint64_t* s_x, int P, int t, int partner,
                                                 bool exchange, bool keep_small) {
#pragma unroll
    for (int i = 0; i < B; ++i) s_x[i * P + t] = x[i];
    __syncthreads();
    if (exchange) {
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const uint64_t y = s_x[(B - 1 - i) * P + partner];
            x[i] = keep_small ? umin64(x[i], y) : umax64(x[i], y);
        }
    }
    __syncthreads();
}

// BTN: p (a power of two) threads; lg p (lg p + 1)/2 merge-split stages.
template <int B>
__global__ void k_btn(uint32_t* keys, uint32_t* vals, uint32_t n, int p, unsigned long long* stage_ctr) {
    extern __shared__ __align__(16) uint64_t s_x[];  // [B][blockDim] when a stage crosses warps
    const int t = threadIdx.x;
    const int P = blockDim.x;
    const bool active = t < p;
    uint64_t x[B];
    load_block<B>(x, keys, n, t);  // threads >= p hold pads only
    local_sort<B>(x);
    for (int k = 2; k <= p; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int partner = t ^ j;
            const bool asc = (t & k) == 0;
            const bool lower = t < partner;
            const bool keep_small = lower == asc;
            if (j < 32) {
                merge_split_shfl<B>(x, j, keep_small);
            } else {
                merge_split_smem<B>(x, s_x, P, t, partner, true, keep_small);
            }
            bitonic_merge<B>(x);
            if (stage_ctr && t == 0) atomicAdd(stage_ctr, 1ull);
        }
    }
    store_block<B>(x, keys, vals, n, t, active);
}

// OET: p threads (any p); p rounds; round r pairs blocks (j, j+1) with
// j = r mod 2, the lower block keeping the smaller half. Exchanges go through
// shared memory.
template <int B>
__global__ void k_oet(uint32_t* keys, uint32_t* vals, uint32_t n, int p, unsigned long long* stage_ctr) {
    extern __shared__ __align__(16) uint64_t s_x[];
    const int t = threadIdx.x;
    const int P = blockDim.x;
    const bool active = t < p;
    uint64_t x[B];
    load_block<B>(x, keys, n, t);
    local_sort<B>(x);
    for (int r = 0; r < p; ++r) {
        const bool lower = ((t - r) & 1) == 0;  // t = j with j = r mod 2
        const int partner = lower ? t + 1 : t - 1;
        const bool exchange = active && partner >= 0 && partner < p;
        merge_split_smem<B>(x, s_x, P, t, partner, exchange, lower);
        if (exchange) bitonic_merge<B>(x);
        if (stage_ctr && t == 0) atomicAdd(stage_ctr, 1ull);
    }
    store_block<B>(x, keys, vals, n, t, active);
}

int next_pow2(uint32_t v) {
    int p = 1;
    while ((uint32_t)p < v) p <<= 1;
    return p;
}

enum class Net { Btn, Oet };

template <int B>
isort_status launch_net(Net net, uint32_t* keys, uint32_t* vals, uint32_t n, int p, unsigned long long* ctr,
                        cudaStream_t s) {
    const int threads = std::max(32, (p + 31) / 32 * 32);
    // shared memory is needed by OET always and by BTN once partners cross warps
    const size_t smem = (net == Net::Oet || p > 32) ? (size_t)B * threads * 8 : 0;
    if (smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    cudaFuncAttributes fa;
    ISORT_TRY_CUDA(cudaFuncGetAttributes(&fa, net == Net::Btn ? (const void*)k_btn<B> : (const void*)k_oet<B>));
    if (threads > fa.maxThreadsPerBlock) return ISORT_ERR_UNSUPPORTED;
    if (net == Net::Btn) {
        ISORT_TRY_CUDA(cudaFuncSetAttribute(k_btn<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        LaunchScope ls("btn", s);
        k_btn<B><<<1, threads, smem, s>>>(keys, vals, n, p, ctr);
    } else {
        ISORT_TRY_CUDA(cudaFuncSetAttribute(k_oet<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        LaunchScope ls("oet", s);
        k_oet<B><<<1, threads, smem, s>>>(keys, vals, n, p, ctr);
    }
    return from_cuda(cudaGetLastError());
}

constexpr uint32_t kNetMaxN = 16384;

// Sorts device buffers with the chosen network on p blocks.
isort_status net_device(Net net, uint32_t* keys, uint32_t* vals, uint32_t n, int p, uint64_t* stages, cudaStream_t s) {
    const uint32_t per = (n + (uint32_t)p - 1) / (uint32_t)p;
    const int B = next_pow2(std::max<uint32_t>(per, 1));
    if (B > 32 || (size_t)B * p > kNetMaxN * 2) return ISORT_ERR_UNSUPPORTED;
    unsigned long long* ctr = nullptr;
    if (stages) {
        isort_status st = scratch_alloc((void**)&ctr, 8, s);
        if (st != ISORT_OK) return st;
        cudaError_t ce = cudaMemsetAsync(ctr, 0, 8, s);
        if (ce != cudaSuccess) {
            scratch_free(ctr, s);
            return from_cuda(ce);
        }
    }
    isort_status st;
    switch (B) {
        case 1: st = launch_net<1>(net, keys, vals, n, p, ctr, s); break;
        case 2: st = launch_net<2>(net, keys, vals, n, p, ctr, s); break;
        case 4: st = launch_net<4>(net, keys, vals, n, p, ctr, s); break;
        case 8: st = launch_net<8>(net, keys, vals, n, p, ctr, s); break;
        case 16: st = launch_net<16>(net, keys, vals, n, p, ctr, s); break;
        default: st = launch_net<32>(net, keys, vals, n, p, ctr, s); break;
    }
    if (stages) {
        if (st == ISORT_OK) {
            unsigned long long h = 0;
            cudaError_t ce = cudaMemcpyAsync(&h, ctr, 8, cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) st = from_cuda(ce);
            *stages = h;
        }
        scratch_free(ctr, s);
    } else if (st == ISORT_OK && sync_mode()) {
        st = from_cuda(cudaStreamSynchronize(s));
    }
    return st;
}

isort_status net_entry(Net net, uint32_t* keys, uint32_t* vals, size_t n, int p, uint64_t* stages, void* stream) {
    if (net == Net::Btn && (p < 1 || p > 1024 || (p & (p - 1)) != 0)) return ISORT_ERR_INVALID_ARG;
    if (net == Net::Oet && (p < 1 || p > 1024)) return ISORT_ERR_INVALID_ARG;
    if (n > (size_t)32 * p || n > kNetMaxN) return ISORT_ERR_UNSUPPORTED;
    if (n > 1 && !keys) return ISORT_ERR_INVALID_ARG;
    if (stages) *stages = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return ISORT_OK;
    const bool host = is_host_pointer(keys) || (vals && is_host_pointer(vals));
    if (!host) return net_device(net, keys, vals, (uint32_t)n, p, stages, s);
    unsigned char* buf = nullptr;
    const size_t kb = align_up(n * 4, 256);
    isort_status st = scratch_alloc((void**)&buf, kb + (vals ? kb : 0), s);
    if (st != ISORT_OK) return st;
    uint32_t* dk = reinterpret_cast<uint32_t*>(buf);
    uint32_t* dv = vals ? reinterpret_cast<uint32_t*>(buf + kb) : nullptr;
    cudaError_t ce = cudaMemcpyAsync(dk, keys, n * 4, cudaMemcpyDefault, s);
    if (ce == cudaSuccess && vals) ce = cudaMemcpyAsync(dv, vals, n * 4, cudaMemcpyDefault, s);
    st = ce == cudaSuccess ? net_device(net, dk, dv, (uint32_t)n, p, stages, s) : from_cuda(ce);
    if (st == ISORT_OK) {
        ce = cudaMemcpyAsync(keys, dk, n * 4, cudaMemcpyDefault, s);
        if (ce == cudaSuccess && vals) ce = cudaMemcpyAsync(vals, dv, n * 4, cudaMemcpyDefault, s);
        if (ce != cudaSuccess) st = from_cuda(ce);
    }
    scratch_free(buf, s);
    cudaError_t se = cudaStreamSynchronize(s);
    if (st == ISORT_OK && se != cudaSuccess) st = from_cuda(se);
    return st;
}

// Default p: 8 keys per block up to 4096 keys, then 16.
int default_p(size_t n) {
    const uint32_t per = n <= 4096 ? 8u : 16u;
    int p = next_pow2((uint32_t)std::max<size_t>(1, (n + per - 1) / per));
    return std::min(p, 1024);
}

}  // namespace
}  // namespace isort

using namespace isort;

extern "C" {

isort_status isort_btn(uint32_t* keys, uint32_t* vals, size_t n, void* stream) {
    return net_entry(Net::Btn, keys, vals, n, default_p(n), nullptr, stream);
}

isort_status isort_oet(uint32_t* keys, uint32_t* vals, size_t n, void* stream) {
    return net_entry(Net::Oet, keys, vals, n, default_p(n), nullptr, stream);
}

isort_status isort_btn_p(uint32_t* keys, uint32_t* vals, size_t n, int p, uint64_t* stages, void* stream) {
    return net_entry(Net::Btn, keys, vals, n, p, stages, stream);
}

isort_status isort_oet_p(uint32_t* keys, uint32_t* vals, size_t n, int p, uint64_t* stages, void* stream) {
    return net_entry(Net::Oet, keys, vals, n, p, stages, stream);
}

}  // extern "C"
