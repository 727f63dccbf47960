// Device code of the paper's block networks (Gerbessiotis, arXiv:1708.09495,
// Section 2; Section 3 eqs. Tb and To), shared by the one-array kernels and the
// segmented router.
//
// Items are 64-bit composites (key << 32 | original index); comparing them
// compares (key, index), so merge-split networks, which are not stable by
// themselves, produce the unique stable order. Thread t holds block t: B
// consecutive items in registers.
//
// Merge-split of two ascending blocks X (this thread) and Y (partner) without
// a serial merge: Z[i] = min(X[i], Y[B-1-i]) is exactly the B smallest items of
// X u Y and forms a bitonic sequence (the first half-cleaner of the bitonic
// sequence X ++ reverse(Y)); max() gives the B largest. A log2(B)-stage
// bitonic merge in registers then sorts Z. The partner's items are fetched one
// at a time (warp shuffle when the partner is in the same warp, shared memory
// otherwise), so a thread never holds two blocks.
#pragma once

#include "common.cuh"

namespace isort {
namespace net {

constexpr uint64_t kPadHi = 0xFFFFFFFFull << 32;

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a < b ? b : a; }

// The networks below work on 64-bit items (key << 32 | index) or on packed
// 32-bit items; T is the item type.
template <typename T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a < b ? b : a; }

template <int B, typename T = uint64_t>
__device__ __forceinline__ void cswap(T (&x)[B], int i, int l, bool asc) {
    const T a = x[i], b = x[l];
    const T lo = tmin(a, b), hi = tmax(a, b);
    x[i] = asc ? lo : hi;
    x[l] = asc ? hi : lo;
}

// Local sort of a block (a register bitonic sorting network, ascending).
template <int B, typename T = uint64_t>
__device__ __forceinline__ void local_sort(T (&x)[B]) {
#pragma unroll
    for (int k = 2; k <= B; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < B; ++i) {
                const int l = i ^ j;
                if (l > i) cswap<B, T>(x, i, l, (i & k) == 0);
            }
}

// Sorts a bitonic block ascending.
template <int B, typename T = uint64_t>
__device__ __forceinline__ void bitonic_merge(T (&x)[B]) {
#pragma unroll
    for (int j = B >> 1; j > 0; j >>= 1)
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int l = i ^ j;
            if (l > i) cswap<B, T>(x, i, l, true);
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
template <int B, bool WARP_ONLY = false>
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
    if constexpr (WARP_ONLY) __syncwarp();
    else __syncthreads();
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
template <int B, typename T = uint64_t>
__device__ __forceinline__ void merge_split_shfl(T (&x)[B], int j, bool keep_small) {
    if constexpr (B == 1) {
        const T y = __shfl_xor_sync(kFullMask, x[0], j);
        x[0] = keep_small ? tmin(x[0], y) : tmax(x[0], y);
    } else {
#pragma unroll
        for (int i = 0; i < B / 2; ++i) {
            const T a = x[i], b = x[B - 1 - i];
            const T ya = __shfl_xor_sync(kFullMask, b, j);  // partner's item B-1-i
            const T yb = __shfl_xor_sync(kFullMask, a, j);  // partner's item i
            x[i] = keep_small ? tmin(a, ya) : tmax(a, ya);
            x[B - 1 - i] = keep_small ? tmin(b, yb) : tmax(b, yb);
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

// BTN over the CTA: p (a power of two) blocks held by threads 0..p-1 (the
// other threads hold pads); lg p (lg p + 1)/2 merge-split stages. s_x holds
// B * blockDim.x items when p > 32. Every thread of the CTA must call it.
// Keys with a bit of range_mask set are out of range: the call then records
// kStatKeyRange in *status and leaves the keys unchanged (range_mask 0: no
// check).
template <int B>
__device__ __forceinline__ uint32_t block_or(const uint64_t (&x)[B], uint32_t n, int t) {
    uint32_t o = 0;
#pragma unroll
    for (int i = 0; i < B; ++i)
        if ((uint32_t)t * B + i < n) o |= (uint32_t)(x[i] >> 32);
    return o;
}

template <int B>
__device__ __forceinline__ void btn_block(uint32_t* keys, uint32_t* vals, uint32_t n, int p, uint64_t* s_x,
                                          unsigned long long* stage_ctr, uint32_t range_mask = 0,
                                          uint32_t* status = nullptr) {
    const int t = threadIdx.x;
    const int P = blockDim.x;
    uint64_t x[B];
    load_block<B>(x, keys, n, t);
    if (range_mask && __syncthreads_or((block_or<B>(x, n, t) & range_mask) != 0)) {
        if (t == 0) set_status(status, kStatKeyRange);
        return;
    }
    local_sort<B>(x);
    for (int k = 2; k <= p; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int partner = t ^ j;
            const bool asc = (t & k) == 0;
            const bool lower = t < partner;
            const bool keep_small = lower == asc;
            if (j < 32) merge_split_shfl<B>(x, j, keep_small);
            else merge_split_smem<B>(x, s_x, P, t, partner, true, keep_small);
            bitonic_merge<B>(x);
            if (stage_ctr && t == 0) atomicAdd(stage_ctr, 1ull);
        }
    }
    store_block<B>(x, keys, vals, n, t, t < p);
}

// BTN inside one warp (p <= 32 blocks, lane = block); shuffles only.
template <int B>
__device__ __forceinline__ void btn_warp(uint32_t* keys, uint32_t* vals, uint32_t n, int p, uint32_t range_mask = 0,
                                         uint32_t* status = nullptr) {
    const int t = threadIdx.x & 31;
    uint64_t x[B];
    load_block<B>(x, keys, n, t);
    if (range_mask && __any_sync(kFullMask, (block_or<B>(x, n, t) & range_mask) != 0)) {
        if (t == 0) set_status(status, kStatKeyRange);
        return;
    }
    local_sort<B>(x);
    for (int k = 2; k <= p; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const bool asc = (t & k) == 0;
            const bool lower = t < (t ^ j);
            merge_split_shfl<B>(x, j, lower == asc);
            bitonic_merge<B>(x);
        }
    }
    store_block<B, true>(x, keys, vals, n, t, t < p);
}

// OET over the CTA: p blocks (any p <= blockDim.x), p rounds; round r pairs
// blocks (j, j+1) with j = r mod 2 and the lower block keeps the smaller half.
// Exchanges go through shared memory (s_x: B * blockDim.x items).
template <int B>
__device__ __forceinline__ void oet_block(uint32_t* keys, uint32_t* vals, uint32_t n, int p, uint64_t* s_x,
                                          unsigned long long* stage_ctr) {
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

// OET inside one warp with one key per lane (n <= 32): n rounds of
// compare-exchange between neighbouring lanes (blocks of one key).
__device__ __forceinline__ void oet_warp1(uint32_t* keys, uint32_t* vals, uint32_t n, uint32_t range_mask = 0,
                                          uint32_t* status = nullptr) {
    const int t = threadIdx.x & 31;
    uint64_t x[1];
    load_block<1>(x, keys, n, t);
    if (range_mask && __any_sync(kFullMask, (block_or<1>(x, n, t) & range_mask) != 0)) {
        if (t == 0) set_status(status, kStatKeyRange);
        return;
    }
    for (uint32_t r = 0; r < n; ++r) {
        const bool lower = ((t - (int)r) & 1) == 0;
        const int partner = lower ? t + 1 : t - 1;
        const uint64_t y = __shfl_sync(kFullMask, x[0], partner & 31);
        const bool exchange = partner >= 0 && partner < 32;
        if (exchange) x[0] = lower ? umin64(x[0], y) : umax64(x[0], y);
    }
    store_block<1, true>(x, keys, vals, n, t, (uint32_t)t < n);
}

}  // namespace net
}  // namespace isort
