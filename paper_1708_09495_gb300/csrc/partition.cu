// Sample-sort steps for sorting across several processors: drawing a sample
// of the keys, and the stable routing of every key to the range of splitters
// chosen regularly from a sorted sample (Section 2, the sample sorts with
// regular sampling; the routing is Section 3's count-sort round with the
// key's range as its digit, the key exchange of eq. Tp). A sort over p
// processes draws a sample on each, gathers and sorts the samples, partitions
// its keys with isort_partition, exchanges the ranges and sorts what it
// receives.
//
// The partition runs as one chunked count-sort round (sweep.cuh): per-chunk
// range counts, chunk offsets, then the rank-and-scatter kernel with the range
// as its digit (the p - 1 splitters sit in shared memory; a key's range is
// found by bisection).
#include <algorithm>

#include "common.cuh"
#include "runtime.h"
#include "sweep.cuh"

namespace isort {

namespace {

constexpr int kMaxParts = 256;

// m sample keys: key at index floor(r_j n / 2^64), r_j = SplitMix64 output j
// from state seed.
template <typename K>
__global__ void k_sample(const K* __restrict__ keys, uint64_t n, uint32_t m, uint64_t seed, K* __restrict__ out) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const uint64_t r = splitmix_mix(seed + (uint64_t)(j + 1) * kSplitmixGamma);
    out[j] = keys[__umul64hi(r, n)];
}

// Digit = the key's range: the number of splitters <= key, splitter j (1 <= j
// < parts) being sorted_sample[floor(j m / parts)].
template <typename K>
struct RangeDigit {
    static constexpr bool kCheap = false;
    static constexpr bool kIndexed = false;
    const K* g_sample;
    uint64_t m;
    int parts;
    K* s_spl;
    __device__ __forceinline__ size_t table_bytes() const { return (size_t)kMaxParts * sizeof(K); }
    __device__ __forceinline__ void setup(unsigned char* p) {
        s_spl = reinterpret_cast<K*>(p);
        for (int j = 1 + (int)threadIdx.x; j < parts; j += blockDim.x)
            s_spl[j - 1] = g_sample[(size_t)((uint64_t)j * m / (uint64_t)parts)];
        __syncthreads();
    }
    __device__ __forceinline__ uint32_t digit(K k) const {
        int lo = 0, hi = parts - 1;  // the answer lies in [0, parts - 1]
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_spl[mid] <= k) lo = mid + 1;
            else hi = mid;
        }
        return (uint32_t)lo;
    }
};

// Per-chunk range counts: each warp adds one count per distinct range of its
// 32 keys (the lanes sharing a range found with one match vote), since a few
// ranges would otherwise take every atomic on the same few words.
constexpr int kPartHistThreads = 512;

template <typename K>
__global__ void __launch_bounds__(kPartHistThreads) k_part_hist(const K* __restrict__ keys, uint32_t n,
                                                                uint32_t chunk_keys, RangeDigit<K> df, int bins,
                                                                uint32_t* __restrict__ hist) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_h = reinterpret_cast<uint32_t*>(smem);  // [bins]
    for (int d = threadIdx.x; d < bins; d += blockDim.x) s_h[d] = 0u;
    df.setup(smem + align_up_dev((size_t)bins * 4, 16));  // synchronises
    const uint32_t lo = blockIdx.x * chunk_keys, hi = min(n, lo + chunk_keys);
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t base = lo + (threadIdx.x & ~31u); base < hi; base += kPartHistThreads) {
        const uint32_t i = base + lane;
        const bool valid = i < hi;
        const uint32_t d = valid ? df.digit(keys[i]) : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(kFullMask, d);
        if (valid && (peers >> lane) == 1u) atomicAdd(&s_h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < bins; d += blockDim.x) hist[(size_t)blockIdx.x * bins + d] = s_h[d];
}

// counts[r] = keys of range r over all chunks.
__global__ void k_part_counts(const uint32_t* __restrict__ hist, uint32_t chunks, int bins, int parts,
                              unsigned long long* __restrict__ counts) {
    for (int d = threadIdx.x; d < parts; d += blockDim.x) {
        unsigned long long t = 0;
        for (uint32_t c = 0; c < chunks; ++c) t += hist[(size_t)c * bins + d];
        counts[d] = t;
    }
}

constexpr int kPartThreads = 512, kPartItems = 8;

template <typename K>
isort_status partition_device(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n,
                              const K* sorted_sample, size_t m, int parts, unsigned long long* counts,
                              cudaStream_t s) {
    int bins = 2;
    while (bins < parts) bins <<= 1;
    const bool hv = vin != nullptr;
    RangeDigit<K> df{sorted_sample, (uint64_t)m, parts, nullptr};
    const size_t tab = (size_t)kMaxParts * sizeof(K);
    const size_t smem = hv ? SweepCfg<K, true, kPartThreads, kPartItems>::smem_bytes(bins, false, tab)
                           : SweepCfg<K, false, kPartThreads, kPartItems>::smem_bytes(bins, false, tab);
    if (smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    auto kern_v = k_downsweep<K, true, kPartThreads, kPartItems, 0, RangeDigit<K>>;
    auto kern_k = k_downsweep<K, false, kPartThreads, kPartItems, 0, RangeDigit<K>>;
    int per_sm = 0;
    if (hv) {
        ISORT_TRY_CUDA(cudaFuncSetAttribute(kern_v, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern_v, kPartThreads, smem));
    } else {
        ISORT_TRY_CUDA(cudaFuncSetAttribute(kern_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern_k, kPartThreads, smem));
    }
    if (per_sm < 1) return ISORT_ERR_UNSUPPORTED;
    const uint32_t tile = (uint32_t)kPartThreads * kPartItems;
    const uint32_t num_tiles = (uint32_t)((n + tile - 1) / tile);
    const uint32_t want = (uint32_t)per_sm * (uint32_t)sm_count();
    const uint32_t chunk_tiles = (num_tiles + want - 1) / want;
    const uint32_t chunks = (num_tiles + chunk_tiles - 1) / chunk_tiles;

    const size_t tbl = align_up((size_t)chunks * bins * 4, 256);
    unsigned char* ws = nullptr;
    isort_status st = scratch_alloc((void**)&ws, 256 + 2 * tbl, s);
    if (st != ISORT_OK) return st;
    uint32_t* status = reinterpret_cast<uint32_t*>(ws);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + 256);
    uint32_t* coff = reinterpret_cast<uint32_t*>(ws + 256 + tbl);
    auto fail = [&](isort_status e) {
        scratch_free(ws, s);
        return e;
    };
    cudaError_t ce = cudaMemsetAsync(ws, 0, 256, s);
    if (ce != cudaSuccess) return fail(from_cuda(ce));
    {
        const size_t hsm = align_up((size_t)bins * 4, 16) + tab;
        ce = cudaFuncSetAttribute(k_part_hist<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
        if (ce != cudaSuccess) return fail(from_cuda(ce));
        LaunchScope ls("part_hist", s);
        k_part_hist<K><<<chunks, kPartHistThreads, hsm, s>>>(kin, (uint32_t)n, chunk_tiles * tile, df, bins, hist);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    {
        LaunchScope ls("chunk_scan", s);
        const int groups = bins >= kChunkScanThreads ? 1 : kChunkScanThreads / bins;
        k_chunk_scan<<<1, kChunkScanThreads, (size_t)(groups + 1) * bins * 4, s>>>(
            hist, (int)chunks, bins, coff, nullptr, 0, (int)sizeof(K) * 8, status);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    {
        SweepArgs a;
        a.keys_in = kin;
        a.vals_in = vin;
        a.keys_out = kout;
        a.vals_out = vout;
        a.n = (uint32_t)n;
        a.shift = 0;
        a.width = 0;
        a.bins = bins;
        a.chunk_off = coff;
        a.chunk_tiles = chunk_tiles;
        a.num_tiles = num_tiles;
        a.status = status;
        a.limit_ns = spin_limit_ns();
        a.use_bulk = (((uintptr_t)kin % 16) == 0) && (!hv || ((uintptr_t)vin % 16) == 0);
        LaunchScope ls("part_sweep", s);
        if (hv) kern_v<<<chunks, kPartThreads, smem, s>>>(a, df);
        else kern_k<<<chunks, kPartThreads, smem, s>>>(a, df);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    {
        LaunchScope ls("part_counts", s);
        k_part_counts<<<1, 256, 0, s>>>(hist, chunks, bins, parts, counts);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    st = finish_status(status, s);
    scratch_free(ws, s);
    return st;
}

template <typename K>
isort_status partition_entry(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n,
                             const K* sorted_sample, size_t m, int parts, uint64_t* counts, void* stream) {
    if (parts < 1 || parts > kMaxParts || !counts || (parts > 1 && (m == 0 || !sorted_sample)))
        return ISORT_ERR_INVALID_ARG;
    if (n >= (size_t(1) << 32)) return ISORT_ERR_UNSUPPORTED;
    if (n > 0 && (!kin || !kout || (const void*)kin == (const void*)kout || (vin && (!vout || vin == vout)) ||
                  (!vin && vout)))
        return ISORT_ERR_INVALID_ARG;
    if (is_host_pointer(counts) || (n > 0 && (is_host_pointer(kin) || is_host_pointer(kout) ||
                                              (vin && (is_host_pointer(vin) || is_host_pointer(vout))))) ||
        (parts > 1 && is_host_pointer(sorted_sample)))
        return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        ISORT_TRY_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint64_t) * (size_t)parts, s));
        return sync_mode() ? from_cuda(cudaStreamSynchronize(s)) : ISORT_OK;
    }
    return partition_device<K>(kin, vin, kout, vout, n, sorted_sample, m, parts,
                               reinterpret_cast<unsigned long long*>(counts), s);
}

}  // namespace
}  // namespace isort

using namespace isort;

extern "C" {

isort_status isort_sample(const void* keys, int key_width, size_t n, uint32_t m, uint64_t seed, void* out,
                          void* stream) {
    if ((key_width != 32 && key_width != 64) || (m > 0 && (n == 0 || !keys || !out))) return ISORT_ERR_INVALID_ARG;
    if (m == 0) return ISORT_OK;
    if (is_host_pointer(keys) || is_host_pointer(out)) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    {
        LaunchScope ls("sample", s);
        if (key_width == 32)
            k_sample<uint32_t><<<(m + 255) / 256, 256, 0, s>>>(static_cast<const uint32_t*>(keys), (uint64_t)n, m, seed,
                                                               static_cast<uint32_t*>(out));
        else
            k_sample<uint64_t><<<(m + 255) / 256, 256, 0, s>>>(static_cast<const uint64_t*>(keys), (uint64_t)n, m, seed,
                                                               static_cast<uint64_t*>(out));
        ISORT_TRY_CUDA(cudaGetLastError());
    }
    return sync_mode() ? from_cuda(cudaStreamSynchronize(s)) : ISORT_OK;
}

isort_status isort_partition(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                             size_t n, const uint32_t* sorted_sample, size_t m, int parts, uint64_t* counts,
                             void* stream) {
    return partition_entry<uint32_t>(keys_in, vals_in, keys_out, vals_out, n, sorted_sample, m, parts, counts, stream);
}

isort_status isort_partition_u64(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                 uint32_t* vals_out, size_t n, const uint64_t* sorted_sample, size_t m, int parts,
                                 uint64_t* counts, void* stream) {
    return partition_entry<uint64_t>(keys_in, vals_in, keys_out, vals_out, n, sorted_sample, m, parts, counts, stream);
}

}  // extern "C"
