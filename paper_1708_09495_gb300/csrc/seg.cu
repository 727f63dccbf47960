// Batched segmented sort: many arrays of uneven size sorted by one launch
// sequence (captured in a CUDA graph). Each segment is routed by its length,
// following the paper's observation that the block networks win for small n
// and count-sort rounds for larger n (Gerbessiotis, arXiv:1708.09495, Section 4,
// Observations 5 and 6):
//   len <= T_oet           OET in one warp, one key per lane (Section 2)
//   len <= T_btn_warp      BTN in one warp, 8 keys per lane (Section 2, eq. Tb)
//   len <= T_btn_cta       BTN over a CTA of p = next_pow2(len / 8) threads,
//                          8 keys per thread (four classes: p = 64 .. 512)
//   len <= 8192            count-sort rounds (8-bit digits, Section 3) entirely
//                          on chip in one CTA (the cluster kernel with C = 1).
//   len <= 8 * 8192        a thread-block cluster of C = 2, 4 or 8 CTAs (8192
//                          keys each) runs one count-sort round on the top 8
//                          bits of the segment's key range, the C digit
//                          histograms exchanged through distributed shared
//                          memory, and writes the result in place; its warps
//                          then finish the 256 digit groups (L2-resident) with
//                          BTN in registers, splitting a group above 512 keys
//                          again on its next 8 bits (MSD order). Segments over
//                          4 * 8192 keys with payloads split on 9 bits.
//   longer                 the global LSD path, one segment at a time (host
//                          driven; only in the synchronous status mode).
// Routing happens on the device: a classification kernel builds one work
// list per class, and persistent kernels walk their list with a static stride
// (warp, CTA or cluster index; no shared work counter).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "net.cuh"
#include "runtime.h"
#include "tune.h"

namespace cg = cooperative_groups;

namespace isort {

isort_status radix_sort_u32_device(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, size_t n,
                                   int key_bits, int rb, cudaStream_t s);

namespace {

constexpr int kSegThreads = 512;
constexpr int kSegItems = 16;
constexpr int kSegChunk = kSegThreads * kSegItems;  // keys per CTA of a cluster
constexpr int kSegChunkLog = 13;
constexpr int kSegBins = 256;
constexpr int kSegWarps = kSegThreads / 32;
static_assert(kSegChunk == 1 << kSegChunkLog, "chunk is a power of two");

enum : int {
    kClsOet = 0,
    kClsBtnWarp,
    kClsCta64,  // BTN over a CTA of p threads, p = next power of two >= len / 8
    kClsCta128,
    kClsCta256,
    kClsCta512,
    kClsC1,
    kClsC2,
    kClsC4,
    kClsC8,
    kClsBig,
    kClsRedo,  // segments the fine finish hands back to the split kernel
    kNumCls
};

struct SegThresholds {
    uint32_t oet;       // <= : OET in a warp (at most 32)
    uint32_t btn_warp;  // <= : BTN in a warp (at most 256)
    uint32_t btn_cta;   // <= : BTN over a CTA (at most 4096)
};

struct SegCtl {
    uint32_t status;
    uint32_t counts[kNumCls];
};

__global__ void k_seg_classify(const uint64_t* off, uint32_t nseg, SegThresholds th, SegCtl* ctl, uint32_t* lists,
                               int big_ok, const uint8_t* seg_bits) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
        const uint64_t lo = off[s], hi = off[s + 1];
        if (hi < lo) {
            set_status(&ctl->status, kStatBadOffsets);
            continue;
        }
        const uint64_t L = hi - lo;
        if (L <= 1) continue;
        if (seg_bits && seg_bits[s] == 0) continue;  // one key value: already in order
        int c;
        if (L <= th.oet) c = kClsOet;
        else if (L <= th.btn_warp) c = kClsBtnWarp;
        else if (L <= th.btn_cta) c = L <= 512 ? kClsCta64 : L <= 1024 ? kClsCta128 : L <= 2048 ? kClsCta256 : kClsCta512;
        else if (L <= (uint64_t)kSegChunk) c = kClsC1;
        else if (L <= 2ull * kSegChunk) c = kClsC2;
        else if (L <= 4ull * kSegChunk) c = kClsC4;
        else if (L <= 8ull * kSegChunk) c = kClsC8;
        else c = kClsBig;
        if (c == kClsBig && !big_ok) set_status(&ctl->status, kStatUnsupported);
        const uint32_t i = atomicAdd(&ctl->counts[c], 1u);
        lists[(size_t)c * nseg + i] = s;
    }
}

// One warp per segment: OET (one key per lane) or BTN (p <= 32 lanes x 8).
template <bool OET>
__global__ void __launch_bounds__(256) k_seg_warp(uint32_t* keys, uint32_t* vals, const uint64_t* off,
                                                  const uint32_t* list, SegCtl* ctl, int cls, uint32_t range_mask) {
    const uint32_t cnt = ctl->counts[cls];
    const uint32_t nwarps = gridDim.x * (blockDim.x / 32);
    for (uint32_t q = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); q < cnt; q += nwarps) {
        const uint32_t s = list[q];
        const uint64_t lo = off[s];
        const uint32_t L = (uint32_t)(off[s + 1] - lo);
        uint32_t* k = keys + lo;
        uint32_t* v = vals ? vals + lo : nullptr;
        if constexpr (OET) {
            net::oet_warp1(k, v, L, range_mask, &ctl->status);
        } else {
            int p = 1;
            while ((uint32_t)(p * 8) < L) p <<= 1;
            net::btn_warp<8>(k, v, L, p, range_mask, &ctl->status);
        }
        __syncwarp();
    }
}

// One CTA of P threads per segment: BTN with p = P blocks of 8 (the class
// holds the segments with next_pow2(len / 8) = P).
template <int P>
__global__ void __launch_bounds__(P) k_seg_btn_cta(uint32_t* keys, uint32_t* vals, const uint64_t* off,
                                                   const uint32_t* list, SegCtl* ctl, int cls, uint32_t range_mask) {
    __shared__ uint64_t s_x[8 * P];
    const uint32_t cnt = ctl->counts[cls];
    for (uint32_t q = blockIdx.x; q < cnt; q += gridDim.x) {
        const uint32_t s = list[q];
        const uint64_t lo = off[s];
        const uint32_t L = (uint32_t)(off[s + 1] - lo);
        net::btn_block<8>(keys + lo, vals ? vals + lo : nullptr, L, P, s_x, nullptr, range_mask, &ctl->status);
        __syncthreads();  // s_x is reused by the next segment
    }
}

template <typename K>
struct SegArgsT {
    K* keys;
    uint32_t* vals;
    const uint64_t* off;
    const uint32_t* list;
    SegCtl* ctl;
    int cls;
    int key_bits;
    const K* seg_lo;          // optional: segment s's keys lie in [seg_lo[s], seg_lo[s] + 2^seg_bits[s])
    const uint8_t* seg_bits;  //   and are sorted on key - seg_lo[s] over seg_bits[s] bits
    uint32_t single_n = 0;    // > 0: one segment [0, single_n) (off, list and counts unused)
    K* keys_out = nullptr;    // single segment: the result goes here (keys / vals only read)
    uint32_t* vals_out = nullptr;
    uint32_t* redo_list = nullptr;  // fine finish: where segments it leaves unsorted are listed
};
using ClusterArgs = SegArgsT<uint32_t>;

constexpr size_t cluster_smem_bytes(bool vals) {
    return (size_t)kSegChunk * 4 * (vals ? 2 : 1) + (size_t)kSegWarps * kSegBins * 2 + (size_t)kSegBins * 4 * 3 +
           64 * 4 + (size_t)kSegWarps * kSegBins * 4;
}

// Count-sort rounds of one segment on a cluster of C CTAs (see file comment).
template <int C, bool VALS>
__global__ void __launch_bounds__(kSegThreads, 2) k_seg_cluster(ClusterArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_keys = reinterpret_cast<uint32_t*>(smem);
    uint32_t* s_vals = s_keys + kSegChunk;
    uint16_t* s_cnt = reinterpret_cast<uint16_t*>(s_keys + kSegChunk * (VALS ? 2 : 1));
    uint32_t* s_cta = reinterpret_cast<uint32_t*>(s_cnt + kSegWarps * kSegBins);  // this CTA's digit totals
    uint32_t* s_pre = s_cta + kSegBins;                                            // earlier CTAs' counts
    uint32_t* s_base = s_pre + kSegBins;                                           // digit start + s_pre
    uint32_t* s_misc = s_base + kSegBins;  // [1] range flag, [8..] warp sums
    uint32_t* s_match = s_misc + 64;       // per warp and digit: lanes holding the digit
    // (the launch always provides cluster_smem_bytes; every CTA of a cluster
    // sees the same size, so a failed check leaves the cluster together)
    if ((size_t)(reinterpret_cast<unsigned char*>(s_match + kSegWarps * kSegBins) - smem) > dynamic_smem_size()) {
        if (threadIdx.x == 0) set_status(&a.ctl->status, kStatBounds);
        return;
    }

    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t r = C == 1 ? 0u : cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t cnt = a.single_n ? 1u : a.ctl->counts[a.cls];

    for (int i = tid; i < kSegWarps * kSegBins; i += kSegThreads) {
        s_cnt[i] = 0;
        s_match[i] = 0;
    }
    __syncthreads();

    // static assignment: cluster c takes list entries c, c + clusters, ...
    // (every CTA of a cluster walks the same entries)
    const uint32_t nclusters = gridDim.x / C;
    for (uint32_t q = blockIdx.x / C; q < cnt; q += nclusters) {
        const uint32_t s = a.single_n ? 0u : a.list[q];
        const uint64_t lo = a.single_n ? 0ull : a.off[s];
        const uint32_t L = a.single_n ? a.single_n : (uint32_t)(a.off[s + 1] - lo);
        const uint32_t kbase = a.seg_lo ? a.seg_lo[s] : 0u;
        const int sbits = a.seg_bits ? (int)a.seg_bits[s] : a.key_bits;
        const int rounds = (sbits + 7) / 8;
        const int check_bits = a.seg_bits ? 32 : a.key_bits;
        const uint32_t my_lo = r * (uint32_t)kSegChunk;
        const uint32_t my_n = L > my_lo ? min(L - my_lo, (uint32_t)kSegChunk) : 0u;
        uint32_t* gk = a.keys + lo + my_lo;
        uint32_t* gv = VALS ? a.vals + lo + my_lo : nullptr;

        uint32_t k[kSegItems], v[kSegItems], rank[kSegItems];
        uint32_t orv = 0;
#pragma unroll
        for (int i = 0; i < kSegItems; ++i) {
            const uint32_t j = (uint32_t)(warp * kSegItems * 32 + i * 32 + lane);
            k[i] = j < my_n ? gk[j] : 0u;
            if constexpr (VALS) v[i] = j < my_n ? gv[j] : 0u;
            orv |= k[i];
        }
        const int bad_local = check_bits < 32 && (orv >> check_bits) != 0;
        const int bad_cta = __syncthreads_or(bad_local);
        if (tid == 0) s_misc[1] = (uint32_t)bad_cta;

        bool bad = false;
        for (int d = 0; d < rounds; ++d) {
            const int shift = d * 8;
            // rank each key among equal digits of its warp, in input order:
            // the lanes holding a digit OR their bit into the warp's word for
            // it, read the word back, and the highest of them advances the
            // digit's count and clears the word
#pragma unroll
            for (int i = 0; i < kSegItems; ++i) {
                const uint32_t j = (uint32_t)(warp * kSegItems * 32 + i * 32 + lane);
                const bool valid = j < my_n;
                const uint32_t dg = ((k[i] - kbase) >> shift) & 0xffu;
                uint32_t* mw = &s_match[warp * kSegBins + dg];
                if (valid) atomicOr(mw, 1u << lane);
                __syncwarp();
                const uint32_t peers = valid ? *mw : 0u;
                const uint32_t below = (uint32_t)__popc(peers & lanemask_lt());
                const uint32_t c = valid ? (uint32_t)s_cnt[warp * kSegBins + dg] : 0u;
                rank[i] = c + below;
                __syncwarp();
                if (valid && below + 1 == (uint32_t)__popc(peers)) {
                    s_cnt[warp * kSegBins + dg] = (uint16_t)(c + below + 1);
                    *mw = 0u;
                }
                __syncwarp();
            }
            __syncthreads();
            if (tid < kSegBins) {
                uint32_t sum = 0;
#pragma unroll 4
                for (int w = 0; w < kSegWarps; ++w) {
                    const uint32_t c = s_cnt[w * kSegBins + tid];
                    s_cnt[w * kSegBins + tid] = (uint16_t)sum;
                    sum += c;
                }
                s_cta[tid] = sum;
            }
            cluster.sync();  // every CTA's digit totals (and range flag) are visible
            if (d == 0 && check_bits < 32) {
                uint32_t any = 0;
                for (int rr = 0; rr < C; ++rr) any |= C == 1 ? s_misc[1] : *cluster.map_shared_rank(&s_misc[1], rr);
                if (any) {
                    bad = true;
                    if (tid == 0 && r == 0) set_status(&a.ctl->status, kStatKeyRange);
                    break;  // the whole cluster leaves the rounds together
                }
            }
            if (tid < kSegBins) {
                uint32_t tot = 0, pre = 0;
#pragma unroll
                for (int rr = 0; rr < C; ++rr) {
                    const uint32_t c = C == 1 ? s_cta[tid] : *cluster.map_shared_rank(&s_cta[tid], rr);
                    tot += c;
                    if constexpr (C > 1) pre += (uint32_t)rr < r ? c : 0u;
                }
                s_pre[tid] = pre;
                s_base[tid] = tot;
            }
            __syncthreads();
            // exclusive scan of the segment's digit totals (256 entries, 8 warps)
            if (warp < kSegBins / 32) {
                const uint32_t x0 = s_base[tid];
                uint32_t x = x0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFullMask, x, o);
                    if (lane >= o) x += y;
                }
                if (lane == 31) s_misc[8 + warp] = x;
                s_base[tid] = x - x0;  // exclusive within the warp
            }
            __syncthreads();
            if (tid < kSegBins) {
                uint32_t add = 0;
                for (int w = 0; w < warp; ++w) add += s_misc[8 + w];
                s_base[tid] += add + s_pre[tid];
            }
            __syncthreads();
            // scatter every key into the shared memory of its new owner
#pragma unroll
            for (int i = 0; i < kSegItems; ++i) {
                const uint32_t j = (uint32_t)(warp * kSegItems * 32 + i * 32 + lane);
                if (j < my_n) {
                    const uint32_t dg = ((k[i] - kbase) >> shift) & 0xffu;
                    const uint32_t pos = s_base[dg] + s_cnt[warp * kSegBins + dg] + rank[i];
                    const uint32_t owner = pos >> kSegChunkLog;
                    const uint32_t o = pos & (kSegChunk - 1);
                    if (owner < (uint32_t)C) {
                        if constexpr (C == 1) {
                            s_keys[o] = k[i];
                            if constexpr (VALS) s_vals[o] = v[i];
                        } else {
                            *cluster.map_shared_rank(&s_keys[o], owner) = k[i];
                            if constexpr (VALS) *cluster.map_shared_rank(&s_vals[o], owner) = v[i];
                        }
                    }
                }
            }
            cluster.sync();  // all keys have arrived
            for (int i = tid; i < kSegWarps * kSegBins; i += kSegThreads) s_cnt[i] = 0;
#pragma unroll
            for (int i = 0; i < kSegItems; ++i) {
                const uint32_t j = (uint32_t)(warp * kSegItems * 32 + i * 32 + lane);
                if (j < my_n) {
                    k[i] = s_keys[j];
                    if constexpr (VALS) v[i] = s_vals[j];
                }
            }
            __syncthreads();
        }
        if (bad) {
            // every CTA of the cluster left the rounds at the same barrier, so
            // they stay in step; the segment is left unchanged
            for (int i = tid; i < kSegWarps * kSegBins; i += kSegThreads) s_cnt[i] = 0;
            __syncthreads();
            continue;
        }
        uint32_t* ok = a.keys_out ? a.keys_out + lo + my_lo : gk;
        uint32_t* ov = VALS ? (a.vals_out ? a.vals_out + lo + my_lo : gv) : nullptr;
#pragma unroll
        for (int i = 0; i < kSegItems; ++i) {
            const uint32_t j = (uint32_t)(warp * kSegItems * 32 + i * 32 + lane);
            if (j < my_n) {
                ok[j] = k[i];
                if constexpr (VALS) ov[j] = v[i];
            }
        }
    }
    cluster.sync();  // no CTA leaves while others may still read its shared memory
}

// ---------------------------------------------------------------- split and finish

// Segments above one CTA's worth of keys (8192 < len <= 8 * 8192): a cluster
// of C CTAs runs ONE count-sort round on the top 8 bits of the segment's key
// range (the MSD digit), writing the result back to HBM in place (coalesced
// runs per digit); every warp of the cluster then sorts some of the 256 digit
// groups (now L2-resident) with BTN in its registers (at most 512 keys, 16 per
// lane). A digit group above 512 keys is split again on its next 8 bits (a
// work stack kept identically by every CTA of the cluster), so a group is
// either finished by a warp, or holds one key value.
constexpr int kSplitWarpMax = 512;  // longest group a warp finishes (BTN, 16 keys per lane)
// Pending groups: they are disjoint parts of one segment (<= 65,536 keys) and
// each holds more than 256 keys, so at most 255 are pending at once.
constexpr int kSplitStack = 512;

__host__ __device__ constexpr size_t split_smem_bytes(bool vals, int bins, size_t key_bytes = 4) {
    return (size_t)kSegChunk * (key_bytes + (vals ? 4 : 0))  // staging
           + (size_t)kSegWarps * bins * 2                    // per-warp digit counts
           + (size_t)kSegWarps * bins * 4                    // per-warp peer masks
           + (size_t)bins * 4 * 5 + 4 * 4                    // cta totals, earlier CTAs, base, local start, starts[bins+1]
           + 64 * 4 + 16                                     // misc (+ alignment)
           + (size_t)kSplitStack * (9 + key_bytes);          // work stack
}

// Exclusive scan of a[0..BINS-1] in place (threads 0..BINS-1, BINS <= 512;
// every thread calls).
template <int BINS>
__device__ __forceinline__ void scan_bins(uint32_t* a, uint32_t* wsum) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t x0 = 0, x = 0;
    if (tid < BINS) {
        x0 = a[tid];
        x = x0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
    }
    __syncthreads();
    if (tid < BINS) {
        uint32_t add = 0;
        for (int w = 0; w < warp; ++w) add += wsum[w];
        a[tid] = add + x - x0;
    }
    __syncthreads();
}

// One warp sorts a group of 2..512 keys: BTN with B keys per lane, B the
// smallest power of two with 32 B >= len (all lanes hold keys).
template <int B>
__device__ __forceinline__ void btn_warp_fill(uint32_t* k, uint32_t* v, uint32_t len) {
    int p = 1;
    while ((uint32_t)(p * B) < len) p <<= 1;
    net::btn_warp<B>(k, v, len, p);
}

// The same network on packed 32-bit items: (key - gkb) << ib | index, with
// ib = bit_length(len) so that every item is below the pad 0xFFFFFFFF (keys
// only: no index, ib = 0). Needs shift + ib <= 32, shift the bits the group's
// keys span above gkb.
// ks / vs: where the group is read (global memory, or the staging buffer in
// shared memory); k / v: where the sorted group is written.
template <int B, bool VALS, typename K>
__device__ __forceinline__ void btn_warp_packed(const K* ks, const uint32_t* vs, K* k, uint32_t* v, uint32_t len,
                                                K gkb, int ib) {
    const int t = threadIdx.x & 31;
    int p = 1;
    while ((uint32_t)(p * B) < len) p <<= 1;
    K x[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const uint32_t g = (uint32_t)t * B + i;
        x[i] = g < len ? (((ks[g] - gkb) << ib) | (VALS ? (K)g : (K)0)) : ~(K)0;
    }
    net::local_sort<B, K>(x);
    for (int kk = 2; kk <= p; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            const bool asc = (t & kk) == 0;
            const bool lower = t < (t ^ j);
            net::merge_split_shfl<B, K>(x, j, lower == asc);
            net::bitonic_merge<B, K>(x);
        }
    }
    uint32_t vv[B];
    if constexpr (VALS) {
        const K m = ((K)1 << ib) - (K)1;
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const uint32_t g = (uint32_t)t * B + i;
            vv[i] = g < len ? vs[(uint32_t)(x[i] & m)] : 0u;
        }
    }
    __syncwarp();  // every payload is read before any is written
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const uint32_t g = (uint32_t)t * B + i;
        if (g < len) {
            k[g] = gkb + (x[i] >> ib);
            if constexpr (VALS) v[g] = vv[i];
        }
    }
}

// A group of len keys spanning `shift` bits above its base packs into one item
// of the key's width when the index fits beside the key bits.
template <bool VALS, typename K>
__device__ __forceinline__ bool group_packs(uint32_t len, int shift) {
    const int ib = VALS ? 32 - __clz(len) : 0;
    return shift + ib <= (int)sizeof(K) * 8;
}

// Whether a warp can finish the group: packed items, or (u32 keys) the 64-bit
// (key, index) items of the block networks. A u64 group that does not pack is
// split again instead.
template <bool VALS, typename K>
__device__ __forceinline__ bool group_warp_ok(uint32_t len, int shift) {
    return len <= (uint32_t)kSplitWarpMax && (sizeof(K) == 4 || group_packs<VALS, K>(len, shift));
}

// ks / vs: the group's source (by default the destination itself).
template <bool VALS, typename K>
__device__ __forceinline__ void finish_group_warp(K* k, uint32_t* v, uint32_t len, K gkb, int shift,
                                                  const K* ks = nullptr, const uint32_t* vs = nullptr) {
    const int ib = VALS ? 32 - __clz(len) : 0;
    if (group_packs<VALS, K>(len, shift)) {
        const K* sk = ks ? ks : k;
        const uint32_t* sv = ks ? vs : v;
        if (len <= 32) btn_warp_packed<1, VALS, K>(sk, sv, k, v, len, gkb, ib);
        else if (len <= 64) btn_warp_packed<2, VALS, K>(sk, sv, k, v, len, gkb, ib);
        else if (len <= 128) btn_warp_packed<4, VALS, K>(sk, sv, k, v, len, gkb, ib);
        else if (len <= 256) btn_warp_packed<8, VALS, K>(sk, sv, k, v, len, gkb, ib);
        else btn_warp_packed<16, VALS, K>(sk, sv, k, v, len, gkb, ib);
        return;
    }
    if constexpr (sizeof(K) == 4) {
        if (ks) {  // the 64-bit item networks sort in place: bring the group over first
            for (uint32_t g = threadIdx.x & 31; g < len; g += 32) {
                k[g] = ks[g];
                if constexpr (VALS) v[g] = vs[g];
            }
            __syncwarp();
        }
        if (len <= 32) btn_warp_fill<1>(k, v, len);
        else if (len <= 64) btn_warp_fill<2>(k, v, len);
        else if (len <= 128) btn_warp_fill<4>(k, v, len);
        else if (len <= 256) btn_warp_fill<8>(k, v, len);
        else btn_warp_fill<16>(k, v, len);
    }
}

// RB: the split's digit width (8, or 9 where groups of about 128 keys let
// payload items pack into 32 bits).
template <int C, bool VALS, int RB, typename K>
__global__ void __launch_bounds__(kSegThreads, (RB == 8 && sizeof(K) == 4) ? 2 : 1) k_seg_split(SegArgsT<K> a) {
    constexpr int BINS = 1 << RB;
    constexpr int KW = (int)sizeof(K) * 8;
    static_assert(BINS <= kSegThreads, "one thread per digit");
    extern __shared__ __align__(16) unsigned char smem[];
    K* s_keys = reinterpret_cast<K*>(smem);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + kSegChunk);
    uint16_t* s_cnt = reinterpret_cast<uint16_t*>(smem + (size_t)kSegChunk * (sizeof(K) + (VALS ? 4 : 0)));
    uint32_t* s_match = reinterpret_cast<uint32_t*>(s_cnt + kSegWarps * BINS);
    uint32_t* s_cta = s_match + kSegWarps * BINS;  // this CTA's digit totals
    uint32_t* s_pre = s_cta + BINS;                 // the digit's keys in lower-ranked CTAs
    uint32_t* s_base = s_pre + BINS;                // group-relative output start of this CTA's run
    uint32_t* s_lst = s_base + BINS;                // local start of the digit in the staging buffer
    uint32_t* s_start = s_lst + BINS;               // [BINS+1] group-relative digit starts (same in every CTA)
    uint32_t* s_misc = s_start + BINS + 4;          // [1] range flag, [2] stack size, [8..23] warp sums
    // work stack: group key base, start (segment-relative), length, span bits
    K* st_kb = reinterpret_cast<K*>(align_up_dev(reinterpret_cast<uintptr_t>(s_misc + 64), sizeof(K)));
    uint32_t* st_lo = reinterpret_cast<uint32_t*>(st_kb + kSplitStack);
    uint32_t* st_len = st_lo + kSplitStack;
    uint8_t* st_bits = reinterpret_cast<uint8_t*>(st_len + kSplitStack);
    if ((size_t)(st_bits + kSplitStack - smem) > dynamic_smem_size()) {
        if (threadIdx.x == 0) set_status(&a.ctl->status, kStatBounds);
        return;  // every CTA of the cluster sees the same size: all leave
    }

    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t r = C == 1 ? 0u : cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t cnt = a.ctl->counts[a.cls];
    for (int i = tid; i < kSegWarps * BINS; i += kSegThreads) {
        s_cnt[i] = 0;
        s_match[i] = 0;
    }
    __syncthreads();

    const uint32_t nclusters = gridDim.x / C;
    for (uint32_t q = blockIdx.x / C; q < cnt; q += nclusters) {
        const uint32_t s = a.list[q];
        const uint64_t seg0 = a.off[s];
        const uint32_t L = (uint32_t)(a.off[s + 1] - seg0);
        const int check_bits = a.seg_bits ? KW : a.key_bits;
        if (tid == 0 && q + nclusters < cnt) {  // this CTA's part of the cluster's next segment: into L2 meanwhile
            const uint32_t s2 = a.list[q + nclusters];
            const uint64_t o2 = a.off[s2], l2 = a.off[s2 + 1] - o2, lo2 = (uint64_t)r * kSegChunk;
            if (l2 > lo2) {
                const uint64_t n2 = min(l2 - lo2, (uint64_t)kSegChunk);
                prefetch_l2(a.keys + o2 + lo2, n2 * sizeof(K));
                if constexpr (VALS) prefetch_l2(a.vals + o2 + lo2, n2 * 4);
            }
        }
        if (tid == 0) {
            st_lo[0] = 0;
            st_len[0] = L;
            st_kb[0] = a.seg_lo ? a.seg_lo[s] : (K)0;
            st_bits[0] = (uint8_t)(a.seg_bits ? (int)a.seg_bits[s] : a.key_bits);
            s_misc[2] = 1;
        }
        __syncthreads();
        bool first = true;
        // every pop removes a group and pushes only narrower ones, so the loop
        // ends; the bound (identical in every CTA) only guards that reasoning
        int guard = 0;
        while (s_misc[2] > 0) {
            if (++guard > 4 * kSplitStack) {
                if (tid == 0 && r == 0) set_status(&a.ctl->status, kStatBounds);
                break;
            }
            // pop (identically in every CTA)
            const uint32_t top = s_misc[2] - 1;
            const uint32_t g_lo = st_lo[top], g_len = st_len[top];
            const K kb = st_kb[top];
            const int bits = st_bits[top];
            __syncthreads();
            if (tid == 0) s_misc[2] = top;
            const int shift = bits > RB ? bits - RB : 0;
            const uint32_t my_lo = r * (uint32_t)kSegChunk;
            const uint32_t my_n = g_len > my_lo ? min(g_len - my_lo, (uint32_t)kSegChunk) : 0u;
            K* gk = a.keys + seg0 + g_lo;
            uint32_t* gv = VALS ? a.vals + seg0 + g_lo : nullptr;

            K k[kSegItems];
            uint32_t v[kSegItems], rank[kSegItems];
            K orv = 0;
#pragma unroll
            for (int i = 0; i < kSegItems; ++i) {
                const uint32_t j = (uint32_t)(warp * kSegItems * 32 + i * 32 + lane);
                k[i] = j < my_n ? gk[my_lo + j] : (K)0;
                if constexpr (VALS) v[i] = j < my_n ? gv[my_lo + j] : 0u;
                orv |= k[i];
            }
            if (first) {
                const int bad = __syncthreads_or(check_bits < KW && (orv >> check_bits) != 0);
                if (tid == 0) s_misc[1] = (uint32_t)bad;
            }
            // rank among equal digits of the warp, in input order (peer masks)
#pragma unroll
            for (int i = 0; i < kSegItems; ++i) {
                const uint32_t j = (uint32_t)(warp * kSegItems * 32 + i * 32 + lane);
                const bool valid = j < my_n;
                const uint32_t dg = (uint32_t)((k[i] - kb) >> shift) & (uint32_t)(BINS - 1);
                uint32_t* mw = &s_match[warp * BINS + dg];
                if (valid) atomicOr(mw, 1u << lane);
                __syncwarp();
                const uint32_t peers = valid ? *mw : 0u;
                const uint32_t below = (uint32_t)__popc(peers & lanemask_lt());
                const uint32_t c = valid ? (uint32_t)s_cnt[warp * BINS + dg] : 0u;
                rank[i] = c + below;
                __syncwarp();
                if (valid && below + 1 == (uint32_t)__popc(peers)) {
                    s_cnt[warp * BINS + dg] = (uint16_t)(c + below + 1);
                    *mw = 0u;
                }
                __syncwarp();
            }
            __syncthreads();
            if (tid < BINS) {  // per-warp counts -> per-warp exclusive prefixes; CTA totals
                uint32_t sum = 0;
#pragma unroll 4
                for (int w = 0; w < kSegWarps; ++w) {
                    const uint32_t c = s_cnt[w * BINS + tid];
                    s_cnt[w * BINS + tid] = (uint16_t)sum;
                    sum += c;
                }
                s_cta[tid] = sum;
                s_lst[tid] = sum;
            }
            cluster.sync();  // (A) every CTA's totals and range flag are visible
            if (first && check_bits < KW) {
                uint32_t any = 0;
                for (int rr = 0; rr < C; ++rr) any |= C == 1 ? s_misc[1] : *cluster.map_shared_rank(&s_misc[1], rr);
                if (any) {  // the whole cluster leaves the segment unchanged
                    if (tid == 0 && r == 0) set_status(&a.ctl->status, kStatKeyRange);
                    for (int i = tid; i < kSegWarps * BINS; i += kSegThreads) s_cnt[i] = 0;
                    if (tid == 0) s_misc[2] = 0;
                    cluster.sync();  // no CTA moves on while another reads its flag
                    break;
                }
            }
            first = false;
            if (tid < BINS) {
                uint32_t tot = 0, pre = 0;
#pragma unroll
                for (int rr = 0; rr < C; ++rr) {
                    const uint32_t c = C == 1 ? s_cta[tid] : *cluster.map_shared_rank(&s_cta[tid], rr);
                    tot += c;
                    if constexpr (C > 1) pre += (uint32_t)rr < r ? c : 0u;
                }
                s_pre[tid] = pre;
                s_start[tid] = tot;
            }
            scan_bins<BINS>(s_start, s_misc + 8);  // group digit starts
            scan_bins<BINS>(s_lst, s_misc + 8);    // local digit starts
            if (tid < BINS) s_base[tid] = s_start[tid] + s_pre[tid];
            if (tid == 0) s_start[BINS] = g_len;
            // stage by digit (stable), then write runs
#pragma unroll
            for (int i = 0; i < kSegItems; ++i) {
                const uint32_t j = (uint32_t)(warp * kSegItems * 32 + i * 32 + lane);
                if (j < my_n) {
                    const uint32_t dg = (uint32_t)((k[i] - kb) >> shift) & (uint32_t)(BINS - 1);
                    const uint32_t p = s_lst[dg] + s_cnt[warp * BINS + dg] + rank[i];
                    s_keys[p] = k[i];
                    if constexpr (VALS) s_vals[p] = v[i];
                }
            }
            __syncthreads();
            for (uint32_t j = tid; j < my_n; j += kSegThreads) {
                const K key = s_keys[j];
                const uint32_t dg = (uint32_t)((key - kb) >> shift) & (uint32_t)(BINS - 1);
                if constexpr (C == 1) {
                    // a group a warp finishes is written once, by that warp, from
                    // this staging buffer
                    const uint32_t len = s_start[dg + 1] - s_start[dg];
                    if (shift > 0 && len > 1 && group_warp_ok<VALS, K>(len, shift)) continue;
                }
                const uint32_t o = s_base[dg] + (j - s_lst[dg]);
                gk[o] = key;
                if constexpr (VALS) gv[o] = s_vals[j];
            }
            for (int i = tid; i < kSegWarps * BINS; i += kSegThreads) s_cnt[i] = 0;
            cluster.sync();  // (B) the whole group is written
            // finish the digit groups: warps take groups, larger ones are pushed
            if (shift > 0) {
                for (int d = (int)r * kSegWarps + warp; d < BINS; d += C * kSegWarps) {
                    const uint32_t c0 = s_start[d], c1 = s_start[d + 1], len = c1 - c0;
                    if (len <= 1 || !group_warp_ok<VALS, K>(len, shift)) continue;
                    if constexpr (C == 1)  // the whole group is in this CTA's staging buffer
                        finish_group_warp<VALS, K>(gk + c0, VALS ? gv + c0 : nullptr, len, kb + ((K)d << shift), shift,
                                                   s_keys + c0, VALS ? s_vals + c0 : nullptr);
                    else
                        finish_group_warp<VALS, K>(gk + c0, VALS ? gv + c0 : nullptr, len, kb + ((K)d << shift),
                                                   shift);
                }
                if (warp == 0) {  // push the groups above a warp's reach, in digit order
                    uint32_t top2 = s_misc[2];
                    for (int d0 = 0; d0 < BINS; d0 += 32) {
                        const int d = d0 + lane;
                        const uint32_t len = s_start[d + 1] - s_start[d];
                        const bool big = len > 1 && !group_warp_ok<VALS, K>(len, shift);
                        const uint32_t m = __ballot_sync(kFullMask, big);
                        const uint32_t slot = top2 + (uint32_t)__popc(m & lanemask_lt());
                        if (big) {
                            if (slot < (uint32_t)kSplitStack) {
                                st_lo[slot] = g_lo + s_start[d];
                                st_len[slot] = len;
                                st_kb[slot] = kb + ((K)d << shift);
                                st_bits[slot] = (uint8_t)shift;
                            } else {  // cannot happen (see kSplitStack)
                                set_status(&a.ctl->status, kStatBounds);
                            }
                        }
                        top2 = min(top2 + (uint32_t)__popc(m), (uint32_t)kSplitStack);
                    }
                    if (lane == 0) s_misc[2] = top2;
                }
            }
            __syncthreads();
        }
        // every thread has read the empty stack before thread 0 starts the next
        // segment's stack (without this a slow warp could see the new size and
        // run one more round of the old segment, out of step with the cluster)
        __syncthreads();
    }
    cluster.sync();  // no CTA leaves while others may still read its shared memory
}

// ---------------------------------------------------------------- fine finish
//
// One CTA per segment of at most 8,192 keys (u32 or u64, optional payload):
// the segment is sorted stably on chip by the top 16 bits of (key - m) over
// the bits its observed range spans (m its smallest key, M its largest): two
// stable count-sort passes of 8 bits, low digit first (Section 3's round, on
// chip). Keys sharing those 16 bits form runs of about n / 65,536 keys; each
// run is then sorted on its remaining low bits: runs of up to kFineThreadRun
// keys by one thread (stable insertion), runs of up to 512 keys by a warp (the
// packed bitonic network, items (low bits << index bits | index)). A segment
// holding a longer run is left unchanged and listed for the split kernel; a
// segment whose keys are all equal is already in order.
constexpr int kFineThreadRun = 16;
constexpr int kFineMaxRuns = 512;  // runs handed to warps per segment
constexpr int kFineBins = 256;

// Threads of a fine-finish CTA: 512 (two CTAs per SM) for u32 keys; 1,024 for
// u64 keys, whose buffers leave one CTA per SM (more warps to cover latency).
template <typename K>
constexpr int fine_threads() {
    return sizeof(K) == 4 ? 512 : 1024;
}
constexpr int kFineMisc = 256;  // words: warp minima and maxima, scan sums, flags

template <typename K, bool VALS>
constexpr size_t fine_smem_bytes() {
    return (size_t)kSegChunk * (sizeof(K) + (VALS ? 4 : 0))           // staging
           + (size_t)(fine_threads<K>() / 32) * kFineBins * 2          // per-warp digit counts
           + (size_t)(fine_threads<K>() / 32) * kFineBins * 4          // per-warp peer masks
           + (size_t)kFineBins * 4 + kFineMisc * 4                     // digit starts, reductions and flags
           + (size_t)kFineMaxRuns * 8;                                 // long runs: start, length
}

template <typename K>
__device__ __forceinline__ K warp_min(K x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const K y = __shfl_xor_sync(kFullMask, x, o);
        x = y < x ? y : x;
    }
    return x;
}

template <typename K>
__device__ __forceinline__ K warp_max(K x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const K y = __shfl_xor_sync(kFullMask, x, o);
        x = y > x ? y : x;
    }
    return x;
}

template <typename K, bool VALS>
__global__ void __launch_bounds__(fine_threads<K>(), sizeof(K) == 4 ? 2 : 1) k_seg_fine(SegArgsT<K> a) {
    constexpr int KW = (int)sizeof(K) * 8;
    constexpr int BINS = kFineBins;
    constexpr int FT = fine_threads<K>(), FW = FT / 32, FI = kSegChunk / FT;  // threads, warps, keys per thread
    static_assert(FI * FT == kSegChunk && 2 * FW * (int)(sizeof(K) / 4) + FW + 2 <= kFineMisc, "fine layout");
    extern __shared__ __align__(16) unsigned char smem[];
    K* s_keys = reinterpret_cast<K*>(smem);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + kSegChunk);
    uint16_t* s_cnt = reinterpret_cast<uint16_t*>(smem + (size_t)kSegChunk * (sizeof(K) + (VALS ? 4 : 0)));
    uint32_t* s_match = reinterpret_cast<uint32_t*>(s_cnt + FW * BINS);
    uint32_t* s_start = s_match + FW * BINS;  // [BINS]
    uint32_t* s_misc = s_start + BINS;        // [kFineMisc]: warp minima / maxima (as K), scan sums, flags
    K* s_wmin = reinterpret_cast<K*>(s_misc);  // [FW]
    K* s_wmax = s_wmin + FW;                   // [FW]
    uint32_t* s_wsum = s_misc + 2 * FW * (int)(sizeof(K) / 4);  // [FW], after the minima and maxima
    uint32_t* s_flag = s_wsum + FW;                             // [0] runs handed to warps, [1] redo
    uint2* s_runs = reinterpret_cast<uint2*>(s_misc + kFineMisc);
    if ((size_t)(reinterpret_cast<unsigned char*>(s_runs + kFineMaxRuns) - smem) > dynamic_smem_size()) {
        if (threadIdx.x == 0) set_status(&a.ctl->status, kStatBounds);
        return;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t cnt = a.ctl->counts[a.cls];
    for (int i = tid; i < FW * BINS; i += FT) {
        s_cnt[i] = 0;
        s_match[i] = 0;
    }
    __syncthreads();
    for (uint32_t q = blockIdx.x; q < cnt; q += gridDim.x) {
        const uint32_t s = a.list[q];
        const uint64_t seg0 = a.off[s];
        const uint32_t L = (uint32_t)(a.off[s + 1] - seg0);
        K* gk = a.keys + seg0;
        uint32_t* gv = VALS ? a.vals + seg0 : nullptr;
        const K base = a.seg_lo ? a.seg_lo[s] : (K)0;
        if (tid == 0 && q + gridDim.x < cnt) {  // the next segment this CTA sorts: into L2 meanwhile
            const uint32_t s2 = a.list[q + gridDim.x];
            const uint64_t o2 = a.off[s2], l2 = min(a.off[s2 + 1] - o2, (uint64_t)kSegChunk);
            prefetch_l2(a.keys + o2, l2 * sizeof(K));
            if constexpr (VALS) prefetch_l2(a.vals + o2, l2 * 4);
        }
        const int check_bits = a.seg_bits ? KW : a.key_bits;
        if (L > (uint32_t)kSegChunk) {  // not this class's segment (never expected)
            if (tid == 0) set_status(&a.ctl->status, kStatBounds);
            continue;
        }
        // load in input order: item i of lane l of warp w is key w * 32 FI + 32 i + l
        K k[FI];
        uint32_t v[FI];
        K mn = ~(K)0, mx = 0, orv = 0;
#pragma unroll
        for (int i = 0; i < FI; ++i) {
            const uint32_t j = (uint32_t)(warp * FI * 32 + i * 32 + lane);
            const bool valid = j < L;
            k[i] = valid ? gk[j] : (K)0;
            if constexpr (VALS) v[i] = valid ? gv[j] : 0u;
            if (valid) {
                orv |= k[i];
                const K x = k[i] - base;
                mn = x < mn ? x : mn;
                mx = x > mx ? x : mx;
            }
        }
        mn = warp_min(mn);
        mx = warp_max(mx);
        if (lane == 0) {
            s_wmin[warp] = mn;
            s_wmax[warp] = mx;
        }
        const int bad = __syncthreads_or(check_bits < KW && (orv >> check_bits) != 0);
        if (bad) {  // a key beyond the declared range: the segment is left unchanged
            if (tid == 0) set_status(&a.ctl->status, kStatKeyRange);
            __syncthreads();
            continue;
        }
        mn = s_wmin[0];
        mx = s_wmax[0];
        for (int w = 1; w < FW; ++w) {
            const K a0 = s_wmin[w], a1 = s_wmax[w];
            mn = a0 < mn ? a0 : mn;
            mx = a1 > mx ? a1 : mx;
        }
        if (tid == 0) {
            s_flag[0] = 0;
            s_flag[1] = 0;
        }
        __syncthreads();
        if (mx == mn) continue;  // every key equal: already in order (uniform)
        const K span = mx - mn;
        const int sbits = KW - (sizeof(K) == 8 ? __clzll((long long)span) : __clz((int)span));
        const int t = sbits > 16 ? sbits - 16 : 0;  // (x - mn) >> t < 2^16
        const int npass = sbits - t > 8 ? 2 : 1;
        for (int pass = 0; pass < npass; ++pass) {
            if (pass == 1) {  // the first pass's order, from the staging buffer
#pragma unroll
                for (int i = 0; i < FI; ++i) {
                    const uint32_t j = (uint32_t)(warp * FI * 32 + i * 32 + lane);
                    k[i] = j < L ? s_keys[j] : (K)0;
                    if constexpr (VALS) v[i] = j < L ? s_vals[j] : 0u;
                }
            }
            const int dsh = t + 8 * pass;
            uint32_t rank[FI];
#pragma unroll
            for (int i = 0; i < FI; ++i) {
                const uint32_t j = (uint32_t)(warp * FI * 32 + i * 32 + lane);
                const bool valid = j < L;
                const uint32_t dg = (uint32_t)((k[i] - base - mn) >> dsh) & (uint32_t)(BINS - 1);
                uint32_t* mw = &s_match[warp * BINS + dg];
                if (valid) atomicOr(mw, 1u << lane);
                __syncwarp();
                const uint32_t peers = valid ? *mw : 0u;
                const uint32_t below = (uint32_t)__popc(peers & lt);
                const uint32_t c = valid ? (uint32_t)s_cnt[warp * BINS + dg] : 0u;
                rank[i] = c + below;
                __syncwarp();
                if (valid && below + 1 == (uint32_t)__popc(peers)) {
                    s_cnt[warp * BINS + dg] = (uint16_t)(c + below + 1);
                    *mw = 0u;
                }
                __syncwarp();
            }
            __syncthreads();
            if (tid < BINS) {  // per-warp counts -> per-warp exclusive prefixes; digit totals
                uint32_t sum = 0;
#pragma unroll 4
                for (int w = 0; w < FW; ++w) {
                    const uint32_t c = s_cnt[w * BINS + tid];
                    s_cnt[w * BINS + tid] = (uint16_t)sum;
                    sum += c;
                }
                s_start[tid] = sum;
            }
            scan_bins<BINS>(s_start, s_wsum);  // synchronises
#pragma unroll
            for (int i = 0; i < FI; ++i) {
                const uint32_t j = (uint32_t)(warp * FI * 32 + i * 32 + lane);
                if (j < L) {
                    const uint32_t dg = (uint32_t)((k[i] - base - mn) >> dsh) & (uint32_t)(BINS - 1);
                    const uint32_t p = s_start[dg] + s_cnt[warp * BINS + dg] + rank[i];
                    if (p < (uint32_t)kSegChunk) {
                        s_keys[p] = k[i];
                        if constexpr (VALS) s_vals[p] = v[i];
                    }
                }
            }
            __syncthreads();
            for (int i = tid; i < FW * BINS; i += FT) s_cnt[i] = 0;
            __syncthreads();  // cleared before the next pass (or segment) ranks
        }
        if (t > 0) {
            // runs of keys sharing the top 16 bits, sorted on the low t bits
            const K lowmask = ((K)1 << t) - (K)1;
            for (uint32_t j = (uint32_t)tid; j < L; j += FT) {
                const K xj = s_keys[j] - base - mn;
                const K dj = xj >> t;
                if (j > 0 && ((s_keys[j - 1] - base - mn) >> t) == dj) continue;  // not a run start
                uint32_t e = j + 1;
                while (e < L && e - j <= (uint32_t)kSplitWarpMax && ((s_keys[e] - base - mn) >> t) == dj) ++e;
                const uint32_t r = e - j;
                if (r < 2) continue;
                if (r <= (uint32_t)kFineThreadRun) {  // stable insertion on the low bits
                    for (uint32_t u = j + 1; u < e; ++u) {
                        const K ku = s_keys[u];
                        uint32_t vu = 0;
                        if constexpr (VALS) vu = s_vals[u];
                        const K lu = (ku - base - mn) & lowmask;
                        uint32_t w = u;
                        while (w > j && ((s_keys[w - 1] - base - mn) & lowmask) > lu) {
                            s_keys[w] = s_keys[w - 1];
                            if constexpr (VALS) s_vals[w] = s_vals[w - 1];
                            --w;
                        }
                        s_keys[w] = ku;
                        if constexpr (VALS) s_vals[w] = vu;
                    }
                } else if (r > (uint32_t)kSplitWarpMax || !group_packs<VALS, K>(r, t)) {
                    s_flag[1] = 1;  // beyond a warp's network: the split kernel takes the segment
                } else {
                    const uint32_t slot = atomicAdd(&s_flag[0], 1u);
                    if (slot < (uint32_t)kFineMaxRuns) s_runs[slot] = make_uint2(j, r);
                    else s_flag[1] = 1;
                }
            }
            __syncthreads();
            if (s_flag[1]) {  // uniform: hand the whole segment to the split kernel
                if (tid == 0) {
                    const uint32_t slot = atomicAdd(&a.ctl->counts[kClsRedo], 1u);
                    a.redo_list[slot] = s;
                }
                __syncthreads();
                continue;
            }
            const uint32_t nruns = s_flag[0];
            for (uint32_t ri = (uint32_t)warp; ri < nruns; ri += FW) {
                const uint2 run = s_runs[ri];
                K* rk = s_keys + run.x;
                uint32_t* rv = VALS ? s_vals + run.x : nullptr;
                const K gkb = base + mn + (((rk[0] - base - mn) >> t) << t);
                const int ib = VALS ? 32 - __clz(run.y) : 0;
                if (run.y <= 32) btn_warp_packed<1, VALS, K>(rk, rv, rk, rv, run.y, gkb, ib);
                else if (run.y <= 64) btn_warp_packed<2, VALS, K>(rk, rv, rk, rv, run.y, gkb, ib);
                else if (run.y <= 128) btn_warp_packed<4, VALS, K>(rk, rv, rk, rv, run.y, gkb, ib);
                else if (run.y <= 256) btn_warp_packed<8, VALS, K>(rk, rv, rk, rv, run.y, gkb, ib);
                else btn_warp_packed<16, VALS, K>(rk, rv, rk, rv, run.y, gkb, ib);
                __syncwarp();
            }
            __syncthreads();
        }
        for (uint32_t j = (uint32_t)tid; j < L; j += FT) {
            gk[j] = s_keys[j];
            if constexpr (VALS) gv[j] = s_vals[j];
        }
        __syncthreads();  // the staging buffer is refilled by the next segment
    }
}

// ---------------------------------------------------------------- host side


template <int C>
isort_status launch_cluster(bool vals, const ClusterArgs& a, cudaStream_t s) {
    const size_t smem = cluster_smem_bytes(vals);
    auto kern = vals ? k_seg_cluster<C, true> : k_seg_cluster<C, false>;
    ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(kSegThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    cfg.gridDim = dim3(C);
    ISORT_TRY_CUDA(cudaOccupancyMaxActiveClusters(&clusters, (void*)kern, &cfg));
    if (clusters < 1) return ISORT_ERR_UNSUPPORTED;
    cfg.gridDim = dim3(C * clusters);
    LaunchScope ls(C == 1 ? "seg_cluster1" : C == 2 ? "seg_cluster2" : C == 4 ? "seg_cluster4" : "seg_cluster8", s);
    ISORT_TRY_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
    return ISORT_OK;
}

// One cluster of C CTAs sorting the single segment a.single_n keys long.
template <int C>
isort_status launch_cluster_single(bool vals, const ClusterArgs& a, cudaStream_t s) {
    const size_t smem = cluster_smem_bytes(vals);
    auto kern = vals ? k_seg_cluster<C, true> : k_seg_cluster<C, false>;
    ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(kSegThreads);
    cfg.gridDim = dim3(C);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    LaunchScope ls(C == 1 ? "small_sort1" : C == 2 ? "small_sort2" : C == 4 ? "small_sort4" : "small_sort8", s);
    ISORT_TRY_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
    return ISORT_OK;
}

template <int P>
isort_status launch_btn_cta(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint32_t* lists, uint32_t nseg,
                            SegCtl* ctl, int cls, uint32_t range_mask, cudaStream_t s) {
    int per_sm = 0;
    ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seg_btn_cta<P>, P, 0));
    k_seg_btn_cta<P><<<std::max(1, per_sm) * sm_count(), P, 0, s>>>(keys, vals, off, lists + (size_t)cls * nseg, ctl,
                                                                     cls, range_mask);
    return from_cuda(cudaGetLastError());
}

template <int C, typename K = uint32_t>
isort_status launch_split(bool vals, const SegArgsT<K>& a, cudaStream_t s) {
    // u32 payload groups pack into 32-bit items when the index fits next to
    // the key's remaining bits: 9-bit digits for the largest segments
    constexpr int kRbVals = (C == 8 && sizeof(K) == 4) ? 9 : 8;
    const size_t smem = split_smem_bytes(vals, vals ? 1 << kRbVals : 256, sizeof(K));
    auto kern = vals ? k_seg_split<C, true, kRbVals, K> : k_seg_split<C, false, 8, K>;
    ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(kSegThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    cfg.gridDim = dim3(C);
    ISORT_TRY_CUDA(cudaOccupancyMaxActiveClusters(&clusters, (void*)kern, &cfg));
    if (clusters < 1) return ISORT_ERR_UNSUPPORTED;
    cfg.gridDim = dim3(C * clusters);
    LaunchScope ls(C == 1 ? "seg_split1" : C == 2 ? "seg_split2" : C == 4 ? "seg_split4" : "seg_split8", s);
    ISORT_TRY_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
    return ISORT_OK;
}

template <typename K>
isort_status launch_fine(bool vals, const SegArgsT<K>& a, cudaStream_t s) {
    const size_t smem = vals ? fine_smem_bytes<K, true>() : fine_smem_bytes<K, false>();
    auto kern = vals ? k_seg_fine<K, true> : k_seg_fine<K, false>;
    ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, fine_threads<K>(), smem));
    if (per_sm < 1) return ISORT_ERR_UNSUPPORTED;
    LaunchScope ls("seg_fine", s);
    kern<<<per_sm * sm_count(), fine_threads<K>(), smem, s>>>(a);
    return from_cuda(cudaGetLastError());
}

// Enqueues classification and every class kernel on `s`.
isort_status enqueue_segmented(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint32_t nseg, int key_bits,
                               SegCtl* ctl, uint32_t* lists, int big_ok, const SegThresholds& th, cudaStream_t s,
                               const uint32_t* seg_lo = nullptr, const uint8_t* seg_bits = nullptr) {
    const uint32_t range_mask = (key_bits >= 32 || seg_bits) ? 0u : ~((1u << key_bits) - 1u);
    ISORT_TRY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(SegCtl), s));
    {
        LaunchScope ls("seg_classify", s);
        const unsigned grid = (unsigned)std::max<uint32_t>(1, std::min<uint32_t>((nseg + 255) / 256, 4 * sm_count()));
        k_seg_classify<<<grid, 256, 0, s>>>(off, nseg, th, ctl, lists, big_ok, seg_bits);
        ISORT_TRY_CUDA(cudaGetLastError());
    }
    ClusterArgs a;
    a.keys = keys;
    a.vals = vals;
    a.off = off;
    a.ctl = ctl;
    a.key_bits = key_bits;
    a.seg_lo = seg_lo;
    a.seg_bits = seg_bits;
    const bool v = vals != nullptr;
    // largest segments first: they take longest
    const int order[4] = {kClsC8, kClsC4, kClsC2, kClsC1};
    for (int c : order) {
        a.cls = c;
        a.list = lists + (size_t)c * nseg;
        isort_status st;
        if (c == kClsC1 && tune().fine) {  // the fine finish; what it hands back takes the on-chip rounds
            a.redo_list = lists + (size_t)kClsRedo * nseg;
            st = launch_fine<uint32_t>(v, a, s);
            if (st == ISORT_OK) {
                a.cls = kClsRedo;
                a.list = a.redo_list;
                st = launch_cluster<1>(v, a, s);
            }
        } else {
            st = c == kClsC8   ? launch_split<8>(v, a, s)
                 : c == kClsC4 ? launch_split<4>(v, a, s)
                 : c == kClsC2 ? launch_split<2>(v, a, s)
                               : launch_cluster<1>(v, a, s);
        }
        if (st != ISORT_OK) return st;
    }
    {
        LaunchScope ls("seg_btn_cta", s);
        ISORT_TRY(launch_btn_cta<512>(keys, vals, off, lists, nseg, ctl, kClsCta512, range_mask, s));
        ISORT_TRY(launch_btn_cta<256>(keys, vals, off, lists, nseg, ctl, kClsCta256, range_mask, s));
        ISORT_TRY(launch_btn_cta<128>(keys, vals, off, lists, nseg, ctl, kClsCta128, range_mask, s));
        ISORT_TRY(launch_btn_cta<64>(keys, vals, off, lists, nseg, ctl, kClsCta64, range_mask, s));
    }
    {
        int per_sm = 0;
        ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seg_warp<false>, 256, 0));
        LaunchScope ls("seg_btn_warp", s);
        k_seg_warp<false><<<std::max(1, per_sm) * sm_count(), 256, 0, s>>>(
            keys, vals, off, lists + (size_t)kClsBtnWarp * nseg, ctl, kClsBtnWarp, range_mask);
        ISORT_TRY_CUDA(cudaGetLastError());
    }
    {
        int per_sm = 0;
        ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seg_warp<true>, 256, 0));
        LaunchScope ls("seg_oet_warp", s);
        k_seg_warp<true><<<std::max(1, per_sm) * sm_count(), 256, 0, s>>>(keys, vals, off, lists + (size_t)kClsOet * nseg,
                                                                          ctl, kClsOet, range_mask);
        ISORT_TRY_CUDA(cudaGetLastError());
    }
    return ISORT_OK;
}

// Per-thread cached graph of the launch sequence (updated in place per call).
struct GraphCache {
    int device = -1;
    uint32_t nseg = 0;
    bool vals = false;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
};

thread_local GraphCache g_graph;

isort_status launch_via_graph(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint32_t nseg, int key_bits,
                              SegCtl* ctl, uint32_t* lists, int big_ok, const SegThresholds& th, cudaStream_t s,
                              const uint32_t* seg_lo = nullptr, const uint8_t* seg_bits = nullptr) {
    int dev = 0;
    ISORT_TRY_CUDA(cudaGetDevice(&dev));
    GraphCache& gc = g_graph;
    if (gc.device != dev) {
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        if (gc.cap) cudaStreamDestroy(gc.cap);
        gc = GraphCache();
        ISORT_TRY_CUDA(cudaStreamCreateWithFlags(&gc.cap, cudaStreamNonBlocking));
        gc.device = dev;
    }
    cudaGraph_t graph = nullptr;
    ISORT_TRY_CUDA(cudaStreamBeginCapture(gc.cap, cudaStreamCaptureModeThreadLocal));
    isort_status st;
    {
        CaptureScope cs;  // launches are counted, not timed, while capturing
        st = enqueue_segmented(keys, vals, off, nseg, key_bits, ctl, lists, big_ok, th, gc.cap, seg_lo, seg_bits);
    }
    cudaError_t ce = cudaStreamEndCapture(gc.cap, &graph);
    if (st != ISORT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess) return from_cuda(ce);
    bool updated = false;
    if (gc.exec && gc.vals == (vals != nullptr)) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(gc.exec, graph, &info) == cudaSuccess) updated = true;
        else cudaGetLastError();
    }
    if (!updated) {
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
        ce = cudaGraphInstantiate(&gc.exec, graph, 0);
        if (ce != cudaSuccess) {
            cudaGraphDestroy(graph);
            return from_cuda(ce);
        }
        gc.vals = vals != nullptr;
    }
    cudaGraphDestroy(graph);
    LaunchScope ls("segmented_graph", s, /*count=*/false);
    ISORT_TRY_CUDA(cudaGraphLaunch(gc.exec, s));
    return ISORT_OK;
}

// ---------------------------------------------------------------- router autotuning
//
// The length cut-offs between the classes are where one method overtakes the
// next (Section 4, Observations 5-6: the networks win for small n, the
// count-sort rounds for larger n; where is machine-dependent). The built-in
// cut-offs {32, 256, 4096} are the largest lengths each network kernel takes.
// With isort_autotune on, the first segmented sort of each kind (keys only or
// with payloads) times each method -- OET in a warp, BTN in a warp, BTN over a
// CTA, the one-CTA on-chip count-sort rounds -- on synthetic batches of 2^20
// keys in segments of one length, for lengths from 8 to 4096, and takes as
// each cut-off the largest length at which that method was the fastest; the
// choice is appended to the cache file as "router <payload> <oet> <btn_warp>
// <btn_cta>" and read from it later. Every method sorts every length it is
// given stably, so the output does not depend on the cut-offs.
constexpr SegThresholds kDefaultThresholds{32, 256, 4096};
constexpr uint32_t kMaxOet = 32, kMaxBtnWarp = 256, kMaxBtnCta = 4096;

struct RouterTune {
    std::mutex mu;
    bool done[2] = {false, false};
    SegThresholds th[2] = {kDefaultThresholds, kDefaultThresholds};
};

RouterTune& router_state() {
    static RouterTune r;
    return r;
}

bool valid_thresholds(const SegThresholds& t) {
    return t.oet <= kMaxOet && t.btn_warp <= kMaxBtnWarp && t.btn_cta <= kMaxBtnCta && t.oet <= t.btn_warp &&
           t.btn_warp <= t.btn_cta;
}

__global__ void k_router_fill(uint32_t* keys, uint32_t* vals, uint32_t n, uint64_t* off, uint32_t nseg, uint32_t len) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        keys[i] = (uint32_t)(splitmix_mix(0x5E6Dull + (uint64_t)(i + 1) * kSplitmixGamma) >> 32);
        if (vals) vals[i] = i;
    }
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= nseg; q += gridDim.x * blockDim.x)
        off[q] = (uint64_t)q * len;
}

// Times each method on segments of each length; *out gets the cut-offs.
isort_status measure_router(bool with_vals, cudaStream_t s, SegThresholds* out) {
    constexpr uint32_t kN = 1u << 20;
    constexpr uint32_t kLens[] = {8, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096};
    constexpr uint32_t kMaxSeg = kN / 8;
    const size_t kb = (size_t)kN * 4, ob = align_up((size_t)(kMaxSeg + 1) * 8, 256);
    const size_t ctl_bytes = align_up(sizeof(SegCtl), 256), list_bytes = align_up((size_t)kNumCls * kMaxSeg * 4, 256);
    const size_t total = 4 * kb + ob + ctl_bytes + list_bytes;
    unsigned char* ws = nullptr;
    ISORT_TRY(scratch_alloc((void**)&ws, total, s));
    uint32_t* k0 = reinterpret_cast<uint32_t*>(ws);
    uint32_t* v0 = reinterpret_cast<uint32_t*>(ws + kb);
    uint32_t* k = reinterpret_cast<uint32_t*>(ws + 2 * kb);
    uint32_t* v = reinterpret_cast<uint32_t*>(ws + 3 * kb);
    uint64_t* off = reinterpret_cast<uint64_t*>(ws + 4 * kb);
    SegCtl* ctl = reinterpret_cast<SegCtl*>(ws + 4 * kb + ob);
    uint32_t* lists = reinterpret_cast<uint32_t*>(ws + 4 * kb + ob + ctl_bytes);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // method m: the thresholds that send every segment of up to its limit to it
    const SegThresholds route[4] = {{kMaxOet, kMaxOet, kMaxOet}, {0, kMaxBtnWarp, kMaxBtnWarp}, {0, 0, kMaxBtnCta},
                                    {0, 0, 0}};
    const uint32_t limit[4] = {kMaxOet, kMaxBtnWarp, kMaxBtnCta, (uint32_t)kSegChunk};
    uint32_t best_len[3] = {0, 0, 0};  // largest length where OET / BTN warp / BTN CTA was the fastest
    isort_status st = ISORT_OK;
    for (uint32_t len : kLens) {
        const uint32_t nseg = kN / len;
        k_router_fill<<<4 * sm_count(), 256, 0, s>>>(k0, with_vals ? v0 : nullptr, kN, off, nseg, len);
        float best = 1e30f;
        int win = -1;
        for (int m = 0; m < 4 && st == ISORT_OK; ++m) {
            if (len > limit[m]) continue;
            float t_best = 1e30f;
            for (int rep = 0; rep < 3 && st == ISORT_OK; ++rep) {
                cudaMemcpyAsync(k, k0, kb, cudaMemcpyDeviceToDevice, s);
                if (with_vals) cudaMemcpyAsync(v, v0, kb, cudaMemcpyDeviceToDevice, s);
                cudaEventRecord(e0, s);
                st = enqueue_segmented(k, with_vals ? v : nullptr, off, nseg, 32, ctl, lists, 0, route[m], s);
                cudaEventRecord(e1, s);
                if (st == ISORT_OK && cudaEventSynchronize(e1) == cudaSuccess) {
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    t_best = std::min(t_best, t);
                } else if (st == ISORT_OK) {
                    st = ISORT_ERR_CUDA;
                }
            }
            if (t_best < best) {
                best = t_best;
                win = m;
            }
        }
        if (st != ISORT_OK) break;
        if (win >= 0 && win < 3) best_len[win] = len;
    }
    uint32_t dev_status = 0;
    if (st == ISORT_OK) {
        if (cudaMemcpyAsync(&dev_status, &ctl->status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = ISORT_ERR_CUDA;
        else if (dev_status)
            st = map_bits(dev_status);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    scratch_free(ws, s);
    cudaStreamSynchronize(s);
    if (st != ISORT_OK) return st;
    SegThresholds t;
    t.oet = best_len[0];
    t.btn_warp = std::max(t.oet, best_len[1]);
    t.btn_cta = std::max(t.btn_warp, best_len[2]);
    *out = t;
    return ISORT_OK;
}

// The cut-offs a segmented sort uses (the built-in ones unless autotuning is on).
isort_status router_thresholds(bool with_vals, cudaStream_t s, SegThresholds* th) {
    std::string path;
    *th = kDefaultThresholds;
    if (!autotune_config(&path)) return ISORT_OK;
    RouterTune& rt = router_state();
    std::lock_guard<std::mutex> lk(rt.mu);
    const int kind = with_vals ? 1 : 0;
    if (rt.done[kind]) {
        *th = rt.th[kind];
        return ISORT_OK;
    }
    if (!path.empty()) {
        if (FILE* f = std::fopen(path.c_str(), "r")) {
            char ln[256];
            while (std::fgets(ln, sizeof(ln), f)) {
                int pv = -1;
                SegThresholds t{};
                if (std::sscanf(ln, "router %d %u %u %u", &pv, &t.oet, &t.btn_warp, &t.btn_cta) == 4 && pv == kind &&
                    valid_thresholds(t)) {
                    rt.th[kind] = t;
                    rt.done[kind] = true;
                }
            }
            std::fclose(f);
        }
        if (rt.done[kind]) {
            *th = rt.th[kind];
            return ISORT_OK;
        }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    if (cap != cudaStreamCaptureStatusNone) return ISORT_OK;  // no timing inside a capture: built-in cut-offs
    SegThresholds t;
    ISORT_TRY(measure_router(with_vals, s, &t));
    rt.th[kind] = t;
    rt.done[kind] = true;
    *th = t;
    if (!path.empty()) {
        if (FILE* f = std::fopen(path.c_str(), "a")) {
            std::fprintf(f, "router %d %u %u %u\n", kind, t.oet, t.btn_warp, t.btn_cta);
            std::fclose(f);
        }
    }
    return ISORT_OK;
}

isort_status segmented_entry(uint32_t* keys, uint32_t* vals, const uint64_t* off, size_t nseg, int key_bits,
                             void* stream, const uint32_t* seg_lo = nullptr, const uint8_t* seg_bits = nullptr) {
    if (key_bits == 0) key_bits = 32;
    if (key_bits < 1 || key_bits > 32) return ISORT_ERR_INVALID_ARG;
    if (nseg == 0) return ISORT_OK;
    if (nseg >= (size_t(1) << 31)) return ISORT_ERR_UNSUPPORTED;
    if (!keys || !off) return ISORT_ERR_INVALID_ARG;
    if (is_host_pointer(keys) || is_host_pointer(off) || (vals && is_host_pointer(vals))) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t ns = (uint32_t)nseg;
    SegThresholds th;
    ISORT_TRY(router_thresholds(vals != nullptr, s, &th));
    const size_t ctl_bytes = align_up(sizeof(SegCtl), 256);
    const size_t list_bytes = align_up((size_t)kNumCls * ns * 4, 256);
    unsigned char* ws = nullptr;
    isort_status st = scratch_alloc((void**)&ws, ctl_bytes + list_bytes, s);
    if (st != ISORT_OK) return st;
    SegCtl* ctl = reinterpret_cast<SegCtl*>(ws);
    uint32_t* lists = reinterpret_cast<uint32_t*>(ws + ctl_bytes);

    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    const int big_ok = sync_mode() && cap != cudaStreamCaptureStatusActive;
    if (cap == cudaStreamCaptureStatusActive || trace_on()) {
        // the caller is building its own graph (or launches are traced): enqueue directly
        st = enqueue_segmented(keys, vals, off, ns, key_bits, ctl, lists, big_ok, th, s, seg_lo, seg_bits);
    } else {
        st = launch_via_graph(keys, vals, off, ns, key_bits, ctl, lists, big_ok, th, s, seg_lo, seg_bits);
    }
    if (st != ISORT_OK) {
        scratch_free(ws, s);
        return st;
    }
    // segments beyond the on-chip classes: global rounds, one segment at a time
    if (big_ok) {
        SegCtl h;
        cudaError_t ce = cudaMemcpyAsync(&h, ctl, sizeof(SegCtl), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) {
            scratch_free(ws, s);
            return from_cuda(ce);
        }
        if (h.counts[kClsBig] > 0) {
            std::vector<uint32_t> ids(h.counts[kClsBig]);
            std::vector<uint64_t> hoff(nseg + 1);
            ce = cudaMemcpyAsync(ids.data(), lists + (size_t)kClsBig * ns, ids.size() * 4, cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(hoff.data(), off, (nseg + 1) * 8, cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) {
                scratch_free(ws, s);
                return from_cuda(ce);
            }
            for (uint32_t id : ids) {
                const size_t len = (size_t)(hoff[id + 1] - hoff[id]);
                uint32_t* k = keys + hoff[id];
                uint32_t* v = vals ? vals + hoff[id] : nullptr;
                st = radix_sort_u32_device(k, v, k, v, len, key_bits, 8, s);
                if (st != ISORT_OK) break;
            }
        }
        if (st == ISORT_OK) st = finish_status(&ctl->status, s);
    } else {
        st = finish_status(&ctl->status, s);
    }
    scratch_free(ws, s);
    return st;
}

}  // namespace

void router_autotune_reset() {
    RouterTune& rt = router_state();
    std::lock_guard<std::mutex> lk(rt.mu);
    rt.done[0] = rt.done[1] = false;
    rt.th[0] = rt.th[1] = kDefaultThresholds;
}

// The finishing step of the learned-bucket sort: every bucket is a segment
// whose keys lie in [seg_lo[s], seg_lo[s] + 2^seg_bits[s]).
// The whole radix-2^8 sort of n <= 8 * 8192 u32 keys (+ payload) in one
// launch, from kin/vin to kout/vout (the same buffers: in place): the
// count-sort rounds run on chip on one cluster of C = 1, 2, 4 or 8 CTAs (8192
// keys each), keys exchanged through distributed shared memory between
// rounds. A key >= 2^key_bits: ISORT_ERR_KEY_RANGE, buffers unchanged.
isort_status radix_small_u32(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, uint32_t n,
                             int key_bits, cudaStream_t s) {
    if (n == 0 || n > 8u * kSegChunk) return ISORT_ERR_INVALID_ARG;
    SegCtl* ctl = nullptr;
    ISORT_TRY(scratch_alloc((void**)&ctl, sizeof(SegCtl), s));
    isort_status st = from_cuda(cudaMemsetAsync(ctl, 0, sizeof(SegCtl), s));
    ClusterArgs a{};
    a.keys = const_cast<uint32_t*>(kin);  // only read when kout is set
    a.vals = const_cast<uint32_t*>(vin);
    a.keys_out = kout;
    a.vals_out = vout;
    a.ctl = ctl;
    a.key_bits = key_bits;
    a.single_n = n;
    const bool hv = vin != nullptr;
    if (st == ISORT_OK) {
        if (n <= (uint32_t)kSegChunk) st = launch_cluster_single<1>(hv, a, s);
        else if (n <= 2u * kSegChunk) st = launch_cluster_single<2>(hv, a, s);
        else if (n <= 4u * kSegChunk) st = launch_cluster_single<4>(hv, a, s);
        else st = launch_cluster_single<8>(hv, a, s);
    }
    if (st == ISORT_OK) st = finish_status(&ctl->status, s);
    scratch_free(ctl, s);
    return st;
}

isort_status segmented_finish_u32(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint32_t nseg,
                                  const uint32_t* seg_lo, const uint8_t* seg_bits, cudaStream_t s) {
    return segmented_entry(keys, vals, off, nseg, 32, (void*)s, seg_lo, seg_bits);
}

// The same for u64 keys, segments of at most 8 x 8192 keys: every segment of
// two or more keys (and more than one key value) goes to the split kernel of
// its size class (one CTA up to 8192 keys, then clusters of 2, 4, 8), whose
// warps finish the digit groups on packed 64-bit items. Synchronises.
isort_status segmented_finish_u64(uint64_t* keys, uint32_t* vals, const uint64_t* off, uint32_t nseg,
                                  const uint64_t* seg_lo, const uint8_t* seg_bits, cudaStream_t s) {
    if (nseg == 0) return ISORT_OK;
    const size_t ctl_bytes = align_up(sizeof(SegCtl), 256);
    const size_t list_bytes = align_up((size_t)kNumCls * nseg * 4, 256);
    unsigned char* ws = nullptr;
    isort_status st = scratch_alloc((void**)&ws, ctl_bytes + list_bytes, s);
    if (st != ISORT_OK) return st;
    SegCtl* ctl = reinterpret_cast<SegCtl*>(ws);
    uint32_t* lists = reinterpret_cast<uint32_t*>(ws + ctl_bytes);
    cudaError_t ce = cudaMemsetAsync(ctl, 0, sizeof(SegCtl), s);
    if (ce == cudaSuccess) {
        LaunchScope ls("seg_classify", s);
        const SegThresholds none{0, 0, 0};  // no network classes: the split kernels take every length
        const unsigned grid = (unsigned)std::max<uint32_t>(1, std::min<uint32_t>((nseg + 255) / 256, 4 * sm_count()));
        k_seg_classify<<<grid, 256, 0, s>>>(off, nseg, none, ctl, lists, 0, seg_bits);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) {
        scratch_free(ws, s);
        return from_cuda(ce);
    }
    SegArgsT<uint64_t> a;
    a.keys = keys;
    a.vals = vals;
    a.off = off;
    a.ctl = ctl;
    a.key_bits = 64;
    a.seg_lo = seg_lo;
    a.seg_bits = seg_bits;
    const bool v = vals != nullptr;
    const int order[4] = {kClsC8, kClsC4, kClsC2, kClsC1};
    for (int c : order) {
        a.cls = c;
        a.list = lists + (size_t)c * nseg;
        if (c == kClsC1 && tune().fine) {  // the fine finish; what it hands back takes the split kernel
            a.redo_list = lists + (size_t)kClsRedo * nseg;
            st = launch_fine<uint64_t>(v, a, s);
            if (st == ISORT_OK) {
                a.cls = kClsRedo;
                a.list = a.redo_list;
                st = launch_split<1, uint64_t>(v, a, s);
            }
        } else {
            st = c == kClsC8   ? launch_split<8, uint64_t>(v, a, s)
                 : c == kClsC4 ? launch_split<4, uint64_t>(v, a, s)
                 : c == kClsC2 ? launch_split<2, uint64_t>(v, a, s)
                               : launch_split<1, uint64_t>(v, a, s);
        }
        if (st != ISORT_OK) break;
    }
    if (st == ISORT_OK) st = finish_status(&ctl->status, s);  // a longer segment sets "unsupported"
    scratch_free(ws, s);
    return st;
}

}  // namespace isort

using namespace isort;

extern "C" {

isort_status isort_segmented(uint32_t* keys, uint32_t* vals, const uint64_t* seg_offsets, size_t nseg, int key_bits,
                             void* stream) {
    return segmented_entry(keys, vals, seg_offsets, nseg, key_bits, stream);
}

}  // extern "C"
