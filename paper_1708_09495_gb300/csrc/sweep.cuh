// The chunked count-sort round (reduce-then-scan), shared by the LSD radix
// rounds and the learned-bucket distribution passes. A round is generic over
// how a key's digit is computed (a digit function object):
//   RadixDigit   (key >> shift) & mask          -- Section 3's count-sort round
//   BucketDigit  a sub-field of the key's learned bucket (learned.cu)
#pragma once

#include "common.cuh"
#include "runtime.h"

#include <type_traits>

namespace isort {

// Digit = (key >> shift) & mask. Cheap: recomputed wherever needed.
struct RadixDigit {
    static constexpr bool kCheap = true;
    static constexpr bool kIndexed = false;  // the digit comes from the key (see sweep_tile)
    int shift;
    uint32_t mask;
    __device__ __forceinline__ size_t table_bytes() const { return 0; }
    __device__ __forceinline__ void setup(unsigned char*) {}
    template <typename K>
    __device__ __forceinline__ uint32_t digit(K k) const {
        return (uint32_t)(k >> shift) & mask;
    }
};

template <int THREADS>
__device__ void block_exclusive_scan(uint32_t* data, int count, uint32_t* s_warp) {
    constexpr int WARPS = THREADS / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ipt = (count + THREADS - 1) / THREADS;
    const int base = tid * ipt;
    uint32_t local = 0;
    for (int i = 0; i < ipt; ++i)
        if (base + i < count) local += data[base + i];
    uint32_t x = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(kFullMask, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < WARPS ? s_warp[lane] : 0;
        uint32_t z = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(kFullMask, z, d);
            if (lane >= d) z += y;
        }
        if (lane < WARPS) s_warp[lane] = z - w;
    }
    __syncthreads();
    uint32_t run = s_warp[warp] + x - local;
    for (int i = 0; i < ipt; ++i)
        if (base + i < count) {
            const uint32_t v = data[base + i];
            data[base + i] = run;
            run += v;
        }
    __syncthreads();
}

// ----------------------------------------------------------------------------
// Count-sort rounds by chunked reduce-then-scan.
//
// The round's input is cut into C contiguous chunks of whole tiles, one per
// persistent CTA. k_chunk_hist counts each chunk's digits (one read of the
// keys); k_chunk_scan turns the C x 2^rb counts into the first output position
// of every digit for every chunk (digit-major prefix, then chunk order);
// k_downsweep then streams its chunk tile by tile -- the next tile's keys and
// payloads copied into shared memory by the bulk-copy engine while the current
// tile is ranked -- and keeps one running output position per digit in shared
// memory. Chunks never wait for one another, so the round runs at the rate of
// the memory system; the price is the extra read of the keys per round.
// ----------------------------------------------------------------------------
constexpr int kChunkHistThreads = 512;

// parts CTAs share a chunk (each counts a contiguous part of it and adds its
// counts to the chunk's row, which starts zeroed); parts == 1 stores the row.
template <typename K>
__global__ void __launch_bounds__(kChunkHistThreads) k_chunk_hist(const K* __restrict__ keys, uint32_t n, int shift,
                                                                  int width, uint32_t chunk_keys, int nsub,
                                                                  uint32_t* __restrict__ hist,
                                                                  unsigned long long* key_or, int parts = 1) {
    extern __shared__ __align__(16) uint32_t s_h[];  // [nsub][bins]
    const int bins = 1 << width;
    const uint32_t mask = (uint32_t)bins - 1u;
    const int tid = threadIdx.x;
    for (int i = tid; i < nsub * bins; i += kChunkHistThreads) s_h[i] = 0;
    __syncthreads();
    uint32_t* my = s_h + (size_t)((tid >> 5) % nsub) * bins;
    const uint32_t chunk = blockIdx.x / (uint32_t)parts, part = blockIdx.x % (uint32_t)parts;
    const uint32_t part_keys = (chunk_keys / (uint32_t)parts + 3u) & ~3u;  // parts start 16-byte aligned
    const uint32_t c_lo = chunk * chunk_keys, c_hi = min(n, c_lo + chunk_keys);
    const uint32_t lo = min(c_hi, c_lo + part * part_keys);
    const uint32_t hi = part + 1 == (uint32_t)parts ? c_hi : min(c_hi, lo + part_keys);
    K acc = 0;
    if (lo < hi) {
        const K* base = keys + lo;
        const uint32_t cnt = hi - lo;
        constexpr int per_vec = 16 / sizeof(K);
        const bool vec = ((uintptr_t)base % 16) == 0;
        const uint32_t nvec = vec ? cnt / per_vec : 0;
        const uint4* v4 = reinterpret_cast<const uint4*>(base);
#pragma unroll 4
        for (uint32_t i = tid; i < nvec; i += kChunkHistThreads) {
            const uint4 v = __ldg(&v4[i]);
            if constexpr (sizeof(K) == 4) {
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    acc |= (K)w[e];
                    atomicAdd(&my[(w[e] >> shift) & mask], 1u);
                }
            } else if constexpr (sizeof(K) == 2) {
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint32_t x = (w[e >> 1] >> ((e & 1) * 16)) & 0xFFFFu;
                    acc |= (K)x;
                    atomicAdd(&my[(x >> shift) & mask], 1u);
                }
            } else {
                const K w[2] = {((K)v.y << 32) | v.x, ((K)v.w << 32) | v.z};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    acc |= w[e];
                    atomicAdd(&my[(uint32_t)(w[e] >> shift) & mask], 1u);
                }
            }
        }
        for (uint32_t i = nvec * per_vec + tid; i < cnt; i += kChunkHistThreads) {
            const K k = base[i];
            acc |= k;
            atomicAdd(&my[(uint32_t)(k >> shift) & mask], 1u);
        }
    }
    __syncthreads();
    uint32_t* out = hist + (size_t)chunk * bins;
    for (int d = tid; d < bins; d += kChunkHistThreads) {
        uint32_t sum = 0;
        for (int q = 0; q < nsub; ++q) sum += s_h[q * bins + d];
        if (parts == 1) out[d] = sum;
        else if (sum) atomicAdd(&out[d], sum);
    }
    if (key_or) {
        const unsigned long long o = (unsigned long long)acc;
        const uint32_t l = __reduce_or_sync(kFullMask, (uint32_t)o);
        const uint32_t h = __reduce_or_sync(kFullMask, (uint32_t)(o >> 32));
        if ((tid & 31) == 0 && (l | h)) atomicOr(key_or, ((unsigned long long)h << 32) | l);
    }
}

// chunk_off[c][d] = (keys with a smaller digit) + (keys with digit d in chunks < c).
// The 1024 threads form G = max(1, 1024 / bins) groups; group g owns a
// contiguous run of chunks, so each thread sums (and later prefixes) only
// C / G counts, with independent loads.
constexpr int kChunkScanThreads = 1024;

static __global__ void __launch_bounds__(kChunkScanThreads) k_chunk_scan(const uint32_t* __restrict__ hist, int chunks,
                                                                  int bins, uint32_t* __restrict__ chunk_off,
                                                                  const unsigned long long* key_or, int key_bits,
                                                                  int key_width, uint32_t* status,
                                                                  uint32_t* heavy = nullptr) {
    extern __shared__ __align__(16) uint32_t s_dyn[];  // [G][bins] group sums, then [bins] digit totals
    __shared__ uint32_t s_warp[kChunkScanThreads / 32];
    const int tid = threadIdx.x;
    const int G = bins >= kChunkScanThreads ? 1 : kChunkScanThreads / bins;
    const int per = (chunks + G - 1) / G;
    uint32_t* s_part = s_dyn;
    uint32_t* s_tot = s_dyn + (size_t)G * bins;
    for (int x = tid; x < G * bins; x += kChunkScanThreads) {
        const int g = x / bins, d = x % bins;
        const int c0 = g * per, c1 = min(chunks, c0 + per);
        uint32_t t = 0;
#pragma unroll 8
        for (int c = c0; c < c1; ++c) t += hist[(size_t)c * bins + d];
        s_part[x] = t;
    }
    __syncthreads();
    __shared__ uint32_t s_hmax[kChunkScanThreads / 32], s_hsum[kChunkScanThreads / 32];
    uint32_t hmax = 0, hsum = 0;
    for (int d = tid; d < bins; d += kChunkScanThreads) {
        uint32_t t = 0;
        for (int g = 0; g < G; ++g) t += s_part[g * bins + d];
        s_tot[d] = t;
        hmax = max(hmax, t);
        hsum += t;
    }
    hmax = __reduce_max_sync(kFullMask, hmax);
    hsum = __reduce_add_sync(kFullMask, hsum);
    if ((tid & 31) == 0) {
        s_hmax[tid >> 5] = hmax;
        s_hsum[tid >> 5] = hsum;
    }
    __syncthreads();
    block_exclusive_scan<kChunkScanThreads>(s_tot, bins, s_warp);
    if (heavy && tid == 0) {  // the round has a digit holding over four times its mean share of the keys
        uint32_t m = 0, n = 0;
        for (int w = 0; w < kChunkScanThreads / 32; ++w) {
            m = max(m, s_hmax[w]);
            n += s_hsum[w];
        }
        *heavy = (unsigned long long)m * (unsigned)bins > 4ull * n ? 1u : 0u;
    }
    for (int x = tid; x < G * bins; x += kChunkScanThreads) {
        const int g = x / bins, d = x % bins;
        uint32_t run = s_tot[d];
        for (int q = 0; q < g; ++q) run += s_part[q * bins + d];
        const int c0 = g * per, c1 = min(chunks, c0 + per);
#pragma unroll 8
        for (int c = c0; c < c1; ++c) {
            const uint32_t h = hist[(size_t)c * bins + d];
            chunk_off[(size_t)c * bins + d] = run;
            run += h;
        }
    }
    if (key_or && tid == 0 && key_bits < key_width && ((*key_or) >> key_bits)) set_status(status, kStatKeyRange);
}

struct SweepArgs {
    const void* keys_in;
    const uint32_t* vals_in;
    void* keys_out;
    uint32_t* vals_out;
    uint32_t n;
    int shift;
    int width;
    int bins;
    const uint32_t* chunk_off;  // [chunks][bins]
    uint32_t chunk_tiles;
    uint32_t num_tiles;
    uint32_t* status;
    uint64_t limit_ns;
    int use_bulk;
    // when set: the launch runs only if (*heavy != 0) == (run_if_heavy != 0)
    // (two forms of one round launched back to back; the digit counts pick one)
    const uint32_t* heavy = nullptr;
    int run_if_heavy = 0;
};

// Whether this launch of a round is the form the round's digit counts picked
// (uniform over the grid).
__device__ __forceinline__ bool round_form_selected(const SweepArgs& a) {
    return a.heavy == nullptr || ((*a.heavy != 0u) == (a.run_if_heavy != 0));
}

template <typename K, bool VALS, int THREADS, int ITEMS>
struct SweepCfg {
    static constexpr int kWarps = THREADS / 32;
    static constexpr int kTile = THREADS * ITEMS;
    static constexpr size_t kBufBytes = (size_t)kTile * sizeof(K) + (VALS ? (size_t)kTile * 4 : 0);
    // with a digit function that is not cheap: staged digits and its tables
    static size_t smem_bytes(int bins, bool cheap, size_t table_bytes) {
        return align_up(smem_bytes(bins) + (cheap ? 0 : align_up((size_t)kTile * 2, 16)) + table_bytes, 128);
    }
    static size_t smem_bytes(int bins) {
        size_t b = 2 * kBufBytes;
        b += align_up((size_t)kWarps * bins * 2, 16);  // per-warp digit counts (u16)
        b += (size_t)kWarps * bins * 4;                // per-warp peer masks
        b += (size_t)bins * 4 * 4;                     // tile digit starts, totals, running positions, deltas
        b += 2 * 8 + (size_t)kWarps * 4 + 16;          // mbarriers, warp sums, tile flags
        return align_up(b, 128);
    }
};

// One tile of a chunked round: rank, stage by digit, write out, advance the
// chunk's running positions. FULL: the tile holds TILE keys (no bounds tests
// on the tile's own indices). WIDTH > 0: the digit width at compile time.
//
// Ranking: peers (the lanes of a warp holding the same digit) come from a
// per-warp mask word per digit: every lane ORs its lane bit into its digit's
// word and, after a warp barrier, reads the word back. The result does not
// depend on the order in which the atomics land. A per-warp 16-bit count per
// digit carries the rank across the warp's items (input order: stable).
template <typename K, bool VALS, int THREADS, int ITEMS, int WIDTH, bool FULL, typename DF>
__device__ __forceinline__ void sweep_tile(const SweepArgs& a, const DF& df, K* s_keys, uint32_t* s_vals,
                                           uint16_t* s_cnt, uint32_t* s_match, uint32_t* s_start, uint32_t* s_tot,
                                           uint32_t* s_run, uint32_t* s_delta, uint32_t* s_warp_scan,
                                           uint16_t* s_dig, uint32_t* s_skew, int par, uint32_t tile_base,
                                           uint32_t tile_n) {
    constexpr int WARPS = THREADS / 32;
    constexpr int TILE = THREADS * ITEMS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bins = WIDTH > 0 ? (1 << WIDTH) : a.bins;
    // the previous tile had a digit over four times its mean count: look for
    // warps whose keys share one digit (flag set in the previous tile's
    // bookkeeping; this tile's flag is cleared here, before its barrier)
    const bool skew = s_skew[par ^ 1] != 0u;
    if (tid == 0) s_skew[par] = 0u;
    uint16_t* my_cnt = s_cnt + warp * bins;
    uint32_t* my_match = s_match + warp * bins;
    const uint32_t lt = lanemask_lt();
    K kreg[ITEMS];
    uint32_t vreg[ITEMS];
    uint32_t rank[ITEMS];
    uint32_t dreg[ITEMS];
    // the ranking loop in two compiled forms (the check below only where a
    // tile before showed a heavy digit)
    // an indexed digit function reads a 16-bit value stored per input position
    // (the value moves with its key; the digit is part of it): all of a
    // thread's values are loaded before the ranking starts
    uint32_t auxv[ITEMS];
    if constexpr (DF::kIndexed) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t j = (uint32_t)(warp * ITEMS * 32 + i * 32 + lane);
            auxv[i] = (FULL || j < tile_n) ? df.load(tile_base + j) : 0u;
        }
    }
    auto rank_items = [&](auto skew_c) {
        constexpr bool SKEW = decltype(skew_c)::value;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t j = (uint32_t)(warp * ITEMS * 32 + i * 32 + lane);
            const bool valid = FULL || j < tile_n;
            const K k = valid ? s_keys[j] : (K)0;
            kreg[i] = k;
            if constexpr (VALS) vreg[i] = valid ? s_vals[j] : 0u;
            uint32_t d, aux = 0;
            if constexpr (DF::kIndexed) {
                aux = auxv[i];
                d = valid ? df.digit_of(aux) : 0u;
            } else {
                d = valid ? df.digit(k) : 0u;
            }
            // a warp whose 32 keys share one digit (runs of a repeated key) skips
            // the mask atomics, which would all land on one word and serialize
            bool uni = false;
            if constexpr (SKEW) {
                const uint32_t d0 = __shfl_sync(kFullMask, d, 0);  // every lane takes part (also invalid ones)
                uni = __all_sync(kFullMask, valid && d == d0);
            }
            if (valid && !uni) atomicOr(&my_match[d], 1u << lane);
            __syncwarp();
            const uint32_t peers = uni ? kFullMask : (valid ? my_match[d] : 0u);
            const uint32_t c = valid ? (uint32_t)my_cnt[d] : 0u;
            __syncwarp();
            rank[i] = c + (uint32_t)__popc(peers & lt);
            dreg[i] = DF::kIndexed ? aux : d;
            if (valid && (peers >> lane) == 1u) {  // the group's highest lane
                my_cnt[d] = (uint16_t)(c + (uint32_t)__popc(peers));
                if (!uni) my_match[d] = 0u;
            }
            __syncwarp();
        }
    };
    if (skew) rank_items(std::true_type{});  // uniform over the CTA
    else rank_items(std::false_type{});
    __syncthreads();
    for (int d = tid; d < bins; d += THREADS) {
        uint32_t sum = 0;
#pragma unroll 4
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t c = s_cnt[w * bins + d];
            s_cnt[w * bins + d] = (uint16_t)sum;
            sum += c;
        }
        s_start[d] = sum;
        s_tot[d] = sum;
        if (sum * (uint32_t)bins > 4u * (uint32_t)TILE) s_skew[par] = 1u;
    }
    __syncthreads();
    block_exclusive_scan<THREADS>(s_start, bins, s_warp_scan);
    for (int d = tid; d < bins; d += THREADS) s_delta[d] = s_run[d] - s_start[d];
    // stage keys by digit (over the tile's own buffer: its keys are in registers)
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = (uint32_t)(warp * ITEMS * 32 + i * 32 + lane);
        if (FULL || j < tile_n) {
            uint32_t d = dreg[i];
            if constexpr (DF::kIndexed) d = df.digit_of(d);
            const uint32_t pos = s_start[d] + my_cnt[d] + rank[i];
            if (pos < (uint32_t)TILE) {
                s_keys[pos] = kreg[i];
                if constexpr (VALS) s_vals[pos] = vreg[i];
                if constexpr (!DF::kCheap) s_dig[pos] = (uint16_t)dreg[i];  // the digit, or the indexed value
            }
        }
    }
    __syncthreads();
    K* keys_out = static_cast<K*>(a.keys_out);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = (uint32_t)(tid + i * THREADS);
        if (FULL || j < tile_n) {
            const K k = s_keys[j];
            uint32_t sd = 0, d;
            if constexpr (DF::kCheap) {
                d = df.digit(k);
            } else {
                sd = s_dig[j];
                if constexpr (DF::kIndexed) d = df.digit_of(sd);
                else d = sd;
            }
            const uint32_t dst = s_delta[d] + j;
            if (dst < a.n) {
                keys_out[dst] = k;
                if constexpr (VALS) a.vals_out[dst] = s_vals[j];
                if constexpr (DF::kIndexed) df.store(dst, sd);
            } else {
                set_status(a.status, kStatBounds);
            }
        }
    }
    __syncthreads();
    for (int d = tid; d < bins; d += THREADS) s_run[d] += s_tot[d];
    for (int i = tid; i < WARPS * bins; i += THREADS) s_cnt[i] = 0;
    __syncthreads();
}

template <typename K, bool VALS, int THREADS, int ITEMS, int WIDTH, typename DF>
__global__ void __launch_bounds__(THREADS, (1024 / THREADS) > 0 ? (1024 / THREADS) : 1)
    k_downsweep(SweepArgs a, DF df) {
    if (!round_form_selected(a)) return;
    using Cfg = SweepCfg<K, VALS, THREADS, ITEMS>;
    constexpr int WARPS = Cfg::kWarps;
    constexpr int TILE = Cfg::kTile;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x;
    const int bins = a.bins;
    unsigned char* buf0 = smem;
    uint16_t* s_cnt = reinterpret_cast<uint16_t*>(smem + 2 * Cfg::kBufBytes);
    uint32_t* s_match = reinterpret_cast<uint32_t*>(smem + 2 * Cfg::kBufBytes +
                                                    align_up_dev((size_t)WARPS * bins * 2, 16));
    uint32_t* s_start = s_match + (size_t)WARPS * bins;
    uint32_t* s_tot = s_start + bins;
    uint32_t* s_run = s_tot + bins;
    uint32_t* s_delta = s_run + bins;
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_delta + bins);
    uint32_t* s_warp_scan = reinterpret_cast<uint32_t*>(bars + 2);
    uint32_t* s_skew = s_warp_scan + WARPS;  // two tile flags (the words after the scan's)
    uint16_t* s_dig = reinterpret_cast<uint16_t*>(s_warp_scan + WARPS + 4);  // staged digits (costly digits only)
    unsigned char* s_tab = reinterpret_cast<unsigned char*>(s_dig) + (DF::kCheap ? 0 : align_up_dev((size_t)TILE * 2, 16));
    // the layout must fit the launch's shared memory (uniform check)
    if ((size_t)(s_tab + df.table_bytes() - smem) > dynamic_smem_size()) {
        if (threadIdx.x == 0) set_status(a.status, kStatBounds);
        return;
    }

    // an earlier step failed: leave (one read, shared by the CTA, so that all
    // of its threads leave together)
    if (__syncthreads_or(tid == 0 && *(volatile uint32_t*)a.status != 0)) return;
    const uint32_t t_begin = blockIdx.x * a.chunk_tiles;
    const uint32_t t_end = min(a.num_tiles, t_begin + a.chunk_tiles);
    if (t_begin >= t_end) return;
    const K* keys_in = static_cast<const K*>(a.keys_in);

    for (int i = tid; i < WARPS * bins; i += THREADS) {
        s_cnt[i] = 0;
        s_match[i] = 0;
    }
    for (int d = tid; d < bins; d += THREADS) s_run[d] = a.chunk_off[(size_t)blockIdx.x * bins + d];
    if (tid < 2) s_skew[tid] = 0u;
    df.setup(s_tab);  // copies the digit function's tables into shared memory
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto full_bulk_tile = [&](uint32_t t) -> bool { return a.use_bulk && (size_t)(t + 1) * TILE <= a.n; };
    auto issue_tile = [&](uint32_t t, int b) {
        unsigned char* dst = buf0 + (size_t)b * Cfg::kBufBytes;
        constexpr uint32_t kb = TILE * sizeof(K);
        constexpr uint32_t vb = VALS ? TILE * 4 : 0;
        mbar_arrive_expect_tx(&bars[b], kb + vb);
        bulk_load(dst, keys_in + (size_t)t * TILE, kb, &bars[b]);
        if constexpr (VALS) bulk_load(dst + kb, a.vals_in + (size_t)t * TILE, vb, &bars[b]);
    };
    if (tid == 0 && full_bulk_tile(t_begin)) issue_tile(t_begin, 0);
    uint32_t phase = 0u;
    int b = 0;
    for (uint32_t tile = t_begin; tile < t_end; ++tile, b ^= 1) {
        if (tid == 0 && tile + 1 < t_end && full_bulk_tile(tile + 1)) {
            fence_proxy_async_smem();
            issue_tile(tile + 1, b ^ 1);
        }
        K* s_keys = reinterpret_cast<K*>(buf0 + (size_t)b * Cfg::kBufBytes);
        uint32_t* s_vals = reinterpret_cast<uint32_t*>(buf0 + (size_t)b * Cfg::kBufBytes + (size_t)TILE * sizeof(K));
        const uint32_t tile_base = tile * (uint32_t)TILE;
        const uint32_t tile_n = min((uint32_t)TILE, a.n - tile_base);
        bool ok = true;
        if (full_bulk_tile(tile)) {
            ok = mbar_wait_bounded(&bars[b], (phase >> b) & 1u, a.limit_ns);
            phase ^= 1u << b;
        } else {
            for (uint32_t j = tid; j < tile_n; j += THREADS) {
                s_keys[j] = keys_in[tile_base + j];
                if constexpr (VALS) s_vals[j] = a.vals_in[tile_base + j];
            }
        }
        if (__syncthreads_or(!ok)) {
            // a bulk copy never completed: record it, wait (bounded) for the
            // copy issued into the other buffer, and stop
            if (tid == 0) set_status(a.status, kStatTimeout);
            if (tile + 1 < t_end && full_bulk_tile(tile + 1))
                mbar_wait_bounded(&bars[b ^ 1], (phase >> (b ^ 1)) & 1u, a.limit_ns);
            return;
        }
        if (tile_n == (uint32_t)TILE)
            sweep_tile<K, VALS, THREADS, ITEMS, WIDTH, true>(a, df, s_keys, s_vals, s_cnt, s_match, s_start, s_tot,
                                                             s_run, s_delta, s_warp_scan, s_dig, s_skew, b, tile_base,
                                                             TILE);
        else
            sweep_tile<K, VALS, THREADS, ITEMS, WIDTH, false>(a, df, s_keys, s_vals, s_cnt, s_match, s_start, s_tot,
                                                              s_run, s_delta, s_warp_scan, s_dig, s_skew, b, tile_base,
                                                              tile_n);
    }
}

}  // namespace isort

namespace isort {

// ---------------------------------------------------------------- half-warp ranking
//
// A variant of the chunked round for 8-bit digits (512 threads, 8 keys per
// thread) whose ranking state is ONE 32-bit word per (half-warp, digit): bits
// [16, 32) count the digit's keys the half-warp has seen, bits [0, 16) collect
// the lanes holding the digit in the current item. A key costs one atomicAdd,
// one read and (for the group's highest lane) one write, against five
// accesses with separate count and peer-mask arrays; after ranking the same
// words hold each (half-warp, digit)'s output base, so staging reads one word.
// Each half-warp owns 128 consecutive keys of the tile (8 items of 16 keys);
// blocks sit 144 elements apart in shared memory so that the two half-warps of
// a warp read disjoint banks.
constexpr int kHwBins = 256;

// THREADS x ITEMS keys per tile; THREADS / 16 half-warps each own 16 x ITEMS
// consecutive keys (ITEMS even, so that the 16-element pitch shift puts the
// two half-warps of a warp on disjoint banks); counts per half-warp and digit
// stay below 2^16.
template <typename K, bool VALS, int THREADS, int ITEMS>
struct HwCfg {
    static_assert(THREADS == 256 || THREADS == 512, "one or two threads per digit");
    static_assert(ITEMS % 2 == 0 && 16 * ITEMS < 65536, "pitch and count width");
    static constexpr int kTile = THREADS * ITEMS;
    static constexpr int kGroups = THREADS / 16;
    static constexpr int kBlock = 16 * ITEMS;
    static constexpr int kPitch = kBlock + 16;
    static constexpr int kHalves = THREADS / kHwBins;  // threads per digit in the per-digit steps
    static constexpr size_t kKeyBytes = (size_t)kGroups * kPitch * sizeof(K);
    static constexpr size_t kValBytes = VALS ? (size_t)kGroups * kPitch * 4 : 0;
    static constexpr size_t kBufBytes = kKeyBytes + kValBytes;
    static size_t smem_bytes() {
        return 2 * kBufBytes + (size_t)kGroups * kHwBins * 4  // buffers, ranking words
               + (size_t)kHwBins * 4 * 6                     // start, tot, run, delta, half totals (2)
               + 2 * 8 + 32 * 4 + 16;                        // mbarriers, scan scratch
    }
};

template <typename K, bool VALS, int THREADS, int ITEMS, bool FULL>
__device__ __forceinline__ void hw_tile(const SweepArgs& a, K* s_keys, uint32_t* s_vals, uint32_t* s_word,
                                       uint32_t* s_start, uint32_t* s_tot, uint32_t* s_run, uint32_t* s_delta,
                                       uint32_t* s_half, uint32_t* s_warp_scan, uint32_t tile_n) {
    using Cfg = HwCfg<K, VALS, THREADS, ITEMS>;
    constexpr int kTile = Cfg::kTile, kBlock = Cfg::kBlock, kPitch = Cfg::kPitch, kGroups = Cfg::kGroups;
    constexpr int kPerHalf = kGroups / Cfg::kHalves;
    const int tid = threadIdx.x, lane = tid & 31, hw = tid >> 4, l16 = lane & 15;
    const int shift = a.shift;
    const uint32_t dmask = (uint32_t)a.bins - 1u;  // digits of up to 8 bits
    uint32_t* my_w = s_word + hw * kHwBins;
    const uint32_t bit = 1u << l16, lt16 = bit - 1u;
    K kreg[ITEMS];
    uint32_t vreg[ITEMS];
    uint32_t rank[ITEMS];
    uint32_t dreg[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = (uint32_t)(hw * kBlock + i * 16 + l16);  // position in the tile (input order)
        const bool valid = FULL || j < tile_n;
        const int p = hw * kPitch + i * 16 + l16;
        const K k = valid ? s_keys[p] : (K)0;
        kreg[i] = k;
        if constexpr (VALS) vreg[i] = valid ? s_vals[p] : 0u;
        const uint32_t d = valid ? (uint32_t)(k >> shift) & dmask : 0u;
        if (valid) atomicAdd(&my_w[d], 0x10000u | bit);
        __syncwarp();
        const uint32_t x = valid ? my_w[d] : 0u;
        const uint32_t m = x & 0xFFFFu;
        rank[i] = (x >> 16) - (uint32_t)__popc(m) + (uint32_t)__popc(m & lt16);
        dreg[i] = d;
        __syncwarp();
        if (valid && (m >> l16) == 1u) my_w[d] = x & 0xFFFF0000u;  // the group's highest lane clears the lanes
        __syncwarp();
    }
    __syncthreads();
    {  // per digit: counts -> exclusive prefixes over half-warps, in two halves of 16
        const int half = tid >> 8, d = tid & (kHwBins - 1);
        uint32_t sum = 0;
#pragma unroll 4
        for (int h = half * kPerHalf; h < half * kPerHalf + kPerHalf; ++h) {
            const uint32_t c = s_word[h * kHwBins + d] >> 16;
            s_word[h * kHwBins + d] = sum;
            sum += c;
        }
        s_half[half * kHwBins + d] = sum;
    }
    __syncthreads();
    if (tid < kHwBins) {
        const uint32_t t = Cfg::kHalves == 2 ? s_half[tid] + s_half[kHwBins + tid] : s_half[tid];
        s_tot[tid] = t;
        s_start[tid] = t;
    }
    __syncthreads();
    block_exclusive_scan<THREADS>(s_start, kHwBins, s_warp_scan);
    {  // bases of every (half-warp, digit); the round's output offsets
        const int half = tid >> 8, d = tid & (kHwBins - 1);
        const uint32_t add = s_start[d] + (half ? s_half[d] : 0u);
#pragma unroll 4
        for (int h = half * kPerHalf; h < half * kPerHalf + kPerHalf; ++h) s_word[h * kHwBins + d] += add;
        if (tid < kHwBins) s_delta[tid] = s_run[tid] - s_start[tid];
    }
    __syncthreads();
    // stage by digit (linear, over the tile's own buffer: its keys are in registers)
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = (uint32_t)(hw * kBlock + i * 16 + l16);
        if (FULL || j < tile_n) {
            const uint32_t pos = my_w[dreg[i]] + rank[i];
            if (pos < (uint32_t)kTile) {
                s_keys[pos] = kreg[i];
                if constexpr (VALS) s_vals[pos] = vreg[i];
            }
        }
    }
    __syncthreads();
    K* keys_out = static_cast<K*>(a.keys_out);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = (uint32_t)(tid + i * THREADS);
        if (FULL || j < tile_n) {
            const K k = s_keys[j];
            const uint32_t d = (uint32_t)(k >> shift) & dmask;
            const uint32_t dst = s_delta[d] + j;
            if (dst < a.n) {
                keys_out[dst] = k;
                if constexpr (VALS) a.vals_out[dst] = s_vals[j];
            } else {
                set_status(a.status, kStatBounds);
            }
        }
    }
    {  // clear the ranking words for the next tile (16-byte stores)
        uint4* w4 = reinterpret_cast<uint4*>(s_word);
        for (int i = tid; i < kGroups * kHwBins / 4; i += THREADS) w4[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid < kHwBins) s_run[tid] += s_tot[tid];
    __syncthreads();
}

template <typename K, bool VALS, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, (THREADS == 512 && ITEMS <= 8) || THREADS == 256 ? 2 : 1)
    k_downsweep_hw(SweepArgs a) {
    if (!round_form_selected(a)) return;
    using Cfg = HwCfg<K, VALS, THREADS, ITEMS>;
    constexpr int kTile = Cfg::kTile, kBlock = Cfg::kBlock, kPitch = Cfg::kPitch, kGroups = Cfg::kGroups;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned char* buf0 = smem;
    uint32_t* s_word = reinterpret_cast<uint32_t*>(smem + 2 * Cfg::kBufBytes);
    uint32_t* s_start = s_word + kGroups * kHwBins;
    uint32_t* s_tot = s_start + kHwBins;
    uint32_t* s_run = s_tot + kHwBins;
    uint32_t* s_delta = s_run + kHwBins;
    uint32_t* s_half = s_delta + kHwBins;
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_half + 2 * kHwBins);
    uint32_t* s_warp_scan = reinterpret_cast<uint32_t*>(bars + 2);
    if ((size_t)(reinterpret_cast<unsigned char*>(s_warp_scan + 32) - smem) > dynamic_smem_size()) {
        if (tid == 0) set_status(a.status, kStatBounds);
        return;
    }
    if (__syncthreads_or(tid == 0 && *(volatile uint32_t*)a.status != 0)) return;
    const uint32_t t_begin = blockIdx.x * a.chunk_tiles;
    const uint32_t t_end = min(a.num_tiles, t_begin + a.chunk_tiles);
    if (t_begin >= t_end) return;
    const K* keys_in = static_cast<const K*>(a.keys_in);

    for (int i = tid; i < kGroups * kHwBins; i += THREADS) s_word[i] = 0u;
    for (int d = tid; d < kHwBins; d += THREADS)
        s_run[d] = d < a.bins ? a.chunk_off[(size_t)blockIdx.x * a.bins + d] : 0u;  // [chunks][bins]
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto full_bulk_tile = [&](uint32_t t) -> bool { return a.use_bulk && (size_t)(t + 1) * kTile <= a.n; };
    // warp 0: lane 0 announces the bytes, then lane l copies half-warp blocks l, l + 32, ...
    auto issue_tile = [&](uint32_t t, int b) {
        unsigned char* dst = buf0 + (size_t)b * Cfg::kBufBytes;
        constexpr uint32_t kb = kBlock * sizeof(K);
        if (lane == 0) mbar_arrive_expect_tx(&bars[b], kTile * (uint32_t)sizeof(K) + (VALS ? kTile * 4u : 0u));
        __syncwarp();
        fence_proxy_async_smem();
        for (int g = lane; g < kGroups; g += 32) {
            bulk_load(dst + (size_t)g * kPitch * sizeof(K), keys_in + (size_t)t * kTile + (size_t)g * kBlock, kb,
                      &bars[b]);
            if constexpr (VALS)
                bulk_load(dst + Cfg::kKeyBytes + (size_t)g * kPitch * 4,
                          a.vals_in + (size_t)t * kTile + (size_t)g * kBlock, kBlock * 4, &bars[b]);
        }
    };
    if (warp == 0 && full_bulk_tile(t_begin)) issue_tile(t_begin, 0);
    uint32_t phase = 0u;
    int b = 0;
    for (uint32_t tile = t_begin; tile < t_end; ++tile, b ^= 1) {
        if (warp == 0 && tile + 1 < t_end && full_bulk_tile(tile + 1)) issue_tile(tile + 1, b ^ 1);
        K* s_keys = reinterpret_cast<K*>(buf0 + (size_t)b * Cfg::kBufBytes);
        uint32_t* s_vals = reinterpret_cast<uint32_t*>(buf0 + (size_t)b * Cfg::kBufBytes + Cfg::kKeyBytes);
        const uint32_t tile_base = tile * (uint32_t)kTile;
        const uint32_t tile_n = min((uint32_t)kTile, a.n - tile_base);
        bool ok = true;
        if (full_bulk_tile(tile)) {
            ok = mbar_wait_bounded(&bars[b], (phase >> b) & 1u, a.limit_ns);
            phase ^= 1u << b;
        } else {
            for (uint32_t j = tid; j < tile_n; j += THREADS) {
                const uint32_t p = (j / kBlock) * kPitch + (j % kBlock);
                s_keys[p] = keys_in[tile_base + j];
                if constexpr (VALS) s_vals[p] = a.vals_in[tile_base + j];
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) set_status(a.status, kStatTimeout);
            if (tile + 1 < t_end && full_bulk_tile(tile + 1))
                mbar_wait_bounded(&bars[b ^ 1], (phase >> (b ^ 1)) & 1u, a.limit_ns);
            return;
        }
        if (tile_n == (uint32_t)kTile)
            hw_tile<K, VALS, THREADS, ITEMS, true>(a, s_keys, s_vals, s_word, s_start, s_tot, s_run, s_delta, s_half,
                                                   s_warp_scan, kTile);
        else
            hw_tile<K, VALS, THREADS, ITEMS, false>(a, s_keys, s_vals, s_word, s_start, s_tot, s_run, s_delta, s_half,
                                                    s_warp_scan, tile_n);
    }
}

}  // namespace isort
