// LSD radix sort on sm_103a: the count-sort rounds of Gerbessiotis,
// arXiv:1708.09495, Section 3 ("Serial radix-r radix-sort", eq. Ts; "Parallel
// radix-r radix-sort", eq. Tp).
//
// The paper's round reads its input twice (count, then output) and writes it
// once (3Ng per round). The default rounds are the chunked reduce-then-scan
// rounds (rts.cu, kernels in sweep.cuh: per-chunk counts, chunk offsets, rank
// and scatter). This file holds the entry points and the single-pass rounds,
// taken for digits whose per-tile tables do not fit the chunked round, by the
// allocation-free entry point, and by the stalled-tile fault test:
//   k_digit_hist  one streaming read of the keys (bulk copies into shared
//                 memory, 128-bit shared loads) counts the digits of EVERY
//                 round at once, and ORs the keys for the key-range check;
//   k_digit_scan  turns each round's counts into exclusive global offsets (the
//                 paper's counts scatter/gather, 2rpg, becomes a table in HBM);
//   k_onesweep    one launch per round: persistent CTAs take tiles in order,
//                 prefetch the next tile with bulk copies, rank each key among
//                 equal digits of its warp with one ballot per digit bit
//                 (input order, so the round is stable), publish the tile's
//                 digit counts and resolve the tile's global offsets with a
//                 bounded decoupled look-back over earlier tiles, then stage
//                 keys by digit in shared memory and write them out in runs.
// So each round costs one read and one write of the keys (and payloads).
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "runtime.h"
#include "sweep.cuh"
#include "tune.h"

namespace isort {

static Tune load_tune() {
    Tune t;
    const char* e = getenv("ISORT_TUNE");
    if (!e) return t;
    char key[32];
    int val;
    const char* p = e;
    while (*p) {
        int used = 0;
        if (sscanf(p, "%31[a-z_0-9]=%d%n", key, &val, &used) != 2 || used == 0) break;
        if (!strcmp(key, "hist_agg")) t.hist_agg = val;
        else if (!strcmp(key, "rank")) t.rank_mode = val;
        else if (!strcmp(key, "shape8")) t.shape_small = val;
        else if (!strcmp(key, "shape11")) t.shape_large = val;
        else if (!strcmp(key, "algo")) t.algo = val;
        else if (!strcmp(key, "sweep8")) t.sweep_small = val;
        else if (!strcmp(key, "sweep11")) t.sweep_large = val;
        else if (!strcmp(key, "sweepk")) t.sweep_keys = val;
        else if (!strcmp(key, "heavy")) t.heavy = val;
        else if (!strcmp(key, "split")) t.split = val;
        else if (!strcmp(key, "copy_pieces")) t.copy_pieces = val;
        else if (!strcmp(key, "small")) t.small = val;
        else if (!strcmp(key, "fine")) t.fine = val;
        p += used;
        if (*p == ',') ++p;
    }
    if (t.sweep_small < 0 || t.sweep_small >= 6) t.sweep_small = 4;
    if (t.sweep_keys < 0 || t.sweep_keys >= 6) t.sweep_keys = 3;
    if (t.sweep_large < 0 || t.sweep_large >= 4) t.sweep_large = 2;
    if (t.split < 8 || t.split > 16) t.split = 8;
    auto built = [](int sh) { return sh == 0 || sh == 1 || sh == 4 || sh == 9 || sh == 10; };
    if (!built(t.shape_small)) t.shape_small = 4;
    if (!built(t.shape_large)) t.shape_large = 1;
    return t;
}

const Tune& tune() {
    static const Tune t = load_tune();
    return t;
}

// ----------------------------------------------------------------------------
// Digit histogram of all rounds (one read).
// ----------------------------------------------------------------------------
constexpr int kHistThreads = 512;
constexpr int kHistStages = 3;
constexpr uint32_t kHistChunkBytes = 16384;

struct HistArgs {
    const void* keys;
    size_t n;
    int shift0;                      // first digit starts at this bit
    int radix_bits;
    int key_bits;                    // digits cover bits [shift0, shift0 + key_bits)
    int rounds;
    uint32_t* hist;                  // [rounds][2^radix_bits]
    unsigned long long* key_or;      // OR of all keys
    uint32_t* status;
    uint64_t limit_ns;
    int use_bulk;                    // keys 16-byte aligned
};

template <typename K>
__device__ __forceinline__ void hist_count_key(K k, uint32_t* s_hist, int shift0, int rounds, int rb, int key_bits,
                                               int bins) {
    for (int d = 0; d < rounds; ++d) {
        const int sh = d * rb;
        const int w = min(rb, key_bits - sh);
        const uint32_t dig = (uint32_t)(k >> (shift0 + sh)) & ((1u << w) - 1u);
        atomicAdd(&s_hist[d * bins + dig], 1u);
    }
}

// Full-warp form: equal digits in a warp are merged with one match-any vote,
// so one lane adds the group's size (heavy duplicates cost one atomic).
template <typename K>
__device__ __forceinline__ void hist_count_key_warp(K k, uint32_t* s_hist, int shift0, int rounds, int rb,
                                                    int key_bits, int bins) {
    for (int d = 0; d < rounds; ++d) {
        const int sh = d * rb;
        const int w = min(rb, key_bits - sh);
        const uint32_t dig = (uint32_t)(k >> (shift0 + sh)) & ((1u << w) - 1u);
        const uint32_t peers = __match_any_sync(kFullMask, dig);
        if ((peers & lanemask_lt()) == 0) atomicAdd(&s_hist[d * bins + dig], (uint32_t)__popc(peers));
    }
}

// Compile-time form for the common (radix bits, key bits) pairs: the digit
// shifts and masks fold into constants.
template <typename K, int RB, int KB>
__device__ __forceinline__ void hist_count_key_c(K k, uint32_t* s_hist) {
    constexpr int R = (KB + RB - 1) / RB;
#pragma unroll
    for (int d = 0; d < R; ++d) {
        const int w = (KB - d * RB) < RB ? (KB - d * RB) : RB;
        const uint32_t dig = (uint32_t)(k >> (d * RB)) & ((1u << w) - 1u);
        atomicAdd(&s_hist[d * (1 << RB) + dig], 1u);
    }
}

// RB, KB > 0: compile-time digit layout (shift0 must be 0); 0: runtime.
template <typename K, bool AGG, int RB = 0, int KB = 0>
__global__ void __launch_bounds__(kHistThreads) k_digit_hist(HistArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int bins = 1 << a.radix_bits;
    const int nh = a.rounds * bins;
    uint32_t* s_hist = reinterpret_cast<uint32_t*>(smem + kHistStages * kHistChunkBytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_hist + align_up_dev(nh, 2));
    const K* keys = static_cast<const K*>(a.keys);
    const int tid = threadIdx.x;
    if ((size_t)(reinterpret_cast<unsigned char*>(bars + kHistStages) - smem) > dynamic_smem_size()) {
        if (tid == 0) set_status(a.status, kStatBounds);
        return;
    }

    for (int i = tid; i < nh; i += kHistThreads) s_hist[i] = 0;
    if (tid == 0) {
        for (int s = 0; s < kHistStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    constexpr uint32_t kpc = kHistChunkBytes / sizeof(K);  // keys per chunk
    const size_t nchunks = a.use_bulk ? a.n / kpc : 0;
    const size_t G = gridDim.x;
    K acc = 0;

    if (tid == 0) {
        for (int s = 0; s < kHistStages; ++s) {
            size_t c = blockIdx.x + (size_t)s * G;
            if (c < nchunks) {
                mbar_arrive_expect_tx(&bars[s], kHistChunkBytes);
                bulk_load(smem + s * kHistChunkBytes, keys + c * kpc, kHistChunkBytes, &bars[s]);
            }
        }
    }
    size_t k = 0;
    for (;; ++k) {
        const size_t c = blockIdx.x + k * G;
        if (c >= nchunks) break;
        const int s = (int)(k % kHistStages);
        const uint32_t parity = (uint32_t)((k / kHistStages) & 1);
        const bool ok = mbar_wait_bounded(&bars[s], parity, a.limit_ns);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) set_status(a.status, kStatTimeout);
            // wait (bounded) for copies this CTA still has in flight
            for (size_t q = k; q < k + kHistStages; ++q) {
                const size_t cq = blockIdx.x + q * G;
                if (cq >= nchunks) break;
                mbar_wait_bounded(&bars[q % kHistStages], (uint32_t)((q / kHistStages) & 1), a.limit_ns);
            }
            return;
        }
        const uint4* v4 = reinterpret_cast<const uint4*>(smem + s * kHistChunkBytes);
        constexpr int nv = kHistChunkBytes / 16;
#pragma unroll
        for (int i = tid; i < nv; i += kHistThreads) {
            const uint4 v = v4[i];
            if constexpr (sizeof(K) == 4) {
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    acc |= (K)w[e];
                    if constexpr (RB > 0)
                        hist_count_key_c<K, RB, KB>((K)w[e], s_hist);
                    else if constexpr (AGG)
                        hist_count_key_warp<K>((K)w[e], s_hist, a.shift0, a.rounds, a.radix_bits, a.key_bits, bins);
                    else
                        hist_count_key<K>((K)w[e], s_hist, a.shift0, a.rounds, a.radix_bits, a.key_bits, bins);
                }
            } else {
                const K w[2] = {((K)v.y << 32) | v.x, ((K)v.w << 32) | v.z};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    acc |= w[e];
                    if constexpr (RB > 0)
                        hist_count_key_c<K, RB, KB>(w[e], s_hist);
                    else if constexpr (AGG)
                        hist_count_key_warp<K>(w[e], s_hist, a.shift0, a.rounds, a.radix_bits, a.key_bits, bins);
                    else
                        hist_count_key<K>(w[e], s_hist, a.shift0, a.rounds, a.radix_bits, a.key_bits, bins);
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            const size_t cn = c + (size_t)kHistStages * G;
            if (cn < nchunks) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bars[s], kHistChunkBytes);
                bulk_load(smem + s * kHistChunkBytes, keys + cn * kpc, kHistChunkBytes, &bars[s]);
            }
        }
    }
    // the tail not covered by whole chunks (everything if keys are unaligned)
    for (size_t i = nchunks * kpc + blockIdx.x * (size_t)kHistThreads + tid; i < a.n; i += G * kHistThreads) {
        const K key = keys[i];
        acc |= key;
        hist_count_key<K>(key, s_hist, a.shift0, a.rounds, a.radix_bits, a.key_bits, bins);
    }
    __syncthreads();
    for (int i = tid; i < nh; i += kHistThreads) {
        const uint32_t v = s_hist[i];
        if (v) atomicAdd(&a.hist[i], v);
    }
    // OR of the keys (key-range check)
    unsigned long long o = (unsigned long long)acc;
    uint32_t lo = __reduce_or_sync(kFullMask, (uint32_t)o);
    uint32_t hi = __reduce_or_sync(kFullMask, (uint32_t)(o >> 32));
    if ((tid & 31) == 0 && (lo | hi)) atomicOr(a.key_or, ((unsigned long long)hi << 32) | lo);
}

// ----------------------------------------------------------------------------
// Exclusive scan of each round's digit counts -> global digit offsets.
// One CTA per round. Block 0 also checks the key range.
// ----------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_digit_scan(const uint32_t* hist, uint32_t* offs, int bins,
                                                             const unsigned long long* key_or, int key_bits,
                                                             int key_width, uint32_t* status) {
    __shared__ uint32_t s_warp[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t* h = hist + (size_t)blockIdx.x * bins;
    uint32_t* o = offs + (size_t)blockIdx.x * bins;
    const int ipt = (bins + kScanThreads - 1) / kScanThreads;
    const int base = tid * ipt;
    uint32_t local = 0;
    for (int i = 0; i < ipt; ++i)
        if (base + i < bins) local += h[base + i];
    uint32_t x = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(kFullMask, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_warp[lane];
        uint32_t z = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(kFullMask, z, d);
            if (lane >= d) z += y;
        }
        s_warp[lane] = z - w;
    }
    __syncthreads();
    uint32_t run = s_warp[warp] + x - local;
    for (int i = 0; i < ipt; ++i)
        if (base + i < bins) {
            o[base + i] = run;
            run += h[base + i];
        }
    if (blockIdx.x == 0 && tid == 0 && key_bits < key_width) {
        if ((*key_or) >> key_bits) set_status(status, kStatKeyRange);
    }
}

// ----------------------------------------------------------------------------
// One count-sort round: rank within tiles, decoupled look-back, scatter.
// ----------------------------------------------------------------------------
// Look-back word: [31:30] flag, [29:0] count (n < 2^30).
constexpr uint32_t kFlagAgg = 1u << 30;   // tile's own digit count is published
constexpr uint32_t kFlagInc = 2u << 30;   // count of this and all earlier tiles
constexpr uint32_t kCountMask = (1u << 30) - 1;

struct PassArgs {
    const void* keys_in;
    const uint32_t* vals_in;
    void* keys_out;
    uint32_t* vals_out;
    uint32_t n;
    int shift;
    int width;                 // digit bits of this round
    int bins;                  // 2^width
    const uint32_t* bin_off;   // [bins] exclusive global offsets
    uint32_t* lookback;        // [num_tiles][bins]
    uint32_t* tile_counter;
    uint32_t* status;
    uint32_t num_tiles;
    uint64_t limit_ns;
    long long stall_tile;
    int use_bulk;
};

template <typename K, bool VALS, int THREADS, int ITEMS>
struct OnesweepCfg {
    static constexpr int kWarps = THREADS / 32;
    static constexpr int kTile = THREADS * ITEMS;
    static constexpr size_t kBufBytes = (size_t)kTile * sizeof(K) + (VALS ? (size_t)kTile * 4 : 0);
    static size_t smem_bytes(int bins) {
        size_t b = 2 * kBufBytes;
        b += align_up((size_t)kWarps * bins * 2, 16);  // per-warp digit counters (u16)
        b += (size_t)bins * 4 * 2;                     // tile digit starts, output deltas
        b += 2 * 8;                                    // mbarriers
        b += (size_t)kWarps * 4 + 16;                  // warp partial sums, next tile id
        return align_up(b, 128);
    }
};

// Peers of this lane: the lanes of the warp holding a valid key with the
// same digit. RANK 0 uses one match-any vote; RANK 1 intersects one ballot per
// digit bit (no match unit involved).
template <int RANK>
__device__ __forceinline__ uint32_t warp_peers(uint32_t d, bool valid, int width) {
    if constexpr (RANK == 0) {
        return __match_any_sync(kFullMask, valid ? d : 0xffffffffu);
    } else {
        uint32_t peers = __ballot_sync(kFullMask, valid);
#pragma unroll 4
        for (int b = 0; b < width; ++b) {
            const bool bit = (d >> b) & 1u;
            const uint32_t bal = __ballot_sync(kFullMask, bit);
            peers &= bit ? bal : ~bal;
        }
        return peers;
    }
}

template <typename K, bool VALS, int THREADS, int ITEMS, int RANK>
__global__ void __launch_bounds__(THREADS, (1024 / THREADS) > 0 ? (1024 / THREADS) : 1) k_onesweep(PassArgs a) {
    using Cfg = OnesweepCfg<K, VALS, THREADS, ITEMS>;
    constexpr int WARPS = Cfg::kWarps;
    constexpr int TILE = Cfg::kTile;
    extern __shared__ __align__(128) unsigned char smem[];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bins = a.bins;
    const uint32_t dmask = (uint32_t)bins - 1u;
    unsigned char* buf0 = smem;
    uint16_t* s_cnt = reinterpret_cast<uint16_t*>(smem + 2 * Cfg::kBufBytes);
    uint32_t* s_bin_start = reinterpret_cast<uint32_t*>(
        smem + 2 * Cfg::kBufBytes + align_up_dev((size_t)WARPS * bins * 2, 16));
    uint32_t* s_delta = s_bin_start + bins;
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_delta + bins);
    uint32_t* s_warp_scan = reinterpret_cast<uint32_t*>(bars + 2);
    volatile uint32_t& s_next_tile = s_warp_scan[WARPS];
    if ((size_t)(reinterpret_cast<unsigned char*>(s_warp_scan + WARPS + 1) - smem) > dynamic_smem_size()) {
        if (threadIdx.x == 0) set_status(a.status, kStatBounds);
        return;
    }

    // An earlier step (the key-range check) failed: do nothing. One read,
    // shared by the CTA, so that its threads leave together.
    if (__syncthreads_or(tid == 0 && *(volatile uint32_t*)a.status != 0)) return;

    const K* keys_in = static_cast<const K*>(a.keys_in);
    K* keys_out = static_cast<K*>(a.keys_out);

    for (int i = tid; i < WARPS * bins; i += THREADS) s_cnt[i] = 0;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_next_tile = atomicAdd(a.tile_counter, 1u);
    }
    __syncthreads();

    auto full_bulk_tile = [&](uint32_t t) -> bool {
        return a.use_bulk && (size_t)(t + 1) * TILE <= a.n;
    };
    auto issue_tile = [&](uint32_t t, int b) {
        unsigned char* dst = buf0 + (size_t)b * Cfg::kBufBytes;
        constexpr uint32_t kb = TILE * sizeof(K);
        constexpr uint32_t vb = VALS ? TILE * 4 : 0;
        mbar_arrive_expect_tx(&bars[b], kb + vb);
        bulk_load(dst, keys_in + (size_t)t * TILE, kb, &bars[b]);
        if constexpr (VALS) bulk_load(dst + kb, a.vals_in + (size_t)t * TILE, vb, &bars[b]);
    };

    uint32_t tile = s_next_tile;
    if (tid == 0 && tile < a.num_tiles && full_bulk_tile(tile)) issue_tile(tile, 0);
    uint32_t phase = 0u;  // bit b: parity of the next completion of buffer b's barrier
    int b = 0;

    while (tile < a.num_tiles) {
        // Take the next tile now and start copying it into the other buffer.
        if (tid == 0) {
            const uint32_t nt = atomicAdd(a.tile_counter, 1u);
            s_next_tile = nt;
            if (nt < a.num_tiles && full_bulk_tile(nt)) {
                fence_proxy_async_smem();
                issue_tile(nt, b ^ 1);
            }
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
        int fail = __syncthreads_or(!ok);
        const uint32_t next_tile = s_next_tile;
        if (fail) {
            // a bulk copy never completed: record it, wait (bounded) for the
            // copy this CTA issued into the other buffer, and stop
            if (tid == 0) set_status(a.status, kStatTimeout);
            if (next_tile < a.num_tiles && full_bulk_tile(next_tile))
                mbar_wait_bounded(&bars[b ^ 1], (phase >> (b ^ 1)) & 1u, a.limit_ns);
            return;
        }
        const bool stalled = (long long)tile == a.stall_tile;  // fault injection: never publish

        if (!fail && !stalled) {
            // ---- rank every key among equal digits of its warp, in input order
            K kreg[ITEMS];
            uint32_t vreg[ITEMS];
            uint32_t rank[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t j = (uint32_t)(warp * ITEMS * 32 + i * 32 + lane);
                const bool valid = j < tile_n;
                const K k = valid ? s_keys[j] : (K)0;
                kreg[i] = k;
                if constexpr (VALS) vreg[i] = valid ? s_vals[j] : 0u;
                const uint32_t d = (uint32_t)(k >> a.shift) & dmask;
                const uint32_t peers = warp_peers<RANK>(d, valid, a.width);
                const uint32_t below = (uint32_t)__popc(peers & lanemask_lt());
                const uint32_t c = valid ? (uint32_t)s_cnt[warp * bins + d] : 0u;
                rank[i] = c + below;
                __syncwarp();
                if (valid && below + 1 == (uint32_t)__popc(peers))  // highest lane of the group
                    s_cnt[warp * bins + d] = (uint16_t)(c + below + 1);
                __syncwarp();
            }
            __syncthreads();

            // ---- per digit: offsets of each warp inside the tile, tile totals,
            //      publish the tile's count (aggregate) for later tiles
            uint32_t* lb_tile = a.lookback + (size_t)tile * bins;
            for (int d = tid; d < bins; d += THREADS) {
                uint32_t sum = 0;
#pragma unroll 4
                for (int w = 0; w < WARPS; ++w) {
                    const uint32_t c = s_cnt[w * bins + d];
                    s_cnt[w * bins + d] = (uint16_t)sum;
                    sum += c;
                }
                s_bin_start[d] = sum;
                s_delta[d] = sum;
                st_relaxed(&lb_tile[d], (tile == 0 ? kFlagInc : kFlagAgg) | sum);
            }
            __syncthreads();
            block_exclusive_scan<THREADS>(s_bin_start, bins, s_warp_scan);

            // ---- decoupled look-back: sum earlier tiles' counts per digit.
            //      A window of kWin predecessors is read at once (the reads are
            //      independent), then consumed nearest first until a tile with
            //      an inclusive count is met; a predecessor that has published
            //      nothing yet is re-read after a short sleep (bounded).
            constexpr int kWin = 16;
            int lfail = 0;
            for (int d = tid; d < bins; d += THREADS) {
                const uint32_t total = s_delta[d];
                uint32_t excl = 0;
                if (tile > 0) {
                    long long t = (long long)tile - 1;
                    uint64_t t0 = 0;
                    uint32_t spins = 0;
                    bool done = false;
                    while (!done && t >= 0) {
                        uint32_t w[kWin];
#pragma unroll
                        for (int q = 0; q < kWin; ++q)
                            w[q] = t - q >= 0 ? ld_relaxed(&a.lookback[(size_t)(t - q) * bins + d]) : kFlagInc;
                        int used = 0;
                        bool stall = false;
#pragma unroll
                        for (int q = 0; q < kWin; ++q) {
                            if (done || stall) continue;
                            const uint32_t flag = w[q] & ~kCountMask;
                            if (flag == 0) { stall = true; continue; }
                            excl += w[q] & kCountMask;
                            ++used;
                            if (flag == kFlagInc) done = true;
                        }
                        t -= used;
                        if (stall && !done) {
                            if (t0 == 0) t0 = global_timer_ns();
                            else if (global_timer_ns() - t0 > a.limit_ns) { lfail = 1; break; }
                            if ((++spins & 31u) == 0 && ld_relaxed(a.status) != 0) { lfail = 1; break; }
                            __nanosleep(20);
                        }
                    }
                    if (lfail) set_status(a.status, kStatTimeout);
                    __threadfence();
                    st_relaxed(&lb_tile[d], kFlagInc | ((excl + total) & kCountMask));
                }
                s_delta[d] = a.bin_off[d] + excl - s_bin_start[d];
            }
            if (tid == 0 && ld_relaxed(a.status) != 0) lfail = 1;
            fail = __syncthreads_or(lfail);

            if (!fail) {
                // ---- stage keys by digit in shared memory (tile-local order)
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    const uint32_t j = (uint32_t)(warp * ITEMS * 32 + i * 32 + lane);
                    if (j < tile_n) {
                        const uint32_t d = (uint32_t)(kreg[i] >> a.shift) & dmask;
                        const uint32_t pos = s_bin_start[d] + s_cnt[warp * bins + d] + rank[i];
                        if (pos < (uint32_t)TILE) {
                            s_keys[pos] = kreg[i];
                            if constexpr (VALS) s_vals[pos] = vreg[i];
                        }
                    }
                }
                __syncthreads();
                // ---- write runs of equal digits to their global places
                for (uint32_t j = tid; j < tile_n; j += THREADS) {
                    const K k = s_keys[j];
                    const uint32_t d = (uint32_t)(k >> a.shift) & dmask;
                    const uint32_t dst = s_delta[d] + j;
                    if (dst < a.n) {
                        keys_out[dst] = k;
                        if constexpr (VALS) a.vals_out[dst] = s_vals[j];
                    } else {
                        set_status(a.status, kStatBounds);
                    }
                }
            }
        }
        for (int i = tid; i < WARPS * bins; i += THREADS) s_cnt[i] = 0;
        __syncthreads();
        tile = next_tile;
        b ^= 1;
    }
}

// ----------------------------------------------------------------------------
// One count-sort round, second form: one CTA per tile (tiles taken in order
// from an atomic counter), keys and payloads loaded straight into registers,
// several CTAs per SM so that one CTA's look-back wait overlaps another's
// ranking. The tile's digit counts are taken first with shared atomics
// ("early counts") and published before the ranking, so later tiles rarely
// wait on this one.
// ----------------------------------------------------------------------------
template <typename K, bool VALS, int THREADS, int ITEMS>
struct DirectCfg {
    static constexpr int kWarps = THREADS / 32;
    static constexpr int kTile = THREADS * ITEMS;
    static size_t smem_bytes(int bins) {
        size_t b = (size_t)kTile * sizeof(K) + (VALS ? (size_t)kTile * 4 : 0);  // staging
        b += (size_t)kWarps * bins * 4;                                          // per-warp counts -> offsets
        b += align_up((size_t)kWarps * bins * 2, 16);                            // per-warp running ranks
        b += (size_t)bins * 4 * 2;                                               // digit starts, deltas
        b += (size_t)kWarps * 4 + 16;
        return align_up(b, 128);
    }
};

template <typename K, bool VALS, int THREADS, int ITEMS, int RANK>
__global__ void __launch_bounds__(THREADS, ((ITEMS >= 24 ? 512 : 1024) / THREADS) > 0
                                                ? ((ITEMS >= 24 ? 512 : 1024) / THREADS)
                                                : 1) k_onesweep_direct(PassArgs a) {
    using Cfg = DirectCfg<K, VALS, THREADS, ITEMS>;
    constexpr int WARPS = Cfg::kWarps;
    constexpr int TILE = Cfg::kTile;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bins = a.bins;
    const uint32_t dmask = (uint32_t)bins - 1u;
    K* s_keys = reinterpret_cast<K*>(smem);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(smem + (size_t)TILE * sizeof(K));
    uint32_t* s_whist = reinterpret_cast<uint32_t*>(smem + (size_t)TILE * sizeof(K) + (VALS ? (size_t)TILE * 4 : 0));
    uint16_t* s_cnt = reinterpret_cast<uint16_t*>(s_whist + (size_t)WARPS * bins);
    uint32_t* s_bin_start = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(s_cnt) +
                                                        align_up_dev((size_t)WARPS * bins * 2, 16));
    uint32_t* s_delta = s_bin_start + bins;
    uint32_t* s_warp_scan = s_delta + bins;
    volatile uint32_t& s_tile = s_warp_scan[WARPS];
    if ((size_t)(reinterpret_cast<unsigned char*>(s_warp_scan + WARPS + 1) - smem) > dynamic_smem_size()) {
        if (threadIdx.x == 0) set_status(a.status, kStatBounds);
        return;
    }

    // an earlier step failed (one read, shared by the CTA)
    if (__syncthreads_or(tid == 0 && *(volatile uint32_t*)a.status != 0)) return;
    if (tid == 0) s_tile = atomicAdd(a.tile_counter, 1u);
    for (int i = tid; i < WARPS * bins; i += THREADS) {
        s_whist[i] = 0;
        s_cnt[i] = 0;
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= a.num_tiles) return;
    const uint32_t tile_base = tile * (uint32_t)TILE;
    const uint32_t tile_n = min((uint32_t)TILE, a.n - tile_base);
    const K* keys_in = static_cast<const K*>(a.keys_in) + tile_base;
    const uint32_t* vals_in = VALS ? a.vals_in + tile_base : nullptr;
    K* keys_out = static_cast<K*>(a.keys_out);

    K kreg[ITEMS];
    uint32_t vreg[ITEMS];
    uint32_t rank[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = (uint32_t)(warp * ITEMS * 32 + i * 32 + lane);
        kreg[i] = j < tile_n ? keys_in[j] : (K)0;
        if constexpr (VALS) vreg[i] = j < tile_n ? vals_in[j] : 0u;
    }
    const bool stalled = (long long)tile == a.stall_tile;  // fault injection: never publish
    // early counts
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = (uint32_t)(warp * ITEMS * 32 + i * 32 + lane);
        if (j < tile_n) atomicAdd(&s_whist[warp * bins + ((uint32_t)(kreg[i] >> a.shift) & dmask)], 1u);
    }
    __syncthreads();
    uint32_t* lb_tile = a.lookback + (size_t)tile * bins;
    for (int d = tid; d < bins; d += THREADS) {
        uint32_t sum = 0;
#pragma unroll 4
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t c = s_whist[w * bins + d];
            s_whist[w * bins + d] = sum;
            sum += c;
        }
        s_bin_start[d] = sum;
        s_delta[d] = sum;
        if (!stalled) st_relaxed(&lb_tile[d], (tile == 0 ? kFlagInc : kFlagAgg) | sum);
    }
    if (stalled) {
        __syncthreads();
        block_exclusive_scan<THREADS>(s_bin_start, bins, s_warp_scan);
        return;
    }
    // decoupled look-back (windowed, bounded), right after publishing, so that
    // this tile's inclusive counts appear as early as possible; the warps
    // without look-back work go on to rank their keys meanwhile
    constexpr int kWin = 8;
    int lfail = 0;
    for (int d = tid; d < bins; d += THREADS) {
        const uint32_t total = s_delta[d];
        uint32_t excl = 0;
        if (tile > 0) {
            long long t = (long long)tile - 1;
            uint64_t t0 = 0;
            uint32_t spins = 0;
            bool done = false;
            while (!done && t >= 0) {
                uint32_t w[kWin];
#pragma unroll
                for (int q = 0; q < kWin; ++q)
                    w[q] = t - q >= 0 ? ld_relaxed(&a.lookback[(size_t)(t - q) * bins + d]) : kFlagInc;
                int used = 0;
                bool stall = false;
#pragma unroll
                for (int q = 0; q < kWin; ++q) {
                    if (done || stall) continue;
                    const uint32_t flag = w[q] & ~kCountMask;
                    if (flag == 0) { stall = true; continue; }
                    excl += w[q] & kCountMask;
                    ++used;
                    if (flag == kFlagInc) done = true;
                }
                t -= used;
                if (stall && !done) {
                    if (t0 == 0) t0 = global_timer_ns();
                    else if (global_timer_ns() - t0 > a.limit_ns) { lfail = 1; break; }
                    if ((++spins & 31u) == 0 && ld_relaxed(a.status) != 0) { lfail = 1; break; }
                    __nanosleep(64);
                }
            }
            if (lfail) set_status(a.status, kStatTimeout);
            __threadfence();
            st_relaxed(&lb_tile[d], kFlagInc | ((excl + total) & kCountMask));
        }
        s_delta[d] = a.bin_off[d] + excl;  // the tile's digit start is subtracted after the scan
    }
    // rank each key among equal digits of its warp, in input order
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = (uint32_t)(warp * ITEMS * 32 + i * 32 + lane);
        const bool valid = j < tile_n;
        const uint32_t d = (uint32_t)(kreg[i] >> a.shift) & dmask;
        const uint32_t peers = warp_peers<RANK>(d, valid, a.width);
        const uint32_t below = (uint32_t)__popc(peers & lanemask_lt());
        const uint32_t c = valid ? (uint32_t)s_cnt[warp * bins + d] : 0u;
        rank[i] = c + below;
        __syncwarp();
        if (valid && below + 1 == (uint32_t)__popc(peers)) s_cnt[warp * bins + d] = (uint16_t)(c + below + 1);
        __syncwarp();
    }
    __syncthreads();
    block_exclusive_scan<THREADS>(s_bin_start, bins, s_warp_scan);
    for (int d = tid; d < bins; d += THREADS) s_delta[d] -= s_bin_start[d];
    if (tid == 0 && ld_relaxed(a.status) != 0) lfail = 1;
    if (__syncthreads_or(lfail)) return;
    // stage by digit
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t j = (uint32_t)(warp * ITEMS * 32 + i * 32 + lane);
        if (j < tile_n) {
            const uint32_t d = (uint32_t)(kreg[i] >> a.shift) & dmask;
            const uint32_t pos = s_bin_start[d] + s_whist[warp * bins + d] + rank[i];
            if (pos < (uint32_t)TILE) {
                s_keys[pos] = kreg[i];
                if constexpr (VALS) s_vals[pos] = vreg[i];
            }
        }
    }
    __syncthreads();
    for (uint32_t j = tid; j < tile_n; j += THREADS) {
        const K k = s_keys[j];
        const uint32_t d = (uint32_t)(k >> a.shift) & dmask;
        const uint32_t dst = s_delta[d] + j;
        if (dst < a.n) {
            keys_out[dst] = k;
            if constexpr (VALS) a.vals_out[dst] = s_vals[j];
        } else {
            set_status(a.status, kStatBounds);
        }
    }
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
namespace {

// Launch shapes of a round (threads x keys per thread).
// 0-5: persistent bulk-copy kernel; 6-9: one CTA per tile.
constexpr int kShapeThreads[] = {512, 256, 256, 128, 512, 1024, 256, 256, 384, 512, 512, 1024, 256};
constexpr int kShapeItems[] = {8, 16, 8, 16, 16, 8, 16, 12, 12, 8, 16, 16, 32};

int shape_tile(int sh) { return kShapeThreads[sh] * kShapeItems[sh]; }

template <typename K, bool VALS, int THREADS, int ITEMS, int RANK>
isort_status launch_round(PassArgs a, cudaStream_t s) {
    using Cfg = OnesweepCfg<K, VALS, THREADS, ITEMS>;
    auto kern = k_onesweep<K, VALS, THREADS, ITEMS, RANK>;
    const size_t smem = Cfg::smem_bytes(a.bins);
    if (smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem));
    if (per_sm < 1) return ISORT_ERR_UNSUPPORTED;
    const uint32_t grid = (uint32_t)std::min<size_t>(a.num_tiles, (size_t)per_sm * sm_count());
    LaunchScope ls("onesweep", s);
    kern<<<grid, THREADS, smem, s>>>(a);
    return from_cuda(cudaGetLastError());
}

template <typename K, bool VALS, int THREADS, int ITEMS, int RANK>
isort_status launch_round_direct(PassArgs a, cudaStream_t s) {
    using Cfg = DirectCfg<K, VALS, THREADS, ITEMS>;
    auto kern = k_onesweep_direct<K, VALS, THREADS, ITEMS, RANK>;
    const size_t smem = Cfg::smem_bytes(a.bins);
    if (smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LaunchScope ls("onesweep", s);
    kern<<<a.num_tiles, THREADS, smem, s>>>(a);
    return from_cuda(cudaGetLastError());
}

template <typename K, bool VALS, int RANK>
isort_status launch_round_shape(int sh, PassArgs a, cudaStream_t s) {
    // the shapes kept built (others measured slower; load_tune maps them here)
    switch (sh) {
        case 0: return launch_round<K, VALS, 512, 8, RANK>(a, s);
        case 1: return launch_round<K, VALS, 256, 16, RANK>(a, s);
        case 9: return launch_round_direct<K, VALS, 512, 8, RANK>(a, s);
        case 10: return launch_round_direct<K, VALS, 512, 16, RANK>(a, s);
        default: return launch_round<K, VALS, 512, 16, RANK>(a, s);  // shape 4
    }
}

template <typename K>
isort_status launch_round_dispatch(int sh, bool vals, PassArgs a, cudaStream_t s) {
    // per-bit ballot ranking (match-any ranking measured slower and is not built)
    if (vals) return launch_round_shape<K, true, 1>(sh, a, s);
    return launch_round_shape<K, false, 1>(sh, a, s);
}

template <typename K>
isort_status launch_hist(const K* keys, size_t n, int shift0, int rb, int key_bits, int rounds, uint32_t* hist,
                         unsigned long long* key_or, uint32_t* status, cudaStream_t s) {
    HistArgs a;
    a.keys = keys;
    a.n = n;
    a.shift0 = shift0;
    a.radix_bits = rb;
    a.key_bits = key_bits;
    a.rounds = rounds;
    a.hist = hist;
    a.key_or = key_or;
    a.status = status;
    a.limit_ns = spin_limit_ns();
    a.use_bulk = ((uintptr_t)keys % 16) == 0;
    const int bins = 1 << rb;
    const size_t smem = kHistStages * kHistChunkBytes + align_up((size_t)rounds * bins * 4, 8) + kHistStages * 8;
    if (smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    void (*kern)(HistArgs) = tune().hist_agg ? k_digit_hist<K, true> : k_digit_hist<K, false>;
    if (shift0 == 0 && !tune().hist_agg) {
        if constexpr (sizeof(K) == 4) {
            if (rb == 8 && key_bits == 32) kern = k_digit_hist<K, false, 8, 32>;
            else if (rb == 11 && key_bits == 32) kern = k_digit_hist<K, false, 11, 32>;
            else if (rb == 8 && key_bits == 20) kern = k_digit_hist<K, false, 8, 20>;
            else if (rb == 11 && key_bits == 20) kern = k_digit_hist<K, false, 11, 20>;
        } else {
            if (rb == 8 && key_bits == 64) kern = k_digit_hist<K, false, 8, 64>;
            else if (rb == 8 && key_bits == 48) kern = k_digit_hist<K, false, 8, 48>;
        }
    }
    ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kHistThreads, smem));
    per_sm = std::max(1, std::min(per_sm, 2));
    const size_t chunks = n * sizeof(K) / kHistChunkBytes;
    const size_t want = std::max<size_t>(1, std::min<size_t>((size_t)per_sm * sm_count(),
                                                            std::max<size_t>(chunks, (n + kHistThreads - 1) / kHistThreads)));
    LaunchScope ls("digit_hist", s);
    kern<<<(unsigned)want, kHistThreads, smem, s>>>(a);
    return from_cuda(cudaGetLastError());
}

isort_status launch_scan(const uint32_t* hist, uint32_t* offs, int rounds, int bins, const unsigned long long* key_or,
                         int key_bits, int key_width, uint32_t* status, cudaStream_t s) {
    LaunchScope ls("digit_scan", s);
    k_digit_scan<<<rounds, kScanThreads, 0, s>>>(hist, offs, bins, key_or, key_bits, key_width, status);
    return from_cuda(cudaGetLastError());
}

// Control block at the head of the scratch allocation.
struct Ctl {
    uint32_t* status;
    unsigned long long* key_or;
    uint32_t* hist;
    uint32_t* offs;
    uint32_t* tile_ctr;
    uint32_t* lookback;
    size_t zero_bytes;   // bytes to clear from the start
    size_t bytes;        // total control bytes
    uint32_t num_tiles;
};

Ctl layout_ctl(unsigned char* base, int rounds, int bins, uint32_t num_tiles, bool with_lookback) {
    Ctl c;
    size_t off = 0;
    c.status = reinterpret_cast<uint32_t*>(base + off);
    off += 8;
    c.key_or = reinterpret_cast<unsigned long long*>(base + off);
    off += 8;
    c.hist = reinterpret_cast<uint32_t*>(base + off);
    off += align_up((size_t)rounds * bins * 4, 16);
    c.tile_ctr = reinterpret_cast<uint32_t*>(base + off);
    off += align_up((size_t)rounds * 4, 16);
    c.lookback = reinterpret_cast<uint32_t*>(base + off);
    if (with_lookback) off += align_up((size_t)rounds * num_tiles * bins * 4, 16);
    c.zero_bytes = off;
    c.offs = reinterpret_cast<uint32_t*>(base + off);
    off += align_up((size_t)rounds * bins * 4, 16);
    c.bytes = align_up(off, 256);
    c.num_tiles = num_tiles;
    return c;
}

bool valid_widths(int key_width, int& key_bits, int rb) {
    if (key_bits == 0) key_bits = key_width;
    return key_bits >= 1 && key_bits <= key_width && rb >= 1 && rb <= 16;
}

}  // namespace

// The whole sort of up to 8 x 8192 u32 keys on one cluster (seg.cu).
constexpr size_t kSmallSortMax = 8 * 8192;
isort_status radix_small_u32(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, uint32_t n,
                             int key_bits, cudaStream_t s);

// The chunked reduce-then-scan rounds (rts.cu).
template <typename K>
isort_status radix_device_rts(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n, int key_bits,
                              int rb, cudaStream_t s, int shape = -1);
extern template isort_status radix_device_rts<uint32_t>(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, size_t,
                                                        int, int, cudaStream_t, int);
extern template isort_status radix_device_rts<uint64_t>(const uint64_t*, const uint32_t*, uint64_t*, uint32_t*, size_t,
                                                        int, int, cudaStream_t, int);

namespace {

template <typename K>
isort_status radix_device(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n, int key_bits, int rb,
                          cudaStream_t s) {
    const int key_width = (int)sizeof(K) * 8;
    const int rounds = (key_bits + rb - 1) / rb;
    const int bins = 1 << rb;
    if constexpr (sizeof(K) == 4) {
        // up to 65,536 keys: all rounds on chip in one launch
        if (n <= kSmallSortMax && rb == 8 && tune().small && peek_stall_tile() < 0)
            return radix_small_u32(kin, vin, kout, vout, (uint32_t)n, key_bits, s);
    }
    if (rb > 12 || (tune().algo == 1 && peek_stall_tile() < 0)) {
        // chunked rounds (which also take radix 2^13..2^16, as two passes per
        // round); wide digits whose tables do not fit on chip take the
        // single-pass rounds below (refused before any work is enqueued)
        const isort_status st = radix_device_rts<K>(kin, vin, kout, vout, n, key_bits, rb, s);
        if (st != ISORT_ERR_UNSUPPORTED || rb > 12) return st;
    }
    const bool vals = vin != nullptr;
    const bool inplace = (const void*)kin == (const void*)kout;
    const int sh = bins <= 256 ? tune().shape_small : tune().shape_large;
    const uint32_t tile = (uint32_t)shape_tile(sh);
    const uint32_t num_tiles = (uint32_t)((n + tile - 1) / tile);

    // ping-pong buffers needed besides kout
    int nbuf;
    if (inplace) nbuf = (rounds % 2 == 0) ? 1 : (rounds == 1 ? 1 : 2);
    else nbuf = rounds == 1 ? 0 : 1;
    const size_t buf_bytes = align_up(n * sizeof(K), 256) + (vals ? align_up(n * 4, 256) : 0);

    unsigned char* ws = nullptr;
    Ctl probe = layout_ctl(nullptr, rounds, bins, num_tiles, true);
    const size_t total = probe.bytes + (size_t)nbuf * buf_bytes;
    isort_status st = scratch_alloc((void**)&ws, total, s);
    if (st != ISORT_OK) return st;
    Ctl c = layout_ctl(ws, rounds, bins, num_tiles, true);
    K* wk[2] = {nullptr, nullptr};
    uint32_t* wv[2] = {nullptr, nullptr};
    for (int i = 0; i < nbuf; ++i) {
        unsigned char* p = ws + c.bytes + (size_t)i * buf_bytes;
        wk[i] = reinterpret_cast<K*>(p);
        wv[i] = vals ? reinterpret_cast<uint32_t*>(p + align_up(n * sizeof(K), 256)) : nullptr;
    }

    auto fail = [&](isort_status e) {
        scratch_free(ws, s);
        return e;
    };
    cudaError_t ce = cudaMemsetAsync(ws, 0, c.zero_bytes, s);
    if (ce != cudaSuccess) return fail(from_cuda(ce));
    st = launch_hist<K>(kin, n, 0, rb, key_bits, rounds, c.hist, c.key_or, c.status, s);
    if (st != ISORT_OK) return fail(st);
    st = launch_scan(c.hist, c.offs, rounds, bins, c.key_or, key_bits, key_width, c.status, s);
    if (st != ISORT_OK) return fail(st);

    // Source/destination of every round.
    const K* src_k = kin;
    const uint32_t* src_v = vin;
    const long long stall = take_stall_tile();
    for (int d = 0; d < rounds; ++d) {
        K* dk;
        uint32_t* dv;
        const bool last = d == rounds - 1;
        if (!inplace) {
            // rounds - 1 - d even -> kout, odd -> buffer 0
            const bool to_out = ((rounds - 1 - d) % 2) == 0;
            dk = to_out ? kout : wk[0];
            dv = to_out ? vout : wv[0];
        } else if (rounds == 1) {
            dk = wk[0];
            dv = wv[0];
        } else if (rounds % 2 == 0) {
            const bool to_out = (d % 2) == 1;
            dk = to_out ? kout : wk[0];
            dv = to_out ? vout : wv[0];
        } else {
            if (last) { dk = kout; dv = vout; }
            else { dk = wk[d % 2]; dv = wv[d % 2]; }
        }
        const int shift = d * rb;
        const int width = std::min(rb, key_bits - shift);
        PassArgs a;
        a.keys_in = src_k;
        a.vals_in = src_v;
        a.keys_out = dk;
        a.vals_out = dv;
        a.n = (uint32_t)n;
        a.shift = shift;
        a.width = width;
        a.bins = 1 << width;
        a.bin_off = c.offs + (size_t)d * bins;
        a.lookback = c.lookback + (size_t)d * num_tiles * bins;
        a.tile_counter = c.tile_ctr + d;
        a.status = c.status;
        a.num_tiles = num_tiles;
        a.limit_ns = spin_limit_ns();
        a.stall_tile = d == 0 ? stall : -1;
        a.use_bulk = (((uintptr_t)src_k % 16) == 0) && (!vals || ((uintptr_t)src_v % 16) == 0);
        st = launch_round_dispatch<K>(sh, vals, a, s);
        if (st != ISORT_OK) return fail(st);
        src_k = dk;
        src_v = dv;
    }
    if (inplace && rounds == 1) {
        ce = cudaMemcpyAsync(kout, wk[0], n * sizeof(K), cudaMemcpyDeviceToDevice, s);
        if (ce == cudaSuccess && vals) ce = cudaMemcpyAsync(vout, wv[0], n * 4, cudaMemcpyDeviceToDevice, s);
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    st = finish_status(c.status, s);
    scratch_free(ws, s);
    return st;
}

// Entry: validates, stages host buffers through device memory if needed.
// A copy ordered on `s`, cut into up to kCopyStreams pieces of at least 64 MiB
// that run on auxiliary streams kept per (thread, device, calling stream), so
// that the copies of calls made on different streams can overlap.
constexpr int kCopyStreams = 4;
constexpr size_t kMaxCopySets = 16;  // calling streams with their own auxiliary streams, per thread

struct CopyStreams {
    cudaStream_t st[kCopyStreams] = {};
    cudaEvent_t ev[kCopyStreams + 1] = {};
};

thread_local std::map<std::pair<int, cudaStream_t>, CopyStreams> t_copy;

cudaError_t copy_split(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    // pieces help a call that runs alone; with calls in flight on several
    // streams (the asynchronous status mode) one copy per buffer is faster
    const size_t piece_min = size_t(64) << 20;
    const int max_pieces = sync_mode() ? std::min(kCopyStreams, tune().copy_pieces) : 1;
    const int pieces = (int)std::min<size_t>(max_pieces, std::max<size_t>(1, bytes / piece_min));
    if (pieces <= 1) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return ce;
    auto it = t_copy.find({dev, s});
    if (it == t_copy.end()) {
        if (t_copy.size() >= kMaxCopySets) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
        CopyStreams cs;  // created once per (thread, device, stream), kept for the process
        for (int i = 0; i < kCopyStreams; ++i) {
            if (cudaStreamCreateWithFlags(&cs.st[i], cudaStreamNonBlocking) != cudaSuccess) return cudaGetLastError();
        }
        for (int i = 0; i <= kCopyStreams; ++i) {
            if (cudaEventCreateWithFlags(&cs.ev[i], cudaEventDisableTiming) != cudaSuccess) return cudaGetLastError();
        }
        it = t_copy.emplace(std::make_pair(dev, s), cs).first;
    }
    CopyStreams& cs = it->second;
    ce = cudaEventRecord(cs.ev[kCopyStreams], s);  // the copies start after the work before them
    const size_t step = align_up((bytes + pieces - 1) / pieces, 4096);
    for (int i = 0; i < pieces && ce == cudaSuccess; ++i) {
        const size_t off = (size_t)i * step;
        if (off >= bytes) break;
        const size_t len = std::min(step, bytes - off);
        ce = cudaStreamWaitEvent(cs.st[i], cs.ev[kCopyStreams], 0);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(static_cast<char*>(dst) + off, static_cast<const char*>(src) + off, len,
                                 cudaMemcpyDefault, cs.st[i]);
        if (ce == cudaSuccess) ce = cudaEventRecord(cs.ev[i], cs.st[i]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, cs.ev[i], 0);  // the work after them waits
    }
    return ce;
}

template <typename K>
isort_status radix_entry(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n, int key_bits, int rb,
                         void* stream) {
    const int key_width = (int)sizeof(K) * 8;
    if (!valid_widths(key_width, key_bits, rb)) return ISORT_ERR_INVALID_ARG;
    if ((vin == nullptr) != (vout == nullptr)) return ISORT_ERR_INVALID_ARG;
    if (n >= (size_t(1) << 30)) return ISORT_ERR_UNSUPPORTED;
    if (n > 1 && (!kin || !kout)) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool inplace = (const void*)kin == (const void*)kout;
    if (inplace && vin != vout) return ISORT_ERR_INVALID_ARG;
    if (n <= 1) {
        if (!inplace && n == 1) {
            // keys_out = keys_in for a single element
            ISORT_TRY_CUDA(cudaMemcpyAsync(kout, kin, sizeof(K), cudaMemcpyDefault, s));
            if (vin) ISORT_TRY_CUDA(cudaMemcpyAsync(vout, vin, 4, cudaMemcpyDefault, s));
            if (sync_mode()) ISORT_TRY_CUDA(cudaStreamSynchronize(s));
        }
        return ISORT_OK;
    }
    const bool host = is_host_pointer(kin) || is_host_pointer(kout) || (vin && (is_host_pointer(vin) || is_host_pointer(vout)));
    if (!host) return radix_device<K>(kin, vin, kout, vout, n, key_bits, rb, s);

    // Host buffers: copy in, sort in place on the device, copy out. The copies
    // are cut into pieces spread over a few streams (several DMA transfers at
    // once), joined to `s` by events.
    const size_t kb = align_up(n * sizeof(K), 256);
    unsigned char* st_buf = nullptr;
    isort_status st = scratch_alloc((void**)&st_buf, kb + (vin ? align_up(n * 4, 256) : 0), s);
    if (st != ISORT_OK) return st;
    K* dk = reinterpret_cast<K*>(st_buf);
    uint32_t* dv = vin ? reinterpret_cast<uint32_t*>(st_buf + kb) : nullptr;
    cudaError_t ce = copy_split(dk, kin, n * sizeof(K), s);
    if (ce == cudaSuccess && vin) ce = copy_split(dv, vin, n * 4, s);
    if (ce != cudaSuccess) {
        scratch_free(st_buf, s);
        return from_cuda(ce);
    }
    const int was_sync = sync_mode();
    st = radix_device<K>(dk, dv, dk, dv, n, key_bits, rb, s);
    if (st == ISORT_OK || st == ISORT_ERR_TIMEOUT) {
        if (st == ISORT_OK) {
            ce = copy_split(kout, dk, n * sizeof(K), s);
            if (ce == cudaSuccess && vin) ce = copy_split(vout, dv, n * 4, s);
            if (ce != cudaSuccess) st = from_cuda(ce);
        }
    }
    scratch_free(st_buf, s);
    // asynchronous status mode: the call returns once everything is enqueued;
    // the host buffers are in use until `s` reaches this point
    if (!was_sync) return st;
    cudaError_t se = cudaStreamSynchronize(s);
    if (st == ISORT_OK && se != cudaSuccess) st = from_cuda(se);
    return st;
}

}  // namespace

// Used by other translation units (segmented / learned paths).
isort_status radix_sort_u32_device(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, size_t n,
                                   int key_bits, int rb, cudaStream_t s) {
    if (key_bits == 0) key_bits = 32;
    return radix_device<uint32_t>(kin, vin, kout, vout, n, key_bits, rb, s);
}

isort_status radix_sort_u64_device(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout, size_t n,
                                   int key_bits, int rb, cudaStream_t s) {
    if (key_bits == 0) key_bits = 64;
    return radix_device<uint64_t>(kin, vin, kout, vout, n, key_bits, rb, s);
}

// Scratch an in-place sort of n u32 keys (+ payload) needs when the caller
// provides it: the control block followed by the ping-pong buffers.
size_t radix_u32_inplace_workspace_bytes(size_t n, int key_bits, int rb, bool vals) {
    const int rounds = (key_bits + rb - 1) / rb;
    const int bins = 1 << rb;
    const int sh = bins <= 256 ? tune().shape_small : tune().shape_large;
    const uint32_t tile = (uint32_t)shape_tile(sh);
    const uint32_t num_tiles = (uint32_t)((n + tile - 1) / tile);
    const int nbuf = (rounds % 2 == 0 || rounds == 1) ? 1 : 2;
    const size_t buf_bytes = align_up(n * 4, 256) + (vals ? align_up(n * 4, 256) : 0);
    return layout_ctl(nullptr, rounds, bins, num_tiles, true).bytes + (size_t)nbuf * buf_bytes;
}

// The in-place sort of isort_radix, with `ws` (ws_bytes, 256-byte aligned,
// device memory) as its only scratch: no memory is allocated. The control
// block at the head of ws is cleared here. *d_status points at the call's
// device status word inside ws once the work is enqueued.
isort_status radix_u32_inplace_in_workspace(uint32_t* keys, uint32_t* vals, size_t n, int key_bits, int rb,
                                            unsigned char* ws, size_t ws_bytes, cudaStream_t s,
                                            const uint32_t** d_status) {
    const int rounds = (key_bits + rb - 1) / rb;
    const int bins = 1 << rb;
    const bool hv = vals != nullptr;
    const int sh = bins <= 256 ? tune().shape_small : tune().shape_large;
    const uint32_t tile = (uint32_t)shape_tile(sh);
    const uint32_t num_tiles = (uint32_t)((n + tile - 1) / tile);
    if (radix_u32_inplace_workspace_bytes(n, key_bits, rb, hv) > ws_bytes) return ISORT_ERR_UNSUPPORTED;
    Ctl c = layout_ctl(ws, rounds, bins, num_tiles, true);
    const size_t buf_bytes = align_up(n * 4, 256) + (hv ? align_up(n * 4, 256) : 0);
    uint32_t* wk[2];
    uint32_t* wv[2];
    for (int i = 0; i < 2; ++i) {
        unsigned char* p = ws + c.bytes + (size_t)i * buf_bytes;
        wk[i] = reinterpret_cast<uint32_t*>(p);
        wv[i] = hv ? reinterpret_cast<uint32_t*>(p + align_up(n * 4, 256)) : nullptr;
    }
    *d_status = c.status;
    ISORT_TRY_CUDA(cudaMemsetAsync(ws, 0, c.zero_bytes, s));
    isort_status st = launch_hist<uint32_t>(keys, n, 0, rb, key_bits, rounds, c.hist, c.key_or, c.status, s);
    if (st != ISORT_OK) return st;
    st = launch_scan(c.hist, c.offs, rounds, bins, c.key_or, key_bits, 32, c.status, s);
    if (st != ISORT_OK) return st;
    const uint32_t* src_k = keys;
    const uint32_t* src_v = vals;
    for (int d = 0; d < rounds; ++d) {
        uint32_t* dk;
        uint32_t* dv;
        if (rounds == 1) {
            dk = wk[0];
            dv = wv[0];
        } else if (rounds % 2 == 0) {
            dk = (d % 2) == 1 ? keys : wk[0];
            dv = (d % 2) == 1 ? vals : wv[0];
        } else if (d == rounds - 1) {
            dk = keys;
            dv = vals;
        } else {
            dk = wk[d % 2];
            dv = wv[d % 2];
        }
        const int shift = d * rb;
        const int width = std::min(rb, key_bits - shift);
        PassArgs a;
        a.keys_in = src_k;
        a.vals_in = src_v;
        a.keys_out = dk;
        a.vals_out = dv;
        a.n = (uint32_t)n;
        a.shift = shift;
        a.width = width;
        a.bins = 1 << width;
        a.bin_off = c.offs + (size_t)d * bins;
        a.lookback = c.lookback + (size_t)d * num_tiles * bins;
        a.tile_counter = c.tile_ctr + d;
        a.status = c.status;
        a.num_tiles = num_tiles;
        a.limit_ns = spin_limit_ns();
        a.stall_tile = -1;
        a.use_bulk = (((uintptr_t)src_k % 16) == 0) && (!hv || ((uintptr_t)src_v % 16) == 0);
        st = launch_round_dispatch<uint32_t>(sh, hv, a, s);
        if (st != ISORT_OK) return st;
        src_k = dk;
        src_v = dv;
    }
    if (rounds == 1) {
        ISORT_TRY_CUDA(cudaMemcpyAsync(keys, wk[0], n * 4, cudaMemcpyDeviceToDevice, s));
        if (hv) ISORT_TRY_CUDA(cudaMemcpyAsync(vals, wv[0], n * 4, cudaMemcpyDeviceToDevice, s));
    }
    return ISORT_OK;
}

template <typename K>
isort_status count_round_entry(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n, int shift,
                                      int width, void* stream) {
    const int key_width = (int)sizeof(K) * 8;
    if (width < 1 || width > 16 || shift < 0 || shift + width > key_width) return ISORT_ERR_INVALID_ARG;
    if ((vin == nullptr) != (vout == nullptr)) return ISORT_ERR_INVALID_ARG;
    if (n >= (size_t(1) << 30)) return ISORT_ERR_UNSUPPORTED;
    if (width > 12) return ISORT_ERR_UNSUPPORTED;
    if (n == 0) return ISORT_OK;
    if (!kin || !kout || (const void*)kin == (const void*)kout) return ISORT_ERR_INVALID_ARG;
    if (is_host_pointer(kin) || is_host_pointer(kout) || (vin && (is_host_pointer(vin) || is_host_pointer(vout))))
        return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int bins = 1 << width;
    const int sh = bins <= 256 ? tune().shape_small : tune().shape_large;
    const uint32_t tile = (uint32_t)shape_tile(sh);
    const uint32_t num_tiles = (uint32_t)((n + tile - 1) / tile);
    Ctl probe = layout_ctl(nullptr, 1, bins, num_tiles, true);
    unsigned char* ws = nullptr;
    isort_status st = scratch_alloc((void**)&ws, probe.bytes, s);
    if (st != ISORT_OK) return st;
    Ctl c = layout_ctl(ws, 1, bins, num_tiles, true);
    auto fail = [&](isort_status e) {
        scratch_free(ws, s);
        return e;
    };
    cudaError_t ce = cudaMemsetAsync(ws, 0, c.zero_bytes, s);
    if (ce != cudaSuccess) return fail(from_cuda(ce));
    // the one digit as a single round starting at bit `shift`
    st = launch_hist<K>(kin, n, shift, width, width, 1, c.hist, c.key_or, c.status, s);
    if (st != ISORT_OK) return fail(st);
    st = launch_scan(c.hist, c.offs, 1, bins, c.key_or, key_width, key_width, c.status, s);
    if (st != ISORT_OK) return fail(st);
    PassArgs a;
    a.keys_in = kin;
    a.vals_in = vin;
    a.keys_out = kout;
    a.vals_out = vout;
    a.n = (uint32_t)n;
    a.shift = shift;
    a.width = width;
    a.bins = bins;
    a.bin_off = c.offs;
    a.lookback = c.lookback;
    a.tile_counter = c.tile_ctr;
    a.status = c.status;
    a.num_tiles = num_tiles;
    a.limit_ns = spin_limit_ns();
    a.stall_tile = take_stall_tile();
    a.use_bulk = (((uintptr_t)kin % 16) == 0) && (!vin || ((uintptr_t)vin % 16) == 0);
    st = launch_round_dispatch<K>(sh, vin != nullptr, a, s);
    if (st != ISORT_OK) return fail(st);
    st = finish_status(c.status, s);
    scratch_free(ws, s);
    return st;
}

}  // namespace isort

using namespace isort;

extern "C" {

isort_status isort_radix(uint32_t* keys, uint32_t* vals, size_t n, int key_bits, int radix_bits, void* stream) {
    return radix_entry<uint32_t>(keys, vals, keys, vals, n, key_bits, radix_bits, stream);
}

isort_status isort_radix_u64(uint64_t* keys, uint32_t* vals, size_t n, int key_bits, int radix_bits, void* stream) {
    return radix_entry<uint64_t>(keys, vals, keys, vals, n, key_bits, radix_bits, stream);
}

isort_status isort_radix_copy(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                              size_t n, int key_bits, int radix_bits, void* stream) {
    if (keys_in == keys_out && n > 0) return ISORT_ERR_INVALID_ARG;
    return radix_entry<uint32_t>(keys_in, vals_in, keys_out, vals_out, n, key_bits, radix_bits, stream);
}

isort_status isort_radix_copy_u64(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                  uint32_t* vals_out, size_t n, int key_bits, int radix_bits, void* stream) {
    if (keys_in == keys_out && n > 0) return ISORT_ERR_INVALID_ARG;
    return radix_entry<uint64_t>(keys_in, vals_in, keys_out, vals_out, n, key_bits, radix_bits, stream);
}

isort_status isort_digit_hist(const void* keys, int key_width, size_t n, int key_bits, int radix_bits, uint32_t* hist,
                              void* stream) {
    if (key_width != 32 && key_width != 64) return ISORT_ERR_INVALID_ARG;
    if (!valid_widths(key_width, key_bits, radix_bits) || !hist || (n && !keys)) return ISORT_ERR_INVALID_ARG;
    if (radix_bits > 12) return ISORT_ERR_UNSUPPORTED;
    if (n >= (size_t(1) << 32)) return ISORT_ERR_UNSUPPORTED;
    if (is_host_pointer(keys) || is_host_pointer(hist)) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int rounds = (key_bits + radix_bits - 1) / radix_bits;
    const int bins = 1 << radix_bits;
    unsigned char* ws = nullptr;
    isort_status st = scratch_alloc((void**)&ws, 64, s);
    if (st != ISORT_OK) return st;
    uint32_t* status = reinterpret_cast<uint32_t*>(ws);
    unsigned long long* kor = reinterpret_cast<unsigned long long*>(ws + 8);
    cudaError_t ce = cudaMemsetAsync(ws, 0, 64, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(hist, 0, (size_t)rounds * bins * 4, s);
    if (ce != cudaSuccess) {
        scratch_free(ws, s);
        return from_cuda(ce);
    }
    if (key_width == 32)
        st = launch_hist<uint32_t>((const uint32_t*)keys, n, 0, radix_bits, key_bits, rounds, hist, kor, status, s);
    else
        st = launch_hist<uint64_t>((const uint64_t*)keys, n, 0, radix_bits, key_bits, rounds, hist, kor, status, s);
    if (st == ISORT_OK) {
        // key-range check only (scan of round 0 into scratch is not needed): reuse the scan kernel's check
        LaunchScope ls("range_check", s);
        k_digit_scan<<<1, kScanThreads, 0, s>>>(hist, reinterpret_cast<uint32_t*>(ws + 0), 0, kor, key_bits,
                                                key_width, status);
        st = from_cuda(cudaGetLastError());
    }
    if (st == ISORT_OK) st = finish_status(status, s);
    scratch_free(ws, s);
    return st;
}

isort_status isort_count_round(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                               size_t n, int shift, int width, void* stream) {
    return count_round_entry<uint32_t>(keys_in, vals_in, keys_out, vals_out, n, shift, width, stream);
}

isort_status isort_count_round_u64(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                   uint32_t* vals_out, size_t n, int shift, int width, void* stream) {
    return count_round_entry<uint64_t>(keys_in, vals_in, keys_out, vals_out, n, shift, width, stream);
}


}  // extern "C"
