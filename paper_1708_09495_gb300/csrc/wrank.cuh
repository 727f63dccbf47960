// The count-sort round with warp ranking (u32 keys, digits of up to 8 bits):
// the rank-and-scatter step of one round of Section 3's serial radix-r sort
// (eq. Ts, output phase), run over chunks of whole tiles as in the chunked
// reduce-then-scan rounds of sweep.cuh. An alternative to the half-warp round
// of sweep.cuh (a launch shape the autotuner may pick).
//
// Per tile of THREADS x ITEMS keys:
//   1. the bulk-copy engine has put the tile's keys and payloads in shared
//      memory (two contiguous copies, issued two tiles ahead);
//   2. every warp ranks its 32 x ITEMS keys in input order. The eight ballots
//      of a digit's bits are the bit planes of the warp's 32 digits; lane x
//      forms the mask of the lanes whose low nibble equals x & 15 (and the one
//      for the high nibble), and every lane fetches the two masks of its own
//      nibbles with two shuffles: their AND is the set of its peers (the lanes
//      holding the same digit). The peers' highest lane adds their number to
//      the warp's counter of the digit with one shared-memory atomic, whose
//      old value (passed on by a shuffle) is the count of earlier keys of the
//      digit in the warp. Counters are 16 bits, two digits to a 32-bit word;
//   3. per word, an exclusive prefix over the warps plus the tile's digit
//      starts turn the counters into each (warp, digit)'s staging base;
//   4. keys with their payloads (one 64-bit pair) are staged by digit, read
//      back in order and written out: each digit's keys form one run that
//      lands at the chunk's running position of that digit.
// Shared-memory accesses indexed by digit: one atomic per group of peers, one
// base read and one staging store per key (the half-warp round makes five),
// at the price of the ballots and shuffles on the ALU side.
#pragma once

#include "common.cuh"
#include "runtime.h"
#include "sweep.cuh"

namespace isort {

constexpr int kWrBins = 256;
constexpr int kWrWords = kWrBins / 2;  // two 16-bit digit counters per word

// Four barriers per tile, and none between a tile's write-out and the next
// tile's ranking: a warp that has written its share of tile t goes on to rank
// tile t + 1 while others are still writing. What makes that safe: keys are
// staged into a buffer of their own (the input buffer is read again when
// staging, and is refilled with tile t + 2 only after tile t's staging
// barrier); each warp clears its own counters right after the staging barrier
// (no other warp touches them until the next tile's first barrier); the output
// offsets of tile t are replaced only after the next tile's first barrier,
// which every warp reaches after its write-out of tile t. The digit starts are
// formed by every warp from the group totals (no single-warp scan between
// barriers).
template <bool VALS, int THREADS, int ITEMS>
struct WpCfg {
    static_assert(THREADS % 128 == 0 && THREADS <= 1024 && ITEMS % 2 == 0, "groups of four warps; rank pairs");
    static constexpr int kWarps = THREADS / 32;
    static constexpr int kTile = THREADS * ITEMS;
    static_assert(kTile < 65536, "tile positions fit 16 bits");
    static constexpr int kGroups = THREADS / kWrWords;
    static constexpr size_t kBufBytes = (size_t)kTile * 4 * (VALS ? 2 : 1);
    static constexpr size_t kCntBytes = (size_t)kWarps * kWrWords * 4;
    // [input 0 | input 1 | staging | counters | group totals | run, delta | mbarriers]
    static constexpr size_t kStgOff = 2 * kBufBytes;
    static constexpr size_t kCntOff = 3 * kBufBytes;
    static constexpr size_t kGrpOff = kCntOff + kCntBytes;
    static constexpr size_t kTabOff = kGrpOff + (size_t)kGroups * kWrWords * 4;
    static constexpr size_t kBarOff = kTabOff + (size_t)2 * kWrBins * 4;
    static constexpr size_t kBytes = kBarOff + 2 * 8;
    static size_t smem_bytes() { return align_up(kBytes, 128); }
};

template <bool VALS, int THREADS, int ITEMS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_downsweep_wp(SweepArgs a) {
    using Cfg = WpCfg<VALS, THREADS, ITEMS>;
    constexpr int kTile = Cfg::kTile, kGroups = Cfg::kGroups;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned char* stg = smem + Cfg::kStgOff;
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + Cfg::kCntOff);
    uint32_t* my_cnt = s_cnt + warp * kWrWords;
    uint32_t* s_grp = reinterpret_cast<uint32_t*>(smem + Cfg::kGrpOff);
    uint32_t* s_run = reinterpret_cast<uint32_t*>(smem + Cfg::kTabOff);
    uint32_t* s_delta = s_run + kWrBins;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::kBarOff);
    if (Cfg::kBytes > dynamic_smem_size()) {  // the layout must fit the launch (uniform check)
        if (tid == 0) set_status(a.status, kStatBounds);
        return;
    }
    if (__syncthreads_or(tid == 0 && *(volatile uint32_t*)a.status != 0)) return;
    const uint32_t t_begin = blockIdx.x * a.chunk_tiles;
    const uint32_t t_end = min(a.num_tiles, t_begin + a.chunk_tiles);
    if (t_begin >= t_end) return;
    const uint32_t* keys_in = static_cast<const uint32_t*>(a.keys_in);
    uint32_t* keys_out = static_cast<uint32_t*>(a.keys_out);
    const int shift = a.shift;
    const uint32_t dmask = (uint32_t)a.bins - 1u;  // digits of up to 8 bits
    const uint32_t lt = lanemask_lt();
    uint32_t e[4];  // all ones where bit b of (lane & 15) is clear
#pragma unroll
    for (int b = 0; b < 4; ++b) e[b] = ((lane >> b) & 1) ? 0u : kFullMask;

    for (int i = tid; i < Cfg::kWarps * kWrWords; i += THREADS) s_cnt[i] = 0u;
    for (int d = tid; d < kWrBins; d += THREADS)
        s_run[d] = d < a.bins ? a.chunk_off[(size_t)blockIdx.x * a.bins + d] : 0u;  // [chunks][bins]
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto full_bulk_tile = [&](uint32_t t) -> bool { return a.use_bulk && (size_t)(t + 1) * kTile <= a.n; };
    auto issue_tile = [&](uint32_t t, int b) {
        unsigned char* dst = smem + (size_t)b * Cfg::kBufBytes;
        mbar_arrive_expect_tx(&bars[b], (uint32_t)Cfg::kBufBytes);
        bulk_load(dst, keys_in + (size_t)t * kTile, kTile * 4u, &bars[b]);
        if constexpr (VALS) bulk_load(dst + (size_t)kTile * 4, a.vals_in + (size_t)t * kTile, kTile * 4u, &bars[b]);
    };
    if (tid == 0) {
        if (full_bulk_tile(t_begin)) issue_tile(t_begin, 0);
        if (t_begin + 1 < t_end && full_bulk_tile(t_begin + 1)) issue_tile(t_begin + 1, 1);
    }
    uint32_t phase = 0u;  // bit b: parity of the next completion of buffer b's barrier
    for (uint32_t tile = t_begin; tile < t_end; ++tile) {
        const int b = (int)((tile - t_begin) & 1u);
        unsigned char* buf = smem + (size_t)b * Cfg::kBufBytes;
        const uint32_t* s_keys = reinterpret_cast<const uint32_t*>(buf);
        const uint32_t* s_vals = reinterpret_cast<const uint32_t*>(buf + (size_t)kTile * 4);
        const uint32_t tile_base = tile * (uint32_t)kTile;
        const uint32_t tile_n = min((uint32_t)kTile, a.n - tile_base);
        const bool bulk = full_bulk_tile(tile);
        bool ok = true;
        if (bulk) {
            ok = mbar_wait_bounded(&bars[b], (phase >> b) & 1u, a.limit_ns);
            phase ^= 1u << b;
            ok = __all_sync(kFullMask, ok);  // the ranking's votes need the whole warp
        } else {
            // the ragged tail (or unaligned input): plain loads, then a barrier
            uint32_t* sk = reinterpret_cast<uint32_t*>(buf);
            for (uint32_t j = tid; j < tile_n; j += THREADS) {
                sk[j] = keys_in[tile_base + j];
                if constexpr (VALS) sk[kTile + j] = a.vals_in[tile_base + j];
            }
            __syncthreads();
        }
        const bool full = tile_n == (uint32_t)kTile;

        // ---- rank in input order (item i of lane l is key warp*32*ITEMS + 32 i + l)
        uint32_t rank2[ITEMS / 2];
        if (ok) {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t j = (uint32_t)(warp * ITEMS * 32 + i * 32 + lane);
                const bool valid = full || j < tile_n;
                const uint32_t d = valid ? (s_keys[j] >> shift) & dmask : 0u;
                uint32_t bp[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) bp[q] = __ballot_sync(kFullMask, (d >> q) & 1u);
                const uint32_t ml = (bp[0] ^ e[0]) & (bp[1] ^ e[1]) & (bp[2] ^ e[2]) & (bp[3] ^ e[3]);
                const uint32_t mh = (bp[4] ^ e[0]) & (bp[5] ^ e[1]) & (bp[6] ^ e[2]) & (bp[7] ^ e[3]);
                uint32_t peers = __shfl_sync(kFullMask, ml, (int)(d & 15u)) & __shfl_sync(kFullMask, mh, (int)(d >> 4));
                if (!full) peers &= __ballot_sync(kFullMask, valid);
                const int leader = 31 - __clz(peers);
                const uint32_t hsh = (d & 1u) * 16u;
                uint32_t old = 0;
                if (valid && lane == leader) old = atomicAdd(&my_cnt[d >> 1], (uint32_t)__popc(peers) << hsh);
                old = __shfl_sync(kFullMask, old, leader);
                const uint32_t r = ((old >> hsh) & 0xFFFFu) + (uint32_t)__popc(peers & lt);
                if (i & 1) rank2[i / 2] |= r << 16;
                else rank2[i / 2] = r;
                __syncwarp();
            }
        }
        // (A) every warp has ranked this tile and written out the previous one
        if (__syncthreads_or(!ok)) {
            // a bulk copy never completed: record it, wait (bounded) for the
            // copies still in flight into either buffer, and stop
            if (tid == 0) {
                set_status(a.status, kStatTimeout);
                // this tile's copy (the phase already waited for), unless this
                // thread saw it complete, and the next tile's copy
                if (bulk && !ok) mbar_wait_bounded(&bars[b], ((phase >> b) & 1u) ^ 1u, a.limit_ns);
                if (tile + 1 < t_end && full_bulk_tile(tile + 1))
                    mbar_wait_bounded(&bars[b ^ 1], (phase >> (b ^ 1)) & 1u, a.limit_ns);
            }
            return;
        }

        // ---- per word (two digits): prefix over the four warps of each group
        {
            const int q = tid & (kWrWords - 1), g = tid >> 7;
            uint32_t sum = 0;
#pragma unroll
            for (int w = g * 4; w < g * 4 + 4; ++w) {
                const uint32_t c = s_cnt[w * kWrWords + q];
                s_cnt[w * kWrWords + q] = sum;
                sum += c;  // each half stays below 2^16 (a tile has fewer keys)
            }
            s_grp[g * kWrWords + q] = sum;
        }
        __syncthreads();  // (B)
        {
            // every warp forms the word starts: lane l sums words 4l..4l+3 over
            // the groups, then a warp scan; thread (q, g) takes word q's start
            uint32_t wt[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int g = 0; g < kGroups; ++g) {
                const uint4 x = reinterpret_cast<const uint4*>(s_grp + g * kWrWords)[lane];
                wt[0] += x.x;
                wt[1] += x.y;
                wt[2] += x.z;
                wt[3] += x.w;
            }
            // packed word totals hold two 16-bit digit totals: digit starts need
            // a carry from the low digit to the high one, so scan digit totals
            uint32_t dt[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                dt[2 * k] = wt[k] & 0xFFFFu;
                dt[2 * k + 1] = wt[k] >> 16;
            }
            uint32_t loc = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) loc += dt[k];
            uint32_t x = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFullMask, x, o);
                if (lane >= o) x += y;
            }
            uint32_t st[4];  // word starts, packed (start of digit 2w | start of digit 2w + 1 << 16)
            uint32_t r = x - loc;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                st[k] = r | ((r + dt[2 * k]) << 16);
                r += dt[2 * k] + dt[2 * k + 1];
            }
            const int q = tid & (kWrWords - 1), g = tid >> 7;
            const int src = q >> 2, slot = q & 3;
            const uint32_t s0 = __shfl_sync(kFullMask, st[0], src);
            const uint32_t s1 = __shfl_sync(kFullMask, st[1], src);
            const uint32_t s2 = __shfl_sync(kFullMask, st[2], src);
            const uint32_t s3 = __shfl_sync(kFullMask, st[3], src);
            const uint32_t wst = slot == 0 ? s0 : slot == 1 ? s1 : slot == 2 ? s2 : s3;
            uint32_t gp = 0;  // this group's prefix over earlier groups (packed)
            for (int gg = 0; gg < g; ++gg) gp += s_grp[gg * kWrWords + q];
            const uint32_t add = wst + gp;
#pragma unroll
            for (int w = g * 4; w < g * 4 + 4; ++w) s_cnt[w * kWrWords + q] += add;
            if (g == 0) {  // output offsets of the word's two digits; advance the running positions
                uint32_t tot = 0;
                for (int gg = 0; gg < kGroups; ++gg) tot += s_grp[gg * kWrWords + q];
                const uint32_t d0 = 2 * q, d1 = 2 * q + 1;
                const uint32_t r0 = s_run[d0], r1 = s_run[d1];
                s_delta[d0] = r0 - (wst & 0xFFFFu);
                s_delta[d1] = r1 - (wst >> 16);
                s_run[d0] = r0 + (tot & 0xFFFFu);
                s_run[d1] = r1 + (tot >> 16);
            }
        }
        __syncthreads();  // (C)

        // ---- stage by digit (keys and payloads read again from the input buffer)
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t j = (uint32_t)(warp * ITEMS * 32 + i * 32 + lane);
            if (full || j < tile_n) {
                const uint32_t k = s_keys[j];
                const uint32_t d = (k >> shift) & dmask;
                const uint32_t pos = ((my_cnt[d >> 1] >> ((d & 1u) * 16u)) & 0xFFFFu) +
                                     ((rank2[i / 2] >> ((i & 1) * 16)) & 0xFFFFu);
                if (pos < (uint32_t)kTile) {
                    if constexpr (VALS) reinterpret_cast<uint2*>(stg)[pos] = make_uint2(k, s_vals[j]);
                    else reinterpret_cast<uint32_t*>(stg)[pos] = k;
                }
            }
        }
        __syncthreads();  // (D)
        // the input buffer is free: start copying tile + 2 into it
        if (tid == 0 && tile + 2 < t_end && full_bulk_tile(tile + 2)) {
            fence_proxy_async_smem();
            issue_tile(tile + 2, b);
        }
        // this warp's counters are read for the last time in staging: clear them
        reinterpret_cast<uint4*>(my_cnt)[lane] = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();  // the clears are seen by the next tile's atomics of any lane
        // ---- write runs of equal digits to their places
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t j = (uint32_t)(tid + i * THREADS);
            if (full || j < tile_n) {
                uint32_t k, v = 0;
                if constexpr (VALS) {
                    const uint2 p = reinterpret_cast<const uint2*>(stg)[j];
                    k = p.x;
                    v = p.y;
                } else {
                    k = reinterpret_cast<const uint32_t*>(stg)[j];
                }
                const uint32_t dst = s_delta[(k >> shift) & dmask] + j;
                if (dst < a.n) {
                    keys_out[dst] = k;
                    if constexpr (VALS) a.vals_out[dst] = v;
                } else {
                    set_status(a.status, kStatBounds);
                }
            }
        }
    }
}

}  // namespace isort
