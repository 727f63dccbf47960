// The count-sort rounds by chunked reduce-then-scan (the default radix path):
// per-chunk digit counts, chunk offsets, and the rank-and-scatter round in one
// of its launch shapes, with the optional launch-shape autotuning.
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "runtime.h"
#include "sweep.cuh"
#include "tune.h"
#include "wrank.cuh"

namespace isort {

template <typename K>
isort_status radix_device_rts(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n, int key_bits,
                              int rb, cudaStream_t s, int shape = -1);

namespace {

// ---- chunked reduce-then-scan rounds
// shapes 0-3: the generic chunked round; 4: the half-warp ranking variant (u32
// keys and 8-bit digits; other cases take the generic round of the same tile).
// Half-warp shapes 256 x 16 and 512 x 16 measured slower and are not built.
// 5: the warp-ranked round (wrank.cuh; u32 keys and digits of up to 8 bits;
// other cases take shape 4).
constexpr int kSweepThreads[] = {256, 512, 256, 512, 512, 512};
constexpr int kSweepItems[] = {16, 16, 8, 8, 8, 8};
constexpr int kNumShapes = (int)(sizeof(kSweepThreads) / sizeof(kSweepThreads[0]));

int sweep_tile(int sh) { return kSweepThreads[sh] * kSweepItems[sh]; }

template <typename K, bool VALS, int THREADS, int ITEMS>
isort_status sweep_occupancy(int bins, int* per_sm) {
    using Cfg = SweepCfg<K, VALS, THREADS, ITEMS>;
    const size_t smem = Cfg::smem_bytes(bins);
    if (smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    auto k8 = k_downsweep<K, VALS, THREADS, ITEMS, 8, RadixDigit>;
    auto k0 = k_downsweep<K, VALS, THREADS, ITEMS, 0, RadixDigit>;
    ISORT_TRY_CUDA(cudaFuncSetAttribute(k8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ISORT_TRY_CUDA(cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int p8 = 0, p0 = 0;
    ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p8, k8, THREADS, smem));
    ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p0, k0, THREADS, smem));
    *per_sm = std::min(p8, p0);
    return *per_sm >= 1 ? ISORT_OK : ISORT_ERR_UNSUPPORTED;
}

template <typename K, bool VALS, int THREADS, int ITEMS>
isort_status launch_sweep(const SweepArgs& a, uint32_t chunks, cudaStream_t s, const char* name = "downsweep") {
    using Cfg = SweepCfg<K, VALS, THREADS, ITEMS>;
    LaunchScope ls(name, s);
    RadixDigit df;
    df.shift = a.shift;
    df.mask = (uint32_t)a.bins - 1u;
    if (a.width == 8)
        k_downsweep<K, VALS, THREADS, ITEMS, 8, RadixDigit><<<chunks, THREADS, Cfg::smem_bytes(a.bins), s>>>(a, df);
    else
        k_downsweep<K, VALS, THREADS, ITEMS, 0, RadixDigit><<<chunks, THREADS, Cfg::smem_bytes(a.bins), s>>>(a, df);
    return from_cuda(cudaGetLastError());
}

template <typename K, bool VALS, int THREADS, int ITEMS>
isort_status sweep_occupancy_hw(int* per_sm) {
    const size_t smem = HwCfg<K, VALS, THREADS, ITEMS>::smem_bytes();
    if (smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    auto kern = k_downsweep_hw<K, VALS, THREADS, ITEMS>;
    ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, THREADS, smem));
    return *per_sm >= 1 ? ISORT_OK : ISORT_ERR_UNSUPPORTED;
}

template <typename K, bool VALS, int THREADS, int ITEMS>
isort_status launch_sweep_hw(const SweepArgs& a, uint32_t chunks, cudaStream_t s) {
    LaunchScope ls("downsweep", s);
    k_downsweep_hw<K, VALS, THREADS, ITEMS><<<chunks, THREADS, HwCfg<K, VALS, THREADS, ITEMS>::smem_bytes(), s>>>(a);
    return from_cuda(cudaGetLastError());
}

// The half-warp round for u32 keys and 8-bit digits; other cases take the
// generic round of the same tile.
template <typename K, bool VALS, int THREADS, int ITEMS>
isort_status sweep_hw_or_generic(bool occupancy_only, int bins, int* per_sm, const SweepArgs* a, uint32_t chunks,
                                 cudaStream_t s) {
    if constexpr (sizeof(K) == 4) {  // with u64 keys the padded buffers leave one CTA per SM
        if (bins <= kHwBins) {
            if (occupancy_only) return sweep_occupancy_hw<K, VALS, THREADS, ITEMS>(per_sm);
            int tmp = 0;  // sets the kernel's shared-memory attribute (the sizing may have been for a wider pass)
            const isort_status so = sweep_occupancy_hw<K, VALS, THREADS, ITEMS>(&tmp);
            if (so != ISORT_OK) return so;
            return launch_sweep_hw<K, VALS, THREADS, ITEMS>(*a, chunks, s);
        }
    }
    if (occupancy_only) return sweep_occupancy<K, VALS, THREADS, ITEMS>(bins, per_sm);
    int tmp = 0;
    const isort_status so = sweep_occupancy<K, VALS, THREADS, ITEMS>(bins, &tmp);  // sets the kernel's attribute
    if (so != ISORT_OK) return so;
    return launch_sweep<K, VALS, THREADS, ITEMS>(*a, chunks, s);
}

// The pipelined warp-ranked round (u32 keys, digits of up to 8 bits).
template <bool VALS, int THREADS, int ITEMS, int MINB>
isort_status sweep_wp(bool occupancy_only, int* per_sm, const SweepArgs* a, uint32_t chunks, cudaStream_t s) {
    using Cfg = WpCfg<VALS, THREADS, ITEMS>;
    const size_t smem = Cfg::smem_bytes();
    if (smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    auto kern = k_downsweep_wp<VALS, THREADS, ITEMS, MINB>;
    ISORT_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (occupancy_only) {
        ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, THREADS, smem));
        return *per_sm >= 1 ? ISORT_OK : ISORT_ERR_UNSUPPORTED;
    }
    LaunchScope ls("downsweep", s);
    kern<<<chunks, THREADS, smem, s>>>(*a);
    return from_cuda(cudaGetLastError());
}

// name: the launch's name in the library's profile ("downsweep"; the second
// form of a two-form round is "downsweep_heavy")
template <typename K, bool VALS>
isort_status sweep_dispatch(int sh, bool occupancy_only, int bins, int* per_sm, const SweepArgs* a, uint32_t chunks,
                            cudaStream_t s, const char* name = "downsweep") {
    if constexpr (sizeof(K) == 4) {
        if (sh == 5) return sweep_wp<VALS, 512, 8, 2>(occupancy_only, per_sm, a, chunks, s);
    }
    switch (sh) {
        case 0:
            return occupancy_only ? sweep_occupancy<K, VALS, 256, 16>(bins, per_sm)
                                  : launch_sweep<K, VALS, 256, 16>(*a, chunks, s, name);
        case 1:
            return occupancy_only ? sweep_occupancy<K, VALS, 512, 16>(bins, per_sm)
                                  : launch_sweep<K, VALS, 512, 16>(*a, chunks, s, name);
        case 2:
            return occupancy_only ? sweep_occupancy<K, VALS, 256, 8>(bins, per_sm)
                                  : launch_sweep<K, VALS, 256, 8>(*a, chunks, s, name);
        case 4:
            return sweep_hw_or_generic<K, VALS, 512, 8>(occupancy_only, bins, per_sm, a, chunks, s);
        default:
            return occupancy_only ? sweep_occupancy<K, VALS, 512, 8>(bins, per_sm)
                                  : launch_sweep<K, VALS, 512, 8>(*a, chunks, s, name);
    }
}


template <typename K>
int autotuned_shape(const K* kin, bool vals, size_t n, int key_bits, int rb, cudaStream_t s);

// ---------------------------------------------------------------- autotuning
//
// With autotuning on, the first chunked-round sort of each kind (key width,
// payload or not, narrow or wide digits, log2 n; n >= 2^20) times the
// candidate launch shapes once on synthetic keys of the same size and keeps
// the fastest; choices are read from and appended to a cache file.
struct AutoKey {
    int key_bytes, vals, wide, log2n;
    bool operator<(const AutoKey& o) const {
        return std::tie(key_bytes, vals, wide, log2n) < std::tie(o.key_bytes, o.vals, o.wide, o.log2n);
    }
};

struct AutoState {
    std::mutex mu;
    bool enabled = false;
    std::string path;
    std::map<AutoKey, int> shapes;
};

AutoState& auto_state() {
    static AutoState st;
    return st;
}

template <typename K>
__global__ void k_fill_random(K* k, uint32_t* v, size_t n, uint64_t seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;  // SplitMix64 (Steele, Lea & Flood 2014)
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        k[i] = sizeof(K) == 4 ? (K)(z >> 32) : (K)z;
        if (v) v[i] = (uint32_t)i;
    }
}

template <typename K>
int autotuned_shape(const K* kin, bool vals, size_t n, int key_bits, int rb, cudaStream_t s) {
    (void)kin;
    const int bins = 1 << rb;
    const int fixed = bins <= 256 ? (vals ? tune().sweep_small : tune().sweep_keys) : tune().sweep_large;
    AutoState& as = auto_state();
    std::lock_guard<std::mutex> lk(as.mu);
    if (!as.enabled || n < (size_t(1) << 20)) return fixed;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    if (cap == cudaStreamCaptureStatusActive) return fixed;  // no timing inside a capture
    int log2n = 0;
    while ((size_t(1) << (log2n + 1)) <= n) ++log2n;
    const AutoKey key{(int)sizeof(K), vals ? 1 : 0, bins > 256 ? 1 : 0, log2n};
    const auto it = as.shapes.find(key);
    if (it != as.shapes.end()) return it->second;

    std::vector<int> cands = bins <= 256 ? std::vector<int>{4, 5, 3, 1} : std::vector<int>{2, 0};
    const size_t m = size_t(1) << log2n;
    const size_t kb = align_up(m * sizeof(K), 256);
    unsigned char* buf = nullptr;
    if (scratch_alloc((void**)&buf, 2 * kb + (vals ? 2 * align_up(m * 4, 256) : 0), s) != ISORT_OK) return fixed;
    K* k0 = reinterpret_cast<K*>(buf);
    K* k1 = reinterpret_cast<K*>(buf + kb);
    uint32_t* v0 = vals ? reinterpret_cast<uint32_t*>(buf + 2 * kb) : nullptr;
    uint32_t* v1 = vals ? reinterpret_cast<uint32_t*>(buf + 2 * kb + align_up(m * 4, 256)) : nullptr;
    k_fill_random<K><<<sm_count() * 4, 256, 0, s>>>(k0, v0, m, 0x5EEDull + (uint64_t)log2n);
    int best = fixed;
    float best_ms = 1e30f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int c : cands) {
        float ms = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {  // one warm-up, two timed
            cudaEventRecord(e0, s);
            ok = radix_device_rts<K>(k0, v0, k1, v1, m, key_bits, rb, s, c) == ISORT_OK;
            cudaEventRecord(e1, s);
            if (ok && cudaEventSynchronize(e1) == cudaSuccess) {
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms += t;
            } else {
                ok = false;
            }
        }
        if (ok && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    scratch_free(buf, s);
    cudaStreamSynchronize(s);
    as.shapes[key] = best;
    if (!as.path.empty()) {
        if (FILE* f = std::fopen(as.path.c_str(), "a")) {
            std::fprintf(f, "%d %d %d %d %d\n", key.key_bytes, key.vals, key.wide, key.log2n, best);
            std::fclose(f);
        }
    }
    return best;
}


}  // namespace

template <typename K>
isort_status radix_device_rts(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n, int key_bits,
                              int rb, cudaStream_t s, int shape) {
    const int key_width = (int)sizeof(K) * 8;
    // The passes: one per round of ceil(key_bits / rb); a round whose digit is
    // wider than 8 bits runs as two stable passes over its low and high
    // halves (11 = 6 + 5, 16 = 8 + 8): together they are the round's stable
    // count-sort on the whole digit. A one-pass round of 9..12 bits scans
    // 2^w counters per warp on every tile and keeps one CTA per SM (measured
    // slower than its two passes); a one-pass 2^16-way round would need 2^16
    // counters per chunk (256 KB, above the shared memory of an SM).
    const int split = std::min(tune().split, 12);
    int pass_shift[64], pass_width[64];
    int rounds = 0, max_width = 0;
    for (int shift = 0; shift < key_bits; shift += rb) {
        const int w = std::min(rb, key_bits - shift);
        const int lo = w > split ? (w + 1) / 2 : w;
        pass_shift[rounds] = shift;
        pass_width[rounds++] = lo;
        if (w > lo) {
            pass_shift[rounds] = shift + lo;
            pass_width[rounds++] = w - lo;
        }
        max_width = std::max(max_width, lo);
    }
    const int bins = 1 << max_width;
    const bool vals = vin != nullptr;
    const bool inplace = (const void*)kin == (const void*)kout;
    int sh = shape >= 0 ? shape : autotuned_shape<K>(kin, vals, n, key_bits, max_width, s);
    if (sh == 5 && (sizeof(K) != 4 || bins > kWrBins)) sh = bins <= 256 ? 4 : 2;  // warp-ranked: u32, <= 8 bits
    int per_sm = 0;
    isort_status st = vals ? sweep_dispatch<K, true>(sh, true, bins, &per_sm, nullptr, 0, s)
                           : sweep_dispatch<K, false>(sh, true, bins, &per_sm, nullptr, 0, s);
    if (st != ISORT_OK) return st;
    // pairs at the half-warp shape: every round launches the half-warp form
    // and the per-warp-mask form of the same tile (3) back to back, and the
    // round's digit counts pick the one that runs. Runs of repeated keys put
    // a half-warp's 16 atomics on one ranking word; the per-warp form then
    // takes such a warp in one step.
    const bool dual = sh == 4 && vals && sizeof(K) == 4 && bins <= kHwBins && tune().heavy != 0 &&
                      sweep_tile(3) == sweep_tile(4);
    if (dual) {
        int per_sm3 = 0;  // sets the second form's shared-memory attribute
        st = sweep_dispatch<K, true>(3, true, bins, &per_sm3, nullptr, 0, s);
        if (st != ISORT_OK) return st;
    }
    const uint32_t tile = (uint32_t)sweep_tile(sh);
    const uint32_t num_tiles = (uint32_t)((n + tile - 1) / tile);
    const uint32_t want = (uint32_t)per_sm * (uint32_t)sm_count();
    const uint32_t chunk_tiles = (num_tiles + want - 1) / want;
    const uint32_t chunks = (num_tiles + chunk_tiles - 1) / chunk_tiles;
    const int nsub = bins <= 256 ? 16 : (bins <= 1024 ? 4 : 1);

    int nbuf;
    if (inplace) nbuf = (rounds % 2 == 0) ? 1 : (rounds == 1 ? 1 : 2);
    else nbuf = rounds == 1 ? 0 : 1;
    const size_t buf_bytes = align_up(n * sizeof(K), 256) + (vals ? align_up(n * 4, 256) : 0);
    const size_t ctl = 256 + 2 * align_up((size_t)chunks * bins * 4, 256);
    unsigned char* ws = nullptr;
    st = scratch_alloc((void**)&ws, ctl + (size_t)nbuf * buf_bytes, s);
    if (st != ISORT_OK) return st;
    uint32_t* status = reinterpret_cast<uint32_t*>(ws);
    unsigned long long* key_or = reinterpret_cast<unsigned long long*>(ws + 8);
    uint32_t* heavy = reinterpret_cast<uint32_t*>(ws + 16);  // the round's digit counts have a heavy digit
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + 256);
    uint32_t* coff = reinterpret_cast<uint32_t*>(ws + 256 + align_up((size_t)chunks * bins * 4, 256));
    K* wk[2] = {nullptr, nullptr};
    uint32_t* wv[2] = {nullptr, nullptr};
    for (int i = 0; i < nbuf; ++i) {
        unsigned char* p = ws + ctl + (size_t)i * buf_bytes;
        wk[i] = reinterpret_cast<K*>(p);
        wv[i] = vals ? reinterpret_cast<uint32_t*>(p + align_up(n * sizeof(K), 256)) : nullptr;
    }
    auto fail = [&](isort_status e) {
        scratch_free(ws, s);
        return e;
    };
    cudaError_t ce = cudaMemsetAsync(ws, 0, 256, s);
    if (ce != cudaSuccess) return fail(from_cuda(ce));
    const size_t hist_smem = (size_t)nsub * bins * 4;
    ce = cudaFuncSetAttribute(k_chunk_hist<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hist_smem);
    if (ce != cudaSuccess) return fail(from_cuda(ce));
    const K* src_k = kin;
    const uint32_t* src_v = vin;
    for (int d = 0; d < rounds; ++d) {
        K* dk;
        uint32_t* dv;
        if (!inplace) {
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
        } else if (d == rounds - 1) {
            dk = kout;
            dv = vout;
        } else {
            dk = wk[d % 2];
            dv = wv[d % 2];
        }
        const int shift = pass_shift[d];
        const int width = pass_width[d];
        {
            // several CTAs per chunk when chunks are fewer than two per SM
            const int parts = std::max(1, (2 * sm_count() + (int)chunks - 1) / (int)chunks);
            if (parts > 1) {
                ce = cudaMemsetAsync(hist, 0, (size_t)chunks * (1u << width) * 4, s);
                if (ce != cudaSuccess) return fail(from_cuda(ce));
            }
            LaunchScope ls("chunk_hist", s);
            k_chunk_hist<K><<<chunks * parts, kChunkHistThreads, hist_smem, s>>>(
                src_k, (uint32_t)n, shift, width, chunk_tiles * tile, nsub, hist, d == 0 ? key_or : nullptr, parts);
            ce = cudaGetLastError();
            if (ce != cudaSuccess) return fail(from_cuda(ce));
        }
        {
            LaunchScope ls("chunk_scan", s);
            const int sbins = 1 << width;
            const int groups = sbins >= kChunkScanThreads ? 1 : kChunkScanThreads / sbins;
            k_chunk_scan<<<1, kChunkScanThreads, (size_t)(groups + 1) * sbins * 4, s>>>(
                hist, (int)chunks, 1 << width, coff, d == 0 ? key_or : nullptr, key_bits, key_width, status,
                dual ? heavy : nullptr);
            ce = cudaGetLastError();
            if (ce != cudaSuccess) return fail(from_cuda(ce));
        }
        SweepArgs a;
        a.keys_in = src_k;
        a.vals_in = src_v;
        a.keys_out = dk;
        a.vals_out = dv;
        a.n = (uint32_t)n;
        a.shift = shift;
        a.width = width;
        a.bins = 1 << width;
        a.chunk_off = coff;
        a.chunk_tiles = chunk_tiles;
        a.num_tiles = num_tiles;
        a.status = status;
        a.limit_ns = spin_limit_ns();
        a.use_bulk = (((uintptr_t)src_k % 16) == 0) && (!vals || ((uintptr_t)src_v % 16) == 0);
        if (dual) {
            a.heavy = heavy;
            a.run_if_heavy = 0;
        }
        st = vals ? sweep_dispatch<K, true>(sh, false, a.bins, &per_sm, &a, chunks, s)
                  : sweep_dispatch<K, false>(sh, false, a.bins, &per_sm, &a, chunks, s);
        if (st != ISORT_OK) return fail(st);
        if (dual) {
            a.run_if_heavy = 1;
            st = sweep_dispatch<K, true>(3, false, a.bins, &per_sm, &a, chunks, s, "downsweep_heavy");
            if (st != ISORT_OK) return fail(st);
        }
        src_k = dk;
        src_v = dv;
    }
    if (inplace && rounds == 1) {
        ce = cudaMemcpyAsync(kout, wk[0], n * sizeof(K), cudaMemcpyDeviceToDevice, s);
        if (ce == cudaSuccess && vals) ce = cudaMemcpyAsync(vout, wv[0], n * 4, cudaMemcpyDeviceToDevice, s);
        if (ce != cudaSuccess) return fail(from_cuda(ce));
    }
    st = finish_status(status, s);
    scratch_free(ws, s);
    return st;
}

// Sorts device buffers. kin/vin are read; the result lands in kout/vout.
// If kin == kout the sort is in place (vin == vout then too).

template isort_status radix_device_rts<uint32_t>(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, size_t, int,
                                                 int, cudaStream_t, int);
template isort_status radix_device_rts<uint64_t>(const uint64_t*, const uint32_t*, uint64_t*, uint32_t*, size_t, int,
                                                 int, cudaStream_t, int);

bool autotune_config(std::string* path) {
    AutoState& as = auto_state();
    std::lock_guard<std::mutex> lk(as.mu);
    if (path) *path = as.path;
    return as.enabled;
}

}  // namespace isort

using namespace isort;

extern "C" {

isort_status isort_autotune(int enable, const char* cache_path) {
    if (enable != 0 && enable != 1) return ISORT_ERR_INVALID_ARG;
    {
        AutoState& as = auto_state();
        std::lock_guard<std::mutex> lk(as.mu);
        as.enabled = enable == 1;
        as.shapes.clear();
        as.path = cache_path ? cache_path : "";
        if (as.enabled && cache_path) {
            if (FILE* f = std::fopen(cache_path, "r")) {
                // "key_bytes payload wide log2n shape" lines; lines of other
                // kinds (the segmented router's) are read by their owner
                char ln[256];
                while (std::fgets(ln, sizeof(ln), f)) {
                    AutoKey k;
                    int shape = 0;
                    if (std::sscanf(ln, "%d %d %d %d %d", &k.key_bytes, &k.vals, &k.wide, &k.log2n, &shape) == 5 &&
                        shape >= 0 && shape < kNumShapes)
                        as.shapes[k] = shape;
                }
                std::fclose(f);
            }
        }
    }
    router_autotune_reset();
    return ISORT_OK;
}

}  // extern "C"
