// Batched segmented sort: many arrays of uneven size sorted by one launch
// sequence (captured in a CUDA graph). Each segment is routed by its length,
// following the paper's observation that the block networks win for small n
// and count-sort rounds for larger n (Gerbessiotis, arXiv:1708.09495, Section 4,
// Observations 5 and 6):
//   len <= T_oet           OET in one warp, one key per lane (Section 2)
//   len <= T_btn_warp      BTN in one warp, 8 keys per lane (Section 2, eq. Tb)
//   len <= T_btn_cta       BTN over a 512-thread CTA, 8 keys per thread
//   len <= 8 * 8192        count-sort rounds (8-bit digits, Section 3) entirely
//                          on chip: a thread-block cluster of C = 1, 2, 4 or 8
//                          CTAs holds the segment, 8192 keys per CTA; each round
//                          ranks keys per CTA, exchanges the C digit histograms
//                          through distributed shared memory, and scatters
//                          every key straight into the shared memory of the CTA
//                          that owns its new position. HBM sees one read and
//                          one write per key.
//   longer                 the global LSD path, one segment at a time (host
//                          driven; only in the synchronous status mode).
// Routing happens on the device: a classification kernel builds one work
// list per class, and persistent kernels pull segments from their list.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "net.cuh"
#include "runtime.h"

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

enum : int { kClsOet = 0, kClsBtnWarp, kClsBtnCta, kClsC1, kClsC2, kClsC4, kClsC8, kClsBig, kNumCls };

struct SegThresholds {
    uint32_t oet;       // <= : OET in a warp (at most 32)
    uint32_t btn_warp;  // <= : BTN in a warp (at most 256)
    uint32_t btn_cta;   // <= : BTN over a CTA (at most 4096)
};

struct SegCtl {
    uint32_t status;
    uint32_t counts[kNumCls];
    uint32_t work[kNumCls];
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
        else if (L <= th.btn_cta) c = kClsBtnCta;
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
    const int lane = threadIdx.x & 31;
    const uint32_t cnt = ctl->counts[cls];
    while (true) {
        uint32_t q = 0;
        if (lane == 0) q = atomicAdd(&ctl->work[cls], 1u);
        q = __shfl_sync(kFullMask, q, 0);
        if (q >= cnt) break;
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

// One CTA per segment: BTN with p = next_pow2(len / 8) <= 512 blocks of 8.
__global__ void __launch_bounds__(512) k_seg_btn_cta(uint32_t* keys, uint32_t* vals, const uint64_t* off,
                                                     const uint32_t* list, SegCtl* ctl, int cls, uint32_t range_mask) {
    extern __shared__ __align__(16) uint64_t s_x[];
    __shared__ uint32_t s_q;
    const uint32_t cnt = ctl->counts[cls];
    while (true) {
        if (threadIdx.x == 0) s_q = atomicAdd(&ctl->work[cls], 1u);
        __syncthreads();
        const uint32_t q = s_q;
        __syncthreads();
        if (q >= cnt) break;
        const uint32_t s = list[q];
        const uint64_t lo = off[s];
        const uint32_t L = (uint32_t)(off[s + 1] - lo);
        int p = 1;
        while ((uint32_t)(p * 8) < L) p <<= 1;
        net::btn_block<8>(keys + lo, vals ? vals + lo : nullptr, L, p, s_x, nullptr, range_mask, &ctl->status);
    }
}

struct ClusterArgs {
    uint32_t* keys;
    uint32_t* vals;
    const uint64_t* off;
    const uint32_t* list;
    SegCtl* ctl;
    int cls;
    int key_bits;
    const uint32_t* seg_lo;   // optional: segment s's keys lie in [seg_lo[s], seg_lo[s] + 2^seg_bits[s])
    const uint8_t* seg_bits;  //   and are sorted on key - seg_lo[s] over seg_bits[s] bits
};

constexpr size_t cluster_smem_bytes(bool vals) {
    return (size_t)kSegChunk * 4 * (vals ? 2 : 1) + (size_t)kSegWarps * kSegBins * 2 + (size_t)kSegBins * 4 * 3 +
           64 * 4;
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
    uint32_t* s_misc = s_base + kSegBins;  // [0] work item, [1] range flag, [8..] warp sums
    // (the launch always provides cluster_smem_bytes; every CTA of a cluster
    // sees the same size, so a failed check leaves the cluster together)
    if ((size_t)(reinterpret_cast<unsigned char*>(s_misc + 64) - smem) > dynamic_smem_size()) {
        if (threadIdx.x == 0) set_status(&a.ctl->status, kStatBounds);
        return;
    }

    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t r = C == 1 ? 0u : cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t cnt = a.ctl->counts[a.cls];

    for (int i = tid; i < kSegWarps * kSegBins; i += kSegThreads) s_cnt[i] = 0;

    while (true) {
        if (r == 0 && tid == 0) s_misc[0] = atomicAdd(&a.ctl->work[a.cls], 1u);
        cluster.sync();
        const uint32_t q = C == 1 ? s_misc[0] : *cluster.map_shared_rank(&s_misc[0], 0);
        if (q >= cnt) break;
        const uint32_t s = a.list[q];
        const uint64_t lo = a.off[s];
        const uint32_t L = (uint32_t)(a.off[s + 1] - lo);
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
            // rank each key among equal digits of its warp, in input order
#pragma unroll
            for (int i = 0; i < kSegItems; ++i) {
                const uint32_t j = (uint32_t)(warp * kSegItems * 32 + i * 32 + lane);
                const bool valid = j < my_n;
                const uint32_t dg = ((k[i] - kbase) >> shift) & 0xffu;
                uint32_t peers = __ballot_sync(kFullMask, valid);
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const bool bit = (dg >> b) & 1u;
                    const uint32_t bal = __ballot_sync(kFullMask, bit);
                    peers &= bit ? bal : ~bal;
                }
                const uint32_t below = (uint32_t)__popc(peers & lanemask_lt());
                const uint32_t c = valid ? (uint32_t)s_cnt[warp * kSegBins + dg] : 0u;
                rank[i] = c + below;
                __syncwarp();
                if (valid && below + 1 == (uint32_t)__popc(peers)) s_cnt[warp * kSegBins + dg] = (uint16_t)(c + below + 1);
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
#pragma unroll
        for (int i = 0; i < kSegItems; ++i) {
            const uint32_t j = (uint32_t)(warp * kSegItems * 32 + i * 32 + lane);
            if (j < my_n) {
                gk[j] = k[i];
                if constexpr (VALS) gv[j] = v[i];
            }
        }
    }
    cluster.sync();  // no CTA leaves while others may still read its shared memory
}

// ---------------------------------------------------------------- host side

struct Tuned {
    SegThresholds th{32, 256, 4096};
};

Tuned& seg_tune() {
    static Tuned t;
    return t;
}

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

// Enqueues classification and every class kernel on `s`.
isort_status enqueue_segmented(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint32_t nseg, int key_bits,
                               SegCtl* ctl, uint32_t* lists, int big_ok, cudaStream_t s,
                               const uint32_t* seg_lo = nullptr, const uint8_t* seg_bits = nullptr) {
    const SegThresholds th = seg_tune().th;
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
        isort_status st = c == kClsC8   ? launch_cluster<8>(v, a, s)
                          : c == kClsC4 ? launch_cluster<4>(v, a, s)
                          : c == kClsC2 ? launch_cluster<2>(v, a, s)
                                        : launch_cluster<1>(v, a, s);
        if (st != ISORT_OK) return st;
    }
    {
        const size_t smem = (size_t)8 * 512 * 8;
        ISORT_TRY_CUDA(cudaFuncSetAttribute(k_seg_btn_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        ISORT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seg_btn_cta, 512, smem));
        LaunchScope ls("seg_btn_cta", s);
        k_seg_btn_cta<<<std::max(1, per_sm) * sm_count(), 512, smem, s>>>(keys, vals, off, lists + (size_t)kClsBtnCta * nseg,
                                                                         ctl, kClsBtnCta, range_mask);
        ISORT_TRY_CUDA(cudaGetLastError());
    }
    {
        LaunchScope ls("seg_btn_warp", s);
        k_seg_warp<false><<<4 * sm_count(), 256, 0, s>>>(keys, vals, off, lists + (size_t)kClsBtnWarp * nseg, ctl,
                                                        kClsBtnWarp, range_mask);
        ISORT_TRY_CUDA(cudaGetLastError());
    }
    {
        LaunchScope ls("seg_oet_warp", s);
        k_seg_warp<true><<<4 * sm_count(), 256, 0, s>>>(keys, vals, off, lists + (size_t)kClsOet * nseg, ctl, kClsOet, range_mask);
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
                              SegCtl* ctl, uint32_t* lists, int big_ok, cudaStream_t s,
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
        st = enqueue_segmented(keys, vals, off, nseg, key_bits, ctl, lists, big_ok, gc.cap, seg_lo, seg_bits);
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
    if (cap == cudaStreamCaptureStatusActive) {
        // the caller is building its own graph: enqueue directly
        st = enqueue_segmented(keys, vals, off, ns, key_bits, ctl, lists, big_ok, s, seg_lo, seg_bits);
    } else {
        st = launch_via_graph(keys, vals, off, ns, key_bits, ctl, lists, big_ok, s, seg_lo, seg_bits);
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

// The finishing step of the learned-bucket sort: every bucket is a segment
// whose keys lie in [seg_lo[s], seg_lo[s] + 2^seg_bits[s]).
isort_status segmented_finish_u32(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint32_t nseg,
                                  const uint32_t* seg_lo, const uint8_t* seg_bits, cudaStream_t s) {
    return segmented_entry(keys, vals, off, nseg, 32, (void*)s, seg_lo, seg_bits);
}

}  // namespace isort

using namespace isort;

extern "C" {

isort_status isort_segmented(uint32_t* keys, uint32_t* vals, const uint64_t* seg_offsets, size_t nseg, int key_bits,
                             void* stream) {
    return segmented_entry(keys, vals, seg_offsets, nseg, key_bits, stream);
}

}  // extern "C"
