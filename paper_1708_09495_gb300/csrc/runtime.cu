// Host-side runtime: scratch pool, status handling, launch accounting and
// per-kernel event timing.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "runtime.h"

namespace isort {

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};
size_t g_smem_optin[kMaxDevices] = {};

std::atomic<int> g_sync{1};
std::atomic<uint64_t> g_spin_ns{2000000000ull};
std::atomic<int64_t> g_stall{-1};
std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_profile{0};

struct ProfRec {
    const char* name;
    cudaEvent_t e0, e1;
};
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof;

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

cudaMemPool_t pool_for(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~0ull;  // keep freed blocks for reuse by later calls
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = p;
    }
    return g_pools[dev];
}

}  // namespace

// Device errors of asynchronous calls accumulate here (one word per device).
__device__ uint32_t g_sticky_status;

__global__ void k_fold_status(const uint32_t* st) {
    if (threadIdx.x == 0) {
        uint32_t v = *st;
        if (v) atomicOr(&g_sticky_status, v);
    }
}

thread_local char t_last_error[160] = "";

static void note_error(const char* what) {
    std::snprintf(t_last_error, sizeof(t_last_error), "%s", what);
}

isort_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return ISORT_OK;
    note_error(cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return ISORT_ERR_NO_MEMORY;
    }
    return ISORT_ERR_CUDA;
}

isort_status scratch_alloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) return ISORT_OK;
    cudaMemPool_t pool = pool_for(current_device());
    if (!pool) return ISORT_ERR_CUDA;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? ISORT_ERR_NO_MEMORY : ISORT_ERR_CUDA;
    }
    return ISORT_OK;
}

void scratch_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int sm_count() {
    int d = current_device();
    if (d >= 0 && d < kMaxDevices && g_sms[d]) return g_sms[d];
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    if (d >= 0 && d < kMaxDevices) g_sms[d] = v;
    return v > 0 ? v : 1;
}

size_t max_smem_optin() {
    int d = current_device();
    if (d >= 0 && d < kMaxDevices && g_smem_optin[d]) return g_smem_optin[d];
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, d);
    if (d >= 0 && d < kMaxDevices) g_smem_optin[d] = (size_t)v;
    return (size_t)v;
}

bool sync_mode() { return g_sync.load() != 0; }
uint64_t spin_limit_ns() { return g_spin_ns.load(); }
int64_t take_stall_tile() { return g_stall.exchange(-1); }
int64_t peek_stall_tile() { return g_stall.load(); }

isort_status map_bits(uint32_t v) {
    if (v) {
        char buf[96];
        std::snprintf(buf, sizeof(buf), "device status bits 0x%x (1 key range, 2 timeout, 4 output index, 8 offsets)", v);
        note_error(buf);
    }
    if (v & kStatTimeout) return ISORT_ERR_TIMEOUT;
    if (v & kStatBadOffsets) return ISORT_ERR_INVALID_ARG;
    if (v & kStatUnsupported) return ISORT_ERR_UNSUPPORTED;
    if (v & kStatKeyRange) return ISORT_ERR_KEY_RANGE;
    if (v & kStatBounds) return ISORT_ERR_CUDA;
    return ISORT_OK;
}

isort_status fold_status(const uint32_t* d_status, cudaStream_t s) {
    LaunchScope ls("fold_status", s);
    k_fold_status<<<1, 32, 0, s>>>(d_status);
    return from_cuda(cudaGetLastError());
}

isort_status finish_status(const uint32_t* d_status, cudaStream_t s) {
    if (!sync_mode()) return fold_status(d_status, s);
    static thread_local uint32_t* host_slot = nullptr;
    if (!host_slot) {
        if (cudaHostAlloc((void**)&host_slot, 64, cudaHostAllocDefault) != cudaSuccess) {
            host_slot = nullptr;
            return ISORT_ERR_CUDA;
        }
    }
    ISORT_TRY_CUDA(cudaMemcpyAsync(host_slot, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    ISORT_TRY_CUDA(cudaStreamSynchronize(s));
    return map_bits(*host_slot);
}

bool is_host_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return true;  // unknown to CUDA: ordinary pageable host memory
    }
    return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

thread_local int t_capturing = 0;

CaptureScope::CaptureScope() { ++t_capturing; }
CaptureScope::~CaptureScope() { --t_capturing; }

// ISORT_TRACE=1: every launch scope names itself on stderr as it opens and,
// outside stream capture, waits for its work when it closes (a debugging aid
// that shows which step a stalled call is in).
bool trace_on() {
    static const bool on = [] {
        const char* e = std::getenv("ISORT_TRACE");
        return e && e[0] == '1';
    }();
    return on;
}

LaunchScope::LaunchScope(const char* name, cudaStream_t s, bool count) : name_(name), s_(s) {
    if (count) g_launches.fetch_add(1);
    if (trace_on()) {
        std::fprintf(stderr, "[isort] %s\n", name);
        std::fflush(stderr);
    }
    if (g_profile.load() && t_capturing == 0) {
        if (cudaEventCreate(&e0_) == cudaSuccess) cudaEventRecord(e0_, s_);
        else e0_ = nullptr;
    }
}

LaunchScope::~LaunchScope() {
    if (trace_on() && t_capturing == 0) {
        const cudaError_t e = cudaStreamSynchronize(s_);
        std::fprintf(stderr, "[isort] %s done (%s)\n", name_, cudaGetErrorString(e));
        std::fflush(stderr);
    }
    if (!e0_) return;
    cudaEvent_t e1 = nullptr;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0_);
        return;
    }
    cudaEventRecord(e1, s_);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back({name_, e0_, e1});
}

}  // namespace isort

using namespace isort;

extern "C" {

const char* isort_status_string(isort_status s) {
    switch (s) {
        case ISORT_OK: return "ISORT_OK";
        case ISORT_ERR_INVALID_ARG: return "ISORT_ERR_INVALID_ARG";
        case ISORT_ERR_KEY_RANGE: return "ISORT_ERR_KEY_RANGE";
        case ISORT_ERR_NO_MEMORY: return "ISORT_ERR_NO_MEMORY";
        case ISORT_ERR_CUDA: return "ISORT_ERR_CUDA";
        case ISORT_ERR_TIMEOUT: return "ISORT_ERR_TIMEOUT";
        case ISORT_ERR_UNSUPPORTED: return "ISORT_ERR_UNSUPPORTED";
    }
    return "ISORT_UNKNOWN_STATUS";
}

isort_status isort_set_sync(int on) {
    g_sync.store(on ? 1 : 0);
    return ISORT_OK;
}

isort_status isort_set_spin_limit(uint64_t microseconds) {
    if (microseconds == 0 || microseconds > 3600ull * 1000000ull) return ISORT_ERR_INVALID_ARG;
    g_spin_ns.store(microseconds * 1000ull);
    return ISORT_OK;
}

isort_status isort_device_status(int clear, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    ISORT_TRY_CUDA(cudaStreamSynchronize(s));
    uint32_t v = 0;
    ISORT_TRY_CUDA(cudaMemcpyFromSymbol(&v, g_sticky_status, sizeof(v)));
    if (clear) {
        uint32_t z = 0;
        ISORT_TRY_CUDA(cudaMemcpyToSymbol(g_sticky_status, &z, sizeof(z)));
    }
    return map_bits(v);
}

isort_status isort_debug_stall_tile(int64_t tile) {
    g_stall.store(tile < 0 ? -1 : tile);
    return ISORT_OK;
}

uint64_t isort_launch_count(void) { return g_launches.load(); }

const char* isort_last_error_string(void) { return t_last_error; }

isort_status isort_profile_enable(int on) {
    g_profile.store(on ? 1 : 0);
    return ISORT_OK;
}

int isort_profile_read(isort_kernel_time* out, int max) {
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        recs.swap(g_prof);
    }
    std::vector<isort_kernel_time> agg;
    for (auto& r : recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.e1) == cudaSuccess) cudaEventElapsedTime(&ms, r.e0, r.e1);
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
        isort_kernel_time* slot = nullptr;
        for (auto& a : agg)
            if (std::strncmp(a.name, r.name, sizeof(a.name)) == 0) slot = &a;
        if (!slot) {
            isort_kernel_time t;
            std::memset(&t, 0, sizeof(t));
            std::strncpy(t.name, r.name, sizeof(t.name) - 1);
            agg.push_back(t);
            slot = &agg.back();
        }
        slot->launches += 1;
        slot->total_ms += ms;
    }
    int k = 0;
    for (auto& a : agg) {
        if (k >= max || !out) break;
        out[k++] = a;
    }
    return k;
}

}  // extern "C"
