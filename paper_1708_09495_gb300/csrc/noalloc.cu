// isort_radix_noalloc: the in-place LSD radix sort for callers that must not
// allocate memory.
//
// Some callers cannot let a library allocate device memory: processes whose
// device memory is entirely reserved up front by another allocator, and
// latency-critical loops that cannot afford the implicit synchronisation an
// allocation may cause. For them this entry
// point takes all of its scratch from one fixed array in device memory that
// the library declares at file scope, so no call allocates anything.
//
// The array is kNoAllocScratchBytes (5 MiB) on every GPU that loads the
// library, for the life of the process, which bounds the problem size:
// at most kNoAllocMaxKeys (262,144) uint32 keys, with or without a uint32
// payload, radix_bits 1..8. All calls on a device share the array: calls whose
// work overlaps on the GPU (different streams, or a second call enqueued before
// the first one finished in the asynchronous status mode) race and corrupt each
// other's results. The control part of the array is cleared at the start of
// every call; the rest is overwritten before it is read.
#include <mutex>

#include "common.cuh"
#include "runtime.h"

namespace isort {

size_t radix_u32_inplace_workspace_bytes(size_t n, int key_bits, int rb, bool vals);
isort_status radix_u32_inplace_in_workspace(uint32_t* keys, uint32_t* vals, size_t n, int key_bits, int rb,
                                            unsigned char* ws, size_t ws_bytes, cudaStream_t s,
                                            const uint32_t** d_status);

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(5) << 20;
constexpr size_t kNoAllocMaxKeys = size_t(1) << 18;
constexpr int kNoAllocMaxRadixBits = 8;
constexpr int kMaxDevices = 64;

// The scratch memory. In host code this name is only a stand-in for the
// device array: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Once per device, with that device current: the array's device address.
isort_status scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    ISORT_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return ISORT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return ISORT_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return ISORT_OK;
}

}  // namespace
}  // namespace isort

using namespace isort;

extern "C" {

isort_status isort_radix_noalloc(uint32_t* keys, uint32_t* vals, size_t n, int key_bits, int radix_bits,
                                 void* stream) {
    if (key_bits == 0) key_bits = 32;
    if (key_bits < 1 || key_bits > 32 || radix_bits < 1 || radix_bits > 16) return ISORT_ERR_INVALID_ARG;
    if (radix_bits > kNoAllocMaxRadixBits || n > kNoAllocMaxKeys) return ISORT_ERR_UNSUPPORTED;
    if (n <= 1) return ISORT_OK;
    if (!keys) return ISORT_ERR_INVALID_ARG;
    if (is_host_pointer(keys) || (vals && is_host_pointer(vals))) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* ws = nullptr;
    isort_status st = scratch_for_current_device(&ws);
    if (st != ISORT_OK) return st;
    if (radix_u32_inplace_workspace_bytes(n, key_bits, radix_bits, vals != nullptr) > kNoAllocScratchBytes)
        return ISORT_ERR_UNSUPPORTED;
    const uint32_t* d_status = nullptr;
    st = radix_u32_inplace_in_workspace(keys, vals, n, key_bits, radix_bits, ws, kNoAllocScratchBytes, s, &d_status);
    if (st != ISORT_OK) return st;
    if (!sync_mode()) return finish_status(d_status, s);  // folds into the device's sticky status; no allocation
    // A stream that reports an active capture is not waited for: the device
    // status is then folded into the sticky word, as in the asynchronous mode.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ISORT_TRY_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return fold_status(d_status, s);
    // synchronous mode: read the status word into this stack variable and map
    // it as isort_radix does
    uint32_t h = 0;
    ISORT_TRY_CUDA(cudaMemcpyAsync(&h, d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
    ISORT_TRY_CUDA(cudaStreamSynchronize(s));
    return map_bits(h);
}

}  // extern "C"
