// Host-side runtime shared by the entry points: the per-device scratch pool,
// the status mode, launch accounting and optional per-kernel event timing.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "isort.h"

namespace isort {

// Scratch memory, stream-ordered, from a pool owned by the library.
isort_status scratch_alloc(void** p, size_t bytes, cudaStream_t s);
void scratch_free(void* p, cudaStream_t s);

int sm_count();                 // SMs of the current device
size_t max_smem_optin();        // opt-in dynamic shared memory per block
bool sync_mode();
uint64_t spin_limit_ns();
int64_t take_stall_tile();      // consumes the injected stall (-1 if none)
int64_t peek_stall_tile();      // the injected stall without consuming it

// Finishes a call whose kernels recorded device errors into d_status:
// in synchronous mode waits for `s` and maps the bits to a status; in
// asynchronous mode folds them into the device's sticky status word.
isort_status finish_status(const uint32_t* d_status, cudaStream_t s);
// ISORT_TRACE=1 in the environment: launches are named on stderr and waited for.
bool trace_on();

// Folds a call's device status word into the device's sticky status word
// (what the asynchronous status mode does), whatever the mode.
isort_status fold_status(const uint32_t* d_status, cudaStream_t s);

// The status of a device status word already read on the host.
isort_status map_bits(uint32_t v);

isort_status from_cuda(cudaError_t e);

// True when p points to host memory (pinned or pageable).
bool is_host_pointer(const void* p);

// Launch accounting / profiling: construct before a launch, destroy after.
// count = false times a launch (e.g. of a graph) without counting it as a
// kernel. While a CaptureScope is alive on this thread, launches are counted
// but not timed (events cannot bracket captured work).
class LaunchScope {
   public:
    LaunchScope(const char* name, cudaStream_t s, bool count = true);
    ~LaunchScope();

   private:
    const char* name_;
    cudaStream_t s_;
    cudaEvent_t e0_ = nullptr;
};

class CaptureScope {
   public:
    CaptureScope();
    ~CaptureScope();
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace isort

#define ISORT_TRY_CUDA(expr)                                 \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return ::isort::from_cuda(e_); \
    } while (0)

#define ISORT_TRY(expr)                       \
    do {                                      \
        isort_status s_ = (expr);             \
        if (s_ != ISORT_OK) return s_;        \
    } while (0)
