// Typed keys: signed integers and IEEE 754 floats sorted by the unsigned
// count-sort rounds through an order-preserving bijection on the key's bits
// (applied in place before the rounds and undone after them):
//   signed (two's complement):  u = x ^ sign bit;
//   float (binary32/binary64):  u = x ^ (all ones if the sign bit is set,
//                               else the sign bit),
// so that unsigned order of u is the integer order, or IEEE 754 totalOrder
// (-NaN < -Inf < ... < -0 < +0 < ... < +Inf < +NaN). A stable sort of u is
// the stable sort of the keys in their own order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "isort.h"
#include "runtime.h"

namespace isort {

isort_status radix_sort_u32_device(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, size_t n,
                                   int key_bits, int rb, cudaStream_t s);
isort_status radix_sort_u64_device(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout, size_t n,
                                   int key_bits, int rb, cudaStream_t s);

namespace {

enum KeyType { kU32 = 0, kI32 = 1, kF32 = 2, kU64 = 3, kI64 = 4, kF64 = 5 };

template <typename K, bool FLOAT, bool FORWARD>
__device__ __forceinline__ K order_bits(K x) {
    constexpr K sign = (K)1 << (sizeof(K) * 8 - 1);
    if constexpr (!FLOAT) return x ^ sign;
    // forward: decide on the key's sign; inverse: on the transformed top bit
    // (set exactly for keys whose sign was clear)
    const bool neg = FORWARD ? (x & sign) != 0 : (x & sign) == 0;
    return x ^ (neg ? ~(K)0 : sign);
}

// In place over n keys; 16-byte accesses over the aligned body.
template <typename K, bool FLOAT, bool FORWARD>
__global__ void k_order_bits(K* __restrict__ keys, size_t n) {
    constexpr int kPerVec = 16 / sizeof(K);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t head = std::min(n, (size_t)((16 - ((uintptr_t)keys % 16)) % 16) / sizeof(K));
    const size_t body = (n - head) / kPerVec;
    for (size_t i = t0; i < head; i += stride) keys[i] = order_bits<K, FLOAT, FORWARD>(keys[i]);
    uint4* v = reinterpret_cast<uint4*>(keys + head);
    for (size_t i = t0; i < body; i += stride) {
        union {
            uint4 q;
            K k[kPerVec];
        } u;
        u.q = v[i];
#pragma unroll
        for (int e = 0; e < kPerVec; ++e) u.k[e] = order_bits<K, FLOAT, FORWARD>(u.k[e]);
        v[i] = u.q;
    }
    for (size_t i = head + body * kPerVec + t0; i < n; i += stride) keys[i] = order_bits<K, FLOAT, FORWARD>(keys[i]);
}

template <typename K, bool FLOAT, bool FORWARD>
isort_status launch_order_bits(K* keys, size_t n, cudaStream_t s) {
    LaunchScope ls(FORWARD ? "order_bits" : "order_bits_inverse", s);
    const unsigned grid = (unsigned)std::max<size_t>(1, std::min<size_t>((n + 1023) / 1024, (size_t)sm_count() * 8));
    k_order_bits<K, FLOAT, FORWARD><<<grid, 256, 0, s>>>(keys, n);
    return from_cuda(cudaGetLastError());
}

template <typename K>
isort_status typed_sort(K* keys, uint32_t* vals, size_t n, bool is_float, int rb, cudaStream_t s) {
    constexpr int kw = (int)sizeof(K) * 8;
    auto to_order = [&](bool forward) {
        if (is_float) return forward ? launch_order_bits<K, true, true>(keys, n, s)
                                     : launch_order_bits<K, true, false>(keys, n, s);
        return forward ? launch_order_bits<K, false, true>(keys, n, s) : launch_order_bits<K, false, false>(keys, n, s);
    };
    ISORT_TRY(to_order(true));
    isort_status st;
    if constexpr (sizeof(K) == 4) st = radix_sort_u32_device(keys, vals, keys, vals, n, kw, rb, s);
    else st = radix_sort_u64_device(keys, vals, keys, vals, n, kw, rb, s);
    // undone whatever the sort returned, so that the keys keep their type
    const isort_status back = to_order(false);
    if (st != ISORT_OK) return st;
    if (back != ISORT_OK) return back;
    if (sync_mode()) ISORT_TRY_CUDA(cudaStreamSynchronize(s));
    return ISORT_OK;
}

}  // namespace
}  // namespace isort

using namespace isort;

extern "C" isort_status isort_radix_typed(void* keys, int key_type, uint32_t* vals, size_t n, int radix_bits,
                                          void* stream) {
    if (key_type < kU32 || key_type > kF64 || radix_bits < 1 || radix_bits > 16) return ISORT_ERR_INVALID_ARG;
    if (n >= (size_t(1) << 30)) return ISORT_ERR_UNSUPPORTED;
    if (n > 1 && !keys) return ISORT_ERR_INVALID_ARG;
    if (n <= 1) return ISORT_OK;
    if (is_host_pointer(keys) || (vals && is_host_pointer(vals))) return ISORT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    switch (key_type) {
        case kU32: return radix_sort_u32_device((uint32_t*)keys, vals, (uint32_t*)keys, vals, n, 32, radix_bits, s);
        case kU64: return radix_sort_u64_device((uint64_t*)keys, vals, (uint64_t*)keys, vals, n, 64, radix_bits, s);
        case kI32: return typed_sort<uint32_t>((uint32_t*)keys, vals, n, false, radix_bits, s);
        case kF32: return typed_sort<uint32_t>((uint32_t*)keys, vals, n, true, radix_bits, s);
        case kI64: return typed_sort<uint64_t>((uint64_t*)keys, vals, n, false, radix_bits, s);
        default: return typed_sort<uint64_t>((uint64_t*)keys, vals, n, true, radix_bits, s);
    }
}
