// BTN and OET: the paper's small-n block networks (Gerbessiotis,
// arXiv:1708.09495, Section 2; Section 3 "Bitonic Sort" eq. Tb and "Odd-even
// transposition sort" eq. To).
//
// p "processors" are p threads of one CTA; the device code is in net.cuh.
#include <algorithm>

#include "common.cuh"
#include "net.cuh"
#include "runtime.h"

namespace isort {
namespace {

// BTN: one CTA, p (a power of two) threads hold the blocks.
template <int B>
__global__ void __launch_bounds__(B <= 16 ? 1024 : 512)
    k_btn(uint32_t* keys, uint32_t* vals, uint32_t n, int p, unsigned long long* stage_ctr) {
    extern __shared__ __align__(16) uint64_t s_x[];  // [B][blockDim] when a stage crosses warps
    net::btn_block<B>(keys, vals, n, p, s_x, stage_ctr);
}

// OET: one CTA, p threads hold the blocks.
template <int B>
__global__ void __launch_bounds__(B <= 16 ? 1024 : 512)
    k_oet(uint32_t* keys, uint32_t* vals, uint32_t n, int p, unsigned long long* stage_ctr) {
    extern __shared__ __align__(16) uint64_t s_x[];
    net::oet_block<B>(keys, vals, n, p, s_x, stage_ctr);
}

int next_pow2(uint32_t v) {
    int p = 1;
    while ((uint32_t)p < v) p <<= 1;
    return p;
}

enum class Net { Btn, Oet };

template <int B>
isort_status launch_net(Net net, uint32_t* keys, uint32_t* vals, uint32_t n, int p, unsigned long long* ctr,
                        cudaStream_t s) {
    const int threads = std::max(32, (p + 31) / 32 * 32);
    // shared memory is needed by OET always and by BTN once partners cross warps
    const size_t smem = (net == Net::Oet || p > 32) ? (size_t)B * threads * 8 : 0;
    if (smem > max_smem_optin()) return ISORT_ERR_UNSUPPORTED;
    cudaFuncAttributes fa;
    ISORT_TRY_CUDA(cudaFuncGetAttributes(&fa, net == Net::Btn ? (const void*)k_btn<B> : (const void*)k_oet<B>));
    if (threads > fa.maxThreadsPerBlock) return ISORT_ERR_UNSUPPORTED;
    if (net == Net::Btn) {
        ISORT_TRY_CUDA(cudaFuncSetAttribute(k_btn<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        LaunchScope ls("btn", s);
        k_btn<B><<<1, threads, smem, s>>>(keys, vals, n, p, ctr);
    } else {
        ISORT_TRY_CUDA(cudaFuncSetAttribute(k_oet<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        LaunchScope ls("oet", s);
        k_oet<B><<<1, threads, smem, s>>>(keys, vals, n, p, ctr);
    }
    return from_cuda(cudaGetLastError());
}

constexpr uint32_t kNetMaxN = 16384;

// Sorts device buffers with the chosen network on p blocks.
isort_status net_device(Net net, uint32_t* keys, uint32_t* vals, uint32_t n, int p, uint64_t* stages, cudaStream_t s) {
    const uint32_t per = (n + (uint32_t)p - 1) / (uint32_t)p;
    const int B = next_pow2(std::max<uint32_t>(per, 1));
    if (B > 32 || (size_t)B * p > kNetMaxN * 2) return ISORT_ERR_UNSUPPORTED;
    unsigned long long* ctr = nullptr;
    if (stages) {
        isort_status st = scratch_alloc((void**)&ctr, 8, s);
        if (st != ISORT_OK) return st;
        cudaError_t ce = cudaMemsetAsync(ctr, 0, 8, s);
        if (ce != cudaSuccess) {
            scratch_free(ctr, s);
            return from_cuda(ce);
        }
    }
    isort_status st;
    switch (B) {
        case 1: st = launch_net<1>(net, keys, vals, n, p, ctr, s); break;
        case 2: st = launch_net<2>(net, keys, vals, n, p, ctr, s); break;
        case 4: st = launch_net<4>(net, keys, vals, n, p, ctr, s); break;
        case 8: st = launch_net<8>(net, keys, vals, n, p, ctr, s); break;
        case 16: st = launch_net<16>(net, keys, vals, n, p, ctr, s); break;
        default: st = launch_net<32>(net, keys, vals, n, p, ctr, s); break;
    }
    if (stages) {
        if (st == ISORT_OK) {
            unsigned long long h = 0;
            cudaError_t ce = cudaMemcpyAsync(&h, ctr, 8, cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) st = from_cuda(ce);
            *stages = h;
        }
        scratch_free(ctr, s);
    } else if (st == ISORT_OK && sync_mode()) {
        st = from_cuda(cudaStreamSynchronize(s));
    }
    return st;
}

isort_status net_entry(Net net, uint32_t* keys, uint32_t* vals, size_t n, int p, uint64_t* stages, void* stream) {
    if (net == Net::Btn && (p < 1 || p > 1024 || (p & (p - 1)) != 0)) return ISORT_ERR_INVALID_ARG;
    if (net == Net::Oet && (p < 1 || p > 1024)) return ISORT_ERR_INVALID_ARG;
    if (n > (size_t)32 * p || n > kNetMaxN) return ISORT_ERR_UNSUPPORTED;
    if (n > 1 && !keys) return ISORT_ERR_INVALID_ARG;
    if (stages) *stages = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return ISORT_OK;
    const bool host = is_host_pointer(keys) || (vals && is_host_pointer(vals));
    if (!host) return net_device(net, keys, vals, (uint32_t)n, p, stages, s);
    unsigned char* buf = nullptr;
    const size_t kb = align_up(n * 4, 256);
    isort_status st = scratch_alloc((void**)&buf, kb + (vals ? kb : 0), s);
    if (st != ISORT_OK) return st;
    uint32_t* dk = reinterpret_cast<uint32_t*>(buf);
    uint32_t* dv = vals ? reinterpret_cast<uint32_t*>(buf + kb) : nullptr;
    cudaError_t ce = cudaMemcpyAsync(dk, keys, n * 4, cudaMemcpyDefault, s);
    if (ce == cudaSuccess && vals) ce = cudaMemcpyAsync(dv, vals, n * 4, cudaMemcpyDefault, s);
    st = ce == cudaSuccess ? net_device(net, dk, dv, (uint32_t)n, p, stages, s) : from_cuda(ce);
    if (st == ISORT_OK) {
        ce = cudaMemcpyAsync(keys, dk, n * 4, cudaMemcpyDefault, s);
        if (ce == cudaSuccess && vals) ce = cudaMemcpyAsync(vals, dv, n * 4, cudaMemcpyDefault, s);
        if (ce != cudaSuccess) st = from_cuda(ce);
    }
    scratch_free(buf, s);
    cudaError_t se = cudaStreamSynchronize(s);
    if (st == ISORT_OK && se != cudaSuccess) st = from_cuda(se);
    return st;
}

// Default p: 8 keys per block up to 4096 keys, then 16.
int default_p(size_t n) {
    const uint32_t per = n <= 4096 ? 8u : 16u;
    int p = next_pow2((uint32_t)std::max<size_t>(1, (n + per - 1) / per));
    return std::min(p, 1024);
}

}  // namespace
}  // namespace isort

using namespace isort;

extern "C" {

isort_status isort_btn(uint32_t* keys, uint32_t* vals, size_t n, void* stream) {
    return net_entry(Net::Btn, keys, vals, n, default_p(n), nullptr, stream);
}

isort_status isort_oet(uint32_t* keys, uint32_t* vals, size_t n, void* stream) {
    return net_entry(Net::Oet, keys, vals, n, default_p(n), nullptr, stream);
}

isort_status isort_btn_p(uint32_t* keys, uint32_t* vals, size_t n, int p, uint64_t* stages, void* stream) {
    return net_entry(Net::Btn, keys, vals, n, p, stages, stream);
}

isort_status isort_oet_p(uint32_t* keys, uint32_t* vals, size_t n, int p, uint64_t* stages, void* stream) {
    return net_entry(Net::Oet, keys, vals, n, p, stages, stream);
}

}  // extern "C"
