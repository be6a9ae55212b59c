// ch_chain_noalloc: the chain step (Lemma 1 scan of L) for callers that
// cannot hand over a workspace: plain C callers that hold no device
// allocator of their own, and loops that must not allocate because
// cudaMalloc/cudaFree synchronise the whole device.  The only scratch the
// chain step needs is its look-back state (one ticket word plus one word per
// 1024-column tile); here it lives in a fixed device array of this file
// instead of caller memory, so the call allocates nothing.
//
// The array holds the state of p <= CH_CHAIN_NOALLOC_MAX_P (16385 words,
// 128 KiB).  The state must be zero when the kernel starts; every call
// clears the words it uses with cudaMemsetAsync on the caller's stream first.
// One array serves every call on a device, so calls that overlap in time
// (other streams, other host threads) race on it: the caller serialises them.
#include <mutex>

#include "ch_internal.cuh"

namespace {

constexpr int NOALLOC_TILE = 1024;  // columns per chain tile (the chain kernel's)
constexpr size_t NOALLOC_WORDS = (CH_CHAIN_NOALLOC_MAX_P + NOALLOC_TILE - 1) / NOALLOC_TILE + 1;

static __device__ __align__(256) unsigned long long g_chain_scratch[NOALLOC_WORDS];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {};

// Address of this device's scratch array, resolved once per device while
// that device is current.
void *scratch_ptr()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return nullptr;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_chain_scratch) != cudaSuccess)
            return nullptr;
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" int ch_chain_noalloc(const int32_t *L, int32_t p, int32_t *lower, int32_t *upper,
                                int32_t *counts, uint32_t *mask, ch_stream_t stream)
{
    if (!L || !lower || !upper || !counts || p < 1 || ((uintptr_t)L & 7) ||
        ((uintptr_t)lower & 7) || ((uintptr_t)upper & 7))
        return CH_ERR_ARG;
    if (p > CH_CHAIN_NOALLOC_MAX_P)
        return CH_ERR_CAPACITY;
    if (ch::chain_state_bytes(p) > sizeof(g_chain_scratch))
        return CH_ERR_CAPACITY;
    void *state = scratch_ptr();
    unsigned *st = ch::device_status_ptr(reinterpret_cast<cudaStream_t>(stream));
    if (!state || !st)
        return CH_ERR_CUDA;
    const cudaError_t e = ch::chain_launch(L, p, lower, upper, counts, mask, state, false, nullptr,
                                           nullptr, st, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? CH_OK : CH_ERR_CUDA;
}
