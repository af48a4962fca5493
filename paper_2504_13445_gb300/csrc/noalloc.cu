// Top-N selection from a caller's score array without any device allocation.
//
// Some callers cannot call cudaMalloc: for example a host process that reserves all device
// memory up front and forbids later allocations, or code running inside another library's
// memory manager with only the buffers it was handed.  rkm_topn_scores_noalloc serves them:
// its only scratch is the file-scope device array below, created when the library is
// loaded, so the call allocates nothing.  Inputs and outputs stay the caller's.
//
// The scratch array is shared by every call on a device and keeps the last call's contents;
// each call clears the words that must start at zero.  Calls that overlap on the GPU (on
// different streams, or from different host threads) race on it and must be serialised by
// the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rkm.h"
#include "common.cuh"
#include "kernels.h"

namespace rkm {

namespace {

constexpr int NOALLOC_MAX_N = 4096;     // the largest N the scratch holds
constexpr int NOALLOC_WORDS = 2 + NOALLOC_MAX_N;
constexpr int NOALLOC_THREADS = 1024;
constexpr int NOALLOC_MAX_DEVICES = 64;

// Word 0: error flag, word 1: number of selected keys, words 2..: the selected keys.
// 32 KB per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned long long g_topn_scratch[NOALLOC_WORDS];

// The score's sign bit is flipped so that signed scores order correctly as unsigned keys
// (a negative score sorts below every non-negative one); the top-N writer flips it back.
__device__ __forceinline__ unsigned long long score_key(const int* scores, int64_t i) {
    return ((unsigned long long)((unsigned)scores[i] ^ 0x80000000u) << 32) |
           (unsigned long long)(0xFFFFFFFFu - (unsigned)i);
}

// Same selection as k_topn (most-significant-digit radix select over the unique keys
// (score << 32) | (0xFFFFFFFF - id), then a rank sort), with the selected keys and the
// status kept in the scratch array instead of shared memory and a status word.
__global__ void __launch_bounds__(NOALLOC_THREADS) k_topn_noalloc(const int* __restrict__ scores, int64_t m,
                                                                   int N, int* __restrict__ ids,
                                                                   int* __restrict__ top_scores,
                                                                   unsigned long long* scratch) {
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned s_need;
    const int t = threadIdx.x;
    unsigned long long* err = scratch;
    unsigned long long* nsel = scratch + 1;
    unsigned long long* sel = scratch + 2;
    if (t == 0) {
        s_prefix = 0ull;
        s_need = (unsigned)N;
    }
    unsigned long long mask = 0ull;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = t; b < 256; b += NOALLOC_THREADS) hist[b] = 0u;
        __syncthreads();
        const unsigned long long prefix = s_prefix;
        for (int64_t p = t; p < m; p += NOALLOC_THREADS) {
            const unsigned long long key = score_key(scores, p);
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (t == 0) {
            unsigned need = s_need, cum = 0u;
            int dg = 255;
            for (; dg > 0; --dg) {
                if (cum + hist[dg] >= need) break;
                cum += hist[dg];
            }
            s_need = need - cum;
            s_prefix = prefix | ((unsigned long long)dg << shift);
        }
        mask |= (0xFFull << shift);
        __syncthreads();
    }
    const unsigned long long kth = s_prefix;
    for (int64_t p = t; p < m; p += NOALLOC_THREADS) {
        const unsigned long long key = score_key(scores, p);
        if (key >= kth) {
            const unsigned long long slot = atomicAdd(nsel, 1ull);
            if (slot < (unsigned long long)NOALLOC_MAX_N) sel[slot] = key;
        }
    }
    __threadfence_block();
    __syncthreads();
    if (*reinterpret_cast<volatile unsigned long long*>(nsel) != (unsigned long long)N) {
        if (t == 0) *err = 1ull;
        return;
    }
    for (int j = t; j < N; j += NOALLOC_THREADS) {
        const unsigned long long key = sel[j];
        int rank = 0;
        for (int r = 0; r < N; ++r) rank += sel[r] > key;
        ids[rank] = (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
        top_scores[rank] = (int)((unsigned)(key >> 32) ^ 0x80000000u);
    }
}

std::mutex g_setup_mutex;
unsigned long long* g_scratch_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once per device and
// kept for the life of the process.  The lookup is a runtime call, so the first call on a
// device should precede any stream capture on that device.  A device reset
// (cudaDeviceReset) reloads the library's module and moves the array: the library must not
// be used on a device across a reset.
cudaError_t scratch_address(int dev, unsigned long long** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_topn_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace rkm

extern "C" rkm_status rkm_topn_scores_noalloc(const int32_t* scores, int64_t m, int N, int32_t* ids,
                                              int32_t* top_scores, void* stream) {
    using namespace rkm;
    auto set_error = [](rkm_status s, const char* msg) { return (rkm_status)rkm::set_error((int)s, msg); };
    if (!scores || !ids || !top_scores) return set_error(RKM_EINVAL, "null pointer argument");
    if (m < 1 || m > (int64_t)INT32_MAX) return set_error(RKM_EINVAL, "m must be in [1, 2^31-1]");
    if (N < 1 || N > m) return set_error(RKM_EINVAL, "N must satisfy 1 <= N <= m");
    if (N > NOALLOC_MAX_N)
        return set_error(RKM_EINVAL, "N exceeds 4096, the capacity of the fixed scratch array");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return set_error(RKM_ECUDA, "no usable current CUDA device");
    unsigned long long* scratch = nullptr;
    cudaError_t e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return set_error(RKM_ECUDA, cudaGetErrorString(e));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Clear the error flag and the selection counter left by the previous call.
    e = cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return set_error(RKM_ECUDA, cudaGetErrorString(e));
    note_launch();
    k_topn_noalloc<<<1, NOALLOC_THREADS, 0, s>>>(scores, m, N, ids, top_scores, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(RKM_ECUDA, cudaGetErrorString(e));
    unsigned long long err = 0ull;  // host stack word: the copy allocates nothing
    e = cudaMemcpyAsync(&err, scratch, sizeof err, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(RKM_ECUDA, cudaGetErrorString(e));
    if (err) return set_error(RKM_EINTERNAL, "top-N selection found an inconsistent key count");
    return RKM_OK;
}
