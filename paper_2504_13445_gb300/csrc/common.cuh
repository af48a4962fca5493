// Shared definitions for the reverse k-MIPS kernels (device side).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

namespace rkm {

// Tile shapes.  BU users (TMEM lanes / SIMT rows) by BI items per product tile.
constexpr int BU = 128;
constexpr int BI_SIMT = 128;
constexpr int BI_TC = 256;
constexpr int KMAX = 64;          // largest k the on-chip heaps hold
constexpr int NMAX_TOPN = 4096;   // largest N the single-CTA top-N select holds
constexpr int NBUCKET = 65536;    // buckets of the 16-bit float keys
constexpr int SCAN_BLOCK = 1024;  // buckets per block of the bucket-count prefix scan
constexpr int SCAN_BLOCKS = NBUCKET / SCAN_BLOCK;
constexpr int HIST_WORDS = NBUCKET + SCAN_BLOCKS;  // bucket counts, then per-block totals

// Device-side status and counters of one call.  Zeroed before each call.
struct DevStatus {
    unsigned int cand_overflow;   // a user's candidate list stayed full after compaction
    unsigned int band_overflow;   // the band queue was full
    unsigned int internal_error;  // a consistency check failed (e.g. < k candidates)
    unsigned int timeout;         // a bounded wait gave up
    unsigned int off_grid;        // set when a user or item row is not on the 2^-12 grid
    unsigned int debug_line;      // debug builds: source line of the first failed index check
    unsigned int band_count;      // pairs pushed to the band queue (may exceed capacity)
    unsigned int band_done;       // pairs of the queue already rescored
    unsigned int ticket;          // work ticket of the persistent counting kernel
    unsigned int units_total;     // work units of the current counting stage
    int t_end;                    // one past the last item tile of the filtered stage
    int m_counted;                // items whose scores are complete (rkm_topn)
    unsigned long long cand_total;      // candidates kept for exact rescoring
    unsigned long long pairs_evaluated; // products computed by the counting pass
    unsigned long long launch_units;    // work units of the current tensor-core counting launch
    unsigned long long thr_pairs;       // user-item products computed by the threshold pass
    unsigned long long pad[2];
};

// Debug builds (-DRKM_DEBUG): index checks on the gathers and scatters whose index comes from
// device data.  A failed check records its source line in the status word (the first one
// wins), raises internal_error and skips the access; the call returns RKM_EINTERNAL.  Release
// builds compile the checks away.
#ifdef RKM_DEBUG
__device__ __forceinline__ bool rkm_dcheck(bool ok, DevStatus* st, int line) {
    if (!ok) {
        atomicCAS(&st->debug_line, 0u, (unsigned)line);
        st->internal_error = 1u;
    }
    return ok;
}
#define RKM_DCHECK(cond, st) ::rkm::rkm_dcheck((cond), (st), __LINE__)
#else
#define RKM_DCHECK(cond, st) true
#endif

// Per-user data of the counting pass, one 32-byte record per user in ratio order:
// tau_u rounded up and down to FP32, ||u||, ||u^||, ||u^ - u|| (rounded up), original id.
struct __align__(16) UserMeta {
    float tau_hi, tau_lo, un, unh, ud;
    int uorig;
    int uexp;  // row exponent e (max|u| <= 2^e); scales the FP8 operand
    float pad1;
};

// Candidate of the threshold pass: an upper bound of u.p and the item's sorted position.
struct Cand {
    float ub;
    int pos;
};

// Monotone map float -> uint32 (total order of non-NaN floats, -0 < +0).
__host__ __device__ __forceinline__ uint32_t float_key(float x) {
    uint32_t b;
#ifdef __CUDA_ARCH__
    b = __float_as_uint(x);
#else
    memcpy(&b, &x, 4);
#endif
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Inverse of float_key; the key 0 (nothing recorded) reads as -inf.
__device__ __forceinline__ float key_float(uint32_t k) {
    if (k == 0u) return -INFINITY;
    const uint32_t b = (k & 0x80000000u) ? (k ^ 0x80000000u) : ~k;
    return __uint_as_float(b);
}

// 16-bit bucket of a float, monotone non-decreasing in x.
__host__ __device__ __forceinline__ uint32_t bucket16(float x) { return float_key(x) >> 16; }

// Monotone map double -> uint64 for the exact scores; callers add +0.0 first so
// that -0.0 and +0.0 share one key.
__device__ __forceinline__ unsigned long long double_key(double s) {
    unsigned long long b = (unsigned long long)__double_as_longlong(s);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Error bound of one approximate product v of u^ . p^ (operands u^, p^ rounded from u, p):
//   |v - u.p| <= |u^.p^ - u.p| + |v - u^.p^|
//             <= ||u^ - u|| ||p^|| + ||u|| ||p^ - p|| + cacc ||u^|| ||p^|| + eabs
// by Cauchy-Schwarz on (u^ - u).p^ + u.(p^ - p), with the tile maxima of the item
// terms; every operation rounds up.
__device__ __forceinline__ float err_bound(float cacc, float eabs, float un, float unhat, float udel,
                                           float pnhat, float pdel) {
    const float rep = __fadd_ru(__fmul_ru(udel, pnhat), __fmul_ru(un, pdel));
    return __fadd_ru(__fadd_ru(rep, __fmul_ru(cacc, __fmul_ru(unhat, pnhat))), eabs);
}

// Exponent of the FP8 operand scale 2^(8 - e) of a row (or tile) with max|x| <= 2^e, clamped
// to [-60, 60] so that the scale, the descaled operand and the product factor
// 2^(e_u + e_T - 16) are exact FP32 powers of two.  Rows outside that range saturate (at
// 448) or underflow in FP8; the norms ||x^ - x|| of the actual rounding carry that error
// into the guard band, so results stay exact.
__host__ __device__ __forceinline__ int fp8_exp(int e) { return e < -60 ? -60 : (e > 60 ? 60 : e); }

// Three-input maximum (sm_100 and later).
__device__ __forceinline__ float fmax3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

}  // namespace rkm
