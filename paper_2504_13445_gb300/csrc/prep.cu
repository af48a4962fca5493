// K1 (prep) and K4 (Eq. 2 bounds) kernels, plus the 16-bit bucket counting sort.
//
// Prep follows step (1) of Algorithm 1 (norms of every vector, items ordered by
// descending norm) and adds what the GPU path needs: the exact grid codes for
// exact rescoring and zero-padded operand copies for the product kernels.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace rkm {

namespace {

// x^ of the FP8 operand with scale 2^(8-e) (e already clamped by fp8_exp): e4m3
// round-to-nearest-even (saturating at 448) of x * 2^(8-e), as a float; descaled by the
// caller (exact in FP32).
__device__ __forceinline__ float fp8_scaled(float v, int e, __nv_fp8_storage_t* code) {
    const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(ldexpf(v, 8 - e), __NV_SATFINITE, __NV_E4M3);
    if (code) *code = c;
    const __half_raw h = __nv_cvt_fp8_to_halfraw(c, __NV_E4M3);
    return __half2float(__half(h));
}

inline int grid_for(int64_t work, int per_block, int cap = 1 << 20) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// A segment of lpr lanes per row (lpr a power of two, 32 / lpr rows per warp, so that short
// rows do not leave most of a warp's reductions idle).  The row is on the grid iff every
// x * 2^(12-e) is an integer of magnitude <= 4096; then ||x||^2 = sum(q^2) * 2^(2e-24) exactly.
__global__ void k_prep_rows(const float* __restrict__ X, int64_t rows, int64_t ld, int d,
                            int* __restrict__ ex, int16_t* __restrict__ q, int dq,
                            double* __restrict__ norm2, float* __restrict__ nrm_hi,
                            float* __restrict__ nhat_hi, float* __restrict__ del_hi, int operand,
                            unsigned* grid_flag, int lpr) {
    const int lane = threadIdx.x & 31;
    const int sub = lane & (lpr - 1);
    const int rpw = 32 / lpr;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * rpw; r0 < rows; r0 += warps * rpw) {
        const int64_t row = r0 + lane / lpr;
        const bool valid = row < rows;
        const float* x = X + (valid ? row : 0) * ld;
        float mx = 0.f;
        if (valid)
            for (int j = sub; j < d; j += lpr) mx = fmaxf(mx, fabsf(x[j]));
        for (int o = lpr >> 1; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int e = 0;
        if (mx > 0.f) {
            int E;
            float f = frexpf(mx, &E);
            e = (f == 0.5f) ? E - 1 : E;
        }
        int ok = 1;
        long long s2 = 0;
        // Upper bounds of sums of squares: every FP32 operation rounds up.
        float d2 = 0.f, h2 = 0.f, e2 = 0.f;
        if (valid) {
            for (int j = sub; j < dq; j += lpr) {
                float v = (j < d) ? x[j] : 0.f;
                float t = ldexpf(v, 12 - e);
                bool gi = (t == rintf(t)) && fabsf(t) <= 4096.f;
                ok = ok & (gi ? 1 : 0);
                int qi = gi ? (int)t : 0;
                q[row * dq + j] = (int16_t)qi;
                s2 += (long long)qi * qi;
                d2 = __fmaf_ru(v, v, d2);
                // Operand the product kernels see, and its rounding error (exact in FP32).
                float vh = v;
                if (operand == OPERAND_BF16) vh = __bfloat162float(__float2bfloat16_rn(v));
                if (operand == OPERAND_FP8_ROW) vh = ldexpf(fp8_scaled(v, fp8_exp(e), nullptr), fp8_exp(e) - 8);
                const float dv = vh - v;
                h2 = __fmaf_ru(vh, vh, h2);
                e2 = __fmaf_ru(dv, dv, e2);
            }
        }
        for (int o = lpr >> 1; o > 0; o >>= 1) {
            ok &= __shfl_xor_sync(0xffffffffu, ok, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            d2 = __fadd_ru(d2, __shfl_xor_sync(0xffffffffu, d2, o));
            h2 = __fadd_ru(h2, __shfl_xor_sync(0xffffffffu, h2, o));
            e2 = __fadd_ru(e2, __shfl_xor_sync(0xffffffffu, e2, o));
        }
        if (valid && sub == 0) {
            double n2;
            if (ok) {
                n2 = ldexp((double)s2, 2 * e - 24);  // exact
            } else {
                n2 = (double)d2;                     // an upper bound
                atomicOr(grid_flag, 1u);
            }
            ex[row] = e;
            norm2[row] = n2;
            nrm_hi[row] = ok ? __double2float_ru(__dsqrt_ru(n2)) : __fsqrt_ru(d2);
            nhat_hi[row] = __fsqrt_ru(h2);
            del_hi[row] = __fsqrt_ru(e2);
        }
    }
}

template <typename T>
__device__ __forceinline__ T cvt_from_float(float v);
template <>
__device__ __forceinline__ float cvt_from_float<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_from_float<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// Eight consecutive columns per thread (dp is a multiple of 8), written as one 16-byte
// (BF16) or two 16-byte (FP32) stores.
template <typename T>
__global__ void k_pack(const float* __restrict__ X, int64_t rows, int64_t ld, int d,
                       const int* __restrict__ perm, T* __restrict__ dst, int64_t rows_pad, int dp) {
    const int cpr = dp >> 3;  // 8-column chunks per row
    const int64_t total = rows_pad * cpr;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / cpr;
        const int c0 = (int)(idx - r * cpr) * 8;
        float v[8];
        const float* x = (r < rows) ? X + (perm ? (int64_t)perm[r] : r) * ld : nullptr;
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (x && c0 + j < d) ? x[c0 + j] : 0.f;
        T out[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) out[j] = cvt_from_float<T>(v[j]);
        uint4* o = reinterpret_cast<uint4*>(dst + r * dp + c0);
        const uint4* src = reinterpret_cast<const uint4*>(out);
#pragma unroll
        for (int w = 0; w < (int)(8 * sizeof(T) / 16); ++w) o[w] = src[w];
    }
}

// One warp per packed row: e4m3 codes of the row scaled by 2^(8 - e) (e = its tile's or its
// own exponent), zero padding, and the norms of the descaled operand at the source row.
__global__ void k_pack_fp8(const float* __restrict__ X, int64_t rows, int64_t ld, int d,
                           const int* __restrict__ perm, const int* __restrict__ row_exp,
                           const int* __restrict__ tile_exp, int tile, uint8_t* __restrict__ dst, int64_t rows_pad,
                           int dp, float* __restrict__ nhat, float* __restrict__ del) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows_pad; r += warps) {
        uint8_t* out = dst + r * dp;
        if (r >= rows) {
            for (int c = lane; c < dp; c += 32) out[c] = 0;
            continue;
        }
        const int64_t src = perm ? (int64_t)perm[r] : r;
        const int e = tile_exp ? tile_exp[r / tile] : fp8_exp(row_exp[src]);
        const float* x = X + src * ld;
        float h2 = 0.f, e2 = 0.f;
        for (int c = lane; c < dp; c += 32) {
            __nv_fp8_storage_t code = 0;
            if (c < d) {
                const float v = x[c];
                const float vh = ldexpf(fp8_scaled(v, e, &code), e - 8);
                const float dv = vh - v;
                h2 = __fmaf_ru(vh, vh, h2);
                e2 = __fmaf_ru(dv, dv, e2);
            }
            out[c] = (uint8_t)code;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            h2 = __fadd_ru(h2, __shfl_xor_sync(0xffffffffu, h2, o));
            e2 = __fadd_ru(e2, __shfl_xor_sync(0xffffffffu, e2, o));
        }
        if (lane == 0) {
            if (nhat) nhat[src] = __fsqrt_ru(h2);
            if (del) del[src] = __fsqrt_ru(e2);
        }
    }
}

// Largest row exponent of each tile of sorted rows.
__global__ void k_tile_exp(const int* __restrict__ ex, const int* __restrict__ perm, int64_t count, int tile,
                           int64_t tiles, int* __restrict__ texp) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tiles; t += warps) {
        int mx = INT_MIN;
        int64_t i0 = t * tile, i1 = i0 + tile;
        if (i1 > count) i1 = count;
        for (int64_t i = i0 + lane; i < i1; i += 32) mx = max(mx, ex[perm[i]]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) texp[t] = (mx == INT_MIN) ? 0 : fp8_exp(mx);
    }
}

__global__ void k_hist(const float* __restrict__ keys, int64_t count, bool desc,
                       unsigned* __restrict__ hist) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned b = bucket16(keys[i]);
        if (desc) b = (NBUCKET - 1) - b;
        atomicAdd(&hist[b], 1u);
    }
}

// Exclusive scan of the bucket counts hist into offs and inclusive into cum (if non-null), in
// two launches of SCAN_BLOCKS blocks with coalesced accesses: each block scans its SCAN_BLOCK
// buckets (warp shuffles, then the warp totals) and records its total; then each block adds
// the totals of the blocks before it.
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_part(const unsigned* __restrict__ hist,
                                                          unsigned* __restrict__ offs,
                                                          unsigned* __restrict__ totals) {
    __shared__ unsigned wsum[SCAN_BLOCK / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int i = blockIdx.x * SCAN_BLOCK + t;
    const unsigned h = hist[i];
    unsigned x = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned z = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        wsum[lane] = z;
    }
    __syncthreads();
    offs[i] = (w > 0 ? wsum[w - 1] : 0u) + x - h;
    if (t == SCAN_BLOCK - 1) totals[blockIdx.x] = wsum[SCAN_BLOCK / 32 - 1];
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_fix(const unsigned* __restrict__ hist,
                                                         unsigned* __restrict__ offs, unsigned* __restrict__ cum,
                                                         const unsigned* __restrict__ totals) {
    __shared__ unsigned base;
    const int t = threadIdx.x;
    if (t < 32) {
        unsigned z = 0u;
        for (int j = t; j < (int)blockIdx.x; j += 32) z += totals[j];
        z = warp_sum(z);
        if (t == 0) base = z;
    }
    __syncthreads();
    const int i = blockIdx.x * SCAN_BLOCK + t;
    const unsigned o = offs[i] + base;
    offs[i] = o;
    if (cum) cum[i] = o + hist[i];
}

__global__ void k_scatter(const float* __restrict__ keys, int64_t count, bool desc,
                          unsigned* __restrict__ offs, int* __restrict__ perm) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned b = bucket16(keys[i]);
        if (desc) b = (NBUCKET - 1) - b;
        unsigned pos = atomicAdd(&offs[b], 1u);
        perm[pos] = (int)i;
    }
}

template <typename T>
__global__ void k_gather(const T* __restrict__ src, const int* __restrict__ perm, int64_t count,
                         T* __restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

// Per tile of `tile` consecutive sorted rows: max ||p||, max ||p^||, max ||p^ - p||.
__global__ void k_tile_max(const float* __restrict__ nrm, const float* __restrict__ nhat,
                           const float* __restrict__ del, const int* __restrict__ perm, int64_t count, int tile,
                           int64_t tiles, float* __restrict__ tmax, float* __restrict__ thmax,
                           float* __restrict__ tdel) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tiles; t += warps) {
        float a = 0.f, b = 0.f, c = 0.f;
        int64_t i0 = t * tile, i1 = i0 + tile;
        if (i1 > count) i1 = count;
        for (int64_t i = i0 + lane; i < i1; i += 32) {
            const int src = perm[i];
            a = fmaxf(a, nrm[src]);
            b = fmaxf(b, nhat[src]);
            c = fmaxf(c, del[src]);
        }
        a = warp_max(a);
        b = warp_max(b);
        c = warp_max(c);
        if (lane == 0) {
            tmax[t] = a;
            thmax[t] = b;
            tdel[t] = c;
        }
    }
}

// r_u <= tau_u / ||u||: divide by an upper bound of ||u|| rounding down, then round the
// FP64 quotient down to FP32.  Users with tau_u <= 0 keep every item (r = -inf).
__global__ void k_user_ratio(const double* __restrict__ tau, const double* __restrict__ norm2,
                             int64_t n, float* __restrict__ r) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        double t = tau[u];
        float v = -INFINITY;
        if (t > 0.0) {
            double nu = __dsqrt_ru(norm2[u]);
            v = __double2float_rd(__ddiv_rd(t, nu));
        }
        r[u] = v;
    }
}

__global__ void k_user_meta(const double* __restrict__ tau, const float* __restrict__ nrm,
                            const float* __restrict__ nhat, const float* __restrict__ del,
                            const int* __restrict__ ex, const int* __restrict__ perm, int64_t n,
                            UserMeta* __restrict__ meta) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int u = perm[i];
        const double t = tau[u];
        UserMeta r;
        r.tau_hi = __double2float_ru(t);
        r.tau_lo = __double2float_rd(t);
        r.un = nrm[u];
        r.unh = nhat[u];
        r.ud = del[u];
        r.uorig = u;
        r.uexp = ex[u];
        r.pad1 = 0.f;
        meta[i] = r;
    }
}

__global__ void k_item_uscore(const float* __restrict__ nrm_hi, int64_t m,
                              const unsigned* __restrict__ ucum, int* __restrict__ uscore) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        uscore[i] = (int)ucum[bucket16(nrm_hi[i])];
}

}  // namespace

void launch_prep_rows(const float* X, int64_t rows, int64_t ld, int d, int* ex, int16_t* q, int dq,
                      double* norm2, float* nrm_hi, float* nhat_hi, float* del_hi, int operand,
                      DevStatus* st, cudaStream_t s) {
    if (rows <= 0) return;
    // Lanes per row: about 8 elements per lane, between 4 and 32 lanes.
    int lpr = 4;
    while (lpr < 32 && lpr * 8 < dq) lpr <<= 1;
    const int64_t warps = (rows + (32 / lpr) - 1) / (32 / lpr);
    note_launch();
    k_prep_rows<<<grid_for(warps * 32, 256, 65536), 256, 0, s>>>(X, rows, ld, d, ex, q, dq, norm2,
                                                                  nrm_hi, nhat_hi, del_hi, operand,
                                                                  &st->off_grid, lpr);
}

void launch_pack_fp8(const float* X, int64_t rows, int64_t ld, int d, const int* perm, const int* row_exp,
                     const int* tile_exp, int tile, uint8_t* dst, int64_t rows_pad, int dp, float* nhat,
                     float* del, cudaStream_t s) {
    if (rows_pad <= 0) return;
    note_launch();
    k_pack_fp8<<<grid_for(rows_pad * 32, 256, 65536), 256, 0, s>>>(X, rows, ld, d, perm, row_exp, tile_exp, tile,
                                                                     dst, rows_pad, dp, nhat, del);
}

void launch_tile_exp(const int* ex, const int* perm, int64_t count, int tile, int64_t tiles, int* texp,
                     cudaStream_t s) {
    if (tiles <= 0) return;
    note_launch();
    k_tile_exp<<<grid_for(tiles * 32, 256, 65536), 256, 0, s>>>(ex, perm, count, tile, tiles, texp);
}

void launch_pack_f32(const float* X, int64_t rows, int64_t ld, int d, const int* perm, float* dst,
                     int64_t rows_pad, int dp, cudaStream_t s) {
    if (rows_pad <= 0) return;
    note_launch();
    k_pack<float><<<grid_for(rows_pad * (dp / 8), 256, 65536), 256, 0, s>>>(X, rows, ld, d, perm, dst,
                                                                            rows_pad, dp);
}

void launch_pack_bf16(const float* X, int64_t rows, int64_t ld, int d, const int* perm,
                      __nv_bfloat16* dst, int64_t rows_pad, int dp, cudaStream_t s) {
    if (rows_pad <= 0) return;
    note_launch();
    k_pack<__nv_bfloat16><<<grid_for(rows_pad * (dp / 8), 256, 65536), 256, 0, s>>>(X, rows, ld, d, perm,
                                                                                    dst, rows_pad, dp);
}

void launch_bucket_sort(const float* keys, int64_t count, bool descending, unsigned* hist,
                        unsigned* offs, int* perm, unsigned* cum, cudaStream_t s) {
    cudaMemsetAsync(hist, 0, NBUCKET * sizeof(unsigned), s);
    if (count > 0) {
        note_launch();
        k_hist<<<grid_for(count, 256, 4096), 256, 0, s>>>(keys, count, descending, hist);
    }
    note_launch();
    k_scan_part<<<SCAN_BLOCKS, SCAN_BLOCK, 0, s>>>(hist, offs, hist + NBUCKET);
    note_launch();
    k_scan_fix<<<SCAN_BLOCKS, SCAN_BLOCK, 0, s>>>(hist, offs, cum, hist + NBUCKET);
    if (count > 0) {
        note_launch();
        k_scatter<<<grid_for(count, 256, 4096), 256, 0, s>>>(keys, count, descending, offs, perm);
    }
}

void launch_gather_f32(const float* src, const int* perm, int64_t count, float* dst, cudaStream_t s) {
    if (count > 0) {
        note_launch();
        k_gather<float><<<grid_for(count, 256, 65536), 256, 0, s>>>(src, perm, count, dst);
    }
}
void launch_gather_f64(const double* src, const int* perm, int64_t count, double* dst, cudaStream_t s) {
    if (count > 0) {
        note_launch();
        k_gather<double><<<grid_for(count, 256, 65536), 256, 0, s>>>(src, perm, count, dst);
    }
}
void launch_gather_i32(const int* src, const int* perm, int64_t count, int* dst, cudaStream_t s) {
    if (count > 0) {
        note_launch();
        k_gather<int><<<grid_for(count, 256, 65536), 256, 0, s>>>(src, perm, count, dst);
    }
}

void launch_tile_max(const float* nrm, const float* nhat, const float* del, const int* perm, int64_t count,
                     int tile, int64_t tiles, float* tmax, float* thmax, float* tdel, cudaStream_t s) {
    if (tiles > 0) {
        note_launch();
        k_tile_max<<<grid_for(tiles * 32, 256, 65536), 256, 0, s>>>(nrm, nhat, del, perm, count, tile, tiles,
                                                                     tmax, thmax, tdel);
    }
}

__global__ void k_seed_ratio(const unsigned* __restrict__ lkey, const float* __restrict__ nrm, int64_t n,
                             float* __restrict__ r) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const float L = key_float(lkey[u]);
        r[u] = (L > 0.f && nrm[u] > 0.f) ? L / nrm[u] : -INFINITY;
    }
}

void launch_seed_ratio(const unsigned* lkey, const float* nrm, int64_t n, float* r, cudaStream_t s) {
    if (n > 0) {
        note_launch();
        k_seed_ratio<<<grid_for(n, 256, 65536), 256, 0, s>>>(lkey, nrm, n, r);
    }
}

void launch_user_ratio(const double* tau, const double* norm2, int64_t n, float* r, cudaStream_t s) {
    if (n > 0) {
        note_launch();
        k_user_ratio<<<grid_for(n, 256, 65536), 256, 0, s>>>(tau, norm2, n, r);
    }
}

void launch_user_meta(const double* tau, const float* nrm, const float* nhat, const float* del, const int* ex,
                      const int* perm, int64_t n, UserMeta* meta, cudaStream_t s) {
    if (n > 0) {
        note_launch();
        k_user_meta<<<grid_for(n, 256, 65536), 256, 0, s>>>(tau, nrm, nhat, del, ex, perm, n, meta);
    }
}

void launch_item_uscore(const float* nrm_hi, int64_t m, const unsigned* ucum, int* uscore,
                        cudaStream_t s) {
    if (m > 0) {
        note_launch();
        k_item_uscore<<<grid_for(m, 256, 65536), 256, 0, s>>>(nrm_hi, m, ucum, uscore);
    }
}

}  // namespace rkm
