// FP32 CUDA-core product kernels: the plain exact path of the threshold pass (K2)
// and the counting pass (K5).  Each 128-user x 128-item tile is computed with
// sequential FP32 FMAs (so |v - u.p| <= gamma_d * ||u|| ||p||, Higham, "Accuracy and
// Stability of Numerical Algorithms", 2nd ed., Section 3.1), staged through shared
// memory and handed row by row to the per-user epilogues of epilogue.cuh.
#include <cuda_runtime.h>

#include "common.cuh"
#include "count_units.cuh"
#include "epilogue.cuh"
#include "kernels.h"

namespace rkm {

namespace {

constexpr int KC = 32;          // k-chunk of the product loop
constexpr int ASTR = 132;       // row stride (floats) of the transposed operand chunks
constexpr int CSTR = 132;       // row stride of the staged score tile
constexpr int SIMT_THREADS = 256;

struct SimtSmem {
    float As[KC * ASTR];        // users chunk, [k][user]
    float Bs[KC * ASTR];        // items chunk, [k][item]
    float Cs[BU * CSTR];        // scores, [user][item]
};

// Load a 128-row x 32-k chunk of a packed operand (row stride dp) transposed into S[k][row].
__device__ __forceinline__ void load_chunk_t(const float* __restrict__ X, int64_t row0, int dp, int k0,
                                             float* S) {
    const int t = threadIdx.x;
    const int r = t & 127;
    const int kq0 = t >> 7;  // 0 or 1
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int kq = kq0 + 2 * i;  // float4 index within the chunk, 0..7
        const float4 x = *reinterpret_cast<const float4*>(X + (row0 + r) * (int64_t)dp + k0 + kq * 4);
        S[(kq * 4 + 0) * ASTR + r] = x.x;
        S[(kq * 4 + 1) * ASTR + r] = x.y;
        S[(kq * 4 + 2) * ASTR + r] = x.z;
        S[(kq * 4 + 3) * ASTR + r] = x.w;
    }
}

// Cs = A[row0a .. +128) . B[row0b .. +128)^T over the padded depth dp (multiple of 32).
__device__ void simt_tile(const float* __restrict__ A, int64_t row0a, const float* __restrict__ B,
                          int64_t row0b, int dp, SimtSmem& sm) {
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < dp; k0 += KC) {
        load_chunk_t(A, row0a, dp, k0, sm.As);
        load_chunk_t(B, row0b, dp, k0, sm.Bs);
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KC; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&sm.As[kk * ASTR + ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&sm.As[kk * ASTR + 64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&sm.Bs[kk * ASTR + tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&sm.Bs[kk * ASTR + 64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = (i < 4) ? (ty * 4 + i) : (64 + ty * 4 + i - 4);
        *reinterpret_cast<float4*>(&sm.Cs[row * CSTR + tx * 4]) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        *reinterpret_cast<float4*>(&sm.Cs[row * CSTR + 64 + tx * 4]) =
            make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
    __syncthreads();
}

__device__ __forceinline__ void load_row_chunk(const SimtSmem& sm, int row, int c0, float (&v)[32]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 x = *reinterpret_cast<const float4*>(&sm.Cs[row * CSTR + c0 + q * 4]);
        v[q * 4 + 0] = x.x;
        v[q * 4 + 1] = x.y;
        v[q * 4 + 2] = x.z;
        v[q * 4 + 3] = x.w;
    }
}

// K2: persistent over user tiles; every CTA scans all item tiles for its users.
__global__ void __launch_bounds__(SIMT_THREADS, 1) k_threshold_simt(ThresholdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SimtSmem& sm = *reinterpret_cast<SimtSmem*>(smem_raw);
    float* heap = reinterpret_cast<float*>(smem_raw + sizeof(SimtSmem));  // [k][BU]
    const float* A = static_cast<const float*>(a.A);
    const float* B = static_cast<const float*>(a.B);
    const int t = threadIdx.x;
    const int64_t user_tiles = (a.n + BU - 1) / BU;
    const int64_t item_tiles = (a.m + BI_SIMT - 1) / BI_SIMT;
    for (int64_t ut = blockIdx.x; ut < user_tiles; ut += gridDim.x) {
        const int64_t u = ut * BU + t;
        const bool owner = t < BU;
        const bool active = owner && u < a.n;
        SelState s;
        s.L = -INFINITY;
        s.hn = 0;
        s.Lw = -INFINITY;
        s.Lx = -INFINITY;
        s.thr = -INFINITY;
        s.cnt = 0;
        s.pub = nullptr;
        s.tag = 0u;
        s.defer = 0;
        s.mark = 0;
        float un = 0.f, unh = 0.f, ud = 0.f;
        Cand* mycand = nullptr;
        if (owner) {
            for (int j = 0; j < a.k; ++j) heap[j * BU + t] = -INFINITY;
            if (active) {
                un = a.unrm[u];
                unh = a.unhat[u];
                ud = a.udel[u];
                mycand = a.cand + u * (int64_t)a.nseg * a.cap;
            }
        }
        int64_t tiles_done = 0;
        for (int64_t it = 0; it < item_tiles; ++it) {
            simt_tile(A, ut * BU, B, it * BI_SIMT, a.dp, sm);
            bool need_next = false;
            if (owner) {
                const float E = err_bound(a.cacc, a.eabs, un, unh, ud, a.thmax[it], a.tdel[it]);
                s.thr = __fsub_rd(sel_bound(s), E);
#pragma unroll 1
                for (int c0 = 0; c0 < BI_SIMT; c0 += 32) {
                    float v[32];
                    load_row_chunk(sm, t, c0, v);
                    sel_chunk(v, active, (int)(it * BI_SIMT + c0), a.m, E, s, mycand, a.cap, heap, t,
                              a.k, a.st);
                }
                // Algorithm 1's stop by Cauchy-Schwarz: items come in descending norm order, so
                // once ||u|| max||p|| of the next tile (rounded up) is below a lower bound of
                // tau_u, no later item can reach tau_u or tie it.
                need_next = active && it + 1 < item_tiles && !(__fmul_ru(un, a.tmax[it + 1]) < sel_bound(s));
            }
            ++tiles_done;
            if (!__syncthreads_or(need_next)) break;
        }
        if (t == 0) {
            const int64_t rows = (a.n - ut * BU < BU) ? a.n - ut * BU : BU;
            const int64_t items = (tiles_done * BI_SIMT < a.m) ? tiles_done * BI_SIMT : a.m;
            atomicAdd(&a.st->thr_pairs, (unsigned long long)(rows * items));
        }
        if (active) {
            atomicMax(&a.lfin_key[u], float_key(fmaxf(s.L, s.Lw)));
            a.cand_cnt[u * a.nseg] = s.cnt;
        }
    }
}

// K5: persistent over work units (item tile, group of user tiles) taken from a ticket.
__global__ void __launch_bounds__(SIMT_THREADS, 1) k_count_simt(CountArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SimtSmem& sm = *reinterpret_cast<SimtSmem*>(smem_raw);
    int* cnt_s = reinterpret_cast<int*>(smem_raw + sizeof(SimtSmem));  // [BI_SIMT]
    __shared__ unsigned s_unit;
    const float* A = static_cast<const float*>(a.A);
    const float* B = static_cast<const float*>(a.B);
    const int t = threadIdx.x;
    const unsigned total = a.st->units_total;
    while (true) {
        if (t == 0) s_unit = atomicAdd(&a.st->ticket, 1u);
        __syncthreads();
        const unsigned w = s_unit;
        __syncthreads();
        if (w >= total) break;
        int T;
        int64_t ut0, ut1;
        decode_count_unit(a, w, T, ut0, ut1);
        if (t < BI_SIMT) cnt_s[t] = 0;
        __syncthreads();
        const float pnh = a.thmax[T], pd = a.tdel[T];
        const int pos0 = T * BI_SIMT;
        for (int64_t ut = ut0; ut < ut1; ++ut) {
            simt_tile(A, ut * BU, B, (int64_t)T * BI_SIMT, a.dp, sm);
            if (t < BU) {
                const int64_t us = ut * BU + t;
                const bool active = us < a.n;
                float hi_t = 0.f, lo_t = 0.f;
                int u_orig = 0;
                if (active) {
                    const UserMeta um = a.meta[us];
                    const float E = err_bound(a.cacc, a.eabs, um.un, um.unh, um.ud, pnh, pd);
                    hi_t = __fadd_ru(um.tau_hi, E);
                    lo_t = __fsub_rd(um.tau_lo, E);
                    u_orig = um.uorig;
                }
#pragma unroll 1
                for (int c0 = 0; c0 < BI_SIMT; c0 += 32) {
                    float v[32];
                    load_row_chunk(sm, t, c0, v);
                    count_chunk(v, active, c0, pos0 + c0, a.m, hi_t, lo_t, cnt_s, u_orig, a.band,
                                a.band_cap, a.st);
                }
            }
            __syncthreads();
        }
        if (t == 0 && ut1 > ut0) {
            unsigned long long users = (unsigned long long)((ut1 * BU < a.n ? ut1 * BU : a.n) - ut0 * BU);
            atomicAdd(&a.st->pairs_evaluated, users * (unsigned long long)BI_SIMT);
        }
        if (t < BI_SIMT && cnt_s[t] != 0 && pos0 + t < a.m) atomicAdd(&a.counts[pos0 + t], cnt_s[t]);
        __syncthreads();
    }
}

}  // namespace

void launch_threshold_simt(const ThresholdArgs& a, cudaStream_t s) {
    const size_t smem = sizeof(SimtSmem) + (size_t)KMAX * BU * sizeof(float);
    cudaFuncSetAttribute(k_threshold_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t user_tiles = (a.n + BU - 1) / BU;
    int grid = (int)(user_tiles < a.num_sms ? user_tiles : a.num_sms);
    if (grid < 1) return;
    note_launch();
    k_threshold_simt<<<grid, SIMT_THREADS, smem, s>>>(a);
}

void launch_count_simt(const CountArgs& a, cudaStream_t s) {
    const size_t smem = sizeof(SimtSmem) + BI_SIMT * sizeof(int);
    cudaFuncSetAttribute(k_count_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    k_count_simt<<<a.num_sms, SIMT_THREADS, smem, s>>>(a);
}

}  // namespace rkm
