// K7: top-N items (Definition 3, ties by smaller id) by a most-significant-digit radix
// select over the unique 64-bit keys (score << 32) | (0xFFFFFFFF - id), then a rank sort
// of the N selected keys.  Also the filter cut of the counting pass (the stopping rule of
// Algorithm 2 applied to whole item tiles with an exact lower bound of the N-th score).
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace rkm {

namespace {

constexpr int TOPN_THREADS = 1024;

__device__ __forceinline__ unsigned long long topn_key(const int* counts, const int* item_id, int64_t pos) {
    const unsigned id = item_id ? (unsigned)item_id[pos] : (unsigned)pos;
    return ((unsigned long long)(unsigned)counts[pos] << 32) | (unsigned long long)(0xFFFFFFFFu - id);
}

__global__ void __launch_bounds__(TOPN_THREADS) k_topn(const int* __restrict__ counts,
                                                       const int* __restrict__ item_id, int64_t m,
                                                       const int* m_lim_dev, int N, int* __restrict__ ids,
                                                       int* __restrict__ scores, DevStatus* st) {
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned s_need;
    __shared__ unsigned s_sel;
    __shared__ unsigned long long sel[NMAX_TOPN];
    const int t = threadIdx.x;
    int64_t M = m;
    if (m_lim_dev) {
        const int64_t lim = *m_lim_dev;
        if (lim < M) M = lim;
    }
    if (M < N || N > NMAX_TOPN) {
        if (t == 0) st->internal_error = 1u;
        return;
    }
    if (t == 0) {
        s_prefix = 0ull;
        s_need = (unsigned)N;
        s_sel = 0u;
    }
    unsigned long long mask = 0ull;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = t; b < 256; b += TOPN_THREADS) hist[b] = 0u;
        __syncthreads();
        const unsigned long long prefix = s_prefix;
        for (int64_t p = t; p < M; p += TOPN_THREADS) {
            const unsigned long long key = topn_key(counts, item_id, p);
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
    // s_prefix is now the N-th largest key; keys are unique, so exactly N keys are >= it.
    const unsigned long long kth = s_prefix;
    for (int64_t p = t; p < M; p += TOPN_THREADS) {
        const unsigned long long key = topn_key(counts, item_id, p);
        if (key >= kth) {
            const unsigned slot = atomicAdd(&s_sel, 1u);
            if (slot < (unsigned)NMAX_TOPN) sel[slot] = key;
        }
    }
    __syncthreads();
    if (s_sel != (unsigned)N) {
        if (t == 0) st->internal_error = 1u;
        return;
    }
    for (int j = t; j < N; j += TOPN_THREADS) {
        const unsigned long long key = sel[j];
        int rank = 0;
        for (int r = 0; r < N; ++r) rank += sel[r] > key;
        ids[rank] = (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
        scores[rank] = (int)(key >> 32);
    }
}

// One thread: LB = N-th score of the first stage; cut at the first tile whose Eq. 2 bound
// (users in ratio buckets up to the tile's largest norm) is below LB.  The bound of a
// tile never increases along the norm order, so a binary search applies.
__global__ void k_filter_cut(const int* __restrict__ top_scores_c0, int N, const float* __restrict__ tmax,
                             const unsigned* __restrict__ ucum, int64_t tiles, int t_begin, int tile_items,
                             int64_t m, DevStatus* st) {
    const unsigned lb = (unsigned)top_scores_c0[N - 1];
    int64_t lo = t_begin, hi = tiles;  // answer in [t_begin, tiles]
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (ucum[bucket16(tmax[mid])] < lb) hi = mid; else lo = mid + 1;
    }
    st->t_end = (int)lo;
    const int64_t mc = lo * (int64_t)tile_items;
    st->m_counted = (int)(mc < m ? mc : m);
}

// Single block: per item tile of [t_begin, t_end) its user prefix and work units, and
// the exclusive scan of the units.
__global__ void k_build_units(const float* __restrict__ tmax, const unsigned* __restrict__ ucum, int t_begin,
                              int t_end_host, const int* t_end_dev, int tile_users, int group,
                              int* __restrict__ nprefix, unsigned* __restrict__ unit_off, DevStatus* st) {
    constexpr int T = 1024;
    __shared__ unsigned part[T];
    const int t = threadIdx.x;
    const int t_end = t_end_dev ? *t_end_dev : t_end_host;
    const int len = t_end > t_begin ? t_end - t_begin : 0;
    const int per = (len + T - 1) / T;
    const int b0 = t * per;
    const int b1 = (b0 + per < len) ? b0 + per : len;
    unsigned local = 0;
    for (int j = b0; j < b1; ++j) {
        const int tile = t_begin + j;
        const unsigned np = ucum[bucket16(tmax[tile])];
        nprefix[tile] = (int)np;
        const unsigned ut = (np + tile_users - 1) / tile_users;
        local += (ut + group - 1) / group;
    }
    part[t] = local;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        unsigned v = (t >= o) ? part[t - o] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned run = part[t] - local;
    for (int j = b0; j < b1; ++j) {
        const unsigned np = (unsigned)nprefix[t_begin + j];
        const unsigned ut = (np + tile_users - 1) / tile_users;
        unit_off[j] = run;
        run += (ut + group - 1) / group;
    }
    if (t == T - 1) {
        unit_off[len] = part[T - 1];
        st->units_total = part[T - 1];
        st->ticket = 0u;
        st->t_end = t_end;
    }
}

}  // namespace

void launch_topn(const int* counts, const int* item_id, int64_t m, const int* m_lim_dev, int N, int* ids,
                 int* scores, DevStatus* st, cudaStream_t s) {
    note_launch();
    k_topn<<<1, TOPN_THREADS, 0, s>>>(counts, item_id, m, m_lim_dev, N, ids, scores, st);
}

void launch_filter_cut(const int* top_scores_c0, int N, const float* tmax, const unsigned* ucum, int64_t tiles,
                       int t_begin, int tile_items, int64_t m, DevStatus* st, cudaStream_t s) {
    note_launch();
    k_filter_cut<<<1, 1, 0, s>>>(top_scores_c0, N, tmax, ucum, tiles, t_begin, tile_items, m, st);
}

void launch_build_units(const float* tmax, const unsigned* ucum, int t_begin, int t_end, const int* t_end_dev,
                        int tile_users, int group, int* nprefix, unsigned* unit_off, DevStatus* st,
                        cudaStream_t s) {
    note_launch();
    k_build_units<<<1, 1024, 0, s>>>(tmax, ucum, t_begin, t_end, t_end_dev, tile_users, group, nprefix,
                                     unit_off, st);
}

}  // namespace rkm
