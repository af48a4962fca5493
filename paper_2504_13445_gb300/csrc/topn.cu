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

// Shared memory of one top-N select (one CTA of TOPN_THREADS threads).
struct TopnSmem {
    unsigned hist[256];
    unsigned long long prefix;
    unsigned need;
    unsigned sel_count;
    unsigned long long sel[NMAX_TOPN];
};

// Top N of positions [0, M) (all threads of the CTA call it).
__device__ __forceinline__ void topn_select(TopnSmem& sm, const int* __restrict__ counts,
                                            const int* __restrict__ item_id, int64_t M, int N, int* __restrict__ ids,
                                            int* __restrict__ scores, DevStatus* st) {
    const int t = threadIdx.x;
    if (M < N || N > NMAX_TOPN) {
        if (t == 0) st->internal_error = 1u;
        return;
    }
    if (t == 0) {
        sm.prefix = 0ull;
        sm.need = (unsigned)N;
        sm.sel_count = 0u;
    }
    unsigned long long mask = 0ull;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = t; b < 256; b += TOPN_THREADS) sm.hist[b] = 0u;
        __syncthreads();
        const unsigned long long prefix = sm.prefix;
        for (int64_t p = t; p < M; p += TOPN_THREADS) {
            const unsigned long long key = topn_key(counts, item_id, p);
            if ((key & mask) == prefix) atomicAdd(&sm.hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (t == 0) {
            unsigned need = sm.need, cum = 0u;
            int dg = 255;
            for (; dg > 0; --dg) {
                if (cum + sm.hist[dg] >= need) break;
                cum += sm.hist[dg];
            }
            sm.need = need - cum;
            sm.prefix = prefix | ((unsigned long long)dg << shift);
        }
        mask |= (0xFFull << shift);
        __syncthreads();
    }
    // sm.prefix is now the N-th largest key; keys are unique, so exactly N keys are >= it.
    const unsigned long long kth = sm.prefix;
    for (int64_t p = t; p < M; p += TOPN_THREADS) {
        const unsigned long long key = topn_key(counts, item_id, p);
        if (key >= kth) {
            const unsigned slot = atomicAdd(&sm.sel_count, 1u);
            if (slot < (unsigned)NMAX_TOPN) sm.sel[slot] = key;
        }
    }
    __syncthreads();
    if (sm.sel_count != (unsigned)N) {
        if (t == 0) st->internal_error = 1u;
        return;
    }
    for (int j = t; j < N; j += TOPN_THREADS) {
        const unsigned long long key = sm.sel[j];
        int rank = 0;
        for (int r = 0; r < N; ++r) rank += sm.sel[r] > key;
        ids[rank] = (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
        scores[rank] = (int)(key >> 32);
    }
}

__global__ void __launch_bounds__(TOPN_THREADS) k_topn(const int* __restrict__ counts,
                                                       const int* __restrict__ item_id, int64_t m,
                                                       const int* m_lim_dev, int N, int* __restrict__ ids,
                                                       int* __restrict__ scores, DevStatus* st) {
    __shared__ TopnSmem sm;
    int64_t M = m;
    if (m_lim_dev) {
        const int64_t lim = *m_lim_dev;
        if (lim < M) M = lim;
    }
    topn_select(sm, counts, item_id, M, N, ids, scores, st);
}

// Top N of job blockIdx.x: stage 1 over the first-stage items, stage 2 over the counted ones.
__global__ void __launch_bounds__(TOPN_THREADS) k_topn_multi(const BatchJob* __restrict__ jobs, int stage) {
    __shared__ TopnSmem sm;
    const BatchJob& J = jobs[blockIdx.x];
    if (stage == 1) {
        const int64_t m0 = (int64_t)J.t0 * J.tile_items;
        topn_select(sm, J.counts, J.item_perm, m0 < J.m ? m0 : J.m, J.N, J.top_ids_c0, J.top_sc_c0, J.st);
    } else {
        const int64_t lim = J.st->m_counted;
        topn_select(sm, J.counts, J.item_perm, lim < J.m ? lim : J.m, J.N, J.ids, J.top_scores, J.st);
    }
}

// LB = N-th score of the first stage; cut at the first tile whose Eq. 2 bound (users in
// ratio buckets up to the tile's largest norm) is below LB.  The bound of a tile never
// increases along the norm order, so a binary search applies.
__device__ __forceinline__ void filter_cut(const int* __restrict__ top_scores_c0, int N,
                                           const float* __restrict__ tmax, const unsigned* __restrict__ ucum,
                                           int64_t tiles, int t_begin, int tile_items, int64_t m, DevStatus* st) {
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

__global__ void k_filter_cut(const int* __restrict__ top_scores_c0, int N, const float* __restrict__ tmax,
                             const unsigned* __restrict__ ucum, int64_t tiles, int t_begin, int tile_items,
                             int64_t m, DevStatus* st) {
    filter_cut(top_scores_c0, N, tmax, ucum, tiles, t_begin, tile_items, m, st);
}

__global__ void k_filter_cut_multi(const BatchJob* __restrict__ jobs, int count) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    const BatchJob& J = jobs[j];
    filter_cut(J.top_sc_c0, J.N, J.tmax, J.ucum, J.tiles, J.t0, J.tile_items, J.m, J.st);
}

// Work units of a counting stage over item tiles [t_begin, t_end) (one CTA of 1024 threads).
// Tile T needs the users of ratio-order prefix nprefix[T], i.e. ceil(nprefix[T] / tile_users)
// user tiles, cut into groups of `group` user tiles; the units are numbered tile-major, (T, g)
// for the groups g of tile T, and unit_off[j] is the first unit of tile t_begin + j
// (unit_off[len] = total).  Concurrent CTAs then hold one item tile (shared through L2) and
// stream different users.  (Numbering them group-major instead, so that concurrent CTAs
// share user tiles, was measured on GB300: 3 % faster on 2,000,000 users, 22 % slower on
// 500,000 and 36 % slower in the serving loop.)
__device__ __forceinline__ void build_units(const float* __restrict__ tmax, const unsigned* __restrict__ ucum,
                                            int t_begin, int t_end, int tile_users, int group,
                                            int* __restrict__ nprefix, unsigned* __restrict__ unit_off,
                                            DevStatus* st) {
    constexpr int T = 1024;
    __shared__ unsigned part[T];
    const int t = threadIdx.x;
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

__global__ void k_build_units(const float* __restrict__ tmax, const unsigned* __restrict__ ucum, int t_begin,
                              int t_end_host, const int* t_end_dev, int tile_users, int group,
                              int* __restrict__ nprefix, unsigned* __restrict__ unit_off, DevStatus* st) {
    build_units(tmax, ucum, t_begin, t_end_dev ? *t_end_dev : t_end_host, tile_users, group, nprefix, unit_off, st);
}

// Unit lists of job blockIdx.x: stage 1 over tiles [0, t0), stage 2 over [t0, st->t_end).
__global__ void k_build_units_multi(const BatchJob* __restrict__ jobs, int stage) {
    const BatchJob& J = jobs[blockIdx.x];
    const int t_begin = stage == 1 ? 0 : J.t0;
    const int t_end = stage == 1 ? J.t0 : J.st->t_end;
    build_units(J.tmax, J.ucum, t_begin, t_end, BU, J.group, J.nprefix, J.unit_off, J.st);
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

void launch_topn_multi(const BatchJob* jobs, int count, int stage, cudaStream_t s) {
    note_launch();
    k_topn_multi<<<count, TOPN_THREADS, 0, s>>>(jobs, stage);
}

void launch_filter_cut_multi(const BatchJob* jobs, int count, cudaStream_t s) {
    note_launch();
    k_filter_cut_multi<<<(count + 127) / 128, 128, 0, s>>>(jobs, count);
}

void launch_build_units_multi(const BatchJob* jobs, int count, int stage, cudaStream_t s) {
    note_launch();
    k_build_units_multi<<<count, 1024, 0, s>>>(jobs, stage);
}

}  // namespace rkm
