// Per-user epilogues of the fused product kernels.
//
// Both product passes see approximate scores v ~ u.p with a proven error bound E
// (|v - u.p| <= E for every pair of the tile).  One thread owns one user row of
// the tile and consumes it 32 columns at a time.
//
// Threshold pass (K2, Definition 1).  The thread keeps a min-heap of the k largest
// lower bounds v - E seen so far; its root L never exceeds tau_u, because k items
// have u.p >= L.  Any item with u.p >= tau_u has v + E >= u.p >= L, so keeping every
// item with v >= L - E as a candidate (with its upper bound v + E) keeps all of
// S_k(u) and every item tied with t_u.  Candidates whose upper bound fell below the
// current L can never be needed and are compacted away when the list fills.
//
// Counting pass (K5, Eq. 1).  v > tau_u + E proves u.p > tau_u (member); v < tau_u - E
// proves u.p < tau_u (not a member); anything between is queued for exact rescoring.
#pragma once

#include "common.cuh"

namespace rkm {

// Heap element j of user-thread t lives at heap[j * BU + t] (conflict-free per warp).
__device__ __forceinline__ void heap_replace_root(float* heap, int t, int k, float v) {
    int j = 0;
    while (true) {
        int l = 2 * j + 1;
        if (l >= k) break;
        int c = l;
        float cv = heap[l * BU + t];
        int r = l + 1;
        if (r < k) {
            float rv = heap[r * BU + t];
            if (rv < cv) { c = r; cv = rv; }
        }
        if (cv >= v) break;
        heap[j * BU + t] = cv;
        j = c;
    }
    heap[j * BU + t] = v;
}

static __device__ __noinline__ int compact_candidates(Cand* c, int cnt, float L) {
    int w = 0;
    for (int r = 0; r < cnt; ++r) {
        Cand x = c[r];
        if (x.ub >= L) c[w++] = x;
    }
    return w;
}

struct SelState {
    float L;    // root of the lower-bound heap (k-th largest v - E so far)
    float thr;  // L - E of the current tile, rounded down
    int cnt;    // candidates stored
};

__device__ __forceinline__ void sel_insert(float v, int pos, float E, SelState& s, Cand* mycand, int cap,
                                        float* heap, int t, int k, DevStatus* st) {
    const float ub = __fadd_ru(v, E);
    const float lb = __fsub_rd(v, E);
    if (s.cnt >= cap) s.cnt = compact_candidates(mycand, s.cnt, s.L);
    if (s.cnt < cap) {
        Cand c;
        c.ub = ub;
        c.pos = pos;
        mycand[s.cnt++] = c;
    } else {
        st->cand_overflow = 1u;
    }
    if (lb > s.L) {
        heap_replace_root(heap, t, k, lb);
        s.L = heap[t];
        s.thr = __fsub_rd(s.L, E);
    }
}

__device__ __forceinline__ float max32(const float (&v)[32]) {
    float a = fmaxf(v[0], v[1]), b = fmaxf(v[2], v[3]);
#pragma unroll
    for (int c = 4; c < 32; c += 4) {
        a = fmaxf(a, fmaxf(v[c], v[c + 1]));
        b = fmaxf(b, fmaxf(v[c + 2], v[c + 3]));
    }
    return fmaxf(a, b);
}

// Threshold-pass epilogue of one 32-column chunk.  Must be called by all 32 lanes of
// the warp (warp-uniform fast path); `active` masks lanes without a valid user.
__device__ __forceinline__ void sel_chunk(const float (&v)[32], bool active, int pos0, int64_t m,
                                          float E, SelState& s, Cand* mycand, int cap, float* heap,
                                          int t, int k, DevStatus* st) {
    const bool hit = active && (max32(v) >= s.thr);
    if (!__any_sync(0xffffffffu, hit)) return;
    if (hit) {
#pragma unroll
        for (int c = 0; c < 32; ++c)
            if (v[c] >= s.thr && pos0 + c < m) sel_insert(v[c], pos0 + c, E, s, mycand, cap, heap, t, k, st);
    }
}

// Counting-pass epilogue of one 32-column chunk; same calling rule as sel_chunk.
// cnt_s: per-column member counters of the tile (shared memory), indexed by column.
__device__ __forceinline__ void count_chunk(const float (&v)[32], bool active, int col0, int pos0,
                                            int64_t mlim, float hi, float lo, int* cnt_s,
                                            int u_orig, int2* band, unsigned band_cap,
                                            DevStatus* st) {
    const bool hit = active && (max32(v) >= lo);
    if (!__any_sync(0xffffffffu, hit)) return;
    if (hit) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const float x = v[c];
            if (x >= lo && pos0 + c < mlim) {
                if (x > hi) {
                    atomicAdd(&cnt_s[col0 + c], 1);
                } else {
                    unsigned idx = atomicAdd(&st->band_count, 1u);
                    if (idx < band_cap) band[idx] = make_int2(u_orig, pos0 + c);
                    else st->band_overflow = 1u;
                }
            }
        }
    }
}

}  // namespace rkm
