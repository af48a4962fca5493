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
    // Keep the candidates whose upper bound still reaches the bound L <= tau_u.
    int w = 0;
    for (int r = 0; r < cnt; ++r) {
        Cand x = c[r];
        if (x.ub >= L) c[w++] = x;
    }
    return w;
}

struct SelState {
    float L;     // heap root once the heap holds k lower bounds (-inf while it fills)
    int hn;      // lower bounds held in the heap (<= k)
    float Lw;    // warm-start bound of this group (-inf if none)
    float Lx;    // a lower bound of tau_u published by the other epilogue group (or -inf)
    float thr;   // max(L, Lw, Lx) - E of the current tile, rounded down
    int cnt;     // candidates stored
    unsigned long long* pub;  // where this group publishes its bound for the other (null: none)
    unsigned tag;             // user tile the published bound belongs to
    int defer;   // 1: hits only record candidates; sel_merge_tile admits them at the tile's end
    int mark;    // first candidate recorded in the current tile (-1 after a compaction in it)
};

// The best lower bound of tau_u this group knows.
__device__ __forceinline__ float sel_bound(const SelState& s) { return fmaxf(fmaxf(s.L, s.Lw), s.Lx); }

// A published bound: (user tile << 32) | bits of the bound, written and read as one 64-bit
// word so a reader never mixes a bound with the tag of another user tile.
__device__ __forceinline__ void publish_bound(unsigned long long* p, unsigned tag, float L) {
    *reinterpret_cast<volatile unsigned long long*>(p) =
        ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(L);
}

__device__ __forceinline__ float read_bound(const unsigned long long* p, unsigned tag) {
    const unsigned long long x = *reinterpret_cast<const volatile unsigned long long*>(p);
    return ((unsigned)(x >> 32) == tag) ? __uint_as_float((unsigned)(x & 0xffffffffull)) : -INFINITY;
}

// Min-heap order over heap[0 .. k) of user-thread t (bottom-up construction).
__device__ __forceinline__ void heapify(float* heap, int t, int k) {
    for (int i = k / 2 - 1; i >= 0; --i) {
        const float v = heap[i * BU + t];
        int j = i;
        while (true) {
            const int l = 2 * j + 1;
            if (l >= k) break;
            int c = l;
            float cv = heap[l * BU + t];
            if (l + 1 < k) {
                const float rv = heap[(l + 1) * BU + t];
                if (rv < cv) { c = l + 1; cv = rv; }
            }
            if (cv >= v) break;
            heap[j * BU + t] = cv;
            j = c;
        }
        heap[j * BU + t] = v;
    }
}

// Record a value that reached the threshold: store it as a candidate (with its upper bound),
// and admit its lower bound into the heap when it raises the best bound known here.  Any k
// lower bounds held in the heap make its root a valid lower bound of tau_u, so skipping an
// admission is sound; while the heap fills, admission is an append, and the heap is built
// once when it holds k values.
__device__ __forceinline__ void sel_insert(float v, int pos, float E, SelState& s, Cand* mycand, int cap,
                                           float* heap, int t, int k, DevStatus* st) {
    const float ub = __fadd_ru(v, E);
    const float lb = __fsub_rd(v, E);
    if (s.cnt >= cap) {
        s.cnt = compact_candidates(mycand, s.cnt, sel_bound(s));
        s.mark = -1;
    }
    if (s.cnt < cap) {
        Cand c;
        c.ub = ub;
        c.pos = pos;
        mycand[s.cnt++] = c;
    } else {
        st->cand_overflow = 1u;
    }
    if (s.defer) return;
    if (lb > sel_bound(s)) {
        if (s.hn < k) {
            heap[s.hn * BU + t] = lb;
            if (++s.hn < k) return;
            heapify(heap, t, k);
        } else {
            heap_replace_root(heap, t, k, lb);
        }
        s.L = heap[t];
        if (s.pub) publish_bound(s.pub, s.tag, fmaxf(s.L, s.Lw));
        s.thr = __fsub_rd(sel_bound(s), E);
    }
}

// A lower bound of u.p for a candidate recorded with ub = RU(v + E) in a tile whose products
// have error bound E: v >= ub - E - ulp(ub), so u.p >= v - E >= ub - 2E - ulp(ub) (the ulp
// taken as |ub| 2^-23 + 2^-149, every step rounded down).
__device__ __forceinline__ float cand_lower(float ub, float E) {
    const float d = __fadd_ru(__fmul_ru(fabsf(ub), 0x1p-23f), 0x1p-149f);
    return __fsub_rd(__fsub_rd(__fsub_rd(ub, E), E), d);
}

// Deferred admissions: the lower bounds of the candidates recorded since the tile started
// enter the heap at the tile's end, with every lane of the warp stepping through its own
// list together (the heap is built at most once per lane, in one place, instead of at the
// hit that completes it).  Skipping admissions is sound (see sel_insert), so a tile whose
// entries a compaction moved admits nothing.
__device__ __forceinline__ void sel_merge_tile(SelState& s, const Cand* mycand, float* heap, int t, int k, float E,
                                               bool active) {
    const int j0 = s.mark, j1 = s.cnt;
    s.mark = s.cnt;
    if (!active || j0 < 0 || j0 >= j1) return;
    const float L0 = sel_bound(s);
    int j = j0;
    bool filled = false;
    for (; j < j1 && s.hn < k; ++j) {
        const float lb = cand_lower(mycand[j].ub, E);
        if (lb > L0) {
            heap[s.hn * BU + t] = lb;
            if (++s.hn == k) filled = true;
        }
    }
    if (filled) {
        heapify(heap, t, k);
        s.L = heap[t];
    }
    for (; j < j1; ++j) {
        const float lb = cand_lower(mycand[j].ub, E);
        if (lb > sel_bound(s)) {
            heap_replace_root(heap, t, k, lb);
            s.L = heap[t];
        }
    }
    if (s.hn == k && s.pub) publish_bound(s.pub, s.tag, fmaxf(s.L, s.Lw));
}

// x = v[c] for a run-time c in [0, 32): a five-level select tree (no local memory).
__device__ __forceinline__ float select32(const float (&v)[32], int c) {
    float l1[16], l2[8], l3[4], l4[2];
#pragma unroll
    for (int i = 0; i < 16; ++i) l1[i] = (c & 1) ? v[2 * i + 1] : v[2 * i];
#pragma unroll
    for (int i = 0; i < 8; ++i) l2[i] = (c & 2) ? l1[2 * i + 1] : l1[2 * i];
#pragma unroll
    for (int i = 0; i < 4; ++i) l3[i] = (c & 4) ? l2[2 * i + 1] : l2[2 * i];
#pragma unroll
    for (int i = 0; i < 2; ++i) l4[i] = (c & 8) ? l3[2 * i + 1] : l3[2 * i];
    return (c & 16) ? l4[1] : l4[0];
}

// Maxima of the four 8-column groups of a chunk.
__device__ __forceinline__ void group_max8(const float (&v)[32], float (&g)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        g[q] = fmax3f(fmax3f(v[8 * q], v[8 * q + 1], v[8 * q + 2]), fmax3f(v[8 * q + 3], v[8 * q + 4], v[8 * q + 5]),
                      fmaxf(v[8 * q + 6], v[8 * q + 7]));
}

// Bit c of the result is set when v[c] >= thr, for the 8-column groups whose maximum g[q]
// reaches thr in some lane of the warp (all 32 lanes must call it).
__device__ __forceinline__ unsigned hit_mask(const float (&v)[32], const float (&g)[4], bool active, float thr) {
    unsigned mask = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool hq = active && g[q] >= thr;
        if (__any_sync(0xffffffffu, hq) && hq) {
#pragma unroll
            for (int j = 0; j < 8; ++j) mask |= (v[8 * q + j] >= thr ? 1u : 0u) << (8 * q + j);
        }
    }
    return mask;
}

// Threshold-pass epilogue of one 32-column chunk, called when the pair vote of the product
// kernel found a value reaching some lane's threshold.  Must be called by all 32 lanes of the
// warp: a maximum tree and a vote skip a chunk without hits; 8-column groups in which some
// lane reaches its threshold are compared element by element, and the hits are inserted one
// by one through a single call site.  `active` masks lanes without a valid user.
__device__ __forceinline__ void sel_chunk(const float (&v)[32], bool active, int pos0, int64_t m,
                                          float E, SelState& s, Cand* mycand, int cap, float* heap,
                                          int t, int k, DevStatus* st) {
    float g[4];
    group_max8(v, g);
    const float mx = fmax3f(g[0], g[1], fmaxf(g[2], g[3]));
    if (!__any_sync(0xffffffffu, active && mx >= s.thr)) return;
    unsigned mask = hit_mask(v, g, active, s.thr);
    while (mask) {
        const int c = __ffs(mask) - 1;
        mask &= mask - 1u;
        const float x = select32(v, c);
        // s.thr only grows, so skipping values now below it is still sound.
        if (x >= s.thr && pos0 + c < m) sel_insert(x, pos0 + c, E, s, mycand, cap, heap, t, k, st);
    }
}

// Counting-pass epilogue of one 32-column chunk; same calling rule as sel_chunk.
// cnt_s: per-column member counters of the tile (shared memory), indexed by column.
__device__ __forceinline__ void count_chunk(const float (&v)[32], bool active, int col0, int pos0,
                                            int64_t mlim, float hi, float lo, int* cnt_s,
                                            int u_orig, int2* band, unsigned band_cap,
                                            DevStatus* st) {
    float g[4];
    group_max8(v, g);
    const float mx = fmax3f(g[0], g[1], fmaxf(g[2], g[3]));
    if (!__any_sync(0xffffffffu, active && mx >= lo)) return;
    unsigned mask = hit_mask(v, g, active, lo);
    while (mask) {
        const int c = __ffs(mask) - 1;
        mask &= mask - 1u;
        if (pos0 + c >= mlim) continue;
        const float x = select32(v, c);
        if (x > hi) {
            atomicAdd(&cnt_s[col0 + c], 1);
        } else {
            unsigned idx = atomicAdd(&st->band_count, 1u);
            if (idx < band_cap) band[idx] = make_int2(u_orig, pos0 + c);
            else st->band_overflow = 1u;
        }
    }
}

// Warm-start bound from COLS columns of one accumulator row held in TMEM: the maxima of
// the NG column groups of width COLS/NG, sorted by a bitonic network in registers; the k-th
// largest (k <= NG) minus E bounds tau_u from below, because k distinct items reach it.
// Columns at or beyond m count as -inf.  Returns -inf when fewer than k groups are valid.
template <int NG, int COLS, typename LoadChunk>
__device__ __forceinline__ float warm_bound(LoadChunk load, int pos0, int64_t m, int k, float E) {
    constexpr int GW = COLS / NG;  // group width
    float g[NG];
#pragma unroll
    for (int c0 = 0; c0 < COLS; c0 += 32) {
        float v[32];
        load(c0, v);
#pragma unroll
        for (int q = 0; q < 32 / GW; ++q) {
            float x = -INFINITY;
#pragma unroll
            for (int j = 0; j < GW; ++j)
                if (pos0 + c0 + q * GW + j < m) x = fmaxf(x, v[q * GW + j]);
            g[(c0 / GW) + q] = x;
        }
    }
#pragma unroll
    for (int size = 2; size <= NG; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
            for (int i = 0; i < NG; ++i) {
                const int j = i ^ stride;
                if (j > i) {
                    const float hi = fmaxf(g[i], g[j]), lo = fminf(g[i], g[j]);
                    const bool desc = (i & size) == 0;
                    g[i] = desc ? hi : lo;
                    g[j] = desc ? lo : hi;
                }
            }
        }
    }
    float kth = -INFINITY;
#pragma unroll
    for (int j = 0; j < NG; ++j)
        if (j == k - 1) kth = g[j];
    return (kth == -INFINITY) ? -INFINITY : __fsub_rd(kth, E);
}

}  // namespace rkm
