// Exact rescoring: K3 (exact tau_u, t_u and S_k(u) from the candidate lists, Definition 1),
// K6 (exact membership of the counting pass's band pairs, Eq. 1) and K8 (scores as the
// histogram of S_k(u), the first Section 2.2 baseline).
//
// Exact inner products.  When every row is on the grid 2^e * q / 4096, u.p equals
// 2^(e_u + e_p - 24) * sum_j q_u[j] q_p[j]; the integer sum is formed in 32-bit chunks of
// 64 terms (each |term| <= 2^24, so a chunk stays below 2^30) added in 64 bits, then
// scaled exactly into FP64.  Otherwise u.p is the left-to-right FP64 sum of the exact
// FP64 products of the FP32 inputs.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace rkm {

namespace {

__device__ __forceinline__ double exact_dot(const ExactData& x, bool grid, int64_t u, int64_t i) {
    double s;
    if (grid) {
        const int4* a = reinterpret_cast<const int4*>(x.qu + u * x.dq);
        const int4* b = reinterpret_cast<const int4*>(x.qp + i * x.dq);
        long long acc = 0;
        const int vecs = x.dq >> 3;  // 8 int16 per int4
        for (int v0 = 0; v0 < vecs; v0 += 8) {
            int part = 0;
            const int v1 = (v0 + 8 < vecs) ? v0 + 8 : vecs;  // 8 vectors = 64 terms
            for (int v = v0; v < v1; ++v) {
                const int4 av = a[v], bv = b[v];
                const int aw[4] = {av.x, av.y, av.z, av.w};
                const int bw[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int alo = (int)(int16_t)(aw[h] & 0xffff), ahi = aw[h] >> 16;
                    const int blo = (int)(int16_t)(bw[h] & 0xffff), bhi = bw[h] >> 16;
                    part += alo * blo + ahi * bhi;
                }
            }
            acc += part;
        }
        s = ldexp((double)acc, x.eu[u] + x.ep[i] - 24);
    } else {
        const float* a = x.U + u * x.ldu;
        const float* b = x.P + i * x.ldp;
        s = 0.0;
        for (int j = 0; j < x.d; ++j) s = fma((double)a[j], (double)b[j], s);
    }
    return s + 0.0;  // -0.0 -> +0.0
}

__device__ __forceinline__ double key_to_double(unsigned long long k) {
    unsigned long long b = (k & 0x8000000000000000ull) ? (k ^ 0x8000000000000000ull) : ~k;
    return __longlong_as_double((long long)b);
}

// One warp per user.
__device__ __forceinline__ float key_to_float(unsigned k) {
    if (k == 0u) return -INFINITY;
    const unsigned b = (k & 0x80000000u) ? (k ^ 0x80000000u) : ~k;
    return __uint_as_float(b);
}

// Number of keys[0 .. cnt) >= K, summed over the warp.
__device__ __forceinline__ int count_at_least(const unsigned long long* keys, int cnt, unsigned long long K, int lane) {
    int c = 0;
    for (int j = lane; j < cnt; j += 32) c += keys[j] >= K;
    return warp_sum(c);
}

// Moves the candidates whose exact key is at least the k-th largest key K to the front of
// keys/ids and returns how many there are (k, plus any ties with K).  K is built one bit at a
// time from the top: a bit is kept when at least k keys reach the prefix with it set.  The
// full ranking then runs over about k candidates instead of all of them (a wide guard band,
// as on the FP8 path, keeps hundreds per user).  All 32 lanes call it.
__device__ __forceinline__ int keep_top_keys(unsigned long long* keys, int* ids, int cnt, int k, int lane) {
    unsigned long long K = 0ull;
    for (int b = 63; b >= 0; --b) {
        const unsigned long long t = K | (1ull << b);
        if (count_at_least(keys, cnt, t, lane) >= k) K = t;
    }
    const unsigned lt_mask = (1u << lane) - 1u;
    int out = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int j = base + lane;
        const unsigned long long key = j < cnt ? keys[j] : 0ull;
        const int id = j < cnt ? ids[j] : 0;
        const bool take = j < cnt && key >= K;
        const unsigned mask = __ballot_sync(0xffffffffu, take);
        // Every lane has read its entry (the ballot orders it before the writes), and writes
        // go to slots at or before the ones read in this round.
        if (take) {
            const int slot = out + __popc(mask & lt_mask);
            keys[slot] = key;
            ids[slot] = id;
        }
        out += __popc(mask);
        __syncwarp();
    }
    return out;
}

// Exact tau_u, t_u (and S_k(u) when topk != null) of user u from its candidate lists; one
// warp per user, all 32 lanes call it.  Returns the number of candidates kept.
__device__ __forceinline__ int exact_user(const ExactData& x, bool grid, const Cand* __restrict__ cand,
                                          const int* __restrict__ cand_cnt, const unsigned* __restrict__ lfin_key,
                                          int cap, int nseg, const int* __restrict__ item_perm, int k,
                                          unsigned long long* __restrict__ keys, int* __restrict__ kid,
                                          double* __restrict__ tau, int* __restrict__ tid, int* __restrict__ topk,
                                          DevStatus* st, int64_t u, int lane, const int* __restrict__ uperm) {
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t uo = uperm ? (int64_t)uperm[u] : u;  // row of the lists -> original user
    if (!RKM_DCHECK(uo >= 0 && (x.n_users == 0 || uo < x.n_users), st)) return k;
    const float L = key_to_float(lfin_key[u]);
    unsigned long long* kk = keys + u * (int64_t)nseg * cap;
    int* ki = kid + u * (int64_t)nseg * cap;
    int kept = 0;
    for (int h = 0; h < nseg; ++h) {
        const int cnt = cand_cnt[u * nseg + h];
        const Cand* c = cand + (u * nseg + h) * (int64_t)cap;
        for (int base = 0; base < cnt; base += 32) {
            const int j = base + lane;
            bool keep = false;
            Cand cj;
            cj.ub = 0.f;
            cj.pos = 0;
            if (j < cnt) {
                cj = c[j];
                keep = cj.ub >= L && RKM_DCHECK(cj.pos >= 0 && (x.m_items == 0 || cj.pos < x.m_items), st);
            }
            const unsigned mask = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int slot = kept + __popc(mask & lt_mask);
                const int io = item_perm[cj.pos];
                RKM_DCHECK(io >= 0 && (x.m_items == 0 || io < x.m_items), st);
                kk[slot] = double_key(exact_dot(x, grid, uo, io));
                ki[slot] = io;
            }
            kept += __popc(mask);
        }
    }
    __syncwarp();
    if (kept < k) {
        if (lane == 0) st->internal_error = 1u;
        return kept;
    }
    const int kept_all = kept;
    if (kept > 2 * 32) kept = keep_top_keys(kk, ki, kept, k, lane);
    // Rank of each kept candidate under (score desc, id asc) = the number of candidates
    // before it.  Candidates are visited 32 at a time and broadcast by shuffles.
    for (int j0 = 0; j0 < kept; j0 += 32) {
        const int j = j0 + lane;
        const bool mine = j < kept;
        const unsigned long long key = mine ? kk[j] : 0ull;
        const int id = mine ? ki[j] : 0x7fffffff;
        int rank = 0;
        for (int r0 = 0; r0 < kept; r0 += 32) {
            const int rn = (kept - r0 < 32) ? kept - r0 : 32;
            const unsigned long long k2l = (r0 + lane < kept) ? kk[r0 + lane] : 0ull;
            const int i2l = (r0 + lane < kept) ? ki[r0 + lane] : 0x7fffffff;
            for (int r = 0; r < rn; ++r) {
                const unsigned long long k2 = __shfl_sync(0xffffffffu, k2l, r);
                const int i2 = __shfl_sync(0xffffffffu, i2l, r);
                rank += (k2 > key) || (k2 == key && i2 < id);
            }
        }
        if (mine && rank < k) {
            if (topk) topk[uo * (int64_t)k + rank] = id;
            if (rank == k - 1) {
                tau[uo] = key_to_double(key);
                tid[uo] = id;
            }
        }
    }
    __syncwarp();
    return kept_all;
}

// Latency-bound (dependent loads of each user's candidates, ids and codes): six blocks per
// SM (40 registers, a few spilled) hide more of it than the four that 63 registers allow.
__global__ void __launch_bounds__(256, 6) k_exact_tau(ExactData x, const Cand* __restrict__ cand, const int* __restrict__ cand_cnt,
                            const unsigned* __restrict__ lfin_key, int cap, int nseg,
                            const int* __restrict__ item_perm,
                            int64_t n, int k, unsigned long long* __restrict__ keys,
                            int* __restrict__ kid, double* __restrict__ tau, int* __restrict__ tid,
                            int* __restrict__ topk, DevStatus* st, const int* __restrict__ uperm) {
    const int lane = threadIdx.x & 31;
    const bool grid = *x.off_grid == 0u;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long kept_total = 0;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps)
        kept_total += (unsigned long long)exact_user(x, grid, cand, cand_cnt, lfin_key, cap, nseg, item_perm, k, keys,
                                                     kid, tau, tid, topk, st, u, lane, uperm);
    if (lane == 0 && kept_total) atomicAdd(&st->cand_total, kept_total);
}

// The same over the users of many problems: global user g belongs to the last job whose
// user_begin is <= g.
__global__ void __launch_bounds__(256, 6) k_exact_tau_multi(const BatchJob* __restrict__ jobs, int count,
                                                            int64_t total_users) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long kept_total = 0;
    int cur = -1;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < total_users; g += warps) {
        int lo = 0, hi = count;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (jobs[mid].user_begin <= g) lo = mid; else hi = mid;
        }
        if (lo != cur) {
            if (lane == 0 && cur >= 0 && kept_total) atomicAdd(&jobs[cur].st->cand_total, kept_total);
            kept_total = 0;
            cur = lo;
        }
        const BatchJob& J = jobs[lo];
        const bool grid = *J.x.off_grid == 0u;
        kept_total += (unsigned long long)exact_user(J.x, grid, J.cand, J.cand_cnt, J.lfin, J.cap, J.nseg,
                                                     J.item_perm, J.k, J.keys, J.kid, J.tau, J.tid, nullptr, J.st,
                                                     g - J.user_begin, lane, nullptr);
    }
    if (lane == 0 && cur >= 0 && kept_total) atomicAdd(&jobs[cur].st->cand_total, kept_total);
}

// Exact membership of band pairs [st->band_done, min(st->band_count, cap)) taken with
// stride `stride` from `first`; members add one to their item's count.
__device__ __forceinline__ void band_pairs(const ExactData& x, const int2* __restrict__ band, unsigned band_cap,
                                           const int* __restrict__ item_perm, const double* __restrict__ tau,
                                           const int* __restrict__ tid, bool new_items, int* __restrict__ counts,
                                           const DevStatus* st, unsigned first, unsigned stride) {
    const bool grid = *x.off_grid == 0u;
    const unsigned begin = st->band_done;
    unsigned end = st->band_count;
    if (end > band_cap) end = band_cap;
    for (unsigned e = begin + first; e < end; e += stride) {
        const int2 b = band[e];
        if (!RKM_DCHECK(b.x >= 0 && (x.n_users == 0 || b.x < x.n_users) && b.y >= 0 &&
                            (x.m_items == 0 || b.y < x.m_items),
                        const_cast<DevStatus*>(st)))
            continue;
        const int64_t u = b.x;
        const int io = item_perm[b.y];
        const double s = exact_dot(x, grid, u, io);
        const double t = tau[u];
        const bool member = (s > t) || (!new_items && s == t && io <= tid[u]);
        if (member) atomicAdd(&counts[b.y], 1);
    }
}

__global__ void k_band_rescore(ExactData x, const int2* __restrict__ band, unsigned band_cap,
                               const int* __restrict__ item_perm, const double* __restrict__ tau,
                               const int* __restrict__ tid, bool new_items, int* __restrict__ counts,
                               DevStatus* st) {
    band_pairs(x, band, band_cap, item_perm, tau, tid, new_items, counts, st, blockIdx.x * blockDim.x + threadIdx.x,
               gridDim.x * blockDim.x);
}

__global__ void k_band_mark(DevStatus* st, unsigned band_cap) {
    unsigned end = st->band_count;
    st->band_done = end > band_cap ? band_cap : end;
}

// Band rescoring of job blockIdx.y (catalogue items: ties at tau_u are decided by t_u).
__global__ void k_band_rescore_multi(const BatchJob* __restrict__ jobs) {
    const BatchJob& J = jobs[blockIdx.y];
    band_pairs(J.x, J.band, J.band_cap, J.item_perm, J.tau, J.tid, false, J.counts, J.st,
               blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void k_band_mark_multi(const BatchJob* __restrict__ jobs, int count) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    DevStatus* st = jobs[j].st;
    const unsigned end = st->band_count, cap = jobs[j].band_cap;
    st->band_done = end > cap ? cap : end;
}

// Zero the counts of job blockIdx.y and its band counters.
__global__ void k_batch_reset(const BatchJob* __restrict__ jobs) {
    const BatchJob& J = jobs[blockIdx.y];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < J.m; i += (int64_t)gridDim.x * blockDim.x)
        J.counts[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        J.st->band_count = 0u;
        J.st->band_done = 0u;
    }
}

__global__ void k_histogram(const int* __restrict__ topk, int64_t nk, int* __restrict__ scores) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nk; j += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&scores[topk[j]], 1);
}

// Histogram of the first k ids of every row of lists [n][kmax] (S_k(u) is the first k
// entries of S_kmax(u) in order).  An id outside [0, m) flags an internal error.
__global__ void k_histogram_prefix(const int* __restrict__ lists, int64_t n, int kmax, int k, int64_t m,
                                   int* __restrict__ scores, DevStatus* st) {
    const int64_t total = n * k;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = j / k;
        const int id = lists[u * kmax + (j - u * k)];
        if (id >= 0 && id < m) atomicAdd(&scores[id], 1);
        else st->internal_error = 1u;
    }
}

}  // namespace

void launch_histogram_prefix(const int* lists, int64_t n, int kmax, int k, int64_t m, int* scores, DevStatus* st,
                             cudaStream_t s) {
    if (n <= 0 || k <= 0) return;
    int64_t blocks = (n * k + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    note_launch();
    k_histogram_prefix<<<(int)blocks, 256, 0, s>>>(lists, n, kmax, k, m, scores, st);
}

void launch_exact_tau(const ExactData& x, const Cand* cand, const int* cand_cnt, const unsigned* lfin_key,
                      int cap, int nseg, const int* item_perm, int64_t n, int k, unsigned long long* keys, int* kid,
                      double* tau, int* tid, int* topk, DevStatus* st, cudaStream_t s, const int* uperm) {
    if (n <= 0) return;
    int64_t blocks = (n * 32 + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    note_launch();
    k_exact_tau<<<(int)blocks, 256, 0, s>>>(x, cand, cand_cnt, lfin_key, cap, nseg, item_perm, n, k, keys, kid, tau,
                                            tid, topk, st, uperm);
}

void launch_band_rescore(const ExactData& x, const int2* band, unsigned band_cap, const int* item_perm,
                         int64_t m_ids, const double* tau, const int* tid, bool new_items, int* counts,
                         DevStatus* st, cudaStream_t s) {
    (void)m_ids;
    note_launch();
    k_band_rescore<<<1184, 256, 0, s>>>(x, band, band_cap, item_perm, tau, tid, new_items, counts, st);
    note_launch();
    k_band_mark<<<1, 1, 0, s>>>(st, band_cap);
}

void launch_exact_tau_multi(const BatchJob* jobs, int count, int64_t total_users, cudaStream_t s) {
    if (total_users <= 0) return;
    int64_t blocks = (total_users * 32 + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    note_launch();
    k_exact_tau_multi<<<(int)blocks, 256, 0, s>>>(jobs, count, total_users);
}

void launch_band_multi(const BatchJob* jobs, int count, cudaStream_t s) {
    note_launch();
    k_band_rescore_multi<<<dim3(64, (unsigned)count), 256, 0, s>>>(jobs);
    note_launch();
    k_band_mark_multi<<<(count + 127) / 128, 128, 0, s>>>(jobs, count);
}

void launch_batch_reset(const BatchJob* jobs, int count, int64_t max_m, cudaStream_t s) {
    int64_t bx = (max_m + 255) / 256;
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    note_launch();
    k_batch_reset<<<dim3((unsigned)bx, (unsigned)count), 256, 0, s>>>(jobs);
}

void launch_histogram(const int* topk, int64_t nk, int* scores, cudaStream_t s) {
    if (nk <= 0) return;
    int64_t blocks = (nk + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    note_launch();
    k_histogram<<<(int)blocks, 256, 0, s>>>(topk, nk, scores);
}

}  // namespace rkm
