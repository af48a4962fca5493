// Internal launchers of the reverse k-MIPS kernels (host side, not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "common.cuh"

namespace rkm {

// Record the message returned by rkm_last_error() on this host thread; returns s.
int set_error(int s, const char* msg);

// Kernels launched by this library since load (each launcher calls note_launch()).
extern std::atomic<unsigned long long> g_launches;
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---- prep.cu (K1 prep, K4 bounds and the bucket sort) ------------------------------

// Per row: exponent e (max|x| <= 2^e), integer grid codes q = x * 2^(12-e) (int16,
// row stride dq), exact/upper-bound squared norm, ||x|| rounded up; st->off_grid is set
// when a row is not on the grid.
// Also ||x^|| and ||x^ - x|| (rounded up) of the operand x^ the product kernels see:
// OPERAND_F32: x itself; OPERAND_BF16: BF16 round-to-nearest of x; OPERAND_FP8_ROW: x scaled
// by 2^(8-e), rounded to FP8 e4m3 (nearest even) and scaled back (per-row scale).  Operands
// with a per-tile scale get their norms from launch_pack_fp8 instead.
enum OperandKind { OPERAND_F32 = 0, OPERAND_BF16 = 1, OPERAND_FP8_ROW = 2 };
void launch_prep_rows(const float* X, int64_t rows, int64_t ld, int d, int* ex, int16_t* q,
                      int dq, double* norm2, float* nrm_hi, float* nhat_hi, float* del_hi,
                      int operand, DevStatus* st, cudaStream_t s);

// FP8 e4m3 operand copy dst[r][c] (rows_pad x dp bytes) of X (row perm[r] if perm != null):
// row r holds e4m3(x * 2^(8 - e_r)) with e_r = tile_exp[r / tile] when tile_exp != null,
// else fp8_exp(row_exp[src]) (the row's own exponent).  Since max|x| <= 2^e, scaled values
// stay within +-256 (e4m3 saturates at 448) unless the exponent was clamped.  When
// nhat/del are non-null, also writes ||x^|| and ||x^ - x|| (rounded up) of the descaled
// operand at the source row.
void launch_pack_fp8(const float* X, int64_t rows, int64_t ld, int d, const int* perm, const int* row_exp,
                     const int* tile_exp, int tile, uint8_t* dst, int64_t rows_pad, int dp, float* nhat,
                     float* del, cudaStream_t s);

// Per tile of `tile` consecutive sorted rows: fp8_exp of the largest row exponent ex[perm[i]]
// (0 for an empty tile).
void launch_tile_exp(const int* ex, const int* perm, int64_t count, int tile, int64_t tiles, int* texp,
                     cudaStream_t s);

// Zero-padded operand copy dst[r][c] (rows_pad x dp) of X (row perm[r] if perm != null).
void launch_pack_f32(const float* X, int64_t rows, int64_t ld, int d, const int* perm,
                     float* dst, int64_t rows_pad, int dp, cudaStream_t s);
void launch_pack_bf16(const float* X, int64_t rows, int64_t ld, int d, const int* perm,
                      __nv_bfloat16* dst, int64_t rows_pad, int dp, cudaStream_t s);

// Counting sort of `count` float keys by their 16-bit bucket (ascending, or descending
// when `descending`).  Writes perm[pos] = source index and, if cum != null, the
// inclusive prefix count of each bucket (in sort order).  hist: HIST_WORDS uints scratch.
void launch_bucket_sort(const float* keys, int64_t count, bool descending, unsigned* hist,
                        unsigned* offs, int* perm, unsigned* cum, cudaStream_t s);

// gathered[i] = src[perm[i]] for float / double / int arrays.
void launch_gather_f32(const float* src, const int* perm, int64_t count, float* dst, cudaStream_t s);
void launch_gather_f64(const double* src, const int* perm, int64_t count, double* dst, cudaStream_t s);
void launch_gather_i32(const int* src, const int* perm, int64_t count, int* dst, cudaStream_t s);

// Per tile t of sorted positions [t*tile, min(count,(t+1)*tile)): the maxima of nrm, nhat and
// del over the rows perm[pos] (0 for an empty tile).
void launch_tile_max(const float* nrm, const float* nhat, const float* del, const int* perm, int64_t count,
                     int tile, int64_t tiles, float* tmax, float* thmax, float* tdel, cudaStream_t s);

// K4: r_u = tau_u / ||u|| rounded down (-inf when tau_u <= 0).
void launch_user_ratio(const double* tau, const double* norm2, int64_t n, float* r, cudaStream_t s);

// Ordering key of the threshold pass: r[u] = L_u / ||u|| for a lower bound L_u of tau_u given
// as float_key (key 0 or L_u <= 0 gives -inf).  Only an order, not a bound.
void launch_seed_ratio(const unsigned* lkey, const float* nrm, int64_t n, float* r, cudaStream_t s);

// K4: per-user records of the counting pass, in ratio order (perm: ratio order -> user).
void launch_user_meta(const double* tau, const float* nrm, const float* nhat, const float* del, const int* ex,
                      const int* perm, int64_t n, UserMeta* meta, cudaStream_t s);

// K4: uscore[i] = number of users whose ratio bucket <= bucket(||p_i||) (ucum lookup).
void launch_item_uscore(const float* nrm_hi, int64_t m, const unsigned* ucum, int* uscore,
                        cudaStream_t s);

// ---- threshold pass (K2) ------------------------------------------------------------

struct ThresholdArgs {
    const void* A;        // users, packed [n_pad][dp] (fp32 or bf16), original order
    const void* B;        // items, packed [m_pad][dp], sorted by norm (descending)
    int64_t n, m;
    int dp, k, cap;
    const float* unrm;    // [n] ||u|| rounded up
    const float* unhat;   // [n] ||u^|| rounded up (u^ = operand seen by the product)
    const float* udel;    // [n] ||u^ - u|| rounded up
    const float* tmax;    // [item tiles] max ||p|| of the tile, rounded up
    const float* thmax;   // [item tiles] max ||p^||
    const float* tdel;    // [item tiles] max ||p^ - p||
    float cacc, eabs;     // accumulation coefficient and absolute (underflow) term of the bound
    const int* uexp;      // [n] FP8: user row exponents (operand scale 2^(8-e)); else unused
    const int* texp;      // [item tiles] FP8: item tile exponents; else unused
    Cand* cand;           // [n][nseg][cap]
    int* cand_cnt;        // [n][nseg]
    unsigned* lfin_key;   // [n] float_key of the final lower threshold L_u (atomic max; 0 = none)
    int nseg;             // candidate segments per user (epilogue groups of the kernel)
    DevStatus* st;
    int num_sms;
    // Tensor-core kernel, optional: the users packed in A are in this order (packed row ->
    // original user; the per-user norms and exponents above are by original user, the outputs
    // cand / cand_cnt / lfin_key by packed row), and a lower bound of tau_u per original
    // user (float_key, 0 = none) that seeds the selector.
    const int* uperm;
    const unsigned* lfin_seed;
};
void launch_threshold_simt(const ThresholdArgs& a, cudaStream_t s);

// One problem of the tensor-core threshold pass: its TMA descriptors (users, items), its
// arguments, and the index of its first work unit (user tile) in the launch.
struct __align__(64) TcInstance {
    CUtensorMap tmA;
    CUtensorMap tmB;
    ThresholdArgs a;
    long long unit_begin;
};
// Tensor-core threshold pass over `count` instances in one persistent launch.  inst: device
// array; total_units = sum of the instances' user tiles; kheap = largest k; max_dp = largest
// padded depth (elements).  fp8: operands are e4m3 (128 per K-block) with power-of-two
// scales, else BF16 (64 per K-block); every instance of a launch has the same kind.
// Epilogue warpgroups (= candidate segments per user) of the tensor-core threshold launch for
// the largest k, padded depth and operand kind of its instances.  want = 2 or 4 asks for that
// many, 0 chooses; 4 only when four per-user heaps of kheap bounds (kheap <= 32) still leave
// the shared-memory ring enough slots, else 2.
int threshold_groups(int kheap, int max_dp, bool fp8, int want);
// Epilogue warpgroups of the tensor-core counting kernel for padded depth dp (want as above).
int count_groups(int dp, bool fp8, int want);
// ng: epilogue warpgroups, as threshold_groups returned for these instances.
void launch_threshold_tc(const TcInstance* inst, int count, long long total_units, int kheap, int max_dp,
                         bool fp8, int ng, int num_sms, cudaStream_t s);

// Approximate products of the tensor-core paths with their guard band, for validating the
// error bound: v[u * ldo + perm[pos]] = the product the threshold and counting kernels see
// for user u and the item at sorted position pos (FP8: descaled), E[...] = its bound.
struct ProductsArgs {
    int64_t n, m, ldo;
    int dp;
    const int* perm;                      // sorted pos -> original item id
    const float *unrm, *unhat, *udel;     // [n] user norms (as ThresholdArgs)
    const int* uexp;                      // [n] FP8 user row exponents
    const float *thmax, *tdel;            // [item tiles] item norm maxima
    const int* texp;                      // [item tiles] FP8 tile exponents
    float cacc, eabs;
    float* v;                             // [n][ldo]
    float* E;                             // [n][ldo]
    DevStatus* st;
};
void launch_products_tc(const ProductsArgs& a, const void* tmapA, const void* tmapB, bool fp8, cudaStream_t s);

// A bounded mbarrier wait (the product kernels' own) on a phase nothing completes, with a
// limit of `limit` SM clocks: sets st->timeout and returns.
void launch_wait_timeout(long long limit, DevStatus* st, cudaStream_t s);

// ---- exact rescoring (K3, K6, K8) ---------------------------------------------------

struct ExactData {
    // user side (original order)
    const float* U; int64_t ldu;
    const int* eu; const int16_t* qu;
    // item side (original order)
    const float* P; int64_t ldp;
    const int* ep; const int16_t* qp;
    int d, dq;
    const unsigned* off_grid;  // device flag: zero = every row on the grid, use the integer path
    // Debug builds check gathered indices against these (0 = unchecked).
    int64_t n_users = 0, m_items = 0;
};

// K3: exact tau_u, t_u and (optionally) S_k(u) from the candidate lists.  With uperm, the
// lists are by threshold-pass row and uperm[row] is the original user (rows, outputs).
void launch_exact_tau(const ExactData& x, const Cand* cand, const int* cand_cnt, const unsigned* lfin_key,
                      int cap, int nseg, const int* item_perm, int64_t n, int k,
                      unsigned long long* keys, int* kid, double* tau, int* tid, int* topk,
                      DevStatus* st, cudaStream_t s, const int* uperm = nullptr);

// K6: rescore queued band pairs (orig user, sorted item pos) and add members to counts.
void launch_band_rescore(const ExactData& x, const int2* band, unsigned band_cap,
                         const int* item_perm, int64_t m_ids, const double* tau, const int* tid,
                         bool new_items, int* counts, DevStatus* st, cudaStream_t s);

// K8: scores by histogram of S_k(u) (the first Section 2.2 baseline).
void launch_histogram(const int* topk, int64_t nk, int* scores, cudaStream_t s);
// Same over the first k entries of each row of lists [n][kmax] (ids checked against [0, m)).
void launch_histogram_prefix(const int* lists, int64_t n, int kmax, int k, int64_t m, int* scores, DevStatus* st,
                             cudaStream_t s);

// ---- counting pass (K5) -------------------------------------------------------------

struct CountArgs {
    const void* A;          // users packed in ratio order [n_pad][dp]
    const void* B;          // items packed sorted [m_pad][dp]
    int64_t n, m;
    int dp;
    const UserMeta* meta;   // [n] per-user record, ratio order
    const int* item_id;     // sorted pos -> original item id (null for new items)
    bool new_items;         // strict rule u.p > tau_u (new ids beat no tie)
    const float* tmax;      // per item tile: max ||p||
    const float* thmax;     // per item tile: max ||p^||
    const float* tdel;      // per item tile: max ||p^ - p||
    const int* texp;        // per item tile: FP8 tile exponent (unused for BF16 / FP32)
    const int* nprefix;     // per item tile: users needed (ratio-order prefix length)
    const unsigned* unit_off;  // [tiles+1] first unit of each item tile (exclusive scan)
    int t_begin;            // first item tile of the stage
    int group;              // user tiles per work unit
    int groups;             // tensor-core kernel: epilogue warpgroups (2 or 4)
    float cacc, eabs;
    int* counts;            // [m] by sorted position
    int2* band; unsigned band_cap;
    DevStatus* st;
    int num_sms;
};
// Work list of a counting stage over item tiles [t_begin, t_end or *t_end_dev).
void launch_build_units(const float* tmax, const unsigned* ucum, int t_begin, int t_end,
                        const int* t_end_dev, int tile_users, int group, int* nprefix,
                        unsigned* unit_off, DevStatus* st, cudaStream_t s);
void launch_count_simt(const CountArgs& a, cudaStream_t s);

// One problem of a tensor-core counting launch: its TMA maps (users in ratio order, items
// sorted), its arguments (its own status word, counts, band queue, unit list), and its first
// work unit in the launch (written by launch_count_prefix).
struct __align__(64) CountInstance {
    CUtensorMap tmA;
    CUtensorMap tmB;
    CountArgs a;
    long long unit_begin;
};
// inst: device array; every instance's unit list must have been built (st->units_total).
// Writes inst[i].unit_begin and *total (device word) on the stream.
void launch_count_prefix(CountInstance* inst, int count, unsigned long long* total, cudaStream_t s);
// Tensor-core counting of one problem (arguments and TMA maps passed by value; its unit list
// built on the stream), with a.groups epilogue warpgroups.
void launch_count_tc(const CountArgs& a, const void* tmapA, const void* tmapB, bool fp8, cudaStream_t s);
// Tensor-core counting over the units of all instances (persistent, num_sms CTAs); total:
// device word from launch_count_prefix; max_dp: largest padded depth.
void launch_count_tc_multi(const CountInstance* inst, int count, const unsigned long long* total, int max_dp,
                           bool fp8, int num_sms, cudaStream_t s);

// ---- batches: the steps after the threshold launch, one launch over all problems ----

// Everything the multi-problem launches of a batch need about one problem.
struct BatchJob {
    // K3: exact thresholds from the candidate lists of the persistent threshold launch
    ExactData x;                  // rows and grid codes of users and items (original order)
    const Cand* cand;
    const int* cand_cnt;
    const unsigned* lfin;
    int cap, nseg;
    const int* item_perm;         // sorted pos -> item id
    int64_t n, m;
    int k, N;
    unsigned long long* keys;
    int* kid;
    double* tau;
    int* tid;
    int64_t user_begin;           // first user of this problem in the launch's numbering
    // K4-K6: counting stages over item tiles [0, t0) and [t0, cut)
    const float* tmax;
    const unsigned* ucum;
    int tiles, t0, tile_items, group;
    int* nprefix;
    unsigned* unit_off;
    int* counts;                  // by sorted position
    int2* band;
    unsigned band_cap;
    // K7
    int* top_ids_c0;
    int* top_sc_c0;
    int* ids;
    int* top_scores;
    DevStatus* st;
};
// jobs: device array of `count` problems, user_begin = exclusive prefix of n (total_users).
void launch_exact_tau_multi(const BatchJob* jobs, int count, int64_t total_users, cudaStream_t s);
// Zero every problem's counts and band counters (max_m: largest m).
void launch_batch_reset(const BatchJob* jobs, int count, int64_t max_m, cudaStream_t s);
// Unit lists of counting stage 1 (tiles [0, t0)) or 2 (tiles [t0, st->t_end)) of every problem.
void launch_build_units_multi(const BatchJob* jobs, int count, int stage, cudaStream_t s);
// Exact rescoring of every problem's new band pairs, then marks them done.
void launch_band_multi(const BatchJob* jobs, int count, cudaStream_t s);
// Top-N of every problem: stage 1 over the first-stage items into top_ids_c0/top_sc_c0,
// stage 2 over the counted items into ids/top_scores.
void launch_topn_multi(const BatchJob* jobs, int count, int stage, cudaStream_t s);
// Filter cut of every problem from its stage-1 top-N.
void launch_filter_cut_multi(const BatchJob* jobs, int count, cudaStream_t s);

// ---- top-N (K7) ---------------------------------------------------------------------

// Top N of key = (count << 32) | (0xFFFFFFFF - id) over positions [0, m_lim) where
// m_lim = *m_lim_dev if non-null else m.  ids/scores in order.
void launch_topn(const int* counts, const int* item_id, int64_t m, const int* m_lim_dev, int N,
                 int* ids, int* scores, DevStatus* st, cudaStream_t s);

// Filter cut: with LB = N-th score among the first c0 positions (from ids/scores of a
// top-N over them), set st->t_end to the first item tile whose uscore bound is < LB.
void launch_filter_cut(const int* top_scores_c0, int N, const float* tmax, const unsigned* ucum,
                       int64_t tiles, int t_begin, int tile_items, int64_t m, DevStatus* st,
                       cudaStream_t s);

}  // namespace rkm
