// C ABI of librkm: argument checks, workspace, and the order of the kernels of each call.
//
// rkm_thresholds:  K1 prep (users, items) -> item bucket sort by norm -> operand packs
//                  -> K2 product + per-user selector -> K3 exact tau_u, t_u, S_k(u).
// rkm_scores:      K1 -> K4 ratios tau_u/||u|| and their bucket sort -> K5 product +
//                  classify against (tau_u, t_u) -> K6 exact band rescoring.
// rkm_topn:        thresholds, then K4/K5/K6 over a first stage of items, K7 on it, the
//                  filter cut (Algorithm 2's stop rule on Eq. 2 bounds), K5/K6 over the
//                  items left before the cut, K7 over every counted item.
// Serving:         resident users + K4 once; per query batch K1 -> K5 -> K6.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <atomic>

#include "../../include/rkm.h"
#include "common.cuh"
#include "kernels.h"
#include "tmap.h"

using rkm::TmapPair;
using rkm::make_tmaps;
using rkm::rkm_tc_available;

using namespace rkm;

std::atomic<unsigned long long> rkm::g_launches{0};

namespace {

thread_local std::string g_err;

rkm_status fail(rkm_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
rkm_status fail(rkm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

}  // namespace

int rkm::set_error(int s, const char* msg) {
    g_err = msg;
    return s;
}

namespace {

#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(RKM_ECUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),    \
                        __FILE__, __LINE__);                                                  \
    } while (0)

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

int64_t round_up(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

}  // namespace

struct rkm_ctx {
    int device = 0;
    int num_sms = 0;
    rkm_opts opts{};
    rkm_stats stats{};
    DevStatus* st = nullptr;     // device status word
    DevStatus* st_host = nullptr;  // pinned mirror
    // users (original order)
    Buf u_e, u_q, u_n2, u_nrm, u_nhat, u_del, u_pack;
    // items (original order; sorted copies)
    Buf p_e, p_q, p_n2, p_nrm, p_nhat, p_del, p_perm, p_pack, tmax, thmax, tdel;
    // bucket sort scratch
    Buf hist, offs;
    // threshold pass
    Buf cand, cand_cnt, lfin, keys, kid;
    // counting pass
    Buf r_u, uperm, ucum, us_pack, us_meta, nprefix, unit_off, band, cnt_s, top_ids, top_sc, tau_tmp,
        tid_tmp;
    // serving (resident users)
    bool resident = false;
    int64_t res_n = 0;
    int res_d = 0;
    unsigned res_grid = 0;
    Buf res_U, res_e, res_q, res_tau, res_tid, res_uperm, res_ucum, res_pack, res_meta;
    // query scratch
    Buf q_e, q_q, q_n2, q_nrm, q_nhat, q_del, q_perm, q_pack, q_tmax, q_thmax, q_tdel, q_cnt;
    // host staging for rkm_topn_host
    Buf h_U, h_P, h_ids, h_sc;
    int cand_cap = 0;
    int cand_k = 0;
    int64_t band_cap = 0;
    // phase timing (opts.profile)
    struct Pending {
        int phase;
        cudaEvent_t e0, e1;
    };
    std::vector<cudaEvent_t> ev_pool;
    std::vector<Pending> pending;
    unsigned long long launches_at_start = 0;

    cudaEvent_t take_event() {
        if (ev_pool.empty()) {
            cudaEvent_t e = nullptr;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = ev_pool.back();
        ev_pool.pop_back();
        return e;
    }

    template <typename T>
    rkm_status ensure(Buf& b, int64_t count, T** out) {
        size_t need = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
        need = (need + 255) & ~(size_t)255;
        if (b.bytes < need) {
            if (b.p) cudaFree(b.p);
            b.p = nullptr;
            b.bytes = 0;
            size_t alloc = need + need / 8;
            cudaError_t e = cudaMalloc(&b.p, alloc);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(RKM_ENOMEM, "cudaMalloc(%zu) failed: %s", alloc, cudaGetErrorString(e));
            }
            b.bytes = alloc;
        }
        *out = static_cast<T*>(b.p);
        return RKM_OK;
    }

    void free_all() {
        Buf* all[] = {&u_e, &u_q, &u_n2, &u_nrm, &u_nhat, &u_del, &u_pack, &p_e, &p_q, &p_n2, &p_nrm,
                      &p_nhat, &p_del, &p_perm, &p_pack, &tmax, &thmax, &tdel, &hist, &offs, &cand,
                      &cand_cnt, &lfin, &keys, &kid, &r_u, &uperm, &ucum, &us_pack, &us_meta,
                      &nprefix, &unit_off, &band, &cnt_s, &top_ids, &top_sc,
                      &tau_tmp, &tid_tmp, &res_U, &res_e, &res_q, &res_tau, &res_tid, &res_uperm, &res_ucum,
                      &res_pack, &res_meta, &q_e, &q_q,
                      &q_n2, &q_nrm, &q_nhat, &q_del, &q_perm, &q_pack, &q_tmax, &q_thmax, &q_tdel, &q_cnt,
                      &h_U, &h_P, &h_ids, &h_sc};
        for (Buf* b : all) {
            if (b->p) cudaFree(b->p);
            b->p = nullptr;
            b->bytes = 0;
        }
        for (auto& p : pending) {
            ev_pool.push_back(p.e0);
            ev_pool.push_back(p.e1);
        }
        pending.clear();
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        ev_pool.clear();
    }
};

namespace {

// Records CUDA events around one phase on the call's stream when profiling is on.
struct Phase {
    rkm_ctx* c;
    cudaStream_t s;
    int ph;
    cudaEvent_t e0 = nullptr;
    Phase(rkm_ctx* c_, cudaStream_t s_, int ph_) : c(c_), s(s_), ph(ph_) {
        if (c->opts.profile) {
            e0 = c->take_event();
            cudaEventRecord(e0, s);
        }
    }
    ~Phase() {
        if (c->opts.profile) {
            cudaEvent_t e1 = c->take_event();
            cudaEventRecord(e1, s);
            c->pending.push_back({ph, e0, e1});
        }
    }
};

// After a stream synchronisation: fold the recorded phases into the stats.
void collect_phases(rkm_ctx* c) {
    for (auto& p : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) c->stats.phase_ms[p.phase] += ms;
        c->ev_pool.push_back(p.e0);
        c->ev_pool.push_back(p.e1);
    }
    c->pending.clear();
    c->stats.kernel_launches = g_launches.load() - c->launches_at_start;
}

}  // namespace

namespace {

#define TRY(expr)                          \
    do {                                   \
        rkm_status s_ = (expr);            \
        if (s_ != RKM_OK) return s_;       \
    } while (0)

// Operand layout of one precision path.
struct PathShape {
    bool tc;        // tensor-core kernels
    int item_tile;  // BI of the product kernels
    int dp;         // padded depth (elements)
    float cacc, eabs;
};

// Error bound of the approximate products (err_bound in common.cuh):
//   |v - u.p| <= ||u^ - u|| ||p^|| + ||u|| ||p^ - p|| + cacc ||u^|| ||p^|| + eabs,
// where u^, p^ are the operands the product kernel multiplies exactly (BF16 products are
// exact in FP32; FP32 operands are used as they are) and cacc bounds the accumulation.
// FP32 CUDA cores: sequential FMA, so the accumulation error is at most gamma_d sum|u^ p^|,
// gamma_d = d 2^-24 / (1 - d 2^-24) (Higham, "Accuracy and Stability of Numerical
// Algorithms", Section 3.1); cacc = 2 gamma_d.  Tensor cores: the order and rounding of the
// FP32 accumulation are not specified; cacc = d 2^-22, four times gamma_d (measured tensor-core
// accumulation truncates, Fasi, Higham, Mikaitis and Pranesh, PeerJ Comput. Sci. 2021, which
// needs at most twice gamma_d).  A further d 2^-50 covers the gap between the FP64 reference
// sum and the exact value for off-grid inputs; eabs covers FP32 underflow of products.
PathShape path_shape(rkm_precision prec, int d) {
    PathShape ps{};
    const double dd = (double)d;
    const double g32 = dd * 0x1p-24 / (1.0 - dd * 0x1p-24);
    if (prec == RKM_FP32) {
        ps.tc = false;
        ps.item_tile = BI_SIMT;
        ps.dp = (int)round_up(d, 32);
        ps.cacc = (float)((2.0 * g32 + dd * 0x1p-50) * (1.0 + 0x1p-20));
    } else {
        ps.tc = true;
        ps.item_tile = BI_TC;
        ps.dp = (int)round_up(d, 64);
        ps.cacc = (float)((dd * 0x1p-22 + dd * 0x1p-50) * (1.0 + 0x1p-20));
    }
    ps.cacc = nextafterf(ps.cacc, INFINITY);
    ps.eabs = (float)(dd * 0x1p-126);
    return ps;
}

rkm_status check_matrix(const float* X, int64_t rows, int64_t ld, int d, const char* name) {
    if (rows < 0) return fail(RKM_EINVAL, "%s: negative row count", name);
    if (rows > 0 && !X) return fail(RKM_EINVAL, "%s: null pointer", name);
    if (ld < d) return fail(RKM_EINVAL, "%s: ld (%lld) < d (%d)", name, (long long)ld, d);
    if (rows > (int64_t)INT32_MAX) return fail(RKM_EINVAL, "%s: more than 2^31-1 rows", name);
    return RKM_OK;
}

rkm_status check_common(rkm_ctx* c, int d) {
    if (!c) return fail(RKM_EINVAL, "null context");
    if (d < 1 || d > 256) return fail(RKM_EINVAL, "d must be in [1, 256] (got %d)", d);
    if (c->opts.precision == RKM_FP8) return fail(RKM_EINVAL, "FP8 precision is not built");
    if (c->opts.precision == RKM_BF16 && !rkm_tc_available())
        return fail(RKM_EINVAL, "BF16 tensor-core kernels are not built into this library");
    CUDA_TRY(cudaSetDevice(c->device));
    return RKM_OK;
}

rkm_status begin_call(rkm_ctx* c, cudaStream_t s) {
    CUDA_TRY(cudaMemsetAsync(c->st, 0, sizeof(DevStatus), s));
    const unsigned one = 1u;
    CUDA_TRY(cudaMemcpyAsync(&c->st->grid_u, &one, sizeof(unsigned), cudaMemcpyHostToDevice, s));
    return RKM_OK;
}

rkm_status read_status(rkm_ctx* c, cudaStream_t s) {
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    collect_phases(c);
    if (c->st_host->timeout) return fail(RKM_ETIMEOUT, "a bounded device wait gave up (kernel aborted)");
    return RKM_OK;
}

void reset_stats(rkm_ctx* c) {
    c->stats = rkm_stats{};
    c->launches_at_start = g_launches.load();
}

// Prepared side of a product: per-row codes and norms in original order.
struct RowPrep {
    int* e;
    int16_t* q;
    double* n2;
    float* nrm;   // ||x|| rounded up
    float* nhat;  // ||x^|| rounded up (x^ = operand of the product kernels)
    float* del;   // ||x^ - x|| rounded up
};

rkm_status prep_rows(rkm_ctx* c, const PathShape& ps, const float* X, int64_t rows, int64_t ld, int d, Buf& be,
                     Buf& bq, Buf& bn2, Buf& bnrm, Buf& bnhat, Buf& bdel, RowPrep* out, cudaStream_t s) {
    const int dq = (int)round_up(d, 8);
    TRY(c->ensure(be, rows, &out->e));
    TRY(c->ensure(bq, rows * dq, &out->q));
    TRY(c->ensure(bn2, rows, &out->n2));
    TRY(c->ensure(bnrm, rows, &out->nrm));
    TRY(c->ensure(bnhat, rows, &out->nhat));
    TRY(c->ensure(bdel, rows, &out->del));
    launch_prep_rows(X, rows, ld, d, out->e, out->q, dq, out->n2, out->nrm, out->nhat, out->del, ps.tc,
                     &c->st->grid_u, s);
    return RKM_OK;
}

rkm_status pack(rkm_ctx* c, const PathShape& ps, const float* X, int64_t rows, int64_t ld, int d,
                const int* perm, int64_t rows_pad, Buf& b, void** out, cudaStream_t s) {
    if (ps.tc) {
        __nv_bfloat16* p;
        TRY(c->ensure(b, rows_pad * ps.dp, &p));
        launch_pack_bf16(X, rows, ld, d, perm, p, rows_pad, ps.dp, s);
        *out = p;
    } else {
        float* p;
        TRY(c->ensure(b, rows_pad * ps.dp, &p));
        launch_pack_f32(X, rows, ld, d, perm, p, rows_pad, ps.dp, s);
        *out = p;
    }
    return RKM_OK;
}

// Items: prep, sort by norm (descending), packed sorted operand, tile maxima of the norms.
struct ItemSide {
    RowPrep rp;
    int* perm;       // sorted pos -> original id
    void* pack;      // [m_pad][dp]
    float* tmax;     // [tiles] max ||p||
    float* thmax;    // [tiles] max ||p^||
    float* tdel;     // [tiles] max ||p^ - p||
    int64_t m, m_pad, tiles;
};

struct ItemBufs {
    Buf &e, &q, &n2, &nrm, &nhat, &del, &perm, &pack, &tmax, &thmax, &tdel;
};

rkm_status prep_items(rkm_ctx* c, const PathShape& ps, const float* P, int64_t m, int64_t ldp, int d,
                      const ItemBufs& bb, ItemSide* it, cudaStream_t s) {
    it->m = m;
    it->m_pad = round_up(std::max<int64_t>(m, 1), BI_TC);
    it->tiles = (m + ps.item_tile - 1) / ps.item_tile;
    TRY(prep_rows(c, ps, P, m, ldp, d, bb.e, bb.q, bb.n2, bb.nrm, bb.nhat, bb.del, &it->rp, s));
    unsigned *hist, *offs;
    TRY(c->ensure(c->hist, NBUCKET, &hist));
    TRY(c->ensure(c->offs, NBUCKET, &offs));
    TRY(c->ensure(bb.perm, m, &it->perm));
    launch_bucket_sort(it->rp.nrm, m, true, hist, offs, it->perm, nullptr, s);
    TRY(pack(c, ps, P, m, ldp, d, it->perm, it->m_pad, bb.pack, &it->pack, s));
    const int64_t nt = std::max<int64_t>(it->tiles, 1);
    TRY(c->ensure(bb.tmax, nt, &it->tmax));
    TRY(c->ensure(bb.thmax, nt, &it->thmax));
    TRY(c->ensure(bb.tdel, nt, &it->tdel));
    launch_tile_max(it->rp.nrm, it->rp.nhat, it->rp.del, it->perm, m, ps.item_tile, it->tiles, it->tmax,
                    it->thmax, it->tdel, s);
    return RKM_OK;
}

ItemBufs catalogue_bufs(rkm_ctx* c) {
    return ItemBufs{c->p_e, c->p_q, c->p_n2, c->p_nrm, c->p_nhat, c->p_del, c->p_perm, c->p_pack, c->tmax,
                    c->thmax, c->tdel};
}

ItemBufs query_bufs(rkm_ctx* c) {
    return ItemBufs{c->q_e, c->q_q, c->q_n2, c->q_nrm, c->q_nhat, c->q_del, c->q_perm, c->q_pack, c->q_tmax,
                    c->q_thmax, c->q_tdel};
}

rkm_status thresholds_core(rkm_ctx* c, const PathShape& ps, const float* U, int64_t n, int64_t ldu,
                           const float* P, int64_t ldp, int d, int k, const RowPrep& up, const ItemSide& it,
                           double* tau, int* tid, int* topk, cudaStream_t s) {
    const int64_t n_pad = round_up(std::max<int64_t>(n, 1), BU);
    void* apack;
    {
        Phase ph(c, s, RKM_PHASE_PREP);
        TRY(pack(c, ps, U, n, ldu, d, nullptr, n_pad, c->u_pack, &apack, s));
    }
    int cap = c->cand_cap;
    for (int attempt = 0;; ++attempt) {
        const int nseg = ps.tc ? 2 : 1;
        Cand* cand;
        int *cand_cnt, *kid;
        unsigned* lfin;
        unsigned long long* keys;
        TRY(c->ensure(c->cand, n * (int64_t)nseg * cap, &cand));
        TRY(c->ensure(c->cand_cnt, n * (int64_t)nseg, &cand_cnt));
        TRY(c->ensure(c->lfin, n, &lfin));
        TRY(c->ensure(c->keys, n * (int64_t)nseg * cap, &keys));
        TRY(c->ensure(c->kid, n * (int64_t)nseg * cap, &kid));
        CUDA_TRY(cudaMemsetAsync(lfin, 0, n * sizeof(unsigned), s));
        CUDA_TRY(cudaMemsetAsync(cand_cnt, 0, n * nseg * sizeof(int), s));
        ThresholdArgs a{};
        a.A = apack;
        a.B = it.pack;
        a.n = n;
        a.m = it.m;
        a.dp = ps.dp;
        a.k = k;
        a.cap = cap;
        a.unrm = up.nrm;
        a.unhat = up.nhat;
        a.udel = up.del;
        a.tmax = it.tmax;
        a.thmax = it.thmax;
        a.tdel = it.tdel;
        a.cacc = ps.cacc;
        a.eabs = ps.eabs;
        a.cand = cand;
        a.cand_cnt = cand_cnt;
        a.lfin_key = lfin;
        a.nseg = nseg;
        a.st = c->st;
        a.num_sms = c->num_sms;
        {
            Phase ph(c, s, RKM_PHASE_THRESHOLD);
            c->stats.threshold_launches++;
            if (ps.tc) {
                TmapPair tm;
                TRY(make_tmaps(apack, n_pad, it.pack, it.m_pad, ps.dp, BI_TC, &tm));
                launch_threshold_tc(a, &tm.a, &tm.b, s);
            } else {
                launch_threshold_simt(a, s);
            }
        }
        {
            Phase ph(c, s, RKM_PHASE_EXACT);
            ExactData x{U, ldu, up.e, up.q, P, ldp, it.rp.e, it.rp.q, d, (int)round_up(d, 8), &c->st->grid_u};
            launch_exact_tau(x, cand, cand_cnt, lfin, cap, nseg, it.perm, n, k, keys, kid, tau, tid, topk, c->st,
                             s);
        }
        TRY(read_status(c, s));
        if (!c->st_host->cand_overflow) break;
        if (cap >= it.m || attempt >= 3)
            return fail(RKM_EOVERFLOW, "candidate capacity %d overflowed after %d retries", cap, attempt);
        const int64_t next = std::min<int64_t>(it.m, (int64_t)cap * 4);
        if ((double)n * next * 20.0 * (ps.tc ? 2 : 1) > 64e9)
            return fail(RKM_EOVERFLOW, "candidate lists need more than 64 GB (n=%lld, cap=%lld)",
                        (long long)n, (long long)next);
        cap = (int)round_up(next, 32);
        c->cand_cap = cap;
        c->stats.retries++;
        CUDA_TRY(cudaMemsetAsync(&c->st->cand_overflow, 0, sizeof(unsigned), s));
        CUDA_TRY(cudaMemsetAsync(&c->st->internal_error, 0, sizeof(unsigned), s));
        CUDA_TRY(cudaMemsetAsync(&c->st->cand_total, 0, sizeof(unsigned long long), s));
    }
    if (c->st_host->internal_error) return fail(RKM_EINTERNAL, "threshold pass: fewer than k candidates");
    c->stats.candidates = c->st_host->cand_total;
    c->stats.exact_integer_path = c->st_host->grid_u ? 1 : 0;
    return RKM_OK;
}

// K4 for users: ratios, bucket sort, ratio-order copies.
struct UserOrder {
    int* uperm;       // ratio order -> original user
    unsigned* ucum;   // users per ratio bucket, inclusive prefix
    void* pack;       // users packed in ratio order
    UserMeta* meta;   // per-user records, ratio order
};

struct UserBufs {
    Buf &perm, &cum, &pack, &meta;
};

rkm_status order_users(rkm_ctx* c, const PathShape& ps, const float* U, int64_t n, int64_t ldu, int d,
                       const RowPrep& up, const double* tau, const int* tid, const UserBufs& bb, UserOrder* uo,
                       cudaStream_t s) {
    float* r;
    unsigned *hist, *offs;
    TRY(c->ensure(c->r_u, n, &r));
    TRY(c->ensure(c->hist, NBUCKET, &hist));
    TRY(c->ensure(c->offs, NBUCKET, &offs));
    TRY(c->ensure(bb.perm, n, &uo->uperm));
    TRY(c->ensure(bb.cum, NBUCKET, &uo->ucum));
    launch_user_ratio(tau, up.n2, n, r, s);
    launch_bucket_sort(r, n, false, hist, offs, uo->uperm, uo->ucum, s);
    const int64_t n_pad = round_up(std::max<int64_t>(n, 1), BU);
    TRY(pack(c, ps, U, n, ldu, d, uo->uperm, n_pad, bb.pack, &uo->pack, s));
    TRY(c->ensure(bb.meta, n, &uo->meta));
    launch_user_meta(tau, up.nrm, up.nhat, up.del, uo->uperm, n, uo->meta, s);
    return RKM_OK;
}

// One counting stage over item tiles [t_begin, t_end) (t_end from the device if t_end_dev).
rkm_status count_stage(rkm_ctx* c, const PathShape& ps, int64_t n, const UserOrder& uo, const ItemSide& it,
                       bool new_items, int t_begin, int t_end, bool t_end_from_dev, const ExactData& x,
                       const double* tau, const int* tid, int* cnt, int2* band, cudaStream_t s) {
    int* nprefix;
    unsigned* unit_off;
    TRY(c->ensure(c->nprefix, std::max<int64_t>(it.tiles, 1), &nprefix));
    TRY(c->ensure(c->unit_off, it.tiles + 2, &unit_off));
    const int group = 32;  // user tiles per work unit (4096 users against one item tile)
    Phase ph_count(c, s, RKM_PHASE_COUNT);
    launch_build_units(it.tmax, uo.ucum, t_begin, t_end, t_end_from_dev ? &c->st->t_end : nullptr, BU, group,
                       nprefix, unit_off, c->st, s);
    CountArgs a{};
    a.A = uo.pack;
    a.B = it.pack;
    a.n = n;
    a.m = it.m;
    a.dp = ps.dp;
    a.meta = uo.meta;
    a.item_id = new_items ? nullptr : it.perm;
    a.new_items = new_items;
    a.tmax = it.tmax;
    a.thmax = it.thmax;
    a.tdel = it.tdel;
    a.nprefix = nprefix;
    a.unit_off = unit_off;
    a.t_begin = t_begin;
    a.group = group;
    a.cacc = ps.cacc;
    a.eabs = ps.eabs;
    a.counts = cnt;
    a.band = band;
    a.band_cap = (unsigned)c->band_cap;
    a.st = c->st;
    a.num_sms = c->num_sms;
    if (ps.tc) {
        TmapPair tm;
        const int64_t n_pad = round_up(std::max<int64_t>(n, 1), BU);
        TRY(make_tmaps(uo.pack, n_pad, it.pack, it.m_pad, ps.dp, BI_TC, &tm));
        launch_count_tc(a, &tm.a, &tm.b, s);
    } else {
        launch_count_simt(a, s);
    }
    return RKM_OK;
}

rkm_status band_stage(rkm_ctx* c, const ItemSide& it, bool new_items, const ExactData& x, const double* tau,
                      const int* tid, int* cnt, int2* band, cudaStream_t s) {
    Phase ph(c, s, RKM_PHASE_BAND);
    launch_band_rescore(x, band, (unsigned)c->band_cap, it.perm, it.m, tau, tid, new_items, cnt, c->st, s);
    return RKM_OK;
}

__global__ void k_scatter_i32(const int* __restrict__ src, const int* __restrict__ perm, int64_t count,
                              int* __restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[perm[i]] = src[i];
}

void scatter_i32(const int* src, const int* perm, int64_t count, int* dst, cudaStream_t s) {
    if (count <= 0) return;
    int64_t blocks = std::min<int64_t>((count + 255) / 256, 65536);
    note_launch();
    k_scatter_i32<<<(int)blocks, 256, 0, s>>>(src, perm, count, dst);
}

rkm_status ensure_band(rkm_ctx* c, int2** band) { return c->ensure(c->band, c->band_cap, band); }

// Initial capacities of a call: the option (or a default sized from n and k), or the
// capacity a previous call on this context grew to, whichever is larger.
void init_caps(rkm_ctx* c, int64_t n, int k) {
    int cap = c->opts.cand_capacity > 0 ? c->opts.cand_capacity : (int)round_up(2 * k + 96, 32);
    cap = (int)round_up(cap, 32);
    if (c->cand_k == k) cap = std::max(cap, c->cand_cap);
    c->cand_cap = cap;
    c->cand_k = k;
    int64_t band = c->opts.band_capacity > 0 ? c->opts.band_capacity : std::max<int64_t>(1 << 22, 16 * n);
    band = std::max<int64_t>(band, c->band_cap);
    c->band_cap = std::min<int64_t>(band, (int64_t)UINT32_MAX - 1);
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

extern "C" {

void rkm_default_opts(rkm_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = RKM_BF16;
    o->k_max = KMAX;
    o->cand_capacity = 0;
    o->band_capacity = 0;
    o->filter = 1;
}

const char* rkm_last_error(void) { return g_err.c_str(); }

const char* rkm_version(void) { return "rkm 0.1 (sm_103a)"; }

rkm_status rkm_create(rkm_ctx** out, const rkm_opts* opts, int device) {
    if (!out) return fail(RKM_EINVAL, "null output pointer");
    *out = nullptr;
    rkm_opts o;
    rkm_default_opts(&o);
    if (opts) o = *opts;
    if (o.k_max < 1 || o.k_max > KMAX) return fail(RKM_EINVAL, "k_max must be in [1, %d]", KMAX);
    if (o.precision < RKM_FP32 || o.precision > RKM_FP8) return fail(RKM_EINVAL, "unknown precision");
    if (o.cand_capacity < 0 || o.band_capacity < 0) return fail(RKM_EINVAL, "negative capacity");
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(RKM_EINVAL, "device %d out of range (%d devices)", device, ndev);
    CUDA_TRY(cudaSetDevice(device));
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return fail(RKM_ECUDA, "device %d is sm_%d%d; this library is built for sm_103a", device, prop.major,
                    prop.minor);
    rkm_ctx* c = new rkm_ctx();
    c->device = device;
    c->opts = o;
    c->num_sms = prop.multiProcessorCount;
    cudaError_t e = cudaMalloc(&c->st, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost(&c->st_host, sizeof(DevStatus));
    if (e != cudaSuccess) {
        if (c->st) cudaFree(c->st);
        delete c;
        return fail(RKM_ENOMEM, "status allocation failed: %s", cudaGetErrorString(e));
    }
    *out = c;
    return RKM_OK;
}

void rkm_destroy(rkm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    c->free_all();
    if (c->st) cudaFree(c->st);
    if (c->st_host) cudaFreeHost(c->st_host);
    delete c;
}

rkm_status rkm_get_stats(const rkm_ctx* c, rkm_stats* out) {
    if (!c || !out) return fail(RKM_EINVAL, "null argument");
    *out = c->stats;
    return RKM_OK;
}

rkm_status rkm_thresholds(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, const float* P, int64_t m,
                          int64_t ldp, int d, int k, double* tau, int32_t* tid, int32_t* topk, void* stream) {
    TRY(check_common(c, d));
    TRY(check_matrix(U, n, ldu, d, "U"));
    TRY(check_matrix(P, m, ldp, d, "P"));
    if (k < 1 || k > m || k > c->opts.k_max)
        return fail(RKM_EINVAL, "k must satisfy 1 <= k <= min(m, k_max) (k=%d, m=%lld)", k, (long long)m);
    if (n > 0 && (!tau || !tid)) return fail(RKM_EINVAL, "null tau/tid");
    const double t0 = now_ms();
    reset_stats(c);
    if (n == 0) return RKM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const PathShape ps = path_shape(c->opts.precision, d);
    init_caps(c, n, k);
    TRY(begin_call(c, s));
    RowPrep up;
    ItemSide it;
    {
        Phase ph(c, s, RKM_PHASE_PREP);
        TRY(prep_rows(c, ps, U, n, ldu, d, c->u_e, c->u_q, c->u_n2, c->u_nrm, c->u_nhat, c->u_del, &up, s));
        TRY(prep_items(c, ps, P, m, ldp, d, catalogue_bufs(c), &it, s));
    }
    TRY(thresholds_core(c, ps, U, n, ldu, P, ldp, d, k, up, it, tau, tid, topk, s));
    c->stats.pairs_total = (uint64_t)n * (uint64_t)m;
    c->stats.last_ms = now_ms() - t0;
    return RKM_OK;
}

static rkm_status scores_impl(rkm_ctx* c, const PathShape& ps, const float* U, int64_t n, int64_t ldu,
                              const float* P, int64_t ldp, int d, const RowPrep& up, const ItemSide& it,
                              const double* tau, const int32_t* tid, int N, int32_t* scores, int32_t* ids,
                              int32_t* top_scores, bool filter, cudaStream_t s) {
    UserOrder uo;
    {
        Phase ph(c, s, RKM_PHASE_BOUNDS);
        TRY(order_users(c, ps, U, n, ldu, d, up, tau, tid,
                        UserBufs{c->uperm, c->ucum, c->us_pack, c->us_meta},
                        &uo, s));
    }
    ExactData x{U, ldu, up.e, up.q, P, ldp, it.rp.e, it.rp.q, d, (int)round_up(d, 8), &c->st->grid_u};
    int* cnt;
    TRY(c->ensure(c->cnt_s, it.m, &cnt));
    for (int attempt = 0;; ++attempt) {
        int2* band;
        TRY(ensure_band(c, &band));
        CUDA_TRY(cudaMemsetAsync(cnt, 0, it.m * sizeof(int), s));
        CUDA_TRY(cudaMemsetAsync(&c->st->band_count, 0, 2 * sizeof(unsigned), s));  // band_count, band_done
        const int tiles = (int)it.tiles;
        if (!filter) {
            TRY(count_stage(c, ps, n, uo, it, false, 0, tiles, false, x, tau, tid, cnt, band, s));
            TRY(band_stage(c, it, false, x, tau, tid, cnt, band, s));
            Phase ph(c, s, RKM_PHASE_TOPN);
            if (scores) scatter_i32(cnt, it.perm, it.m, scores, s);
            if (ids) launch_topn(cnt, it.perm, it.m, nullptr, N, ids, top_scores, c->st, s);
        } else {
            // First stage: enough leading tiles (largest norms, so largest bounds) to hold
            // N items and a few thousand more; its N-th score is an exact lower bound.
            int64_t c0 = std::max<int64_t>(4 * (int64_t)N, 8192);
            int t0 = (int)std::min<int64_t>(tiles, (c0 + ps.item_tile - 1) / ps.item_tile);
            TRY(count_stage(c, ps, n, uo, it, false, 0, t0, false, x, tau, tid, cnt, band, s));
            TRY(band_stage(c, it, false, x, tau, tid, cnt, band, s));
            int *tids_c0, *tsc_c0;
            TRY(c->ensure(c->top_ids, N, &tids_c0));
            TRY(c->ensure(c->top_sc, N, &tsc_c0));
            const int64_t m0 = std::min<int64_t>(it.m, (int64_t)t0 * ps.item_tile);
            if (t0 < tiles) {
                {
                    Phase ph(c, s, RKM_PHASE_TOPN);
                    launch_topn(cnt, it.perm, m0, nullptr, N, tids_c0, tsc_c0, c->st, s);
                    launch_filter_cut(tsc_c0, N, it.tmax, uo.ucum, it.tiles, t0, ps.item_tile, it.m, c->st, s);
                }
                TRY(count_stage(c, ps, n, uo, it, false, t0, 0, true, x, tau, tid, cnt, band, s));
                TRY(band_stage(c, it, false, x, tau, tid, cnt, band, s));
                Phase ph(c, s, RKM_PHASE_TOPN);
                launch_topn(cnt, it.perm, it.m, &c->st->m_counted, N, ids, top_scores, c->st, s);
            } else {
                Phase ph(c, s, RKM_PHASE_TOPN);
                launch_topn(cnt, it.perm, it.m, nullptr, N, ids, top_scores, c->st, s);
            }
        }
        TRY(read_status(c, s));
        if (!c->st_host->band_overflow) break;
        if (attempt >= 3) return fail(RKM_EOVERFLOW, "band queue (%lld pairs) overflowed", (long long)c->band_cap);
        c->band_cap = std::min<int64_t>((int64_t)UINT32_MAX - 1,
                                        std::max<int64_t>(c->band_cap * 2, (int64_t)c->st_host->band_count + 1024));
        c->stats.retries++;
        CUDA_TRY(cudaMemsetAsync(&c->st->band_overflow, 0, sizeof(unsigned), s));
    }
    if (c->st_host->internal_error) return fail(RKM_EINTERNAL, "counting pass: device consistency check failed");
    c->stats.band_pairs = c->st_host->band_count;
    c->stats.pairs_evaluated += c->st_host->pairs_evaluated;
    c->stats.items_counted = filter ? (uint64_t)(c->st_host->m_counted ? c->st_host->m_counted : it.m)
                                    : (uint64_t)it.m;
    return RKM_OK;
}

rkm_status rkm_scores(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, const float* P, int64_t m, int64_t ldp,
                      int d, const double* tau, const int32_t* tid, int32_t* scores, void* stream) {
    TRY(check_common(c, d));
    TRY(check_matrix(U, n, ldu, d, "U"));
    TRY(check_matrix(P, m, ldp, d, "P"));
    if (m > 0 && !scores) return fail(RKM_EINVAL, "null scores");
    if (n > 0 && (!tau || !tid)) return fail(RKM_EINVAL, "null tau/tid");
    const double t0 = now_ms();
    reset_stats(c);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (m == 0) return RKM_OK;
    if (n == 0) {
        CUDA_TRY(cudaMemsetAsync(scores, 0, m * sizeof(int32_t), s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return RKM_OK;
    }
    const PathShape ps = path_shape(c->opts.precision, d);
    init_caps(c, n, 1);
    TRY(begin_call(c, s));
    RowPrep up;
    ItemSide it;
    {
        Phase ph(c, s, RKM_PHASE_PREP);
        TRY(prep_rows(c, ps, U, n, ldu, d, c->u_e, c->u_q, c->u_n2, c->u_nrm, c->u_nhat, c->u_del, &up, s));
        TRY(prep_items(c, ps, P, m, ldp, d, catalogue_bufs(c), &it, s));
    }
    TRY(scores_impl(c, ps, U, n, ldu, P, ldp, d, up, it, tau, tid, 0, scores, nullptr, nullptr, false, s));
    c->stats.pairs_total = (uint64_t)n * (uint64_t)m;
    c->stats.exact_integer_path = c->st_host->grid_u ? 1 : 0;
    c->stats.last_ms = now_ms() - t0;
    return RKM_OK;
}

rkm_status rkm_topn(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, const float* P, int64_t m, int64_t ldp,
                    int d, int k, int N, int32_t* ids, int32_t* top_scores, double* tau_out, int32_t* tid_out,
                    void* stream) {
    TRY(check_common(c, d));
    TRY(check_matrix(U, n, ldu, d, "U"));
    TRY(check_matrix(P, m, ldp, d, "P"));
    if (k < 1 || k > m || k > c->opts.k_max)
        return fail(RKM_EINVAL, "k must satisfy 1 <= k <= min(m, k_max) (k=%d, m=%lld)", k, (long long)m);
    if (N < 1 || N > m || N > NMAX_TOPN)
        return fail(RKM_EINVAL, "N must satisfy 1 <= N <= min(m, %d) (N=%d)", NMAX_TOPN, N);
    if (!ids || !top_scores) return fail(RKM_EINVAL, "null ids/top_scores");
    const double t0 = now_ms();
    reset_stats(c);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const PathShape ps = path_shape(c->opts.precision, d);
    init_caps(c, n, k);
    TRY(begin_call(c, s));
    if (n == 0) {
        int* cnt;
        TRY(c->ensure(c->cnt_s, m, &cnt));
        CUDA_TRY(cudaMemsetAsync(cnt, 0, m * sizeof(int), s));
        launch_topn(cnt, nullptr, m, nullptr, N, ids, top_scores, c->st, s);
        TRY(read_status(c, s));
        return RKM_OK;
    }
    double* tau = tau_out;
    int* tid = tid_out;
    if (!tau) TRY(c->ensure(c->tau_tmp, n, &tau));
    if (!tid) TRY(c->ensure(c->tid_tmp, n, &tid));
    RowPrep up;
    ItemSide it;
    {
        Phase ph(c, s, RKM_PHASE_PREP);
        TRY(prep_rows(c, ps, U, n, ldu, d, c->u_e, c->u_q, c->u_n2, c->u_nrm, c->u_nhat, c->u_del, &up, s));
        TRY(prep_items(c, ps, P, m, ldp, d, catalogue_bufs(c), &it, s));
    }
    TRY(thresholds_core(c, ps, U, n, ldu, P, ldp, d, k, up, it, tau, tid, nullptr, s));
    const uint64_t cands = c->stats.candidates;
    TRY(scores_impl(c, ps, U, n, ldu, P, ldp, d, up, it, tau, tid, N, nullptr, ids, top_scores,
                    c->opts.filter != 0, s));
    c->stats.candidates = cands;
    c->stats.pairs_total = 2ull * (uint64_t)n * (uint64_t)m;
    c->stats.pairs_evaluated += (uint64_t)n * (uint64_t)m;
    c->stats.last_ms = now_ms() - t0;
    return RKM_OK;
}

rkm_status rkm_topn_host(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, const float* P, int64_t m,
                         int64_t ldp, int d, int k, int N, int32_t* ids, int32_t* top_scores, void* stream) {
    TRY(check_common(c, d));
    TRY(check_matrix(U, n, ldu, d, "U"));
    TRY(check_matrix(P, m, ldp, d, "P"));
    if (N < 1 || N > m || N > NMAX_TOPN) return fail(RKM_EINVAL, "bad N");
    if (!ids || !top_scores) return fail(RKM_EINVAL, "null ids/top_scores");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *dU, *dP;
    int *dids, *dsc;
    TRY(c->ensure(c->h_U, std::max<int64_t>(n * ldu, 1), &dU));
    TRY(c->ensure(c->h_P, std::max<int64_t>(m * ldp, 1), &dP));
    TRY(c->ensure(c->h_ids, N, &dids));
    TRY(c->ensure(c->h_sc, N, &dsc));
    if (n > 0) CUDA_TRY(cudaMemcpyAsync(dU, U, n * ldu * sizeof(float), cudaMemcpyHostToDevice, s));
    if (m > 0) CUDA_TRY(cudaMemcpyAsync(dP, P, m * ldp * sizeof(float), cudaMemcpyHostToDevice, s));
    TRY(rkm_topn(c, dU, n, ldu, dP, m, ldp, d, k, N, dids, dsc, nullptr, nullptr, stream));
    CUDA_TRY(cudaMemcpyAsync(ids, dids, N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(top_scores, dsc, N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return RKM_OK;
}

rkm_status rkm_item_bounds(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, const float* P, int64_t m,
                           int64_t ldp, int d, const double* tau, int32_t* uscore, void* stream) {
    TRY(check_common(c, d));
    TRY(check_matrix(U, n, ldu, d, "U"));
    TRY(check_matrix(P, m, ldp, d, "P"));
    if (m > 0 && !uscore) return fail(RKM_EINVAL, "null uscore");
    if (n > 0 && !tau) return fail(RKM_EINVAL, "null tau");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    reset_stats(c);
    if (m == 0) return RKM_OK;
    TRY(begin_call(c, s));
    RowPrep up, pp;
    const PathShape ps = path_shape(c->opts.precision, d);
    TRY(prep_rows(c, ps, U, n, ldu, d, c->u_e, c->u_q, c->u_n2, c->u_nrm, c->u_nhat, c->u_del, &up, s));
    TRY(prep_rows(c, ps, P, m, ldp, d, c->p_e, c->p_q, c->p_n2, c->p_nrm, c->p_nhat, c->p_del, &pp, s));
    float* r;
    unsigned *hist, *offs, *ucum;
    int* uperm;
    TRY(c->ensure(c->r_u, std::max<int64_t>(n, 1), &r));
    TRY(c->ensure(c->hist, NBUCKET, &hist));
    TRY(c->ensure(c->offs, NBUCKET, &offs));
    TRY(c->ensure(c->uperm, std::max<int64_t>(n, 1), &uperm));
    TRY(c->ensure(c->ucum, NBUCKET, &ucum));
    launch_user_ratio(tau, up.n2, n, r, s);
    launch_bucket_sort(r, n, false, hist, offs, uperm, ucum, s);
    launch_item_uscore(pp.nrm, m, ucum, uscore, s);
    TRY(read_status(c, s));
    return RKM_OK;
}

rkm_status rkm_resident_set(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, int d, const double* tau,
                            const int32_t* tid, void* stream) {
    TRY(check_common(c, d));
    TRY(check_matrix(U, n, ldu, d, "U"));
    if (n > 0 && (!tau || !tid)) return fail(RKM_EINVAL, "null tau/tid");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    c->resident = false;
    const PathShape ps = path_shape(c->opts.precision, d);
    TRY(begin_call(c, s));
    float* Uc;
    double* tau_c;
    int* tid_c;
    TRY(c->ensure(c->res_U, std::max<int64_t>(n * d, 1), &Uc));
    TRY(c->ensure(c->res_tau, std::max<int64_t>(n, 1), &tau_c));
    TRY(c->ensure(c->res_tid, std::max<int64_t>(n, 1), &tid_c));
    if (n > 0) {
        CUDA_TRY(cudaMemcpy2DAsync(Uc, d * sizeof(float), U, ldu * sizeof(float), d * sizeof(float), n,
                                   cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(tau_c, tau, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(tid_c, tid, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    }
    RowPrep up;
    TRY(prep_rows(c, ps, Uc, n, d, d, c->res_e, c->res_q, c->u_n2, c->u_nrm, c->u_nhat, c->u_del, &up, s));
    UserOrder uo;
    TRY(order_users(c, ps, Uc, n, d, d, up, tau_c, tid_c,
                    UserBufs{c->res_uperm, c->res_ucum, c->res_pack, c->res_meta},
                    &uo, s));
    TRY(read_status(c, s));
    c->res_grid = c->st_host->grid_u;
    c->res_n = n;
    c->res_d = d;
    c->resident = true;
    return RKM_OK;
}

rkm_status rkm_query_new_items(rkm_ctx* c, const float* Q, int64_t q, int64_t ldq, int32_t* counts, void* stream) {
    if (!c) return fail(RKM_EINVAL, "null context");
    if (!c->resident) return fail(RKM_ESTATE, "rkm_query_new_items before rkm_resident_set");
    const int d = c->res_d;
    TRY(check_common(c, d));
    TRY(check_matrix(Q, q, ldq, d, "Q"));
    if (q > 0 && !counts) return fail(RKM_EINVAL, "null counts");
    const double t0 = now_ms();
    reset_stats(c);
    if (q == 0) return RKM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = c->res_n;
    if (n == 0) {
        CUDA_TRY(cudaMemsetAsync(counts, 0, q * sizeof(int32_t), s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return RKM_OK;
    }
    const PathShape ps = path_shape(c->opts.precision, d);
    init_caps(c, std::max<int64_t>(n / 64, q * 64), 1);
    TRY(begin_call(c, s));
    CUDA_TRY(cudaMemcpyAsync(&c->st->grid_u, &c->res_grid, sizeof(unsigned), cudaMemcpyHostToDevice, s));
    ItemSide it;
    {
        Phase ph(c, s, RKM_PHASE_PREP);
        TRY(prep_items(c, ps, Q, q, ldq, d, query_bufs(c), &it, s));
    }
    UserOrder uo{static_cast<int*>(c->res_uperm.p), static_cast<unsigned*>(c->res_ucum.p), c->res_pack.p,
                 static_cast<UserMeta*>(c->res_meta.p)};
    ExactData x{static_cast<const float*>(c->res_U.p), d, static_cast<const int*>(c->res_e.p),
                static_cast<const int16_t*>(c->res_q.p), Q, ldq, it.rp.e, it.rp.q, d, (int)round_up(d, 8),
                &c->st->grid_u};
    int* cnt;
    TRY(c->ensure(c->q_cnt, q, &cnt));
    for (int attempt = 0;; ++attempt) {
        int2* band;
        TRY(ensure_band(c, &band));
        CUDA_TRY(cudaMemsetAsync(cnt, 0, q * sizeof(int), s));
        CUDA_TRY(cudaMemsetAsync(&c->st->band_count, 0, 2 * sizeof(unsigned), s));
        const double* rtau = static_cast<const double*>(c->res_tau.p);
        const int* rtid = static_cast<const int*>(c->res_tid.p);
        TRY(count_stage(c, ps, n, uo, it, true, 0, (int)it.tiles, false, x, rtau, rtid, cnt, band, s));
        TRY(band_stage(c, it, true, x, rtau, rtid, cnt, band, s));
        scatter_i32(cnt, it.perm, q, counts, s);
        TRY(read_status(c, s));
        if (!c->st_host->band_overflow) break;
        if (attempt >= 3) return fail(RKM_EOVERFLOW, "band queue overflowed");
        c->band_cap = std::min<int64_t>((int64_t)UINT32_MAX - 1,
                                        std::max<int64_t>(c->band_cap * 2, (int64_t)c->st_host->band_count + 1024));
        c->stats.retries++;
        CUDA_TRY(cudaMemsetAsync(&c->st->band_overflow, 0, sizeof(unsigned), s));
    }
    if (c->st_host->internal_error) return fail(RKM_EINTERNAL, "query: device consistency check failed");
    c->stats.pairs_total = (uint64_t)n * (uint64_t)q;
    c->stats.pairs_evaluated = c->st_host->pairs_evaluated;
    c->stats.band_pairs = c->st_host->band_count;
    c->stats.exact_integer_path = c->st_host->grid_u ? 1 : 0;
    c->stats.last_ms = now_ms() - t0;
    return RKM_OK;
}

}  // extern "C"
