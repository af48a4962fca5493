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
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdarg>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <atomic>
#include <map>
#include <mutex>
#include <fstream>
#include <sstream>

#include "../../include/rkm.h"
#include "common.cuh"
#include "internal.h"
#include "kernels.h"
#include "state_io.h"
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
    // Serialises the calls made on this context from different host threads (a call that
    // enters another entry point on the same context re-locks it).
    mutable std::recursive_mutex mu;
    int device = 0;
    int num_sms = 0;
    rkm_opts opts{};
    rkm_stats stats{};
    DevStatus* st = nullptr;     // device status word
    DevStatus* st_host = nullptr;  // pinned mirror
    // users (original order)
    Buf u_e, u_q, u_n2, u_nrm, u_nhat, u_del, u_pack;
    // items (original order; sorted copies)
    Buf p_e, p_q, p_n2, p_nrm, p_nhat, p_del, p_perm, p_pack, tmax, thmax, tdel, p_texp;
    // bucket sort scratch
    Buf hist, offs;
    // threshold pass
    Buf cand, cand_cnt, lfin, keys, kid, topk_tmp;
    // threshold pass: seed bounds and user order
    Buf lseed, thr_perm;
    // counting pass
    Buf r_u, uperm, ucum, us_pack, us_meta, nprefix, unit_off, band, cnt_s, top_ids, top_sc, tau_tmp,
        tid_tmp;
    // serving (resident users)
    bool resident = false;
    std::atomic<int> servers{0};  // serving loops borrowing the resident set
    int64_t res_n = 0;
    int res_d = 0;
    unsigned res_off_grid = 0;
    Buf res_U, res_e, res_q, res_tau, res_tid, res_uperm, res_ucum, res_pack, res_meta;
    // query scratch
    Buf q_e, q_q, q_n2, q_nrm, q_nhat, q_del, q_perm, q_pack, q_tmax, q_thmax, q_tdel, q_cnt, q_texp;
    // host staging for rkm_topn_host
    Buf h_U, h_P, h_ids, h_sc;
    int cand_cap = 0;
    int cand_k = 0;
    // Batches: one sub-context per instance (its own workspace and status), the captured graph
    // and the layout it was captured for, the batch's launch descriptors.
    std::vector<rkm_ctx*> sub;
    std::vector<rkm_instance> graph_key;
    int graph_opts_key = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    unsigned long long graph_kernels = 0;
    TcInstance* batch_host = nullptr;
    int batch_host_cap = 0;
    Buf batch_dev;
    // Batches: per-problem descriptors of the launches after the threshold pass (pinned host
    // staging, stable while a captured graph replays them, and device copies): the jobs and
    // the counting descriptors of both stages.
    BatchJob* jobs_host = nullptr;
    CountInstance* bcount_host = nullptr;
    int jobs_cap = 0;
    Buf jobs_dev, bcount_dev;
    std::string tune_cache;
    struct TuneEntry {
        int group;        // user tiles per counting work unit
        int64_t stage1;   // minimum items of the first counting stage
    };
    std::map<std::string, TuneEntry> tune;  // size bucket -> choices
    bool tune_loaded = false;
    // Batches run on an internal stream joined to the caller's stream by events, so that the
    // graph can be captured whatever stream the caller uses.
    cudaStream_t bstream = nullptr;
    cudaEvent_t bev_in = nullptr, bev_out = nullptr;
    // Tunables (set by the autotuner for batches): user tiles per counting work unit, and the
    // minimum number of items in the first counting stage of the filtered top-N.
    int count_group = 32;
    int64_t stage1_items = 8192;
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

    // Descriptors of the tensor-core threshold launch: pinned host staging and device copy.
    TcInstance* inst_host = nullptr;
    int inst_host_cap = 0;
    Buf inst_dev;

    rkm_status instances(int count, TcInstance** host, TcInstance** dev) {
        if (inst_host_cap < count) {
            if (inst_host) cudaFreeHost(inst_host);
            inst_host = nullptr;
            inst_host_cap = 0;
            if (cudaMallocHost(&inst_host, (size_t)count * sizeof(TcInstance)) != cudaSuccess) {
                cudaGetLastError();
                return fail(RKM_ENOMEM, "pinned descriptor staging of %d instances failed", count);
            }
            inst_host_cap = count;
        }
        *host = inst_host;
        return ensure(inst_dev, count, dev);
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
        Buf* all[] = {&topk_tmp, &u_e, &u_q, &u_n2, &u_nrm, &u_nhat, &u_del, &u_pack, &p_e, &p_q, &p_n2, &p_nrm,
                      &p_nhat, &p_del, &p_perm, &p_pack, &tmax, &thmax, &tdel, &hist, &offs, &cand,
                      &cand_cnt, &lfin, &keys, &kid, &r_u, &uperm, &ucum, &us_pack, &us_meta,
                      &nprefix, &unit_off, &band, &cnt_s, &top_ids, &top_sc, &lseed, &thr_perm,
                      &tau_tmp, &tid_tmp, &res_U, &res_e, &res_q, &res_tau, &res_tid, &res_uperm, &res_ucum,
                      &res_pack, &res_meta, &q_e, &q_q,
                      &q_n2, &q_nrm, &q_nhat, &q_del, &q_perm, &q_pack, &q_tmax, &q_thmax, &q_tdel, &q_cnt,
                      &q_texp, &p_texp,
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
        if (inst_dev.p) cudaFree(inst_dev.p);
        inst_dev = Buf{};
        if (inst_host) cudaFreeHost(inst_host);
        inst_host = nullptr;
        inst_host_cap = 0;
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        graph_exec = nullptr;
        graph = nullptr;
        if (batch_dev.p) cudaFree(batch_dev.p);
        batch_dev = Buf{};
        if (bstream) cudaStreamDestroy(bstream);
        if (bev_in) cudaEventDestroy(bev_in);
        if (bev_out) cudaEventDestroy(bev_out);
        bstream = nullptr;
        bev_in = bev_out = nullptr;
        if (batch_host) cudaFreeHost(batch_host);
        batch_host = nullptr;
        batch_host_cap = 0;
        if (jobs_host) cudaFreeHost(jobs_host);
        if (bcount_host) cudaFreeHost(bcount_host);
        jobs_host = nullptr;
        bcount_host = nullptr;
        jobs_cap = 0;
        if (jobs_dev.p) cudaFree(jobs_dev.p);
        if (bcount_dev.p) cudaFree(bcount_dev.p);
        jobs_dev = Buf{};
        bcount_dev = Buf{};
    }
};

namespace {

// Holds a context's call mutex for the duration of an entry point (nothing for NULL).
struct CtxLock {
    std::unique_lock<std::recursive_mutex> lk;
    explicit CtxLock(const rkm_ctx* c) {
        if (c) lk = std::unique_lock<std::recursive_mutex>(c->mu);
    }
};

// Names of the phases in NVTX ranges (indices RKM_PHASE_*).
const char* const PHASE_NAMES[RKM_PHASES] = {"rkm prep (K1)",   "rkm threshold (K2)", "rkm exact tau (K3)",
                                             "rkm bounds (K4)", "rkm count (K5)",     "rkm band (K6)",
                                             "rkm top-N (K7)",  "rkm host copies"};

// One phase of a call: an NVTX range on the host thread (seen by Nsight tools when they are
// attached; a no-op otherwise), and CUDA events around it on the call's stream when
// profiling is on.
struct Phase {
    rkm_ctx* c;
    cudaStream_t s;
    int ph;
    cudaEvent_t e0 = nullptr;
    Phase(rkm_ctx* c_, cudaStream_t s_, int ph_) : c(c_), s(s_), ph(ph_) {
        nvtxRangePushA(PHASE_NAMES[ph]);
        if (c->opts.profile) {
            e0 = c->take_event();
            cudaEventRecord(e0, s);
        }
    }
    ~Phase() {
        nvtxRangePop();
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
    bool tc;         // tensor-core kernels
    bool fp8;        // FP8 e4m3 operands (tensor cores) with power-of-two scales
    int elem_bytes;  // bytes per packed operand element (4 FP32, 2 BF16, 1 FP8)
    int item_tile;   // BI of the product kernels
    int dp;          // padded depth (elements)
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
// FP8 e4m3 products are exact (4-bit significands), but the internal accumulation of
// kind::f8f6f4 is not documented either; FP8 accumulation on the previous generation kept
// only about 14 bits (DeepSeek-AI, "DeepSeek-V3 Technical Report", 2024, Section 3.3).
// Measured on GB300 through rkm_debug_products, on operands that e4m3 represents exactly
// (so the accumulation is the only error) with partial sums spanning more than 24 bits, the
// largest error of kind::f8f6f4 was 1.1 * 2^-24 ||u|| ||p|| at d = 128 and 256: FP32-like, no
// narrow accumulator.  So FP8 takes the BF16 constant, cacc = d 2^-22, which is still about
// 100 times the largest error measured at d = 128.  The FP8 representation error (3 mantissa
// bits, ||x^ - x|| near 2^-5 ||x||) dominates the band anyway.
PathShape path_shape(rkm_precision prec, int d) {
    PathShape ps{};
    const double dd = (double)d;
    const double g32 = dd * 0x1p-24 / (1.0 - dd * 0x1p-24);
    if (prec == RKM_FP32) {
        ps.tc = false;
        ps.elem_bytes = 4;
        ps.item_tile = BI_SIMT;
        ps.dp = (int)round_up(d, 32);
        ps.cacc = (float)((2.0 * g32 + dd * 0x1p-50) * (1.0 + 0x1p-20));
    } else if (prec == RKM_FP8) {
        ps.tc = true;
        ps.fp8 = true;
        ps.elem_bytes = 1;
        ps.item_tile = BI_TC;
        ps.dp = (int)round_up(d, 128);
        ps.cacc = (float)((dd * 0x1p-22 + dd * 0x1p-50) * (1.0 + 0x1p-20));
    } else {
        ps.tc = true;
        ps.elem_bytes = 2;
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
    if (c->opts.precision != RKM_FP32 && !rkm_tc_available())
        return fail(RKM_EINVAL, "tensor-core kernels are not built into this library");
    CUDA_TRY(cudaSetDevice(c->device));
    return RKM_OK;
}

rkm_status begin_call(rkm_ctx* c, cudaStream_t s) {
    CUDA_TRY(cudaMemsetAsync(c->st, 0, sizeof(DevStatus), s));
    return RKM_OK;
}

rkm_status read_status(rkm_ctx* c, cudaStream_t s) {
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    collect_phases(c);
    if (c->st_host->timeout) return fail(RKM_ETIMEOUT, "a bounded device wait gave up (kernel aborted)");
    if (c->st_host->debug_line)
        return fail(RKM_EINTERNAL, "debug build: a device index check failed (source line %u)", c->st_host->debug_line);
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

// Users get the norms of their product operand here; items on the FP8 path get them from
// their pack, whose scale is per item tile (items = true).
rkm_status prep_rows(rkm_ctx* c, const PathShape& ps, const float* X, int64_t rows, int64_t ld, int d, Buf& be,
                     Buf& bq, Buf& bn2, Buf& bnrm, Buf& bnhat, Buf& bdel, RowPrep* out, cudaStream_t s,
                     bool items = false) {
    const int dq = (int)round_up(d, 8);
    TRY(c->ensure(be, rows, &out->e));
    TRY(c->ensure(bq, rows * dq, &out->q));
    TRY(c->ensure(bn2, rows, &out->n2));
    TRY(c->ensure(bnrm, rows, &out->nrm));
    TRY(c->ensure(bnhat, rows, &out->nhat));
    TRY(c->ensure(bdel, rows, &out->del));
    const int operand = !ps.tc ? OPERAND_F32 : !ps.fp8 ? OPERAND_BF16 : items ? OPERAND_F32 : OPERAND_FP8_ROW;
    launch_prep_rows(X, rows, ld, d, out->e, out->q, dq, out->n2, out->nrm, out->nhat, out->del, operand, c->st, s);
    return RKM_OK;
}

// Operand pack (row perm[r] if perm != null).  FP8: each row scaled by 2^(8 - e) with e its
// tile's exponent (tile_exp) or its own (row_exp); nhat/del, when given, receive the norms of
// the descaled operand.
rkm_status pack(rkm_ctx* c, const PathShape& ps, const float* X, int64_t rows, int64_t ld, int d,
                const int* perm, int64_t rows_pad, Buf& b, void** out, cudaStream_t s, const int* row_exp = nullptr,
                const int* tile_exp = nullptr, float* nhat = nullptr, float* del = nullptr) {
    if (ps.fp8) {
        uint8_t* p;
        TRY(c->ensure(b, rows_pad * ps.dp, &p));
        launch_pack_fp8(X, rows, ld, d, perm, row_exp, tile_exp, ps.item_tile, p, rows_pad, ps.dp, nhat, del, s);
        *out = p;
    } else if (ps.tc) {
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
    int* texp;       // [tiles] FP8 tile exponents (null otherwise)
    int* perm;       // sorted pos -> original id
    void* pack;      // [m_pad][dp]
    float* tmax;     // [tiles] max ||p||
    float* thmax;    // [tiles] max ||p^||
    float* tdel;     // [tiles] max ||p^ - p||
    int64_t m, m_pad, tiles;
};

struct ItemBufs {
    Buf &e, &q, &n2, &nrm, &nhat, &del, &perm, &pack, &tmax, &thmax, &tdel, &texp;
};

rkm_status prep_items(rkm_ctx* c, const PathShape& ps, const float* P, int64_t m, int64_t ldp, int d,
                      const ItemBufs& bb, ItemSide* it, cudaStream_t s) {
    it->m = m;
    it->m_pad = round_up(std::max<int64_t>(m, 1), BI_TC);
    it->tiles = (m + ps.item_tile - 1) / ps.item_tile;
    TRY(prep_rows(c, ps, P, m, ldp, d, bb.e, bb.q, bb.n2, bb.nrm, bb.nhat, bb.del, &it->rp, s, true));
    unsigned *hist, *offs;
    TRY(c->ensure(c->hist, HIST_WORDS, &hist));
    TRY(c->ensure(c->offs, NBUCKET, &offs));
    TRY(c->ensure(bb.perm, m, &it->perm));
    launch_bucket_sort(it->rp.nrm, m, true, hist, offs, it->perm, nullptr, s);
    const int64_t nt = std::max<int64_t>(it->tiles, 1);
    it->texp = nullptr;
    if (ps.fp8) {
        TRY(c->ensure(bb.texp, nt, &it->texp));
        launch_tile_exp(it->rp.e, it->perm, m, ps.item_tile, it->tiles, it->texp, s);
    }
    TRY(pack(c, ps, P, m, ldp, d, it->perm, it->m_pad, bb.pack, &it->pack, s, nullptr, it->texp, it->rp.nhat,
             it->rp.del));
    TRY(c->ensure(bb.tmax, nt, &it->tmax));
    TRY(c->ensure(bb.thmax, nt, &it->thmax));
    TRY(c->ensure(bb.tdel, nt, &it->tdel));
    launch_tile_max(it->rp.nrm, it->rp.nhat, it->rp.del, it->perm, m, ps.item_tile, it->tiles, it->tmax,
                    it->thmax, it->tdel, s);
    return RKM_OK;
}

ItemBufs catalogue_bufs(rkm_ctx* c) {
    return ItemBufs{c->p_e, c->p_q, c->p_n2, c->p_nrm, c->p_nhat, c->p_del, c->p_perm, c->p_pack, c->tmax,
                    c->thmax, c->tdel, c->p_texp};
}

ItemBufs query_bufs(rkm_ctx* c) {
    return ItemBufs{c->q_e, c->q_q, c->q_n2, c->q_nrm, c->q_nhat, c->q_del, c->q_perm, c->q_pack, c->q_tmax,
                    c->q_thmax, c->q_tdel, c->q_texp};
}

// Threshold pass of one problem, split so that a batch can put many problems into one
// launch of the tensor-core kernel: prepare (user pack, candidate buffers, arguments),
// launch the product, then exact rescoring.  None of these waits for the device.
struct ThrPlan {
    ThresholdArgs a;
    void* apack;
    int64_t n_pad;
    Cand* cand;
    int* cand_cnt;
    unsigned* lfin;
    unsigned long long* keys;
    int* kid;
    int nseg, cap;
};

// Candidate segments per user of a threshold launch with the largest k `kheap` (one per
// epilogue warpgroup of the tensor-core kernel; one on the FP32 path).  want_groups: the
// context's epilogue_groups option (0 = auto).
int threshold_segments(const PathShape& ps, int kheap, int want_groups) {
    return ps.tc ? threshold_groups(kheap, ps.dp, ps.fp8, want_groups) : 1;
}

// nseg: candidate segments of the launch this problem joins (0 = a launch of its own).
rkm_status threshold_prepare(rkm_ctx* c, const PathShape& ps, const float* U, int64_t n, int64_t ldu, int d, int k,
                             const RowPrep& up, const ItemSide& it, ThrPlan* pl, cudaStream_t s, int nseg = 0) {
    pl->n_pad = round_up(std::max<int64_t>(n, 1), BU);
    {
        Phase ph(c, s, RKM_PHASE_PREP);
        TRY(pack(c, ps, U, n, ldu, d, nullptr, pl->n_pad, c->u_pack, &pl->apack, s, up.e));
    }
    pl->cap = c->cand_cap;
    pl->nseg = nseg > 0 ? nseg : threshold_segments(ps, k, c->opts.epilogue_groups);
    TRY(c->ensure(c->cand, n * (int64_t)pl->nseg * pl->cap, &pl->cand));
    TRY(c->ensure(c->cand_cnt, n * (int64_t)pl->nseg, &pl->cand_cnt));
    TRY(c->ensure(c->lfin, n, &pl->lfin));
    TRY(c->ensure(c->keys, n * (int64_t)pl->nseg * pl->cap, &pl->keys));
    TRY(c->ensure(c->kid, n * (int64_t)pl->nseg * pl->cap, &pl->kid));
    CUDA_TRY(cudaMemsetAsync(pl->lfin, 0, n * sizeof(unsigned), s));
    CUDA_TRY(cudaMemsetAsync(pl->cand_cnt, 0, n * pl->nseg * sizeof(int), s));
    ThresholdArgs& a = pl->a;
    a = ThresholdArgs{};
    a.A = pl->apack;
    a.B = it.pack;
    a.n = n;
    a.m = it.m;
    a.dp = ps.dp;
    a.k = k;
    a.cap = pl->cap;
    a.unrm = up.nrm;
    a.unhat = up.nhat;
    a.udel = up.del;
    a.tmax = it.tmax;
    a.thmax = it.thmax;
    a.tdel = it.tdel;
    a.cacc = ps.cacc;
    a.eabs = ps.eabs;
    a.uexp = up.e;
    a.texp = it.texp;
    a.cand = pl->cand;
    a.cand_cnt = pl->cand_cnt;
    a.lfin_key = pl->lfin;
    a.nseg = pl->nseg;
    a.st = c->st;
    a.num_sms = c->num_sms;
    return RKM_OK;
}

rkm_status threshold_descriptor(const PathShape& ps, const ThrPlan& pl, const ItemSide& it, TcInstance* out) {
    TmapPair tm;
    TRY(make_tmaps(pl.apack, pl.n_pad, it.pack, it.m_pad, ps.dp, BI_TC, ps.elem_bytes, &tm));
    out->tmA = tm.a;
    out->tmB = tm.b;
    out->a = pl.a;
    out->unit_begin = 0;
    return RKM_OK;
}

// slot: descriptor slot (0 or 1; the seed pass and the main pass of one call use different
// slots, since the pinned staging of the first may not have been copied yet).
rkm_status threshold_launch_one(rkm_ctx* c, const PathShape& ps, const ThrPlan& pl, const ItemSide& it,
                                cudaStream_t s, int slot = 0) {
    Phase ph(c, s, RKM_PHASE_THRESHOLD);
    c->stats.threshold_launches++;
    if (ps.tc) {
        TcInstance* hi;
        TcInstance* di;
        TRY(c->instances(2, &hi, &di));
        TRY(threshold_descriptor(ps, pl, it, hi + slot));
        CUDA_TRY(cudaMemcpyAsync(di + slot, hi + slot, sizeof(TcInstance), cudaMemcpyHostToDevice, s));
        launch_threshold_tc(di + slot, 1, (pl.a.n + BU - 1) / BU, pl.a.k, ps.dp, ps.fp8, pl.nseg, c->num_sms, s);
    } else {
        launch_threshold_simt(pl.a, s);
    }
    return RKM_OK;
}

void threshold_exact(rkm_ctx* c, const float* U, int64_t ldu, const float* P, int64_t ldp, int d,
                     const RowPrep& up, const ItemSide& it, const ThrPlan& pl, double* tau, int* tid, int* topk,
                     cudaStream_t s) {
    Phase ph(c, s, RKM_PHASE_EXACT);
    ExactData x{U, ldu, up.e, up.q, P, ldp, it.rp.e, it.rp.q, d, (int)round_up(d, 8), &c->st->off_grid,
                pl.a.n, it.m};
    launch_exact_tau(x, pl.cand, pl.cand_cnt, pl.lfin, pl.cap, pl.nseg, it.perm, pl.a.n, pl.a.k, pl.keys, pl.kid,
                     tau, tid, topk, c->st, s, pl.a.uperm);
}

// Seed order of the tensor-core threshold pass.  Items arrive in descending norm order and a
// user tile stops once no user of it can still reach its bound (Algorithm 1's Cauchy-Schwarz
// stop), so a tile stops as late as its user with the smallest tau_u / ||u||.  A first pass
// of the same kernel over the SEED_TILES highest-norm item tiles gives every user a lower
// bound L_u of tau_u (the k-th largest lower bound over those items); users are then packed
// in the order of L_u / ||u||, so that the users of a tile stop at about the same item, and
// L_u seeds the selector of the main pass.  The results do not depend on the order.  Used when
// a tile's product is two K-blocks deep or more (BF16 d > 64): measured on GB300 at
// 2M x 500K, d = 128, the products computed fell from 59 % to 52 % of n*m and the threshold
// phase from 116 to 104 ms; at 500K x 100K, d = 64, where the epilogue bounds the kernel, the
// phase grew from 7.9 to 8.9 ms.
#ifndef RKM_SEED_TILES
#define RKM_SEED_TILES 8
#endif
constexpr int64_t SEED_TILES = RKM_SEED_TILES;

rkm_status threshold_seed_order(rkm_ctx* c, const PathShape& ps, const float* U, int64_t n, int64_t ldu, int d,
                                const RowPrep& up, const ItemSide& it, ThrPlan* pl, cudaStream_t s) {
    unsigned *seed, *hist, *offs;
    float* r;
    int* perm;
    TRY(c->ensure(c->lseed, n, &seed));
    TRY(c->ensure(c->r_u, n, &r));
    TRY(c->ensure(c->hist, HIST_WORDS, &hist));
    TRY(c->ensure(c->offs, NBUCKET, &offs));
    TRY(c->ensure(c->thr_perm, n, &perm));
    CUDA_TRY(cudaMemsetAsync(seed, 0, n * sizeof(unsigned), s));
    ThrPlan pre = *pl;
    pre.a.m = std::min<int64_t>(it.m, SEED_TILES * BI_TC);
    pre.a.lfin_key = seed;
    TRY(threshold_launch_one(c, ps, pre, it, s, 1));
    {
        Phase ph(c, s, RKM_PHASE_PREP);
        launch_seed_ratio(seed, up.nrm, n, r, s);
        launch_bucket_sort(r, n, false, hist, offs, perm, nullptr, s);
        TRY(pack(c, ps, U, n, ldu, d, perm, pl->n_pad, c->u_pack, &pl->apack, s, up.e));
    }
    pl->a.A = pl->apack;
    pl->a.uperm = perm;
    pl->a.lfin_seed = seed;
    return RKM_OK;
}

// Grow the candidate capacity after an overflow; fails after three retries.
rkm_status grow_candidates(rkm_ctx* c, int64_t m, int attempt) {
    const int cap = c->cand_cap;
    if (cap >= m || attempt >= 3)
        return fail(RKM_EOVERFLOW, "candidate capacity %d overflowed after %d retries", cap, attempt);
    c->cand_cap = (int)round_up(std::min<int64_t>(m, (int64_t)cap * 4), 32);
    c->stats.retries++;
    return RKM_OK;
}

// Device bytes the candidate lists of one threshold launch may take (20 bytes per slot:
// the candidate, its exact key and its id): half of the device memory, at most 48 GB.
int64_t candidate_budget(const rkm_ctx* c) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        total_b = (size_t)16 << 30;
    }
    return std::min<int64_t>((int64_t)48 << 30, (int64_t)(total_b / 2));
}

// Rows [u0, u0 + rows) of a prepared side.
RowPrep row_slice(const RowPrep& r, int64_t u0, int d) {
    const int64_t dq = round_up(d, 8);
    return RowPrep{r.e + u0, r.q + u0 * dq, r.n2 + u0, r.nrm + u0, r.nhat + u0, r.del + u0};
}

// Thresholds of every user, in slices of users small enough that their candidate lists fit
// the candidate budget (a wide guard band, as on the FP8 path, keeps many candidates per
// user).  A capacity overflow in any slice grows the capacity and restarts the pass.
rkm_status thresholds_core(rkm_ctx* c, const PathShape& ps, const float* U, int64_t n, int64_t ldu,
                           const float* P, int64_t ldp, int d, int k, const RowPrep& up, const ItemSide& it,
                           double* tau, int* tid, int* topk, cudaStream_t s) {
    for (int attempt = 0;; ++attempt) {
        const int64_t per_user = (int64_t)threshold_segments(ps, k, c->opts.epilogue_groups) * c->cand_cap * 20;
        const int64_t slice = std::min<int64_t>(n, std::max<int64_t>(BU, candidate_budget(c) / per_user / BU * BU));
        bool overflow = false;
        for (int64_t u0 = 0; u0 < n && !overflow; u0 += slice) {
            const int64_t un = std::min<int64_t>(slice, n - u0);
            const RowPrep us = row_slice(up, u0, d);
            ThrPlan pl;
            TRY(threshold_prepare(c, ps, U + u0 * ldu, un, ldu, d, k, us, it, &pl, s));
            if (ps.tc && c->opts.seed_order && slice >= n && it.tiles >= 2 * SEED_TILES &&
                ps.dp * ps.elem_bytes >= 256)
                TRY(threshold_seed_order(c, ps, U, n, ldu, d, up, it, &pl, s));
            TRY(threshold_launch_one(c, ps, pl, it, s));
            threshold_exact(c, U + u0 * ldu, ldu, P, ldp, d, us, it, pl, tau + u0, tid + u0,
                            topk ? topk + u0 * k : nullptr, s);
            if (slice < n) TRY(read_status(c, s));  // a single slice is checked below
            if (slice < n) overflow = c->st_host->cand_overflow != 0;
        }
        if (slice >= n) {
            TRY(read_status(c, s));
            overflow = c->st_host->cand_overflow != 0;
        }
        if (!overflow) break;
        TRY(grow_candidates(c, it.m, attempt));
        CUDA_TRY(cudaMemsetAsync(&c->st->cand_overflow, 0, sizeof(unsigned), s));
        CUDA_TRY(cudaMemsetAsync(&c->st->internal_error, 0, sizeof(unsigned), s));
        CUDA_TRY(cudaMemsetAsync(&c->st->cand_total, 0, sizeof(unsigned long long), s));
        CUDA_TRY(cudaMemsetAsync(&c->st->thr_pairs, 0, sizeof(unsigned long long), s));
    }
    if (c->st_host->internal_error) return fail(RKM_EINTERNAL, "threshold pass: fewer than k candidates");
    c->stats.candidates = c->st_host->cand_total;
    c->stats.threshold_pairs = c->st_host->thr_pairs;  // products the threshold kernels computed
    c->stats.exact_integer_path = c->st_host->off_grid ? 0 : 1;
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
    TRY(c->ensure(c->hist, HIST_WORDS, &hist));
    TRY(c->ensure(c->offs, NBUCKET, &offs));
    TRY(c->ensure(bb.perm, n, &uo->uperm));
    TRY(c->ensure(bb.cum, NBUCKET, &uo->ucum));
    launch_user_ratio(tau, up.n2, n, r, s);
    launch_bucket_sort(r, n, false, hist, offs, uo->uperm, uo->ucum, s);
    const int64_t n_pad = round_up(std::max<int64_t>(n, 1), BU);
    TRY(pack(c, ps, U, n, ldu, d, uo->uperm, n_pad, bb.pack, &uo->pack, s, up.e));
    TRY(c->ensure(bb.meta, n, &uo->meta));
    launch_user_meta(tau, up.nrm, up.nhat, up.del, up.e, uo->uperm, n, uo->meta, s);
    return RKM_OK;
}

// Arguments and TMA maps of a tensor-core counting launch over one problem (unit_begin is
// written on the device).
rkm_status count_descriptor(const PathShape& ps, int64_t n, const UserOrder& uo, const ItemSide& it,
                            const CountArgs& a, CountInstance* out) {
    TmapPair tm;
    const int64_t n_pad = round_up(std::max<int64_t>(n, 1), BU);
    TRY(make_tmaps(uo.pack, n_pad, it.pack, it.m_pad, ps.dp, BI_TC, ps.elem_bytes, &tm));
    out->tmA = tm.a;
    out->tmB = tm.b;
    out->a = a;
    out->unit_begin = 0;
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
    const int group = c->count_group;  // user tiles per work unit
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
    a.texp = it.texp;
    a.nprefix = nprefix;
    a.unit_off = unit_off;
    a.t_begin = t_begin;
    a.group = group;
    a.groups = count_groups(ps.dp, ps.fp8, c->opts.epilogue_groups);
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
        TRY(make_tmaps(uo.pack, n_pad, it.pack, it.m_pad, ps.dp, BI_TC, ps.elem_bytes, &tm));
        launch_count_tc(a, &tm.a, &tm.b, ps.fp8, s);
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

// The band queue's size after an overflow: twice the old one, or the pairs the call pushed
// plus an eighth.  The margin matters for later calls on the same inputs: the bucket sorts
// do not fix the order of users (or items) within a bucket, so which users share the last
// user tile of a counting unit, and with it the band of a repeated call, varies by a few
// pairs in 10^4.
int64_t grown_band_cap(const rkm_ctx* c) {
    const int64_t pushed = (int64_t)c->st_host->band_count;
    return std::min<int64_t>((int64_t)UINT32_MAX - 1, std::max<int64_t>(c->band_cap * 2, pushed + pushed / 8 + 1024));
}

// Initial capacities of a call: the option (or a default sized from n and k), or the
// capacity a previous call on this context grew to, whichever is larger.
void init_caps(rkm_ctx* c, int64_t n, int k) {
    // FP8's guard band is about eight times BF16's, so its lists start larger.
    const int dflt = c->opts.precision == RKM_FP8 ? 8 * k + 256 : 2 * k + 96;
    int cap = c->opts.cand_capacity > 0 ? c->opts.cand_capacity : (int)round_up(dflt, 32);
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

rkm_status rkm::query_resident(rkm_ctx* c, const rkm_ctx* r, const float* Q, int64_t q, int64_t ldq, int32_t* counts,
                               cudaStream_t s) {
    if (!c || !r) return fail(RKM_EINVAL, "null context");
    if (!r->resident) return fail(RKM_ESTATE, "rkm_query_new_items before rkm_resident_set");
    const int d = r->res_d;
    TRY(check_common(c, d));
    TRY(check_matrix(Q, q, ldq, d, "Q"));
    if (q > 0 && !counts) return fail(RKM_EINVAL, "null counts");
    const double t0 = now_ms();
    reset_stats(c);
    if (q == 0) return RKM_OK;
    const int64_t n = r->res_n;
    if (n == 0) {
        CUDA_TRY(cudaMemsetAsync(counts, 0, q * sizeof(int32_t), s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return RKM_OK;
    }
    const PathShape ps = path_shape(c->opts.precision, d);
    init_caps(c, std::max<int64_t>(n / 64, q * 64), 1);
    TRY(begin_call(c, s));
    if (r->res_off_grid) CUDA_TRY(cudaMemsetAsync(&c->st->off_grid, 1, 1, s));
    ItemSide it;
    {
        Phase ph(c, s, RKM_PHASE_PREP);
        TRY(prep_items(c, ps, Q, q, ldq, d, query_bufs(c), &it, s));
    }
    UserOrder uo{static_cast<int*>(r->res_uperm.p), static_cast<unsigned*>(r->res_ucum.p), r->res_pack.p,
                 static_cast<UserMeta*>(r->res_meta.p)};
    ExactData x{static_cast<const float*>(r->res_U.p), d, static_cast<const int*>(r->res_e.p),
                static_cast<const int16_t*>(r->res_q.p), Q, ldq, it.rp.e, it.rp.q, d, (int)round_up(d, 8),
                &c->st->off_grid, n, q};
    int* cnt;
    TRY(c->ensure(c->q_cnt, q, &cnt));
    for (int attempt = 0;; ++attempt) {
        int2* band;
        TRY(ensure_band(c, &band));
        CUDA_TRY(cudaMemsetAsync(cnt, 0, q * sizeof(int), s));
        CUDA_TRY(cudaMemsetAsync(&c->st->band_count, 0, 2 * sizeof(unsigned), s));
        const double* rtau = static_cast<const double*>(r->res_tau.p);
        const int* rtid = static_cast<const int*>(r->res_tid.p);
        TRY(count_stage(c, ps, n, uo, it, true, 0, (int)it.tiles, false, x, rtau, rtid, cnt, band, s));
        TRY(band_stage(c, it, true, x, rtau, rtid, cnt, band, s));
        scatter_i32(cnt, it.perm, q, counts, s);
        TRY(read_status(c, s));
        if (!c->st_host->band_overflow) break;
        if (attempt >= 3) return fail(RKM_EOVERFLOW, "band queue overflowed");
        c->band_cap = grown_band_cap(c);
        c->stats.retries++;
        CUDA_TRY(cudaMemsetAsync(&c->st->band_overflow, 0, sizeof(unsigned), s));
    }
    if (c->st_host->internal_error) return fail(RKM_EINTERNAL, "query: device consistency check failed");
    c->stats.pairs_total = (uint64_t)n * (uint64_t)q;
    c->stats.pairs_evaluated = c->st_host->pairs_evaluated;
    c->stats.band_pairs = c->st_host->band_count;
    c->stats.exact_integer_path = c->st_host->off_grid ? 0 : 1;
    c->stats.last_ms = now_ms() - t0;
    return RKM_OK;
}


extern "C" {

void rkm_default_opts(rkm_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = RKM_BF16;
    o->k_max = KMAX;
    o->cand_capacity = 0;
    o->band_capacity = 0;
    o->filter = 1;
    o->profile = 0;
    o->autotune = 0;
    o->tune_cache = nullptr;
    o->scores_from_topk = 0;
    o->epilogue_groups = 0;
    o->seed_order = 1;
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
    if (o.epilogue_groups != 0 && o.epilogue_groups != 2 && o.epilogue_groups != 4)
        return fail(RKM_EINVAL, "epilogue_groups must be 0, 2 or 4");
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
    if (o.tune_cache) c->tune_cache = o.tune_cache;
    c->opts.tune_cache = nullptr;
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
    for (rkm_ctx* sc : c->sub) rkm_destroy(sc);
    c->sub.clear();
    c->free_all();
    if (c->st) cudaFree(c->st);
    if (c->st_host) cudaFreeHost(c->st_host);
    delete c;
}

rkm_status rkm_get_stats(const rkm_ctx* c, rkm_stats* out) {
    CtxLock lock_(c);
    if (!c || !out) return fail(RKM_EINVAL, "null argument");
    *out = c->stats;
    return RKM_OK;
}

rkm_status rkm_thresholds(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, const float* P, int64_t m,
                          int64_t ldp, int d, int k, double* tau, int32_t* tid, int32_t* topk, void* stream) {
    CtxLock lock_(c);
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

// Counting pass of one problem, split like the threshold pass: prepare (user ratios, their
// bucket order, packs and records), then enqueue one attempt (stages, band rescoring, top-N)
// without waiting for the device.
struct CountPlan {
    UserOrder uo;
    ExactData x;
    int* cnt;
};

rkm_status count_prepare(rkm_ctx* c, const PathShape& ps, const float* U, int64_t n, int64_t ldu, const float* P,
                         int64_t ldp, int d, const RowPrep& up, const ItemSide& it, const double* tau,
                         const int32_t* tid, CountPlan* cp, cudaStream_t s) {
    {
        Phase ph(c, s, RKM_PHASE_BOUNDS);
        TRY(order_users(c, ps, U, n, ldu, d, up, tau, tid, UserBufs{c->uperm, c->ucum, c->us_pack, c->us_meta},
                        &cp->uo, s));
    }
    cp->x = ExactData{U, ldu, up.e, up.q, P, ldp, it.rp.e, it.rp.q, d, (int)round_up(d, 8), &c->st->off_grid,
                      n, it.m};
    TRY(c->ensure(c->cnt_s, it.m, &cp->cnt));
    return RKM_OK;
}

rkm_status count_enqueue(rkm_ctx* c, const PathShape& ps, int64_t n, const ItemSide& it, const CountPlan& cp,
                         const double* tau, const int32_t* tid, int N, int32_t* scores, int32_t* ids,
                         int32_t* top_scores, bool filter, cudaStream_t s) {
    const UserOrder& uo = cp.uo;
    const ExactData& x = cp.x;
    int* cnt = cp.cnt;
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
        return RKM_OK;
    }
    // First stage: enough leading tiles (largest norms, so largest bounds) to hold N items
    // and a few thousand more; its N-th score is an exact lower bound of the final one.
    const int64_t c0 = std::max<int64_t>(4 * (int64_t)N, c->stage1_items);
    const int t0 = (int)std::min<int64_t>(tiles, (c0 + ps.item_tile - 1) / ps.item_tile);
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
    return RKM_OK;
}

// Grow the band queue after an overflow.
rkm_status grow_band(rkm_ctx* c, int attempt) {
    if (attempt >= 3) return fail(RKM_EOVERFLOW, "band queue (%lld pairs) overflowed", (long long)c->band_cap);
    c->band_cap = grown_band_cap(c);
    c->stats.retries++;
    return RKM_OK;
}

static rkm_status scores_impl(rkm_ctx* c, const PathShape& ps, const float* U, int64_t n, int64_t ldu,
                              const float* P, int64_t ldp, int d, const RowPrep& up, const ItemSide& it,
                              const double* tau, const int32_t* tid, int N, int32_t* scores, int32_t* ids,
                              int32_t* top_scores, bool filter, cudaStream_t s) {
    CountPlan cp;
    TRY(count_prepare(c, ps, U, n, ldu, P, ldp, d, up, it, tau, tid, &cp, s));
    for (int attempt = 0;; ++attempt) {
        TRY(count_enqueue(c, ps, n, it, cp, tau, tid, N, scores, ids, top_scores, filter, s));
        TRY(read_status(c, s));
        if (!c->st_host->band_overflow) break;
        TRY(grow_band(c, attempt));
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
    CtxLock lock_(c);
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
    c->stats.exact_integer_path = c->st_host->off_grid ? 0 : 1;
    c->stats.last_ms = now_ms() - t0;
    return RKM_OK;
}

rkm_status rkm_topn(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, const float* P, int64_t m, int64_t ldp,
                    int d, int k, int N, int32_t* ids, int32_t* top_scores, double* tau_out, int32_t* tid_out,
                    void* stream) {
    CtxLock lock_(c);
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
    if (c->opts.scores_from_topk) {
        // Scores as the histogram of S_k(u) (the first Section 2.2 baseline): the threshold
        // pass already ranks every user's candidates exactly, so it writes S_k(u) and the
        // counting pass is not needed.
        int *topk, *cnt;
        TRY(c->ensure(c->topk_tmp, n * (int64_t)k, &topk));
        TRY(c->ensure(c->cnt_s, m, &cnt));
        TRY(thresholds_core(c, ps, U, n, ldu, P, ldp, d, k, up, it, tau, tid, topk, s));
        {
            Phase ph(c, s, RKM_PHASE_COUNT);
            CUDA_TRY(cudaMemsetAsync(cnt, 0, m * sizeof(int), s));
            launch_histogram(topk, n * (int64_t)k, cnt, s);
        }
        {
            Phase ph(c, s, RKM_PHASE_TOPN);
            launch_topn(cnt, nullptr, m, nullptr, N, ids, top_scores, c->st, s);
        }
        TRY(read_status(c, s));
        if (c->st_host->internal_error) return fail(RKM_EINTERNAL, "top-N: device consistency check failed");
        c->stats.items_counted = (uint64_t)m;
        c->stats.pairs_total = (uint64_t)n * (uint64_t)m;
        c->stats.pairs_evaluated = c->stats.threshold_pairs;
        c->stats.last_ms = now_ms() - t0;
        return RKM_OK;
    }
    TRY(thresholds_core(c, ps, U, n, ldu, P, ldp, d, k, up, it, tau, tid, nullptr, s));
    const uint64_t cands = c->stats.candidates, thr_pairs = c->stats.threshold_pairs;
    TRY(scores_impl(c, ps, U, n, ldu, P, ldp, d, up, it, tau, tid, N, nullptr, ids, top_scores,
                    c->opts.filter != 0, s));
    c->stats.candidates = cands;
    c->stats.threshold_pairs = thr_pairs;
    c->stats.pairs_total = 2ull * (uint64_t)n * (uint64_t)m;
    c->stats.pairs_evaluated += thr_pairs;
    c->stats.last_ms = now_ms() - t0;
    return RKM_OK;
}

rkm_status rkm_topn_from_topk(rkm_ctx* c, const int32_t* lists, int64_t n, int kmax, int k, int64_t m, int N,
                              int32_t* ids, int32_t* top_scores, void* stream) {
    CtxLock lock_(c);
    if (!c) return fail(RKM_EINVAL, "null context");
    if (n < 0 || n > (int64_t)INT32_MAX) return fail(RKM_EINVAL, "n must be in [0, 2^31-1]");
    if (n > 0 && !lists) return fail(RKM_EINVAL, "null lists");
    if (m < 1 || m > (int64_t)INT32_MAX) return fail(RKM_EINVAL, "m must be in [1, 2^31-1]");
    if (kmax < 1 || k < 1 || k > kmax || k > m)
        return fail(RKM_EINVAL, "k must satisfy 1 <= k <= min(kmax, m) (k=%d, kmax=%d)", k, kmax);
    if (N < 1 || N > m || N > NMAX_TOPN)
        return fail(RKM_EINVAL, "N must satisfy 1 <= N <= min(m, %d) (N=%d)", NMAX_TOPN, N);
    if (!ids || !top_scores) return fail(RKM_EINVAL, "null ids/top_scores");
    CUDA_TRY(cudaSetDevice(c->device));
    const double t0 = now_ms();
    reset_stats(c);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TRY(begin_call(c, s));
    int* cnt;
    TRY(c->ensure(c->cnt_s, m, &cnt));
    {
        Phase ph(c, s, RKM_PHASE_COUNT);
        CUDA_TRY(cudaMemsetAsync(cnt, 0, m * sizeof(int), s));
        launch_histogram_prefix(lists, n, kmax, k, m, cnt, c->st, s);
    }
    {
        Phase ph(c, s, RKM_PHASE_TOPN);
        launch_topn(cnt, nullptr, m, nullptr, N, ids, top_scores, c->st, s);
    }
    TRY(read_status(c, s));
    if (c->st_host->internal_error) return fail(RKM_EINVAL, "lists hold an id outside [0, m) or top-N failed");
    c->stats.items_counted = (uint64_t)m;
    c->stats.last_ms = now_ms() - t0;
    return RKM_OK;
}

rkm_status rkm_topn_host(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, const float* P, int64_t m,
                         int64_t ldp, int d, int k, int N, int32_t* ids, int32_t* top_scores, void* stream) {
    CtxLock lock_(c);
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
    {
        Phase ph(c, s, RKM_PHASE_TRANSFER);
        if (n > 0) CUDA_TRY(cudaMemcpyAsync(dU, U, n * ldu * sizeof(float), cudaMemcpyHostToDevice, s));
        if (m > 0) CUDA_TRY(cudaMemcpyAsync(dP, P, m * ldp * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    TRY(rkm_topn(c, dU, n, ldu, dP, m, ldp, d, k, N, dids, dsc, nullptr, nullptr, stream));
    {
        Phase ph(c, s, RKM_PHASE_TRANSFER);
        CUDA_TRY(cudaMemcpyAsync(ids, dids, N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaMemcpyAsync(top_scores, dsc, N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    collect_phases(c);
    return RKM_OK;
}

rkm_status rkm_item_bounds(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, const float* P, int64_t m,
                           int64_t ldp, int d, const double* tau, int32_t* uscore, void* stream) {
    CtxLock lock_(c);
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
    TRY(prep_rows(c, ps, P, m, ldp, d, c->p_e, c->p_q, c->p_n2, c->p_nrm, c->p_nhat, c->p_del, &pp, s, true));
    float* r;
    unsigned *hist, *offs, *ucum;
    int* uperm;
    TRY(c->ensure(c->r_u, std::max<int64_t>(n, 1), &r));
    TRY(c->ensure(c->hist, HIST_WORDS, &hist));
    TRY(c->ensure(c->offs, NBUCKET, &offs));
    TRY(c->ensure(c->uperm, std::max<int64_t>(n, 1), &uperm));
    TRY(c->ensure(c->ucum, NBUCKET, &ucum));
    launch_user_ratio(tau, up.n2, n, r, s);
    launch_bucket_sort(r, n, false, hist, offs, uperm, ucum, s);
    launch_item_uscore(pp.nrm, m, ucum, uscore, s);
    TRY(read_status(c, s));
    return RKM_OK;
}

rkm_status rkm_debug_products(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, const float* P, int64_t m,
                              int64_t ldp, int d, float* v, float* E, int64_t ldo, void* stream) {
    CtxLock lock_(c);
    TRY(check_common(c, d));
    TRY(check_matrix(U, n, ldu, d, "U"));
    TRY(check_matrix(P, m, ldp, d, "P"));
    if (c->opts.precision == RKM_FP32) return fail(RKM_EINVAL, "rkm_debug_products: tensor-core paths only");
    if (n > 65536 || m > 1048576) return fail(RKM_EINVAL, "rkm_debug_products: n <= 65536 and m <= 2^20");
    if (ldo < m) return fail(RKM_EINVAL, "rkm_debug_products: ldo < m");
    if (n > 0 && m > 0 && (!v || !E)) return fail(RKM_EINVAL, "null v/E");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    reset_stats(c);
    if (n == 0 || m == 0) return RKM_OK;
    TRY(begin_call(c, s));
    const PathShape ps = path_shape(c->opts.precision, d);
    RowPrep up;
    ItemSide it;
    TRY(prep_rows(c, ps, U, n, ldu, d, c->u_e, c->u_q, c->u_n2, c->u_nrm, c->u_nhat, c->u_del, &up, s));
    TRY(prep_items(c, ps, P, m, ldp, d, catalogue_bufs(c), &it, s));
    const int64_t n_pad = round_up(n, BU);
    void* apack;
    TRY(pack(c, ps, U, n, ldu, d, nullptr, n_pad, c->u_pack, &apack, s, up.e));
    TmapPair tm;
    TRY(make_tmaps(apack, n_pad, it.pack, it.m_pad, ps.dp, BI_TC, ps.elem_bytes, &tm));
    ProductsArgs a{};
    a.n = n;
    a.m = m;
    a.ldo = ldo;
    a.dp = ps.dp;
    a.perm = it.perm;
    a.unrm = up.nrm;
    a.unhat = up.nhat;
    a.udel = up.del;
    a.uexp = up.e;
    a.thmax = it.thmax;
    a.tdel = it.tdel;
    a.texp = it.texp;
    a.cacc = ps.cacc;
    a.eabs = ps.eabs;
    a.v = v;
    a.E = E;
    a.st = c->st;
    launch_products_tc(a, &tm.a, &tm.b, ps.fp8, s);
    TRY(read_status(c, s));
    if (c->st_host->internal_error)
        return fail(RKM_EINTERNAL, "rkm_debug_products: a TMEM load's row maximum differs from its values");
    return RKM_OK;
}

rkm_status rkm_debug_wait_timeout(rkm_ctx* c, int64_t wait_cycles, void* stream) {
    CtxLock lock_(c);
    if (!c) return fail(RKM_EINVAL, "null context");
    if (wait_cycles < 1 || wait_cycles > ((int64_t)1 << 32))
        return fail(RKM_EINVAL, "wait_cycles must be in [1, 2^32]");
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    reset_stats(c);
    TRY(begin_call(c, s));
    launch_wait_timeout((long long)wait_cycles, c->st, s);
    return read_status(c, s);
}

rkm_status rkm_resident_set(rkm_ctx* c, const float* U, int64_t n, int64_t ldu, int d, const double* tau,
                            const int32_t* tid, void* stream) {
    CtxLock lock_(c);
    TRY(check_common(c, d));
    TRY(check_matrix(U, n, ldu, d, "U"));
    if (n > 0 && (!tau || !tid)) return fail(RKM_EINVAL, "null tau/tid");
    if (c->servers.load() != 0) return fail(RKM_ESTATE, "the resident set is in use by a serving loop");
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
    c->res_off_grid = c->st_host->off_grid;
    c->res_n = n;
    c->res_d = d;
    c->resident = true;
    return RKM_OK;
}

rkm_status rkm_state_save(const rkm_ctx* c, const char* path) {
    CtxLock lock_(c);
    if (!c || !path) return fail(RKM_EINVAL, "null context or path");
    if (!c->resident) return fail(RKM_ESTATE, "rkm_state_save before rkm_resident_set");
    CUDA_TRY(cudaSetDevice(c->device));
    const int64_t n = c->res_n;
    const int d = c->res_d;
    std::vector<float> U((size_t)n * d);
    std::vector<double> tau((size_t)n);
    std::vector<int32_t> tid((size_t)n);
    if (n > 0) {
        CUDA_TRY(cudaMemcpy(U.data(), c->res_U.p, U.size() * sizeof(float), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(tau.data(), c->res_tau.p, tau.size() * sizeof(double), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(tid.data(), c->res_tid.p, tid.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    }
    std::string err;
    if (!state::write(path, n, d, U.data(), tau.data(), tid.data(), &err)) return fail(RKM_EIO, "%s", err.c_str());
    return RKM_OK;
}

rkm_status rkm_state_load(rkm_ctx* c, const char* path, void* stream) {
    CtxLock lock_(c);
    if (!c || !path) return fail(RKM_EINVAL, "null context or path");
    if (c->servers.load() != 0) return fail(RKM_ESTATE, "the resident set is in use by a serving loop");
    int64_t n = 0;
    int d = 0;
    std::vector<float> U;
    std::vector<double> tau;
    std::vector<int32_t> tid;
    std::string err;
    if (!state::read(path, &n, &d, &U, &tau, &tid, &err)) return fail(RKM_EIO, "%s", err.c_str());
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* Ud;
    double* taud;
    int* tidd;
    TRY(c->ensure(c->h_U, std::max<int64_t>(n * d, 1), &Ud));
    TRY(c->ensure(c->tau_tmp, std::max<int64_t>(n, 1), &taud));
    TRY(c->ensure(c->tid_tmp, std::max<int64_t>(n, 1), &tidd));
    if (n > 0) {
        CUDA_TRY(cudaMemcpyAsync(Ud, U.data(), U.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(taud, tau.data(), tau.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(tidd, tid.data(), tid.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    // rkm_resident_set synchronises the stream before it returns, so the host vectors
    // outlive the copies.
    return rkm_resident_set(c, Ud, n, d, d, taud, tidd, stream);
}

rkm_status rkm_query_new_items(rkm_ctx* c, const float* Q, int64_t q, int64_t ldq, int32_t* counts, void* stream) {
    CtxLock lock_(c);
    if (!c) return fail(RKM_EINVAL, "null context");
    return rkm::query_resident(c, c, Q, q, ldq, counts, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

// ---------------------------------------------------------------- batches

namespace {

rkm_ctx* make_sub(const rkm_ctx* parent) {
    rkm_ctx* c = new rkm_ctx();
    c->device = parent->device;
    c->opts = parent->opts;
    c->opts.profile = 0;
    c->num_sms = parent->num_sms;
    if (cudaMalloc(&c->st, sizeof(DevStatus)) != cudaSuccess ||
        cudaMallocHost(&c->st_host, sizeof(DevStatus)) != cudaSuccess) {
        cudaGetLastError();
        if (c->st) cudaFree(c->st);
        delete c;
        return nullptr;
    }
    return c;
}

}  // namespace

rkm_ctx* rkm::worker_context(const rkm_ctx* parent) { return make_sub(parent); }

bool rkm::resident_shape(const rkm_ctx* c, int64_t* n, int* d, int* device) {
    if (!c || !c->resident) return false;
    *n = c->res_n;
    *d = c->res_d;
    *device = c->device;
    return true;
}

void rkm::attach_server(rkm_ctx* c, int delta) { c->servers.fetch_add(delta); }

rkm_status rkm::fail_with(rkm_status s, const char* msg) { return fail(s, "%s", msg); }

unsigned long long rkm::launch_count() { return g_launches.load(); }

namespace {

struct InstWork {
    PathShape ps;
    RowPrep up;
    ItemSide it;
    ThrPlan pl;
    CountPlan cp;
    double* tau;
    int* tid;
};

int64_t instance_cost(const rkm_instance& I, const PathShape& ps) {
    return ((I.n + BU - 1) / BU) * ((I.m + BI_TC - 1) / BI_TC) * (ps.dp / 64);
}

// Pinned staging and device arrays of a batch's job and counting descriptors.
rkm_status batch_job_arrays(rkm_ctx* c, int count, BatchJob** jd, CountInstance** cd) {
    if (c->jobs_cap < count) {
        if (c->jobs_host) cudaFreeHost(c->jobs_host);
        if (c->bcount_host) cudaFreeHost(c->bcount_host);
        c->jobs_host = nullptr;
        c->bcount_host = nullptr;
        c->jobs_cap = 0;
        if (cudaMallocHost(&c->jobs_host, (size_t)count * sizeof(BatchJob)) != cudaSuccess ||
            cudaMallocHost(&c->bcount_host, 2 * (size_t)count * sizeof(CountInstance)) != cudaSuccess) {
            cudaGetLastError();
            return fail(RKM_ENOMEM, "pinned batch descriptors for %d instances", count);
        }
        c->jobs_cap = count;
    }
    TRY(c->ensure(c->jobs_dev, count, jd));
    TRY(c->ensure(c->bcount_dev, 2 * (int64_t)count, cd));
    return RKM_OK;
}

// The steps after the threshold launch of a tensor-core batch, as launches over all
// instances: exact thresholds (one launch); per instance the K4 user order (it needs that
// instance's thresholds); then one launch each for clearing the counts, the first-stage unit
// lists, the first counting stage (persistent, over every instance's units), band rescoring,
// the first-stage top-N, the filter cut, the second-stage unit lists, the second counting
// stage, band rescoring and the final top-N.
rkm_status batch_enqueue_tc(rkm_ctx* c, const rkm_instance* inst, int count, std::vector<InstWork>& w,
                            int max_dp, cudaStream_t s) {
    BatchJob* jd;
    CountInstance* cd;
    TRY(batch_job_arrays(c, count, &jd, &cd));
    BatchJob* J = c->jobs_host;
    int64_t users = 0, max_m = 1;
    for (int i = 0; i < count; ++i) {
        rkm_ctx* sc = c->sub[i];
        const rkm_instance& I = inst[i];
        const InstWork& x = w[i];
        BatchJob& j = J[i];
        j = BatchJob{};
        j.x = ExactData{I.U, I.ldu, x.up.e, x.up.q, I.P, I.ldp, x.it.rp.e, x.it.rp.q, I.d, (int)round_up(I.d, 8),
                        &sc->st->off_grid, I.n, I.m};
        j.cand = x.pl.cand;
        j.cand_cnt = x.pl.cand_cnt;
        j.lfin = x.pl.lfin;
        j.cap = x.pl.cap;
        j.nseg = x.pl.nseg;
        j.item_perm = x.it.perm;
        j.n = I.n;
        j.m = I.m;
        j.k = I.k;
        j.N = I.N;
        j.keys = x.pl.keys;
        j.kid = x.pl.kid;
        j.tau = x.tau;
        j.tid = x.tid;
        j.user_begin = users;
        j.st = sc->st;
        users += I.n;
        max_m = std::max<int64_t>(max_m, I.m);
    }
    // The exact thresholds read only the fields set so far; the later copy of the completed
    // jobs only adds fields, so either copy may read the staging at any time.
    CUDA_TRY(cudaMemcpyAsync(jd, J, (size_t)count * sizeof(BatchJob), cudaMemcpyHostToDevice, s));
    launch_exact_tau_multi(jd, count, users, s);
    const bool fp8 = w[0].ps.fp8;
    for (int i = 0; i < count; ++i) {
        rkm_ctx* sc = c->sub[i];
        const rkm_instance& I = inst[i];
        InstWork& x = w[i];
        BatchJob& j = J[i];
        TRY(count_prepare(sc, x.ps, I.U, I.n, I.ldu, I.P, I.ldp, I.d, x.up, x.it, x.tau, x.tid, &x.cp, s));
        int2* band;
        TRY(ensure_band(sc, &band));
        TRY(sc->ensure(sc->nprefix, std::max<int64_t>(x.it.tiles, 1), &j.nprefix));
        TRY(sc->ensure(sc->unit_off, x.it.tiles + 2, &j.unit_off));
        TRY(sc->ensure(sc->top_ids, I.N, &j.top_ids_c0));
        TRY(sc->ensure(sc->top_sc, I.N, &j.top_sc_c0));
        const int tiles = (int)x.it.tiles;
        const int64_t c0 = std::max<int64_t>(4 * (int64_t)I.N, sc->stage1_items);
        j.tmax = x.it.tmax;
        j.ucum = x.cp.uo.ucum;
        j.tiles = tiles;
        j.t0 = c->opts.filter ? (int)std::min<int64_t>(tiles, (c0 + x.ps.item_tile - 1) / x.ps.item_tile) : tiles;
        j.tile_items = x.ps.item_tile;
        j.group = sc->count_group;
        j.counts = x.cp.cnt;
        j.band = band;
        j.band_cap = (unsigned)sc->band_cap;
        j.ids = I.ids;
        j.top_scores = I.top_scores;
        CountArgs a{};
        a.A = x.cp.uo.pack;
        a.B = x.it.pack;
        a.n = I.n;
        a.m = x.it.m;
        a.dp = x.ps.dp;
        a.meta = x.cp.uo.meta;
        a.item_id = x.it.perm;
        a.new_items = false;
        a.tmax = x.it.tmax;
        a.thmax = x.it.thmax;
        a.tdel = x.it.tdel;
        a.texp = x.it.texp;
        a.nprefix = j.nprefix;
        a.unit_off = j.unit_off;
        a.group = j.group;
        a.groups = 2;  // the batch's counting launch runs two epilogue warpgroups
        a.cacc = x.ps.cacc;
        a.eabs = x.ps.eabs;
        a.counts = j.counts;
        a.band = band;
        a.band_cap = j.band_cap;
        a.st = sc->st;
        a.num_sms = c->num_sms;
        for (int stage = 0; stage < 2; ++stage) {
            a.t_begin = stage == 0 ? 0 : j.t0;
            TRY(count_descriptor(x.ps, I.n, x.cp.uo, x.it, a, &c->bcount_host[stage * count + i]));
        }
    }
    CUDA_TRY(cudaMemcpyAsync(jd, J, (size_t)count * sizeof(BatchJob), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(cd, c->bcount_host, 2 * (size_t)count * sizeof(CountInstance), cudaMemcpyHostToDevice,
                             s));
    launch_batch_reset(jd, count, max_m, s);
    for (int stage = 1; stage <= 2; ++stage) {
        CountInstance* ci = cd + (stage - 1) * count;
        launch_build_units_multi(jd, count, stage, s);
        launch_count_prefix(ci, count, &c->st->launch_units, s);
        launch_count_tc_multi(ci, count, &c->st->launch_units, max_dp, fp8, c->num_sms, s);
        launch_band_multi(jd, count, s);
        launch_topn_multi(jd, count, stage, s);
        if (stage == 1) launch_filter_cut_multi(jd, count, s);
    }
    return RKM_OK;
}

// Every kernel of a batch, in order, on one stream, without host waits (so that the sequence
// can be captured into a graph): per instance prep and threshold arguments; one threshold
// launch over all instances (largest first); then the remaining steps (one launch over all
// instances each on the tensor-core paths, per instance on the FP32 path).
rkm_status batch_enqueue(rkm_ctx* c, const rkm_instance* inst, int count, cudaStream_t s) {
    std::vector<InstWork> w(count);
    // Every instance of the persistent threshold launch has one candidate segment per
    // epilogue warpgroup of that launch, chosen for the batch's largest k and depth.
    int kheap = 1, max_dp = 64;
    for (int i = 0; i < count; ++i) {
        kheap = std::max(kheap, inst[i].k);
        max_dp = std::max(max_dp, path_shape(c->opts.precision, inst[i].d).dp);
    }
    const PathShape ps0 = path_shape(c->opts.precision, inst[0].d);
    const int nseg = ps0.tc ? threshold_groups(kheap, max_dp, ps0.fp8, c->opts.epilogue_groups) : 1;
    for (int i = 0; i < count; ++i) {
        rkm_ctx* sc = c->sub[i];
        const rkm_instance& I = inst[i];
        InstWork& x = w[i];
        x.ps = path_shape(c->opts.precision, I.d);
        init_caps(sc, I.n, I.k);
        TRY(begin_call(sc, s));
        TRY(prep_rows(sc, x.ps, I.U, I.n, I.ldu, I.d, sc->u_e, sc->u_q, sc->u_n2, sc->u_nrm, sc->u_nhat, sc->u_del,
                      &x.up, s));
        TRY(prep_items(sc, x.ps, I.P, I.m, I.ldp, I.d, catalogue_bufs(sc), &x.it, s));
        TRY(threshold_prepare(sc, x.ps, I.U, I.n, I.ldu, I.d, I.k, x.up, x.it, &x.pl, s, nseg));
        TRY(sc->ensure(sc->tau_tmp, I.n, &x.tau));
        TRY(sc->ensure(sc->tid_tmp, I.n, &x.tid));
    }
    if (w[0].ps.tc) {
        std::vector<int> order(count);
        for (int i = 0; i < count; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return instance_cost(inst[x], w[x].ps) > instance_cost(inst[y], w[y].ps);
        });
        if (c->batch_host_cap < count) {
            if (c->batch_host) cudaFreeHost(c->batch_host);
            c->batch_host = nullptr;
            c->batch_host_cap = 0;
            CUDA_TRY(cudaMallocHost(&c->batch_host, (size_t)count * sizeof(TcInstance)));
            c->batch_host_cap = count;
        }
        TcInstance* dev;
        TRY(c->ensure(c->batch_dev, count, &dev));
        long long units = 0;
        for (int j = 0; j < count; ++j) {
            const int i = order[j];
            TRY(threshold_descriptor(w[i].ps, w[i].pl, w[i].it, &c->batch_host[j]));
            c->batch_host[j].unit_begin = units;
            units += (inst[i].n + BU - 1) / BU;
        }
        CUDA_TRY(cudaMemcpyAsync(dev, c->batch_host, (size_t)count * sizeof(TcInstance), cudaMemcpyHostToDevice, s));
        launch_threshold_tc(dev, count, units, kheap, max_dp, w[0].ps.fp8, nseg, c->num_sms, s);
        return batch_enqueue_tc(c, inst, count, w, max_dp, s);
    } else {
        for (int i = 0; i < count; ++i) launch_threshold_simt(w[i].pl.a, s);
    }
    for (int i = 0; i < count; ++i) {
        rkm_ctx* sc = c->sub[i];
        const rkm_instance& I = inst[i];
        InstWork& x = w[i];
        threshold_exact(sc, I.U, I.ldu, I.P, I.ldp, I.d, x.up, x.it, x.pl, x.tau, x.tid, nullptr, s);
        TRY(count_prepare(sc, x.ps, I.U, I.n, I.ldu, I.P, I.ldp, I.d, x.up, x.it, x.tau, x.tid, &x.cp, s));
        TRY(count_enqueue(sc, x.ps, I.n, x.it, x.cp, x.tau, x.tid, I.N, nullptr, I.ids, I.top_scores,
                          c->opts.filter != 0, s));
    }
    return RKM_OK;
}

bool same_layout(const std::vector<rkm_instance>& key, const rkm_instance* inst, int count) {
    if ((int)key.size() != count) return false;
    for (int i = 0; i < count; ++i) {
        const rkm_instance& a = key[i];
        const rkm_instance& b = inst[i];
        if (a.U != b.U || a.n != b.n || a.ldu != b.ldu || a.P != b.P || a.m != b.m || a.ldp != b.ldp ||
            a.d != b.d || a.k != b.k || a.N != b.N || a.ids != b.ids || a.top_scores != b.top_scores)
            return false;
    }
    return true;
}

void drop_graph(rkm_ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_key.clear();
}

// ---- autotuner: counting work-unit size and first-stage size per size bucket

struct TuneChoice {
    int group;
    int64_t stage1;
};

std::string tune_bucket(const rkm_instance& I, int prec) {
    auto lg = [](int64_t x) { int b = 0; while ((int64_t(1) << (b + 1)) <= x) ++b; return b; };
    char buf[96];
    snprintf(buf, sizeof buf, "p%d_d%d_k%d_n%d_m%d", prec, I.d, I.k, lg(I.n) / 2, lg(I.m) / 2);
    return buf;
}

void load_tune_table(rkm_ctx* c) {
    if (c->tune_loaded) return;
    c->tune_loaded = true;
    if (c->tune_cache.empty()) return;
    // One bucket per line: key, work-unit size, first-stage items.
    std::ifstream f(c->tune_cache);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream ls(line);
        std::string key;
        int g = 0;
        long long s1 = 0;
        if (ls >> key >> g >> s1) c->tune[key] = {g, (int64_t)s1};
    }
}

void save_tune_table(const rkm_ctx* c) {
    if (c->tune_cache.empty()) return;
    std::ofstream f(c->tune_cache);
    for (const auto& kv : c->tune)
        f << kv.first << " " << kv.second.group << " " << kv.second.stage1 << "\n";
}

// Time rkm_topn on this instance for each candidate and keep the fastest.
rkm_status tune_instance(rkm_ctx* sc, const rkm_instance& I, cudaStream_t s, TuneChoice* best) {
    static const int groups[] = {8, 16, 32};
    static const int64_t stages[] = {4096, 16384};
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    auto run = [&](float* ms) -> rkm_status {
        for (int rep = 0; rep < 2; ++rep) {  // the first run may grow the workspace
            cudaEventRecord(e0, s);
            const rkm_status r = rkm_topn(sc, I.U, I.n, I.ldu, I.P, I.m, I.ldp, I.d, I.k, I.N, I.ids, I.top_scores,
                                          nullptr, nullptr, s);
            cudaEventRecord(e1, s);
            if (r != RKM_OK) return r;
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(ms, e0, e1);
        }
        return RKM_OK;
    };
    float best_ms = 1e30f;
    *best = TuneChoice{32, 8192};
    rkm_status r = RKM_OK;
    for (int g : groups) {
        for (int64_t st1 : stages) {
            sc->count_group = g;
            sc->stage1_items = st1;
            float ms = 0.f;
            if ((r = run(&ms)) != RKM_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                *best = TuneChoice{g, st1};
            }
        }
        if (r != RKM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r;
}

}  // namespace

extern "C" rkm_status rkm_topn_batch(rkm_ctx* c, const rkm_instance* inst, int count, void* stream) {
    CtxLock lock_(c);
    if (!c) return fail(RKM_EINVAL, "null context");
    if (!inst || count < 1 || count > 4096) return fail(RKM_EINVAL, "count must be in [1, 4096]");
    const double t0 = now_ms();
    for (int i = 0; i < count; ++i) {
        const rkm_instance& I = inst[i];
        TRY(check_common(c, I.d));
        TRY(check_matrix(I.U, I.n, I.ldu, I.d, "U"));
        TRY(check_matrix(I.P, I.m, I.ldp, I.d, "P"));
        if (I.n < 1) return fail(RKM_EINVAL, "instance %d: n must be >= 1", i);
        if (I.k < 1 || I.k > I.m || I.k > c->opts.k_max) return fail(RKM_EINVAL, "instance %d: bad k", i);
        if (I.N < 1 || I.N > I.m || I.N > NMAX_TOPN) return fail(RKM_EINVAL, "instance %d: bad N", i);
        if (!I.ids || !I.top_scores) return fail(RKM_EINVAL, "instance %d: null outputs", i);
        if (path_shape(c->opts.precision, I.d).tc != path_shape(c->opts.precision, inst[0].d).tc)
            return fail(RKM_EINVAL, "instances must share one precision path");
    }
    reset_stats(c);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    while ((int)c->sub.size() < count) {
        rkm_ctx* sc = make_sub(c);
        if (!sc) return fail(RKM_ENOMEM, "sub-context allocation failed");
        c->sub.push_back(sc);
    }
    // Tunables per instance (autotuned or default).
    load_tune_table(c);
    bool tuned_any = false;
    for (int i = 0; i < count; ++i) {
        rkm_ctx* sc = c->sub[i];
        const std::string key = tune_bucket(inst[i], (int)c->opts.precision);
        auto f = c->tune.find(key);
        if (f == c->tune.end() && c->opts.autotune) {
            TuneChoice ch;
            TRY(tune_instance(sc, inst[i], s, &ch));
            c->tune[key] = {ch.group, ch.stage1};
            tuned_any = true;
            f = c->tune.find(key);
        }
        const int g = (f != c->tune.end()) ? f->second.group : 32;
        const int64_t s1 = (f != c->tune.end()) ? f->second.stage1 : 8192;
        if (sc->count_group != g || sc->stage1_items != s1) drop_graph(c);
        sc->count_group = g;
        sc->stage1_items = s1;
    }
    if (tuned_any) save_tune_table(c);
    if (!c->bstream) {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->bstream, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&c->bev_in, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&c->bev_out, cudaEventDisableTiming));
    }
    // The batch runs on the internal stream after the caller's prior work.
    CUDA_TRY(cudaEventRecord(c->bev_in, s));
    CUDA_TRY(cudaStreamWaitEvent(c->bstream, c->bev_in, 0));
    cudaStream_t caller = s;
    s = c->bstream;
    const unsigned long long l0 = g_launches.load();
    const int okey = (int)c->opts.precision * 2 + (c->opts.filter ? 1 : 0);
    const bool replay = c->graph_exec && c->graph_opts_key == okey && same_layout(c->graph_key, inst, count);
    if (replay) {
        CUDA_TRY(cudaGraphLaunch(c->graph_exec, s));
    } else {
        drop_graph(c);
        TRY(batch_enqueue(c, inst, count, s));
    }
    for (int i = 0; i < count; ++i)
        CUDA_TRY(cudaMemcpyAsync(c->sub[i]->st_host, c->sub[i]->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    unsigned long long launches = replay ? c->graph_kernels : g_launches.load() - l0;
    // Instances that overflowed a buffer (or failed a check) inside the batch are recomputed by
    // the retrying single-instance path; their workspace may grow, so the graph is rebuilt.  A
    // wait that gave up stops a launch shared by every instance (it is recorded in one
    // instance's status), so then every instance is recomputed.
    bool redo = false, any_timeout = false;
    for (int i = 0; i < count; ++i) any_timeout = any_timeout || c->sub[i]->st_host->timeout != 0u;
    for (int i = 0; i < count; ++i) {
        const DevStatus& st = *c->sub[i]->st_host;
        if (st.cand_overflow || st.band_overflow || st.internal_error || any_timeout) {
            const rkm_instance& I = inst[i];
            const unsigned long long l1 = g_launches.load();
            TRY(rkm_topn(c->sub[i], I.U, I.n, I.ldu, I.P, I.m, I.ldp, I.d, I.k, I.N, I.ids, I.top_scores, nullptr,
                         nullptr, s));
            launches += g_launches.load() - l1;
            c->stats.retries++;
            redo = true;
        }
        c->stats.candidates += st.cand_total;
        c->stats.band_pairs += st.band_count;
        c->stats.threshold_pairs += st.thr_pairs;
        c->stats.pairs_evaluated += st.pairs_evaluated + st.thr_pairs;
        c->stats.pairs_total += 2ull * (uint64_t)inst[i].n * (uint64_t)inst[i].m;
    }
    if (redo) drop_graph(c);
    if (!replay && !redo) {
        // Capture the same sequence for the next call with this layout (buffers are in place,
        // so nothing is allocated while capturing).
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c->stats.kernel_launches = launches;
            c->stats.last_ms = now_ms() - t0;
            return RKM_OK;
        }
        const unsigned long long lc = g_launches.load();
        const rkm_status r = batch_enqueue(c, inst, count, s);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        g_launches.fetch_sub(g_launches.load() - lc);  // nothing ran while capturing
        if (r == RKM_OK && e == cudaSuccess && g) {
            cudaGraphExec_t ex = nullptr;
            if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
                c->graph = g;
                c->graph_exec = ex;
                c->graph_key.assign(inst, inst + count);
                c->graph_opts_key = okey;
                c->graph_kernels = 0;  // the kernel nodes of the graph
                size_t nn = 0;
                cudaGraphGetNodes(g, nullptr, &nn);
                std::vector<cudaGraphNode_t> nodes(nn);
                cudaGraphGetNodes(g, nodes.data(), &nn);
                for (cudaGraphNode_t nd : nodes) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
                        ++c->graph_kernels;
                }
            } else {
                cudaGetLastError();
                cudaGraphDestroy(g);
            }
        } else {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
        }
    }
    c->stats.kernel_launches = launches;
    c->stats.last_ms = now_ms() - t0;
    // Later work on the caller's stream follows the batch.
    CUDA_TRY(cudaEventRecord(c->bev_out, s));
    CUDA_TRY(cudaStreamWaitEvent(caller, c->bev_out, 0));
    return RKM_OK;
}
