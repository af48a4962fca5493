// Tensor-core (tcgen05) product kernels of the threshold pass (K2) and the counting
// pass (K5): BF16 or FP8 e4m3 operands staged by TMA into 128-byte-swizzled shared memory
// (a K-block is 128 bytes of every row: 64 BF16 or 128 FP8 values), one thread issuing
// 128 x 256 x 16 (BF16) or 128 x 256 x 32 (FP8) MMAs into a double-buffered FP32 accumulator in TMEM
// (2 x 256 columns), and NG epilogue warpgroups (NG = 2 or 4) that read the accumulator back
// with tcgen05.ld and run the per-user epilogues of epilogue.cuh.  The user x item product
// never leaves the SM.
//
// Roles (64 + 128 NG threads, one CTA per SM, persistent):
//   warp 0      TMA producer: the resident operand once per work unit, then a ring of
//               K-block slots of the streamed operand.
//   warp 1      TMEM allocator and MMA issuer (one thread).
//   warps 2..   NG epilogue warpgroups.  Group g consumes accumulator buffer g % 2, i.e. every
//               other product tile, and of each such tile the columns
//               [(g / 2) * CW, (g / 2 + 1) * CW), CW = 512 / NG.  With NG = 4 every tile is
//               read by eight warps at once (twice the TMEM loads in flight of NG = 2), which
//               is what keeps the epilogue up with the MMA at small d.
// Threshold pass: resident = 128 users, streamed = 256-item tiles.  Each warpgroup keeps
// its own lower-bound heap per user (each is a valid lower bound of tau_u because it is the
// k-th largest lower bound over a subset of the items); the final L_u is their maximum.
// Counting pass: resident = 256 items, streamed = 128-user tiles of the unit's users.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "count_units.cuh"
#include "epilogue.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"
#include "tmap.h"

namespace rkm {

namespace {

// Threads of a product kernel with NG epilogue warpgroups.
constexpr int tc_threads(int ng) { return 64 + 128 * ng; }
constexpr int MAX_SLOTS = 4;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t KB_BYTES_U = 128 * 128;  // one K-block (128 bytes: 64 BF16 / 128 FP8) of 128 user rows
constexpr uint32_t KB_BYTES_I = 256 * 128;  // one K-block of 256 item rows
constexpr int SMEM_LIMIT = 232448;          // 227 KB opt-in maximum per block

struct TcBars {
    uint64_t res_full[2], res_empty[2], drain;
    uint64_t full[MAX_SLOTS], empty[MAX_SLOTS];
    uint64_t tfull[2], tempty[2];
    uint32_t tmem_base;
    int abort;
    // Threshold pass, early end of a unit (see k_threshold_tc): the producer's end marker in
    // the first ring slot of the tile that is not loaded, the MMA issuer's end markers for the
    // epilogue warps, and each epilogue warp's (unit, item tiles its users still need).
    int slot_mark[MAX_SLOTS];
    int tmark[16];
    unsigned long long need_pub[16];
};

// Threshold pass: the item tile at which a unit may stop.  Each epilogue warp publishes how
// many leading item tiles its 32 users still need; a warpgroup covers all 128 users of the
// unit, so the largest value of a group whose four warps all published for this unit bounds
// the tiles needed, and any group's bound is valid (each uses valid lower bounds of tau_u).
__device__ __forceinline__ int unit_stop(const TcBars* B, unsigned tag, int item_tiles, int ng) {
    int stop = item_tiles;
    for (int g = 0; g < ng; ++g) {
        int mg = 0;
        bool all = true;
        for (int j = 0; j < 4; ++j) {
            const unsigned long long x = *reinterpret_cast<const volatile unsigned long long*>(&B->need_pub[4 * g + j]);
            if ((unsigned)(x >> 32) != tag) {
                all = false;
                break;
            }
            const int v = (int)(unsigned)(x & 0xffffffffull);
            mg = v > mg ? v : mg;
        }
        if (all && mg < stop) stop = mg;
    }
    return stop;
}

// Threshold pass: tell the epilogue warps that read accumulator buffer b that the unit ended
// (mark 1 at the position of the first tile not computed, 2 at the next position).
__device__ __forceinline__ void post_unit_end(TcBars* B, uint32_t b, int mark, int ng) {
    for (int g = (int)b; g < ng; g += 2)
        for (int j = 0; j < 4; ++j) *reinterpret_cast<volatile int*>(&B->tmark[4 * g + j]) = mark;
    mbar_arrive(&B->tfull[b]);
}

struct TcLayout {
    uint32_t res_off, ring_off, aux_off, bar_off, bytes;
    uint32_t slot_bytes, res_bytes;  // one ring slot; one resident-operand buffer
    int slots;                       // ring slots
    int nres;                        // resident-operand buffers (2 = next unit loads during this one)
};

// Values per 128-byte K-block row and the MMA of the operand kind.
template <bool FP8>
struct Operand {
    static constexpr int KELEMS = FP8 ? 128 : 64;
    static constexpr int KSHIFT = FP8 ? 7 : 6;
    static __device__ __forceinline__ uint32_t idesc() { return FP8 ? idesc_e4m3_f32(BU, BI_TC) : idesc_bf16_f32(BU, BI_TC); }
    static __device__ __forceinline__ void mma(uint32_t d, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
        if constexpr (FP8) tc_mma_f8(d, ad, bd, id, acc);
        else tc_mma_bf16(d, ad, bd, id, acc);
    }
};

// 2^k as a float (exact; subnormal below 2^-126).  FP8 operands carry the scales 2^(8-e_u)
// and 2^(8-e_T), so an accumulator times 2^(e_u + e_T - 16) is the product of the descaled
// operands; fp8_exp limits the exponents to [-60, 60], so k stays within [-136, 104].
__device__ __forceinline__ float pow2i(int k) { return k >= -126 ? __int_as_float((k + 127) << 23) : ldexpf(1.f, k); }

template <int N>
__device__ __forceinline__ void scale_values(float (&v)[N], float f) {
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] *= f;
}

__device__ __forceinline__ uint8_t* align1024(uint8_t* raw) {
    const uint32_t a = smem_u32(raw);
    return raw + ((1024u - (a & 1023u)) & 1023u);
}

// Bounded wait that ignores the abort flag (used to drain in-flight copies / MMAs at exit).
__device__ __forceinline__ void drain_wait(uint64_t* bar, uint32_t parity, DevStatus* st) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > RKM_WAIT_CYCLES) {
            st->timeout = 1u;
            return;
        }
    }
}

// consumers: warps that release each accumulator buffer (4 per warpgroup reading it).
__device__ __forceinline__ void setup(TcBars* B, int slots, int warp, int consumers) {
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&B->res_full[b], 1);
            mbar_init(&B->res_empty[b], 1);
        }
        mbar_init(&B->drain, 1);
        for (int s = 0; s < slots; ++s) {
            mbar_init(&B->full[s], 1);
            mbar_init(&B->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&B->tfull[b], 1);
            mbar_init(&B->tempty[b], (uint32_t)consumers);
        }
        B->abort = 0;
        mbar_fence_init();
    }
    if (warp == 1) {
        tmem_alloc(&B->tmem_base, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void teardown(TcBars* B, int warp) {
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(B->tmem_base, TMEM_COLS);
    }
}

// ---------------------------------------------------------------- K2

// Instance of a work unit w (its global user-tile index): the last instance whose first unit
// is <= w (instances are few; a binary search over their first units).
__device__ __forceinline__ int unit_instance(const TcInstance* inst, int count, long long w) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (inst[mid].unit_begin <= w) lo = mid; else hi = mid;
    }
    return lo;
}

// Threshold pass over one or many independent problems.  Work units are (instance, user
// tile) pairs numbered consecutively across the instances; CTA b takes units b, b + grid, ...
// A unit streams every item tile of its instance, so the caller orders the instances by
// descending cost to balance the CTAs.
template <bool FP8, int NG>
__global__ void __launch_bounds__(tc_threads(NG), 1)
    k_threshold_tc(const TcInstance* __restrict__ inst, int count, long long total_units, int kheap,
                   const TcLayout L) {
    using Op = Operand<FP8>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint8_t* sA = sm + L.res_off;
    uint8_t* ring = sm + L.ring_off;
    float* heaps = reinterpret_cast<float*>(sm + L.aux_off);
    TcBars* B = reinterpret_cast<TcBars*>(sm + L.bar_off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = L.slots;
    volatile int* abort = &B->abort;
    // Running bounds published per user row by each epilogue group: Lpub[h][row], tagged with
    // the work unit (a bound of another unit is never used).  Initialised before setup's
    // barrier so that no group can read an uninitialised entry.
    unsigned long long* Lpub = reinterpret_cast<unsigned long long*>(heaps + NG * kheap * BU);
    if (warp >= 2) Lpub[threadIdx.x - 64] = 0xFFFFFFFF00000000ull;
    if (threadIdx.x < 16) {
        B->need_pub[threadIdx.x] = 0xFFFFFFFF00000000ull;
        B->tmark[threadIdx.x] = 0;
        if (threadIdx.x < MAX_SLOTS) B->slot_mark[threadIdx.x] = 0;
    }

    setup(B, S, warp, 2 * NG);
    const uint32_t tmem = B->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int slot = 0;
            uint32_t ph = 0;
            int issued[MAX_SLOTS] = {0, 0, 0, 0};
            int res_loads = 0;
            bool ok = true;
            DevStatus* st = inst[0].a.st;
            for (long long w = blockIdx.x; w < total_units && ok; w += gridDim.x) {
                const TcInstance& I = inst[unit_instance(inst, count, w)];
                st = I.a.st;
                const int KB = I.a.dp >> Op::KSHIFT;
                const long long ut = w - I.unit_begin;
                const int item_tiles = (int)((I.a.m + BI_TC - 1) / BI_TC);
                const int rb = res_loads % L.nres, ru = res_loads / L.nres;
                if (ru > 0 && !mbar_wait(&B->res_empty[rb], (ru - 1) & 1, abort, st)) break;
                uint8_t* dst = sA + rb * L.res_bytes;
                mbar_expect_tx(&B->res_full[rb], KB * KB_BYTES_U);
                for (int kb = 0; kb < KB; ++kb)
                    tma_load_2d(dst + kb * KB_BYTES_U, &I.tmA, &B->res_full[rb], kb * Op::KELEMS, (int)(ut * BU));
                ++res_loads;
                int tiles_done = 0;
                for (int it = 0; it < item_tiles && ok; ++it) {
                    // Stop the unit when no user of it needs the remaining tiles (at least two
                    // remaining, so that both end markers fall inside the unit's tile range):
                    // the first ring slot of tile `it` then carries an end marker, no copy.
                    if (it + 1 < item_tiles && it >= unit_stop(B, (unsigned)w, item_tiles, NG)) {
                        if (!mbar_wait(&B->empty[slot], ph ^ 1u, abort, st)) {
                            ok = false;
                            break;
                        }
                        *reinterpret_cast<volatile int*>(&B->slot_mark[slot]) = -1;
                        mbar_arrive(&B->full[slot]);
                        ++issued[slot];
                        if (++slot == S) {
                            slot = 0;
                            ph ^= 1u;
                        }
                        break;
                    }
                    for (int kb = 0; kb < KB; ++kb) {
                        if (!mbar_wait(&B->empty[slot], ph ^ 1u, abort, st)) {
                            ok = false;
                            break;
                        }
                        if (kb == 0) *reinterpret_cast<volatile int*>(&B->slot_mark[slot]) = 0;
                        mbar_expect_tx(&B->full[slot], KB_BYTES_I);
                        tma_load_2d(ring + slot * KB_BYTES_I, &I.tmB, &B->full[slot], kb * Op::KELEMS, it * BI_TC);
                        ++issued[slot];
                        if (++slot == S) {
                            slot = 0;
                            ph ^= 1u;
                        }
                    }
                    ++tiles_done;
                }
                const int64_t urows = (I.a.n - ut * BU < BU) ? I.a.n - ut * BU : BU;
                const int64_t done_items = ((int64_t)tiles_done * BI_TC < I.a.m) ? (int64_t)tiles_done * BI_TC : I.a.m;
                atomicAdd(&st->thr_pairs, (unsigned long long)(urows * done_items));
            }
            // Copies in flight complete on their barriers; wait for them before the CTA exits.
            for (int s = 0; s < S; ++s)
                if (issued[s] > 0) drain_wait(&B->full[s], (uint32_t)(issued[s] - 1) & 1u, st);
            for (int rb = 0; rb < L.nres; ++rb) {
                const int loads = res_loads / L.nres + (rb < res_loads % L.nres ? 1 : 0);
                if (loads > 0) drain_wait(&B->res_full[rb], (uint32_t)(loads - 1) & 1u, st);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = Op::idesc();
            int slot = 0;
            uint32_t ph = 0, tile_j = 0;
            int iter = 0;
            bool ok = true;
            DevStatus* st = inst[0].a.st;
            for (long long w = blockIdx.x; w < total_units && ok; w += gridDim.x, ++iter) {
                const TcInstance& I = inst[unit_instance(inst, count, w)];
                st = I.a.st;
                const int KB = I.a.dp >> Op::KSHIFT;
                const int item_tiles = (int)((I.a.m + BI_TC - 1) / BI_TC);
                const int rb = iter % L.nres;
                if (!mbar_wait(&B->res_full[rb], (iter / L.nres) & 1, abort, st)) break;
                tc_fence_after();
                const uint8_t* sAr = sA + rb * L.res_bytes;
                for (int it = 0; it < item_tiles && ok; ++it) {
                    const uint32_t b = tile_j & 1u, use = tile_j >> 1;
                    if (!mbar_wait(&B->tempty[b], (use & 1u) ^ 1u, abort, st)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (!mbar_wait(&B->full[slot], ph, abort, st)) {
                        ok = false;
                        break;
                    }
                    if (*reinterpret_cast<volatile int*>(&B->slot_mark[slot]) < 0) {
                        // The producer ended the unit here: release the marker's slot and pass
                        // the end to the epilogue warps of both accumulator buffers.
                        mbar_arrive(&B->empty[slot]);
                        if (++slot == S) {
                            slot = 0;
                            ph ^= 1u;
                        }
                        post_unit_end(B, b, 1, NG);
                        ++tile_j;
                        const uint32_t b2 = tile_j & 1u, use2 = tile_j >> 1;
                        if (!mbar_wait(&B->tempty[b2], (use2 & 1u) ^ 1u, abort, st)) {
                            ok = false;
                            break;
                        }
                        post_unit_end(B, b2, 2, NG);
                        ++tile_j;
                        break;
                    }
                    const uint32_t d = tmem + b * BI_TC;
                    for (int kb = 0; kb < KB; ++kb) {
                        if (kb > 0 && !mbar_wait(&B->full[slot], ph, abort, st)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ad = sdesc_sw128(smem_u32(sAr + kb * KB_BYTES_U));
                        const uint64_t bd = sdesc_sw128(smem_u32(ring + slot * KB_BYTES_I));
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            Op::mma(d, ad + 2u * k, bd + 2u * k, idesc, (kb | k) != 0 ? 1u : 0u);
                        tc_commit(&B->empty[slot]);
                        if (++slot == S) {
                            slot = 0;
                            ph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    tc_commit(&B->tfull[b]);
                    ++tile_j;
                }
                if (!ok) break;
                tc_commit(&B->res_empty[rb]);
            }
            tc_commit(&B->drain);
            drain_wait(&B->drain, 0u, st);
        }
    } else {
        constexpr int CW = 2 * BI_TC / NG;  // accumulator columns a group reads per tile
        const int ew = warp - 2;          // 0 .. 4 NG - 1
        const int g = ew >> 2;            // warpgroup
        const int h = g & 1;              // accumulator buffer it consumes
        const int cg = (g >> 1) * CW;     // its first column of each tile
        const int q = warp & 3;           // TMEM lane quarter this warp may access
        const int r = q * 32 + lane;      // user row of the tile
        float* heap = heaps + g * (kheap * BU);
        uint32_t tile_j = 0;
        bool ok = true;
        for (long long w = blockIdx.x; w < total_units && ok; w += gridDim.x) {
            const TcInstance& I = inst[unit_instance(inst, count, w)];
            const ThresholdArgs& a = I.a;
            const long long ut = w - I.unit_begin;
            const int item_tiles = (int)((a.m + BI_TC - 1) / BI_TC);
            const int64_t u = ut * BU + r;
            // The candidate lists have one segment per warpgroup; an instance prepared for
            // another group count is a host bug: flag it and write nothing.
            if (a.nseg != NG && lane == 0 && q == 0) a.st->internal_error = 1u;
            const bool active = u < a.n && a.nseg == NG;
            for (int j = 0; j < a.k; ++j) heap[j * BU + r] = -INFINITY;
            SelState s;
            s.L = -INFINITY;
            s.hn = 0;
            s.Lw = -INFINITY;
            s.Lx = -INFINITY;
            s.thr = -INFINITY;
            s.cnt = 0;
            s.pub = &Lpub[g * BU + r];
            s.tag = (unsigned)w;
            s.defer = 1;
            s.mark = 0;
            bool warm = false;  // warm start done for this unit
            int fb = item_tiles;       // first tile after the last searched one whose
            float bnd_fb = -INFINITY;  // ||u|| max||p|| is below bnd_fb (see the stop below)
            // Packed row u holds original user uo; a seed bound of tau_u (from a pass over the
            // highest-norm items) starts the selector above -inf.
            const int64_t uo = (active && a.uperm) ? (int64_t)a.uperm[u] : u;
            const float seed = (active && a.lfin_seed) ? key_float(a.lfin_seed[uo]) : -INFINITY;
            s.Lw = seed;
            const float un = active ? a.unrm[uo] : 0.f;
            const float unh = active ? a.unhat[uo] : 0.f;
            const float ud = active ? a.udel[uo] : 0.f;
            const int ue = (FP8 && active) ? fp8_exp(a.uexp[uo]) : 0;
            Cand* mycand = a.cand + ((active ? u : 0) * a.nseg + g) * (int64_t)a.cap;
            // This group's first tile of the unit, then every other one: the bound maxima of
            // the next one are loaded while the current one is processed.
            int itn = (int)((tile_j & 1u) == (uint32_t)h ? 0 : 1);
            float thm_next = 0.f, tdl_next = 0.f;
            if (itn < item_tiles) {
                thm_next = a.thmax[itn];
                tdl_next = a.tdel[itn];
            }
            for (int it = 0; it < item_tiles; ++it) {
                const uint32_t b = tile_j & 1u, use = tile_j >> 1;
                ++tile_j;
                if ((int)b != h) continue;
                const float thm = thm_next, tdl = tdl_next;
                if (it + 2 < item_tiles) {
                    thm_next = a.thmax[it + 2];
                    tdl_next = a.tdel[it + 2];
                }
                if (!mbar_wait(&B->tfull[b], use & 1u, abort, a.st)) {
                    ok = false;
                    break;
                }
                __syncwarp();
                tc_fence_after();
                const int mk = *reinterpret_cast<volatile int*>(&B->tmark[ew]);
                if (mk != 0) {
                    // The unit ended early (end marker 1 or 2 of the MMA issuer, no product in
                    // the buffer): release the buffer and continue the tile count where the
                    // issuer did, two positions after the last computed tile.
                    __syncwarp();
                    if (lane == 0) {
                        *reinterpret_cast<volatile int*>(&B->tmark[ew]) = 0;
                        mbar_arrive(&B->tempty[b]);
                    }
                    if (mk == 1) ++tile_j;
                    break;
                }
                const float E = err_bound(a.cacc, a.eabs, un, unh, ud, thm, tdl);
                const float f = FP8 ? pow2i(ue + a.texp[it] - 16) : 1.f;  // descale of the FP8 product
                // The other groups' bounds may be stale or from this unit's start (-inf):
                // any value they held is a valid lower bound of tau_u for the current user.
                float lx = -INFINITY;
#pragma unroll
                for (int o = 0; o < NG; ++o)
                    if (o != g) lx = fmaxf(lx, read_bound(&Lpub[o * BU + r], (unsigned)w));
                s.Lx = lx;
                const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + b * BI_TC + cg;
                if (!warm) {
                    // First tile of this group for these users: a lockstep first pass over the
                    // accumulator gives a lower bound before any candidate is recorded, so the
                    // heap does not fill one divergent insertion at a time: the k-th largest of
                    // CW / 4 maxima of 4 columns (k <= CW / 4 distinct items reach it; -inf for
                    // a larger k).  Hits of this tile are recorded against it until the tile's
                    // end, so its tightness sets how many candidates the first tile records.
                    auto load = [&](int c0, float (&v)[32]) {
                        __syncwarp();
                        tmem_ld32(tb + c0, v);
                        if constexpr (FP8) scale_values(v, f);
                    };
                    const float lw = warm_bound<CW / 4, CW>(load, it * BI_TC + cg, a.m, a.k, E);
                    s.Lw = active ? fmaxf(lw, seed) : -INFINITY;
                    publish_bound(s.pub, s.tag, s.Lw);
                    warm = true;
                }
                s.thr = __fsub_rd(sel_bound(s), E);
                uint32_t ra[32], rb[32];
                // Both 32-column chunks of a 64-column pair in flight, one vote for the pair.  The
                // loads (tcgen05.ld with .red.max, an sm_103a form) return each chunk's row
                // maximum with its values, so the common case (no value of the pair reaches its
                // row's threshold) costs one maximum, one vote and one branch, with no reduction
                // tree.  Measured on GB300 against max trees over the loaded values: threshold
                // phase 8 % shorter at d = 64 and d = 128.  The FP8 descale f is a positive power
                // of two and rounding is monotone, so max(v f) = max(v) f.
#pragma unroll 1
                for (int c0 = 0; c0 < CW; c0 += 64) {
                    __syncwarp();
                    float ma, mb;
                    tmem_ld32_max_issue(tb + c0, ra, ma);
                    tmem_ld32_max_issue(tb + c0 + 32, rb, mb);
                    tmem_wait_bind_max(ra, ma);
                    tmem_wait_bind_max(rb, mb);
                    const float mx = FP8 ? fmaxf(ma, mb) * f : fmaxf(ma, mb);
                    if (__any_sync(0xffffffffu, active && mx >= s.thr)) {
                        float va[32], vb[32];
                        as_floats(ra, va);
                        as_floats(rb, vb);
                        if constexpr (FP8) {
                            scale_values(va, f);
                            scale_values(vb, f);
                        }
                        sel_chunk(va, active, it * BI_TC + cg + c0, a.m, E, s, mycand, a.cap, heap, r, a.k, a.st);
                        sel_chunk(vb, active, it * BI_TC + cg + c0 + 32, a.m, E, s, mycand, a.cap, heap, r, a.k,
                                  a.st);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&B->tempty[b]);
                // The accumulator is released: admit this tile's candidates while the MMA
                // computes the next tiles.
                sel_merge_tile(s, mycand, heap, r, a.k, E, active);
                // Algorithm 1's stop by Cauchy-Schwarz: items arrive in descending norm order,
                // so once ||u|| max||p|| of a tile (rounded up) is below a lower bound of tau_u,
                // no item of that tile or any later one can reach tau_u or tie it.  Publish how
                // many leading tiles this warp's users still need.
                // The first tile below a bound moves back as the bound grows, so the search
                // is skipped while the bound is unchanged and narrowed to [it + 1, fb] when it
                // grew; the other groups' bounds can make it drop (a group that has moved on
                // publishes for its next unit), and then the whole rest is searched.
                {
                    const float bnd = sel_bound(s);
                    int need = 0;
                    if (active) {
                        if (bnd != bnd_fb || fb < it + 1) {
                            int lo = it + 1, hi = item_tiles;  // first tile below the bound
                            if (bnd >= bnd_fb && fb < hi) hi = fb > lo ? fb : lo;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (__fmul_ru(un, a.tmax[mid]) < bnd) hi = mid; else lo = mid + 1;
                            }
                            fb = lo;
                            bnd_fb = bnd;
                        }
                        need = fb;
                    }
                    need = __reduce_max_sync(0xffffffffu, need);
                    if (lane == 0)
                        *reinterpret_cast<volatile unsigned long long*>(&B->need_pub[ew]) =
                            ((unsigned long long)(unsigned)w << 32) | (unsigned)need;
                }
            }
            if (active) {
                atomicMax(&a.lfin_key[u], float_key(fmaxf(s.L, s.Lw)));
                a.cand_cnt[u * a.nseg + g] = s.cnt;
            }
        }
    }
    teardown(B, warp);
}

// ---------------------------------------------------------------- K5

// Instance of global counting unit w: the last instance whose first unit is <= w.
__device__ __forceinline__ int count_instance(const CountInstance* inst, int count, long long w) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (inst[mid].unit_begin <= w) lo = mid; else hi = mid;
    }
    return lo;
}

// The problems of one counting launch: a single problem passed by value (its arguments and
// TMA maps in the parameter space), or an array of problems in global memory.
template <bool MULTI>
struct CountSet {
    const CountArgs& a0;
    const CUtensorMap* mA0;
    const CUtensorMap* mB0;
    const CountInstance* inst;
    int count;
    __device__ __forceinline__ const CountArgs& args(int i) const { return MULTI ? inst[i].a : a0; }
    __device__ __forceinline__ const CUtensorMap* mapA(int i) const { return MULTI ? &inst[i].tmA : mA0; }
    __device__ __forceinline__ const CUtensorMap* mapB(int i) const { return MULTI ? &inst[i].tmB : mB0; }
    // Global unit w -> problem i, item tile T and user tiles [ut0, ut1) of that problem.
    __device__ __forceinline__ void decode(long long w, int& i, int& T, int64_t& ut0, int64_t& ut1) const {
        i = MULTI ? count_instance(inst, count, w) : 0;
        const long long first = MULTI ? inst[i].unit_begin : 0;
        decode_count_unit(args(i), (unsigned)(w - first), T, ut0, ut1);
    }
};

// Position in a CTA's sequence of counting tiles: unit w (problem i, item tile T), user tile
// ut of [ut0, ut1).  Units are taken as blockIdx.x, blockIdx.x + gridDim.x, ...
struct TileCursor {
    long long w;
    int i, T;
    int64_t ut, ut1;
    bool valid;
};

template <bool MULTI>
__device__ __forceinline__ void cursor_unit(const CountSet<MULTI>& cs, long long total, TileCursor& c) {
    c.valid = c.w < total;
    if (!c.valid) return;
    int64_t ut0;
    cs.decode(c.w, c.i, c.T, ut0, c.ut1);
    c.ut = ut0;
}

template <bool MULTI>
__device__ __forceinline__ void cursor_first(const CountSet<MULTI>& cs, long long total, TileCursor& c) {
    c.w = blockIdx.x;
    cursor_unit(cs, total, c);
}

// Every unit holds at least one user tile, so one step never skips a unit.
template <bool MULTI>
__device__ __forceinline__ void cursor_next(const CountSet<MULTI>& cs, long long total, TileCursor& c) {
    if (!c.valid) return;
    if (++c.ut < c.ut1) return;
    c.w += gridDim.x;
    cursor_unit(cs, total, c);
}

// Add a warp's per-item counters of the CW columns starting at pos0 to the global counts.
template <int CW>
__device__ __forceinline__ void flush_counts(int* cw, int lane, int pos0, int64_t m, int* counts) {
    __syncwarp();
    for (int c = lane; c < CW; c += 32) {
        const int x = cw[c];
        if (x != 0) {
            if (pos0 + c < m) atomicAdd(&counts[pos0 + c], x);
            cw[c] = 0;
        }
    }
    __syncwarp();
}

// Fields of a problem the counting epilogue uses on every tile, kept in registers while the
// epilogue stays on that problem.
struct CountHot {
    int64_t n, m;
    float cacc, eabs;
    int* counts;
    int2* band;
    unsigned band_cap;
    DevStatus* st;
};

__device__ __forceinline__ CountHot count_hot(const CountArgs& a) {
    return CountHot{a.n, a.m, a.cacc, a.eabs, a.counts, a.band, a.band_cap, a.st};
}

// Counting pass over the work units of one problem (MULTI = false: arguments and TMA maps by
// value, units [0, st->units_total)) or of many (MULTI = true: unit w of the launch belongs to
// the problem whose unit range holds it; the ranges are written on the device by
// k_count_prefix from each problem's unit count, so one launch serves every instance of a
// batch).  Resident = 256 items of the unit's tile, streamed = the unit's 128-user tiles.
// Bounded waits record a timeout in the first problem's status word.
template <bool FP8, int NG, bool MULTI>
__global__ void __launch_bounds__(tc_threads(NG), 1)
    k_count_tc(const CountArgs a0, const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmB0,
               const CountInstance* __restrict__ inst, int count, const unsigned long long* __restrict__ total_dev,
               const TcLayout L) {
    using Op = Operand<FP8>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint8_t* sB = sm + L.res_off;
    uint8_t* ring = sm + L.ring_off;
    int* cnt_all = reinterpret_cast<int*>(sm + L.aux_off);
    TcBars* B = reinterpret_cast<TcBars*>(sm + L.bar_off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = L.slots;
    const CountSet<MULTI> cs{a0, &tmA0, &tmB0, inst, count};
    const long long total = MULTI ? (long long)*total_dev : (long long)a0.st->units_total;
    DevStatus* st0 = cs.args(0).st;
    volatile int* abort = &B->abort;

    setup(B, S, warp, 2 * NG);
    const uint32_t tmem = B->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int slot = 0;
            uint32_t ph = 0;
            int issued[MAX_SLOTS] = {0, 0, 0, 0};
            int res_loads = 0;
            bool ok = true;
            int last_i = -1;
            unsigned long long pairs = 0;
            for (long long w = blockIdx.x; w < total && ok; w += gridDim.x) {
                int i, T;
                int64_t ut0, ut1;
                cs.decode(w, i, T, ut0, ut1);
                const CountArgs& a = cs.args(i);
                if (i != last_i) {
                    if (pairs) atomicAdd(&cs.args(last_i).st->pairs_evaluated, pairs);
                    pairs = 0;
                    last_i = i;
                    tma_prefetch_desc(cs.mapA(i));
                    tma_prefetch_desc(cs.mapB(i));
                }
                const CUtensorMap* mA = cs.mapA(i);
                const CUtensorMap* mB = cs.mapB(i);
                const int KB = a.dp >> Op::KSHIFT;
                const int rb = res_loads % L.nres, ru = res_loads / L.nres;
                if (ru > 0 && !mbar_wait(&B->res_empty[rb], (ru - 1) & 1, abort, st0)) break;
                uint8_t* dst = sB + rb * L.res_bytes;
                mbar_expect_tx(&B->res_full[rb], KB * KB_BYTES_I);
                for (int kb = 0; kb < KB; ++kb)
                    tma_load_2d(dst + kb * KB_BYTES_I, mB, &B->res_full[rb], kb * Op::KELEMS, T * BI_TC);
                ++res_loads;
                for (int64_t ut = ut0; ut < ut1 && ok; ++ut) {
                    for (int kb = 0; kb < KB; ++kb) {
                        if (!mbar_wait(&B->empty[slot], ph ^ 1u, abort, st0)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&B->full[slot], KB_BYTES_U);
                        tma_load_2d(ring + slot * KB_BYTES_U, mA, &B->full[slot], kb * Op::KELEMS, (int)(ut * BU));
                        ++issued[slot];
                        if (++slot == S) {
                            slot = 0;
                            ph ^= 1u;
                        }
                    }
                }
                const int64_t uend = (ut1 * BU < a.n) ? ut1 * BU : a.n;
                if (ut1 > ut0) pairs += (unsigned long long)(uend - ut0 * BU) * BI_TC;
            }
            if (pairs && last_i >= 0) atomicAdd(&cs.args(last_i).st->pairs_evaluated, pairs);
            for (int s = 0; s < S; ++s)
                if (issued[s] > 0) drain_wait(&B->full[s], (uint32_t)(issued[s] - 1) & 1u, st0);
            for (int rb = 0; rb < L.nres; ++rb) {
                const int loads = res_loads / L.nres + (rb < res_loads % L.nres ? 1 : 0);
                if (loads > 0) drain_wait(&B->res_full[rb], (uint32_t)(loads - 1) & 1u, st0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = Op::idesc();
            int slot = 0;
            uint32_t ph = 0, tile_j = 0;
            int iter = 0;
            bool ok = true;
            for (long long w = blockIdx.x; w < total && ok; w += gridDim.x, ++iter) {
                int i, T;
                int64_t ut0, ut1;
                cs.decode(w, i, T, ut0, ut1);
                const int KB = cs.args(i).dp >> Op::KSHIFT;
                const int rb = iter % L.nres;
                if (!mbar_wait(&B->res_full[rb], (iter / L.nres) & 1, abort, st0)) break;
                tc_fence_after();
                const uint8_t* sBr = sB + rb * L.res_bytes;
                for (int64_t ut = ut0; ut < ut1 && ok; ++ut) {
                    const uint32_t b = tile_j & 1u, use = tile_j >> 1;
                    if (!mbar_wait(&B->tempty[b], (use & 1u) ^ 1u, abort, st0)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + b * BI_TC;
                    for (int kb = 0; kb < KB; ++kb) {
                        if (!mbar_wait(&B->full[slot], ph, abort, st0)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ad = sdesc_sw128(smem_u32(ring + slot * KB_BYTES_U));
                        const uint64_t bd = sdesc_sw128(smem_u32(sBr + kb * KB_BYTES_I));
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            Op::mma(d, ad + 2u * k, bd + 2u * k, idesc, (kb | k) != 0 ? 1u : 0u);
                        tc_commit(&B->empty[slot]);
                        if (++slot == S) {
                            slot = 0;
                            ph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    tc_commit(&B->tfull[b]);
                    ++tile_j;
                }
                if (!ok) break;
                tc_commit(&B->res_empty[rb]);
            }
            tc_commit(&B->drain);
            drain_wait(&B->drain, 0u, st0);
        }
    } else {
        constexpr int CW = 2 * BI_TC / NG;  // accumulator columns a group reads per tile
        const int ew = warp - 2;
        const int g = ew >> 2;
        const int h = g & 1;
        const int cg = (g >> 1) * CW;
        const int q = warp & 3;
        const int r = q * 32 + lane;
        int* cw = cnt_all + ew * CW;  // this warp's per-item member counters (its CW columns)
        for (int c = lane; c < CW; c += 32) cw[c] = 0;
        __syncwarp();
        // This group consumes global tiles h, h+2, h+4, ... of the CTA's sequence.  `cur` is
        // the current one, `nxt` the one after it, whose per-user record is loaded one tile
        // ahead so that its latency hides behind the current tile.
        TileCursor cur;
        cursor_first(cs, total, cur);
        if (h == 1) cursor_next(cs, total, cur);
        TileCursor nxt = cur;
        cursor_next(cs, total, nxt);
        cursor_next(cs, total, nxt);
        UserMeta um_cur{}, um_nxt{};
        if (cur.valid && cur.ut * BU + r < cs.args(cur.i).n) um_cur = cs.args(cur.i).meta[cur.ut * BU + r];
        uint32_t use = 0;
        int curT = -1, curI = -1;
        float pnh = 0.f, pd = 0.f;
        int te = 0;
        CountHot hot = count_hot(cs.args(0));
        while (cur.valid) {
            if (nxt.valid && nxt.ut * BU + r < cs.args(nxt.i).n) um_nxt = cs.args(nxt.i).meta[nxt.ut * BU + r];
            if (cur.T != curT || cur.i != curI) {
                if (curT >= 0) flush_counts<CW>(cw, lane, curT * BI_TC + cg, hot.m, hot.counts);
                if (MULTI && cur.i != curI) hot = count_hot(cs.args(cur.i));
                const CountArgs& a = cs.args(cur.i);
                curT = cur.T;
                curI = cur.i;
                pnh = a.thmax[cur.T];
                pd = a.tdel[cur.T];
                if constexpr (FP8) te = a.texp[cur.T];
            }
            if (!mbar_wait(&B->tfull[h], use & 1u, abort, st0)) break;
            __syncwarp();
            tc_fence_after();
            const int64_t us = cur.ut * BU + r;
            const bool active = us < hot.n;
            float hi_t = 0.f, lo_t = 0.f;
            int u_orig = 0;
            const float f = (FP8 && active) ? pow2i(fp8_exp(um_cur.uexp) + te - 16) : 1.f;  // descale of the FP8 product
            if (active) {
                const float E = err_bound(hot.cacc, hot.eabs, um_cur.un, um_cur.unh, um_cur.ud, pnh, pd);
                hi_t = __fadd_ru(um_cur.tau_hi, E);
                lo_t = __fsub_rd(um_cur.tau_lo, E);
                u_orig = um_cur.uorig;
            }
            const int pos0 = cur.T * BI_TC + cg;
            const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)h * BI_TC + cg;
            uint32_t ra[32], rb[32];
            // One vote per 64-column pair on the row maxima the two loads return, as in the
            // threshold epilogue.
#pragma unroll 1
            for (int c0 = 0; c0 < CW; c0 += 64) {
                __syncwarp();
                float ma, mb;
                tmem_ld32_max_issue(tb + c0, ra, ma);
                tmem_ld32_max_issue(tb + c0 + 32, rb, mb);
                tmem_wait_bind_max(ra, ma);
                tmem_wait_bind_max(rb, mb);
                const float mx = FP8 ? fmaxf(ma, mb) * f : fmaxf(ma, mb);
                if (__any_sync(0xffffffffu, active && mx >= lo_t)) {
                    float va[32], vb[32];
                    as_floats(ra, va);
                    as_floats(rb, vb);
                    if constexpr (FP8) {
                        scale_values(va, f);
                        scale_values(vb, f);
                    }
                    count_chunk(va, active, c0, pos0 + c0, hot.m, hi_t, lo_t, cw, u_orig, hot.band,
                                hot.band_cap, hot.st);
                    count_chunk(vb, active, c0 + 32, pos0 + c0 + 32, hot.m, hi_t, lo_t, cw, u_orig, hot.band,
                                hot.band_cap, hot.st);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B->tempty[h]);
            ++use;
            cur = nxt;
            um_cur = um_nxt;
            cursor_next(cs, total, nxt);
            cursor_next(cs, total, nxt);
        }
        if (curT >= 0) flush_counts<CW>(cw, lane, curT * BI_TC + cg, hot.m, hot.counts);
    }
    teardown(B, warp);
}

// First global unit of every instance of a counting launch (exclusive scan of the unit
// counts that k_build_units left in each instance's status word) and the launch's total.
__global__ void k_count_prefix(CountInstance* inst, int count, unsigned long long* total) {
    constexpr int T = 1024;
    __shared__ unsigned long long part[T];
    const int t = threadIdx.x;
    const int per = (count + T - 1) / T;
    const int b0 = t * per, b1 = (b0 + per < count) ? b0 + per : count;
    unsigned long long local = 0;
    for (int i = b0; i < b1; ++i) local += inst[i].a.st->units_total;
    part[t] = local;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        const unsigned long long v = (t >= o) ? part[t - o] : 0ull;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned long long run = part[t] - local;
    for (int i = b0; i < b1; ++i) {
        inst[i].unit_begin = (long long)run;
        run += inst[i].a.st->units_total;
    }
    if (t == T - 1) *total = part[T - 1];
}

// ---------------------------------------------------------------- guard-band check

// One 128-user x 256-item tile per CTA, computed with the operands, TMA boxes, swizzle,
// descriptors, MMA shape and FP8 descale of the product kernels above, written out with the
// error bound E of its row instead of being consumed by an epilogue.  128 threads: thread 0
// loads every K-block at once and issues the MMAs; warp 1 owns the TMEM columns; all four
// warps read back their 32 accumulator lanes.
template <bool FP8>
__global__ void __launch_bounds__(128, 1)
    k_products_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const ProductsArgs a) {
    using Op = Operand<FP8>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    const int KB = a.dp >> Op::KSHIFT;
    uint8_t* sA = sm;
    uint8_t* sB = sm + KB * KB_BYTES_U;
    __shared__ uint64_t full, done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ut = blockIdx.x, it = blockIdx.y;
    if (threadIdx.x == 0) {
        mbar_init(&full, 1);
        mbar_init(&done, 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) {
        tmem_alloc(&tmem_base, BI_TC);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int* abort = &abort_flag;
    bool issued = false;
    if (threadIdx.x == 0) {
        mbar_expect_tx(&full, KB * (KB_BYTES_U + KB_BYTES_I));
        for (int kb = 0; kb < KB; ++kb) {
            tma_load_2d(sA + kb * KB_BYTES_U, &tmA, &full, kb * Op::KELEMS, ut * BU);
            tma_load_2d(sB + kb * KB_BYTES_I, &tmB, &full, kb * Op::KELEMS, it * BI_TC);
        }
        if (mbar_wait(&full, 0u, abort, a.st)) {
            tc_fence_after();
            const uint32_t idesc = Op::idesc();
            for (int kb = 0; kb < KB; ++kb) {
                const uint64_t ad = sdesc_sw128(smem_u32(sA + kb * KB_BYTES_U));
                const uint64_t bd = sdesc_sw128(smem_u32(sB + kb * KB_BYTES_I));
#pragma unroll
                for (int k = 0; k < 4; ++k) Op::mma(tmem, ad + 2u * k, bd + 2u * k, idesc, (kb | k) != 0 ? 1u : 0u);
            }
            tc_commit(&done);
            issued = true;
        } else {
            drain_wait(&full, 0u, a.st);  // the copies must land before the CTA exits
        }
    }
    __syncwarp();
    if (mbar_wait(&done, 0u, abort, a.st)) {
        tc_fence_after();
        const int r = warp * 32 + lane;
        const int64_t u = (int64_t)ut * BU + r;
        const bool active = u < a.n;
        const float thm = a.thmax[it], tdl = a.tdel[it];
        const float E = active ? err_bound(a.cacc, a.eabs, a.unrm[u], a.unhat[u], a.udel[u], thm, tdl) : 0.f;
        const float f = (FP8 && active) ? pow2i(fp8_exp(a.uexp[u]) + a.texp[it] - 16) : 1.f;
        for (int c0 = 0; c0 < BI_TC; c0 += 32) {
            uint32_t rv[32];
            float v[32], mx;
            __syncwarp();
            tmem_ld32_max_issue(tmem + ((uint32_t)(warp * 32) << 16) + c0, rv, mx);
            tmem_wait_bind_max(rv, mx);
            as_floats(rv, v);
            // The product kernels vote on the maximum returned by the load itself: check it
            // against the loaded values (a mismatch makes the call return RKM_EINTERNAL).
            float ref = v[0];
#pragma unroll
            for (int j = 1; j < 32; ++j) ref = fmaxf(ref, v[j]);
            if (!(mx == ref)) a.st->internal_error = 1u;
            if (!active) continue;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int64_t pos = (int64_t)it * BI_TC + c0 + j;
                if (pos < a.m) {
                    const int64_t o = u * a.ldo + a.perm[pos];
                    a.v[o] = FP8 ? v[j] * f : v[j];
                    a.E[o] = E;
                }
            }
        }
    }
    if (threadIdx.x == 0 && issued) drain_wait(&done, 0u, a.st);  // no MMA in flight at exit
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, BI_TC);
    }
}

// ---------------------------------------------------------------- timeout path check

// One warp waits, with the product kernels' bounded wait and a given limit, on an mbarrier
// whose phase nothing completes (no arrival, no copy): the wait gives up, raises the abort
// flag and records the timeout in the status word, and the kernel returns normally.  The
// other lanes then see the abort flag and leave their waits at once.
__global__ void k_wait_timeout(long long limit, DevStatus* st) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    mbar_wait(&bar, 0u, &abort_flag, st, limit);
}

// Shared-memory plan: two resident buffers when that still leaves two ring slots, else one;
// then as many ring slots (up to max_slots) as fit in the 227 KB opt-in limit.
TcLayout make_layout(uint32_t res_bytes, uint32_t slot_bytes, uint32_t aux_bytes, int max_slots) {
    TcLayout L{};
    aux_bytes = (aux_bytes + 1023u) & ~1023u;
    const uint32_t fixed = 1024u + aux_bytes + 1024u;  // align slack + barriers
    L.nres = (fixed + 2u * res_bytes + 2u * slot_bytes <= (uint32_t)SMEM_LIMIT) ? 2 : 1;
    int slots = max_slots;
    while (slots > 1 && fixed + L.nres * res_bytes + slots * slot_bytes > (uint32_t)SMEM_LIMIT) --slots;
    L.slots = slots;
    L.res_bytes = res_bytes;
    L.slot_bytes = slot_bytes;
    L.res_off = 0;
    L.ring_off = L.nres * res_bytes;
    L.aux_off = L.ring_off + slots * slot_bytes;
    L.bar_off = L.aux_off + aux_bytes;
    L.bytes = 1024u + L.bar_off + (uint32_t)sizeof(TcBars);
    return L;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tiled map of a packed operand: rows x dp elements of elem_bytes (2 = BF16, 1 = FP8 codes),
// boxes of box_rows rows x 128 bytes with the 128-byte swizzle.
bool encode_operand(CUtensorMap* map, const void* base, int64_t rows, int dp, int box_rows, int elem_bytes) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)dp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)dp * (cuuint64_t)elem_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1u, 1u};
    const CUtensorMapDataType dt = elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

bool rkm_tc_available() { return true; }

rkm_status make_tmaps(const void* A, int64_t a_rows, const void* B, int64_t b_rows, int dp, int item_tile,
                      int elem_bytes, TmapPair* out) {
    if (elem_bytes != 1 && elem_bytes != 2) return RKM_EINVAL;
    if ((dp * elem_bytes) % 128 != 0 || a_rows % BU != 0 || b_rows % item_tile != 0 || item_tile != BI_TC)
        return RKM_EINVAL;
    if ((reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(B) & 15u)) return RKM_EINVAL;
    if (!encode_operand(&out->a, A, a_rows, dp, BU, elem_bytes)) return RKM_ECUDA;
    if (!encode_operand(&out->b, B, b_rows, dp, item_tile, elem_bytes)) return RKM_ECUDA;
    return RKM_OK;
}

namespace {

TcLayout threshold_layout(int ng, int kheap, int max_dp, bool fp8) {
    const int KB = fp8 ? max_dp / 128 : max_dp / 64;
    return make_layout(KB * KB_BYTES_U, KB_BYTES_I, (uint32_t)ng * BU * kheap * 4u + (uint32_t)ng * BU * 8u,
                       MAX_SLOTS);
}

template <bool FP8, int NG>
void launch_threshold_ng(const TcInstance* inst, int count, long long total_units, int kheap, const TcLayout& L,
                         int grid, cudaStream_t s) {
    cudaFuncSetAttribute(k_threshold_tc<FP8, NG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
    k_threshold_tc<FP8, NG><<<grid, tc_threads(NG), L.bytes, s>>>(inst, count, total_units, kheap, L);
}

}  // namespace

// Two groups unless four are asked for: measured on GB300 (BF16, d = 64 and 128), four
// groups made the threshold pass 1.5-1.8x slower.  Each group's heap then sees a quarter of
// the items, so its bound is lower and it records more candidates (exact rescoring took 2.4x
// longer), and 18 warps leave 96 registers per thread, so the hit path spills.
int threshold_groups(int kheap, int max_dp, bool fp8, int want) {
    if (want != 4 || kheap > 32) return 2;
    return threshold_layout(4, kheap, max_dp, fp8).slots >= 2 ? 4 : 2;
}

// Four groups for BF16 tiles one K-block deep (d <= 64): the MMA of a tile is then shortest and
// eight warps reading each tile made the counting pass 15 % faster at d = 64 on GB300; at two
// K-blocks and more the two were equal.  FP8 keeps two: its descale multiplies make the
// four-group kernel (96 registers per thread) spill, and it ran 2.7x slower.
int count_groups(int dp, bool fp8, int want) {
    if (want == 2 || want == 4) return want;
    return (!fp8 && dp <= 64) ? 4 : 2;
}

void launch_threshold_tc(const TcInstance* inst, int count, long long total_units, int kheap, int max_dp,
                         bool fp8, int ng, int num_sms, cudaStream_t s) {
    if (ng != 4) ng = 2;
    const TcLayout L = threshold_layout(ng, kheap, max_dp, fp8);
    const int grid = (int)(total_units < num_sms ? total_units : num_sms);
    if (grid < 1) return;
    note_launch();
    if (fp8) {
        if (ng == 4) launch_threshold_ng<true, 4>(inst, count, total_units, kheap, L, grid, s);
        else launch_threshold_ng<true, 2>(inst, count, total_units, kheap, L, grid, s);
    } else {
        if (ng == 4) launch_threshold_ng<false, 4>(inst, count, total_units, kheap, L, grid, s);
        else launch_threshold_ng<false, 2>(inst, count, total_units, kheap, L, grid, s);
    }
}

void launch_wait_timeout(long long limit, DevStatus* st, cudaStream_t s) {
    note_launch();
    k_wait_timeout<<<1, 32, 0, s>>>(limit, st);
}

void launch_products_tc(const ProductsArgs& a, const void* tmapA, const void* tmapB, bool fp8, cudaStream_t s) {
    const int KB = fp8 ? a.dp / 128 : a.dp / 64;
    // At least 120 KB of shared memory, so one CTA per SM: no CTA waits for TMEM columns.
    uint32_t bytes = 1024u + (uint32_t)KB * (KB_BYTES_U + KB_BYTES_I);
    if (bytes < 120u * 1024u) bytes = 120u * 1024u;
    const dim3 grid((unsigned)((a.n + BU - 1) / BU), (unsigned)((a.m + BI_TC - 1) / BI_TC));
    if (grid.x == 0 || grid.y == 0) return;
    const CUtensorMap& mA = *static_cast<const CUtensorMap*>(tmapA);
    const CUtensorMap& mB = *static_cast<const CUtensorMap*>(tmapB);
    note_launch();
    if (fp8) {
        cudaFuncSetAttribute(k_products_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        k_products_tc<true><<<grid, 128, bytes, s>>>(mA, mB, a);
    } else {
        cudaFuncSetAttribute(k_products_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        k_products_tc<false><<<grid, 128, bytes, s>>>(mA, mB, a);
    }
}

namespace {

template <bool FP8, int NG, bool MULTI>
void launch_count_ng(const CountArgs& a0, const CUtensorMap& mA, const CUtensorMap& mB, const CountInstance* inst,
                     int count, const unsigned long long* total, int max_dp, int grid, cudaStream_t s) {
    const int KB = FP8 ? max_dp / 128 : max_dp / 64;
    // per-warp member counters: 4 NG warps x (512 / NG) columns
    const TcLayout L = make_layout(KB * KB_BYTES_I, KB_BYTES_U, 4u * NG * (2u * BI_TC / NG) * 4u, MAX_SLOTS);
    cudaFuncSetAttribute(k_count_tc<FP8, NG, MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
    k_count_tc<FP8, NG, MULTI><<<grid, tc_threads(NG), L.bytes, s>>>(a0, mA, mB, inst, count, total, L);
}

}  // namespace

void launch_count_prefix(CountInstance* inst, int count, unsigned long long* total, cudaStream_t s) {
    note_launch();
    k_count_prefix<<<1, 1024, 0, s>>>(inst, count, total);
}

void launch_count_tc(const CountArgs& a, const void* tmapA, const void* tmapB, bool fp8, cudaStream_t s) {
    note_launch();
    const CUtensorMap& mA = *static_cast<const CUtensorMap*>(tmapA);
    const CUtensorMap& mB = *static_cast<const CUtensorMap*>(tmapB);
    if (fp8) {
        if (a.groups == 4) launch_count_ng<true, 4, false>(a, mA, mB, nullptr, 1, nullptr, a.dp, a.num_sms, s);
        else launch_count_ng<true, 2, false>(a, mA, mB, nullptr, 1, nullptr, a.dp, a.num_sms, s);
    } else {
        if (a.groups == 4) launch_count_ng<false, 4, false>(a, mA, mB, nullptr, 1, nullptr, a.dp, a.num_sms, s);
        else launch_count_ng<false, 2, false>(a, mA, mB, nullptr, 1, nullptr, a.dp, a.num_sms, s);
    }
}

// Always two epilogue warpgroups: with the arguments read from device memory, four would
// spill registers.
void launch_count_tc_multi(const CountInstance* inst, int count, const unsigned long long* total, int max_dp,
                           bool fp8, int num_sms, cudaStream_t s) {
    note_launch();
    CountArgs none{};
    CUtensorMap nomap{};
    if (fp8) launch_count_ng<true, 2, true>(none, nomap, nomap, inst, count, total, max_dp, num_sms, s);
    else launch_count_ng<false, 2, true>(none, nomap, nomap, inst, count, total, max_dp, num_sms, s);
}

}  // namespace rkm
