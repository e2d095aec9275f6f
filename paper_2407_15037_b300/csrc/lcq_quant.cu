// lcq_quant.cu -- single-array quantize / verify / compact, NOA range
// reduction and dequantize kernels, and the C-ABI entry points declared in
// include/lcq.h.
//
// Data path of one lcq_quantize call (Fallin & Burtscher, arXiv 2407.15037):
//   [NOA only] k_minmax: finite min/max (ordered-integer keys, warp + block
//       reductions, per-block partials, last block combines) -> R, eb*R and
//       the ABS constants, written to the header in device memory (Sec. 2.1.3).
//   k_quantize: persistent CTAs of 8 compute warps and 1 scan warp.  Stages
//       of the input arrive in shared memory by bulk asynchronous copies
//       (cp.async.bulk + mbarrier) in a ring; scan tiles (several stages) are
//       handed out by an atomic ticket.  Compute warps quantize, verify and
//       store bins per value (Sec. 2.2, 3.1-3.3) and build the outlier mask
//       words; the scan warp stores each finished tile's mask words and its
//       outlier count, and adds the count into its group of 64 tiles.  No
//       CTA waits for another.
//   k_compact: the outliers' raw bits to payload[offset + rank], ascending
//       index order (Sec. 3.1), one warp per tile that has outliers; each
//       CTA takes its first offset from the group and tile counts, the last
//       CTA writes the header's outlier count.
// The kernels are launched with programmatic stream serialisation, so each
// one is scheduled while the one before it drains.
// Decoding: k_tile_counts (outliers per tile and per group of 64 tiles,
// from the mask); k_dequantize streams bins and mask words by bulk copies,
// reconstructs the values with the encoder's exact operations (Sec. 3.1; no
// double-check on decode, Sec. 6), and patches the outliers from the payload
// at offsets its scan warp adds up from those counts.
//
// Arrays longer than kChunk values are processed as several launches; the
// running outlier count carries from one chunk to the next in device memory,
// so a call never waits on the host.  lcq_quantize_host / _host_batch use the
// same per-range launches to pipeline host copies with the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>

#include "lcq_device.cuh"
#include "lcq_pipe.cuh"
#include "lcq_tile.cuh"
#include "lcq_host.h"

namespace lcq {

constexpr int kBlock = 256;
constexpr uint64_t kChunk = 1ull << 31;         // values per launch at most
constexpr uint32_t kDefaultSpin = 1u << 20;     // default of the test hook's poll limit
constexpr uint32_t kMbarLimit = 1u << 22;       // bulk-copy completion polls (seconds)
constexpr uint32_t kGroupTiles = 64;            // scan tiles per group count of the compaction
constexpr uint64_t kMaxSub = 8;                 // ring stages per scan tile, at most (staging table)
constexpr uint64_t kStageNone = ~0ull;          // staging table: a stage left to k_compact's walk

// Tile shapes: 4-value vectors per thread (tile = 256 x 4 x VPT values) and
// the depth of the shared-memory stage ring.
// Tile shapes ("variants"): VPT 4-value vectors per compute thread per stage
// (stage = 1024 VPT values), STAGES ring depth, SUB stages per scan tile,
// MINB CTAs per SM the register budget must allow.  lcq_tune_* selects one
// per (kernel, dtype, bound type); lcq_autotune_quantize times them all.
struct Variant {
    int vpt, stages, sub, minb;
};
constexpr Variant kVariants[] = {
    {8, 3, 4, 2},  // 0: 32 KB float stages, 2 CTAs/SM
    {4, 3, 8, 3},  // 1: 16 KB float stages, 3 CTAs/SM
    {4, 3, 4, 4},  // 2: 16 KB float stages, 4 CTAs/SM
    {4, 4, 4, 3},  // 3
    {2, 6, 8, 4},  // 4: 8 KB float stages, 4 CTAs/SM
    {8, 2, 4, 2},  // 5
    {2, 3, 8, 4},  // 6: 8 KB float / 16 KB double stages: 4 CTAs/SM also for float64
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

static ScanCfg g_scan = {kDefaultSpin, ~0ull};  // the test hook (lcq_debug_set_scan)

// ---------------------------------------------------------------------------
// Quantize kernel: persistent CTAs; input tiles stream into a ring of
// shared-memory stages by bulk asynchronous copies, so that the next tiles
// are in flight while the current tile is quantized.
// ---------------------------------------------------------------------------
template <typename T>
struct QParams {
    const T* in;          // chunk start
    int32_t* bins;        // chunk start
    uint32_t* mask;       // chunk start (chunk offsets are multiples of 32)
    uint32_t* counts;     // outliers per scan tile of this chunk
    uint32_t* groups;     // outliers per kGroupTiles scan tiles (added up; zero on entry)
    uint64_t* stab;       // float32 REL outlier staging: entry per stage (null: no staging)
    uint32_t* stg;        // staging area (raw bits), stage_cap values
    uint64_t scap;        // staging area capacity in values
    lcq_header* hdr;
    WsHead* ws;
    uint64_t n;           // values in this chunk
    uint32_t num_tiles;
    uint32_t first_chunk;
    uint32_t consts_from_hdr;  // NOA: constants written by k_minmax
    Consts<CT<T>> c;
    ScanCfg hook;              // test hook of the bounded tile handoff
    // header fields (written by the CTA that owns tile 0 of the first chunk)
    uint32_t dtype, bound;
    double eb, eb_abs;
    uint64_t n_total;
};

// Warp-specialised streaming kernels.  A CTA has 8 compute warps and one
// scan warp.  The compute warps stream the CTA's tiles through a ring of
// shared-memory stages (bulk asynchronous copies, one sub-tile per stage):
// when a scan tile (SUB sub-tiles) is done they hand its mask words to the
// scan warp and go on.  The scan warp stores the words and the tile's count
// (quantize) or their in-tile prefix counts and the tile's payload offset
// (dequantize: the compute warps then patch that tile's outliers one scan
// tile later).  Tickets are taken one scan tile at a time as the ring fills.


template <typename T, int MODE, int VPT, int STAGES, int SUB, int MINB>
__global__ void __launch_bounds__(kSpecThreads, MINB) k_quantize(QParams<T> p) {
    using F = Ty<T>;
    constexpr int STILE = kComputeThreads * 4 * VPT;  // values per stage (sub-tile)
    constexpr int TILE = STILE * SUB;                  // values per scan tile
    constexpr int SWORDS = STILE / 32;
    constexpr int WORDS = TILE / 32;
    constexpr int WPL = WORDS / 32;
    static_assert(WPL % 4 == 0, "whole uint4 mask stores per lane");
    static_assert(SUB <= (int)kMaxSub, "staging table: at most kMaxSub stages per scan tile");
    extern __shared__ __align__(128) unsigned char dsmem[];
    T* sbuf = reinterpret_cast<T*>(dsmem);
    __shared__ __align__(8) uint64_t s_stage_bar[STAGES];
    __shared__ __align__(8) uint64_t s_full[2];
    __shared__ __align__(8) uint64_t s_done[2];
    __shared__ uint32_t s_stage_ticket[STAGES];
    __shared__ uint32_t s_mask[2][WORDS];
    __shared__ uint32_t s_wpre[2][WORDS];
    __shared__ uint32_t s_jt[2];
    __shared__ uint32_t s_epoch, s_filled;
    __shared__ volatile uint32_t s_abort;
    // float32 REL outlier staging: the compute warps hand each consumed stage
    // to the scan warp (s_cons), which copies its outliers out and refills
    // the slot itself; s_cons_end = k + 1 marks that the stages end before
    // stage k (a lagging scan warp must not stop early).
    constexpr bool STG = MODE == LCQ_REL && std::is_same<T, float>::value;
    __shared__ __align__(8) uint64_t s_cons[STG ? STAGES : 1];
    __shared__ volatile uint32_t s_cons_end;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t full_sub = p.n / STILE;
    const bool stg = STG && p.stab != nullptr;  // uniform over the launch
    pdl_wait();  // the compaction is let in only when this CTA's tiles are done (below)

    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) mbar_init(&s_stage_bar[s], 1);
        for (int b = 0; b < 2; b++) {
            mbar_init(&s_full[b], 1);
            mbar_init(&s_done[b], 1);
        }
        if constexpr (STG) {
            for (int s = 0; s < STAGES; s++) mbar_init(&s_cons[s], 1);
        }
        mbar_init_fence();
        s_epoch = ld_relaxed_u32(&p.ws->epoch);
        s_abort = 0;
        s_filled = 0;
        s_cons_end = 0;
    }
    const Consts<CT<T>> c = p.consts_from_hdr ? consts_from_header<CT<T>>(p.hdr) : p.c;
    __syncthreads();

    // One thread: the next sub-tile of this CTA into the next stage (f:
    // stages issued so far).  Without staging, thread 0 issues every stage
    // and a stage past the last tile arms nothing (the compute warps read its
    // ticket first and stop); with staging, lane 0 of the scan warp issues
    // every stage and a stage past the last tile completes its barrier
    // phase, as the compute warps read its ticket after the wait.
    auto issue = [&](uint32_t& f, bool arm_end) {
        const int s = (int)(f % STAGES);
        const uint32_t sub = f % SUB;
        const uint32_t t = sub == 0 ? atomicAdd(&p.ws->ticket, 1u) : s_stage_ticket[(f - 1) % STAGES];
        s_stage_ticket[s] = t;
        f = f + 1;
        if (t < p.num_tiles) {
            const uint64_t g = (uint64_t)t * SUB + sub;
            if (g < full_sub) {
                mbar_arrive_expect_tx(&s_stage_bar[s], STILE * sizeof(T));
                bulk_g2s(sbuf + (size_t)s * STILE, p.in + g * STILE, STILE * sizeof(T), &s_stage_bar[s]);
            } else {
                mbar_arrive(&s_stage_bar[s]);  // ragged or empty sub-tile: global reads
            }
        } else if (arm_end) {
            mbar_arrive(&s_stage_bar[s]);
        }
    };

    if (warp < kComputeThreads / 32) {
        // ------------------------------------------------ compute warps --
        // Wait until the scan warp has taken scan tile jj's mask words, so
        // that its buffer may be reused.  Returns true if the kernel must
        // stop (uniform over the compute warps).
        auto release_tile = [&](uint32_t jj) -> bool {  // all compute threads
            const int bb = (int)(jj & 1u);
            const uint32_t limit = (uint64_t)s_jt[bb] == p.hook.drop_tile ? p.hook.spin_limit : kMbarLimit;
            bool ok = mbar_wait_or_abort(&s_done[bb], (jj >> 1) & 1u, limit, &s_abort);
            if (!ok && !s_abort) {
                atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT);
                s_abort = 1;
            }
            return named_barrier_or(1, kComputeThreads, !ok);
        };

        if (tid == 0 && !stg) {
            uint32_t f = s_filled;
            issue(f, false);
            s_filled = f;
        }
        named_barrier_sync(1, kComputeThreads);
        uint32_t k = 0;
        for (;; k++) {
            const int s = (int)(k % STAGES);
            const uint32_t sub = k % SUB;
            const uint32_t j = k / SUB;
            const int b = (int)(j & 1u);
            uint32_t t;
            bool end = false;  // with staging: no stage k (decided at the consumed barrier)
            if (!stg) {
                if (tid == 0 && s_filled < k + STAGES) {  // ring fill
                    uint32_t f = s_filled;
                    issue(f, false);
                    s_filled = f;
                }
                t = s_stage_ticket[s];  // written stages ago, before a barrier
                if (t >= p.num_tiles) break;
            }
            if (!mbar_wait_or_abort(&s_stage_bar[s], (k / STAGES) & 1u, kMbarLimit, &s_abort)) {
                if (!s_abort) { atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT); s_abort = 1; }
            }
            if (stg) {
                // written by the scan warp before the stage's barrier phase
                // completed; a thread whose wait gave up has set the abort
                // flag, so the stop below is uniform either way
                t = s_stage_ticket[s];
                end = t >= p.num_tiles;
            }
            if (!end) {
                const uint64_t g = (uint64_t)t * SUB + sub;
                const T* st = sbuf + (size_t)s * STILE;
                const uint64_t sbase = g * STILE;
                quantize_subtile<T, MODE, VPT>(st, p.in + sbase, g < full_sub, p.n > sbase ? p.n - sbase : 0,
                                               p.bins + sbase, s_mask[b], (int)sub * SWORDS, c);
            }
            fence_proxy_async_smem();
            bool stop = named_barrier_or(1, kComputeThreads, s_abort != 0 || end);  // stage s consumed
            if (stop) break;
            if (stg && tid == 0) mbar_arrive(&s_cons[s]);  // to the scan warp: outliers, then refill
            if (!stg && tid == 0 && s_filled < k + 1 + STAGES) {  // refill stage s
                uint32_t f = s_filled;
                issue(f, false);
                s_filled = f;
            }
            if (sub == SUB - 1) {
                if (tid == 0) {
                    s_jt[b] = t;
                    mbar_arrive(&s_full[b]);  // hand the scan tile to the scan warp
                }
                if (j >= 1 && release_tile(j - 1)) {
                    stop = true;
                    break;
                }
            }
        }
        // k is uniform here; an aborted loop leaves the scan warp to notice
        // the abort flag by itself
        if (!named_barrier_or(1, kComputeThreads, s_abort != 0)) {
            const uint32_t J = k / SUB;  // scan tiles handled by this CTA
            if (!(J >= 1 && release_tile(J - 1)) && tid == 0) {
                // With staging: no stage k, the stages end here.  Only now, once
                // the scan warp has finished tile J - 1 (and so taken in every
                // stage before k), may slot k % STAGES take this extra arrival:
                // earlier, its barrier could run two phases ahead of the scan
                // warp's wait for the slot's previous stage.
                if (stg) {
                    s_cons_end = k + 1;
                    mbar_arrive(&s_cons[k % STAGES]);
                }
                s_jt[J & 1u] = kNoTile;
                mbar_arrive(&s_full[J & 1u]);
            }
        }
        // no bulk copy outstanding at CTA exit (also after an abort)
        if (tid == 0 &&
            !drain_stages<STAGES>(s_stage_bar, s_filled,
                                  [&](uint32_t f) { return s_stage_ticket[f % STAGES] < p.num_tiles; },
                                  kMbarLimit))
            atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT);
    } else {
        // --------------------------------------------------- scan warp --
        const uint64_t nwords = (p.n + 31) / 32;
        // Staging (float32 REL): this CTA's share of the staging area, and
        // how much of it is used.  Each consumed stage comes here before its
        // slot is refilled: its outliers, read from the stage in shared
        // memory, go to the staging area in index order; the stage's table
        // entry records where (k_compact then copies them to the payload).
        // A stage read from global memory (ragged), with more than half of
        // its values outliers, or that would overflow the CTA's share is left
        // to k_compact's own walk (entry kStageNone).  Lane 0 issues every
        // stage: the first STAGES here, each later one into the slot of the
        // stage just taken out.
        constexpr int SWPL = SWORDS / 32;  // mask words per lane of a stage
        const uint64_t region = stg ? p.scap / gridDim.x : 0;
        const uint64_t sbeg = (uint64_t)blockIdx.x * region;
        uint64_t sused = 0;
        uint32_t kk = 0;      // the next stage to take in
        uint32_t filled = 0;  // stages issued (lane 0)
        if (stg && lane == 0)
            while (filled < (uint32_t)STAGES) issue(filled, true);
        auto stage_out = [&](int sl, uint32_t sub, int b) {
            const uint64_t g = (uint64_t)s_stage_ticket[sl] * SUB + sub;
            uint32_t w[SWPL], cnt = 0;
#pragma unroll
            for (int i = 0; i < SWPL; i++) {
                w[i] = s_mask[b][sw((int)sub * SWORDS + lane * SWPL + i)];
                cnt += __popc(w[i]);
            }
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            uint64_t entry = 0;
            if (total != 0u) {
                if (g >= full_sub || total > (uint32_t)(STILE / 2) || sused + total > region) {
                    entry = kStageNone;
                } else {
                    // each word from both ends: its lowest outlier to the next
                    // slot of its run, its highest to the last free one, so a
                    // word takes ceil(bits / 2) steps
                    const uint32_t* sv = reinterpret_cast<const uint32_t*>(sbuf + (size_t)sl * STILE) +
                                         (size_t)lane * SWPL * 32;
                    uint32_t* dst = p.stg + (sbeg + sused + (incl - cnt));
#pragma unroll
                    for (int i = 0; i < SWPL; i++) {
                        uint32_t m = w[i];
                        const uint32_t* svi = sv + i * 32;
                        uint32_t* lo = dst;
                        uint32_t* hi = dst + __popc(m);  // one past the word's run
                        dst = hi;
                        while (m) {
                            const int bl = __ffs(m) - 1;
                            const int bh = 31 - __clz(m);
                            *lo++ = svi[bl];
                            if (bh != bl) *--hi = svi[bh];
                            m &= m - 1u;
                            m &= ~(1u << bh);
                        }
                    }
                    entry = ((uint64_t)total << 32) | (sbeg + sused);
                    sused += total;
                }
            }
            if (lane == 0) p.stab[g] = entry;
            fence_proxy_async_smem();  // the stage was read; it may be refilled
            __syncwarp();
            if (lane == 0) issue(filled, true);  // stage kk + STAGES into slot sl
        };
        for (uint32_t j = 0;; j++) {
            const int b = (int)(j & 1u);
            if (stg) {  // the stages of tile j first
                bool out = false;
                for (uint32_t sub = 0; sub < (uint32_t)SUB; sub++, kk++) {
                    const int sl = (int)(kk % STAGES);
                    if (!mbar_wait_or_abort(&s_cons[sl], (kk / STAGES) & 1u, kMbarLimit, &s_abort)) {
                        if (!s_abort) { atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT); s_abort = 1; }
                        out = true;
                        break;
                    }
                    if (s_cons_end == kk + 1) break;  // no stage kk: the next handover is the end
                    stage_out(sl, sub, b);
                }
                if (out) break;
            }
            if (!mbar_wait_or_abort(&s_full[b], (j >> 1) & 1u, kMbarLimit, &s_abort)) {
                if (!s_abort) { atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT); s_abort = 1; }
                break;
            }
            const uint32_t t = s_jt[b];
            if (t == kNoTile) break;
            const uint32_t agg = scan_mask_words<WPL>(s_mask[b], s_wpre[b], p.mask,
                                                      (uint64_t)t * WORDS + (uint64_t)lane * WPL, nwords, true);
            if (lane == 0) {
                p.counts[t] = agg;
                if (agg) atomicAdd(&p.groups[t / kGroupTiles], agg);
                if (t == 0 && p.first_chunk) {
                    lcq_header* h = p.hdr;
                    h->magic = LCQ_MAGIC;
                    h->dtype = p.dtype;
                    h->bound_type = p.bound;
                    h->n = p.n_total;
                    h->eb = p.eb;
                    if (!p.consts_from_hdr) {
                        h->mode = MODE == kModeRelLib ? 2u : 0u;
                        h->range = 0.0;
                        h->eb_abs = p.eb_abs;
                        using FC = Ty<CT<T>>;
                        h->ebT_bits = (uint64_t)FC::bits(p.c.ebT);
                        h->scale_bits = (uint64_t)FC::bits(p.c.scale);
                        h->inv_bits = (uint64_t)FC::bits(p.c.inv);
                        h->chk_bits = (uint64_t)FC::bits(p.c.chk);
                    }
                    h->reserved = 0;
                }
            }
            __syncwarp();
            if (lane == 0 && (uint64_t)t != p.hook.drop_tile) mbar_arrive(&s_done[b]);  // test hook: never handed back
        }
        // with staging, no bulk copy of this warp's outstanding at CTA exit
        if (stg && lane == 0 &&
            !drain_stages<STAGES>(s_stage_bar, filled,
                                  [&](uint32_t f) { return s_stage_ticket[f % STAGES] < p.num_tiles; },
                                  kMbarLimit))
            atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT);
    }
    pdl_trigger();
    __syncthreads();
    if (tid == 0) finish_launch(p.ws, s_epoch, &p.hdr->status, p.first_chunk != 0);
}

// Header for an empty input (no tiles to launch).
__global__ void k_header_empty(lcq_header* h, uint32_t dtype, uint32_t bound, double eb,
                               double eb_abs, uint64_t ebT, uint64_t scale, uint64_t inv,
                               uint64_t chk, uint32_t mode) {
    h->magic = LCQ_MAGIC;
    h->dtype = dtype;
    h->bound_type = bound;
    h->mode = mode;
    h->n = 0;
    h->eb = eb;
    h->range = 0.0;
    h->eb_abs = eb_abs;
    h->ebT_bits = ebT;
    h->scale_bits = scale;
    h->inv_bits = inv;
    h->chk_bits = chk;
    h->outlier_count = 0;
    h->status = 0;
    h->reserved = 0;
}

// ---------------------------------------------------------------------------
// Outlier compaction (after k_quantize): k_compact places the outliers of a
// chunk.  Each CTA takes a run of consecutive scan tiles; its first payload
// offset is the count of the earlier chunks plus the outliers of all tiles
// before the run, which it adds up from the group counts (k_quantize's scan
// warps add every tile's count into the count of its group of kGroupTiles
// tiles) and the tile counts of the group it starts in.  It scans its own
// tiles' counts, and each warp walks the mask words of one tile with
// outliers and writes their raw bits to payload[offset + rank], in index
// order.  The last CTA to finish writes the header's outlier count and
// zeroes the group counts for the next call.  Keeping this out of
// k_quantize leaves the streaming CTAs without any dependence on one another
// (an in-kernel lookback made every CTA wait for the slowest ones).
//
// The decoder takes each tile's outlier count from the mask (k_tile_counts,
// which adds the group counts too), and its scan warp adds up a tile's
// payload offset the same way.
// ---------------------------------------------------------------------------

// Outliers per scan tile of WORDS mask words (the decoder's counts), one
// warp per tile; each count is also added into its group count.
template <int WORDS>
__global__ void __launch_bounds__(256) k_tile_counts(const uint32_t* mask, uint64_t n, uint32_t tiles,
                                                     uint32_t* counts, uint32_t* groups) {
    pdl_wait();
    pdl_trigger();
    constexpr int WPL = WORDS / 32;
    const int lane = threadIdx.x & 31;
    const uint64_t nwords = (n + 31) / 32;
    const uint32_t wstride = gridDim.x * (blockDim.x / 32);
    for (uint32_t t = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); t < tiles; t += wstride) {
        const uint64_t gw = (uint64_t)t * WORDS + (uint64_t)lane * WPL;
        uint32_t c = 0;
#pragma unroll
        for (int j = 0; j < WPL; j += 4) {
            if (gw + j + 4 <= nwords) {
                const uint4 a = *reinterpret_cast<const uint4*>(mask + gw + j);
                c += __popc(a.x) + __popc(a.y) + __popc(a.z) + __popc(a.w);
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++) c += gw + j + i < nwords ? __popc(mask[gw + j + i]) : 0;
            }
        }
        c = __reduce_add_sync(0xFFFFFFFFu, c);
        if (lane == 0) {
            counts[t] = c;
            if (c) atomicAdd(&groups[t / kGroupTiles], c);
        }
    }
}

constexpr int kCompactThreads = 256;
constexpr int kCompactWarps = kCompactThreads / 32;

template <typename T>
struct CParams {
    const T* in;               // chunk start
    const uint32_t* mask;      // chunk start
    uint64_t n;                // values in this chunk
    const uint32_t* counts;    // outliers per scan tile
    uint32_t* groups;          // outliers per kGroupTiles scan tiles
    const uint64_t* stab;      // staged outliers per ring stage (null: none staged)
    const uint32_t* stg;       // the staging area
    uint32_t sub;              // ring stages per scan tile
    uint32_t tiles, per;       // scan tiles of the chunk; consecutive tiles per CTA
    typename Ty<T>::U* out;    // payload
    uint64_t cap;              // payload capacity
    lcq_header* hdr;
    WsHead* ws;
    uint32_t first_chunk;
};

// Sum over the CTA's threads (every thread gets it); s_red: kCompactWarps words.
__device__ __forceinline__ uint32_t cta_sum(uint32_t v, uint32_t* s_red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = __reduce_add_sync(0xFFFFFFFFu, v);
    __syncthreads();  // s_red may still be read from the previous call
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < kCompactWarps; w++) t += s_red[w];
    return t;
}

// Dense tiles (at least 1/16 outliers, whole) stream through a stage of
// shared memory per warp, kCompactChunk values and their 32 mask words at a
// time, by bulk asynchronous copies (the CTA's other warps keep the memory
// busy meanwhile); the warp then writes each word's outliers with one
// coalesced store.  The bytes of one stage.
constexpr int kCompactChunk = 1024;
template <typename T>
__host__ __device__ constexpr size_t compact_stage_bytes() {
    return (size_t)kCompactChunk * sizeof(T) + kCompactChunk / 8;
}
constexpr int kCompactStages = 1;

template <typename T, int WORDS>
__global__ void __launch_bounds__(kCompactThreads, sizeof(T) == 8 ? 3 : 4) k_compact(CParams<T> p) {
    using F = Ty<T>;
    pdl_wait();
    pdl_trigger();
    constexpr int TILE = WORDS * 32;
    constexpr size_t SB = compact_stage_bytes<T>();
    static_assert(TILE % kCompactChunk == 0 && SB % 16 == 0, "whole chunks, 16-byte stages");
    extern __shared__ __align__(128) unsigned char dsmem[];
    __shared__ uint32_t s_red[kCompactWarps];
    __shared__ uint32_t s_wsum[kCompactWarps];
    __shared__ uint32_t s_cnt[kCompactThreads];
    __shared__ uint64_t s_off[kCompactThreads];
    __shared__ __align__(8) uint64_t s_cbar[kCompactWarps][kCompactStages];
    __shared__ bool s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t nwords = (p.n + 31) / 32;
    if (tid == 0) {
        for (int w = 0; w < kCompactWarps; w++)
            for (int s = 0; s < kCompactStages; s++) mbar_init(&s_cbar[w][s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    // this warp's stages; issued / used count its copies (uniform in the warp)
    unsigned char* wbuf = dsmem + (size_t)warp * kCompactStages * SB;
    uint64_t* wbar = s_cbar[warp];
    uint32_t issued = 0, used = 0;
    bool failed = false;
    auto cissue = [&](const T* tin, const uint32_t* tmask, int c) {
        if (lane == 0) {
            uint64_t* bar = &wbar[issued % kCompactStages];
            unsigned char* dst = wbuf + (issued % kCompactStages) * SB;
            mbar_arrive_expect_tx(bar, (uint32_t)SB);
            bulk_g2s(dst, tin + (size_t)c * kCompactChunk, kCompactChunk * sizeof(T), bar);
            bulk_g2s(dst + kCompactChunk * sizeof(T), tmask + (size_t)c * (kCompactChunk / 32), kCompactChunk / 8, bar);
        }
        issued++;
    };
    // One dense whole tile: its outliers to out[pbase + rank], rank in index order.
    auto compact_dense = [&](const T* tin, const uint32_t* tmask, uint64_t pbase) {
        constexpr int NCH = TILE / kCompactChunk;
        // one chunk in flight per stage: a stage's barrier takes one arrival per phase
#pragma unroll
        for (int c0 = 0; c0 < kCompactStages && c0 < NCH; c0++) cissue(tin, tmask, c0);
        uint64_t run = pbase;
        for (int c = 0; c < NCH; c++) {
            const uint32_t u = used;
            const bool arrived = mbar_wait(&wbar[u % kCompactStages], (u / kCompactStages) & 1u, kMbarLimit);
            if (!__all_sync(0xFFFFFFFFu, arrived)) {  // uniform in the warp
                failed = true;
                return;
            }
            used = u + 1;
            const unsigned char* src = wbuf + (u % kCompactStages) * SB;
            const T* vals = reinterpret_cast<const T*>(src);
            const uint32_t w = reinterpret_cast<const uint32_t*>(src + kCompactChunk * sizeof(T))[lane];
            const uint32_t cnt = (uint32_t)__popc(w);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t ex = incl - cnt, below = (1u << lane) - 1u;
            // word by word, lane i the word's value i: the outliers of a word
            // go to consecutive payload entries, one coalesced store
#pragma unroll 8
            for (int j = 0; j < 32; j++) {
                const uint32_t m = __shfl_sync(0xFFFFFFFFu, w, j);
                const uint32_t pre = __shfl_sync(0xFFFFFFFFu, ex, j);
                if ((m >> lane) & 1u) {
                    const uint64_t r = run + pre + (uint32_t)__popc(m & below);
                    if (r < p.cap) p.out[r] = F::bits(vals[j * 32 + lane]);
                }
            }
            run += __shfl_sync(0xFFFFFFFFu, incl, 31);
            fence_proxy_async_smem();  // the stage is read; it may be refilled
            __syncwarp();
            if (c + kCompactStages < NCH) cissue(tin, tmask, c + kCompactStages);
        }
    };

    // outliers of the earlier chunks (the header's count, written by the
    // last CTA of the previous chunk's compaction)
    const uint64_t carry = p.first_chunk ? 0ull : p.hdr->outlier_count;
    const uint32_t t0 = blockIdx.x * p.per < p.tiles ? blockIdx.x * p.per : p.tiles;
    const uint32_t t1 = t0 + p.per < p.tiles ? t0 + p.per : p.tiles;
    // outliers of the tiles before t0: whole groups, then single tiles
    const uint32_t g0 = t0 / kGroupTiles;
    uint32_t before = 0;
    for (uint32_t g = tid; g < g0; g += kCompactThreads) before += p.groups[g];
    for (uint32_t t = g0 * kGroupTiles + tid; t < t0; t += kCompactThreads) before += p.counts[t];
    uint64_t base = carry + cta_sum(before, s_red);
    for (uint32_t b = t0; b < t1; b += kCompactThreads) {
        // exclusive scan of up to kCompactThreads tile counts
        const uint32_t c = b + tid < t1 ? p.counts[b + tid] : 0u;
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        __syncthreads();
        uint32_t wpre = 0, pass = 0;
#pragma unroll
        for (int w = 0; w < kCompactWarps; w++) {
            const uint32_t v = s_wsum[w];
            wpre += w < warp ? v : 0u;
            pass += v;
        }
        s_cnt[tid] = c;
        s_off[tid] = base + wpre + x - c;
        __syncthreads();
        const uint32_t m = t1 - b < (uint32_t)kCompactThreads ? t1 - b : (uint32_t)kCompactThreads;
        for (uint32_t i = (uint32_t)warp; i < m; i += kCompactWarps) {
            const uint32_t tcount = s_cnt[i];
            const uint64_t pbase = s_off[i];
            if (tcount == 0u || pbase >= p.cap) continue;  // the same in every lane
            const uint64_t t = b + i;
            if constexpr (sizeof(T) == 4 && !is16<T>()) {
                // Every stage of the tile staged by k_quantize: its stages are
                // consecutive stages of one quantize CTA, whose staged runs
                // follow one another, so the tile's outliers are one run of
                // tcount values starting at its first non-empty stage's run.
                if (p.stab) {
                    const uint64_t e = lane < (int)p.sub ? p.stab[t * p.sub + lane] : 0ull;
                    const uint32_t nz = __ballot_sync(0xFFFFFFFFu, (e >> 32) != 0ull);
                    if (!__any_sync(0xFFFFFFFFu, e == kStageNone) && nz != 0u) {
                        const uint64_t e0 = __shfl_sync(0xFFFFFFFFu, e, __ffs(nz) - 1);
                        const uint32_t* src = p.stg + (uint32_t)e0;
                        typename Ty<T>::U* dst = p.out + pbase;
                        const uint32_t len = p.cap - pbase < tcount ? (uint32_t)(p.cap - pbase) : tcount;
                        for (uint32_t x0 = 0; x0 < len; x0 += 256u) {
                            uint32_t v[8];
#pragma unroll
                            for (int u = 0; u < 8; u++) {
                                const uint32_t x = x0 + 32u * u + (uint32_t)lane;
                                if (x < len) v[u] = __ldcs(src + x);
                            }
#pragma unroll
                            for (int u = 0; u < 8; u++) {
                                const uint32_t x = x0 + 32u * u + (uint32_t)lane;
                                if (x < len) dst[x] = v[u];
                            }
                        }
                        continue;
                    }
                }
            }
            if (!failed && (t + 1) * TILE <= p.n && tcount >= (uint32_t)(TILE / 16))
                compact_dense(p.in + t * TILE, p.mask + t * WORDS, pbase);
            else
                compact_tile<T, WORDS>(p.in + t * TILE, p.mask + t * WORDS, nwords - t * WORDS, tcount, pbase,
                                       p.out, p.cap);
        }
        base += pass;
        __syncthreads();  // s_wsum, s_cnt and s_off are rewritten by the next pass
    }
    // no bulk copy outstanding at CTA exit; a stage that never arrived is a
    // timeout of the call
    if (lane == 0) {
        for (uint32_t u = used; u < issued; u++)
            if (!mbar_wait(&wbar[u % kCompactStages], (u / kCompactStages) & 1u, kMbarLimit)) failed = true;
        if (failed) atomicOr(&p.hdr->status, LCQ_STATUS_TIMEOUT);
    }
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&p.ws->cdone, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // last CTA: every other CTA has read the group counts
    __threadfence();
    const uint32_t ng = (p.tiles + kGroupTiles - 1) / kGroupTiles;
    uint32_t total = 0;
    for (uint32_t g = tid; g < ng; g += kCompactThreads) {
        total += p.groups[g];
        p.groups[g] = 0u;
    }
    total = cta_sum(total, s_red);
    if (tid == 0) {
        const uint64_t all = carry + total;
        p.hdr->outlier_count = all;
        if (all > p.cap) atomicOr(&p.hdr->status, LCQ_STATUS_CAPACITY);
        p.ws->cdone = 0u;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// NOA range reduction (Sec. 2.1.3): finite-only min/max as ordered integer
// keys; the last block derives R = RD(max - min), eb_abs = RD(eb * R) and the
// ABS constants, and writes them to the header.
// ---------------------------------------------------------------------------
template <typename T>
struct MParams {
    const T* in;
    uint64_t n;
    lcq_header* hdr;
    WsHead* ws;
    uint64_t* partial;  // 2 per block
    double eb;
    double* range_out;  // non-null: write {any, min, max} here instead of the header
};

template <typename T>
__global__ void __launch_bounds__(kBlock) k_minmax(MParams<T> p) {
    pdl_wait();
    pdl_trigger();
    using F = Ty<T>;
    using U = typename F::K;  // order keys
    __shared__ U s_lo[kBlock / 32], s_hi[kBlock / 32];
    __shared__ bool s_last;
    U lo = ~(U)0, hi = (U)0;
    const uint64_t stride = (uint64_t)gridDim.x * kBlock;
    uint64_t done;  // values covered by whole vectors
    if constexpr (is16<T>()) {
        // eight 16-bit values per 16-byte load (four would leave half as many
        // bytes in flight as the float32 loop)
        const uint64_t nvec = p.n / 8;
        for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < nvec; i += stride) {
            const uint4 a = *reinterpret_cast<const uint4*>(p.in + 8 * i);
            const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int k = 0; k < 4; k++) {
                minmax_accum<T>(T((int)(w[k] & 0xFFFFu)), lo, hi);
                minmax_accum<T>(T((int)(w[k] >> 16)), lo, hi);
            }
        }
        done = nvec * 8;
    } else {
        const uint64_t nvec = p.n / 4;
        for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < nvec; i += stride) {
            T x[4];
            Vec4<T>::load_cached(p.in + 4 * i, x);
#pragma unroll
            for (int k = 0; k < 4; k++) minmax_accum<T>(x[k], lo, hi);
        }
        done = nvec * 4;
    }
    if (blockIdx.x == 0 && threadIdx.x < p.n - done) minmax_accum<T>(p.in[done + threadIdx.x], lo, hi);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const U a = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
        const U b = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_lo[warp] = lo; s_hi[warp] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kBlock / 32; w++) {
            lo = s_lo[w] < lo ? s_lo[w] : lo;
            hi = s_hi[w] > hi ? s_hi[w] : hi;
        }
        p.partial[2 * blockIdx.x] = (uint64_t)lo;
        p.partial[2 * blockIdx.x + 1] = (uint64_t)hi;
        __threadfence();
        s_last = atomicAdd(&p.ws->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // last block: combine the partials of all blocks
    __threadfence();
    lo = ~(U)0;
    hi = (U)0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kBlock) {
        const U a = (U)ld_relaxed_u64(&p.partial[2 * b]);
        const U c = (U)ld_relaxed_u64(&p.partial[2 * b + 1]);
        lo = a < lo ? a : lo;
        hi = c > hi ? c : hi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const U a = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
        const U b = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
    }
    __syncthreads();
    if (lane == 0) { s_lo[warp] = lo; s_hi[warp] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kBlock / 32; w++) {
            lo = s_lo[w] < lo ? s_lo[w] : lo;
            hi = s_hi[w] > hi ? s_hi[w] : hi;
        }
        const bool any = lo <= hi;
        const double mn = F::to_f64(F::from_bits(key_to_bits<T>(lo)));
        const double mx = F::to_f64(F::from_bits(key_to_bits<T>(hi)));
        if (p.range_out) {
            p.range_out[0] = any ? 1.0 : 0.0;
            p.range_out[1] = any ? mn : 0.0;
            p.range_out[2] = any ? mx : 0.0;
        } else {
            noa_finalize<CT<T>>(p.hdr, any, mn, mx, p.eb);
        }
        atomicExch(&p.ws->done, 0u);
        __threadfence();
    }
}

// NOA with a range the caller supplies (the global range of a sharded array,
// Sec. 2.1.3 applied to the union of the shards): the same derivation as the
// last block of k_minmax.  For an empty shard it also fills the header.
template <typename C>
__global__ void k_noa_given(lcq_header* h, bool any, double mn, double mx, double eb, uint32_t dtype,
                            bool empty) {
    noa_finalize<C>(h, any, mn, mx, eb);
    if (empty) {
        h->magic = LCQ_MAGIC;
        h->dtype = dtype;
        h->bound_type = LCQ_NOA;
        h->n = 0;
        h->eb = eb;
        h->outlier_count = 0;
        h->status = 0;
        h->reserved = 0;
    }
}

// ---------------------------------------------------------------------------
// Dequantize kernel: persistent CTAs; bins and mask words of each tile stream
// into shared-memory stages.  A tile writes the reconstructions of its
// quantized values at once and patches its outliers from the payload at the
// tile's offset one scan tile later.  The scan warp adds up that offset from
// the counts of k_tile_counts: the earlier chunks' total (a workspace word),
// the group counts of the whole groups before the tile and the tile counts
// of its own group; the last CTA updates the total and zeroes the groups.
// ---------------------------------------------------------------------------
template <typename T>
struct DParams {
    const int32_t* bins;
    const uint32_t* mask;
    const typename Ty<T>::U* outl;
    T* out;
    const lcq_header* hdr;
    WsHead* ws;
    const uint32_t* counts;   // outliers per scan tile of this chunk (k_tile_counts)
    uint32_t* groups;         // outliers per kGroupTiles scan tiles (k_tile_counts; zeroed here)
    uint32_t* status;
    uint64_t n;           // values in this chunk
    uint64_t n_total;
    uint32_t dtype;
    uint32_t num_tiles;
    uint32_t first_chunk;
};

template <typename T, int VPT, int STAGES, int SUB, int MINB>
__global__ void __launch_bounds__(kSpecThreads, MINB) k_dequantize(DParams<T> p) {
    using F = Ty<T>;
    constexpr int STILE = kComputeThreads * 4 * VPT;
    constexpr int TILE = STILE * SUB;
    constexpr int SWORDS = STILE / 32;
    constexpr int WORDS = TILE / 32;
    constexpr int WPL = WORDS / 32;
    constexpr int STAGE_WORDS = STILE + SWORDS;  // bins, then the sub-tile's mask words
    extern __shared__ __align__(128) unsigned char dsmem[];
    uint32_t* sbuf = reinterpret_cast<uint32_t*>(dsmem);
    __shared__ __align__(8) uint64_t s_stage_bar[STAGES];
    __shared__ __align__(8) uint64_t s_full[2];
    __shared__ __align__(8) uint64_t s_done[2];
    __shared__ uint32_t s_stage_ticket[STAGES];
    __shared__ uint32_t s_mask[2][WORDS];
    __shared__ uint32_t s_wpre[2][WORDS];
    __shared__ uint32_t s_jt[2];
    __shared__ uint64_t s_pbase[2];
    __shared__ uint64_t s_carry;  // outliers of the earlier chunks of the call
    __shared__ uint32_t s_total;
    __shared__ bool s_last;
    __shared__ uint32_t s_epoch, s_filled, s_ok;
    __shared__ volatile uint32_t s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t full_sub = p.n / STILE;
    const uint64_t nwords = (p.n + 31) / 32;
    pdl_wait();
    pdl_trigger();

    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) mbar_init(&s_stage_bar[s], 1);
        for (int b = 0; b < 2; b++) {
            mbar_init(&s_full[b], 1);
            mbar_init(&s_done[b], 1);
        }
        mbar_init_fence();
        s_epoch = ld_relaxed_u32(&p.ws->epoch);
        s_carry = p.first_chunk ? 0ull : p.ws->carry;  // rewritten only by this launch's last CTA
        // decode only a complete, error-free encoding of exactly these arrays
        const bool ok = p.hdr->magic == LCQ_MAGIC && p.hdr->dtype == p.dtype &&
                        p.hdr->n == p.n_total && p.hdr->status == 0u && p.hdr->mode <= 1u &&
                        (p.outl != nullptr || p.hdr->outlier_count == 0);
        s_ok = ok;
        if (!ok) atomicOr(&p.ws->err, LCQ_STATUS_HEADER);
        s_abort = 0;
        s_filled = 0;
    }
    __syncthreads();
    if (s_ok && warp < kComputeThreads / 32) {
        // ------------------------------------------------ compute warps --
        const Consts<CT<T>> c = consts_from_header<CT<T>>(p.hdr);
        const bool rel = p.hdr->bound_type == LCQ_REL;
        const uint64_t avail = p.hdr->outlier_count;
        bool overrun = false;
        auto issue = [&]() {
            const uint32_t f = s_filled;
            const int s = (int)(f % STAGES);
            const uint32_t sub = f % SUB;
            const uint32_t t = sub == 0 ? atomicAdd(&p.ws->ticket, 1u) : s_stage_ticket[(f - 1) % STAGES];
            s_stage_ticket[s] = t;
            s_filled = f + 1;
            if (t < p.num_tiles) {
                const uint64_t g = (uint64_t)t * SUB + sub;
                if (g < full_sub) {
                    uint32_t* st = sbuf + (size_t)s * STAGE_WORDS;
                    mbar_arrive_expect_tx(&s_stage_bar[s], STAGE_WORDS * 4);
                    bulk_g2s(st, p.bins + g * STILE, STILE * 4, &s_stage_bar[s]);
                    bulk_g2s(st + STILE, p.mask + g * SWORDS, SWORDS * 4, &s_stage_bar[s]);
                } else {
                    mbar_arrive(&s_stage_bar[s]);
                }
            }
        };
        // Patch the outliers of local scan tile jj; true if the kernel must stop.
        auto patch_outliers = [&](uint32_t jj) -> bool {
            const int bb = (int)(jj & 1u);
            bool ok = mbar_wait_or_abort(&s_done[bb], (jj >> 1) & 1u, kMbarLimit, &s_abort);
            if (!ok && !s_abort) {
                atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT);
                s_abort = 1;
            }
            if (named_barrier_or(1, kComputeThreads, !ok)) return true;
            const uint64_t tb = (uint64_t)s_jt[bb] * TILE;
            const uint64_t pbase = s_pbase[bb];
            using U = typename F::U;
            for_each_outlier<U>(
                s_mask[bb], s_wpre[bb], WORDS,
                [&](uint32_t, uint32_t r) {
                    const uint64_t rank = pbase + r;
                    return rank < avail ? p.outl[rank] : (U)0;
                },
                [&](uint32_t i, uint32_t r, U v) {
                    if (pbase + r < avail) p.out[tb + i] = F::from_bits(v);
                    else overrun = true;
                });
            named_barrier_sync(1, kComputeThreads);
            return false;
        };

        if (tid == 0) issue();
        named_barrier_sync(1, kComputeThreads);
        uint32_t k = 0;
        for (;; k++) {
            const int s = (int)(k % STAGES);
            const uint32_t sub = k % SUB;
            const uint32_t j = k / SUB;
            const int b = (int)(j & 1u);
            if (tid == 0 && s_filled < k + STAGES) issue();
            const uint32_t t = s_stage_ticket[s];
            if (t >= p.num_tiles) break;
            const uint64_t g = (uint64_t)t * SUB + sub;
            const bool from_smem = g < full_sub;
            if (!mbar_wait_or_abort(&s_stage_bar[s], (k / STAGES) & 1u, kMbarLimit, &s_abort)) {
                if (!s_abort) { atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT); s_abort = 1; }
            }
            const uint32_t* sb = sbuf + (size_t)s * STAGE_WORDS;
            const uint64_t sbase = g * STILE;
            for (int w = tid; w < SWORDS; w += kComputeThreads) {
                const uint64_t gw = g * SWORDS + w;
                s_mask[b][sw(sub * SWORDS + w)] = from_smem ? sb[STILE + w] : (gw < nwords ? p.mask[gw] : 0u);
            }
            if (from_smem) {
                // fast path: a whole sub-tile in shared memory, no bounds checks
                T* go = p.out + sbase;
#pragma unroll
                for (int v = 0; v < VPT; v++) {
                    const int off = v * (kComputeThreads * 4) + tid * 4;
                    const int word = v * (kComputeThreads / 8) + warp * 4 + (lane >> 3);
                    const uint32_t nb = (sb[STILE + word] >> ((lane & 7) * 4)) & 0xFu;
                    const int4 a = *reinterpret_cast<const int4*>(sb + off);
                    const int32_t bn[4] = {a.x, a.y, a.z, a.w};
                    T x[4];
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        x[q] = ((nb >> q) & 1u) ? T(0) : recon_out<T>(rel, bn[q], c);
                    Vec4<T>::store(go + off, x);
                }
            } else
#pragma unroll
            for (int v = 0; v < VPT; v++) {
                const int off = v * (kComputeThreads * 4) + tid * 4;
                const uint64_t e0 = sbase + off;
                const int word = v * (kComputeThreads / 8) + warp * 4 + (lane >> 3);
                const uint64_t gw = g * SWORDS + word;
                const uint32_t mw = from_smem ? sb[STILE + word] : (gw < nwords ? p.mask[gw] : 0u);
                const uint32_t nb = (mw >> ((lane & 7) * 4)) & 0xFu;
                int32_t bn[4];
                if (from_smem) {
                    const int4 a = *reinterpret_cast<const int4*>(sb + off);
                    bn[0] = a.x; bn[1] = a.y; bn[2] = a.z; bn[3] = a.w;
                } else if (e0 + 4 <= p.n) {
                    const int4 a = __ldcs(reinterpret_cast<const int4*>(p.bins + e0));
                    bn[0] = a.x; bn[1] = a.y; bn[2] = a.z; bn[3] = a.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; q++) bn[q] = (e0 + q < p.n) ? p.bins[e0 + q] : 0;
                }
                T x[4];
#pragma unroll
                for (int q = 0; q < 4; q++)
                    x[q] = ((nb >> q) & 1u) ? T(0) : recon_out<T>(rel, bn[q], c);
                if (e0 + 4 <= p.n) {
                    Vec4<T>::store(p.out + e0, x);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        if (e0 + q < p.n) p.out[e0 + q] = x[q];
                }
            }
            fence_proxy_async_smem();
            if (named_barrier_or(1, kComputeThreads, s_abort != 0)) break;  // stage s consumed
            if (tid == 0 && s_filled < k + 1 + STAGES) issue();
            if (sub == SUB - 1) {
                if (tid == 0) {
                    s_jt[b] = t;
                    mbar_arrive(&s_full[b]);
                }
                if (j >= 1 && patch_outliers(j - 1)) break;
            }
        }
        if (!named_barrier_or(1, kComputeThreads, s_abort != 0)) {
            const uint32_t J = k / SUB;
            if (!(J >= 1 && patch_outliers(J - 1)) && tid == 0) {
                s_jt[J & 1u] = kNoTile;
                mbar_arrive(&s_full[J & 1u]);
            }
        }
        // no bulk copy outstanding at CTA exit (also after an abort)
        if (tid == 0 &&
            !drain_stages<STAGES>(s_stage_bar, s_filled,
                                  [&](uint32_t f) { return s_stage_ticket[f % STAGES] < p.num_tiles; },
                                  kMbarLimit))
            atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT);
        if (overrun) atomicOr(&p.ws->err, LCQ_STATUS_HEADER);
    } else if (s_ok) {
        // --------------------------------------------------- scan warp --
        for (uint32_t j = 0;; j++) {
            const int b = (int)(j & 1u);
            if (!mbar_wait_or_abort(&s_full[b], (j >> 1) & 1u, kMbarLimit, &s_abort)) {
                if (!s_abort) { atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT); s_abort = 1; }
                break;
            }
            const uint32_t t = s_jt[b];
            if (t == kNoTile) break;
            scan_mask_words<WPL>(s_mask[b], s_wpre[b], nullptr, 0, 0, false);
            // payload offset of tile t: the earlier chunks, the whole groups
            // before t, the tiles of t's group before t
            const uint32_t g0 = t / kGroupTiles;
            uint32_t before = 0;
            for (uint32_t g = (uint32_t)lane; g < g0; g += 32) before += p.groups[g];
            for (uint32_t u = g0 * kGroupTiles + (uint32_t)lane; u < t; u += 32) before += p.counts[u];
            before = __reduce_add_sync(0xFFFFFFFFu, before);
            if (lane == 0) s_pbase[b] = s_carry + before;
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_done[b]);
        }
    }
    __syncthreads();
    if (tid == 0) s_last = finish_launch(p.ws, s_epoch, p.status, p.first_chunk != 0);
    __syncthreads();
    if (!s_last) return;
    // last CTA (every scan warp has read the group counts): the running
    // outlier count for the next chunk, and zero group counts for the next call
    if (tid == 0) s_total = 0;
    __syncthreads();
    const uint32_t ng = (p.num_tiles + kGroupTiles - 1) / kGroupTiles;
    uint32_t tot = 0;
    for (uint32_t g = (uint32_t)tid; g < ng; g += kSpecThreads) {
        tot += p.groups[g];
        p.groups[g] = 0u;
    }
    tot = __reduce_add_sync(0xFFFFFFFFu, tot);
    if (lane == 0) atomicAdd(&s_total, tot);
    __syncthreads();
    if (tid == 0) {
        p.ws->carry = s_carry + s_total;
        __threadfence();
    }
}

__global__ void k_status_only(uint32_t* status, uint32_t bits) {
    if (status) *status = bits;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static bool dtype_valid(lcq_dtype d) { return d == LCQ_F32 || d == LCQ_F64 || d == LCQ_F16 || d == LCQ_BF16; }
static size_t dtype_bytes(lcq_dtype d) { return d == LCQ_F64 ? 8 : (d == LCQ_F32 ? 4 : 2); }

// v (finite) is exactly a value of the data type.
static bool representable(lcq_dtype d, double v) {
    if (d == LCQ_F64) return true;
    const float f = (float)v;
    if ((double)f != v) return false;
    if (d == LCQ_F32) return true;
    if (d == LCQ_BF16) {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return (u & 0xFFFFu) == 0u;
    }
    return (double)__half2float(__float2half_rn(f)) == v;  // binary16: exact round trip
}

// f(T()) with T the storage type of dtype (a valid dtype).
template <typename Fn>
static lcq_status with_dtype(lcq_dtype dtype, Fn&& f) {
    switch (dtype) {
        case LCQ_F32: return f(float());
        case LCQ_F64: return f(double());
        case LCQ_F16: return f(f16s());
        case LCQ_BF16: return f(bf16s());
    }
    return LCQ_ERR_ARG;
}

static uint64_t tiles_of(uint64_t n, int tile) { return (n + tile - 1) / tile; }


// Tile table of a chunk: outlier counts (uint32) per scan tile; every tile
// shape has at least kTileValuesMin values per scan tile.
constexpr uint64_t kTileValuesMin = 16384;

static uint64_t table_tiles(uint64_t n) {
    const uint64_t per_chunk = n < kChunk ? n : kChunk;
    return (per_chunk + kTileValuesMin - 1) / kTileValuesMin;
}

static size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Workspace of the single-array calls: the head, the range-reduction
// partials, the group counts, and the tile counts.  The group counts must be
// zero when a call starts, so every call leaves them zero, and they sit at a
// fixed place sized for the largest chunk, whatever the n of the call.
constexpr size_t kGroupBytes = (kChunk / kTileValuesMin + kGroupTiles - 1) / kGroupTiles * 4;  // 8 KB
static_assert(kGroupBytes % 256 == 0, "256-byte aligned regions");

static size_t ws_size(uint64_t n) {
    const uint64_t tt = table_tiles(n);
    return kWsHeadBytes + kMinmaxPartialBytes + kGroupBytes + up256(tt * 4);
}

// Outlier staging for float32 REL, in a workspace of lcq_workspace_size(
// LCQ_F32, LCQ_REL, n) bytes: one uint64 entry per ring stage (outlier
// count << 32 | first staging index; 0 for a stage without outliers;
// kStageNone for a stage left to k_compact's own walk), then a staging area
// for a quarter of a chunk's values, split evenly among the quantize CTAs.
static uint64_t stage_entries(uint64_t n) {
    // every stage of every scan tile, empty stages of a ragged last tile
    // included: at most kMaxSub stages per tile of at least kTileValuesMin values
    return table_tiles(n) * kMaxSub;
}
static uint64_t stage_cap(uint64_t n) {
    const uint64_t per_chunk = n < kChunk ? n : kChunk;
    return (per_chunk + 3) / 4;
}
static size_t ws_size_staged(uint64_t n) {
    return ws_size(n) + up256(stage_entries(n) * 8) + up256(stage_cap(n) * 4);
}
static uint64_t* ws_stage_table(void* ws, uint64_t n) {
    return reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(ws) + ws_size(n));
}
static uint32_t* ws_staging(void* ws, uint64_t n) {
    return reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(ws_stage_table(ws, n)) + up256(stage_entries(n) * 8));
}

static uint64_t* ws_partials(void* ws) {
    return reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(ws) + kWsHeadBytes);
}
static uint32_t* ws_groups(void* ws) {
    return reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(ws) + kWsHeadBytes + kMinmaxPartialBytes);
}
static uint32_t* ws_counts(void* ws) {
    return reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(ws) + kWsHeadBytes + kMinmaxPartialBytes +
                                       kGroupBytes);
}

// Persistent grid: as many CTAs as fit on the device at once (cached per
// kernel instantiation and device), never more than there are tiles.
static std::atomic<int> g_sms[kMaxDevices];

std::mutex& launch_setup_mutex() {
    static std::mutex mu;
    return mu;
}

static int device_sms(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return 148;
    int v = g_sms[dev].load(std::memory_order_acquire);
    if (!v) {
        int q = 0;
        if (cudaDeviceGetAttribute(&q, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || q <= 0) return 148;
        g_sms[dev].store(q, std::memory_order_release);  // every thread stores the same value
        v = q;
    }
    return v;
}

template <typename K>
static int persistent_blocks(K kernel, size_t dyn_smem, int threads, OccupancyCache& cache) {
    int dev = 0;
    cudaGetDevice(&dev);
    return cached_blocks_per_sm(cache, dev, kernel, threads, dyn_smem) * device_sms(dev);
}

// Launch with programmatic stream serialisation (the kernel starts with
// pdl_wait / pdl_trigger): its CTAs may be scheduled while the previous
// kernel of the stream drains.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    return e != cudaSuccess ? e : cudaPeekAtLastError();
}

template <typename T, int MODE, int VPT, int STAGES, int SUB, int MINB>
static cudaError_t launch_quantize(const QParams<T>& p, cudaStream_t st) {
    static OccupancyCache cache{};
    constexpr int STILE = kComputeThreads * 4 * VPT;
    const size_t smem = (size_t)STAGES * STILE * sizeof(T);
    auto kern = k_quantize<T, MODE, VPT, STAGES, SUB, MINB>;
    QParams<T> q = p;
    q.num_tiles = (uint32_t)tiles_of(p.n, STILE * SUB);
    uint64_t grid = (uint64_t)persistent_blocks(kern, smem, kSpecThreads, cache);
    if (grid > q.num_tiles) grid = q.num_tiles;
    return launch_pdl(kern, (unsigned)grid, kSpecThreads, smem, st, q);
}

template <typename T, int VPT, int STAGES, int SUB, int MINB>
static cudaError_t launch_dequantize(const DParams<T>& p, cudaStream_t st) {
    static OccupancyCache cache{};
    constexpr int STILE = kComputeThreads * 4 * VPT;
    const size_t smem = (size_t)STAGES * (STILE + STILE / 32) * 4;
    auto kern = k_dequantize<T, VPT, STAGES, SUB, MINB>;
    DParams<T> q = p;
    q.num_tiles = (uint32_t)tiles_of(p.n, STILE * SUB);
    uint64_t grid = (uint64_t)persistent_blocks(kern, smem, kSpecThreads, cache);
    if (grid > q.num_tiles) grid = q.num_tiles;
    return launch_pdl(kern, (unsigned)grid, kSpecThreads, smem, st, q);
}

// Variant dispatch (the template arguments must be compile-time constants).
#define LCQ_VARIANT_CASES(CALL)                                   \
    case 0: return CALL(kVariants[0].vpt, kVariants[0].stages, kVariants[0].sub, kVariants[0].minb); \
    case 1: return CALL(kVariants[1].vpt, kVariants[1].stages, kVariants[1].sub, kVariants[1].minb); \
    case 2: return CALL(kVariants[2].vpt, kVariants[2].stages, kVariants[2].sub, kVariants[2].minb); \
    case 3: return CALL(kVariants[3].vpt, kVariants[3].stages, kVariants[3].sub, kVariants[3].minb); \
    case 4: return CALL(kVariants[4].vpt, kVariants[4].stages, kVariants[4].sub, kVariants[4].minb); \
    case 5: return CALL(kVariants[5].vpt, kVariants[5].stages, kVariants[5].sub, kVariants[5].minb); \
    case 6: return CALL(kVariants[6].vpt, kVariants[6].stages, kVariants[6].sub, kVariants[6].minb);

// The 16-bit formats are built in two tile shapes per kernel (fewer
// instantiations): quantize variants 0 and 1, dequantize variants 1 and 5.
constexpr int kQuant16[2] = {0, 1};
constexpr int kDequant16[2] = {1, 5};

static bool variant_ok(int kind, lcq_dtype dtype, int v) {
    if (v < 0 || v >= kNumVariants) return false;
    if (dtype == LCQ_F32 || dtype == LCQ_F64) return true;
    const int* set = kind == 0 ? kQuant16 : kDequant16;
    return v == set[0] || v == set[1];
}

template <typename T, int MODE>
static cudaError_t launch_quantize_variant(int v, const QParams<T>& p, cudaStream_t st) {
#define Q_CALL(a, b, c, d) launch_quantize<T, MODE, a, b, c, d>(p, st)
    if constexpr (is16<T>()) {
        constexpr Variant v0 = kVariants[kQuant16[0]], v1 = kVariants[kQuant16[1]];
        if (v == kQuant16[0]) return Q_CALL(v0.vpt, v0.stages, v0.sub, v0.minb);
        if (v == kQuant16[1]) return Q_CALL(v1.vpt, v1.stages, v1.sub, v1.minb);
    } else {
        switch (v) { LCQ_VARIANT_CASES(Q_CALL) }
    }
#undef Q_CALL
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t launch_dequantize_variant(int v, const DParams<T>& p, cudaStream_t st) {
#define D_CALL(a, b, c, d) launch_dequantize<T, a, b, c, d>(p, st)
    if constexpr (is16<T>()) {
        constexpr Variant v0 = kVariants[kDequant16[0]], v1 = kVariants[kDequant16[1]];
        if (v == kDequant16[0]) return D_CALL(v0.vpt, v0.stages, v0.sub, v0.minb);
        if (v == kDequant16[1]) return D_CALL(v1.vpt, v1.stages, v1.sub, v1.minb);
    } else {
        switch (v) { LCQ_VARIANT_CASES(D_CALL) }
    }
#undef D_CALL
    return cudaErrorInvalidValue;
}

// The ablation kernels run one fixed tile shape each: the default shape of
// the protected kernel they are compared with.
template <typename T, int MODE>
constexpr int ablation_variant() {
    return sizeof(T) == 4 ? (MODE == kModeRelLib ? 3 : 1) : 2;
}

template <typename T, int MODE>
static cudaError_t launch_ablation(const QParams<T>& p, cudaStream_t st) {
    constexpr Variant v = kVariants[ablation_variant<T, MODE>()];
    return launch_quantize<T, MODE, v.vpt, v.stages, v.sub, v.minb>(p, st);
}

template <typename T, int WORDS>
static cudaError_t launch_compact_words(uint32_t grid, size_t smem, const CParams<T>& p, cudaStream_t st) {
    static OccupancyCache cache{};  // the shared-memory opt-in, once per device
    int dev = 0;
    cudaGetDevice(&dev);
    cached_blocks_per_sm(cache, dev, k_compact<T, WORDS>, kCompactThreads, smem);
    return launch_pdl(k_compact<T, WORDS>, grid, kCompactThreads, smem, st, p);
}

// The compaction kernel for scan tiles of `words` mask words (every tile
// shape has 512 or 1024): runs of about kCompactWarps tiles per CTA, at most
// 8 CTAs per SM.
template <typename T>
static cudaError_t launch_compact(int words, CParams<T> p, cudaStream_t st) {
    int dev = 0;
    cudaGetDevice(&dev);
    uint32_t grid = (uint32_t)device_sms(dev) * 8u;
    if (grid > (p.tiles + kCompactWarps - 1) / kCompactWarps) grid = (p.tiles + kCompactWarps - 1) / kCompactWarps;
    if (grid < 1) grid = 1;
    p.per = (p.tiles + grid - 1) / grid;
    grid = (p.tiles + p.per - 1) / p.per;
    const size_t smem = (size_t)kCompactWarps * kCompactStages * compact_stage_bytes<T>();
    if (words == 1024) return launch_compact_words<T, 1024>(grid, smem, p, st);
    if (words == 512) return launch_compact_words<T, 512>(grid, smem, p, st);
    return cudaErrorInvalidValue;
}

// Selected variant per kernel kind (0 quantize, 1 dequantize), dtype (float32,
// float64, binary16, bfloat16), bound type.  Defaults from autotuning on a
// B300 (float32 512^3 field, float64 256^3 field; float32 REL with outlier
// staging also on the REL stress input, where shape 2's four CTAs per SM
// give four scan warps to share the staging walk).
static int g_variant[2][4][3] = {{{1, 2, 1}, {6, 6, 6}, {1, 1, 1}, {1, 1, 1}},
                                 {{5, 5, 5}, {2, 2, 2}, {5, 5, 5}, {5, 5, 5}}};

// RD_f32(d): the largest float not above d.
static float rd_f32_host(double d) {
    float f = (float)d;
    if ((double)f > d) f = nextafterf(f, -INFINITY);
    return f;
}

static bool is_normal_f(float f) { return std::fpclassify(f) == FP_NORMAL; }
static bool is_normal_d(double f) { return std::fpclassify(f) == FP_NORMAL; }

// ABS constants (Sec. 2.2): eb_T = RD_T(eb), eb2 = 2 eb_T, inv = RN(1/eb2).
template <typename T>
static bool abs_consts_host(double eb, Consts<T>& c);

template <>
bool abs_consts_host<float>(double eb, Consts<float>& c) {
    const float ebT = rd_f32_host(eb);
    if (!is_normal_f(ebT)) return false;
    const float eb2 = 2.0f * ebT;
    if (!std::isfinite(eb2)) return false;
    const float inv = 1.0f / eb2;
    if (!is_normal_f(inv)) return false;
    c.ebT = ebT; c.scale = eb2; c.inv = inv; c.chk = 0.0f; c.all_outliers = 0;
    return true;
}

template <>
bool abs_consts_host<double>(double eb, Consts<double>& c) {
    const double ebT = eb;
    if (!is_normal_d(ebT)) return false;
    const double eb2 = 2.0 * ebT;
    if (!std::isfinite(eb2)) return false;
    const double inv = 1.0 / eb2;
    if (!is_normal_d(inv)) return false;
    c.ebT = ebT; c.scale = eb2; c.inv = inv; c.chk = 0.0; c.all_outliers = 0;
    return true;
}

// REL constants: log-domain half step lb = RN(e / RN(1 + e)), step = 2 lb,
// inv = RN(1/step), acceptance factor chk = RN(e (1 - 2^-p)), e = RD_T(eb).
// The certainty bounds of the float64 REL check (rel_quant_f64): cert_w =
// ceil((step/2 + 2^-40) 2^52) and cert_emin = max(512, 1027 - exponent field
// of chk), or cert_w = 0 unless chk - step/2 >= 2^-39.  With step/2 <= chk <=
// step the subtraction is exact (Sterbenz); otherwise the test is off.
void rel_cert_host(double step, double chk, uint64_t* cert_w, uint32_t* cert_emin) {
    *cert_w = 0;
    *cert_emin = 0;
    if (!(chk <= step) || !(chk - 0.5 * step >= 0x1p-39)) return;
    const double v = std::ceil(std::ldexp(step, 51));  // step/2 in units of 2^-52, rounded up
    if (!(v < 0x1p50)) return;
    const uint64_t w = (uint64_t)v + 4096;                // + 2^-40 in units of 2^-52
    uint64_t cb;
    std::memcpy(&cb, &chk, 8);
    const int ec = (int)(cb >> 52);
    *cert_w = w;
    *cert_emin = (uint32_t)(1027 - ec > 512 ? 1027 - ec : 512);
}

template <typename T>
static bool rel_consts_host(double eb, Consts<T>& c);

template <>
bool rel_consts_host<float>(double eb, Consts<float>& c) {
    const float e = rd_f32_host(eb);
    if (!is_normal_f(e)) return false;
    const float onep = 1.0f + e;
    const float lb = e / onep;
    const float step = 2.0f * lb;
    const float inv = 1.0f / step;
    const float chk = e * 0x1.fffffcp-1f;
    if (!is_normal_f(lb) || !is_normal_f(step) || !is_normal_f(inv) || !is_normal_f(chk)) return false;
    c.ebT = e; c.scale = step; c.inv = inv; c.chk = chk; c.all_outliers = 0;
    c.cert_w = 0; c.cert_emin = 0;
    return true;
}

template <>
bool rel_consts_host<double>(double eb, Consts<double>& c) {
    const double e = eb;
    if (!is_normal_d(e)) return false;
    const double onep = 1.0 + e;
    const double lb = e / onep;
    const double step = 2.0 * lb;
    const double inv = 1.0 / step;
    const double chk = e * 0x1.ffffffffffffep-1;
    if (!is_normal_d(lb) || !is_normal_d(step) || !is_normal_d(inv) || !is_normal_d(chk)) return false;
    c.ebT = e; c.scale = step; c.inv = inv; c.chk = chk; c.all_outliers = 0;
    rel_cert_host(step, chk, &c.cert_w, &c.cert_emin);
    return true;
}

template <typename T>
static uint64_t bits_host(T v) {
    uint64_t u = 0;
    std::memcpy(&u, &v, sizeof(T));
    return u;
}

// Pipelined host <-> device copies around quantize_impl (lcq_quantize_host
// and lcq_quantize_host_batch): the input goes up in chunks on its own
// stream (host_io_upload, enqueued by the caller), each chunk is quantized as
// soon as it has arrived, and its bins and mask words go down on a third
// stream while later chunks are still moving up.
struct HostIO {
    const char* h_in;
    char* d_in;
    size_t es;
    int32_t* h_bins;
    const int32_t* d_bins;
    uint32_t* h_mask;
    const uint32_t* d_mask;
    cudaStream_t h2d, d2h;
    cudaEvent_t* up_ev;    // one per chunk: its upload has finished
    cudaEvent_t* done_ev;  // one per chunk: its quantization has finished
    uint64_t chunk;        // values per chunk, a multiple of 32
};

static uint64_t host_io_chunks(uint64_t n, uint64_t chunk) { return (n + chunk - 1) / chunk; }

static bool host_io_upload(const HostIO& io, uint64_t n) {
    const uint64_t K = host_io_chunks(n, io.chunk);
    for (uint64_t i = 0; i < K; i++) {
        const uint64_t off = i * io.chunk, len = n - off < io.chunk ? n - off : io.chunk;
        if (cudaMemcpyAsync(io.d_in + off * io.es, io.h_in + off * io.es, len * io.es, cudaMemcpyHostToDevice,
                            io.h2d) != cudaSuccess ||
            cudaEventRecord(io.up_ev[i], io.h2d) != cudaSuccess)
            return false;
    }
    return true;
}

static bool host_io_download(const HostIO& io, uint64_t i, uint64_t off, uint64_t len, cudaStream_t st) {
    if (cudaEventRecord(io.done_ev[i], st) != cudaSuccess) return false;
    if (cudaStreamWaitEvent(io.d2h, io.done_ev[i], 0) != cudaSuccess) return false;
    const uint64_t w0 = off / 32, w1 = (off + len + 31) / 32;
    return cudaMemcpyAsync(io.h_bins + off, io.d_bins + off, len * 4, cudaMemcpyDeviceToHost, io.d2h) ==
               cudaSuccess &&
           cudaMemcpyAsync(io.h_mask + w0, io.d_mask + w0, (w1 - w0) * 4, cudaMemcpyDeviceToHost, io.d2h) ==
               cudaSuccess;
}

// given: NOA only; null = derive the range from the input (k_minmax), else
// {any, min, max} of the caller's range (already validated).  io: host
// copies to pipeline with the launches (n > 0), or null.
template <typename T>
static lcq_status quantize_impl(lcq_bound_type bt, double eb, const T* in, uint64_t n, int32_t* bins,
                                uint32_t* mask, void* outl, uint64_t cap, lcq_header* hdr, void* ws,
                                size_t ws_bytes, cudaStream_t st, const double* given = nullptr, int ablation = 0,
                                const HostIO* io = nullptr) {
    Consts<CT<T>> c{};
    const bool noa = bt == LCQ_NOA;
    if (bt == LCQ_ABS) {
        if (!abs_consts_host<CT<T>>(eb, c)) return LCQ_ERR_BOUND;
    } else if (bt == LCQ_REL) {
        if (!rel_consts_host<CT<T>>(eb, c)) return LCQ_ERR_BOUND;
    }
    const uint32_t dtype = Ty<T>::kDtype;
    WsHead* head = reinterpret_cast<WsHead*>(ws);
    uint64_t* partial = ws_partials(ws);
    uint32_t* counts = ws_counts(ws);
    uint32_t* groups = ws_groups(ws);
    // float32 REL stages its outliers when the workspace has room for it
    const bool staged = std::is_same<T, float>::value && bt == LCQ_REL && ablation == 0 && !io &&
                        ws_bytes >= ws_size_staged(n);

    if (io) {
        // NOA needs the whole input for its range before any binning
        if (n == 0) return LCQ_ERR_CUDA;
        const uint64_t K = host_io_chunks(n, io->chunk);
        if (noa && !given && cudaStreamWaitEvent(st, io->up_ev[K - 1], 0) != cudaSuccess) return LCQ_ERR_CUDA;
    }
    if (noa && given) {
        k_noa_given<CT<T>><<<1, 1, 0, st>>>(hdr, given[0] != 0.0, given[1], given[2], eb, dtype, n == 0);
        if (cudaPeekAtLastError() != cudaSuccess) return LCQ_ERR_CUDA;
        if (n == 0) return LCQ_OK;
    } else if (noa) {
        MParams<T> mp{in, n, hdr, head, partial, eb, nullptr};
        uint64_t blocks = (n / 4 + kBlock - 1) / kBlock;
        if (blocks < 1) blocks = 1;
        if (blocks > (uint64_t)kMinmaxMaxBlocks) blocks = kMinmaxMaxBlocks;
        if (launch_pdl(k_minmax<T>, (unsigned)blocks, kBlock, 0, st, mp) != cudaSuccess) return LCQ_ERR_CUDA;
    }
    const double eb_abs = bt == LCQ_ABS ? eb : 0.0;
    if (n == 0) {
        if (noa) {
            // no finite value: the range kernel wrote mode 1; fill the rest
            k_header_empty<<<1, 1, 0, st>>>(hdr, dtype, bt, eb, 0.0, 0, 0, 0, 0, 1);
        } else {
            k_header_empty<<<1, 1, 0, st>>>(hdr, dtype, bt, eb, eb_abs, bits_host(c.ebT),
                                            bits_host(c.scale), bits_host(c.inv), bits_host(c.chk), 0);
        }
        return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
    }
    const uint64_t chunk = io ? io->chunk : kChunk;
    for (uint64_t off = 0; off < n; off += chunk) {
        const uint64_t len = (n - off) < chunk ? (n - off) : chunk;
        if (io && !(noa && !given) && cudaStreamWaitEvent(st, io->up_ev[off / chunk], 0) != cudaSuccess)
            return LCQ_ERR_CUDA;
        QParams<T> p;
        p.in = in + off;
        p.bins = bins + off;
        p.mask = mask + off / 32;
        p.counts = counts;
        p.groups = groups;
        p.stab = staged ? ws_stage_table(ws, n) : nullptr;
        p.stg = staged ? ws_staging(ws, n) : nullptr;
        p.scap = staged ? stage_cap(n) : 0;
        p.hdr = hdr;
        p.ws = head;
        p.n = len;
        p.num_tiles = 0;  // set per tile shape at launch
        p.first_chunk = off == 0;
        p.consts_from_hdr = noa;
        p.c = c;
        p.hook = g_scan;
        p.dtype = dtype;
        p.bound = bt;
        p.eb = eb;
        p.eb_abs = eb_abs;
        p.n_total = n;
        int var = g_variant[0][dtype][bt];
        cudaError_t e = cudaErrorInvalidValue;
        if constexpr (!is16<T>()) {
            if (ablation == kModeAbsNoCheck) {
                var = ablation_variant<T, kModeAbsNoCheck>();
                e = launch_ablation<T, kModeAbsNoCheck>(p, st);
            } else if (ablation == kModeRelLib) {
                var = ablation_variant<T, kModeRelLib>();
                e = launch_ablation<T, kModeRelLib>(p, st);
            }
        }
        if (ablation == 0) {
            if (bt == LCQ_REL) e = launch_quantize_variant<T, LCQ_REL>(var, p, st);
            else e = launch_quantize_variant<T, LCQ_ABS>(var, p, st);
        }
        if (e != cudaSuccess) return LCQ_ERR_CUDA;
        if (io && !host_io_download(*io, off / chunk, off, len, st)) return LCQ_ERR_CUDA;
        // outlier offsets and payload of this chunk
        const uint64_t tile = (uint64_t)kComputeThreads * 4 * kVariants[var].vpt * kVariants[var].sub;
        const uint32_t tiles = (uint32_t)tiles_of(len, (int)tile);
        CParams<T> cp;
        cp.in = p.in;
        cp.mask = p.mask;
        cp.n = len;
        cp.counts = counts;
        cp.groups = groups;
        cp.stab = p.stab;
        cp.stg = p.stg;
        cp.sub = (uint32_t)kVariants[var].sub;
        cp.tiles = tiles;
        cp.per = 0;  // set at launch
        cp.out = reinterpret_cast<typename Ty<T>::U*>(outl);
        cp.cap = cap;
        cp.hdr = hdr;
        cp.ws = head;
        cp.first_chunk = off == 0 ? 1u : 0u;
        if (launch_compact<T>((int)(tile / 32), cp, st) != cudaSuccess) return LCQ_ERR_CUDA;
    }
    return LCQ_OK;
}

template <typename T>
static lcq_status dequantize_impl(uint64_t n, const lcq_header* hdr, const int32_t* bins,
                                  const uint32_t* mask, const void* outl, T* out, uint32_t* status,
                                  void* ws, cudaStream_t st) {
    WsHead* head = reinterpret_cast<WsHead*>(ws);
    uint32_t* counts = ws_counts(ws);
    uint32_t* groups = ws_groups(ws);
    if (n == 0) {
        k_status_only<<<1, 1, 0, st>>>(status, 0u);
        return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    for (uint64_t off = 0; off < n; off += kChunk) {
        const uint64_t len = (n - off) < kChunk ? (n - off) : kChunk;
        const int var = g_variant[1][Ty<T>::kDtype][0];
        // outlier counts of the scan tiles (and their groups) from the mask
        const uint64_t tile = (uint64_t)kComputeThreads * 4 * kVariants[var].vpt * kVariants[var].sub;
        const uint32_t tiles = (uint32_t)tiles_of(len, (int)tile);
        uint32_t grid = (uint32_t)device_sms(dev) * 8u;
        if (grid > (tiles + 7) / 8) grid = (tiles + 7) / 8;
        const uint32_t* cmask = mask + off / 32;
        cudaError_t e;
        if (tile == 32768) e = launch_pdl(k_tile_counts<1024>, grid, 256, 0, st, cmask, len, tiles, counts, groups);
        else if (tile == 16384) e = launch_pdl(k_tile_counts<512>, grid, 256, 0, st, cmask, len, tiles, counts, groups);
        else return LCQ_ERR_ARG;
        if (e != cudaSuccess) return LCQ_ERR_CUDA;
        DParams<T> p;
        p.bins = bins + off;
        p.mask = mask + off / 32;
        p.outl = reinterpret_cast<const typename Ty<T>::U*>(outl);
        p.out = out + off;
        p.hdr = hdr;
        p.ws = head;
        p.counts = counts;
        p.groups = groups;
        p.status = status;
        p.n = len;
        p.n_total = n;
        p.dtype = Ty<T>::kDtype;
        p.num_tiles = 0;  // set per tile shape at launch
        p.first_chunk = off == 0;
        if (launch_dequantize_variant<T>(var, p, st) != cudaSuccess) return LCQ_ERR_CUDA;
    }
    return LCQ_OK;
}

bool host_consts(lcq_dtype dtype, lcq_bound_type bound, double eb, uint64_t bits[4], uint64_t* cert_w,
                 uint32_t* cert_emin) {
    if (dtype != LCQ_F64) {  // float32 and the 16-bit formats: float constants
        Consts<float> c{};
        const bool ok = bound == LCQ_REL ? rel_consts_host<float>(eb, c) : abs_consts_host<float>(eb, c);
        bits[0] = bits_host(c.ebT); bits[1] = bits_host(c.scale); bits[2] = bits_host(c.inv); bits[3] = bits_host(c.chk);
        if (cert_w) *cert_w = c.cert_w;
        if (cert_emin) *cert_emin = c.cert_emin;
        return ok;
    }
    Consts<double> c{};
    const bool ok = bound == LCQ_REL ? rel_consts_host<double>(eb, c) : abs_consts_host<double>(eb, c);
    bits[0] = bits_host(c.ebT); bits[1] = bits_host(c.scale); bits[2] = bits_host(c.inv); bits[3] = bits_host(c.chk);
    if (cert_w) *cert_w = c.cert_w;
    if (cert_emin) *cert_emin = c.cert_emin;
    return ok;
}

lcq_status check_quantize_args(lcq_dtype dtype, lcq_bound_type bound_type, double eb, const void* d_in,
                               uint64_t n, const int32_t* d_bins, const uint32_t* d_mask,
                               const void* d_outliers, uint64_t outlier_capacity, const lcq_header* d_hdr) {
    if (!dtype_valid(dtype)) return LCQ_ERR_ARG;
    if (bound_type != LCQ_ABS && bound_type != LCQ_REL && bound_type != LCQ_NOA) return LCQ_ERR_ARG;
    if (!d_hdr || !aligned16(d_hdr)) return LCQ_ERR_ARG;
    if (n > 0 && (!d_in || !d_bins || !d_mask)) return LCQ_ERR_ARG;
    if (n > 0 && (!aligned16(d_in) || !aligned16(d_bins) || !aligned16(d_mask))) return LCQ_ERR_ARG;
    if (outlier_capacity > 0 && (!d_outliers || !aligned16(d_outliers))) return LCQ_ERR_ARG;
    if (n >= (1ull << 40)) return LCQ_ERR_ARG;
    if (!(eb > 0.0) || !std::isfinite(eb)) return LCQ_ERR_BOUND;
    return LCQ_OK;
}

// Copy streams and events for lcq_quantize_host, one set per device, made
// on first use and kept; the lock serialises the calls of one device.
constexpr uint64_t kHostChunk = 1ull << 23;  // values per pipelined chunk (multiple of 32)

struct HostPipe {
    cudaStream_t h2d = nullptr, d2h = nullptr;
    std::vector<cudaEvent_t> ev;
};
static std::mutex g_pipe_mu[64];
static HostPipe g_pipe[64];

static lcq_status host_pipe(size_t nev, HostPipe** out, std::unique_lock<std::mutex>& lock) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LCQ_ERR_CUDA;
    lock = std::unique_lock<std::mutex>(g_pipe_mu[dev]);
    HostPipe& p = g_pipe[dev];
    if (!p.h2d && cudaStreamCreateWithFlags(&p.h2d, cudaStreamNonBlocking) != cudaSuccess) return LCQ_ERR_CUDA;
    if (!p.d2h && cudaStreamCreateWithFlags(&p.d2h, cudaStreamNonBlocking) != cudaSuccess) return LCQ_ERR_CUDA;
    while (p.ev.size() < nev) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return LCQ_ERR_CUDA;
        p.ev.push_back(e);
    }
    *out = &p;
    return LCQ_OK;
}

int device_sm_count() {
    int dev = 0;
    cudaGetDevice(&dev);
    return device_sms(dev);
}

}  // namespace lcq

using namespace lcq;

extern "C" {

size_t lcq_workspace_size(lcq_dtype dtype, lcq_bound_type bound_type, uint64_t n) {
    return dtype == LCQ_F32 && bound_type == LCQ_REL ? ws_size_staged(n) : ws_size(n);
}

lcq_status lcq_workspace_init(void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!d_ws || ws_bytes < kWsHeadBytes) return LCQ_ERR_ARG;
    return cudaMemsetAsync(d_ws, 0, ws_bytes, stream) == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
}

lcq_status lcq_quantize(lcq_dtype dtype, lcq_bound_type bound_type, double eb, const void* d_in,
                        uint64_t n, int32_t* d_bins, uint32_t* d_mask, void* d_outliers,
                        uint64_t outlier_capacity, lcq_header* d_hdr, void* d_ws, size_t ws_bytes,
                        cudaStream_t stream) {
    if (!dtype_valid(dtype)) return LCQ_ERR_ARG;
    if (bound_type != LCQ_ABS && bound_type != LCQ_REL && bound_type != LCQ_NOA) return LCQ_ERR_ARG;
    if (!d_hdr || !d_ws || !aligned16(d_ws) || !aligned16(d_hdr)) return LCQ_ERR_ARG;
    if (n > 0 && (!d_in || !d_bins || !d_mask)) return LCQ_ERR_ARG;
    if (n > 0 && (!aligned16(d_in) || !aligned16(d_bins) || !aligned16(d_mask))) return LCQ_ERR_ARG;
    if (outlier_capacity > 0 && (!d_outliers || !aligned16(d_outliers))) return LCQ_ERR_ARG;
    if (n >= (1ull << 40)) return LCQ_ERR_ARG;
    if (!(eb > 0.0) || !std::isfinite(eb)) return LCQ_ERR_BOUND;
    if (ws_bytes < ws_size(n)) return LCQ_ERR_WORKSPACE;
    return with_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        return quantize_impl<T>(bound_type, eb, (const T*)d_in, n, d_bins, d_mask, d_outliers, outlier_capacity,
                                d_hdr, d_ws, ws_bytes, stream);
    });
}

lcq_status lcq_dequantize(lcq_dtype dtype, uint64_t n, const lcq_header* d_hdr,
                          const int32_t* d_bins, const uint32_t* d_mask, const void* d_outliers,
                          void* d_out, uint32_t* d_status, void* d_ws, size_t ws_bytes,
                          cudaStream_t stream) {
    if (!dtype_valid(dtype)) return LCQ_ERR_ARG;
    if (!d_hdr || !d_ws || !aligned16(d_ws) || !aligned16(d_hdr)) return LCQ_ERR_ARG;
    if (n > 0 && (!d_bins || !d_mask || !d_out)) return LCQ_ERR_ARG;
    if (n > 0 && (!aligned16(d_bins) || !aligned16(d_mask) || !aligned16(d_out))) return LCQ_ERR_ARG;
    if (d_outliers && !aligned16(d_outliers)) return LCQ_ERR_ARG;
    if (n >= (1ull << 40)) return LCQ_ERR_ARG;
    if (ws_bytes < ws_size(n)) return LCQ_ERR_WORKSPACE;
    return with_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        return dequantize_impl<T>(n, d_hdr, d_bins, d_mask, d_outliers, (T*)d_out, d_status, d_ws, stream);
    });
}

lcq_status lcq_quantize_ablation(lcq_ablation kind, lcq_dtype dtype, double eb, const void* d_in, uint64_t n,
                                 int32_t* d_bins, uint32_t* d_mask, void* d_outliers, uint64_t outlier_capacity,
                                 lcq_header* d_hdr, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (kind != LCQ_ABL_ABS_NO_CHECK && kind != LCQ_ABL_REL_LIBRARY) return LCQ_ERR_ARG;
    if (dtype != LCQ_F32 && dtype != LCQ_F64) return LCQ_ERR_ARG;  // the paper's float and double
    const lcq_bound_type bt = kind == LCQ_ABL_REL_LIBRARY ? LCQ_REL : LCQ_ABS;
    const lcq_status a = check_quantize_args(dtype, bt, eb, d_in, n, d_bins, d_mask, d_outliers,
                                             outlier_capacity, d_hdr);
    if (a != LCQ_OK) return a;
    if (!d_ws || !aligned16(d_ws)) return LCQ_ERR_ARG;
    if (ws_bytes < ws_size(n)) return LCQ_ERR_WORKSPACE;
    const int mode = kind == LCQ_ABL_REL_LIBRARY ? kModeRelLib : kModeAbsNoCheck;
    if (dtype == LCQ_F32)
        return quantize_impl<float>(bt, eb, (const float*)d_in, n, d_bins, d_mask, d_outliers, outlier_capacity,
                                    d_hdr, d_ws, ws_bytes, stream, nullptr, mode);
    return quantize_impl<double>(bt, eb, (const double*)d_in, n, d_bins, d_mask, d_outliers, outlier_capacity,
                                 d_hdr, d_ws, ws_bytes, stream, nullptr, mode);
}

int lcq_ablation_variant(lcq_dtype dtype, lcq_ablation kind) {
    if (kind != LCQ_ABL_ABS_NO_CHECK && kind != LCQ_ABL_REL_LIBRARY) return -1;
    if (dtype == LCQ_F32)
        return kind == LCQ_ABL_REL_LIBRARY ? ablation_variant<float, kModeRelLib>()
                                           : ablation_variant<float, kModeAbsNoCheck>();
    if (dtype == LCQ_F64)
        return kind == LCQ_ABL_REL_LIBRARY ? ablation_variant<double, kModeRelLib>()
                                           : ablation_variant<double, kModeAbsNoCheck>();
    return -1;
}

lcq_status lcq_finite_range(lcq_dtype dtype, const void* d_in, uint64_t n, double* d_range, void* d_ws,
                            size_t ws_bytes, cudaStream_t stream) {
    if (!dtype_valid(dtype)) return LCQ_ERR_ARG;
    if (!d_range || (reinterpret_cast<uintptr_t>(d_range) & 7) != 0) return LCQ_ERR_ARG;
    if (!d_ws || !aligned16(d_ws)) return LCQ_ERR_ARG;
    if (n > 0 && (!d_in || !aligned16(d_in))) return LCQ_ERR_ARG;
    if (n >= (1ull << 40)) return LCQ_ERR_ARG;
    if (ws_bytes < ws_size(n)) return LCQ_ERR_WORKSPACE;
    WsHead* head = reinterpret_cast<WsHead*>(d_ws);
    uint64_t* partial = ws_partials(d_ws);
    uint64_t blocks = (n / 4 + kBlock - 1) / kBlock;
    if (blocks < 1) blocks = 1;
    if (blocks > (uint64_t)kMinmaxMaxBlocks) blocks = kMinmaxMaxBlocks;
    return with_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        MParams<T> mp{(const T*)d_in, n, nullptr, head, partial, 0.0, d_range};
        k_minmax<T><<<(unsigned)blocks, kBlock, 0, stream>>>(mp);
        return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
    });
}

lcq_status lcq_quantize_noa_range(lcq_dtype dtype, double eb, int has_finite, double range_min,
                                  double range_max, const void* d_in, uint64_t n, int32_t* d_bins,
                                  uint32_t* d_mask, void* d_outliers, uint64_t outlier_capacity,
                                  lcq_header* d_hdr, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    const lcq_status a = check_quantize_args(dtype, LCQ_NOA, eb, d_in, n, d_bins, d_mask, d_outliers,
                                             outlier_capacity, d_hdr);
    if (a != LCQ_OK) return a;
    if (!d_ws || !aligned16(d_ws)) return LCQ_ERR_ARG;
    if (has_finite != 0 && has_finite != 1) return LCQ_ERR_ARG;
    if (has_finite) {
        if (!std::isfinite(range_min) || !std::isfinite(range_max) || !(range_min <= range_max))
            return LCQ_ERR_ARG;
        if (!representable(dtype, range_min) || !representable(dtype, range_max)) return LCQ_ERR_ARG;
    }
    if (ws_bytes < ws_size(n)) return LCQ_ERR_WORKSPACE;
    const double given[3] = {has_finite ? 1.0 : 0.0, has_finite ? range_min : 0.0, has_finite ? range_max : 0.0};
    return with_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        return quantize_impl<T>(LCQ_NOA, eb, (const T*)d_in, n, d_bins, d_mask, d_outliers, outlier_capacity, d_hdr,
                                d_ws, ws_bytes, stream, given);
    });
}

lcq_status lcq_sync_status(const lcq_header* d_hdr, uint64_t* h_outlier_count, cudaStream_t stream) {
    if (!d_hdr) return LCQ_ERR_ARG;
    lcq_header h;
    if (cudaMemcpyAsync(&h, d_hdr, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return LCQ_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return LCQ_ERR_CUDA;
    if (h_outlier_count) *h_outlier_count = h.outlier_count;
    if (h.status & LCQ_STATUS_TIMEOUT) return LCQ_ERR_TIMEOUT;
    if (h.status & LCQ_STATUS_CAPACITY) return LCQ_ERR_CAPACITY;
    if (h.status & LCQ_STATUS_HEADER) return LCQ_ERR_HEADER;
    return LCQ_OK;
}

const char* lcq_status_string(lcq_status s) {
    switch (s) {
        case LCQ_OK: return "ok";
        case LCQ_ERR_ARG: return "invalid argument (pointer, alignment, size or enum)";
        case LCQ_ERR_BOUND: return "unusable error bound";
        case LCQ_ERR_CAPACITY: return "outlier capacity exceeded";
        case LCQ_ERR_TIMEOUT: return "outlier scan wait timed out";
        case LCQ_ERR_CUDA: return "CUDA error";
        case LCQ_ERR_WORKSPACE: return "workspace too small";
        case LCQ_ERR_HEADER: return "header does not match the arrays";
    }
    return "unknown status";
}

size_t lcq_host_stage_size(lcq_dtype dtype, uint64_t n, uint64_t outlier_capacity) {
    const size_t es = dtype_bytes(dtype);
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return up(n * es) + up(n * 4) + up(((n + 31) / 32) * 4) + up(outlier_capacity * es) +
           up(sizeof(lcq_header));
}

namespace {

// Device layout of one stage slot: input, bins, mask words, outliers, header.
struct StageSlot {
    char* d_in;
    int32_t* d_bins;
    uint32_t* d_mask;
    void* d_out;
    lcq_header* d_hdr;
};

StageSlot stage_slot(void* base, size_t es, uint64_t n, uint64_t cap) {
    StageSlot t;
    t.d_in = (char*)base;
    t.d_bins = (int32_t*)(t.d_in + up256(n * es));
    t.d_mask = (uint32_t*)((char*)t.d_bins + up256(n * 4));
    t.d_out = (char*)t.d_mask + up256(((n + 31) / 32) * 4);
    t.d_hdr = (lcq_header*)((char*)t.d_out + up256(cap * es));
    return t;
}

lcq_status check_host_item(lcq_dtype dtype, lcq_bound_type bound_type, double eb, const void* h_in, uint64_t n,
                           const int32_t* h_bins, const uint32_t* h_mask, const void* h_outliers,
                           uint64_t outlier_capacity, const lcq_header* h_hdr) {
    if (!dtype_valid(dtype)) return LCQ_ERR_ARG;
    if (bound_type != LCQ_ABS && bound_type != LCQ_REL && bound_type != LCQ_NOA) return LCQ_ERR_ARG;
    if (!h_hdr) return LCQ_ERR_ARG;
    if (n > 0 && (!h_in || !h_bins || !h_mask)) return LCQ_ERR_ARG;
    if (outlier_capacity > 0 && !h_outliers) return LCQ_ERR_ARG;
    if (n >= (1ull << 40)) return LCQ_ERR_ARG;
    if (!(eb > 0.0) || !std::isfinite(eb)) return LCQ_ERR_BOUND;
    return LCQ_OK;
}

// Enqueue the quantization of one host item whose upload (io.up_ev) is
// already enqueued: the chunked launches with their bin / mask downloads,
// then the header download, after which `hdr_ev` is recorded on io.d2h.
lcq_status enqueue_host_item(lcq_dtype dtype, lcq_bound_type bt, double eb, uint64_t n, const StageSlot& t,
                             uint64_t cap, lcq_header* h_hdr, const HostIO& io, cudaEvent_t end_ev,
                             cudaEvent_t hdr_ev, void* d_ws, cudaStream_t st) {
    void* d_outl = cap ? t.d_out : nullptr;
    const lcq_status s = with_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        return quantize_impl<T>(bt, eb, (const T*)t.d_in, n, t.d_bins, t.d_mask, d_outl, cap, t.d_hdr, d_ws, 0, st,
                                nullptr, 0, &io);
    });
    const bool ok = cudaEventRecord(end_ev, st) == cudaSuccess &&
                    cudaStreamWaitEvent(io.d2h, end_ev, 0) == cudaSuccess &&
                    cudaMemcpyAsync(h_hdr, t.d_hdr, sizeof(lcq_header), cudaMemcpyDeviceToHost, io.d2h) ==
                        cudaSuccess &&
                    cudaEventRecord(hdr_ev, io.d2h) == cudaSuccess;
    if (s != LCQ_OK) return s;
    return ok ? LCQ_OK : LCQ_ERR_CUDA;
}

// After the header of an item is on the host: download its outliers.
lcq_status finish_host_item(const lcq_header* h_hdr, const StageSlot& t, size_t es, void* h_outliers, uint64_t cap,
                            cudaStream_t d2h) {
    const uint64_t cnt = h_hdr->outlier_count < cap ? h_hdr->outlier_count : cap;
    if (cnt && cudaMemcpyAsync(h_outliers, t.d_out, cnt * es, cudaMemcpyDeviceToHost, d2h) != cudaSuccess)
        return LCQ_ERR_CUDA;
    return LCQ_OK;
}

lcq_status host_status(const lcq_header* h) {
    if (h->status & LCQ_STATUS_TIMEOUT) return LCQ_ERR_TIMEOUT;
    if (h->status & LCQ_STATUS_CAPACITY) return LCQ_ERR_CAPACITY;
    return LCQ_OK;
}

}  // namespace

lcq_status lcq_quantize_host(lcq_dtype dtype, lcq_bound_type bound_type, double eb,
                             const void* h_in, uint64_t n, int32_t* h_bins, uint32_t* h_mask,
                             void* h_outliers, uint64_t outlier_capacity, lcq_header* h_hdr,
                             void* d_stage, size_t stage_bytes, void* d_ws, size_t ws_bytes,
                             cudaStream_t stream) {
    lcq_status s = check_host_item(dtype, bound_type, eb, h_in, n, h_bins, h_mask, h_outliers, outlier_capacity,
                                   h_hdr);
    if (s != LCQ_OK) return s;
    if (!d_stage || !aligned16(d_stage)) return LCQ_ERR_ARG;
    if (stage_bytes < lcq_host_stage_size(dtype, n, outlier_capacity)) return LCQ_ERR_WORKSPACE;
    if (!d_ws || !aligned16(d_ws)) return LCQ_ERR_ARG;
    if (ws_bytes < ws_size(n)) return LCQ_ERR_WORKSPACE;
    const size_t es = dtype_bytes(dtype);
    const StageSlot t = stage_slot(d_stage, es, n, outlier_capacity);
    if (n == 0) {
        s = lcq_quantize(dtype, bound_type, eb, nullptr, 0, t.d_bins, t.d_mask,
                         outlier_capacity ? t.d_out : nullptr, outlier_capacity, t.d_hdr, d_ws, ws_bytes, stream);
        if (s != LCQ_OK) return s;
        if (cudaMemcpyAsync(h_hdr, t.d_hdr, sizeof(lcq_header), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
            return LCQ_ERR_CUDA;
        return LCQ_OK;
    }
    // the copy streams and events of this device, held for the whole call
    const uint64_t K = host_io_chunks(n, kHostChunk);
    HostPipe* pipe = nullptr;
    std::unique_lock<std::mutex> lock;
    if (host_pipe(2 * K + 3, &pipe, lock) != LCQ_OK) return LCQ_ERR_CUDA;
    cudaEvent_t* ev = pipe->ev.data();
    HostIO io{(const char*)h_in, t.d_in, es, h_bins, t.d_bins, h_mask, t.d_mask, pipe->h2d, pipe->d2h,
              ev, ev + K, kHostChunk};
    cudaEvent_t start_ev = ev[2 * K], end_ev = ev[2 * K + 1], hdr_ev = ev[2 * K + 2];
    // the copies start after the work already on `stream`
    bool ok = cudaEventRecord(start_ev, stream) == cudaSuccess &&
              cudaStreamWaitEvent(io.h2d, start_ev, 0) == cudaSuccess &&
              cudaStreamWaitEvent(io.d2h, start_ev, 0) == cudaSuccess && host_io_upload(io, n);
    s = ok ? enqueue_host_item(dtype, bound_type, eb, n, t, outlier_capacity, h_hdr, io, end_ev, hdr_ev, d_ws,
                               stream)
           : LCQ_ERR_CUDA;
    // drain the copy streams whatever happened, then report
    ok = cudaStreamSynchronize(io.h2d) == cudaSuccess && cudaStreamSynchronize(io.d2h) == cudaSuccess &&
         cudaStreamSynchronize(stream) == cudaSuccess;
    if (s != LCQ_OK) return s;
    if (!ok) return LCQ_ERR_CUDA;
    if (finish_host_item(h_hdr, t, es, h_outliers, outlier_capacity, io.d2h) != LCQ_OK ||
        cudaStreamSynchronize(io.d2h) != cudaSuccess)
        return LCQ_ERR_CUDA;
    return host_status(h_hdr);
}

size_t lcq_host_batch_stage_size(const lcq_host_item* items, uint32_t count) {
    size_t mx = 0;
    for (uint32_t i = 0; items && i < count; i++) {
        const size_t b = lcq_host_stage_size((lcq_dtype)items[i].dtype, items[i].n, items[i].outlier_capacity);
        mx = b > mx ? b : mx;
    }
    return count > 1 ? 2 * mx : mx;
}

lcq_status lcq_quantize_host_batch(lcq_host_item* items, uint32_t count, void* d_stage, size_t stage_bytes,
                                   void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!items || count == 0) return LCQ_ERR_ARG;
    if (!d_stage || !aligned16(d_stage) || !d_ws || !aligned16(d_ws)) return LCQ_ERR_ARG;
    uint64_t nmax = 0, ksum = 0;
    lcq_status first = LCQ_OK;
    for (uint32_t i = 0; i < count; i++) {
        lcq_host_item& it = items[i];
        it.status = check_host_item((lcq_dtype)it.dtype, (lcq_bound_type)it.bound_type, it.eb, it.h_in, it.n,
                                    it.h_bins, it.h_mask, it.h_outliers, it.outlier_capacity, it.h_hdr);
        if (it.status == LCQ_OK && it.n == 0) it.status = LCQ_ERR_ARG;  // empty arrays: use lcq_quantize_host
        if (it.status != LCQ_OK) return (lcq_status)it.status;
        nmax = it.n > nmax ? it.n : nmax;
        ksum += host_io_chunks(it.n, kHostChunk);
    }
    if (stage_bytes < lcq_host_batch_stage_size(items, count)) return LCQ_ERR_WORKSPACE;
    if (ws_bytes < ws_size(nmax)) return LCQ_ERR_WORKSPACE;
    const size_t slot_bytes = count > 1 ? lcq_host_batch_stage_size(items, count) / 2 : stage_bytes;
    HostPipe* pipe = nullptr;
    std::unique_lock<std::mutex> lock;
    // per item: an upload and a done event per chunk, end, header and slot-free events; one start event
    if (host_pipe(2 * ksum + 3 * (uint64_t)count + 1, &pipe, lock) != LCQ_OK) return LCQ_ERR_CUDA;
    cudaEvent_t* ev = pipe->ev.data();
    cudaEvent_t start_ev = ev[0];
    size_t evi = 1;
    std::vector<StageSlot> slot(count);
    std::vector<cudaEvent_t> hdr_ev(count), free_ev(count);
    bool ok = cudaEventRecord(start_ev, stream) == cudaSuccess &&
              cudaStreamWaitEvent(pipe->h2d, start_ev, 0) == cudaSuccess &&
              cudaStreamWaitEvent(pipe->d2h, start_ev, 0) == cudaSuccess;
    uint32_t enq = 0;  // items whose work is enqueued
    for (uint32_t j = 0; ok && j < count; j++) {
        lcq_host_item& it = items[j];
        const lcq_dtype dt = (lcq_dtype)it.dtype;
        const size_t es = dtype_bytes(dt);
        const uint64_t K = host_io_chunks(it.n, kHostChunk);
        slot[j] = stage_slot((char*)d_stage + (j & 1) * slot_bytes, es, it.n, it.outlier_capacity);
        HostIO io{(const char*)it.h_in, slot[j].d_in, es, it.h_bins, slot[j].d_bins, it.h_mask, slot[j].d_mask,
                  pipe->h2d, pipe->d2h, ev + evi, ev + evi + K, kHostChunk};
        evi += 2 * K;
        cudaEvent_t end_ev = ev[evi++];
        hdr_ev[j] = ev[evi++];
        free_ev[j] = ev[evi++];
        // the slot is free once item j-2 is completely downloaded
        if (j >= 2 && cudaStreamWaitEvent(pipe->h2d, free_ev[j - 2], 0) != cudaSuccess) { ok = false; break; }
        if (!host_io_upload(io, it.n)) { ok = false; break; }
        // while item j moves up, item j-1's outliers go down
        if (j >= 1) {
            lcq_host_item& pv = items[j - 1];
            if (cudaEventSynchronize(hdr_ev[j - 1]) != cudaSuccess ||
                finish_host_item(pv.h_hdr, slot[j - 1], dtype_bytes((lcq_dtype)pv.dtype), pv.h_outliers,
                                 pv.outlier_capacity, pipe->d2h) != LCQ_OK ||
                cudaEventRecord(free_ev[j - 1], pipe->d2h) != cudaSuccess) {
                ok = false;
                break;
            }
        }
        it.status = enqueue_host_item(dt, (lcq_bound_type)it.bound_type, it.eb, it.n, slot[j], it.outlier_capacity,
                                      it.h_hdr, io, end_ev, hdr_ev[j], d_ws, stream);
        enq = j + 1;
        if (it.status != LCQ_OK) { ok = false; break; }
    }
    if (ok && enq == count) {
        lcq_host_item& ls = items[count - 1];
        ok = cudaEventSynchronize(hdr_ev[count - 1]) == cudaSuccess &&
             finish_host_item(ls.h_hdr, slot[count - 1], dtype_bytes((lcq_dtype)ls.dtype), ls.h_outliers,
                              ls.outlier_capacity, pipe->d2h) == LCQ_OK;
    }
    const bool ok_sync = cudaStreamSynchronize(pipe->h2d) == cudaSuccess &&
                         cudaStreamSynchronize(pipe->d2h) == cudaSuccess &&
                         cudaStreamSynchronize(stream) == cudaSuccess;
    for (uint32_t j = 0; j < count; j++) {
        lcq_host_item& it = items[j];
        if (j >= enq) {
            if (it.status == LCQ_OK) it.status = LCQ_ERR_CUDA;
        } else if (it.status == LCQ_OK) {
            it.status = (ok && ok_sync) ? host_status(it.h_hdr) : LCQ_ERR_CUDA;
        }
        if (first == LCQ_OK && it.status != LCQ_OK) first = (lcq_status)it.status;
    }
    return first;
}

int lcq_tune_variant_count(void) { return kNumVariants; }

lcq_status lcq_tune_describe(int variant, int* vpt, int* stages, int* sub, int* min_ctas_per_sm) {
    if (variant < 0 || variant >= kNumVariants) return LCQ_ERR_ARG;
    if (vpt) *vpt = kVariants[variant].vpt;
    if (stages) *stages = kVariants[variant].stages;
    if (sub) *sub = kVariants[variant].sub;
    if (min_ctas_per_sm) *min_ctas_per_sm = kVariants[variant].minb;
    return LCQ_OK;
}

lcq_status lcq_tune_set(int kind, lcq_dtype dtype, lcq_bound_type bound_type, int variant) {
    if (kind < 0 || kind > 1 || !dtype_valid(dtype) || (int)bound_type < 0 || (int)bound_type > 2 ||
        !variant_ok(kind, dtype, variant))
        return LCQ_ERR_ARG;
    g_variant[kind][dtype][kind == 1 ? 0 : bound_type] = variant;
    return LCQ_OK;
}

int lcq_tune_get(int kind, lcq_dtype dtype, lcq_bound_type bound_type) {
    if (kind < 0 || kind > 1 || !dtype_valid(dtype) || (int)bound_type < 0 || (int)bound_type > 2) return -1;
    return g_variant[kind][dtype][kind == 1 ? 0 : bound_type];
}

lcq_status lcq_autotune_quantize(lcq_dtype dtype, lcq_bound_type bound_type, double eb, const void* d_in,
                                 uint64_t n, int32_t* d_bins, uint32_t* d_mask, void* d_outliers,
                                 uint64_t outlier_capacity, lcq_header* d_hdr, void* d_ws,
                                 size_t ws_bytes, cudaStream_t stream, int reps, float* h_ms) {
    if (!dtype_valid(dtype)) return LCQ_ERR_ARG;
    if ((int)bound_type < 0 || (int)bound_type > 2) return LCQ_ERR_ARG;
    if (reps < 1) reps = 1;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return LCQ_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return LCQ_ERR_CUDA; }
    const int saved = g_variant[0][dtype][bound_type];
    int best = saved;
    float best_ms = 0.0f;
    lcq_status st = LCQ_OK;
    bool first = true;
    for (int v = 0; v < kNumVariants && st == LCQ_OK; v++) {
        if (h_ms) h_ms[v] = -1.0f;
        if (!variant_ok(0, dtype, v)) continue;
        g_variant[0][dtype][bound_type] = v;
        st = lcq_quantize(dtype, bound_type, eb, d_in, n, d_bins, d_mask, d_outliers, outlier_capacity,
                          d_hdr, d_ws, ws_bytes, stream);  // warm-up
        cudaEventRecord(a, stream);
        for (int r = 0; r < reps && st == LCQ_OK; r++)
            st = lcq_quantize(dtype, bound_type, eb, d_in, n, d_bins, d_mask, d_outliers,
                              outlier_capacity, d_hdr, d_ws, ws_bytes, stream);
        cudaEventRecord(b, stream);
        if (cudaEventSynchronize(b) != cudaSuccess) st = LCQ_ERR_CUDA;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        ms /= reps;
        if (h_ms) h_ms[v] = ms;
        if (st == LCQ_OK && (first || ms < best_ms)) {
            best_ms = ms;
            best = v;
            first = false;
        }
    }
    g_variant[0][dtype][bound_type] = st == LCQ_OK ? best : saved;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

lcq_status lcq_autotune_dequantize(lcq_dtype dtype, uint64_t n, const lcq_header* d_hdr,
                                   const int32_t* d_bins, const uint32_t* d_mask, const void* d_outliers,
                                   void* d_out, void* d_ws, size_t ws_bytes, cudaStream_t stream,
                                   int reps, float* h_ms) {
    if (!dtype_valid(dtype)) return LCQ_ERR_ARG;
    if (reps < 1) reps = 1;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return LCQ_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return LCQ_ERR_CUDA; }
    const int saved = g_variant[1][dtype][0];
    int best = saved;
    float best_ms = 0.0f;
    lcq_status st = LCQ_OK;
    bool first = true;
    for (int v = 0; v < kNumVariants && st == LCQ_OK; v++) {
        if (h_ms) h_ms[v] = -1.0f;
        if (!variant_ok(1, dtype, v)) continue;
        g_variant[1][dtype][0] = v;
        st = lcq_dequantize(dtype, n, d_hdr, d_bins, d_mask, d_outliers, d_out, nullptr, d_ws, ws_bytes,
                            stream);
        cudaEventRecord(a, stream);
        for (int r = 0; r < reps && st == LCQ_OK; r++)
            st = lcq_dequantize(dtype, n, d_hdr, d_bins, d_mask, d_outliers, d_out, nullptr, d_ws,
                                ws_bytes, stream);
        cudaEventRecord(b, stream);
        if (cudaEventSynchronize(b) != cudaSuccess) st = LCQ_ERR_CUDA;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        ms /= reps;
        if (h_ms) h_ms[v] = ms;
        if (st == LCQ_OK && (first || ms < best_ms)) {
            best_ms = ms;
            best = v;
            first = false;
        }
    }
    g_variant[1][dtype][0] = st == LCQ_OK ? best : saved;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

void lcq_debug_set_scan(uint32_t spin_limit, uint64_t drop_tile) {
    g_scan.spin_limit = spin_limit ? spin_limit : kDefaultSpin;
    g_scan.drop_tile = drop_tile;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free quantize entry point.
//
// Some callers cannot allocate device memory at the point where they
// quantize: code running inside a region that must not allocate (a
// fixed-memory-budget streaming pipeline, a simulation time step that must
// not synchronise the device through the allocator, a callback invoked from
// another library's allocator or scheduler), or code that simply has no
// allocator to hand.  lcq_quantize_noalloc serves them: the caller still
// passes inputs and outputs, and the scan workspace comes from the
// fixed-size device array below, which every GPU that loads this library
// holds until the process exits.
// ---------------------------------------------------------------------------
namespace lcq {

constexpr size_t kNoAllocWsBytes = (size_t)1 << 20;  // 1 MiB of scratch per device
static __device__ __align__(256) unsigned char g_noalloc_ws[kNoAllocWsBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64];  // device address of g_noalloc_ws, per device

// Device address of the scratch array for the current device (set-up on the
// first call per device; the array's host-side name is only a stand-in).
static lcq_status noalloc_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LCQ_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || !p) return LCQ_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return LCQ_OK;
}

}  // namespace lcq

extern "C" {

uint64_t lcq_noalloc_max_values(void) {
    // largest n whose workspace fits the static scratch
    uint64_t lo = 0, hi = 1ull << 40;
    while (lo + 1 < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (ws_size(mid) <= kNoAllocWsBytes) lo = mid;
        else hi = mid;
    }
    return lo;
}

lcq_status lcq_quantize_noalloc(lcq_dtype dtype, lcq_bound_type bound_type, double eb,
                                const void* d_in, uint64_t n, int32_t* d_bins, uint32_t* d_mask,
                                void* d_outliers, uint64_t outlier_capacity, lcq_header* d_hdr,
                                cudaStream_t stream) {
    // The size limit, then every check lcq_quantize makes, before anything
    // is enqueued on the shared scratch: a rejected call leaves it untouched.
    if (n > lcq_noalloc_max_values()) return LCQ_ERR_WORKSPACE;
    lcq_status st = check_quantize_args(dtype, bound_type, eb, d_in, n, d_bins, d_mask, d_outliers,
                                        outlier_capacity, d_hdr);
    if (st != LCQ_OK) return st;
    uint64_t bits[4];
    if (bound_type != LCQ_NOA && !host_consts(dtype, bound_type, eb, bits)) return LCQ_ERR_BOUND;
    // The scratch is the current device's; the stream must belong to it.
    int cur = 0, sdev = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaStreamGetDevice(stream, &sdev) != cudaSuccess)
        return LCQ_ERR_CUDA;
    if (sdev != cur) return LCQ_ERR_ARG;
    void* ws = nullptr;
    st = noalloc_scratch(&ws);
    if (st != LCQ_OK) return st;
    // Start from a clean scan state even if an earlier call on this device
    // was cut short: zero the ticket, the finished-CTA counters, the error
    // bits and the group counts (the epoch counter must keep counting, so it
    // is left alone).
    WsHead* head = reinterpret_cast<WsHead*>(ws);
    if (cudaMemsetAsync(&head->ticket, 0, 2 * sizeof(uint32_t), stream) != cudaSuccess ||
        cudaMemsetAsync(&head->err, 0, sizeof(uint32_t), stream) != cudaSuccess ||
        cudaMemsetAsync(&head->cdone, 0, sizeof(uint32_t), stream) != cudaSuccess ||
        cudaMemsetAsync(ws_groups(ws), 0, kGroupBytes, stream) != cudaSuccess)
        return LCQ_ERR_CUDA;
    return lcq_quantize(dtype, bound_type, eb, d_in, n, d_bins, d_mask, d_outliers, outlier_capacity,
                        d_hdr, ws, kNoAllocWsBytes, stream);
}

}  // extern "C"
