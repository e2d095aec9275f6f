// lcq_batch.cu -- batched quantization: many arrays of different sizes, data
// types, bound types and bounds in one header/range pass, ONE persistent
// quantize launch and two compaction launches (the method per array is that
// of lcq_quant.cu, Fallin & Burtscher, arXiv 2407.15037, Sec. 2.1-3.3; the
// batching itself has no counterpart in the paper).
//
// Every array is cut into scan tiles of 16384 values.  A global ticket hands
// out scan tiles of all arrays in array order; a CTA maps its ticket to the
// array by binary search over the plan's tile prefix, streams the tile's
// stages through its shared-memory ring (16 KB stages by default: 4096
// float32 or 2048 float64 values each; a 16-bit stage holds 4096 values in
// 8 KB), quantizes them with the same
// per-value code as the single-array kernel, and its scan warp stores the
// tile's mask words and outlier count; no CTA waits for another.  Then
// k_batch_offsets scans each array's tile counts into payload offsets (one
// CTA per array) and k_batch_compact writes the outliers, one warp per tile.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "lcq_device.cuh"
#include "lcq_host.h"
#include "lcq_pipe.cuh"
#include "lcq_tile.cuh"

namespace lcq {
namespace batch {

constexpr int kScanTile = 16384;        // values per scan tile, every dtype
constexpr int kWords = kScanTile / 32;  // mask words per scan tile
constexpr int kWpl = kWords / 32;       // per scan-warp lane
constexpr int kRangeChunk = 16384;      // values per range-reduction chunk
constexpr int kRangeBlock = 256;
constexpr uint32_t kMbarLimit = 1u << 22;

// One array of the plan (device memory, read-only for the kernels).
struct alignas(16) Array {
    const void* in;
    int32_t* bins;
    uint32_t* mask;
    void* out;
    lcq_header* hdr;
    uint64_t n;
    uint64_t cap;
    uint64_t tile_begin;  // first global scan tile
    uint32_t num_tiles;
    uint32_t dtype;
    uint32_t bound;
    uint32_t pad;
    double eb;
    uint64_t bits[4];  // ABS/REL constants: ebT, scale, inv, chk (NOA: in the header)
    uint64_t cert_w;   // float64 REL certainty bounds (Consts::cert_w / cert_emin)
    uint32_t cert_emin;
    uint32_t pad2;
};

struct PlanHead {
    uint32_t count, noa_count;
    uint64_t total_tiles, noa_chunks;
    uint64_t pad[5];
};

// Plan layout: PlanHead | Array[count] | uint64 tile_begin[count+1] |
//              uint32 noa_index[noa_count] | uint64 noa_begin[noa_count+1]
static size_t plan_bytes_for(uint32_t count) {
    return sizeof(PlanHead) + (size_t)count * sizeof(Array) + ((size_t)count + 1) * 8 + (size_t)count * 4 +
           ((size_t)count + 1) * 8 + 64;
}

struct PlanView {
    const Array* arr;
    const uint64_t* tile_begin;
    const uint32_t* noa_index;
    const uint64_t* noa_begin;
};

__host__ __device__ inline PlanView plan_view(const void* plan, uint32_t count, uint32_t noa_count) {
    const char* p = reinterpret_cast<const char*>(plan);
    const size_t off_arr = sizeof(PlanHead);
    const size_t off_tiles = off_arr + (size_t)count * sizeof(Array);
    const size_t off_noa = off_tiles + ((size_t)count + 1) * 8;
    const size_t off_noa_begin = (off_noa + (size_t)count * 4 + 7) & ~(size_t)7;
    PlanView v;
    v.arr = reinterpret_cast<const Array*>(p + off_arr);
    v.tile_begin = reinterpret_cast<const uint64_t*>(p + off_tiles);
    v.noa_index = reinterpret_cast<const uint32_t*>(p + off_noa);
    v.noa_begin = reinterpret_cast<const uint64_t*>(p + off_noa_begin);
    (void)noa_count;
    return v;
}

// Workspace: WsHead (256 B) | per-tile count / offset[total_tiles] | keys: min[count], max[count]
static size_t ws_bytes_for(uint64_t total_tiles, uint32_t count) {
    size_t d = (size_t)total_tiles * 8;
    d = (d + 255) & ~(size_t)255;
    return kWsHeadBytes + d + (size_t)count * 16;
}

// Index i with begin[i] <= x < begin[i+1] (begin has m+1 entries).
__device__ __forceinline__ uint32_t find_slot(const uint64_t* begin, uint32_t m, uint64_t x) {
    uint32_t lo = 0, hi = m;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (begin[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Pass 1: headers of every array, and the NOA ranges.
// ---------------------------------------------------------------------------
struct RParams {
    PlanView v;
    uint32_t count, noa_count;
    uint64_t noa_chunks;
    WsHead* ws;
    uint64_t* kmin;
    uint64_t* kmax;
};

template <typename T>
__device__ void range_chunk(const Array& A, uint64_t lc, uint64_t* kmin, uint64_t* kmax, uint32_t a) {
    using K = typename Ty<T>::K;  // order keys (32-bit for the 16-bit formats)
    __shared__ K s_lo[kRangeBlock / 32], s_hi[kRangeBlock / 32];
    const T* in = reinterpret_cast<const T*>(A.in);
    const uint64_t b0 = lc * kRangeChunk;
    const uint64_t e = A.n < b0 + kRangeChunk ? A.n : b0 + kRangeChunk;
    K lo = ~(K)0, hi = (K)0;
    // four values per load (chunks start at multiples of 16384 values, so
    // every vector is aligned), then the ragged end of the array
    const uint64_t nv = (e - b0) / 4;
    for (uint64_t v = threadIdx.x; v < nv; v += kRangeBlock) {
        T x[4];
        Vec4<T>::load_cached(in + b0 + 4 * v, x);
#pragma unroll
        for (int k = 0; k < 4; k++) minmax_accum<T>(x[k], lo, hi);
    }
    for (uint64_t i = b0 + 4 * nv + threadIdx.x; i < e; i += kRangeBlock) minmax_accum<T>(in[i], lo, hi);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const K x = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
        const K y = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
        lo = x < lo ? x : lo;
        hi = y > hi ? y : hi;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_lo[warp] = lo; s_hi[warp] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kRangeBlock / 32; w++) {
            lo = s_lo[w] < lo ? s_lo[w] : lo;
            hi = s_hi[w] > hi ? s_hi[w] : hi;
        }
        if (lo <= hi) {
            atomicMin(reinterpret_cast<unsigned long long*>(&kmin[a]), (unsigned long long)lo);
            atomicMax(reinterpret_cast<unsigned long long*>(&kmax[a]), (unsigned long long)hi);
        }
    }
    __syncthreads();
}

// The NOA bound of one array from its range keys (Sec. 2.1.3).
template <typename T>
__device__ void range_finalize(const Array& A, uint64_t lo, uint64_t hi) {
    using F = Ty<T>;
    using K = typename F::K;
    const bool any = lo <= hi;
    const double mn = any ? F::to_f64(F::from_bits(key_to_bits<T>((K)lo))) : 0.0;
    const double mx = any ? F::to_f64(F::from_bits(key_to_bits<T>((K)hi))) : 0.0;
    noa_finalize<CT<T>>(A.hdr, any, mn, mx, A.eb);
}

__global__ void __launch_bounds__(kRangeBlock) k_batch_range(RParams p) {
    // headers of every array (NOA constants come later, from the last block)
    for (uint64_t a = (uint64_t)blockIdx.x * kRangeBlock + threadIdx.x; a < p.count;
         a += (uint64_t)gridDim.x * kRangeBlock) {
        const Array& A = p.v.arr[a];
        lcq_header* h = A.hdr;
        h->magic = LCQ_MAGIC;
        h->dtype = A.dtype;
        h->bound_type = A.bound;
        h->n = A.n;
        h->eb = A.eb;
        h->range = 0.0;
        h->outlier_count = 0;
        h->status = 0;
        h->reserved = 0;
        if (A.bound != LCQ_NOA) {
            h->mode = 0;
            h->eb_abs = A.bound == LCQ_ABS ? A.eb : 0.0;
            h->ebT_bits = A.bits[0];
            h->scale_bits = A.bits[1];
            h->inv_bits = A.bits[2];
            h->chk_bits = A.bits[3];
        }
    }
    // NOA min/max over finite values, one 16384-value chunk per step
    for (uint64_t c = blockIdx.x; c < p.noa_chunks; c += gridDim.x) {
        const uint32_t i = find_slot(p.v.noa_begin, p.noa_count, c);
        const uint32_t a = p.v.noa_index[i];
        const Array& A = p.v.arr[a];
        const uint64_t lc = c - p.v.noa_begin[i];
        switch (A.dtype) {
            case LCQ_F32: range_chunk<float>(A, lc, p.kmin, p.kmax, a); break;
            case LCQ_F64: range_chunk<double>(A, lc, p.kmin, p.kmax, a); break;
            case LCQ_F16: range_chunk<f16s>(A, lc, p.kmin, p.kmax, a); break;
            default: range_chunk<bf16s>(A, lc, p.kmin, p.kmax, a); break;
        }
    }
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&p.ws->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last block: derive every NOA array's bound and reset its keys
    for (uint32_t i = threadIdx.x; i < p.noa_count; i += kRangeBlock) {
        const uint32_t a = p.v.noa_index[i];
        const Array& A = p.v.arr[a];
        const uint64_t lo = ld_relaxed_u64(&p.kmin[a]);
        const uint64_t hi = ld_relaxed_u64(&p.kmax[a]);
        switch (A.dtype) {
            case LCQ_F32: range_finalize<float>(A, lo, hi); break;
            case LCQ_F64: range_finalize<double>(A, lo, hi); break;
            case LCQ_F16: range_finalize<f16s>(A, lo, hi); break;
            default: range_finalize<bf16s>(A, lo, hi); break;
        }
        p.kmin[a] = ~0ull;
        p.kmax[a] = 0ull;
    }
    if (threadIdx.x == 0) atomicExch(&p.ws->done, 0u);
    __threadfence();
}

// ---------------------------------------------------------------------------
// Pass 2: one persistent, warp-specialised quantize launch over all tiles.
// ---------------------------------------------------------------------------
struct BParams {
    PlanView v;
    uint32_t count;
    uint64_t total_tiles;
    WsHead* ws;
    uint64_t* tiles;  // per global scan tile: outlier count, then (k_batch_offsets) payload offset
};

template <typename T, int MODE, int VPT>
__device__ __forceinline__ void batch_subtile(const Array& A, const void* stage, uint64_t first,
                                              uint32_t* s_words, int word_base) {
    constexpr int STILE = kComputeThreads * 4 * VPT;
    using C = CT<T>;  // float constants for float32 and the 16-bit formats
    Consts<C> c;
    if (A.bound == LCQ_NOA) {
        c = consts_from_header<C>(A.hdr);
    } else {
        using U = typename Ty<C>::U;
        c.ebT = Ty<C>::from_bits((U)A.bits[0]);
        c.scale = Ty<C>::from_bits((U)A.bits[1]);
        c.inv = Ty<C>::from_bits((U)A.bits[2]);
        c.chk = Ty<C>::from_bits((U)A.bits[3]);
        c.all_outliers = 0;
        c.cert_w = A.cert_w;
        c.cert_emin = A.cert_emin;
    }
    const bool full = first + STILE <= A.n;
    const uint64_t nvalid = A.n > first ? A.n - first : 0;
    quantize_subtile<T, MODE, VPT>(reinterpret_cast<const T*>(stage), reinterpret_cast<const T*>(A.in) + first,
                                   full, nvalid, A.bins + first, s_words, word_base, c);
}

template <int SB, int STAGES, int MINB>
__global__ void __launch_bounds__(kSpecThreads, MINB) k_batch_quantize(BParams p) {
    constexpr int VF = SB / 4 / (kComputeThreads * 4);  // float32 vectors per thread per stage
    constexpr int VD = SB / 8 / (kComputeThreads * 4);  // float64
    constexpr int STILE_F = SB / 4, STILE_D = SB / 8;   // values per stage
    // a 16-bit stage holds as many values as a float32 stage (half its bytes),
    // so its per-thread work is the float32 one
    static_assert(VD >= 1, "a stage must hold at least one float64 vector per thread");
    extern __shared__ __align__(128) unsigned char dsmem[];
    __shared__ __align__(8) uint64_t s_stage_bar[STAGES];
    __shared__ __align__(8) uint64_t s_full[2];
    __shared__ __align__(8) uint64_t s_done[2];
    __shared__ uint32_t s_st_tile[STAGES], s_st_arr[STAGES], s_st_sub[STAGES];
    __shared__ uint32_t s_mask[2][kWords];
    __shared__ uint32_t s_wpre[2][kWords];
    __shared__ uint32_t s_jt[2], s_ja[2];
    __shared__ uint32_t s_epoch, s_filled, s_cur_tile, s_cur_arr, s_cur_sub, s_cur_subs;
    __shared__ volatile uint32_t s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) mbar_init(&s_stage_bar[s], 1);
        for (int b = 0; b < 2; b++) {
            mbar_init(&s_full[b], 1);
            mbar_init(&s_done[b], 1);
        }
        mbar_init_fence();
        s_epoch = ld_relaxed_u32(&p.ws->epoch);
        s_abort = 0;
        s_filled = 0;
        s_cur_sub = 0;
        s_cur_subs = 0;
        s_cur_tile = kNoTile;
        s_cur_arr = 0;
    }
    __syncthreads();

    if (warp < kComputeThreads / 32) {
        // ------------------------------------------------ compute warps --
        auto issue = [&]() {  // thread 0: the next stage of this CTA's work
            const uint32_t f = s_filled;
            const int s = (int)(f % STAGES);
            if (s_cur_sub == s_cur_subs) {  // next scan tile
                const uint32_t t = atomicAdd(&p.ws->ticket, 1u);
                if (t < p.total_tiles) {
                    const uint32_t a = find_slot(p.v.tile_begin, p.count, t);
                    s_cur_tile = t;
                    s_cur_arr = a;
                    s_cur_subs = p.v.arr[a].dtype == LCQ_F64 ? kScanTile / STILE_D : kScanTile / STILE_F;
                } else {
                    s_cur_tile = kNoTile;
                    s_cur_subs = 1;
                }
                s_cur_sub = 0;
            }
            const uint32_t t = s_cur_tile, a = s_cur_arr, sub = s_cur_sub;
            s_st_tile[s] = t;
            s_st_arr[s] = a;
            s_st_sub[s] = sub;
            s_cur_sub = sub + 1;
            s_filled = f + 1;
            if (t != kNoTile) {
                const Array& A = p.v.arr[a];
                const bool f64 = A.dtype == LCQ_F64;
                const uint32_t es = f64 ? 8u : A.dtype == LCQ_F32 ? 4u : 2u;
                const uint64_t stile = f64 ? STILE_D : STILE_F;
                const uint32_t bytes = (uint32_t)(stile * es);
                const uint64_t first = (t - A.tile_begin) * (uint64_t)kScanTile + (uint64_t)sub * stile;
                void* dst = dsmem + (size_t)s * SB;
                if (first + stile <= A.n) {
                    mbar_arrive_expect_tx(&s_stage_bar[s], bytes);
                    bulk_g2s(dst, reinterpret_cast<const char*>(A.in) + first * es, bytes, &s_stage_bar[s]);
                } else {
                    mbar_arrive(&s_stage_bar[s]);  // ragged or empty stage: global reads
                }
            }
        };
        // Wait until the scan warp has taken local scan tile jj's mask words
        // (their buffer may then be reused); true if the kernel must stop.
        auto release_tile = [&](uint32_t jj) -> bool {
            const int bb = (int)(jj & 1u);
            bool ok = mbar_wait_or_abort(&s_done[bb], (jj >> 1) & 1u, kMbarLimit, &s_abort);
            if (!ok && !s_abort) {
                atomicOr(&p.v.arr[s_ja[bb]].hdr->status, LCQ_STATUS_TIMEOUT);
                s_abort = 1;
            }
            return named_barrier_or(1, kComputeThreads, !ok);
        };

        if (tid == 0) issue();
        named_barrier_sync(1, kComputeThreads);
        uint32_t j = 0;  // scan tiles completed by this CTA
        for (uint32_t k = 0;; k++) {
            const int s = (int)(k % STAGES);
            if (tid == 0 && s_filled < k + STAGES) issue();
            const uint32_t t = s_st_tile[s];
            if (t == kNoTile) break;
            const uint32_t a = s_st_arr[s], sub = s_st_sub[s];
            const int b = (int)(j & 1u);
            const Array& A = p.v.arr[a];
            if (!mbar_wait_or_abort(&s_stage_bar[s], (k / STAGES) & 1u, kMbarLimit, &s_abort)) {
                if (!s_abort) { atomicOr(&A.hdr->status, LCQ_STATUS_TIMEOUT); s_abort = 1; }
            }
            const void* stage = dsmem + (size_t)s * SB;
            const uint64_t tfirst = (t - A.tile_begin) * (uint64_t)kScanTile;
            const bool f64 = A.dtype == LCQ_F64;
            const uint32_t subs = f64 ? kScanTile / STILE_D : kScanTile / STILE_F;
            const uint64_t first = tfirst + (uint64_t)sub * (f64 ? STILE_D : STILE_F);
            const int wb = (int)sub * ((f64 ? STILE_D : STILE_F) / 32);
            const bool rel = A.bound == LCQ_REL;
            switch (A.dtype) {
                case LCQ_F32:
                    if (rel) batch_subtile<float, LCQ_REL, VF>(A, stage, first, s_mask[b], wb);
                    else batch_subtile<float, LCQ_ABS, VF>(A, stage, first, s_mask[b], wb);
                    break;
                case LCQ_F64:
                    if (rel) batch_subtile<double, LCQ_REL, VD>(A, stage, first, s_mask[b], wb);
                    else batch_subtile<double, LCQ_ABS, VD>(A, stage, first, s_mask[b], wb);
                    break;
                case LCQ_F16:
                    if (rel) batch_subtile<f16s, LCQ_REL, VF>(A, stage, first, s_mask[b], wb);
                    else batch_subtile<f16s, LCQ_ABS, VF>(A, stage, first, s_mask[b], wb);
                    break;
                default:
                    if (rel) batch_subtile<bf16s, LCQ_REL, VF>(A, stage, first, s_mask[b], wb);
                    else batch_subtile<bf16s, LCQ_ABS, VF>(A, stage, first, s_mask[b], wb);
                    break;
            }
            fence_proxy_async_smem();
            if (named_barrier_or(1, kComputeThreads, s_abort != 0)) break;  // stage s consumed
            if (tid == 0 && s_filled < k + 1 + STAGES) issue();
            if (sub == subs - 1) {
                if (tid == 0) {
                    s_jt[b] = t;
                    s_ja[b] = a;
                    mbar_arrive(&s_full[b]);
                }
                if (j >= 1 && release_tile(j - 1)) break;
                j++;
            }
        }
        if (!named_barrier_or(1, kComputeThreads, s_abort != 0)) {
            if (!(j >= 1 && release_tile(j - 1)) && tid == 0) {
                s_jt[j & 1u] = kNoTile;
                mbar_arrive(&s_full[j & 1u]);
            }
        }
        // no bulk copy outstanding at CTA exit (also after an abort)
        if (tid == 0 &&
            !drain_stages<STAGES>(s_stage_bar, s_filled,
                                  [&](uint32_t f) { return s_st_tile[f % STAGES] != kNoTile; }, kMbarLimit))
            atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT);
    } else {
        // --------------------------------------------------- scan warp --
        for (uint32_t jj = 0;; jj++) {
            const int b = (int)(jj & 1u);
            if (!mbar_wait_or_abort(&s_full[b], (jj >> 1) & 1u, kMbarLimit, &s_abort)) {
                if (!s_abort) { atomicOr(&p.ws->err, LCQ_STATUS_TIMEOUT); s_abort = 1; }
                break;
            }
            const uint32_t t = s_jt[b];
            if (t == kNoTile) break;
            const Array& A = p.v.arr[s_ja[b]];
            const uint32_t lt = (uint32_t)(t - A.tile_begin);
            const uint64_t nwords = (A.n + 31) / 32;
            const uint32_t agg = scan_mask_words<kWpl>(s_mask[b], s_wpre[b], A.mask,
                                                       (uint64_t)lt * kWords + (uint64_t)lane * kWpl, nwords, true);
            if (lane == 0) p.tiles[t] = agg;
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_done[b]);
        }
    }
    __syncthreads();
    if (tid == 0) finish_launch(p.ws, s_epoch, nullptr, false);
}

// ---------------------------------------------------------------------------
// Pass 3: payload offsets per array (one CTA per array: exclusive scan of its
// tiles' counts in place, the header's outlier count and capacity status).
// Pass 4: the outliers' raw bits, one warp per tile (compact_tile).
// ---------------------------------------------------------------------------
constexpr int kOffThreads = 256;

__global__ void __launch_bounds__(kOffThreads) k_batch_offsets(PlanView v, uint64_t* tiles) {
    __shared__ unsigned long long s_warp[kOffThreads / 32];
    __shared__ unsigned long long s_carry;
    const Array& A = v.arr[blockIdx.x];
    uint64_t* c = tiles + A.tile_begin;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t t0 = 0; t0 < A.num_tiles; t0 += kOffThreads) {
        const uint32_t t = t0 + (uint32_t)tid;
        const unsigned long long x0 = t < A.num_tiles ? c[t] : 0ull;
        unsigned long long x = x0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = lane < kOffThreads / 32 ? s_warp[lane] : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < kOffThreads / 32) s_warp[lane] = w;
        }
        __syncthreads();
        const unsigned long long excl = s_carry + (warp ? s_warp[warp - 1] : 0ull) + x - x0;
        if (t < A.num_tiles) c[t] = excl;  // every count of this pass was read above
        __syncthreads();
        if (tid == kOffThreads - 1) s_carry = excl + x0;
        __syncthreads();
    }
    if (tid == 0) {
        A.hdr->outlier_count = s_carry;
        if (s_carry > A.cap) atomicOr(&A.hdr->status, LCQ_STATUS_CAPACITY);
    }
}

template <typename T>
__device__ __forceinline__ void batch_compact_tile(const Array& A, uint32_t lt, uint64_t w0, uint64_t nwords,
                                                   uint32_t tcount, uint64_t off) {
    compact_tile<T, kWords>(reinterpret_cast<const T*>(A.in) + (uint64_t)lt * kScanTile, A.mask + w0, nwords - w0,
                            tcount, off, reinterpret_cast<typename Ty<T>::U*>(A.out), A.cap);
}

__global__ void __launch_bounds__(256) k_batch_compact(PlanView v, uint32_t count, uint64_t total_tiles,
                                                       const uint64_t* tiles) {
    const uint64_t wstride = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); t < total_tiles; t += wstride) {
        const uint32_t a = find_slot(v.tile_begin, count, t);
        const Array& A = v.arr[a];
        const uint32_t lt = (uint32_t)(t - A.tile_begin);
        const uint64_t off = tiles[t];
        const uint64_t next = lt + 1 < A.num_tiles ? tiles[t + 1] : A.hdr->outlier_count;
        const uint32_t tcount = (uint32_t)(next - off);
        if (tcount == 0u || off >= A.cap) continue;  // the same in every lane
        const uint64_t nwords = (A.n + 31) / 32;
        const uint64_t w0 = (uint64_t)lt * kWords;
        switch (A.dtype) {
            case LCQ_F32: batch_compact_tile<float>(A, lt, w0, nwords, tcount, off); break;
            case LCQ_F64: batch_compact_tile<double>(A, lt, w0, nwords, tcount, off); break;
            case LCQ_F16: batch_compact_tile<f16s>(A, lt, w0, nwords, tcount, off); break;
            default: batch_compact_tile<bf16s>(A, lt, w0, nwords, tcount, off); break;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct BVariant {
    int sb, stages, minb;
};
constexpr BVariant kBVariants[] = {
    {16384, 3, 4},  // 0
    {16384, 4, 3},  // 1
    {32768, 3, 2},  // 2
    {8192, 6, 4},   // 3
    {32768, 2, 3},  // 4
};
constexpr int kNumBVariants = sizeof(kBVariants) / sizeof(kBVariants[0]);
static int g_bvariant = 0;

template <int SB, int STAGES, int MINB>
static cudaError_t launch_batch(const BParams& p, cudaStream_t st) {
    static OccupancyCache cache{};
    auto kern = k_batch_quantize<SB, STAGES, MINB>;
    const size_t smem = (size_t)STAGES * SB;
    int dev = 0;
    cudaGetDevice(&dev);
    uint64_t grid = (uint64_t)cached_blocks_per_sm(cache, dev, kern, kSpecThreads, smem) * device_sm_count();
    if (grid > p.total_tiles) grid = p.total_tiles;
    if (grid == 0) return cudaSuccess;
    kern<<<(unsigned)grid, kSpecThreads, smem, st>>>(p);
    return cudaPeekAtLastError();
}

static cudaError_t launch_batch_variant(int v, const BParams& p, cudaStream_t st) {
    switch (v) {
#define B_CASE(i) \
    case i: return launch_batch<kBVariants[i].sb, kBVariants[i].stages, kBVariants[i].minb>(p, st);
        B_CASE(0) B_CASE(1) B_CASE(2) B_CASE(3) B_CASE(4)
#undef B_CASE
    }
    return cudaErrorInvalidValue;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace batch
}  // namespace lcq

using namespace lcq;
using namespace lcq::batch;

extern "C" {

size_t lcq_batch_plan_size(uint32_t count) { return plan_bytes_for(count); }

size_t lcq_batch_workspace_size(const lcq_batch_item* h_items, uint32_t count) {
    uint64_t tiles = 0;
    for (uint32_t i = 0; h_items && i < count; i++) tiles += (h_items[i].n + kScanTile - 1) / kScanTile;
    return ws_bytes_for(tiles, count);
}

lcq_status lcq_batch_prepare(const lcq_batch_item* h_items, uint32_t count, void* d_plan, size_t plan_bytes,
                             void* d_ws, size_t ws_bytes, lcq_batch_info* h_info, cudaStream_t stream) {
    if (!h_info) return LCQ_ERR_ARG;
    std::memset(h_info, 0, sizeof(*h_info));
    h_info->bad_item = 0xFFFFFFFFu;
    if (!h_items || count == 0 || !d_plan || !d_ws || !aligned16(d_plan) || !aligned16(d_ws))
        return LCQ_ERR_ARG;
    if (plan_bytes < plan_bytes_for(count)) return LCQ_ERR_WORKSPACE;
    std::vector<char> host(plan_bytes_for(count), 0);
    PlanHead* head = reinterpret_cast<PlanHead*>(host.data());
    Array* arr = reinterpret_cast<Array*>(host.data() + sizeof(PlanHead));
    std::vector<uint64_t> tile_begin(count + 1);
    std::vector<uint32_t> noa_index;
    std::vector<uint64_t> noa_begin(1, 0);
    uint64_t tiles = 0;
    for (uint32_t i = 0; i < count; i++) {
        const lcq_batch_item& it = h_items[i];
        lcq_status st = check_quantize_args((lcq_dtype)it.dtype, (lcq_bound_type)it.bound_type, it.eb,
                                            it.d_in, it.n, it.d_bins, it.d_mask, it.d_outliers,
                                            it.outlier_capacity, it.d_hdr);
        if (st != LCQ_OK) {
            h_info->bad_item = i;
            return st;
        }
        Array& A = arr[i];
        A.in = it.d_in;
        A.bins = it.d_bins;
        A.mask = it.d_mask;
        A.out = it.d_outliers;
        A.hdr = it.d_hdr;
        A.n = it.n;
        A.cap = it.outlier_capacity;
        A.tile_begin = tiles;
        A.num_tiles = (uint32_t)((it.n + kScanTile - 1) / kScanTile);
        A.dtype = it.dtype;
        A.bound = it.bound_type;
        A.eb = it.eb;
        if (it.bound_type != LCQ_NOA) {
            if (!host_consts((lcq_dtype)it.dtype, (lcq_bound_type)it.bound_type, it.eb, A.bits, &A.cert_w,
                             &A.cert_emin)) {
                h_info->bad_item = i;
                return LCQ_ERR_BOUND;
            }
        } else {
            noa_index.push_back(i);
            noa_begin.push_back(noa_begin.back() + (it.n + kRangeChunk - 1) / kRangeChunk);
        }
        tile_begin[i] = tiles;
        tiles += A.num_tiles;
        h_info->total_values += it.n;
        h_info->total_bytes_in += it.n * (it.dtype == LCQ_F64 ? 8 : it.dtype == LCQ_F32 ? 4 : 2);
    }
    tile_begin[count] = tiles;
    if (tiles >= 0xFFFFFFFFull) return LCQ_ERR_ARG;  // tickets are 32-bit
    head->count = count;
    head->noa_count = (uint32_t)noa_index.size();
    head->total_tiles = tiles;
    head->noa_chunks = noa_begin.back();
    PlanView v = plan_view(host.data(), count, head->noa_count);
    std::memcpy((void*)v.tile_begin, tile_begin.data(), tile_begin.size() * 8);
    if (!noa_index.empty()) std::memcpy((void*)v.noa_index, noa_index.data(), noa_index.size() * 4);
    std::memcpy((void*)v.noa_begin, noa_begin.data(), noa_begin.size() * 8);
    if (ws_bytes < ws_bytes_for(tiles, count)) return LCQ_ERR_WORKSPACE;
    if (cudaMemcpyAsync(d_plan, host.data(), host.size(), cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return LCQ_ERR_CUDA;
    // workspace: zero head and descriptors; NOA min keys start at all ones
    const size_t keys_off = ws_bytes_for(tiles, count) - (size_t)count * 16;
    if (cudaMemsetAsync(d_ws, 0, ws_bytes_for(tiles, count), stream) != cudaSuccess ||
        cudaMemsetAsync((char*)d_ws + keys_off, 0xFF, (size_t)count * 8, stream) != cudaSuccess)
        return LCQ_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return LCQ_ERR_CUDA;
    h_info->count = count;
    h_info->noa_count = head->noa_count;
    h_info->total_tiles = tiles;
    h_info->noa_chunks = head->noa_chunks;
    return LCQ_OK;
}

lcq_status lcq_quantize_batched(const lcq_batch_info* h_info, const void* d_plan, void* d_ws, size_t ws_bytes,
                                cudaStream_t stream) {
    if (!h_info || !d_plan || !d_ws || h_info->count == 0) return LCQ_ERR_ARG;
    if (ws_bytes < ws_bytes_for(h_info->total_tiles, h_info->count)) return LCQ_ERR_WORKSPACE;
    const PlanView v = plan_view(d_plan, h_info->count, h_info->noa_count);
    WsHead* ws = reinterpret_cast<WsHead*>(d_ws);
    const size_t keys_off = ws_bytes_for(h_info->total_tiles, h_info->count) - (size_t)h_info->count * 16;
    uint64_t* kmin = reinterpret_cast<uint64_t*>((char*)d_ws + keys_off);
    RParams rp{v, h_info->count, h_info->noa_count, h_info->noa_chunks, ws, kmin, kmin + h_info->count};
    uint64_t rgrid = std::max<uint64_t>(h_info->noa_chunks, (h_info->count + kRangeBlock - 1) / kRangeBlock);
    const uint64_t rcap = (uint64_t)device_sm_count() * 8;
    if (rgrid > rcap) rgrid = rcap;
    if (rgrid < 1) rgrid = 1;
    k_batch_range<<<(unsigned)rgrid, kRangeBlock, 0, stream>>>(rp);
    if (cudaPeekAtLastError() != cudaSuccess) return LCQ_ERR_CUDA;
    BParams bp;
    bp.v = v;
    bp.count = h_info->count;
    bp.total_tiles = h_info->total_tiles;
    bp.ws = ws;
    bp.tiles = reinterpret_cast<uint64_t*>((char*)d_ws + kWsHeadBytes);
    if (launch_batch_variant(g_bvariant, bp, stream) != cudaSuccess) return LCQ_ERR_CUDA;
    if (h_info->count > 0) {
        k_batch_offsets<<<h_info->count, kOffThreads, 0, stream>>>(v, bp.tiles);
        uint64_t cgrid = (uint64_t)device_sm_count() * 8;
        const uint64_t need = (h_info->total_tiles + 7) / 8;
        if (cgrid > need) cgrid = need;
        if (cgrid < 1) cgrid = 1;
        k_batch_compact<<<(unsigned)cgrid, 256, 0, stream>>>(v, h_info->count, h_info->total_tiles, bp.tiles);
        if (cudaPeekAtLastError() != cudaSuccess) return LCQ_ERR_CUDA;
    }
    return LCQ_OK;
}

int lcq_batch_tune_variant_count(void) { return kNumBVariants; }

lcq_status lcq_batch_tune_set(int variant) {
    if (variant < 0 || variant >= kNumBVariants) return LCQ_ERR_ARG;
    g_bvariant = variant;
    return LCQ_OK;
}

int lcq_batch_tune_get(void) { return g_bvariant; }

lcq_status lcq_autotune_batched(const lcq_batch_info* h_info, const void* d_plan, void* d_ws, size_t ws_bytes,
                                cudaStream_t stream, int reps, float* h_ms) {
    if (reps < 1) reps = 1;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return LCQ_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return LCQ_ERR_CUDA; }
    const int saved = g_bvariant;
    int best = saved;
    float best_ms = 0.0f;
    lcq_status st = LCQ_OK;
    for (int v = 0; v < kNumBVariants && st == LCQ_OK; v++) {
        g_bvariant = v;
        st = lcq_quantize_batched(h_info, d_plan, d_ws, ws_bytes, stream);
        cudaEventRecord(a, stream);
        for (int r = 0; r < reps && st == LCQ_OK; r++) st = lcq_quantize_batched(h_info, d_plan, d_ws, ws_bytes, stream);
        cudaEventRecord(b, stream);
        if (cudaEventSynchronize(b) != cudaSuccess) st = LCQ_ERR_CUDA;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        ms /= reps;
        if (h_ms) h_ms[v] = ms;
        if (st == LCQ_OK && (v == 0 || ms < best_ms)) {
            best_ms = ms;
            best = v;
        }
    }
    g_bvariant = st == LCQ_OK ? best : saved;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

}  // extern "C"
