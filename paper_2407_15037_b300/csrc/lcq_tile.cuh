// lcq_tile.cuh -- per-tile building blocks shared by the single-array and the
// batched streaming kernels: vector access, the 4-value quantize of one ring
// stage ("sub-tile") into bins and shared-memory mask words, the warp scan of
// a scan tile's mask words, the decoder's outlier walk, the per-tile
// compaction after quantization, and the NOA range helpers.
#pragma once

#include <cstdint>

#include "lcq_device.cuh"

namespace lcq {

constexpr int kComputeThreads = 256;               // 8 compute warps
constexpr int kSpecThreads = kComputeThreads + 32;  // + 1 scan warp
constexpr uint32_t kNoTile = 0xFFFFFFFFu;

// Shared-memory position of mask word w of a scan tile: the low 5 bits are
// XOR-ed with the row (w / 32), so that the scan warp's lanes, which read 16
// or 32 consecutive words each, hit 32 different banks.
__device__ __forceinline__ int sw(int w) { return w ^ ((w >> 5) & 31); }

// ---------------------------------------------------------------------------
// Vector access helpers: 4 consecutive values per thread per step.
// ---------------------------------------------------------------------------
template <typename T>
struct Vec4;

template <>
struct Vec4<float> {
    static __device__ __forceinline__ void load(const float* p, float v[4]) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(p));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    static __device__ __forceinline__ void load_shared(const float* p, float v[4]) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    static __device__ __forceinline__ void load_cached(const float* p, float v[4]) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    static __device__ __forceinline__ void store(float* p, const float v[4]) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
    }
};

template <>
struct Vec4<double> {
    static __device__ __forceinline__ void load(const double* p, double v[4]) {
        const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
        const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void load_shared(const double* p, double v[4]) {
        const double2 a = reinterpret_cast<const double2*>(p)[0];
        const double2 b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void load_cached(const double* p, double v[4]) {
        const double2 a = reinterpret_cast<const double2*>(p)[0];
        const double2 b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void store(double* p, const double v[4]) {
        __stcs(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
        __stcs(reinterpret_cast<double2*>(p) + 1, make_double2(v[2], v[3]));
    }
};

// 16-bit formats: 4 values = 8 bytes.
template <typename T>
struct Vec4x16 {
    static __device__ __forceinline__ void split(uint2 a, T v[4]) {
        v[0] = T((int)(a.x & 0xFFFFu)); v[1] = T((int)(a.x >> 16));
        v[2] = T((int)(a.y & 0xFFFFu)); v[3] = T((int)(a.y >> 16));
    }
    static __device__ __forceinline__ void load(const T* p, T v[4]) {
        split(__ldcs(reinterpret_cast<const uint2*>(p)), v);
    }
    static __device__ __forceinline__ void load_shared(const T* p, T v[4]) {
        split(*reinterpret_cast<const uint2*>(p), v);
    }
    static __device__ __forceinline__ void load_cached(const T* p, T v[4]) {
        split(*reinterpret_cast<const uint2*>(p), v);
    }
    static __device__ __forceinline__ void store(T* p, const T v[4]) {
        __stcs(reinterpret_cast<uint2*>(p), make_uint2((uint32_t)v[0].u | ((uint32_t)v[1].u << 16),
                                                      (uint32_t)v[2].u | ((uint32_t)v[3].u << 16)));
    }
};
template <>
struct Vec4<f16s> : Vec4x16<f16s> {};
template <>
struct Vec4<bf16s> : Vec4x16<bf16s> {};

template <typename T, int VPT>
__device__ __forceinline__ void load4(const T* sbuf_tile, const T* gin, bool from_smem, int off,
                                      uint64_t e0, uint64_t n, T x[4]) {
    if (from_smem) {
        Vec4<T>::load_shared(sbuf_tile + off, x);
    } else if (e0 + 4 <= n) {
        Vec4<T>::load(gin + e0, x);
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) x[k] = (e0 + k < n) ? gin[e0 + k] : T(0);
    }
}

// Mask words of one tile -> global, 16-byte stores where the tile is whole.
template <int WPL>
__device__ __forceinline__ void store_mask_words(uint32_t* gmask, uint64_t gw, uint64_t nwords,
                                                 const uint32_t* wv) {
#pragma unroll
    for (int j = 0; j < WPL; j += 4) {
        if (gw + j + 4 <= nwords) {
            __stcs(reinterpret_cast<uint4*>(gmask + gw + j), make_uint4(wv[j], wv[j + 1], wv[j + 2], wv[j + 3]));
        } else {
#pragma unroll
            for (int i = 0; i < 4; i++)
                if (gw + j + i < nwords) gmask[gw + j + i] = wv[j + i];
        }
    }
}

// Warp 0: exclusive prefix popcounts of the tile's mask words into s_wpre;
// returns the tile's outlier count.  Also stores the words to global memory.
template <int WPL>
__device__ __forceinline__ uint32_t scan_mask_words(const uint32_t* s_words, uint32_t* s_wpre,
                                                    uint32_t* gmask, uint64_t gw, uint64_t nwords,
                                                    bool store) {
    const int lane = threadIdx.x & 31;
    uint32_t wv[WPL], loc[WPL], cnt = 0;
#pragma unroll
    for (int j = 0; j < WPL; j++) {
        wv[j] = s_words[sw(lane * WPL + j)];
        loc[j] = cnt;
        cnt += __popc(wv[j]);
    }
    if (store) store_mask_words<WPL>(gmask, gw, nwords, wv);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t ex = incl - cnt;
#pragma unroll
    for (int j = 0; j < WPL; j++) s_wpre[sw(lane * WPL + j)] = ex + loc[j];
    return __shfl_sync(0xFFFFFFFFu, incl, 31);
}

// Quantize one sub-tile of kComputeThreads x 4 x VPT values: from the
// shared-memory stage st (from_smem, a whole sub-tile) or else from global
// memory gin (a ragged or empty sub-tile with nvalid valid values).  Bins go
// to gbins (the sub-tile's first bin); the sub-tile's mask words go to
// s_words[sw(word_base + i)].  Called by the kComputeThreads compute threads.
template <typename T, int MODE, int VPT>
__device__ __forceinline__ void quantize_subtile(const T* st, const T* gin, bool from_smem,
                                                 uint64_t nvalid, int32_t* gbins, uint32_t* s_words,
                                                 int word_base, const Consts<CT<T>>& c) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wbase = word_base + warp * 4 + (lane >> 3);
    // 4-value outlier nibbles of 8 lanes -> one mask word
    auto put_word = [&](int v, uint32_t nb) {
        uint32_t w = nb << ((lane & 7) * 4);
        w |= __shfl_xor_sync(0xFFFFFFFFu, w, 1);
        w |= __shfl_xor_sync(0xFFFFFFFFu, w, 2);
        w |= __shfl_xor_sync(0xFFFFFFFFu, w, 4);
        if ((lane & 7) == 0) s_words[sw(wbase + v * (kComputeThreads / 8))] = w;
    };
    if (from_smem && !c.all_outliers) {
        // fast path: a whole sub-tile in shared memory, no bounds checks
#pragma unroll
        for (int v = 0; v < VPT; v++) {
            const int off = v * (kComputeThreads * 4) + tid * 4;
            T x[4];
            Vec4<T>::load_shared(st + off, x);
            int32_t bn[4];
            const uint32_t nb = quant4<T, MODE>(x, c, bn);
            __stcs(reinterpret_cast<int4*>(gbins + off), make_int4(bn[0], bn[1], bn[2], bn[3]));
            put_word(v, nb);
        }
    } else {
#pragma unroll
        for (int v = 0; v < VPT; v++) {
            const int off = v * (kComputeThreads * 4) + tid * 4;
            const uint64_t e0 = (uint64_t)off;
            T x[4];
            load4<T, VPT>(st, gin, from_smem, off, e0, nvalid, x);
            int32_t bn[4];
            uint32_t nb = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                int32_t bin = 0;
                bool ok = false;
                if (!c.all_outliers) ok = quant1<T, MODE>(x[q], c, bin);
                if (!ok && e0 + q < nvalid) nb |= 1u << q;
                bn[q] = ok ? bin : 0;
            }
            if (e0 + 4 <= nvalid) {
                __stcs(reinterpret_cast<int4*>(gbins + e0), make_int4(bn[0], bn[1], bn[2], bn[3]));
            } else {
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (e0 + q < nvalid) gbins[e0 + q] = bn[q];
            }
            put_word(v, nb);
        }
    }
}

// Every set bit of a scan tile's mask words (s_words, with the exclusive
// in-tile prefix counts s_wpre) in index order: for the tile's value i whose
// outlier rank within the tile is r, v = ld(i, r), then st(i, r, v).  Called
// by the kComputeThreads compute threads.  Each warp takes 32 consecutive
// words at a time and walks them one of two ways: each lane its own word (as
// many steps as the fullest word has bits; every load and store of a step
// touches a different line per lane), or all 32 words one by one with one
// lane per value (32 steps; loads and stores coalesced).  It takes the
// cheaper by a cost in issued instructions plus memory wavefronts: 14 per
// lane-walk step and 2 per outlier, against 13 per word step.  Either walk
// takes U steps at a time and issues their U loads before the U stores, so
// that the loads' latencies overlap.
template <typename V, int U = 4, typename LD, typename ST>
__device__ __forceinline__ void for_each_outlier(const uint32_t* s_words, const uint32_t* s_wpre, int words,
                                                 LD&& ld, ST&& st) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w0 = warp * 32; w0 < words; w0 += kComputeThreads) {
        const int w = w0 + lane;
        const uint32_t mw = w < words ? s_words[sw(w)] : 0u;
        const uint32_t pre = w < words ? s_wpre[sw(w)] : 0u;
        const uint32_t cnt = (uint32_t)__popc(mw);
        const uint32_t tot = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if (tot == 0) continue;
        const uint32_t maxc = __reduce_max_sync(0xFFFFFFFFu, cnt);
        if (14u * maxc + 2u * tot <= 13u * 32u + 2u * 32u) {
            uint32_t m = mw, r = pre;
            while (m) {
                uint32_t iu[U], ru[U];
                bool on[U];
                V v[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    on[u] = m != 0u;
                    iu[u] = (uint32_t)w * 32 + (on[u] ? (uint32_t)(__ffs(m) - 1) : 0u);
                    ru[u] = r;
                    r += on[u] ? 1u : 0u;
                    m &= m - 1u;
                }
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (on[u]) v[u] = ld(iu[u], ru[u]);
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (on[u]) st(iu[u], ru[u], v[u]);
            }
        } else {
            const uint32_t bit = 1u << lane, below = bit - 1u;
            const uint32_t i0 = (uint32_t)w0 * 32 + lane;
            for (int j0 = 0; j0 < 32; j0 += U) {
                uint32_t ru[U];
                bool on[U];
                V v[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const uint32_t mj = __shfl_sync(0xFFFFFFFFu, mw, j0 + u);
                    const uint32_t pj = __shfl_sync(0xFFFFFFFFu, pre, j0 + u);
                    on[u] = (mj & bit) != 0u;
                    ru[u] = pj + __popc(mj & below);
                }
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (on[u]) v[u] = ld(i0 + 32u * (j0 + u), ru[u]);
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (on[u]) st(i0 + 32u * (j0 + u), ru[u], v[u]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Outlier payload of one scan tile after quantization, by one warp (all 32
// lanes): the raw bits of the tile's outliers (tcount of them, tcount > 0) to
// out[pbase + rank], ranks in index order, writes stopping at cap.  tin: the
// tile's first value; tmask: its first mask word, of which words_left are
// valid (the rest count as 0).  The warp reads the mask in parts of up to
// 512 words, up to 16 per lane, and a warp scan of the lanes' bit counts gives each
// lane its first rank.  In a sparse tile each lane walks its own words in
// index order and issues the loads of up to eight outliers (across words)
// before their stores, so that the latencies overlap.  In a dense tile (more
// than 1/8 outliers) the warp takes the words one by one with one lane per
// bit, so that its loads and stores are coalesced.
// ---------------------------------------------------------------------------
template <typename T, int WORDS>
__device__ __forceinline__ void compact_tile(const T* tin, const uint32_t* tmask, uint64_t words_left,
                                             uint32_t tcount, uint64_t pbase, typename Ty<T>::U* out,
                                             uint64_t cap) {
    using U = typename Ty<T>::U;
    // parts of up to 512 words: 16 (or, for smaller tiles, 4 or 8) words per lane
    constexpr int TILE = WORDS * 32, PART = WORDS < 512 ? WORDS : 512, WPL = PART / 32;
    static_assert(WORDS % PART == 0 && WPL % 4 == 0, "whole parts of whole uint4 loads per lane");
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    const bool dense = tcount > (uint32_t)(TILE / 8);
    for (int part = 0; part < WORDS / PART; part++) {
        const uint64_t lw = (uint64_t)part * PART + (uint64_t)lane * WPL;  // the lane's first word
        uint32_t wv[WPL];
        uint32_t cnt = 0;
#pragma unroll
        for (int j = 0; j < WPL; j += 4) {
            if (lw + j + 4 <= words_left) {
                const uint4 a = *reinterpret_cast<const uint4*>(tmask + lw + j);
                wv[j] = a.x; wv[j + 1] = a.y; wv[j + 2] = a.z; wv[j + 3] = a.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++) wv[j + i] = lw + j + i < words_left ? tmask[lw + j + i] : 0u;
            }
#pragma unroll
            for (int i = 0; i < 4; i++) cnt += __popc(wv[j + i]);
        }
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        const T* gp = tin + (uint64_t)part * PART * 32;  // first value of the part
        if (dense) {
            for (int L = 0; L < 32; L++) {
                uint32_t run = __shfl_sync(0xFFFFFFFFu, incl - cnt, L);
#pragma unroll
                for (int j0 = 0; j0 < WPL; j0 += 4) {
                    uint32_t w[4], r[4];
                    U v[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        w[u] = __shfl_sync(0xFFFFFFFFu, wv[j0 + u], L);
                        r[u] = run + __popc(w[u] & below);
                        run += __popc(w[u]);
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++)
                        if ((w[u] >> lane) & 1u) v[u] = Ty<T>::bits(gp[(uint32_t)(L * WPL + j0 + u) * 32u + lane]);
#pragma unroll
                    for (int u = 0; u < 4; u++)
                        if (((w[u] >> lane) & 1u) && pbase + r[u] < cap) out[pbase + r[u]] = v[u];
                }
            }
        } else {
            constexpr int Q = 8;
            uint64_t rank = pbase + (incl - cnt);
            const T* gin = gp + (uint64_t)lane * WPL * 32;
            uint32_t qi[Q] = {0, 0, 0, 0, 0, 0, 0, 0};
            int qn = 0;
            auto flush = [&]() {
                U v[Q];
#pragma unroll
                for (int u = 0; u < Q; u++)
                    if (u < qn) v[u] = Ty<T>::bits(gin[qi[u]]);
#pragma unroll
                for (int u = 0; u < Q; u++)
                    if (u < qn && rank + u < cap) out[rank + u] = v[u];
                rank += (uint64_t)qn;
                qn = 0;
            };
#pragma unroll
            for (int jw = 0; jw < WPL; jw++) {
                uint32_t m = wv[jw];
                while (m) {
                    const uint32_t idx = (uint32_t)jw * 32u + (uint32_t)(__ffs(m) - 1);
                    m &= m - 1u;
#pragma unroll
                    for (int u = 0; u < Q; u++) qi[u] = qn == u ? idx : qi[u];
                    if (++qn == Q) flush();
                }
            }
            flush();
        }
        pbase += __shfl_sync(0xFFFFFFFFu, incl, 31);  // outliers of this part
    }
}

// ---------------------------------------------------------------------------
// NOA range (Sec. 2.1.3): finite values as order-preserving integer keys, and
// the bound derived from the range on the device.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ typename Ty<T>::K order_key(typename Ty<T>::U u) {
    using U = typename Ty<T>::U;
    constexpr U sign = (U)((U)1 << (sizeof(U) * 8 - 1));
    return (typename Ty<T>::K)((u & sign) ? (U)~u : (U)(u | sign));
}
template <typename T>
__device__ __forceinline__ typename Ty<T>::U key_to_bits(typename Ty<T>::K key) {
    using U = typename Ty<T>::U;
    constexpr U sign = (U)((U)1 << (sizeof(U) * 8 - 1));
    const U k = (U)key;
    return (k & sign) ? (U)(k & (U)~sign) : (U)~k;
}

template <typename T>
__device__ __forceinline__ void minmax_accum(T x, typename Ty<T>::K& lo, typename Ty<T>::K& hi) {
    using F = Ty<T>;
    using U = typename F::U;
    const U u = F::bits(x);
    if (((u >> F::kP) & F::kExpAll) == F::kExpAll) return;  // Inf / NaN
    const typename F::K k = order_key<T>(u);
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
}

// C: the arithmetic type (float constants for float32 and the 16-bit
// formats, double constants for float64); mn, mx: the finite range, exact.
template <typename C>
__device__ __forceinline__ void noa_finalize(lcq_header* h, bool any, double mn, double mx, double eb) {
    uint32_t mode = 1;
    double R = 0.0, eb_abs = 0.0;
    uint64_t ebT_b = 0, eb2_b = 0, inv_b = 0;
    if (any) {
        R = __dsub_rd(mx, mn);
        if (R == 0.0) R = 0.0;  // a zero range is +0, whichever signed zeros min and max are
        eb_abs = __dmul_rd(eb, R);
        if (sizeof(C) == 4) {
            const float ebT = __double2float_rd(eb_abs);
            const float eb2 = __fmul_rn(2.0f, ebT);
            const float inv = __fdiv_rn(1.0f, eb2);
            const bool ok = (ebT >= FLT_MIN && ebT <= FLT_MAX) && (eb2 <= FLT_MAX) &&
                            (inv >= FLT_MIN && inv <= FLT_MAX);
            if (ok) {
                mode = 0;
                ebT_b = __float_as_uint(ebT);
                eb2_b = __float_as_uint(eb2);
                inv_b = __float_as_uint(inv);
            }
        } else {
            const double ebT = eb_abs;
            const double eb2 = __dmul_rn(2.0, ebT);
            const double inv = __ddiv_rn(1.0, eb2);
            const bool ok = (ebT >= DBL_MIN && ebT <= DBL_MAX) && (eb2 <= DBL_MAX) &&
                            (inv >= DBL_MIN && inv <= DBL_MAX);
            if (ok) {
                mode = 0;
                ebT_b = (uint64_t)__double_as_longlong(ebT);
                eb2_b = (uint64_t)__double_as_longlong(eb2);
                inv_b = (uint64_t)__double_as_longlong(inv);
            }
        }
    }
    h->mode = mode;
    h->range = R;
    h->eb_abs = eb_abs;
    h->ebT_bits = ebT_b;
    h->scale_bits = eb2_b;
    h->inv_bits = inv_b;
    h->chk_bits = 0;
}

}  // namespace lcq
