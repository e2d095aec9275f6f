// lcq_pack.cu -- lossless stage after quantization (no counterpart in the
// paper, which hands its bins to LC's lossless stages): bit-plane packing of
// int32 codes (bins or predictor residuals).
//
// Format for n codes, nb = ceil(n / 32) blocks of 32 codes (the last padded
// with zeros):
//   z = zigzag(code) = (code << 1) ^ (code >> 31)  (uint32);
//   w_b = bit width of the OR of the block's z (0..32);
//   bytes [0, align16(nb))           : w_b as uint8, zero padding;
//   then uint32 words, block after block: block b holds w_b bit-planes, word
//   j of the block has bit i = bit j of z of code 32 b + i.
// Total size align16(nb) + 4 sum(w_b).
//
// Encoding: k_pack_widths (widths and per-chunk sums), k_scan_chunks (one
// CTA: exclusive scan of the chunk sums, total size), k_pack_write (bit-planes
// by a warp bit transpose at the scanned offsets).  Decoding: k_unpack_sums
// (chunk sums from the widths), k_scan_chunks, k_unpack (bit-planes back to
// codes by the same transpose).  A chunk is 256 blocks (8192 codes), one CTA of 8 warps.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lcq.h"
#include "lcq_host.h"

namespace lcq {
namespace {

constexpr int kPackThreads = 256;
constexpr int kChunkBlocks = 256;  // blocks of 32 codes per chunk: 32 per warp, 8 warps
constexpr int kScanThreads = 1024;

__device__ __forceinline__ uint32_t zigzag(int32_t v) { return ((uint32_t)v << 1) ^ (uint32_t)(v >> 31); }
__device__ __forceinline__ int32_t unzigzag(uint32_t z) { return (int32_t)(z >> 1) ^ -(int32_t)(z & 1u); }

__host__ __device__ inline uint64_t num_blocks(uint64_t n) { return (n + 31) / 32; }
__host__ __device__ inline uint64_t num_chunks(uint64_t n) { return (num_blocks(n) + kChunkBlocks - 1) / kChunkBlocks; }
__host__ __device__ inline uint64_t align16(uint64_t b) { return (b + 15) & ~(uint64_t)15; }

// 32 x 32 bit transpose across a warp: on return lane p holds the word whose
// bit i is bit p of lane i's input (and, the transpose being its own inverse,
// the same call turns bit-planes back into values).  Five rounds of
// swapping the off-diagonal s x s blocks with the lane s apart.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x) {
    const int lane = threadIdx.x & 31;
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int r = 0; r < 5; r++) {
        const int sft = 16 >> r;
        const uint32_t m = masks[r];
        const uint32_t other = __shfl_xor_sync(0xFFFFFFFFu, x, sft);
        x = (lane & sft) ? ((x & ~m) | ((other & ~m) >> sft)) : ((x & m) | ((other & m) << sft));
    }
    return x;
}

// Sum of a CTA's per-warp values; every thread gets the total and its warp's
// exclusive prefix.
__device__ __forceinline__ uint32_t cta_exclusive(uint32_t warp_total, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_warp[warp] = warp_total;
    __syncthreads();
    uint32_t pre = 0, tot = 0;
    for (int i = 0; i < kPackThreads / 32; i++) {
        const uint32_t v = s_warp[i];
        pre += i < warp ? v : 0u;
        tot += v;
    }
    __syncthreads();
    total = tot;
    return pre;
}

// Zigzagged codes of one chunk (8192 codes) into shared memory: coalesced
// 16-byte loads, the ragged tail (and the padding past n) as zeros.
__device__ __forceinline__ void load_chunk_z(const int32_t* __restrict__ codes, uint64_t n, uint32_t* s_z) {
    const uint64_t base = (uint64_t)blockIdx.x * kChunkBlocks * 32;
#pragma unroll
    for (int k = 0; k < kChunkBlocks * 32 / 4 / kPackThreads; k++) {
        const int v = k * kPackThreads + threadIdx.x;  // int4 index within the chunk
        const uint64_t i = base + 4 * (uint64_t)v;
        uint32_t z0 = 0, z1 = 0, z2 = 0, z3 = 0;
        if (i + 4 <= n) {
            const int4 c = __ldcs(reinterpret_cast<const int4*>(codes + i));
            z0 = zigzag(c.x); z1 = zigzag(c.y); z2 = zigzag(c.z); z3 = zigzag(c.w);
        } else {
            if (i < n) z0 = zigzag(codes[i]);
            if (i + 1 < n) z1 = zigzag(codes[i + 1]);
            if (i + 2 < n) z2 = zigzag(codes[i + 2]);
        }
        reinterpret_cast<uint4*>(s_z)[v] = make_uint4(z0, z1, z2, z3);
    }
}

// Width of each block and the chunk's sum of widths: 16-byte loads, 8 lanes
// per block of 32 codes, the OR by three shuffles.
__global__ void __launch_bounds__(kPackThreads) k_pack_widths(const int32_t* __restrict__ codes, uint64_t n,
                                                              uint8_t* __restrict__ widths,
                                                              uint32_t* __restrict__ chunk_sum) {
    __shared__ uint32_t s_warp[kPackThreads / 32];
    const uint64_t nb = num_blocks(n);
    const uint64_t base = (uint64_t)blockIdx.x * kChunkBlocks * 32;
    uint32_t wsum = 0;
#pragma unroll
    for (int k = 0; k < kChunkBlocks * 32 / 4 / kPackThreads; k++) {
        const int v = k * kPackThreads + threadIdx.x;
        const uint64_t i = base + 4 * (uint64_t)v;
        uint32_t m = 0;
        if (i + 4 <= n) {
            const int4 c = __ldcs(reinterpret_cast<const int4*>(codes + i));
            m = zigzag(c.x) | zigzag(c.y) | zigzag(c.z) | zigzag(c.w);
        } else {
            if (i < n) m |= zigzag(codes[i]);
            if (i + 1 < n) m |= zigzag(codes[i + 1]);
            if (i + 2 < n) m |= zigzag(codes[i + 2]);
        }
        m |= __shfl_xor_sync(0xFFFFFFFFu, m, 1);
        m |= __shfl_xor_sync(0xFFFFFFFFu, m, 2);
        m |= __shfl_xor_sync(0xFFFFFFFFu, m, 4);
        const uint64_t b = (uint64_t)blockIdx.x * kChunkBlocks + (uint64_t)(v >> 3);
        const uint32_t w = 32u - (uint32_t)__clz((int)m);
        if ((threadIdx.x & 7) == 0) {
            if (b < align16(nb)) widths[b] = (uint8_t)(b < nb ? w : 0u);  // 0 on the padding
            wsum += b < nb ? w : 0u;
        }
    }
    uint32_t total;
    cta_exclusive(__reduce_add_sync(0xFFFFFFFFu, wsum), s_warp, total);
    if (threadIdx.x == 0) chunk_sum[blockIdx.x] = total;
}

// Exclusive scan of the chunk sums into 64-bit word offsets (one CTA);
// out[nchunks] = the total.  *total_bytes (optional) = the encoded size.
__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(const uint32_t* chunk_sum, uint64_t nchunks,
                                                              uint64_t* out, uint64_t nb, uint64_t* total_bytes) {
    __shared__ uint64_t s_part[kScanThreads / 32];
    __shared__ uint64_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < nchunks; base += kScanThreads) {
        const uint64_t i = base + threadIdx.x;
        const uint64_t v = i < nchunks ? chunk_sum[i] : 0u;
        uint64_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_part[warp] = incl;
        __syncthreads();
        uint64_t wpre = 0, tot = 0;
        for (int k = 0; k < kScanThreads / 32; k++) {
            wpre += k < warp ? s_part[k] : 0u;
            tot += s_part[k];
        }
        const uint64_t carry = s_carry;
        if (i < nchunks) out[i] = carry + wpre + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[nchunks] = s_carry;
        if (total_bytes) *total_bytes = align16(nb) + 4 * s_carry;
    }
}

// Bit-planes of each block at its offset.  The chunk's codes are staged in
// shared memory; a warp bit transpose puts plane p of a block in lane p, so
// that the block's planes are written by one coalesced store of w words.
__global__ void __launch_bounds__(kPackThreads) k_pack_write(const int32_t* __restrict__ codes, uint64_t n,
                                                             const uint8_t* __restrict__ widths,
                                                             const uint64_t* __restrict__ chunk_off,
                                                             uint32_t* __restrict__ words) {
    __shared__ uint32_t s_warp[kPackThreads / 32];
    __shared__ __align__(16) uint32_t s_z[kChunkBlocks * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nb = num_blocks(n);
    load_chunk_z(codes, n, s_z);
    const uint64_t b0 = (uint64_t)blockIdx.x * kChunkBlocks + (uint64_t)warp * 32;
    const uint32_t wl = b0 + lane < nb ? widths[b0 + lane] : 0u;  // width of block b0 + lane
    uint32_t incl = wl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    uint32_t total;  // cta_exclusive also orders the shared-memory stores above
    const uint32_t wpre = cta_exclusive(__shfl_sync(0xFFFFFFFFu, incl, 31), s_warp, total);
    const uint64_t off = chunk_off[blockIdx.x] + wpre + (incl - wl);  // word offset of block b0 + lane
    const int jn = b0 >= nb ? 0 : (nb - b0 < 32 ? (int)(nb - b0) : 32);
    for (int j = 0; j < jn; j++) {
        const uint32_t w = __shfl_sync(0xFFFFFFFFu, wl, j);
        const uint64_t o = __shfl_sync(0xFFFFFFFFu, off, j);
        const uint32_t plane = warp_transpose32(s_z[(warp * 32 + j) * 32 + lane]);  // lane p: plane p
        if ((uint32_t)lane < w) words[o + lane] = plane;
    }
}

// Chunk sums of the stored widths (decoding).
__global__ void __launch_bounds__(kPackThreads) k_unpack_sums(const uint8_t* widths, uint64_t nb, uint32_t* chunk_sum) {
    __shared__ uint32_t s_warp[kPackThreads / 32];
    const uint64_t b = (uint64_t)blockIdx.x * kChunkBlocks + threadIdx.x;  // kChunkBlocks == kPackThreads
    const uint32_t w = b < nb ? widths[b] : 0u;
    uint32_t total;
    cta_exclusive(__reduce_add_sync(0xFFFFFFFFu, w), s_warp, total);
    if (threadIdx.x == 0) chunk_sum[blockIdx.x] = total;
}

// Codes back from the bit-planes: the chunk's words (contiguous, at most 32
// per block) are staged in shared memory, then a warp bit transpose of a
// block's planes (planes past w are 0) gives lane i its value.  *status gets LCQ_STATUS_HEADER (and the block decodes as
// zeros) if a stored width exceeds 32 or a block's planes would lie beyond
// the avail words.
__global__ void __launch_bounds__(kPackThreads) k_unpack(const uint8_t* __restrict__ widths,
                                                         const uint32_t* __restrict__ words, uint64_t avail,
                                                         const uint64_t* __restrict__ chunk_off, uint64_t n,
                                                         int32_t* __restrict__ codes, uint32_t* status) {
    __shared__ uint32_t s_warp[kPackThreads / 32];
    __shared__ uint32_t s_w[kChunkBlocks * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nb = num_blocks(n);
    const uint64_t b0 = (uint64_t)blockIdx.x * kChunkBlocks + (uint64_t)warp * 32;
    uint32_t wl = b0 + lane < nb ? widths[b0 + lane] : 0u;
    if (wl > 32u) {
        if (status) atomicOr(status, LCQ_STATUS_HEADER);
        wl = 0;
    }
    uint32_t incl = wl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    uint32_t total;
    const uint32_t wpre = cta_exclusive(__shfl_sync(0xFFFFFFFFu, incl, 31), s_warp, total);
    // the chunk's planes: words [base, base + total) of the stream
    const uint64_t base = chunk_off[blockIdx.x];
    const uint32_t have = base >= avail ? 0u : (avail - base < total ? (uint32_t)(avail - base) : total);
    if (have < total && status && threadIdx.x == 0) atomicOr(status, LCQ_STATUS_HEADER);
    for (uint32_t k = threadIdx.x; k < have; k += kPackThreads) s_w[k] = __ldcs(words + base + k);
    __syncthreads();
    const uint32_t loc = wpre + (incl - wl);  // block b0 + lane: its first word within the chunk
    const int jn = b0 >= nb ? 0 : (nb - b0 < 32 ? (int)(nb - b0) : 32);
    for (int j = 0; j < jn; j++) {
        uint32_t w = __shfl_sync(0xFFFFFFFFu, wl, j);
        const uint32_t o = __shfl_sync(0xFFFFFFFFu, loc, j);
        if (o + w > have) w = 0;  // planes missing from the stream (reported above)
        const uint32_t z = warp_transpose32((uint32_t)lane < w ? s_w[o + lane] : 0u);
        const uint64_t i = (b0 + j) * 32 + lane;
        if (i < n) codes[i] = unzigzag(z);
    }
}

size_t pack_ws_bytes(uint64_t n) {
    const uint64_t nc = num_chunks(n);
    return align16(nc * 4) + (nc + 1) * 8;
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace
}  // namespace lcq

using namespace lcq;

extern "C" {

size_t lcq_pack_bound(uint64_t n) { return align16(num_blocks(n)) + 4 * 32 * num_blocks(n); }

size_t lcq_pack_workspace_size(uint64_t n) { return pack_ws_bytes(n); }

lcq_status lcq_pack(const int32_t* d_codes, uint64_t n, void* d_out, size_t out_bytes, uint64_t* d_out_bytes,
                    void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (n == 0 || n >= (1ull << 40)) return LCQ_ERR_ARG;
    if (!d_codes || !d_out || !d_ws || !al16(d_codes) || !al16(d_out) || !al16(d_ws)) return LCQ_ERR_ARG;
    if (d_out_bytes && (reinterpret_cast<uintptr_t>(d_out_bytes) & 7) != 0) return LCQ_ERR_ARG;
    if (out_bytes < lcq_pack_bound(n)) return LCQ_ERR_CAPACITY;
    if (ws_bytes < pack_ws_bytes(n)) return LCQ_ERR_WORKSPACE;
    const uint64_t nb = num_blocks(n), nc = num_chunks(n);
    uint8_t* widths = (uint8_t*)d_out;
    uint32_t* words = (uint32_t*)((char*)d_out + align16(nb));
    uint32_t* chunk_sum = (uint32_t*)d_ws;
    uint64_t* chunk_off = (uint64_t*)((char*)d_ws + align16(nc * 4));
    k_pack_widths<<<(unsigned)nc, kPackThreads, 0, stream>>>(d_codes, n, widths, chunk_sum);
    k_scan_chunks<<<1, kScanThreads, 0, stream>>>(chunk_sum, nc, chunk_off, nb, d_out_bytes);
    k_pack_write<<<(unsigned)nc, kPackThreads, 0, stream>>>(d_codes, n, widths, chunk_off, words);
    return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
}

lcq_status lcq_unpack(const void* d_in, size_t in_bytes, uint64_t n, int32_t* d_codes, uint32_t* d_status,
                      void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (n == 0 || n >= (1ull << 40)) return LCQ_ERR_ARG;
    if (!d_in || !d_codes || !d_ws || !al16(d_in) || !al16(d_codes) || !al16(d_ws)) return LCQ_ERR_ARG;
    if (d_status && (reinterpret_cast<uintptr_t>(d_status) & 3) != 0) return LCQ_ERR_ARG;
    if (ws_bytes < pack_ws_bytes(n)) return LCQ_ERR_WORKSPACE;
    const uint64_t nb = num_blocks(n), nc = num_chunks(n);
    if (in_bytes < align16(nb)) return LCQ_ERR_ARG;
    const uint64_t avail = (in_bytes - align16(nb)) / 4;
    const uint8_t* widths = (const uint8_t*)d_in;
    const uint32_t* words = (const uint32_t*)((const char*)d_in + align16(nb));
    uint32_t* chunk_sum = (uint32_t*)d_ws;
    uint64_t* chunk_off = (uint64_t*)((char*)d_ws + align16(nc * 4));
    if (d_status && cudaMemsetAsync(d_status, 0, 4, stream) != cudaSuccess) return LCQ_ERR_CUDA;
    k_unpack_sums<<<(unsigned)nc, kPackThreads, 0, stream>>>(widths, nb, chunk_sum);
    k_scan_chunks<<<1, kScanThreads, 0, stream>>>(chunk_sum, nc, chunk_off, nb, nullptr);
    k_unpack<<<(unsigned)nc, kPackThreads, 0, stream>>>(widths, words, avail, chunk_off, n, d_codes, d_status);
    return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
}

}  // extern "C"
