/*
 * lcq.h -- C ABI of liblcq.so: guaranteed-error-bound ABS / REL / NOA
 * quantizers on NVIDIA B300 (sm_103a).
 *
 * The method is that of Fallin & Burtscher, "Lessons Learned on the Path to
 * Guaranteeing the Error Bound in Lossy Quantizers" (arXiv 2407.15037):
 *   - error-bound types ABS, REL and NOA as defined in Sec. 2.1.1-2.1.3;
 *   - ABS quantization by multiplying with the inverse of twice the bound and
 *     rounding to the nearest bin (Sec. 2.2);
 *   - an immediate reconstruction of every value and a check against the
 *     bound; values that fail are stored losslessly (Sec. 3.1);
 *   - IEEE-754 operations only, no FMA contraction (Sec. 3.2);
 *   - the bit-level log2/pow2 approximations for REL (Sec. 3.2);
 *   - a two-sided bin-range test instead of abs() (Sec. 2.4, 3.3).
 * Results are bit-identical to a plain CPU implementation of the same recipe.
 *
 * Conventions shared by every entry point
 *   - Ownership: the caller allocates and owns every buffer; the library never
 *     allocates device or host memory and never synchronises inside the
 *     device-buffer entry points (they only enqueue work on `stream`).
 *   - Pointers named d_* are device pointers, h_* host pointers.  Every device
 *     array pointer must be 16-byte aligned (LCQ_ERR_ARG otherwise).
 *   - Argument and bound errors are returned synchronously.  Errors found on
 *     the device are OR-ed into a status word (lcq_header.status or the
 *     d_status argument) as LCQ_STATUS_* bits; read them after the stream has
 *     reached the call, e.g. with lcq_sync_status().
 *   - A workspace (d_ws) must be zero-filled once before its first use
 *     (lcq_workspace_init or cudaMemsetAsync); the kernels leave it ready for
 *     the next call.  One workspace must not be used by two calls that can run
 *     concurrently.  After a call that reported LCQ_STATUS_TIMEOUT, or a CUDA
 *     error, re-initialise the workspace; also before a single-array call
 *     uses a workspace that the batched calls used (their layout differs).
 *   - n = 0 is legal.
 *
 * Compressed representation of an array of n values of type T (float, double,
 * or a 16-bit format, see lcq_dtype):
 *   bins     int32[n]      quantization bins; 0 where the value is an outlier.
 *                          ABS/NOA: the bin b; REL: 2*b + signbit(x).
 *   mask     uint32[ceil(n/32)]  bit (i & 31) of word (i >> 5) is 1 iff value i
 *                          is an outlier; unused bits of the last word are 0.
 *   outliers T-sized raw bit patterns of the outliers, in ascending index
 *                          order (NaN payloads and the sign of zero preserved).
 *   header   lcq_header    the exact constants used, so the decoder
 *                          reconstructs exactly what the encoder verified.
 */
#ifndef LCQ_H
#define LCQ_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Data types.  LCQ_F32 and LCQ_F64 are the paper's float and double.  The
 * 16-bit formats LCQ_F16 (IEEE binary16) and LCQ_BF16 (bfloat16) go beyond
 * the paper: each value widens exactly to a float and takes the float recipe
 * with float constants; the check of Sec. 3.1 tests the value the decoder
 * outputs, i.e. the float reconstruction rounded to nearest-even in the
 * 16-bit format.  REL treats the widened float's zeros, denormals (so
 * bfloat16 subnormals), Inf and NaN as outliers.  Outliers are stored as raw
 * 16-bit patterns.  The 16-bit formats are accepted by lcq_quantize,
 * lcq_dequantize, lcq_quantize_noalloc, lcq_finite_range,
 * lcq_quantize_noa_range, lcq_quantize_host(_batch), the batched launch
 * (any mix of the four types) and the tuning calls (quantize tile shapes 0
 * and 1, dequantize shapes 1 and 5); the ablations take LCQ_F32 / LCQ_F64
 * only (LCQ_ERR_ARG). */
typedef enum { LCQ_F32 = 0, LCQ_F64 = 1, LCQ_F16 = 2, LCQ_BF16 = 3 } lcq_dtype;

/* Error-bound types, Sec. 2.1: point-wise absolute (ABS), relative (REL) and
 * normalised absolute (NOA, the ABS bound eb * (max - min)). */
typedef enum { LCQ_ABS = 0, LCQ_REL = 1, LCQ_NOA = 2 } lcq_bound_type;

typedef enum {
    LCQ_OK = 0,
    LCQ_ERR_ARG = 1,       /* null/misaligned pointer, bad enum, size too large */
    LCQ_ERR_BOUND = 2,     /* eb <= 0, NaN or Inf; ABS/REL: derived constants not finite-normal */
    LCQ_ERR_CAPACITY = 3,  /* more outliers than outlier_capacity (device-side) */
    LCQ_ERR_TIMEOUT = 4,   /* a bounded wait in the outlier scan gave up (device-side) */
    LCQ_ERR_CUDA = 5,      /* a CUDA launch or copy failed */
    LCQ_ERR_WORKSPACE = 6, /* workspace smaller than lcq_workspace_size() */
    LCQ_ERR_HEADER = 7     /* header does not describe the arrays given to the decoder */
} lcq_status;

/* Device-side status bits (lcq_header.status, dequantize d_status). */
#define LCQ_STATUS_CAPACITY 1u
#define LCQ_STATUS_TIMEOUT 2u
#define LCQ_STATUS_HEADER 4u

#define LCQ_MAGIC 0x3151434Cu /* "LCQ1" */

/* Quantizer header, written to device memory by lcq_quantize.  Float
 * constants are stored as raw bits (a float's bits in the low 32 bits). */
typedef struct lcq_header {
    uint32_t magic;         /* LCQ_MAGIC */
    uint32_t dtype;         /* lcq_dtype */
    uint32_t bound_type;    /* lcq_bound_type */
    uint32_t mode;          /* 0: quantized; 1: every value stored as an outlier
                               (NOA without a usable range); 2: the REL
                               library ablation (see lcq_quantize_ablation) */
    uint64_t n;             /* number of values */
    double eb;              /* the bound passed by the caller */
    double range;           /* NOA: R = RD(max - min) over the finite values, else 0 */
    double eb_abs;          /* ABS: eb; NOA: RD(eb * R); REL: 0 */
    uint64_t ebT_bits;      /* ABS/NOA: eb_T = RD_T(eb_abs); REL: RD_T(eb) */
    uint64_t scale_bits;    /* ABS/NOA: eb2 = 2 eb_T; REL: log-domain step */
    uint64_t inv_bits;      /* ABS/NOA: RN_T(1 / eb2); REL: RN_T(1 / step) */
    uint64_t chk_bits;      /* REL: acceptance factor RN_T(eb_T (1 - 2^-p)); else 0 */
    uint64_t outlier_count; /* total outliers (complete even past capacity) */
    uint32_t status;        /* OR of LCQ_STATUS_* */
    uint32_t reserved;
} lcq_header;

/* Bytes of workspace for lcq_quantize / lcq_dequantize on n values.  For
 * LCQ_F32 with LCQ_REL this includes room for staging outliers: the quantize
 * kernel then copies the outliers of each shared-memory stage out as it
 * streams, and the compaction copies them instead of reading the input a
 * second time.  Any workspace of at least lcq_workspace_size(dtype,
 * LCQ_ABS, n) bytes is accepted for every bound type; with less than this
 * size a float32 REL call simply does not stage (same results). */
size_t lcq_workspace_size(lcq_dtype dtype, lcq_bound_type bound_type, uint64_t n);

/* Zero-fill a workspace on `stream` (needed once before first use). */
lcq_status lcq_workspace_init(void* d_ws, size_t ws_bytes, cudaStream_t stream);

/*
 * Quantize and verify n values (Sec. 2.1-3.3).
 *   dtype, bound_type, eb  the problem as the paper states it: data type, bound
 *                          type and bound (ABS: |x - x'| <= eb; REL:
 *                          |x|/(1+eb) <= |x'| <= |x|(1+eb) with the sign kept;
 *                          NOA: |x - x'| <= eb * (max - min) over finite x).
 *   d_in         T[n]      input values.
 *   d_bins       int32[n]  output bins.
 *   d_mask       uint32[ceil(n/32)] output outlier mask.
 *   d_outliers   T[outlier_capacity] output outlier bit patterns.  Writes stop
 *                          at the capacity; header.outlier_count is complete and
 *                          LCQ_STATUS_CAPACITY is set if it exceeds the capacity.
 *   d_hdr        lcq_header* output header (device memory).
 *   d_ws, ws_bytes         workspace of at least lcq_workspace_size(...) bytes.
 * Each value becomes either a bin whose reconstruction was verified against
 * the bound with the exact IEEE operations the decoder uses, or an outlier
 * (NaN, Inf, values whose bin is out of range, values that fail the check;
 * for REL also zeros and denormals).  Stream-ordered; no host synchronisation.
 * Returns LCQ_ERR_BOUND synchronously for an unusable ABS/REL bound; a NOA
 * range that gives no usable bound makes every value an outlier instead.
 */
lcq_status lcq_quantize(lcq_dtype dtype, lcq_bound_type bound_type, double eb, const void* d_in,
                        uint64_t n, int32_t* d_bins, uint32_t* d_mask, void* d_outliers,
                        uint64_t outlier_capacity, lcq_header* d_hdr, void* d_ws, size_t ws_bytes,
                        cudaStream_t stream);

/*
 * Reconstruct n values from a header written by lcq_quantize (the decoder of
 * Sec. 3.1, without a double-check, Sec. 6): x'_i is the outlier bit pattern
 * if mask bit i is set, else bin_i * eb2 (ABS/NOA) or the pow2 approximation
 * of the stored log-domain bin with the stored sign (REL).  dtype and n must
 * match the header; if they do not, d_status gets LCQ_STATUS_HEADER and
 * d_out is not written.  d_status (uint32, device) may be NULL.
 */
lcq_status lcq_dequantize(lcq_dtype dtype, uint64_t n, const lcq_header* d_hdr,
                          const int32_t* d_bins, const uint32_t* d_mask, const void* d_outliers,
                          void* d_out, uint32_t* d_status, void* d_ws, size_t ws_bytes,
                          cudaStream_t stream);

/*
 * Sharded arrays (Sec. 2.1.3 over the union of contiguous shards held by
 * several ranks).  ABS and REL need no exchange: each shard quantizes alone
 * and the outlier payloads concatenate in rank order.  NOA needs the global
 * finite range before binning:
 *   lcq_finite_range   writes {has_finite (0 or 1), min, max} of the finite
 *       values of d_in to d_range (3 doubles, device, 8-byte aligned; min and
 *       max are exact: values of dtype).  {0, 0, 0} when no value is finite.
 *       Needs a workspace of lcq_workspace_size(dtype, LCQ_NOA, n) bytes.
 *   lcq_quantize_noa_range   lcq_quantize with LCQ_NOA, but R = RD(max - min)
 *       is taken from the caller's range (the combination over all shards:
 *       has_finite = OR, min = MIN, max = MAX) instead of from d_in.  With
 *       has_finite = 0 every value becomes an outlier, as for an input with
 *       no finite value.  Errors: LCQ_ERR_ARG if has_finite is not 0/1, or if
 *       it is 1 and min/max are not finite, min > max, or (LCQ_F32) min/max
 *       are not float values; the other errors as lcq_quantize.
 * Every shard then holds exactly the bins, mask words and outliers that the
 * unsharded call gives for its index range when shard boundaries are
 * multiples of 32 values; its header differs only in n and outlier_count.
 */
lcq_status lcq_finite_range(lcq_dtype dtype, const void* d_in, uint64_t n, double* d_range, void* d_ws,
                            size_t ws_bytes, cudaStream_t stream);
lcq_status lcq_quantize_noa_range(lcq_dtype dtype, double eb, int has_finite, double range_min,
                                  double range_max, const void* d_in, uint64_t n, int32_t* d_bins,
                                  uint32_t* d_mask, void* d_outliers, uint64_t outlier_capacity,
                                  lcq_header* d_hdr, void* d_ws, size_t ws_bytes, cudaStream_t stream);

/*
 * Lossless stage after quantization (no counterpart in the paper, which
 * hands its bins to LC's lossless stages): bit-plane packing of int32 codes
 * (bins or predictor residuals).  For n codes in nb = ceil(n/32) blocks of
 * 32 (the last padded with zeros), z = zigzag(code) = (code << 1) ^ (code >>
 * 31) and w_b = the bit width of the OR of the block's z (0..32).  Layout:
 * w_b as uint8 for every block, zero-padded to a multiple of 16 bytes, then
 * for each block in order w_b uint32 words, word j holding bit j of the
 * block's 32 z values (bit i = code 32 b + i).  Size 16-aligned(nb) +
 * 4 sum(w_b) <= lcq_pack_bound(n).
 *   lcq_pack      d_codes int32[n] -> d_out (at least lcq_pack_bound(n) bytes,
 *       else LCQ_ERR_CAPACITY); *d_out_bytes (uint64, device, may be NULL)
 *       receives the size.  Stream-ordered, no host synchronisation.
 *   lcq_unpack    d_in (in_bytes bytes) -> d_codes int32[n].  A width above
 *       32 or planes beyond in_bytes set LCQ_STATUS_HEADER in *d_status (which
 *       the call first zeroes; may be NULL) and decode as zeros.
 * Both need a workspace of lcq_pack_workspace_size(n) bytes; n > 0; all
 * pointers 16-byte aligned.
 */
size_t lcq_pack_bound(uint64_t n);
size_t lcq_pack_workspace_size(uint64_t n);
lcq_status lcq_pack(const int32_t* d_codes, uint64_t n, void* d_out, size_t out_bytes, uint64_t* d_out_bytes,
                    void* d_ws, size_t ws_bytes, cudaStream_t stream);
lcq_status lcq_unpack(const void* d_in, size_t in_bytes, uint64_t n, int32_t* d_codes, uint32_t* d_status,
                      void* d_ws, size_t ws_bytes, cudaStream_t stream);

/*
 * Ablations of the paper's experiments (not for production use).
 *   LCQ_ABL_ABS_NO_CHECK  ABS without the reconstruct-and-check step: the
 *       unprotected quantizer that Sec. 6 (Tables 7-8) measures against.  Bins
 *       are rint(x / (2 eb_T)) wherever the range tests of Sec. 2.4 / 3.3
 *       pass; NaN, Inf and out-of-range values are still outliers.  The header
 *       is an ordinary ABS header, so lcq_dequantize decodes the result, which
 *       may break the bound (lcq_count_abs_violations counts where).
 *   LCQ_ABL_REL_LIBRARY   REL with the CUDA math library's log2 / exp2 in
 *       place of the Sec. 3.2 approximations (the library variant of Sec. 2.3,
 *       Tables 4-6), still checked on the device with exp2.  Its header has
 *       mode 2; lcq_dequantize refuses it (LCQ_STATUS_HEADER) and only
 *       lcq_rel_library_reconstruct (the same library) decodes it.
 * lcq_quantize_ablation   as lcq_quantize; outputs in the same layout.
 * lcq_ablation_variant    the tile-shape variant (see lcq_tune_*) the ablation
 *       kernel runs, -1 for bad arguments; time the protected kernel on the same
 *       variant for a like-for-like comparison.
 * lcq_rel_library_reconstruct  d_out[i] = the library decode of bin i where
 *       mask bit i is clear, 0 where it is set (outliers are not gathered).
 *       A header that is not an LCQ_ABL_REL_LIBRARY header of n values of
 *       dtype sets LCQ_STATUS_HEADER in *d_status (if not NULL), d_out untouched.
 * lcq_count_abs_violations  *d_count (uint64, device, 8-byte aligned) = the
 *       number of i with |x_i - xr_i| > eb in exact arithmetic; identical bit
 *       patterns (NaN included) never count, any other non-finite pair does.
 *       eb >= 0 (LCQ_ERR_BOUND otherwise).  Stream-ordered.
 */
typedef enum { LCQ_ABL_ABS_NO_CHECK = 0, LCQ_ABL_REL_LIBRARY = 1 } lcq_ablation;
lcq_status lcq_quantize_ablation(lcq_ablation kind, lcq_dtype dtype, double eb, const void* d_in, uint64_t n,
                                 int32_t* d_bins, uint32_t* d_mask, void* d_outliers, uint64_t outlier_capacity,
                                 lcq_header* d_hdr, void* d_ws, size_t ws_bytes, cudaStream_t stream);
int lcq_ablation_variant(lcq_dtype dtype, lcq_ablation kind);
lcq_status lcq_rel_library_reconstruct(lcq_dtype dtype, uint64_t n, const lcq_header* d_hdr,
                                       const int32_t* d_bins, const uint32_t* d_mask, void* d_out,
                                       uint32_t* d_status, cudaStream_t stream);
lcq_status lcq_count_abs_violations(lcq_dtype dtype, double eb, const void* d_x, const void* d_xr, uint64_t n,
                                    unsigned long long* d_count, cudaStream_t stream);

/* Synchronise `stream`, read d_hdr->status and map it to an lcq_status
 * (LCQ_ERR_TIMEOUT before LCQ_ERR_CAPACITY before LCQ_ERR_HEADER).
 * Optionally returns the outlier count.  This one does block the host. */
lcq_status lcq_sync_status(const lcq_header* d_hdr, uint64_t* h_outlier_count,
                           cudaStream_t stream);

/* Static description of a status code. */
const char* lcq_status_string(lcq_status status);

/*
 * End-to-end form for host-resident data: copies h_in to the device, runs
 * lcq_quantize, and copies bins, mask, header and the outliers back into
 * the host buffers; returns once everything is back on the host (it
 * synchronises `stream`).  d_stage is a device buffer of at least
 * lcq_host_stage_size(dtype, n, outlier_capacity) bytes (caller-owned).
 * The work is pipelined in chunks of 2^23 values: the input goes up on one
 * copy stream, each chunk is quantized on `stream` once it has arrived (NOA:
 * once all of it has, for the range), and its bins and mask words come down
 * on another copy stream meanwhile; the outliers come down at the end.  The
 * result is the one lcq_quantize gives.  The two copy streams and their
 * events belong to the library (one set per device, made on first use);
 * calls for one device run one at a time.  For full copy bandwidth the host
 * buffers should be page-locked.
 */
size_t lcq_host_stage_size(lcq_dtype dtype, uint64_t n, uint64_t outlier_capacity);
lcq_status lcq_quantize_host(lcq_dtype dtype, lcq_bound_type bound_type, double eb,
                             const void* h_in, uint64_t n, int32_t* h_bins, uint32_t* h_mask,
                             void* h_outliers, uint64_t outlier_capacity, lcq_header* h_hdr,
                             void* d_stage, size_t stage_bytes, void* d_ws, size_t ws_bytes,
                             cudaStream_t stream);

/*
 * Many host arrays end to end (no counterpart in the paper): each item is
 * quantized exactly as lcq_quantize_host would quantize it, and the items
 * are pipelined across two device stage slots, so that the upload of item
 * j + 1 overlaps the download of item j.  Items must have n > 0.  d_stage:
 * at least lcq_host_batch_stage_size(items, count) device bytes (two slots
 * of the largest item); d_ws: lcq_workspace_size of the largest n.  Each
 * item's status receives its result; the call returns the first error, or
 * LCQ_OK, once everything is on the host.  Calls for one device run one at
 * a time (the copy streams are the library's).
 */
typedef struct lcq_host_item {
    uint32_t dtype;            /* lcq_dtype */
    uint32_t bound_type;       /* lcq_bound_type */
    double eb;
    const void* h_in;          /* host input (page-locked for full bandwidth) */
    uint64_t n;
    int32_t* h_bins;           /* host outputs, as lcq_quantize_host */
    uint32_t* h_mask;
    void* h_outliers;
    uint64_t outlier_capacity;
    lcq_header* h_hdr;
    int32_t status;            /* out: lcq_status of this item */
    uint32_t reserved;
} lcq_host_item;
size_t lcq_host_batch_stage_size(const lcq_host_item* items, uint32_t count);
lcq_status lcq_quantize_host_batch(lcq_host_item* items, uint32_t count, void* d_stage, size_t stage_bytes,
                                   void* d_ws, size_t ws_bytes, cudaStream_t stream);

/*
 * Batched quantization (no counterpart in the paper, which quantizes one file
 * at a time): many arrays of different sizes, data types, bound types and
 * bounds in one persistent launch.  Each array gets exactly the result that
 * lcq_quantize gives it alone (same bins, mask, outliers and header).
 *
 *   lcq_batch_item   one array: the arguments of lcq_quantize.
 *   lcq_batch_plan_size(count)            device bytes of the plan.
 *   lcq_batch_workspace_size(items, count) device bytes of the workspace.
 *   lcq_batch_prepare(...)  validates the items, derives the ABS/REL constants
 *       on the host, writes the plan (a descriptor table and the scan-tile
 *       prefix) to d_plan, initialises the workspace, and fills *h_info.  It
 *       synchronises `stream`.  Errors: LCQ_ERR_ARG / LCQ_ERR_BOUND for the
 *       first bad item (its index in h_info->bad_item).
 *   lcq_quantize_batched(info, plan, ws, stream)  enqueues four kernels: a
 *       header / NOA range pass over all arrays (min/max over finite values
 *       of every NOA array, its bound derived on the device), one persistent
 *       quantize launch over every array's tiles (bins, mask words and each
 *       tile's outlier count), the payload offsets of every array (an
 *       exclusive scan of its tiles' counts, the header's outlier count) and
 *       the outliers' raw bits in index order.  No host work,
 *       no synchronisation, no allocation: it can be captured in a CUDA graph
 *       and replayed; each replay re-reads the inputs and rewrites every
 *       output.  Per-array device errors go to that array's header status.
 *   lcq_batch_tune_*  tile-shape variants of the batched kernel (as for the
 *       single-array kernels below); lcq_autotune_batched times each on the
 *       batch itself and keeps the fastest (synchronises the stream).
 */
typedef struct lcq_batch_item {
    uint32_t dtype;            /* lcq_dtype */
    uint32_t bound_type;       /* lcq_bound_type */
    double eb;
    uint64_t n;
    const void* d_in;
    int32_t* d_bins;
    uint32_t* d_mask;
    void* d_outliers;
    uint64_t outlier_capacity;
    lcq_header* d_hdr;
} lcq_batch_item;

typedef struct lcq_batch_info {
    uint32_t count;            /* arrays */
    uint32_t noa_count;        /* NOA arrays */
    uint64_t total_tiles;      /* 16384-value scan tiles over all arrays */
    uint64_t noa_chunks;       /* 16384-value range chunks over the NOA arrays */
    uint64_t total_values;
    uint64_t total_bytes_in;
    uint32_t bad_item;         /* index of the first rejected item, or UINT32_MAX */
    uint32_t reserved;
} lcq_batch_info;

size_t lcq_batch_plan_size(uint32_t count);
size_t lcq_batch_workspace_size(const lcq_batch_item* h_items, uint32_t count);
lcq_status lcq_batch_prepare(const lcq_batch_item* h_items, uint32_t count, void* d_plan,
                             size_t plan_bytes, void* d_ws, size_t ws_bytes, lcq_batch_info* h_info,
                             cudaStream_t stream);
lcq_status lcq_quantize_batched(const lcq_batch_info* h_info, const void* d_plan, void* d_ws,
                                size_t ws_bytes, cudaStream_t stream);
int lcq_batch_tune_variant_count(void);
lcq_status lcq_batch_tune_set(int variant);
int lcq_batch_tune_get(void);
lcq_status lcq_autotune_batched(const lcq_batch_info* h_info, const void* d_plan, void* d_ws,
                                size_t ws_bytes, cudaStream_t stream, int reps, float* h_ms);

/*
 * Hierarchical-grid predictor of quantization bins (no counterpart in the
 * paper, which keeps the bins and leaves decorrelation to later lossless
 * stages).  The error guarantee is untouched: prediction works on the exact
 * integer bins produced and verified by lcq_quantize, and reconstruction
 * gives back exactly those bins.
 *   Grid: N^3 int32 bins, index (i*N + j)*N + k, 1 <= N <= 2048, every bin
 *   in (-2^30, 2^30) as lcq_quantize produces them (the kernels add pairs of
 *   bins in int32; other values give unspecified residuals, never a fault;
 *   reconstruction of residuals from lcq_pred_residuals stays in range).  Anchors
 *   (coordinates multiples of 8) are kept; a point of stride s = 4, 2, 1
 *   (level 1, 2, 3: multiples of s, not all multiples of 2s) is predicted from
 *   bins of coarser levels: interpolation over the 2^c coarse corners along
 *   its c odd axes, (sum + 2^(c-1)) >> c, coarse positions clamped to the
 *   last multiple of 2s below N; with a network, plus the int8 correction
 *     x_t = clamp((stencil bin t - base) >> s_in[level-1], -128, 127) (3x3x3
 *           coarse stencil around the point rounded down to the coarse grid),
 *     h_u = clamp((W1 x + b1 + 2^(s1-1)) >> s1, 0, 127),
 *     o   = (W2 h + b2 + 2^(s2-1)) >> s2,
 *   one weight set per (level, class of odd axes).  Residual = bin - pred
 *   modulo 2^32 (anchors: the bin).  Supported parameters (lcq_pred_freeze
 *   produces them): |b1|, |b2| <= 2^22, 1 <= s1, s2 <= 24, 0 <= s_in <= 30;
 *   then every sum above fits int32 and the tensor-core products are exact
 *   (other values give unspecified predictions, never a fault).
 * lcq_pred_residuals   bins -> residuals (d_params NULL: interpolation only).
 * lcq_pred_reconstruct residuals -> bins, level by level (exact inverse).
 * lcq_pred_histogram   counts of residual values in [-2^20, 2^20):
 *   d_hist[lcq_pred_histogram_words()] = anchors' counts at value + 2^20, then
 *   predicted points' counts at 2^21 + value + 2^20; values outside the range
 *   are counted in d_over[0] (anchors) / d_over[1]; points whose bit is set
 *   in d_mask (the quantizer's outlier mask; may be NULL) are skipped.
 * Training (straight-through quantisation-aware, all on the device):
 *   shadow parameters float[lcq_train_param_count()] = 21 networks x 465
 *   (w1[16][27], b1[16], w2[16], b2 in integer units).  lcq_train_gradients
 *   takes samples (uint64 (field << 32) | point index into the fields of
 *   d_bins laid back to back), grouped by network and cut into items of at
 *   most 256 samples (struct {uint32 net, start, count, pad}; d_item_begin
 *   [22]: first item of each network); it writes per-item partial sums to
 *   d_partial[num_items * 466], then d_grad[21 * 465] (gradient of the mean
 *   squared residual of each network, summed in item order: deterministic)
 *   and d_loss[21] (sum of squared residuals).  lcq_train_adam applies one
 *   Adam step (Kingma & Ba) with bias corrections for `step` >= 1.
 *   lcq_pred_freeze rounds and clamps the shadow parameters into an
 *   lcq_pred_params block (synchronises the stream).
 */
typedef struct lcq_pred_params {
    int8_t w1[3][7][16][28]; /* [level-1][class-1][hidden][input]; input 27 is padding, 0 */
    int32_t b1[3][7][16];
    int8_t w2[3][7][16];
    int32_t b2[3][7];
    int32_t s_in[3];
    int32_t s1, s2;
    int32_t reserved;
} lcq_pred_params;

lcq_status lcq_pred_residuals(const int32_t* d_bins, uint32_t N, const lcq_pred_params* d_params,
                              int32_t* d_res, cudaStream_t stream);
lcq_status lcq_pred_reconstruct(const int32_t* d_res, uint32_t N, const lcq_pred_params* d_params,
                                int32_t* d_bins, cudaStream_t stream);
size_t lcq_pred_histogram_words(void);
lcq_status lcq_pred_histogram(const int32_t* d_res, uint32_t N, const uint32_t* d_mask, uint32_t* d_hist,
                              unsigned long long* d_over, cudaStream_t stream);
uint32_t lcq_train_param_count(void);
lcq_status lcq_train_gradients(const int32_t* d_bins, uint32_t N, const uint64_t* d_samples, const void* d_items,
                               uint32_t num_items, const uint32_t* d_item_begin, const float* d_shadow,
                               const float* d_inv_count, const int32_t* h_s_in, int32_t s1, int32_t s2,
                               float* d_partial, float* d_grad, float* d_loss, cudaStream_t stream);
lcq_status lcq_train_adam(float* d_shadow, float* d_m, float* d_v, const float* d_grad, float lr, float beta1,
                          float beta2, float eps, uint32_t step, cudaStream_t stream);
lcq_status lcq_pred_freeze(const float* d_shadow, const int32_t* h_s_in, int32_t s1, int32_t s2,
                           lcq_pred_params* d_params, cudaStream_t stream);

/*
 * Tile-shape tuning (no counterpart in the paper; it only affects speed, never
 * results).  The streaming kernels come in lcq_tune_variant_count() tile
 * shapes ("variants"): lcq_tune_describe gives a variant's 4-value vectors per
 * thread per stage (a stage holds 1024 * vpt values), its ring depth, the
 * number of stages per scan tile and the CTAs per SM its register budget
 * allows.  kind: 0 = quantize, 1 = dequantize (the dequantize choice is per
 * dtype; bound_type is ignored).  Choices are process-wide and affect later
 * launches.  lcq_autotune_quantize / lcq_autotune_dequantize run the given
 * call once per variant as warm-up plus `reps` timed times (CUDA events on
 * `stream`), select the fastest, and write the per-variant milliseconds to
 * h_ms[lcq_tune_variant_count()] if it is not NULL.  They synchronise the
 * stream and overwrite the outputs of the call.
 */
int lcq_tune_variant_count(void);
lcq_status lcq_tune_describe(int variant, int* vpt, int* stages, int* sub, int* min_ctas_per_sm);
lcq_status lcq_tune_set(int kind, lcq_dtype dtype, lcq_bound_type bound_type, int variant);
int lcq_tune_get(int kind, lcq_dtype dtype, lcq_bound_type bound_type);
lcq_status lcq_autotune_quantize(lcq_dtype dtype, lcq_bound_type bound_type, double eb, const void* d_in,
                                 uint64_t n, int32_t* d_bins, uint32_t* d_mask, void* d_outliers,
                                 uint64_t outlier_capacity, lcq_header* d_hdr, void* d_ws,
                                 size_t ws_bytes, cudaStream_t stream, int reps, float* h_ms);
lcq_status lcq_autotune_dequantize(lcq_dtype dtype, uint64_t n, const lcq_header* d_hdr,
                                   const int32_t* d_bins, const uint32_t* d_mask, const void* d_outliers,
                                   void* d_out, void* d_ws, size_t ws_bytes, cudaStream_t stream,
                                   int reps, float* h_ms);

/*
 * Allocation-free variant of lcq_quantize.  The paper has no counterpart;
 * this entry point exists for callers that cannot allocate device memory
 * where they quantize (code inside a no-allocation region such as a fixed
 * memory budget streaming pipeline or a simulation step that must not
 * synchronise through the allocator, or code running inside another
 * library's callback), so it takes no workspace argument.
 *   - Arguments, outputs and results are those of lcq_quantize.
 *   - The scan workspace is a fixed 1 MiB device array inside the library,
 *     held by every GPU that loads the library until the process exits.
 *     lcq_noalloc_max_values() is the largest n whose workspace fits it
 *     (with the current layout every n below 2^40 fits); larger n returns
 *     LCQ_ERR_WORKSPACE.  The array has no room for float32 REL outlier
 *     staging, so such a call compacts without it (same results, the
 *     compaction reads the input again).  Every argument is checked before anything is
 *     enqueued: a rejected call (LCQ_ERR_ARG, LCQ_ERR_BOUND,
 *     LCQ_ERR_WORKSPACE) enqueues nothing and leaves the array as it was.
 *   - The array used is the current device's: `stream` must belong to the
 *     current device (LCQ_ERR_ARG otherwise).
 *   - It allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 *     routine.  The first call on each device looks up the device address of
 *     that array (cudaGetSymbolAddress) with the device current; make that
 *     first call before any stream capture.
 *   - Every call on a device shares the one array: calls that can overlap on
 *     the GPU (other streams, other host threads) race and must not be made;
 *     serialise them on one stream.  Each call clears the scan counters and
 *     the group counts it needs at zero before launching, so a call that was
 *     cut short leaves nothing behind for the next one.
 */
uint64_t lcq_noalloc_max_values(void);
lcq_status lcq_quantize_noalloc(lcq_dtype dtype, lcq_bound_type bound_type, double eb,
                                const void* d_in, uint64_t n, int32_t* d_bins, uint32_t* d_mask,
                                void* d_outliers, uint64_t outlier_capacity, lcq_header* d_hdr,
                                cudaStream_t stream);

/*
 * Measurement probe (no counterpart in the paper): enqueue a kernel that
 * issues float64 multiplications as fast as the GPU allows, so that the
 * float64 quantizers can be reported against their FP64 roof as well as
 * HBM bandwidth.  ctas_per_sm (1..64) CTAs of 256 threads per SM, each thread
 * `iters` (1..2^24) rounds of eight independent multiplications; the number
 * of multiplications is written to *h_mults (host, may be NULL) at once, and
 * one double to d_sink (device).  Time it with CUDA events on `stream`.
 */
lcq_status lcq_probe_fp64_mul(uint32_t ctas_per_sm, uint32_t iters, double* d_sink, uint64_t* h_mults,
                              cudaStream_t stream);

/*
 * Test hook for the bounded waits inside the quantize kernel (no counterpart
 * in the paper).  drop_tile: index of a scan tile, within a launch, whose
 * buffers the kernel's scan warp never hands back to the compute warps, so
 * that their wait for it runs out after spin_limit polls and the call
 * reports LCQ_STATUS_TIMEOUT (UINT64_MAX: none; spin_limit 0 restores the
 * default).  Affects subsequent lcq_quantize calls of this process; after a
 * timeout, re-initialise the workspace.
 */
void lcq_debug_set_scan(uint32_t spin_limit, uint64_t drop_tile);

#ifdef __cplusplus
}
#endif

#endif /* LCQ_H */
