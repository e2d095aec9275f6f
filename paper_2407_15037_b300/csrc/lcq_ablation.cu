// lcq_ablation.cu -- device support for the two ablations of the paper's
// experiments (neither is on the production path):
//   k_rel_lib_reconstruct  decoder of the REL variant that uses the CUDA math
//       library's exp2 (Sec. 2.3: a library result depends on the device and
//       library that computes it, so only the same library decodes it);
//   k_count_abs_violations counts values whose reconstruction breaks the ABS
//       bound in exact arithmetic (the violations of the unprotected
//       quantizer, Sec. 6 / Table 7).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/lcq.h"
#include "lcq_device.cuh"
#include "lcq_host.h"

namespace lcq {
namespace {

constexpr int kAblBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kAblBlock) k_rel_lib_reconstruct(const lcq_header* h, const int32_t* bins,
                                                                   const uint32_t* mask, uint64_t n, T* out,
                                                                   uint32_t* status) {
    const bool ok = h->magic == LCQ_MAGIC && h->dtype == (sizeof(T) == 4 ? LCQ_F32 : LCQ_F64) &&
                    h->bound_type == LCQ_REL && h->mode == 2u && h->n == n;
    if (!ok) {
        if (status && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, LCQ_STATUS_HEADER);
        return;
    }
    const Consts<T> c = consts_from_header<T>(h);
    const uint64_t stride = (uint64_t)gridDim.x * kAblBlock;
    for (uint64_t i = (uint64_t)blockIdx.x * kAblBlock + threadIdx.x; i < n; i += stride) {
        const bool outlier = (mask[i >> 5] >> (i & 31)) & 1u;
        out[i] = outlier ? T(0) : rel_recon_lib<T>(bins[i], c);
    }
}

// Exact test of |x - xr| <= eb (eb a double): with a, b the values as
// doubles, s = RN(a - b) and its rounding error e from the two-sum
// transformation (exact: a - b = s + e).  |s| > eb or |s| < eb decide alone
// (rounding to nearest is monotone and eb is a double); |s| == eb is a
// violation iff e points away from zero like s.  Identical bit patterns
// (lossless outliers, NaN included) never violate; otherwise a non-finite
// value on either side does.
__device__ __forceinline__ bool abs_violates(double a, double b, bool same_bits, double eb) {
    if (same_bits) return false;
    if (!isfinite(a) || !isfinite(b)) return true;
    const double s = __dsub_rn(a, b);
    if (!isfinite(s)) return true;  // |a - b| > DBL_MAX > eb
    const double as = fabs(s);
    if (as != eb) return as > eb;
    const double bv = __dsub_rn(s, a);
    const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bv)), __dsub_rn(-b, bv));
    return e != 0.0 && ((e > 0.0) == (s > 0.0));
}

template <typename T>
__global__ void __launch_bounds__(kAblBlock) k_count_abs_violations(const T* x, const T* xr, uint64_t n, double eb,
                                                                    unsigned long long* count) {
    __shared__ unsigned int s_cnt[kAblBlock / 32];
    unsigned int local = 0;
    const uint64_t stride = (uint64_t)gridDim.x * kAblBlock;
    for (uint64_t i = (uint64_t)blockIdx.x * kAblBlock + threadIdx.x; i < n; i += stride) {
        const T a = x[i], b = xr[i];
        local += abs_violates((double)a, (double)b, Ty<T>::bits(a) == Ty<T>::bits(b), eb) ? 1u : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xFFFFFFFFu, local, o);
    if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kAblBlock / 32; w++) t += s_cnt[w];
        if (t) atomicAdd(count, t);
    }
}

unsigned grid_for(uint64_t n) {
    const uint64_t want = (n + kAblBlock - 1) / kAblBlock;
    const uint64_t cap = (uint64_t)device_sm_count() * 8;
    return (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace
}  // namespace lcq

using namespace lcq;

extern "C" {

lcq_status lcq_rel_library_reconstruct(lcq_dtype dtype, uint64_t n, const lcq_header* d_hdr,
                                       const int32_t* d_bins, const uint32_t* d_mask, void* d_out,
                                       uint32_t* d_status, cudaStream_t stream) {
    if (dtype != LCQ_F32 && dtype != LCQ_F64) return LCQ_ERR_ARG;
    if (!d_hdr || !al16(d_hdr) || n >= (1ull << 40)) return LCQ_ERR_ARG;
    if (n > 0 && (!d_bins || !d_mask || !d_out || !al16(d_bins) || !al16(d_mask) || !al16(d_out)))
        return LCQ_ERR_ARG;
    if (n == 0) return LCQ_OK;
    if (dtype == LCQ_F32)
        k_rel_lib_reconstruct<float><<<grid_for(n), kAblBlock, 0, stream>>>(d_hdr, d_bins, d_mask, n, (float*)d_out,
                                                                           d_status);
    else
        k_rel_lib_reconstruct<double><<<grid_for(n), kAblBlock, 0, stream>>>(d_hdr, d_bins, d_mask, n,
                                                                            (double*)d_out, d_status);
    return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
}

lcq_status lcq_count_abs_violations(lcq_dtype dtype, double eb, const void* d_x, const void* d_xr, uint64_t n,
                                    unsigned long long* d_count, cudaStream_t stream) {
    if (dtype != LCQ_F32 && dtype != LCQ_F64) return LCQ_ERR_ARG;
    if (!(eb >= 0.0) || !std::isfinite(eb)) return LCQ_ERR_BOUND;
    if (!d_count || (reinterpret_cast<uintptr_t>(d_count) & 7) != 0 || n >= (1ull << 40)) return LCQ_ERR_ARG;
    if (n > 0 && (!d_x || !d_xr || !al16(d_x) || !al16(d_xr))) return LCQ_ERR_ARG;
    if (cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), stream) != cudaSuccess) return LCQ_ERR_CUDA;
    if (n == 0) return LCQ_OK;
    if (dtype == LCQ_F32)
        k_count_abs_violations<float><<<grid_for(n), kAblBlock, 0, stream>>>((const float*)d_x, (const float*)d_xr,
                                                                            n, eb, d_count);
    else
        k_count_abs_violations<double><<<grid_for(n), kAblBlock, 0, stream>>>(
            (const double*)d_x, (const double*)d_xr, n, eb, d_count);
    return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
}

}  // extern "C"
