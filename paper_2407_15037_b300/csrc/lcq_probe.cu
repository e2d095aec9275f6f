// lcq_probe.cu -- a measurement probe, not part of the quantizer: the rate at
// which this GPU issues float64 multiplications (DMUL), the second roof of
// the float64 quantizers besides HBM bandwidth.  Every thread runs eight
// independent chains of multiplications by a constant just below 1 (no
// overflow, no subnormals within the iteration counts used), so that the
// FP64 pipe, not latency, limits the rate; one store of a combined result
// keeps the work from being removed.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lcq.h"
#include "lcq_host.h"

namespace lcq {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_mul_probe(uint32_t iters, double m, double* sink) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = 1.0 + (double)(threadIdx.x + k) * 0x1p-20;
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = __dmul_rn(a[k], m);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s = __dadd_rn(s, a[k]);
    if (blockIdx.x == 0 && threadIdx.x == 0) *sink = s;
}

}  // namespace
}  // namespace lcq

extern "C" {

lcq_status lcq_probe_fp64_mul(uint32_t ctas_per_sm, uint32_t iters, double* d_sink, uint64_t* h_mults,
                              cudaStream_t stream) {
    if (!d_sink || ctas_per_sm == 0 || ctas_per_sm > 64 || iters == 0 || iters > (1u << 24)) return LCQ_ERR_ARG;
    const uint64_t grid = (uint64_t)lcq::device_sm_count() * ctas_per_sm;
    lcq::k_fp64_mul_probe<<<(unsigned)grid, lcq::kProbeThreads, 0, stream>>>(iters, 0.99999999, d_sink);
    if (cudaPeekAtLastError() != cudaSuccess) return LCQ_ERR_CUDA;
    if (h_mults) *h_mults = grid * lcq::kProbeThreads * (uint64_t)iters * lcq::kChains;
    return LCQ_OK;
}

}  // extern "C"
