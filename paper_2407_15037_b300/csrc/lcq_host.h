// lcq_host.h -- host-side helpers shared between the library's translation
// units (not part of the C ABI).
#pragma once

#include <atomic>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/lcq.h"

namespace lcq {

// ABS/REL constants of Sec. 2.2 and the REL reading, as the raw bits stored
// in lcq_header (ebT, scale, inv, chk), and the certainty bounds of the
// float64 REL check (0 otherwise); false if the bound is unusable.
bool host_consts(lcq_dtype dtype, lcq_bound_type bound, double eb, uint64_t bits[4],
                 uint64_t* cert_w = nullptr, uint32_t* cert_emin = nullptr);

// Validation shared by lcq_quantize and the batch planner.
lcq_status check_quantize_args(lcq_dtype dtype, lcq_bound_type bound_type, double eb, const void* d_in,
                               uint64_t n, const int32_t* d_bins, const uint32_t* d_mask,
                               const void* d_outliers, uint64_t outlier_capacity, const lcq_header* d_hdr);

int device_sm_count();

// Host-side launch set-up done once per (kernel, device) -- the dynamic
// shared-memory opt-in and the occupancy query -- is cached.  Host threads
// may launch on several devices at once, so each fill happens under one
// library-wide lock and is published with a release store; readers take the
// lock-free path once it is set.
constexpr int kMaxDevices = 64;
std::mutex& launch_setup_mutex();

struct OccupancyCache {
    std::atomic<int> per_sm[kMaxDevices];  // CTAs per SM; 0 = not set up on that device
};

// CTAs of `kernel` (threads per CTA, dyn_smem bytes of dynamic shared
// memory) that fit on one SM of device dev, the opt-in to dyn_smem included.
template <typename K>
int cached_blocks_per_sm(OccupancyCache& cache, int dev, K kernel, int threads, size_t dyn_smem) {
    auto setup = [&]() {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, dyn_smem);
        return b > 0 ? b : 1;
    };
    if (dev < 0 || dev >= kMaxDevices) {
        std::lock_guard<std::mutex> g(launch_setup_mutex());
        return setup();
    }
    int v = cache.per_sm[dev].load(std::memory_order_acquire);
    if (v) return v;
    std::lock_guard<std::mutex> g(launch_setup_mutex());
    v = cache.per_sm[dev].load(std::memory_order_relaxed);
    if (!v) {
        v = setup();
        cache.per_sm[dev].store(v, std::memory_order_release);
    }
    return v;
}

}  // namespace lcq
