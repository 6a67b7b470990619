// gcm_ctx.h -- the session object behind the opaque gcm_ctx handle.
// Internal to the library (shared by the C-ABI implementation files).
#pragma once
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "gcm_internal.h"

struct gcm_ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;          // 0 = unlimited
    size_t in_flight = 0;       // scratch bytes held by calls not yet returned
    cudaMemPool_t pool = nullptr;
    gcmgpu::DevTables *tabs = nullptr;
    std::mutex mu;
    // measurement hooks
    std::atomic<int> profiling{0};
    std::atomic<uint64_t> launches{0};
    struct Timed {
        cudaEvent_t start, stop;
        uint64_t bytes;
    };
    std::vector<Timed> timed;       // recorded, not yet read
    std::vector<cudaEvent_t> spare; // recycled events
    double fused_ms = 0.0;
    uint64_t fused_launches = 0, fused_bytes = 0;
};

