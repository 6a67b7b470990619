// gcm_ctx.h -- the session object behind the opaque gcm_ctx handle.
// Internal to the library (shared by the C-ABI implementation files).
#pragma once
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <thread>
#include <utility>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "gcm_internal.h"
#include "gcmgpu.h"

namespace gcmgpu {
// A named NVTX range over a scope: the library's public calls and the
// server's waves show up by name in a profiler timeline (a no-op unless a
// tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
}  // namespace gcmgpu

struct gcm_ctx {
    int device = 0;
    int num_sms = 0;
    // Host buffers are read and written by the kernels themselves over the
    // CPU-GPU link (coherent access, e.g. NVLink-C2C with address translation)
    // instead of being copied through device staging buffers.
    bool host_direct = false;
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
    // host-mode streaming (created on first use)
    size_t chunk_bytes = (size_t)256 << 20;
    int n_buffers = 3;
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    std::vector<cudaEvent_t> ev_h2d, ev_comp, ev_d2h;
    std::mutex stream_mu;  // one streamed call at a time per context
    uint8_t *ring = nullptr;        // n_buffers x chunk_bytes device chunk buffers
    size_t ring_bytes = 0;
    uint8_t *staging = nullptr;     // pinned host staging for tags / status words
    size_t staging_bytes = 0;
    // registered keys (gcm_key_register)
    std::vector<gcmgpu::KeyMat *> keys;
    std::vector<uint32_t> key_nr;
    // Key material of the single-message calls, cached per key on the device
    // (least recently used entry replaced; guarded by mu).  An entry is only
    // overwritten when no call holds it and every stream that used it has
    // passed its last use.
    struct KeyCacheEntry {
        uint8_t key[32];
        uint32_t key_len = 0;
        gcmgpu::KeyMat *km = nullptr;
        uint64_t tick = 0;            // last use, for LRU
        int holders = 0;              // calls between acquire and release
        cudaEvent_t ready = nullptr;  // recorded after the entry's key setup
        std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;  // last use per stream
    };
    std::vector<KeyCacheEntry> key_cache;
    size_t key_cache_cap = 64;
    uint64_t key_cache_tick = 0;
    // Tile size of the single-message path: forced (gcm_ctx_set_tile_log2),
    // else the autotuned choice for the sequence's size class
    // (tuned_lg[floor(log2(blocks))], 0 = not tuned), else the built-in rule.
    int forced_tile_log2 = 0;
    uint8_t tuned_lg[64] = {};
    // AES engine of the single-message fused pass (GCM_AES_TABLES / _BITSLICED).
    int aes_impl = 0;
    // Ticket words of fused launches that finish their own message (the
    // last CTA runs the combine and the tag): one zero word per stream the
    // calls use (keyed by the runtime's stream id, never reused), so that
    // only launches ordered on one stream share a word; a launch leaves its
    // word at zero.  The per-thread default stream is one handle for many
    // streams, so its words are per calling thread too.  Once every slot is
    // taken, calls on further streams use the separate combine kernel.
    static constexpr int TICKET_SLOTS = 4096;
    uint32_t *tickets = nullptr;
    std::map<std::pair<unsigned long long, std::thread::id>, int> ticket_slot;  // guarded by mu
};

namespace gcmgpu {
// Shared between the C-ABI implementation files.
int ctx_fail(int code, const char *msg);
// gcm_encrypt / gcm_decrypt_verify that also return the FITS DATASUM of the
// ciphertext side (when the data goes through the device pass; *datasum_done
// tells).  Waits for the stream.
int ctx_run_with_datasum(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *iv, size_t iv_len,
                         const uint8_t *aad, size_t aad_len, const uint8_t *in, size_t len, uint8_t *out,
                         uint8_t *tag, bool decrypt, int mem, void *stream, uint32_t *datasum, bool *datasum_done);
int ctx_cuda_fail(cudaError_t e, const char *where);
uint32_t choose_tile_log2(uint64_t M, int num_sms);
void ctx_record_fused(gcm_ctx *ctx, cudaEvent_t start, cudaEvent_t stop, uint64_t bytes);
cudaEvent_t ctx_take_event(gcm_ctx *ctx);
// Host-memory messages streamed through device chunk buffers (gcm_stream.cu).
int stream_host(gcm_ctx *ctx, const gcm_msg *msgs, size_t n, bool decrypt, int32_t *status);
void stream_release(gcm_ctx *ctx);
// Device-memory messages in one persistent batched launch (gcm_batch.cu).
// host_mem: the buffers are host memory the kernels reach directly.
int batch_device(gcm_ctx *ctx, const gcm_msg *msgs, size_t n, bool decrypt, int32_t *status, uint64_t *done_ns,
                 cudaStream_t s, bool host_mem = false);
}  // namespace gcmgpu

