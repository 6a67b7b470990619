// gcm_batch.cu -- gcm_batch with GCM_MEM_DEVICE: many independent messages,
// each with its own key schedule and IV, in one persistent launch.
//
// Host side: validates the messages, lays out one scratch allocation
// (message descriptors, key/IV records, per-message key material, tile
// partials and tree scratch, counters), copies the descriptors in with one
// transfer from pinned staging, and enqueues three kernels: key setup for
// all messages (one CTA each), the persistent batched kernel over
// (message, tile) items, and -- for decryption -- the zero-fill of messages
// whose tag failed.  The verdicts come back with one small copy.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "gcm_ctx.h"
#include "gcm_internal.h"
#include "gcmgpu.h"

namespace gcmgpu {

namespace {

size_t al(size_t x) { return (x + 255) / 256 * 256; }

int check_device_msg(const gcm_msg &m)
{
    if (!m.key || (m.key_len != 16 && m.key_len != 24 && m.key_len != 32))
        return ctx_fail(GCM_ERR_INVALID_ARG, "key must be 16, 24 or 32 bytes");
    if (!m.iv || m.iv_len == 0) return ctx_fail(GCM_ERR_INVALID_ARG, "IV must be at least one byte");
    if (m.iv_len > 65536) return ctx_fail(GCM_ERR_LENGTH_LIMIT, "IV longer than 65536 bytes");
    if (m.len > (1ull << 36) - 32) return ctx_fail(GCM_ERR_LENGTH_LIMIT, "payload longer than 2^36 - 32 bytes");
    if ((uint64_t)m.aad_len > (1ull << 40)) return ctx_fail(GCM_ERR_LENGTH_LIMIT, "AAD too long for a batch");
    if (m.aad_len && !m.aad) return ctx_fail(GCM_ERR_INVALID_ARG, "aad is NULL with a nonzero length");
    if (m.len && (!m.in || !m.out)) return ctx_fail(GCM_ERR_INVALID_ARG, "payload pointer is NULL with a nonzero length");
    if (!m.tag) return ctx_fail(GCM_ERR_INVALID_ARG, "tag pointer is NULL");
    if (m.len && ((((uintptr_t)m.in) & 15u) || (((uintptr_t)m.out) & 15u)))
        return ctx_fail(GCM_ERR_ALIGNMENT, "device payload pointers must be 16-byte aligned");
    return GCM_OK;
}

}  // namespace

int batch_device(gcm_ctx *ctx, const gcm_msg *msgs, size_t n, bool decrypt, int32_t *status, uint64_t *done_ns,
                 cudaStream_t s)
{
    for (size_t i = 0; i < n; i++) {
        int rc = check_device_msg(msgs[i]);
        if (rc) return rc;
    }
    if (n == 0) return GCM_OK;
    if (n > 0x7FFFFFFFu) return ctx_fail(GCM_ERR_INVALID_ARG, "too many messages in one batch");
    std::lock_guard<std::mutex> lk(ctx->stream_mu);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    struct Restore {
        int d;
        ~Restore()
        {
            if (d >= 0) cudaSetDevice(d);
        }
    } restore{prev};

    // Work items go out shortest message first: slot j of the launch holds
    // message order[j], so short messages finish early and the median
    // completion time drops (results do not depend on the order).  Verdicts
    // and completion times are mapped back to the caller's order.
    std::vector<uint64_t> Mlen(n);
    for (size_t i = 0; i < n; i++) Mlen[i] = (msgs[i].aad_len + 15) / 16 + (msgs[i].len + 15) / 16;
    std::vector<size_t> order(n);
    std::iota(order.begin(), order.end(), (size_t)0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return Mlen[a] < Mlen[b]; });

    // Sizes and the layout of one scratch allocation (indexed by slot).
    std::vector<uint64_t> K(n), base(n), o_km(n), o_part(n), o_tree(n), o_iv(n);
    uint64_t items = 0;
    for (size_t j = 0; j < n; j++) {
        const uint64_t M = Mlen[order[j]];
        uint64_t k = (M + (1ull << BATCH_TILE_LOG2) - 1) >> BATCH_TILE_LOG2;
        if (k == 0) k = 1;  // an empty message still has one (empty) tile, so its tag gets computed
        K[j] = k;
        base[j] = items;
        items += k;
    }
    size_t off = 0;
    const size_t o_msgs = off;
    off = al(off + n * sizeof(BatchMsg));
    const size_t o_keys = off;
    off = al(off + n * sizeof(BatchKey));
    const size_t o_ivs = off;
    size_t iv_total = 0;
    for (size_t j = 0; j < n; j++) {
        o_iv[j] = iv_total;
        iv_total += msgs[order[j]].iv_len;
    }
    off = al(off + iv_total);
    const size_t host_bytes = off;  // everything above is filled on the host
    const size_t o_done = off;
    off = al(off + n * sizeof(uint32_t));
    const size_t o_counter = off;
    off = al(off + sizeof(unsigned long long));
    const size_t o_status = off;
    off = al(off + n * sizeof(int32_t));
    const size_t counters_bytes = off - o_done;
    const size_t o_times = off;  // t_start, then one completion time per message
    off = al(off + (n + 1) * sizeof(uint64_t));
    for (size_t i = 0; i < n; i++) {
        o_km[i] = off;
        off = al(off + sizeof(KeyMat) + sizeof(MsgMat));
        o_part[i] = off;
        off = al(off + K[i] * sizeof(gf128));
        o_tree[i] = off;
        off = al(off + (K[i] / 2 + 1) * sizeof(gf128));
    }
    const size_t total = off;
    if (ctx->budget && total > ctx->budget)
        return ctx_fail(GCM_ERR_NO_MEMORY, "batch scratch would exceed the context's HBM budget");

    // Pinned staging for the descriptors and for the verdicts coming back.
    const size_t stage_need = al(host_bytes) + al(n * sizeof(int32_t)) + al((n + 1) * sizeof(uint64_t));
    if (ctx->staging_bytes < stage_need) {
        if (ctx->staging) cudaFreeHost(ctx->staging);
        ctx->staging = nullptr;
        ctx->staging_bytes = 0;
        if (cudaMallocHost(reinterpret_cast<void **>(&ctx->staging), stage_need) != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(GCM_ERR_NO_MEMORY, "cannot allocate pinned staging");
        }
        ctx->staging_bytes = stage_need;
    }
    uint8_t *dev = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&dev), total, ctx->pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(GCM_ERR_NO_MEMORY, "batch scratch allocation failed");
    }
    uint8_t *stage = ctx->staging;
    BatchMsg *hm = reinterpret_cast<BatchMsg *>(stage + o_msgs);
    BatchKey *hk = reinterpret_cast<BatchKey *>(stage + o_keys);
    uint8_t *hiv = stage + o_ivs;
    for (size_t i = 0; i < n; i++) {  // i = slot
        const gcm_msg &m = msgs[order[i]];
        BatchMsg &b = hm[i];
        memset(&b, 0, sizeof(b));
        b.in = m.in;
        b.out = m.out;
        b.aad = m.aad;
        b.len = m.len;
        b.aad_len = m.aad_len;
        b.K = K[i];
        b.item_base = base[i];
        b.nr = (uint32_t)m.key_len / 4 + 6;
        b.dec = decrypt ? 1u : 0u;
        b.km = reinterpret_cast<KeyMat *>(dev + o_km[i]);
        b.mm = reinterpret_cast<MsgMat *>(dev + o_km[i] + sizeof(KeyMat));
        b.partials = reinterpret_cast<gf128 *>(dev + o_part[i]);
        b.tree = reinterpret_cast<gf128 *>(dev + o_tree[i]);
        b.tag = m.tag;
        b.status = reinterpret_cast<int32_t *>(dev + o_status) + i;
        b.t_done = done_ns ? reinterpret_cast<uint64_t *>(dev + o_times) + 1 + i : nullptr;
        BatchKey &k = hk[i];
        memset(&k, 0, sizeof(k));
        memcpy(k.key, m.key, m.key_len);
        k.key_len = (uint32_t)m.key_len;
        k.iv_len = (uint32_t)m.iv_len;
        memcpy(hiv + o_iv[i], m.iv, m.iv_len);
        k.iv = dev + o_ivs + o_iv[i];
    }
    e = cudaMemcpyAsync(dev, stage, host_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev + o_done, 0, counters_bytes, s);
    if (e == cudaSuccess)
        e = launch_batch_key_setup(reinterpret_cast<const BatchMsg *>(dev + o_msgs),
                                   reinterpret_cast<const BatchKey *>(dev + o_keys), (uint32_t)n, ctx->tabs,
                                   done_ns ? reinterpret_cast<uint64_t *>(dev + o_times) : nullptr, s);
    ctx->launches += 1;
    BatchParams bp;
    memset(&bp, 0, sizeof(bp));
    bp.msgs = reinterpret_cast<const BatchMsg *>(dev + o_msgs);
    bp.n = (uint32_t)n;
    bp.decrypt = decrypt ? 1u : 0u;
    bp.total_items = items;
    bp.item_counter = reinterpret_cast<unsigned long long *>(dev + o_counter);
    bp.done = reinterpret_cast<uint32_t *>(dev + o_done);
    bp.tabs = ctx->tabs;
    const bool prof = ctx->profiling.load() != 0;
    cudaEvent_t p0 = nullptr, p1 = nullptr;
    if (prof) {
        p0 = ctx_take_event(ctx);
        p1 = ctx_take_event(ctx);
        cudaEventRecord(p0, s);
    }
    if (e == cudaSuccess) e = launch_batch(bp, ctx->num_sms, s);
    if (prof) {
        cudaEventRecord(p1, s);
        uint64_t bytes = 0;
        for (size_t i = 0; i < n; i++) bytes += 2 * msgs[i].len + msgs[i].aad_len;  // order-free
        ctx_record_fused(ctx, p0, p1, bytes);
    }
    ctx->launches += 1;
    if (e == cudaSuccess && decrypt) {
        e = launch_batch_zero(bp.msgs, (uint32_t)n, s);
        ctx->launches += 1;
    }
    int32_t *hstat = reinterpret_cast<int32_t *>(stage + al(host_bytes));
    uint64_t *htimes = reinterpret_cast<uint64_t *>(stage + al(host_bytes) + al(n * sizeof(int32_t)));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hstat, dev + o_status, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && done_ns)
        e = cudaMemcpyAsync(htimes, dev + o_times, (n + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaFreeAsync(dev, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ctx_cuda_fail(e, "batched launch");
    if (status)
        for (size_t j = 0; j < n; j++) status[order[j]] = hstat[j] ? GCM_ERR_AUTH : 0;
    if (done_ns)
        for (size_t j = 0; j < n; j++) done_ns[order[j]] = htimes[1 + j] - htimes[0];
    return GCM_OK;
}

}  // namespace gcmgpu
