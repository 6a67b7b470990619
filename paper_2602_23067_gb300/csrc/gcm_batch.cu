// gcm_batch.cu -- gcm_batch with GCM_MEM_DEVICE: many independent messages,
// each with its own key schedule and IV, in one persistent launch; and the
// same batch prepared once and replayed as a CUDA graph (gcm_batch_plan_*).
//
// Host side: validates the messages, lays out one scratch allocation
// (message descriptors, key/IV records, per-message key material, tile
// partials and tree scratch, counters), copies the descriptors in with one
// transfer from pinned staging, and enqueues three kernels: key setup for
// all messages (one CTA each), the persistent batched kernel over
// (message, tile) items, and -- for decryption -- the zero-fill of messages
// whose tag failed.  The verdicts come back with one small copy.
//
// A plan does the layout, the allocations and the descriptor image once and
// captures that whole sequence (upload, counter reset, three kernels,
// verdict download) into a CUDA graph; every replay re-reads the descriptor
// image from pinned memory, so keys, IVs and buffers can change between
// replays as long as every message keeps its lengths.  A second capture
// replaces the key setup by the per-message J0 / E_K(J0) step and serves the
// replays whose keys did not change.
#include <algorithm>
#include <cmath>
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

// Where one batch lives: the slot order of its messages (shortest first),
// the tiles of each slot, and the offsets inside one scratch allocation.
// Everything below host_bytes is the descriptor image filled on the host.
struct BatchLayout {
    size_t n = 0;
    uint32_t tile_log2 = BATCH_TILE_LOG2;  // tile size of every message of the batch
    std::vector<size_t> order;  // slot -> caller's index
    std::vector<uint64_t> K, base, o_km, o_part, o_tree, o_iv;
    uint64_t items = 0;
    size_t o_msgs = 0, o_keys = 0, o_ivs = 0, host_bytes = 0;
    size_t o_done = 0, o_counter = 0, o_status = 0, counters_bytes = 0, o_times = 0, total = 0;
};

namespace {

// Tile size of a batch in device memory: the size that balances the fixed
// work of a tile (the item fetch, the message's constants, the closing
// multiplies and reductions: about as long as 2,400 blocks of table work)
// against the tail of the last tiles, sqrt(blocks per SM x 2,400), rounded
// to a power of two in 2^9..2^16.  Fitted on batches of 16, 128 and 1024
// small messages: the fastest forced size at 16 and 1024 messages, within
// 8-10% of it at 128; 2^16 for the 10,000-message mix.
uint32_t device_batch_tile_log2(uint64_t total_blocks, int num_sms)
{
    const double w = (double)total_blocks / (double)(num_sms > 0 ? num_sms : 1);
    if (w < 1.0) return SEGF_MIN_LOG2;
    long lg = lround(0.5 * log2(w * 2400.0));
    if (lg < (long)SEGF_MIN_LOG2) lg = SEGF_MIN_LOG2;
    if (lg > (long)BATCH_TILE_LOG2) lg = BATCH_TILE_LOG2;
    return (uint32_t)lg;
}

// tile_log2: the batch's tile size, forced (9..16) or 0 for a rule: the one
// above for device memory, and for host memory the single-message rule (the
// largest tile that gives every SM four tiles), whose extra tiles in flight
// keep more reads crossing the CPU-GPU link at once.
void make_layout(const gcm_msg *msgs, size_t n, int num_sms, int tile_log2, bool host_mem, BatchLayout &L)
{
    L.n = n;
    // Work items go out shortest message first: slot j of the launch holds
    // message order[j], so short messages finish early and the median
    // completion time drops (results do not depend on the order).  Verdicts
    // and completion times are mapped back to the caller's order.
    std::vector<uint64_t> Mlen(n);
    for (size_t i = 0; i < n; i++) Mlen[i] = (msgs[i].aad_len + 15) / 16 + (msgs[i].len + 15) / 16;
    L.order.resize(n);
    std::iota(L.order.begin(), L.order.end(), (size_t)0);
    std::stable_sort(L.order.begin(), L.order.end(), [&](size_t a, size_t b) { return Mlen[a] < Mlen[b]; });

    // One tile size for the batch, so that a batch of short messages spreads
    // over the SMs (a message shorter than a tile runs on one SM) and large
    // batches keep the largest tiles.
    uint64_t total = 0;
    for (size_t i = 0; i < n; i++) total += Mlen[i];
    L.tile_log2 = tile_log2 ? (uint32_t)tile_log2
                            : (host_mem ? choose_tile_log2(total, num_sms) : device_batch_tile_log2(total, num_sms));
    const uint32_t lg = L.tile_log2;
    L.K.assign(n, 0);
    L.base.assign(n, 0);
    L.o_km.assign(n, 0);
    L.o_part.assign(n, 0);
    L.o_tree.assign(n, 0);
    L.o_iv.assign(n, 0);
    L.items = 0;
    for (size_t j = 0; j < n; j++) {
        const uint64_t M = Mlen[L.order[j]];
        uint64_t k = (M + (1ull << lg) - 1) >> lg;
        if (k == 0) k = 1;  // an empty message still has one (empty) tile, so its tag gets computed
        L.K[j] = k;
        L.base[j] = L.items;
        L.items += k;
    }
    size_t off = 0;
    L.o_msgs = off;
    off = al(off + n * sizeof(BatchMsg));
    L.o_keys = off;
    off = al(off + n * sizeof(BatchKey));
    L.o_ivs = off;
    size_t iv_total = 0;
    for (size_t j = 0; j < n; j++) {
        L.o_iv[j] = iv_total;
        iv_total += msgs[L.order[j]].iv_len;
    }
    off = al(off + iv_total);
    L.host_bytes = off;  // everything above is filled on the host
    L.o_done = off;
    off = al(off + n * sizeof(uint32_t));
    L.o_counter = off;
    off = al(off + sizeof(unsigned long long));
    L.o_status = off;
    off = al(off + n * sizeof(int32_t));
    L.counters_bytes = off - L.o_done;
    L.o_times = off;  // t_start, then one completion time per message
    off = al(off + (n + 1) * sizeof(uint64_t));
    for (size_t j = 0; j < n; j++) {
        L.o_km[j] = off;
        off = al(off + sizeof(KeyMat) + sizeof(MsgMat));
        L.o_part[j] = off;
        off = al(off + L.K[j] * sizeof(gf128));
        L.o_tree[j] = off;
        off = al(off + (L.K[j] / 2 + 1) * sizeof(gf128));
    }
    L.total = off;
}

// Writes slot j's records (message m) into the descriptor image `image`;
// the device pointers inside refer to the scratch allocation `dev`.
void fill_slot(const BatchLayout &L, size_t j, const gcm_msg &m, bool decrypt, bool timed, uint8_t *dev,
               uint8_t *image)
{
    BatchMsg &b = reinterpret_cast<BatchMsg *>(image + L.o_msgs)[j];
    memset(&b, 0, sizeof(b));
    b.in = m.in;
    b.out = m.out;
    b.aad = m.aad;
    b.len = m.len;
    b.aad_len = m.aad_len;
    b.K = L.K[j];
    b.item_base = L.base[j];
    b.nr = (uint32_t)m.key_len / 4 + 6;
    b.dec = decrypt ? 1u : 0u;
    b.tile_log2 = L.tile_log2;
    b.km = reinterpret_cast<KeyMat *>(dev + L.o_km[j]);
    b.mm = reinterpret_cast<MsgMat *>(dev + L.o_km[j] + sizeof(KeyMat));
    b.partials = reinterpret_cast<gf128 *>(dev + L.o_part[j]);
    b.tree = reinterpret_cast<gf128 *>(dev + L.o_tree[j]);
    b.tag = m.tag;
    b.status = reinterpret_cast<int32_t *>(dev + L.o_status) + j;
    b.t_done = timed ? reinterpret_cast<uint64_t *>(dev + L.o_times) + 1 + j : nullptr;
    BatchKey &k = reinterpret_cast<BatchKey *>(image + L.o_keys)[j];
    memset(&k, 0, sizeof(k));
    memcpy(k.key, m.key, m.key_len);
    k.key_len = (uint32_t)m.key_len;
    k.iv_len = (uint32_t)m.iv_len;
    memcpy(image + L.o_ivs + L.o_iv[j], m.iv, m.iv_len);
    k.iv = dev + L.o_ivs + L.o_iv[j];
}

// Enqueues one run of the batch on s: descriptor image in, counters zeroed,
// key setup (or, with key_setup false, only J0 and E_K(J0) from the key
// material already in the scratch), the persistent kernel, the zero-fill of
// failed messages (decrypt), verdicts (and, when timed, completion times)
// out to the pinned host words.  *kernels receives the number of kernels
// enqueued.  With prof the persistent kernel is bracketed by profiling
// events (prof_bytes: the bytes it moves).
cudaError_t enqueue_batch(gcm_ctx *ctx, const BatchLayout &L, uint8_t *dev, const uint8_t *image, bool decrypt,
                          bool key_setup, bool timed, bool prof, uint64_t prof_bytes, int32_t *hstat,
                          uint64_t *htimes, cudaStream_t s, int *kernels)
{
    const size_t n = L.n;
    *kernels = 0;
    cudaError_t e = cudaMemcpyAsync(dev, image, L.host_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev + L.o_done, 0, L.counters_bytes, s);
    const BatchMsg *dmsgs = reinterpret_cast<const BatchMsg *>(dev + L.o_msgs);
    const BatchKey *dkeys = reinterpret_cast<const BatchKey *>(dev + L.o_keys);
    if (e == cudaSuccess)
        e = key_setup ? launch_batch_key_setup(dmsgs, dkeys, (uint32_t)n, ctx->tabs,
                                               timed ? reinterpret_cast<uint64_t *>(dev + L.o_times) : nullptr, s)
                      : launch_msg_setup(dmsgs, dkeys, (uint32_t)n, ctx->tabs, s);
    *kernels += 1;
    BatchParams bp;
    memset(&bp, 0, sizeof(bp));
    bp.msgs = reinterpret_cast<const BatchMsg *>(dev + L.o_msgs);
    bp.n = (uint32_t)n;
    bp.decrypt = decrypt ? 1u : 0u;
    bp.total_items = L.items;
    bp.item_counter = reinterpret_cast<unsigned long long *>(dev + L.o_counter);
    bp.done = reinterpret_cast<uint32_t *>(dev + L.o_done);
    bp.tabs = ctx->tabs;
    cudaEvent_t p0 = nullptr, p1 = nullptr;
    if (prof) {
        p0 = ctx_take_event(ctx);
        p1 = ctx_take_event(ctx);
        cudaEventRecord(p0, s);
    }
    if (e == cudaSuccess) e = launch_batch(bp, ctx->num_sms, s);
    if (prof) {
        cudaEventRecord(p1, s);
        ctx_record_fused(ctx, p0, p1, prof_bytes);
    }
    *kernels += 1;
    if (e == cudaSuccess && decrypt) {
        e = launch_batch_zero(bp.msgs, (uint32_t)n, s);
        *kernels += 1;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hstat, dev + L.o_status, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && timed)
        e = cudaMemcpyAsync(htimes, dev + L.o_times, (n + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    return e;
}

}  // namespace

int batch_device(gcm_ctx *ctx, const gcm_msg *msgs, size_t n, bool decrypt, int32_t *status, uint64_t *done_ns,
                 cudaStream_t s, bool host_mem)
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

    BatchLayout L;
    make_layout(msgs, n, ctx->num_sms, ctx->forced_tile_log2, host_mem, L);
    if (ctx->budget && L.total > ctx->budget)
        return ctx_fail(GCM_ERR_NO_MEMORY, "batch scratch would exceed the context's HBM budget");

    // Pinned staging for the descriptors and for the verdicts coming back.
    const size_t stage_need = al(L.host_bytes) + al(n * sizeof(int32_t)) + al((n + 1) * sizeof(uint64_t));
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
    cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&dev), L.total, ctx->pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(GCM_ERR_NO_MEMORY, "batch scratch allocation failed");
    }
    uint8_t *stage = ctx->staging;
    for (size_t j = 0; j < n; j++) fill_slot(L, j, msgs[L.order[j]], decrypt, done_ns != nullptr, dev, stage);
    const bool prof = ctx->profiling.load() != 0;
    uint64_t prof_bytes = 0;
    if (prof)
        for (size_t i = 0; i < n; i++) prof_bytes += 2 * msgs[i].len + msgs[i].aad_len;  // order-free
    int32_t *hstat = reinterpret_cast<int32_t *>(stage + al(L.host_bytes));
    uint64_t *htimes = reinterpret_cast<uint64_t *>(stage + al(L.host_bytes) + al(n * sizeof(int32_t)));
    int kernels = 0;
    e = enqueue_batch(ctx, L, dev, stage, decrypt, true, done_ns != nullptr, prof, prof_bytes, hstat, htimes, s,
                      &kernels);
    ctx->launches += kernels;
    if (e == cudaSuccess) e = cudaFreeAsync(dev, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ctx_cuda_fail(e, "batched launch");
    if (status)
        for (size_t j = 0; j < n; j++) status[L.order[j]] = hstat[j] ? GCM_ERR_AUTH : 0;
    if (done_ns)
        for (size_t j = 0; j < n; j++) done_ns[L.order[j]] = htimes[1 + j] - htimes[0];
    return GCM_OK;
}

}  // namespace gcmgpu

// A batch prepared for repeated runs (the opaque gcm_batch_plan handle).
struct gcm_batch_plan {
    gcm_ctx *ctx = nullptr;
    int device = 0;
    bool decrypt = false;
    gcmgpu::BatchLayout L;
    std::vector<size_t> slot_of;  // caller's index -> slot
    std::vector<gcm_msg> shape;   // lengths fixed at creation (caller's order; pointers unused)
    uint8_t *dev = nullptr;       // scratch, held until destroy
    size_t held = 0;              // bytes of it counted in the context's scratch in flight
    uint8_t *pinned = nullptr;    // descriptor image read by every replay, then the verdict words
    int32_t *hstat = nullptr;
    std::vector<uint8_t> pending;  // descriptor image edited by gcm_batch_plan_set
    bool dirty = false;
    bool in_flight = false;
    // Two captures of the run: [1] sets up every message's key material,
    // [0] derives only J0 and E_K(J0) from the key material a [1] run left in
    // the scratch; [0] runs when no key changed since the last [1] run.
    bool keys_built = false, keys_changed = false;
    int kernels[2] = {0, 0};
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaEvent_t done = nullptr;
    std::mutex mu;
};

namespace {

using gcmgpu::ctx_cuda_fail;
using gcmgpu::ctx_fail;

struct OnDevice {
    int prev = -1;
    explicit OnDevice(int dev)
    {
        cudaGetDevice(&prev);
        cudaSetDevice(dev);
    }
    ~OnDevice()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

void plan_free(gcm_batch_plan *P)
{
    for (int g = 0; g < 2; g++) {
        if (P->exec[g]) cudaGraphExecDestroy(P->exec[g]);
        if (P->graph[g]) cudaGraphDestroy(P->graph[g]);
    }
    if (P->done) cudaEventDestroy(P->done);
    if (P->dev) cudaFree(P->dev);
    if (P->held) {
        std::lock_guard<std::mutex> lk(P->ctx->mu);
        P->ctx->in_flight -= P->held;
    }
    if (P->pinned) {
        memset(P->pinned, 0, P->L.host_bytes);  // the image holds the keys
        cudaFreeHost(P->pinned);
    }
    if (!P->pending.empty()) memset(P->pending.data(), 0, P->pending.size());
    delete P;
}

}  // namespace

extern "C" {

int gcm_batch_plan_create(gcm_ctx *ctx, const gcm_msg *msgs, size_t n, int decrypt, gcm_batch_plan **out)
{
    using namespace gcmgpu;
    TraceRange trace_("gcm_batch_plan_create");
    if (!out) return ctx_fail(GCM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx) return ctx_fail(GCM_ERR_INVALID_ARG, "context is NULL");
    if (n == 0 || !msgs) return ctx_fail(GCM_ERR_INVALID_ARG, "a plan needs at least one message");
    if (n > 0x7FFFFFFFu) return ctx_fail(GCM_ERR_INVALID_ARG, "too many messages in one batch");
    for (size_t i = 0; i < n; i++) {
        int rc = check_device_msg(msgs[i]);
        if (rc) return rc;
    }
    OnDevice on(ctx->device);
    gcm_batch_plan *P = new gcm_batch_plan();
    P->ctx = ctx;
    P->device = ctx->device;
    P->decrypt = decrypt != 0;
    make_layout(msgs, n, ctx->num_sms, ctx->forced_tile_log2, false, P->L);
    const BatchLayout &L = P->L;
    {
        // Held for the plan's lifetime, like the scratch of calls in flight.
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (!ctx->budget || ctx->in_flight + L.total <= ctx->budget) {
            ctx->in_flight += L.total;
            P->held = L.total;
        }
    }
    if (!P->held) {
        plan_free(P);
        return ctx_fail(GCM_ERR_NO_MEMORY, "the plan's scratch would exceed the context's HBM budget");
    }
    P->shape.assign(msgs, msgs + n);
    P->slot_of.assign(n, 0);
    for (size_t j = 0; j < n; j++) P->slot_of[L.order[j]] = j;

    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&P->dev), L.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        plan_free(P);
        return ctx_fail(GCM_ERR_NO_MEMORY, "plan scratch allocation failed");
    }
    e = cudaHostAlloc(reinterpret_cast<void **>(&P->pinned), al(L.host_bytes) + al(n * sizeof(int32_t)),
                      cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        P->pinned = nullptr;
        plan_free(P);
        return ctx_fail(GCM_ERR_NO_MEMORY, "cannot allocate the plan's page-locked descriptor image");
    }
    P->hstat = reinterpret_cast<int32_t *>(P->pinned + al(L.host_bytes));
    P->pending.assign(L.host_bytes, 0);
    for (size_t j = 0; j < n; j++) fill_slot(L, j, msgs[L.order[j]], P->decrypt, false, P->dev, P->pending.data());
    memcpy(P->pinned, P->pending.data(), L.host_bytes);

    // Capture the whole run once per form; the capture only records the work.
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int g = 0; g < 2 && e == cudaSuccess; g++) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = enqueue_batch(ctx, L, P->dev, P->pinned, P->decrypt, g == 1, false, false, 0, P->hstat,
                                           nullptr, cs, &P->kernels[g]);
            cudaError_t e2 = cudaStreamEndCapture(cs, &P->graph[g]);
            e = e1 != cudaSuccess ? e1 : e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec[g], P->graph[g], 0);
    }
    if (cs) cudaStreamDestroy(cs);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        int rc = ctx_cuda_fail(e, "capturing the batch plan");
        plan_free(P);
        return rc;
    }
    *out = P;
    return GCM_OK;
}

int gcm_batch_plan_set(gcm_batch_plan *P, size_t first, const gcm_msg *msgs, size_t count)
{
    using namespace gcmgpu;
    if (!P || (count && !msgs)) return ctx_fail(GCM_ERR_INVALID_ARG, "plan or messages are NULL");
    if (first > P->L.n || count > P->L.n - first) return ctx_fail(GCM_ERR_INVALID_ARG, "message index out of range");
    for (size_t k = 0; k < count; k++) {
        const gcm_msg &m = msgs[k];
        int rc = check_device_msg(m);
        if (rc) return rc;
        const gcm_msg &s = P->shape[first + k];
        if (m.len != s.len || m.aad_len != s.aad_len || m.key_len != s.key_len || m.iv_len != s.iv_len)
            return ctx_fail(GCM_ERR_INVALID_ARG,
                            "a plan's message keeps the payload, AAD, key and IV lengths it was created with");
    }
    std::lock_guard<std::mutex> lk(P->mu);
    for (size_t k = 0; k < count; k++) {
        const size_t j = P->slot_of[first + k];
        const BatchKey &old = reinterpret_cast<const BatchKey *>(P->pending.data() + P->L.o_keys)[j];
        if (memcmp(old.key, msgs[k].key, msgs[k].key_len) != 0) P->keys_changed = true;
        fill_slot(P->L, j, msgs[k], P->decrypt, false, P->dev, P->pending.data());
    }
    if (count) P->dirty = true;
    return GCM_OK;
}

int gcm_batch_plan_launch(gcm_batch_plan *P, void *stream)
{
    using namespace gcmgpu;
    TraceRange trace_("gcm_batch_plan_launch");
    if (!P) return ctx_fail(GCM_ERR_INVALID_ARG, "plan is NULL");
    std::lock_guard<std::mutex> lk(P->mu);
    if (P->in_flight) return ctx_fail(GCM_ERR_BUSY, "the plan's previous run has not been waited for");
    OnDevice on(P->device);
    // The previous run has been waited for, so nothing reads the image now.
    if (P->dirty) {
        memcpy(P->pinned, P->pending.data(), P->L.host_bytes);
        P->dirty = false;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int g = (!P->keys_built || P->keys_changed) ? 1 : 0;
    cudaError_t e = cudaGraphLaunch(P->exec[g], s);
    if (e == cudaSuccess) e = cudaEventRecord(P->done, s);
    if (e != cudaSuccess) return ctx_cuda_fail(e, "launching the batch plan");
    if (g == 1) {
        P->keys_built = true;
        P->keys_changed = false;
    }
    P->ctx->launches += P->kernels[g];
    P->in_flight = true;
    return GCM_OK;
}

int gcm_batch_plan_wait(gcm_batch_plan *P, int32_t *status)
{
    using namespace gcmgpu;
    if (!P) return ctx_fail(GCM_ERR_INVALID_ARG, "plan is NULL");
    std::lock_guard<std::mutex> lk(P->mu);
    if (!P->in_flight) return ctx_fail(GCM_ERR_INVALID_ARG, "the plan has no run in flight");
    OnDevice on(P->device);
    cudaError_t e = cudaEventSynchronize(P->done);
    P->in_flight = false;
    if (e != cudaSuccess) return ctx_cuda_fail(e, "batch plan run");
    if (status)
        for (size_t j = 0; j < P->L.n; j++) status[P->L.order[j]] = P->hstat[j] ? GCM_ERR_AUTH : 0;
    return GCM_OK;
}

void gcm_batch_plan_destroy(gcm_batch_plan *P)
{
    if (!P) return;
    OnDevice on(P->device);
    if (P->in_flight) cudaEventSynchronize(P->done);
    plan_free(P);
}

}  // extern "C"
