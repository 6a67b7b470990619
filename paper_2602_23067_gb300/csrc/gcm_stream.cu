// gcm_stream.cu -- host-memory messages streamed through device chunk buffers.
//
// The paper overlaps host<->device transfers with the GCM kernels on CUDA
// streams with pinned buffers (Sec. 3.3.2, "Asynchronous Streams Pipeline";
// Sec. 5.2.3).  Here every message's GHASH sequence is cut into chunks of
// whole tiles; chunk c is copied into ring slot c mod R on the copy-in
// stream, processed by the fused kernel (restricted to the chunk's tiles) on
// the compute stream, and copied back on the copy-out stream, each step
// waiting on the previous one through events, and a slot is refilled only
// after its copy-out finished.  So copies in both directions and the
// kernels of neighbouring chunks run at the same time, and the device
// footprint is R chunk buffers however large the catalog is.  The tile
// partials stay in per-message scratch until the message's combine runs.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "gcm_ctx.h"
#include "gcm_internal.h"
#include "gcmgpu.h"

namespace gcmgpu {

namespace {

struct Guard {
    int prev = -1;
    explicit Guard(int dev)
    {
        cudaGetDevice(&prev);
        cudaSetDevice(dev);
    }
    ~Guard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int ensure_resources(gcm_ctx *ctx, size_t n_msgs)
{
    cudaError_t e = cudaSuccess;
    if (!ctx->s_h2d) {
        e = cudaStreamCreateWithFlags(&ctx->s_h2d, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->s_comp, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->s_d2h, cudaStreamNonBlocking);
        if (e != cudaSuccess) return ctx_cuda_fail(e, "creating the streaming streams");
    }
    const size_t want_ring = (size_t)ctx->n_buffers * ctx->chunk_bytes;
    if (ctx->ring_bytes != want_ring) {
        if (ctx->ring) {
            cudaFree(ctx->ring);
            ctx->ring = nullptr;
            ctx->ring_bytes = 0;
        }
        if (ctx->budget && want_ring > ctx->budget) return ctx_fail(GCM_ERR_NO_MEMORY, "chunk ring exceeds the HBM budget");
        e = cudaMalloc(&ctx->ring, want_ring);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(GCM_ERR_NO_MEMORY, "cannot allocate the device chunk ring");
        }
        ctx->ring_bytes = want_ring;
    }
    while ((int)ctx->ev_h2d.size() < ctx->n_buffers) {
        cudaEvent_t a, b, c;
        e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c, cudaEventDisableTiming);
        if (e != cudaSuccess) return ctx_cuda_fail(e, "creating streaming events");
        ctx->ev_h2d.push_back(a);
        ctx->ev_comp.push_back(b);
        ctx->ev_d2h.push_back(c);
    }
    const size_t want_stage = align256(n_msgs * 32 + 32);
    if (ctx->staging_bytes < want_stage) {
        if (ctx->staging) cudaFreeHost(ctx->staging);
        ctx->staging = nullptr;
        ctx->staging_bytes = 0;
        e = cudaMallocHost(reinterpret_cast<void **>(&ctx->staging), want_stage);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(GCM_ERR_NO_MEMORY, "cannot allocate pinned staging");
        }
        ctx->staging_bytes = want_stage;
    }
    return GCM_OK;
}

int check_msg(const gcm_msg &m)
{
    if (!m.key || (m.key_len != 16 && m.key_len != 24 && m.key_len != 32))
        return ctx_fail(GCM_ERR_INVALID_ARG, "key must be 16, 24 or 32 bytes");
    if (!m.iv || m.iv_len == 0) return ctx_fail(GCM_ERR_INVALID_ARG, "IV must be at least one byte");
    if (m.iv_len > 65536) return ctx_fail(GCM_ERR_LENGTH_LIMIT, "IV longer than 65536 bytes");
    if (m.len > (1ull << 36) - 32) return ctx_fail(GCM_ERR_LENGTH_LIMIT, "payload longer than 2^36 - 32 bytes");
    if ((uint64_t)m.aad_len > (1ull << 61) - 1) return ctx_fail(GCM_ERR_LENGTH_LIMIT, "AAD longer than 2^61 - 1 bytes");
    if (m.aad_len && !m.aad) return ctx_fail(GCM_ERR_INVALID_ARG, "aad is NULL with a nonzero length");
    if (m.len && (!m.in || !m.out)) return ctx_fail(GCM_ERR_INVALID_ARG, "payload pointer is NULL with a nonzero length");
    if (!m.tag) return ctx_fail(GCM_ERR_INVALID_ARG, "tag pointer is NULL");
    return GCM_OK;
}

}  // namespace

void stream_release(gcm_ctx *ctx)
{
    if (ctx->s_h2d) {
        cudaStreamSynchronize(ctx->s_h2d);
        cudaStreamSynchronize(ctx->s_comp);
        cudaStreamSynchronize(ctx->s_d2h);
        cudaStreamDestroy(ctx->s_h2d);
        cudaStreamDestroy(ctx->s_comp);
        cudaStreamDestroy(ctx->s_d2h);
        ctx->s_h2d = ctx->s_comp = ctx->s_d2h = nullptr;
    }
    for (auto e : ctx->ev_h2d) cudaEventDestroy(e);
    for (auto e : ctx->ev_comp) cudaEventDestroy(e);
    for (auto e : ctx->ev_d2h) cudaEventDestroy(e);
    ctx->ev_h2d.clear();
    ctx->ev_comp.clear();
    ctx->ev_d2h.clear();
    if (ctx->ring) cudaFree(ctx->ring);
    ctx->ring = nullptr;
    ctx->ring_bytes = 0;
    if (ctx->staging) cudaFreeHost(ctx->staging);
    ctx->staging = nullptr;
    ctx->staging_bytes = 0;
}

int stream_host(gcm_ctx *ctx, const gcm_msg *msgs, size_t n, bool decrypt, int32_t *status)
{
    for (size_t i = 0; i < n; i++) {
        int rc = check_msg(msgs[i]);
        if (rc) return rc;
    }
    std::lock_guard<std::mutex> lk(ctx->stream_mu);
    Guard guard(ctx->device);
    int rc = ensure_resources(ctx, n);
    if (rc) return rc;
    const int R = ctx->n_buffers;
    const size_t C = ctx->chunk_bytes;
    cudaStream_t sh = ctx->s_h2d, sc = ctx->s_comp, sd = ctx->s_d2h;
    std::vector<bool> slot_used(R, false);
    int slot_next = 0;
    uint8_t *stage = ctx->staging;  // per message: 16 tag bytes + 4 status bytes at 32*i
    cudaError_t e = cudaSuccess;
    const bool prof = ctx->profiling.load() != 0;

    for (size_t mi = 0; mi < n && e == cudaSuccess; mi++) {
        const gcm_msg &m = msgs[mi];
        const uint64_t a = (m.aad_len + 15) / 16, nb = (m.len + 15) / 16, M = a + nb;
        // Tiles no larger than a chunk, so chunks are whole tiles.
        uint32_t lg = choose_tile_log2(M, ctx->num_sms);
        while (lg > 10 && ((size_t)16 << lg) > C) lg--;
        const uint64_t K = (M + (1ull << lg) - 1) >> lg;
        uint32_t levels = 0;
        while ((1ull << levels) < K) levels++;
        if (lg + levels >= (uint32_t)H2K_COUNT) return ctx_fail(GCM_ERR_LENGTH_LIMIT, "message too long for the power table");
        const uint64_t tiles_per_chunk = (C / 16) >> lg;

        // Per-message scratch: KeyMat | MsgMat | partials | tree | aad | iv | tag | status.
        const size_t o_km = 0, o_mm = align256(sizeof(KeyMat)), o_part = align256(o_mm + sizeof(MsgMat));
        const size_t o_tree = align256(o_part + K * sizeof(gf128));
        const size_t o_aad = align256(o_tree + (K / 2 + 1) * sizeof(gf128));
        const size_t o_iv = align256(o_aad + m.aad_len);
        const size_t o_tag = align256(o_iv + (m.iv_len > IV_INLINE_MAX ? m.iv_len : 0));
        const size_t total = o_tag + 256;
        uint8_t *sb = nullptr;
        e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&sb), total, ctx->pool, sc);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(GCM_ERR_NO_MEMORY, "per-message scratch allocation failed");
        }
        KeyMat *km = reinterpret_cast<KeyMat *>(sb + o_km);
        MsgMat *mm = reinterpret_cast<MsgMat *>(sb + o_mm);
        gf128 *part = reinterpret_cast<gf128 *>(sb + o_part);
        uint8_t *d_tag = sb + o_tag;
        int32_t *d_status = reinterpret_cast<int32_t *>(sb + o_tag + 16);
        if (m.aad_len) e = cudaMemcpyAsync(sb + o_aad, m.aad, m.aad_len, cudaMemcpyHostToDevice, sc);
        if (e == cudaSuccess && decrypt) e = cudaMemcpyAsync(d_tag, m.tag, 16, cudaMemcpyHostToDevice, sc);

        KsParams ks;
        memset(&ks, 0, sizeof(ks));
        memcpy(ks.key, m.key, m.key_len);
        ks.key_len = (uint32_t)m.key_len;
        ks.iv_len = (uint32_t)m.iv_len;
        if (m.iv_len <= (size_t)IV_INLINE_MAX) {
            memcpy(ks.iv_inline, m.iv, m.iv_len);
        } else if (e == cudaSuccess) {
            e = cudaMemcpyAsync(sb + o_iv, m.iv, m.iv_len, cudaMemcpyHostToDevice, sc);
            ks.iv_dev = sb + o_iv;
        }
        ks.km = km;
        ks.mm = mm;
        ks.tabs = ctx->tabs;
        if (e == cudaSuccess) e = launch_key_setup(ks, sc);
        ctx->launches += 1;

        KfParams kf;
        memset(&kf, 0, sizeof(kf));
        kf.aad = sb + o_aad;
        kf.len = m.len;
        kf.aad_len = m.aad_len;
        kf.a_blocks = a;
        kf.n_full = m.len / 16;
        kf.M = M;
        kf.K = K;
        kf.tile_log2 = lg;
        kf.decrypt = decrypt ? 1u : 0u;
        kf.km = km;
        kf.mm = mm;
        kf.tabs = ctx->tabs;
        kf.partials = part;
        const int nr = (int)m.key_len / 4 + 6;
        for (uint64_t t0 = 0; t0 < K && e == cudaSuccess; t0 += tiles_per_chunk) {
            const uint64_t t1 = (t0 + tiles_per_chunk < K) ? t0 + tiles_per_chunk : K;
            const int64_t s_lo_raw = (int64_t)M - (int64_t)((K - t0) << lg);
            const uint64_t s_lo = s_lo_raw > 0 ? (uint64_t)s_lo_raw : 0;
            const uint64_t s_hi = M - ((K - t1) << lg);
            const uint64_t jb = s_lo > a ? s_lo - a : 0, je = s_hi > a ? s_hi - a : 0;
            const uint64_t b0 = 16 * jb;
            const uint64_t b1 = (16 * je < m.len) ? 16 * je : m.len;
            kf.tile_begin = t0;
            kf.tile_end = t1;
            const int grid = (int)((t1 - t0) < (uint64_t)ctx->num_sms ? (t1 - t0) : (uint64_t)ctx->num_sms);
            cudaEvent_t p0 = nullptr, p1 = nullptr;
            if (b1 > b0) {
                const int slot = slot_next;
                slot_next = (slot_next + 1) % R;
                uint8_t *buf = ctx->ring + (size_t)slot * C;
                if (slot_used[slot]) e = cudaStreamWaitEvent(sh, ctx->ev_d2h[slot], 0);
                if (e == cudaSuccess) e = cudaMemcpyAsync(buf, m.in + b0, b1 - b0, cudaMemcpyHostToDevice, sh);
                if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_h2d[slot], sh);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(sc, ctx->ev_h2d[slot], 0);
                kf.in = buf - b0;
                kf.out = buf - b0;
                if (prof) {
                    p0 = ctx_take_event(ctx);
                    p1 = ctx_take_event(ctx);
                    cudaEventRecord(p0, sc);
                }
                if (e == cudaSuccess) e = launch_fused(kf, nr, grid, sc);
                if (prof) {
                    cudaEventRecord(p1, sc);
                    ctx_record_fused(ctx, p0, p1, 2 * (b1 - b0));
                }
                ctx->launches += 1;
                if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_comp[slot], sc);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(sd, ctx->ev_comp[slot], 0);
                if (e == cudaSuccess) e = cudaMemcpyAsync(m.out + b0, buf, b1 - b0, cudaMemcpyDeviceToHost, sd);
                if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_d2h[slot], sd);
                slot_used[slot] = true;
            } else {
                // A chunk of AAD blocks only.
                kf.in = ctx->ring;
                kf.out = ctx->ring;
                if (e == cudaSuccess) e = launch_fused(kf, nr, grid, sc);
                ctx->launches += 1;
            }
        }

        KcParams kc;
        memset(&kc, 0, sizeof(kc));
        kc.partials = part;
        kc.scratch = reinterpret_cast<gf128 *>(sb + o_tree);
        kc.K = K;
        kc.tile_log2 = lg;
        kc.aad_len = m.aad_len;
        kc.len = m.len;
        kc.km = km;
        kc.mm = mm;
        kc.tag_out = decrypt ? nullptr : d_tag;
        kc.tag_expected = decrypt ? d_tag : nullptr;
        kc.status = d_status;
        if (e == cudaSuccess) e = launch_combine(kc, sc);
        ctx->launches += 1;
        if (e == cudaSuccess) e = cudaMemcpyAsync(stage + 32 * mi, d_tag, 20, cudaMemcpyDeviceToHost, sc);
        if (e == cudaSuccess) e = cudaFreeAsync(sb, sc);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(sc);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sd);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sh);
    if (e != cudaSuccess) return ctx_cuda_fail(e, "streamed host pipeline");
    for (size_t mi = 0; mi < n; mi++) {
        int32_t st = 0;
        if (decrypt) {
            memcpy(&st, stage + 32 * mi + 16, 4);
            if (st != 0) {
                st = GCM_ERR_AUTH;
                if (msgs[mi].len) memset(msgs[mi].out, 0, msgs[mi].len);  // payload suppression
            }
        } else {
            memcpy(msgs[mi].tag, stage + 32 * mi, 16);
        }
        if (status) status[mi] = st;
    }
    return GCM_OK;
}

}  // namespace gcmgpu
