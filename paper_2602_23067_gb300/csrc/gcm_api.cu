// gcm_api.cu -- C ABI of the library (declared in include/gcmgpu.h).
//
// Host code only validates arguments, sizes the tiling, takes per-call device
// scratch from a stream-ordered pool and enqueues the kernels of
// gcm_kernels.cu.  Every step of the method runs on the device.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "gcm_ctx.h"
#include "gcm_internal.h"
#include "gcmgpu.h"

using namespace gcmgpu;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, const char *detail = nullptr)
{
    char buf[512];
    if (detail)
        snprintf(buf, sizeof(buf), fmt, detail);
    else
        snprintf(buf, sizeof(buf), "%s", fmt);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    g_last_error = buf;
    return GCM_ERR_CUDA;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

constexpr uint64_t MAX_PAYLOAD = (1ull << 36) - 32;  // 2^39 - 256 bits
constexpr uint64_t MAX_AAD = (1ull << 61) - 1;       // 2^64 - 1 bits
constexpr uint64_t MAX_IV = 65536;                    // library cap

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

cudaEvent_t take_event(gcm_ctx *ctx)
{
    // caller holds ctx->mu
    if (!ctx->spare.empty()) {
        cudaEvent_t e = ctx->spare.back();
        ctx->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Tile size: 2^16 blocks (1 MiB) for large sequences; smaller for short ones
// so that there are at least a few tiles per SM.
uint32_t tile_log2_for(uint64_t M, int num_sms)
{
    uint32_t lg = 16;
    while (lg > (uint32_t)SEGF_MIN_LOG2 && (M >> lg) < (uint64_t)num_sms * 4) lg--;
    return lg;
}

int size_class(uint64_t M)
{
    int c = 0;
    while (c < 63 && (M >> (c + 1)) != 0) c++;
    return c;
}

// Tile sizes found by gcm_ctx_autotune on a GB300 (152 SMs, compute
// capability 10.3), 16 KiB .. 1 GiB, indexed by floor(log2(blocks));
// installed by default on that device.  AES-128 and AES-256 give the same
// table since messages of up to 1024 tiles finish inside the fused launch
// (up to 4 MiB the smallest tiles win: more CTAs, no combine launch).
// Medium messages prefer about one tile per SM over the rule's four.
const uint8_t kTunedGB300[64] = {
    0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  9,  9,  9,  9,  9,  9,  9,  9,  11, 11, 13, 13,
    15, 15, 14, 14, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16,
    16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16};

uint32_t tile_log2_ctx(const gcm_ctx *ctx, uint64_t M)
{
    if (ctx->forced_tile_log2) return (uint32_t)ctx->forced_tile_log2;
    const uint8_t t = ctx->tuned_lg[size_class(M)];
    return t ? t : tile_log2_for(M, ctx->num_sms);
}

struct Scratch {
    void *base = nullptr;
    size_t bytes = 0;
};

// The ticket word of `s` for fused launches that finish their message, or
// null when every slot is taken or `s` is being captured into a graph (the
// call then uses the combine kernel: replays of a graph on several streams
// at once would share one word).  Slots are keyed by the stream's id, which
// the runtime never reuses (a stream handle can be reused after
// cudaStreamDestroy while the destroyed stream's work is still running, so
// the handle cannot be the key).
uint32_t *ticket_for(gcm_ctx *ctx, cudaStream_t s)
{
    if (!ctx->tickets) return nullptr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;
    }
    unsigned long long id = 0;
    if (cudaStreamGetId(s, &id) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const std::thread::id who = (s == cudaStreamPerThread) ? std::this_thread::get_id() : std::thread::id();
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->ticket_slot.find({id, who});
    if (it != ctx->ticket_slot.end()) return ctx->tickets + it->second;
    const int n = (int)ctx->ticket_slot.size();
    if (n >= gcm_ctx::TICKET_SLOTS) return nullptr;
    ctx->ticket_slot.emplace(std::make_pair(id, who), n);
    return ctx->tickets + n;
}

int scratch_alloc(gcm_ctx *ctx, size_t bytes, cudaStream_t s, Scratch &out)
{
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->budget && ctx->in_flight + bytes > ctx->budget)
            return fail(GCM_ERR_NO_MEMORY, "device scratch would exceed the context's HBM budget");
        ctx->in_flight += bytes;
    }
    cudaError_t e = cudaMallocFromPoolAsync(&out.base, bytes, ctx->pool, s);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->in_flight -= bytes;
        cudaGetLastError();
        return fail(GCM_ERR_NO_MEMORY, "device scratch allocation failed: %s", cudaGetErrorString(e));
    }
    out.bytes = bytes;
    return GCM_OK;
}

void scratch_free(gcm_ctx *ctx, Scratch &sc, cudaStream_t s)
{
    if (sc.base) cudaFreeAsync(sc.base, s);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->in_flight -= sc.bytes;
    sc.base = nullptr;
    sc.bytes = 0;
}

int check_common(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *iv, size_t iv_len,
                 const uint8_t *aad, size_t aad_len, const uint8_t *in, size_t len, const uint8_t *out,
                 const uint8_t *tag, int mem)
{
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    if (mem != GCM_MEM_DEVICE && mem != GCM_MEM_HOST) return fail(GCM_ERR_INVALID_ARG, "mem must be GCM_MEM_DEVICE or GCM_MEM_HOST");
    if (!key || (key_len != 16 && key_len != 24 && key_len != 32))
        return fail(GCM_ERR_INVALID_ARG, "key must be 16, 24 or 32 bytes");
    if (!iv || iv_len == 0) return fail(GCM_ERR_INVALID_ARG, "IV must be at least one byte");
    if (iv_len > MAX_IV) return fail(GCM_ERR_LENGTH_LIMIT, "IV longer than 65536 bytes");
    if (len > MAX_PAYLOAD) return fail(GCM_ERR_LENGTH_LIMIT, "payload longer than 2^36 - 32 bytes");
    if ((uint64_t)aad_len > MAX_AAD) return fail(GCM_ERR_LENGTH_LIMIT, "AAD longer than 2^61 - 1 bytes");
    if (aad_len && !aad) return fail(GCM_ERR_INVALID_ARG, "aad is NULL with a nonzero length");
    if (len && (!in || !out)) return fail(GCM_ERR_INVALID_ARG, "payload pointer is NULL with a nonzero length");
    if (!tag) return fail(GCM_ERR_INVALID_ARG, "tag pointer is NULL");
    if (mem == GCM_MEM_DEVICE && len &&
        (((uintptr_t)in & 15u) != 0 || ((uintptr_t)out & 15u) != 0))
        return fail(GCM_ERR_ALIGNMENT, "device payload pointers must be 16-byte aligned");
    return GCM_OK;
}

// The context's key-material cache.  key_cache_acquire returns the slot of
// `ks.key` with ks.km pointing at its device key material and this
// message's J0 / E_K(J0) setup already enqueued on s: the full key setup
// when the key is new to the cache, only the message part when it is cached
// (after waiting for the stream that set it up).  It returns -1 when the key
// cannot be cached now (cache disabled or every entry in use); the caller
// then sets up private key material.  A held slot is released, after the
// call's last kernel that reads it, by key_cache_release.
int key_cache_acquire(gcm_ctx *ctx, KsParams &ks, cudaStream_t s, cudaError_t &err, int &launched)
{
    err = cudaSuccess;
    launched = 0;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->key_cache_cap == 0) return -1;
    auto &C = ctx->key_cache;
    int slot = -1;
    for (size_t i = 0; i < C.size(); i++)
        if (C[i].key_len == ks.key_len && memcmp(C[i].key, ks.key, ks.key_len) == 0) {
            slot = (int)i;
            break;
        }
    bool fresh = false;
    if (slot < 0) {
        if (C.size() < ctx->key_cache_cap) {
            gcm_ctx::KeyCacheEntry e;
            // The entry's KeyMat is followed by its flat-reduce weights.
            if (cudaMalloc(reinterpret_cast<void **>(&e.km), sizeof(KeyMat) + sizeof(KeyFin)) != cudaSuccess) {
                cudaGetLastError();
                return -1;
            }
            if (cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming) != cudaSuccess) {
                cudaFree(e.km);
                cudaGetLastError();
                return -1;
            }
            C.push_back(e);
            slot = (int)C.size() - 1;
        } else {
            // Least recently used entry that no call holds and whose last
            // use has completed on every stream.
            uint64_t best = UINT64_MAX;
            for (size_t i = 0; i < C.size(); i++) {
                if (C[i].holders || C[i].tick >= best) continue;
                bool idle = cudaEventQuery(C[i].ready) == cudaSuccess;
                for (auto &u : C[i].uses) idle = idle && cudaEventQuery(u.second) == cudaSuccess;
                if (idle) {
                    best = C[i].tick;
                    slot = (int)i;
                }
            }
            cudaGetLastError();  // clears cudaErrorNotReady left by the queries
            if (slot < 0) return -1;
        }
        fresh = true;
    }
    auto &e = C[slot];
    ks.km = e.km;
    ks.fin = reinterpret_cast<KeyFin *>(e.km + 1);
    if (fresh) {
        memcpy(e.key, ks.key, ks.key_len);
        e.key_len = ks.key_len;
        err = launch_key_setup(ks, s);
        launched = 1;
        if (err == cudaSuccess) err = cudaEventRecord(e.ready, s);
        if (err != cudaSuccess) {
            memset(e.key, 0, sizeof(e.key));
            e.key_len = 0;
            return -1;
        }
    } else {
        // With a 96-bit IV the caller forms J0 on the host and the kernel
        // that computes the tag (the finishing CTA of the fused launch, or
        // the combine kernel) derives E_K(J0), so nothing per message is
        // needed here.
        err = cudaStreamWaitEvent(s, e.ready, 0);
        if (err == cudaSuccess && ks.iv_len != 12) {
            err = launch_msg_only(ks, s);
            launched = 1;
        }
        if (err != cudaSuccess) return -1;
    }
    e.tick = ++ctx->key_cache_tick;
    e.holders++;
    return slot;
}

void key_cache_release(gcm_ctx *ctx, int slot, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto &e = ctx->key_cache[slot];
    cudaEvent_t ev = nullptr;
    for (auto &u : e.uses)
        if (u.first == s) ev = u.second;
    if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) e.uses.push_back({s, ev});
    if (ev) cudaEventRecord(ev, s);
    e.holders--;
}

// Enqueues the whole device path for one message whose aad/in/out/tag live
// in device memory.  For decryption `tag_dev` is the expected tag and
// `status_dev` receives 0 or GCM_ERR_AUTH; for encryption the tag is written.
// mode 1 (CTR only) writes out = in xor keystream and no tag; mode 2 (GHASH
// only) writes GHASH_H(aad, in) to tag_dev and no payload output.
int enqueue_device(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *iv, size_t iv_len,
                   const uint8_t *aad, size_t aad_len, const uint8_t *in, size_t len, uint8_t *out,
                   uint8_t *tag_dev, bool decrypt, int32_t *status_dev, Scratch &sc, cudaStream_t s,
                   int mode = 0, uint32_t *datasum_dev = nullptr)
{
    if (datasum_dev && mode == 0) mode = 3;  // GCM plus the DATASUM of the ciphertext side
    const uint64_t a_blocks = (aad_len + 15) / 16;
    const uint64_t n_blocks = (len + 15) / 16;
    const uint64_t M = a_blocks + n_blocks;
    const uint32_t lg = tile_log2_ctx(ctx, M);
    const uint64_t K = (M + (1ull << lg) - 1) >> lg;
    uint32_t levels = 0;
    while ((1ull << levels) < K) levels++;
    if (lg + levels >= (uint32_t)H2K_COUNT) return fail(GCM_ERR_LENGTH_LIMIT, "message too long for the power table");

    // Scratch layout: KeyMat + KeyFin | MsgMat | partials[K] | tree scratch | IV copy
    const size_t off_km = 0;
    const size_t off_mm = align_up(off_km + sizeof(KeyMat) + sizeof(KeyFin), 256);
    const size_t off_part = align_up(off_mm + sizeof(MsgMat), 256);
    const size_t off_tree = align_up(off_part + (size_t)K * sizeof(gf128), 256);
    const size_t off_iv = align_up(off_tree + (size_t)(K / 2 + 1) * sizeof(gf128), 256);
    const size_t off_ds = align_up(off_iv + (iv_len > IV_INLINE_MAX ? iv_len : 0), 256);
    const size_t total = align_up(off_ds + (mode == 3 ? (size_t)K * sizeof(uint32_t) : 0), 256);
    int rc = scratch_alloc(ctx, total, s, sc);
    if (rc) return rc;
    uint8_t *base = static_cast<uint8_t *>(sc.base);
    KeyMat *km = reinterpret_cast<KeyMat *>(base + off_km);
    MsgMat *mm = reinterpret_cast<MsgMat *>(base + off_mm);
    gf128 *partials = reinterpret_cast<gf128 *>(base + off_part);
    gf128 *tree = reinterpret_cast<gf128 *>(base + off_tree);

    KsParams ks;
    memset(&ks, 0, sizeof(ks));
    memcpy(ks.key, key, key_len);
    ks.key_len = (uint32_t)key_len;
    ks.iv_len = (uint32_t)iv_len;
    if (iv_len <= IV_INLINE_MAX) {
        memcpy(ks.iv_inline, iv, iv_len);
    } else {
        uint8_t *div = base + off_iv;
        cudaError_t e = cudaMemcpyAsync(div, iv, iv_len, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "IV copy");
        ks.iv_dev = div;
    }
    ks.mm = mm;
    ks.tabs = ctx->tabs;
    cudaError_t e = cudaSuccess;
    int setup_launches = 0;
    const int slot = key_cache_acquire(ctx, ks, s, e, setup_launches);
    if (e != cudaSuccess) return cuda_fail(e, "key setup launch");
    if (slot >= 0) {
        km = ks.km;
    } else {
        ks.km = km;
        ks.fin = reinterpret_cast<KeyFin *>(km + 1);
        e = launch_key_setup(ks, s);
        if (e != cudaSuccess) return cuda_fail(e, "key setup launch");
        setup_launches = 1;
    }
    ctx->launches += setup_launches;
    // Releases the cache slot after the last kernel of this call that reads
    // the key material has been enqueued (on every return path below).
    struct SlotGuard {
        gcm_ctx *ctx;
        int slot;
        cudaStream_t s;
        ~SlotGuard()
        {
            if (slot >= 0) key_cache_release(ctx, slot, s);
        }
    } slot_guard{ctx, slot, s};

    const int nr = (int)key_len / 4 + 6;
    KfParams kf;
    memset(&kf, 0, sizeof(kf));
    kf.in = in;
    kf.out = out;
    kf.aad = aad;
    kf.len = len;
    kf.aad_len = aad_len;
    kf.a_blocks = a_blocks;
    kf.n_full = len / 16;
    kf.M = M;
    kf.K = K;
    kf.tile_begin = 0;
    kf.tile_end = K;
    kf.tile_log2 = lg;
    kf.decrypt = decrypt ? 1u : 0u;
    kf.km = km;
    kf.mm = mm;
    kf.tabs = ctx->tabs;
    kf.partials = partials;
    if (mode == 3) kf.dsums = reinterpret_cast<uint32_t *>(base + off_ds);
    if (iv_len == 12) {
        // J0 = IV || 0^31 || 1 (SP 800-38D Alg. 4 step 2), as memory words.
        kf.j0_given = 1u;
        for (int i = 0; i < 3; i++)
            kf.j0[i] = (uint32_t)iv[4 * i] | ((uint32_t)iv[4 * i + 1] << 8) | ((uint32_t)iv[4 * i + 2] << 16) |
                       ((uint32_t)iv[4 * i + 3] << 24);
        kf.j0[3] = 0x01000000u;
    }
    // Messages of a few tiles are finished by the fused launch itself (its
    // last CTA runs the reduce, the tag and the verify gate): no combine or
    // zero-fill launch follows.
    const bool can_finish = (mode == 2) || (mode != 1 && ctx->aes_impl == 0);
    if (can_finish && K >= 1 && K <= FINISH_MAX_TILES && M <= FINISH_MAX_BLOCKS) {
        kf.ticket = ticket_for(ctx, s);
        if (kf.ticket) {
            kf.fin = reinterpret_cast<const KeyFin *>(km + 1);
            kf.tag_out = decrypt ? nullptr : tag_dev;
            kf.tag_expected = decrypt ? tag_dev : nullptr;
            kf.status = status_dev;
            if (mode == 3) kf.datasum_out = datasum_dev;
        }
    }
    const int grid = (int)((K < (uint64_t)ctx->num_sms) ? K : (uint64_t)ctx->num_sms);
    const bool prof = ctx->profiling.load() != 0 && K > 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (prof) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ev0 = take_event(ctx);
        ev1 = take_event(ctx);
    }
    if (prof) cudaEventRecord(ev0, s);
    e = launch_fused(kf, nr, grid, s, mode, ctx->aes_impl);
    if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
    if (prof) {
        cudaEventRecord(ev1, s);
        std::lock_guard<std::mutex> lk(ctx->mu);
        const uint64_t moved = (mode == 2 ? (uint64_t)len : (uint64_t)len * 2u) + (mode == 1 ? 0u : (uint64_t)aad_len);
        ctx->timed.push_back({ev0, ev1, moved});
    }
    ctx->launches += (K > 0) ? 1 : 0;
    if (mode == 1) return GCM_OK;  // CTR only: no authenticator
    if (kf.ticket) return GCM_OK;  // finished by the fused launch

    KcParams kc;
    memset(&kc, 0, sizeof(kc));
    kc.partials = partials;
    kc.scratch = tree;
    kc.K = K;
    kc.tile_log2 = lg;
    kc.aad_len = aad_len;
    kc.len = len;
    kc.km = km;
    kc.mm = mm;
    kc.tag_out = decrypt ? nullptr : tag_dev;
    kc.tag_expected = decrypt ? tag_dev : nullptr;
    kc.status = status_dev;
    kc.raw = (mode == 2) ? 1 : 0;
    kc.tabs = ctx->tabs;
    if (mode == 3 && K > 0) {
        kc.dsums = kf.dsums;
        kc.datasum_out = datasum_dev;
    }
    if (kf.j0_given) {
        kc.ej0_from_j0 = 1u;
        for (int i = 0; i < 4; i++) kc.j0[i] = kf.j0[i];
    }
    e = launch_combine(kc, s);
    if (e != cudaSuccess) return cuda_fail(e, "combine kernel launch");
    ctx->launches += 1;

    if (decrypt && len) {
        KzParams kz;
        kz.out = out;
        kz.len = len;
        kz.status = status_dev;
        const uint64_t nvec = len / 16 + 1;
        uint64_t g = (nvec + 255) / 256;
        if (g > (uint64_t)ctx->num_sms * 8) g = (uint64_t)ctx->num_sms * 8;
        e = launch_zero_on_fail(kz, (int)g, s);
        if (e != cudaSuccess) return cuda_fail(e, "zero-fill launch");
        ctx->launches += 1;
    }
    return GCM_OK;
}

// datasum (optional, host): receives the FITS DATASUM of the ciphertext side
// computed in the same pass, and the call then waits for its stream; it is
// left untouched (and *datasum_done false) on the staged host path.
int run_call(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *iv, size_t iv_len,
             const uint8_t *aad, size_t aad_len, const uint8_t *in, size_t len, uint8_t *out, uint8_t *tag,
             bool decrypt, int mem, void *stream, uint32_t *datasum = nullptr, bool *datasum_done = nullptr)
{
    if (datasum_done) *datasum_done = false;
    int rc = check_common(ctx, key, key_len, iv, iv_len, aad, aad_len, in, len, out, tag, mem);
    if (rc) return rc;
    const bool aligned = ((((uintptr_t)in) | ((uintptr_t)out)) & 15u) == 0;
    if (mem == GCM_MEM_HOST && ctx->host_direct && aligned) {
        // The kernels read the host buffers and write the host output
        // directly over the CPU-GPU link; only the tag / verdict pass
        // through device scratch.
        DeviceGuard guard(ctx->device);
        if (!guard.ok) return fail(GCM_ERR_CUDA, "cannot select the context's device");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        Scratch io;
        rc = scratch_alloc(ctx, 256, s, io);
        if (rc) return rc;
        uint8_t *iob = static_cast<uint8_t *>(io.base);
        int32_t *d_status = reinterpret_cast<int32_t *>(iob);
        uint8_t *d_tag = iob + 64;
        uint32_t *d_sum = datasum ? reinterpret_cast<uint32_t *>(iob + 128) : nullptr;
        cudaError_t e = cudaSuccess;
        if (decrypt) e = cudaMemcpyAsync(d_tag, tag, 16, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && d_sum) e = cudaMemsetAsync(d_sum, 0, 4, s);
        if (e != cudaSuccess) {
            scratch_free(ctx, io, s);
            return cuda_fail(e, "tag copy");
        }
        Scratch sc;
        rc = enqueue_device(ctx, key, key_len, iv, iv_len, aad, aad_len, in, len, out, d_tag, decrypt, d_status, sc, s,
                            0, d_sum);
        if (rc) {
            if (sc.base) scratch_free(ctx, sc, s);
            scratch_free(ctx, io, s);
            return rc;
        }
        scratch_free(ctx, sc, s);
        int32_t status = 0;
        uint8_t htag[16];
        e = cudaMemcpyAsync(decrypt ? (void *)&status : (void *)htag, decrypt ? (void *)d_status : (void *)d_tag,
                            decrypt ? sizeof(int32_t) : 16, cudaMemcpyDeviceToHost, s);
        uint32_t hsum = 0;
        if (e == cudaSuccess && d_sum) e = cudaMemcpyAsync(&hsum, d_sum, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        scratch_free(ctx, io, s);
        if (e != cudaSuccess) return cuda_fail(e, "host-direct call");
        if (!decrypt) memcpy(tag, htag, 16);
        if (d_sum) {
            *datasum = hsum;
            if (datasum_done) *datasum_done = true;
        }
        if (decrypt && status != 0) return fail(GCM_ERR_AUTH, "authentication tag mismatch: output zero-filled");
        return GCM_OK;
    }
    if (mem == GCM_MEM_HOST) {
        // Host buffers are streamed through the context's chunk ring.
        gcm_msg m;
        m.key = key;
        m.key_len = key_len;
        m.iv = iv;
        m.iv_len = iv_len;
        m.aad = aad;
        m.aad_len = aad_len;
        m.in = in;
        m.out = out;
        m.len = len;
        m.tag = tag;
        int32_t st = 0;
        rc = stream_host(ctx, &m, 1, decrypt, &st);
        if (rc) return rc;
        if (decrypt && st != 0) return fail(GCM_ERR_AUTH, "authentication tag mismatch: output zero-filled");
        return GCM_OK;
    }
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(GCM_ERR_CUDA, "cannot select the context's device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // Per-call device buffers: status word, and in host mode the staged data.
    const bool host = (mem == GCM_MEM_HOST);
    const size_t off_status = 0;
    const size_t off_tag = 256;
    const size_t off_aad = 512;
    const size_t off_data = align_up(off_aad + (host ? aad_len : 0), 256);
    const size_t total = align_up(off_data + (host ? len : 0), 256);
    Scratch io;
    rc = scratch_alloc(ctx, total, s, io);
    if (rc) return rc;
    uint8_t *iob = static_cast<uint8_t *>(io.base);
    int32_t *d_status = reinterpret_cast<int32_t *>(iob + off_status);
    uint32_t *d_sum = datasum ? reinterpret_cast<uint32_t *>(iob + off_status + 128) : nullptr;
    uint8_t *d_tag = host ? iob + off_tag : tag;
    const uint8_t *d_aad = host ? iob + off_aad : aad;
    uint8_t *d_data = host ? iob + off_data : nullptr;
    const uint8_t *d_in = host ? d_data : in;
    uint8_t *d_out = host ? d_data : out;
    cudaError_t e = cudaSuccess;

    if (host) {
        if (aad_len) e = cudaMemcpyAsync(iob + off_aad, aad, aad_len, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && len) e = cudaMemcpyAsync(d_data, in, len, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && decrypt) e = cudaMemcpyAsync(d_tag, tag, 16, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            scratch_free(ctx, io, s);
            return cuda_fail(e, "host-to-device copy");
        }
    }

    if (d_sum) {
        e = cudaMemsetAsync(d_sum, 0, 4, s);
        if (e != cudaSuccess) {
            scratch_free(ctx, io, s);
            return cuda_fail(e, "memset");
        }
    }
    Scratch sc;
    rc = enqueue_device(ctx, key, key_len, iv, iv_len, d_aad, aad_len, d_in, len, d_out, d_tag, decrypt,
                        d_status, sc, s, 0, d_sum);
    if (rc) {
        if (sc.base) scratch_free(ctx, sc, s);
        scratch_free(ctx, io, s);
        return rc;
    }
    scratch_free(ctx, sc, s);

    if (host) {
        if (len) e = cudaMemcpyAsync(out, d_data, len, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && !decrypt) e = cudaMemcpyAsync(tag, d_tag, 16, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) {
            scratch_free(ctx, io, s);
            return cuda_fail(e, "device-to-host copy");
        }
    }
    int32_t status = 0;
    uint32_t hsum = 0;
    if (d_sum) e = cudaMemcpyAsync(&hsum, d_sum, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && decrypt) {
        e = cudaMemcpyAsync(&status, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    } else if (e == cudaSuccess && (host || d_sum)) {
        e = cudaStreamSynchronize(s);
    }
    scratch_free(ctx, io, s);
    if (e != cudaSuccess) return cuda_fail(e, "synchronisation");
    if (d_sum) {
        *datasum = hsum;
        if (datasum_done) *datasum_done = true;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "asynchronous kernel error");
    if (decrypt && status != 0) return fail(GCM_ERR_AUTH, "authentication tag mismatch: output zero-filled");
    return GCM_OK;
}

}  // namespace

namespace gcmgpu {
int ctx_fail(int code, const char *msg) { return fail(code, "%s", msg); }
int ctx_run_with_datasum(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *iv, size_t iv_len,
                         const uint8_t *aad, size_t aad_len, const uint8_t *in, size_t len, uint8_t *out,
                         uint8_t *tag, bool decrypt, int mem, void *stream, uint32_t *datasum, bool *datasum_done)
{
    return run_call(ctx, key, key_len, iv, iv_len, aad, aad_len, in, len, out, tag, decrypt, mem, stream, datasum,
                    datasum_done);
}
int ctx_cuda_fail(cudaError_t e, const char *where) { return cuda_fail(e, where); }
uint32_t choose_tile_log2(uint64_t M, int num_sms) { return tile_log2_for(M, num_sms); }
cudaEvent_t ctx_take_event(gcm_ctx *ctx)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    return take_event(ctx);
}
void ctx_record_fused(gcm_ctx *ctx, cudaEvent_t start, cudaEvent_t stop, uint64_t bytes)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->timed.push_back({start, stop, bytes});
}
}  // namespace gcmgpu

extern "C" {

const char *gcm_last_error(void) { return g_last_error.c_str(); }

int gcm_ctx_create(gcm_ctx **out, int device, size_t hbm_budget_bytes)
{
    if (!out) return fail(GCM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(GCM_ERR_INVALID_ARG, "no such CUDA device");
    DeviceGuard guard(device);
    if (!guard.ok) return fail(GCM_ERR_CUDA, "cannot select the device");
    gcm_ctx *ctx = new gcm_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        int pageable = 0;
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device);
        ctx->host_direct = pageable != 0;
    }
    if (e == cudaSuccess) e = configure_kernels();
    if (e == cudaSuccess) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        e = cudaMemPoolCreate(&ctx->pool, &props);
    }
    if (e == cudaSuccess) {
        uint64_t keep = UINT64_MAX;  // keep freed scratch cached for later calls
        e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) {
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
        if (major == 10 && minor == 3 && ctx->num_sms == 152) memcpy(ctx->tuned_lg, kTunedGB300, sizeof(kTunedGB300));
    }
    if (e == cudaSuccess) e = cudaMalloc(&ctx->tabs, sizeof(DevTables));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->tickets, gcm_ctx::TICKET_SLOTS * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->tickets, 0, gcm_ctx::TICKET_SLOTS * sizeof(uint32_t));
    if (e == cudaSuccess) e = launch_build_tables(ctx->tabs, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "context creation");
        gcm_ctx_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return GCM_OK;
}

int gcm_host_alloc(int device, size_t bytes, void **out)
{
    if (!out) return fail(GCM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (bytes == 0) return fail(GCM_ERR_INVALID_ARG, "bytes must be positive");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(GCM_ERR_INVALID_ARG, "no such CUDA device");
    DeviceGuard guard(device);
    if (!guard.ok) return fail(GCM_ERR_CUDA, "cannot select the device");
    void *p = nullptr;
    e = cudaHostAlloc(&p, bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GCM_ERR_NO_MEMORY, "page-locked host allocation failed");
    }
    *out = p;
    return GCM_OK;
}

int gcm_host_free(void *p)
{
    if (!p) return GCM_OK;
    cudaError_t e = cudaFreeHost(p);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFreeHost");
    return GCM_OK;
}

int gcm_ctx_set_host_access(gcm_ctx *ctx, int mode)
{
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    if (mode < 0 || mode > 2) return fail(GCM_ERR_INVALID_ARG, "mode must be 0 (auto), 1 (direct) or 2 (staged)");
    int pageable = 0;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, ctx->device);
    }
    if (mode == 1 && !pageable) return fail(GCM_ERR_INVALID_ARG, "the device cannot access host memory directly");
    ctx->host_direct = (mode == 2) ? false : (pageable != 0);
    return GCM_OK;
}

int gcm_ctx_set_streaming(gcm_ctx *ctx, size_t chunk_bytes, int n_buffers)
{
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    if (chunk_bytes < ((size_t)16 << 10) || n_buffers < 2 || n_buffers > 64)
        return fail(GCM_ERR_INVALID_ARG, "chunk_bytes must be >= 16 KiB (whole 16 KiB tiles) and n_buffers 2..64");
    std::lock_guard<std::mutex> lk(ctx->stream_mu);
    ctx->chunk_bytes = chunk_bytes / ((size_t)16 << 10) * ((size_t)16 << 10);
    ctx->n_buffers = n_buffers;
    return GCM_OK;
}

int gcm_batch(gcm_ctx *ctx, const gcm_msg *msgs, size_t n, int decrypt, int32_t *status, int mem, void *stream)
{
    gcmgpu::TraceRange trace_("gcm_batch");
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    if (n && !msgs) return fail(GCM_ERR_INVALID_ARG, "msgs is NULL");
    if (mem == GCM_MEM_HOST) {
        bool aligned = true;
        for (size_t i = 0; i < n && aligned; i++)
            aligned = ((((uintptr_t)msgs[i].in) | ((uintptr_t)msgs[i].out)) & 15u) == 0;
        if (ctx->host_direct && aligned) {
            // One persistent launch straight over the host buffers.
            cudaStream_t s = nullptr;
            {
                std::lock_guard<std::mutex> lk(ctx->stream_mu);
                if (!ctx->s_comp) {
                    DeviceGuard g(ctx->device);
                    cudaError_t e = cudaStreamCreateWithFlags(&ctx->s_comp, cudaStreamNonBlocking);
                    if (e != cudaSuccess) return cuda_fail(e, "creating a stream");
                }
                s = ctx->s_comp;
            }
            return batch_device(ctx, msgs, n, decrypt != 0, status, nullptr, s, true);
        }
        return stream_host(ctx, msgs, n, decrypt != 0, status);
    }
    if (mem == GCM_MEM_DEVICE)
        return batch_device(ctx, msgs, n, decrypt != 0, status, nullptr, static_cast<cudaStream_t>(stream));
    return fail(GCM_ERR_INVALID_ARG, "mem must be GCM_MEM_DEVICE or GCM_MEM_HOST");
}

int gcm_batch_timed(gcm_ctx *ctx, const gcm_msg *msgs, size_t n, int decrypt, int32_t *status, uint64_t *done_ns,
                    void *stream)
{
    gcmgpu::TraceRange trace_("gcm_batch_timed");
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    if (n && !msgs) return fail(GCM_ERR_INVALID_ARG, "msgs is NULL");
    return batch_device(ctx, msgs, n, decrypt != 0, status, done_ns, static_cast<cudaStream_t>(stream));
}

int gcm_profile_enable(gcm_ctx *ctx, int enable)
{
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    ctx->profiling = enable ? 1 : 0;
    return GCM_OK;
}

int gcm_profile_read(gcm_ctx *ctx, int reset, double *fused_ms, uint64_t *fused_launches,
                     uint64_t *fused_bytes, uint64_t *launches)
{
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    DeviceGuard guard(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (auto &t : ctx->timed) {
        cudaError_t e = cudaEventSynchronize(t.stop);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.start, t.stop);
        if (e != cudaSuccess) return cuda_fail(e, "reading profile events");
        ctx->fused_ms += ms;
        ctx->fused_launches += 1;
        ctx->fused_bytes += t.bytes;
        ctx->spare.push_back(t.start);
        ctx->spare.push_back(t.stop);
    }
    ctx->timed.clear();
    if (fused_ms) *fused_ms = ctx->fused_ms;
    if (fused_launches) *fused_launches = ctx->fused_launches;
    if (fused_bytes) *fused_bytes = ctx->fused_bytes;
    if (launches) *launches = ctx->launches.load();
    if (reset) {
        ctx->fused_ms = 0.0;
        ctx->fused_launches = 0;
        ctx->fused_bytes = 0;
        ctx->launches = 0;
    }
    return GCM_OK;
}

void gcm_ctx_destroy(gcm_ctx *ctx)
{
    if (!ctx) return;
    {
        DeviceGuard guard(ctx->device);
        cudaDeviceSynchronize();
        for (auto &t : ctx->timed) {
            cudaEventDestroy(t.start);
            cudaEventDestroy(t.stop);
        }
        for (auto e : ctx->spare) cudaEventDestroy(e);
        stream_release(ctx);
        for (auto k : ctx->keys) cudaFree(k);
        for (auto &c : ctx->key_cache) {
            memset(c.key, 0, sizeof(c.key));
            cudaFree(c.km);
            cudaEventDestroy(c.ready);
            for (auto &u : c.uses) cudaEventDestroy(u.second);
        }
        ctx->key_cache.clear();
        if (ctx->tabs) cudaFree(ctx->tabs);
        if (ctx->tickets) cudaFree(ctx->tickets);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    }
    delete ctx;
}

int gcm_ctx_set_key_cache(gcm_ctx *ctx, size_t entries)
{
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    if (entries > 4096) return fail(GCM_ERR_INVALID_ARG, "at most 4096 cached keys");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (entries < ctx->key_cache.size()) {
        for (auto &c : ctx->key_cache)
            if (c.holders) return fail(GCM_ERR_BUSY, "cached keys are in use by calls in flight");
        DeviceGuard guard(ctx->device);
        for (auto &c : ctx->key_cache) {
            cudaEventSynchronize(c.ready);
            for (auto &u : c.uses) cudaEventSynchronize(u.second);
            memset(c.key, 0, sizeof(c.key));
            cudaFree(c.km);
            cudaEventDestroy(c.ready);
            for (auto &u : c.uses) cudaEventDestroy(u.second);
        }
        ctx->key_cache.clear();
    }
    ctx->key_cache_cap = entries;
    return GCM_OK;
}

int gcm_ctx_set_tile_log2(gcm_ctx *ctx, int tile_log2)
{
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    if (tile_log2 != 0 && (tile_log2 < SEGF_MIN_LOG2 || tile_log2 > 16))
        return fail(GCM_ERR_INVALID_ARG, "tile_log2 must be 0 (automatic) or 9..16");
    ctx->forced_tile_log2 = tile_log2;
    return GCM_OK;
}

int gcm_ctx_set_aes_impl(gcm_ctx *ctx, int impl)
{
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    if (impl != GCM_AES_TABLES && impl != GCM_AES_BITSLICED)
        return fail(GCM_ERR_INVALID_ARG, "AES engine must be GCM_AES_TABLES (0) or GCM_AES_BITSLICED (1)");
    ctx->aes_impl = impl;
    return GCM_OK;
}

int gcm_ctx_autotune(gcm_ctx *ctx, size_t key_len, size_t max_bytes, uint8_t *table_out)
{
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    if (key_len != 16 && key_len != 24 && key_len != 32) return fail(GCM_ERR_INVALID_ARG, "key must be 16, 24 or 32 bytes");
    if (max_bytes < ((size_t)16 << 10)) return fail(GCM_ERR_INVALID_ARG, "max_bytes must be at least 16 KiB");
    if (max_bytes > ((size_t)1 << 30)) max_bytes = (size_t)1 << 30;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(GCM_ERR_CUDA, "cannot select the context's device");
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "creating the tuning stream");
    Scratch buf;
    int rc = scratch_alloc(ctx, 2 * max_bytes + 256, s, buf);
    if (rc) {
        cudaStreamDestroy(s);
        return rc;
    }
    uint8_t *in = static_cast<uint8_t *>(buf.base), *out = in + max_bytes, *tag = out + max_bytes;
    e = cudaMemsetAsync(in, 0, max_bytes, s);
    uint8_t key[32], iv[12];
    for (int i = 0; i < 32; i++) key[i] = (uint8_t)(0x5A ^ (17 * i));
    for (int i = 0; i < 12; i++) iv[i] = (uint8_t)(0xC3 ^ (29 * i));
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    const int saved_forced = ctx->forced_tile_log2;
    uint8_t found[64] = {};
    int prev_class = -1;
    uint8_t prev_lg = 0;
    // Sizes 16 KiB, 64 KiB, ... (x4) up to max_bytes; each measured size
    // decides the classes from its own up to the next measured size.
    for (size_t S = (size_t)16 << 10; e == cudaSuccess && rc == GCM_OK && S <= max_bytes; S *= 4) {
        const uint64_t M = S / 16;
        float best = 1e30f;
        uint8_t best_lg = 0;
        for (int lg = SEGF_MIN_LOG2; lg <= 16 && rc == GCM_OK && e == cudaSuccess; lg++) {
            if ((M >> lg) == 0 && lg > SEGF_MIN_LOG2) break;  // one tile already
            ctx->forced_tile_log2 = lg;
            float t_best = 1e30f;
            for (int rep = 0; rep < 4 && rc == GCM_OK && e == cudaSuccess; rep++) {
                Scratch sc;
                e = cudaEventRecord(ev0, s);
                if (e != cudaSuccess) break;
                rc = enqueue_device(ctx, key, key_len, iv, sizeof(iv), nullptr, 0, in, S, out, tag, false, nullptr,
                                    sc, s);
                if (sc.base) scratch_free(ctx, sc, s);
                if (rc) break;
                e = cudaEventRecord(ev1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
                if (rep > 0 && ms < t_best) t_best = ms;  // rep 0 warms up
            }
            if (t_best < best) {
                best = t_best;
                best_lg = (uint8_t)lg;
            }
        }
        const int c = size_class(M);
        if (best_lg) {
            for (int k = prev_class + 1; k <= c && prev_class >= 0; k++) found[k] = prev_lg;
            found[c] = best_lg;
            prev_class = c;
            prev_lg = best_lg;
        }
    }
    for (int k = prev_class + 1; k < 64 && prev_class >= 0; k++) found[k] = prev_lg;
    ctx->forced_tile_log2 = saved_forced;
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    scratch_free(ctx, buf, s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "autotuning");
    memcpy(ctx->tuned_lg, found, sizeof(found));
    if (table_out) memcpy(table_out, found, sizeof(found));
    return GCM_OK;
}

int gcm_ctx_set_tuning(gcm_ctx *ctx, const uint8_t *table)
{
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    uint8_t t[64] = {};
    if (table) {
        for (int i = 0; i < 64; i++) {
            if (table[i] != 0 && (table[i] < SEGF_MIN_LOG2 || table[i] > 16))
                return fail(GCM_ERR_INVALID_ARG, "tuning entries must be 0 or 9..16");
            t[i] = table[i];
        }
    }
    memcpy(ctx->tuned_lg, t, sizeof(t));
    return GCM_OK;
}

int gcm_sync(gcm_ctx *ctx, void *stream)
{
    if (!ctx) return fail(GCM_ERR_INVALID_ARG, "context is NULL");
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(GCM_ERR_CUDA, "cannot select the context's device");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronisation");
    return GCM_OK;
}

int gcm_ctr_xor(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *iv, size_t iv_len,
                const uint8_t *in, size_t len, uint8_t *out, void *stream)
{
    gcmgpu::TraceRange trace_("gcm_ctr_xor");
    static const uint8_t no_tag[1] = {0};
    int rc = check_common(ctx, key, key_len, iv, iv_len, nullptr, 0, in, len, out, no_tag, GCM_MEM_DEVICE);
    if (rc) return rc;
    if (len == 0) return GCM_OK;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(GCM_ERR_CUDA, "cannot select the context's device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc;
    rc = enqueue_device(ctx, key, key_len, iv, iv_len, nullptr, 0, in, len, out, nullptr, false, nullptr, sc, s, 1);
    if (sc.base) scratch_free(ctx, sc, s);
    return rc;
}

int gcm_ghash(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *aad, size_t aad_len,
              const uint8_t *data, size_t len, uint8_t *out16, void *stream)
{
    gcmgpu::TraceRange trace_("gcm_ghash");
    static const uint8_t iv96[12] = {0};  // H does not depend on the IV; J0 is unused
    int rc = check_common(ctx, key, key_len, iv96, sizeof(iv96), aad, aad_len, data, len, data, out16,
                          GCM_MEM_DEVICE);
    if (rc) return rc;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(GCM_ERR_CUDA, "cannot select the context's device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc;
    rc = enqueue_device(ctx, key, key_len, iv96, sizeof(iv96), aad, aad_len, data, len, nullptr, out16, false,
                        nullptr, sc, s, 2);
    if (sc.base) scratch_free(ctx, sc, s);
    return rc;
}

int gcm_encrypt(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *iv, size_t iv_len,
                const uint8_t *aad, size_t aad_len, const uint8_t *pt, size_t len, uint8_t *ct, uint8_t *tag,
                int mem, void *stream)
{
    gcmgpu::TraceRange trace_("gcm_encrypt");
    return run_call(ctx, key, key_len, iv, iv_len, aad, aad_len, pt, len, ct, tag, false, mem, stream);
}

int gcm_decrypt_verify(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *iv, size_t iv_len,
                       const uint8_t *aad, size_t aad_len, const uint8_t *ct, size_t len, const uint8_t *tag,
                       uint8_t *pt, int mem, void *stream)
{
    gcmgpu::TraceRange trace_("gcm_decrypt_verify");
    return run_call(ctx, key, key_len, iv, iv_len, aad, aad_len, ct, len, pt, const_cast<uint8_t *>(tag), true,
                    mem, stream);
}

}  // extern "C"
