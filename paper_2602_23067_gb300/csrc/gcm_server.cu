// gcm_server.cu -- key cache and the continuous-batching request server.
//
// Keys are registered once: their key material (round keys, H, powers of H,
// the GHASH table) is built on the device and kept for later requests.
//
// The server takes encrypt / decrypt-verify requests on host buffers from
// any thread.  Its own thread forms "waves" out of the requests waiting at
// that moment (first come first served, as many as fit the HBM budget and
// the wave size), and runs each wave as: copy-in of payloads, AAD and
// descriptors on a copy stream; J0/E_K(J0) per message, the persistent
// batched kernel (each message with its cached key) and the zero-fill of
// failed decryptions on a compute stream; copy-out of payloads, tags and
// verdicts on a third stream.  Up to `max_inflight` waves are in flight, so
// requests that arrive while others are on the GPU are admitted as soon as
// a slot and memory free up, and their copies overlap the other waves'
// kernels (continuous batching).  Completions carry the request's arrival
// and completion times on the host's monotonic clock.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "gcm_ctx.h"
#include "gcm_internal.h"
#include "gcmgpu.h"

using namespace gcmgpu;

namespace {

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t al(size_t x) { return (x + 255) / 256 * 256; }

struct Pending {
    gcm_request r;
    uint64_t ticket;
    uint64_t t_arrival;
    std::vector<uint8_t> iv;
    uint8_t tag_in[16];
    bool waited = false;  // once held back because the HBM budget was taken
};

struct Wave {
    std::vector<Pending> reqs;
    uint8_t *arena = nullptr;
    size_t arena_bytes = 0;
    uint8_t *stage = nullptr;  // pinned: descriptors out, then tags+status back
    int slot = 0;
    cudaEvent_t done = nullptr;
};

}  // namespace

struct gcm_server;
namespace {
bool is_direct(const gcm_server *S, const gcm_request &r);
}

struct gcm_server {
    gcm_ctx *ctx = nullptr;
    size_t budget = 0;
    size_t max_wave = 0;
    int max_inflight = 0;
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    std::vector<uint8_t *> stages;  // one pinned staging buffer per in-flight slot
    size_t stage_bytes = 0;
    std::vector<cudaEvent_t> ev_start, ev_in, ev_comp, ev_done;
    std::vector<bool> slot_busy;
    // timing of the pipeline stages (summed over waves)
    double t_launch_host_ms = 0, t_in_ms = 0, t_comp_ms = 0, t_out_ms = 0;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> queue;
    size_t queue_cap = 0;
    std::deque<gcm_completion> completions;
    std::atomic<uint64_t> next_ticket{1};
    std::atomic<bool> stop{false};
    std::thread worker;
    size_t bytes_in_flight = 0;
    size_t peak_bytes_in_flight = 0;  // largest bytes_in_flight after an admission
    uint64_t budget_waits = 0;        // requests held back at least once for memory
    std::atomic<uint64_t> waves{0}, launched_msgs{0};
    int fatal = 0;
};

namespace {

bool is_direct(const gcm_server *S, const gcm_request &r)
{
    return S->ctx->host_direct && ((((uintptr_t)r.in) | ((uintptr_t)r.out)) & 15u) == 0;
}

// Whether the kernels work on this request's host buffers in place (the
// device reaches host memory directly and the payload is 16-byte aligned).
bool is_direct(const gcm_server *S, const gcm_request &r);

// Device bytes a request needs inside a wave arena, at most: its tile
// partials are counted at the smallest tile a wave may choose.
size_t request_bytes(const gcm_server *S, const gcm_request &r)
{
    const uint64_t M = (r.aad_len + 15) / 16 + (r.len + 15) / 16;
    uint64_t K = (M + (1ull << SEGF_MIN_LOG2) - 1) >> SEGF_MIN_LOG2;
    if (K == 0) K = 1;
    const size_t data = is_direct(S, r) ? 0 : al(r.len) + al(r.aad_len);
    return data + al(sizeof(MsgMat)) + al(K * sizeof(gf128)) + al((K / 2 + 1) * sizeof(gf128)) +
           al(sizeof(BatchMsg) + sizeof(BatchKey) + 64) + 64;
}

int launch_wave(gcm_server *S, Wave &w)
{
    gcm_ctx *ctx = S->ctx;
    const size_t n = w.reqs.size();
    // Arena layout: descriptors | keys | ivs | counters | status | tags | per message scratch | payloads | aads
    size_t off = 0;
    const size_t o_msgs = off;
    off = al(off + n * sizeof(BatchMsg));
    const size_t o_keys = off;
    off = al(off + n * sizeof(BatchKey));
    const size_t o_ivs = off;
    std::vector<size_t> o_iv(n);
    size_t ivt = 0;
    for (size_t i = 0; i < n; i++) {
        o_iv[i] = ivt;
        ivt += w.reqs[i].iv.size();
    }
    off = al(off + ivt);
    const size_t o_exp = off;  // expected tags (decrypt)
    off = al(off + 16 * n);
    const size_t host_bytes = off;
    const size_t o_done = off;
    off = al(off + 4 * n);
    const size_t o_ctr = off;
    off = al(off + 8);
    const size_t o_ret = off;  // returned: 16-byte tag + 16 bytes (status) per message
    off = al(off + 32 * n);
    const size_t zero_bytes = off - o_done;
    std::vector<size_t> o_mm(n), o_part(n), o_tree(n), o_pay(n), o_aad(n);
    std::vector<uint64_t> K(n), base(n);
    // One tile size for the wave: the largest that gives every SM four tiles'
    // worth of its blocks, so a light wave spreads over the SMs.
    uint64_t total = 0;
    for (size_t i = 0; i < n; i++) total += (w.reqs[i].r.aad_len + 15) / 16 + (w.reqs[i].r.len + 15) / 16;
    const uint32_t lg = ctx->forced_tile_log2 ? (uint32_t)ctx->forced_tile_log2 : choose_tile_log2(total, ctx->num_sms);
    uint64_t items = 0;
    for (size_t i = 0; i < n; i++) {
        const gcm_request &r = w.reqs[i].r;
        const uint64_t M = (r.aad_len + 15) / 16 + (r.len + 15) / 16;
        uint64_t k = (M + (1ull << lg) - 1) >> lg;
        if (k == 0) k = 1;
        K[i] = k;
        base[i] = items;
        items += k;
        o_mm[i] = off;
        off = al(off + sizeof(MsgMat));
        o_part[i] = off;
        off = al(off + k * sizeof(gf128));
        o_tree[i] = off;
        off = al(off + (k / 2 + 1) * sizeof(gf128));
        if (!is_direct(S, r)) {
            o_pay[i] = off;
            off = al(off + r.len);
            o_aad[i] = off;
            off = al(off + r.aad_len);
        }
    }
    w.arena_bytes = off;
    cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&w.arena), off, ctx->pool, S->s_in);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GCM_ERR_NO_MEMORY;
    }
    uint8_t *dev = w.arena;
    uint8_t *st = w.stage;
    BatchMsg *hm = reinterpret_cast<BatchMsg *>(st + o_msgs);
    BatchKey *hk = reinterpret_cast<BatchKey *>(st + o_keys);
    for (size_t i = 0; i < n; i++) {
        const Pending &p = w.reqs[i];
        const gcm_request &r = p.r;
        const KeyMat *km = ctx->keys[r.key];
        BatchMsg &b = hm[i];
        memset(&b, 0, sizeof(b));
        if (is_direct(S, r)) {
            b.in = r.in;
            b.out = r.out;
            b.aad = r.aad;
        } else {
            b.in = dev + o_pay[i];
            b.out = dev + o_pay[i];
            b.aad = dev + o_aad[i];
        }
        b.len = r.len;
        b.aad_len = r.aad_len;
        b.tile_log2 = lg;
        b.K = K[i];
        b.item_base = base[i];
        b.nr = ctx->key_nr[r.key];
        b.dec = r.op ? 1u : 0u;
        b.km = const_cast<KeyMat *>(km);
        b.mm = reinterpret_cast<MsgMat *>(dev + o_mm[i]);
        b.partials = reinterpret_cast<gf128 *>(dev + o_part[i]);
        b.tree = reinterpret_cast<gf128 *>(dev + o_tree[i]);
        b.tag = r.op ? dev + o_exp + 16 * i : dev + o_ret + 32 * i;
        b.status = reinterpret_cast<int32_t *>(dev + o_ret + 32 * i + 16);
        b.t_done = nullptr;
        BatchKey &k = hk[i];
        memset(&k, 0, sizeof(k));
        k.iv_len = (uint32_t)p.iv.size();
        k.iv = dev + o_ivs + o_iv[i];
        memcpy(st + o_ivs + o_iv[i], p.iv.data(), p.iv.size());
        memcpy(st + o_exp + 16 * i, p.tag_in, 16);
    }
    // Copy-in stream: descriptors, payloads, AADs.
    cudaEventRecord(S->ev_start[w.slot], S->s_in);
    e = cudaMemcpyAsync(dev, st, host_bytes, cudaMemcpyHostToDevice, S->s_in);
    for (size_t i = 0; i < n && e == cudaSuccess; i++) {
        const gcm_request &r = w.reqs[i].r;
        if (is_direct(S, r)) continue;
        if (r.len) e = cudaMemcpyAsync(dev + o_pay[i], r.in, r.len, cudaMemcpyHostToDevice, S->s_in);
        if (e == cudaSuccess && r.aad_len) e = cudaMemcpyAsync(dev + o_aad[i], r.aad, r.aad_len, cudaMemcpyHostToDevice, S->s_in);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(dev + o_done, 0, zero_bytes, S->s_in);
    if (e == cudaSuccess) e = cudaEventRecord(S->ev_in[w.slot], S->s_in);
    // Compute stream.
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->s_comp, S->ev_in[w.slot], 0);
    const BatchMsg *dmsgs = reinterpret_cast<const BatchMsg *>(dev + o_msgs);
    if (e == cudaSuccess)
        e = launch_msg_setup(dmsgs, reinterpret_cast<const BatchKey *>(dev + o_keys), (uint32_t)n, ctx->tabs, S->s_comp);
    BatchParams bp;
    memset(&bp, 0, sizeof(bp));
    bp.msgs = dmsgs;
    bp.n = (uint32_t)n;
    bp.total_items = items;
    bp.item_counter = reinterpret_cast<unsigned long long *>(dev + o_ctr);
    bp.done = reinterpret_cast<uint32_t *>(dev + o_done);
    bp.tabs = ctx->tabs;
    if (e == cudaSuccess) e = launch_batch(bp, ctx->num_sms, S->s_comp);
    bool any_dec = false;
    for (auto &p : w.reqs) any_dec |= (p.r.op != 0);
    if (e == cudaSuccess && any_dec) e = launch_batch_zero(dmsgs, (uint32_t)n, S->s_comp);
    ctx->launches += any_dec ? 3 : 2;
    if (e == cudaSuccess) e = cudaEventRecord(S->ev_comp[w.slot], S->s_comp);
    // Copy-out stream.
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->s_out, S->ev_comp[w.slot], 0);
    for (size_t i = 0; i < n && e == cudaSuccess; i++) {
        const gcm_request &r = w.reqs[i].r;
        if (is_direct(S, r)) continue;
        if (r.len) e = cudaMemcpyAsync(r.out, dev + o_pay[i], r.len, cudaMemcpyDeviceToHost, S->s_out);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(st + host_bytes, dev + o_ret, 32 * n, cudaMemcpyDeviceToHost, S->s_out);
    if (e == cudaSuccess) e = cudaFreeAsync(dev, S->s_out);
    if (e == cudaSuccess) e = cudaEventRecord(w.done, S->s_out);
    return e == cudaSuccess ? GCM_OK : GCM_ERR_CUDA;
}

void finish_wave(gcm_server *S, Wave &w)
{
    const size_t n = w.reqs.size();
    // The returned block sits right after the descriptors in the staging buffer.
    size_t host_bytes = al(n * sizeof(BatchMsg)) + al(n * sizeof(BatchKey));
    size_t ivt = 0;
    for (auto &p : w.reqs) ivt += p.iv.size();
    host_bytes = al(host_bytes + ivt);
    host_bytes = al(host_bytes + 16 * n);
    const uint8_t *ret = w.stage + host_bytes;
    const uint64_t t = now_ns();
    float a = 0, b = 0, c = 0;
    cudaEventElapsedTime(&a, S->ev_start[w.slot], S->ev_in[w.slot]);
    cudaEventElapsedTime(&b, S->ev_in[w.slot], S->ev_comp[w.slot]);
    cudaEventElapsedTime(&c, S->ev_comp[w.slot], w.done);
    std::lock_guard<std::mutex> lk(S->mu);
    S->t_in_ms += a;
    S->t_comp_ms += b;
    S->t_out_ms += c;
    for (size_t i = 0; i < n; i++) {
        const Pending &p = w.reqs[i];
        int32_t status;
        memcpy(&status, ret + 32 * i + 16, 4);
        if (p.r.op == 0) {
            if (p.r.tag) memcpy(p.r.tag, ret + 32 * i, 16);
            status = 0;
        } else {
            status = status ? GCM_ERR_AUTH : 0;
        }
        gcm_completion c;
        c.ticket = p.ticket;
        c.status = status;
        c.arrival_ns = p.t_arrival;
        c.complete_ns = t;
        c.user = p.r.user;
        S->completions.push_back(c);
        S->bytes_in_flight -= request_bytes(S, p.r);
    }
    S->slot_busy[w.slot] = false;
}

void worker_loop(gcm_server *S)
{
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->ctx->device);
    std::deque<Wave> inflight;
    std::deque<Pending> pending;
    while (true) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (pending.empty() && inflight.empty() && S->queue.empty() && !S->stop.load())
                S->cv.wait_for(lk, std::chrono::microseconds(200));
            while (!S->queue.empty()) {
                pending.push_back(std::move(S->queue.front()));
                S->queue.pop_front();
            }
            if (S->stop.load() && pending.empty() && inflight.empty()) break;
        }
        // Retire finished waves in order.
        while (!inflight.empty() && cudaEventQuery(inflight.front().done) == cudaSuccess) {
            finish_wave(S, inflight.front());
            inflight.pop_front();
        }
        // Admit new waves while there is a free slot.
        while (!pending.empty() && (int)inflight.size() < S->max_inflight) {
            int slot = -1;
            for (int i = 0; i < S->max_inflight; i++)
                if (!S->slot_busy[i]) {
                    slot = i;
                    break;
                }
            if (slot < 0) break;
            Wave w;
            size_t wave_bytes = 0, n = 0;
            size_t avail;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                avail = S->budget > S->bytes_in_flight ? S->budget - S->bytes_in_flight : 0;
            }
            size_t ivt = 0;
            while (n < pending.size() && n < S->max_wave) {
                const size_t b = request_bytes(S, pending[n].r);
                const size_t m = n + 1, iv2 = ivt + pending[n].iv.size();
                const size_t sn = al(m * sizeof(BatchMsg)) + al(m * sizeof(BatchKey)) + al(iv2) + al(16 * m) + 32 * m;
                if (wave_bytes + b > avail) {
                    // Held back until waves in flight release their memory.
                    if (!pending[n].waited) {
                        pending[n].waited = true;
                        std::lock_guard<std::mutex> lk(S->mu);
                        S->budget_waits++;
                    }
                    break;
                }
                if (sn > S->stage_bytes) break;
                wave_bytes += b;
                ivt = iv2;
                n++;
            }
            if (n == 0) break;  // wait for memory to free up
            for (size_t i = 0; i < n; i++) {
                w.reqs.push_back(std::move(pending.front()));
                pending.pop_front();
            }
            w.slot = slot;
            w.stage = S->stages[slot];
            w.done = S->ev_done[slot];
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->bytes_in_flight += wave_bytes;
                if (S->bytes_in_flight > S->peak_bytes_in_flight) S->peak_bytes_in_flight = S->bytes_in_flight;
                S->slot_busy[slot] = true;
            }
            const uint64_t th0 = now_ns();
            int lrc;
            {
                gcmgpu::TraceRange trace_("gcm_server wave launch");
                lrc = launch_wave(S, w);
            }
            S->t_launch_host_ms += (now_ns() - th0) / 1e6;
            if (lrc != GCM_OK) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->fatal = GCM_ERR_CUDA;
                for (auto &p : w.reqs) {
                    gcm_completion c;
                    c.ticket = p.ticket;
                    c.status = GCM_ERR_CUDA;
                    c.arrival_ns = p.t_arrival;
                    c.complete_ns = now_ns();
                    c.user = p.r.user;
                    S->completions.push_back(c);
                    S->bytes_in_flight -= request_bytes(S, p.r);
                }
                S->slot_busy[slot] = false;
                continue;
            }
            S->waves++;
            S->launched_msgs += n;
            inflight.push_back(std::move(w));
        }
        if (!inflight.empty()) {
            // Poll the oldest wave without burning a whole core.
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
}

}  // namespace

extern "C" {

uint64_t gcm_now_ns(void) { return now_ns(); }

int gcm_key_register(gcm_ctx *ctx, const uint8_t *key, size_t key_len, uint32_t *handle)
{
    if (!ctx || !handle) return ctx_fail(GCM_ERR_INVALID_ARG, "context or handle is NULL");
    if (!key || (key_len != 16 && key_len != 24 && key_len != 32))
        return ctx_fail(GCM_ERR_INVALID_ARG, "key must be 16, 24 or 32 bytes");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    KeyMat *km = nullptr;
    MsgMat *mm = nullptr;
    cudaError_t e = cudaMalloc(&km, sizeof(KeyMat));
    if (e == cudaSuccess) e = cudaMalloc(&mm, sizeof(MsgMat));
    if (e == cudaSuccess) {
        KsParams ks;
        memset(&ks, 0, sizeof(ks));
        memcpy(ks.key, key, key_len);
        ks.key_len = (uint32_t)key_len;
        ks.iv_len = 12;  // any IV: only the key material is kept
        ks.km = km;
        ks.mm = mm;
        ks.tabs = ctx->tabs;
        e = launch_key_setup(ks, nullptr);
        if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    }
    if (mm) cudaFree(mm);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        if (km) cudaFree(km);
        cudaGetLastError();
        return ctx_cuda_fail(e, "registering a key");
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->keys.push_back(km);
    ctx->key_nr.push_back((uint32_t)key_len / 4 + 6);
    *handle = (uint32_t)(ctx->keys.size() - 1);
    return GCM_OK;
}

int gcm_server_create(gcm_ctx *ctx, size_t hbm_budget_bytes, size_t max_wave_msgs, int max_inflight,
                      gcm_server **out)
{
    if (!ctx || !out) return ctx_fail(GCM_ERR_INVALID_ARG, "context or out is NULL");
    *out = nullptr;
    if (max_wave_msgs == 0 || max_inflight < 1 || max_inflight > 8)
        return ctx_fail(GCM_ERR_INVALID_ARG, "max_wave_msgs >= 1 and 1 <= max_inflight <= 8");
    gcm_server *S = new gcm_server();
    S->ctx = ctx;
    S->budget = hbm_budget_bytes ? hbm_budget_bytes : ((size_t)40 << 30);
    S->max_wave = max_wave_msgs;
    S->max_inflight = max_inflight;
    S->queue_cap = 1u << 20;
    S->stage_bytes = max_wave_msgs * (sizeof(BatchMsg) + sizeof(BatchKey) + 16 + 32 + 512) + 65536 + (1u << 20);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamCreateWithFlags(&S->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_comp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_out, cudaStreamNonBlocking);
    for (int i = 0; i < max_inflight && e == cudaSuccess; i++) {
        uint8_t *st = nullptr;
        e = cudaMallocHost(reinterpret_cast<void **>(&st), S->stage_bytes);
        if (e != cudaSuccess) break;
        S->stages.push_back(st);
        cudaEvent_t a, b, c, d;
        e = cudaEventCreate(&a);
        if (e == cudaSuccess) e = cudaEventCreate(&b);
        if (e == cudaSuccess) e = cudaEventCreate(&c);
        if (e == cudaSuccess) e = cudaEventCreate(&d);
        S->ev_start.push_back(d);
        S->ev_in.push_back(a);
        S->ev_comp.push_back(b);
        S->ev_done.push_back(c);
        S->slot_busy.push_back(false);
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        gcm_server_destroy(S);
        return ctx_cuda_fail(e, "creating the server");
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return GCM_OK;
}

int gcm_server_submit(gcm_server *S, const gcm_request *r, uint64_t *ticket)
{
    if (!S || !r) return ctx_fail(GCM_ERR_INVALID_ARG, "server or request is NULL");
    if (r->op != 0 && r->op != 1) return ctx_fail(GCM_ERR_INVALID_ARG, "op must be 0 (encrypt) or 1 (decrypt-verify)");
    if (r->key >= S->ctx->keys.size()) return ctx_fail(GCM_ERR_INVALID_ARG, "unknown key handle");
    if (!r->iv || r->iv_len == 0 || r->iv_len > 65536) return ctx_fail(GCM_ERR_INVALID_ARG, "IV must be 1..65536 bytes");
    if (r->len > (1ull << 36) - 32) return ctx_fail(GCM_ERR_LENGTH_LIMIT, "payload too long");
    if (r->len && (!r->in || !r->out)) return ctx_fail(GCM_ERR_INVALID_ARG, "payload pointer is NULL");
    if (r->aad_len && !r->aad) return ctx_fail(GCM_ERR_INVALID_ARG, "aad is NULL with a nonzero length");
    if (!r->tag) return ctx_fail(GCM_ERR_INVALID_ARG, "tag pointer is NULL");
    if (request_bytes(S, *r) > S->budget) return ctx_fail(GCM_ERR_NO_MEMORY, "request larger than the server's HBM budget");
    Pending p;
    p.r = *r;
    p.t_arrival = r->arrival_ns ? r->arrival_ns : now_ns();
    p.iv.assign(r->iv, r->iv + r->iv_len);
    if (r->op == 1) memcpy(p.tag_in, r->tag, 16);
    else memset(p.tag_in, 0, 16);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->queue.size() >= S->queue_cap) return ctx_fail(GCM_ERR_BUSY, "server queue full");
        p.ticket = S->next_ticket++;
        if (ticket) *ticket = p.ticket;
        S->queue.push_back(std::move(p));
    }
    S->cv.notify_one();
    return GCM_OK;
}

int gcm_server_submit_batch(gcm_server *S, const gcm_request *reqs, size_t n, uint64_t *first_ticket)
{
    if (!S || (n && !reqs)) return ctx_fail(GCM_ERR_INVALID_ARG, "server or requests are NULL");
    std::vector<Pending> ps(n);
    for (size_t i = 0; i < n; i++) {
        const gcm_request *r = &reqs[i];
        if (r->op != 0 && r->op != 1) return ctx_fail(GCM_ERR_INVALID_ARG, "op must be 0 (encrypt) or 1 (decrypt-verify)");
        if (r->key >= S->ctx->keys.size()) return ctx_fail(GCM_ERR_INVALID_ARG, "unknown key handle");
        if (!r->iv || r->iv_len == 0 || r->iv_len > 65536) return ctx_fail(GCM_ERR_INVALID_ARG, "IV must be 1..65536 bytes");
        if (r->len > (1ull << 36) - 32) return ctx_fail(GCM_ERR_LENGTH_LIMIT, "payload too long");
        if (r->len && (!r->in || !r->out)) return ctx_fail(GCM_ERR_INVALID_ARG, "payload pointer is NULL");
        if (r->aad_len && !r->aad) return ctx_fail(GCM_ERR_INVALID_ARG, "aad is NULL with a nonzero length");
        if (!r->tag) return ctx_fail(GCM_ERR_INVALID_ARG, "tag pointer is NULL");
        if (request_bytes(S, *r) > S->budget) return ctx_fail(GCM_ERR_NO_MEMORY, "request larger than the server's HBM budget");
        Pending &p = ps[i];
        p.r = *r;
        p.t_arrival = r->arrival_ns ? r->arrival_ns : now_ns();
        p.iv.assign(r->iv, r->iv + r->iv_len);
        if (r->op == 1) memcpy(p.tag_in, r->tag, 16);
        else memset(p.tag_in, 0, 16);
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->queue.size() + n > S->queue_cap) return ctx_fail(GCM_ERR_BUSY, "server queue full");
        if (first_ticket) *first_ticket = S->next_ticket.load();
        for (size_t i = 0; i < n; i++) {
            ps[i].ticket = S->next_ticket++;
            S->queue.push_back(std::move(ps[i]));
        }
    }
    S->cv.notify_one();
    return GCM_OK;
}

size_t gcm_server_poll(gcm_server *S, gcm_completion *out, size_t max)
{
    if (!S || !out) return 0;
    std::lock_guard<std::mutex> lk(S->mu);
    size_t n = 0;
    while (n < max && !S->completions.empty()) {
        out[n++] = S->completions.front();
        S->completions.pop_front();
    }
    return n;
}

int gcm_server_stats(gcm_server *S, uint64_t *waves, uint64_t *messages, size_t *queued, size_t *bytes_in_flight)
{
    if (!S) return ctx_fail(GCM_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    if (waves) *waves = S->waves.load();
    if (messages) *messages = S->launched_msgs.load();
    if (queued) *queued = S->queue.size();
    if (bytes_in_flight) *bytes_in_flight = S->bytes_in_flight;
    return S->fatal;
}

int gcm_server_admission(gcm_server *S, size_t *budget, size_t *peak_bytes_in_flight, uint64_t *budget_waits)
{
    if (!S) return ctx_fail(GCM_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    if (budget) *budget = S->budget;
    if (peak_bytes_in_flight) *peak_bytes_in_flight = S->peak_bytes_in_flight;
    if (budget_waits) *budget_waits = S->budget_waits;
    return GCM_OK;
}

int gcm_server_timing(gcm_server *S, double out[4])
{
    if (!S || !out) return ctx_fail(GCM_ERR_INVALID_ARG, "server or out is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    out[0] = S->t_launch_host_ms;
    out[1] = S->t_in_ms;
    out[2] = S->t_comp_ms;
    out[3] = S->t_out_ms;
    return GCM_OK;
}

void gcm_server_destroy(gcm_server *S)
{
    if (!S) return;
    S->stop = true;
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->ctx->device);
    if (S->s_in) cudaStreamSynchronize(S->s_in);
    if (S->s_comp) cudaStreamSynchronize(S->s_comp);
    if (S->s_out) cudaStreamSynchronize(S->s_out);
    for (auto p : S->stages) cudaFreeHost(p);
    for (auto e : S->ev_start) cudaEventDestroy(e);
    for (auto e : S->ev_in) cudaEventDestroy(e);
    for (auto e : S->ev_comp) cudaEventDestroy(e);
    for (auto e : S->ev_done) cudaEventDestroy(e);
    if (S->s_in) cudaStreamDestroy(S->s_in);
    if (S->s_comp) cudaStreamDestroy(S->s_comp);
    if (S->s_out) cudaStreamDestroy(S->s_out);
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
}

}  // extern "C"
