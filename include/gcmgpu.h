/*
 * gcmgpu.h -- C ABI of the GB300 AES-GCM library.
 *
 * The library implements AES-GCM authenticated encryption and decryption
 * (NIST SP 800-38D over the FIPS-197 block cipher) as adopted by the paper
 * "GpuFitsCrypt" (Sec. 3.2.1): the AES-CTR keystream fused, in one pass over
 * the data, with GHASH recast as the paper's parallel reduction (Sec. 3.3.1,
 * Eq. 1 and Fig. 3b; Sec. 5.2.1-5.2.3): per-chunk Horner, a device table of
 * powers of H, and a log-depth combination of chunk partials.  The session
 * object mirrors the paper's context API (Table "Core functions",
 * gfc_context_create / gfc_context_destroy) and the FITS entry points follow
 * its FitsOperationResult convention (same table).
 *
 * Conventions that hold for every call below:
 *   - Every function declared to return int returns a gcm_status (0 =
 *     success, negative = error); the others say what they return.  The
 *     message of the last error on the calling thread is available from
 *     gcm_last_error().
 *   - key and iv are always HOST pointers; the library copies them.
 *   - Buffers named "data" (aad, pt, ct, tag) are DEVICE pointers when
 *     mem == GCM_MEM_DEVICE and HOST pointers when mem == GCM_MEM_HOST.
 *     Device data buffers for pt/ct must be 16-byte aligned; aad and tag
 *     buffers have no alignment requirement.
 *   - The caller owns all buffers it passes.  ct may equal pt (in place).
 *   - stream is a cudaStream_t (NULL = the legacy default stream).  Device
 *     mode encryption is asynchronous on that stream; the tag is valid once
 *     the stream reaches the point of the call.
 *   - A length of zero is valid for aad and for the payload.  A NULL
 *     pointer is accepted only together with a zero length.
 *   - Limits (SP 800-38D sec. 5.2.1.1): payload <= 2^36 - 32 bytes, aad <=
 *     2^61 - 1 bytes.  IVs must be 1..65536 bytes (the standard allows
 *     longer IVs; this library caps them and reports GCM_ERR_LENGTH_LIMIT).
 */
#ifndef GCMGPU_H
#define GCMGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- */
/* Status codes (the paper's convention: 0 success, < 0 error;      */
/* Table "Core functions", error_code row)                          */
/* ---------------------------------------------------------------- */
typedef enum {
    GCM_OK = 0,
    GCM_ERR_INVALID_ARG = -1,   /* bad key/IV length, NULL with nonzero length, bad mode */
    GCM_ERR_LENGTH_LIMIT = -2,  /* payload, AAD or IV beyond the limits above */
    GCM_ERR_AUTH = -3,          /* tag mismatch: the output was zero-filled (Sec. 4.2) */
    GCM_ERR_NO_MEMORY = -4,     /* device/pinned allocation failed or HBM budget exceeded */
    GCM_ERR_CUDA = -5,          /* a CUDA runtime call failed */
    GCM_ERR_TIMEOUT = -6,       /* a bounded device-side wait gave up */
    GCM_ERR_ALIGNMENT = -7,     /* a device pt/ct pointer is not 16-byte aligned */
    GCM_ERR_BUSY = -8           /* serving queue full, or a run in flight; retry later */
} gcm_status;

/* Where the data buffers of a call live. */
typedef enum {
    GCM_MEM_DEVICE = 0,
    GCM_MEM_HOST = 1
} gcm_mem;

/* Opaque session: device scratch pools, streams, the key cache and the HBM
 * budget.  One context serves one device.  Calls on one context may come
 * from several host threads at once, each on its own stream: the key cache,
 * the scratch accounting and the profiling state are guarded inside the
 * context, and per-call scratch is stream-ordered.  Changing a setting
 * (gcm_ctx_set_*) while calls are in flight is not supported, except as
 * gcm_ctx_set_key_cache documents. */
typedef struct gcm_ctx gcm_ctx;

/* Creates a session on CUDA device `device`.  hbm_budget_bytes caps the
 * device scratch the session may hold (0 = no cap).  Builds the AES round
 * tables on the device.  *out receives the context; it is NULL on error.
 * Mirrors gfc_context_create (Table "Core functions"). */
int gcm_ctx_create(gcm_ctx **out, int device, size_t hbm_budget_bytes);

/* Releases every device and host resource of the session (mirrors
 * gfc_context_destroy).  Waits for the session's own streams.  NULL is a
 * no-op. */
void gcm_ctx_destroy(gcm_ctx *ctx);

/* Message of the last error seen on the calling thread ("" if none). */
const char *gcm_last_error(void);

/* GCM-AE (SP 800-38D Algorithm 4; the paper's AES-GCM, Sec. 3.2.1).
 *   key/key_len : 16 or 32 bytes (AES-128 / AES-256), 24 (AES-192) also works.
 *   iv/iv_len   : 12 bytes is the fast path J0 = IV || 0^31 || 1; any other
 *                 length uses J0 = GHASH(IV || pad || [len(IV)]_64).
 *   aad/aad_len : additional authenticated data (e.g. a FITS header).
 *   pt/len      : plaintext;  ct receives len bytes of ciphertext.
 *   tag         : receives the 16-byte tag T = E_K(J0) xor GHASH_H(A, C).
 * Device mode: returns once the work is enqueued on `stream`.
 * Host mode:   returns when done.  Where the device reads host memory
 *              directly (gcm_ctx_set_host_access) and pt/ct are 16-byte
 *              aligned, the kernels run on the host buffers on `stream`;
 *              otherwise the buffers stream through the context's device
 *              chunk buffers (see gcm_batch) and `stream` is not used. */
int gcm_encrypt(gcm_ctx *ctx, const uint8_t *key, size_t key_len,
                const uint8_t *iv, size_t iv_len,
                const uint8_t *aad, size_t aad_len,
                const uint8_t *pt, size_t len, uint8_t *ct, uint8_t *tag,
                int mem, void *stream);

/* GCM-AD (SP 800-38D Algorithm 5) with the paper's validation gate
 * (Sec. 3.3.2 item 4): the GHASH is taken over the input ciphertext in the
 * same pass that writes the plaintext; the tag is then compared in constant
 * time and, on a mismatch, the plaintext buffer is zero-filled on the device
 * (the payload suppression of Sec. 4.2) before the call returns
 * GCM_ERR_AUTH.  The call synchronises `stream` to read the verdict.
 * `tag` holds the 16 expected tag bytes (a device pointer in device mode). */
int gcm_decrypt_verify(gcm_ctx *ctx, const uint8_t *key, size_t key_len,
                       const uint8_t *iv, size_t iv_len,
                       const uint8_t *aad, size_t aad_len,
                       const uint8_t *ct, size_t len, const uint8_t *tag,
                       uint8_t *pt, int mem, void *stream);

/* Sets how many keys the session keeps set up on the device for
 * gcm_encrypt / gcm_decrypt_verify / gcm_ctr_xor / gcm_ghash (default 64;
 * 0 disables the cache).  A call whose key is cached skips the key setup
 * (round keys, H and its power tables, the weights of the reduce that
 * finishes messages of at most 1024 tiles inside the fused launch:
 * 75.4 KiB per key) and only derives
 * J0 and E_K(J0) for its IV; a new key replaces the least recently used entry
 * that no call in flight still reads.  The cache holds key material on the
 * device and the key bytes in host memory until the entry is replaced, the
 * cache is shrunk, or the context is destroyed (the bytes are zeroed then).
 * Shrinking waits for the cached entries' last uses; it returns
 * GCM_ERR_BUSY if another thread's call holds an entry at that moment.  No
 * counterpart in the paper, which sets up the key per call. */
int gcm_ctx_set_key_cache(gcm_ctx *ctx, size_t entries);

/* Tile size of the single-message calls.  The fused pass splits the GHASH
 * input sequence A || C into tiles of 2^t 16-byte blocks (the paper's chunks,
 * Sec. 5.2.2 map phase); any t gives the same ciphertext and tag.  By
 * default t comes from the context's tuning table (on a GB300 with 152 SMs a
 * table measured there with gcm_ctx_autotune is installed at creation),
 * else from a rule (t = 16, lowered down to 9 while there are fewer than 4
 * tiles per SM).  A batch (gcm_batch, a batch plan, a server wave) uses one
 * t for all its messages, from the batch's total blocks: in device memory
 * the t that balances a tile's fixed work against the tail of the last
 * tiles, for host memory and the server the rule above.
 * gcm_ctx_set_tile_log2 forces t = tile_log2 (9..16) for every call and
 * every batch or plan created afterwards; 0 returns to the default. */
int gcm_ctx_set_tile_log2(gcm_ctx *ctx, int tile_log2);

/* AES engine of the single-message device pass (gcm_encrypt,
 * gcm_decrypt_verify, gcm_ctr_xor, the FITS calls).  The paper builds on a
 * bit-sliced AES-CTR core (Sec. 5.2, citing Lee et al. 2024); this library
 * defaults to round tables in shared memory and offers the bit-sliced form:
 *   GCM_AES_TABLES    (0, default) T-table rounds, one block per lane, with
 *                     counter-mode caching of rounds 1-2;
 *   GCM_AES_BITSLICED (1) 32 counter blocks per thread as 128 bitsliced words
 *                     (the S-box as a 129-gate AND/XOR circuit derived from
 *                     the tower field GF(((2^2)^2)^2)), 256 threads per SM.
 * Ciphertexts and tags are identical; only speed differs.  GHASH uses the
 * same shared-memory table in both.  Segments that touch the AAD or a final
 * partial block, the GHASH-only pass, gcm_batch, the staged host-memory
 * pipeline and gcm_encrypt_noalloc always use the tables.
 * Returns GCM_ERR_INVALID_ARG for another value. */
#define GCM_AES_TABLES 0
#define GCM_AES_BITSLICED 1
int gcm_ctx_set_aes_impl(gcm_ctx *ctx, int impl);

/* Autotuner (the analogue of the paper's per-GPU (TS, R) search, Sec. 5.4,
 * Table 3, "Kernel-optimal parameters"): times a GCM encryption of
 * 16 KiB, 64 KiB, 256 KiB, ... (x4) up to max_bytes (at most 1 GiB) of
 * device-resident zeros with a key of key_len bytes for every tile size
 * 2^9..2^16 blocks, and keeps the fastest per size class: table[c] is the
 * chosen t for sequences of 2^c .. 2^(c+1)-1 blocks (0 = not tuned, the rule
 * applies).  Classes between two measured sizes take the smaller size's
 * choice; classes above the largest take the largest's.  Uses a private
 * stream, about 2 x max_bytes of device scratch from the context's pool
 * (subject to its budget) and synchronises.  table_out (64 bytes, may be
 * NULL) receives the table.  No counterpart in the paper beyond its search. */
int gcm_ctx_autotune(gcm_ctx *ctx, size_t key_len, size_t max_bytes, uint8_t *table_out);

/* Installs a tuning table (64 entries, each 0 or 9..16), e.g. one saved
 * from gcm_ctx_autotune on the same GPU model; NULL clears it. */
int gcm_ctx_set_tuning(gcm_ctx *ctx, const uint8_t *table);

/* Waits until everything enqueued on `stream` (a cudaStream_t; NULL is the
 * legacy default stream) has finished on the context's device, and reports
 * an asynchronous CUDA error from that work as GCM_ERR_CUDA.  The
 * asynchronous device-mode calls (gcm_encrypt, gcm_ctr_xor, gcm_ghash) need
 * it, or any other synchronisation of the stream, before their outputs are
 * read on the host. */
int gcm_sync(gcm_ctx *ctx, void *stream);

/* ---------------------------------------------------------------- */
/* The two halves of the fused pass on their own                    */
/* ---------------------------------------------------------------- */

/* CTR keystream XOR alone (SP 800-38D GCTR started at inc32(J0), the
 * ciphertext half of GCM-AE; the paper's CTR kernel, Sec. 3.3.2, and its
 * unauthenticated CTR comparison, Sec. 5.4, Table 4).  out = in xor E_K(inc32^i(J0)),
 * byte for byte the ciphertext gcm_encrypt would write; no tag.  Same key
 * and IV rules as gcm_encrypt.  in/out are DEVICE pointers, 16-byte aligned,
 * out may equal in; key and iv are host pointers.  Enqueues on `stream` and
 * returns.  Applying it twice with the same key and IV restores the input. */
int gcm_ctr_xor(gcm_ctx *ctx, const uint8_t *key, size_t key_len,
                const uint8_t *iv, size_t iv_len,
                const uint8_t *in, size_t len, uint8_t *out, void *stream);

/* GHASH alone (SP 800-38D Sec. 6.4 / Algorithm 2 over A || 0^v || C || 0^u ||
 * [len(A)]_64 || [len(C)]_64, with H = E_K(0^128); the paper's GHASH-only
 * throughput measurement, Sec. 5.4, Table 5).  Runs the same parallel
 * reduction as the fused pass -- per-chunk Horner, H-power table,
 * log-depth combine (Sec. 3.3.1, Fig. 3b) -- but no AES on the payload
 * and no payload output.
 * out16 receives the 16-byte GHASH value S, so that the GCM tag of the same
 * (A, C) is S xor E_K(J0).  aad, data and out16 are DEVICE pointers (data
 * 16-byte aligned); key is a host pointer.  Enqueues on `stream` and
 * returns. */
int gcm_ghash(gcm_ctx *ctx, const uint8_t *key, size_t key_len,
              const uint8_t *aad, size_t aad_len,
              const uint8_t *data, size_t len, uint8_t *out16, void *stream);

/* ---------------------------------------------------------------- */
/* Many messages: batched device launch and streamed host catalogs   */
/* ---------------------------------------------------------------- */

/* One independent message.  key and iv are host pointers; aad, in, out and
 * tag follow the mem argument of gcm_batch.  out may equal in.  For
 * encryption tag receives the 16-byte tag, for decryption it holds the
 * expected tag. */
typedef struct {
    const uint8_t *key;
    size_t key_len;
    const uint8_t *iv;
    size_t iv_len;
    const uint8_t *aad;
    size_t aad_len;
    const uint8_t *in;
    uint8_t *out;
    size_t len;
    uint8_t *tag;
} gcm_msg;

/* Processes n independent messages (encrypt if decrypt == 0, else
 * decrypt-verify) and returns when all are done.  status (host array of n)
 * receives 0 or GCM_ERR_AUTH per message; the call returns GCM_OK if the
 * batch ran (individual tag failures are only in status), or the first
 * argument/CUDA error.  Outputs of messages whose tag failed are zero-filled.
 *
 * GCM_MEM_DEVICE: all messages go into ONE persistent launch that splits the
 *   work into (message, tile) items taken from an atomic counter; each
 *   message's GHASH partials are reduced across its tiles by the CTA that
 *   finishes the message's last tile (no spin-waits).  Key setup for all
 *   messages is one launch.  Messages of different key sizes mix freely.
 *   Items are handed out shortest message first (status stays in the
 *   caller's order), which lowers the median completion time.
 * GCM_MEM_HOST: where the device reads host memory directly
 *   (gcm_ctx_set_host_access) and every message's in/out is 16-byte
 *   aligned, the same persistent launch runs over the host buffers (page-
 *   locked ones, e.g. from gcm_host_alloc, are reached fastest).  Otherwise
 *   the buffers are streamed through a ring of device chunk buffers: host-
 *   to-device copies, the fused kernel and device-to-host copies of
 *   successive chunks overlap on three streams (the paper's asynchronous
 *   stream pipeline, Sec. 3.3.2), so catalogs larger than device memory
 *   pass through a fixed device footprint.
 * stream: the stream the device-mode launch is ordered on (host mode uses
 *   the context's own streams). */
int gcm_batch(gcm_ctx *ctx, const gcm_msg *msgs, size_t n, int decrypt,
              int32_t *status, int mem, void *stream);

/* gcm_batch in device memory that also reports, per message, the device
 * time (ns, from the GPU's global timer) between the start of the batch's
 * key setup and the completion of that message's tag (done_ns: host array
 * of n).  Used to measure per-message latency inside one persistent launch. */
int gcm_batch_timed(gcm_ctx *ctx, const gcm_msg *msgs, size_t n, int decrypt,
                    int32_t *status, uint64_t *done_ns, void *stream);

/* A device-memory batch prepared once and replayed as a CUDA graph.  The
 * paper launches its kernels file by file (Sec. 3.3.2) and has no
 * counterpart.  A plan serves pipelines that run batches of one shape over
 * and over (the same message lengths, new IVs and data each time, the same
 * or new keys).  It does gcm_batch's per-call host work (validation,
 * ordering, layout, scratch allocation, the enqueued operations) once, and
 * keeps the key material between runs whose keys do not change.
 *
 * gcm_batch_plan_create validates msgs exactly like gcm_batch in
 * GCM_MEM_DEVICE mode (n >= 1).  It allocates the batch's scratch (device
 * memory, held until the plan is destroyed and counted against the
 * context's HBM budget meanwhile, like the scratch of calls in flight) and
 * a page-locked image of its descriptors.  It captures the whole run into
 * a CUDA graph: descriptor upload, counter reset, key setup for every
 * message, the persistent (message, tile) kernel, for decrypt the zero-fill
 * of failed messages, and the verdict download.  A second graph is the same
 * run with the key setup replaced by the per-message J0 / E_K(J0) step.
 * The plan copies the messages' keys and IVs; the device buffers (aad, in,
 * out, tag) must stay valid while a run uses them.  *out receives the plan,
 * or NULL on failure (GCM_ERR_INVALID_ARG, GCM_ERR_LENGTH_LIMIT,
 * GCM_ERR_ALIGNMENT as for gcm_batch; GCM_ERR_NO_MEMORY; GCM_ERR_CUDA).
 * The plan belongs to ctx and must be destroyed before it.
 *
 * gcm_batch_plan_set replaces messages first .. first + count - 1 (the
 * caller's indices at creation) by msgs[0 .. count - 1] for the following
 * runs: any keys, IVs and device buffers, with the payload, AAD, key and IV
 * lengths each message was created with.  All are checked before any is
 * replaced (GCM_ERR_INVALID_ARG / GCM_ERR_ALIGNMENT otherwise, and nothing
 * changes).  It may be called while a run is in flight.
 *
 * gcm_batch_plan_launch enqueues one run on `stream` (a cudaStream_t; NULL
 * is the legacy default stream) and returns.  The first run, and every run
 * after gcm_batch_plan_set changed a key, replays the first graph and builds
 * all messages' key material (round keys, powers of H, GHASH table).  The
 * other runs replay the second graph: they keep that material and derive
 * only each message's J0 and E_K(J0), as the server does for registered
 * keys.  gcm_batch_plan_wait waits for
 * it and writes the per-message verdicts (0 or GCM_ERR_AUTH, the caller's
 * order) to status (host array of n, may be NULL).  Runs of one plan share
 * its scratch, so a plan has at most one run in flight: launch returns
 * GCM_ERR_BUSY until the previous run has been waited for.  Results are
 * those of gcm_batch on the same messages.  A plan is used by one thread at
 * a time; different plans are independent. */
typedef struct gcm_batch_plan gcm_batch_plan;
int gcm_batch_plan_create(gcm_ctx *ctx, const gcm_msg *msgs, size_t n, int decrypt,
                          gcm_batch_plan **out);
int gcm_batch_plan_set(gcm_batch_plan *plan, size_t first, const gcm_msg *msgs, size_t count);
int gcm_batch_plan_launch(gcm_batch_plan *plan, void *stream);
int gcm_batch_plan_wait(gcm_batch_plan *plan, int32_t *status);
/* Waits for a run in flight, then releases the plan's graph, scratch and
 * descriptor image (cleared first: it holds the keys).  NULL is a no-op. */
void gcm_batch_plan_destroy(gcm_batch_plan *plan);

/* How host buffers (GCM_MEM_HOST, host batches, the server) reach the GPU.
 * mode 0 (default, auto): when the device can access host memory directly
 *   (cudaDevAttrPageableMemoryAccess, e.g. Grace-Blackwell over NVLink-C2C
 *   with address translation), the kernels read the host input and write
 *   the host output themselves -- no copies, no staging -- for buffers that
 *   are 16-byte aligned; otherwise the staged pipeline below is used.
 * mode 1: require direct access (GCM_ERR_INVALID_ARG if unsupported).
 * mode 2: always stage through device chunk buffers. */
int gcm_ctx_set_host_access(gcm_ctx *ctx, int mode);

/* Page-locked host memory of exactly `bytes` (cudaHostAlloc, default
 * flags, made under CUDA device `device`) for GCM_MEM_HOST calls, host
 * batches and the server.  The GPU reaches page-locked memory through its
 * own page tables (no per-page address translation over the CPU-GPU link),
 * and the staged pipeline's copies from it run asynchronously.  The caller
 * owns the memory and releases it with gcm_host_free.  *out receives the
 * pointer, or NULL on failure.  Returns GCM_ERR_INVALID_ARG for out == NULL,
 * bytes == 0 or a bad device, GCM_ERR_NO_MEMORY when the allocation fails. */
int gcm_host_alloc(int device, size_t bytes, void **out);

/* Releases memory from gcm_host_alloc; p == NULL is a no-op.  Returns
 * GCM_ERR_CUDA if the runtime refuses the pointer. */
int gcm_host_free(void *p);

/* Host-mode streaming geometry: chunk_bytes of payload per chunk (rounded
 * to whole tiles) and n_buffers device chunk buffers in the ring (>= 2).
 * Defaults: 256 MiB and 3. */
int gcm_ctx_set_streaming(gcm_ctx *ctx, size_t chunk_bytes, int n_buffers);

/* ---------------------------------------------------------------- */
/* Key cache and the continuous-batching server                     */
/* ---------------------------------------------------------------- */

/* Builds a key's material once on the device (round keys, H, powers of H,
 * the GHASH table: 67.4 KiB) and returns a handle for server requests.
 * Register keys before submitting requests that use them. */
int gcm_key_register(gcm_ctx *ctx, const uint8_t *key, size_t key_len, uint32_t *handle);

typedef struct gcm_server gcm_server;

/* One request.  All pointers are host pointers; in/out/aad/tag must stay
 * valid until the request completes (pinned memory lets the copies run
 * asynchronously).  tag receives the tag (op 0) or holds the expected tag
 * (op 1, read at submit).  arrival_ns (the library clock, gcm_now_ns) is the
 * arrival time used for latency; 0 means "now". */
typedef struct {
    int op;                 /* 0 = encrypt, 1 = decrypt-verify */
    uint32_t key;           /* handle from gcm_key_register */
    const uint8_t *iv;
    size_t iv_len;
    const uint8_t *aad;
    size_t aad_len;
    const uint8_t *in;
    uint8_t *out;
    size_t len;
    uint8_t *tag;
    uint64_t arrival_ns;
    uint64_t user;          /* copied to the completion */
} gcm_request;

typedef struct {
    uint64_t ticket;
    int32_t status;         /* 0, GCM_ERR_AUTH (output zero-filled) or an error */
    uint64_t arrival_ns;
    uint64_t complete_ns;   /* library clock when the outputs were in host memory */
    uint64_t user;
} gcm_completion;

/* Starts a server thread on the context's device.  hbm_budget_bytes bounds
 * the device memory of all waves in flight (0 = 40 GB); max_wave_msgs bounds
 * the requests per wave; max_inflight (1..8) waves may be in flight at once.
 * max_wave_msgs = max_inflight = 1 gives a one-request-per-launch server. */
int gcm_server_create(gcm_ctx *ctx, size_t hbm_budget_bytes, size_t max_wave_msgs, int max_inflight,
                      gcm_server **out);

/* Queues a request (thread-safe, does not block on the GPU).  Returns
 * GCM_ERR_BUSY when the queue is full, GCM_ERR_NO_MEMORY when the request
 * alone exceeds the HBM budget. */
int gcm_server_submit(gcm_server *srv, const gcm_request *req, uint64_t *ticket);

/* Queues n requests at once (same rules as gcm_server_submit; all or none
 * are queued).  Their tickets are first_ticket, first_ticket + 1, ... */
int gcm_server_submit_batch(gcm_server *srv, const gcm_request *reqs, size_t n, uint64_t *first_ticket);

/* Moves up to max completions into out; returns how many. */
size_t gcm_server_poll(gcm_server *srv, gcm_completion *out, size_t max);

/* Counters: waves launched, requests launched, requests queued, device
 * bytes held by waves in flight.  Returns 0, or the error that stopped the
 * server. */
int gcm_server_stats(gcm_server *srv, uint64_t *waves, uint64_t *messages, size_t *queued,
                     size_t *bytes_in_flight);

/* Admission under the HBM budget (spec serving: requests are admitted
 * as memory frees up): the budget in force, the largest number of device
 * bytes that waves in flight held at once (never above the budget), and
 * how many requests were held back at least once because the next wave
 * would have exceeded the budget.  Any pointer may be NULL.  Returns 0, or
 * GCM_ERR_INVALID_ARG for a NULL server. */
int gcm_server_admission(gcm_server *srv, size_t *budget, size_t *peak_bytes_in_flight,
                         uint64_t *budget_waits);

/* Time spent so far, summed over waves (ms): out[0] host time issuing
 * waves, out[1] copy-in stage, out[2] compute stage (from copy-in done to
 * kernels done, queueing included), out[3] copy-out stage. */
int gcm_server_timing(gcm_server *srv, double out[4]);

/* Finishes the queued requests, stops the thread, frees the server. */
void gcm_server_destroy(gcm_server *srv);

/* The library's monotonic clock in nanoseconds (for arrival_ns). */
uint64_t gcm_now_ns(void);

/* ---------------------------------------------------------------- */
/* Measurement hooks (used by the benchmark; no counterpart in the  */
/* paper beyond its cudaEventRecord protocol, Sec. 5.3.1)           */
/* ---------------------------------------------------------------- */

/* When enabled, every launch of the fused CTR+GHASH kernel is bracketed by
 * CUDA events recorded on the stream it is launched on, and every kernel the
 * library launches is counted.  Costs two event records per call. */
int gcm_profile_enable(gcm_ctx *ctx, int enable);

/* Waits for the recorded events and returns, since the last reset:
 * fused_ms: summed device time of the fused kernel launches;
 * fused_launches: their number; fused_bytes: algorithmic bytes they moved
 * (payload read + payload written + AAD read); launches: all kernels
 * launched by the library.  Any output pointer may be NULL.  reset != 0
 * clears the totals afterwards. */
int gcm_profile_read(gcm_ctx *ctx, int reset, double *fused_ms, uint64_t *fused_launches,
                     uint64_t *fused_bytes, uint64_t *launches);

/* ---------------------------------------------------------------- */
/* FITS wrapper (Sec. 3.2.2-3.2.3; Table "Core functions")          */
/* ---------------------------------------------------------------- */

/* Which bytes authenticate the data unit.
 *   GFC_AAD_HEADER     : the header records exactly as in the file (every
 *                        2880-byte record through the one holding END,
 *                        blank padding included); the header stays in clear.
 *   GFC_AAD_STRUCTURAL : the paper's AAD_Data = NONCE || Serialize(BITPIX)
 *                        || Serialize(NAXIS) || Serialize(NAXIS1) || ... with
 *                        Serialize = strict ASCII decimal and no separators
 *                        (Sec. 3.2.3). */
typedef enum {
    GFC_AAD_HEADER = 0,
    GFC_AAD_STRUCTURAL = 1
} gfc_aad_mode;

#define GFC_MAX_AXES 999

/* The FITS layout of a single-HDU file, from its header (FITS standard:
 * 2880-byte records of 80-character cards). */
typedef struct {
    size_t header_bytes;      /* records up to and including the END record */
    size_t data_bytes;        /* |BITPIX|/8 * NAXIS1 * ... * NAXISn (0 if NAXIS = 0) */
    size_t data_padded_bytes; /* data_bytes rounded up to whole 2880-byte records */
    int bitpix;
    int naxis;
    int64_t naxes[16];        /* the first 16 axis lengths */
} gfc_layout;

/* Parses the header at `fits` (host memory, `len` bytes available).
 * Returns GCM_ERR_INVALID_ARG if no END card is found, or if SIMPLE,
 * BITPIX or NAXISn are missing or malformed. */
int gfc_fits_layout(const uint8_t *fits, size_t len, gfc_layout *out);

/* The paper's FitsOperationResult (Table "Core functions").
 * data_buffer / buffer_size: the processed file (header records in clear,
 *   then the processed record-padded data unit); owned by the library until
 *   gfc_result_free; in device memory when the call was made with
 *   GCM_MEM_DEVICE, else in pinned host memory.
 * error_code: 0, or the negative gcm_status of the call.
 * warning_code: 0 full access; 2 payload suppressed (tag mismatch: the data
 *   unit in data_buffer is zero-filled and the header is returned as is).
 * error_message: text of the failure ("" on success).
 * datasum / datasum_valid: the FITS DATASUM (32-bit ones' complement sum of
 *   the big-endian 32-bit words; the keyword the paper's container writes,
 *   Sec. 3.2.2) of the ENCRYPTED data unit -- the one written by
 *   gfc_fits_encrypt, or the one read by gfc_fits_decrypt_verify, so that a
 *   container's stored DATASUM can be checked -- computed in the same pass as
 *   the cipher (no extra read of the data).  datasum_valid is 1 when it was
 *   computed (device memory, or host memory the GPU reads directly), 0 on the
 *   staged host path. */
typedef struct {
    uint8_t *data_buffer;
    size_t buffer_size;
    int error_code;
    int warning_code;
    char error_message[200];
    int mem;
    void *stream;
    uint32_t datasum;
    int datasum_valid;
} gfc_result;

/* Encrypts the data unit of a single-HDU FITS file and authenticates it
 * together with the AAD chosen by aad_mode.  iv12 is a 12-byte IV, or NULL
 * to draw one from the operating system's entropy source (Sec. 3.2.2:
 * 96-bit nonces from /dev/urandom); the IV used is written to iv_out (host,
 * 12 bytes) and the tag to tag_out (host, 16 bytes).  fits points to
 * fits_len bytes in the memory space given by mem (device pointers must be
 * 16-byte aligned).  A file whose data unit lacks its final padding is
 * zero-padded; bytes after the padded data unit (further HDUs) are
 * rejected with GCM_ERR_INVALID_ARG.  Returns the status also stored in
 * out->error_code; on success out holds the encrypted file. */
int gfc_fits_encrypt(gcm_ctx *ctx, const uint8_t *key, size_t key_len,
                     const uint8_t *fits, size_t fits_len, const uint8_t *iv12,
                     uint8_t *iv_out, uint8_t *tag_out, int aad_mode, int mem,
                     void *stream, gfc_result *out);

/* Decrypts and verifies a file produced by gfc_fits_encrypt (the paper's
 * gfc_decrypt_frame with the validation gate, Sec. 3.3.2 item 4, and the
 * payload suppression of Sec. 4.2).  iv12 and tag are host pointers.  On a
 * tag mismatch the call returns GCM_ERR_AUTH, out->warning_code is 2 and the
 * data unit of out->data_buffer is all zero bytes. */
int gfc_fits_decrypt_verify(gcm_ctx *ctx, const uint8_t *key, size_t key_len,
                            const uint8_t *fits_enc, size_t len, const uint8_t *iv12,
                            const uint8_t *tag, int aad_mode, int mem, void *stream,
                            gfc_result *out);

/* The paper's dual-key authenticated container (Sec. 3.2.2, Fig.
 * "Structure of the Authenticated FITS Format").  gfc_container_encrypt turns
 * a single-HDU FITS image into two HDUs:
 *   HDU 0 (NAXIS = 0): NONCE_H, NONCE_D (12-byte nonces as lowercase hex),
 *     AUTHTG_H, AUTHTG_D (the paper's AUTHTAG_H / AUTHTAG_D, shortened to the
 *     8-character keyword limit; 16-byte tags as hex), ORIG_BPX, ORIG_NAX,
 *     ORIG_NA1.. (the original BITPIX, NAXIS, NAXISn, abbreviated as in the
 *     paper), and ENCHDR: the original header records encrypted with the
 *     header key under NONCE_H (no AAD), as a hex long string (CONTINUE
 *     cards of 64 characters).
 *   HDU 1: a one-row binary table (TFORM1 = '<N>B', TTYPE1 = 'ENCDATA')
 *     holding the N pixel bytes encrypted with the data key under NONCE_D
 *     with AAD_D = NONCE_D || Serialize(ORIG_BITPIX) || Serialize(ORIG_NAXIS)
 *     || Serialize(ORIG_NAXIS1) || ... (Sec. 3.2.3).
 *   Both HDUs end with the FITS-standard DATASUM and CHECKSUM keywords
 *   (Sec. 3.2.2; FITS checksum convention): DATASUM is the 32-bit ones'
 *   complement sum of the data unit ('0' for HDU 0, which has none; for
 *   HDU 1 computed in the encryption pass) and CHECKSUM the 16-character
 *   encoding of the complement of the HDU's sum, so that each HDU sums to
 *   -0.  On the staged host path, which computes no data sum, HDU 1 carries
 *   neither.
 * key_h/key_d: 16/24/32-byte keys (host).  nonce_h/nonce_d: 12 host bytes,
 * or NULL to draw them from the operating system's entropy source.  fits is
 * in the memory given by mem; out->data_buffer receives the container.
 *
 * gfc_decrypt_frame is the paper's gfc_decrypt_frame(ctx, file, key_h,
 * key_d) (Table "Core functions"; Sec. 3.3.2 pipeline; Sec. 4.2 access
 * behaviour).  key_h / key_d may be NULL (key not provisioned).  The output
 * is always a structurally valid FITS file: the original header when key_h
 * is given and AUTHTG_H verifies, else a minimal header from ORIG_* (header
 * fallback, warning_code 1); the pixels when key_d is given and AUTHTG_D
 * verifies over the pixels and the structural keywords, else zero bytes
 * (payload suppression, warning_code 2, which takes precedence).  As in the
 * paper, error_code is 0 in all of these cases; it is negative only for
 * system errors or a malformed container.  out->datasum is the DATASUM of the
 * stored (encrypted) table data, when the data key was used. */
int gfc_container_encrypt(gcm_ctx *ctx, const uint8_t *key_h, size_t key_h_len,
                          const uint8_t *key_d, size_t key_d_len,
                          const uint8_t *fits, size_t fits_len,
                          const uint8_t *nonce_h, const uint8_t *nonce_d,
                          int mem, void *stream, gfc_result *out);

int gfc_decrypt_frame(gcm_ctx *ctx, const uint8_t *container, size_t len,
                      const uint8_t *key_h, size_t key_h_len,
                      const uint8_t *key_d, size_t key_d_len,
                      int mem, void *stream, gfc_result *out);

/* Releases out->data_buffer (mirrors the teardown side of the paper's API).
 * Safe on a zeroed or already released result. */
void gfc_result_free(gcm_ctx *ctx, gfc_result *res);

/* ---------------------------------------------------------------- */
/* Allocation-free encryption (the paper has no counterpart)        */
/* ---------------------------------------------------------------- */

/* GCM-AE like gcm_encrypt in device mode, but without a context and without
 * allocating any device memory.  It is meant for callers that cannot call
 * cudaMalloc at call time: a process whose device memory is already handed
 * out by another allocator (for example a framework's caching pool that owns
 * almost all of HBM), or a latency-critical loop that must not risk the
 * implicit device-wide synchronisation that cudaMalloc/cudaFree can cause.
 *
 * All scratch (round tables, key material, tile partials) lives in one
 * fixed device array of about 268 KiB inside the library, which every GPU
 * that loads the library keeps until the process exits.  The caller still
 * passes its own buffers: aad, pt, ct and tag are DEVICE pointers (pt/ct
 * 16-byte aligned, ct may equal pt); key and iv are host pointers.
 *
 * Limits: payload + AAD of at most 8 GiB (2^29 blocks) and IVs of at most
 * 256 bytes; larger requests return GCM_ERR_LENGTH_LIMIT without touching
 * the GPU.  Works on the caller's current CUDA device.
 *
 * The first call on each device sets that device up (finds the array's
 * device address, builds the round tables in it) and synchronises `stream`;
 * make that first call before any stream capture.  Later calls only enqueue
 * work on `stream` and return.  The set-up belongs to the CUDA context it
 * was made in: after a device reset (or under another context) the next
 * call detects the new context and sets up again, synchronising as the
 * first call does.
 *
 * Every call shares the one array and the array keeps the last call's
 * contents, so calls whose work overlaps on the GPU (e.g. issued on two
 * streams without ordering) race and can produce wrong tags; order them on
 * one stream.  No part of the array needs clearing between calls: each call
 * writes everything it reads.  Error text: gcm_noalloc_last_error(). */
int gcm_encrypt_noalloc(const uint8_t *key, size_t key_len,
                        const uint8_t *iv, size_t iv_len,
                        const uint8_t *aad, size_t aad_len,
                        const uint8_t *pt, size_t len, uint8_t *ct, uint8_t *tag,
                        void *stream);

/* Message of the last gcm_encrypt_noalloc error on the calling thread. */
const char *gcm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GCMGPU_H */
