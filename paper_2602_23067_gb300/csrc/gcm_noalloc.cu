// gcm_noalloc.cu -- gcm_encrypt_noalloc: GCM encryption that allocates no
// device memory.
//
// The regular entry points take their per-call scratch (key material, tile
// partials, tree scratch) from the context's stream-ordered pool.  Some
// callers cannot allocate at call time: a process whose device memory is
// already carved up by another allocator, or a latency-critical loop that
// must not risk the implicit device synchronisation of cudaMalloc/cudaFree.
// This entry point runs the same kernels with all scratch in one file-scope
// device array of fixed size, which every GPU that loads the library holds
// until the process exits.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda.h>
#include <cuda_runtime.h>

#include "gcm_internal.h"
#include "gcmgpu.h"

using namespace gcmgpu;

namespace {

// Largest number of tiles the static scratch holds.  With 2^16-block tiles
// this bounds payload + AAD to 8192 * 2^16 * 16 bytes = 8 GiB.
constexpr uint64_t NA_MAX_TILES = 8192;
constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t NA_OFF_TABS = 0;
constexpr size_t NA_OFF_KM = na_align(NA_OFF_TABS + sizeof(DevTables));
constexpr size_t NA_OFF_MM = na_align(NA_OFF_KM + sizeof(KeyMat));
constexpr size_t NA_OFF_PART = na_align(NA_OFF_MM + sizeof(MsgMat));
constexpr size_t NA_OFF_TREE = na_align(NA_OFF_PART + NA_MAX_TILES * sizeof(gf128));
constexpr size_t NA_BYTES = na_align(NA_OFF_TREE + (NA_MAX_TILES / 2 + 1) * sizeof(gf128));

}  // namespace

// The scratch itself (about 268 KiB; see NA_BYTES).  In host code this name
// is only a stand-in for the device symbol, never a device address: the
// address each device uses is taken with cudaGetSymbolAddress below.
static __device__ __align__(256) uint8_t g_noalloc_scratch[NA_BYTES];

namespace {

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
uint8_t *g_na_ptr[NA_MAX_DEVICES] = {};
int g_na_sms[NA_MAX_DEVICES] = {};
unsigned long long g_na_ctx[NA_MAX_DEVICES] = {};  // context the set-up was done in

// Identity of the calling thread's current CUDA context (driver entry points
// cuCtxGetCurrent / cuCtxGetId, resolved once through the runtime); 0 when
// there is none yet or the driver cannot tell.  A device reset or a new
// primary context gets a new identity, so the set-up below is redone.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

thread_local std::string g_na_error;

int na_fail(int code, const char *msg)
{
    g_na_error = msg;
    return code;
}

int na_cuda_fail(cudaError_t e, const char *where)
{
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    g_na_error = buf;
    return GCM_ERR_CUDA;
}

// Tile size for a sequence of M blocks: the same rule as the pooled path.
uint32_t na_tile_log2(uint64_t M, int num_sms)
{
    uint32_t lg = 16;
    while (lg > (uint32_t)SEGF_MIN_LOG2 && (M >> lg) < (uint64_t)num_sms * 4) lg--;
    return lg;
}

// One-time set-up on the current device: the device address of the scratch,
// the fused kernel's shared-memory limit, and the AES round tables (built on
// `stream`, which is then synchronised so that later calls on any stream see
// them).
// Set-up is per device and per CUDA context: the cache entry records the
// context it was made in and is redone when the current context differs
// (after cudaDeviceReset, for example).
int na_setup(int dev, cudaStream_t stream, uint8_t **base, int *num_sms)
{
    std::lock_guard<std::mutex> lk(g_na_mu);
    unsigned long long cid = current_context_id();
    if (g_na_ptr[dev] && cid != 0 && cid == g_na_ctx[dev]) {
        *base = g_na_ptr[dev];
        *num_sms = g_na_sms[dev];
        return GCM_OK;
    }
    uint8_t *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&ptr), g_noalloc_scratch);
    if (e != cudaSuccess) return na_cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    cid = current_context_id();  // the runtime has bound a context by now
    if (g_na_ptr[dev] == ptr && cid == g_na_ctx[dev]) {
        *base = ptr;
        *num_sms = g_na_sms[dev];
        return GCM_OK;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return na_cuda_fail(e, "cudaDeviceGetAttribute");
    e = configure_kernels();
    if (e != cudaSuccess) return na_cuda_fail(e, "configuring the fused kernel");
    e = launch_build_tables(reinterpret_cast<DevTables *>(ptr + NA_OFF_TABS), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return na_cuda_fail(e, "building the round tables in the static scratch");
    g_na_ptr[dev] = ptr;
    g_na_sms[dev] = sms;
    g_na_ctx[dev] = cid;
    *base = ptr;
    *num_sms = sms;
    return GCM_OK;
}

}  // namespace

extern "C" const char *gcm_noalloc_last_error(void) { return g_na_error.c_str(); }

extern "C" int gcm_encrypt_noalloc(const uint8_t *key, size_t key_len, const uint8_t *iv, size_t iv_len,
                                   const uint8_t *aad, size_t aad_len, const uint8_t *pt, size_t len,
                                   uint8_t *ct, uint8_t *tag, void *stream)
{
    if (!key || (key_len != 16 && key_len != 24 && key_len != 32))
        return na_fail(GCM_ERR_INVALID_ARG, "key must be 16, 24 or 32 bytes");
    if (!iv || iv_len == 0) return na_fail(GCM_ERR_INVALID_ARG, "IV must be at least one byte");
    if (iv_len > (size_t)IV_INLINE_MAX)
        return na_fail(GCM_ERR_LENGTH_LIMIT, "gcm_encrypt_noalloc takes IVs of at most 256 bytes");
    if (aad_len && !aad) return na_fail(GCM_ERR_INVALID_ARG, "aad is NULL with a nonzero length");
    if (len && (!pt || !ct)) return na_fail(GCM_ERR_INVALID_ARG, "payload pointer is NULL with a nonzero length");
    if (!tag) return na_fail(GCM_ERR_INVALID_ARG, "tag pointer is NULL");
    if (len && ((((uintptr_t)pt) & 15u) || (((uintptr_t)ct) & 15u)))
        return na_fail(GCM_ERR_ALIGNMENT, "device payload pointers must be 16-byte aligned");
    const uint64_t a_blocks = ((uint64_t)aad_len + 15) / 16;
    const uint64_t n_blocks = ((uint64_t)len + 15) / 16;
    const uint64_t M = a_blocks + n_blocks;
    if (len > (1ull << 36) - 32 || M > (NA_MAX_TILES << 16))
        return na_fail(GCM_ERR_LENGTH_LIMIT,
                       "gcm_encrypt_noalloc: payload + AAD exceed the static scratch (at most 8 GiB)");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(GCM_ERR_INVALID_ARG, "device ordinal out of range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *base = nullptr;
    int sms = 0;
    int rc = na_setup(dev, s, &base, &sms);
    if (rc) return rc;

    const uint32_t lg = na_tile_log2(M, sms);
    const uint64_t K = (M + (1ull << lg) - 1) >> lg;
    if (K > NA_MAX_TILES)
        return na_fail(GCM_ERR_LENGTH_LIMIT, "gcm_encrypt_noalloc: too many tiles for the static scratch");
    const DevTables *tabs = reinterpret_cast<const DevTables *>(base + NA_OFF_TABS);
    KeyMat *km = reinterpret_cast<KeyMat *>(base + NA_OFF_KM);
    MsgMat *mm = reinterpret_cast<MsgMat *>(base + NA_OFF_MM);
    gf128 *partials = reinterpret_cast<gf128 *>(base + NA_OFF_PART);
    gf128 *tree = reinterpret_cast<gf128 *>(base + NA_OFF_TREE);
    // Every word of the scratch that a call reads is first written by the
    // same call (key setup fills KeyMat/MsgMat, every tile writes its
    // partial, each tree level writes before the next reads), so nothing has
    // to be cleared between calls.

    KsParams ks;
    memset(&ks, 0, sizeof(ks));
    memcpy(ks.key, key, key_len);
    ks.key_len = (uint32_t)key_len;
    ks.iv_len = (uint32_t)iv_len;
    memcpy(ks.iv_inline, iv, iv_len);
    ks.km = km;
    ks.mm = mm;
    ks.tabs = tabs;
    e = launch_key_setup(ks, s);
    if (e != cudaSuccess) return na_cuda_fail(e, "key setup launch");

    KfParams kf;
    memset(&kf, 0, sizeof(kf));
    kf.in = pt;
    kf.out = ct;
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
    kf.decrypt = 0;
    kf.km = km;
    kf.mm = mm;
    kf.tabs = tabs;
    kf.partials = partials;
    const int grid = (int)(K < (uint64_t)sms ? K : (uint64_t)sms);
    e = launch_fused(kf, (int)key_len / 4 + 6, grid, s);
    if (e != cudaSuccess) return na_cuda_fail(e, "fused kernel launch");

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
    kc.tag_out = tag;
    e = launch_combine(kc, s);
    if (e != cudaSuccess) return na_cuda_fail(e, "combine kernel launch");
    return GCM_OK;
}
