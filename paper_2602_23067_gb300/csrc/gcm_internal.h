// gcm_internal.h -- device data layouts and kernel launchers shared by the
// kernel file and the C-ABI implementation.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "gcm_device.cuh"

namespace gcmgpu {

// Threads per CTA of the fused map kernel (16 warps).  Each warp walks one
// contiguous segment of a tile in windows of 32 consecutive blocks, lane l
// taking the l-th block of every window, so each lane's Horner chain has
// stride GH_STRIDE = 32 and the key setup builds its table for H^32.
constexpr int KF_THREADS = 512;
constexpr int KF_WARPS = KF_THREADS / 32;
constexpr int KF_LOG2_WARPS = 4;
constexpr int GH_STRIDE = 32;
constexpr int GH_LOG2_STRIDE = 5;
constexpr int SEGF_MIN_LOG2 = 9;   // smallest tile: 2^9 blocks (32 per warp)
constexpr int SEGF_SIZES = 8;      // tile sizes 2^9 .. 2^16
constexpr int H2K_COUNT = 40;  // H^(2^k), k = 0..39 (covers 2^39 blocks)
constexpr uint32_t BATCH_TILE_LOG2 = 16;  // largest tile of the batched kernel (2^16 blocks)
constexpr int GTAB_ENTRIES = 4096;  // 256 byte values x 16 byte positions
// Warps of the fused kernel that run their GHASH chains through the integer
// field multiply instead of the table (a measured alternative; 0 = none).
// Set at build time, e.g. GCMGPU_NVCC_FLAGS=-DGH_IMAD_WARPS=2.
#ifndef GH_IMAD_WARPS
#define GH_IMAD_WARPS 0
#endif

// Shared-memory map of the fused kernel (byte offsets into dynamic smem).
constexpr uint32_t SM_T01 = 0;         // rows v: [T0[v] x 32 lanes | T1[v] x 32 lanes]
constexpr uint32_t SM_T23 = 65536;     // rows v: [T2[v] x 32 lanes | T3[v] x 32 lanes]
constexpr uint32_t SM_GTAB = 131072;   // rows v: 16 positions x 16 bytes
constexpr uint32_t SM_RED = 196608;    // cross-warp reduction slots (16 x 16 B)
constexpr uint32_t SM_SEGF = SM_RED + 256;  // per-warp segment factors H^((15-w)S)
constexpr uint32_t SM_WSCR = SM_SEGF + KF_WARPS * 16;  // per-warp scratch of gf_mul_warp (16 x 128 B)
constexpr uint32_t SM_DSUM = SM_WSCR + KF_WARPS * 128;  // per-warp DATASUM partials (16 x 8 B)
constexpr uint32_t KF_SMEM_BYTES = SM_DSUM + KF_WARPS * 8;
// The bitsliced-AES form of the fused kernel (gcm_ctx_set_aes_impl = 1):
// 256 threads (each holds 32 blocks as 128 bitsliced words, so it needs far
// more registers than a table thread), every warp walking two of the tile's
// 16 segments; the same shared memory plus the bitsliced round keys
// (128 words per round, up to 15 rounds).
constexpr int KBS_THREADS = 256;
constexpr uint32_t SM_KBS = (KF_SMEM_BYTES + 15u) & ~15u;
constexpr uint32_t KBS_SMEM_BYTES = SM_KBS + 128 * 15 * 4;

// Per-key material, built on the device by the key-setup kernel.
struct KeyMat {
    uint32_t rk[60];            // round keys, memory words (FIPS-197 sec. 5.2)
    uint32_t nr;                // 10, 12 or 14
    uint32_t pad_[3];
    gf128 H;                    // hash subkey E_K(0^128), poly words
    gf128 h2k[H2K_COUNT];       // H^(2^k): the stride table of the tree (Sec. 3.3.1)
    gf128 hpow[GH_STRIDE];      // H^1 .. H^32: per-lane closing factors
    gf128 segf[SEGF_SIZES][KF_WARPS];  // [lg - SEGF_MIN_LOG2][w] = H^((15-w) * 2^(lg-4)): warp
                                        // factors for tiles of 2^lg blocks, lg = 9..16
    uint4 gtab[GTAB_ENTRIES];   // entry v*16+k = (byte v at position k) * H^32, memory words
};

// Weights of the flat reduce that finishes a message of at most 1024 tiles
// of 2^lg blocks inside the fused launch: the partial of the tile g tiles
// before the last one moves to the sequence end by
// H^(2^lg * g) = w1[g mod 32] * w2[g / 32].  Built by the single-message key
// setup only, and stored right after that path's KeyMat.
struct KeyFin {
    gf128 w1[SEGF_SIZES][32];  // [lg - SEGF_MIN_LOG2][j] = H^(2^lg * j)
    gf128 w2[SEGF_SIZES][32];  // [lg - SEGF_MIN_LOG2][q] = H^(2^lg * 32 q)
};

// Per-message material.
struct MsgMat {
    uint32_t j0[4];   // pre-counter block J0, memory words
    uint32_t ej0[4];  // E_K(J0), memory words
};

// Device-resident constants built once per context.
struct DevTables {
    uint8_t sbox[256];
    uint32_t ttab[4 * 256];  // T0..T3
};

constexpr int IV_INLINE_MAX = 256;

struct KsParams {
    uint8_t key[32];
    uint32_t key_len;
    uint32_t iv_len;
    uint8_t iv_inline[IV_INLINE_MAX];
    const uint8_t *iv_dev;      // used when iv_len > IV_INLINE_MAX
    KeyMat *km;
    MsgMat *mm;
    const DevTables *tabs;
    KeyFin *fin;                // non-null: also build the flat-reduce weights here
};

struct KfParams {
    const uint8_t *in;      // payload read (pt for encrypt, ct for decrypt)
    uint8_t *out;           // payload written
    const uint8_t *aad;
    uint64_t len;           // payload bytes
    uint64_t aad_len;
    uint64_t a_blocks;      // ceil(aad_len / 16)
    uint64_t n_full;        // len / 16 (whole payload blocks)
    uint64_t M;             // a_blocks + ceil(len / 16): GHASH blocks before the length block
    uint64_t K;             // number of tiles
    uint64_t tile_begin;    // this launch processes tiles [tile_begin, tile_end)
    uint64_t tile_end;
    uint32_t tile_log2;     // tile = 2^tile_log2 blocks, aligned to the end of the sequence
    uint32_t decrypt;
    const KeyMat *km;
    const MsgMat *mm;
    const DevTables *tabs;
    gf128 *partials;        // K tile partials, poly words
    uint32_t j0_given;      // 1: J0 is j0 below (96-bit IV, formed on the host), else mm->j0
    uint32_t j0[4];         // memory words
    uint32_t *dsums;        // K per-tile DATASUM partials (mode 3 only)
    // Finishing in the same launch (1 <= K <= FINISH_MAX_TILES, M <=
    // FINISH_MAX_BLOCKS; modes 0, 2, 3): the last CTA to finish runs the
    // combine, the length block, the tag and the verify gate.  ticket is a
    // zero word that only launches on one stream share (left at zero).
    uint32_t *ticket;       // null: a separate combine kernel follows
    const KeyFin *fin;      // flat-reduce weights of the key (with ticket)
    uint8_t *tag_out;       // 16 bytes (device): the tag, or GHASH_H(A, C) in mode 2
    const uint8_t *tag_expected;  // 16 bytes (device) for decryption, else null
    int32_t *status;        // device verdict word (decryption), may be null
    uint32_t *datasum_out;  // mode 3: the message's DATASUM
};
// Largest message finished by the fused launch itself: the tile partials fit
// in shared memory and a failed tag's zero-fill by one CTA stays short.
constexpr uint64_t FINISH_MAX_TILES = 1024;
constexpr uint64_t FINISH_MAX_BLOCKS = 1ull << 22;  // 64 MiB of payload + AAD

// One message of a device-memory batch (gcm_batch with GCM_MEM_DEVICE).
struct BatchMsg {
    const uint8_t *in;
    uint8_t *out;
    const uint8_t *aad;
    uint64_t len;
    uint64_t aad_len;
    uint64_t K;             // tiles of 2^tile_log2 blocks
    uint64_t item_base;     // index of the message's first work item
    uint32_t nr;
    uint32_t dec;           // 1: decrypt-verify this message (GHASH over the input)
    uint32_t tile_log2;     // SEGF_MIN_LOG2 .. BATCH_TILE_LOG2
    KeyMat *km;
    MsgMat *mm;
    gf128 *partials;        // K entries
    gf128 *tree;            // K/2 + 1 entries
    uint8_t *tag;           // device: written (encrypt) or expected (decrypt)
    int32_t *status;        // device verdict word
    uint64_t *t_done;       // device: %globaltimer when the message completed (or null)
};

struct BatchKey {
    uint8_t key[32];
    uint32_t key_len;
    uint32_t iv_len;
    const uint8_t *iv;      // device copy of the IV
};

struct BatchParams {
    const BatchMsg *msgs;
    uint32_t n;
    uint32_t decrypt;
    uint64_t total_items;
    unsigned long long *item_counter;  // zeroed before the launch
    uint32_t *done;                    // n counters, zeroed before the launch
    const DevTables *tabs;
};

struct KcParams {
    gf128 *partials;        // K partials (overwritten: used as the tree's scratch)
    gf128 *scratch;         // K/2 + 1 entries
    uint64_t K;
    uint32_t tile_log2;
    uint64_t aad_len;
    uint64_t len;
    const KeyMat *km;
    const MsgMat *mm;
    uint8_t *tag_out;       // 16 bytes (device), may be null
    const uint8_t *tag_expected;  // 16 bytes (device) for decrypt, else null
    int32_t *status;        // device status word (decrypt), may be null
    int raw;                // 1: output GHASH_H(A, C) itself (no E_K(J0) mask)
    uint32_t ej0_from_j0;   // 1: compute E_K(J0) here from j0 below, else read mm->ej0
    uint32_t j0[4];         // memory words
    const DevTables *tabs;  // round tables (for E_K(J0))
    const uint32_t *dsums;  // K per-tile DATASUM partials, or null
    uint32_t *datasum_out;  // device: the message's DATASUM (when dsums is set)
};

struct KzParams {
    uint8_t *out;
    uint64_t len;
    const int32_t *status;
};

// Launchers (defined in gcm_kernels.cu).  All are asynchronous on `stream`.
cudaError_t launch_build_tables(DevTables *tabs, cudaStream_t stream);
cudaError_t launch_key_setup(const KsParams &p, cudaStream_t stream);
// J0 and E_K(J0) only, into p.mm, for key material p.km set up earlier.
cudaError_t launch_msg_only(const KsParams &p, cudaStream_t stream);
// mode: 0 full GCM, 1 CTR keystream only, 2 GHASH only (no AES, no output),
// 3 full GCM plus the per-tile DATASUM partials of the ciphertext side
// impl: 0 round tables in shared memory, 1 bitsliced AES (modes 0, 1, 3)
cudaError_t launch_fused(const KfParams &p, int nr, int grid, cudaStream_t stream, int mode = 0, int impl = 0);
cudaError_t launch_combine(const KcParams &p, cudaStream_t stream);
cudaError_t launch_zero_on_fail(const KzParams &p, int grid, cudaStream_t stream);
cudaError_t launch_batch_key_setup(const BatchMsg *msgs, const BatchKey *keys, uint32_t n,
                                   const DevTables *tabs, uint64_t *t_start, cudaStream_t stream);
cudaError_t launch_batch(const BatchParams &p, int grid, cudaStream_t stream);
// J0 and E_K(J0) for messages whose key material is already built (cached keys).
cudaError_t launch_msg_setup(const BatchMsg *msgs, const BatchKey *keys, uint32_t n, const DevTables *tabs,
                             cudaStream_t stream);
cudaError_t launch_batch_zero(const BatchMsg *msgs, uint32_t n, cudaStream_t stream);
cudaError_t configure_kernels();  // sets the dynamic shared memory limit

}  // namespace gcmgpu
