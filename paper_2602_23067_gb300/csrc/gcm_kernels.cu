// gcm_kernels.cu -- the AES-GCM hot path on sm_103a.
//
// Kernels (one pass over the payload; the paper's CTR kernel and GHASH map
// kernel, Sec. 3.3.2 and 5.2.2, are fused into KF):
//   build_tables  once per context: S-box from GF(2^8) and the four AES
//                 round tables T0..T3 (FIPS-197 sec. 5.1).
//   KS  key_setup per key/message: key expansion (FIPS-197 sec. 5.2),
//                 H = E_K(0^128), J0 (SP 800-38D Alg. 4 step 2), E_K(J0),
//                 the stride table H^(2^k) (Sec. 3.3.1), H^1..H^T and the
//                 8-bit multiplication table of H^T.
//   KF  fused     AES-CTR keystream + XOR (geometry-agnostic counters,
//                 Sec. 5.2: block j always uses inc32^(j+1)(J0)) fused with
//                 the GHASH map: every CTA reduces tiles of the GHASH input
//                 sequence A||C to 16-byte partials (Sec. 5.2.2, map phase).
//   KF' fused_bs  the same pass with the CTR keystream from bitsliced AES
//                 (32 blocks per thread; the paper's own AES core is
//                 bit-sliced, Sec. 5.2), selected per context.
//   KC  combine   log-depth tree over the tile partials with multipliers
//                 H^(2^k) (Sec. 3.3.1, Fig. 3b; Sec. 5.2.2 reduce phase),
//                 the length block and T = E_K(J0) xor GHASH; for decryption
//                 the constant-time tag check (Sec. 3.3.2 item 4).
//   KZ  zero_fill on an authentication failure the output payload is zeroed
//                 (payload suppression, Sec. 4.2).
#include <cstdint>
#include <cuda_runtime.h>

#include "gcm_bitsliced.cuh"
#include "gcm_internal.h"

namespace gcmgpu {

// ---------------------------------------------------------------------
// Tables, once per context
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(256) build_tables_kernel(DevTables *tabs)
{
    __shared__ uint8_t sbox[256], ex[256], lg[256];
    build_sbox_block(sbox, ex, lg);
    const int t = threadIdx.x;
    tabs->sbox[t] = sbox[t];
#pragma unroll
    for (int r = 0; r < 4; r++) tabs->ttab[r * 256 + t] = ttable_entry(r, sbox[t]);
}

// ---------------------------------------------------------------------
// Single-block AES for the setup kernels (H = E_K(0^128) and E_K(J0)):
// round tables T0..T3 and S-box given by pointer (the context's tables in
// global memory, or a copy in shared memory).  State: four memory words, word c = column c, byte r = row r;
// column c of a round takes row r from column c + r (ShiftRows).
// ---------------------------------------------------------------------
__device__ void aes_block_tt(const uint32_t *rk, int nr, const uint32_t *T, const uint8_t *sbox,
                             const uint32_t in[4], uint32_t out[4])
{
    uint32_t s0 = in[0] ^ rk[0], s1 = in[1] ^ rk[1], s2 = in[2] ^ rk[2], s3 = in[3] ^ rk[3];
#define TT(k, w, B) T[(k) * 256 + (((w) >> (8 * (B))) & 0xFFu)]
    for (int r = 1; r < nr; r++) {
        const uint32_t n0 = TT(0, s0, 0) ^ TT(1, s1, 1) ^ TT(2, s2, 2) ^ TT(3, s3, 3) ^ rk[4 * r];
        const uint32_t n1 = TT(0, s1, 0) ^ TT(1, s2, 1) ^ TT(2, s3, 2) ^ TT(3, s0, 3) ^ rk[4 * r + 1];
        const uint32_t n2 = TT(0, s2, 0) ^ TT(1, s3, 1) ^ TT(2, s0, 2) ^ TT(3, s1, 3) ^ rk[4 * r + 2];
        const uint32_t n3 = TT(0, s3, 0) ^ TT(1, s0, 1) ^ TT(2, s1, 2) ^ TT(3, s2, 3) ^ rk[4 * r + 3];
        s0 = n0; s1 = n1; s2 = n2; s3 = n3;
    }
#undef TT
#define SB(w, B) ((uint32_t)sbox[((w) >> (8 * (B))) & 0xFFu] << (8 * (B)))
    out[0] = (SB(s0, 0) | SB(s1, 1) | SB(s2, 2) | SB(s3, 3)) ^ rk[4 * nr];
    out[1] = (SB(s1, 0) | SB(s2, 1) | SB(s3, 2) | SB(s0, 3)) ^ rk[4 * nr + 1];
    out[2] = (SB(s2, 0) | SB(s3, 1) | SB(s0, 2) | SB(s1, 3)) ^ rk[4 * nr + 2];
    out[3] = (SB(s3, 0) | SB(s0, 1) | SB(s1, 2) | SB(s2, 3)) ^ rk[4 * nr + 3];
#undef SB
}

// Key expansion (FIPS-197 sec. 5.2) into memory words.  Word i holds bytes
// 4i..4i+3 of the schedule with the first byte in the low bits, so RotWord is
// a right rotation by 8 and Rcon enters the low byte.
__device__ int key_expand_words(const uint8_t *key, int key_len, const uint8_t *sbox, uint32_t *w)
{
    const int nk = key_len / 4;
    const int nr = nk + 6;
    for (int i = 0; i < nk; i++)
        w[i] = (uint32_t)key[4 * i] | ((uint32_t)key[4 * i + 1] << 8) |
               ((uint32_t)key[4 * i + 2] << 16) | ((uint32_t)key[4 * i + 3] << 24);
    uint8_t rcon = 1;
    for (int i = nk; i < 4 * (nr + 1); i++) {
        uint32_t t = w[i - 1];
        if (i % nk == 0) {
            t = (t >> 8) | (t << 24);
            t = (uint32_t)sbox[t & 0xFF] | ((uint32_t)sbox[(t >> 8) & 0xFF] << 8) |
                ((uint32_t)sbox[(t >> 16) & 0xFF] << 16) | ((uint32_t)sbox[t >> 24] << 24);
            t ^= rcon;
            rcon = gf8_xtime(rcon);
        } else if (nk > 6 && i % nk == 4) {
            t = (uint32_t)sbox[t & 0xFF] | ((uint32_t)sbox[(t >> 8) & 0xFF] << 8) |
                ((uint32_t)sbox[(t >> 16) & 0xFF] << 16) | ((uint32_t)sbox[t >> 24] << 24);
        }
        w[i] = w[i - nk] ^ t;
    }
    return nr;
}

// ---------------------------------------------------------------------
// KS: per-key / per-message setup (one CTA of 256 threads)
// ---------------------------------------------------------------------
// The whole per-key / per-message setup, run by one CTA of 256 threads.
// iv points to iv_len bytes (device or kernel-parameter memory).
__device__ void key_setup_body(const uint8_t *key, uint32_t key_len, const uint8_t *iv, uint32_t iv_len, KeyMat *km,
                               MsgMat *mm, const DevTables *tabs, KeyFin *fin = nullptr)
{
    __shared__ uint8_t sbox[256];
    __shared__ uint32_t stt[4 * 256];  // T0..T3: the two single-block AES calls read them here
    __shared__ uint32_t rkw[60];
    __shared__ gf128 sH;
    __shared__ gf128 sh2k[H2K_COUNT];
    __shared__ gf128 basis[128];
    __shared__ int s_nr;
    const int t = threadIdx.x;

    sbox[t] = tabs->sbox[t];
#pragma unroll
    for (int r = 0; r < 4; r++) stt[r * 256 + t] = tabs->ttab[r * 256 + t];
    __syncthreads();
    if (t == 0) {
        int nr = key_expand_words(key, (int)key_len, sbox, rkw);
        s_nr = nr;
        uint32_t zero[4] = {0u, 0u, 0u, 0u}, h[4];
        aes_block_tt(rkw, nr, stt, sbox, zero, h);
        sH = gf_from_mem(h[0], h[1], h[2], h[3]);
    }
    __syncthreads();
    const int nr = s_nr;
    if (t == 0) {
        // Stride table H^(2^k) by repeated squaring.
        gf128 cur = sH;
        for (int k = 0; k < H2K_COUNT; k++) {
            sh2k[k] = cur;
            km->h2k[k] = cur;
            cur = gf_sqr(cur);
        }
        km->H = sH;
        km->nr = (uint32_t)nr;
    } else if (t == 32) {
        // J0: IV || 0^31 || 1 for a 96-bit IV, else GHASH_H(IV || pad || [len(IV)]_64).
        uint32_t j0[4];
        if (iv_len == 12) {
            for (int i = 0; i < 3; i++)
                j0[i] = (uint32_t)iv[4 * i] | ((uint32_t)iv[4 * i + 1] << 8) |
                        ((uint32_t)iv[4 * i + 2] << 16) | ((uint32_t)iv[4 * i + 3] << 24);
            j0[3] = 0x01000000u;  // bytes 12..15 = 00 00 00 01
        } else {
            gf128 y = gf_zero();
            for (uint32_t off = 0; off < iv_len; off += 16) {
                uint32_t m[4] = {0u, 0u, 0u, 0u};
                for (uint32_t b = 0; b < 16 && off + b < iv_len; b++)
                    m[b >> 2] |= (uint32_t)iv[off + b] << (8 * (b & 3));
                y = gf_mul(gf_xor(y, gf_from_mem(m[0], m[1], m[2], m[3])), sH);
            }
            gf128 lb = gf_zero();
            const uint64_t bits = (uint64_t)iv_len * 8u;
            lb.w[2] = (uint32_t)(bits >> 32);
            lb.w[3] = (uint32_t)bits;
            y = gf_mul(gf_xor(y, lb), sH);
            uint4 jm = gf_to_mem(y);
            j0[0] = jm.x; j0[1] = jm.y; j0[2] = jm.z; j0[3] = jm.w;
        }
        uint32_t e[4];
        aes_block_tt(rkw, nr, stt, sbox, j0, e);
        for (int i = 0; i < 4; i++) {
            mm->j0[i] = j0[i];
            mm->ej0[i] = e[i];
        }
    } else if (t >= 64 && t < 64 + 60) {
        km->rk[t - 64] = (t - 64 < 4 * (nr + 1)) ? rkw[t - 64] : 0u;
    }
    __syncthreads();
    // All multiplications below are branch-free selects of a factor, so the
    // threads of a warp multiply in lockstep.
    gf128 one;
    one.w[0] = 0x80000000u;
    one.w[1] = one.w[2] = one.w[3] = 0u;
    if (t < 128) {
        // basis[i] = x^i * H^32: the 128 single-coefficient products.
        gf128 xi = gf_zero();
        xi.w[t >> 5] = 0x80000000u >> (t & 31);
        basis[t] = gf_mul(xi, sh2k[GH_LOG2_STRIDE]);
    }
    if (t < GH_STRIDE) {
        // H^e for e = 1..32 as a product of stride-table entries.
        const int e = t + 1;
        gf128 acc = one;
        for (int k = 0; k <= GH_LOG2_STRIDE; k++) acc = gf_mul(acc, ((e >> k) & 1) ? sh2k[k] : one);
        km->hpow[e - 1] = acc;
    }
    if (t >= 128 && t < 128 + SEGF_SIZES * KF_WARPS) {
        // H^((15-w) * 2^(lg-4)) for every tile size 2^lg the kernels use.
        const int w = (t - 128) & (KF_WARPS - 1), sz = (t - 128) / KF_WARPS;
        const int steps = KF_WARPS - 1 - w;
        const int base = SEGF_MIN_LOG2 + sz - KF_LOG2_WARPS;
        gf128 f = one;
        for (int b = 0; b < KF_LOG2_WARPS; b++) f = gf_mul(f, ((steps >> b) & 1) ? sh2k[base + b] : one);
        km->segf[sz][w] = f;
    }
    if (fin) {
        // Flat-reduce weights for tiles of 2^lg blocks, lg = 9..16: entry j of
        // w1 is H^(2^lg * j) (bits of j select H^(2^(lg+b))), entry q of w2
        // is H^(2^lg * 32 q) (H^(2^(lg+5+b))); two entries per thread.
        for (int idx = t; idx < 2 * SEGF_SIZES * 32; idx += blockDim.x) {
            const int which = idx / (SEGF_SIZES * 32), r = idx % (SEGF_SIZES * 32);
            const int sz = r / 32, e = r % 32;
            const int base = SEGF_MIN_LOG2 + sz + (which ? 5 : 0);
            gf128 f = one;
            for (int b = 0; b < 5; b++) f = gf_mul(f, ((e >> b) & 1) ? sh2k[base + b] : one);
            if (which) fin->w2[sz][e] = f;
            else fin->w1[sz][e] = f;
        }
    }
    __syncthreads();
    // 8-bit table: entry (v, k) = (byte value v at byte position k) * H^32,
    // stored at v * 16 + k.  Bit b of v (LSB = 0) is the coefficient of
    // x^(8k + 7 - b).  The lanes of a warp share k, so their basis reads are
    // broadcasts (lanes on different k would read entries 128 bytes apart,
    // all in one bank group).
    for (int idx = t; idx < GTAB_ENTRIES; idx += blockDim.x) {
        const int k = idx >> 8, v = idx & 255;
        gf128 acc = gf_zero();
        for (int b = 0; b < 8; b++) {
            const uint32_t m = 0u - (uint32_t)((v >> b) & 1);
            const gf128 &bv = basis[8 * k + 7 - b];
            for (int i = 0; i < 4; i++) acc.w[i] ^= bv.w[i] & m;
        }
        km->gtab[v * 16 + k] = gf_to_mem(acc);
    }
}

__global__ void __launch_bounds__(256) key_setup_kernel(const __grid_constant__ KsParams p)
{
    const uint8_t *iv = (p.iv_len <= IV_INLINE_MAX) ? p.iv_inline : p.iv_dev;
    key_setup_body(p.key, p.key_len, iv, p.iv_len, p.km, p.mm, p.tabs, p.fin);
}

// ---------------------------------------------------------------------
// KF: fused CTR + GHASH map
// ---------------------------------------------------------------------
__device__ __forceinline__ uint32_t lds32(const uint8_t *base, uint32_t off)
{
    return *reinterpret_cast<const uint32_t *>(base + off);
}

__device__ __forceinline__ uint4 lds128(const uint8_t *base, uint32_t off)
{
    return *reinterpret_cast<const uint4 *>(base + off);
}

__device__ __forceinline__ void xor4(uint4 &a, const uint4 &b)
{
    a.x ^= b.x; a.y ^= b.y; a.z ^= b.z; a.w ^= b.w;
}

// Address of a round-table entry: byte `BYTE` of w selects the row (bits
// 8..15 of the address) and c holds this lane's column inside the row
// (lane * 4, plus 128 for the odd table of the pair).  Every lane reads its
// own bank, so a warp-wide lookup never conflicts.
#define TADDR(w, BYTE, c) __byte_perm((w), (c), 0x5504u | ((BYTE) << 4))

struct LaneConst {
    uint32_t cA, cB;        // round-table lane offsets
    uint32_t selA, selB;    // byte rotations for the GHASH lookups
    uint32_t cg[8];         // GHASH table slot offsets per lookup step
};

__device__ __forceinline__ LaneConst make_lane_const(int lane)
{
    LaneConst L;
    L.cA = (uint32_t)lane * 4u;
    L.cB = 128u + (uint32_t)lane * 4u;
    const uint32_t r8 = (uint32_t)lane & 7u;
    L.selA = 0u;
    L.selB = 0u;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        L.selA |= ((r8 + j) & 7u) << (4 * j);
        L.selB |= ((r8 + 4 + j) & 7u) << (4 * j);
    }
#pragma unroll
    for (int i = 0; i < 8; i++) L.cg[i] = ((i + r8) & 7u) << 4;
    return L;
}

// a * H^T through the shared 8-bit table: the XOR of 16 entries, one per
// byte position.  Lanes of a quarter-warp visit the positions of each half
// in rotated order, so their 16-byte reads fall in 8 distinct bank groups.
__device__ __forceinline__ uint4 ghash_mul_table(const uint8_t *smem, const uint4 &a, const LaneConst &L)
{
    const uint8_t *g = smem + SM_GTAB;
    const uint32_t y0 = __byte_perm(a.x, a.y, L.selA);
    const uint32_t y1 = __byte_perm(a.x, a.y, L.selB);
    const uint32_t y2 = __byte_perm(a.z, a.w, L.selA);
    const uint32_t y3 = __byte_perm(a.z, a.w, L.selB);
    uint4 r = lds128(g, TADDR(y0, 0, L.cg[0]));
    xor4(r, lds128(g, TADDR(y0, 1, L.cg[1])));
    xor4(r, lds128(g, TADDR(y0, 2, L.cg[2])));
    xor4(r, lds128(g, TADDR(y0, 3, L.cg[3])));
    xor4(r, lds128(g, TADDR(y1, 0, L.cg[4])));
    xor4(r, lds128(g, TADDR(y1, 1, L.cg[5])));
    xor4(r, lds128(g, TADDR(y1, 2, L.cg[6])));
    xor4(r, lds128(g, TADDR(y1, 3, L.cg[7])));
    const uint8_t *g2 = g + 128;
    xor4(r, lds128(g2, TADDR(y2, 0, L.cg[0])));
    xor4(r, lds128(g2, TADDR(y2, 1, L.cg[1])));
    xor4(r, lds128(g2, TADDR(y2, 2, L.cg[2])));
    xor4(r, lds128(g2, TADDR(y2, 3, L.cg[3])));
    xor4(r, lds128(g2, TADDR(y3, 0, L.cg[4])));
    xor4(r, lds128(g2, TADDR(y3, 1, L.cg[5])));
    xor4(r, lds128(g2, TADDR(y3, 2, L.cg[6])));
    xor4(r, lds128(g2, TADDR(y3, 3, L.cg[7])));
    return r;
}

// Round-table lookups: T0/T1 live in the first 64 KiB region, T2/T3 in the
// second; the lane's column is cA (even table) or cB (odd table).
#define LT0(w, B) lds32(t01, TADDR((w), B, L.cA))
#define LT1(w, B) lds32(t01, TADDR((w), B, L.cB))
#define LT2(w, B) lds32(t23, TADDR((w), B, L.cA))
#define LT3(w, B) lds32(t23, TADDR((w), B, L.cB))

// One full AES round (SubBytes, ShiftRows, MixColumns, AddRoundKey) on the
// state s0..s3 (memory words = columns): column c takes row r from column c+r.
__device__ __forceinline__ void aes_round(const uint8_t *t01, const uint8_t *t23, const LaneConst &L,
                                          uint32_t &s0, uint32_t &s1, uint32_t &s2, uint32_t &s3,
                                          uint32_t k0, uint32_t k1, uint32_t k2, uint32_t k3)
{
    const uint32_t n0 = LT0(s0, 0) ^ LT1(s1, 1) ^ LT2(s2, 2) ^ LT3(s3, 3) ^ k0;
    const uint32_t n1 = LT0(s1, 0) ^ LT1(s2, 1) ^ LT2(s3, 2) ^ LT3(s0, 3) ^ k1;
    const uint32_t n2 = LT0(s2, 0) ^ LT1(s3, 1) ^ LT2(s0, 2) ^ LT3(s1, 3) ^ k2;
    const uint32_t n3 = LT0(s3, 0) ^ LT1(s0, 1) ^ LT2(s1, 2) ^ LT3(s2, 3) ^ k3;
    s0 = n0; s1 = n1; s2 = n2; s3 = n3;
}

// Final round (no MixColumns).  S[v] is byte 0 of T2[v], byte 1 of T3[v],
// byte 2 of T0[v] and byte 3 of T1[v].
__device__ __forceinline__ uint32_t aes_last_col(const uint8_t *t01, const uint8_t *t23, const LaneConst &L,
                                                 uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t k)
{
    const uint32_t e0 = LT2(a, 0), e1 = LT3(b, 1), e2 = LT0(c, 2), e3 = LT1(d, 3);
    return __byte_perm(__byte_perm(e0, e1, 0x3250u), __byte_perm(e2, e3, 0x7210u), 0x7610u) ^ k;
}

// Rounds 3..NR on a state that already went through rounds 0..2.
template <int NR>
__device__ __forceinline__ uint4 aes_rounds_from3(const uint8_t *t01, const uint8_t *t23, const LaneConst &L,
                                                  uint32_t s0, uint32_t s1, uint32_t s2, uint32_t s3,
                                                  const uint32_t *rk)
{
#pragma unroll
    for (int r = 3; r < NR; r++)
        aes_round(t01, t23, L, s0, s1, s2, s3, rk[4 * r], rk[4 * r + 1], rk[4 * r + 2], rk[4 * r + 3]);
    uint4 o;
    o.x = aes_last_col(t01, t23, L, s0, s1, s2, s3, rk[4 * NR + 0]);
    o.y = aes_last_col(t01, t23, L, s1, s2, s3, s0, rk[4 * NR + 1]);
    o.z = aes_last_col(t01, t23, L, s2, s3, s0, s1, rk[4 * NR + 2]);
    o.w = aes_last_col(t01, t23, L, s3, s0, s1, s2, rk[4 * NR + 3]);
    return o;
}

__device__ __forceinline__ uint4 load_partial(const uint8_t *src, uint32_t nbytes)
{
    uint32_t m[4] = {0u, 0u, 0u, 0u};
    for (uint32_t b = 0; b < nbytes; b++) m[b >> 2] |= (uint32_t)src[b] << (8 * (b & 3));
    return make_uint4(m[0], m[1], m[2], m[3]);
}

__device__ __forceinline__ void store_partial(uint8_t *dst, const uint4 &v, uint32_t nbytes)
{
    const uint32_t m[4] = {v.x, v.y, v.z, v.w};
    for (uint32_t b = 0; b < nbytes; b++) dst[b] = (uint8_t)(m[b >> 2] >> (8 * (b & 3)));
}

__device__ __forceinline__ uint4 keep_bytes(const uint4 &v, uint32_t nbytes)
{
    uint32_t m[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint32_t lo = 4u * i;
        if (nbytes <= lo) m[i] = 0u;
        else if (nbytes < lo + 4) m[i] &= (1u << (8 * (nbytes - lo))) - 1u;
    }
    return make_uint4(m[0], m[1], m[2], m[3]);
}

// What a fused pass computes: full GCM (CTR keystream + GHASH), the CTR
// keystream XOR alone, or GHASH alone over the input (no AES, no output).
constexpr int MODE_GCM = 0;
constexpr int MODE_CTR = 1;
constexpr int MODE_GHASH = 2;
// Full GCM plus the FITS DATASUM of the ciphertext side: the 32-bit ones'
// complement sum of the payload as big-endian words (zero-padded to a word),
// taken over the same blocks GHASH hashes, so it costs no extra load.
constexpr int MODE_GCM_SUM = 3;

// Sum of the four big-endian 32-bit words of a 16-byte block.
__device__ __forceinline__ uint64_t word_sum_be(const uint4 &x)
{
    return (uint64_t)bswap32(x.x) + bswap32(x.y) + (uint64_t)bswap32(x.z) + bswap32(x.w);
}

// Folds a 64-bit sum of 32-bit words into their 32-bit ones' complement sum
// (end-around carry): the result is 0 only for a zero sum, else the sum
// mod 2^32 - 1 with 0xFFFFFFFF standing for a nonzero multiple.
__device__ __forceinline__ uint32_t ones_fold(uint64_t s)
{
    while (s >> 32) s = (s & 0xFFFFFFFFull) + (s >> 32);
    return (uint32_t)s;
}

// Everything a tile needs to know about its message.
struct MsgView {
    const uint8_t *in;
    uint8_t *out;
    const uint8_t *aad;
    uint64_t len, aad_len, a_blocks, n_full, M, K;
    uint32_t tile_log2;
    bool dec;
    const KeyMat *km;
    const MsgMat *mm;
    gf128 *partials;
    uint32_t *dsums;  // per-tile DATASUM partials (MODE_GCM_SUM)
};

// Per-message constants of AES round 1: everything except the lookups of
// counter bytes 12..15 (K0 misses byte 15, K1..K3 bytes 14, 13, 12).
struct MsgConst {
    uint32_t j0w0, j0w1, j0w2, ctr0, rk3, k15, K0, K1, K2, K3;
};

__device__ __forceinline__ MsgConst make_msg_const(const uint8_t *t01, const uint8_t *t23, const LaneConst &L,
                                                   const KeyMat *km, uint32_t j0w0, uint32_t j0w1, uint32_t j0w2,
                                                   uint32_t j0w3)
{
    MsgConst c;
    c.j0w0 = j0w0;
    c.j0w1 = j0w1;
    c.j0w2 = j0w2;
    c.ctr0 = bswap32(j0w3);
    const uint32_t x0 = c.j0w0 ^ __ldg(&km->rk[0]);
    const uint32_t x1 = c.j0w1 ^ __ldg(&km->rk[1]);
    const uint32_t x2 = c.j0w2 ^ __ldg(&km->rk[2]);
    c.rk3 = __ldg(&km->rk[3]);
    c.K0 = LT0(x0, 0) ^ LT1(x1, 1) ^ LT2(x2, 2) ^ __ldg(&km->rk[4]);
    c.K1 = LT0(x1, 0) ^ LT1(x2, 1) ^ LT3(x0, 3) ^ __ldg(&km->rk[5]);
    c.K2 = LT0(x2, 0) ^ LT2(x0, 2) ^ LT3(x1, 3) ^ __ldg(&km->rk[6]);
    c.K3 = LT1(x0, 1) ^ LT2(x1, 2) ^ LT3(x2, 3) ^ __ldg(&km->rk[7]);
    c.k15 = c.rk3 >> 24;
    return c;
}

// Stages the replicated round tables into shared memory.
__device__ __forceinline__ void stage_round_tables(uint8_t *smem, const DevTables *tabs)
{
    // Row v of a region holds T_even[v] for the 32 lanes, then T_odd[v]:
    // 16 vectors of four equal words.
    const uint32_t *tt = tabs->ttab;
    uint4 *s128 = reinterpret_cast<uint4 *>(smem);
#pragma unroll 4
    for (int q = threadIdx.x; q < 8192; q += blockDim.x) {
        const int region = q >> 12, v = (q >> 4) & 255, odd = (q >> 3) & 1;
        const uint32_t t = __ldg(&tt[(2 * region + odd) * 256 + v]);
        s128[q] = make_uint4(t, t, t, t);
    }
}

__device__ __forceinline__ void stage_ghash_table(uint8_t *smem, const KeyMat *km)
{
    const uint4 *g = km->gtab;
    uint4 *sg = reinterpret_cast<uint4 *>(smem + SM_GTAB);
    for (int i = threadIdx.x; i < GTAB_ENTRIES; i += blockDim.x) sg[i] = __ldg(&g[i]);
}

// The same for a block of NT threads with every load of a thread in flight
// before its first store: one memory round trip per staging instead of one
// per entry (the batched kernel restages at every change of message).
template <int NT>
__device__ __forceinline__ void stage_ghash_table_in_flight(uint8_t *smem, const KeyMat *km)
{
    constexpr int GT = GTAB_ENTRIES / NT;
    const uint4 *g = km->gtab;
    uint4 *sg = reinterpret_cast<uint4 *>(smem + SM_GTAB);
    uint4 e[GT];
#pragma unroll
    for (int k = 0; k < GT; k++) e[k] = __ldg(&g[threadIdx.x + k * NT]);
#pragma unroll
    for (int k = 0; k < GT; k++) sg[threadIdx.x + k * NT] = e[k];
}

// Both tables of the fused kernel (KF_THREADS threads), with every global
// load of a thread issued before its first shared-memory store, so that the
// staging costs about one memory round trip instead of one per loop trip.
__device__ __forceinline__ void stage_fused_tables(uint8_t *smem, const DevTables *tabs, const KeyMat *km)
{
    constexpr int RT = 8192 / KF_THREADS, GT = GTAB_ENTRIES / KF_THREADS;
    const uint32_t *tt = tabs->ttab;
    const uint4 *g = km->gtab;
    uint32_t w[RT];
    uint4 e[GT];
#pragma unroll
    for (int k = 0; k < RT; k++) {
        const int q = threadIdx.x + k * KF_THREADS;
        const int region = q >> 12, v = (q >> 4) & 255, odd = (q >> 3) & 1;
        w[k] = __ldg(&tt[(2 * region + odd) * 256 + v]);
    }
#pragma unroll
    for (int k = 0; k < GT; k++) e[k] = __ldg(&g[threadIdx.x + k * KF_THREADS]);
    uint4 *s128 = reinterpret_cast<uint4 *>(smem);
    uint4 *sg = reinterpret_cast<uint4 *>(smem + SM_GTAB);
#pragma unroll
    for (int k = 0; k < RT; k++) s128[threadIdx.x + k * KF_THREADS] = make_uint4(w[k], w[k], w[k], w[k]);
#pragma unroll
    for (int k = 0; k < GT; k++) sg[threadIdx.x + k * KF_THREADS] = e[k];
}

// H^((15-w) * S) for every warp w, S = 2^(tile_log2 - 4): moves a warp's
// segment partial to the tile end.  Lane 0 of each warp copies its own from
// the key material.
__device__ __forceinline__ void stage_segment_factors(uint8_t *smem, const KeyMat *km, uint32_t tile_log2)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    gf128 *segf = reinterpret_cast<gf128 *>(smem + SM_SEGF);
    if (lane == 0) segf[warp] = km->segf[tile_log2 - SEGF_MIN_LOG2][warp];
}

// Per-lane cache of the counter-group constants of AES round 2: G0..G3 for
// the lane's 256-counter group, and P0..P3, their parts that depend only on
// counter bytes 12 and 13 (and round-key words 8..11), for its 65536-counter
// group.
struct GroupCache {
    uint32_t grp, G0, G1, G2, G3;
    uint32_t grp_hi, P0, P1, P2, P3;
};

// A segment that touches the AAD or the final partial block: lane l takes
// blocks l, l + 32, ... of the segment, each with a whole AES computation
// (counter = inc32^(j+1)(J0) for payload block j), and chains them into its
// Horner accumulator (acc <- acc * H^32 xor X).  rk holds the round keys (at
// least words 12 .. 4 NR + 3).
template <int NR, int MODE>
__device__ __forceinline__ void segment_general(const uint8_t *smem, const MsgView &v, const MsgConst &c,
                                                const uint32_t *rk, const LaneConst &L, int64_t seg_lo,
                                                uint32_t seg_len, uint4 &acc, uint32_t &dlast, bool &have,
                                                uint64_t &dsum)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint8_t *t01 = smem + SM_T01;
    const uint8_t *t23 = smem + SM_T23;
    const KeyMat *km = v.km;
    uint32_t rlo[12];
#pragma unroll
    for (int i = 0; i < 12; i++) rlo[i] = __ldg(&km->rk[i]);
    for (uint32_t q = lane; q < seg_len; q += 32) {
        const uint64_t s = (uint64_t)seg_lo + q;
        uint4 x;
        if (s < v.a_blocks) {
            const uint64_t off = s * 16u;
            const uint64_t rem = v.aad_len - off;
            const uint8_t *src = v.aad + off;
            if (rem >= 16 && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0))
                x = *reinterpret_cast<const uint4 *>(src);
            else
                x = load_partial(src, rem >= 16 ? 16u : (uint32_t)rem);
        } else if (MODE == MODE_GHASH) {
            const uint64_t j = s - v.a_blocks;
            x = (j < v.n_full) ? __ldcs(reinterpret_cast<const uint4 *>(v.in) + j)
                               : load_partial(v.in + j * 16u, (uint32_t)(v.len - j * 16u));
        } else {
            const uint64_t j = s - v.a_blocks;
            const uint32_t ctr = c.ctr0 + 1u + (uint32_t)j;
            uint32_t s0 = c.j0w0 ^ rlo[0], s1 = c.j0w1 ^ rlo[1], s2 = c.j0w2 ^ rlo[2];
            uint32_t s3 = bswap32(ctr) ^ rlo[3];
            aes_round(t01, t23, L, s0, s1, s2, s3, rlo[4], rlo[5], rlo[6], rlo[7]);
            aes_round(t01, t23, L, s0, s1, s2, s3, rlo[8], rlo[9], rlo[10], rlo[11]);
            uint4 ks = aes_rounds_from3<NR>(t01, t23, L, s0, s1, s2, s3, rk);
            if (j < v.n_full) {
                const uint4 din = __ldcs(reinterpret_cast<const uint4 *>(v.in) + j);
                ks.x ^= din.x; ks.y ^= din.y; ks.z ^= din.z; ks.w ^= din.w;
                __stcs(reinterpret_cast<uint4 *>(v.out) + j, ks);
                x = v.dec ? din : ks;
            } else {
                const uint32_t nb = (uint32_t)(v.len - j * 16u);
                const uint4 din = load_partial(v.in + j * 16u, nb);
                ks.x ^= din.x; ks.y ^= din.y; ks.z ^= din.z; ks.w ^= din.w;
                const uint4 cb = keep_bytes(ks, nb);
                store_partial(v.out + j * 16u, cb, nb);
                x = v.dec ? din : cb;
            }
        }
        if (MODE != MODE_CTR) {
            uint4 m = ghash_mul_table(smem, acc, L);
            xor4(m, x);
            acc = m;
            dlast = q;
            have = true;
            if (MODE == MODE_GCM_SUM && s >= v.a_blocks) dsum += word_sum_be(x);
        }
    }
}

// One tile: Tiles of 2^tile_log2 blocks of the GHASH input sequence A||C
// are aligned to its end (the first tile is the short one; it is treated as
// the smallest tile of 2^lg >= its length blocks, left-padded with zero
// blocks).  Warp w owns segment w of the tile (S = 2^lg/16 blocks).  On
// whole-payload segments the warp walks windows of 32 blocks from the
// segment start (no partial windows).  Rounds 1 and 2 of AES need only the
// lookups that depend on the counter's low byte (counter-mode caching): the
// rest are per-lane constants of the lane's 256-counter group, refreshed
// when its counter enters a new group.  Lane l chains the
// l-th block of every window through acc <- acc*H^32 xor X and closes the
// chain with H^e, e = distance of its last block from the segment end; the
// warp's partial then moves to the tile end with H^((15-w)*S) and the CTA
// reduces the 16 warp partials into v.partials[tile].
// Needs the round tables, the message's GHASH table and segment factors in
// shared memory; contains two __syncthreads.
template <int NR, int MODE = MODE_GCM>
__device__ __forceinline__ void tile_body(uint8_t *smem, const MsgView &v, const MsgConst &c, const uint32_t *rk,
                                          const LaneConst &L, uint64_t tile, GroupCache &gc)
{
    const uint32_t lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint8_t *t01 = smem + SM_T01;
    const uint8_t *t23 = smem + SM_T23;
    const KeyMat *km = v.km;
    const gf128 *segf = reinterpret_cast<const gf128 *>(smem + SM_SEGF);
    gf128 *red = reinterpret_cast<gf128 *>(smem + SM_RED);
    const int64_t tend = (int64_t)v.M - (int64_t)((v.K - 1 - tile) << v.tile_log2);
    // The first tile is the short one.  It is laid out as the smallest tile
    // size 2^lg (lg >= SEGF_MIN_LOG2) that holds it, so that all warps share
    // its blocks; its end, and so its partial, is the same at any size.
    uint32_t lg = v.tile_log2;
    if (tile == 0)
        while (lg > (uint32_t)SEGF_MIN_LOG2 && ((int64_t)1 << (lg - 1)) >= tend) lg--;
    const int64_t seg_blocks = (int64_t)1 << (lg - KF_LOG2_WARPS);
    const int64_t tv_lo = tend - ((int64_t)1 << lg);
    const int64_t seg_hi = tv_lo + (int64_t)(warp + 1) * seg_blocks;
    int64_t seg_lo = tv_lo + (int64_t)warp * seg_blocks;
    if (seg_lo < 0) seg_lo = 0;
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
    uint32_t dlast = 0;
    bool have = false;
    uint32_t seg_len = 0;
    uint64_t dsum = 0;  // MODE_GCM_SUM: this lane's word sum (< 2^45 per tile)
#if GH_IMAD_WARPS > 0
    // Measured alternative (off by default): the last GH_IMAD_WARPS warps
    // multiply their Horner chains by H^32 with the integer-product field
    // multiply instead of the shared-memory table, to move GHASH work off the
    // shared-memory pipe onto the logic and multiply pipes.  Bit-exact, but
    // slower at every warp count tried.
    const bool imad = (MODE == MODE_GCM || MODE == MODE_GCM_SUM) && warp >= KF_WARPS - GH_IMAD_WARPS;
    bool poly = false;
    gf128 accp = gf_zero(), h32 = gf_zero();
    if (imad) {
        const uint4 g = __ldg(reinterpret_cast<const uint4 *>(&km->h2k[GH_LOG2_STRIDE]));
        h32.w[0] = g.x; h32.w[1] = g.y; h32.w[2] = g.z; h32.w[3] = g.w;
    }
#endif

    if (seg_hi > seg_lo) {
        seg_len = (uint32_t)(seg_hi - seg_lo);
        if ((uint64_t)seg_lo >= v.a_blocks && (uint64_t)seg_hi <= v.a_blocks + v.n_full) {
            // Whole payload blocks: windows of 32 from the segment start.
            const uint64_t j_lo = (uint64_t)seg_lo - v.a_blocks;
            const uint32_t c_lo = c.ctr0 + 1u + (uint32_t)j_lo;
            const uint32_t nwin = (seg_len + 31u) >> 5;
            const uint4 *in = reinterpret_cast<const uint4 *>(v.in) + j_lo;
            uint4 *out = reinterpret_cast<uint4 *>(v.out) + j_lo;
            // The next window's input is loaded one window ahead, so a load's
            // latency (long when the payload is in host memory across the
            // CPU-GPU link) overlaps a window of AES work.
            uint4 din_next = make_uint4(0u, 0u, 0u, 0u);
            if (lane < seg_len) din_next = __ldcs(in + lane);
            for (uint32_t wi = 0; wi < nwin; wi++) {
                const uint32_t d = (wi << 5) + lane;
                const bool active = d < seg_len;
                // This lane's counter word (inc32 arithmetic: wraps mod 2^32).
                const uint32_t ctr = c_lo + d;
                const uint4 din = din_next;
                const uint32_t dn = d + 32u;
                if (dn < seg_len) din_next = __ldcs(in + dn);
                if (MODE == MODE_GHASH) {
                    if (active) {
                        uint4 m = ghash_mul_table(smem, acc, L);
                        xor4(m, din);
                        acc = m;
                        dlast = d;
                        have = true;
                    }
                    continue;
                }
                if ((ctr >> 8) != gc.grp) {
                    // Per-group constants of rounds 1-2 (counter bytes 12..14
                    // fixed).  A window that straddles a 256-counter boundary
                    // refreshes only the lanes past it (the others refresh one
                    // window later): two divergent refreshes per 8 windows.
                    // Between consecutive groups only counter byte 14 (u1)
                    // changes, so the terms of bytes 12 and 13 (u2, u3) are
                    // kept in P0..P3 and rebuilt once per 65536 counters.
                    gc.grp = ctr >> 8;
                    const uint32_t x3g = bswap32(ctr) ^ c.rk3;
                    if ((ctr >> 16) != gc.grp_hi) {
                        gc.grp_hi = ctr >> 16;
                        const uint32_t u2 = c.K2 ^ LT1(x3g, 1);
                        const uint32_t u3 = c.K3 ^ LT0(x3g, 0);
                        gc.P0 = LT2(u2, 2) ^ LT3(u3, 3) ^ __ldg(&km->rk[8]);
                        gc.P1 = LT1(u2, 1) ^ LT2(u3, 2) ^ __ldg(&km->rk[9]);
                        gc.P2 = LT0(u2, 0) ^ LT1(u3, 1) ^ __ldg(&km->rk[10]);
                        gc.P3 = LT0(u3, 0) ^ LT3(u2, 3) ^ __ldg(&km->rk[11]);
                    }
                    const uint32_t u1 = c.K1 ^ LT2(x3g, 2);
                    gc.G0 = gc.P0 ^ LT1(u1, 1);
                    gc.G1 = gc.P1 ^ LT0(u1, 0);
                    gc.G2 = gc.P2 ^ LT3(u1, 3);
                    gc.G3 = gc.P3 ^ LT2(u1, 2);
                }
                // Round 1 column 0 (the only column that sees counter byte 15),
                // then round 2 (one varying lookup per column).
                const uint32_t x15 = (ctr & 0xFFu) ^ c.k15;
                const uint32_t v0 = c.K0 ^ LT3(x15, 0);
                uint4 ks = aes_rounds_from3<NR>(t01, t23, L, gc.G0 ^ LT0(v0, 0), gc.G1 ^ LT3(v0, 3),
                                                gc.G2 ^ LT2(v0, 2), gc.G3 ^ LT1(v0, 1), rk);
                if (active) {
                    ks.x ^= din.x; ks.y ^= din.y; ks.z ^= din.z; ks.w ^= din.w;
                    __stcs(out + d, ks);
                    if (MODE == MODE_GCM || MODE == MODE_GCM_SUM) {
                        const uint4 x = v.dec ? din : ks;
#if GH_IMAD_WARPS > 0
                        if (imad) {
                            accp = gf_xor(gf_mul(accp, h32), gf_from_mem(x.x, x.y, x.z, x.w));
                            poly = true;
                        } else
#endif
                        {
                            uint4 m = ghash_mul_table(smem, acc, L);
                            xor4(m, x);
                            acc = m;
                        }
                        dlast = d;
                        have = true;
                        if (MODE == MODE_GCM_SUM) dsum += word_sum_be(x);
                    }
                }
            }
        } else {
            // Segments that touch the AAD or the final partial block.
            segment_general<NR, MODE>(smem, v, c, rk, L, seg_lo, seg_len, acc, dlast, have, dsum);
        }
    }
    if (MODE == MODE_CTR) return;  // no authenticator: nothing to reduce

    // Close the lane's chain (its last block is e = seg_len - dlast blocks
    // before the segment end, 1 <= e <= 32), reduce the warp, move the
    // warp's partial to the tile end, reduce the CTA.
    gf128 z = gf_zero();
#if GH_IMAD_WARPS > 0
    if (have && poly) z = gf_mul(accp, km->hpow[seg_len - dlast - 1]);
    else
#endif
    if (have) z = gf_mul(gf_from_mem(acc.x, acc.y, acc.z, acc.w), km->hpow[seg_len - dlast - 1]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < 4; k++) z.w[k] ^= __shfl_xor_sync(0xFFFFFFFFu, z.w[k], off);
    // Every lane holds the warp's sum z; the whole warp multiplies it by the
    // segment factor (warp-uniform branch).
    if (warp != KF_WARPS - 1) {
        // The staged factor, or for a first tile laid out smaller the one of
        // its size from the key material.
        gf128 f = segf[warp];
        if (lg != v.tile_log2) {
            const uint4 g = __ldg(reinterpret_cast<const uint4 *>(&km->segf[lg - SEGF_MIN_LOG2][warp]));
            f.w[0] = g.x; f.w[1] = g.y; f.w[2] = g.z; f.w[3] = g.w;
        }
        z = gf_mul_warp(z, f, reinterpret_cast<uint64_t *>(smem + SM_WSCR) + 16 * warp);
    }
    if (lane == 0) red[warp] = z;
    uint64_t *dred = reinterpret_cast<uint64_t *>(smem + SM_DSUM);
    if (MODE == MODE_GCM_SUM) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) dsum += __shfl_xor_sync(0xFFFFFFFFu, dsum, off);
        if (lane == 0) dred[warp] = dsum;
    }
    __syncthreads();
    if (warp == 0) {
        z = (lane < KF_WARPS) ? red[lane] : gf_zero();
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < 4; k++) z.w[k] ^= __shfl_xor_sync(0xFFFFFFFFu, z.w[k], off);
        if (lane == 0) v.partials[tile] = z;
        if (MODE == MODE_GCM_SUM) {
            dsum = (lane < KF_WARPS) ? dred[lane] : 0ull;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) dsum += __shfl_xor_sync(0xFFFFFFFFu, dsum, off);
            if (lane == 0) v.dsums[tile] = ones_fold(dsum);
        }
    }
    __syncthreads();
}

// E_K(J0) through the replicated round tables in shared memory (every lane
// of the calling warp computes the same block; each reads its own bank).
// rk holds round-key words 12 .. 4 NR + 3.
template <int NR>
__device__ __forceinline__ uint4 aes_block_smem(const uint8_t *smem, const LaneConst &L, const KeyMat *km,
                                                const uint32_t *rk, const uint32_t j0[4])
{
    const uint8_t *t01 = smem + SM_T01;
    const uint8_t *t23 = smem + SM_T23;
    uint32_t s0 = j0[0] ^ __ldg(&km->rk[0]), s1 = j0[1] ^ __ldg(&km->rk[1]);
    uint32_t s2 = j0[2] ^ __ldg(&km->rk[2]), s3 = j0[3] ^ __ldg(&km->rk[3]);
    aes_round(t01, t23, L, s0, s1, s2, s3, __ldg(&km->rk[4]), __ldg(&km->rk[5]), __ldg(&km->rk[6]),
              __ldg(&km->rk[7]));
    aes_round(t01, t23, L, s0, s1, s2, s3, __ldg(&km->rk[8]), __ldg(&km->rk[9]), __ldg(&km->rk[10]),
              __ldg(&km->rk[11]));
    return aes_rounds_from3<NR>(t01, t23, L, s0, s1, s2, s3, rk);
}

// The reduce phase of a message with few tiles, run by the last CTA of the
// fused launch to finish (Sec. 5.2.2; the same tree, length block, tag and
// verify gate as the separate combine kernel, without its launch):
//   * warp 0 computes E_K(J0) from the round tables still in shared memory;
//   * the K <= FINISH_MAX_TILES tile partials (written by every CTA before
//     its ticket) are staged into shared memory over the round tables, and
//     reduced level by level with Combine(L, R) = L * H^(2^(lg + level)) xor
//     R, R read from the end of the sequence (the tiles are end-aligned, so
//     every right operand is a full group of 2^level tiles);
//   * GHASH = (P xor [len A]_64 || [len C]_64) * H, T = E_K(J0) xor GHASH;
//     decryption compares T with the expected tag in constant time and, on a
//     mismatch, zero-fills the whole payload before the kernel ends.
// Kept out of line so that it does not take registers from the tile loop.
template <int NR, int MODE>
__device__ __noinline__ void finish_message(uint8_t *smem, const KfParams &p)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = blockDim.x >> 5;
    const KeyMat *km = p.km;
    uint32_t *sej0 = reinterpret_cast<uint32_t *>(smem + SM_RED);
    int32_t *sfail = reinterpret_cast<int32_t *>(smem + SM_RED + 16);
    // The reduce's buffers take the place of the GHASH table (no longer
    // read), so the last warp can compute E_K(J0) from the round tables while
    // the other warps stage the partials and H.
    gf128 *sgrp = reinterpret_cast<gf128 *>(smem + SM_GTAB);  // group sums, then G
    gf128 *spart = reinterpret_cast<gf128 *>(smem + SM_GTAB + 16 * FINISH_MAX_TILES);
    gf128 *sH = reinterpret_cast<gf128 *>(smem + SM_GTAB + 32 * FINISH_MAX_TILES);
    uint64_t *wscr = reinterpret_cast<uint64_t *>(smem + SM_WSCR) + 16 * warp;
    const uint64_t K = p.K;
    if (warp == nwarps - 1) {
        uint4 e = make_uint4(0u, 0u, 0u, 0u);
        if (MODE != MODE_GHASH) {
            if (p.j0_given) {
                uint32_t rk[4 * (NR + 1)];
#pragma unroll
                for (int i = 12; i < 4 * (NR + 1); i++) rk[i] = __ldg(&km->rk[i]);
                e = aes_block_smem<NR>(smem, make_lane_const(lane), km, rk, p.j0);
            } else {
                e.x = __ldg(&p.mm->ej0[0]);
                e.y = __ldg(&p.mm->ej0[1]);
                e.z = __ldg(&p.mm->ej0[2]);
                e.w = __ldg(&p.mm->ej0[3]);
            }
        }
        if (lane == 0) {
            sej0[0] = e.x; sej0[1] = e.y; sej0[2] = e.z; sej0[3] = e.w;
            *sfail = 0;
        }
    } else {
        for (uint64_t i = t; i < K; i += blockDim.x - 32)
            for (int k = 0; k < 4; k++) spart[i].w[k] = __ldcg(&p.partials[i].w[k]);
        if (t == 0) *sH = km->H;
    }
    __syncthreads();
    // Flat reduce: with g = K - 1 - i the distance of partial i from the last
    // tile, G = sum_g P_i * H^(2^lg g) = sum_q (sum_j P * w1[j]) * w2[q]
    // (g = 32 q + j): one product per partial, a warp XOR, one product per
    // group of 32.  Thread t handles g = t and g = t + 512 (K <= 1024).
    const int sz = (int)p.tile_log2 - SEGF_MIN_LOG2;
    for (int pass = 0; pass < (int)((FINISH_MAX_TILES + blockDim.x - 1) / blockDim.x); pass++) {
        const uint64_t g = (uint64_t)t + (uint64_t)pass * blockDim.x;
        gf128 u = gf_zero();
        if (g < K) u = gf_mul(spart[K - 1 - g], p.fin->w1[sz][g & 31]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < 4; k++) u.w[k] ^= __shfl_xor_sync(0xFFFFFFFFu, u.w[k], off);
        if (lane == 0 && (g >> 5) < 32) sgrp[g >> 5] = u;  // the warp of g holds group g / 32
    }
    __syncthreads();
    const uint64_t ngrp = (K + 31) / 32;
    gf128 G = gf_zero();  // meaningful in warp 0
    if (warp == 0) {
        if ((uint64_t)lane < ngrp) G = gf_mul(sgrp[lane], p.fin->w2[sz][lane]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < 4; k++) G.w[k] ^= __shfl_xor_sync(0xFFFFFFFFu, G.w[k], off);
    }
    if (MODE == MODE_GCM_SUM) {
        uint64_t *dred = reinterpret_cast<uint64_t *>(smem + SM_DSUM);
        uint64_t acc = 0;
        for (uint64_t i = t; i < K; i += blockDim.x) acc += __ldcg(&p.dsums[i]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
        if (lane == 0) dred[warp] = acc;
        __syncthreads();
        if (t == 0) {
            uint64_t tot = 0;
            for (int w = 0; w < nwarps; w++) tot += dred[w];
            *p.datasum_out = ones_fold(tot);
        }
    }
    if (warp == 0) {
        gf128 lb;
        const uint64_t abits = p.aad_len * 8u, cbits = p.len * 8u;
        lb.w[0] = (uint32_t)(abits >> 32);
        lb.w[1] = (uint32_t)abits;
        lb.w[2] = (uint32_t)(cbits >> 32);
        lb.w[3] = (uint32_t)cbits;
        const gf128 gh = gf_mul_warp(gf_xor(G, lb), *sH, wscr);
        if (lane == 0) {
            const uint4 gm = gf_to_mem(gh);
            const uint32_t tw[4] = {gm.x ^ sej0[0], gm.y ^ sej0[1], gm.z ^ sej0[2], gm.w ^ sej0[3]};
            if (p.tag_out)
                for (int b = 0; b < 16; b++) p.tag_out[b] = (uint8_t)(tw[b >> 2] >> (8 * (b & 3)));
            if (p.tag_expected) {
                uint32_t diff = 0;
                for (int b = 0; b < 16; b++)
                    diff |= (uint32_t)((uint8_t)(tw[b >> 2] >> (8 * (b & 3))) ^ p.tag_expected[b]);
                if (p.status) *p.status = diff ? -3 : 0;
                *sfail = diff ? 1 : 0;
            } else if (p.status) {
                *p.status = 0;
            }
        }
    }
    __syncthreads();
    if (*sfail) {
        // Payload suppression: the whole output is zeroed before the kernel
        // ends (messages on this path hold at most FINISH_MAX_BLOCKS blocks).
        const uint64_t nvec = p.len / 16;
        uint4 *o = reinterpret_cast<uint4 *>(p.out);
        for (uint64_t i = t; i < nvec; i += blockDim.x) o[i] = make_uint4(0u, 0u, 0u, 0u);
        if (t < (int)(p.len & 15)) p.out[nvec * 16 + t] = 0;
    }
}

// KF: one message, tiles [tile_begin, tile_end) over a persistent grid.
template <int NR, int MODE = MODE_GCM>
__global__ void __launch_bounds__(KF_THREADS, 1) fused_kernel(const __grid_constant__ KfParams p)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint8_t *t01 = smem + SM_T01;
    const uint8_t *t23 = smem + SM_T23;
    stage_fused_tables(smem, p.tabs, p.km);
    stage_segment_factors(smem, p.km, p.tile_log2);
    uint32_t rk[4 * (NR + 1)];
#pragma unroll
    for (int i = 12; i < 4 * (NR + 1); i++) rk[i] = __ldg(&p.km->rk[i]);
    const LaneConst L = make_lane_const((int)(threadIdx.x & 31));
    MsgView v;
    v.in = p.in;
    v.out = p.out;
    v.aad = p.aad;
    v.len = p.len;
    v.aad_len = p.aad_len;
    v.a_blocks = p.a_blocks;
    v.n_full = p.n_full;
    v.M = p.M;
    v.K = p.K;
    v.tile_log2 = p.tile_log2;
    v.dec = p.decrypt != 0;
    v.km = p.km;
    v.mm = p.mm;
    v.partials = p.partials;
    v.dsums = p.dsums;
    __syncthreads();
    const MsgConst c = p.j0_given ? make_msg_const(t01, t23, L, p.km, p.j0[0], p.j0[1], p.j0[2], p.j0[3])
                                  : make_msg_const(t01, t23, L, p.km, __ldg(&p.mm->j0[0]), __ldg(&p.mm->j0[1]),
                                                   __ldg(&p.mm->j0[2]), __ldg(&p.mm->j0[3]));
    GroupCache gc;
    gc.grp = gc.grp_hi = 0xFFFFFFFFu;  // no counter group matches (ctr >> 8 < 2^24)
    gc.G0 = gc.G1 = gc.G2 = gc.G3 = 0u;
    gc.P0 = gc.P1 = gc.P2 = gc.P3 = 0u;
    for (uint64_t tile = p.tile_begin + blockIdx.x; tile < p.tile_end; tile += gridDim.x)
        tile_body<NR, MODE>(smem, v, c, rk, L, tile, gc);
    if (MODE != MODE_CTR && p.ticket) {
        // Thread 0 wrote this CTA's partials (tile_body ends with a barrier);
        // make them visible device-wide, then take a ticket.  atomicInc wraps
        // the counter back to 0 on the last ticket, so the word is ready for
        // the next launch on the same stream.
        __shared__ int s_last;
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = (atomicInc(p.ticket, gridDim.x - 1) == gridDim.x - 1) ? 1 : 0;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            finish_message<NR, MODE>(smem, p);
        }
    }
}

// ---------------------------------------------------------------------
// KF, bitsliced: the same tiles, segments and GHASH chains, with the CTR
// keystream of whole-payload segments computed by bitsliced AES
// ---------------------------------------------------------------------
// A warp walks a whole-payload segment in windows of 1024 blocks from the
// segment start; lane l holds blocks l, l + 32, ..., l + 992 of a window as
// one bitsliced state (block k of the lane = bit k of every word), so the
// lane's blocks are exactly the next 32 links of its stride-32 Horner chain.
// Counters come from the segment's first counter (inc32 arithmetic, any
// alignment); they are transposed into bytes 12..15 of the state.  After the
// rounds the state is transposed back to 32 blocks of four memory words,
// which are xored with the input, stored and hashed in chain order.
// Segments touching the AAD or the final partial block use the table path.
// Each of the 8 warps walks segments w and w + 8 of the tile.
template <int NR, int MODE>
__device__ __forceinline__ void tile_body_bs(uint8_t *smem, const MsgView &v, const MsgConst &c, const LaneConst &L,
                                             uint64_t tile)
{
    const uint32_t lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const KeyMat *km = v.km;
    const uint32_t *kbs = reinterpret_cast<const uint32_t *>(smem + SM_KBS);
    const gf128 *segf = reinterpret_cast<const gf128 *>(smem + SM_SEGF);
    gf128 *red = reinterpret_cast<gf128 *>(smem + SM_RED);
    const int64_t tend = (int64_t)v.M - (int64_t)((v.K - 1 - tile) << v.tile_log2);
    uint32_t lg = v.tile_log2;
    if (tile == 0)
        while (lg > (uint32_t)SEGF_MIN_LOG2 && ((int64_t)1 << (lg - 1)) >= tend) lg--;
    const int64_t seg_blocks = (int64_t)1 << (lg - KF_LOG2_WARPS);
    const int64_t tv_lo = tend - ((int64_t)1 << lg);
    gf128 zw = gf_zero();
    uint64_t dsum = 0;

    for (int sw = warp; sw < KF_WARPS; sw += nwarps) {
        const int64_t seg_hi = tv_lo + (int64_t)(sw + 1) * seg_blocks;
        int64_t seg_lo = tv_lo + (int64_t)sw * seg_blocks;
        if (seg_lo < 0) seg_lo = 0;
        uint4 acc = make_uint4(0u, 0u, 0u, 0u);
        uint32_t dlast = 0, seg_len = 0;
        bool have = false;
        if (seg_hi > seg_lo) {
            seg_len = (uint32_t)(seg_hi - seg_lo);
            if ((uint64_t)seg_lo >= v.a_blocks && (uint64_t)seg_hi <= v.a_blocks + v.n_full) {
                const uint64_t j_lo = (uint64_t)seg_lo - v.a_blocks;
                const uint32_t c_lo = c.ctr0 + 1u + (uint32_t)j_lo;
                const uint4 *in = reinterpret_cast<const uint4 *>(v.in) + j_lo;
                uint4 *out = reinterpret_cast<uint4 *>(v.out) + j_lo;
                for (uint32_t base = 0; base < seg_len; base += 1024u) {
                    uint32_t s[128];
                    {
                        uint32_t ctr[32];
#pragma unroll
                        for (int k = 0; k < 32; k++) ctr[k] = c_lo + base + lane + 32u * (uint32_t)k;
                        load_counters_bs(s, c.j0w0, c.j0w1, c.j0w2, ctr, kbs);
                    }
                    aes_rounds_bs<NR>(s, kbs);
                    unload_blocks_bs(s);
#pragma unroll
                    for (int k = 0; k < 32; k++) {
                        const uint32_t d = base + lane + 32u * (uint32_t)k;
                        if (d < seg_len) {
                            const uint4 din = __ldcs(in + d);
                            const uint4 ks = make_uint4(s[k] ^ din.x, s[32 + k] ^ din.y, s[64 + k] ^ din.z,
                                                        s[96 + k] ^ din.w);
                            __stcs(out + d, ks);
                            if (MODE == MODE_GCM || MODE == MODE_GCM_SUM) {
                                const uint4 x = v.dec ? din : ks;
                                uint4 m = ghash_mul_table(smem, acc, L);
                                xor4(m, x);
                                acc = m;
                                dlast = d;
                                have = true;
                                if (MODE == MODE_GCM_SUM) dsum += word_sum_be(x);
                            }
                        }
                    }
                }
            } else {
                segment_general<NR, MODE>(smem, v, c, km->rk, L, seg_lo, seg_len, acc, dlast, have, dsum);
            }
        }
        if (MODE != MODE_CTR) {
            // Close the lane chains, reduce the warp, move the segment's
            // partial to the tile end and add it to the warp's sum.
            gf128 z = gf_zero();
            if (have) z = gf_mul(gf_from_mem(acc.x, acc.y, acc.z, acc.w), km->hpow[seg_len - dlast - 1]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int k = 0; k < 4; k++) z.w[k] ^= __shfl_xor_sync(0xFFFFFFFFu, z.w[k], off);
            if (sw != KF_WARPS - 1) {
                gf128 f = segf[sw];
                if (lg != v.tile_log2) {
                    const uint4 g = __ldg(reinterpret_cast<const uint4 *>(&km->segf[lg - SEGF_MIN_LOG2][sw]));
                    f.w[0] = g.x; f.w[1] = g.y; f.w[2] = g.z; f.w[3] = g.w;
                }
                z = gf_mul_warp(z, f, reinterpret_cast<uint64_t *>(smem + SM_WSCR) + 16 * warp);
            }
            zw = gf_xor(zw, z);
        }
    }
    if (MODE == MODE_CTR) return;  // no authenticator: nothing to reduce
    if (lane == 0) red[warp] = zw;
    uint64_t *dred = reinterpret_cast<uint64_t *>(smem + SM_DSUM);
    if (MODE == MODE_GCM_SUM) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) dsum += __shfl_xor_sync(0xFFFFFFFFu, dsum, off);
        if (lane == 0) dred[warp] = dsum;
    }
    __syncthreads();
    if (warp == 0) {
        gf128 z = (lane < (uint32_t)nwarps) ? red[lane] : gf_zero();
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < 4; k++) z.w[k] ^= __shfl_xor_sync(0xFFFFFFFFu, z.w[k], off);
        if (lane == 0) v.partials[tile] = z;
        if (MODE == MODE_GCM_SUM) {
            dsum = (lane < (uint32_t)nwarps) ? dred[lane] : 0ull;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) dsum += __shfl_xor_sync(0xFFFFFFFFu, dsum, off);
            if (lane == 0) v.dsums[tile] = ones_fold(dsum);
        }
    }
    __syncthreads();
}

template <int NR, int MODE>
__global__ void __launch_bounds__(KBS_THREADS, 1) fused_bs_kernel(const __grid_constant__ KfParams p)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint8_t *t01 = smem + SM_T01;
    const uint8_t *t23 = smem + SM_T23;
    stage_round_tables(smem, p.tabs);
    if (MODE != MODE_CTR) stage_ghash_table(smem, p.km);
    if (threadIdx.x < KF_WARPS)
        reinterpret_cast<gf128 *>(smem + SM_SEGF)[threadIdx.x] =
            p.km->segf[p.tile_log2 - SEGF_MIN_LOG2][threadIdx.x];
    uint32_t *kbs = reinterpret_cast<uint32_t *>(smem + SM_KBS);
    for (int q = threadIdx.x; q < 128 * (NR + 1); q += blockDim.x) kbs[q] = round_key_word_bs(p.km->rk, q);
    const LaneConst L = make_lane_const((int)(threadIdx.x & 31));
    MsgView v;
    v.in = p.in;
    v.out = p.out;
    v.aad = p.aad;
    v.len = p.len;
    v.aad_len = p.aad_len;
    v.a_blocks = p.a_blocks;
    v.n_full = p.n_full;
    v.M = p.M;
    v.K = p.K;
    v.tile_log2 = p.tile_log2;
    v.dec = p.decrypt != 0;
    v.km = p.km;
    v.mm = p.mm;
    v.partials = p.partials;
    v.dsums = p.dsums;
    __syncthreads();
    const MsgConst c = p.j0_given ? make_msg_const(t01, t23, L, p.km, p.j0[0], p.j0[1], p.j0[2], p.j0[3])
                                  : make_msg_const(t01, t23, L, p.km, __ldg(&p.mm->j0[0]), __ldg(&p.mm->j0[1]),
                                                   __ldg(&p.mm->j0[2]), __ldg(&p.mm->j0[3]));
    for (uint64_t tile = p.tile_begin + blockIdx.x; tile < p.tile_end; tile += gridDim.x)
        tile_body_bs<NR, MODE>(smem, v, c, L, tile);
}

// ---------------------------------------------------------------------
// KB: many messages in one persistent launch
// ---------------------------------------------------------------------
template <int NR>
__device__ __forceinline__ void batch_tile(uint8_t *smem, const MsgView &v, const LaneConst &L, uint64_t tile,
                                        GroupCache &gc)
{
    const uint8_t *t01 = smem + SM_T01;
    const uint8_t *t23 = smem + SM_T23;
    uint32_t rk[4 * (NR + 1)];
#pragma unroll
    for (int i = 12; i < 4 * (NR + 1); i++) rk[i] = __ldg(&v.km->rk[i]);
    const MsgConst c = make_msg_const(t01, t23, L, v.km, __ldg(&v.mm->j0[0]), __ldg(&v.mm->j0[1]),
                                      __ldg(&v.mm->j0[2]), __ldg(&v.mm->j0[3]));
    tile_body<NR>(smem, v, c, rk, L, tile, gc);
}

// The CTA that finishes a message's last tile combines its partials (the
// same right-to-left tree as combine_kernel, inside one CTA) and writes the
// tag, or the verdict for decryption.
// Levels with few products give each product to a whole warp
// (gf_mul_warp, scratch in smem at SM_WSCR), which has a much shorter
// latency than one thread's multiply; so does the tag's product.
__device__ void batch_combine(uint8_t *smem, const BatchMsg &m, bool dec)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = blockDim.x >> 5;
    uint64_t *wscr = reinterpret_cast<uint64_t *>(smem + SM_WSCR) + 16 * warp;
    uint64_t cnt = m.K;
    int level = 0;
    gf128 *src = m.partials;
    gf128 *dst = m.tree;
    bool reversed = true;
    while (cnt > 1) {
        const uint64_t half = (cnt + 1) / 2;
        const gf128 mult = m.km->h2k[m.tile_log2 + level];
        const bool by_warp = half <= (uint64_t)nwarps * 4;
        const uint64_t first = by_warp ? (uint64_t)warp : (uint64_t)t;
        const uint64_t step = by_warp ? (uint64_t)nwarps : (uint64_t)blockDim.x;
        for (uint64_t g = first; g < half; g += step) {
            const uint64_t ri = 2 * g, li = 2 * g + 1;
            gf128 right, left;
            const gf128 *pr = reversed ? &src[cnt - 1 - ri] : &src[ri];
            for (int k = 0; k < 4; k++) right.w[k] = __ldcg(&pr->w[k]);
            gf128 val = right;
            if (li < cnt) {
                const gf128 *pl = reversed ? &src[cnt - 1 - li] : &src[li];
                for (int k = 0; k < 4; k++) left.w[k] = __ldcg(&pl->w[k]);
                val = gf_xor(by_warp ? gf_mul_warp(left, mult, wscr) : gf_mul(left, mult), right);
            }
            if (!by_warp || lane == 0)
                for (int k = 0; k < 4; k++) __stcg(&dst[g].w[k], val.w[k]);
        }
        __threadfence_block();
        __syncthreads();
        gf128 *tmp = src;
        src = dst;
        dst = tmp;
        reversed = false;
        cnt = half;
        level++;
    }
    if (warp != 0) return;
    gf128 s = gf_zero();
    if (cnt == 1)
        for (int k = 0; k < 4; k++) s.w[k] = __ldcg(&src[0].w[k]);
    gf128 lb;
    const uint64_t abits = m.aad_len * 8u, cbits = m.len * 8u;
    lb.w[0] = (uint32_t)(abits >> 32);
    lb.w[1] = (uint32_t)abits;
    lb.w[2] = (uint32_t)(cbits >> 32);
    lb.w[3] = (uint32_t)cbits;
    const gf128 gh = gf_mul_warp(gf_xor(s, lb), m.km->H, wscr);
    if (lane != 0) return;
    const uint4 gm = gf_to_mem(gh);
    const uint32_t tw[4] = {gm.x ^ m.mm->ej0[0], gm.y ^ m.mm->ej0[1], gm.z ^ m.mm->ej0[2], gm.w ^ m.mm->ej0[3]};
    uint32_t diff = 0;
    for (int b = 0; b < 16; b++) {
        const uint8_t tb = (uint8_t)(tw[b >> 2] >> (8 * (b & 3)));
        if (dec)
            diff |= (uint32_t)(tb ^ m.tag[b]);
        else
            m.tag[b] = tb;
    }
    *m.status = dec ? (diff ? -3 : 0) : 0;
    if (m.t_done) {
        uint64_t now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        *m.t_done = now;
    }
}

__global__ void __launch_bounds__(KF_THREADS, 1) batch_kernel(const __grid_constant__ BatchParams p)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t s_item;
    __shared__ uint32_t s_msg;
    __shared__ int s_last;
    stage_round_tables(smem, p.tabs);
    const LaneConst L = make_lane_const((int)(threadIdx.x & 31));
    uint32_t cur = 0xFFFFFFFFu;
    GroupCache gc;
    for (;;) {
        __syncthreads();  // previous item (and its tables) fully done
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            uint64_t item = 0;
            if (lane == 0) item = atomicAdd(p.item_counter, 1ull);
            item = __shfl_sync(0xFFFFFFFFu, item, 0);
            if (lane == 0) s_item = item;
            if (item < p.total_items) {
                // The message whose item range holds `item` (item_base is
                // strictly increasing): a 32-way search, each lane probing one
                // point of the range, so 10^4 messages take 3 rounds.
                uint32_t lo = 0, hi = p.n - 1;
                while (lo < hi) {
                    const uint32_t step = (hi - lo) / 32 + 1;
                    const uint64_t probe = (uint64_t)lo + (uint64_t)(lane + 1) * step;
                    const bool le = probe <= hi && p.msgs[probe].item_base <= item;
                    const uint32_t c = (uint32_t)__popc(__ballot_sync(0xFFFFFFFFu, le));
                    const uint64_t nhi = (uint64_t)lo + (uint64_t)(c + 1) * step - 1;
                    lo += c * step;
                    hi = nhi < hi ? (uint32_t)nhi : hi;
                }
                if (lane == 0) s_msg = lo;
            }
        }
        __syncthreads();
        const uint64_t item = s_item;
        if (item >= p.total_items) break;
        const uint32_t mi = s_msg;
        const BatchMsg &bm = p.msgs[mi];
        MsgView v;
        v.dsums = nullptr;
        v.in = bm.in;
        v.out = bm.out;
        v.aad = bm.aad;
        v.len = bm.len;
        v.aad_len = bm.aad_len;
        v.a_blocks = (bm.aad_len + 15) / 16;
        v.n_full = bm.len / 16;
        v.M = v.a_blocks + (bm.len + 15) / 16;
        v.K = bm.K;
        v.tile_log2 = bm.tile_log2;
        v.dec = bm.dec != 0;
        v.km = bm.km;
        v.mm = bm.mm;
        v.partials = bm.partials;
        if (mi != cur) {
            // New message: its key's GHASH table and segment factors.
            stage_ghash_table_in_flight<KF_THREADS>(smem, bm.km);
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            if (lane == 0)
                reinterpret_cast<gf128 *>(smem + SM_SEGF)[warp] = bm.km->segf[bm.tile_log2 - SEGF_MIN_LOG2][warp];
            cur = mi;
            gc.grp = gc.grp_hi = 0xFFFFFFFFu;  // the constants belong to the previous message
            __syncthreads();
        }
        const uint64_t tile = item - bm.item_base;
        if (bm.nr == 14)
            batch_tile<14>(smem, v, L, tile, gc);
        else if (bm.nr == 10)
            batch_tile<10>(smem, v, L, tile, gc);
        else
            batch_tile<12>(smem, v, L, tile, gc);
        // tile_body ended with __syncthreads after warp 0 lane 0 stored the
        // partial; publish it and count the message's finished tiles.
        if (threadIdx.x == 0) {
            __threadfence();
            const uint32_t prev = atomicAdd(&p.done[mi], 1u);
            s_last = (prev + 1 == (uint32_t)bm.K) ? 1 : 0;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            batch_combine(smem, bm, bm.dec != 0);
        }
    }
}

// Zero-fills the outputs of messages whose tag failed (one CTA per message).
__global__ void __launch_bounds__(256) batch_zero_kernel(const BatchMsg *msgs, uint32_t n)
{
    const uint32_t mi = blockIdx.x;
    if (mi >= n) return;
    const BatchMsg &m = msgs[mi];
    if (*m.status == 0) return;
    const uint64_t nvec = m.len / 16;
    uint4 *o = reinterpret_cast<uint4 *>(m.out);
    for (uint64_t i = threadIdx.x; i < nvec; i += blockDim.x) o[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x < (m.len & 15)) m.out[nvec * 16 + threadIdx.x] = 0;
}

// J0 and E_K(J0) of one message whose key material is already set up
// (SP 800-38D Alg. 4 step 2 and the tag's E_K(J0)); one thread.
__device__ void msg_material(const uint8_t *iv, uint32_t iv_len, const KeyMat *km, const DevTables *tabs, MsgMat *mm)
{
    uint32_t j0[4];
    if (iv_len == 12) {
        for (int i = 0; i < 3; i++)
            j0[i] = (uint32_t)iv[4 * i] | ((uint32_t)iv[4 * i + 1] << 8) | ((uint32_t)iv[4 * i + 2] << 16) |
                    ((uint32_t)iv[4 * i + 3] << 24);
        j0[3] = 0x01000000u;
    } else {
        const gf128 H = km->H;
        gf128 y = gf_zero();
        for (uint32_t off = 0; off < iv_len; off += 16) {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            for (uint32_t b = 0; b < 16 && off + b < iv_len; b++) w[b >> 2] |= (uint32_t)iv[off + b] << (8 * (b & 3));
            y = gf_mul(gf_xor(y, gf_from_mem(w[0], w[1], w[2], w[3])), H);
        }
        gf128 lb = gf_zero();
        const uint64_t bits = (uint64_t)iv_len * 8u;
        lb.w[2] = (uint32_t)(bits >> 32);
        lb.w[3] = (uint32_t)bits;
        y = gf_mul(gf_xor(y, lb), H);
        const uint4 jm = gf_to_mem(y);
        j0[0] = jm.x; j0[1] = jm.y; j0[2] = jm.z; j0[3] = jm.w;
    }
    uint32_t e[4];
    aes_block_tt(km->rk, (int)km->nr, tabs->ttab, tabs->sbox, j0, e);
    for (int i = 0; i < 4; i++) {
        mm->j0[i] = j0[i];
        mm->ej0[i] = e[i];
    }
}

// Batched form: one thread per message.
__global__ void __launch_bounds__(128) msg_setup_kernel(const BatchMsg *msgs, const BatchKey *keys, uint32_t n,
                                                        const DevTables *tabs)
{
    const uint32_t mi = blockIdx.x * blockDim.x + threadIdx.x;
    if (mi >= n) return;
    msg_material(keys[mi].iv, keys[mi].iv_len, msgs[mi].km, tabs, msgs[mi].mm);
}

// Single-message form for cached key material (one warp).
__global__ void __launch_bounds__(32) msg_only_kernel(const __grid_constant__ KsParams p)
{
    if (threadIdx.x != 0) return;
    const uint8_t *iv = (p.iv_len <= IV_INLINE_MAX) ? p.iv_inline : p.iv_dev;
    msg_material(iv, p.iv_len, p.km, p.tabs, p.mm);
}

// Key setup for many messages: one CTA each.
__global__ void __launch_bounds__(256) batch_key_setup_kernel(const BatchMsg *msgs, const BatchKey *keys,
                                                              const DevTables *tabs, uint64_t *t_start)
{
    if (t_start && blockIdx.x == 0 && threadIdx.x == 0) {
        uint64_t now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        *t_start = now;
    }
    const BatchMsg &m = msgs[blockIdx.x];
    const BatchKey &k = keys[blockIdx.x];
    key_setup_body(k.key, k.key_len, k.iv, k.iv_len, m.km, m.mm, tabs);
}

#undef LT0
#undef LT1
#undef LT2
#undef LT3

// ---------------------------------------------------------------------
// KC: log-depth combine + tag (one CTA)
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(512) combine_kernel(const __grid_constant__ KcParams p)
{
    // Levels whose output fits (at most 1024 entries) run in shared memory;
    // larger ones go through the global scratch.  Levels with many products
    // give one product to each thread; levels with few give each product to
    // a whole warp (gf_mul_warp), which has a much shorter latency.
    // Everything the serial path reads -- the partials (up to 1024), the
    // multipliers H^(2^(tile_log2 + level)), H, the round keys and tables of
    // E_K(J0) -- is staged into shared memory first, in one parallel step,
    // and E_K(J0) is computed by the last warp while the others run the tree.
    __shared__ gf128 sbuf[2][1024];
    __shared__ uint64_t wscr[16][16];
    __shared__ uint32_t stab[1024];
    __shared__ uint8_t ssbox[256];
    __shared__ uint32_t srk[60];
    __shared__ gf128 smult[H2K_COUNT];
    __shared__ gf128 sH;
    __shared__ uint32_t sej0[4];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = blockDim.x >> 5;
    const KeyMat *km = p.km;
    const bool aes_warp = p.ej0_from_j0 && !p.raw;  // the last warp computes E_K(J0)
    const int tree_warps = aes_warp ? nwarps - 1 : nwarps;
    const uint64_t K = p.K;
    if (aes_warp) {
        for (int i = t; i < 1024; i += blockDim.x) stab[i] = __ldg(&p.tabs->ttab[i]);
        for (int i = t; i < 256; i += blockDim.x) ssbox[i] = __ldg(&p.tabs->sbox[i]);
        if (t < 60) srk[t] = __ldg(&km->rk[t]);
    } else if (!p.raw && t < 4) {
        sej0[t] = __ldg(&p.mm->ej0[t]);
    }
    if (t >= 64 && t < 64 + H2K_COUNT && (uint32_t)(t - 64) + p.tile_log2 < (uint32_t)H2K_COUNT)
        smult[t - 64] = km->h2k[p.tile_log2 + (t - 64)];
    if (t == 128) sH = km->H;
    const bool staged = K <= 1024;
    if (staged)
        for (uint64_t i = t; i < K; i += blockDim.x) sbuf[1][i] = p.partials[i];
    __syncthreads();
    if (aes_warp && warp == nwarps - 1 && lane == 0) aes_block_tt(srk, (int)km->nr, stab, ssbox, p.j0, sej0);

    uint64_t cnt = K;
    int level = 0;
    // Level 0 reads the partials right to left (index g counts tiles from
    // the end of the sequence), so every right-hand operand is a full group
    // of 2^level tiles and its multiplier is exactly H^(2^(tile_log2+level)).
    const gf128 *src = staged ? sbuf[1] : p.partials;
    bool reversed = true;
    int flip = 0;
    while (cnt > 1) {
        const uint64_t half = (cnt + 1) / 2;
        const gf128 mult = smult[level];
        gf128 *dst = (half <= 1024) ? sbuf[flip] : ((src == p.scratch) ? p.partials : p.scratch);
        if (half > (uint64_t)tree_warps * 4) {
            for (uint64_t g = t; g < half; g += blockDim.x) {
                const uint64_t ri = 2 * g, li = 2 * g + 1;
                gf128 v = reversed ? src[cnt - 1 - ri] : src[ri];
                if (li < cnt) v = gf_xor(gf_mul(reversed ? src[cnt - 1 - li] : src[li], mult), v);
                dst[g] = v;
            }
        } else if (warp < tree_warps) {
            for (uint64_t g = warp; g < half; g += tree_warps) {
                const uint64_t ri = 2 * g, li = 2 * g + 1;
                gf128 v = reversed ? src[cnt - 1 - ri] : src[ri];
                if (li < cnt) v = gf_xor(gf_mul_warp(reversed ? src[cnt - 1 - li] : src[li], mult, wscr[warp]), v);
                if (lane == 0) dst[g] = v;
            }
        }
        __syncthreads();
        if (half <= 1024) flip ^= 1;
        src = dst;
        reversed = false;
        cnt = half;
        level++;
    }
    __syncthreads();  // E_K(J0) is in sej0 (also when there was no tree level)
    if (p.dsums) {
        // DATASUM: ones' complement total of the tile partials (each < 2^32,
        // so a 64-bit sum cannot overflow for any supported length).
        __shared__ uint64_t dpart[16];
        uint64_t acc = 0;
        for (uint64_t i = t; i < K; i += blockDim.x) acc += p.dsums[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
        if (lane == 0) dpart[warp] = acc;
        __syncthreads();
        if (t == 0) {
            uint64_t tot = 0;
            for (int w = 0; w < nwarps; w++) tot += dpart[w];
            *p.datasum_out = ones_fold(tot);
        }
    }
    if (warp != 0) return;
    gf128 s = (cnt == 1) ? src[0] : gf_zero();
    // Length block [len(A)]_64 || [len(C)]_64 in bits (SP 800-38D Alg. 4 step 5).
    gf128 lb;
    const uint64_t abits = p.aad_len * 8u, cbits = p.len * 8u;
    lb.w[0] = (uint32_t)(abits >> 32);
    lb.w[1] = (uint32_t)abits;
    lb.w[2] = (uint32_t)(cbits >> 32);
    lb.w[3] = (uint32_t)cbits;
    const gf128 gh = gf_mul_warp(gf_xor(s, lb), sH, wscr[0]);
    if (lane != 0) return;
    const uint4 gm = gf_to_mem(gh);
    uint32_t ej0[4] = {0u, 0u, 0u, 0u};
    if (!p.raw)
        for (int i = 0; i < 4; i++) ej0[i] = sej0[i];
    const uint32_t tw[4] = {gm.x ^ ej0[0], gm.y ^ ej0[1], gm.z ^ ej0[2], gm.w ^ ej0[3]};
    if (p.tag_out)
        for (int b = 0; b < 16; b++) p.tag_out[b] = (uint8_t)(tw[b >> 2] >> (8 * (b & 3)));
    if (p.tag_expected) {
        uint32_t diff = 0;
        for (int b = 0; b < 16; b++) diff |= (uint32_t)((uint8_t)(tw[b >> 2] >> (8 * (b & 3))) ^ p.tag_expected[b]);
        if (p.status) *p.status = diff ? -3 : 0;
    } else if (p.status) {
        *p.status = 0;
    }
}

// ---------------------------------------------------------------------
// KZ: zero-fill the payload when the tag check failed
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(256) zero_on_fail_kernel(const __grid_constant__ KzParams p)
{
    if (*p.status == 0) return;
    const uint64_t nvec = p.len / 16;
    uint4 *o = reinterpret_cast<uint4 *>(p.out);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += stride)
        o[i] = make_uint4(0u, 0u, 0u, 0u);
    if (blockIdx.x == 0 && threadIdx.x < (p.len & 15)) p.out[nvec * 16 + threadIdx.x] = 0;
}

// ---------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------
cudaError_t launch_batch_key_setup(const BatchMsg *msgs, const BatchKey *keys, uint32_t n,
                                   const DevTables *tabs, uint64_t *t_start, cudaStream_t stream)
{
    if (n == 0) return cudaSuccess;
    batch_key_setup_kernel<<<n, 256, 0, stream>>>(msgs, keys, tabs, t_start);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchParams &p, int grid, cudaStream_t stream)
{
    if (p.total_items == 0) return cudaSuccess;
    batch_kernel<<<grid, KF_THREADS, KF_SMEM_BYTES, stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_msg_setup(const BatchMsg *msgs, const BatchKey *keys, uint32_t n, const DevTables *tabs,
                             cudaStream_t stream)
{
    if (n == 0) return cudaSuccess;
    msg_setup_kernel<<<(n + 127) / 128, 128, 0, stream>>>(msgs, keys, n, tabs);
    return cudaGetLastError();
}

cudaError_t launch_batch_zero(const BatchMsg *msgs, uint32_t n, cudaStream_t stream)
{
    if (n == 0) return cudaSuccess;
    batch_zero_kernel<<<n, 256, 0, stream>>>(msgs, n);
    return cudaGetLastError();
}

cudaError_t configure_kernels()
{
    cudaError_t e;
    e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, KF_SMEM_BYTES);
    if (e != cudaSuccess) return e;
#define SET_SMEM(K)                                                                         \
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, KF_SMEM_BYTES); \
    if (e != cudaSuccess) return e;
    SET_SMEM((fused_kernel<10, MODE_GCM>));
    SET_SMEM((fused_kernel<12, MODE_GCM>));
    SET_SMEM((fused_kernel<14, MODE_GCM>));
    SET_SMEM((fused_kernel<10, MODE_CTR>));
    SET_SMEM((fused_kernel<12, MODE_CTR>));
    SET_SMEM((fused_kernel<14, MODE_CTR>));
    SET_SMEM((fused_kernel<14, MODE_GHASH>));
    SET_SMEM((fused_kernel<10, MODE_GCM_SUM>));
    SET_SMEM((fused_kernel<12, MODE_GCM_SUM>));
    SET_SMEM((fused_kernel<14, MODE_GCM_SUM>));
#undef SET_SMEM
#define SET_SMEM_BS(K)                                                                          \
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, KBS_SMEM_BYTES); \
    if (e != cudaSuccess) return e;
    SET_SMEM_BS((fused_bs_kernel<10, MODE_GCM>));
    SET_SMEM_BS((fused_bs_kernel<12, MODE_GCM>));
    SET_SMEM_BS((fused_bs_kernel<14, MODE_GCM>));
    SET_SMEM_BS((fused_bs_kernel<10, MODE_CTR>));
    SET_SMEM_BS((fused_bs_kernel<12, MODE_CTR>));
    SET_SMEM_BS((fused_bs_kernel<14, MODE_CTR>));
    SET_SMEM_BS((fused_bs_kernel<10, MODE_GCM_SUM>));
    SET_SMEM_BS((fused_bs_kernel<12, MODE_GCM_SUM>));
    SET_SMEM_BS((fused_bs_kernel<14, MODE_GCM_SUM>));
#undef SET_SMEM_BS
    return cudaSuccess;
}

cudaError_t launch_build_tables(DevTables *tabs, cudaStream_t stream)
{
    build_tables_kernel<<<1, 256, 0, stream>>>(tabs);
    return cudaGetLastError();
}

cudaError_t launch_msg_only(const KsParams &p, cudaStream_t stream)
{
    msg_only_kernel<<<1, 32, 0, stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_key_setup(const KsParams &p, cudaStream_t stream)
{
    key_setup_kernel<<<1, 256, 0, stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fused(const KfParams &p, int nr, int grid, cudaStream_t stream, int mode, int impl)
{
    if (p.tile_end <= p.tile_begin) return cudaSuccess;
    if (impl == 1 && mode != MODE_GHASH) {
#define KBS_LAUNCH(NRV)                                                                                             \
    if (mode == MODE_CTR) fused_bs_kernel<NRV, MODE_CTR><<<grid, KBS_THREADS, KBS_SMEM_BYTES, stream>>>(p);         \
    else if (mode == MODE_GCM_SUM) fused_bs_kernel<NRV, MODE_GCM_SUM><<<grid, KBS_THREADS, KBS_SMEM_BYTES, stream>>>(p); \
    else fused_bs_kernel<NRV, MODE_GCM><<<grid, KBS_THREADS, KBS_SMEM_BYTES, stream>>>(p);
        switch (nr) {
        case 10: KBS_LAUNCH(10); break;
        case 12: KBS_LAUNCH(12); break;
        case 14: KBS_LAUNCH(14); break;
        default: return cudaErrorInvalidValue;
        }
#undef KBS_LAUNCH
        return cudaGetLastError();
    }
    if (mode == MODE_GHASH) {
        fused_kernel<14, MODE_GHASH><<<grid, KF_THREADS, KF_SMEM_BYTES, stream>>>(p);
        return cudaGetLastError();
    }
#define KF_LAUNCH(NRV)                                                                        \
    if (mode == MODE_CTR) fused_kernel<NRV, MODE_CTR><<<grid, KF_THREADS, KF_SMEM_BYTES, stream>>>(p);         \
    else if (mode == MODE_GCM_SUM) fused_kernel<NRV, MODE_GCM_SUM><<<grid, KF_THREADS, KF_SMEM_BYTES, stream>>>(p); \
    else fused_kernel<NRV, MODE_GCM><<<grid, KF_THREADS, KF_SMEM_BYTES, stream>>>(p);
    switch (nr) {
    case 10: KF_LAUNCH(10); break;
    case 12: KF_LAUNCH(12); break;
    case 14: KF_LAUNCH(14); break;
    default: return cudaErrorInvalidValue;
    }
#undef KF_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_combine(const KcParams &p, cudaStream_t stream)
{
    combine_kernel<<<1, 512, 0, stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_zero_on_fail(const KzParams &p, int grid, cudaStream_t stream)
{
    zero_on_fail_kernel<<<grid, 256, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace gcmgpu
