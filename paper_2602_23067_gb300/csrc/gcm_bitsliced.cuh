// gcm_bitsliced.cuh -- bitsliced AES for the CTR keystream (FIPS-197 Cipher
// on 32 counter blocks per thread at once).
//
// Layout: a thread holds 32 blocks as 128 words s[8 p + i]: bit k of that
// word is bit i (LSB = 0) of byte p of block k.  In that form SubBytes is the
// S-box circuit of bitsliced_sbox.cuh applied to the 8 words of each byte
// position, ShiftRows is a renaming of byte positions, MixColumns is XOR
// arithmetic on whole bytes (xtime = a shift of bit positions with the
// reduction bits x^8 = x^4 + x^3 + x + 1), and AddRoundKey is an XOR with an
// all-zeros / all-ones word per key bit.  Every operation works on 32 blocks
// per instruction.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "bitsliced_sbox.cuh"

namespace gcmgpu {

// In-place transpose of a 32 x 32 bit matrix: afterwards bit k of a[j] is
// what bit j of a[k] was.  Five rounds of block swaps (16, 8, 4, 2, 1): for
// a row pair (k, k + j) the upper j-block of row k trades places with the
// lower j-block of row k + j.  The byte-granular rounds are byte permutes.
__host__ __device__ __forceinline__ void transpose32(uint32_t a[32])
{
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const uint32_t x = a[k], y = a[k + 16];
#ifdef __CUDA_ARCH__
        a[k] = __byte_perm(x, y, 0x5410);
        a[k + 16] = __byte_perm(x, y, 0x7632);
#else
        a[k] = (x & 0x0000FFFFu) | (y << 16);
        a[k + 16] = (x >> 16) | (y & 0xFFFF0000u);
#endif
    }
#pragma unroll
    for (int k0 = 0; k0 < 32; k0 += 16)
#pragma unroll
        for (int k = k0; k < k0 + 8; k++) {
            const uint32_t x = a[k], y = a[k + 8];
#ifdef __CUDA_ARCH__
            a[k] = __byte_perm(x, y, 0x6240);
            a[k + 8] = __byte_perm(x, y, 0x7351);
#else
            a[k] = (x & 0x00FF00FFu) | ((y << 8) & 0xFF00FF00u);
            a[k + 8] = ((x >> 8) & 0x00FF00FFu) | (y & 0xFF00FF00u);
#endif
        }
#pragma unroll
    for (int js = 2; js >= 0; js--) {  // j = 4, 2, 1 (a linear counter, so the loop unrolls)
        const int j = 1 << js;
        const uint32_t m = (js == 2) ? 0x0F0F0F0Fu : (js == 1) ? 0x33333333u : 0x55555555u;
#pragma unroll
        for (int k = 0; k < 32; k++) {
            if (k & j) continue;
            const uint32_t t = ((a[k] >> j) ^ a[k + j]) & m;
            a[k + j] ^= t;
            a[k] ^= t << j;
        }
    }
}

// MixColumns on one column (bytes a, b, c, d, 8 words each, bit i at [i]):
// out_r = xtime(a_r + a_{r+1}) + a_{r+1} + a_{r+2} + a_{r+3} (FIPS-197
// sec. 5.1.3 rows 2 3 1 1).  xtime(u) has bits (u7, u0+u7, u1, u2+u7,
// u3+u7, u4, u5, u6).
__host__ __device__ __forceinline__ void mixcolumn_bs(const uint32_t *a, const uint32_t *b, const uint32_t *c,
                                                      const uint32_t *d, uint32_t *o0, uint32_t *o1, uint32_t *o2,
                                                      uint32_t *o3)
{
    uint32_t t[8], u[4][8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        t[i] = a[i] ^ b[i] ^ c[i] ^ d[i];
        u[0][i] = a[i] ^ b[i];
        u[1][i] = b[i] ^ c[i];
        u[2][i] = c[i] ^ d[i];
        u[3][i] = d[i] ^ a[i];
    }
    const uint32_t *src[4] = {a, b, c, d};
    uint32_t *dst[4] = {o0, o1, o2, o3};
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const uint32_t *x = src[r];
        const uint32_t *v = u[r];
        // out = xtime(v) + (t + x)
        dst[r][0] = v[7] ^ t[0] ^ x[0];
        dst[r][1] = v[0] ^ v[7] ^ t[1] ^ x[1];
        dst[r][2] = v[1] ^ t[2] ^ x[2];
        dst[r][3] = v[2] ^ v[7] ^ t[3] ^ x[3];
        dst[r][4] = v[3] ^ v[7] ^ t[4] ^ x[4];
        dst[r][5] = v[4] ^ t[5] ^ x[5];
        dst[r][6] = v[5] ^ t[6] ^ x[6];
        dst[r][7] = v[6] ^ t[7] ^ x[7];
    }
}

// ShiftRows source: byte 4c + r of the result is byte 4((c + r) mod 4) + r.
__host__ __device__ constexpr int shiftrows_src(int p)
{
    return 4 * (((p >> 2) + (p & 3)) & 3) + (p & 3);
}

// Rounds 1..NR on a bitsliced state that already holds input xor round key
// 0.  km_bs holds the bitsliced round keys: word 128 r + 8 p + i is all ones
// when bit i of byte p of round key r (xor 0x63 in every byte for r >= 1,
// the S-box constant the circuit leaves out) is set.  The words of a round
// are read as 16-byte vectors that every lane reads at the same address.
template <int NR>
__host__ __device__ __forceinline__ void aes_rounds_bs(uint32_t s[128], const uint32_t *km_bs)
{
#pragma unroll 1
    for (int r = 1; r <= NR; r++) {
#pragma unroll
        for (int p = 0; p < 16; p++)
            sbox_bitsliced(s[8 * p + 0], s[8 * p + 1], s[8 * p + 2], s[8 * p + 3], s[8 * p + 4], s[8 * p + 5],
                           s[8 * p + 6], s[8 * p + 7]);
        uint32_t t[128];
#pragma unroll
        for (int p = 0; p < 16; p++)
#pragma unroll
            for (int i = 0; i < 8; i++) t[8 * p + i] = s[8 * shiftrows_src(p) + i];
        if (r != NR) {
#pragma unroll
            for (int c = 0; c < 4; c++)
                mixcolumn_bs(&t[32 * c], &t[32 * c + 8], &t[32 * c + 16], &t[32 * c + 24], &s[32 * c],
                             &s[32 * c + 8], &s[32 * c + 16], &s[32 * c + 24]);
        } else {
#pragma unroll
            for (int q = 0; q < 128; q++) s[q] = t[q];
        }
        const uint4 *kr = reinterpret_cast<const uint4 *>(km_bs + 128 * r);
#pragma unroll
        for (int q = 0; q < 32; q++) {
            const uint4 k4 = kr[q];
            s[4 * q + 0] ^= k4.x;
            s[4 * q + 1] ^= k4.y;
            s[4 * q + 2] ^= k4.z;
            s[4 * q + 3] ^= k4.w;
        }
    }
}

// Word q (0 <= q < 128 (NR + 1)) of the bitsliced round keys, from the round
// keys as memory words (rk[4 r + c] = bytes 4c..4c+3 of round key r, first
// byte in the low bits): all ones when bit i = q mod 8 of byte p = (q / 8)
// mod 16 of round key r = q / 128 is set, the S-box constant 0x63 xored into
// every byte of the keys of rounds 1..NR.
__host__ __device__ __forceinline__ uint32_t round_key_word_bs(const uint32_t *rk, int q)
{
    const int r = q >> 7, p = (q >> 3) & 15, i = q & 7;
    uint32_t byte = (rk[4 * r + (p >> 2)] >> (8 * (p & 3))) & 0xFFu;
    if (r >= 1) byte ^= 0x63u;
    return ((byte >> i) & 1u) ? 0xFFFFFFFFu : 0u;
}

// Bitsliced AES input for 32 counter blocks xor round key 0: bytes 0..11 are
// those of J0 (memory words j0w0..j0w2, the same for every block), bytes
// 12..15 the big-endian counter ctr[k] of block k.
__host__ __device__ __forceinline__ void load_counters_bs(uint32_t s[128], uint32_t j0w0, uint32_t j0w1,
                                                          uint32_t j0w2, uint32_t ctr[32], const uint32_t *km_bs)
{
    const uint32_t jw[3] = {j0w0, j0w1, j0w2};
#pragma unroll
    for (int p = 0; p < 12; p++)
#pragma unroll
        for (int i = 0; i < 8; i++)
            s[8 * p + i] = (((jw[p >> 2] >> (8 * (p & 3) + i)) & 1u) ? 0xFFFFFFFFu : 0u) ^ km_bs[8 * p + i];
    transpose32(ctr);  // ctr[j] bit k = bit j of block k's counter
#pragma unroll
    for (int i = 0; i < 8; i++) {
        s[8 * 12 + i] = ctr[24 + i] ^ km_bs[8 * 12 + i];
        s[8 * 13 + i] = ctr[16 + i] ^ km_bs[8 * 13 + i];
        s[8 * 14 + i] = ctr[8 + i] ^ km_bs[8 * 14 + i];
        s[8 * 15 + i] = ctr[i] ^ km_bs[8 * 15 + i];
    }
}

// The 32 output blocks as memory words: afterwards s[32 w + k] is word w
// (bytes 4w..4w+3) of block k.  Byte p = 4w + j, bit i sits at s[32 w + 8 j + i]
// before the transpose, which is bit 8 j + i of that word.
__host__ __device__ __forceinline__ void unload_blocks_bs(uint32_t s[128])
{
#pragma unroll
    for (int w = 0; w < 4; w++) transpose32(&s[32 * w]);
}

}  // namespace gcmgpu
