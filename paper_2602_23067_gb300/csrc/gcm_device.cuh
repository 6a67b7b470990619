// gcm_device.cuh -- device-side building blocks of the AES-GCM hot path.
//
// Representations used on the device:
//   * "memory words": a 16-byte block loaded as four little-endian uint32
//     (word i = bytes 4i..4i+3).  Data, keystream and the GHASH table entries
//     stay in this layout so that XOR-accumulation needs no byte swapping.
//   * "poly words" (gf128): the same block with every word byte-swapped, so
//     that the coefficient of x^i (GCM's bit-reflected convention, SP 800-38D
//     sec. 6.3: bit 0 of the block is the MSB of byte 0 and is x^0) sits at
//     bit 31 - (i mod 32) of word i/32.  Multiplication by x is then a
//     right shift of the 128-bit value, with x^128 = x^7 + x^2 + x + 1
//     folding back as R = 0xE1000000 into word 0.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gcmgpu {

struct gf128 {
    uint32_t w[4];
};

__host__ __device__ __forceinline__ uint32_t bswap32(uint32_t x)
{
#ifdef __CUDA_ARCH__
    return __byte_perm(x, 0, 0x0123);
#else
    return (x >> 24) | ((x >> 8) & 0xFF00u) | ((x << 8) & 0xFF0000u) | (x << 24);
#endif
}

__device__ __forceinline__ gf128 gf_zero()
{
    gf128 r;
    r.w[0] = r.w[1] = r.w[2] = r.w[3] = 0u;
    return r;
}

__device__ __forceinline__ gf128 gf_xor(const gf128 &a, const gf128 &b)
{
    gf128 r;
#pragma unroll
    for (int i = 0; i < 4; i++) r.w[i] = a.w[i] ^ b.w[i];
    return r;
}

// memory words <-> poly words
__device__ __forceinline__ gf128 gf_from_mem(uint32_t m0, uint32_t m1, uint32_t m2, uint32_t m3)
{
    gf128 r;
    r.w[0] = bswap32(m0);
    r.w[1] = bswap32(m1);
    r.w[2] = bswap32(m2);
    r.w[3] = bswap32(m3);
    return r;
}

__device__ __forceinline__ uint4 gf_to_mem(const gf128 &a)
{
    return make_uint4(bswap32(a.w[0]), bswap32(a.w[1]), bswap32(a.w[2]), bswap32(a.w[3]));
}

// a * x (one step of the V chain of the shift-and-add multiplier).
__device__ __forceinline__ gf128 gf_mul_x(const gf128 &v)
{
    gf128 r;
    uint32_t carry = 0u - (v.w[3] & 1u);
    r.w[3] = __funnelshift_r(v.w[3], v.w[2], 1);
    r.w[2] = __funnelshift_r(v.w[2], v.w[1], 1);
    r.w[1] = __funnelshift_r(v.w[1], v.w[0], 1);
    r.w[0] = (v.w[0] >> 1) ^ (carry & 0xE1000000u);
    return r;
}

// ---------------------------------------------------------------------
// General product a * b (the rare multiplications: key setup, the closing of
// a lane's chain, segment factors, the tree combine).  The per-block
// multiplications of the hot loop go through the shared-memory table.
//
// Carry-less multiplication from integer multiplication: split a 32-bit
// operand into four "sparse" parts holding only the bits at positions
// = i (mod 4).  In the integer product of two sparse parts every position of
// one residue class receives the count of bit pairs that land there (at most
// 8), which needs 4 bits, so the counts of neighbouring positions of the class
// (4 apart) never overlap and no carry reaches another position of the class:
// the bit at each such position is the count mod 2, i.e. the carry-less
// product.  XOR of the four products per class and a mask per class give the
// 64-bit carry-less product.  Two levels of Karatsuba build the 128 x 128
// product from nine such multiplies; the 255-bit product is then reduced
// modulo x^128 + x^7 + x^2 + x + 1.  Everything is data-independent (no
// branches, no table), so the latency is a few hundred cycles instead of the
// 128 dependent steps of shift-and-add.
// ---------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t brev32(uint32_t x)
{
#ifdef __CUDA_ARCH__
    return __brev(x);
#else
    uint32_t r = 0u;
    for (int i = 0; i < 32; i++) r |= ((x >> i) & 1u) << (31 - i);
    return r;
#endif
}

// 32 x 32 -> 64-bit carry-less product; bit i of x is the coefficient of t^i.
__host__ __device__ __forceinline__ uint64_t clmul32(uint32_t x, uint32_t y)
{
    const uint32_t x0 = x & 0x11111111u, x1 = x & 0x22222222u, x2 = x & 0x44444444u, x3 = x & 0x88888888u;
    const uint32_t y0 = y & 0x11111111u, y1 = y & 0x22222222u, y2 = y & 0x44444444u, y3 = y & 0x88888888u;
    const uint64_t z0 = ((uint64_t)x0 * y0) ^ ((uint64_t)x1 * y3) ^ ((uint64_t)x2 * y2) ^ ((uint64_t)x3 * y1);
    const uint64_t z1 = ((uint64_t)x0 * y1) ^ ((uint64_t)x1 * y0) ^ ((uint64_t)x2 * y3) ^ ((uint64_t)x3 * y2);
    const uint64_t z2 = ((uint64_t)x0 * y2) ^ ((uint64_t)x1 * y1) ^ ((uint64_t)x2 * y0) ^ ((uint64_t)x3 * y3);
    const uint64_t z3 = ((uint64_t)x0 * y3) ^ ((uint64_t)x1 * y2) ^ ((uint64_t)x2 * y1) ^ ((uint64_t)x3 * y0);
    return (z0 & 0x1111111111111111ull) | (z1 & 0x2222222222222222ull) | (z2 & 0x4444444444444444ull) |
           (z3 & 0x8888888888888888ull);
}

// 64 x 64 -> 128-bit carry-less product (one Karatsuba level).
__host__ __device__ __forceinline__ void clmul64(uint64_t a, uint64_t b, uint64_t &lo, uint64_t &hi)
{
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    const uint64_t p0 = clmul32(a0, b0), p2 = clmul32(a1, b1);
    const uint64_t p1 = clmul32(a0 ^ a1, b0 ^ b1) ^ p0 ^ p2;
    lo = p0 ^ (p1 << 32);
    hi = p2 ^ (p1 >> 32);
}

// Reduces the 255-bit carry-less product P3:P2:P1:P0 (64-bit words, bit i =
// coefficient of x^i, P3 < 2^63) modulo x^128 + x^7 + x^2 + x + 1 and returns
// it as poly words.  x^128 = x^7 + x^2 + x + 1: the high half Q = P3:P2 folds
// back as Q * (1 + x + x^2 + x^7).  Its bits pushed above x^127 (the top 7
// bits of Q shifted by 1, 2, 7) fold once more; adding them into the low bits
// of Q first (T) makes one pass of shifts do both folds.
__host__ __device__ __forceinline__ void gf_reduce256(uint64_t P0, uint64_t P1, uint64_t P2, uint64_t P3,
                                                      uint32_t out[4])
{
    const uint64_t T0 = P2 ^ (P3 >> 63) ^ (P3 >> 62) ^ (P3 >> 57);
    const uint64_t T1 = P3;
    const uint64_t R0 = T0 ^ (T0 << 1) ^ (T0 << 2) ^ (T0 << 7);
    const uint64_t R1 = T1 ^ ((T1 << 1) | (T0 >> 63)) ^ ((T1 << 2) | (T0 >> 62)) ^ ((T1 << 7) | (T0 >> 57));
    const uint64_t Z0 = P0 ^ R0, Z1 = P1 ^ R1;
    out[0] = brev32((uint32_t)Z0);
    out[1] = brev32((uint32_t)(Z0 >> 32));
    out[2] = brev32((uint32_t)Z1);
    out[3] = brev32((uint32_t)(Z1 >> 32));
}

// Product of two field elements given as poly words (see the top of this
// file): out = a * b mod x^128 + x^7 + x^2 + x + 1.
__host__ __device__ __forceinline__ void gf_mul_words(const uint32_t a[4], const uint32_t b[4], uint32_t out[4])
{
    // Bit-reversing each poly word puts the coefficient of x^i at bit i of
    // the 128-bit little-endian integer (A0 = x^0..x^63, A1 = x^64..x^127).
    const uint64_t A0 = (uint64_t)brev32(a[0]) | ((uint64_t)brev32(a[1]) << 32);
    const uint64_t A1 = (uint64_t)brev32(a[2]) | ((uint64_t)brev32(a[3]) << 32);
    const uint64_t B0 = (uint64_t)brev32(b[0]) | ((uint64_t)brev32(b[1]) << 32);
    const uint64_t B1 = (uint64_t)brev32(b[2]) | ((uint64_t)brev32(b[3]) << 32);
    uint64_t l0, h0, l2, h2, l1, h1;
    clmul64(A0, B0, l0, h0);
    clmul64(A1, B1, l2, h2);
    clmul64(A0 ^ A1, B0 ^ B1, l1, h1);
    l1 ^= l0 ^ l2;
    h1 ^= h0 ^ h2;
    gf_reduce256(l0, h0 ^ l1, l2 ^ h1, h2, out);
}

__device__ __forceinline__ gf128 gf_mul(const gf128 &a, const gf128 &b)
{
    gf128 r;
    gf_mul_words(a.w, b.w, r.w);
    return r;
}

// The same product computed by a whole warp, for a multiply on a serial
// path (the tree combine, the tag): every lane passes the same a and b and
// receives a * b.  Lanes 0..15 each form one of the 16 schoolbook products
// of 32-bit words, A_i * B_j at bit offset 32 (i + j); every lane then sums
// them from `scratch` (16 x 8 bytes of shared memory owned by this warp) and
// reduces the 255-bit product.  Several hundred cycles instead of the
// several thousand of one thread doing all nine Karatsuba products.
// Word i (0..3, not a compile-time constant) of a, by selects, so that a
// can stay in registers.
__device__ __forceinline__ uint32_t gf_word(const gf128 &a, int i)
{
    const uint32_t lo = (i & 1) ? a.w[1] : a.w[0];
    const uint32_t hi = (i & 1) ? a.w[3] : a.w[2];
    return (i & 2) ? hi : lo;
}

__device__ __forceinline__ gf128 gf_mul_warp(const gf128 &a, const gf128 &b, uint64_t *scratch)
{
    const int lane = threadIdx.x & 31;
    if (lane < 16) {
        const int i = lane >> 2, j = lane & 3;
        scratch[lane] = clmul32(brev32(gf_word(a, i)), brev32(gf_word(b, j)));
    }
    __syncwarp();
    uint32_t p[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint64_t v = scratch[4 * i + j];
            p[i + j] ^= (uint32_t)v;
            p[i + j + 1] ^= (uint32_t)(v >> 32);
        }
    __syncwarp();  // scratch may be reused by the next call
    gf128 r;
    gf_reduce256((uint64_t)p[0] | ((uint64_t)p[1] << 32), (uint64_t)p[2] | ((uint64_t)p[3] << 32),
                 (uint64_t)p[4] | ((uint64_t)p[5] << 32), (uint64_t)p[6] | ((uint64_t)p[7] << 32), r.w);
    return r;
}

// Spreads the 16 bits of x so that bit q lands on bit 2q (zeros between).
__device__ __forceinline__ uint32_t spread16(uint32_t x)
{
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// a^2.  Squaring is linear over GF(2): (sum a_i x^i)^2 = sum a_i x^(2i).
// The 128 coefficients are spread into a 256-coefficient product, whose
// upper half is folded back with x^128 = 1 + x + x^2 + x^7.
__device__ __forceinline__ gf128 gf_sqr(const gf128 &a)
{
    // In poly words, coefficient 32*wi + j sits at bit 31 - j of word wi and
    // goes to coefficient 64*wi + 2j: the upper 16 bits of word wi fill word
    // 2wi of the product and the lower 16 bits fill word 2wi + 1, each bit p
    // moving to bit 2(p mod 16) + 1.
    uint32_t p[8];
#pragma unroll
    for (int wi = 0; wi < 4; wi++) {
        p[2 * wi] = spread16(a.w[wi] >> 16) << 1;
        p[2 * wi + 1] = spread16(a.w[wi]) << 1;
    }
    // High half h (coefficients 128..255 as a 128-bit poly value) times
    // (1 + x + x^2 + x^7) added into the low half.
    const uint32_t h0 = p[4], h1 = p[5], h2 = p[6], h3 = p[7];
    gf128 r;
    r.w[3] = p[3] ^ h3 ^ __funnelshift_r(h3, h2, 1) ^ __funnelshift_r(h3, h2, 2) ^ __funnelshift_r(h3, h2, 7);
    r.w[2] = p[2] ^ h2 ^ __funnelshift_r(h2, h1, 1) ^ __funnelshift_r(h2, h1, 2) ^ __funnelshift_r(h2, h1, 7);
    r.w[1] = p[1] ^ h1 ^ __funnelshift_r(h1, h0, 1) ^ __funnelshift_r(h1, h0, 2) ^ __funnelshift_r(h1, h0, 7);
    r.w[0] = p[0] ^ h0 ^ (h0 >> 1) ^ (h0 >> 2) ^ (h0 >> 7);
    // Coefficients pushed past x^127 by the shifts (the low 7 bits of h3)
    // come back once more: coefficient 128 + e folds to x^e (1+x+x^2+x^7).
    uint32_t ov = ((h3 & 1u) << 31) ^ ((h3 & 3u) << 30) ^ ((h3 & 0x7Fu) << 25);
    r.w[0] ^= ov ^ (ov >> 1) ^ (ov >> 2) ^ (ov >> 7);
    return r;
}

// ---------------------------------------------------------------------
// AES: S-box from GF(2^8) (FIPS-197 sec. 5.1.1), built with log/antilog
// tables over the generator 0x03 and the affine map written as rotations.
// ---------------------------------------------------------------------
__device__ __forceinline__ uint8_t gf8_xtime(uint8_t a)
{
    return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1B : 0x00));
}

__device__ __forceinline__ uint8_t rotl8(uint8_t x, int s)
{
    return (uint8_t)((x << s) | (x >> (8 - s)));
}

// Fills sbox[256] (call with one block of >= 256 threads; uses smem scratch
// of 512 bytes passed in).
__device__ inline void build_sbox_block(uint8_t *sbox, uint8_t *scratch_exp, uint8_t *scratch_log)
{
    if (threadIdx.x == 0) {
        uint8_t x = 1;
        for (int i = 0; i < 255; i++) {
            scratch_exp[i] = x;
            scratch_log[x] = (uint8_t)i;
            x = (uint8_t)(x ^ gf8_xtime(x)); // x * 0x03
        }
        scratch_exp[255] = 1;
        scratch_log[0] = 0;
    }
    __syncthreads();
    int t = threadIdx.x;
    if (t < 256) {
        uint8_t inv = (t == 0) ? 0 : scratch_exp[(255 - scratch_log[t]) % 255];
        uint8_t s = (uint8_t)(inv ^ rotl8(inv, 1) ^ rotl8(inv, 2) ^ rotl8(inv, 3) ^ rotl8(inv, 4) ^ 0x63);
        sbox[t] = s;
    }
    __syncthreads();
}

// Round-table entry for table r (0..3) and S-box output s, as a little-endian
// word whose byte i is row i of the MixColumns column: T_r[v] is column r of
// the matrix [2 3 1 1; 1 2 3 1; 1 1 2 3; 3 1 1 2] times S[v].
__device__ __forceinline__ uint32_t ttable_entry(int r, uint8_t s)
{
    uint32_t s1 = s, s2 = gf8_xtime(s), s3 = s2 ^ s1;
    uint32_t t0 = s2 | (s1 << 8) | (s1 << 16) | (s3 << 24);
    return (t0 << (8 * r)) | (r ? (t0 >> (32 - 8 * r)) : 0u);
}

} // namespace gcmgpu
