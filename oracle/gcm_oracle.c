/*
 * gcm_oracle.c -- plain, slow, byte-at-a-time AES-GCM on the CPU.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the
 * GPU library.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may build, load or call it.  The product path
 * (the CUDA library and its Python binding) never links or imports it, and
 * it shares no code, table or constant generator with the product.
 *
 * What it computes, and where each step comes from:
 *   - AES forward and inverse cipher, key expansion: FIPS-197 sections 5.1-5.3.
 *     The S-box is derived at start-up from its definition (multiplicative
 *     inverse in GF(2^8) modulo x^8+x^4+x^3+x+1, then the affine map with
 *     constant 0x63), not typed in.
 *   - GF(2^128) multiplication: NIST SP 800-38D section 6.3, Algorithm 1
 *     (bit-reflected convention, R = 11100001 || 0^120).
 *   - GHASH: SP 800-38D Algorithm 2, which is the serial recurrence
 *     Y_i = (Y_{i-1} xor X_i) * H of the paper (Sec. 3.3.1, Eq. 1).
 *   - inc32 and GCTR: SP 800-38D sections 6.2 and 6.5 (Algorithm 3).
 *   - GCM-AE / GCM-AD: SP 800-38D sections 7.1 and 7.2 (Algorithms 4, 5),
 *     the AES-GCM mode the paper adopts (Sec. 3.2.1).  On an authentication
 *     failure the output buffer is zero-filled, the payload suppression the
 *     paper describes (Sec. 4.2).
 *
 * Everything works on byte arrays in the standards' own bit order, with no
 * blocking, no lookup tables beyond the S-box, and no reordering of the
 * steps.  Speed is not a goal.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* GF(2^8) arithmetic and the S-box (FIPS-197 sections 4.2 and 5.1.1)   */
/* ------------------------------------------------------------------ */

/* Multiplication in GF(2^8) modulo m(x) = x^8 + x^4 + x^3 + x + 1 (0x11B),
 * shift-and-add (FIPS-197 section 4.2 / 4.2.1 xtime). */
static uint8_t gf8_mul(uint8_t a, uint8_t b)
{
    uint8_t p = 0;
    for (int i = 0; i < 8; i++) {
        if (b & 1) p ^= a;
        uint8_t hi = (uint8_t)(a & 0x80);
        a = (uint8_t)(a << 1);
        if (hi) a ^= 0x1B;
        b >>= 1;
    }
    return p;
}

/* Multiplicative inverse by exhaustive search; 0 maps to 0 (FIPS-197 5.1.1). */
static uint8_t gf8_inv(uint8_t a)
{
    if (a == 0) return 0;
    for (int c = 1; c < 256; c++)
        if (gf8_mul(a, (uint8_t)c) == 1) return (uint8_t)c;
    return 0; /* unreachable: every nonzero element has an inverse */
}

static uint8_t g_sbox[256];
static uint8_t g_inv_sbox[256];
static int g_ready = 0;

/* S-box: affine transformation of the inverse (FIPS-197 eq. 5.1):
 * b'_i = b_i ^ b_{(i+4)%8} ^ b_{(i+5)%8} ^ b_{(i+6)%8} ^ b_{(i+7)%8} ^ c_i,
 * c = 0x63. */
static void build_sbox(void)
{
    for (int x = 0; x < 256; x++) {
        uint8_t b = gf8_inv((uint8_t)x);
        uint8_t s = 0;
        for (int i = 0; i < 8; i++) {
            int bit = ((b >> i) & 1) ^ ((b >> ((i + 4) % 8)) & 1) ^
                      ((b >> ((i + 5) % 8)) & 1) ^ ((b >> ((i + 6) % 8)) & 1) ^
                      ((b >> ((i + 7) % 8)) & 1) ^ ((0x63 >> i) & 1);
            s |= (uint8_t)(bit << i);
        }
        g_sbox[x] = s;
    }
    for (int x = 0; x < 256; x++) g_inv_sbox[g_sbox[x]] = (uint8_t)x;
    g_ready = 1;
}

static void ensure_ready(void)
{
    if (!g_ready) build_sbox();
}

void oracle_sbox(uint8_t out[256], uint8_t inv_out[256])
{
    ensure_ready();
    memcpy(out, g_sbox, 256);
    if (inv_out) memcpy(inv_out, g_inv_sbox, 256);
}

uint8_t oracle_gf8_mul(uint8_t a, uint8_t b) { return gf8_mul(a, b); }

/* ------------------------------------------------------------------ */
/* AES (FIPS-197 sections 5.1 - 5.3)                                    */
/* ------------------------------------------------------------------ */

/* Key expansion (FIPS-197 section 5.2).  Returns Nr, or -1 on a bad key
 * length.  w receives 4*(Nr+1) words as 16*(Nr+1) bytes. */
int oracle_aes_key_expansion(const uint8_t *key, int key_len, uint8_t *w)
{
    ensure_ready();
    int Nk, Nr;
    if (key_len == 16) { Nk = 4; Nr = 10; }
    else if (key_len == 24) { Nk = 6; Nr = 12; }
    else if (key_len == 32) { Nk = 8; Nr = 14; }
    else return -1;

    for (int i = 0; i < 4 * Nk; i++) w[i] = key[i];
    uint8_t rcon = 0x01; /* Rcon[i/Nk] = x^(i/Nk - 1) in GF(2^8) */
    for (int i = Nk; i < 4 * (Nr + 1); i++) {
        uint8_t t[4];
        memcpy(t, &w[4 * (i - 1)], 4);
        if (i % Nk == 0) {
            uint8_t r0 = t[0]; /* RotWord */
            t[0] = t[1]; t[1] = t[2]; t[2] = t[3]; t[3] = r0;
            for (int j = 0; j < 4; j++) t[j] = g_sbox[t[j]]; /* SubWord */
            t[0] ^= rcon;
            rcon = gf8_mul(rcon, 0x02);
        } else if (Nk > 6 && i % Nk == 4) {
            for (int j = 0; j < 4; j++) t[j] = g_sbox[t[j]];
        }
        for (int j = 0; j < 4; j++) w[4 * i + j] = (uint8_t)(w[4 * (i - Nk) + j] ^ t[j]);
    }
    return Nr;
}

/* The state is s[r][c] with input byte in[r + 4c] (FIPS-197 section 3.4). */
static void add_round_key(uint8_t s[4][4], const uint8_t *rk)
{
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) s[r][c] ^= rk[4 * c + r];
}

static void sub_bytes(uint8_t s[4][4], const uint8_t *box)
{
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) s[r][c] = box[s[r][c]];
}

/* ShiftRows: row r is rotated left by r (FIPS-197 5.1.2). */
static void shift_rows(uint8_t s[4][4])
{
    for (int r = 1; r < 4; r++) {
        uint8_t t[4];
        for (int c = 0; c < 4; c++) t[c] = s[r][(c + r) % 4];
        for (int c = 0; c < 4; c++) s[r][c] = t[c];
    }
}

/* InvShiftRows: row r is rotated right by r (FIPS-197 5.3.1). */
static void inv_shift_rows(uint8_t s[4][4])
{
    for (int r = 1; r < 4; r++) {
        uint8_t t[4];
        for (int c = 0; c < 4; c++) t[(c + r) % 4] = s[r][c];
        for (int c = 0; c < 4; c++) s[r][c] = t[c];
    }
}

/* MixColumns with the fixed polynomial {03}x^3+{01}x^2+{01}x+{02}
 * (FIPS-197 5.1.3), or InvMixColumns with {0b}x^3+{0d}x^2+{09}x+{0e}
 * (5.3.3).  m[] is the first row of the circulant matrix. */
static void mix_columns_with(uint8_t s[4][4], const uint8_t m[4])
{
    for (int c = 0; c < 4; c++) {
        uint8_t a[4];
        for (int r = 0; r < 4; r++) a[r] = s[r][c];
        for (int r = 0; r < 4; r++) {
            uint8_t v = 0;
            for (int k = 0; k < 4; k++) v ^= gf8_mul(m[(k - r + 4) % 4], a[k]);
            s[r][c] = v;
        }
    }
}

void oracle_aes_encrypt_block(const uint8_t *w, int Nr, const uint8_t in[16], uint8_t out[16])
{
    static const uint8_t mix[4] = {0x02, 0x03, 0x01, 0x01};
    ensure_ready();
    uint8_t s[4][4];
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) s[r][c] = in[r + 4 * c];
    add_round_key(s, w);
    for (int round = 1; round < Nr; round++) {
        sub_bytes(s, g_sbox);
        shift_rows(s);
        mix_columns_with(s, mix);
        add_round_key(s, w + 16 * round);
    }
    sub_bytes(s, g_sbox);
    shift_rows(s);
    add_round_key(s, w + 16 * Nr);
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) out[r + 4 * c] = s[r][c];
}

void oracle_aes_decrypt_block(const uint8_t *w, int Nr, const uint8_t in[16], uint8_t out[16])
{
    static const uint8_t inv_mix[4] = {0x0e, 0x0b, 0x0d, 0x09};
    ensure_ready();
    uint8_t s[4][4];
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) s[r][c] = in[r + 4 * c];
    add_round_key(s, w + 16 * Nr);
    for (int round = Nr - 1; round >= 1; round--) {
        inv_shift_rows(s);
        sub_bytes(s, g_inv_sbox);
        add_round_key(s, w + 16 * round);
        mix_columns_with(s, inv_mix);
    }
    inv_shift_rows(s);
    sub_bytes(s, g_inv_sbox);
    add_round_key(s, w);
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) out[r + 4 * c] = s[r][c];
}

/* ------------------------------------------------------------------ */
/* GF(2^128) and GHASH (SP 800-38D sections 6.3, 6.4)                   */
/* ------------------------------------------------------------------ */

/* Bit i of a block (i = 0 is the leftmost bit, the MSB of byte 0). */
static int bit_at(const uint8_t x[16], int i)
{
    return (x[i / 8] >> (7 - (i % 8))) & 1;
}

/* Algorithm 1: Z = X * Y.  Z_0 = 0, V_0 = Y; for i = 0..127:
 *   Z_{i+1} = Z_i xor V_i if x_i = 1;
 *   V_{i+1} = V_i >> 1 if LSB_1(V_i) = 0, else (V_i >> 1) xor R. */
void oracle_gf128_mul(const uint8_t x[16], const uint8_t y[16], uint8_t z[16])
{
    uint8_t Z[16], V[16];
    memset(Z, 0, 16);
    memcpy(V, y, 16);
    for (int i = 0; i < 128; i++) {
        if (bit_at(x, i))
            for (int k = 0; k < 16; k++) Z[k] ^= V[k];
        int lsb = V[15] & 1;
        for (int k = 15; k > 0; k--) V[k] = (uint8_t)((V[k] >> 1) | (V[k - 1] << 7));
        V[0] >>= 1;
        if (lsb) V[0] ^= 0xE1; /* R = 11100001 || 0^120 */
    }
    memcpy(z, Z, 16);
}

/* Algorithm 2: GHASH_H(X_1 || ... || X_m); Y_0 = 0, Y_i = (Y_{i-1} xor X_i) * H. */
void oracle_ghash(const uint8_t H[16], const uint8_t *X, size_t m, uint8_t out[16])
{
    uint8_t Y[16];
    memset(Y, 0, 16);
    for (size_t i = 0; i < m; i++) {
        for (int k = 0; k < 16; k++) Y[k] ^= X[16 * i + k];
        oracle_gf128_mul(Y, H, Y);
    }
    memcpy(out, Y, 16);
}

/* ------------------------------------------------------------------ */
/* inc32, GCTR (SP 800-38D sections 6.2, 6.5)                           */
/* ------------------------------------------------------------------ */

/* inc_32(X): the rightmost 32 bits, read as a big-endian integer, are
 * incremented modulo 2^32; the leftmost 96 bits are unchanged. */
void oracle_inc32(uint8_t b[16])
{
    for (int k = 15; k >= 12; k--) {
        b[k] = (uint8_t)(b[k] + 1);
        if (b[k] != 0) break;
    }
}

/* Algorithm 3: GCTR_K(ICB, X).  CB_1 = ICB, CB_i = inc_32(CB_{i-1}),
 * Y_i = X_i xor CIPH_K(CB_i); the final partial block uses the leftmost
 * bits of the last keystream block. */
void oracle_gctr(const uint8_t *w, int Nr, const uint8_t icb[16],
                 const uint8_t *X, size_t len, uint8_t *Y)
{
    uint8_t cb[16], ks[16];
    memcpy(cb, icb, 16);
    for (size_t off = 0; off < len; off += 16) {
        oracle_aes_encrypt_block(w, Nr, cb, ks);
        size_t n = (len - off < 16) ? (len - off) : 16;
        for (size_t k = 0; k < n; k++) Y[off + k] = (uint8_t)(X[off + k] ^ ks[k]);
        oracle_inc32(cb);
    }
}

/* ------------------------------------------------------------------ */
/* GCM-AE and GCM-AD (SP 800-38D sections 7.1, 7.2)                     */
/* ------------------------------------------------------------------ */

static void put_be64(uint8_t *p, uint64_t v)
{
    for (int k = 7; k >= 0; k--) { p[k] = (uint8_t)(v & 0xFF); v >>= 8; }
}

/* Serial GHASH over A || 0^v || C || 0^u || [len(A)]_64 || [len(C)]_64,
 * fed block by block in exactly that order (step 5 of Algorithm 4). */
static void ghash_aad_ct(const uint8_t H[16], const uint8_t *A, size_t alen,
                         const uint8_t *C, size_t clen, uint8_t S[16])
{
    uint8_t Y[16], blk[16];
    memset(Y, 0, 16);
    for (size_t off = 0; off < alen; off += 16) {
        memset(blk, 0, 16);
        size_t n = (alen - off < 16) ? (alen - off) : 16;
        memcpy(blk, A + off, n);
        for (int k = 0; k < 16; k++) Y[k] ^= blk[k];
        oracle_gf128_mul(Y, H, Y);
    }
    for (size_t off = 0; off < clen; off += 16) {
        memset(blk, 0, 16);
        size_t n = (clen - off < 16) ? (clen - off) : 16;
        memcpy(blk, C + off, n);
        for (int k = 0; k < 16; k++) Y[k] ^= blk[k];
        oracle_gf128_mul(Y, H, Y);
    }
    put_be64(blk, (uint64_t)alen * 8u);
    put_be64(blk + 8, (uint64_t)clen * 8u);
    for (int k = 0; k < 16; k++) Y[k] ^= blk[k];
    oracle_gf128_mul(Y, H, Y);
    memcpy(S, Y, 16);
}

/* Hash subkey H = CIPH_K(0^128) (Algorithm 4 step 1). */
void oracle_hash_subkey(const uint8_t *w, int Nr, uint8_t H[16])
{
    uint8_t zero[16];
    memset(zero, 0, 16);
    oracle_aes_encrypt_block(w, Nr, zero, H);
}

/* Pre-counter block J0 (Algorithm 4 step 2):
 *   len(IV) = 96:  J0 = IV || 0^31 || 1;
 *   otherwise:     J0 = GHASH_H(IV || 0^(s+64) || [len(IV)]_64),
 *                  s = 128*ceil(len(IV)/128) - len(IV). */
void oracle_j0(const uint8_t H[16], const uint8_t *iv, size_t iv_len, uint8_t J0[16])
{
    if (iv_len == 12) {
        memcpy(J0, iv, 12);
        J0[12] = 0; J0[13] = 0; J0[14] = 0; J0[15] = 1;
        return;
    }
    uint8_t Y[16], blk[16];
    memset(Y, 0, 16);
    for (size_t off = 0; off < iv_len; off += 16) {
        memset(blk, 0, 16);
        size_t n = (iv_len - off < 16) ? (iv_len - off) : 16;
        memcpy(blk, iv + off, n);
        for (int k = 0; k < 16; k++) Y[k] ^= blk[k];
        oracle_gf128_mul(Y, H, Y);
    }
    memset(blk, 0, 16);
    put_be64(blk + 8, (uint64_t)iv_len * 8u);
    for (int k = 0; k < 16; k++) Y[k] ^= blk[k];
    oracle_gf128_mul(Y, H, Y);
    memcpy(J0, Y, 16);
}

/* Algorithm 4 (GCM-AE).  Returns 0, or -1 on a bad key length or an
 * empty IV. */
int oracle_gcm_encrypt(const uint8_t *key, size_t key_len,
                       const uint8_t *iv, size_t iv_len,
                       const uint8_t *aad, size_t aad_len,
                       const uint8_t *pt, size_t len,
                       uint8_t *ct, uint8_t tag[16])
{
    uint8_t w[240], H[16], J0[16], icb[16], S[16];
    int Nr = oracle_aes_key_expansion(key, (int)key_len, w);
    if (Nr < 0 || iv_len == 0) return -1;
    oracle_hash_subkey(w, Nr, H);
    oracle_j0(H, iv, iv_len, J0);
    memcpy(icb, J0, 16);
    oracle_inc32(icb);
    oracle_gctr(w, Nr, icb, pt, len, ct);
    ghash_aad_ct(H, aad, aad_len, ct, len, S);
    oracle_gctr(w, Nr, J0, S, 16, tag);
    return 0;
}

/* Algorithm 5 (GCM-AD).  Returns 0 when the tag verifies; 1 on an
 * authentication failure, in which case pt is zero-filled; -1 on a bad
 * key length or an empty IV.  The tag comparison looks at every byte. */
int oracle_gcm_decrypt(const uint8_t *key, size_t key_len,
                       const uint8_t *iv, size_t iv_len,
                       const uint8_t *aad, size_t aad_len,
                       const uint8_t *ct, size_t len,
                       const uint8_t tag[16], uint8_t *pt)
{
    uint8_t w[240], H[16], J0[16], icb[16], S[16], T[16];
    int Nr = oracle_aes_key_expansion(key, (int)key_len, w);
    if (Nr < 0 || iv_len == 0) return -1;
    oracle_hash_subkey(w, Nr, H);
    oracle_j0(H, iv, iv_len, J0);
    memcpy(icb, J0, 16);
    oracle_inc32(icb);
    ghash_aad_ct(H, aad, aad_len, ct, len, S);
    oracle_gctr(w, Nr, J0, S, 16, T);
    uint8_t diff = 0;
    for (int k = 0; k < 16; k++) diff |= (uint8_t)(T[k] ^ tag[k]);
    if (diff != 0) {
        if (len) memset(pt, 0, len);
        return 1;
    }
    oracle_gctr(w, Nr, icb, ct, len, pt);
    return 0;
}

/* Keystream block CIPH_K(inc_32^i(J0)) for one block index i >= 1: the
 * counter of the i-th data block of GCTR(inc32(J0), .).  Applying inc_32
 * i times adds i to the rightmost 32 bits modulo 2^32; that closed form
 * is what is used here so that single blocks deep into a large message
 * can be checked one by one. */
void oracle_keystream_block(const uint8_t *key, size_t key_len,
                            const uint8_t J0[16], uint64_t i, uint8_t out[16])
{
    uint8_t w[240], cb[16];
    int Nr = oracle_aes_key_expansion(key, (int)key_len, w);
    memcpy(cb, J0, 16);
    uint32_t lo = ((uint32_t)cb[12] << 24) | ((uint32_t)cb[13] << 16) |
                  ((uint32_t)cb[14] << 8) | (uint32_t)cb[15];
    lo = (uint32_t)(lo + (uint32_t)(i & 0xFFFFFFFFu));
    cb[12] = (uint8_t)(lo >> 24); cb[13] = (uint8_t)(lo >> 16);
    cb[14] = (uint8_t)(lo >> 8);  cb[15] = (uint8_t)lo;
    oracle_aes_encrypt_block(w, Nr, cb, out);
}

/* Convenience: H and J0 for a key and IV (Algorithm 4 steps 1-2). */
int oracle_gcm_h_j0(const uint8_t *key, size_t key_len, const uint8_t *iv,
                    size_t iv_len, uint8_t H[16], uint8_t J0[16], uint8_t EJ0[16])
{
    uint8_t w[240];
    int Nr = oracle_aes_key_expansion(key, (int)key_len, w);
    if (Nr < 0 || iv_len == 0) return -1;
    oracle_hash_subkey(w, Nr, H);
    oracle_j0(H, iv, iv_len, J0);
    if (EJ0) oracle_aes_encrypt_block(w, Nr, J0, EJ0);
    return 0;
}

/* FITS DATASUM (the FITS checksum convention of Seaman, Pence and Rots,
 * which the paper's container writes through cfitsio, Sec. 3.2.2): the
 * 32-bit ones' complement sum of the data read as big-endian 32-bit words,
 * accumulated one word at a time with end-around carry.  A trailing partial
 * word is padded with zero bytes. */
uint32_t oracle_datasum(const uint8_t *data, size_t len)
{
    uint32_t sum = 0;
    for (size_t i = 0; i < len; i += 4) {
        uint32_t w = 0;
        for (size_t b = 0; b < 4; b++)
            w = (w << 8) | (i + b < len ? data[i + b] : 0u);
        uint32_t t = sum + w;
        if (t < w) t += 1; /* carry out of bit 31 wraps around to bit 0 */
        sum = t;
    }
    return sum;
}
