// Host build of the bitsliced AES (gcm_bitsliced.cuh + the generated S-box
// circuit), for the CPU test that compares it with the oracle's cipher.
// Reads lines "NR ROUNDKEYS_HEX J0_HEX CTR_0 ... CTR_31" (round keys as
// bytes in FIPS-197 order, the first 12 bytes of J0, 32 decimal counters)
// and prints the 32 keystream blocks in hex, one line per block.
#include <cstdio>
#include <cstring>

#include "gcm_bitsliced.cuh"

template <int NR>
static void run(const uint32_t *rk, const uint32_t j0w[3], uint32_t ctr[32])
{
    uint32_t km[128 * 15];
    for (int q = 0; q < 128 * (NR + 1); q++) km[q] = gcmgpu::round_key_word_bs(rk, q);
    uint32_t s[128];
    gcmgpu::load_counters_bs(s, j0w[0], j0w[1], j0w[2], ctr, km);
    gcmgpu::aes_rounds_bs<NR>(s, km);
    gcmgpu::unload_blocks_bs(s);
    for (int k = 0; k < 32; k++) {
        for (int w = 0; w < 4; w++)
            for (int b = 0; b < 4; b++) printf("%02x", (s[32 * w + k] >> (8 * b)) & 0xFFu);
        printf("\n");
    }
}

static uint32_t word_le(const unsigned char *b)
{
    return (uint32_t)b[0] | ((uint32_t)b[1] << 8) | ((uint32_t)b[2] << 16) | ((uint32_t)b[3] << 24);
}

int main()
{
    int nr;
    static char hk[1024], hj[64];
    while (scanf("%d %1023s %63s", &nr, hk, hj) == 3) {
        unsigned char kb[240], jb[12];
        const int nk = 16 * (nr + 1);
        for (int i = 0; i < nk; i++) {
            unsigned x;
            sscanf(hk + 2 * i, "%2x", &x);
            kb[i] = (unsigned char)x;
        }
        for (int i = 0; i < 12; i++) {
            unsigned x;
            sscanf(hj + 2 * i, "%2x", &x);
            jb[i] = (unsigned char)x;
        }
        uint32_t rk[60], j0w[3], ctr[32];
        for (int i = 0; i < 4 * (nr + 1); i++) rk[i] = word_le(kb + 4 * i);
        for (int i = 0; i < 3; i++) j0w[i] = word_le(jb + 4 * i);
        for (int k = 0; k < 32; k++) {
            unsigned long long c;
            if (scanf("%llu", &c) != 1) return 1;
            ctr[k] = (uint32_t)c;
        }
        if (nr == 10) run<10>(rk, j0w, ctr);
        else if (nr == 12) run<12>(rk, j0w, ctr);
        else run<14>(rk, j0w, ctr);
    }
    return 0;
}
