// Host build of the library's field multiplier (gcm_device.cuh), for the CPU
// test that compares it with the oracle.  Reads lines "A B" (two 16-byte
// blocks in hex, GCM byte order) from stdin and prints A*B in hex per line.
#include <cstdio>
#include <cstring>

#include "gcm_device.cuh"

static void to_words(const unsigned char *b, uint32_t w[4])
{
    for (int i = 0; i < 4; i++)
        w[i] = ((uint32_t)b[4 * i] << 24) | ((uint32_t)b[4 * i + 1] << 16) | ((uint32_t)b[4 * i + 2] << 8) |
               (uint32_t)b[4 * i + 3];
}

int main()
{
    char ha[64], hb[64];
    while (scanf("%63s %63s", ha, hb) == 2) {
        unsigned char a[16], b[16];
        for (int i = 0; i < 16; i++) {
            unsigned x, y;
            sscanf(ha + 2 * i, "%2x", &x);
            sscanf(hb + 2 * i, "%2x", &y);
            a[i] = (unsigned char)x;
            b[i] = (unsigned char)y;
        }
        uint32_t wa[4], wb[4], wz[4];
        to_words(a, wa);
        to_words(b, wb);
        gcmgpu::gf_mul_words(wa, wb, wz);
        for (int i = 0; i < 4; i++) printf("%08x", wz[i]);
        printf("\n");
    }
    return 0;
}
