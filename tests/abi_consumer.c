/* A C99 program that uses the library through include/gcmgpu.h alone (no
 * Python, no C++): GCM-AE of a deterministic message in host memory,
 * GCM-AD of the result, and a tampered tag that must be refused with the
 * output zero-filled.  Usage: abi_consumer <len> <ciphertext-out-file>;
 * prints the tag in hex.  Exit status 0 only if every step behaved. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "gcmgpu.h"

static int fail(const char *what)
{
    fprintf(stderr, "%s: %s\n", what, gcm_last_error());
    return 1;
}

int main(int argc, char **argv)
{
    uint8_t key[32], iv[12], aad[20], tag[16];
    uint8_t *pt, *ct, *back;
    size_t len, i;
    gcm_ctx *ctx = NULL;
    int rc;
    FILE *f;

    if (argc != 3) {
        fprintf(stderr, "usage: %s <len> <ciphertext-out-file>\n", argv[0]);
        return 2;
    }
    len = (size_t)strtoull(argv[1], NULL, 10);
    for (i = 0; i < sizeof key; i++) key[i] = (uint8_t)(11u * i + 1u);
    for (i = 0; i < sizeof iv; i++) iv[i] = (uint8_t)(0xA0u + i);
    for (i = 0; i < sizeof aad; i++) aad[i] = (uint8_t)(3u * i);
    /* 16-byte aligned buffers, as the host fast path wants */
    pt = (uint8_t *)calloc(len / 16 + 2, 16);
    ct = (uint8_t *)calloc(len / 16 + 2, 16);
    back = (uint8_t *)calloc(len / 16 + 2, 16);
    if (!pt || !ct || !back) return 1;
    for (i = 0; i < len; i++) pt[i] = (uint8_t)(7u * i + 3u);

    if (gcm_ctx_create(&ctx, 0, 0) != GCM_OK) return fail("gcm_ctx_create");
    rc = gcm_encrypt(ctx, key, sizeof key, iv, sizeof iv, aad, sizeof aad, pt, len, ct, tag, GCM_MEM_HOST, NULL);
    if (rc != GCM_OK) return fail("gcm_encrypt");
    rc = gcm_decrypt_verify(ctx, key, sizeof key, iv, sizeof iv, aad, sizeof aad, ct, len, tag, back, GCM_MEM_HOST,
                            NULL);
    if (rc != GCM_OK) return fail("gcm_decrypt_verify");
    if (len && memcmp(back, pt, len) != 0) {
        fprintf(stderr, "round trip differs\n");
        return 1;
    }
    tag[15] ^= 0x01u;
    memset(back, 0x55, len);
    rc = gcm_decrypt_verify(ctx, key, sizeof key, iv, sizeof iv, aad, sizeof aad, ct, len, tag, back, GCM_MEM_HOST,
                            NULL);
    tag[15] ^= 0x01u;
    if (rc != GCM_ERR_AUTH) {
        fprintf(stderr, "tampered tag: status %d\n", rc);
        return 1;
    }
    for (i = 0; i < len; i++)
        if (back[i] != 0) {
            fprintf(stderr, "output not zero-filled at %lu\n", (unsigned long)i);
            return 1;
        }
    gcm_ctx_destroy(ctx);

    f = fopen(argv[2], "wb");
    if (!f || fwrite(ct, 1, len, f) != len || fclose(f) != 0) return 1;
    for (i = 0; i < 16; i++) printf("%02x", tag[i]);
    printf("\n");
    free(pt);
    free(ct);
    free(back);
    return 0;
}
