// gfc_fits.cu -- the FITS-aware wrapper of the C ABI (Sec. 3.2.2-3.2.3 and
// the API table of the paper).  Host code: it parses the header, chooses the
// AAD, and runs the data unit through gcm_encrypt / gcm_decrypt_verify.
//
// FITS framing (FITS standard): a header is a sequence of 2880-byte records
// of 80-character cards ending with the END card; the data unit that follows
// holds |BITPIX|/8 * NAXIS1 * ... * NAXISn bytes and is padded to whole
// records.  The data unit is encrypted with its padding (the padding is
// zero bytes in a plain file), the header stays in clear.
#include <cctype>
#include <cerrno>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <sys/random.h>

#include <cuda_runtime.h>

#include "gcm_ctx.h"
#include "gcmgpu.h"

namespace {

constexpr size_t REC = 2880;
constexpr size_t CARD = 80;

int set_result(gfc_result *out, int code, int warning, const char *msg)
{
    if (out) {
        out->error_code = code;
        out->warning_code = warning;
        snprintf(out->error_message, sizeof(out->error_message), "%s", msg ? msg : "");
    }
    return code;
}

// Keyword of a card: columns 1-8 without trailing blanks.
std::string keyword(const uint8_t *card)
{
    size_t n = 8;
    while (n > 0 && card[n - 1] == ' ') n--;
    return std::string(reinterpret_cast<const char *>(card), n);
}

// Integer value of a "KEY     = value / comment" card.
bool card_int(const uint8_t *card, int64_t *v)
{
    if (card[8] != '=' || card[9] != ' ') return false;
    size_t i = 10;
    while (i < CARD && card[i] == ' ') i++;
    bool neg = false;
    if (i < CARD && (card[i] == '-' || card[i] == '+')) {
        neg = card[i] == '-';
        i++;
    }
    if (i >= CARD || !isdigit(card[i])) return false;
    int64_t x = 0;
    while (i < CARD && isdigit(card[i])) {
        if (x > (INT64_MAX - 9) / 10) return false;
        x = x * 10 + (card[i] - '0');
        i++;
    }
    while (i < CARD && card[i] == ' ') i++;
    if (i < CARD && card[i] != '/') return false;
    *v = neg ? -x : x;
    return true;
}

bool card_logical_true(const uint8_t *card)
{
    if (card[8] != '=' || card[9] != ' ') return false;
    size_t i = 10;
    while (i < CARD && card[i] == ' ') i++;
    return i < CARD && card[i] == 'T';
}

int parse_layout(const uint8_t *fits, size_t len, gfc_layout *out, std::string *err)
{
    memset(out, 0, sizeof(*out));
    if (len < REC) {
        *err = "input shorter than one FITS record";
        return GCM_ERR_INVALID_ARG;
    }
    if (keyword(fits) != "SIMPLE" || !card_logical_true(fits)) {
        *err = "first card is not SIMPLE = T";
        return GCM_ERR_INVALID_ARG;
    }
    size_t end = 0;
    for (size_t off = 0; off + CARD <= len; off += CARD) {
        if (keyword(fits + off) == "END") {
            end = (off / REC + 1) * REC;
            break;
        }
    }
    if (!end || end > len) {
        *err = "no END card in the header";
        return GCM_ERR_INVALID_ARG;
    }
    int64_t bitpix = 0, naxis = -1;
    int64_t naxes[GFC_MAX_AXES + 1];
    bool have_bitpix = false;
    for (int i = 0; i <= GFC_MAX_AXES; i++) naxes[i] = -1;
    for (size_t off = 0; off < end; off += CARD) {
        const uint8_t *c = fits + off;
        const std::string k = keyword(c);
        int64_t v;
        if (k == "BITPIX" && card_int(c, &v)) {
            bitpix = v;
            have_bitpix = true;
        } else if (k == "NAXIS" && card_int(c, &v)) {
            naxis = v;
        } else if (k.size() > 5 && k.compare(0, 5, "NAXIS") == 0 && card_int(c, &v)) {
            const int idx = atoi(k.c_str() + 5);
            if (idx >= 1 && idx <= GFC_MAX_AXES) naxes[idx] = v;
        }
    }
    if (!have_bitpix || (bitpix != 8 && bitpix != 16 && bitpix != 32 && bitpix != 64 && bitpix != -32 &&
                         bitpix != -64)) {
        *err = "missing or invalid BITPIX";
        return GCM_ERR_INVALID_ARG;
    }
    if (naxis < 0 || naxis > GFC_MAX_AXES) {
        *err = "missing or invalid NAXIS";
        return GCM_ERR_INVALID_ARG;
    }
    uint64_t bytes = naxis > 0 ? (uint64_t)(bitpix < 0 ? -bitpix : bitpix) / 8 : 0;
    for (int i = 1; i <= naxis; i++) {
        if (naxes[i] < 0) {
            *err = "missing or negative NAXISn";
            return GCM_ERR_INVALID_ARG;
        }
        if (naxes[i] && bytes > (UINT64_MAX >> 2) / (uint64_t)naxes[i]) {
            *err = "data unit size overflows";
            return GCM_ERR_LENGTH_LIMIT;
        }
        bytes *= (uint64_t)naxes[i];
        if (i <= 16) out->naxes[i - 1] = naxes[i];
    }
    out->header_bytes = end;
    out->data_bytes = bytes;
    out->data_padded_bytes = (bytes + REC - 1) / REC * REC;
    out->bitpix = (int)bitpix;
    out->naxis = (int)naxis;
    return GCM_OK;
}

// AAD_Data = NONCE || Serialize(BITPIX) || Serialize(NAXIS) || Serialize(NAXIS1) ...
std::string structural_aad(const uint8_t iv[12], const gfc_layout &L, const uint8_t *hdr, size_t hdr_len)
{
    std::string a(reinterpret_cast<const char *>(iv), 12);
    a += std::to_string(L.bitpix);
    a += std::to_string(L.naxis);
    // Every axis, including those past the first 16 kept in the layout.
    for (int i = 1; i <= L.naxis; i++) {
        int64_t v = (i <= 16) ? L.naxes[i - 1] : 0;
        if (i > 16) {
            for (size_t off = 0; off < hdr_len; off += CARD) {
                if (keyword(hdr + off) == "NAXIS" + std::to_string(i)) {
                    card_int(hdr + off, &v);
                    break;
                }
            }
        }
        a += std::to_string(v);
    }
    return a;
}

// Reads the header of a file in device memory: copies records to the host
// until the END record.
int read_device_header(const uint8_t *dev, size_t len, cudaStream_t s, std::string *hdr, std::string *err)
{
    hdr->clear();
    std::string rec(REC, '\0');
    for (size_t off = 0; off + REC <= len; off += REC) {
        cudaError_t e = cudaMemcpyAsync(&rec[0], dev + off, REC, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            *err = std::string("reading the header from the device: ") + cudaGetErrorString(e);
            return GCM_ERR_CUDA;
        }
        *hdr += rec;
        for (size_t c = 0; c < REC; c += CARD)
            if (keyword(reinterpret_cast<const uint8_t *>(rec.data()) + c) == "END") return GCM_OK;
        if (hdr->size() > (64u << 20)) break;
    }
    *err = "no END card in the header";
    return GCM_ERR_INVALID_ARG;
}

int fits_call(gcm_ctx *ctx, bool decrypt, const uint8_t *key, size_t key_len, const uint8_t *fits, size_t fits_len,
              const uint8_t *iv_in, uint8_t *iv_out, const uint8_t *tag_in, uint8_t *tag_out, int aad_mode, int mem,
              void *stream, gfc_result *out)
{
    if (!out) return GCM_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->mem = mem;
    out->stream = stream;
    if (!ctx) return set_result(out, GCM_ERR_INVALID_ARG, 0, "context is NULL");
    if (!fits) return set_result(out, GCM_ERR_INVALID_ARG, 0, "input file is NULL");
    if (mem != GCM_MEM_DEVICE && mem != GCM_MEM_HOST)
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "mem must be GCM_MEM_DEVICE or GCM_MEM_HOST");
    if (aad_mode != GFC_AAD_HEADER && aad_mode != GFC_AAD_STRUCTURAL)
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "unknown AAD mode");
    if (decrypt && (!iv_in || !tag_in)) return set_result(out, GCM_ERR_INVALID_ARG, 0, "IV and tag are required");
    if (!decrypt && (!iv_out || !tag_out))
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "iv_out and tag_out are required");
    if (mem == GCM_MEM_DEVICE && ((uintptr_t)fits & 15u))
        return set_result(out, GCM_ERR_ALIGNMENT, 0, "device FITS buffer must be 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // Header and layout.
    std::string err;
    std::string dev_hdr;
    const uint8_t *hdr = fits;
    int rc;
    if (mem == GCM_MEM_DEVICE) {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(ctx->device);
        rc = read_device_header(fits, fits_len, s, &dev_hdr, &err);
        if (prev >= 0) cudaSetDevice(prev);
        if (rc) return set_result(out, rc, 0, err.c_str());
        hdr = reinterpret_cast<const uint8_t *>(dev_hdr.data());
    }
    gfc_layout L;
    rc = parse_layout(hdr, mem == GCM_MEM_DEVICE ? dev_hdr.size() : fits_len, &L, &err);
    if (rc) return set_result(out, rc, 0, err.c_str());
    const size_t total = L.header_bytes + L.data_padded_bytes;
    if (fits_len < L.header_bytes + L.data_bytes)
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "file shorter than its data unit");
    if (fits_len > total)
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "bytes after the primary data unit (only single-HDU files)");
    if (decrypt && fits_len != total)
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "encrypted file must hold the whole padded data unit");
    const bool padded_in_file = (fits_len == total);

    // IV.
    uint8_t iv[12];
    if (decrypt) {
        memcpy(iv, iv_in, 12);
    } else if (iv_in) {
        memcpy(iv, iv_in, 12);
    } else {
        ssize_t got = getrandom(iv, sizeof(iv), 0);
        if (got != (ssize_t)sizeof(iv)) return set_result(out, GCM_ERR_INVALID_ARG, 0, "getrandom failed");
    }
    if (!decrypt) memcpy(iv_out, iv, 12);

    // AAD bytes (host) for the structural mode.
    std::string aad_s;
    if (aad_mode == GFC_AAD_STRUCTURAL) aad_s = structural_aad(iv, L, hdr, L.header_bytes);

    // Output buffer: header | data unit | (device mode) AAD copy | tag slot.
    const size_t aad_dev_len = (mem == GCM_MEM_DEVICE && aad_mode == GFC_AAD_STRUCTURAL) ? aad_s.size() : 0;
    const size_t off_aad = (total + 255) / 256 * 256;
    const size_t off_tag = (off_aad + aad_dev_len + 255) / 256 * 256;
    const size_t alloc = off_tag + 256;
    uint8_t *buf = nullptr;
    cudaError_t e;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    if (mem == GCM_MEM_DEVICE)
        e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&buf), alloc, ctx->pool, s);
    else
        e = cudaMallocHost(reinterpret_cast<void **>(&buf), alloc);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (prev >= 0) cudaSetDevice(prev);
        return set_result(out, GCM_ERR_NO_MEMORY, 0, "cannot allocate the result buffer");
    }
    out->data_buffer = buf;
    out->buffer_size = total;
    uint8_t *data_out = buf + L.header_bytes;
    const uint8_t *data_in = fits + L.header_bytes;
    if (mem == GCM_MEM_DEVICE) {
        e = cudaMemcpyAsync(buf, fits, L.header_bytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && !padded_in_file) {
            e = cudaMemcpyAsync(data_out, data_in, L.data_bytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(data_out + L.data_bytes, 0, L.data_padded_bytes - L.data_bytes, s);
            data_in = data_out;
        }
        if (e == cudaSuccess && aad_dev_len)
            e = cudaMemcpyAsync(buf + off_aad, aad_s.data(), aad_dev_len, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && decrypt) e = cudaMemcpyAsync(buf + off_tag, tag_in, 16, cudaMemcpyHostToDevice, s);
    } else {
        memcpy(buf, fits, L.header_bytes);
        if (!padded_in_file) {
            memcpy(data_out, data_in, L.data_bytes);
            memset(data_out + L.data_bytes, 0, L.data_padded_bytes - L.data_bytes);
            data_in = data_out;
        }
        e = cudaSuccess;
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        gfc_result_free(ctx, out);
        return set_result(out, GCM_ERR_CUDA, 0, cudaGetErrorString(e));
    }

    const uint8_t *aad;
    size_t aad_len;
    if (aad_mode == GFC_AAD_HEADER) {
        aad = (mem == GCM_MEM_DEVICE) ? buf : fits;
        aad_len = L.header_bytes;
    } else {
        aad = (mem == GCM_MEM_DEVICE) ? buf + off_aad : reinterpret_cast<const uint8_t *>(aad_s.data());
        aad_len = aad_s.size();
    }
    uint8_t *tag_slot = (mem == GCM_MEM_DEVICE) ? buf + off_tag : nullptr;
    uint8_t host_tag[16];
    uint32_t datasum = 0;
    bool datasum_done = false;
    if (!decrypt) {
        rc = gcmgpu::ctx_run_with_datasum(ctx, key, key_len, iv, 12, aad, aad_len, data_in, L.data_padded_bytes, data_out,
                                  mem == GCM_MEM_DEVICE ? tag_slot : host_tag, false, mem, stream, &datasum,
                                  &datasum_done);
        if (rc == GCM_OK && mem == GCM_MEM_DEVICE) {
            cudaGetDevice(&prev);
            cudaSetDevice(ctx->device);
            e = cudaMemcpyAsync(host_tag, tag_slot, 16, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (prev >= 0) cudaSetDevice(prev);
            if (e != cudaSuccess) rc = GCM_ERR_CUDA;
        }
        if (rc == GCM_OK) memcpy(tag_out, host_tag, 16);
    } else {
        memcpy(host_tag, tag_in, 16);
        rc = gcmgpu::ctx_run_with_datasum(ctx, key, key_len, iv, 12, aad, aad_len, data_in, L.data_padded_bytes, data_out,
                                  mem == GCM_MEM_DEVICE ? tag_slot : host_tag, true, mem, stream, &datasum,
                                  &datasum_done);
    }
    out->datasum = datasum;
    out->datasum_valid = datasum_done ? 1 : 0;
    if (rc == GCM_ERR_AUTH)
        return set_result(out, rc, 2, "authentication tag mismatch: payload suppressed (data unit zero-filled)");
    if (rc != GCM_OK) {
        std::string m = gcm_last_error();
        gfc_result_free(ctx, out);
        return set_result(out, rc, 0, m.c_str());
    }
    return set_result(out, GCM_OK, 0, "");
}

}  // namespace

extern "C" {

int gfc_fits_layout(const uint8_t *fits, size_t len, gfc_layout *out)
{
    if (!fits || !out) return GCM_ERR_INVALID_ARG;
    std::string err;
    return parse_layout(fits, len, out, &err);
}

int gfc_fits_encrypt(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *fits, size_t fits_len,
                     const uint8_t *iv12, uint8_t *iv_out, uint8_t *tag_out, int aad_mode, int mem, void *stream,
                     gfc_result *out)
{
    return fits_call(ctx, false, key, key_len, fits, fits_len, iv12, iv_out, nullptr, tag_out, aad_mode, mem,
                     stream, out);
}

int gfc_fits_decrypt_verify(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *fits_enc, size_t len,
                            const uint8_t *iv12, const uint8_t *tag, int aad_mode, int mem, void *stream,
                            gfc_result *out)
{
    return fits_call(ctx, true, key, key_len, fits_enc, len, iv12, nullptr, tag, nullptr, aad_mode, mem, stream,
                     out);
}

void gfc_result_free(gcm_ctx *ctx, gfc_result *res)
{
    if (!res || !res->data_buffer) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (ctx) cudaSetDevice(ctx->device);
    if (res->mem == GCM_MEM_DEVICE)
        cudaFreeAsync(res->data_buffer, static_cast<cudaStream_t>(res->stream));
    else
        cudaFreeHost(res->data_buffer);
    if (prev >= 0) cudaSetDevice(prev);
    res->data_buffer = nullptr;
    res->buffer_size = 0;
}

}  // extern "C"
