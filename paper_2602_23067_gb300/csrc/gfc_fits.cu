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
#include <map>
#include <string>
#include <sys/random.h>
#include <vector>

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

// ---------------------------------------------------------------------
// The paper's dual-key container (Sec. 3.2.2): HDU 0 holds the nonces, the
// two tags, the ORIG_* structural keywords and ENCHDR (the original header
// encrypted with the header key); HDU 1 is a one-row binary table whose
// single column holds the pixel bytes encrypted with the data key, with
// AAD_D = NONCE_D || Serialize(ORIG_BITPIX) || Serialize(ORIG_NAXIS) || ...
// Encodings where the paper is silent: nonces and tags as lowercase hex
// strings, the tag keywords shortened to AUTHTG_H / AUTHTG_D (eight
// characters), ENCHDR as a lowercase hex long string of 64 characters per
// card (CONTINUE convention), ENCHDR authenticated without AAD.
// ---------------------------------------------------------------------
std::string pad80(const std::string &t) { return t + std::string(CARD - t.size(), ' '); }

std::string kcard_int(const char *key, int64_t v)
{
    char b[96];
    snprintf(b, sizeof(b), "%-8s= %20lld", key, (long long)v);
    return pad80(b);
}

std::string kcard_logical(const char *key, bool v)
{
    char b[96];
    snprintf(b, sizeof(b), "%-8s= %20s", key, v ? "T" : "F");
    return pad80(b);
}

std::string kcard_str(const char *key, const std::string &v)
{
    std::string t = v;
    if (t.size() < 8) t += std::string(8 - t.size(), ' ');
    char b[96];
    snprintf(b, sizeof(b), "%-8s= '%s'", key, t.c_str());
    return pad80(b);
}

std::string hexs(const uint8_t *p, size_t n)
{
    static const char *d = "0123456789abcdef";
    std::string s(2 * n, '0');
    for (size_t i = 0; i < n; i++) {
        s[2 * i] = d[p[i] >> 4];
        s[2 * i + 1] = d[p[i] & 15];
    }
    return s;
}

bool unhex(const std::string &s, std::string *out)
{
    if (s.size() % 2) return false;
    out->assign(s.size() / 2, '\0');
    for (size_t i = 0; i < s.size(); i += 2) {
        int v = 0;
        for (int k = 0; k < 2; k++) {
            const char c = s[i + k];
            const int x = (c >= '0' && c <= '9') ? c - '0' : (c >= 'a' && c <= 'f') ? c - 'a' + 10 : -1;
            if (x < 0) return false;
            v = v * 16 + x;
        }
        (*out)[i / 2] = (char)v;
    }
    return true;
}

// Cards + END, blank-filled to whole records.
std::string header_records(const std::vector<std::string> &cards)
{
    std::string h;
    for (const auto &c : cards) h += c;
    h += pad80("END");
    h += std::string((REC - h.size() % REC) % REC, ' ');
    return h;
}

size_t header_records_size(size_t n_cards) { return ((n_cards + 1) * CARD + REC - 1) / REC * REC; }

// FITS checksum convention (the CHECKSUM / DATASUM keywords the container
// carries in both HDUs, Sec. 3.2.2): 32-bit ones' complement arithmetic on
// big-endian words.
uint32_t ones_add32(uint32_t a, uint32_t b)
{
    uint64_t t = (uint64_t)a + b;
    while (t >> 32) t = (t & 0xFFFFFFFFull) + (t >> 32);
    return (uint32_t)t;
}

uint32_t ones_sum_words(const std::string &bytes)  // length a multiple of 4
{
    uint64_t t = 0;
    for (size_t i = 0; i + 4 <= bytes.size(); i += 4) {
        const uint8_t *q = reinterpret_cast<const uint8_t *>(bytes.data()) + i;
        t += ((uint32_t)q[0] << 24) | ((uint32_t)q[1] << 16) | ((uint32_t)q[2] << 8) | (uint32_t)q[3];
    }
    while (t >> 32) t = (t & 0xFFFFFFFFull) + (t >> 32);
    return (uint32_t)t;
}

// The CHECKSUM value for a 32-bit v (the complement of the HDU's sum): every
// byte of v, most significant first, gives four characters 0x30 + byte / 4
// with the first one raised by byte % 4, so their codes add up to the byte
// plus 4 * 0x30; characters in the punctuation ranges 0x3A..0x40 and
// 0x5B..0x60 are avoided by shifting one unit inside the pairs (0,1) and
// (2,3).  Byte i's characters go to positions i, i + 4, i + 8, i + 12, and
// the string is rotated right by one place: the value starts at column 12
// of its card, one byte before a 4-byte boundary of the header.
std::string checksum_value(uint32_t v)
{
    auto punct = [](int c) { return (c >= 0x3A && c <= 0x40) || (c >= 0x5B && c <= 0x60); };
    char plain[16];
    for (int i = 0; i < 4; i++) {
        const int byte = (int)((v >> (24 - 8 * i)) & 0xFFu);
        int c[4] = {0x30 + byte / 4 + byte % 4, 0x30 + byte / 4, 0x30 + byte / 4, 0x30 + byte / 4};
        for (int j = 0; j < 4; j += 2)
            while (punct(c[j]) || punct(c[j + 1])) {
                c[j]++;
                c[j + 1]--;
            }
        for (int j = 0; j < 4; j++) plain[4 * j + i] = (char)c[j];
    }
    std::string out(16, '0');
    for (int k = 0; k < 16; k++) out[k] = plain[(k + 15) % 16];
    return out;
}

// Header records of `cards` followed by DATASUM (data_sum_text) and a
// CHECKSUM whose value makes the header together with a data unit of sum
// data_sum add up to -0 (0xFFFFFFFF).
std::string header_records_checksummed(std::vector<std::string> cards, uint32_t data_sum,
                                       const std::string &data_sum_text)
{
    cards.push_back(kcard_str("DATASUM", data_sum_text));
    const size_t at = cards.size() * CARD + 11;  // the CHECKSUM value's first byte
    cards.push_back(kcard_str("CHECKSUM", std::string(16, '0')));
    std::string h = header_records(cards);
    const uint32_t total = ones_add32(ones_sum_words(h), data_sum);
    h.replace(at, 16, checksum_value(~total));
    return h;
}

constexpr size_t HEX_PER_CARD = 64;

// Keyword -> value text (strings unquoted and right-trimmed, long strings
// joined over CONTINUE cards, comments dropped) of the header at hdr.
std::map<std::string, std::string> header_keys(const std::string &hdr)
{
    std::map<std::string, std::string> k;
    std::string last;
    for (size_t off = 0; off + CARD <= hdr.size(); off += CARD) {
        const std::string card = hdr.substr(off, CARD);
        const std::string name = keyword(reinterpret_cast<const uint8_t *>(card.data()));
        if (name == "END") break;
        if (name == "CONTINUE" && !last.empty()) {
            const size_t q0 = card.find('\''), q1 = card.rfind('\'');
            std::string &v = k[last];
            if (q0 != std::string::npos && q1 > q0 && !v.empty() && v.back() == '&') {
                v.pop_back();
                v += card.substr(q0 + 1, q1 - q0 - 1);
            }
            continue;
        }
        if (card.compare(8, 2, "= ") != 0) {
            last.clear();
            continue;
        }
        std::string v = card.substr(10);
        const size_t a = v.find_first_not_of(' ');
        v = (a == std::string::npos) ? "" : v.substr(a);
        if (!v.empty() && v[0] == '\'') {
            const size_t q1 = v.rfind('\'');
            v = v.substr(1, q1 > 0 ? q1 - 1 : 0);
            while (!v.empty() && v.back() == ' ') v.pop_back();
        } else {
            const size_t sl = v.find('/');
            if (sl != std::string::npos) v = v.substr(0, sl);
            while (!v.empty() && v.back() == ' ') v.pop_back();
        }
        k[name] = v;
        last = name;
    }
    return k;
}

bool key_int(const std::map<std::string, std::string> &k, const std::string &name, int64_t *v)
{
    auto it = k.find(name);
    if (it == k.end() || it->second.empty()) return false;
    char *end = nullptr;
    const long long x = strtoll(it->second.c_str(), &end, 10);
    if (*end) return false;
    *v = x;
    return true;
}

bool check_key(const uint8_t *key, size_t key_len)
{
    return key && (key_len == 16 || key_len == 24 || key_len == 32);
}

// Copies host bytes into the result buffer (device or pinned host).
cudaError_t put_bytes(uint8_t *dst, const void *src, size_t n, int mem, cudaStream_t s)
{
    if (!n) return cudaSuccess;
    if (mem == GCM_MEM_DEVICE) return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s);
    memcpy(dst, src, n);
    return cudaSuccess;
}

cudaError_t zero_bytes(uint8_t *dst, size_t n, int mem, cudaStream_t s)
{
    if (!n) return cudaSuccess;
    if (mem == GCM_MEM_DEVICE) return cudaMemsetAsync(dst, 0, n, s);
    memset(dst, 0, n);
    return cudaSuccess;
}

struct DevSel {
    int prev = -1;
    explicit DevSel(int d)
    {
        cudaGetDevice(&prev);
        cudaSetDevice(d);
    }
    ~DevSel()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int container_encrypt(gcm_ctx *ctx, const uint8_t *key_h, size_t key_h_len, const uint8_t *key_d, size_t key_d_len,
                      const uint8_t *fits, size_t fits_len, const uint8_t *nonce_h_in, const uint8_t *nonce_d_in,
                      int mem, void *stream, gfc_result *out)
{
    if (!out) return GCM_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->mem = mem;
    out->stream = stream;
    if (!ctx || !fits) return set_result(out, GCM_ERR_INVALID_ARG, 0, "context or input is NULL");
    if (!check_key(key_h, key_h_len) || !check_key(key_d, key_d_len))
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "header and data keys must be 16, 24 or 32 bytes");
    if (mem != GCM_MEM_DEVICE && mem != GCM_MEM_HOST)
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "mem must be GCM_MEM_DEVICE or GCM_MEM_HOST");
    if (mem == GCM_MEM_DEVICE && ((uintptr_t)fits & 15u))
        return set_result(out, GCM_ERR_ALIGNMENT, 0, "device FITS buffer must be 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevSel sel(ctx->device);
    std::string err, hdr_s;
    int rc;
    if (mem == GCM_MEM_DEVICE) {
        rc = read_device_header(fits, fits_len, s, &hdr_s, &err);
        if (rc) return set_result(out, rc, 0, err.c_str());
    } else {
        gfc_layout L0;
        rc = parse_layout(fits, fits_len, &L0, &err);
        if (rc) return set_result(out, rc, 0, err.c_str());
        hdr_s.assign(reinterpret_cast<const char *>(fits), L0.header_bytes);
    }
    gfc_layout L;
    rc = parse_layout(reinterpret_cast<const uint8_t *>(hdr_s.data()), hdr_s.size(), &L, &err);
    if (rc) return set_result(out, rc, 0, err.c_str());
    hdr_s.resize(L.header_bytes);
    if (fits_len < L.header_bytes + L.data_bytes)
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "file shorter than its data unit");
    if (fits_len > L.header_bytes + L.data_padded_bytes)
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "bytes after the primary data unit (only single-HDU files)");
    if (L.naxis > 9) return set_result(out, GCM_ERR_INVALID_ARG, 0, "at most 9 axes (ORIG_NA1..ORIG_NA9)");

    uint8_t nonce_h[12], nonce_d[12];
    if (nonce_h_in) memcpy(nonce_h, nonce_h_in, 12);
    if (nonce_d_in) memcpy(nonce_d, nonce_d_in, 12);
    if ((!nonce_h_in && getrandom(nonce_h, 12, 0) != 12) || (!nonce_d_in && getrandom(nonce_d, 12, 0) != 12))
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "getrandom failed");

    // ENCHDR: the header records under the header key (host memory, small).
    std::string enchdr(hdr_s.size(), '\0');
    uint8_t tag_h[16];
    rc = gcm_encrypt(ctx, key_h, key_h_len, nonce_h, 12, nullptr, 0, reinterpret_cast<const uint8_t *>(hdr_s.data()),
                     hdr_s.size(), reinterpret_cast<uint8_t *>(&enchdr[0]), tag_h, GCM_MEM_HOST, nullptr);
    if (rc) return set_result(out, rc, 0, gcm_last_error());

    // Layout of the container.
    const std::string hx = hexs(reinterpret_cast<const uint8_t *>(enchdr.data()), enchdr.size());
    const size_t n_hex_cards = (hx.size() + HEX_PER_CARD - 1) / HEX_PER_CARD;
    const size_t prim_cards = 12 + (size_t)L.naxis + (n_hex_cards ? n_hex_cards : 1);  // + DATASUM, CHECKSUM
    const size_t prim_bytes = header_records_size(prim_cards);
    const size_t ext_bytes = header_records_size(12);
    const size_t N = L.data_bytes;
    const size_t blob_off = prim_bytes + ext_bytes;
    const size_t total = blob_off + (N + REC - 1) / REC * REC;
    const std::string aad = structural_aad(nonce_d, L, reinterpret_cast<const uint8_t *>(hdr_s.data()), hdr_s.size());
    const size_t off_aad = (total + 255) / 256 * 256;
    const size_t off_tag = (off_aad + aad.size() + 255) / 256 * 256;
    const size_t alloc = off_tag + 256;
    uint8_t *buf = nullptr;
    cudaError_t e = (mem == GCM_MEM_DEVICE)
                        ? cudaMallocFromPoolAsync(reinterpret_cast<void **>(&buf), alloc, ctx->pool, s)
                        : cudaMallocHost(reinterpret_cast<void **>(&buf), alloc);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_result(out, GCM_ERR_NO_MEMORY, 0, "cannot allocate the result buffer");
    }
    out->data_buffer = buf;
    out->buffer_size = total;

    // Pixels under the data key with AAD_D, straight into the table's data
    // unit; the DATASUM of the ciphertext comes from the same pass.
    const uint8_t *aad_p = reinterpret_cast<const uint8_t *>(aad.data());
    if (mem == GCM_MEM_DEVICE) {
        e = put_bytes(buf + off_aad, aad.data(), aad.size(), mem, s);
        aad_p = buf + off_aad;
    }
    if (e == cudaSuccess) e = zero_bytes(buf + blob_off + N, total - blob_off - N, mem, s);
    if (e != cudaSuccess) {
        gfc_result_free(ctx, out);
        return set_result(out, GCM_ERR_CUDA, 0, cudaGetErrorString(e));
    }
    uint8_t tag_d[16];
    uint8_t *tag_slot = (mem == GCM_MEM_DEVICE) ? buf + off_tag : tag_d;
    uint32_t dsum = 0;
    bool dsum_done = false;
    rc = gcmgpu::ctx_run_with_datasum(ctx, key_d, key_d_len, nonce_d, 12, aad_p, aad.size(), fits + L.header_bytes, N,
                                      buf + blob_off, tag_slot, false, mem, stream, &dsum, &dsum_done);
    if (rc == GCM_OK && mem == GCM_MEM_DEVICE) {
        e = cudaMemcpyAsync(tag_d, tag_slot, 16, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = GCM_ERR_CUDA;
    }
    if (rc != GCM_OK) {
        std::string m = gcm_last_error();
        gfc_result_free(ctx, out);
        return set_result(out, rc, 0, m.c_str());
    }

    // The two headers, now that both tags are known.
    std::vector<std::string> pc = {kcard_logical("SIMPLE", true), kcard_int("BITPIX", 8), kcard_int("NAXIS", 0),
                                   kcard_logical("EXTEND", true), kcard_str("NONCE_H", hexs(nonce_h, 12)),
                                   kcard_str("NONCE_D", hexs(nonce_d, 12)), kcard_str("AUTHTG_H", hexs(tag_h, 16)),
                                   kcard_str("AUTHTG_D", hexs(tag_d, 16)), kcard_int("ORIG_BPX", L.bitpix),
                                   kcard_int("ORIG_NAX", L.naxis)};
    for (int i = 1; i <= L.naxis; i++) {
        const std::string name = "ORIG_NA" + std::to_string(i);
        pc.push_back(kcard_int(name.c_str(), L.naxes[i - 1]));
    }
    for (size_t i = 0; i < (n_hex_cards ? n_hex_cards : 1); i++) {
        const std::string part = hx.substr(i * HEX_PER_CARD, HEX_PER_CARD);
        const std::string amp = (i + 1 < n_hex_cards) ? "&" : "";
        pc.push_back(pad80(i == 0 ? std::string("ENCHDR  = '") + part + amp + "'"
                                  : std::string("CONTINUE  '") + part + amp + "'"));
    }
    const std::string prim = header_records_checksummed(pc, 0, "0");  // no data unit
    std::vector<std::string> xc = {kcard_str("XTENSION", "BINTABLE"), kcard_int("BITPIX", 8), kcard_int("NAXIS", 2),
                                   kcard_int("NAXIS1", (int64_t)N), kcard_int("NAXIS2", 1), kcard_int("PCOUNT", 0),
                                   kcard_int("GCOUNT", 1), kcard_int("TFIELDS", 1), kcard_str("TTYPE1", "ENCDATA"),
                                   kcard_str("TFORM1", std::to_string(N) + "B")};
    // DATASUM and CHECKSUM need the data unit's sum, which the staged
    // host-memory path does not compute: there both cards are left out.
    const std::string ext = dsum_done ? header_records_checksummed(xc, dsum, std::to_string(dsum)) : header_records(xc);
    e = put_bytes(buf, prim.data(), prim.size(), mem, s);
    if (e == cudaSuccess) e = put_bytes(buf + prim_bytes, ext.data(), ext.size(), mem, s);
    if (e == cudaSuccess && mem == GCM_MEM_DEVICE) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        gfc_result_free(ctx, out);
        return set_result(out, GCM_ERR_CUDA, 0, cudaGetErrorString(e));
    }
    out->datasum = dsum;
    out->datasum_valid = dsum_done ? 1 : 0;
    return set_result(out, GCM_OK, 0, "");
}

int decrypt_frame(gcm_ctx *ctx, const uint8_t *cont, size_t len, const uint8_t *key_h, size_t key_h_len,
                  const uint8_t *key_d, size_t key_d_len, int mem, void *stream, gfc_result *out)
{
    if (!out) return GCM_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->mem = mem;
    out->stream = stream;
    if (!ctx || !cont) return set_result(out, GCM_ERR_INVALID_ARG, 0, "context or input is NULL");
    if ((key_h && !check_key(key_h, key_h_len)) || (key_d && !check_key(key_d, key_d_len)))
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "keys must be 16, 24 or 32 bytes (or NULL: not provisioned)");
    if (mem != GCM_MEM_DEVICE && mem != GCM_MEM_HOST)
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "mem must be GCM_MEM_DEVICE or GCM_MEM_HOST");
    if (mem == GCM_MEM_DEVICE && ((uintptr_t)cont & 15u))
        return set_result(out, GCM_ERR_ALIGNMENT, 0, "device container buffer must be 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevSel sel(ctx->device);
    std::string err, prim, ext;
    int rc;
    // The two headers (host copies).
    auto read_hdr = [&](size_t off, std::string *h) -> int {
        if (off >= len) return GCM_ERR_INVALID_ARG;
        if (mem == GCM_MEM_DEVICE) return read_device_header(cont + off, len - off, s, h, &err);
        h->clear();
        for (size_t o = off; o + REC <= len; o += REC) {
            h->append(reinterpret_cast<const char *>(cont + o), REC);
            for (size_t c = 0; c < REC; c += CARD)
                if (keyword(cont + o + c) == "END") return GCM_OK;
        }
        err = "no END card";
        return GCM_ERR_INVALID_ARG;
    };
    rc = read_hdr(0, &prim);
    if (rc == GCM_OK) rc = read_hdr(prim.size(), &ext);
    if (rc) return set_result(out, rc, 0, err.empty() ? "not a container" : err.c_str());
    const auto P = header_keys(prim), X = header_keys(ext);
    int64_t n = 0, bitpix = 0, naxis = -1;
    std::string nonce_h, nonce_d, tag_h, tag_d, enchdr;
    const auto str = [](const std::map<std::string, std::string> &k, const char *name) {
        auto it = k.find(name);
        return it == k.end() ? std::string() : it->second;
    };
    if (str(X, "XTENSION") != "BINTABLE" || !key_int(X, "NAXIS1", &n) || n < 0 ||
        !unhex(str(P, "NONCE_H"), &nonce_h) || nonce_h.size() != 12 || !unhex(str(P, "NONCE_D"), &nonce_d) ||
        nonce_d.size() != 12 || !unhex(str(P, "AUTHTG_H"), &tag_h) || tag_h.size() != 16 ||
        !unhex(str(P, "AUTHTG_D"), &tag_d) || tag_d.size() != 16 || !key_int(P, "ORIG_BPX", &bitpix) ||
        !key_int(P, "ORIG_NAX", &naxis) || naxis < 0 || naxis > 9 || !unhex(str(P, "ENCHDR"), &enchdr))
        return set_result(out, GCM_ERR_INVALID_ARG, 0, "missing or malformed container keywords");
    gfc_layout L;
    memset(&L, 0, sizeof(L));
    L.bitpix = (int)bitpix;
    L.naxis = (int)naxis;
    for (int i = 1; i <= naxis; i++) {
        int64_t v;
        if (!key_int(P, ("ORIG_NA" + std::to_string(i)).c_str(), &v) || v < 0)
            return set_result(out, GCM_ERR_INVALID_ARG, 0, "missing ORIG_NAn");
        L.naxes[i - 1] = v;
    }
    const size_t blob_off = prim.size() + ext.size();
    if (blob_off + (size_t)n > len) return set_result(out, GCM_ERR_INVALID_ARG, 0, "container shorter than its table");

    // Header: ENCHDR under the header key, else the fallback from ORIG_*.
    int warning = 0;
    std::string header;
    if (key_h && !enchdr.empty() && enchdr.size() % REC == 0) {
        std::string h(enchdr.size(), '\0');
        rc = gcm_decrypt_verify(ctx, key_h, key_h_len, reinterpret_cast<const uint8_t *>(nonce_h.data()), 12, nullptr,
                                0, reinterpret_cast<const uint8_t *>(enchdr.data()), enchdr.size(),
                                reinterpret_cast<const uint8_t *>(tag_h.data()), reinterpret_cast<uint8_t *>(&h[0]),
                                GCM_MEM_HOST, nullptr);
        if (rc == GCM_OK) header = h;
        else if (rc != GCM_ERR_AUTH) return set_result(out, rc, 0, gcm_last_error());
    }
    if (header.empty()) {
        std::vector<std::string> c = {kcard_logical("SIMPLE", true), kcard_int("BITPIX", bitpix),
                                      kcard_int("NAXIS", naxis)};
        for (int i = 1; i <= naxis; i++)
            c.push_back(kcard_int(("NAXIS" + std::to_string(i)).c_str(), L.naxes[i - 1]));
        header = header_records(c);
        warning = 1;
    }
    const size_t total = header.size() + ((size_t)n + REC - 1) / REC * REC;
    const std::string aad = structural_aad(reinterpret_cast<const uint8_t *>(nonce_d.data()), L, nullptr, 0);
    const size_t off_aad = (total + 255) / 256 * 256;
    const size_t off_tag = (off_aad + aad.size() + 255) / 256 * 256;
    const size_t alloc = off_tag + 256;
    uint8_t *buf = nullptr;
    cudaError_t e = (mem == GCM_MEM_DEVICE)
                        ? cudaMallocFromPoolAsync(reinterpret_cast<void **>(&buf), alloc, ctx->pool, s)
                        : cudaMallocHost(reinterpret_cast<void **>(&buf), alloc);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_result(out, GCM_ERR_NO_MEMORY, 0, "cannot allocate the result buffer");
    }
    out->data_buffer = buf;
    out->buffer_size = total;
    e = put_bytes(buf, header.data(), header.size(), mem, s);
    if (e == cudaSuccess) e = zero_bytes(buf + header.size() + n, total - header.size() - n, mem, s);
    const uint8_t *aad_p = reinterpret_cast<const uint8_t *>(aad.data());
    uint8_t *tag_p = reinterpret_cast<uint8_t *>(&tag_d[0]);
    if (e == cudaSuccess && mem == GCM_MEM_DEVICE) {
        e = put_bytes(buf + off_aad, aad.data(), aad.size(), mem, s);
        if (e == cudaSuccess) e = put_bytes(buf + off_tag, tag_d.data(), 16, mem, s);
        aad_p = buf + off_aad;
        tag_p = buf + off_tag;
    }
    if (e != cudaSuccess) {
        gfc_result_free(ctx, out);
        return set_result(out, GCM_ERR_CUDA, 0, cudaGetErrorString(e));
    }
    // Pixels: decrypted and verified under the data key (zero-filled by the
    // library on a tag mismatch), or suppressed without one.
    bool data_ok = false;
    uint32_t dsum = 0;
    bool dsum_done = false;
    if (key_d) {
        rc = gcmgpu::ctx_run_with_datasum(ctx, key_d, key_d_len, reinterpret_cast<const uint8_t *>(nonce_d.data()), 12,
                                          aad_p, aad.size(), cont + blob_off, (size_t)n, buf + header.size(), tag_p,
                                          true, mem, stream, &dsum, &dsum_done);
        if (rc == GCM_OK) data_ok = true;
        else if (rc != GCM_ERR_AUTH) {
            std::string m = gcm_last_error();
            gfc_result_free(ctx, out);
            return set_result(out, rc, 0, m.c_str());
        }
    } else {
        e = zero_bytes(buf + header.size(), (size_t)n, mem, s);
        if (e == cudaSuccess && mem == GCM_MEM_DEVICE) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            gfc_result_free(ctx, out);
            return set_result(out, GCM_ERR_CUDA, 0, cudaGetErrorString(e));
        }
    }
    if (mem == GCM_MEM_DEVICE) cudaStreamSynchronize(s);
    if (!data_ok) warning = 2;
    out->datasum = dsum;
    out->datasum_valid = dsum_done ? 1 : 0;
    return set_result(out, GCM_OK, warning,
                      warning == 2 ? "payload suppressed (data key missing or tag mismatch)"
                                   : warning == 1 ? "header fallback (header key missing or tag mismatch)" : "");
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
    gcmgpu::TraceRange trace_("gfc_fits_encrypt");
    return fits_call(ctx, false, key, key_len, fits, fits_len, iv12, iv_out, nullptr, tag_out, aad_mode, mem,
                     stream, out);
}

int gfc_fits_decrypt_verify(gcm_ctx *ctx, const uint8_t *key, size_t key_len, const uint8_t *fits_enc, size_t len,
                            const uint8_t *iv12, const uint8_t *tag, int aad_mode, int mem, void *stream,
                            gfc_result *out)
{
    gcmgpu::TraceRange trace_("gfc_fits_decrypt_verify");
    return fits_call(ctx, true, key, key_len, fits_enc, len, iv12, nullptr, tag, nullptr, aad_mode, mem, stream,
                     out);
}

int gfc_container_encrypt(gcm_ctx *ctx, const uint8_t *key_h, size_t key_h_len, const uint8_t *key_d,
                          size_t key_d_len, const uint8_t *fits, size_t fits_len, const uint8_t *nonce_h,
                          const uint8_t *nonce_d, int mem, void *stream, gfc_result *out)
{
    gcmgpu::TraceRange trace_("gfc_container_encrypt");
    return container_encrypt(ctx, key_h, key_h_len, key_d, key_d_len, fits, fits_len, nonce_h, nonce_d, mem, stream,
                             out);
}

int gfc_decrypt_frame(gcm_ctx *ctx, const uint8_t *container, size_t len, const uint8_t *key_h, size_t key_h_len,
                      const uint8_t *key_d, size_t key_d_len, int mem, void *stream, gfc_result *out)
{
    gcmgpu::TraceRange trace_("gfc_decrypt_frame");
    return decrypt_frame(ctx, container, len, key_h, key_h_len, key_d, key_d_len, mem, stream, out);
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
