/*
 * Plain scalar base64 codec: the ORACLE for parity tests.
 *
 * This file is test infrastructure. Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline leg may load it. The GPU library shares no code,
 * header, table or constant with it: the two are written independently and
 * only compared.
 *
 * It is the textbook definition written out, one character at a time, in the
 * order the paper states it (Mula & Lemire, "Base64 encoding and decoding at
 * almost the speed of a memory copy", arXiv:1910.05109):
 *   - Sec. 2, Table 1: the 64-character alphabet, a bijection between 6-bit
 *     values and ASCII characters. Any other 64-character table (base64url,
 *     Sec. 2) is passed in the same way.
 *   - Sec. 2: three bytes s1,s2,s3 map to the four 6-bit values
 *       s1 div 4, (s2 div 16) + (s1*16) mod 64,
 *       (s2*4) mod 64 + (s3 div 64), s3 mod 64.
 *   - Sec. 2: '=' padding makes the encoded length a multiple of four.
 *   - Sec. 2: four 6-bit values a,b,c,d give back the three bytes
 *       a*4 + b div 16, (b*16) mod 256 + c div 4, (c*64) mod 256 + d,
 *     and characters outside the table map to a special value (an error).
 *
 * Where the paper is silent the following readings are used (they are the
 * library's documented contract as well):
 *   R1  Any byte that is neither in the alphabet nor a permitted '=' is an
 *       error at its own index. Bytes >= 0x80 are never alphabet characters
 *       (Sec. 3.2, Fig. 2: the input's top bit is part of the error test).
 *   R2  Padded mode: '=' is permitted only as the last character, or as the
 *       second-to-last when the last is also '='. The length must be a
 *       multiple of 4, else the error is at offset m (the input length).
 *       Unpadded mode: every '=' is an error; a length of 1 mod 4 is an error
 *       at offset m.
 *   R3  Trailing bits of the last data character that do not reach an output
 *       byte are ignored (non-canonical encodings are accepted).
 *   R4  The reported error is the smallest offset among all errors.
 *   R5  MIME mode (not in the paper): CR, LF and SP are removed first; R1-R4
 *       apply to what is left; error offsets are given in the original
 *       (uncompacted) coordinates and a length error is at offset m.
 *   R6  A partial final group of k data characters (k = 2 or 3) is completed
 *       with zero 6-bit values and yields k-1 bytes; a partial final group of
 *       encoder input (1 or 2 bytes) is completed with zero bytes (RFC 4648
 *       Sec. 4, the standard the paper cites for base64url).
 *   R7  Canonical mode (optional, flag bit 1; RFC 4648 Sec. 3.5 lets a decoder
 *       reject what an encoder never emits): R3 is replaced by this rule. When
 *       the final group is partial (k = 2 or 3 data characters once the
 *       padding is removed), the bits of its last data character that reach
 *       no output byte (the low 4 bits for k = 2, the low 2 bits for k = 3)
 *       must be zero; otherwise that character is an error at its own index.
 *       It competes with the length error of R2 under R4.
 *
 * The decoders' `padded` argument carries flags: bit 0 = padded (R2),
 * bit 1 = canonical (R7).
 *
 * Return values: encode returns the number of characters written; decode
 * returns the number of bytes written (>= 0) or -(offset+1) for the first
 * error. Nothing is written past the returned length on success.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_NOT_IN_TABLE (-1)

/* Table 1 (Sec. 2): value k <-> character, read row by row. */
static const char oracle_table1[64] = {
    'A', 'B', 'C', 'D', 'E', 'F', 'G', 'H', 'I', 'J', 'K', 'L', 'M', 'N', 'O', 'P',
    'Q', 'R', 'S', 'T', 'U', 'V', 'W', 'X', 'Y', 'Z', 'a', 'b', 'c', 'd', 'e', 'f',
    'g', 'h', 'i', 'j', 'k', 'l', 'm', 'n', 'o', 'p', 'q', 'r', 's', 't', 'u', 'v',
    'w', 'x', 'y', 'z', '0', '1', '2', '3', '4', '5', '6', '7', '8', '9', '+', '/'};

/* Copies Table 1 into out[64]. */
void oracle_standard_alphabet(uint8_t out[64]) {
    for (int k = 0; k < 64; ++k) out[k] = (uint8_t)oracle_table1[k];
}

/* base64url (Sec. 2, RFC 4648): Table 1 with '+' -> '-' and '/' -> '_'. */
void oracle_url_alphabet(uint8_t out[64]) {
    oracle_standard_alphabet(out);
    out[62] = (uint8_t)'-';
    out[63] = (uint8_t)'_';
}

/* The inverse of the alphabet (Table 1 is invertible, Sec. 2): for every byte
 * value, its 6-bit value, or ORACLE_NOT_IN_TABLE. */
static void oracle_inverse(const uint8_t alph[64], int inv[256]) {
    for (int c = 0; c < 256; ++c) inv[c] = ORACLE_NOT_IN_TABLE;
    for (int k = 0; k < 64; ++k) inv[alph[k]] = k;
}

/* 6-bit value of byte c under alph, or -1 (the "special value", Sec. 2). */
int oracle_value_of(const uint8_t alph[64], uint8_t c) {
    for (int k = 0; k < 64; ++k)
        if (alph[k] == c) return k;
    return ORACLE_NOT_IN_TABLE;
}

/* Encoded length: four characters per three bytes; with padding the last
 * partial group also takes four characters (Sec. 2), without it a group of
 * r bytes takes r+1 characters. */
size_t oracle_encoded_length(size_t n, int padded) {
    size_t groups = n / 3, r = n % 3;
    if (r == 0) return 4 * groups;
    return 4 * groups + (padded ? 4 : r + 1);
}

int64_t oracle_encode(const uint8_t* src, size_t n, uint8_t* dst,
                      const uint8_t alph[64], int padded) {
    size_t o = 0, i = 0;
    for (; i + 3 <= n; i += 3) {
        unsigned s1 = src[i], s2 = src[i + 1], s3 = src[i + 2];
        dst[o++] = alph[s1 / 4];
        dst[o++] = alph[(s2 / 16) + (s1 * 16) % 64];
        dst[o++] = alph[(s2 * 4) % 64 + (s3 / 64)];
        dst[o++] = alph[s3 % 64];
    }
    size_t r = n - i;
    if (r == 1) { /* s2 = s3 = 0 (R6): two characters, then "==" */
        unsigned s1 = src[i];
        dst[o++] = alph[s1 / 4];
        dst[o++] = alph[(s1 * 16) % 64];
        if (padded) { dst[o++] = '='; dst[o++] = '='; }
    } else if (r == 2) { /* s3 = 0 (R6): three characters, then "=" */
        unsigned s1 = src[i], s2 = src[i + 1];
        dst[o++] = alph[s1 / 4];
        dst[o++] = alph[(s2 / 16) + (s1 * 16) % 64];
        dst[o++] = alph[(s2 * 4) % 64];
        if (padded) dst[o++] = '=';
    }
    return (int64_t)o;
}

static int oracle_is_mime_space(uint8_t c) {
    return c == '\r' || c == '\n' || c == ' ';
}

int64_t oracle_decode(const uint8_t* src, size_t m, uint8_t* dst,
                      const uint8_t alph[64], int flags, int mime) {
    const int padded = flags & 1, canonical = (flags >> 1) & 1;
    int inv[256];
    oracle_inverse(alph, inv);

    /* R5: the positions of the characters that take part in decoding (in
     * MIME mode a list; otherwise every position, POS(j) = j). */
    size_t* pos = NULL;
    size_t mc = m;
    if (mime) {
        pos = (size_t*)malloc((m ? m : 1) * sizeof(size_t));
        if (!pos) return INT64_MIN;
        mc = 0;
        for (size_t i = 0; i < m; ++i) {
            if (oracle_is_mime_space(src[i])) continue;
            pos[mc++] = i;
        }
    }
#define POS(j) (pos ? pos[(j)] : (j))

    /* R1, R2, R4: scan in order; the first bad character is the smallest
     * offset, and the length error (offset m) is larger than any index. */
    int has_err = 0;
    size_t err = 0;
    for (size_t j = 0; j < mc; ++j) {
        uint8_t ch = src[POS(j)];
        if (inv[ch] != ORACLE_NOT_IN_TABLE) continue;
        int pad_ok = 0;
        if (ch == '=' && padded) {
            if (j == mc - 1) pad_ok = 1;
            if (j + 2 == mc && src[POS(mc - 1)] == '=') pad_ok = 1;
        }
        if (!pad_ok) { has_err = 1; err = POS(j); break; }
    }
    size_t pads = 0;
    if (padded) {
        if (mc >= 1 && src[POS(mc - 1)] == '=') pads = 1;
        if (mc >= 2 && src[POS(mc - 2)] == '=') pads = 2;
    }
    size_t d = mc - pads;
    if (!has_err) {
        if (padded && mc % 4 != 0) { has_err = 1; err = m; }
        if (!padded && mc % 4 == 1) { has_err = 1; err = m; }
        /* R7: the unused low bits of a partial final group's last character */
        if (canonical && (d % 4 == 2 || d % 4 == 3)) {
            unsigned low = d % 4 == 2 ? 15u : 3u;
            size_t at = POS(d - 1);
            if (((unsigned)inv[src[at]] & low) != 0 && (!has_err || at < err)) {
                has_err = 1;
                err = at;
            }
        }
    }
    if (has_err) {
        free(pos);
        return -(int64_t)err - 1;
    }

    /* Sec. 2: four 6-bit values a,b,c,d -> three bytes; a short final group
     * is completed with zero values and emits one byte fewer than it has
     * characters (R6). */
    size_t o = 0;
    for (size_t j = 0; j < d; j += 4) {
        unsigned v[4] = {0, 0, 0, 0};
        size_t k = d - j < 4 ? d - j : 4;
        for (size_t t = 0; t < k; ++t) v[t] = (unsigned)inv[src[POS(j + t)]];
        unsigned a = v[0], b = v[1], c = v[2], dd = v[3];
        unsigned bytes[3];
        bytes[0] = (a * 4) + (b / 16);
        bytes[1] = (b * 16) % 256 + (c / 4);
        bytes[2] = (c * 64) % 256 + dd;
        for (size_t t = 0; t + 1 < k; ++t) dst[o++] = (uint8_t)bytes[t];
    }
    free(pos);
    return (int64_t)o;
#undef POS
}

/* Batched forms: string i occupies src[src_off[i] .. src_off[i+1]) and is
 * written at dst + dst_off[i]; alph_id[i] selects one of the alphabets
 * (64 bytes each, contiguous in alphs) and padded[i] its flags (bit 0
 * padded, bit 1 canonical; encode reads bit 0 only).
 * results[i] gets what the single-string call returns. */
void oracle_encode_batch(const uint8_t* src, const int64_t* src_off, uint8_t* dst,
                         const int64_t* dst_off, const uint8_t* alphs,
                         const int32_t* alph_id, const int32_t* padded, int64_t n,
                         int64_t* results) {
    for (int64_t i = 0; i < n; ++i) {
        results[i] = oracle_encode(src + src_off[i], (size_t)(src_off[i + 1] - src_off[i]),
                                   dst + dst_off[i], alphs + 64 * alph_id[i], padded[i] & 1);
    }
}

void oracle_decode_batch(const uint8_t* src, const int64_t* src_off, uint8_t* dst,
                         const int64_t* dst_off, const uint8_t* alphs,
                         const int32_t* alph_id, const int32_t* padded, int32_t mime,
                         int64_t n, int64_t* results) {
    for (int64_t i = 0; i < n; ++i) {
        results[i] = oracle_decode(src + src_off[i], (size_t)(src_off[i + 1] - src_off[i]),
                                   dst + dst_off[i], alphs + 64 * alph_id[i], padded[i], mime);
    }
}
