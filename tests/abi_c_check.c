/* A plain C99 caller of the library's C ABI, built and run by
 * tests/test_abi_c.py without a GPU: it includes include/b64gpu.h as C,
 * links libb64gpu.so and exercises the entry points that need no device
 * (alphabet handles, length helpers, argument checks). Prints the failed
 * check and exits non-zero on the first failure. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "b64gpu.h"

#define CHECK(cond)                                                          \
    do {                                                                     \
        if (!(cond)) {                                                       \
            fprintf(stderr, "%s:%d: check failed: %s (last error: %s)\n",    \
                    __FILE__, __LINE__, #cond, b64_last_error());            \
            return 1;                                                        \
        }                                                                    \
    } while (0)

static const char kTable1[] =
    "ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789+/";

int main(void) {
    uint8_t chars[64];
    size_t n;
    int64_t r;

    /* Table 1 and its base64url variant (Sec. 2) */
    CHECK(b64_alphabet_chars(b64_alphabet_standard(), chars) == 1);
    CHECK(memcmp(chars, kTable1, 64) == 0);
    CHECK(b64_alphabet_chars(b64_alphabet_url(), chars) == 0);
    CHECK(memcmp(chars, kTable1, 62) == 0 && chars[62] == '-' && chars[63] == '_');

    /* a custom table; invalid ones are refused with a message */
    {
        uint8_t custom[64];
        b64_alphabet* a;
        memcpy(custom, kTable1, 64);
        custom[62] = '.';
        custom[63] = '_';
        a = b64_alphabet_create_flags(custom, B64_FLAG_PADDED | B64_FLAG_CANONICAL);
        CHECK(a != NULL);
        CHECK(b64_alphabet_flags(a) == (B64_FLAG_PADDED | B64_FLAG_CANONICAL));
        CHECK(b64_alphabet_chars(a, chars) == 1 && memcmp(chars, custom, 64) == 0);
        b64_alphabet_destroy(a);
        custom[5] = custom[6];
        CHECK(b64_alphabet_create(custom, 1) == NULL);
        CHECK(strstr(b64_last_error(), "twice") != NULL);
        custom[5] = '=';
        CHECK(b64_alphabet_create(custom, 1) == NULL);
        custom[5] = 0xC3;
        CHECK(b64_alphabet_create(custom, 1) == NULL);
        CHECK(b64_alphabet_create_flags((const uint8_t*)kTable1, 4) == NULL); /* unknown flag */
        b64_alphabet_destroy(NULL);
        b64_alphabet_destroy((b64_alphabet*)b64_alphabet_standard()); /* ignored */
    }

    /* lengths (Sec. 2) */
    for (n = 0; n < 1000; ++n) {
        CHECK(b64_encoded_length(n, 1) == (n + 2) / 3 * 4);
        CHECK(b64_encoded_length(n, 0) == (4 * n + 2) / 3);
        CHECK(b64_decoded_max_length(n) == (n + 3) / 4 * 3);
    }

    /* argument errors are reported before any device work */
    r = b64_encode(NULL, 16, NULL, NULL, NULL);
    CHECK(r == B64_E_INVAL);
    CHECK(b64_encode(NULL, 0, NULL, b64_alphabet_standard(), NULL) == 0);
    CHECK(b64_decode_async(NULL, 4, NULL, b64_alphabet_standard(), NULL, NULL) ==
          B64_ERR_INVALID_ARGUMENT);
    CHECK(b64_decode_async((const uint8_t*)16, 4, (uint8_t*)64, b64_alphabet_standard(),
                           (int64_t*)12, NULL) == B64_ERR_INVALID_ARGUMENT);
    CHECK(strstr(b64_last_error(), "aligned") != NULL);
    CHECK(b64_decode_async((const uint8_t*)64, 64, (uint8_t*)80, b64_alphabet_standard(),
                           (int64_t*)256, NULL) == B64_ERR_INVALID_ARGUMENT);
    CHECK(strstr(b64_last_error(), "overlap") != NULL);
    CHECK(b64_batch_workspace_size(0) == 0 && b64_batch_workspace_size(10) >= 80);
    CHECK(b64_encode_batch(NULL, NULL, -1, NULL, NULL, NULL, 0, NULL, NULL, 0, NULL, 0, NULL) ==
          B64_ERR_INVALID_ARGUMENT);
    CHECK(b64_mime_workspace_size(1 << 20) > 0);
    CHECK(b64_selftest_wait_timeout(NULL, 1000, NULL) == B64_ERR_INVALID_ARGUMENT);
    CHECK(b64_server_create(1000, 1, 0, NULL, 0) == NULL);
    CHECK(b64_host_codec_create(0, 99) == NULL);
    CHECK(b64_version() >= 100);
    puts("C ABI checks passed");
    return 0;
}
