// C ABI of the library (declared in include/b64gpu.h): alphabet handles,
// length helpers, argument checks, and the launches of the codec kernels.
// Host code only; the kernels live in b64_encode.cu and b64_decode.cu.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "b64gpu.h"
#include "b64_internal.h"

namespace b64 {
namespace {

thread_local std::string t_last_error;

struct DeviceSlot {
    std::once_flag once;
    DeviceInfo info;
};
DeviceSlot g_devices[64];

bool valid_chars(const uint8_t chars[64], char* why, size_t why_len) {
    bool seen[256] = {false};
    for (int k = 0; k < 64; ++k) {
        const uint8_t c = chars[k];
        if (c >= 0x80 || c == '=' || c == '\r' || c == '\n' || c == ' ') {
            snprintf(why, why_len, "alphabet character %d (0x%02x) is reserved or not ASCII", k, c);
            return false;
        }
        if (seen[c]) {
            snprintf(why, why_len, "alphabet character 0x%02x appears twice", c);
            return false;
        }
        seen[c] = true;
    }
    return true;
}

void fill_tables(b64_alphabet* a) {
    memset(&a->enc, 0, sizeof(a->enc));
    uint8_t* e = reinterpret_cast<uint8_t*>(a->enc.w);
    uint8_t* d = reinterpret_cast<uint8_t*>(a->dec.w);
    for (int c = 0; c < 256; ++c) d[c] = uint8_t(kBad);
    for (int k = 0; k < 64; ++k) {
        e[k] = a->chars[k];
        d[a->chars[k]] = uint8_t(k);
    }
}

b64_alphabet make_builtin(bool url) {
    b64_alphabet a;
    int k = 0;
    for (char c = 'A'; c <= 'Z'; ++c) a.chars[k++] = uint8_t(c);
    for (char c = 'a'; c <= 'z'; ++c) a.chars[k++] = uint8_t(c);
    for (char c = '0'; c <= '9'; ++c) a.chars[k++] = uint8_t(c);
    a.chars[62] = url ? '-' : '+';
    a.chars[63] = url ? '_' : '/';
    a.padded = url ? 0 : 1;
    a.canonical = 0;
    fill_tables(&a);
    return a;
}

const b64_alphabet g_standard = make_builtin(false);
const b64_alphabet g_url = make_builtin(true);

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return na && nb && x < y + nb && y < x + na;
}

// Per-thread, per-device scratch of the synchronous decode: one device word
// for the result and one pinned host word to read it back into.
struct SyncScratch {
    int64_t* d_word = nullptr;
    int64_t* h_word = nullptr;
};
thread_local SyncScratch t_scratch[64];

}  // namespace

const DeviceInfo& device_info(int device) {
    if (device < 0) cudaGetDevice(&device);
    DeviceSlot& slot = g_devices[device & 63];
    std::call_once(slot.once, [&] {
        slot.info.device = device;
        cudaDeviceGetAttribute(&slot.info.sm_count, cudaDevAttrMultiProcessorCount, device);
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
        slot.info.smem_optin = size_t(optin);
    });
    return slot.info;
}

static void vset(const char* fmt, va_list ap) {
    char buf[512];
    vsnprintf(buf, sizeof(buf), fmt, ap);
    t_last_error = buf;
}

int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vset(fmt, ap);
    va_end(ap);
    return code;
}

int64_t set_error64(int64_t code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vset(fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { t_last_error.clear(); }

}  // namespace b64

using namespace b64;

namespace b64 {

int batch_tables(const char* fn, const b64_alphabet* const* alphabets, int n_alphabets,
                 BatchTables* t) {
    if (!alphabets || n_alphabets < 1 || n_alphabets > B64_BATCH_MAX_ALPHABETS)
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: need 1..%d alphabets", fn,
                         B64_BATCH_MAX_ALPHABETS);
    for (int k = 0; k < kMaxAlphabets; ++k) {
        const b64_alphabet* a = alphabets[k < n_alphabets ? k : 0];
        if (!a) return set_error(B64_ERR_INVALID_ARGUMENT, "%s: alphabet %d is NULL", fn, k);
        t->enc[k] = a->enc;
        t->dec[k] = a->dec;
        t->padded[k] = a->padded;
        t->canonical[k] = a->canonical;
    }
    t->n_alph = n_alphabets;
    return B64_SUCCESS;
}

}  // namespace b64

extern "C" {

b64_alphabet* b64_alphabet_create_flags(const uint8_t chars[64], int flags) {
    if (!chars) {
        set_error(0, "b64_alphabet_create: chars is NULL");
        return nullptr;
    }
    if (flags & ~(B64_FLAG_PADDED | B64_FLAG_CANONICAL)) {
        set_error(0, "b64_alphabet_create_flags: unknown flag bits 0x%x", flags);
        return nullptr;
    }
    char why[160];
    if (!valid_chars(chars, why, sizeof(why))) {
        set_error(0, "b64_alphabet_create: %s", why);
        return nullptr;
    }
    b64_alphabet* a = new b64_alphabet;
    memcpy(a->chars, chars, 64);
    a->padded = (flags & B64_FLAG_PADDED) ? 1 : 0;
    a->canonical = (flags & B64_FLAG_CANONICAL) ? 1 : 0;
    fill_tables(a);
    return a;
}

b64_alphabet* b64_alphabet_create(const uint8_t chars[64], int padded) {
    return b64_alphabet_create_flags(chars, padded ? B64_FLAG_PADDED : 0);
}

int b64_alphabet_flags(const b64_alphabet* a) {
    if (!a) return set_error(B64_ERR_INVALID_ARGUMENT, "b64_alphabet_flags: NULL alphabet");
    return (a->padded ? B64_FLAG_PADDED : 0) | (a->canonical ? B64_FLAG_CANONICAL : 0);
}

const b64_alphabet* b64_alphabet_standard(void) { return &g_standard; }
const b64_alphabet* b64_alphabet_url(void) { return &g_url; }

void b64_alphabet_destroy(b64_alphabet* a) {
    if (!a || a == &g_standard || a == &g_url) return;
    delete a;
}

int b64_alphabet_chars(const b64_alphabet* a, uint8_t out[64]) {
    if (!a || !out) return set_error(B64_ERR_INVALID_ARGUMENT, "b64_alphabet_chars: NULL argument");
    memcpy(out, a->chars, 64);
    return a->padded;
}

size_t b64_encoded_length(size_t n, int padded) {
    const size_t g = n / 3, r = n % 3;
    if (r == 0) return 4 * g;
    return 4 * g + (padded ? 4 : r + 1);
}

size_t b64_decoded_max_length(size_t m) { return (m / 4 + (m % 4 ? 1 : 0)) * 3; }

int64_t b64_encode(const uint8_t* src, size_t len, uint8_t* dst, const b64_alphabet* a,
                   void* stream) {
    if (!a) return set_error64(B64_E_INVAL, "b64_encode: alphabet is NULL");
    if (len == 0) return 0;
    if (!src || !dst) return set_error64(B64_E_INVAL, "b64_encode: NULL src or dst");
    if (len > (size_t(1) << 62)) return set_error64(B64_E_INVAL, "b64_encode: len too large");
    const size_t out = b64_encoded_length(len, a->padded);
    if (overlaps(src, len, dst, out)) return set_error64(B64_E_INVAL, "b64_encode: src and dst overlap");
    const cudaError_t e =
        launch_encode(src, len, dst, a->enc, a->padded, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return set_error64(B64_E_CUDA, "b64_encode: %s", cudaGetErrorString(e));
    return int64_t(out);
}

int b64_decode_async(const uint8_t* src, size_t len, uint8_t* dst, const b64_alphabet* a,
                     int64_t* d_result, void* stream) {
    if (!a || !d_result)
        return set_error(B64_ERR_INVALID_ARGUMENT, "b64_decode_async: NULL alphabet or d_result");
    if (reinterpret_cast<uintptr_t>(d_result) & 7u)
        return set_error(B64_ERR_INVALID_ARGUMENT, "b64_decode_async: d_result not 8-byte aligned");
    if (len > 0 && (!src || !dst))
        return set_error(B64_ERR_INVALID_ARGUMENT, "b64_decode_async: NULL src or dst");
    if (len > (size_t(1) << 62))
        return set_error(B64_ERR_INVALID_ARGUMENT, "b64_decode_async: len too large");
    if (overlaps(src, len, dst, b64_decoded_max_length(len)))
        return set_error(B64_ERR_INVALID_ARGUMENT, "b64_decode_async: src and dst overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaError_t e = launch_decode(src, len, dst, a->dec, decode_flags(a), d_result, s);
    if (e != cudaSuccess)
        return set_error(B64_ERR_CUDA, "b64_decode_async: %s", cudaGetErrorString(e));
    return B64_SUCCESS;
}

int64_t b64_decode(const uint8_t* src, size_t len, uint8_t* dst, const b64_alphabet* a,
                   void* stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error64(B64_E_CUDA, "b64_decode: %s", cudaGetErrorString(e));
    SyncScratch& sc = t_scratch[dev & 63];
    if (!sc.d_word) {
        e = cudaMalloc(&sc.d_word, sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMallocHost(&sc.h_word, sizeof(int64_t));
        if (e != cudaSuccess) {
            if (sc.d_word) cudaFree(sc.d_word);
            sc.d_word = nullptr;
            return set_error64(B64_E_CUDA, "b64_decode: scratch allocation: %s",
                               cudaGetErrorString(e));
        }
    }
    const int rc = b64_decode_async(src, len, dst, a, sc.d_word, stream);
    if (rc == B64_ERR_INVALID_ARGUMENT) return B64_E_INVAL;
    if (rc != B64_SUCCESS) return B64_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(sc.h_word, sc.d_word, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error64(B64_E_CUDA, "b64_decode: %s", cudaGetErrorString(e));
    return *sc.h_word;
}

size_t b64_batch_workspace_size(int64_t n) { return n > 0 ? batch_workspace_bytes(n) : 0; }


static int batch_common(bool decode, const uint8_t* src, const int64_t* src_off, int64_t n,
                        uint8_t* dst, const int64_t* dst_off, const b64_alphabet* const* alphabets,
                        int n_alphabets, const uint8_t* alph_id, int64_t* results, int tile_units,
                        void* workspace, size_t workspace_bytes, void* stream) {
    const char* fn = decode ? "b64_decode_batch" : "b64_encode_batch";
    if (n < 0) return set_error(B64_ERR_INVALID_ARGUMENT, "%s: n < 0", fn);
    BatchTables tabs;
    const int rc = batch_tables(fn, alphabets, n_alphabets, &tabs);
    if (rc != B64_SUCCESS) return rc;
    if (n == 0) return B64_SUCCESS;
    // src and dst may be NULL when every string is empty (nothing reads them).
    if (!src_off || !dst_off || !results || !workspace)
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: NULL pointer argument", fn);
    int units = tile_units & 0xFF;
    if (units == 0) units = 8;
    if ((units != 1 && units != 2 && units != 4 && units != 8) || tile_units < 0 ||
        (tile_units & ~(0xFFFF | B64_TILE_PAIRS)))
        return set_error(B64_ERR_INVALID_ARGUMENT,
                         "%s: tile_units must be 0, 1, 2, 4 or 8, optionally OR-ed with "
                         "(blocks per SM << 8) and B64_TILE_PAIRS", fn);
    tile_units = units | (tile_units & (0xFF00 | B64_TILE_PAIRS));
    if (workspace_bytes < batch_workspace_bytes(n))
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: workspace holds %zu bytes, %zu needed", fn,
                         workspace_bytes, batch_workspace_bytes(n));
    if (reinterpret_cast<uintptr_t>(workspace) & 255)
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: workspace not 256-byte aligned", fn);
    BatchArgs a{src, src_off, n, dst, dst_off, alph_id, results};
    const cudaError_t e =
        launch_batch(decode, a, tabs, tile_units, workspace, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_error(B64_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return B64_SUCCESS;
}

int b64_encode_batch(const uint8_t* src, const int64_t* src_off, int64_t n, uint8_t* dst,
                     const int64_t* dst_off, const b64_alphabet* const* alphabets,
                     int n_alphabets, const uint8_t* alph_id, int64_t* results, int tile_units,
                     void* workspace, size_t workspace_bytes, void* stream) {
    return batch_common(false, src, src_off, n, dst, dst_off, alphabets, n_alphabets, alph_id,
                        results, tile_units, workspace, workspace_bytes, stream);
}

int b64_decode_batch(const uint8_t* src, const int64_t* src_off, int64_t n, uint8_t* dst,
                     const int64_t* dst_off, const b64_alphabet* const* alphabets,
                     int n_alphabets, const uint8_t* alph_id, int64_t* results, int tile_units,
                     void* workspace, size_t workspace_bytes, void* stream) {
    return batch_common(true, src, src_off, n, dst, dst_off, alphabets, n_alphabets, alph_id,
                        results, tile_units, workspace, workspace_bytes, stream);
}

int b64_batch_offsets(const int64_t* src_off, int64_t n, const b64_alphabet* const* alphabets,
                      int n_alphabets, const uint8_t* alph_id, int flags, int64_t* dst_off,
                      void* stream) {
    if (n < 0 || !src_off || !dst_off)
        return set_error(B64_ERR_INVALID_ARGUMENT, "b64_batch_offsets: bad argument");
    if (flags & ~(B64_OFFSETS_DECODE | B64_OFFSETS_ALIGN16))
        return set_error(B64_ERR_INVALID_ARGUMENT, "b64_batch_offsets: unknown flags %d", flags);
    BatchTables tabs;
    const int rc = batch_tables("b64_batch_offsets", alphabets, n_alphabets, &tabs);
    if (rc != B64_SUCCESS) return rc;
    const cudaError_t e =
        launch_batch_offsets((flags & B64_OFFSETS_DECODE) != 0, (flags & B64_OFFSETS_ALIGN16) != 0,
                             src_off, n, tabs, alph_id, dst_off, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return set_error(B64_ERR_CUDA, "b64_batch_offsets: %s", cudaGetErrorString(e));
    return B64_SUCCESS;
}

size_t b64_mime_workspace_size(size_t len) { return mime_workspace_bytes(len); }

static int mime_common(const char* fn, const uint8_t* src, size_t len, uint8_t* dst,
                       const b64_alphabet* a, int64_t* d_result, void* workspace,
                       size_t workspace_bytes, uint64_t limit_ns, void* stream) {
    if (!a || !d_result || !workspace)
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: NULL alphabet, d_result or workspace", fn);
    if ((reinterpret_cast<uintptr_t>(d_result) | reinterpret_cast<uintptr_t>(workspace)) & 7u)
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: d_result/workspace not 8-byte aligned", fn);
    if (len > 0 && (!src || !dst))
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: NULL src or dst", fn);
    if (len > (size_t(1) << 62)) return set_error(B64_ERR_INVALID_ARGUMENT, "%s: len too large", fn);
    if (workspace_bytes < mime_workspace_bytes(len))
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: workspace holds %zu bytes, %zu needed", fn,
                         workspace_bytes, mime_workspace_bytes(len));
    if (overlaps(src, len, dst, b64_decoded_max_length(len)))
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: src and dst overlap", fn);
    const cudaError_t e = launch_mime_decode(src, len, dst, a->dec, decode_flags(a), d_result,
                                             workspace, limit_ns, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_error(B64_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return B64_SUCCESS;
}

int b64_mime_decode_async(const uint8_t* src, size_t len, uint8_t* dst, const b64_alphabet* a,
                          int64_t* d_result, void* workspace, size_t workspace_bytes,
                          void* stream) {
    return mime_common("b64_mime_decode_async", src, len, dst, a, d_result, workspace,
                       workspace_bytes, kWaitLimitNs, stream);
}

size_t b64_mime_batch_workspace_size(int64_t n, uint64_t total_bytes) {
    return n > 0 ? mime_batch_workspace_bytes(n, total_bytes) : 0;
}

int b64_mime_decode_batch(const uint8_t* src, const int64_t* src_off, int64_t n, uint8_t* dst,
                          const int64_t* dst_off, const b64_alphabet* const* alphabets,
                          int n_alphabets, const uint8_t* alph_id, int64_t* results,
                          void* workspace, size_t workspace_bytes, void* stream) {
    const char* fn = "b64_mime_decode_batch";
    if (n < 0) return set_error(B64_ERR_INVALID_ARGUMENT, "%s: n < 0", fn);
    BatchTables tabs;
    const int rc = batch_tables(fn, alphabets, n_alphabets, &tabs);
    if (rc != B64_SUCCESS) return rc;
    if (n == 0) return B64_SUCCESS;
    if (!src_off || !dst_off || !results || !workspace)
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: NULL pointer argument", fn);
    if (reinterpret_cast<uintptr_t>(workspace) & 7u)
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: workspace not 8-byte aligned", fn);
    if (workspace_bytes < mime_batch_workspace_bytes(n, 0))
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: workspace holds %zu bytes, at least %zu needed",
                         fn, workspace_bytes, mime_batch_workspace_bytes(n, 0));
    BatchArgs a{src, src_off, n, dst, dst_off, alph_id, results};
    const cudaError_t e = launch_mime_decode_batch(a, tabs, workspace, workspace_bytes,
                                                   static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_error(B64_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return B64_SUCCESS;
}

int b64_selftest_wait_timeout(int64_t* d_result, uint64_t wait_limit_ns, void* stream) {
    if (!d_result || (reinterpret_cast<uintptr_t>(d_result) & 7u))
        return set_error(B64_ERR_INVALID_ARGUMENT,
                         "b64_selftest_wait_timeout: d_result NULL or not 8-byte aligned");
    if (wait_limit_ns == 0 || wait_limit_ns > kWaitLimitNs)
        return set_error(B64_ERR_INVALID_ARGUMENT,
                         "b64_selftest_wait_timeout: wait_limit_ns must be 1..%llu",
                         (unsigned long long)kWaitLimitNs);
    const cudaError_t e = launch_selftest_wait(d_result, wait_limit_ns, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return set_error(B64_ERR_CUDA, "b64_selftest_wait_timeout: %s", cudaGetErrorString(e));
    return B64_SUCCESS;
}

const char* b64_last_error(void) { return t_last_error.c_str(); }

int b64_device_fault_flag(int clear) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_error(B64_ERR_CUDA, "b64_device_fault_flag: %s", cudaGetErrorString(e));
    uint32_t f = encode_fault_flag(clear != 0) | decode_fault_flag(clear != 0) |
                 mime_fault_flag(clear != 0) | batch_fault_flag(clear != 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(B64_ERR_CUDA, "b64_device_fault_flag: %s", cudaGetErrorString(e));
    return int(f);
}

int b64_version(void) { return 100; }

}  // extern "C"
