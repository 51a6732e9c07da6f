// Host-buffer codec: encode or strictly decode a buffer in host memory with
// the device kernels, the host-to-device copy, the kernel and the
// device-to-host copy of consecutive pieces overlapped on several streams
// (the copy engines of the two directions and the SMs then work at once).
// Not in the paper, which codes buffers that are already in the processor's
// memory; this is how such a buffer reaches the GPU and comes back.
//
// Encode pieces are P input bytes (P a multiple of 12), so every piece but
// the last is whole 3-byte groups and its output starts at 4/3 of its input
// offset. Decode pieces are P characters, except that the last piece always
// holds the last two characters of the input (it is P + 1 characters when
// that needs it): '=' may only stand at the last two positions of the whole
// input (Sec. 2), so the inner pieces are decoded with the padding rule off
// (every '=' is an error there, as it is at that position in the whole
// input) and the final piece with the alphabet's own rule. Offsets inside a
// piece are shifted by the piece's start; pieces are checked in order, so
// the first piece with an error holds the smallest offset.
#include <cstring>
#include <mutex>
#include <vector>

#include "b64gpu.h"
#include "b64_internal.h"

namespace b64 {
namespace {
constexpr int kMaxHostStreams = 8;
constexpr size_t kDefaultPiece = size_t(48) << 20;
}  // namespace
}  // namespace b64

struct b64_host_codec {
    int device = 0;
    int n_streams = 0;
    size_t piece = 0;                  // P: input bytes per piece
    cudaStream_t st[b64::kMaxHostStreams] = {};
    cudaEvent_t ready = nullptr;       // results memset done (stream 0)
    uint8_t* d_in[b64::kMaxHostStreams] = {};
    uint8_t* d_out[b64::kMaxHostStreams] = {};
    int64_t* d_res = nullptr;          // one result word per decode piece
    int64_t* h_res = nullptr;          // pinned copy of d_res
    size_t res_cap = 0;
    std::mutex mu;                     // one call at a time
};

namespace b64 {
namespace {

size_t in_bytes(size_t P) { return P + 16; }            // decode's last piece: P + 1
size_t out_bytes(size_t P) { return P / 3 * 4 + 16; }    // encode output of P bytes

void release(b64_host_codec* c) {
    for (int s = 0; s < kMaxHostStreams; ++s) {
        if (c->st[s]) cudaStreamDestroy(c->st[s]);
        if (c->d_in[s]) cudaFree(c->d_in[s]);
        if (c->d_out[s]) cudaFree(c->d_out[s]);
    }
    if (c->ready) cudaEventDestroy(c->ready);
    if (c->d_res) cudaFree(c->d_res);
    if (c->h_res) cudaFreeHost(c->h_res);
}

// Makes the codec's device current for the scope.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

cudaError_t grow_results(b64_host_codec* c, size_t pieces) {
    if (pieces <= c->res_cap) return cudaSuccess;
    size_t cap = c->res_cap ? c->res_cap : 64;
    while (cap < pieces) cap *= 2;
    int64_t *d = nullptr, *h = nullptr;
    cudaError_t e = cudaMalloc(&d, cap * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMallocHost(&h, cap * sizeof(int64_t));
    if (e != cudaSuccess) {
        if (d) cudaFree(d);
        return e;
    }
    if (c->d_res) cudaFree(c->d_res);
    if (c->h_res) cudaFreeHost(c->h_res);
    c->d_res = d;
    c->h_res = h;
    c->res_cap = cap;
    return cudaSuccess;
}

cudaError_t drain(b64_host_codec* c) {
    cudaError_t first = cudaSuccess;
    for (int s = 0; s < c->n_streams; ++s) {
        const cudaError_t e = cudaStreamSynchronize(c->st[s]);
        if (first == cudaSuccess) first = e;
    }
    return first;
}

}  // namespace
}  // namespace b64

using namespace b64;

extern "C" {

b64_host_codec* b64_host_codec_create(size_t piece_bytes, int n_streams) {
    if (n_streams == 0) n_streams = 3;
    if (n_streams < 1 || n_streams > kMaxHostStreams) {
        set_error(0, "b64_host_codec_create: n_streams must be 0..%d", kMaxHostStreams);
        return nullptr;
    }
    size_t P = piece_bytes ? piece_bytes / 12 * 12 : kDefaultPiece;
    if (P < 12) P = 12;
    if (P > (size_t(1) << 40)) {
        set_error(0, "b64_host_codec_create: piece_bytes too large");
        return nullptr;
    }
    b64_host_codec* c = new b64_host_codec;
    c->n_streams = n_streams;
    c->piece = P;
    cudaError_t e = cudaGetDevice(&c->device);
    for (int s = 0; s < n_streams && e == cudaSuccess; ++s) {
        e = cudaStreamCreateWithFlags(&c->st[s], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&c->d_in[s], in_bytes(P));
        if (e == cudaSuccess) e = cudaMalloc(&c->d_out[s], out_bytes(P));
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = grow_results(c, 64);
    if (e != cudaSuccess) {
        set_error(0, "b64_host_codec_create: %s", cudaGetErrorString(e));
        release(c);
        delete c;
        return nullptr;
    }
    return c;
}

size_t b64_host_codec_device_bytes(const b64_host_codec* c) {
    return c ? size_t(c->n_streams) * (in_bytes(c->piece) + out_bytes(c->piece)) +
                   c->res_cap * sizeof(int64_t)
             : 0;
}

void b64_host_codec_destroy(b64_host_codec* c) {
    if (!c) return;
    {
        DeviceGuard g(c->device);
        drain(c);
        release(c);
    }
    delete c;
}

int64_t b64_host_encode(b64_host_codec* c, const uint8_t* src, size_t len, uint8_t* dst,
                        const b64_alphabet* a) {
    const char* fn = "b64_host_encode";
    if (!c || !a) return set_error64(B64_E_INVAL, "%s: NULL codec or alphabet", fn);
    if (len == 0) return 0;
    if (!src || !dst) return set_error64(B64_E_INVAL, "%s: NULL src or dst", fn);
    if (len > (size_t(1) << 62)) return set_error64(B64_E_INVAL, "%s: len too large", fn);
    std::lock_guard<std::mutex> lock(c->mu);
    DeviceGuard g(c->device);
    if (g.err != cudaSuccess) return set_error64(B64_E_CUDA, "%s: %s", fn, cudaGetErrorString(g.err));
    const size_t P = c->piece;
    const size_t pieces = (len + P - 1) / P;
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < pieces && e == cudaSuccess; ++i) {
        const int s = int(i % size_t(c->n_streams));
        const size_t off = i * P, n = len - off < P ? len - off : P;
        const size_t out = b64_encoded_length(n, a->padded);
        e = cudaMemcpyAsync(c->d_in[s], src + off, n, cudaMemcpyHostToDevice, c->st[s]);
        if (e == cudaSuccess) e = launch_encode(c->d_in[s], n, c->d_out[s], a->enc, a->padded, c->st[s]);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dst + off / 3 * 4, c->d_out[s], out, cudaMemcpyDeviceToHost, c->st[s]);
    }
    const cudaError_t d = drain(c);
    if (e == cudaSuccess) e = d;
    if (e != cudaSuccess) return set_error64(B64_E_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return int64_t(b64_encoded_length(len, a->padded));
}

int64_t b64_host_decode(b64_host_codec* c, const uint8_t* src, size_t len, uint8_t* dst,
                        const b64_alphabet* a) {
    const char* fn = "b64_host_decode";
    if (!c || !a) return set_error64(B64_E_INVAL, "%s: NULL codec or alphabet", fn);
    if (len == 0) return 0;
    if (!src || !dst) return set_error64(B64_E_INVAL, "%s: NULL src or dst", fn);
    if (len > (size_t(1) << 62)) return set_error64(B64_E_INVAL, "%s: len too large", fn);
    std::lock_guard<std::mutex> lock(c->mu);
    DeviceGuard g(c->device);
    if (g.err != cudaSuccess) return set_error64(B64_E_CUDA, "%s: %s", fn, cudaGetErrorString(g.err));
    const size_t P = c->piece;
    // Inner pieces cover [0, B), B the largest multiple of P with B <= len - 2.
    const size_t inner = len >= 2 ? (len - 2) / P : 0;
    const size_t pieces = inner + 1;
    cudaError_t e = grow_results(c, pieces);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->d_res, 0xFF, pieces * sizeof(int64_t), c->st[0]);
    if (e == cudaSuccess) e = cudaEventRecord(c->ready, c->st[0]);
    for (int s = 1; s < c->n_streams && e == cudaSuccess; ++s)
        e = cudaStreamWaitEvent(c->st[s], c->ready, 0);
    b64_alphabet inner_a;
    memcpy(&inner_a, a, sizeof(inner_a));
    inner_a.padded = 0;     // every '=' in an inner piece is an error
    inner_a.canonical = 0;  // inner pieces hold whole groups only
    for (size_t i = 0; i < pieces && e == cudaSuccess; ++i) {
        const int s = int(i % size_t(c->n_streams));
        const size_t off = i * P, n = i < inner ? P : len - off;
        const b64_alphabet& pa = i < inner ? inner_a : *a;
        e = cudaMemcpyAsync(c->d_in[s], src + off, n, cudaMemcpyHostToDevice, c->st[s]);
        if (e == cudaSuccess)
            e = launch_decode(c->d_in[s], n, c->d_out[s], pa.dec, decode_flags(&pa), c->d_res + i,
                              c->st[s]);
        // The piece's output is copied whole (its bytes past an error are
        // unspecified, as for the single-buffer decode).
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dst + off / 4 * 3, c->d_out[s], i < inner ? P / 4 * 3 : b64_decoded_max_length(n),
                                cudaMemcpyDeviceToHost, c->st[s]);
    }
    const cudaError_t d = drain(c);
    if (e == cudaSuccess) e = d;
    if (e == cudaSuccess)
        e = cudaMemcpy(c->h_res, c->d_res, pieces * sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_error64(B64_E_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    int64_t total = 0;
    for (size_t i = 0; i < pieces; ++i) {
        const int64_t r = c->h_res[i];
        if (r >= 0) {
            total += r;
            continue;
        }
        if (r == B64_E_TIMEOUT || r == B64_E_CUDA || r == B64_E_INVAL) return r;
        return r - int64_t(i * P);  // -(offset+1) shifted by the piece's start
    }
    return total;
}

}  // extern "C"
