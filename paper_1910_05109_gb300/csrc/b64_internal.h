// Host-side declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "b64_device.cuh"
#include "b64gpu.h"

// The alphabet handle behind the C ABI's opaque pointer.
struct b64_alphabet {
    uint8_t chars[64];
    int padded;     // '=' emitted by encode, required by decode
    int canonical;  // decode rejects non-zero unused bits in a partial final group
    b64::EncodeTable enc;
    b64::DecodeTable dec;
};

// The decode kernels' mode word: bit 0 padded, bit 1 canonical.
inline int decode_flags(const b64_alphabet* a) { return (a->padded ? 1 : 0) | (a->canonical ? 2 : 0); }

namespace b64 {

struct DeviceInfo {
    int device = -1;
    int sm_count = 0;
    size_t smem_optin = 0;
};

// Cached per device; the current device if `device` < 0.
const DeviceInfo& device_info(int device = -1);

// Records a message for b64_last_error() and returns `code`.
int set_error(int code, const char* fmt, ...);
int64_t set_error64(int64_t code, const char* fmt, ...);
void clear_error();

// ---- encode (b64_encode.cu)
// Enqueues the encode of n bytes (n > 0). Returns cudaSuccess or the launch error.
cudaError_t launch_encode(const uint8_t* src, uint64_t n, uint8_t* dst, const EncodeTable& tab,
                          int padded, cudaStream_t stream);
uint32_t encode_fault_flag(bool clear);

// ---- decode (b64_decode.cu)
// Enqueues the strict decode of m characters; *d_result receives the length
// or -(offset+1). Up to 512 KiB of input takes one launch (one block, or one
// cluster of up to 16 blocks); larger inputs take a kernel that initialises
// *d_result, then the body kernel and the tail kernel.
cudaError_t launch_decode(const uint8_t* src, uint64_t m, uint8_t* dst, const DecodeTable& tab,
                          int flags, int64_t* d_result, cudaStream_t stream);
uint32_t decode_fault_flag(bool clear);

// ---- batches (b64_batch.cu)
constexpr int kMaxAlphabets = 4;

// The alphabets of one batched call, passed by value in the kernel
// parameters. Slots past the caller's count repeat alphabet 0, and alphabet
// ids are taken modulo kMaxAlphabets, so no id reads outside the table.
struct BatchTables {
    EncodeTable enc[kMaxAlphabets];
    DecodeTable dec[kMaxAlphabets];
    int padded[kMaxAlphabets];
    int canonical[kMaxAlphabets];
    int n_alph;  // distinct alphabets the caller gave (slots past them repeat alphabet 0)
};

struct BatchArgs {
    const uint8_t* src;
    const int64_t* src_off;  // n+1 device offsets
    int64_t n;
    uint8_t* dst;
    const int64_t* dst_off;  // n+1 device offsets (only the first n are read)
    const uint8_t* alph_id;  // n device ids, or NULL (all alphabet 0)
    int64_t* results;        // n device results
};

size_t batch_workspace_bytes(int64_t n);
uint32_t batch_fault_flag(bool clear);
// Fills the by-value tables of a batched call from 1..kMaxAlphabets handles
// (later slots repeat alphabet 0). Returns B64_SUCCESS or sets the error.
int batch_tables(const char* fn, const b64_alphabet* const* alphabets, int n_alphabets,
                 BatchTables* t);
// Enqueues prep + tile kernel (+ decode finalize). `tile`: units a lane
// (1, 2, 4 or 8) in bits 0..7; resident blocks an SM in bits 8..15 (0: as
// many as fit).
cudaError_t launch_batch(bool decode, const BatchArgs& a, const BatchTables& tabs, int tile,
                         void* workspace, cudaStream_t stream);
// dst_off[0..n] = exclusive scan of per-string output capacities (encoded
// length, or 3*ceil(m/4) for decode; each rounded up to 16 bytes with align16).
cudaError_t launch_batch_offsets(bool decode, bool align16, const int64_t* src_off, int64_t n,
                                 const BatchTables& tabs, const uint8_t* alph_id,
                                 int64_t* dst_off, cudaStream_t stream);

// ---- MIME decode (b64_mime.cu)
size_t mime_workspace_bytes(uint64_t m);
// Enqueues the whitespace-skipping strict decode; its bulk-copy waits give
// up after wait_limit_ns.
cudaError_t launch_mime_decode(const uint8_t* src, uint64_t m, uint8_t* dst,
                               const DecodeTable& tab, int flags, int64_t* d_result,
                               void* workspace, uint64_t wait_limit_ns, cudaStream_t stream);
// Self-test of the bounded wait: a barrier armed for a copy that never comes.
cudaError_t launch_selftest_wait(int64_t* d_result, uint64_t wait_limit_ns, cudaStream_t stream);
// Many MIME documents (BatchArgs: document i is src[src_off[i] .. src_off[i+1])
// -> dst + dst_off[i], results[i]); the workspace holds 8 * (5 n + slots)
// bytes, slots = total_bytes / 4096 + n + 1 (a smaller one makes every result
// B64_E_INVAL on the device).
size_t mime_batch_workspace_bytes(int64_t n, uint64_t total_bytes);
cudaError_t launch_mime_decode_batch(const BatchArgs& a, const BatchTables& tabs, void* workspace,
                                     size_t workspace_bytes, cudaStream_t stream);
uint32_t mime_fault_flag(bool clear);

// ---- programmatic dependent launch (the decode and MIME launch chains)
// A kernel launched by launch_dependent may start while the kernel before it
// on the stream finishes; wait_prior_grid waits until that kernel has
// completed and its writes are visible, and makes this kernel's own
// completion imply it, so a dependent kernel calls it before it reads what
// the kernel before wrote, and on every path before it exits. Launched
// plainly, the wait returns at once.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class... KArgs, class... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                             cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace b64
