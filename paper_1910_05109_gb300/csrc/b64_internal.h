// Host-side declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "b64_device.cuh"

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
// or -(offset+1). d_result must already hold ~0 (no error) if m > 0.
cudaError_t launch_decode(const uint8_t* src, uint64_t m, uint8_t* dst, const DecodeTable& tab,
                          int padded, int64_t* d_result, cudaStream_t stream);

}  // namespace b64
