// Batched strict decode that allocates nothing.
//
// b64_decode_batch needs a device workspace (one error word per string) that
// its caller allocates. Some callers cannot
// allocate device memory at the point where they decode: a plugin or
// extension that is handed only its input and output buffers, code that runs
// while another component owns the whole device-memory budget (a fixed pool,
// or a serving process whose memory is already spent), and latency-critical
// paths that must never enter an allocator. This entry point gives them the
// same decode with its workspace in a file-scope device array of the library.
//
// Limits and rules:
//   - at most kNoAllocMaxStrings strings per call; larger batches are refused
//     with an error (use b64_decode_batch with your own workspace);
//   - every GPU that loads the library's device code keeps this array
//     (512 KiB) until the process exits;
//   - all calls share the one array, so calls whose work overlaps on the GPU
//     (different streams, or different host threads) race and corrupt each
//     other's results: serialise them, e.g. on one stream;
//   - the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current. Under CUDA's default
//     lazy loading, that first call is also when the driver loads this
//     library's device code (the array and the kernels) onto the device,
//     which takes device memory; the calls after it allocate nothing. Make
//     that first call early, before the device-memory budget is spent, and
//     before any stream capture on the device.
#include <cinttypes>
#include <mutex>

#include "b64_internal.h"

namespace b64 {
namespace {

constexpr int64_t kNoAllocMaxStrings = 65536;
// Same layout as batch_workspace_bytes(kNoAllocMaxStrings): one error word
// per string (512 KiB).
constexpr size_t kNoAllocBytes = size_t(kNoAllocMaxStrings) * sizeof(uint64_t);

// The shared workspace. In host code this name only stands for the device
// array; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_workspace[kNoAllocBytes];

struct DeviceAddress {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    void* ptr = nullptr;
};
DeviceAddress g_address[64];

// The array's device address on the current device (set up once per device).
cudaError_t workspace_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    DeviceAddress& slot = g_address[dev & 63];
    std::call_once(slot.once, [&] {
        void* p = nullptr;
        slot.err = cudaGetSymbolAddress(&p, g_noalloc_workspace);
        slot.ptr = p;
    });
    *out = slot.ptr;
    return slot.err;
}

}  // namespace
}  // namespace b64

using namespace b64;

extern "C" int b64_decode_batch_noalloc(const uint8_t* src, const int64_t* src_off, int64_t n,
                                        uint8_t* dst, const int64_t* dst_off,
                                        const b64_alphabet* const* alphabets, int n_alphabets,
                                        const uint8_t* alph_id, int64_t* results, int tile_units,
                                        void* stream) {
    const char* fn = "b64_decode_batch_noalloc";
    if (n < 0) return set_error(B64_ERR_INVALID_ARGUMENT, "%s: n < 0", fn);
    if (n > kNoAllocMaxStrings)
        return set_error(B64_ERR_INVALID_ARGUMENT,
                         "%s: %" PRId64 " strings exceed the built-in workspace limit of %" PRId64
                         " strings per call; use b64_decode_batch with a caller workspace",
                         fn, n, kNoAllocMaxStrings);
    if (batch_workspace_bytes(n > 0 ? n : 1) > kNoAllocBytes)
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: workspace layout mismatch", fn);
    BatchTables tabs;
    const int rc = batch_tables(fn, alphabets, n_alphabets, &tabs);
    if (rc != B64_SUCCESS) return rc;
    if (n == 0) return B64_SUCCESS;
    if (!src_off || !dst_off || !results)
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: NULL pointer argument", fn);
    if (tile_units == 0) tile_units = 4;
    if (tile_units != 1 && tile_units != 2 && tile_units != 4 && tile_units != 8)
        return set_error(B64_ERR_INVALID_ARGUMENT, "%s: tile_units must be 0, 1, 2, 4 or 8", fn);
    void* ws = nullptr;
    cudaError_t e = workspace_address(&ws);
    if (e != cudaSuccess)
        return set_error(B64_ERR_CUDA, "%s: workspace address: %s", fn, cudaGetErrorString(e));
    // The call sets all n error words before the tile kernel reads them, so
    // nothing left by an earlier call leaks in.
    BatchArgs a{src, src_off, n, dst, dst_off, alph_id, results};
    e = launch_batch(true, a, tabs, tile_units, ws, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_error(B64_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return B64_SUCCESS;
}
