/*
 * b64gpu: base64 encode and strict decode on one NVIDIA GB300 GPU (sm_103a).
 *
 * The operations are those of Mula & Lemire, "Base64 encoding and decoding at
 * almost the speed of a memory copy" (arXiv:1910.05109):
 *   - encode (Sec. 2 and Sec. 3.1): every 3 input bytes s1,s2,s3 become the
 *     characters of the 6-bit values s1 div 4, (s2 div 16) + (s1*16) mod 64,
 *     (s2*4) mod 64 + (s3 div 64), s3 mod 64, looked up in a 64-entry
 *     alphabet (Table 1, or any other table given at run time, Sec. 3.1);
 *     '=' pads the output to a multiple of 4 characters (Sec. 2);
 *   - strict decode (Sec. 2 and Sec. 3.2): every 4 characters a,b,c,d become
 *     a*4 + b div 16, (b*16) mod 256 + c div 4, (c*64) mod 256 + d; any byte
 *     outside the alphabet is an error (Sec. 3.2, Fig. 2).
 *
 * Decoding rules where the paper is silent (the library's contract):
 *   - the error reported is the smallest offset among all errors;
 *   - a byte >= 0x80, or any byte not in the alphabet, is an error at its index;
 *   - padded alphabets: '=' is allowed only as the last character, or as the
 *     second-to-last when the last is '='; any other '=' is an error at its
 *     index; a length that is not a multiple of 4 is an error at offset len;
 *   - unpadded alphabets: every '=' is an error; a length of 1 mod 4 is an
 *     error at offset len;
 *   - bits of the last character that reach no output byte are ignored,
 *     unless the alphabet was made with B64_FLAG_CANONICAL: then, when the
 *     final group is partial (2 or 3 data characters once the padding is
 *     removed), its last data character must have those bits (the low 4 for
 *     2 characters, the low 2 for 3) at zero, else it is an error at its own
 *     offset (RFC 4648 Sec. 3.5, canonical encoding);
 *   - MIME mode (b64_mime_decode*): CR, LF and space are skipped first, the
 *     rules above apply to the rest, and offsets are in the original input.
 *
 * Conventions for every call below:
 *   - Data pointers (src, dst, offsets, results) are DEVICE pointers on the
 *     current CUDA device, owned by the caller. The library keeps no pointer
 *     after a call returns and never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Calls enqueue work on it and return without waiting, except
 *     where a call says it synchronises.
 *   - The library writes nothing past the output length it returns; on a
 *     decode error the content of dst is unspecified but nothing past
 *     b64_decoded_max_length(len) is written. One exception, stated at
 *     b64_mime_decode_async: a MIME input whose line layout breaks part way
 *     may leave bytes past the returned length (within
 *     b64_decoded_max_length(len)) overwritten.
 *   - src and dst must not overlap.
 *   - Any alignment is accepted; 16-byte aligned src and dst take the fast
 *     path.
 *   - Errors in arguments or CUDA calls are reported through the return value;
 *     b64_last_error() then gives a message for the calling thread.
 */
#ifndef B64GPU_H
#define B64GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Codes returned by calls that return int (0 = success). */
#define B64_SUCCESS 0
#define B64_ERR_INVALID_ARGUMENT (-1)
#define B64_ERR_CUDA (-2)

/* Codes returned by calls that return int64_t in place of a length. They are
 * far below -(len+1) for any possible len, so they cannot be mistaken for a
 * decode error offset. */
#define B64_E_INVAL (INT64_MIN + 1)
#define B64_E_CUDA (INT64_MIN + 2)
/* A device-side wait inside the call ran out of time (see
 * b64_device_fault_flag); the output is incomplete. */
#define B64_E_TIMEOUT (INT64_MIN + 3)

/* ---------------------------------------------------------------- alphabets
 * A 64-character table (Table 1 and its base64url variant, Sec. 2; any other
 * table at run time, Sec. 3.1) plus a padding mode. Handles are host objects,
 * immutable after creation and safe to share between threads. */
typedef struct b64_alphabet b64_alphabet;

/* chars: 64 distinct bytes, each < 0x80 and none of '=', CR, LF or space
 * (those have fixed meanings). padded: 1 = encode appends '=' and decode
 * requires it; 0 = no padding. Returns NULL (and sets b64_last_error) if chars
 * is invalid. Free with b64_alphabet_destroy. */
b64_alphabet* b64_alphabet_create(const uint8_t chars[64], int padded);

/* Alphabet flags: B64_FLAG_PADDED ('=' emitted by encode and required by
 * decode) and B64_FLAG_CANONICAL (decode rejects non-zero unused bits in a
 * partial final group, as stated at the top of this file). Not in the paper;
 * b64_alphabet_create(chars, padded) is the same as flags = padded ?
 * B64_FLAG_PADDED : 0. Returns NULL on invalid characters or unknown flag
 * bits (b64_last_error). */
#define B64_FLAG_PADDED 1
#define B64_FLAG_CANONICAL 2
b64_alphabet* b64_alphabet_create_flags(const uint8_t chars[64], int flags);

/* The alphabet's flags, or B64_ERR_INVALID_ARGUMENT for NULL. */
int b64_alphabet_flags(const b64_alphabet* a);

/* Table 1 (A-Z a-z 0-9 + /), padded. Static; never destroy. */
const b64_alphabet* b64_alphabet_standard(void);

/* base64url (Sec. 2: '+' and '/' replaced by '-' and '_'), unpadded. Static. */
const b64_alphabet* b64_alphabet_url(void);

/* Destroys a handle made by b64_alphabet_create (NULL and the static tables
 * are ignored). The caller must make sure no enqueued call still needs it:
 * calls copy the table into their launch parameters, so it may be destroyed
 * as soon as the call has returned. */
void b64_alphabet_destroy(b64_alphabet* a);

/* Copies the 64 characters into out and returns the padding mode. */
int b64_alphabet_chars(const b64_alphabet* a, uint8_t out[64]);

/* ---------------------------------------------------------------- lengths */

/* Encoded length of n bytes: 4*ceil(n/3) when padded, ceil(4n/3) when not
 * (Sec. 2). */
size_t b64_encoded_length(size_t n, int padded);

/* Capacity a decode output needs for m input characters: 3*ceil(m/4). */
size_t b64_decoded_max_length(size_t m);

/* ---------------------------------------------------------------- single buffer */

/* Encodes len bytes at src into dst (capacity >= b64_encoded_length(len,
 * padded)). Enqueues on stream and returns the output length immediately, or
 * B64_E_INVAL / B64_E_CUDA. */
int64_t b64_encode(const uint8_t* src, size_t len, uint8_t* dst, const b64_alphabet* a,
                   void* stream);

/* Strict decode of len characters at src into dst (capacity >=
 * b64_decoded_max_length(len)). Enqueues, writes the result to the device
 * int64 *d_result (8-byte aligned, caller-owned) and returns B64_SUCCESS
 * without waiting. *d_result becomes the decoded length (>= 0) or
 * -(offset+1), offset in [0, len] being the first error (offset == len: bad
 * length), or B64_E_TIMEOUT if a bounded wait on one of the kernel's bulk
 * copies ran out (the output is then incomplete). If such a wait ran out
 * while another part of the input held a bad character, *d_result is that
 * character's offset, which then need not be the first; b64_device_fault_flag
 * reports the timeout in both cases. Returns B64_ERR_INVALID_ARGUMENT /
 * B64_ERR_CUDA on failure to enqueue. */
int b64_decode_async(const uint8_t* src, size_t len, uint8_t* dst, const b64_alphabet* a,
                     int64_t* d_result, void* stream);

/* As b64_decode_async, then waits for the stream and returns *d_result's
 * value (which may be B64_E_TIMEOUT), or B64_E_INVAL / B64_E_CUDA. Uses one 8-byte device word and one
 * pinned host word per calling thread and device, allocated on the thread's
 * first call and kept until the process exits. */
int64_t b64_decode(const uint8_t* src, size_t len, uint8_t* dst, const b64_alphabet* a,
                   void* stream);

/* ---------------------------------------------------------------- MIME
 * Strict decode that first skips CR, LF and space anywhere in the input
 * (line-wrapped base64 as in MIME; the paper names MIME only as motivation,
 * Sec. 1). The remaining characters are decoded exactly as b64_decode_async
 * decodes them (Sec. 2, Sec. 3.2, and the rules at the top of this file);
 * error offsets are offsets into the original input, and a bad length is
 * reported at offset len. Five kernels on `stream`. First a one-pass decode:
 * if the input starts with a line of L data characters (L a multiple of 4,
 * below 1024) and a CR LF or LF break, every 4 KiB segment is decoded at
 * the output offset that this line layout gives it, and checks that its
 * whitespace sits exactly where the layout puts breaks. Only if a segment
 * does not (or there is no layout) do the next three kernels run: a count of
 * the data characters of every segment, a scan of those counts, and the
 * decode of every segment at its counted output offset; otherwise they
 * return at once. A one-thread kernel then writes *d_result: the decoded
 * length, -(offset+1), or B64_E_TIMEOUT (a bounded wait ran out). When the
 * layout breaks part way, the one-pass kernel may already have written the
 * segments after the break at their layout offsets: bytes past the returned
 * length, within b64_decoded_max_length(len), can then be overwritten.
 * workspace: device memory of b64_mime_workspace_size(len) bytes, 8-byte
 * aligned, caller-owned, busy until the work completes (one call at a time per
 * workspace). dst needs b64_decoded_max_length(len) bytes. */
size_t b64_mime_workspace_size(size_t len);

int b64_mime_decode_async(const uint8_t* src, size_t len, uint8_t* dst, const b64_alphabet* a,
                          int64_t* d_result, void* workspace, size_t workspace_bytes,
                          void* stream);

/* Many MIME documents in one launch sequence (not in the paper): document i
 * is src[src_off[i] .. src_off[i+1]) (device int64[n+1], any alignment),
 * decoded exactly as b64_mime_decode_async decodes it, to dst + dst_off[i]
 * (room for b64_decoded_max_length of its length, e.g. from
 * b64_batch_offsets with decode != 0), with alphabets[alph_id[i]] (alph_id
 * NULL: alphabet 0); results[i] receives its length or -(offset+1), offset
 * within the document, or B64_E_TIMEOUT (a bounded wait on one of its
 * segments' bulk copies ran out; if another of its segments held a bad
 * character, that offset is reported instead and need not be the first;
 * b64_device_fault_flag reports the timeout in both cases). workspace: device memory of
 * b64_mime_batch_workspace_size(n, src_off[n] - src_off[0]) bytes, 8-byte
 * aligned; if the documents' total turns out larger than the size was
 * computed for, every results[i] becomes B64_E_INVAL and nothing else is
 * written. Seven launches on `stream`, no waits between blocks: a memset,
 * per-document line layout, a one-pass decode of the documents laid out as
 * lines (as b64_mime_decode_async decodes them, so the same note on bytes past
 * the result holds), then count, per-document scan and decode for the others
 * (each returning at once when every document kept its line layout), and the
 * results; each kernel after the layout kernel is a programmatic dependent
 * of the one before (it may start while that one finishes, and waits for it
 * before reading its results). Returns B64_SUCCESS or an error code; n == 0
 * enqueues nothing. */
size_t b64_mime_batch_workspace_size(int64_t n, uint64_t total_bytes);

int b64_mime_decode_batch(const uint8_t* src, const int64_t* src_off, int64_t n, uint8_t* dst,
                          const int64_t* dst_off, const b64_alphabet* const* alphabets,
                          int n_alphabets, const uint8_t* alph_id, int64_t* results,
                          void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- batches
 * Many independent strings in one launch sequence (a per-string results
 * kernel or error-word memset, one persistent tile kernel, and for decode a
 * per-string finalize kernel), all
 * on `stream`, so it can be recorded in a CUDA graph. Batching is not in the
 * paper; each string is coded exactly as the single-buffer calls code it.
 *
 * String i is src[src_off[i] .. src_off[i+1]) (src_off: n+1 device int64,
 * non-decreasing, src_off[0] may be > 0) and is written at dst + dst_off[i]
 * (dst_off: n device int64; each string needs its capacity, see
 * b64_batch_offsets). alph_id: n device bytes selecting one of the
 * n_alphabets (1..B64_BATCH_MAX_ALPHABETS) handles, or NULL for alphabet 0;
 * an id >= n_alphabets is a caller error (it is taken modulo
 * B64_BATCH_MAX_ALPHABETS and reads a repeat of alphabet 0). results: n
 * device int64, receiving what the single-buffer call returns for that string
 * (encode: output length; decode: length or -(offset+1), offset within the
 * string). tile_units: bytes per thread of a tile as 1, 2, 4 or 8 units of
 * 12 input bytes (encode) or 16 characters (decode), 0 picks 8; optionally
 * OR-ed with (b << 8), b resident blocks of 8 warps per SM (at most as many
 * as fit; 0: as many as fit), the number of warps the batch is spread over,
 * and with B64_TILE_PAIRS (encode with 8 units, at most 2 alphabets; ignored
 * otherwise): tiles of one string's full units are encoded through 4096-entry
 * tables of character pairs built per block (faster for long strings, slower
 * where tiles are shared by many strings). All are the autotuner's choices;
 * any value gives the same results. workspace:
 * device memory of at least b64_batch_workspace_size(n) bytes, 256-byte
 * aligned, owned by the caller and busy until the enqueued work completes.
 * Strings may start at any alignment; src and dst may be NULL only if every
 * string is empty. If a bounded wait on a tile's bulk copy runs out, the
 * kernel stops early and sets the flag b64_device_fault_flag reads; results
 * and output are then incomplete. Returns B64_SUCCESS or an error code;
 * nothing is enqueued on error. n == 0 enqueues nothing. */
#define B64_BATCH_MAX_ALPHABETS 4
#define B64_TILE_PAIRS (1 << 16)

size_t b64_batch_workspace_size(int64_t n);

int b64_encode_batch(const uint8_t* src, const int64_t* src_off, int64_t n, uint8_t* dst,
                     const int64_t* dst_off, const b64_alphabet* const* alphabets,
                     int n_alphabets, const uint8_t* alph_id, int64_t* results, int tile_units,
                     void* workspace, size_t workspace_bytes, void* stream);

int b64_decode_batch(const uint8_t* src, const int64_t* src_off, int64_t n, uint8_t* dst,
                     const int64_t* dst_off, const b64_alphabet* const* alphabets,
                     int n_alphabets, const uint8_t* alph_id, int64_t* results, int tile_units,
                     void* workspace, size_t workspace_bytes, void* stream);

/* Batched strict decode for callers that cannot allocate device memory where
 * they decode (a plugin handed only its buffers, a process whose memory budget
 * another component owns, a path that must never enter an allocator). The
 * paper has no counterpart; this is b64_decode_batch with its workspace in a
 * file-scope device array of the library (512 KiB on every GPU that loads the
 * library's device code, kept until exit) instead of caller memory. Same
 * arguments and results as b64_decode_batch, without workspace. At most 65536
 * strings per call (more returns B64_ERR_INVALID_ARGUMENT). The call itself
 * calls no allocator. All calls share the one array: calls whose work
 * overlaps on the GPU race, so serialise them (e.g. one stream). The first
 * call on each device looks up the array's device address, and under CUDA's
 * default lazy loading it is also where the driver loads the library's
 * device code (the array and the kernels), which takes device memory: make
 * that first call early, before the device-memory budget is spent, and
 * outside any stream capture. */
int b64_decode_batch_noalloc(const uint8_t* src, const int64_t* src_off, int64_t n,
                             uint8_t* dst, const int64_t* dst_off,
                             const b64_alphabet* const* alphabets, int n_alphabets,
                             const uint8_t* alph_id, int64_t* results, int tile_units,
                             void* stream);

/* dst_off[0..n] (n+1 device int64) = exclusive scan of each string's output
 * capacity: its encoded length, or 3*ceil(len/4) with B64_OFFSETS_DECODE.
 * With B64_OFFSETS_ALIGN16 each capacity is rounded up to a multiple of 16
 * bytes, so that with a 16-byte aligned dst every string's output starts
 * 16-byte aligned; the batched kernels then store each string's output
 * straight from registers (with any other layout they realign it through
 * shared memory first). The bytes between one string's output and the next
 * string are left untouched. dst_off[n] is the total. flags: 0 or the two
 * flags OR-ed (0 and 1 as the encode / decode switch of earlier versions);
 * other bits are B64_ERR_INVALID_ARGUMENT. Three kernels on `stream`. */
#define B64_OFFSETS_DECODE 1
#define B64_OFFSETS_ALIGN16 2
int b64_batch_offsets(const int64_t* src_off, int64_t n, const b64_alphabet* const* alphabets,
                      int n_alphabets, const uint8_t* alph_id, int flags, int64_t* dst_off,
                      void* stream);

/* ---------------------------------------------------------------- host buffers
 * Encode or strictly decode a buffer that lives in host memory (not in the
 * paper, which codes buffers already in the processor's memory). The codec
 * owns n_streams streams and, per stream, one device piece buffer for input
 * and one for output, allocated once here; a call copies consecutive pieces
 * of piece_bytes to the device, codes them and copies the results back, the
 * three steps of different pieces overlapping on the streams. Host buffers
 * that are page-locked (cudaHostAlloc / cudaHostRegister, torch
 * pin_memory) give full overlap; pageable ones work, with copies the CUDA
 * driver stages itself. Results are those of b64_encode / b64_decode on the whole
 * buffer: decode pieces after the first are offset-shifted, inner pieces
 * treat every '=' as an error and the last piece always holds the last two
 * characters, so the padding and length rules apply to the whole input
 * (Sec. 2). A codec serves one call at a time (calls from several threads
 * take turns) and stays on the device that was current when it was made. */
typedef struct b64_host_codec b64_host_codec;

/* piece_bytes: input bytes per piece, rounded down to a multiple of 12
 * (0 picks 48 MiB); n_streams: 1..8 (0 picks 3). Device memory used:
 * b64_host_codec_device_bytes. Returns NULL on failure (b64_last_error). */
b64_host_codec* b64_host_codec_create(size_t piece_bytes, int n_streams);

size_t b64_host_codec_device_bytes(const b64_host_codec* c);

/* Host src (len bytes) -> host dst (b64_encoded_length(len, padded) bytes).
 * Blocks until the output is in dst. Returns the output length, B64_E_INVAL
 * or B64_E_CUDA. */
int64_t b64_host_encode(b64_host_codec* c, const uint8_t* src, size_t len, uint8_t* dst,
                        const b64_alphabet* a);

/* Host src (len characters) -> host dst (b64_decoded_max_length(len) bytes,
 * contents past an error unspecified). Blocks until done. Returns the decoded
 * length, -(offset+1) of the first invalid character, B64_E_TIMEOUT,
 * B64_E_INVAL or B64_E_CUDA. */
int64_t b64_host_decode(b64_host_codec* c, const uint8_t* src, size_t len, uint8_t* dst,
                        const b64_alphabet* a);

/* Waits for the codec's streams, then frees it. */
void b64_host_codec_destroy(b64_host_codec* c);

/* ---------------------------------------------------------------- serving
 * A request engine with continuous batching (not in the paper; it drives the
 * codec above). The server owns a device arena of budget_bytes and a pinned
 * host staging area of the same size, allocated once here. b64_server_submit
 * queues a request (host input and output buffers, owned by the caller and
 * untouched until the request completes). b64_server_poll makes progress
 * without blocking: it hands back finished requests and, whenever one of the
 * n_streams streams is idle and arena space is free, launches the queued
 * requests in arrival order (up to max_batch_bytes of input+output, 0 = 64
 * MiB) as one batched encode and/or one batched decode: a host-to-device
 * copy, the batched kernels, device-to-host copies. Batches on different
 * streams overlap, and requests that arrive while others run join the next
 * batch. Host copies into and out of the staging area are spread over up to
 * eight worker threads the server starts (half the hardware threads). A
 * server is used by one thread at a time. */
typedef struct b64_server b64_server;

typedef struct {
    uint64_t tag;      /* the caller's tag from b64_server_submit */
    int64_t result;    /* as b64_encode / b64_decode return for this request */
    double latency_us; /* from submit to the poll that handed it back */
} b64_completion;

/* Returns NULL on failure (b64_last_error). alphabets: 1..B64_BATCH_MAX_ALPHABETS. */
b64_server* b64_server_create(size_t budget_bytes, int n_streams, size_t max_batch_bytes,
                              const b64_alphabet* const* alphabets, int n_alphabets);

/* op: 0 = encode, 1 = strict decode; alph_id indexes the server's alphabets
 * (0 .. n_alphabets - 1; others are refused). out_cap: at least
 * b64_encoded_length (encode) or b64_decoded_max_length (decode) of len. A
 * request that could never fit the budget is refused. */
int b64_server_submit(b64_server* s, uint64_t tag, int op, int alph_id, const uint8_t* in,
                      size_t len, uint8_t* out, size_t out_cap);

/* Queues n requests in one call (fewer crossings for callers that collect
 * arrivals): request i is (tags[i], ops[i], alph_ids[i], ins[i], lens[i],
 * outs[i], out_caps[i]), each checked as b64_server_submit checks one, in
 * order. Returns how many were queued: n, or the index of the first refused
 * request (b64_last_error says why; none after it is queued); an error code
 * < 0 for a NULL array with n > 0. */
int b64_server_submit_many(b64_server* s, int n, const uint64_t* tags, const int32_t* ops,
                           const int32_t* alph_ids, const uint8_t* const* ins,
                           const uint64_t* lens, uint8_t* const* outs, const uint64_t* out_caps);

/* Writes up to max_out completions; returns how many (or an error code < 0). */
int b64_server_poll(b64_server* s, b64_completion* out, int max_out);

/* Requests submitted and not yet handed back. */
int b64_server_outstanding(const b64_server* s);

/* Batches launched so far. */
uint64_t b64_server_batches(const b64_server* s);

/* Waits for in-flight work, then frees the server. */
void b64_server_destroy(b64_server* s);

/* ---------------------------------------------------------------- diagnostics */

/* Thread-local message for the last failed call of this thread ("" if none). */
const char* b64_last_error(void);

/* Every wait inside the library's kernels is bounded in time; a kernel whose
 * wait runs out sets a per-device flag and returns early (its output is then
 * incomplete). Returns the flag of the current device (0 = never set) and
 * clears it if clear != 0. Synchronises the device. Negative on CUDA error. */
int b64_device_fault_flag(int clear);

/* Self-test of the bounded device waits: runs the wait the kernels use for
 * their bulk (TMA) copies on a barrier armed for a copy that is never issued,
 * giving up after wait_limit_ns (1 .. 2e9). *d_result then becomes
 * B64_E_TIMEOUT and b64_device_fault_flag reports the timeout; the wait lasts
 * no longer than the limit and the context stays usable. Returns B64_SUCCESS
 * if the work was enqueued. */
int b64_selftest_wait_timeout(int64_t* d_result, uint64_t wait_limit_ns, void* stream);

/* Library version: major*10000 + minor*100 + patch. */
int b64_version(void);

#ifdef __cplusplus
}
#endif

#endif /* B64GPU_H */
