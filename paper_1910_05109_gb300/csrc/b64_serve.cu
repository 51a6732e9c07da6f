// Serving engine: continuous batching of encode/decode requests under a
// device-memory budget (not in the paper; it drives the paper's codec).
//
// The engine owns one device arena (the budget) and a pinned host staging
// area of the same size, both allocated once by b64_server_create. Each poll:
//   1. reaps batches whose completion event has fired, copies each
//      request's result from staging into the caller's output buffer and
//      releases, in allocation order, the arena blocks of the finished
//      prefix;
//   2. while a stream is idle and requests are queued, takes queued requests
//      in arrival order up to max_batch_bytes, splits them by operation, and
//      for each part reserves one contiguous block of the ring (payload,
//      outputs, offsets, alphabet ids, results, batch workspace), packs the
//      payloads into staging, and enqueues on that stream: one host-to-device
//      copy, the batched kernels, the device-to-host copies, an event.
// Batches on different streams overlap (copies of one with kernels of
// another); requests that arrive while batches run are admitted as soon as a
// stream and ring space are free. One thread at a time may use a server.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "b64_internal.h"
#include "b64_serve_plan.h"

using Clock = std::chrono::steady_clock;

namespace {

using b64serve::align_up;
using b64serve::Ring;
constexpr size_t kMaxBatchRequests = 16384;

// Host copies of one poll (packing payloads into staging, unpacking
// results into the callers' buffers) spread over worker threads: the tasks
// are cut into pieces of at most kPiece bytes and taken from a shared index
// by the workers and the calling thread. Each run is its own job object, so
// a worker that wakes late only ever sees a finished job. Small jobs run on
// the caller alone.
class CopyPool {
public:
    struct Task {
        void* dst;
        const void* src;
        size_t len;
    };
    static constexpr size_t kPiece = size_t(1) << 20;
    static constexpr size_t kInline = size_t(512) << 10;

    explicit CopyPool(int threads) {
        for (int i = 0; i < threads; ++i) workers_.emplace_back([this] { work(); });
    }
    ~CopyPool() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto& t : workers_) t.join();
    }

    void run(const std::vector<Task>& tasks) {
        size_t total = 0;
        for (const auto& t : tasks) total += t.len;
        if (workers_.empty() || total <= kInline) {
            for (const auto& t : tasks)
                if (t.len) memcpy(t.dst, t.src, t.len);
            return;
        }
        auto job = std::make_shared<Job>();
        for (const auto& t : tasks)
            for (size_t o = 0; o < t.len; o += kPiece)
                job->pieces.push_back({static_cast<uint8_t*>(t.dst) + o,
                                       static_cast<const uint8_t*>(t.src) + o,
                                       std::min(kPiece, t.len - o)});
        job->left.store(job->pieces.size());
        {
            std::lock_guard<std::mutex> g(mu_);
            job_ = job;
            ++generation_;
        }
        cv_.notify_all();
        drain(*job);
        std::unique_lock<std::mutex> g(mu_);
        done_cv_.wait(g, [&] { return job->left.load() == 0; });
    }

private:
    struct Job {
        std::vector<Task> pieces;
        std::atomic<size_t> next{0}, left{0};
    };
    void drain(Job& j) {
        for (;;) {
            const size_t i = j.next.fetch_add(1);
            if (i >= j.pieces.size()) return;
            memcpy(j.pieces[i].dst, j.pieces[i].src, j.pieces[i].len);
            if (j.left.fetch_sub(1) == 1) {
                std::lock_guard<std::mutex> g(mu_);
                done_cv_.notify_all();
            }
        }
    }
    void work() {
        uint64_t seen = 0;
        for (;;) {
            std::shared_ptr<Job> job;
            {
                std::unique_lock<std::mutex> g(mu_);
                cv_.wait(g, [&] { return stop_ || generation_ != seen; });
                if (stop_) return;
                seen = generation_;
                job = job_;
            }
            drain(*job);
        }
    }

    std::vector<std::thread> workers_;
    std::shared_ptr<Job> job_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    uint64_t generation_ = 0;
    bool stop_ = false;
};

int default_copy_threads() {
    const unsigned hw = std::thread::hardware_concurrency();
    const int n = hw > 2 ? int(hw / 2) : 0;
    return n > 8 ? 8 : n;
}

}  // namespace

struct b64_server_req {
    uint64_t tag;
    int op;
    int alph;
    const uint8_t* in;
    size_t len;
    uint8_t* out;
    size_t out_cap;
    size_t cap;  // device output capacity of this request
    Clock::time_point t0;
};

struct b64_server_batch {
    int op = 0;
    int stream = 0;
    std::vector<b64_server_req> reqs;
    size_t off = 0, bytes = 0;  // ring block
    size_t o_in = 0, o_out = 0, o_meta = 0, o_res = 0, o_ws = 0, meta_bytes = 0;
    std::vector<int64_t> dst_off;
    cudaEvent_t done = nullptr;
    bool ready = false;     // event fired; results are in staging
    size_t reported = 0;    // requests already handed back by poll
    bool finished = false;  // every request handed back
};

struct b64_server {
    size_t budget = 0, max_batch_bytes = 0;
    uint8_t* d_arena = nullptr;
    uint8_t* h_stage = nullptr;
    Ring ring{0};
    b64::BatchTables tabs{};
    int padded[b64::kMaxAlphabets] = {0, 0, 0, 0};
    std::vector<cudaStream_t> streams;
    std::vector<int> busy;  // batches in flight per stream
    std::deque<b64_server_req> queue;
    std::deque<b64_server_batch> inflight;
    int device = 0;
    uint64_t launched_batches = 0;
    CopyPool* copies = nullptr;
    std::vector<CopyPool::Task> tasks;  // scratch of one poll
};

namespace {

size_t out_capacity(const b64_server* s, int op, int alph, size_t len) {
    return op == 0 ? b64_encoded_length(len, s->padded[alph]) : b64_decoded_max_length(len);
}

// Layout of a batch block: [src_off n+1][dst_off n+1][ids n][payload]
// [outputs][results n][workspace], sections 256-byte aligned, so that one
// host-to-device copy moves the offsets and the payload, and one
// device-to-host copy the outputs and the results.
size_t workspace_bytes(size_t n) { return b64::batch_workspace_bytes(int64_t(n)); }

// Section offsets of the block; the total is b64serve::block_bytes.
size_t batch_layout(b64_server_batch& b, size_t in_bytes, size_t out_bytes) {
    const size_t n = b.reqs.size();
    b.o_meta = 0;
    b.meta_bytes = b64serve::meta_bytes(n);
    b.o_in = b.meta_bytes;
    b.o_out = b.o_in + align_up(in_bytes);
    b.o_res = b.o_out + align_up(out_bytes);
    b.o_ws = b.o_res + align_up(n * sizeof(int64_t));
    return b64serve::block_bytes(n, in_bytes, out_bytes, workspace_bytes(n));
}

size_t single_request_bytes(size_t len, size_t cap) {
    return b64serve::block_bytes(1, len, cap, workspace_bytes(1));
}

int launch(b64_server* s, b64_server_batch& b) {
    const size_t n = b.reqs.size();
    size_t in_bytes = 0, out_bytes = 0;
    for (auto& r : b.reqs) {
        in_bytes += r.len;
        out_bytes += r.cap;
    }
    const size_t bytes = batch_layout(b, in_bytes, out_bytes);
    if (!s->ring.reserve(bytes, &b.off)) return 1;  // no room yet
    b.bytes = bytes;
    uint8_t* h = s->h_stage + b.off;
    uint8_t* d = s->d_arena + b.off;
    int64_t* h_src_off = reinterpret_cast<int64_t*>(h + b.o_meta);
    int64_t* h_dst_off = h_src_off + (n + 1);
    uint8_t* h_ids = reinterpret_cast<uint8_t*>(h_dst_off + (n + 1));
    b.dst_off.resize(n + 1);
    s->tasks.clear();
    size_t pi = 0, po = 0;
    for (size_t i = 0; i < n; ++i) {
        const auto& r = b.reqs[i];
        if (r.len) s->tasks.push_back({h + b.o_in + pi, r.in, r.len});
        h_src_off[i] = int64_t(pi);
        h_dst_off[i] = int64_t(po);
        b.dst_off[i] = int64_t(po);
        h_ids[i] = uint8_t(r.alph);
        pi += r.len;
        po += r.cap;
    }
    h_src_off[n] = int64_t(pi);
    h_dst_off[n] = int64_t(po);
    b.dst_off[n] = int64_t(po);
    s->copies->run(s->tasks);
    cudaStream_t st = s->streams[b.stream];
    cudaError_t e = cudaMemcpyAsync(d, h, b.o_in + in_bytes, cudaMemcpyHostToDevice, st);
    b64::BatchArgs a{d + b.o_in, reinterpret_cast<const int64_t*>(d + b.o_meta), int64_t(n),
                     d + b.o_out, reinterpret_cast<const int64_t*>(d + b.o_meta) + (n + 1),
                     d + b.o_meta + 2 * (n + 1) * sizeof(int64_t),
                     reinterpret_cast<int64_t*>(d + b.o_res)};
    if (e == cudaSuccess) e = b64::launch_batch(b.op == 1, a, s->tabs, 4, d + b.o_ws, st);
    if (e == cudaSuccess)  // outputs and results in one copy
        e = cudaMemcpyAsync(h + b.o_out, d + b.o_out, b.o_res - b.o_out + n * sizeof(int64_t),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(b.done, st);
    if (e != cudaSuccess) {
        // Whatever was enqueued finishes before the block is handed out again.
        cudaStreamSynchronize(st);
        s->ring.release_back();
        return -1;
    }
    return 0;
}

}  // namespace

using namespace b64;

extern "C" {

b64_server* b64_server_create(size_t budget_bytes, int n_streams, size_t max_batch_bytes,
                              const b64_alphabet* const* alphabets, int n_alphabets) {
    if (budget_bytes < (size_t(1) << 20) || n_streams < 1 || n_streams > 16) {
        set_error(0, "b64_server_create: budget must be >= 1 MiB and streams in 1..16");
        return nullptr;
    }
    b64_server* s = new b64_server;
    if (batch_tables("b64_server_create", alphabets, n_alphabets, &s->tabs) != B64_SUCCESS) {
        delete s;
        return nullptr;
    }
    for (int k = 0; k < kMaxAlphabets; ++k) s->padded[k] = s->tabs.padded[k];
    s->budget = budget_bytes & ~(b64serve::kAlign - 1);
    s->max_batch_bytes = max_batch_bytes ? max_batch_bytes : (size_t(64) << 20);
    s->ring = Ring(s->budget);
    cudaGetDevice(&s->device);
    cudaError_t e = cudaMalloc(&s->d_arena, s->budget);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_stage, s->budget);
    for (int i = 0; e == cudaSuccess && i < n_streams; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->streams.push_back(st);
    }
    s->busy.assign(s->streams.size(), 0);
    s->copies = new CopyPool(default_copy_threads());
    if (e != cudaSuccess) {
        set_error(0, "b64_server_create: %s", cudaGetErrorString(e));
        b64_server_destroy(s);
        return nullptr;
    }
    return s;
}

int b64_server_submit(b64_server* s, uint64_t tag, int op, int alph_id, const uint8_t* in,
                      size_t len, uint8_t* out, size_t out_cap) {
    if (!s || (op != 0 && op != 1) || alph_id < 0 || alph_id >= s->tabs.n_alph ||
        (len && (!in || !out)))
        return set_error(B64_ERR_INVALID_ARGUMENT, "b64_server_submit: bad argument");
    b64_server_req r{tag, op, alph_id, in, len, out, out_cap, 0, Clock::now()};
    r.cap = out_capacity(s, op, alph_id, len);
    if (out_cap < (op == 0 ? r.cap : b64_decoded_max_length(len)))
        return set_error(B64_ERR_INVALID_ARGUMENT, "b64_server_submit: out_cap below %zu", r.cap);
    if (single_request_bytes(len, r.cap) > s->budget)
        return set_error(B64_ERR_INVALID_ARGUMENT,
                         "b64_server_submit: request needs more than the device budget");
    s->queue.push_back(r);
    return B64_SUCCESS;
}

int b64_server_submit_many(b64_server* s, int n, const uint64_t* tags, const int32_t* ops,
                           const int32_t* alph_ids, const uint8_t* const* ins,
                           const uint64_t* lens, uint8_t* const* outs, const uint64_t* out_caps) {
    if (!s || n < 0 ||
        (n > 0 && (!tags || !ops || !alph_ids || !ins || !lens || !outs || !out_caps)))
        return set_error(B64_ERR_INVALID_ARGUMENT, "b64_server_submit_many: bad argument");
    for (int i = 0; i < n; ++i)
        if (b64_server_submit(s, tags[i], ops[i], alph_ids[i], ins[i], size_t(lens[i]), outs[i],
                              size_t(out_caps[i])) != B64_SUCCESS)
            return i;
    return n;
}

int b64_server_poll(b64_server* s, b64_completion* out, int max_out) {
    if (!s || max_out < 0 || (max_out > 0 && !out))
        return set_error(B64_ERR_INVALID_ARGUMENT, "b64_server_poll: bad argument");
    int nout = 0;
    // 1. reap finished batches (results in staging), release the ring prefix
    for (auto& b : s->inflight) {
        if (b.finished) continue;
        if (!b.ready) {
            const cudaError_t q = cudaEventQuery(b.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess)
                return set_error(B64_ERR_CUDA, "b64_server_poll: %s", cudaGetErrorString(q));
            b.ready = true;
        }
        const uint8_t* h = s->h_stage + b.off;
        const int64_t* res = reinterpret_cast<const int64_t*>(h + b.o_res);
        const auto now = Clock::now();
        const size_t first = b.reported;
        const size_t take = std::min(b.reqs.size() - first, size_t(max_out - nout));
        s->tasks.clear();
        for (size_t i = first; i < first + take; ++i)
            if (res[i] > 0) s->tasks.push_back({b.reqs[i].out, h + b.o_out + b.dst_off[i], size_t(res[i])});
        s->copies->run(s->tasks);
        for (size_t i = first; i < first + take; ++i) {
            const auto& r = b.reqs[i];
            out[nout].tag = r.tag;
            out[nout].result = res[i];
            out[nout].latency_us = std::chrono::duration<double, std::micro>(now - r.t0).count();
            ++nout;
        }
        b.reported = first + take;
        if (b.reported == b.reqs.size()) {
            b.finished = true;
            s->busy[b.stream] -= 1;
        }
        if (nout == max_out) break;
    }
    while (!s->inflight.empty() && s->inflight.front().finished) {
        cudaEventDestroy(s->inflight.front().done);
        s->inflight.pop_front();
        s->ring.release_front();
    }
    // 2. launch queued requests on idle streams
    for (size_t si = 0; si < s->streams.size() && !s->queue.empty(); ++si) {
        if (s->busy[si]) continue;
        b64_server_batch parts[2];
        const size_t taken = b64serve::plan_take(s->queue, s->max_batch_bytes, s->budget,
                                                 kMaxBatchRequests, workspace_bytes);
        for (size_t k = 0; k < taken; ++k) parts[s->queue[k].op].reqs.push_back(s->queue[k]);
        bool sent[2] = {false, false}, stalled = false;
        for (int op = 0; op < 2; ++op) {
            b64_server_batch& b = parts[op];
            if (b.reqs.empty()) continue;
            b.op = op;
            b.stream = int(si);
            if (cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess)
                return set_error(B64_ERR_CUDA, "b64_server_poll: event creation failed");
            const int rc = launch(s, b);
            if (rc != 0) {
                cudaEventDestroy(b.done);
                if (rc < 0) return set_error(B64_ERR_CUDA, "b64_server_poll: launch failed");
                stalled = true;  // no ring space now: wait for completions
                break;
            }
            sent[op] = true;
            s->busy[si] += 1;
            s->launched_batches += 1;
            s->inflight.push_back(std::move(b));
        }
        if (sent[0] || sent[1]) {  // drop what was sent; keep the rest in order
            std::deque<b64_server_req> rest;
            for (size_t k = 0; k < s->queue.size(); ++k)
                if (!(k < taken && sent[s->queue[k].op])) rest.push_back(s->queue[k]);
            s->queue.swap(rest);
        }
        if (stalled) break;
    }
    return nout;
}

int b64_server_outstanding(const b64_server* s) {
    if (!s) return set_error(B64_ERR_INVALID_ARGUMENT, "b64_server_outstanding: NULL");
    size_t n = s->queue.size();
    for (auto& b : s->inflight)
        if (!b.finished) n += b.reqs.size();
    return int(n);
}

uint64_t b64_server_batches(const b64_server* s) { return s ? s->launched_batches : 0; }

void b64_server_destroy(b64_server* s) {
    if (!s) return;
    for (auto st : s->streams) cudaStreamSynchronize(st);
    for (auto& b : s->inflight)
        if (b.done) cudaEventDestroy(b.done);
    for (auto st : s->streams) cudaStreamDestroy(st);
    if (s->d_arena) cudaFree(s->d_arena);
    if (s->h_stage) cudaFreeHost(s->h_stage);
    delete s->copies;
    delete s;
}

}  // extern "C"
