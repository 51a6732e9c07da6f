// Host-only planning of the serving engine (no CUDA): the arena ring that
// hands out batch blocks, the size of one batch block, and how many queued
// requests the next batch takes. Kept free of CUDA types so that it can be
// compiled and checked on a machine without a GPU.
#ifndef B64_SERVE_PLAN_H
#define B64_SERVE_PLAN_H

#include <cstddef>
#include <cstdint>
#include <deque>
#include <utility>

namespace b64serve {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Bytes of the arena block of one batch of n requests with in_bytes of
// payload, out_bytes of output capacity and ws_bytes of kernel workspace:
// [src_off n+1][dst_off n+1][ids n][payload][outputs][results n][workspace],
// every section 256-byte aligned.
inline size_t meta_bytes(size_t n) { return align_up(2 * (n + 1) * sizeof(int64_t) + n); }
inline size_t block_bytes(size_t n, size_t in_bytes, size_t out_bytes, size_t ws_bytes) {
    return meta_bytes(n) + align_up(in_bytes) + align_up(out_bytes) +
           align_up(n * sizeof(int64_t)) + align_up(ws_bytes);
}

// Contiguous blocks of [0, cap), released in the order they were reserved
// (or the newest one taken back).
class Ring {
public:
    explicit Ring(size_t cap) : cap_(cap) {}
    bool reserve(size_t size, size_t* off) {
        size_t at;
        if (blocks_.empty()) {
            at = 0;
            if (size > cap_) return false;
        } else {
            const size_t first = blocks_.front().first;
            const size_t end = blocks_.back().first + blocks_.back().second;
            // Wrapped: the newest block starts before the oldest. Its end can
            // then equal the oldest block's start (no room left), so the
            // order of the blocks, not end against first, tells the cases apart.
            if (blocks_.back().first >= first) {  // room after the end, or before the first
                if (end + size <= cap_) at = end;
                else if (size <= first) at = 0;
                else return false;
            } else {  // room between the end and the first
                if (end + size <= first) at = end;
                else return false;
            }
        }
        blocks_.emplace_back(at, size);
        *off = at;
        return true;
    }
    void release_front() { blocks_.pop_front(); }
    void release_back() { blocks_.pop_back(); }
    size_t blocks() const { return blocks_.size(); }

private:
    size_t cap_;
    std::deque<std::pair<size_t, size_t>> blocks_;
};

// How many requests, from the front of `queue` (arrival order), the next
// batch takes. A batch is split by operation into two parts, each reserved
// as one block. Taking stops at max_requests, before the input + output
// bytes pass max_batch_bytes (the first request is always taken), and before
// either part's block would exceed the budget, so that each part fits an
// empty arena and a batch can always start once the batches before it have
// finished. A single request must fit the budget (the submit check).
// Q is a sequence of requests with fields op (0 or 1), len and cap; ws(n)
// gives the kernel workspace bytes of a batch of n requests.
template <class Q, class Ws>
size_t plan_take(const Q& queue, size_t max_batch_bytes, size_t budget, size_t max_requests,
                 Ws ws) {
    size_t taken = 0, bytes = 0;
    size_t n[2] = {0, 0}, in[2] = {0, 0}, out[2] = {0, 0};
    while (taken < queue.size() && taken < max_requests) {
        const auto& r = queue[taken];
        const int op = r.op ? 1 : 0;
        const size_t add = r.len + r.cap;
        if (taken > 0 && bytes + add > max_batch_bytes) break;
        if (taken > 0 &&
            block_bytes(n[op] + 1, in[op] + r.len, out[op] + r.cap, ws(n[op] + 1)) > budget)
            break;
        bytes += add;
        n[op] += 1;
        in[op] += r.len;
        out[op] += r.cap;
        ++taken;
    }
    return taken;
}

}  // namespace b64serve

#endif  // B64_SERVE_PLAN_H
