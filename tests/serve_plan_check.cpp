// Checks of the serving engine's host-only planning (b64_serve_plan.h):
// the arena ring never hands out overlapping or out-of-range blocks, and the
// batch planner never builds a part that could not fit an empty arena, so a
// queue always drains. Built and run by tests/test_serve_plan.py; prints the
// failed check and exits non-zero on the first failure.
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <map>
#include <random>
#include <vector>

#include "b64_serve_plan.h"

using namespace b64serve;

#define CHECK(cond)                                                         \
    do {                                                                    \
        if (!(cond)) {                                                      \
            std::fprintf(stderr, "%s:%d: check failed: %s\n", __FILE__,     \
                         __LINE__, #cond);                                  \
            std::exit(1);                                                   \
        }                                                                   \
    } while (0)

struct Req {
    int op;
    size_t len, cap;
};

static size_t ws(size_t n) { return 8 * n; }

static void ring_full_after_wrap() {
    Ring r(1024);
    size_t at = 1;
    CHECK(r.reserve(256, &at) && at == 0);
    CHECK(r.reserve(256, &at) && at == 256);
    r.release_front();                        // oldest block now starts at 256
    CHECK(r.reserve(256, &at) && at == 512);
    CHECK(r.reserve(256, &at) && at == 768);
    CHECK(r.reserve(256, &at) && at == 0);    // wraps; ends where the oldest starts
    CHECK(!r.reserve(256, &at));              // full
    CHECK(!r.reserve(1, &at));
    r.release_back();                         // the newest block taken back
    CHECK(r.reserve(256, &at) && at == 0);
    CHECK(!r.reserve(2048, &at));
}

static void ring_random_never_overlaps() {
    std::mt19937_64 g(5);
    const size_t cap = 1 << 16;
    Ring r(cap);
    std::deque<std::pair<size_t, size_t>> live;   // in reservation order
    for (int step = 0; step < 200000; ++step) {
        const unsigned roll = unsigned(g() % 100);
        if (!live.empty() && roll < 40) {
            r.release_front();
            live.pop_front();
            continue;
        }
        if (!live.empty() && roll < 43) {
            r.release_back();
            live.pop_back();
            continue;
        }
        const size_t size = align_up(1 + g() % (cap / 3));
        size_t at = 0;
        if (!r.reserve(size, &at)) continue;
        CHECK(at + size <= cap);
        for (const auto& b : live) CHECK(at + size <= b.first || b.first + b.second <= at);
        live.emplace_back(at, size);
        CHECK(r.blocks() == live.size());
    }
}

static void block_layout() {
    CHECK(meta_bytes(1) == 256);
    CHECK(block_bytes(1, 1, 4, ws(1)) == 5 * 256);
    CHECK(block_bytes(100, 1000, 1336, ws(100)) ==
          align_up(2 * 101 * 8 + 100) + 1024 + 1536 + 1024 + 1024);
}

// Simulates the engine: one stream, batches planned from the queue front,
// each op part reserved as one block, parts completing in order.
static void plan_drains_queue(size_t budget, size_t max_batch, std::mt19937_64& g) {
    std::deque<Req> q;
    for (int i = 0; i < 3000; ++i) {
        const int op = int(g() % 2);
        size_t len = 1 + g() % 4096;
        if (g() % 50 == 0) len = 1 + g() % (budget / 4);
        if (op == 1) len = (len + 3) / 4 * 4;
        const size_t cap = op == 0 ? (len + 2) / 3 * 4 : len / 4 * 3;
        if (block_bytes(1, len, cap, ws(1)) > budget) continue;   // refused at submit
        q.push_back({op, len, cap});
    }
    Ring ring(budget);
    std::deque<size_t> inflight;  // parts in reservation order
    int idle_polls = 0;
    while (!q.empty()) {
        const size_t take = plan_take(q, max_batch, budget, 16384, ws);
        CHECK(take >= 1 && take <= q.size());
        size_t n[2] = {0, 0}, in[2] = {0, 0}, out[2] = {0, 0}, bytes = 0;
        for (size_t k = 0; k < take; ++k) {
            n[q[k].op] += 1;
            in[q[k].op] += q[k].len;
            out[q[k].op] += q[k].cap;
            bytes += q[k].len + q[k].cap;
        }
        CHECK(take == 1 || bytes <= max_batch);
        bool sent[2] = {false, false};
        for (int op = 0; op < 2; ++op) {
            if (!n[op]) continue;
            const size_t b = block_bytes(n[op], in[op], out[op], ws(n[op]));
            CHECK(b <= budget);   // every part fits an empty arena
            size_t at = 0;
            if (!ring.reserve(b, &at)) break;
            inflight.push_back(b);
            sent[op] = true;
        }
        if (sent[0] || sent[1]) {
            std::deque<Req> rest;
            for (size_t k = 0; k < q.size(); ++k)
                if (!(k < take && sent[q[k].op])) rest.push_back(q[k]);
            q.swap(rest);
            idle_polls = 0;
        } else {
            CHECK(!inflight.empty());   // nothing fits only while work is in flight
            ++idle_polls;
        }
        // the oldest part completes
        if (!inflight.empty() && (g() % 2 == 0 || !(sent[0] || sent[1]))) {
            ring.release_front();
            inflight.pop_front();
        }
        CHECK(idle_polls < 1000);
    }
}

int main() {
    ring_full_after_wrap();
    ring_random_never_overlaps();
    block_layout();
    std::mt19937_64 g(11);
    // a batch cap far above the budget, and one below it
    plan_drains_queue(size_t(1) << 20, size_t(64) << 20, g);
    plan_drains_queue(size_t(4) << 20, size_t(64) << 20, g);
    plan_drains_queue(size_t(4) << 20, size_t(256) << 10, g);
    // many tiny requests: the per-request sections bound the batch
    {
        // about 38 bytes of block a request: 256 KiB holds fewer than 16384
        std::deque<Req> q(20000, Req{0, 1, 4});
        const size_t budget = size_t(256) << 10;
        const size_t take = plan_take(q, size_t(64) << 20, budget, 16384, ws);
        CHECK(take > 1000 && take < 16384);
        CHECK(block_bytes(take, take, 4 * take, ws(take)) <= budget);
        CHECK(block_bytes(take + 1, take + 1, 4 * (take + 1), ws(take + 1)) > budget);
    }
    std::puts("serve plan checks passed");
    return 0;
}
