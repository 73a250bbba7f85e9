// Host-only checks of the request server's scheduling pieces (tfn_sched.h):
// the ring arena against a brute-force model of live blocks, and the
// admission rule inside a simulated continuous-batching loop.  Prints "ok"
// and exits 0 on success; prints the failed check and exits 1 otherwise.
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <random>
#include <vector>

#include "tfn_sched.h"

using tfn::RingArena;

#define CHECK(c)                                                    \
    do {                                                            \
        if (!(c)) {                                                 \
            std::printf("FAILED %s at line %d\n", #c, __LINE__);    \
            std::exit(1);                                           \
        }                                                           \
    } while (0)

struct Live {
    size_t off, size;
};

// Every live block in range, aligned, disjoint from every other; in_use is the sum.
static void check_blocks(const RingArena &a, const std::deque<Live> &live, size_t align)
{
    size_t sum = 0;
    for (size_t i = 0; i < live.size(); ++i) {
        CHECK(live[i].off % align == 0 && live[i].size % align == 0 && live[i].size > 0);
        CHECK(live[i].off + live[i].size <= a.capacity());
        for (size_t j = i + 1; j < live.size(); ++j)
            CHECK(live[i].off + live[i].size <= live[j].off || live[j].off + live[j].size <= live[i].off);
        sum += live[i].size;
    }
    CHECK(sum == a.in_use());
    CHECK(live.size() == a.live_blocks());
}

static void test_ring_random(unsigned seed, size_t cap, size_t align, size_t max_req)
{
    std::mt19937_64 rng(seed);
    RingArena a(cap, align);
    std::deque<Live> live;
    for (int step = 0; step < 200000; ++step) {
        const bool do_alloc = live.empty() || (rng() % 100) < 55;
        if (do_alloc) {
            const size_t want = 1 + rng() % max_req;
            const size_t fit = a.largest_fit();
            const size_t off = a.alloc(want);
            if (a.round(want) <= fit) {
                CHECK(off != RingArena::kNone);  // largest_fit() is a promise
                live.push_back({off, a.round(want)});
            } else {
                CHECK(off == RingArena::kNone);  // and a bound
            }
        } else {
            a.free_oldest();
            live.pop_front();
        }
        if (step % 97 == 0) check_blocks(a, live, align);
    }
    while (!live.empty()) {
        a.free_oldest();
        live.pop_front();
    }
    CHECK(a.in_use() == 0 && a.largest_fit() == a.capacity());
}

static void test_ring_cases()
{
    RingArena a(1000, 100);  // capacity rounds down to 1000
    CHECK(a.capacity() == 1000);
    CHECK(a.alloc(0) == RingArena::kNone);     // nothing to stage: no block
    CHECK(a.alloc(1001) == RingArena::kNone);  // larger than the ring
    CHECK(a.alloc(1000) == 0);                 // exactly the ring
    CHECK(a.largest_fit() == 0 && a.alloc(1) == RingArena::kNone);
    a.free_oldest();
    CHECK(a.alloc(300) == 0 && a.alloc(300) == 300 && a.alloc(300) == 600);  // [0,300) [300,600) [600,900)
    CHECK(a.largest_fit() == 100);
    a.free_oldest();                         // frees [0,300): runs [900,1000) and [0,300)
    CHECK(a.largest_fit() == 300);
    CHECK(a.alloc(200) == 0);                // wraps: [900,1000) left unused
    CHECK(a.largest_fit() == 100);           // [200,300)
    CHECK(a.alloc(150) == RingArena::kNone);
    a.free_oldest();                         // [300,600) released: [200,600) free
    CHECK(a.largest_fit() == 400);
    a.free_oldest();                         // [600,900) released: only [0,200) live, the tail end is whole again
    CHECK(a.largest_fit() == 800 && a.alloc(800) == 200);
    a.free_oldest();
    a.free_oldest();
    CHECK(a.live_blocks() == 0 && a.in_use() == 0);
}

struct Req {
    int id;
    size_t bytes;
};

static void test_admission()
{
    std::deque<Req> q = {{0, 100}, {1, 200}, {2, 50}, {3, 10}};
    auto by = [](const Req &r) { return r.bytes; };
    size_t tot = 0;
    CHECK(tfn::admit_count(q, 8, 1000, by, &tot) == 4 && tot == 360);
    CHECK(tfn::admit_count(q, 2, 1000, by, &tot) == 2 && tot == 300);  // batch limit
    CHECK(tfn::admit_count(q, 8, 299, by, &tot) == 1 && tot == 100);   // request 1 does not fit: stop (no overtaking)
    CHECK(tfn::admit_count(q, 8, 99, by, &tot) == 0 && tot == 0);
    std::deque<Req> z = {{0, 0}, {1, 0}, {2, 500}};
    CHECK(tfn::admit_count(z, 8, 0, by, &tot) == 2 && tot == 0);  // device-buffer requests need no staging
}

// Simulated server: random arrivals, P pipelines, batches retire in launch
// order after a random delay.  Checks: every request completes, in arrival
// order of admission, staging never exceeds the budget, no batch exceeds the
// batch limit.
static void test_serving_simulation(unsigned seed)
{
    std::mt19937_64 rng(seed);
    const size_t budget = 64 << 20, max_batch = 16;
    const int pipes = 2, nreq = 20000;
    RingArena a(budget, 256);
    std::deque<Req> q;
    struct B {
        std::vector<int> ids;
        bool block;
        int ready;
    };
    std::deque<B> inflight;
    int next_id = 0, next_admit = 0, done = 0, t = 0;
    while (done < nreq) {
        ++t;
        // arrivals
        const int arrivals = (int)(rng() % 4);
        for (int k = 0; k < arrivals && next_id < nreq; ++k) {
            const size_t sizes[4] = {240 * 320 * 17, 480 * 640 * 17, 720 * 1280 * 17, 1080 * 1920 * 17};
            const bool device = rng() % 5 == 0;
            q.push_back({next_id++, device ? 0 : a.round(sizes[rng() % 4])});
        }
        // retire the oldest batch when its time has come
        if (!inflight.empty() && inflight.front().ready <= t) {
            if (inflight.front().block) a.free_oldest();
            done += (int)inflight.front().ids.size();
            inflight.pop_front();
        }
        // launch while a pipeline is free and something is admissible
        while ((int)inflight.size() < pipes && !q.empty()) {
            size_t bytes = 0;
            const size_t k = tfn::admit_count(q, max_batch, a.largest_fit(), [](const Req &r) { return r.bytes; },
                                              &bytes);
            if (k == 0) {
                CHECK(!inflight.empty());  // with nothing in flight the head always fits
                break;
            }
            CHECK(k <= max_batch);
            B b;
            b.block = bytes > 0;
            if (b.block) CHECK(a.alloc(bytes) != RingArena::kNone);
            CHECK(a.in_use() <= budget);
            for (size_t i = 0; i < k; ++i) {
                CHECK(q.front().id == next_admit);  // FIFO admission
                ++next_admit;
                b.ids.push_back(q.front().id);
                q.pop_front();
            }
            b.ready = t + 1 + (int)(rng() % 5);
            inflight.push_back(b);
        }
        CHECK(t < 100 * nreq);  // progress
    }
    CHECK(next_admit == nreq && a.in_use() == 0);
}

int main()
{
    test_ring_cases();
    test_ring_random(1, 1 << 20, 256, 300000);
    test_ring_random(2, 10000, 16, 9000);
    test_ring_random(3, 4096, 1, 64);
    test_admission();
    test_serving_simulation(7);
    test_serving_simulation(8);
    std::printf("ok\n");
    return 0;
}
