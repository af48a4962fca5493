// Checks of the serving scheduler (arena admission and batch formation), host code only.
// Built and run by tests/test_serve_host.py; prints one line per failed check and exits 1 if any.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "serve_sched.h"

using rkm::serve::Arena;
using rkm::serve::batch_bytes;
using rkm::serve::take_batch;

static int failures = 0;
#define CHECK(cond)                                                          \
    do {                                                                     \
        if (!(cond)) {                                                       \
            std::printf("FAILED %s:%d: %s\n", __FILE__, __LINE__, #cond);    \
            ++failures;                                                      \
        }                                                                    \
    } while (0)

static void arena_basics() {
    Arena a(1000);  // rounds down to 768 = 3 granules
    CHECK(a.size() == 768);
    size_t o1, o2, o3, o4;
    CHECK(a.alloc(1, &o1) && o1 == 0);
    CHECK(a.alloc(256, &o2) && o2 == 256);
    CHECK(a.alloc(200, &o3) && o3 == 512);
    CHECK(!a.alloc(1, &o4));
    CHECK(a.in_use() == 768 && a.high_water() == 768);
    a.release(o2, 256);
    CHECK(a.largest_free() == 256);
    CHECK(!a.alloc(300, &o4));  // two granules needed, only one free
    a.release(o1, 1);           // merges with the freed middle granule
    CHECK(a.free_ranges() == 1 && a.largest_free() == 512);
    CHECK(a.alloc(300, &o4) && o4 == 0);
    a.release(o4, 300);
    a.release(o3, 200);
    CHECK(a.free_ranges() == 1 && a.largest_free() == 768 && a.in_use() == 0);
    CHECK(a.high_water() == 768);
}

// Random alloc/release against a byte map: ranges never overlap, accounting matches, and
// after releasing everything the arena is one free range again.
static void arena_random() {
    std::mt19937_64 rng(12345);
    const size_t size = 1 << 20;
    Arena a(size);
    std::vector<int> owner(size / 256, -1);
    std::vector<std::pair<size_t, size_t>> live;
    size_t used = 0;
    for (int step = 0; step < 20000; ++step) {
        if (live.empty() || rng() % 3 != 0) {
            const size_t b = 1 + rng() % 40000;
            size_t off;
            if (a.alloc(b, &off)) {
                const size_t g0 = off / 256, g1 = (off + rkm::serve::round_granule(b)) / 256;
                CHECK(off % 256 == 0 && g1 <= owner.size());
                for (size_t g = g0; g < g1 && g < owner.size(); ++g) {
                    CHECK(owner[g] == -1);
                    owner[g] = step;
                }
                live.push_back({off, b});
                used += rkm::serve::round_granule(b);
            } else {
                CHECK(a.largest_free() < rkm::serve::round_granule(b));
            }
        } else {
            const size_t j = rng() % live.size();
            const auto [off, b] = live[j];
            for (size_t g = off / 256; g < (off + rkm::serve::round_granule(b)) / 256; ++g) owner[g] = -1;
            a.release(off, b);
            used -= rkm::serve::round_granule(b);
            live[j] = live.back();
            live.pop_back();
        }
        CHECK(a.in_use() == used);
    }
    for (const auto& [off, b] : live) a.release(off, b);
    CHECK(a.in_use() == 0 && a.free_ranges() == 1 && a.largest_free() == a.size());
}

static void batches() {
    const int d = 100;
    std::vector<int64_t> q = {3000, 4000, 2000, 500, 4096};
    auto items_of = [&](size_t j) { return q[j]; };
    size_t off;
    int64_t items;
    // item limit: 3000 + 4000 fit 8192, adding 2000 would not
    Arena big(1ull << 30);
    CHECK(take_batch(q.size(), items_of, 8192, d, big, &off, &items) == 2 && items == 7000);
    CHECK(big.in_use() == batch_bytes(7000, d));
    // memory limit: only the oldest request fits
    Arena small(batch_bytes(3500, d));
    CHECK(take_batch(q.size(), items_of, 8192, d, small, &off, &items) == 1 && items == 3000);
    // nothing fits while that batch holds the memory; the oldest is not overtaken by a
    // smaller later request
    std::vector<int64_t> q2 = {3000, 10};
    auto items2 = [&](size_t j) { return q2[j]; };
    CHECK(take_batch(q2.size(), items2, 8192, d, small, &off, &items) == 0 && items == 0);
    small.release(0, batch_bytes(3000, d));
    CHECK(take_batch(q2.size(), items2, 8192, d, small, &off, &items) == 2 && items == 3010);
    // a request larger than the item limit is taken alone
    std::vector<int64_t> q3 = {9000, 1};
    auto items3 = [&](size_t j) { return q3[j]; };
    Arena a3(1ull << 30);
    CHECK(take_batch(q3.size(), items3, 8192, d, a3, &off, &items) == 1 && items == 9000);
    // empty queue
    CHECK(take_batch(0, items3, 8192, d, a3, &off, &items) == 0);
    // bytes: rows and counts each rounded to the granule
    CHECK(batch_bytes(1, 100) == 512 + 256);
    CHECK(batch_bytes(64, 1) == 256 + 256);
}

int main() {
    arena_basics();
    arena_random();
    batches();
    if (failures) return 1;
    std::printf("ok\n");
    return 0;
}
