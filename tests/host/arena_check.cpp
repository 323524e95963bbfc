// Randomised checks of the request server's host bookkeeping (arena.hpp):
// the first-fit arena allocator and the launch packing policy.  Built and run
// by tests/test_serve_host.py with g++; prints "ok" or the first violation.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <vector>

#include "arena.hpp"

#define CHECK(c, ...)                         \
  do {                                        \
    if (!(c)) {                               \
      std::printf("FAIL %s: ", #c);           \
      std::printf(__VA_ARGS__);               \
      std::printf("\n");                      \
      return 1;                               \
    }                                         \
  } while (0)

// Free and live blocks tile [0, capacity) exactly, free blocks never touch.
static int tiles(const locc::Arena& a) {
  std::map<size_t, size_t> all(a.free_blocks());
  for (const auto& kv : a.live_blocks()) {
    CHECK(!all.count(kv.first), "offset %zu both free and live", kv.first);
    all[kv.first] = kv.second;
  }
  size_t pos = 0;
  for (const auto& kv : all) {
    CHECK(kv.first == pos, "gap or overlap at %zu (block at %zu)", pos, kv.first);
    CHECK(kv.second > 0 && kv.second % 256 == 0, "block size %zu", kv.second);
    pos += kv.second;
  }
  CHECK(pos == a.capacity(), "covered %zu of %zu", pos, a.capacity());
  size_t prev_end = (size_t)-1;
  for (const auto& kv : a.free_blocks()) {
    CHECK(kv.first != prev_end, "adjacent free blocks at %zu not merged", kv.first);
    prev_end = kv.first + kv.second;
  }
  size_t used = 0;
  for (const auto& kv : a.live_blocks()) used += kv.second;
  CHECK(used == a.used(), "used %zu vs %zu", used, a.used());
  return 0;
}

static int arena_tests() {
  // exact fills, first fit, alignment, oversize
  locc::Arena a(4096 + 100, 256);
  CHECK(a.capacity() == 4096, "capacity rounds down to the alignment: %zu", a.capacity());
  size_t o1, o2, o3, o4;
  CHECK(a.alloc(1, &o1) && o1 == 0, "first block at 0");
  CHECK(a.alloc(256, &o2) && o2 == 256, "second at 256");
  CHECK(a.alloc(257, &o3) && o3 == 512, "third at 512 (512 bytes)");
  CHECK(a.used() == 1024, "used %zu", a.used());
  CHECK(!a.alloc(3073, &o4), "too large for the rest");
  CHECK(a.alloc(3072, &o4) && o4 == 1024, "exact fill");
  CHECK(a.largest_free() == 0 && !a.alloc(1, &o4), "full");
  CHECK(a.release(o2) && !a.release(o2), "double release refused");
  CHECK(a.alloc(200, &o2) && o2 == 256, "first fit reuses the hole");
  CHECK(!a.fits_empty(4097) && a.fits_empty(4096), "fits_empty");
  CHECK(a.release(0) && a.release(256) && a.release(512) && a.release(1024), "release all");
  CHECK(a.n_free_blocks() == 1 && a.largest_free() == 4096 && a.used() == 0, "merged back");
  CHECK(a.peak() == 4096, "peak %zu", a.peak());
  if (tiles(a)) return 1;

  // random alloc / release against a shadow model
  std::mt19937_64 rng(12345);
  locc::Arena b(1 << 20, 256);
  std::vector<size_t> live;
  for (int it = 0; it < 200000; ++it) {
    if (live.empty() || (rng() % 100) < 55) {
      const size_t want = 1 + rng() % 40000;
      size_t off;
      const bool ok = b.alloc(want, &off);
      if (ok) {
        CHECK(off % 256 == 0, "unaligned offset %zu", off);
        live.push_back(off);
      } else {
        CHECK(b.largest_free() < b.round(want), "alloc of %zu failed with a free block of %zu",
              want, b.largest_free());
      }
    } else {
      const size_t k = rng() % live.size();
      CHECK(b.release(live[k]), "release of live offset %zu", live[k]);
      live[k] = live.back();
      live.pop_back();
    }
    if (it % 997 == 0 && tiles(b)) return 1;
  }
  for (size_t o : live) CHECK(b.release(o), "final release %zu", o);
  CHECK(b.n_free_blocks() == 1 && b.used() == 0, "all merged after random run");
  return tiles(b);
}

static int pack_tests() {
  std::mt19937_64 rng(7);
  for (int it = 0; it < 100000; ++it) {
    const int n = 1 + (int)(rng() % 40);
    const int64_t cap = 1 + (int64_t)(rng() % 5000);
    std::vector<int64_t> rem(n), take(n);
    int64_t sum = 0;
    for (int i = 0; i < n; ++i) {
      rem[i] = (rng() % 4 == 0) ? (int64_t)(rng() % 20000) : (int64_t)(rng() % 300);
      sum += rem[i];
    }
    const int64_t tot = locc::pack_launch(rem.data(), n, cap, take.data());
    int64_t s = 0;
    for (int i = 0; i < n; ++i) {
      CHECK(take[i] >= 0 && take[i] <= rem[i], "take %lld of %lld", (long long)take[i],
            (long long)rem[i]);
      s += take[i];
    }
    CHECK(s == tot && tot == std::min(cap, sum), "total %lld, sum %lld, cap %lld",
          (long long)tot, (long long)sum, (long long)cap);
    // equal share: a request that got less than it had left got at least the
    // share, unless the launch is full
    const int64_t share = std::max<int64_t>(1, cap / n);
    for (int i = 0; i < n; ++i)
      if (take[i] < rem[i] && take[i] < share) CHECK(tot == cap, "request %d starved", i);
  }
  // a small request behind a large one finishes in the first launch
  int64_t rem[2] = {1000000, 100}, take[2];
  locc::pack_launch(rem, 2, 131072, take);
  CHECK(take[1] == 100 && take[0] == 131072 - 100, "small request packed: %lld %lld",
        (long long)take[0], (long long)take[1]);
  return 0;
}

int main() {
  if (arena_tests() || pack_tests()) return 1;
  std::printf("ok\n");
  return 0;
}
