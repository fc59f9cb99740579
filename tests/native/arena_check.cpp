// Randomised check of fp::Arena (the request server's allocator) against a
// plain bitmap model of [0, capacity): every allocation must land where
// first fit in offset order over the model's maximal free runs puts it,
// allocations never overlap, the free list stays sorted, disjoint and
// merged, and releasing everything restores one range.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "../../paper_2101_11408_gb300/csrc/fp_arena.h"

static int fail(const char* what, int step) {
  std::printf("FAIL %s at step %d\n", what, step);
  return 1;
}

int main(int argc, char** argv) {
  const uint64_t cap = argc > 1 ? std::strtoull(argv[1], nullptr, 10) : 4096;
  const int steps = argc > 2 ? std::atoi(argv[2]) : 200000;
  std::mt19937_64 rng(argc > 3 ? std::strtoull(argv[3], nullptr, 10) : 1);
  fp::Arena a(cap);
  std::vector<char> used(cap, 0);
  struct Live { uint64_t off, n; };
  std::vector<Live> live;
  for (int step = 0; step < steps; step++) {
    const bool do_alloc = live.empty() || (rng() % 100) < 55;
    if (do_alloc) {
      // sizes: mostly small, sometimes large, sometimes larger than anything free
      uint64_t n = 1 + rng() % (rng() % 8 == 0 ? cap : 64);
      // model: first maximal free run of length >= n
      uint64_t expect = UINT64_MAX;
      for (uint64_t i = 0; i < cap;) {
        if (used[i]) { i++; continue; }
        uint64_t j = i;
        while (j < cap && !used[j]) j++;
        if (j - i >= n) { expect = i; break; }
        i = j;
      }
      uint64_t off = 0;
      const bool ok = a.alloc(n, &off);
      if (ok != (expect != UINT64_MAX)) return fail("alloc success", step);
      if (ok) {
        if (off != expect) return fail("first-fit offset", step);
        for (uint64_t k = off; k < off + n; k++) {
          if (used[k]) return fail("overlap", step);
          used[k] = 1;
        }
        live.push_back({off, n});
      }
    } else {
      const size_t i = rng() % live.size();
      const Live l = live[i];
      live[i] = live.back();
      live.pop_back();
      a.release(l.off, l.n);
      for (uint64_t k = l.off; k < l.off + l.n; k++) used[k] = 0;
    }
    // free list == model's maximal free runs, in order
    uint64_t free_count = 0;
    for (uint64_t k = 0; k < cap; k++) free_count += !used[k];
    if (a.free_units() != free_count) return fail("free units", step);
    uint64_t pos = 0;
    bool bad = false;
    a.for_each_free([&](uint64_t o, uint64_t n) {
      if (bad) return;
      while (pos < cap && used[pos]) pos++;
      uint64_t end = pos;
      while (end < cap && !used[end]) end++;
      if (o != pos || n != end - pos) bad = true;
      pos = end;
    });
    while (!bad && pos < cap && used[pos]) pos++;
    if (bad || pos != cap) return fail("free list shape", step);
  }
  for (const Live& l : live) a.release(l.off, l.n);
  if (a.fragments() != 1 || a.free_units() != cap || a.largest_free() != cap)
    return fail("restore", steps);
  uint64_t off = 7;
  if (a.alloc(0, &off) || a.alloc(cap + 1, &off)) return fail("degenerate sizes", steps);
  std::printf("ok %llu %d\n", (unsigned long long)cap, steps);
  return 0;
}
