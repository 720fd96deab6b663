// Unit test of the request server's first-fit free list (freelist.h)
// against a brute-force model: a bitmap of used units.  After every random
// take or give the list's runs must be exactly the maximal free runs of the
// bitmap, a take must return the start of the lowest free run that holds it,
// and largest()/fits() must agree with the bitmap.  Prints "ok" and exits 0.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <utility>
#include <vector>

#include "freelist.h"

template <class T>
static int check(const dbn::FreeList<T>& fl, const std::vector<char>& used, T unit, int step) {
  std::map<T, T> runs;
  const T n = (T)used.size();
  for (T a = 0; a < n;) {
    if (used[(size_t)a]) { ++a; continue; }
    T b = a;
    while (b < n && !used[(size_t)b]) ++b;
    runs[a * unit] = (b - a) * unit;
    a = b;
  }
  if (runs != fl.runs()) {
    std::printf("step %d: runs differ from the model\n", step);
    return 1;
  }
  T big = 0;
  for (const auto& kv : runs) big = kv.second > big ? kv.second : big;
  if (fl.largest() != big || !(fl.fits(big) || big == 0) || fl.fits(big + unit)) {
    std::printf("step %d: largest/fits wrong\n", step);
    return 1;
  }
  return 0;
}

template <class T>
static int run(T cap_units, T unit, unsigned seed, int steps) {
  std::mt19937 rng(seed);
  dbn::FreeList<T> fl;
  fl.reset(cap_units * unit);
  std::vector<char> used((size_t)cap_units, 0);
  std::vector<std::pair<T, T>> taken;  // (start unit, units)
  for (int s = 0; s < steps; ++s) {
    const bool do_take = taken.empty() || (rng() % 100) < 55;
    if (do_take) {
      const T n = 1 + (T)(rng() % (unsigned)(cap_units / 4));
      // the model's first fit: the lowest maximal free run of length >= n
      T want = -1;
      for (T a = 0; a < cap_units && want < 0;) {
        if (used[(size_t)a]) { ++a; continue; }
        T b = a;
        while (b < cap_units && !used[(size_t)b]) ++b;
        if (b - a >= n) want = a;
        a = b;
      }
      const T got = fl.take(n * unit);
      if ((want < 0 && got != T(-1)) || (want >= 0 && got != want * unit)) {
        std::printf("step %d: take(%lld) gave %lld, first fit is %lld\n", s, (long long)n,
                    (long long)got, (long long)want);
        return 1;
      }
      if (want >= 0) {
        for (T k = 0; k < n; ++k) used[(size_t)(want + k)] = 1;
        taken.push_back({want, n});
      }
    } else {
      const size_t k = rng() % taken.size();
      const auto r = taken[k];
      taken.erase(taken.begin() + (long)k);
      fl.give(r.first * unit, r.second * unit);
      for (T q = 0; q < r.second; ++q) used[(size_t)(r.first + q)] = 0;
    }
    if (check(fl, used, unit, s)) return 1;
  }
  // everything returned: one run again
  for (const auto& r : taken) fl.give(r.first * unit, r.second * unit);
  if (fl.runs().size() != 1 || fl.runs().begin()->first != 0 ||
      fl.runs().begin()->second != cap_units * unit) {
    std::printf("not one run after returning everything\n");
    return 1;
  }
  if (fl.take(0) != T(-1) || fl.fits(0)) {
    std::printf("zero-length requests must be refused\n");
    return 1;
  }
  return 0;
}

int main() {
  int bad = 0;
  for (unsigned seed = 1; seed <= 20; ++seed) {
    bad |= run<int32_t>(200, 1, seed, 3000);           // tiles, region slots
    bad |= run<int64_t>(300, 256, 100 + seed, 3000);   // arena byte offsets (256-byte granules)
  }
  if (bad) return 1;
  std::printf("ok\n");
  return 0;
}
