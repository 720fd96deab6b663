// First-fit free list over a range of integer units, with neighbouring free
// runs merged on release.  The request server keeps its neuron tiles and
// region slots in one each, and its device arena keeps byte offsets in one.
// Host code only (no CUDA); not thread-safe.
#pragma once

#include <iterator>
#include <map>

namespace dbn {

template <class T>
class FreeList {
 public:
  // Everything free: one run [0, n).
  void reset(T n) {
    free_.clear();
    if (n > 0) free_[0] = n;
  }

  // Take n >= 1 units from the lowest free run that holds them; returns the
  // start of the taken range, or -1 when no run is long enough.
  T take(T n) {
    if (n <= 0) return T(-1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const T at = it->first, len = it->second;
      free_.erase(it);
      if (len > n) free_[at + n] = len - n;
      return at;
    }
    return T(-1);
  }

  bool fits(T n) const { return n > 0 && largest() >= n; }

  // Return [at, at + n), merging it with the free runs it touches.  The
  // range must have been taken and not yet returned.
  void give(T at, T n) {
    if (n <= 0) return;
    auto nx = free_.lower_bound(at);
    if (nx != free_.end() && at + n == nx->first) {
      n += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == at) {
        pv->second += n;
        return;
      }
    }
    free_[at] = n;
  }

  T largest() const {
    T m = 0;
    for (const auto& kv : free_) m = kv.second > m ? kv.second : m;
    return m;
  }

  // The free runs, start -> length, in address order.
  const std::map<T, T>& runs() const { return free_; }

 private:
  std::map<T, T> free_;
};

}  // namespace dbn
