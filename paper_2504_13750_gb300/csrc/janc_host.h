// Host-side logic of the serving loop and of the AMR driver, kept free of
// CUDA so that it runs (and is unit-tested) on a machine without a GPU:
//
//  * Pool: the first-fit allocator over one device memory pool from which
//    the server gives every admitted request its piece;
//  * admission_pass: one pass of the server's admission over its FIFO queue
//    (arrival order with skip-ahead, slot count, cell budget with aging);
#pragma once

#include <cstddef>
#include <deque>
#include <iterator>
#include <map>
#include <vector>

namespace janc {
namespace host {

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// First-fit allocator over [0, size) in 256-byte units; free blocks are kept
// by offset and merged with their neighbours on release.
struct Pool {
  size_t size = 0, used = 0;
  std::map<size_t, size_t> free_;
  void init(size_t s) {
    size = s & ~size_t(255);
    used = 0;
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(size_t n, size_t* off) {
    n = align256(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, o2 = it->first + n;
        free_.erase(it);
        if (rest) free_[o2] = rest;
        used += n;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = align256(n);
    used -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// What the admission pass needs to know of a queued request.
struct Pending {
  long long cells;   // cells of its grid
  size_t footprint;  // device bytes it needs from the pool
  double t_submit;   // arrival time, s
};

// One admission pass over `queue` (request ids in arrival order). For each
// entry in order:
//  - stop when the active set has max_active requests;
//  - with a cell budget, a request that would take the active set over it
//    waits (unless the active set is empty); requests behind it may pass it
//    until it has waited max_skip_s, after which the pass stops, so that the
//    active set drains for it;
//  - otherwise take its footprint from the pool: on success call
//    admit(id, offset), which returns true if the request became active (the
//    caller then counts it in n_active() and active_cells()) and false if it
//    failed, in which case its piece goes back to the pool; either way it
//    leaves the queue. A request the pool cannot hold stays queued and the
//    pass goes on to the next (skip-ahead).
template <class PendingOf, class NActive, class ActiveCells, class Admit>
void admission_pass(std::deque<int>& queue, Pool& pool, int max_active, long long cell_budget, double max_skip_s,
                    double now, PendingOf pending, NActive n_active, ActiveCells active_cells, Admit admit) {
  for (auto it = queue.begin(); it != queue.end();) {
    if (n_active() >= max_active) break;
    const Pending r = pending(*it);
    if (cell_budget > 0 && n_active() > 0 && active_cells() + r.cells > cell_budget) {
      if (now - r.t_submit >= max_skip_s) break;
      ++it;
      continue;
    }
    size_t off;
    if (pool.alloc(r.footprint, &off)) {
      if (!admit(*it, off)) pool.release(off, r.footprint);
      it = queue.erase(it);
    } else {
      ++it;
    }
  }
}

// Neighbour codes of a block side: a block number, or one of these.
constexpr int NB_EXTERNAL = -1;  // no block there: the layer's external boundary (Sec. 3.1.3)
constexpr int NB_PHYSICAL = -2;  // the side lies on the domain's wall or zero-gradient boundary
constexpr int BC_PERIODIC_CODE = 2;

}  // namespace host
}  // namespace janc
