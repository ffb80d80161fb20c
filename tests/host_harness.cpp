// Test harness: the GPU-free host logic of the library (janc_host.h: the
// serving pool and admission pass, the AMR block lists) behind a C ABI, so
// that the CPU tests can drive it through ctypes. Built by the tests with
// the host C++ compiler; not part of the library.
#include <cstring>
#include <deque>
#include <vector>

#include "../paper_2504_13750_gb300/csrc/janc_host.h"

using namespace janc::host;

extern "C" {

// A pool of `size` bytes driven by nops operations: op > 0 allocates op
// bytes (out[i] = offset, or -1 when nothing fits); op = -(j + 1) releases
// the allocation made by operation j, if it succeeded (out[i] = 0). At the
// end *used holds the bytes in use and free_off/free_len (capacity
// max_free) the free blocks in offset order; returns their number.
int hh_pool(long long size, const long long* op, int nops, long long* out, long long* used, long long* free_off,
            long long* free_len, int max_free) {
  Pool p;
  p.init((size_t)size);
  std::vector<long long> sz((size_t)nops, 0);
  for (int i = 0; i < nops; ++i) {
    if (op[i] > 0) {
      size_t off;
      if (p.alloc((size_t)op[i], &off)) {
        out[i] = (long long)off;
        sz[i] = op[i];
      } else {
        out[i] = -1;
      }
    } else {
      const int j = (int)(-op[i] - 1);
      if (out[j] >= 0) p.release((size_t)out[j], (size_t)sz[j]);  // a failed allocation holds nothing
      out[i] = 0;
    }
  }
  *used = (long long)p.used;
  int k = 0;
  for (const auto& f : p.free_) {
    if (k < max_free) {
      free_off[k] = (long long)f.first;
      free_len[k] = (long long)f.second;
    }
    ++k;
  }
  return k;
}

// One admission pass over requests 0..n-1 queued in that order, with
// n_active0 requests already active holding cells0 cells and the first
// pool_used0 bytes of a pool of pool_size bytes. fail[i] != 0 makes the
// admission of request i fail. Writes the admitted ids in admission order
// to out (returns their number) and the ids left queued to left (*nleft);
// *pool_used gets the pool's bytes in use after the pass.
int hh_admission(int n, const long long* cells, const long long* fp, const double* t_submit, const int* fail,
                 long long pool_size, int max_active, long long cell_budget, double max_skip_s, double now,
                 int n_active0, long long cells0, long long pool_used0, int* out, int* left, int* nleft,
                 long long* pool_used) {
  Pool pool;
  pool.init((size_t)pool_size);
  size_t off0;
  if (pool_used0 > 0 && !pool.alloc((size_t)pool_used0, &off0)) return -1;
  std::deque<int> queue;
  for (int i = 0; i < n; ++i) queue.push_back(i);
  int n_active = n_active0;
  long long active_cells = cells0;
  int na = 0;
  admission_pass(
      queue, pool, max_active, cell_budget, max_skip_s, now,
      [&](int id) { return Pending{cells[id], (size_t)fp[id], t_submit[id]}; }, [&] { return n_active; },
      [&] { return active_cells; },
      [&](int id, size_t) {
        if (fail[id]) return false;
        out[na++] = id;
        ++n_active;
        active_cells += cells[id];
        return true;
      });
  *nleft = (int)queue.size();
  int k = 0;
  for (int id : queue) left[k++] = id;
  *pool_used = (long long)pool.used;
  return na;
}


}  // extern "C"
