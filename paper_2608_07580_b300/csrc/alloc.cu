// alloc.cu — the library's device allocations, optionally through a
// caller-supplied allocator (fire_set_allocator). Each block remembers the
// allocator that made it, so it is returned to that one even if the hook
// changes in between.
#include <mutex>
#include <unordered_map>

#include "../../include/firert.h"
#include "internal.cuh"

namespace {

struct Hook {
  fire_alloc_fn alloc = nullptr;
  fire_free_fn free = nullptr;
  void *user = nullptr;
};

std::mutex g_mu;
Hook g_hook;
// blocks made by a caller's allocator, with the free function to return them to
std::unordered_map<void *, Hook> g_owned;

}  // namespace

namespace firert {

cudaError_t dev_malloc(void **p, size_t bytes) {
  Hook h;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    h = g_hook;
  }
  if (!h.alloc) return cudaMalloc(p, bytes);
  void *q = h.alloc(bytes, h.user);
  if (!q) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_owned[q] = h;
  }
  *p = q;
  return cudaSuccess;
}

void dev_free(void *p) {
  if (!p) return;
  Hook h;
  bool mine = false;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_owned.find(p);
    if (it != g_owned.end()) {
      h = it->second;
      mine = true;
      g_owned.erase(it);
    }
  }
  if (mine) {
    if (h.free) h.free(p, h.user);
  } else {
    cudaFree(p);
  }
}

}  // namespace firert

extern "C" void fire_set_allocator(fire_alloc_fn alloc, fire_free_fn free_fn, void *user) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_hook.alloc = alloc;
  g_hook.free = alloc ? free_fn : nullptr;
  g_hook.user = alloc ? user : nullptr;
}
