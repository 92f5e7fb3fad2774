// Host-side cache of the device address of one static __device__ array,
// kept per CUDA context.
//
// The address of a file-scope __device__ array belongs to the module copy
// loaded into one context.  A device reset (cudaDeviceReset) or a second
// context on the same device (cuCtxCreate) loads the module again at another
// address, so an address cached per device ordinal can go stale.  This cache
// is keyed on the context's process-unique id (cuCtxGetId; ids are never
// reused within a process, unlike context handles), so a new context always
// triggers a fresh lookup.  A failed lookup is not cached.
//
// Plain C++ with no CUDA types: the lookup is passed in, which lets the
// cache be checked on a machine without a GPU.
#pragma once

#include <functional>
#include <mutex>
#include <vector>

namespace rteom {

class ContextAddressCache {
 public:
  // Address for the context with id ctx_id: the cached one, or the result
  // of lookup(&addr) (0 = success), stored on success.  Returns lookup's
  // error code on failure.  Thread-safe.
  int get(unsigned long long ctx_id, const std::function<int(void**)>& lookup, void** out) {
    std::lock_guard<std::mutex> lk(mu_);
    for (const Entry& e : entries_)
      if (e.ctx_id == ctx_id) {
        *out = e.addr;
        return 0;
      }
    void* addr = nullptr;
    const int rc = lookup(&addr);
    if (rc != 0) return rc;
    entries_.push_back({ctx_id, addr});
    *out = addr;
    return 0;
  }
  size_t size() {
    std::lock_guard<std::mutex> lk(mu_);
    return entries_.size();
  }

 private:
  struct Entry {
    unsigned long long ctx_id;
    void* addr;
  };
  std::mutex mu_;
  std::vector<Entry> entries_;
};

}  // namespace rteom
