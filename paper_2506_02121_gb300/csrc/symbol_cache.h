// Cache of a __device__ symbol's address, keyed by the CUDA context it was looked up in.
//
// A device symbol's address belongs to the module loaded in one context.  After the
// primary context of a device is reset (cudaDeviceReset, or a context destroyed and made
// again) the module is loaded anew and the symbol may sit elsewhere, so an address cached
// per device index could point into memory that is no longer the symbol.  The key here is
// the context's ID (cuCtxGetId), which the driver never reuses within a process: a new
// context misses the cache and the address is looked up again.
//
// Plain C++ (no CUDA types), so that the host logic can be compiled and tested without a
// GPU.
#pragma once

#include <mutex>

namespace ccg {

template <int kSlots>
class SymbolAddressCache {
  public:
    // Address for context ctx_id: the cached one, else lookup(&addr) (returns 0 on success)
    // is called once and its result kept.  Returns lookup's error code, or 0.
    template <typename Lookup>
    int get(unsigned long long ctx_id, Lookup lookup, void** out) {
        std::lock_guard<std::mutex> lk(mu_);
        for (int i = 0; i < used_; i++)
            if (slot_[i].ctx == ctx_id) {
                *out = slot_[i].addr;
                return 0;
            }
        void* addr = nullptr;
        const int err = lookup(&addr);
        if (err) return err;
        // a full table replaces its entries in turn (contexts of earlier resets are dead)
        const int i = used_ < kSlots ? used_++ : (next_++ % kSlots);
        slot_[i].ctx = ctx_id;
        slot_[i].addr = addr;
        *out = addr;
        return 0;
    }

    int size() {
        std::lock_guard<std::mutex> lk(mu_);
        return used_;
    }

  private:
    struct Slot {
        unsigned long long ctx;
        void* addr;
    };
    std::mutex mu_;
    Slot slot_[kSlots] = {};
    int used_ = 0;
    unsigned next_ = 0;
};

}  // namespace ccg
