// Per-CUDA-context memo of a device address, for the allocation-free entry
// point's scratch array.  Plain C++ with no CUDA types, so that its policy
// can be compiled and checked on a host without a GPU.
//
// A file-scope __device__ array has one address per context that loads the
// library's module: a host application may create its own driver contexts,
// and a context destroyed (cudaDeviceReset) and created again may load the
// module at another address.  So the address is looked up afresh on every
// call that is not being captured into a CUDA graph (the lookup is a cheap
// runtime query) and remembered per context; a call under stream capture
// uses the remembered address of the current context and fails cleanly if
// that context has none yet.
#pragma once

#include <mutex>

namespace sht {

template <int CAP>
class ContextAddressCache {
public:
    // Remember addr for ctx, replacing ctx's previous address; when full,
    // the oldest entry makes room.
    void put(const void* ctx, void* addr) {
        std::lock_guard<std::mutex> lk(mu_);
        for (int i = 0; i < n_; ++i) {
            if (e_[i].ctx == ctx) {
                e_[i].addr = addr;
                return;
            }
        }
        if (n_ < CAP) {
            e_[n_++] = {ctx, addr};
        } else {
            e_[next_] = {ctx, addr};
            next_ = (next_ + 1) % CAP;
        }
    }

    // The remembered address of ctx, or nullptr.
    void* get(const void* ctx) const {
        std::lock_guard<std::mutex> lk(mu_);
        for (int i = 0; i < n_; ++i)
            if (e_[i].ctx == ctx) return e_[i].addr;
        return nullptr;
    }

private:
    struct Entry {
        const void* ctx;
        void* addr;
    };
    Entry e_[CAP] = {};
    int n_ = 0;
    int next_ = 0;
    mutable std::mutex mu_;
};

enum ScratchLookup { kScratchOk = 0, kScratchLookupFailed = 1, kScratchNeedsSetup = 2 };

// The scratch address for the current context `ctx`.  Not capturing:
// lookup(&addr) queries the runtime (returning nonzero on failure), and
// the result is remembered.  Capturing: the remembered address, or
// kScratchNeedsSetup if this context has made no uncaptured call yet.
template <int CAP, class Lookup>
int scratch_for_context(ContextAddressCache<CAP>& cache, const void* ctx, bool capturing,
                        Lookup lookup, void** out) {
    if (capturing) {
        void* a = cache.get(ctx);
        if (!a) return kScratchNeedsSetup;
        *out = a;
        return kScratchOk;
    }
    void* a = nullptr;
    if (lookup(&a) != 0 || !a) return kScratchLookupFailed;
    cache.put(ctx, a);
    *out = a;
    return kScratchOk;
}

}  // namespace sht
