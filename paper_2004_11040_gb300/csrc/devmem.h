// devmem.h -- the library's cache of device allocations (host code only).
//
// Creating a context used to cost a handful of cudaMalloc calls (its pool of
// arrays, the persistent launch's control arrays, the export scratch) and
// destroying it as many cudaFree calls: driver calls of tens to hundreds of
// microseconds each, the largest part of the host time of a short run. Here a
// released block is kept and handed to the next request of about its size:
// at least the size asked for, at most an eighth (plus 64 KiB) more, so a
// cached block never wastes much. The cache holds at most `limit` bytes;
// beyond that the least recently released blocks go back to the device.
// When the backend cannot allocate, every cached block is freed and the
// allocation is tried once more.
//
// The policy is generic over its backend so that it can be checked on the
// host: Backend has `int alloc(void **p, size_t bytes)` (0 on success, an
// error code otherwise) and `void free(void *p)`. All members take one mutex.
#pragma once

#include <cstddef>
#include <cstdint>
#include <list>
#include <mutex>
#include <unordered_map>

struct DevCacheInfo {
    int64_t cached_bytes;  // released blocks held for reuse
    int64_t in_use_bytes;  // blocks handed out and not released
    int64_t hits;          // requests served from the cache
    int64_t misses;        // requests that went to the backend
};

template <class Backend>
class BlockCache {
public:
    explicit BlockCache(size_t limit, Backend be = Backend()) : be_(be), limit_(limit) {}
    ~BlockCache() { trim(); }

    // A block of at least `bytes` (1 if 0) in *p; 0, or the backend's error.
    int acquire(void **p, size_t bytes) {
        if (!p) return -1;
        *p = nullptr;
        if (bytes == 0) bytes = 1;
        std::lock_guard<std::mutex> lock(mu_);
        auto best = free_.end();
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (fits(it->size, bytes) && (best == free_.end() || it->size < best->size)) best = it;
        if (best != free_.end()) {
            *p = best->ptr;
            in_use_[best->ptr] = best->size;
            in_use_bytes_ += best->size;
            cached_ -= best->size;
            free_.erase(best);
            ++hits_;
            return 0;
        }
        ++misses_;
        int rc = be_.alloc(p, bytes);
        if (rc != 0 && !free_.empty()) {
            drop_all();
            rc = be_.alloc(p, bytes);
        }
        if (rc != 0) {
            *p = nullptr;
            return rc;
        }
        in_use_[*p] = bytes;
        in_use_bytes_ += bytes;
        return 0;
    }

    // Gives a block back (null: nothing). A pointer this cache did not hand
    // out goes to the backend directly.
    void release(void *p) {
        if (!p) return;
        std::lock_guard<std::mutex> lock(mu_);
        auto it = in_use_.find(p);
        if (it == in_use_.end()) {
            be_.free(p);
            return;
        }
        const size_t size = it->second;
        in_use_.erase(it);
        in_use_bytes_ -= size;
        if (size > limit_) {
            be_.free(p);
            return;
        }
        free_.push_front(Block{p, size});
        cached_ += size;
        shrink_to(limit_);
    }

    // Bounds the cached bytes (0: keep nothing), freeing blocks beyond it.
    void set_limit(size_t bytes) {
        std::lock_guard<std::mutex> lock(mu_);
        limit_ = bytes;
        shrink_to(limit_);
    }

    // Frees every cached block.
    void trim() {
        std::lock_guard<std::mutex> lock(mu_);
        drop_all();
    }

    DevCacheInfo info() {
        std::lock_guard<std::mutex> lock(mu_);
        return DevCacheInfo{(int64_t)cached_, (int64_t)in_use_bytes_, (int64_t)hits_,
                            (int64_t)misses_};
    }

    static bool fits(size_t block, size_t bytes) {
        return block >= bytes && block - bytes <= bytes / 8 + ((size_t)1 << 16);
    }

private:
    struct Block {
        void *ptr;
        size_t size;
    };
    // (callers hold mu_) least recently released first
    void shrink_to(size_t bound) {
        while (cached_ > bound && !free_.empty()) {
            const Block b = free_.back();
            free_.pop_back();
            cached_ -= b.size;
            be_.free(b.ptr);
        }
    }
    void drop_all() { shrink_to(0); }

    Backend be_;
    size_t limit_;
    std::mutex mu_;
    std::list<Block> free_;  // most recently released first
    std::unordered_map<void *, size_t> in_use_;
    size_t cached_ = 0, in_use_bytes_ = 0;
    uint64_t hits_ = 0, misses_ = 0;
};

// The library's instance (device memory; defined in ecmc.cu): every device
// array of a context, a batch or a launch is taken and given back here.
int dm_alloc(void **p, size_t bytes);  // 0 on success, else a cudaError_t value
void dm_free(void *p);                 // null: nothing
template <class T>
inline int dm_alloc_t(T **p, size_t bytes) {
    return dm_alloc(reinterpret_cast<void **>(p), bytes);
}
