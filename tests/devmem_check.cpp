// Host check of the device memory cache's policy (csrc/devmem.h) with a fake
// backend: plain malloc under a byte capacity, counting live blocks. Prints
// "ok <checks>" and exits 0, or names the first failed check and exits 1.
#include <cstdio>
#include <cstdlib>
#include <set>
#include <thread>
#include <vector>

#include "devmem.h"

namespace {

struct Fake {
    size_t cap = 0, live_bytes = 0;
    long allocs = 0, frees = 0;
    std::set<void *> live;
    std::vector<std::pair<void *, size_t>> sizes;
};
Fake *g_fake = nullptr;

struct FakeBackend {
    int alloc(void **p, size_t bytes) {
        if (g_fake->live_bytes + bytes > g_fake->cap) return 2;  // out of memory
        *p = std::malloc(bytes);
        if (!*p) return 2;
        g_fake->live.insert(*p);
        g_fake->sizes.push_back({*p, bytes});
        g_fake->live_bytes += bytes;
        ++g_fake->allocs;
        return 0;
    }
    void free(void *p) {
        if (!g_fake->live.count(p)) {
            std::printf("FAIL free of a block that is not live\n");
            std::exit(1);
        }
        g_fake->live.erase(p);
        for (auto &e : g_fake->sizes)
            if (e.first == p) {
                g_fake->live_bytes -= e.second;
                e.second = 0;
                e.first = nullptr;
                break;
            }
        ++g_fake->frees;
        std::free(p);
    }
};

int checks = 0;
#define CHECK(cond)                                                       \
    do {                                                                  \
        ++checks;                                                         \
        if (!(cond)) {                                                    \
            std::printf("FAIL line %d: %s\n", __LINE__, #cond);           \
            std::exit(1);                                                 \
        }                                                                 \
    } while (0)

// every live backend block is either handed out or cached
void balanced(BlockCache<FakeBackend> &c) {
    const DevCacheInfo i = c.info();
    CHECK((int64_t)g_fake->live_bytes == i.cached_bytes + i.in_use_bytes);
}

}  // namespace

int main() {
    const size_t MiB = (size_t)1 << 20;
    {
        Fake f;
        f.cap = 1000 * MiB;
        g_fake = &f;
        BlockCache<FakeBackend> c(64 * MiB);
        void *a = nullptr, *b = nullptr, *d = nullptr;
        // a miss, then the same size again after release: the same block
        CHECK(c.acquire(&a, 10 * MiB) == 0 && a);
        c.release(a);
        CHECK(c.info().cached_bytes == (int64_t)(10 * MiB));
        CHECK(c.acquire(&b, 10 * MiB) == 0 && b == a);
        CHECK(c.info().hits == 1 && c.info().misses == 1);
        balanced(c);
        // a little smaller still fits (within an eighth); much smaller does not
        c.release(b);
        CHECK(c.acquire(&d, 9 * MiB) == 0 && d == a);
        c.release(d);
        void *e = nullptr;
        CHECK(c.acquire(&e, 4 * MiB) == 0 && e != a);
        CHECK(c.info().cached_bytes == (int64_t)(10 * MiB));
        balanced(c);
        // a larger request never takes a smaller block
        void *g = nullptr;
        CHECK(c.acquire(&g, 11 * MiB) == 0 && g != a);
        balanced(c);
        // best fit: of two fitting blocks, the smaller
        c.release(g);  // 11 MiB and 10 MiB cached
        void *h = nullptr;
        CHECK(c.acquire(&h, 10 * MiB) == 0 && h == a);
        c.release(h);
        c.release(e);
        balanced(c);
        // the limit: releasing beyond it frees the least recently released
        void *big[8];
        for (auto &p : big) CHECK(c.acquire(&p, 20 * MiB) == 0);
        const long frees0 = f.frees;
        for (auto &p : big) c.release(p);
        CHECK(c.info().cached_bytes <= (int64_t)(64 * MiB));
        CHECK(f.frees > frees0);
        balanced(c);
        // the most recently released blocks stay
        void *q = nullptr;
        CHECK(c.acquire(&q, 20 * MiB) == 0 && q == big[7]);
        c.release(q);
        // a block larger than the limit is not kept
        void *huge = nullptr;
        CHECK(c.acquire(&huge, 100 * MiB) == 0);
        const int64_t cached0 = c.info().cached_bytes;
        c.release(huge);
        CHECK(c.info().cached_bytes == cached0);
        CHECK(f.live.count(huge) == 0);
        balanced(c);
        // limit 0: everything cached goes back, and nothing is kept after
        c.set_limit(0);
        CHECK(c.info().cached_bytes == 0 && f.live_bytes == (size_t)c.info().in_use_bytes);
        void *z = nullptr;
        CHECK(c.acquire(&z, MiB) == 0);
        c.release(z);
        CHECK(c.info().cached_bytes == 0);
        balanced(c);
        // null releases nothing; a foreign pointer goes to the backend
        c.release(nullptr);
        void *foreign = nullptr;
        CHECK(FakeBackend().alloc(&foreign, MiB) == 0);
        c.release(foreign);
        CHECK(f.live.count(foreign) == 0);
        // zero bytes: a valid block of one byte
        void *one = nullptr;
        CHECK(c.acquire(&one, 0) == 0 && one);
        c.release(one);
        balanced(c);
        CHECK(f.live_bytes == 0);
    }
    {
        // out of memory: the cached blocks are freed and the request retried
        Fake f;
        f.cap = 100 * MiB;
        g_fake = &f;
        BlockCache<FakeBackend> c(1000 * MiB);
        void *a = nullptr, *b = nullptr;
        CHECK(c.acquire(&a, 60 * MiB) == 0);
        c.release(a);  // cached: 60 of the 100 MiB
        CHECK(c.acquire(&b, 70 * MiB) == 0);  // fits only after the trim
        CHECK(c.info().cached_bytes == 0);
        void *d = nullptr;
        CHECK(c.acquire(&d, 50 * MiB) != 0 && d == nullptr);  // truly out of memory
        c.release(b);
        c.trim();
        CHECK(f.live_bytes == 0);
        balanced(c);
    }
    {
        // threads: acquire and release concurrently; the books balance
        Fake f;
        f.cap = (size_t)1 << 40;
        g_fake = &f;
        // (the cache calls its backend under its own mutex)
        BlockCache<FakeBackend> c(256 * MiB);
        std::vector<std::thread> ts;
        for (int t = 0; t < 8; ++t)
            ts.emplace_back([&c, t]() {
                for (int i = 0; i < 200; ++i) {
                    void *p = nullptr;
                    const size_t sz = ((size_t)((t * 7 + i) % 5) + 1) << 20;
                    if (c.acquire(&p, sz) != 0) std::abort();
                    c.release(p);
                }
            });
        for (auto &t : ts) t.join();
        const DevCacheInfo i = c.info();
        CHECK(i.in_use_bytes == 0);
        CHECK(i.hits + i.misses == 8 * 200);
        CHECK(i.hits > 0);
        balanced(c);
        c.trim();
        CHECK(f.live_bytes == 0);
    }
    std::printf("ok %d\n", checks);
    return 0;
}
