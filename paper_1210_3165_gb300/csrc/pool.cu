// pool.cu -- host-side first-fit allocator over one caller-owned device
// range, for the serving loop's per-request buffers (no device calls).
#include "bnz.h"
#include "internal.h"

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <new>

struct bnz_pool {
    uintptr_t base = 0;
    size_t bytes = 0;
    std::map<size_t, size_t> free_;  // offset -> size, disjoint, never adjacent
    std::map<size_t, size_t> live_;  // offset -> size
    size_t used = 0, high_water = 0;
    int fail_next = 0;
    mutable std::mutex mu;
};

namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

} // namespace

extern "C" {

int bnz_pool_create(void *base, size_t bytes, bnz_pool **out)
{
    using bnz::fail;
    if (!out)
        return fail(BNZ_EINVAL, "bnz_pool_create: null out");
    *out = nullptr;
    if (!base || (reinterpret_cast<uintptr_t>(base) & (kAlign - 1)))
        return fail(BNZ_EINVAL, "bnz_pool_create: base must be a 256-byte-aligned pointer");
    bytes &= ~(kAlign - 1);
    if (bytes == 0)
        return fail(BNZ_EINVAL, "bnz_pool_create: range smaller than 256 bytes");
    bnz_pool *p = new (std::nothrow) bnz_pool;
    if (!p)
        return fail(BNZ_ENOMEM, "bnz_pool_create: host allocation failed");
    p->base = reinterpret_cast<uintptr_t>(base);
    p->bytes = bytes;
    p->free_.emplace(0, bytes);
    *out = p;
    return BNZ_OK;
}

int bnz_pool_alloc(bnz_pool *p, size_t bytes, void **out)
{
    using bnz::fail;
    if (!p || !out)
        return fail(BNZ_EINVAL, "bnz_pool_alloc: null argument");
    *out = nullptr;
    const size_t need = round_up(std::max<size_t>(bytes, 1));
    std::lock_guard<std::mutex> g(p->mu);
    if (p->fail_next > 0) {
        --p->fail_next;
        return fail(BNZ_ENOMEM, "bnz_pool_alloc: injected failure");
    }
    for (auto it = p->free_.begin(); it != p->free_.end(); ++it) {
        if (it->second < need)
            continue;
        const size_t off = it->first, rest = it->second - need;
        p->free_.erase(it);
        if (rest)
            p->free_.emplace(off + need, rest);
        p->live_.emplace(off, need);
        p->used += need;
        p->high_water = std::max(p->high_water, p->used);
        *out = reinterpret_cast<void *>(p->base + off);
        return BNZ_OK;
    }
    return fail(BNZ_ENOMEM, "bnz_pool_alloc: no free range of %zu bytes", need);
}

int bnz_pool_free(bnz_pool *p, void *ptr)
{
    using bnz::fail;
    if (!p)
        return fail(BNZ_EINVAL, "bnz_pool_free: null pool");
    const uintptr_t a = reinterpret_cast<uintptr_t>(ptr);
    std::lock_guard<std::mutex> g(p->mu);
    if (a < p->base)
        return fail(BNZ_EINVAL, "bnz_pool_free: pointer outside the pool");
    auto lit = p->live_.find(a - p->base);
    if (lit == p->live_.end())
        return fail(BNZ_EINVAL, "bnz_pool_free: not a live block of this pool");
    size_t off = lit->first, size = lit->second;
    p->live_.erase(lit);
    p->used -= size;
    // coalesce with the free neighbours on both sides
    auto next = p->free_.lower_bound(off);
    if (next != p->free_.end() && next->first == off + size) {
        size += next->second;
        next = p->free_.erase(next);
    }
    if (next != p->free_.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            prev->second += size;
            return BNZ_OK;
        }
    }
    p->free_.emplace(off, size);
    return BNZ_OK;
}

int bnz_pool_stats(const bnz_pool *p, size_t *used, size_t *high_water, size_t *largest_free, int *live)
{
    if (!p)
        return bnz::fail(BNZ_EINVAL, "bnz_pool_stats: null pool");
    std::lock_guard<std::mutex> g(p->mu);
    size_t lf = 0;
    for (const auto &f : p->free_)
        lf = std::max(lf, f.second);
    if (used)
        *used = p->used;
    if (high_water)
        *high_water = p->high_water;
    if (largest_free)
        *largest_free = lf;
    if (live)
        *live = static_cast<int>(p->live_.size());
    return BNZ_OK;
}

int bnz_pool_fail_next(bnz_pool *p, int n)
{
    if (!p || n < 0)
        return bnz::fail(BNZ_EINVAL, "bnz_pool_fail_next: bad argument");
    std::lock_guard<std::mutex> g(p->mu);
    p->fail_next = n;
    return BNZ_OK;
}

int bnz_pool_destroy(bnz_pool *p)
{
    delete p;
    return BNZ_OK;
}

} // extern "C"
