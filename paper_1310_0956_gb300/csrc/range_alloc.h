// range_alloc.h -- first-fit allocator of element ranges of a pool, used by
// the request server to place each admitted request's image and sinogram
// state. Plain C++ (no CUDA), so that it also builds into host-only tests.
#pragma once

#include <cstdint>
#include <iterator>
#include <map>

namespace wmg {

// First-fit allocator of element ranges of a pool (offsets aligned to 64
// elements), adjacent free ranges merged on release.
struct RangeAlloc {
    std::map<int64_t, int64_t> free_;   // offset -> length
    int64_t cap = 0, used = 0;
    static int64_t round(int64_t n) { return (n + 63) / 64 * 64; }
    void init(int64_t c)
    {
        cap = c / 64 * 64;
        used = 0;
        free_.clear();
        if (cap > 0) free_[0] = cap;
    }
    int64_t alloc(int64_t n)
    {
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const int64_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[off + n] = len - n;
            used += n;
            return off;
        }
        return -1;
    }
    void release(int64_t off, int64_t n)
    {
        n = round(n);
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

}  // namespace wmg
