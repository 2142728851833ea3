// Host-side first-fit allocator over one device range: the serving engine's
// request pool.  It hands out offsets into a range the caller allocated once;
// it makes no CUDA call, so its logic is testable on the host.
#pragma once

#include <algorithm>
#include <cstddef>
#include <iterator>
#include <map>

namespace csc {

constexpr size_t kAlign = 256;  // every block starts and ends on a 256-byte boundary

inline size_t align_up(size_t x)
{
    return (x + kAlign - 1) & ~(kAlign - 1);
}

// First-fit allocator over one device range, with coalescing of free blocks.
class Pool {
public:
    char *base = nullptr;
    size_t size = 0, in_use = 0, peak = 0;

    void init(char *b, size_t n)
    {
        base = b;
        size = n;
        free_.clear();
        free_[0] = n;
    }
    bool alloc(size_t n, size_t *off)
    {
        n = align_up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n)
                continue;
            const size_t o = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest)
                free_[o + n] = rest;
            *off = o;
            in_use += n;
            peak = std::max(peak, in_use);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = align_up(n);
        in_use -= n;
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

private:
    std::map<size_t, size_t> free_;  // offset -> length
};

}  // namespace csc
