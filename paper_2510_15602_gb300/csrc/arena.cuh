// arena.cuh -- the serving session's device-arena bookkeeping (plain host C++,
// no CUDA): first fit over [0, size) with a free list kept as an ordered map of
// offset -> length; a released block merges with its free neighbours, so the
// free list never holds two adjacent blocks.  Offsets only: the session adds
// them to its one device allocation.
#pragma once

#include <stddef.h>

#include <algorithm>
#include <iterator>
#include <map>

namespace qfca {

struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    void reset(size_t n) {
        size = n;
        free_.clear();
        free_[0] = n;
    }
    // the longest free block
    size_t largest() const {
        size_t m = 0;
        for (auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
    // the lowest-addressed free block of at least n bytes; false when none
    bool alloc(size_t n, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        return false;
    }
    // returns [off, off + n), which alloc handed out
    void release(size_t off, size_t n) {
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

}  // namespace qfca
