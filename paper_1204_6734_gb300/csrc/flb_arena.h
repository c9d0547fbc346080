// flb_arena.h -- first-fit sub-allocator of one device memory pool (host code
// only, no CUDA): hands out aligned byte ranges of [0, size) and coalesces
// freed neighbours. Batches and the request server carve every replica's
// population buffers out of one pool allocated up front, so admitting or
// retiring a lattice never calls cudaMalloc / cudaFree (which synchronise the
// device) and the pool size is the HBM budget admission works against.
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace flb {

class Arena {
public:
    static constexpr size_t kAlign = 256;

    explicit Arena(size_t size = 0) { reset(size); }

    void reset(size_t size) {
        size_ = size / kAlign * kAlign;
        used_bytes_ = 0;
        free_.clear();
        used_.clear();
        if (size_) free_[0] = size_;
    }

    static size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

    // First free range that fits; false (and *off untouched) if none does.
    bool alloc(size_t bytes, size_t* off) {
        if (bytes == 0) bytes = 1;
        const size_t need = round_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t o = it->first, rest = it->second - need;
            free_.erase(it);
            if (rest) free_[o + need] = rest;
            used_[o] = need;
            used_bytes_ += need;
            *off = o;
            return true;
        }
        return false;
    }

    // Return a range from alloc(); false if off is not the start of one.
    bool release(size_t off) {
        auto u = used_.find(off);
        if (u == used_.end()) return false;
        size_t o = off, n = u->second;
        used_.erase(u);
        used_bytes_ -= n;
        auto next = free_.lower_bound(o);
        if (next != free_.end() && next->first == o + n) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == o) {
                prev->second += n;
                return true;
            }
        }
        free_[o] = n;
        return true;
    }

    size_t size() const { return size_; }
    size_t used() const { return used_bytes_; }
    size_t largest_free() const {
        size_t m = 0;
        for (const auto& f : free_) m = f.second > m ? f.second : m;
        return m;
    }
    size_t free_ranges() const { return free_.size(); }
    size_t live_ranges() const { return used_.size(); }

private:
    size_t size_ = 0, used_bytes_ = 0;
    std::map<size_t, size_t> free_;   // offset -> length, disjoint, never adjacent
    std::map<size_t, size_t> used_;   // offset -> length
};

}  // namespace flb
