// Host-side scheduling of the serving loop: the device arena that admits requests by memory
// and the rule that forms the next batch.  Plain C++ with no CUDA, so that it can be
// compiled and checked on a machine without a GPU.
#pragma once

#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace rkm {
namespace serve {

constexpr size_t kGranule = 256;  // arena offsets and sizes are multiples of this

inline size_t round_granule(size_t b) { return (b + kGranule - 1) / kGranule * kGranule; }

// Arena bytes of a batch of `items` candidate rows of dimension d: the FP32 rows (stride d)
// followed by the int32 counts, each part starting on a granule.
inline size_t batch_bytes(int64_t items, int d) {
    return round_granule((size_t)items * (size_t)d * sizeof(float)) + round_granule((size_t)items * sizeof(int32_t));
}

// First-fit allocator over the offsets [0, size) of one device block.  Sizes are rounded up
// to the granule; a released range merges with free neighbours.  Not thread-safe (the
// server calls it under its lock).
class Arena {
public:
    explicit Arena(size_t size = 0) { reset(size); }

    void reset(size_t size) {
        size_ = size / kGranule * kGranule;
        free_.clear();
        if (size_) free_[0] = size_;
        used_ = high_ = 0;
    }

    // Allocate `bytes` (> 0); false when no free range is large enough.
    bool alloc(size_t bytes, size_t* off) {
        bytes = round_granule(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += bytes;
            if (used_ > high_) high_ = used_;
            return true;
        }
        return false;
    }

    // Return a range obtained from alloc with the same `bytes`.
    void release(size_t off, size_t bytes) {
        bytes = round_granule(bytes ? bytes : 1);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                bytes += prev->second;
                free_.erase(prev);
            }
        }
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            free_.erase(next);
        }
        free_[off] = bytes;
    }

    size_t size() const { return size_; }
    size_t in_use() const { return used_; }
    size_t high_water() const { return high_; }
    void reset_high_water() { high_ = used_; }
    size_t free_ranges() const { return free_.size(); }
    size_t largest_free() const {
        size_t best = 0;
        for (const auto& f : free_) best = f.second > best ? f.second : best;
        return best;
    }

private:
    std::map<size_t, size_t> free_;  // offset -> length of each free range
    size_t size_ = 0, used_ = 0, high_ = 0;
};

// The batch a free slot takes next, from the requests waiting in arrival order:
// items_of(j) is the candidate count of the j-th oldest of `waiting` requests.  The batch is
// the longest prefix whose total stays within max_items, shortened from the back until its
// arena bytes can be allocated.  Returns the number of requests taken and sets *off and
// *items; 0 means that not even the oldest request fits in the arena now (the slot waits
// until a running batch releases memory).  Requests are never reordered, so the oldest one
// is always in the next batch that runs.
template <class ItemsOf>
int take_batch(size_t waiting, ItemsOf items_of, int64_t max_items, int d, Arena& arena, size_t* off,
               int64_t* items) {
    int count = 0;
    int64_t total = 0;
    while ((size_t)count < waiting) {
        const int64_t q = items_of((size_t)count);
        if (count > 0 && total + q > max_items) break;
        total += q;
        ++count;
    }
    while (count > 0) {
        if (arena.alloc(batch_bytes(total, d), off)) {
            *items = total;
            return count;
        }
        --count;
        total -= items_of((size_t)count);
    }
    *items = 0;
    return 0;
}

}  // namespace serve
}  // namespace rkm
