// First-fit allocator over one device allocation (host-side bookkeeping
// only): the server carves its HBM budget into per-stream blocks with it.
// Blocks are multiples of 256 bytes; released blocks merge with free
// neighbours, so releasing everything leaves one free block of the full size.
#pragma once

#include <stddef.h>

#include <iterator>
#include <map>

namespace pcal_arena {

constexpr size_t kGrain = 256;  // block granularity (and alignment of every offset)

inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

class Arena {
  public:
    // Forget every block; the whole [0, size) is free.
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        used_ = 0;
    }
    // Lowest-offset free block that holds `bytes` (rounded up to kGrain);
    // false, with nothing changed, when none does.
    bool alloc(size_t bytes, size_t* off) {
        bytes = round_up(bytes, kGrain);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += bytes;
            return true;
        }
        return false;
    }
    // Give back a block alloc returned (same offset and requested size).
    void release(size_t off, size_t bytes) {
        bytes = round_up(bytes, kGrain);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t free_blocks() const { return free_.size(); }

  private:
    std::map<size_t, size_t> free_;  // offset -> bytes, no two adjacent
    size_t used_ = 0;
};

}  // namespace pcal_arena
