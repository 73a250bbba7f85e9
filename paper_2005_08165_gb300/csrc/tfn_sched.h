// tfn_sched.h -- host-only scheduling pieces of the request server: the ring
// arena that hands out device staging memory and the admission rule of the
// continuous batcher.  Plain C++ (no CUDA), so that it can be tested on its
// own.
#pragma once

#include <cstddef>
#include <cstdint>
#include <deque>

namespace tfn {

// First-in first-out allocator over [0, capacity): blocks are carved at the
// head and released oldest first, so free space is always one or two
// contiguous runs and nothing fragments.  Offsets and sizes are multiples of
// `align`.  Not thread-safe.
class RingArena {
public:
    static constexpr size_t kNone = ~(size_t)0;

    explicit RingArena(size_t capacity = 0, size_t align = 256) : cap_(capacity / align * align), align_(align) {}

    size_t capacity() const { return cap_; }
    size_t in_use() const { return used_; }
    size_t live_blocks() const { return live_.size(); }
    size_t round(size_t bytes) const { return (bytes + align_ - 1) / align_ * align_; }

    // Largest block alloc() could return right now.
    size_t largest_fit() const
    {
        if (live_.empty()) return cap_;
        const size_t tail = live_.front().off;
        if (tail < head_) return (cap_ - head_ > tail) ? cap_ - head_ : tail;  // [head, cap) or [0, tail)
        return tail - head_;                                                   // wrapped: [head, tail)
    }

    // Offset of a new block of round(bytes) > 0 bytes, or kNone if it does
    // not fit now (or bytes is 0: callers with nothing to stage take no block).
    size_t alloc(size_t bytes)
    {
        const size_t n = round(bytes);
        if (n == 0) return kNone;
        size_t off;
        if (live_.empty()) {
            if (n > cap_) return kNone;
            off = 0;
        } else {
            // live blocks have positive sizes, so the oldest block starts below
            // head_ exactly when the ring has not wrapped
            const size_t tail = live_.front().off;
            if (tail < head_) {
                if (n <= cap_ - head_)
                    off = head_;
                else if (n <= tail)
                    off = 0;  // wrap: [head_, cap) stays unused until the blocks before it are released
                else
                    return kNone;
            } else {
                if (n > tail - head_) return kNone;
                off = head_;
            }
        }
        live_.push_back({off, n});
        head_ = off + n;
        used_ += n;
        return off;
    }

    // Releases the oldest live block.
    void free_oldest()
    {
        if (live_.empty()) return;
        used_ -= live_.front().size;
        live_.pop_front();
        if (live_.empty()) head_ = 0;
    }

private:
    struct Block {
        size_t off, size;
    };
    std::deque<Block> live_;
    size_t cap_, align_;
    size_t head_ = 0;  // end of the newest block
    size_t used_ = 0;
};

// Admission rule of the continuous batcher: take requests from the front of
// the queue, in order, while the batch holds fewer than `max_batch` and the
// staging bytes of the requests taken so far fit in one block of `fit`
// bytes.  The first request that does not fit stops the batch (no request
// overtakes an earlier one, so a large request cannot starve).  `bytes_of`
// maps a queue element to its staging bytes (already rounded).
template <class Queue, class BytesOf>
size_t admit_count(const Queue &queue, size_t max_batch, size_t fit, BytesOf bytes_of, size_t *total_bytes)
{
    size_t k = 0, sum = 0;
    for (const auto &r : queue) {
        if (k >= max_batch) break;
        const size_t b = bytes_of(r);
        if (sum + b > fit) break;
        sum += b;
        ++k;
    }
    if (total_bytes) *total_bytes = sum;
    return k;
}

}  // namespace tfn
