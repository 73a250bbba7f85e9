// tfn_items.h -- the work-item queue's item -> frame lookup, shared by the
// kernel (device loads) and a host-only test (plain loads).
#pragma once

#ifdef __CUDACC__
#define TFN_HD __host__ __device__ __forceinline__
#else
#define TFN_HD inline
#endif

namespace tfn {

// The frame of work item t: the last frame whose first item is at or below
// t, where first(i) returns frame i's first item (frames are numbered in item
// order, every frame has at least one item).  A warp's items only increase,
// so the search starts at the previous answer `from`.  A warp's next item
// lies about (warps in the grid) / (items per frame) frames further on, so
// stepping one frame at a time would chain dozens of dependent loads per
// item; instead the first guess assumes frames of the size of `from` (exact
// for a batch of equal frames), and a binary search over the rest covers any
// mix.
template <class First>
TFN_HD int frame_of(const First &first, int nframes, int t, int from)
{
    if (from + 1 >= nframes) return from;
    const int b0 = first(from), b1 = first(from + 1);
    if (t < b1) return from;
    int lo = from + 1, hi = nframes - 1;  // the answer lies in [lo, hi] (t >= b1)
    int g = from + (t - b0) / (b1 - b0);
    if (g > hi) g = hi;
    if (g >= lo) {
        if (first(g) <= t) {
            if (g == hi || first(g + 1) > t) return g;
            lo = g + 1;
        } else {
            hi = g - 1;
        }
    }
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first(mid) <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

}  // namespace tfn
