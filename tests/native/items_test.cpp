// Host-only check of the work-item queue's item -> frame lookup (tfn_items.h)
// against a linear scan: random frame sizes (equal runs, mixes, single-item
// frames), random warp counts and warps, each warp's items in increasing
// order as the kernel takes them.  Prints "ok" and exits 0 on success.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "tfn_items.h"

int main()
{
    std::mt19937 rng(12345);
    long long checked = 0;
    for (int trial = 0; trial < 4000; ++trial) {
        const int n = 1 + (int)(rng() % 60);
        std::vector<int> first(n);
        const int kinds[] = {1, 2, 5, 80, 80, 80, 95};
        int acc = 0;
        for (int i = 0; i < n; ++i) {
            first[i] = acc;
            acc += (rng() % 4 == 0) ? 1 + (int)(rng() % 300) : kinds[rng() % 7];
        }
        const int total = acc, nw = 1 + (int)(rng() % 400), gw = (int)(rng() % nw);
        auto get = [&](int i) { return first[i]; };
        int from = 0;
        for (int t = gw; t < total; t += nw) {
            int want = 0;
            while (want + 1 < n && first[want + 1] <= t) ++want;
            from = tfn::frame_of(get, n, t, from);
            if (from != want) {
                std::printf("FAILED trial %d: item %d gives frame %d, not %d\n", trial, t, from, want);
                return 1;
            }
            ++checked;
        }
    }
    std::printf(checked > 50000 ? "ok\n" : "too few checks\n");
    return checked > 50000 ? 0 : 1;
}
