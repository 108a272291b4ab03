// Work lists of the symmetric pair kernels: the runs of rounds of the pair
// schedule that one launch covers, and their decoding into pair blocks (the
// schedule itself is described in hk_internal.cuh).
#pragma once

#include <stdint.h>

namespace hk {

// One pair block of a launch: set, blocks I <= J (J == nblk: the empty
// team), and kind = diagonal | scratch << 1 | slot << 2 (the slot its
// partials are stored in; scratch: a scratch slot of a later phase).
struct WorkItem {
    int32_t set, I, J, kind;
};

// A run of work items of one launch: rounds [r0, r0 + nr) of set `set`,
// either the off-diagonal blocks of each round ((nt - 1) / 2 per round, in
// order j = 1, 2, ...) or its diagonal blocks (one per round).  first: index
// of the run's first item within the launch.
struct ItemRun {
    int32_t set, r0, nr, diag, first, pad_;
};

// The work list of one pair launch: nruns runs (first increasing), nitems
// items in all.
struct Sched {
    const ItemRun *runs;
    int32_t nruns, nitems;
};

#ifdef __CUDACC__
// Item k of a launch (0 <= k < sc.nitems): its run by binary search, then
// its round and blocks by the circle method (sets: the plan's set
// descriptors, of which nblk and nslot are read).
template <typename Set>
__device__ __forceinline__ WorkItem decode_item(const Set *sets, const Sched &sc, int k)
{
    int lo = 0, hi = sc.nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sc.runs[mid].first <= k)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ItemRun ru = sc.runs[lo];
    const int nt = sets[ru.set].nblk | 1, nslot = sets[ru.set].nslot;
    const int local = k - ru.first;
    int r, I, J;
    if (ru.diag) {
        r = ru.r0 + local;
        I = J = r;
    } else {
        const int per = (nt - 1) >> 1;
        r = ru.r0 + local / per;
        const int j = local % per + 1;
        int a = r + j, b = r - j;
        a = a >= nt ? a - nt : a;
        b = b < 0 ? b + nt : b;
        I = min(a, b);
        J = max(a, b);
    }
    const int slot = r < nslot ? r : nslot + r % nslot;
    const int kind = (I == J ? 1 : 0) | (r >= nslot ? 2 : 0) | (slot << 2);
    return WorkItem{ru.set, I, J, kind};
}
#endif

}  // namespace hk
