// Work lists of the symmetric pair kernels: the runs of rounds of the pair
// schedule that one launch covers, and their decoding into pair blocks (the
// schedule itself is described in hk_internal.cuh).
#pragma once

#include <stdint.h>

#include <vector>

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

// The run of one set's rounds in phase `phase` (rounds [phase nslot,
// phase nslot + nslot) of its nblk | 1): its off-diagonal blocks or (diag)
// its diagonal ones, appended to runs with its first item index `first`,
// which advances by the run's item count.  Nothing when the phase holds no
// such item for the set.
inline void append_set_run(int32_t set, int nblk, int nslot, int phase, bool diag, std::vector<ItemRun> &runs,
                           int64_t &first)
{
    const int nt = nblk | 1;
    const int r0 = phase * nslot;
    int r1 = r0 + nslot;
    r1 = r1 < (diag ? nblk : nt) ? r1 : (diag ? nblk : nt);
    const int per = diag ? 1 : (nt - 1) / 2;
    if (r1 <= r0 || per == 0)
        return;
    runs.push_back({set, r0, r1 - r0, diag ? 1 : 0, (int32_t)first, 0});
    first += (int64_t)(r1 - r0) * per;
}

#ifdef __CUDACC__
// Item k of a launch (0 <= k < sc.nitems): its run by binary search, then
// its round and blocks by the circle method (sets: the plan's set
// descriptors, of which nblk and nslot are read).  Host and device.
template <typename Set>
__host__ __device__ __forceinline__ WorkItem decode_item(const Set *sets, const Sched &sc, int k)
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
