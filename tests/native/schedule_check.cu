// Host-side check of the pair schedule (hk_sched.cuh): the runs that the
// plan builder appends and the item decoding that the pair kernels use,
// run on the CPU for many block counts and slot caps.  For one set of nblk
// row blocks and cap G it checks that over all phases every unordered pair
// of distinct blocks and every diagonal block is visited exactly once; that
// every item's blocks lie in range (the empty team only as J = nblk when
// nblk is even); that within a phase no (block, slot) is written twice;
// that phase 0 writes every slot of every block, and later phases use the
// scratch slots nslot .. 2 nslot - 1.  Prints "ok" or the first failure.
// Usage: schedule_check (no arguments).
#include <cstdio>
#include <vector>

#include "hk_sched.cuh"

using namespace hk;

struct TestSet {
    int nblk, nslot;
};

static bool check(int nblk, int G)
{
    const int nt = nblk | 1;
    const int nslot = G < nt ? G : nt;
    const TestSet set{nblk, nslot};
    const int phases = (nt + nslot - 1) / nslot;
    std::vector<int> seen((size_t)(nblk + 1) * (nblk + 1), 0);
    for (int p = 0; p < phases; ++p) {
        std::vector<ItemRun> runs;
        int64_t first = 0;
        append_set_run(0, nblk, nslot, p, false, runs, first);
        append_set_run(0, nblk, nslot, p, true, runs, first);
        if (runs.empty())
            continue;
        const Sched sc{runs.data(), (int32_t)runs.size(), (int32_t)first};
        std::vector<int> written((size_t)nblk * 2 * nslot, 0);
        for (int k = 0; k < sc.nitems; ++k) {
            const WorkItem it = decode_item(&set, sc, k);
            const int slot = it.kind >> 2;
            const bool scratch = (it.kind & 2) != 0, diag = (it.kind & 1) != 0;
            if (it.I < 0 || it.I > it.J || it.J > nblk || (it.J == nblk && (nblk % 2 == 1 || it.I == it.J)) ||
                diag != (it.I == it.J)) {
                std::printf("nblk %d G %d phase %d item %d: blocks %d %d kind %d\n", nblk, G, p, k, it.I, it.J,
                            it.kind);
                return false;
            }
            if (scratch != (p > 0) || (p == 0 ? slot >= nslot : (slot < nslot || slot >= 2 * nslot))) {
                std::printf("nblk %d G %d phase %d item %d: slot %d scratch %d\n", nblk, G, p, k, slot, scratch);
                return false;
            }
            if (it.J < nblk)
                ++seen[(size_t)it.I * (nblk + 1) + it.J];
            // the blocks whose rows this item writes: I, and J unless it is I
            // itself (diagonal) or the empty team
            const int blocks[2] = {it.I, it.J};
            const int nw = (it.I == it.J || it.J == nblk) ? 1 : 2;
            for (int q = 0; q < nw; ++q) {
                const int b = blocks[q];
                if (++written[(size_t)b * 2 * nslot + slot] != 1) {
                    std::printf("nblk %d G %d phase %d: block %d slot %d written twice\n", nblk, G, p, b, slot);
                    return false;
                }
            }
        }
        if (p == 0)
            for (int b = 0; b < nblk; ++b)
                for (int s = 0; s < nslot; ++s)
                    if (written[(size_t)b * 2 * nslot + s] != 1) {
                        std::printf("nblk %d G %d: block %d slot %d not written in phase 0\n", nblk, G, b, s);
                        return false;
                    }
    }
    for (int I = 0; I < nblk; ++I)
        for (int J = I; J < nblk; ++J)
            if (seen[(size_t)I * (nblk + 1) + J] != 1) {
                std::printf("nblk %d G %d: block pair %d %d visited %d times\n", nblk, G, I, J,
                            seen[(size_t)I * (nblk + 1) + J]);
                return false;
            }
    return true;
}

int main()
{
    for (int nblk = 1; nblk <= 130; ++nblk)
        for (int G : {1, 2, 3, 4, 7, 16, 1 << 20})
            if (!check(nblk, G))
                return 1;
    for (int nblk : {391, 392, 977, 1172, 1173})
        for (int G : {27, 55, 83, 1 << 20})
            if (!check(nblk, G))
                return 1;
    std::printf("ok\n");
    return 0;
}
