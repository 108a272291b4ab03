// Host-side check of the pair schedule (hk_sched.cuh): the runs that the
// plan builder appends and the item decoding that the pair kernels use,
// run on the CPU for many block counts and slot caps.  For one set of nblk
// row blocks and cap G it checks that over all phases every unordered pair
// of distinct blocks and every diagonal block is visited exactly once; that
// every item's blocks lie in range (the empty team only as J = nblk when
// nblk is even); that within a phase no (block, slot) is written twice;
// that phase 0 writes every slot of every block, and later phases use the
// scratch slots nslot .. 2 nslot - 1; the same for batches of uneven sets
// whose runs share a launch.  Prints "ok" or the first failure.
// Usage: schedule_check (no arguments).
#include <cstdio>
#include <vector>

#include "hk_sched.cuh"

using namespace hk;

struct TestSet {
    int nblk, nslot;
};

// One launch list per phase over several sets (their off-diagonal runs, then
// their diagonal runs, as the plan builder orders them), every item decoded
// and checked against its own set.
static bool check(const std::vector<int> &nblks, int G)
{
    const int ns = (int)nblks.size();
    std::vector<TestSet> sets(ns);
    int phases = 0;
    for (int s = 0; s < ns; ++s) {
        const int nt = nblks[s] | 1;
        sets[s] = TestSet{nblks[s], G < nt ? G : nt};
        const int ph = (nt + sets[s].nslot - 1) / sets[s].nslot;
        phases = ph > phases ? ph : phases;
    }
    std::vector<std::vector<int>> seen(ns);
    for (int s = 0; s < ns; ++s)
        seen[s].assign((size_t)(nblks[s] + 1) * (nblks[s] + 1), 0);
    for (int p = 0; p < phases; ++p) {
        std::vector<ItemRun> runs;
        int64_t first = 0;
        for (int diag = 0; diag < 2; ++diag)
            for (int s = 0; s < ns; ++s)
                append_set_run(s, sets[s].nblk, sets[s].nslot, p, diag != 0, runs, first);
        if (runs.empty())
            continue;
        const Sched sc{runs.data(), (int32_t)runs.size(), (int32_t)first};
        std::vector<std::vector<int>> written(ns);
        for (int s = 0; s < ns; ++s)
            written[s].assign((size_t)sets[s].nblk * 2 * sets[s].nslot, 0);
        for (int k = 0; k < sc.nitems; ++k) {
            const WorkItem it = decode_item(sets.data(), sc, k);
            if (it.set < 0 || it.set >= ns) {
                std::printf("phase %d item %d: set %d\n", p, k, it.set);
                return false;
            }
            const int nblk = sets[it.set].nblk, nslot = sets[it.set].nslot;
            const int slot = it.kind >> 2;
            const bool scratch = (it.kind & 2) != 0, diag = (it.kind & 1) != 0;
            if (it.I < 0 || it.I > it.J || it.J > nblk || (it.J == nblk && (nblk % 2 == 1 || it.I == it.J)) ||
                diag != (it.I == it.J)) {
                std::printf("set %d nblk %d G %d phase %d item %d: blocks %d %d kind %d\n", it.set, nblk, G, p, k,
                            it.I, it.J, it.kind);
                return false;
            }
            if (scratch != (p > 0) || (p == 0 ? slot >= nslot : (slot < nslot || slot >= 2 * nslot))) {
                std::printf("set %d nblk %d G %d phase %d item %d: slot %d scratch %d\n", it.set, nblk, G, p, k, slot,
                            scratch);
                return false;
            }
            if (it.J < nblk)
                ++seen[it.set][(size_t)it.I * (nblk + 1) + it.J];
            // the blocks whose rows this item writes: I, and J unless it is I
            // itself (diagonal) or the empty team
            const int blocks[2] = {it.I, it.J};
            const int nw = (it.I == it.J || it.J == nblk) ? 1 : 2;
            for (int q = 0; q < nw; ++q) {
                const int b = blocks[q];
                if (++written[it.set][(size_t)b * 2 * nslot + slot] != 1) {
                    std::printf("set %d nblk %d G %d phase %d: block %d slot %d written twice\n", it.set, nblk, G, p,
                                b, slot);
                    return false;
                }
            }
        }
        if (p == 0)
            for (int s = 0; s < ns; ++s)
                for (int b = 0; b < sets[s].nblk; ++b)
                    for (int q = 0; q < sets[s].nslot; ++q)
                        if (written[s][(size_t)b * 2 * sets[s].nslot + q] != 1) {
                            std::printf("set %d nblk %d G %d: block %d slot %d not written in phase 0\n", s,
                                        sets[s].nblk, G, b, q);
                            return false;
                        }
    }
    for (int s = 0; s < ns; ++s)
        for (int I = 0; I < nblks[s]; ++I)
            for (int J = I; J < nblks[s]; ++J)
                if (seen[s][(size_t)I * (nblks[s] + 1) + J] != 1) {
                    std::printf("set %d nblk %d G %d: block pair %d %d visited %d times\n", s, nblks[s], G, I, J,
                                seen[s][(size_t)I * (nblks[s] + 1) + J]);
                    return false;
                }
    return true;
}

int main()
{
    for (int nblk = 1; nblk <= 130; ++nblk)
        for (int G : {1, 2, 3, 4, 7, 16, 1 << 20})
            if (!check({nblk}, G))
                return 1;
    for (int nblk : {391, 392, 977, 1172, 1173})
        for (int G : {27, 55, 83, 1 << 20})
            if (!check({nblk}, G))
                return 1;
    // batches of uneven sets sharing each phase's launch
    for (int G : {1, 2, 3, 5, 8, 1 << 20})
        if (!check({1, 2, 7, 40, 3, 16, 1, 25}, G) || !check({97, 4, 60, 61, 2}, G))
            return 1;
    std::printf("ok\n");
    return 0;
}
