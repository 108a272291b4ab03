// C ABI of libhawkes: context, workspace, validation and the launch
// sequences of the log-likelihood, gradient, HMC and batched entry points.
//
// Every compute entry point builds a list of data sets (one for the single
// calls), lays the sets out in the context's device workspace, and enqueues
//   validate + time sort + pack   (hk_prep.cu)
//   pass 1: rate row sums         (pair kernels)
//   finalize rows, FP64 fixups, ell per set          (hk_finalize.cu)
//   pass 2: gradient row sums     (pair kernels, when a gradient is wanted)
//   finalize gradient, FP64 fixups                   (hk_finalize.cu)
// on the caller's stream without waiting for it.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "hk_internal.cuh"

using namespace hk;

namespace {

std::mutex g_create_err_mu;
std::string g_create_err;

constexpr double kLog2e = 1.4426950408889634073599246810019;
constexpr double kTwoPi = 6.283185307179586476925286766559;

// control block (int32 words): [0] status, [16..34) work/done counters of
// the pair kernel of each dimension, [40..) set flags,
// then one skip bound per set
constexpr int kCtlStatus = 0;
constexpr int kCtlDimCounters = 16;
constexpr int kCtlSetFlags = 40;

// Partial slots of the symmetric pair kernels: at most this many bytes
// (unless one slot per row is already more), and a phase of the pair
// schedule holds at least kMinPhaseItems pair blocks per SM.
constexpr double kSlotBudget = 1024.0 * 1024.0 * 1024.0;
constexpr double kMinPhaseItems = 16.0;

struct DeviceBuffer {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct Carve {
    char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

struct ProfEvent {
    cudaEvent_t a, b;
    int kernel;
    double pairs;
};

// One pair-kernel launch of a pass: runs [run0, run0 + nruns) of the plan's
// run list, nitems work items in all, of dimension d (0: every dimension),
// in phase `phase` of the pair schedule.
struct PairLaunch {
    int d, phase;
    int32_t run0, nruns, nitems;
};

// Host description of one call (a list of sets).
struct Plan {
    std::vector<SetDesc> sets;
    std::vector<ItemRun> runs;           // the pair launches' work lists
    std::vector<PairLaunch> launches;    // in phase order
    std::vector<int64_t> set_ev0;        // nsets+1
    std::vector<int64_t> set_row0;       // nsets+1
    std::vector<int> dims;               // the dimensions present
    int32_t slot_cap = 0;                // G: partial slots per row at most
    int32_t phases = 1;                  // phases of the pair schedule
    std::vector<int> wr_by_d, wc_by_d;  // pair-kernel shape per dimension: row groups, column groups (0 = per pass)
    int64_t n_total = 0, x_total = 0, total_rows = 0, total_rec4 = 0, total_P1 = 0, total_P2 = 0;
    int64_t total_F1 = 0, total_F2 = 0;
    int32_t total_segs = 0, max_fsplit = 1;
    int64_t max_ftiles = 1;
    bool fp64_sym = false;  // FP64 passes: symmetric kernels over the work items
    bool one_launch = false;  // mixed rate and gradient passes: one launch over every dimension
    double pairs = 0.0;  // unordered pairs over all sets
};

struct HmcGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> key;
};

}  // namespace

struct hawkes_ctx {
    int device = 0;
    int sm_count = 0;
    std::string err;
    int32_t *ctl = nullptr;
    int32_t ctl_sets = 0;
    DeviceBuffer ws;
    size_t ws_generation = 0;
    DeviceBuffer bmds_ws;  // BMDS partial-sum slots
    DeviceBuffer bmds_hmc;  // BMDS-Hawkes HMC: locations and BMDS gradient in the caller's order, ell_B
    DeviceBuffer bmds_ys;   // BMDS-Hawkes HMC with the fused gradient pass: Y in time order (FP32)
    // options
    int opt_warps = 0, opt_cols = 0, opt_ctas = 0, opt_profile = 0, opt_sorted = 0, opt_fixup_exp = -76, opt_skip = 0;
    int opt_fp64_ordered = 0, opt_one_launch = 0, opt_slots = 0, opt_bmds_fused = 0;
    int occ_any[3][4] = {};  // CTAs per SM of the one-launch pair kernels: [pass 1..2][log2 warps]
    std::vector<ProfEvent> prof_pending;
    static constexpr int kStages = 5;
    double prof_ms[kStages] = {};
    int64_t prof_launches[kStages] = {};
    double prof_pairs[kStages] = {};
    int64_t launches_own = 0, launches_lib = 0;
    HmcGraph hmc;
    cudaStream_t side[kMaxD + 1] = {};  // forked streams for concurrent per-dimension launches
    cudaEvent_t fork_ev = nullptr, join_ev[kMaxD + 1] = {};
    cudaStream_t bmds_side = nullptr;  // the BMDS branch of a BMDS-Hawkes leapfrog step
    cudaEvent_t bmds_fork = nullptr, bmds_join = nullptr;
    // CTAs per SM of the pair kernels: [d][pass 1..5][log2 wr][log2 wc] (-1: not yet asked)
    int occ[kMaxD + 1][6][4][4];
    static constexpr int kBuckets = 32;
    int tune_warps[kMaxD + 1][kBuckets] = {};  // row groups; 0: no entry
    int tune_cols[kMaxD + 1][kBuckets] = {};   // column groups
    int tune_ctas[kMaxD + 1][kBuckets] = {};
    int cur_ctas_by_d[kMaxD + 1] = {};         // CTA cap per dimension for the current plan
    std::vector<char> uploaded;     // bytes of the plan last copied to the device
    // workspace views of the current plan
    Work w{};
    SetDesc *d_sets = nullptr;
    ItemRun *d_runs = nullptr;
    int64_t *d_set_ev0 = nullptr, *d_set_row0 = nullptr;
    double *keys_a = nullptr, *keys_b = nullptr;
    int32_t *vals_a = nullptr, *vals_b = nullptr;
    void *sort_temp = nullptr;
    size_t sort_bytes = 0;
    // HMC state (sorted rows, stride kMaxD)
    double *hp = nullptr, *hg = nullptr, *hlo = nullptr, *hhi = nullptr;
    double *hscal = nullptr;  // per set: [0, ns) eps, [ns, 2ns) log u, [2ns, 3ns) H0, [3ns, 4ns) H1
    int32_t *hint = nullptr;  // per set: [0, ns) accepted, [ns, 2ns) reflection failure
};

namespace {

hawkes_status fail(hawkes_ctx *c, hawkes_status st, const std::string &msg)
{
    if (c)
        c->err = msg;
    return st;
}

hawkes_status cuda_fail(hawkes_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, HAWKES_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define HK_TRY(expr, where)                      \
    do {                                         \
        cudaError_t e_ = (expr);                 \
        if (e_ != cudaSuccess)                   \
            return cuda_fail(ctx, e_, where);    \
    } while (0)

bool params_ok(const hawkes_params *p)
{
    const double v[6] = {p->mu0, p->tau_x, p->tau_t, p->theta, p->omega, p->h};
    for (double x : v)
        if (!(x > 0.0) || !std::isfinite(x))
            return false;
    return true;
}

// Warps per CTA of the pair kernels for a set of n events in d dimensions:
// the largest count that still gives every SM slot several pair blocks.
int size_bucket(int64_t n)
{
    int b = 0;
    while (((int64_t)1 << b) < n && b < 31)
        ++b;
    return b;
}

int ilog2_small(int v) { return v >= 8 ? 3 : v >= 4 ? 2 : v >= 2 ? 1 : 0; }

// CTAs of shape (wr, wc) that fit on one SM for pass `pass` in d dimensions
// (asked from the runtime once, then cached; 0 if the shape does not fit).
int occupancy(hawkes_ctx *ctx, int d, int pass, int wr, int wc)
{
    int &o = ctx->occ[d][pass][ilog2_small(wr)][ilog2_small(wc)];
    if (o < 0)
        o = pass_max_ctas_per_sm(d, pass, wr, wc);
    return o;
}

// A shape (wr row groups, wc column groups) is valid when it has at most 8
// warps, every column group sweeps whole 32-column chunks, and its shared
// memory lets it run (and, without `tuned`, leaves room for two CTAs per SM).
bool shape_ok(hawkes_ctx *ctx, int d, int wr, int wc, bool theta, size_t smem_cap)
{
    if (wr * wc > 8 || wc > 4 || wc > rows_per_lane(d) * wr)
        return false;
    if (pass_smem_bytes(d, 2, wr, wc) > smem_cap || (theta && pass_smem_bytes(d, 3, wr, wc) > smem_cap))
        return false;
    return occupancy(ctx, d, 2, wr, wc) > 0 && (!theta || occupancy(ctx, d, 3, wr, wc) > 0);
}

// Pair-kernel shape for sets of up to n events in d dimensions: row groups
// (the block size B = 32 rows_per_lane(d) wr is the largest that still gives
// every SM several pair blocks, at least three per SM in all) and column
// groups (0: chosen per pass by pass_cols).  An explicit option, or a tuned
// entry that still gives three blocks per SM at this size, takes precedence.
void choose_shape(hawkes_ctx *ctx, int64_t n, int d, bool theta, int &wr_out, int &wc_out)
{
    const int R = rows_per_lane(d);
    auto items_for = [&](int wv) {
        const int64_t B = 32LL * R * wv;
        const int64_t T = (n + B - 1) / B;
        return T * (T + 1) / 2;
    };
    wc_out = ctx->opt_cols;
    if (ctx->opt_warps > 0) {
        wr_out = ctx->opt_warps;
        return;
    }
    const int tw = ctx->tune_warps[d][size_bucket(n)], tc = ctx->tune_cols[d][size_bucket(n)];
    if (tw > 0 && shape_ok(ctx, d, tw, std::max(1, tc), theta, 200 * 1024) && items_for(tw) >= 3LL * ctx->sm_count) {
        wr_out = tw;
        if (wc_out == 0)
            wc_out = tc;
        return;
    }
    for (int wv : {8, 4, 2, 1}) {
        if (!shape_ok(ctx, d, wv, 1, theta, 110 * 1024))
            continue;
        if (items_for(wv) >= 3LL * ctx->sm_count || wv == 1) {
            wr_out = wv;
            return;
        }
    }
    wr_out = 1;
}

// Column groups of one pair pass with wr row groups over nitems blocks: the
// most (1, 2 or 4; only the rate and gradient passes split columns) that
// keep the warp tasks (blocks x warps) within 48 per SM.  At small N this
// gives the SMs more warps than one warp row per block would (at N = 1e4,
// D = 2 both passes measured fastest with four); at large N the blocks alone
// fill the SMs and the row groups already take all eight warps.
int pass_cols(hawkes_ctx *ctx, int d, int pass, int wr, int64_t nitems)
{
    if (pass != 1 && pass != 2)
        return 1;
    int best = 1;
    for (int wc = 2; wc <= 4; wc *= 2)
        if (shape_ok(ctx, d, wr, wc, false, 110 * 1024) && occupancy(ctx, d, pass, wr, wc) > 0 &&
            nitems * wr * wc <= 48LL * ctx->sm_count)
            best = wc;
    return best;
}

// Fill the derived fields of one set.
void describe_set(SetDesc &S, int64_t n, int d, const hawkes_params &p, double fixup_exp)
{
    S.n = (int32_t)n;
    S.d = d;
    S.mu0 = p.mu0;
    S.tau_x = p.tau_x;
    S.tau_t = p.tau_t;
    S.theta = p.theta;
    S.omega = p.omega;
    S.h = p.h;
    const double k0 = std::sqrt(kLog2e / 2.0);
    S.kx = k0 / p.tau_x;
    S.kt = k0 / p.tau_t;
    S.Pmu = p.mu0 / (std::pow(p.tau_x, d) * p.tau_t * std::pow(kTwoPi, 0.5 * (d + 1)));
    S.iPmu = 1.0 / S.Pmu;
    S.lPmu = std::log(S.Pmu);
    S.Cg = 1.0 / (p.tau_x * p.tau_x * S.kx);
    const double rho = (p.tau_x * p.tau_x) / (p.h * p.h);
    const double cxi1 = std::log2(p.theta * p.omega * std::pow(p.tau_x, d) * p.tau_t * std::sqrt(kTwoPi) /
                                  (p.mu0 * std::pow(p.h, d)));
    S.rho = (float)rho;
    const double kappa = p.omega * kLog2e / S.kt;
    S.kappa = (float)kappa;
    S.kappa_lo = (float)(kappa - (double)S.kappa);
    S.cxi1 = (float)cxi1;
    S.cxi1_lo = (float)(cxi1 - (double)S.cxi1);
    S.bq = (float)(1.0 / (S.kx * S.kx));
    S.bc = (float)(p.tau_x * p.tau_x);
    S.cxi2 = (float)(cxi1 + std::log2(rho));
    S.cxi2_d = cxi1 + std::log2(rho);
    S.s_min = std::ldexp(1.0, (int)fixup_exp);
}

bool mixed_range_ok(const SetDesc &S)
{
    return std::isfinite(S.cxi1) && std::isfinite(S.cxi2) && std::fabs(S.cxi1) < 64.0f &&
           std::fabs(S.cxi2) < 64.0f && S.rho < 1e30f && S.rho > 1e-30f && S.kappa < 1e30f;
}

// Lay out the sets of one call and build the work list.
hawkes_status build_plan(hawkes_ctx *ctx, Plan &pl, int32_t nsets, const int64_t *ev_counts, const int32_t *dims,
                         const hawkes_params *params, bool fp64, bool theta = false, bool xi = false)
{
    pl = Plan();
    pl.sets.resize(nsets);
    pl.set_ev0.resize(nsets + 1);
    pl.set_row0.resize(nsets + 1);
    pl.wr_by_d.assign(kMaxD + 1, 0);
    pl.wc_by_d.assign(kMaxD + 1, 0);
    // the block size is chosen per dimension from the largest set of that dimension
    std::vector<int64_t> nmax_by_d(kMaxD + 1, 0);
    for (int s = 0; s < nsets; ++s)
        nmax_by_d[dims[s]] = std::max(nmax_by_d[dims[s]], ev_counts[s]);
    for (int d = 1; d <= kMaxD; ++d)
        if (nmax_by_d[d] > 0) {
            pl.dims.push_back(d);
            choose_shape(ctx, nmax_by_d[d], d, theta, pl.wr_by_d[d], pl.wc_by_d[d]);
            ctx->cur_ctas_by_d[d] = ctx->tune_ctas[d][size_bucket(nmax_by_d[d])];
        }
    // One launch over every dimension (an option): all dimensions take the
    // row groups of the one with the most pair work, and one column group.
    pl.one_launch = !fp64 && !theta && !xi && ctx->opt_one_launch && pl.dims.size() > 1;
    if (pl.one_launch) {
        std::vector<double> work_by_d(kMaxD + 1, 0.0);
        for (int s = 0; s < nsets; ++s)
            work_by_d[dims[s]] += (double)ev_counts[s] * (double)ev_counts[s] * (6 * dims[s] + 19);
        const int heavy = (int)(std::max_element(work_by_d.begin(), work_by_d.end()) - work_by_d.begin());
        for (int d = 1; d <= kMaxD; ++d)
            if (nmax_by_d[d] > 0) {
                pl.wr_by_d[d] = pl.wr_by_d[heavy];
                pl.wc_by_d[d] = 1;
            }
    }
    pl.fp64_sym = fp64 && ctx->opt_fp64_ordered == 0;
    const bool sym = !fp64 || pl.fp64_sym;  // the symmetric pair kernels and their schedule
    auto block_rows = [&](int d) {
        return fp64 ? (pl.fp64_sym ? kSymRows : kFp64Rows) : 32 * rows_per_lane(d) * pl.wr_by_d[d];
    };
    const int vpc = theta ? kPass1ThetaVals : (xi ? kPass1XiVals : kPass1Vals);
    // Slot cap G of the pair schedule: every round its own slot while all
    // slots fit kSlotBudget bytes; beyond it as many as fit beside as many
    // scratch slots, but at least enough that a phase holds kMinPhaseItems
    // pair blocks per SM.
    if (sym) {
        double per_slot = 0.0, full = 0.0, per_round = 0.0;
        int32_t nt_max = 1;
        for (int s = 0; s < nsets; ++s) {
            const int d = dims[s], B = block_rows(d);
            const int64_t nblk = (ev_counts[s] + B - 1) / B, nt = nblk | 1;
            const double bytes = (double)(nblk * B) * (fp64 ? (kPass1ThetaVals + d) * 8.0 : (vpc + d) * 4.0);
            per_slot += bytes;
            full += (double)nt * bytes;
            per_round += (double)((nt + 1) / 2);
            nt_max = std::max<int32_t>(nt_max, (int32_t)nt);
        }
        int64_t G = nt_max;
        if (ctx->opt_slots > 0) {
            G = ctx->opt_slots;
        } else if (full > kSlotBudget) {
            const int64_t g_fit = (int64_t)(kSlotBudget / std::max(2.0 * per_slot, 1.0));
            const int64_t g_par = (int64_t)std::ceil(kMinPhaseItems * ctx->sm_count / std::max(per_round, 1.0));
            G = std::max<int64_t>(1, std::max(g_fit, g_par));
        }
        pl.slot_cap = (int32_t)std::min<int64_t>(G, nt_max);
    }
    int64_t ev = 0, x = 0, row = 0, rec4 = 0, p1 = 0, p2 = 0, f1 = 0, f2 = 0;
    int32_t seg = 0;
    for (int s = 0; s < nsets; ++s) {
        SetDesc &S = pl.sets[s];
        std::memset(&S, 0, sizeof(S));
        const int d = dims[s];
        const int64_t n = ev_counts[s];
        describe_set(S, n, d, params[s], ctx->opt_fixup_exp);
        if (!fp64 && !mixed_range_ok(S))
            return fail(ctx, HAWKES_ERR_INVALID_ARG,
                        "parameters outside the range of the mixed-precision path; use HAWKES_PREC_FP64");
        const int B = block_rows(d);
        S.B = B;
        S.nblk = (int32_t)((n + B - 1) / B);
        S.npad = S.nblk * B;
        S.nslot = sym ? std::min(S.nblk | 1, pl.slot_cap) : 0;
        S.ev0 = ev;
        S.x0 = x;
        S.row0 = row;
        S.rec0 = rec4;
        S.part0 = p1;
        S.part2_0 = p2;
        S.fpart0 = f1;
        S.fpart2_0 = f2;
        S.vpc = vpc;
        S.seg0 = seg;
        S.nseg = (int32_t)((n + kFinalizeThreads - 1) / kFinalizeThreads);
        // FP64 kernels: enough column splits for about 8 CTAs per SM in total
        const int64_t ftiles = (n + kFp64Rows - 1) / kFp64Rows;
        int64_t fs = std::max<int64_t>(1, (8LL * ctx->sm_count) / std::max<int64_t>(1, ftiles * nsets));
        fs = std::min<int64_t>(fs, ftiles);
        S.fsplit = pl.fp64_sym ? S.nslot : (int32_t)std::max<int64_t>(1, fs);
        pl.max_fsplit = std::max(pl.max_fsplit, S.fsplit);
        pl.max_ftiles = std::max(pl.max_ftiles, ftiles);
        ev += n;
        x += n * d;
        row += S.npad;
        rec4 += (int64_t)nrec(d) * S.npad;
        // partial slots: FP32 for the mixed path, FP64 for the FP64 path
        // (with later phases of the pair schedule, nslot scratch slots too)
        int64_t nalloc = fp64 ? S.fsplit : S.nslot;
        if (sym && (S.nblk | 1) > S.nslot)
            nalloc = 2 * S.nslot;
        if (!fp64) {
            p1 += nalloc * S.npad * S.vpc;
            p2 += nalloc * S.npad * d;
        } else {
            f1 += nalloc * S.npad * kPass1ThetaVals;
            f2 += nalloc * S.npad * d;
        }
        seg += S.nseg;
        pl.pairs += 0.5 * (double)n * (double)(n - 1);
    }
    pl.n_total = ev;
    pl.x_total = x;
    pl.total_rows = row;
    pl.total_rec4 = rec4;
    pl.total_P1 = p1;
    pl.total_P2 = p2;
    pl.total_F1 = f1;
    pl.total_F2 = f2;
    pl.total_segs = seg;
    for (int s = 0; s <= nsets; ++s) {
        pl.set_ev0[s] = s < nsets ? pl.sets[s].ev0 : ev;
        pl.set_row0[s] = s < nsets ? pl.sets[s].row0 : row;
    }
    if (!sym)
        return HAWKES_OK;
    // Work lists of the pair launches, phase by phase: per dimension (or,
    // with one launch, over the dimensions in order of decreasing cost per
    // block, B^2 (6D + 19)), the off-diagonal blocks of every set's rounds
    // in the phase, then their diagonal blocks (half the work), so that the
    // last blocks of a launch are small.
    std::vector<int> order = pl.dims;
    if (pl.one_launch) {
        auto block_cost = [&](int d) {
            const double B = 32.0 * rows_per_lane(d) * pl.wr_by_d[d];
            return B * B * (6 * d + 19);
        };
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return block_cost(a) > block_cost(b); });
    }
    int32_t phases = 0;
    for (int s = 0; s < nsets; ++s) {
        const SetDesc &S = pl.sets[s];
        phases = std::max(phases, ((S.nblk | 1) + S.nslot - 1) / S.nslot);
    }
    pl.phases = phases;
    int64_t first = 0;
    bool overflow = false;
    auto add_runs = [&](int d, int phase, bool diag) {
        for (int s = 0; s < nsets; ++s) {
            const SetDesc &S = pl.sets[s];
            if (S.d != d)
                continue;
            append_set_run(s, S.nblk, S.nslot, phase, diag, pl.runs, first);
            overflow = overflow || first > INT32_MAX;
        }
    };
    auto close_launch = [&](int d, int phase, size_t run0) {
        if (first > 0)
            pl.launches.push_back({d, phase, (int32_t)run0, (int32_t)(pl.runs.size() - run0), (int32_t)first});
        else
            pl.runs.resize(run0);
        first = 0;
    };
    for (int p = 0; p < phases; ++p) {
        if (pl.one_launch) {
            const size_t run0 = pl.runs.size();
            for (int diag = 0; diag < 2; ++diag)
                for (int d : order)
                    add_runs(d, p, diag != 0);
            close_launch(0, p, run0);
        } else {
            for (int d : order) {
                const size_t run0 = pl.runs.size();
                add_runs(d, p, false);
                add_runs(d, p, true);
                close_launch(d, p, run0);
            }
        }
    }
    if (overflow)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "too many pair blocks in one launch");
    return HAWKES_OK;
}

size_t plan_bytes(const Plan &pl, size_t sort_bytes)
{
    Carve c{nullptr};
    const size_t ns = pl.sets.size();
    c.take<SetDesc>(ns);
    c.take<ItemRun>(std::max<size_t>(1, pl.runs.size()));
    c.take<int64_t>(ns + 1);
    c.take<int64_t>(ns + 1);
    c.take<float4>(pl.total_rec4);
    c.take<float>(pl.total_rows);
    c.take<float>(pl.total_rows);
    c.take<int32_t>(pl.total_rows);
    c.take<int32_t>(pl.total_rows);
    for (int k = 0; k < 5; ++k)
        c.take<double>(pl.total_rows);
    c.take<double>(pl.total_rows * kMaxD);
    c.take<double>(pl.total_rows * kPass1ThetaVals);
    c.take<float>(pl.total_P1);
    c.take<float>(pl.total_P2);
    c.take<double>(pl.total_F1);
    c.take<double>(pl.total_F2);
    c.take<int32_t>(pl.total_segs);
    c.take<int32_t>((size_t)pl.total_segs * kFinalizeThreads);
    c.take<double>(pl.total_segs);
    c.take<double>((size_t)kThetaParts * kPass1ThetaVals);
    c.take<double>(ns);
    c.take<double>(pl.n_total);
    c.take<double>(pl.n_total);
    c.take<int32_t>(pl.n_total);
    c.take<int32_t>(pl.n_total);
    c.take<char>(sort_bytes);
    for (int k = 0; k < 4; ++k)
        c.take<double>(pl.total_rows * kMaxD);
    c.take<double>((4 + kEnergyParts) * ns + 8);
    c.take<int32_t>(2 * ns + 8);
    c.take<int32_t>(ns);
    return c.off + 256;
}

// Make the workspace large enough for the plan and point the views at it.
hawkes_status bind_plan(hawkes_ctx *ctx, const Plan &pl, cudaStream_t stream)
{
    const size_t ns = pl.sets.size();
    const size_t sort_bytes = std::max<size_t>(256, sort_temp_bytes(pl.n_total, (int32_t)ns));
    const size_t need = plan_bytes(pl, sort_bytes);
    if (need > ctx->ws.bytes) {
        HK_TRY(cudaDeviceSynchronize(), "synchronize before growing the workspace");
        if (ctx->ws.ptr)
            cudaFree(ctx->ws.ptr);
        ctx->ws.ptr = nullptr;
        ctx->ws.bytes = 0;
        const size_t bytes = need + need / 4;
        if (cudaMalloc(&ctx->ws.ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, HAWKES_ERR_OOM, "device workspace of " + std::to_string(bytes) + " bytes");
        }
        ctx->ws.bytes = bytes;
        ++ctx->ws_generation;
    }
    if ((int32_t)ns > ctx->ctl_sets) {
        HK_TRY(cudaDeviceSynchronize(), "synchronize before growing the control block");
        int32_t *ctl = nullptr;
        const int32_t cap = (int32_t)std::max<size_t>(ns, 64);
        HK_TRY(cudaMalloc(&ctl, sizeof(int32_t) * (kCtlSetFlags + 2 * cap)), "control block");
        HK_TRY(cudaMemset(ctl, 0, sizeof(int32_t) * (kCtlSetFlags + 2 * cap)), "control block");
        if (ctx->ctl) {
            HK_TRY(cudaMemcpy(ctl, ctx->ctl, sizeof(int32_t) * kCtlSetFlags, cudaMemcpyDeviceToDevice), "control");
            cudaFree(ctx->ctl);
        }
        ctx->ctl = ctl;
        ctx->ctl_sets = cap;
        ++ctx->ws_generation;
    }
    Carve c{reinterpret_cast<char *>(ctx->ws.ptr)};
    Work &w = ctx->w;
    ctx->d_sets = c.take<SetDesc>(ns);
    ctx->d_runs = c.take<ItemRun>(std::max<size_t>(1, pl.runs.size()));
    ctx->d_set_ev0 = c.take<int64_t>(ns + 1);
    ctx->d_set_row0 = c.take<int64_t>(ns + 1);
    w.sets = ctx->d_sets;
    w.nsets = (int32_t)ns;
    w.rec = c.take<float4>(pl.total_rec4);
    w.w32 = c.take<float>(pl.total_rows);
    w.cm32 = c.take<float>(pl.total_rows);
    w.tie_end = c.take<int32_t>(pl.total_rows);
    w.perm = c.take<int32_t>(pl.total_rows);
    w.t64 = c.take<double>(pl.total_rows);
    w.lam64 = c.take<double>(pl.total_rows);
    w.w64 = c.take<double>(pl.total_rows);
    w.Lam64 = c.take<double>(pl.total_rows);
    w.lnl = c.take<double>(pl.total_rows);
    w.x64 = c.take<double>(pl.total_rows * kMaxD);
    w.theta_rows = c.take<double>(pl.total_rows * kPass1ThetaVals);
    w.P1 = c.take<float>(pl.total_P1);
    w.P2 = c.take<float>(pl.total_P2);
    w.F1 = c.take<double>(pl.total_F1);
    w.F2 = c.take<double>(pl.total_F2);
    w.seg_count = c.take<int32_t>(pl.total_segs);
    w.seg_rows = c.take<int32_t>((size_t)pl.total_segs * kFinalizeThreads);
    w.seg_sum = c.take<double>(pl.total_segs);
    w.theta_parts = c.take<double>((size_t)kThetaParts * kPass1ThetaVals);
    w.set_loglik = c.take<double>(ns);
    ctx->keys_a = c.take<double>(pl.n_total);
    ctx->keys_b = c.take<double>(pl.n_total);
    ctx->vals_a = c.take<int32_t>(pl.n_total);
    ctx->vals_b = c.take<int32_t>(pl.n_total);
    ctx->sort_temp = c.take<char>(sort_bytes);
    ctx->sort_bytes = sort_bytes;
    ctx->hp = c.take<double>(pl.total_rows * kMaxD);
    ctx->hg = c.take<double>(pl.total_rows * kMaxD);
    ctx->hlo = c.take<double>(pl.total_rows * kMaxD);
    ctx->hhi = c.take<double>(pl.total_rows * kMaxD);
    ctx->hscal = c.take<double>((4 + kEnergyParts) * ns + 8);
    ctx->hint = c.take<int32_t>(2 * ns + 8);
    w.set_done = c.take<int32_t>(ns);
    w.sm_count = ctx->sm_count;
    w.set_flags = ctx->ctl + kCtlSetFlags;
    w.set_cmmax = ctx->ctl + kCtlSetFlags + ctx->ctl_sets;
    w.skip_far = ctx->opt_skip;
    w.status = reinterpret_cast<unsigned *>(ctx->ctl + kCtlStatus);
    // Upload the plan, unless the device already holds exactly this plan at
    // these addresses.  Copies from pageable memory are staged before the
    // call returns, so the host vectors may go away afterwards.
    std::vector<char> bytes;
    auto append = [&bytes](const void *p, size_t n) {
        const char *c = static_cast<const char *>(p);
        bytes.insert(bytes.end(), c, c + n);
    };
    append(&ctx->ws_generation, sizeof(ctx->ws_generation));
    append(&ctx->ws.ptr, sizeof(void *));
    append(pl.sets.data(), sizeof(SetDesc) * ns);
    append(pl.runs.data(), sizeof(ItemRun) * pl.runs.size());
    append(pl.set_ev0.data(), sizeof(int64_t) * (ns + 1));
    append(pl.set_row0.data(), sizeof(int64_t) * (ns + 1));
    if (bytes == ctx->uploaded)
        return HAWKES_OK;
    ctx->uploaded.swap(bytes);
    // the per-set segment tickets start at zero and every evaluation leaves
    // them at zero; a new layout clears them once
    HK_TRY(cudaMemsetAsync(w.set_done, 0, sizeof(int32_t) * ns, stream), "clear tickets");
    HK_TRY(cudaMemcpyAsync(ctx->d_sets, pl.sets.data(), sizeof(SetDesc) * ns, cudaMemcpyHostToDevice, stream),
           "upload set descriptors");
    if (!pl.runs.empty())
        HK_TRY(cudaMemcpyAsync(ctx->d_runs, pl.runs.data(), sizeof(ItemRun) * pl.runs.size(),
                               cudaMemcpyHostToDevice, stream),
               "upload work lists");
    HK_TRY(cudaMemcpyAsync(ctx->d_set_ev0, pl.set_ev0.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice,
                           stream),
           "upload set offsets");
    HK_TRY(cudaMemcpyAsync(ctx->d_set_row0, pl.set_row0.data(), sizeof(int64_t) * (ns + 1),
                           cudaMemcpyHostToDevice, stream),
           "upload set rows");
    return HAWKES_OK;
}

int persistent_grid(hawkes_ctx *ctx, int d, int pass, int wr, int wc, int nitems)
{
    int per_sm = occupancy(ctx, d, pass, wr, wc);
    if (ctx->opt_ctas > 0)
        per_sm = std::min(per_sm, ctx->opt_ctas);
    else if (ctx->cur_ctas_by_d[d] > 0)
        per_sm = std::min(per_sm, ctx->cur_ctas_by_d[d]);
    per_sm = std::max(per_sm, 1);
    return std::max(1, std::min(nitems, per_sm * ctx->sm_count));
}

void prof_begin(hawkes_ctx *ctx, cudaStream_t s, ProfEvent &pe, int kernel, double pairs)
{
    pe.kernel = kernel;
    pe.pairs = pairs;
    cudaEventCreate(&pe.a);
    cudaEventCreate(&pe.b);
    cudaEventRecord(pe.a, s);
}

void prof_end(hawkes_ctx *ctx, cudaStream_t s, ProfEvent &pe)
{
    cudaEventRecord(pe.b, s);
    ctx->prof_pending.push_back(pe);
}

// Validate, sort by time and pack every set of the plan.
hawkes_status enqueue_prep(hawkes_ctx *ctx, const Plan &pl, const double *t, const double *X, cudaStream_t s)
{
    Work &w = ctx->w;
    const int32_t ns = (int32_t)pl.sets.size();
    ProfEvent pe{};
    if (ctx->opt_profile)
        prof_begin(ctx, s, pe, 2, 0.0);
    // per-evaluation control words: the pair kernels' work counters (zero
    // after every launch; cleared here as well), the set flags and bounds
    HK_TRY(cudaMemsetAsync(ctx->ctl + kCtlDimCounters, 0, sizeof(int32_t) * (kCtlSetFlags - kCtlDimCounters + ns), s),
           "reset control words");
    HK_TRY(cudaMemsetAsync(ctx->ctl + kCtlSetFlags + ctx->ctl_sets, 0, sizeof(int32_t) * ns, s), "reset bounds");
    HK_TRY(launch_validate_keys(t, X, pl.n_total, pl.x_total, ctx->keys_a, ctx->vals_a, ctx->d_set_ev0, ns,
                                w.status, s),
           "validate");
    ctx->launches_own += 2;  // validate, pack
    ctx->launches_own += ctx->opt_sorted ? 1 : 0;
    if (ctx->opt_sorted) {
        HK_TRY(launch_identity_order(t, ctx->keys_b, ctx->vals_b, pl.n_total, ctx->d_set_ev0, ns, w.status, s),
               "order check");
    } else {
        HK_TRY(launch_sort(ctx->sort_temp, ctx->sort_bytes, t, ctx->keys_a, ctx->keys_b, ctx->vals_a, ctx->vals_b,
                           pl.n_total, ns, ctx->d_set_ev0, s, &ctx->launches_own, &ctx->launches_lib),
               "time sort");
    }
    HK_TRY(launch_pack_rows(w, X, ctx->keys_b, ctx->vals_b, pl.total_rows, ctx->d_set_row0, s), "pack");
    // a pair schedule with later phases starts with cleared scratch slots
    // (each fold clears them again)
    if (pl.phases > 1) {
        HK_TRY(cudaMemsetAsync(w.P1, 0, sizeof(float) * pl.total_P1, s), "clear slots");
        HK_TRY(cudaMemsetAsync(w.P2, 0, sizeof(float) * pl.total_P2, s), "clear slots");
        HK_TRY(cudaMemsetAsync(w.F1, 0, sizeof(double) * pl.total_F1, s), "clear slots");
        HK_TRY(cudaMemsetAsync(w.F2, 0, sizeof(double) * pl.total_F2, s), "clear slots");
    }
    if (ctx->opt_profile)
        prof_end(ctx, s, pe);
    return HAWKES_OK;
}

// One pair pass (1 rates, 2 gradient, 3 rates with Theta sums, 4 rates with
// the self-excitation sums apart) over every dimension of the plan: the
// plan's pair launches in phase order, each of a later phase followed by a
// fold of its scratch slots.  Each pair launch is persistent with its own
// work counter; with several dimensions each dimension's launches run on its
// own forked stream (joined back into s), so that the GPU fills one
// dimension's tail with another's blocks, while its phases stay in order.
hawkes_status enqueue_pair_pass(hawkes_ctx *ctx, const Plan &pl, int pass, cudaStream_t s)
{
    const int fold_part = pass == 2 || pass == 5 ? 1 : 0;
    if (pl.one_launch && (pass == 1 || pass == 2)) {
        int warps = 1;
        for (int d : pl.dims)
            warps = std::max(warps, pl.wr_by_d[d]);
        int per_sm = ctx->occ_any[pass][ilog2_small(warps)];
        if (ctx->opt_ctas > 0)
            per_sm = std::min(per_sm, ctx->opt_ctas);
        Work wd = ctx->w;
        wd.pair_ctr = ctx->ctl + kCtlDimCounters;  // the slot of dimension 0 (unused otherwise)
        for (const PairLaunch &L : pl.launches) {
            const Sched sc{ctx->d_runs + L.run0, L.nruns, L.nitems};
            const int grid = std::max(1, std::min(L.nitems, std::max(per_sm, 1) * ctx->sm_count));
            HK_TRY(launch_pair_pass_any_d(pass, wd, sc, grid, warps, s), pass == 2 ? "gradient pass" : "rate pass");
            if (L.phase > 0)
                HK_TRY(launch_fold_slots(ctx->w, sc, fold_part, s), "fold slots");
        }
        return HAWKES_OK;
    }
    const bool fork = pl.dims.size() > 1;
    if (fork) {
        if (!ctx->fork_ev) {
            HK_TRY(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming), "fork event");
            for (int d = 1; d <= kMaxD; ++d) {
                HK_TRY(cudaStreamCreateWithFlags(&ctx->side[d], cudaStreamNonBlocking), "side stream");
                HK_TRY(cudaEventCreateWithFlags(&ctx->join_ev[d], cudaEventDisableTiming), "join event");
            }
        }
        HK_TRY(cudaEventRecord(ctx->fork_ev, s), "fork");
        for (int d : pl.dims)
            HK_TRY(cudaStreamWaitEvent(ctx->side[d], ctx->fork_ev, 0), "fork wait");
    }
    for (const PairLaunch &L : pl.launches) {
        const int d = L.d;
        const int wr = pl.wr_by_d[d];
        const int wc = (pass == 1 || pass == 2) && pl.wc_by_d[d] > 0 ? pl.wc_by_d[d]
                                                                      : pass_cols(ctx, d, pass, wr, L.nitems);
        const int grid = persistent_grid(ctx, d, pass, wr, wc, L.nitems);
        Work wd = ctx->w;
        wd.pair_ctr = ctx->ctl + kCtlDimCounters + 2 * d;  // [0] work taken, [1] CTAs done
        const Sched sc{ctx->d_runs + L.run0, L.nruns, L.nitems};
        cudaStream_t ls = fork ? ctx->side[d] : s;
        HK_TRY(launch_pair_pass_mixed(pass, d, wd, sc, grid, wr, wc, ls),
               pass == 2 || pass == 5 ? "gradient pass" : "rate pass");
        if (L.phase > 0)
            HK_TRY(launch_fold_slots(ctx->w, sc, fold_part, ls), "fold slots");
    }
    if (fork)
        for (int d : pl.dims) {
            HK_TRY(cudaEventRecord(ctx->join_ev[d], ctx->side[d]), "join");
            HK_TRY(cudaStreamWaitEvent(s, ctx->join_ev[d], 0), "join wait");
        }
    return HAWKES_OK;
}

// Kernel launches one pair pass makes: the plan's pair launches and a fold
// after each of a later phase (the symmetric kernels), or one (the ordered
// FP64 kernels).
int pass_launches(const Plan &pl)
{
    if (pl.launches.empty())
        return 1;
    int k = 0;
    for (const PairLaunch &L : pl.launches)
        k += L.phase > 0 ? 2 : 1;
    return k;
}

// One FP64 pair pass (1: rates, with the Theta sums when theta; 2: gradient):
// the symmetric kernels over the plan's pair launches (with the folds of the
// later phases), or the ordered kernels over all sets.
hawkes_status enqueue_fp64_pass(hawkes_ctx *ctx, const Plan &pl, int pass, bool theta, cudaStream_t s)
{
    const Work &w = ctx->w;
    const int32_t ns = (int32_t)pl.sets.size();
    if (!pl.fp64_sym) {
        if (pass == 1)
            HK_TRY(launch_pass1_fp64(w, 0, ns, pl.max_fsplit, pl.max_ftiles, theta, s), "FP64 rate pass");
        else
            HK_TRY(launch_pass2_fp64(w, 0, ns, pl.max_fsplit, pl.max_ftiles, s), "FP64 gradient pass");
        return HAWKES_OK;
    }
    for (const PairLaunch &L : pl.launches) {
        const Sched sc{ctx->d_runs + L.run0, L.nruns, L.nitems};
        if (pass == 1)
            HK_TRY(launch_pass1_fp64_sym(L.d, w, sc, theta, s), "FP64 rate pass");
        else
            HK_TRY(launch_pass2_fp64_sym(L.d, w, sc, s), "FP64 gradient pass");
        if (L.phase > 0)
            HK_TRY(launch_fold_slots(w, sc, pass == 2 ? 4 : (theta ? 3 : 2), s), "fold slots");
    }
    return HAWKES_OK;
}

// Pass 1 .. ell (and pass 2 .. gradient) on packed rows:
//   rate pass (with the six Theta sums when wanted), finalize rows (rates,
//   FP64 recompute of flagged rows, ell per set), Theta gradient, gradient
//   pass (grad_pass 5: with the BMDS term), finalize gradient.
hawkes_status enqueue_eval(hawkes_ctx *ctx, const Plan &pl, bool fp64, bool want_grad, double *out_loglik,
                           double *out_grad, double *g_sorted, cudaStream_t s, double *out_grad_params = nullptr,
                           int grad_pass = 2, bool ell = true)
{
    const bool theta = out_grad_params != nullptr;
    Work &w = ctx->w;
    ctx->launches_own += (want_grad ? 2 : 1) * (pass_launches(pl) + 1) + (theta ? 2 : 0);
    hawkes_status st;
    {
        ProfEvent pe{};
        if (ctx->opt_profile)
            prof_begin(ctx, s, pe, 0, pl.pairs);
        st = fp64 ? enqueue_fp64_pass(ctx, pl, 1, theta, s) : enqueue_pair_pass(ctx, pl, theta ? 3 : 1, s);
        if (st != HAWKES_OK)
            return st;
        if (ctx->opt_profile)
            prof_end(ctx, s, pe);
    }
    {
        ProfEvent pf{};
        if (ctx->opt_profile)
            prof_begin(ctx, s, pf, 3, 0.0);
        HK_TRY(launch_finalize_rows(w, pl.total_segs, fp64, theta ? kSumsTheta : kSumsNone, out_loglik, s, ell),
               "finalize rows");
        if (ctx->opt_profile)
            prof_end(ctx, s, pf);
    }
    if (theta)
        HK_TRY(launch_theta_grad(w, pl.n_total, out_grad_params, s), "parameter gradient");
    if (!want_grad)
        return HAWKES_OK;
    {
        ProfEvent pe{};
        if (ctx->opt_profile)
            prof_begin(ctx, s, pe, 1, pl.pairs);
        st = fp64 ? enqueue_fp64_pass(ctx, pl, 2, false, s) : enqueue_pair_pass(ctx, pl, grad_pass, s);
        if (st != HAWKES_OK)
            return st;
        if (ctx->opt_profile)
            prof_end(ctx, s, pe);
    }
    ProfEvent pg{};
    if (ctx->opt_profile)
        prof_begin(ctx, s, pg, 4, 0.0);
    HK_TRY(launch_finalize_grad(w, pl.total_segs, fp64, out_grad, g_sorted, s), "finalize gradient");
    if (ctx->opt_profile)
        prof_end(ctx, s, pg);
    return HAWKES_OK;
}

__global__ void nan_on_invalid_kernel(const unsigned *status, double *a, int64_t na, double *b, int64_t nb)
{
    if ((*status & kStInvalidData) == 0)
        return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < na)
            a[i] = nan("");
        else
            b[i - na] = nan("");
    }
}

hawkes_status enqueue_nan_on_invalid(hawkes_ctx *ctx, double *a, int64_t na, double *b, int64_t nb,
                                     cudaStream_t s)
{
    if (!a)
        na = 0;
    if (!b)
        nb = 0;
    if (na + nb == 0)
        return HAWKES_OK;
    int grid = (int)std::min<int64_t>(1024, (na + nb + 255) / 256);
    ++ctx->launches_own;
    nan_on_invalid_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<unsigned *>(ctx->ctl + kCtlStatus), a, na, b, nb);
    HK_TRY(cudaGetLastError(), "NaN fill");
    return HAWKES_OK;
}

hawkes_status check_common(hawkes_ctx *ctx, const void *t, const void *X, int64_t n, int32_t d,
                           const hawkes_params *params, hawkes_precision prec)
{
    if (!ctx)
        return HAWKES_ERR_INVALID_ARG;
    if (!t || !X)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "t and X must be device pointers");
    if (n < 1 || n > (int64_t)1 << 30)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "n must be in [1, 2^30]");
    if (d < 1 || d > kMaxD)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "d must be in [1, 8]");
    if (!params || !params_ok(params))
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "every parameter must be finite and > 0");
    if (prec != HAWKES_PREC_MIXED && prec != HAWKES_PREC_FP64)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "unknown precision");
    return HAWKES_OK;
}

}  // namespace

// ================================================================ C ABI ==

extern "C" {

const char *hawkes_version(void) { return "hawkes 0.1.0 sm_103a"; }

hawkes_status hawkes_ctx_create(hawkes_ctx **out, int32_t device, int64_t max_n, int32_t max_d)
{
    auto set_err = [](const std::string &m) {
        std::lock_guard<std::mutex> g(g_create_err_mu);
        g_create_err = m;
    };
    if (!out || max_n < 1 || max_d < 1 || max_d > kMaxD) {
        set_err("hawkes_ctx_create: invalid argument");
        return HAWKES_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_err("hawkes_ctx_create: no such CUDA device");
        return HAWKES_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        set_err("hawkes_ctx_create: cudaSetDevice failed");
        return HAWKES_ERR_CUDA;
    }
    hawkes_ctx *ctx = new hawkes_ctx();
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    // control block and a workspace sized for one set of max_n events
    if (cudaMalloc(&ctx->ctl, sizeof(int32_t) * (kCtlSetFlags + 2 * 64)) != cudaSuccess ||
        cudaMemset(ctx->ctl, 0, sizeof(int32_t) * (kCtlSetFlags + 2 * 64)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        set_err("hawkes_ctx_create: control block allocation failed");
        return HAWKES_ERR_OOM;
    }
    ctx->ctl_sets = 64;
    // occupancy of every pair-kernel shape, asked now (it also sets each
    // kernel's shared-memory limit) rather than during a stream capture
    for (int d = 1; d <= kMaxD; ++d)
        for (int pass = 1; pass <= 5; ++pass)
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b)
                    ctx->occ[d][pass][a][b] = (1 << (a + b)) <= 8 ? pass_max_ctas_per_sm(d, pass, 1 << a, 1 << b) : 0;
    for (int pass = 1; pass <= 2; ++pass)
        for (int a = 0; a < 4; ++a)
            ctx->occ_any[pass][a] = pass_any_d_max_ctas_per_sm(pass, 1 << a);
    Plan pl;
    hawkes_params p{1, 1, 1, 1, 1, 1};
    const int64_t n64 = max_n;
    if (build_plan(ctx, pl, 1, &n64, &max_d, &p, false) != HAWKES_OK ||
        bind_plan(ctx, pl, 0) != HAWKES_OK || cudaDeviceSynchronize() != cudaSuccess) {
        set_err("hawkes_ctx_create: " + ctx->err);
        hawkes_ctx_destroy(ctx);
        return HAWKES_ERR_OOM;
    }
    *out = ctx;
    return HAWKES_OK;
}

void hawkes_ctx_destroy(hawkes_ctx *ctx)
{
    if (!ctx)
        return;
    cudaSetDevice(ctx->device);
    for (auto &pe : ctx->prof_pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    if (ctx->hmc.exec)
        cudaGraphExecDestroy(ctx->hmc.exec);
    if (ctx->fork_ev) {
        cudaEventDestroy(ctx->fork_ev);
        for (int d = 1; d <= kMaxD; ++d) {
            cudaStreamDestroy(ctx->side[d]);
            cudaEventDestroy(ctx->join_ev[d]);
        }
    }
    if (ctx->bmds_side) {
        cudaStreamDestroy(ctx->bmds_side);
        cudaEventDestroy(ctx->bmds_fork);
        cudaEventDestroy(ctx->bmds_join);
    }
    if (ctx->ws.ptr)
        cudaFree(ctx->ws.ptr);
    if (ctx->bmds_ws.ptr)
        cudaFree(ctx->bmds_ws.ptr);
    if (ctx->bmds_hmc.ptr)
        cudaFree(ctx->bmds_hmc.ptr);
    if (ctx->bmds_ys.ptr)
        cudaFree(ctx->bmds_ys.ptr);
    if (ctx->ctl)
        cudaFree(ctx->ctl);
    delete ctx;
}

const char *hawkes_last_error(const hawkes_ctx *ctx)
{
    if (!ctx) {
        std::lock_guard<std::mutex> g(g_create_err_mu);
        return g_create_err.c_str();
    }
    return ctx->err.c_str();
}

hawkes_status hawkes_ctx_sync_status(hawkes_ctx *ctx, hawkes_stream stream)
{
    if (!ctx)
        return HAWKES_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    HK_TRY(cudaStreamSynchronize(s), "stream synchronize");
    unsigned st = 0;
    HK_TRY(cudaMemcpy(&st, ctx->ctl + kCtlStatus, sizeof(unsigned), cudaMemcpyDeviceToHost), "read status");
    HK_TRY(cudaMemset(ctx->ctl + kCtlStatus, 0, sizeof(unsigned)), "clear status");
    if (st & kStInvalidData)
        return fail(ctx, HAWKES_ERR_INVALID_DATA,
                    (st & kStNotSorted) ? "times are not sorted although HAWKES_OPT_TIMES_SORTED is set"
                                        : "non-finite location or time, or a negative time");
    if (st & kStZeroRate)
        return fail(ctx, HAWKES_ERR_ZERO_RATE, "some rate lambda_n is zero: ell = -inf, gradient undefined");
    ctx->err.clear();
    return HAWKES_OK;
}

hawkes_status hawkes_ctx_set_option(hawkes_ctx *ctx, int32_t option, int64_t value)
{
    if (!ctx)
        return HAWKES_ERR_INVALID_ARG;
    switch (option) {
    case HAWKES_OPT_BLOCK_WARPS:
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "block warps must be 0, 1, 2, 4 or 8");
        ctx->opt_warps = (int)value;
        return HAWKES_OK;
    case HAWKES_OPT_COL_GROUPS:
        if (value != 0 && value != 1 && value != 2 && value != 4)
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "column groups must be 0, 1, 2 or 4");
        ctx->opt_cols = (int)value;
        return HAWKES_OK;
    case HAWKES_OPT_CTAS_PER_SM:
        if (value < 0 || value > 32)
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "CTAs per SM must be in [0, 32]");
        ctx->opt_ctas = (int)value;
        return HAWKES_OK;
    case HAWKES_OPT_PROFILE:
        ctx->opt_profile = value ? 1 : 0;
        return HAWKES_OK;
    case HAWKES_OPT_TIMES_SORTED:
        ctx->opt_sorted = value ? 1 : 0;
        return HAWKES_OK;
    case HAWKES_OPT_SKIP_FAR_BLOCKS:
        ctx->opt_skip = value ? 1 : 0;
        return HAWKES_OK;
    case HAWKES_OPT_FP64_ORDERED:
        ctx->opt_fp64_ordered = value ? 1 : 0;
        return HAWKES_OK;
    case HAWKES_OPT_ONE_LAUNCH:
        ctx->opt_one_launch = value ? 1 : 0;
        return HAWKES_OK;
    case HAWKES_OPT_BMDS_FUSED:
        ctx->opt_bmds_fused = value ? 1 : 0;
        return HAWKES_OK;
    case HAWKES_OPT_PARTIAL_SLOTS:
        if (value < 0 || value > (int64_t)1 << 30)
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "partial slots must be in [0, 2^30]");
        ctx->opt_slots = (int)value;
        return HAWKES_OK;
    case HAWKES_OPT_MIXED_FIXUP_EXP:
        if (value < -120 || value > 0)
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "fixup exponent must be in [-120, 0]");
        ctx->opt_fixup_exp = (int)value;
        return HAWKES_OK;
    default:
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "unknown option");
    }
}

hawkes_status hawkes_ctx_kernel_stats(hawkes_ctx *ctx, int32_t kernel, double *total_ms, int64_t *launches,
                                      double *pairs)
{
    if (!ctx || kernel < 0 || kernel >= hawkes_ctx::kStages)
        return HAWKES_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    for (auto &pe : ctx->prof_pending) {
        HK_TRY(cudaEventSynchronize(pe.b), "profiling event");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, pe.a, pe.b);
        ctx->prof_ms[pe.kernel] += ms;
        ctx->prof_launches[pe.kernel] += 1;
        ctx->prof_pairs[pe.kernel] += pe.pairs;
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    ctx->prof_pending.clear();
    if (total_ms)
        *total_ms = ctx->prof_ms[kernel];
    if (launches)
        *launches = ctx->prof_launches[kernel];
    if (pairs)
        *pairs = ctx->prof_pairs[kernel];
    return HAWKES_OK;
}

hawkes_status hawkes_ctx_reset_stats(hawkes_ctx *ctx)
{
    if (!ctx)
        return HAWKES_ERR_INVALID_ARG;
    hawkes_ctx_kernel_stats(ctx, 0, nullptr, nullptr, nullptr);
    ctx->launches_own = 0;
    ctx->launches_lib = 0;
    for (int k = 0; k < hawkes_ctx::kStages; ++k) {
        ctx->prof_ms[k] = 0;
        ctx->prof_launches[k] = 0;
        ctx->prof_pairs[k] = 0;
    }
    return HAWKES_OK;
}

hawkes_status hawkes_ctx_launch_count(const hawkes_ctx *ctx, int64_t *own, int64_t *library)
{
    if (!ctx)
        return HAWKES_ERR_INVALID_ARG;
    if (own)
        *own = ctx->launches_own;
    if (library)
        *library = ctx->launches_lib;
    return HAWKES_OK;
}

hawkes_status hawkes_ctx_set_tuning(hawkes_ctx *ctx, int32_t d, int32_t bucket, int32_t warps, int32_t col_groups,
                                    int32_t ctas_per_sm)
{
    if (!ctx)
        return HAWKES_ERR_INVALID_ARG;
    auto pow2_le8 = [](int32_t v) { return v == 1 || v == 2 || v == 4 || v == 8; };
    if (d < 1 || d > kMaxD || bucket < 0 || bucket >= hawkes_ctx::kBuckets || !(warps == 0 || pow2_le8(warps)) ||
        !(col_groups == 0 || (pow2_le8(col_groups) && col_groups <= 4)) ||
        (int64_t)warps * std::max(1, col_groups) > 8 ||
        ctas_per_sm < 0 || ctas_per_sm > 32)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "tuning entry out of range");
    ctx->tune_warps[d][bucket] = warps;
    ctx->tune_cols[d][bucket] = col_groups;
    ctx->tune_ctas[d][bucket] = ctas_per_sm;
    return HAWKES_OK;
}

hawkes_status hawkes_ctx_get_tuning(const hawkes_ctx *ctx, int32_t d, int32_t bucket, int32_t *warps,
                                    int32_t *col_groups, int32_t *ctas_per_sm)
{
    if (!ctx || d < 1 || d > kMaxD || bucket < 0 || bucket >= hawkes_ctx::kBuckets)
        return HAWKES_ERR_INVALID_ARG;
    if (warps)
        *warps = ctx->tune_warps[d][bucket];
    if (col_groups)
        *col_groups = ctx->tune_cols[d][bucket];
    if (ctas_per_sm)
        *ctas_per_sm = ctx->tune_ctas[d][bucket];
    return HAWKES_OK;
}

static hawkes_status loglik_common(hawkes_ctx *ctx, const double *t, const double *X, int64_t n, int32_t d,
                                   const hawkes_params *params, hawkes_precision prec, hawkes_stream stream,
                                   double *out_loglik, double *out_grad_X, double *out_grad_params, bool grad)
{
    hawkes_status st = check_common(ctx, t, X, n, d, params, prec);
    if (st != HAWKES_OK)
        return st;
    if (!out_loglik || (grad && !out_grad_X))
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "output pointers must be device pointers");
    HK_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool fp64 = prec == HAWKES_PREC_FP64;
    Plan pl;
    const bool theta = grad && out_grad_params != nullptr;
    if ((st = build_plan(ctx, pl, 1, &n, &d, params, fp64, theta)) != HAWKES_OK)
        return st;
    if ((st = bind_plan(ctx, pl, s)) != HAWKES_OK)
        return st;
    if ((st = enqueue_prep(ctx, pl, t, X, s)) != HAWKES_OK)
        return st;
    if ((st = enqueue_eval(ctx, pl, fp64, grad, out_loglik, grad ? out_grad_X : nullptr, nullptr, s,
                           theta ? out_grad_params : nullptr)) != HAWKES_OK)
        return st;
    if ((st = enqueue_nan_on_invalid(ctx, out_loglik, 1, grad ? out_grad_X : nullptr, n * d, s)) != HAWKES_OK)
        return st;
    return theta ? enqueue_nan_on_invalid(ctx, out_grad_params, 6, nullptr, 0, s) : HAWKES_OK;
}

hawkes_status hawkes_self_excitation_prob(hawkes_ctx *ctx, const double *t, const double *X, int64_t n, int32_t d,
                                          const hawkes_params *params, hawkes_precision prec, hawkes_stream stream,
                                          double *out_prob)
{
    hawkes_status st = check_common(ctx, t, X, n, d, params, prec);
    if (st != HAWKES_OK)
        return st;
    if (!out_prob)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "out_prob must be a device pointer");
    HK_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool fp64 = prec == HAWKES_PREC_FP64;
    Plan pl;
    // FP64: the rate pass with the parameter-gradient sums carries sum_n' xi_nn';
    // mixed: a rate pass that keeps only that sum apart (two column planes)
    if ((st = build_plan(ctx, pl, 1, &n, &d, params, fp64, fp64, !fp64)) != HAWKES_OK)
        return st;
    if ((st = bind_plan(ctx, pl, s)) != HAWKES_OK)
        return st;
    if ((st = enqueue_prep(ctx, pl, t, X, s)) != HAWKES_OK)
        return st;
    if (fp64) {
        if ((st = enqueue_fp64_pass(ctx, pl, 1, true, s)) != HAWKES_OK)
            return st;
        HK_TRY(launch_finalize_rows(ctx->w, pl.total_segs, true, kSumsTheta, nullptr, s), "finalize rows");
    } else {
        if ((st = enqueue_pair_pass(ctx, pl, 4, s)) != HAWKES_OK)
            return st;
        // flagged rows get all six sums in FP64, the self-excitation one among them
        HK_TRY(launch_finalize_rows(ctx->w, pl.total_segs, false, kSumsXi, nullptr, s), "finalize rows");
    }
    HK_TRY(launch_self_excitation(ctx->w, pl.total_segs, out_prob, s), "self-excitation");
    ctx->launches_own += 2 + pass_launches(pl);
    return enqueue_nan_on_invalid(ctx, out_prob, n, nullptr, 0, s);
}

// Grow-only device buffer; synchronizes the device before replacing it.
static hawkes_status grow_buffer(hawkes_ctx *ctx, DeviceBuffer &b, size_t need, const char *what, size_t zero_head)
{
    if (need <= b.bytes)
        return HAWKES_OK;
    HK_TRY(cudaDeviceSynchronize(), "synchronize before growing a workspace");
    if (b.ptr)
        cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.ptr, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, HAWKES_ERR_OOM, std::string(what) + " of " + std::to_string(need) + " bytes");
    }
    b.bytes = need;
    if (zero_head)
        HK_TRY(cudaMemset(b.ptr, 0, zero_head), "clear workspace head");
    ++ctx->ws_generation;
    return HAWKES_OK;
}

size_t hawkes_bmds_workspace_bytes(int64_t n, int32_t d, hawkes_precision prec)
{
    if (n < 1 || n > (int64_t)1 << 30 || d < 1 || d > kMaxD ||
        (prec != HAWKES_PREC_MIXED && prec != HAWKES_PREC_FP64))
        return 0;
    return bmds_workspace_bytes(n, d, prec == HAWKES_PREC_FP64);
}

hawkes_status hawkes_bmds_loglik_grad(hawkes_ctx *ctx, const void *Y, hawkes_dtype y_type, const double *X, int64_t n,
                                      int32_t d, double sigma2, hawkes_precision prec, hawkes_stream stream,
                                      double *out_loglik, double *out_grad_X, double *out_grad_sigma2)
{
    if (!ctx)
        return HAWKES_ERR_INVALID_ARG;
    if (!Y || !X || !out_loglik)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "Y, X and out_loglik must be device pointers");
    if (n < 1 || n > (int64_t)1 << 30)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "n must be in [1, 2^30]");
    if (d < 1 || d > kMaxD)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "d must be in [1, 8]");
    if (!(sigma2 > 0.0) || !std::isfinite(sigma2))
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "sigma2 must be finite and > 0");
    if (prec != HAWKES_PREC_MIXED && prec != HAWKES_PREC_FP64)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "unknown precision");
    if (y_type != HAWKES_F64 && y_type != HAWKES_F32)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "y_type must be HAWKES_F64 or HAWKES_F32");
    HK_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool fp64 = prec == HAWKES_PREC_FP64;
    hawkes_status gst = grow_buffer(ctx, ctx->bmds_ws, bmds_workspace_bytes(n, d, fp64), "BMDS workspace", 256);
    if (gst != HAWKES_OK)
        return gst;
    HK_TRY(launch_bmds(Y, y_type == HAWKES_F32, X, n, d, sigma2, fp64, ctx->bmds_ws.ptr, reinterpret_cast<unsigned *>(ctx->ctl + kCtlStatus),
                       out_loglik, out_grad_X, out_grad_sigma2, s, &ctx->launches_own),
           "BMDS kernels");
    return HAWKES_OK;  // the finalize kernel writes NaN itself on invalid data
}

hawkes_status hawkes_loglik(hawkes_ctx *ctx, const double *t, const double *X, int64_t n, int32_t d,
                            const hawkes_params *params, hawkes_precision prec, hawkes_stream stream,
                            double *out_loglik)
{
    return loglik_common(ctx, t, X, n, d, params, prec, stream, out_loglik, nullptr, nullptr, false);
}

hawkes_status hawkes_loglik_grad_locations(hawkes_ctx *ctx, const double *t, const double *X, int64_t n, int32_t d,
                                           const hawkes_params *params, hawkes_precision prec, hawkes_stream stream,
                                           double *out_loglik, double *out_grad_X, double *out_grad_params)
{
    return loglik_common(ctx, t, X, n, d, params, prec, stream, out_loglik, out_grad_X, out_grad_params, true);
}

hawkes_status hawkes_autotune(hawkes_ctx *ctx, const double *t, const double *X, int64_t n, int32_t d,
                              const hawkes_params *params, hawkes_stream stream, int32_t *best_warps,
                              int32_t *best_col_groups, int32_t *best_ctas_per_sm, double *out_ms)
{
    hawkes_status st = check_common(ctx, t, X, n, d, params, HAWKES_PREC_MIXED);
    if (st != HAWKES_OK)
        return st;
    HK_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double *out = nullptr;
    HK_TRY(cudaMalloc(&out, sizeof(double) * (1 + n * d)), "autotune output");
    const int saved_w = ctx->opt_warps, saved_wc = ctx->opt_cols, saved_c = ctx->opt_ctas, saved_p = ctx->opt_profile;
    ctx->opt_profile = 0;
    double best = 1e300;
    int bw = 0, bwc = 0, bc = 0;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int wv : {1, 2, 4, 8}) {
        for (int wc : {0, 1, 2, 4}) {  // 0: column groups chosen per pass
            if (!shape_ok(ctx, d, wv, std::max(1, wc), false, 200 * 1024))
                continue;
            const int max_c = std::max(1, occupancy(ctx, d, 2, wv, std::max(1, wc)));
            // caps: as many as fit (0), then powers of two below that
            for (int cv = 0; cv < max_c; cv = cv == 0 ? 1 : 2 * cv) {
                ctx->opt_warps = wv;
                ctx->opt_cols = wc;
                ctx->opt_ctas = cv;
                float ms = 0.0f, tot = 0.0f;
                st = hawkes_loglik_grad_locations(ctx, t, X, n, d, params, HAWKES_PREC_MIXED, stream, out, out + 1,
                                                  nullptr);
                for (int rep = 0; rep < 3 && st == HAWKES_OK; ++rep) {
                    cudaEventRecord(a, s);
                    st = hawkes_loglik_grad_locations(ctx, t, X, n, d, params, HAWKES_PREC_MIXED, stream, out,
                                                      out + 1, nullptr);
                    cudaEventRecord(b, s);
                    cudaEventSynchronize(b);
                    cudaEventElapsedTime(&ms, a, b);
                    tot += ms;
                }
                if (st != HAWKES_OK)
                    break;
                if (tot / 3.0 < best) {
                    best = tot / 3.0;
                    bw = wv;
                    bwc = wc;
                    bc = cv;
                }
            }
            if (st != HAWKES_OK)
                break;
        }
        if (st != HAWKES_OK)
            break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->opt_warps = saved_w;
    ctx->opt_cols = saved_wc;
    ctx->opt_ctas = saved_c;
    ctx->opt_profile = saved_p;
    cudaStreamSynchronize(s);
    cudaFree(out);
    if (st != HAWKES_OK)
        return st;
    if (bw == 0)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "no tile shape fits this dimension");
    ctx->tune_warps[d][size_bucket(n)] = bw;
    ctx->tune_cols[d][size_bucket(n)] = bwc;
    ctx->tune_ctas[d][size_bucket(n)] = bc;
    if (best_warps)
        *best_warps = bw;
    if (best_col_groups)
        *best_col_groups = bwc;
    if (best_ctas_per_sm)
        *best_ctas_per_sm = bc;
    if (out_ms)
        *out_ms = best;
    return HAWKES_OK;
}

// One HMC proposal per set (Section 3), all sets advanced together; the
// trajectory after the prologue is one CUDA graph cached per shape.
// A BMDS term added to the HMC potential (single set): distances Y of
// element type y_f32 ? float : double, variance sigma2.
struct BmdsTerm {
    const void *Y;
    bool y_f32;
    double sigma2;
};

static hawkes_status hmc_common(hawkes_ctx *ctx, int32_t nsets, const int64_t *counts, const int32_t *dims,
                                const double *t, double *X_inout, const double *p0, const double *box_lo,
                                const double *box_hi, const hawkes_params *params, const double *eps,
                                int32_t n_steps, const double *log_u, hawkes_precision prec, hawkes_stream stream,
                                double *out_H0, double *out_H1, int32_t *out_accepted,
                                const BmdsTerm *bmds = nullptr)
{
    hawkes_status st;
    if (!p0 || !log_u || !out_H0 || !out_H1 || !out_accepted)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "p0, log_u and the outputs must be device pointers");
    if ((box_lo == nullptr) != (box_hi == nullptr))
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "box_lo and box_hi must both be given or both be NULL");
    for (int k = 0; k < nsets; ++k)
        if (!(eps[k] > 0.0) || !std::isfinite(eps[k]))
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "eps must be finite and > 0");
    if (n_steps < 0 || n_steps > 100000)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "n_steps must be in [0, 100000]");
    HK_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool fp64 = prec == HAWKES_PREC_FP64;
    Plan pl;
    if ((st = build_plan(ctx, pl, nsets, counts, dims, params, fp64)) != HAWKES_OK)
        return st;
    if ((st = bind_plan(ctx, pl, s)) != HAWKES_OK)
        return st;
    if ((st = enqueue_prep(ctx, pl, t, X_inout, s)) != HAWKES_OK)
        return st;
    Work &w = ctx->w;
    const int ns = nsets;
    double *d_eps = ctx->hscal, *d_logu = ctx->hscal + ns, *d_H0 = ctx->hscal + 2 * ns, *d_H1 = ctx->hscal + 3 * ns;
    int32_t *d_acc = ctx->hint, *d_bad = ctx->hint + ns;
    HK_TRY(launch_gather_sorted(w, ctx->d_set_row0, p0, ctx->hp, pl.total_rows, 0.0, s), "gather momenta");
    const bool box = box_lo != nullptr;
    if (box) {
        HK_TRY(launch_gather_sorted(w, ctx->d_set_row0, box_lo, ctx->hlo, pl.total_rows, 0.0, s), "gather box");
        HK_TRY(launch_gather_sorted(w, ctx->d_set_row0, box_hi, ctx->hhi, pl.total_rows, 0.0, s), "gather box");
    }
    HK_TRY(cudaMemcpyAsync(d_eps, eps, sizeof(double) * ns, cudaMemcpyHostToDevice, s), "step sizes");
    HK_TRY(cudaMemcpyAsync(d_logu, log_u, sizeof(double) * ns, cudaMemcpyDeviceToDevice, s), "log u");
    HK_TRY(cudaMemsetAsync(ctx->hint, 0, sizeof(int32_t) * 2 * ns, s), "flags");

    // BMDS term: its workspace and the caller-order buffers exist before any capture
    double *bx = nullptr, *bg = nullptr, *bl = nullptr;
    // mixed precision, as an option: the gradient pass carries the BMDS term
    // (pass 5), from a time-ordered FP32 copy of Y made here; the BMDS kernels
    // then run only for ell_B at the two ends of the trajectory
    const bool fused = bmds && !fp64 && ctx->opt_bmds_fused && nsets == 1 &&
                       occupancy(ctx, dims[0], 5, pl.wr_by_d[dims[0]], 1) > 0;
    float *ys = nullptr;
    if (fused) {
        const int64_t npad = pl.sets[0].npad;
        if ((st = grow_buffer(ctx, ctx->bmds_ys, sizeof(float) * npad * npad, "time-ordered Y", 0)) != HAWKES_OK)
            return st;
        ys = static_cast<float *>(ctx->bmds_ys.ptr);
        HK_TRY(launch_bmds_sort_y(bmds->Y, bmds->y_f32, w.perm, counts[0], npad, ys, s), "time-ordered Y");
        ++ctx->launches_own;
    }
    if (bmds) {
        const int64_t nd = counts[0] * dims[0];
        if ((st = grow_buffer(ctx, ctx->bmds_ws, bmds_workspace_bytes(counts[0], dims[0], fp64), "BMDS workspace",
                              256)) != HAWKES_OK)
            return st;
        if ((st = grow_buffer(ctx, ctx->bmds_hmc, sizeof(double) * (2 * nd + 32), "BMDS HMC buffers", 0)) !=
            HAWKES_OK)
            return st;
        bx = static_cast<double *>(ctx->bmds_hmc.ptr);
        bg = bx + nd;
        bl = bg + nd;
    }

    // the trajectory itself: captured once per shape, replayed as a graph
    std::vector<int64_t> key = {n_steps, (int64_t)prec, box ? 1 : 0, (int64_t)ctx->ws_generation, ns};
    if (bmds) {
        int64_t sbits;
        std::memcpy(&sbits, &bmds->sigma2, sizeof(sbits));
        key.push_back((int64_t)reinterpret_cast<intptr_t>(bmds->Y));
        key.push_back(bmds->y_f32 ? 2 : 1);
        key.push_back(sbits);
        key.push_back((int64_t)reinterpret_cast<intptr_t>(ys));
    }
    for (int k = 0; k < ns; ++k) {
        key.push_back(counts[k]);
        key.push_back(dims[k]);
        key.push_back(pl.sets[k].B);
    }
    // the options that shape the captured launches or the Work they copy,
    // and the pair launches themselves (a replay must not run another plan's
    // work lists)
    for (int64_t v : {(int64_t)ctx->opt_warps, (int64_t)ctx->opt_cols, (int64_t)ctx->opt_ctas, (int64_t)ctx->opt_skip,
                      (int64_t)ctx->opt_one_launch, (int64_t)ctx->opt_slots, (int64_t)ctx->opt_fp64_ordered,
                      (int64_t)ctx->opt_bmds_fused, (int64_t)pl.slot_cap, (int64_t)pl.phases})
        key.push_back(v);
    for (const PairLaunch &L : pl.launches) {
        key.push_back(L.d);
        key.push_back(L.phase);
        key.push_back(L.run0);
        key.push_back(L.nruns);
        key.push_back(L.nitems);
    }
    // the fused pass's inputs travel in the Work copied into each launch;
    // later calls must not see them
    struct ClearBmdsTerm {
        Work &w;
        ~ClearBmdsTerm() { w.ysort = nullptr; }
    } clear_bmds_term{w};
    if (fused) {
        w.ysort = ys;
        w.bmds_inv_sigma_d = 1.0 / std::sqrt(bmds->sigma2);
        w.bmds_inv_s2_d = 1.0 / bmds->sigma2;
        w.bmds_inv_sigma = (float)w.bmds_inv_sigma_d;
        w.bmds_inv_s2 = (float)w.bmds_inv_s2_d;
    }
    if (!ctx->hmc.exec || ctx->hmc.key != key || ctx->opt_profile) {
        if (ctx->hmc.exec) {
            cudaGraphExecDestroy(ctx->hmc.exec);
            ctx->hmc.exec = nullptr;
        }
        cudaStream_t cs;
        HK_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
        const bool capture = !ctx->opt_profile;  // event timing is not captured
        cudaStream_t es = capture ? cs : s;
        if (capture)
            HK_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
        // the BMDS term of the potential, evaluated at the current locations
        // The BMDS term of a step depends only on the locations, so it runs on a
        // side branch concurrently with the Hawkes evaluation (each leaves SMs
        // idle in its tail at the influenza size); the two gradients meet in
        // add_caller_term.  Neither branch writes what the other reads: the
        // BMDS kernels use their own workspace and buffers, and the Hawkes
        // evaluation's control-word reset leaves the shared status word alone.
        if (bmds && !ctx->bmds_side) {
            HK_TRY(cudaStreamCreateWithFlags(&ctx->bmds_side, cudaStreamNonBlocking), "BMDS stream");
            HK_TRY(cudaEventCreateWithFlags(&ctx->bmds_fork, cudaEventDisableTiming), "BMDS fork event");
            HK_TRY(cudaEventCreateWithFlags(&ctx->bmds_join, cudaEventDisableTiming), "BMDS join event");
        }
        // the BMDS gradient is carried by the fused gradient pass; ell_B is
        // needed only for H0 and H1 (the first and last evaluation)
        auto fork_bmds = [&](bool ends) -> hawkes_status {
            if (!bmds || (fused && !ends))
                return HAWKES_OK;
            cudaStream_t bs = ctx->bmds_side;
            HK_TRY(cudaEventRecord(ctx->bmds_fork, es), "BMDS fork");
            HK_TRY(cudaStreamWaitEvent(bs, ctx->bmds_fork, 0), "BMDS fork wait");
            HK_TRY(launch_to_caller(w, ctx->d_set_row0, w.x64, bx, pl.total_rows, bs), "BMDS locations");
            ++ctx->launches_own;
            // ell_B only where the energy needs it (the first and last
            // evaluation); the steps in between take the gradient alone
            HK_TRY(launch_bmds(bmds->Y, bmds->y_f32, bx, counts[0], dims[0], bmds->sigma2, fp64, ctx->bmds_ws.ptr,
                               reinterpret_cast<unsigned *>(ctx->ctl + kCtlStatus), bl, fused ? nullptr : bg,
                               nullptr, bs, &ctx->launches_own, ends || fp64),
                   "BMDS kernels");
            HK_TRY(cudaEventRecord(ctx->bmds_join, bs), "BMDS join");
            return HAWKES_OK;
        };
        auto join_bmds = [&](bool ends) -> hawkes_status {
            if (!bmds || (fused && !ends))
                return HAWKES_OK;
            HK_TRY(cudaStreamWaitEvent(es, ctx->bmds_join, 0), "BMDS join wait");
            HK_TRY(launch_add_caller_term(w, ctx->d_set_row0, fused ? nullptr : bg, ctx->hg, pl.total_rows,
                                          ends ? bl : nullptr, es),
                   "BMDS gradient");
            ++ctx->launches_own;
            return HAWKES_OK;
        };
        const int grad_pass = fused ? 5 : 2;
        auto body = [&]() -> hawkes_status {
            hawkes_status r;
            // the first evaluation follows the prologue, whose reset of the
            // per-evaluation control words precedes the graph; each later one
            // follows a drift kernel that clears them
            if ((r = fork_bmds(true)) != HAWKES_OK)
                return r;
            if ((r = enqueue_eval(ctx, pl, fp64, true, nullptr, nullptr, ctx->hg, es, nullptr, grad_pass)) != HAWKES_OK)
                return r;
            if ((r = join_bmds(true)) != HAWKES_OK)
                return r;
            HK_TRY(launch_energy(w, ctx->hp, d_H0, ctx->hscal + 4 * ns, es), "H0");
            for (int32_t k = 0; k < n_steps; ++k) {
                HK_TRY(launch_kick_drift(w, ctx->d_set_row0, ctx->hp, ctx->hg, box ? ctx->hlo : nullptr,
                                         box ? ctx->hhi : nullptr, d_eps, pl.total_rows, k == 0 ? 1 : 2, !fp64,
                                         d_bad, es),
                       "leapfrog drift");
                const bool last = k == n_steps - 1;
                if ((r = fork_bmds(last)) != HAWKES_OK)
                    return r;
                // ell (for H1) from the last evaluation only
                if ((r = enqueue_eval(ctx, pl, fp64, true, nullptr, nullptr, ctx->hg, es, nullptr, grad_pass, last)) !=
                    HAWKES_OK)
                    return r;
                if ((r = join_bmds(last)) != HAWKES_OK)
                    return r;
            }
            if (n_steps > 0)
                HK_TRY(launch_kick(w, ctx->d_set_row0, ctx->hp, ctx->hg, d_eps, pl.total_rows, es), "leapfrog kick");
            HK_TRY(launch_energy(w, ctx->hp, d_H1, ctx->hscal + 4 * ns, es), "H1");
            HK_TRY(launch_accept(d_H0, d_H1, d_logu, d_bad, d_acc, ns, es), "accept");
            return HAWKES_OK;
        };
        if (capture) {
            // capture only records; the graph later runs on s after the prologue
            cudaGraph_t graph = nullptr;
            hawkes_status st2 = body();
            cudaError_t ce = cudaStreamEndCapture(cs, &graph);
            if (st2 != HAWKES_OK) {
                if (graph)
                    cudaGraphDestroy(graph);
                cudaStreamDestroy(cs);
                return st2;
            }
            if (ce != cudaSuccess) {
                cudaStreamDestroy(cs);
                return cuda_fail(ctx, ce, "end capture");
            }
            ce = cudaGraphInstantiate(&ctx->hmc.exec, graph, 0);
            cudaGraphDestroy(graph);
            cudaStreamDestroy(cs);
            if (ce != cudaSuccess) {
                ctx->hmc.exec = nullptr;
                return cuda_fail(ctx, ce, "instantiate trajectory graph");
            }
            ctx->hmc.key = key;
        } else {
            cudaStreamDestroy(cs);
            hawkes_status st2 = body();
            if (st2 != HAWKES_OK)
                return st2;
        }
    }
    if (ctx->hmc.exec && !ctx->opt_profile)
        HK_TRY(cudaGraphLaunch(ctx->hmc.exec, s), "launch trajectory graph");
    HK_TRY(launch_scatter(w, ctx->d_set_row0, w.x64, X_inout, d_acc, pl.total_rows, s), "write back");
    HK_TRY(cudaMemcpyAsync(out_H0, d_H0, sizeof(double) * ns, cudaMemcpyDeviceToDevice, s), "H0 out");
    HK_TRY(cudaMemcpyAsync(out_H1, d_H1, sizeof(double) * ns, cudaMemcpyDeviceToDevice, s), "H1 out");
    HK_TRY(cudaMemcpyAsync(out_accepted, d_acc, sizeof(int32_t) * ns, cudaMemcpyDeviceToDevice, s), "accept out");
    return HAWKES_OK;
}

hawkes_status hmc_leapfrog_trajectory(hawkes_ctx *ctx, const double *t, double *X_inout, const double *p0,
                                      const double *box_lo, const double *box_hi, int64_t n, int32_t d,
                                      const hawkes_params *params, double eps, int32_t n_steps, const double *log_u,
                                      hawkes_precision prec, hawkes_stream stream, double *out_H0, double *out_H1,
                                      int32_t *out_accepted)
{
    hawkes_status st = check_common(ctx, t, X_inout, n, d, params, prec);
    if (st != HAWKES_OK)
        return st;
    return hmc_common(ctx, 1, &n, &d, t, X_inout, p0, box_lo, box_hi, params, &eps, n_steps, log_u, prec, stream,
                      out_H0, out_H1, out_accepted);
}

hawkes_status hawkes_bmds_hmc_trajectory(hawkes_ctx *ctx, const double *t, double *X_inout, const double *p0,
                                         int64_t n, int32_t d, const hawkes_params *params, const void *Y,
                                         hawkes_dtype y_type, double sigma2, double eps, int32_t n_steps,
                                         const double *log_u, hawkes_precision prec, hawkes_stream stream,
                                         double *out_H0, double *out_H1, int32_t *out_accepted)
{
    hawkes_status st = check_common(ctx, t, X_inout, n, d, params, prec);
    if (st != HAWKES_OK)
        return st;
    if (!Y)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "Y must be a device pointer");
    if (y_type != HAWKES_F64 && y_type != HAWKES_F32)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "y_type must be HAWKES_F64 or HAWKES_F32");
    if (!(sigma2 > 0.0) || !std::isfinite(sigma2))
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "sigma2 must be finite and > 0");
    const BmdsTerm bt{Y, y_type == HAWKES_F32, sigma2};
    return hmc_common(ctx, 1, &n, &d, t, X_inout, p0, nullptr, nullptr, params, &eps, n_steps, log_u, prec, stream,
                      out_H0, out_H1, out_accepted, &bt);
}

hawkes_status hawkes_batch_hmc_trajectory(hawkes_ctx *ctx, int32_t n_sets, const int64_t *offsets,
                                          const int32_t *dims, const double *t, double *X_inout, const double *p0,
                                          const double *box_lo, const double *box_hi, const hawkes_params *params,
                                          const double *eps, int32_t n_steps, const double *log_u,
                                          hawkes_precision prec, hawkes_stream stream, double *out_H0,
                                          double *out_H1, int32_t *out_accepted)
{
    if (!ctx)
        return HAWKES_ERR_INVALID_ARG;
    if (n_sets < 1 || !offsets || !dims || !params || !eps || !t || !X_inout)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "invalid batch arguments");
    if (prec != HAWKES_PREC_MIXED && prec != HAWKES_PREC_FP64)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "unknown precision");
    if (offsets[0] != 0)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "offsets[0] must be 0");
    std::vector<int64_t> counts(n_sets);
    for (int k = 0; k < n_sets; ++k) {
        counts[k] = offsets[k + 1] - offsets[k];
        if (counts[k] < 1 || counts[k] > (int64_t)1 << 30)
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "every set needs at least one event");
        if (dims[k] < 1 || dims[k] > kMaxD)
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "dims must be in [1, 8]");
        if (!params_ok(&params[k]))
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "every parameter must be finite and > 0");
    }
    return hmc_common(ctx, n_sets, counts.data(), dims, t, X_inout, p0, box_lo, box_hi, params, eps, n_steps, log_u,
                      prec, stream, out_H0, out_H1, out_accepted);
}

hawkes_status hawkes_batch_loglik_grad(hawkes_ctx *ctx, int32_t n_sets, const int64_t *offsets, const int32_t *dims,
                                       const double *t, const double *X, const hawkes_params *params,
                                       hawkes_precision prec, hawkes_stream stream, double *out_loglik,
                                       double *out_grad_X)
{
    if (!ctx)
        return HAWKES_ERR_INVALID_ARG;
    if (n_sets < 1 || !offsets || !dims || !params || !t || !X || !out_loglik || !out_grad_X)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "invalid batch arguments");
    if (prec != HAWKES_PREC_MIXED && prec != HAWKES_PREC_FP64)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "unknown precision");
    if (offsets[0] != 0)
        return fail(ctx, HAWKES_ERR_INVALID_ARG, "offsets[0] must be 0");
    std::vector<int64_t> counts(n_sets);
    int64_t xt = 0;
    for (int s = 0; s < n_sets; ++s) {
        counts[s] = offsets[s + 1] - offsets[s];
        if (counts[s] < 1 || counts[s] > (int64_t)1 << 30)
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "every set needs at least one event");
        if (dims[s] < 1 || dims[s] > kMaxD)
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "dims must be in [1, 8]");
        if (!params_ok(&params[s]))
            return fail(ctx, HAWKES_ERR_INVALID_ARG, "every parameter must be finite and > 0");
        xt += counts[s] * dims[s];
    }
    HK_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool fp64 = prec == HAWKES_PREC_FP64;
    Plan pl;
    hawkes_status st;
    if ((st = build_plan(ctx, pl, n_sets, counts.data(), dims, params, fp64)) != HAWKES_OK)
        return st;
    if ((st = bind_plan(ctx, pl, s)) != HAWKES_OK)
        return st;
    if ((st = enqueue_prep(ctx, pl, t, X, s)) != HAWKES_OK)
        return st;
    if ((st = enqueue_eval(ctx, pl, fp64, true, out_loglik, out_grad_X, nullptr, s)) != HAWKES_OK)
        return st;
    return enqueue_nan_on_invalid(ctx, out_loglik, n_sets, out_grad_X, xt, s);
}

}  // extern "C"
