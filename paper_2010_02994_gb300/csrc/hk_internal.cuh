// Internal declarations shared by the libhawkes translation units.
//
// Data layout (every array lives in the context's device workspace):
//   Events are processed in time-sorted order ("rows").  A call is a list of
//   data sets; set s owns rows [row0, row0 + npad) of every per-row array,
//   npad = nblk * B padded up to whole blocks of B rows.
//   rec   float4 planes: plane p of set s is rec[rec0 + p*npad + i]; the
//         fields of row i are, in order, xh_0, xl_0, ..., xh_{D-1}, xl_{D-1},
//         th, tl: the FP32 hi/lo split of the scaled coordinate kx*x_k and
//         of the scaled time kt*t (nrec(D) planes, unused fields zero).
//   w32   FP32 1/S_n for the gradient pass (0 for rows recomputed in FP64).
//   cm32  FP32 c_xi1 + log2(rho) + log2(w_n), the gradient pass's per-column
//         self-excitation exponent constant (-inf where w_n = 0).
//   tie_end  first set-relative row whose time exceeds this row's time.
//   perm  set-relative caller index of each row.
//   t64, x64  FP64 sorted times and coordinates (x64 row stride kMaxD).
//   P1    pass-1 partial row sums, slot-major: P1[part0 + (slot*vpc + v)*npad + i]
//   P2    pass-2 partial gradients: P2[part2_0 + (slot*D + k)*npad + i]
//   F1, F2  the FP64 path's partials, FP64, in the same slot-major layout
//         (F1[fpart0 + (slot*V + v)*npad + i], V = 6 with the Theta sums,
//         else 1; F2[fpart2_0 + (slot*D + k)*npad + i]), fsplit slots: nslot
//         for the symmetric kernels, a few column splits for the ordered
//         ones.  A plan holds P1/P2 or F1/F2, not both.
//
// Pair schedule.  The pair blocks {I, J} (I <= J) of a set with nblk row
// blocks are dealt out in rounds by the circle method over nt = nblk | 1
// "teams" (one empty team nblk when nblk is even): in round r the team r
// sits out and plays its diagonal block {r, r}, and the pairs {r + j, r - j}
// (mod nt), j = 1 .. (nt - 1) / 2, meet.  Every row block is touched exactly
// once per round, by an off-diagonal block, its diagonal, or a pair with the
// empty team (whose only effect is a zero partial).  With nslot = min(nt, G)
// for the plan's slot cap G, rounds [0, nslot) ("phase 0") store a row's
// partial in slot r; the rounds of a later phase (nslot each) store theirs
// in the scratch slot nslot + (r mod nslot), and a fold kernel then adds
// those into slots [0, nslot) and clears them (a pass starts with cleared
// scratch slots, so a block with zero partials need not store them there).
// Each slot has one writer per launch and the launches run in order, so
// every sum is taken in a fixed order and the results are deterministic;
// the slots take nslot (2 nslot with later phases) x npad values per set,
// which the cap keeps within a byte budget.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hawkes.h"
#include "hk_sched.cuh"

namespace hk {

constexpr int kMaxD = 8;
constexpr float kPadTime = 1.0e18f;  // its square stays finite in FP32
constexpr int kPass1Vals = 1;       // S
constexpr int kPass1ThetaVals = 6;  // M, Xi, sum mu' q, sum mu' dt^2, sum xi'' dt, sum xi'' q
constexpr int kPass1XiVals = 2;     // M, Xi

// What the rate pass keeps per row besides the rate.
enum RateSums : int { kSumsNone = 0, kSumsTheta = 1, kSumsXi = 2 };
constexpr int kSegRows = 64;             // rows per finalize segment
constexpr int kFinalizeThreads = kSegRows;  // threads of a standalone finalize CTA (one segment each)
constexpr int kMaxThetaSets = 1;
constexpr int kThetaParts = 256;  // CTAs of the Theta-gradient reduction

// Bits of the sticky device status word.
enum : unsigned {
    kStInvalidData = 1u,
    kStZeroRate = 2u,
    kStNotSorted = 8u,
};

__host__ __device__ constexpr int nrec(int d) { return (2 * d + 2 + 3) / 4; }
// Rows each lane keeps in registers in the pair kernels.
__host__ __device__ constexpr int rows_per_lane(int d) { return d <= 4 ? 4 : 2; }

struct SetDesc {
    int64_t row0;     // first row of the set in the per-row arrays
    int64_t ev0;      // first event of the set in the caller's t
    int64_t x0;       // first element of the set in the caller's X
    int64_t rec0;     // first float4 of the set's record planes
    int64_t part0;    // first float of the set's pass-1 partial slots
    int64_t part2_0;  // first float of the set's pass-2 partial slots
    int64_t fpart0;   // first double of the set's FP64 rate partial slots
    int64_t fpart2_0; // first double of the set's FP64 gradient partial slots
    int32_t n, d, npad, nblk, B, vpc;
    int32_t item0, nitems;  // the set's work items (in the item list)
    int32_t seg0;           // first finalize segment of the set
    int32_t nseg;           // finalize segments of the set (kSegRows rows each)
    int32_t fsplit;         // column splits of the FP64 pair kernels
    int32_t nslot;          // partial slots per row of the symmetric pair kernels (+ nslot scratch with phases)
    // mixed-path exponent constants (base 2; see the pass kernels)
    float rho, kappa, cxi1, cxi2;
    float kappa_lo, cxi1_lo;  // low words: kappa + kappa_lo and cxi1 + cxi1_lo are the FP64 values
    float bq, bc;     // BMDS term of the gradient pass: 1/kx^2 (scaled q -> squared distance), tau_x^2
    double cxi2_d;    // c_xi1 + log2(rho) in FP64
    // FP64 constants
    double kx, kt;    // coordinate scalings sqrt(log2(e)/2)/tau_x and /tau_t
    double Pmu;       // mu0 / (tau_x^D tau_t (2 pi)^((D+1)/2))
    double iPmu, lPmu;  // 1 / Pmu and log(Pmu), so a row needs one division and one log
    double Cg;        // 1 / (tau_x^2 kx): scaled pass-2 sums -> d ell / d x
    double s_min;     // rows with S_n < s_min are recomputed in FP64
    double mu0, tau_x, tau_t, theta, omega, h;
};


// Device workspace views handed to the kernels.
struct Work {
    const SetDesc *sets;
    int32_t nsets;
    float4 *rec;
    float *w32;
    float *cm32;
    int32_t *tie_end;
    int32_t *perm;
    double *t64;
    double *x64;
    double *lam64;       // lambda_n (FP64) per row
    double *w64;         // 1 / lambda_n per row
    double *Lam64;       // Lambda_n per row
    double *lnl;         // log lambda_n - Lambda_n per row
    float *P1;
    float *P2;
    double *F1;          // FP64 pair-kernel partials (rates)
    double *F2;          // FP64 pair-kernel partials (gradients)
    double *theta_rows;  // per-row Theta-gradient sums (kPass1ThetaVals per row, FP64)
    int32_t *seg_count;  // flagged rows of each finalize segment
    int32_t *seg_rows;   // their set-relative rows (kSegRows slots per segment)
    double *seg_sum;     // each segment's sum of lnl over its unflagged rows
    double *set_loglik;  // ell per set
    double *theta_parts; // kThetaParts x 6 partial sums of the Theta gradient
    int32_t *set_flags;  // bit 0: some rate of the set is zero; bit 1: the set has flagged rows
    int32_t *set_cmmax;  // per set: max(0, max_n cm32[n]) as float bits (gradient-pass skip bound)
    int32_t skip_far;    // skip pair blocks whose kernel values all underflow
    int32_t *pair_ctr;   // a pair launch's own [0] work items taken, [1] CTAs done
    unsigned *status;    // sticky device status
    int32_t *set_done;   // finalizing CTAs done per set: the last one writes ell (returns to zero)
    int32_t sm_count;    // SMs of the device
    // the BMDS term carried by the gradient pass of a BMDS-Hawkes trajectory
    // (one set; null ysort: none): Y in time order (FP32, npad x npad),
    // 1/sigma and 1/sigma2 in FP32 (pair kernel) and FP64 (flagged rows)
    const float *ysort;
    float bmds_inv_sigma, bmds_inv_s2;
    double bmds_inv_sigma_d, bmds_inv_s2_d;
};

// ------------------------------------------------------------ launchers --
// Host functions that enqueue the kernels of one translation unit.  Row
// loops locate their set by binary search in set_row0 (nsets+1 entries).

// hk_prep.cu
cudaError_t launch_validate_keys(const double *t, const double *X, int64_t n_total, int64_t x_total,
                                 double *keys, int32_t *vals, const int64_t *set_ev0, int32_t nsets,
                                 unsigned *status, cudaStream_t s);
size_t sort_temp_bytes(int64_t n_total, int32_t nsets);
cudaError_t launch_sort(void *temp, size_t temp_bytes, const double *t, double *keys_in, double *keys_out,
                        int32_t *vals_in, int32_t *vals_out, int64_t n_total, int32_t nsets,
                        const int64_t *d_set_ev0, cudaStream_t s, int64_t *launches, int64_t *lib_launches);
cudaError_t launch_identity_order(const double *t, double *keys_out, int32_t *vals_out, int64_t n_total,
                                  const int64_t *set_ev0, int32_t nsets, unsigned *status, cudaStream_t s);
cudaError_t launch_pack_rows(const Work &w, const double *X, const double *keys_sorted, const int32_t *vals_sorted,
                             int64_t total_rows, const int64_t *set_row0, cudaStream_t s);

// hk_pairs_mixed_*.cu.  pass: 1 rates, 2 gradient, 3 rates with Theta
// sums, 4 rates with the self-excitation sums apart, 5 gradient with the BMDS
// term.  Shape: wr row groups (block size 32 rows_per_lane(d) wr) and wc
// column groups of warps.
cudaError_t launch_pair_pass_mixed(int pass, int d, const Work &w, const Sched &sc, int grid,
                                   int wr, int wc, cudaStream_t s);
size_t pass_smem_bytes(int d, int pass, int wr, int wc);
int pass_max_ctas_per_sm(int d, int pass, int wr, int wc);
// hk_pairs_mixed_any.cu: the rate (1) or gradient (2) pass over every
// dimension of a plan in one launch (warps row groups, one column group).
cudaError_t launch_pair_pass_any_d(int pass, const Work &w, const Sched &sc, int grid,
                                   int warps, cudaStream_t s);
int pass_any_d_max_ctas_per_sm(int pass, int warps);

// hk_pairs_fp64.cu
constexpr int kFp64Rows = 128;  // rows per CTA of the FP64 pair kernels
cudaError_t launch_pass1_fp64(const Work &w, int32_t set_lo, int32_t set_hi, int32_t max_fsplit, int64_t max_nblk,
                              bool theta, cudaStream_t s);
cudaError_t launch_pass2_fp64(const Work &w, int32_t set_lo, int32_t set_hi, int32_t max_fsplit, int64_t max_nblk,
                              cudaStream_t s);

// hk_pairs_fp64_sym.cu: one CTA per pair block {I, J} (I <= J) of kSymRows
// rows, dimension d, over the items of one launch of the pair schedule
// (fsplit = nslot slots).
constexpr int kSymRows = 256;
cudaError_t launch_pass1_fp64_sym(int d, const Work &w, const Sched &sc, bool theta,
                                  cudaStream_t s);
cudaError_t launch_pass2_fp64_sym(int d, const Work &w, const Sched &sc, cudaStream_t s);

// hk_finalize.cu
// After a later phase of the pair schedule: add the scratch slots of every
// set of the launch's work list (its off-diagonal runs) into its slots and
// clear them.  part: 0 P1 (vpc values per slot), 1 P2 (d), 2 F1 (1), 3 F1
// with the Theta sums (6), 4 F2 (d).
cudaError_t launch_fold_slots(const Work &w, const Sched &sc, int part, cudaStream_t s);
// Rates, ell per set (out_loglik, nullable; not formed when !ell) and the
// FP64 recompute of the flagged rows, one CTA per segment; sums: the rate
// pass's extra row sums.
cudaError_t launch_finalize_rows(const Work &w, int32_t total_segs, bool fp64, int sums, double *out_loglik,
                                 cudaStream_t s, bool ell = true);
cudaError_t launch_theta_grad(const Work &w, int64_t n, double *out6, cudaStream_t s);
// Gradient rows from the pass-2 slots (with the flagged rows' FP64 terms
// and own gradients), in the caller's layout and sorted; one CTA per segment.
cudaError_t launch_finalize_grad(const Work &w, int32_t total_segs, bool fp64, double *out_grad, double *g_sorted,
                                 cudaStream_t s);
cudaError_t launch_self_excitation(const Work &w, int32_t total_segs, double *out, cudaStream_t s);

// hk_hmc.cu
cudaError_t launch_gather_sorted(const Work &w, const int64_t *set_row0, const double *src, double *dst,
                                 int64_t total_rows, double pad, cudaStream_t s);
cudaError_t launch_kick_drift(const Work &w, const int64_t *set_row0, double *p, const double *g, const double *lo,
                              const double *hi, const double *eps_dev, int64_t total_rows, int kicks, bool repack,
                              int32_t *refl_bad, cudaStream_t s);
cudaError_t launch_kick(const Work &w, const int64_t *set_row0, double *p, const double *g, const double *eps_dev,
                        int64_t total_rows, cudaStream_t s);
constexpr int kEnergyParts = 32;  // CTAs per set in the HMC energy reduction
cudaError_t launch_energy(const Work &w, const double *p, double *H_out, double *parts, cudaStream_t s);
cudaError_t launch_accept(const double *H0, const double *H1, const double *log_u, const int32_t *refl_bad,
                          int32_t *accepted, int nsets, cudaStream_t s);
cudaError_t launch_scatter(const Work &w, const int64_t *set_row0, const double *Xs, double *X_out,
                           const int32_t *accepted, int64_t total_rows, cudaStream_t s);
cudaError_t launch_to_caller(const Work &w, const int64_t *set_row0, const double *Xs, double *X_out,
                             int64_t total_rows, cudaStream_t s);
cudaError_t launch_add_caller_term(const Work &w, const int64_t *set_row0, const double *g, double *g_sorted,
                                   int64_t total_rows, const double *ell_add, cudaStream_t s);

// hk_bmds.cu (BMDS likelihood of Eq. (4) and its gradients)
size_t bmds_workspace_bytes(int64_t n, int d, bool fp64);
// Y in time order for the gradient pass with the BMDS term: Ys[i npad + j] =
// Y[perm_i][perm_j] in FP32 (read from the lower triangle), 0 on the
// diagonal and for padded rows or columns (i or j >= n).
cudaError_t launch_bmds_sort_y(const void *Y, bool y_f32, const int32_t *perm, int64_t n, int64_t npad, float *Ys,
                               cudaStream_t s);
// value = false (mixed precision only): the gradient alone; out_loglik and
// out_grad_sigma2 then receive meaningless values.
cudaError_t launch_bmds(const void *Y, bool y_f32, const double *X, int64_t n, int d, double sigma2, bool fp64, void *ws,
                        unsigned *status, double *out_loglik, double *out_grad, double *out_grad_sigma2,
                        cudaStream_t s, int64_t *launches, bool value = true);

}  // namespace hk
