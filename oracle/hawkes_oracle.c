/*
 * FP64 CPU oracle for the spatiotemporal Hawkes log-likelihood and its
 * gradients (Holbrook, Ji & Suchard, "Bayesian mitigation of spatial
 * coarsening for a Hawkes model applied to gunfire, wildfire and viral
 * contagion").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never calls it and shares no code with it.
 *
 * Every quantity is the plain definition from the paper, evaluated in double
 * precision with Neumaier-compensated sums, std libm exp/erfc, and no
 * blocking, fusion or reordering beyond the definition.  Rows are
 * independent, so an optional OpenMP loop over rows does not change any
 * result: each row's sum is taken by one thread in a fixed order.
 *
 * Readings of the paper used here (each one is also listed in the design
 * notes):
 *   - phi is the standard D-variate normal density (2 pi)^(-D/2) exp(-|z|^2/2),
 *     the only reading under which each kernel integrates to exactly 1 over
 *     R^D, as the closed form for Lambda in Section 2.1 requires.
 *   - The sigma_x of the Appendix A gradient is the self-excitation spatial
 *     bandwidth h (it is the only spatial scale in xi).
 *   - T = t_N is the largest event time passed in; the window starts at 0.
 *   - Both indicators act on times: I[t_n != t_n'] on the background term and
 *     I[t_n' < t_n] on the self-excitation term; exactly tied events excite
 *     neither each other's background nor self-excitation rate.
 *   - The Theta-gradient (not printed in the paper) differentiates the rate
 *     and Lambda of Section 2.1 with respect to the natural parameters
 *     (mu0, tau_x, tau_t, theta, omega, h).
 *   - HMC (Section 3, Neal 2011) uses an identity mass matrix, the caller's
 *     momenta and log-uniform draw, and reflection at box walls.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared
 *        (the contraction switch keeps a*b+c unfused on every host).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1

/* Theta = (mu0, tau_x, tau_t, theta, omega, h), in the order of Section 2.1. */
typedef struct {
    double mu0, tau_x, tau_t, theta, omega, h;
} oracle_params;

int oracle_bmds(int64_t n, int32_t d, const double *Y, const double *X, double sigma2, double *out_loglik,
                double *grad, double *grad_sigma2, int32_t nthreads);

static const double kPi = 3.14159265358979323846;

/* ---------------------------------------------------------------- sums -- */

/* Neumaier's compensated summation. */
typedef struct {
    double s, c;
} nsum;

static void nadd(nsum *a, double x)
{
    double t = a->s + x;
    if (!isfinite(t)) {
        /* an infinite term (log of a zero rate) makes the sum infinite; the
           compensation would turn inf - inf into NaN, so it is not kept */
        a->s = t;
        a->c = 0.0;
        return;
    }
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nval(const nsum *a) { return isfinite(a->s) ? a->s + a->c : a->s; }

/* -------------------------------------------------------------- kernels -- */

/* Standard D-variate normal density at a point z with |z|^2 = z2. */
static double phi_d(double z2, int d)
{
    return pow(2.0 * kPi, -0.5 * (double)d) * exp(-0.5 * z2);
}

/* Standard normal CDF through the complementary error function. */
static double Phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

static int params_ok(const oracle_params *p)
{
    return p && p->mu0 > 0 && p->tau_x > 0 && p->tau_t > 0 && p->theta > 0 &&
           p->omega > 0 && p->h > 0 && isfinite(p->mu0) && isfinite(p->tau_x) &&
           isfinite(p->tau_t) && isfinite(p->theta) && isfinite(p->omega) &&
           isfinite(p->h);
}

static double sqdist(int d, const double *a, const double *b)
{
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
        double diff = a[k] - b[k];
        r2 += diff * diff;
    }
    return r2;
}

/*
 * Background term mu_{nn'} of the rate lambda_n (Section 2.1, the kernel
 * smoother with the indicator I[t != t_n], as it appears inside Eq. (1)):
 *   mu0 / (tau_x^D tau_t) * phi((x_n - x_n')/tau_x) * phi((t_n - t_n')/tau_t)
 *   * I[t_n != t_n'].
 */
static double mu_term(int d, const double *xn, double tn, const double *xm,
                      double tm, const oracle_params *p)
{
    if (tn == tm)
        return 0.0;
    double r2 = sqdist(d, xn, xm);
    double dt = tn - tm;
    return p->mu0 / (pow(p->tau_x, (double)d) * p->tau_t) *
           phi_d(r2 / (p->tau_x * p->tau_x), d) *
           phi_d(dt * dt / (p->tau_t * p->tau_t), 1);
}

/*
 * Self-excitation term xi_{nn'} (Section 2.1, exponential in time and
 * Gaussian in space, as it appears inside Eq. (1)):
 *   theta omega / h^D * exp(-omega (t_n - t_n')) * phi((x_n - x_n')/h)
 *   * I[t_n' < t_n].
 */
static double xi_term(int d, const double *xn, double tn, const double *xm,
                      double tm, const oracle_params *p)
{
    if (!(tm < tn))
        return 0.0;
    double r2 = sqdist(d, xn, xm);
    double dt = tn - tm;
    return p->theta * p->omega / pow(p->h, (double)d) * exp(-p->omega * dt) *
           phi_d(r2 / (p->h * p->h), d);
}

/* ------------------------------------------------------------------ rates -- */

/*
 * lambda_n = sum_{n'=1..N} (mu_{nn'} + xi_{nn'})  (Eq. (1); Appendix A defines
 * lambda_n as this row sum).  The n' = n term vanishes through both
 * indicators, so the loop runs over every n'.
 * Optionally returns the two parts M_n = sum mu and X_n = sum xi.
 */
static void rate_row(int64_t n, int d, const double *t, const double *X,
                     const oracle_params *p, int64_t row, double *lam,
                     double *lam_mu, double *lam_xi)
{
    nsum s_mu = {0, 0}, s_xi = {0, 0}, s = {0, 0};
    const double *xn = X + row * d;
    for (int64_t m = 0; m < n; ++m) {
        double mu = mu_term(d, xn, t[row], X + m * d, t[m], p);
        double xi = xi_term(d, xn, t[row], X + m * d, t[m], p);
        nadd(&s_mu, mu);
        nadd(&s_xi, xi);
        nadd(&s, mu + xi);
    }
    *lam = nval(&s);
    if (lam_mu)
        *lam_mu = nval(&s_mu);
    if (lam_xi)
        *lam_xi = nval(&s_xi);
}

/* lambda_n for every row (Eq. (1)). */
int oracle_rates(int64_t n, int32_t d, const double *t, const double *X,
                 const oracle_params *p, double *lam, double *lam_mu,
                 double *lam_xi, int32_t nthreads)
{
    if (n < 0 || d < 1 || !params_ok(p) || (n > 0 && (!t || !X || !lam)))
        return ORACLE_ERR_ARG;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < n; ++i)
        rate_row(n, d, t, X, p, i, &lam[i], lam_mu ? &lam_mu[i] : NULL,
                 lam_xi ? &lam_xi[i] : NULL);
    (void)nthreads;
    return ORACLE_OK;
}

/* lambda_n for a listed subset of rows (same definition). */
int oracle_rates_rows(int64_t n, int32_t d, const double *t, const double *X,
                      const oracle_params *p, int64_t nrows, const int64_t *rows,
                      double *lam, int32_t nthreads)
{
    if (n < 0 || d < 1 || !params_ok(p) || nrows < 0 ||
        (nrows > 0 && (!rows || !lam || !t || !X)))
        return ORACLE_ERR_ARG;
    for (int64_t k = 0; k < nrows; ++k)
        if (rows[k] < 0 || rows[k] >= n)
            return ORACLE_ERR_ARG;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t k = 0; k < nrows; ++k)
        rate_row(n, d, t, X, p, rows[k], &lam[k], NULL, NULL);
    (void)nthreads;
    return ORACLE_OK;
}

/* ----------------------------------------------------------- integrated -- */

static double max_time(int64_t n, const double *t)
{
    double T = t[0];
    for (int64_t i = 1; i < n; ++i)
        if (t[i] > T)
            T = t[i];
    return T;
}

/*
 * Lambda_n of Section 2.1 (closed form of the space-time integral of the
 * rate over R^D x [0, t_N]):
 *   mu0 (Phi((T - t_n)/tau_t) - Phi(-t_n/tau_t)) - theta (exp(-omega (T - t_n)) - 1)
 * with T = t_N the largest time.  Writes every Lambda_n (nullable) and
 * returns their compensated sum.
 */
double oracle_Lambda(int64_t n, const double *t, const oracle_params *p,
                     double *Lambda_n)
{
    if (n <= 0)
        return 0.0;
    double T = max_time(n, t);
    nsum s = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double a = T - t[i];
        double L = p->mu0 * (Phi(a / p->tau_t) - Phi(-t[i] / p->tau_t)) -
                   p->theta * (exp(-p->omega * a) - 1.0);
        if (Lambda_n)
            Lambda_n[i] = L;
        nadd(&s, L);
    }
    return nval(&s);
}

/*
 * Log-likelihood of Eq. (1): ell = sum_n log(lambda_n) - sum_n Lambda_n.
 * A zero rate gives ell = -inf.  lam_out (nullable) receives lambda_n.
 */
int oracle_loglik(int64_t n, int32_t d, const double *t, const double *X,
                  const oracle_params *p, double *out_loglik, double *lam_out,
                  int32_t nthreads)
{
    if (n < 1 || d < 1 || !params_ok(p) || !t || !X || !out_loglik)
        return ORACLE_ERR_ARG;
    double *lam = lam_out ? lam_out : (double *)malloc(sizeof(double) * n);
    if (!lam)
        return ORACLE_ERR_ARG;
    oracle_rates(n, d, t, X, p, lam, NULL, NULL, nthreads);
    nsum s = {0, 0};
    for (int64_t i = 0; i < n; ++i)
        nadd(&s, log(lam[i]));
    double Lam = oracle_Lambda(n, t, p, NULL);
    *out_loglik = nval(&s) - Lam;
    if (!lam_out)
        free(lam);
    return ORACLE_OK;
}

/* ------------------------------------------------------------ gradients -- */

/*
 * d ell / d x_n, Appendix A, with sigma_x read as h:
 *   sum_{n'} [ (mu_{nn'}/lambda_n + mu_{n'n}/lambda_n') / tau_x^2
 *            + (xi_{nn'}/lambda_n + xi_{n'n}/lambda_n') / h^2 ] (x_n' - x_n).
 * Evaluated as the plain ordered double loop: both directions of every term
 * are computed from their own definitions.
 */
static void grad_row(int64_t n, int d, const double *t, const double *X,
                     const oracle_params *p, const double *lam, int64_t row,
                     double *g)
{
    nsum acc[64];
    for (int k = 0; k < d; ++k)
        acc[k].s = acc[k].c = 0.0;
    const double *xn = X + row * d;
    double tx2 = p->tau_x * p->tau_x, h2 = p->h * p->h;
    for (int64_t m = 0; m < n; ++m) {
        const double *xm = X + m * d;
        double mu_nm = mu_term(d, xn, t[row], xm, t[m], p);
        double mu_mn = mu_term(d, xm, t[m], xn, t[row], p);
        double xi_nm = xi_term(d, xn, t[row], xm, t[m], p);
        double xi_mn = xi_term(d, xm, t[m], xn, t[row], p);
        double coef = (mu_nm / lam[row] + mu_mn / lam[m]) / tx2 +
                      (xi_nm / lam[row] + xi_mn / lam[m]) / h2;
        if (coef == 0.0)
            continue;
        for (int k = 0; k < d; ++k)
            nadd(&acc[k], coef * (xm[k] - xn[k]));
    }
    for (int k = 0; k < d; ++k)
        g[k] = nval(&acc[k]);
}

/* Location gradient for every row; lam must hold lambda_n for all rows. */
int oracle_grad_locations(int64_t n, int32_t d, const double *t, const double *X,
                          const oracle_params *p, const double *lam, double *grad,
                          int32_t nthreads)
{
    if (n < 1 || d < 1 || d > 64 || !params_ok(p) || !t || !X || !lam || !grad)
        return ORACLE_ERR_ARG;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < n; ++i)
        grad_row(n, d, t, X, p, lam, i, grad + i * d);
    (void)nthreads;
    return ORACLE_OK;
}

/* Location gradient for a listed subset of rows (lam over all rows). */
int oracle_grad_rows(int64_t n, int32_t d, const double *t, const double *X,
                     const oracle_params *p, const double *lam, int64_t nrows,
                     const int64_t *rows, double *grad, int32_t nthreads)
{
    if (n < 1 || d < 1 || d > 64 || !params_ok(p) || nrows < 0 ||
        (nrows > 0 && (!rows || !grad)) || !t || !X || !lam)
        return ORACLE_ERR_ARG;
    for (int64_t k = 0; k < nrows; ++k)
        if (rows[k] < 0 || rows[k] >= n)
            return ORACLE_ERR_ARG;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t k = 0; k < nrows; ++k)
        grad_row(n, d, t, X, p, lam, rows[k], grad + k * d);
    (void)nthreads;
    return ORACLE_OK;
}

/*
 * Gradient of ell with respect to Theta = (mu0, tau_x, tau_t, theta, omega, h).
 * The paper prints no formula; this differentiates the two rate terms of
 * Section 2.1 and the closed form of Lambda, with a_n = T - t_n:
 *   d/d mu0   = sum_n M_n / (mu0 lambda_n) - sum_n [Phi(a/tau_t) - Phi(-t_n/tau_t)]
 *   d/d tau_x = sum_n lambda_n^-1 sum_n' mu_{nn'} (r^2/tau_x^3 - D/tau_x)
 *   d/d tau_t = sum_n lambda_n^-1 sum_n' mu_{nn'} (dt^2/tau_t^3 - 1/tau_t)
 *               + mu0 sum_n [phi(a/tau_t) a + phi(t_n/tau_t) t_n] / tau_t^2
 *   d/d theta = sum_n X_n / (theta lambda_n) - sum_n [1 - exp(-omega a)]
 *   d/d omega = sum_n lambda_n^-1 sum_n' xi_{nn'} (1/omega - dt)
 *               - theta sum_n a exp(-omega a)
 *   d/d h     = sum_n lambda_n^-1 sum_n' xi_{nn'} (r^2/h^3 - D/h)
 * lam must hold lambda_n for all rows.
 */
/*
 * d ell / d Theta and, when scale6 is not NULL, the magnitude of the terms
 * each component is summed from: for component k, the sum over rows of
 * lambda_n^-1 sum_n' (|first piece| + |second piece|) of the pair terms
 * below, plus the absolute values of the Lambda derivatives.  That is the
 * quantity a rounding error in the row sums is relative to, whatever
 * cancellation the total itself shows (near the data-generating Theta each
 * score is a sum of N terms of either sign).  The total is computed exactly
 * as without the scale.
 */
static int grad_params_impl(int64_t n, int32_t d, const double *t, const double *X,
                            const oracle_params *p, const double *lam, double *out6,
                            double *scale6, int32_t nthreads)
{
    if (n < 1 || d < 1 || !params_ok(p) || !t || !X || !lam || !out6)
        return ORACLE_ERR_ARG;
    double *rowv = (double *)malloc(sizeof(double) * 12 * n);
    if (!rowv)
        return ORACLE_ERR_ARG;
    double *rowm = rowv + 6 * n;
    double tx = p->tau_x, tt = p->tau_t, h = p->h, w = p->omega;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < n; ++i) {
        nsum a[6], b[6];
        for (int k = 0; k < 6; ++k)
            a[k].s = a[k].c = b[k].s = b[k].c = 0.0;
        const double *xi_ = X + i * d;
        for (int64_t m = 0; m < n; ++m) {
            const double *xm = X + m * d;
            double mu = mu_term(d, xi_, t[i], xm, t[m], p);
            double xi = xi_term(d, xi_, t[i], xm, t[m], p);
            double r2 = sqdist(d, xi_, xm);
            double dt = t[i] - t[m];
            nadd(&a[0], mu / p->mu0);
            nadd(&a[1], mu * (r2 / (tx * tx * tx) - (double)d / tx));
            nadd(&a[2], mu * (dt * dt / (tt * tt * tt) - 1.0 / tt));
            nadd(&a[3], xi / p->theta);
            nadd(&a[4], xi * (1.0 / w - dt));
            nadd(&a[5], xi * (r2 / (h * h * h) - (double)d / h));
            if (scale6) {
                nadd(&b[0], mu / p->mu0);
                nadd(&b[1], mu * (r2 / (tx * tx * tx) + (double)d / tx));
                nadd(&b[2], mu * (dt * dt / (tt * tt * tt) + 1.0 / tt));
                nadd(&b[3], xi / p->theta);
                nadd(&b[4], xi * (1.0 / w + fabs(dt)));
                nadd(&b[5], xi * (r2 / (h * h * h) + (double)d / h));
            }
        }
        for (int k = 0; k < 6; ++k) {
            rowv[6 * i + k] = nval(&a[k]) / lam[i];
            rowm[6 * i + k] = scale6 ? nval(&b[k]) / lam[i] : 0.0;
        }
    }
    (void)nthreads;
    double T = max_time(n, t);
    nsum s[6], sm[6];
    for (int k = 0; k < 6; ++k)
        s[k].s = s[k].c = sm[k].s = sm[k].c = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double a_ = T - t[i];
        for (int k = 0; k < 6; ++k)
            nadd(&s[k], rowv[6 * i + k]);
        double l0 = -(Phi(a_ / tt) - Phi(-t[i] / tt));
        double l2 = p->mu0 * (phi_d(a_ * a_ / (tt * tt), 1) * a_ + phi_d(t[i] * t[i] / (tt * tt), 1) * t[i]) /
                    (tt * tt);
        double l3 = -(1.0 - exp(-w * a_));
        double l4 = -p->theta * a_ * exp(-w * a_);
        nadd(&s[0], l0);
        nadd(&s[2], l2);
        nadd(&s[3], l3);
        nadd(&s[4], l4);
        if (scale6) {
            for (int k = 0; k < 6; ++k)
                nadd(&sm[k], rowm[6 * i + k]);
            nadd(&sm[0], fabs(l0));
            nadd(&sm[2], fabs(l2));
            nadd(&sm[3], fabs(l3));
            nadd(&sm[4], fabs(l4));
        }
    }
    for (int k = 0; k < 6; ++k) {
        out6[k] = nval(&s[k]);
        if (scale6)
            scale6[k] = nval(&sm[k]);
    }
    free(rowv);
    return ORACLE_OK;
}

int oracle_grad_params(int64_t n, int32_t d, const double *t, const double *X,
                       const oracle_params *p, const double *lam, double *out6,
                       int32_t nthreads)
{
    return grad_params_impl(n, d, t, X, p, lam, out6, NULL, nthreads);
}

int oracle_grad_params_scaled(int64_t n, int32_t d, const double *t, const double *X,
                              const oracle_params *p, const double *lam, double *out6,
                              double *scale6, int32_t nthreads)
{
    if (!scale6)
        return ORACLE_ERR_ARG;
    return grad_params_impl(n, d, t, X, p, lam, out6, scale6, nthreads);
}

/* ------------------------------------------------------------------ HMC -- */

/*
 * Reflection of one coordinate at the walls of its box [lo, hi] (Neal 2011,
 * Section 5.1): a coordinate that leaves the box is mirrored back across
 * the wall it crossed and its momentum changes sign, repeatedly, until it
 * lies inside.  Returns 0, or 1 when 1000 reflections did not suffice.
 */
static int reflect(double *x, double *pm, double lo, double hi)
{
    for (int it = 0; it < 1000; ++it) {
        if (*x < lo) {
            *x = 2.0 * lo - *x;
            *pm = -*pm;
        } else if (*x > hi) {
            *x = 2.0 * hi - *x;
            *pm = -*pm;
        } else {
            return 0;
        }
    }
    return 1;
}

static int ell_and_grad(int64_t n, int d, const double *t, const double *X,
                        const oracle_params *p, double *lam, double *ell,
                        double *g, int32_t nthreads)
{
    int rc = oracle_loglik(n, d, t, X, p, ell, lam, nthreads);
    if (rc)
        return rc;
    return oracle_grad_locations(n, d, t, X, p, lam, g, nthreads);
}

/*
 * One HMC proposal over the locations (Section 3: HMC over X, Neal 2011).
 * Potential U(X) = -ell(X) (the uniform box prior is constant inside the
 * box), identity mass matrix.  Each of the n_steps leapfrog steps is
 *   p += (eps/2) grad ell(X);  X += eps p;  reflect at box walls;
 *   p += (eps/2) grad ell(X_new)
 * with the gradient at the end of one step reused at the start of the next.
 * H = -ell + |p|^2 / 2.  The proposal is accepted when log_u < H0 - H1 (a
 * non-finite H1 rejects).  X_out receives the accepted state (the proposal,
 * or X0 on rejection); p_out (nullable) the final momenta of the proposal.
 * box_lo/box_hi are n*d arrays or both NULL (unconstrained).
 */
/*
 * Potential energy -U = ell(X) and its gradient for the HMC below: the
 * Hawkes log-likelihood of Eq. (1) alone, or, for the BMDS-Hawkes model of
 * Section 2.2.3, plus the BMDS log-likelihood of Eq. (4) with distances Y
 * and variance sigma2 (both terms' gradients in X add).
 */
static int hmc_potential(int64_t n, int32_t d, const double *t, const double *X, const oracle_params *p,
                         const double *Y, double sigma2, double *lam, double *ell, double *g, int32_t nthreads)
{
    ell_and_grad(n, d, t, X, p, lam, ell, g, nthreads);
    if (!Y)
        return ORACLE_OK;
    double *gb = (double *)malloc(sizeof(double) * n * d);
    double lb = 0.0;
    if (!gb)
        return ORACLE_ERR_ARG;
    int rc = oracle_bmds(n, d, Y, X, sigma2, &lb, gb, NULL, nthreads);
    *ell += lb;
    for (int64_t i = 0; i < n * d; ++i)
        g[i] += gb[i];
    free(gb);
    return rc;
}

static int hmc_core(int64_t n, int32_t d, const double *t, const double *X0, const double *p0,
                    const double *box_lo, const double *box_hi, const oracle_params *p, const double *Y,
                    double sigma2, double eps, int32_t n_steps, double log_u, double *X_out, double *p_out,
                    double *out_H0, double *out_H1, int32_t *out_accepted, int32_t nthreads)
{
    if (n < 1 || d < 1 || !params_ok(p) || !t || !X0 || !p0 || !X_out ||
        n_steps < 0 || !(eps > 0) || ((box_lo == NULL) != (box_hi == NULL)))
        return ORACLE_ERR_ARG;
    int64_t nd = n * d;
    double *X = (double *)malloc(sizeof(double) * nd);
    double *pm = (double *)malloc(sizeof(double) * nd);
    double *g = (double *)malloc(sizeof(double) * nd);
    double *lam = (double *)malloc(sizeof(double) * n);
    if (!X || !pm || !g || !lam) {
        free(X);
        free(pm);
        free(g);
        free(lam);
        return ORACLE_ERR_ARG;
    }
    memcpy(X, X0, sizeof(double) * nd);
    memcpy(pm, p0, sizeof(double) * nd);
    double ell;
    int rc = hmc_potential(n, d, t, X, p, Y, sigma2, lam, &ell, g, nthreads);
    nsum k0 = {0, 0};
    for (int64_t i = 0; i < nd; ++i)
        nadd(&k0, 0.5 * (pm[i] * pm[i]));
    double H0 = -ell + nval(&k0);
    double half = 0.5 * eps;
    int bad = 0;
    for (int32_t s = 0; s < n_steps && rc == ORACLE_OK; ++s) {
        for (int64_t i = 0; i < nd; ++i)
            pm[i] = pm[i] + half * g[i];
        for (int64_t i = 0; i < nd; ++i) {
            X[i] = X[i] + eps * pm[i];
            if (box_lo)
                bad |= reflect(&X[i], &pm[i], box_lo[i], box_hi[i]);
        }
        rc = hmc_potential(n, d, t, X, p, Y, sigma2, lam, &ell, g, nthreads);
        for (int64_t i = 0; i < nd; ++i)
            pm[i] = pm[i] + half * g[i];
    }
    nsum k1 = {0, 0};
    for (int64_t i = 0; i < nd; ++i)
        nadd(&k1, 0.5 * (pm[i] * pm[i]));
    double H1 = -ell + nval(&k1);
    int acc = (!bad && isfinite(H1) && isfinite(H0) && log_u < H0 - H1) ? 1 : 0;
    memcpy(X_out, acc ? X : X0, sizeof(double) * nd);
    if (p_out)
        memcpy(p_out, pm, sizeof(double) * nd);
    if (out_H0)
        *out_H0 = H0;
    if (out_H1)
        *out_H1 = H1;
    if (out_accepted)
        *out_accepted = acc;
    free(X);
    free(pm);
    free(g);
    free(lam);
    return rc;
}

int oracle_hmc_trajectory(int64_t n, int32_t d, const double *t,
                          const double *X0, const double *p0,
                          const double *box_lo, const double *box_hi,
                          const oracle_params *p, double eps, int32_t n_steps,
                          double log_u, double *X_out, double *p_out,
                          double *out_H0, double *out_H1, int32_t *out_accepted,
                          int32_t nthreads)
{
    return hmc_core(n, d, t, X0, p0, box_lo, box_hi, p, NULL, 0.0, eps, n_steps, log_u, X_out, p_out, out_H0,
                    out_H1, out_accepted, nthreads);
}

/* HMC over the latent locations of the BMDS-Hawkes model (Section 3:
 * potential -ell_Hawkes - ell_BMDS, unconstrained locations as in the
 * influenza application), otherwise as oracle_hmc_trajectory. */
int oracle_bmds_hmc_trajectory(int64_t n, int32_t d, const double *t, const double *X0, const double *p0,
                               const oracle_params *p, const double *Y, double sigma2, double eps,
                               int32_t n_steps, double log_u, double *X_out, double *p_out, double *out_H0,
                               double *out_H1, int32_t *out_accepted, int32_t nthreads)
{
    if (!Y || !(sigma2 > 0) || !isfinite(sigma2))
        return ORACLE_ERR_ARG;
    return hmc_core(n, d, t, X0, p0, NULL, NULL, p, Y, sigma2, eps, n_steps, log_u, X_out, p_out, out_H0, out_H1,
                    out_accepted, nthreads);
}

/* ----------------------------------------------------------------- BMDS -- */

/*
 * Bayesian multidimensional scaling likelihood of Section 2.2.3, Eq. (4):
 * observed distances y_nn' (n > n') are truncated normals around the latent
 * distances delta_nn' = |x_n - x_n'| with variance sigma2, so up to an
 * additive constant
 *   ell_B = N (1 - N) / 4 log(sigma2) - sum_{n > n'} r_nn',
 *   r_nn' = (y_nn' - delta_nn')^2 / (2 sigma2) + log Phi(delta_nn' / sigma).
 * Y is N x N row-major; only the entries below the diagonal (n > n') are
 * read.  grad (nullable) receives d ell_B / d x_n:
 *   -sum_{n' != n} dr/d delta (x_n - x_n') / delta,
 *   dr/d delta = -(y - delta)/sigma2 + phi(delta/sigma) / (sigma Phi(delta/sigma)),
 * and grad_sigma2 (nullable) d ell_B / d sigma2:
 *   N (1 - N) / (4 sigma2) + sum (y - delta)^2 / (2 sigma2^2)
 *   + sum phi(delta/sigma) delta / (2 sigma^3 Phi(delta/sigma)).
 */
static double bmds_y(const double *Y, int64_t n, int64_t a, int64_t b)
{
    return a > b ? Y[a * n + b] : Y[b * n + a];
}

int oracle_bmds(int64_t n, int32_t d, const double *Y, const double *X, double sigma2, double *out_loglik,
                double *grad, double *grad_sigma2, int32_t nthreads)
{
    if (n < 1 || d < 1 || d > 64 || !Y || !X || !out_loglik || !(sigma2 > 0) || !isfinite(sigma2))
        return ORACLE_ERR_ARG;
    const double sigma = sqrt(sigma2);
    double *row_r = (double *)malloc(sizeof(double) * n);
    double *row_s = (double *)malloc(sizeof(double) * n);
    if (!row_r || !row_s) {
        free(row_r);
        free(row_s);
        return ORACLE_ERR_ARG;
    }
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < n; ++i) {
        nsum r = {0, 0}, ss = {0, 0};
        nsum g[64];
        for (int k = 0; k < d; ++k)
            g[k].s = g[k].c = 0.0;
        for (int64_t m = 0; m < n; ++m) {
            if (m == i)
                continue;
            const double delta = sqrt(sqdist(d, X + i * d, X + m * d));
            const double y = bmds_y(Y, n, i, m);
            const double z = delta / sigma;
            const double Phi_z = Phi(z);
            const double ratio = phi_d(z * z, 1) / Phi_z;
            if (m < i) {  /* each unordered pair once for the value */
                nadd(&r, (y - delta) * (y - delta) / (2.0 * sigma2) + log(Phi_z));
                nadd(&ss, (y - delta) * (y - delta) / (2.0 * sigma2 * sigma2) + ratio * delta / (2.0 * sigma2 * sigma));
            }
            if (grad && delta > 0.0) {  /* coincident points: no derivative, symmetric subgradient 0 */
                const double drdd = -(y - delta) / sigma2 + ratio / sigma;
                for (int k = 0; k < d; ++k)
                    nadd(&g[k], -drdd * (X[i * d + k] - X[m * d + k]) / delta);
            }
        }
        row_r[i] = nval(&r);
        row_s[i] = nval(&ss);
        if (grad)
            for (int k = 0; k < d; ++k)
                grad[i * d + k] = nval(&g[k]);
    }
    (void)nthreads;
    nsum tot = {0, 0}, tots = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        nadd(&tot, row_r[i]);
        nadd(&tots, row_s[i]);
    }
    const double c = (double)n * (1.0 - (double)n) / 4.0;
    *out_loglik = c * log(sigma2) - nval(&tot);
    if (grad_sigma2)
        *grad_sigma2 = c / sigma2 + nval(&tots);
    free(row_r);
    free(row_s);
    return ORACLE_OK;
}

/* ---------------------------------------------------- MwG proposals -- */

/* x - sin(x) for x in [0, 2 pi], by its Taylor series where the difference
 * would cancel (x < 0.5: terms to x^15, error below 1e-17 x^3). */
static double x_minus_sin(double x)
{
    if (x >= 0.5)
        return x - sin(x);
    const double x2 = x * x;
    double term = x * x2 / 6.0, sum = 0.0;
    for (int k = 1; k <= 7; ++k) {
        sum += term;
        term *= -x2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
    }
    return sum;
}

/*
 * Area of the intersection of two discs with radii R and rho whose centres
 * are c apart (the "asymmetric lens" of the circle proposal, Section 3,
 * Eq. (6)): zero when the discs are apart, the smaller disc when one lies in
 * the other, otherwise the two circular segments cut off by the common
 * chord.  The chord lies at signed distances d1 = (c^2 + R^2 - rho^2)/(2c)
 * and d2 = c - d1 from the centres with half-length h; a segment of a disc
 * of radius r whose chord subtends 2 theta at the centre has area
 * r^2 (2 theta - sin 2 theta) / 2 (sector minus triangle), with
 * theta = atan2(h, d), written so that nothing cancels when one disc is
 * much larger than the other.
 */
double oracle_lens_area(double R, double rho, double c)
{
    if (!(R > 0) || !(rho > 0) || !(c >= 0))
        return NAN;
    if (c >= R + rho)
        return 0.0;
    if (c <= fabs(R - rho)) {
        const double m = R < rho ? R : rho;
        return kPi * m * m;
    }
    const double d1 = (c * c + R * R - rho * rho) / (2.0 * c);
    const double d2 = c - d1;
    double h2 = (R - d1) * (R + d1);
    if (h2 < 0.0)
        h2 = 0.0;
    const double h = sqrt(h2);
    const double th1 = atan2(h, d1), th2 = atan2(h, d2);
    return 0.5 * R * R * x_minus_sin(2.0 * th1) + 0.5 * rho * rho * x_minus_sin(2.0 * th2);
}

/* log of the probability that at least one of `tries` uniform draws from a
 * disc of radius rho lands in a region of area A inside it. */
static double log_success(double A, double rho, int32_t tries)
{
    const double p = A / (kPi * rho * rho);
    if (p >= 1.0)
        return 0.0;
    return log(-expm1((double)tries * log1p(-p)));
}

/*
 * Circle proposals for the D = 2 locations of Eq. (3) (Section 3, Eq. (6)):
 * event b at x_b with prior circle (centre m_b, radius r_b) proposes x*
 * uniform on {|x* - m_b| < r_b, |x* - x_b| < r_b eps}, by rejection from the
 * disc around x_b: try k draws radius r_b eps sqrt(u1) and angle 2 pi u2 from
 * u[(b*tries + k)*2 + {0,1}]; the first draw inside the circle is the
 * proposal.  If all tries miss, the proposal is x_b itself.  Accepted draws
 * are uniform on the lens L(x_b) of area A(x_b), so for x* != x_b
 *   q(x*|x) = (1 - (1 - A(x)/(pi (r eps)^2))^tries) / A(x),
 * and the proposal's log ratio log q(x|x*) - log q(x*|x), summed over the
 * block, is written to *log_q_ratio (0 for events that stay).
 */
int oracle_circle_proposals(int32_t nb, const double *X, const double *centers, const double *radii,
                            double eps, int32_t tries, const double *u, double *X_new, double *log_q_ratio)
{
    if (nb < 0 || tries < 1 || !(eps > 0) || (nb > 0 && (!X || !centers || !radii || !u || !X_new)) ||
        !log_q_ratio)
        return ORACLE_ERR_ARG;
    nsum lq = {0, 0};
    for (int32_t b = 0; b < nb; ++b) {
        const double *x = X + 2 * b, *m = centers + 2 * b;
        const double R = radii[b], rho = R * eps;
        X_new[2 * b] = x[0];
        X_new[2 * b + 1] = x[1];
        for (int32_t k = 0; k < tries; ++k) {
            const double r = rho * sqrt(u[(b * tries + k) * 2]);
            const double ang = 2.0 * kPi * u[(b * tries + k) * 2 + 1];
            const double y0 = x[0] + r * cos(ang), y1 = x[1] + r * sin(ang);
            const double dx = y0 - m[0], dy = y1 - m[1];
            if (dx * dx + dy * dy < R * R) {
                X_new[2 * b] = y0;
                X_new[2 * b + 1] = y1;
                const double A_x = oracle_lens_area(R, rho, hypot(x[0] - m[0], x[1] - m[1]));
                const double A_y = oracle_lens_area(R, rho, hypot(dx, dy));
                nadd(&lq, (log_success(A_y, rho, tries) - log(A_y)) - (log_success(A_x, rho, tries) - log(A_x)));
                break;
            }
        }
    }
    *log_q_ratio = nval(&lq);
    return ORACLE_OK;
}

/* Inverse of the standard normal CDF by bisection on Phi (exact to the last
 * bisection step; slow and plain). */
static double Phi_inv(double p)
{
    if (!(p > 0.0 && p < 1.0))
        return p == 0.0 ? -INFINITY : (p == 1.0 ? INFINITY : NAN);
    double lo = -40.0, hi = 40.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi)
            break;
        if (Phi(mid) < p)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

/*
 * Box proposals for the square priors of Eq. (2) (Section 3: truncated
 * normal proposals): each coordinate k of event b draws
 *   x*_k = x_k + s Phi^{-1}(Phi(a) + u (Phi(b) - Phi(a))),
 *   a = (lo_k - x_k)/s,  b = (hi_k - x_k)/s,
 * from u[b*d + k], i.e. N(x_k, s^2) truncated to [lo_k, hi_k].  The normal
 * parts of q(x|x*) and q(x*|x) cancel, leaving
 *   log q(x|x*) - log q(x*|x) = sum log Z(x) - log Z(x*),
 *   Z(y) = Phi((hi_k - y_k)/s) - Phi((lo_k - y_k)/s),
 * summed over the block into *log_q_ratio.
 */
int oracle_box_proposals(int32_t nb, int32_t d, const double *X, const double *lo, const double *hi, double s,
                         const double *u, double *X_new, double *log_q_ratio)
{
    if (nb < 0 || d < 1 || !(s > 0) || (nb > 0 && (!X || !lo || !hi || !u || !X_new)) || !log_q_ratio)
        return ORACLE_ERR_ARG;
    nsum lq = {0, 0};
    for (int32_t b = 0; b < nb; ++b)
        for (int32_t k = 0; k < d; ++k) {
            const int64_t e = (int64_t)b * d + k;
            const double x = X[e];
            const double Pa = Phi((lo[e] - x) / s), Pb = Phi((hi[e] - x) / s);
            double y = x + s * Phi_inv(Pa + u[e] * (Pb - Pa));
            if (y < lo[e])
                y = lo[e];
            if (y > hi[e])
                y = hi[e];
            X_new[e] = y;
            const double Zx = Pb - Pa;
            const double Zy = Phi((hi[e] - y) / s) - Phi((lo[e] - y) / s);
            nadd(&lq, log(Zx) - log(Zy));
        }
    *log_q_ratio = nval(&lq);
    return ORACLE_OK;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int32_t oracle_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
