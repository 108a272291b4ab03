"""Pins for the FP64 oracle: checks against things other than the oracle itself.

Each pin takes an ``oracle.Oracle`` (the default build, or a deliberately
broken copy in the mutation test) and returns ``(ok, detail)``.  The pins are
chosen so that a plausible mistake anywhere in the oracle -- a dropped term or
indicator, a wrong sign, index or exponent, a transposed operand -- fails at
least one of them (``test_oracle_mutants.py`` plants such mistakes).

What each pin compares against:
  * brute_force   -- the rate as a function of a free point (x, t) from the two
                     sums of Section 2.1, with scipy's normal densities; and the
                     integrated rate by adaptive quadrature in (x, t) (D=1) or
                     in t with the spatial integral checked separately.
  * symbolic_pair -- a two-event case written out by hand and differentiated by
                     sympy at 40 digits (value, location and Theta gradients).
  * finite_diff   -- 4th-order central differences of ell in X and in Theta.
  * invariances   -- translation, spatial and temporal scaling, permutation.
  * euler         -- the two Euler identities implied by the scalings and by
                     linearity of the rate in (mu0, theta).
  * theta_zero    -- with negligible self-excitation, the background weight's
                     score vanishes at mu0* = N / sum_n [Phi(a_n/tau_t) - Phi(-t_n/tau_t)]
                     (Phi from scipy).
  * hmc_*         -- reversibility, O(eps^2) energy error, the accept rule, box
                     walls.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, stats

import synth

P_DEFAULT = {"mu0": 0.6, "tau_x": 0.8, "tau_t": 1.5, "theta": 0.4, "omega": 0.9, "h": 0.3}


def _rel(a, b):
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    den = max(np.max(np.abs(b)), 1e-300)
    return float(np.max(np.abs(a - b)) / den)


# ------------------------------------------------------------ brute force --

def free_point_rate(x, t, T_ev, X_ev, P, parts=False):
    """lambda(x, t) = mu(x, t) + xi(x, t) evaluated at a free point, with the
    sums of Section 2.1 and scipy's standard normal densities (parts=True
    returns (mu, xi))."""
    D = X_ev.shape[1]
    mvn = stats.multivariate_normal(mean=np.zeros(D), cov=np.eye(D))
    mu = 0.0
    xi = 0.0
    for n in range(T_ev.shape[0]):
        if t != T_ev[n]:
            mu += mvn.pdf((x - X_ev[n]) / P["tau_x"]) * stats.norm.pdf((t - T_ev[n]) / P["tau_t"])
        if T_ev[n] < t:
            xi += math.exp(-P["omega"] * (t - T_ev[n])) * mvn.pdf((x - X_ev[n]) / P["h"])
    mu_v = (P["mu0"] / (P["tau_x"] ** D * P["tau_t"])) * mu
    xi_v = (P["theta"] * P["omega"] / P["h"] ** D) * xi
    return (mu_v, xi_v) if parts else mu_v + xi_v


def quad_Lambda_time(T_ev, P):
    """Integral of the rate over [0, T] once the spatial kernels have integrated
    to one: adaptive quadrature in t with breakpoints at the event times."""
    T = float(np.max(T_ev))

    def f(t):
        mu = sum(stats.norm.pdf((t - tn) / P["tau_t"]) for tn in T_ev) / P["tau_t"]
        xi = sum(math.exp(-P["omega"] * (t - tn)) for tn in T_ev if tn < t)
        return P["mu0"] * mu + P["theta"] * P["omega"] * xi

    pts = sorted(set(float(v) for v in T_ev if 0.0 < v < T))
    val, _ = integrate.quad(f, 0.0, T, points=pts or None, limit=400, epsabs=1e-13, epsrel=1e-12)
    return val


def quad_Lambda_space_time_1d(T_ev, X_ev, P):
    """Full two-dimensional quadrature of lambda(x, t) over R x [0, T] (D=1)."""
    T = float(np.max(T_ev))
    w = 14.0 * max(P["tau_x"], P["h"])
    lo, hi = float(X_ev.min()) - w, float(X_ev.max()) + w
    pts = sorted(set(float(v) for v in T_ev if 0.0 < v < T))

    def f(x, t):
        return free_point_rate(np.array([x]), t, T_ev, X_ev, P)

    val, _ = integrate.nquad(f, [[lo, hi], [0.0, T]],
                             opts=[{"limit": 200, "epsabs": 1e-11, "epsrel": 1e-10},
                                   {"limit": 200, "points": pts or None, "epsabs": 1e-11, "epsrel": 1e-10}])
    return val


def pin_brute_force(o):
    worst = worst_rate = 0.0
    zero_ok = True
    cases = [(0, 5, 1, 0), (1, 6, 2, 0), (2, 7, 3, 0), (3, 8, 2, 2), (4, 4, 1, 1), (5, 3, 3, 0), (6, 8, 1, 3)]
    for seed, n, d, ties in cases:
        w = synth.random_case(seed, n, d, ties=ties, shuffle=True, extent=2.0, t_end=4.0)
        lam = o.rates(w.t, w.X, w.params)
        ref = np.array([free_point_rate(w.X[i], w.t[i], w.t, w.X, w.params) for i in range(n)])
        worst_rate = max(worst_rate, _rel(lam, ref))
        Lq = quad_Lambda_time(w.t, w.params)
        L = o.Lambda(w.t, w.params)
        worst = max(worst, abs(L - Lq) / abs(Lq))
        ell = o.loglik(w.t, w.X, w.params)
        if np.any(ref == 0.0):
            # a zero rate (an event tied with every earlier one): ell = -inf
            zero_ok = zero_ok and ell == -np.inf
            continue
        ref_ell = float(np.sum(np.log(ref))) - Lq
        worst = max(worst, abs(ell - ref_ell) / abs(ref_ell))
    ok = worst_rate < 1e-13 and worst < 1e-9 and zero_ok
    return ok, f"rates {worst_rate:.3e}, Lambda/ell {worst:.3e}, zero-rate case ok={zero_ok}"


def pin_rate_parts(o):
    """The background and self-excitation parts of lambda_n separately (they
    give the self-excitation probability xi / (xi + mu) of an event)."""
    worst = 0.0
    for seed, n, d, ties in ((30, 7, 2, 1), (31, 6, 1, 0), (32, 8, 3, 2)):
        w = synth.random_case(seed, n, d, ties=ties, shuffle=True, extent=2.0, t_end=4.0)
        lam, mu, xi = o.rates(w.t, w.X, w.params, parts=True)
        ref = np.array([free_point_rate(w.X[i], w.t[i], w.t, w.X, w.params, parts=True) for i in range(n)])
        worst = max(worst, _rel(mu, ref[:, 0]), _rel(xi, ref[:, 1]), _rel(lam, mu + xi))
    return worst < 1e-13, f"max rel err {worst:.3e}"


def pin_space_time_quadrature(o):
    """D=1: the closed-form Lambda equals the 2-D integral of the rate."""
    w = synth.random_case(11, 3, 1, shuffle=True, extent=1.0, t_end=2.0)
    Lq = quad_Lambda_space_time_1d(w.t, w.X, w.params)
    L = o.Lambda(w.t, w.params)
    err = abs(L - Lq) / abs(Lq)
    return err < 1e-7, f"rel err {err:.3e}"


def pin_spatial_kernel_normalised():
    """The D-variate density integrates to one over R^D (D=1, 2) -- checks the
    reading of phi that the closed-form Lambda relies on."""
    f1, _ = integrate.quad(lambda z: stats.multivariate_normal(mean=[0.0]).pdf([z]), -np.inf, np.inf)
    mvn = stats.multivariate_normal(mean=np.zeros(2), cov=np.eye(2))
    f2, _ = integrate.dblquad(lambda y, x: mvn.pdf([x, y]), -12, 12, -12, 12)
    return abs(f1 - 1) < 1e-10 and abs(f2 - 1) < 1e-8, f"{f1} {f2}"


# -------------------------------------------------------- symbolic pair --

def symbolic_pair_reference(x, t, P, d):
    """Two events written out by hand (t[0] < t[1]); returns (ell, dX, dTheta)
    from sympy at 40 significant digits."""
    import sympy as sp

    mu0, tx, tt, th, om, h = sp.symbols("mu0 tau_x tau_t theta omega h", positive=True)
    xs = sp.symbols(f"x0:{2 * d}", real=True)
    x1, x2 = xs[:d], xs[d:]
    t1, t2 = sp.Float(t[0], 40), sp.Float(t[1], 40)
    r2 = sum((x1[k] - x2[k]) ** 2 for k in range(d))
    dt = t2 - t1
    gauss_d = lambda z2: sp.exp(-z2 / 2) / (2 * sp.pi) ** sp.Rational(d, 2)
    gauss_1 = lambda z2: sp.exp(-z2 / 2) / sp.sqrt(2 * sp.pi)
    Phi = lambda z: sp.erfc(-z / sp.sqrt(2)) / 2
    mu12 = mu0 / (tx ** d * tt) * gauss_d(r2 / tx ** 2) * gauss_1(dt ** 2 / tt ** 2)
    lam1 = mu12                                                    # first event: background only
    lam2 = mu12 + th * om / h ** d * sp.exp(-om * dt) * gauss_d(r2 / h ** 2)
    T = t2
    Lam = sum(mu0 * (Phi((T - tn) / tt) - Phi(-tn / tt)) + th * (1 - sp.exp(-om * (T - tn))) for tn in (t1, t2))
    ell = sp.log(lam1) + sp.log(lam2) - Lam
    subs = {mu0: P["mu0"], tx: P["tau_x"], tt: P["tau_t"], th: P["theta"], om: P["omega"], h: P["h"]}
    subs.update({xs[k]: sp.Float(float(x[k // d][k % d]), 40) for k in range(2 * d)})
    ev = lambda e: float(sp.N(e.subs(subs), 40))
    val = ev(ell)
    gX = np.array([ev(sp.diff(ell, xs[k])) for k in range(2 * d)]).reshape(2, d)
    gT = np.array([ev(sp.diff(ell, s)) for s in (mu0, tx, tt, th, om, h)])
    return val, gX, gT


def pin_symbolic_pair(o):
    worst = 0.0
    for d, seed in ((1, 0), (2, 1)):
        rng = np.random.default_rng(seed)
        t = np.array([0.7, 1.9])
        x = rng.uniform(0, 1, size=(2, d))
        P = dict(P_DEFAULT)
        val, gX, gT = symbolic_pair_reference(x, t, P, d)
        ell, g, lam = o.loglik_and_grad(t, x, P)
        gp = o.grad_params(t, x, P, lam)
        worst = max(worst, abs(ell - val) / abs(val), _rel(g, gX), _rel(gp, gT))
        # same two events passed in reverse order
        ell_r, g_r, lam_r = o.loglik_and_grad(t[::-1], x[::-1], P)
        worst = max(worst, abs(ell_r - val) / abs(val), _rel(g_r[::-1], gX))
    return worst < 1e-12, f"max rel err {worst:.3e}"


# ---------------------------------------------------- finite differences --

def _fd4(f, x0, h):
    return (8.0 * (f(x0 + h) - f(x0 - h)) - (f(x0 + 2 * h) - f(x0 - 2 * h))) / (12.0 * h)


def pin_finite_diff_locations(o):
    worst = 0.0
    for seed, n, d in ((0, 14, 1), (1, 12, 2), (2, 10, 3)):
        w = synth.random_case(100 + seed, n, d, shuffle=True)
        P = w.params
        g = o.grad_locations(w.t, w.X, P)
        fd = np.zeros_like(g)
        step = 1e-4 * min(P["h"], P["tau_x"])
        for i in range(n):
            for k in range(d):
                def f(v, i=i, k=k):
                    X = w.X.copy()
                    X[i, k] = v
                    return o.loglik(w.t, X, P)
                fd[i, k] = _fd4(f, w.X[i, k], step)
        worst = max(worst, float(np.linalg.norm(g - fd) / np.linalg.norm(fd)))
    return worst < 1e-7, f"rel-L2 {worst:.3e}"


def pin_finite_diff_params(o):
    worst = 0.0
    names = synth.PARAM_NAMES
    for seed, n, d in ((3, 12, 1), (4, 10, 2), (5, 9, 3)):
        w = synth.random_case(200 + seed, n, d, shuffle=True)
        P = w.params
        gp = o.grad_params(w.t, w.X, P)
        fd = np.zeros(6)
        for j, name in enumerate(names):
            def f(v, name=name):
                Q = dict(P)
                Q[name] = v
                return o.loglik(w.t, w.X, Q)
            fd[j] = _fd4(f, P[name], 1e-4 * P[name])
        worst = max(worst, float(np.max(np.abs(gp - fd) / np.maximum(np.abs(fd), 1e-3))))
    return worst < 1e-7, f"max rel err {worst:.3e}"


# ------------------------------------------------------------ invariances --

def pin_translation(o):
    worst = 0.0
    for seed, n, d in ((7, 20, 2), (8, 15, 3), (9, 25, 1)):
        w = synth.random_case(seed, n, d)
        ell, g, _ = o.loglik_and_grad(w.t, w.X, w.params)
        worst = max(worst, float(np.max(np.abs(g.sum(axis=0)))) / float(np.abs(g).sum()))
        shift = np.linspace(-3.0, 5.0, d)
        worst = max(worst, abs(o.loglik(w.t, w.X + shift, w.params) - ell) / abs(ell) * 1e-3)
    return worst < 1e-13, f"max {worst:.3e}"


def pin_scaling(o):
    worst = 0.0
    for seed, n, d in ((10, 18, 2), (12, 14, 3), (13, 16, 1)):
        w = synth.random_case(seed, n, d, shuffle=True)
        P = w.params
        ell = o.loglik(w.t, w.X, P)
        for c in (0.37, 2.5):
            Ps = dict(P, tau_x=c * P["tau_x"], h=c * P["h"])
            es = o.loglik(w.t, c * w.X, Ps)
            worst = max(worst, abs(es - (ell - n * d * math.log(c))) / abs(ell))
            Pt = dict(P, tau_t=c * P["tau_t"], omega=P["omega"] / c)
            et = o.loglik(c * w.t, w.X, Pt)
            worst = max(worst, abs(et - (ell - n * math.log(c))) / abs(ell))
    return worst < 1e-12, f"max rel err {worst:.3e}"


def pin_euler(o):
    worst = 0.0
    for seed, n, d in ((14, 16, 2), (15, 11, 3), (16, 13, 1)):
        w = synth.random_case(seed, n, d, shuffle=True)
        P = w.params
        ell, g, lam = o.loglik_and_grad(w.t, w.X, P)
        gp = o.grad_params(w.t, w.X, P, lam)
        lhs = float(np.sum(w.X * g)) + P["tau_x"] * gp[1] + P["h"] * gp[5]
        worst = max(worst, abs(lhs + n * d) / (n * d))
        lhs2 = P["mu0"] * gp[0] + P["theta"] * gp[3]
        Lam = o.Lambda(w.t, P)
        worst = max(worst, abs(lhs2 - (n - Lam)) / n)
    return worst < 1e-11, f"max rel err {worst:.3e}"


def pin_permutation(o):
    w = synth.random_case(17, 21, 2, ties=1)
    P = w.params
    ell, g, lam = o.loglik_and_grad(w.t, w.X, P)
    gp = o.grad_params(w.t, w.X, P, lam)
    perm = np.random.default_rng(5).permutation(w.n)
    ell2, g2, lam2 = o.loglik_and_grad(w.t[perm], w.X[perm], P)
    gp2 = o.grad_params(w.t[perm], w.X[perm], P, lam2)
    err = max(abs(ell2 - ell) / abs(ell), _rel(g2, g[perm]), _rel(lam2, lam[perm]), _rel(gp2, gp))
    return err < 1e-13, f"max rel err {err:.3e}"


def pin_theta_zero(o):
    """Negligible self-excitation: ell(mu0) = N log mu0 + const - mu0 S with
    S = sum_n [Phi(a_n/tau_t) - Phi(-t_n/tau_t)], so the score vanishes at
    mu0* = N/S and ell(2 mu0) - ell(mu0) = N log 2 - mu0 S."""
    worst = 0.0
    for seed, n, d in ((18, 15, 2), (19, 12, 1)):
        w = synth.random_case(seed, n, d, shuffle=True)
        T = w.t.max()
        S = float(np.sum(stats.norm.cdf((T - w.t) / w.params["tau_t"]) - stats.norm.cdf(-w.t / w.params["tau_t"])))
        P = dict(w.params, theta=1e-250)
        mu_star = n / S
        Ps = dict(P, mu0=mu_star)
        gp = o.grad_params(w.t, w.X, Ps)
        worst = max(worst, abs(gp[0]) / (n / mu_star))
        e1 = o.loglik(w.t, w.X, P)
        e2 = o.loglik(w.t, w.X, dict(P, mu0=2 * P["mu0"]))
        worst = max(worst, abs((e2 - e1) - (n * math.log(2) - P["mu0"] * S)) / abs(e1))
    return worst < 1e-12, f"max rel err {worst:.3e}"


def pin_theta_score_scale(o):
    """The magnitude scale of the Theta score (the tolerance scale of the GPU
    comparisons): each component sums the same pieces as the score, with
    absolute values, so score and scale differ by twice the pieces of one
    sign.  Those are fixed by the background and self-excitation parts of
    lambda_n (M_n, Xi_n, pinned by rate_parts) and by closed forms with
    scipy's Phi:
      mu0:   scale - g = 2 sum [Phi(a/tau_t) - Phi(-t/tau_t)],  scale + g = 2 sum M/(mu0 lambda)
      tau_x: (scale - g) tau_x = 2 D sum M/lambda
      tau_t: (scale - g) tau_t = 2 sum M/lambda
      theta: scale - g = 2 sum [1 - e^(-omega a)],             scale + g = 2 sum Xi/(theta lambda)
      omega: (scale + g) omega = 2 sum Xi/lambda
      h:     (scale - g) h = 2 D sum Xi/lambda
    and the scale bounds |g| in every component."""
    worst = 0.0
    bound_ok = True
    for seed, n, d in ((41, 30, 2), (42, 25, 3), (43, 40, 1)):
        w = synth.random_case(seed, n, d, shuffle=True, ties=1)
        P = w.params
        lam, M, Xi = o.rates(w.t, w.X, P, parts=True)
        g, sc = o.grad_params_scaled(w.t, w.X, P, lam)
        g_plain = o.grad_params(w.t, w.X, P, lam)
        bound_ok &= bool(np.array_equal(g, g_plain)) and bool(np.all(sc >= np.abs(g) * (1 - 1e-14)))
        T = w.t.max()
        a = T - w.t
        Sphi = float(np.sum(stats.norm.cdf(a / P["tau_t"]) - stats.norm.cdf(-w.t / P["tau_t"])))
        SM, SX = float(np.sum(M / lam)), float(np.sum(Xi / lam))
        S1 = float(np.sum(1.0 - np.exp(-P["omega"] * a)))
        checks = [
            (sc[0] - g[0], 2 * Sphi), (sc[0] + g[0], 2 * SM / P["mu0"]),
            ((sc[1] - g[1]) * P["tau_x"], 2 * d * SM),
            ((sc[2] - g[2]) * P["tau_t"], 2 * SM),
            (sc[3] - g[3], 2 * S1), (sc[3] + g[3], 2 * SX / P["theta"]),
            ((sc[4] + g[4]) * P["omega"], 2 * SX),
            ((sc[5] - g[5]) * P["h"], 2 * d * SX),
        ]
        for got, ref in checks:
            worst = max(worst, abs(got - ref) / max(abs(ref), 1e-300))
    return bound_ok and worst < 1e-12, f"bound {bound_ok}, max rel err {worst:.3e}"


def pin_row_subsets(o):
    w = synth.random_case(20, 30, 2, shuffle=True)
    lam = o.rates(w.t, w.X, w.params)
    g = o.grad_locations(w.t, w.X, w.params, lam)
    rows = np.array([0, 7, 29, 7, 3])
    e1 = _rel(o.rates_rows(w.t, w.X, w.params, rows), lam[rows])
    e2 = _rel(o.grad_rows(w.t, w.X, w.params, lam, rows), g[rows])
    return max(e1, e2) == 0.0, f"{e1} {e2}"


# ------------------------------------------------------------------- HMC --

def _hmc_case(seed=21, n=12, d=2):
    w = synth.random_case(seed, n, d, shuffle=True, extent=1.5, t_end=3.0)
    rng = np.random.default_rng(seed)
    lo = w.X - rng.uniform(0.02, 0.1, size=w.X.shape)
    hi = w.X + rng.uniform(0.02, 0.1, size=w.X.shape)
    p0 = rng.standard_normal(size=w.X.shape)
    return w, lo, hi, p0


def pin_hmc_reversible(o):
    w, lo, hi, p0 = _hmc_case()
    out = o.hmc_trajectory(w.t, w.X, p0, w.params, 0.01, 15, -np.inf, lo, hi)
    if not out["accepted"]:
        return False, "forward proposal rejected"
    inside = bool(np.all(out["X"] >= lo) and np.all(out["X"] <= hi))
    back = o.hmc_trajectory(w.t, out["X"], -out["p"], w.params, 0.01, 15, -np.inf, lo, hi)
    ex = _rel(back["X"], w.X)
    ep = _rel(-back["p"], p0)
    moved = _rel(out["X"], w.X)
    ok = inside and ex < 1e-9 and ep < 1e-8 and moved > 1e-3 and abs(back["H1"] - out["H0"]) < 1e-8
    return ok, f"inside={inside} dX={ex:.2e} dp={ep:.2e} moved={moved:.2e}"


def pin_hmc_energy_order(o):
    w, _, _, p0 = _hmc_case(22, 10, 2)
    errs = []
    for eps in (0.004, 0.002, 0.001):
        n_steps = int(round(0.04 / eps))
        out = o.hmc_trajectory(w.t, w.X, p0, w.params, eps, n_steps, -np.inf)
        errs.append(abs(out["H1"] - out["H0"]))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    return 3.0 < r1 < 5.3 and 3.0 < r2 < 5.3, f"dH {errs} ratios {r1:.2f} {r2:.2f}"


def pin_hmc_accept_rule(o):
    w, lo, hi, p0 = _hmc_case(23, 9, 2)
    base = o.hmc_trajectory(w.t, w.X, p0, w.params, 0.02, 5, -np.inf, lo, hi)
    dh = base["H0"] - base["H1"]
    a = o.hmc_trajectory(w.t, w.X, p0, w.params, 0.02, 5, dh - 1e-9, lo, hi)
    r = o.hmc_trajectory(w.t, w.X, p0, w.params, 0.02, 5, dh + 1e-9, lo, hi)
    z = o.hmc_trajectory(w.t, w.X, p0, w.params, 0.02, 0, -1e-3, lo, hi)
    ok = (a["accepted"] == 1 and np.array_equal(a["X"], base["X"]) and r["accepted"] == 0
          and np.array_equal(r["X"], w.X) and z["H0"] == z["H1"] and np.array_equal(z["X"], w.X))
    return ok, f"dH={dh:.3e} acc={a['accepted']} rej={r['accepted']}"


# ----------------------------------------------------------------- BMDS --

def bmds_case(seed, n, d, noise=0.2):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, d))
    D = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    Y = np.abs(D + noise * rng.normal(size=(n, n))) + 0.05
    Y = np.tril(Y, -1) + np.tril(Y, -1).T
    Xl = X + 0.1 * rng.normal(size=X.shape)   # latent locations differ from the truth
    return Y, Xl


def pin_bmds_symbolic_pair(o):
    """Two points written out by hand (Eq. (4) with N = 2) and differentiated by sympy."""
    import sympy as sp

    y, s2 = sp.symbols("y sigma2", positive=True)
    xs = sp.symbols("a0 a1 b0 b1", real=True)
    delta = sp.sqrt((xs[0] - xs[2]) ** 2 + (xs[1] - xs[3]) ** 2)
    sigma = sp.sqrt(s2)
    Phi = lambda z: sp.erfc(-z / sp.sqrt(2)) / 2
    ell = sp.Rational(2 * (1 - 2), 4) * sp.log(s2) - ((y - delta) ** 2 / (2 * s2) + sp.log(Phi(delta / sigma)))
    rng = np.random.default_rng(3)
    X = rng.normal(size=(2, 2))
    yv, s2v = 0.9, 0.35
    subs = {y: yv, s2: s2v, xs[0]: X[0, 0], xs[1]: X[0, 1], xs[2]: X[1, 0], xs[3]: X[1, 1]}
    ev = lambda e: float(sp.N(e.subs(subs), 40))
    val = ev(ell)
    gX = np.array([ev(sp.diff(ell, v)) for v in xs]).reshape(2, 2)
    gs = ev(sp.diff(ell, s2))
    Y = np.array([[0.0, yv], [yv, 0.0]])
    e, g, gso = o.bmds(Y, X, s2v)
    err = max(abs(e - val) / abs(val), _rel(g, gX), abs(gso - gs) / abs(gs))
    return err < 1e-12, f"max rel err {err:.3e}"


def pin_bmds_pair_density(o):
    """With N = 2, exp(ell) as a function of the observed distance y is
    sqrt(2 pi) times a normalized truncated normal density on y > 0."""
    X = np.array([[0.0, 0.0], [0.7, 0.2]])
    worst = 0.0
    for s2v in (0.05, 0.4, 2.0):
        f = lambda yv: math.exp(o.bmds(np.array([[0.0, yv], [yv, 0.0]]), X, s2v)[0])
        val, _ = integrate.quad(f, 0.0, np.inf, limit=200, epsabs=1e-13, epsrel=1e-12)
        worst = max(worst, abs(val - math.sqrt(2 * math.pi)) / math.sqrt(2 * math.pi))
    return worst < 1e-9, f"max rel err {worst:.3e}"


def pin_bmds_finite_diff(o):
    worst = 0.0
    for seed, n, d in ((1, 9, 2), (2, 7, 3), (3, 8, 1)):
        Y, X = bmds_case(seed, n, d)
        s2v = 0.3
        e, g, gs = o.bmds(Y, X, s2v)
        fd = np.zeros_like(g)
        for i in range(n):
            for k in range(d):
                def f(v, i=i, k=k):
                    Xp = X.copy()
                    Xp[i, k] = v
                    return o.bmds(Y, Xp, s2v)[0]
                fd[i, k] = _fd4(f, X[i, k], 1e-5)
        fds = _fd4(lambda v: o.bmds(Y, X, v)[0], s2v, 1e-5)
        worst = max(worst, float(np.linalg.norm(g - fd) / np.linalg.norm(fd)), abs(gs - fds) / abs(fds))
    return worst < 1e-7, f"max rel err {worst:.3e}"


def pin_bmds_invariances(o):
    """Translation and rotation leave every distance unchanged (gradient sums
    and torques vanish); scaling X, Y by c and sigma2 by c^2 shifts ell by
    N (1 - N)/2 log c."""
    Y, X = bmds_case(4, 11, 2)
    n = 11
    e, g, _ = o.bmds(Y, X, 0.25)
    worst = float(np.max(np.abs(g.sum(axis=0))) / np.abs(g).sum())
    torque = float(np.sum(X[:, 0] * g[:, 1] - X[:, 1] * g[:, 0]))
    worst = max(worst, abs(torque) / float(np.abs(X).max() * np.abs(g).sum()))
    for c in (0.5, 3.0):
        ec = o.bmds(c * Y, c * X, 0.25 * c * c)[0]
        worst = max(worst, abs(ec - (e + n * (1 - n) / 2 * math.log(c))) / abs(e))
    return worst < 1e-12, f"max {worst:.3e}"


def pin_bmds_coincident(o):
    """Two coincident latent points: |x_n - x_n'| has no derivative there, and
    its central differences vanish, so the symmetric central difference of
    ell_B equals the gradient with that pair's term taken as 0; the value
    stays finite."""
    Y, X = bmds_case(6, 6, 2)
    X[3] = X[0]
    s2v = 0.3
    e, g, _ = o.bmds(Y, X, s2v)
    if not (np.isfinite(e) and np.all(np.isfinite(g))):
        return False, "non-finite value or gradient"
    fd = np.zeros_like(g)
    for i in range(X.shape[0]):
        for k in range(X.shape[1]):
            def f(v, i=i, k=k):
                Xp = X.copy()
                Xp[i, k] = v
                return o.bmds(Y, Xp, s2v)[0]
            fd[i, k] = _fd4(f, X[i, k], 1e-5)
    err = float(np.linalg.norm(g - fd) / np.linalg.norm(fd))
    return err < 1e-7, f"rel err {err:.3e}"


def _lens_quad(R, rho, c):
    """Lens area by quadrature of the overlap of the two chords along the
    line of centres (first circle at 0, second at c)."""
    lo, hi = max(-R, c - rho), min(R, c + rho)
    if hi <= lo:
        return 0.0
    f = lambda x: 2.0 * max(0.0, min(math.sqrt(max(R * R - x * x, 0.0)),
                                     math.sqrt(max(rho * rho - (x - c) ** 2, 0.0))))
    # the chords cross at the discs' common chord, x = (c^2 + R^2 - rho^2) / (2c)
    x_cross = (c * c + R * R - rho * rho) / (2 * c) if c > 0 else lo
    pts = [p for p in (c - rho, c + rho, -R, R, x_cross) if lo < p < hi]
    val, _ = integrate.quad(f, lo, hi, points=pts or None, limit=400, epsabs=1e-14, epsrel=1e-13)
    return val


def pin_lens_area(o):
    """The lens area of Eq. (6) against quadrature, the equal-circle closed
    form 2R^2 acos(c/2R) - (c/2) sqrt(4R^2 - c^2), and the limiting cases."""
    worst = 0.0
    for R, rho, c in ((1.0, 0.5, 0.9), (1.0, 0.5, 1.2), (2.0, 0.3, 1.85), (1.0, 3.0, 2.5), (0.7, 0.7, 0.2),
                      (5.0, 0.01, 4.995), (1.0, 1.0, 1.999)):
        a = o.lens_area(R, rho, c)
        worst = max(worst, abs(a - _lens_quad(R, rho, c)) / max(a, 1e-300))
    for c in (0.1, 0.8, 1.5, 1.9):
        ref = 2 * math.acos(c / 2) - (c / 2) * math.sqrt(4 - c * c)
        worst = max(worst, abs(o.lens_area(1.0, 1.0, c) - ref) / ref)
    ok = o.lens_area(1.0, 0.5, 1.6) == 0.0 and abs(o.lens_area(1.0, 0.5, 0.3) - math.pi * 0.25) < 1e-15
    ok = ok and abs(o.lens_area(0.4, 2.0, 1.0) - math.pi * 0.16) < 1e-15
    return ok and worst < 1e-10, f"max rel err {worst:.3e}"


def pin_circle_proposals(o):
    """The rejection sampler of Eq. (6) by simulation: with `tries` draws from
    the disc of radius r eps, a proposal succeeds with probability
    1 - (1 - A/(pi (r eps)^2))^tries (A from quadrature), successful proposals
    lie in both discs and are uniform on the lens (the share in the half-plane
    y > 0 is 1/2 by symmetry, the share within distance r eps / 2 of x is the
    quadrature area of that smaller lens over A); the log q-ratio of a
    successful single move equals the one built from those pinned pieces."""
    rng = np.random.default_rng(7)
    R, eps, tries = 1.0, 0.6, 2
    x = np.array([0.75, 0.0])
    rho = R * eps
    A = _lens_quad(R, rho, 0.75)
    M = 200_000
    X = np.tile(x, (M, 1))
    u = rng.uniform(size=(M, tries, 2))
    # one event per row: call the oracle in chunks (all rows share the same prior circle)
    Xn, _ = o.circle_proposals(X, np.zeros((M, 2)), np.full(M, R), eps, tries, u)
    moved = np.any(Xn != X, axis=1)
    p_ref = 1.0 - (1.0 - A / (math.pi * rho * rho)) ** tries
    se = math.sqrt(p_ref * (1 - p_ref) / M)
    ok = abs(moved.mean() - p_ref) < 5 * se
    Y = Xn[moved]
    ok = ok and bool(np.all(np.hypot(Y[:, 0], Y[:, 1]) < R)) and bool(np.all(np.hypot(*(Y - x).T) < rho))
    half = (Y[:, 1] > 0).mean()
    near = (np.hypot(*(Y - x).T) < rho / 2).mean()
    near_ref = _lens_quad(R, rho / 2, 0.75) / A
    ok = ok and abs(half - 0.5) < 5 * math.sqrt(0.25 / len(Y)) and abs(near - near_ref) < 5 * math.sqrt(
        near_ref * (1 - near_ref) / len(Y))
    # log q-ratio of one successful move, from the pinned pieces
    u1 = np.array([[[0.3, 0.1], [0.5, 0.5]]])
    y, lq = o.circle_proposals(x[None, :], np.zeros((1, 2)), np.array([R]), eps, tries, u1)
    Ay = _lens_quad(R, rho, float(np.hypot(*y[0])))
    Ps = lambda a: 1.0 - (1.0 - a / (math.pi * rho * rho)) ** tries
    ref = (math.log(Ps(Ay)) - math.log(Ay)) - (math.log(Ps(A)) - math.log(A))
    ok = ok and abs(lq - ref) < 1e-10
    return ok, f"success {moved.mean():.4f} vs {p_ref:.4f}, half {half:.4f}, near {near:.4f} vs {near_ref:.4f}"


def pin_box_proposals(o):
    """Truncated-normal box proposals against scipy: the draw is
    x + s ndtri(Phi(a) + u (Phi(b) - Phi(a))) (scipy's inverse normal CDF),
    stays in the box, and the log q-ratio equals
    truncnorm.logpdf(x | x*) - truncnorm.logpdf(x* | x) summed over coordinates."""
    from scipy import special, stats

    rng = np.random.default_rng(8)
    nb, d, s = 6, 2, 0.03
    X = rng.uniform(0, 1, size=(nb, d))
    lo, hi = X - rng.uniform(0.01, 0.06, size=X.shape), X + rng.uniform(0.01, 0.06, size=X.shape)
    u = rng.uniform(size=(nb, d))
    Xn, lq = o.box_proposals(X, lo, hi, s, u)
    Pa, Pb = special.ndtr((lo - X) / s), special.ndtr((hi - X) / s)
    ref = X + s * special.ndtri(Pa + u * (Pb - Pa))
    err = float(np.max(np.abs(Xn - ref)))
    lp = lambda y, c: stats.truncnorm.logpdf(y, (lo - c) / s, (hi - c) / s, loc=c, scale=s)
    lq_ref = float(np.sum(lp(X, Xn) - lp(Xn, X)))
    ok = err < 1e-12 and bool(np.all((Xn >= lo) & (Xn <= hi))) and abs(lq - lq_ref) < 1e-9
    return ok, f"draw err {err:.2e}, ratio {lq:.6f} vs {lq_ref:.6f}"


def _bmds_hmc_case(seed=41, n=12, d=3):
    w = synth.random_case(seed, n, d, shuffle=True, extent=2.0, t_end=5.0)
    Y, _ = bmds_case(seed, n, d)
    rng = np.random.default_rng(seed)
    return w, Y, rng.standard_normal(size=w.X.shape)


def pin_bmds_hmc_reversible_and_energy(o):
    """HMC on the BMDS-Hawkes potential: the leapfrog is reversible (negated
    final momenta retrace the path) and the energy error falls as eps^2, which
    only holds when the gradient is that of the summed potential."""
    w, Y, p0 = _bmds_hmc_case()
    out = o.bmds_hmc_trajectory(w.t, w.X, p0, w.params, Y, 0.4, 0.005, 12, -np.inf)
    back = o.bmds_hmc_trajectory(w.t, out["X"], -out["p"], w.params, Y, 0.4, 0.005, 12, -np.inf)
    ex, moved = _rel(back["X"], w.X), _rel(out["X"], w.X)
    errs = []
    for eps in (0.002, 0.001, 0.0005):
        r = o.bmds_hmc_trajectory(w.t, w.X, p0, w.params, Y, 0.4, eps, int(round(0.016 / eps)), -np.inf)
        errs.append(abs(r["H1"] - r["H0"]))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    h0 = -(o.loglik(w.t, w.X, w.params) + o.bmds(Y, w.X, 0.4)[0]) + 0.5 * float(np.sum(p0 * p0))
    ok = (out["accepted"] == 1 and ex < 1e-9 and moved > 1e-3 and 3.0 < r1 < 5.3 and 3.0 < r2 < 5.3
          and abs(out["H0"] - h0) <= 1e-10 * abs(h0))
    return ok, f"dX={ex:.2e} moved={moved:.2e} dH ratios {r1:.2f} {r2:.2f}"


ALL_PINS = {
    "brute_force": pin_brute_force,
    "space_time_quadrature": pin_space_time_quadrature,
    "rate_parts": pin_rate_parts,
    "symbolic_pair": pin_symbolic_pair,
    "finite_diff_locations": pin_finite_diff_locations,
    "finite_diff_params": pin_finite_diff_params,
    "translation": pin_translation,
    "scaling": pin_scaling,
    "euler": pin_euler,
    "permutation": pin_permutation,
    "theta_zero": pin_theta_zero,
    "theta_score_scale": pin_theta_score_scale,
    "row_subsets": pin_row_subsets,
    "hmc_reversible": pin_hmc_reversible,
    "hmc_energy_order": pin_hmc_energy_order,
    "hmc_accept_rule": pin_hmc_accept_rule,
    "bmds_symbolic_pair": pin_bmds_symbolic_pair,
    "bmds_pair_density": pin_bmds_pair_density,
    "bmds_finite_diff": pin_bmds_finite_diff,
    "bmds_invariances": pin_bmds_invariances,
    "bmds_coincident": pin_bmds_coincident,
    "lens_area": pin_lens_area,
    "circle_proposals": pin_circle_proposals,
    "box_proposals": pin_box_proposals,
    "bmds_hmc": pin_bmds_hmc_reversible_and_energy,
}
