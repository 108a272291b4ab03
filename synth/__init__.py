"""Seeded synthetic workloads shaped like the paper's data sets.

This module holds no arithmetic of the log-likelihood: it only draws event
times and locations, coarsens them and picks the parameter values at which
the rate is evaluated.  Both the FP64 oracle tests and the GPU path take their
inputs from here.

Events come from the branching (cluster) construction of Zhuang et al. (2004)
that the paper's simulation study uses (Appendix C): background events first,
then generations of offspring, each parent having Poisson(m) children with an
Exp(omega) time lag and a N(0, h^2 I) spatial offset.  Offspring past the time
window are dropped; offspring outside the spatial square are kept.  When the
total falls short of N the background count is raised and the simulation rerun
with the same seed; otherwise the N earliest events are kept.

Coarsening follows Section 2.2: rounding to a 100 m grid (the gunfire data,
Eq. (2)) gives a box of side 0.1 km around each observed location, and the
latent location starts uniform in its box.  The wildfire-like workload draws
box sides from {0.1, 1, 10} km instead (boxes stand in for the circles of
Eq. (3)).

Units: kilometres and days.  Parameters are evaluated at the generating
values: theta = offspring mean, omega = decay rate, h = offspring sd,
mu0 = 1 - theta, with the background bandwidths listed per workload.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PARAM_NAMES = ("mu0", "tau_x", "tau_t", "theta", "omega", "h")


@dataclass
class Workload:
    """One synthetic data set: times t (N,), latent locations X (N, D),
    observed (coarsened) locations X_obs, per-coordinate box walls, and the
    parameter vector Theta at which the rate is evaluated."""

    name: str
    t: np.ndarray
    X: np.ndarray
    X_obs: np.ndarray
    box_lo: np.ndarray | None
    box_hi: np.ndarray | None
    params: dict
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.t.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    def theta_vector(self) -> np.ndarray:
        return np.array([self.params[k] for k in PARAM_NAMES], dtype=np.float64)


def branching_simulation(rng: np.random.Generator, n_background: int, t_end: float, m: float,
                         omega: float, h: float, d: int, background: str, extent: float) -> tuple:
    """Cluster construction: background events, then offspring generations.

    background = "square": uniform on [0, extent]^d; "normal": N(0, I_d).
    Returns (t, X) unsorted, offspring past t_end removed."""
    t0 = rng.uniform(0.0, t_end, size=n_background)
    if background == "square":
        x0 = rng.uniform(0.0, extent, size=(n_background, d))
    elif background == "normal":
        x0 = rng.standard_normal(size=(n_background, d))
    else:
        raise ValueError(background)
    ts, xs = [t0], [x0]
    parents_t, parents_x = t0, x0
    for _generation in range(10_000):
        counts = rng.poisson(m, size=parents_t.shape[0])
        total = int(counts.sum())
        if total == 0:
            break
        ct = np.repeat(parents_t, counts) + rng.exponential(1.0 / omega, size=total)
        cx = np.repeat(parents_x, counts, axis=0) + h * rng.standard_normal(size=(total, d))
        keep = ct <= t_end
        parents_t, parents_x = ct[keep], cx[keep]
        if parents_t.shape[0] == 0:
            break
        ts.append(parents_t)
        xs.append(parents_x)
    return np.concatenate(ts), np.concatenate(xs, axis=0)


def simulate_events(seed: int, n: int, d: int, t_end: float, m: float, omega: float, h: float,
                    background: str = "square", extent: float = 1.0) -> tuple:
    """Exactly n events, time-sorted: rerun with more background events until
    the branching process yields at least n, then keep the n earliest."""
    nb = max(1, int(np.ceil(n * (1.0 - m) * 1.05)))
    for _attempt in range(200):
        rng = np.random.default_rng(seed)
        t, X = branching_simulation(rng, nb, t_end, m, omega, h, d, background, extent)
        if t.shape[0] >= n:
            order = np.argsort(t, kind="stable")[:n]
            return t[order].copy(), X[order].copy(), rng
        nb = int(np.ceil(nb * max(1.02, 1.01 * n / t.shape[0])))
    raise RuntimeError("branching simulation did not reach the requested size")


def grid_boxes(rng: np.random.Generator, X_true: np.ndarray, cell: float):
    """Round to a grid of side `cell`, box = the cell, latent uniform in the cell."""
    X_obs = np.round(X_true / cell) * cell
    lo = X_obs - 0.5 * cell
    hi = X_obs + 0.5 * cell
    X = rng.uniform(lo, hi)
    return X_obs, lo, hi, X


def mixed_boxes(rng: np.random.Generator, X_true: np.ndarray, sides=(0.1, 1.0, 10.0), probs=(0.5, 0.3, 0.2)):
    """Axis-aligned boxes with side drawn per event; centre = truth + U(+-s/2)."""
    n, d = X_true.shape
    s = rng.choice(np.asarray(sides), size=n, p=np.asarray(probs))[:, None]
    centre = X_true + rng.uniform(-0.5, 0.5, size=(n, d)) * s
    lo = centre - 0.5 * s
    hi = centre + 0.5 * s
    X = rng.uniform(lo, hi)
    return centre, lo, hi, X


def _params(m, omega, h, tau_x, tau_t):
    return {"mu0": 1.0 - m, "tau_x": tau_x, "tau_t": tau_t, "theta": m, "omega": omega, "h": h}


def make_c1(seed: int = 0, n: int = 1000) -> Workload:
    """FP64 single evaluation: N=1,000, D=2, 10 km square, 100 days;
    m=0.3, omega=1/day, h=0.2 km; tau_x=1 km, tau_t=7 days; 100 m grid."""
    t, Xt, rng = simulate_events(seed, n, 2, 100.0, 0.3, 1.0, 0.2, "square", 10.0)
    X_obs, lo, hi, X = grid_boxes(rng, Xt, 0.1)
    return Workload("c1_fp64_single_n1000_d2", t, X, X_obs, lo, hi, _params(0.3, 1.0, 0.2, 1.0, 7.0),
                    {"square_km": 10.0, "days": 100.0, "cell_km": 0.1, "seed": seed})


def make_c2(seed: int = 1, n: int = 10_000) -> Workload:
    """Gunfire-like: N=10,000, D=2, 20 km square, 365 days; m=0.5,
    omega=0.5/day, h=0.1 km; tau_x=1 km, tau_t=14 days; 100 m cells as boxes."""
    t, Xt, rng = simulate_events(seed, n, 2, 365.0, 0.5, 0.5, 0.1, "square", 20.0)
    X_obs, lo, hi, X = grid_boxes(rng, Xt, 0.1)
    return Workload("c2_gunfire_like_n10000_d2", t, X, X_obs, lo, hi, _params(0.5, 0.5, 0.1, 1.0, 14.0),
                    {"square_km": 20.0, "days": 365.0, "cell_km": 0.1, "seed": seed, "hmc_steps": 20})


def make_c3(seed: int = 2, n: int = 5000) -> Workload:
    """Wildfire-like: N=5,000, D=2, 200 km square, 3,650 days; m=0.4,
    omega=1/30 per day, h=2 km; tau_x=10 km, tau_t=90 days; box sides
    {0.1, 1, 10} km with probabilities {0.5, 0.3, 0.2}."""
    t, Xt, rng = simulate_events(seed, n, 2, 3650.0, 0.4, 1.0 / 30.0, 2.0, "square", 200.0)
    X_obs, lo, hi, X = mixed_boxes(rng, Xt)
    return Workload("c3_wildfire_like_n5000_d2", t, X, X_obs, lo, hi, _params(0.4, 1.0 / 30.0, 2.0, 10.0, 90.0),
                    {"square_km": 200.0, "days": 3650.0, "seed": seed})


def circle_priors(w: Workload, seed: int = 7) -> tuple[np.ndarray, np.ndarray]:
    """Circle priors of Eq. (3) for the events of w, drawn as the wildfire
    data present them: radii (km, from the fire size at discovery) of 0.05,
    0.5 or 5 with probabilities 0.5, 0.3, 0.2, and each event's latent
    location uniform inside its circle (so the centre is the observed point).
    Returns (centers (N, 2), radii (N,))."""
    rng = np.random.default_rng(seed)
    n = w.n
    radii = rng.choice(np.array([0.05, 0.5, 5.0]), size=n, p=[0.5, 0.3, 0.2])
    ang = rng.uniform(0.0, 2.0 * np.pi, size=n)
    rr = radii * np.sqrt(rng.uniform(size=n)) * 0.999
    centers = w.X - np.stack([rr * np.cos(ang), rr * np.sin(ang)], axis=1)
    return centers, radii


def make_c4(seed: int = 3, n_sets: int = 64, n_min: int = 500, n_max: int = 20_000) -> list:
    """Batched latent-space sets: N log-uniform in [500, 20,000], D uniform in
    {2, 4, 8}, background N(0, I_D) over 365 days; m=0.5, omega=1/day,
    h=0.1; tau_x=0.5, tau_t=14 days; unconstrained.  Set i uses seed 1000+i."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=n_sets)).astype(np.int64)
    dims = rng.choice(np.array([2, 4, 8]), size=n_sets)
    out = []
    for i in range(n_sets):
        n_i, d_i = int(sizes[i]), int(dims[i])
        t, X, _ = simulate_events(1000 + i, n_i, d_i, 365.0, 0.5, 1.0, 0.1, "normal")
        out.append(Workload(f"c4_set{i}_n{n_i}_d{d_i}", t, X, X.copy(), None, None,
                            _params(0.5, 1.0, 0.1, 0.5, 14.0), {"seed": 1000 + i, "days": 365.0}))
    return out


def make_c5(seed: int = 4, n: int = 100_000) -> Workload:
    """Large: N=100,000, D=2, 50 km square, 1,825 days; m=0.6, omega=0.2/day,
    h=0.05 km; tau_x=1 km, tau_t=14 days; 100 m coarsening."""
    t, Xt, rng = simulate_events(seed, n, 2, 1825.0, 0.6, 0.2, 0.05, "square", 50.0)
    X_obs, lo, hi, X = grid_boxes(rng, Xt, 0.1)
    return Workload("c5_large_n100000_d2", t, X, X_obs, lo, hi, _params(0.6, 0.2, 0.05, 1.0, 14.0),
                    {"square_km": 50.0, "days": 1825.0, "cell_km": 0.1, "seed": seed,
                     "oracle_rows": 2000, "oracle_row_seed": 5})


def scaled_down(w: Workload, n: int) -> Workload:
    """The first n events of a workload (same density and parameters over a
    shorter window) -- a bounded sample for the CPU baseline and small tests."""
    sl = slice(0, n)
    lo = None if w.box_lo is None else w.box_lo[sl].copy()
    hi = None if w.box_hi is None else w.box_hi[sl].copy()
    meta = dict(w.meta)
    meta["sample_of"] = w.name
    return Workload(f"{w.name}_first{n}", w.t[sl].copy(), w.X[sl].copy(), w.X_obs[sl].copy(), lo, hi,
                    dict(w.params), meta)


def random_case(seed: int, n: int, d: int, *, ties: int = 0, shuffle: bool = True, extent: float = 3.0,
                t_end: float = 10.0, params: dict | None = None) -> Workload:
    """Small random data for parity and edge-case tests: uniform times and
    locations, optional groups of exactly tied times, optional shuffling so
    that times arrive unsorted."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.0, t_end, size=n)
    X = rng.uniform(0.0, extent, size=(n, d))
    if ties and n >= 2:
        for _ in range(ties):
            k = int(rng.integers(2, min(5, n) + 1))
            idx = rng.choice(n, size=k, replace=False)
            t[idx] = t[idx[0]]
    if not shuffle:
        order = np.argsort(t, kind="stable")
        t, X = t[order], X[order]
    p = params or {"mu0": 0.6, "tau_x": 0.8, "tau_t": 1.5, "theta": 0.4, "omega": 0.9, "h": 0.3}
    return Workload(f"random_s{seed}_n{n}_d{d}", t, X, X.copy(), None, None, dict(p), {"seed": seed})


CONFIGS = {"c1": make_c1, "c2": make_c2, "c3": make_c3, "c5": make_c5}


@dataclass
class BmdsWorkload:
    """Inputs of the BMDS likelihood of Eq. (4): the (N, N) observed distance
    matrix Y (symmetric, zero diagonal), latent locations X (N, D) at which it
    is evaluated, and the variance sigma2."""

    name: str
    Y: np.ndarray
    X: np.ndarray
    sigma2: float
    country: np.ndarray = field(default=None)


def make_bmds(seed: int = 5, n: int = 4733, d: int = 6, n_countries: int = 150, sigma2: float = 0.25,
              spread: float = 2.0, jitter: float = 0.1) -> BmdsWorkload:
    """Shaped like the global influenza application (Section 4.3): cases
    carry a country label, and the distance between two cases is the
    effective air-traffic distance between their countries, so Y is blocky
    and zero within a country.  Country sizes follow a Zipf(1.1) law; country
    positions are N(0, spread^2 I_D); between-country distances are the
    positions' distances plus N(0, sigma2) noise, folded to be >= 0; the
    latent locations sit at their country's position plus N(0, jitter^2 I_D)."""
    rng = np.random.default_rng(seed)
    w = 1.0 / np.arange(1, n_countries + 1) ** 1.1
    country = rng.choice(n_countries, size=n, p=w / w.sum())
    Z = rng.normal(scale=spread, size=(n_countries, d))
    Dc = np.sqrt(((Z[:, None, :] - Z[None, :, :]) ** 2).sum(-1))
    noise = rng.normal(scale=np.sqrt(sigma2), size=(n_countries, n_countries))
    noise = np.triu(noise, 1) + np.triu(noise, 1).T
    Yc = np.abs(Dc + noise)
    np.fill_diagonal(Yc, 0.0)
    Y = Yc[country][:, country]
    X = Z[country] + rng.normal(scale=jitter, size=(n, d))
    return BmdsWorkload(f"bmds_influenza_like_n{n}_d{d}", np.ascontiguousarray(Y), X, float(sigma2), country)


def bmds_random(seed: int, n: int, d: int, noise: float = 0.2, sigma2: float = 0.3) -> BmdsWorkload:
    """Unstructured BMDS case: Y = |true distances + N(0, noise^2)| + 0.05
    (symmetric), latent locations the true ones plus N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    Xt = rng.normal(size=(n, d))
    D = np.sqrt(((Xt[:, None, :] - Xt[None, :, :]) ** 2).sum(-1))
    Y = np.abs(D + noise * rng.normal(size=(n, n))) + 0.05
    Y = np.tril(Y, -1) + np.tril(Y, -1).T
    X = Xt + 0.1 * rng.normal(size=Xt.shape)
    return BmdsWorkload(f"bmds_random_n{n}_d{d}", np.ascontiguousarray(Y), X, float(sigma2))


def make_bmds_hawkes(seed: int = 5, n: int = 4733, d: int = 6) -> tuple:
    """BMDS-Hawkes inputs shaped like the influenza application (Section 4.3:
    4,733 cases over 2000-2012, D = 6): the latent locations and distance
    matrix of make_bmds, and case times spread over 12 years (4,383 days),
    each country's cases clustered around a few seasonal outbreaks.
    Parameters: tau_x = 1 and h = 0.1 in latent units (country scale and
    within-country jitter), tau_t = 30 d, theta = 0.5, omega = 1/7 d^-1,
    mu0 = 0.5.  Returns (Workload, BmdsWorkload)."""
    b = make_bmds(seed, n, d)
    rng = np.random.default_rng(seed + 100)
    n_c = int(b.country.max()) + 1
    waves = rng.uniform(0.0, 4383.0, size=(n_c, 4))
    pick = rng.integers(0, 4, size=n)
    t = np.clip(waves[b.country, pick] + rng.exponential(20.0, size=n), 0.0, 4383.0)
    params = {"mu0": 0.5, "tau_x": 1.0, "tau_t": 30.0, "theta": 0.5, "omega": 1.0 / 7.0, "h": 0.1}
    w = Workload(name=f"influenza_like_n{n}_d{d}", t=t, X=b.X.copy(), X_obs=b.X.copy(),
                 box_lo=None, box_hi=None, params=params)
    return w, b
