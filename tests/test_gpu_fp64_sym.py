"""The FP64 path's two pair layouts against the FP64 oracle.

By default the FP64 path evaluates each unordered pair once (symmetric
kernels over 256-row pair blocks, base-2 exponentials by Tang's
table-driven method); with the option fp64_ordered it evaluates every
ordered pair with CUDA's exp(), the layout it falls back to when the
symmetric kernels' partial slots would not fit.  Both must match the oracle
within 1e-12, and the exponential must stay within 2 ulp of the host's exp2.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2010_02994_gb300 import HawkesContext

    c = HawkesContext(device=0, max_n=20_000, max_d=8)
    yield c
    c.close()


def ulp(x):
    """Spacing of doubles at |x| (2^-1074 in the subnormal range)."""
    x = np.abs(x)
    return np.maximum(np.spacing(x), np.float64(5e-324))


def test_exp2_within_two_ulp_of_host():
    import torch

    from paper_2010_02994_gb300 import probe_exp2_fp64

    rng = np.random.default_rng(11)
    parts = [
        -rng.uniform(0.0, 1.0, 200_000),                     # the table and polynomial range
        -rng.uniform(0.0, 1100.0, 400_000),                  # the whole normal range and beyond
        -1022.0 - rng.uniform(0.0, 54.0, 200_000),           # subnormal results
        -np.ldexp(rng.uniform(0.5, 1.0, 100_000), -rng.integers(1, 60, 100_000)),  # tiny |y|
        -np.arange(0, 1101, dtype=np.float64),               # integers: exact powers of two
        -np.arange(0, 16384, dtype=np.float64) / 2048.0,     # the table's nodes
        -(np.arange(0, 16384, dtype=np.float64) + 0.5) / 2048.0,  # midway between nodes
    ]
    y = np.concatenate(parts)
    got = probe_exp2_fp64(torch.tensor(y, device="cuda")).cpu().numpy()
    ref = np.exp2(y)
    err = np.abs(got - ref) / ulp(ref)
    assert np.all(np.isfinite(got))
    assert float(err.max()) <= 2.0, (y[np.argmax(err)], float(err.max()))
    # exact powers of two, and zero below the subnormal range
    k = -np.arange(0, 1075, dtype=np.float64)
    assert np.array_equal(probe_exp2_fp64(torch.tensor(k, device="cuda")).cpu().numpy(), np.exp2(k))
    special = np.array([-0.0, 0.0, -1075.5, -1100.0, -5000.0, -np.inf, 3.0])
    out = probe_exp2_fp64(torch.tensor(special, device="cuda")).cpu().numpy()
    assert out.tolist() == [1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 1.0]


def eval_both(ctx, w, grad_params=False):
    import torch

    from paper_2010_02994_gb300 import hawkes_loglik_grad_locations

    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda")
    res = {}
    for ordered in (0, 1):
        ctx.set_option("fp64_ordered", ordered)
        try:
            out = hawkes_loglik_grad_locations(ctx, t, X, w.params, precision="fp64", grad_params=grad_params)
        finally:
            ctx.set_option("fp64_ordered", 0)
        res[ordered] = [o.cpu().numpy() if o.dim() else o.item() for o in out]
    return res[0], res[1]


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("seed,n,d,ties", [
    (21, 2, 1, 0), (22, 255, 2, 0), (23, 256, 3, 1), (24, 257, 2, 0), (25, 700, 1, 2), (26, 1300, 4, 0),
    (27, 600, 5, 1), (28, 520, 6, 0), (29, 777, 7, 2), (30, 900, 8, 0), (31, 3000, 2, 3),
])
def test_symmetric_and_ordered_match_oracle(ctx, seed, n, d, ties):
    w = synth.random_case(seed, n, d, ties=ties, shuffle=True)
    ell_ref, g_ref, lam = oracle.loglik_and_grad(w.t, w.X, w.params)
    scale = float(np.sum(np.abs(np.log(lam))) + oracle.Lambda(w.t, w.params))
    sym, ordd = eval_both(ctx, w)
    for name, (ell, g) in (("symmetric", sym), ("ordered", ordd)):
        assert abs(ell - ell_ref) <= 1e-12 * scale, (name, ell, ell_ref)
        assert rel_l2(g, g_ref) <= 1e-12, (name, rel_l2(g, g_ref))
    # the two layouts agree with each other more tightly than with the oracle's tolerance
    assert abs(sym[0] - ordd[0]) <= 1e-13 * scale
    assert rel_l2(sym[1], ordd[1]) <= 1e-13


@pytest.mark.parametrize("seed,n,d", [(41, 300, 2), (42, 1000, 3), (43, 513, 8)])
def test_symmetric_parameter_sums(ctx, seed, n, d):
    w = synth.random_case(seed, n, d, ties=1, shuffle=True)
    _, _, lam = oracle.loglik_and_grad(w.t, w.X, w.params)
    gp_ref = oracle.grad_params(w.t, w.X, w.params, lam)
    sym, ordd = eval_both(ctx, w, grad_params=True)
    for name, res in (("symmetric", sym), ("ordered", ordd)):
        err = np.max(np.abs(res[2] - gp_ref) * w.theta_vector()) / n
        assert err <= 1e-12, (name, res[2], gp_ref)


@pytest.mark.parametrize("seed,d,tau_t,omega", [(51, 2, 1.0, 5.0), (52, 3, 0.5, 0.5), (53, 1, 2.0, 20.0)])
def test_time_gaps_that_zero_whole_chunks(ctx, seed, d, tau_t, omega):
    """Events spread over a long time with a short tau_t (and, in some cases, a
    fast decay omega): most 32 x 32 pair chunks are exactly zero in one or both
    terms and the kernels skip them; the results must not change."""
    rng = np.random.default_rng(seed)
    n = 1500
    t = np.sort(rng.uniform(0.0, 4000.0, n))
    t[rng.integers(0, n, 40)] = t[rng.integers(0, n, 40)]  # some ties
    rng.shuffle(t)
    X = rng.normal(scale=2.0, size=(n, d))
    params = dict(mu0=0.8, tau_x=1.0, tau_t=tau_t, theta=0.5, omega=omega, h=0.7)
    w = synth.Workload(name=f"gaps{seed}", t=t, X=X, X_obs=X, box_lo=None, box_hi=None, params=params)
    ell_ref, g_ref, lam = oracle.loglik_and_grad(w.t, w.X, w.params)
    scale = float(np.sum(np.abs(np.log(lam))) + oracle.Lambda(w.t, w.params))
    sym, ordd = eval_both(ctx, w)
    for name, (ell, g) in (("symmetric", sym), ("ordered", ordd)):
        assert abs(ell - ell_ref) <= 1e-12 * scale, (name, ell, ell_ref)
        assert rel_l2(g, g_ref) <= 1e-12, (name, rel_l2(g, g_ref))


def test_rates_in_the_subnormal_range(ctx):
    """Events about 37.7 tau_x apart: every kernel value is a subnormal double
    (the exponentials' two-step scaling), the rates are subnormal but not zero
    and ell stays finite; the self-excitation terms underflow to zero."""
    import torch

    from paper_2010_02994_gb300 import hawkes_loglik

    X = np.array([[0.0], [37.7], [75.4], [37.69]])
    t = np.array([0.0, 1.0, 2.0, 3.0])
    params = dict(mu0=1.0, tau_x=1.0, tau_t=1000.0, theta=1.0, omega=1.0, h=0.01)
    lam = oracle.rates(t, X, params)
    assert np.all(lam > 0) and np.any(lam < 2.2250738585072014e-308)
    ell_ref = oracle.loglik(t, X, params)
    for ordered in (0, 1):
        ctx.set_option("fp64_ordered", ordered)
        try:
            ell = hawkes_loglik(ctx, torch.tensor(t, device="cuda"), torch.tensor(X, device="cuda"), params,
                                precision="fp64").item()
        finally:
            ctx.set_option("fp64_ordered", 0)
        assert math.isfinite(ell)
        assert abs(ell - ell_ref) <= 1e-12 * abs(ell_ref), (ordered, ell, ell_ref)


def test_all_tied_is_a_zero_rate(ctx):
    """Equal times exclude every pair (both indicators vanish)."""
    import torch

    from paper_2010_02994_gb300 import hawkes_loglik

    rng = np.random.default_rng(3)
    n = 600
    t = np.full(n, 2.5)
    X = rng.normal(size=(n, 2))
    params = dict(mu0=1.0, tau_x=1.0, tau_t=1.0, theta=0.5, omega=1.0, h=0.5)
    ell = hawkes_loglik(ctx, torch.tensor(t, device="cuda"), torch.tensor(X, device="cuda"), params,
                        precision="fp64").item()
    assert ell == -math.inf
