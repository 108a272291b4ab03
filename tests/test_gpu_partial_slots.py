"""The pair schedule under a partial-slot cap (HAWKES_OPT_PARTIAL_SLOTS).

A set's pair blocks are dealt out in rounds that touch every row block once
(the circle method; an even block count adds an empty team whose pairs give
zero partials).  The first G rounds store slots 0 .. G - 1; each later phase
of G rounds is a further launch that stores scratch slots, which a fold
kernel adds into slots 0 .. G - 1 and clears.  Checked here:

  * small caps (G = 1 .. 4: every round, or nearly, its own launch) against
    the FP64 oracle, odd and even block counts, both precisions, the rate
    pass with the parameter-gradient sums, the self-excitation sums, a
    batch (per-dimension and one-launch), an HMC trajectory (the captured
    graph) and the far-block skip (its zero partials stored, or left in the
    cleared scratch slots);
  * the launch count: each pass makes one pair launch per phase and one
    fold per later phase;
  * the default slot budget at sizes where it binds: the FP64 path at
    N = 300,000 runs on the symmetric kernels in phases and agrees with a
    single phase (every round its own slot, 22.5 GB of slots) to rounding,
    and so does the mixed path at N = 1,000,000.

Tolerances are those of the other parity tests: FP64 1e-12, mixed 1e-6 on
ell (relative to the sum of |log lambda| and Lambda) and 1e-5 relative L2 on
the gradient.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    from paper_2010_02994_gb300 import HawkesContext

    c = HawkesContext(device=0, max_n=20_000, max_d=8)
    yield c
    c.close()


def _eval(ctx, w, prec, grad_params=False):
    import torch

    from paper_2010_02994_gb300 import hawkes_loglik_grad_locations

    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda")
    out = hawkes_loglik_grad_locations(ctx, t, X, w.params, precision=prec, grad_params=grad_params)
    return tuple(o.item() if o.dim() == 0 else o.cpu().numpy() for o in out)


def _with(ctx, opts, fn):
    for k, v in opts.items():
        ctx.set_option(k, v)
    try:
        return fn()
    finally:
        for k in opts:
            ctx.set_option(k, 0)


def _blocks(n, d, prec, warps):
    B = 256 if prec == "fp64" else 32 * (4 if d <= 4 else 2) * warps
    return -(-n // B)


# (seed, n, d, ties, cap): with two row groups of warps the mixed blocks are
# 256 (D <= 4) or 128 rows, the FP64 blocks 256 rows; the block counts below
# are odd and even in both precisions
CASES = [(1, 2500, 2, 0, 1), (2, 3000, 3, 1, 2), (3, 1700, 5, 0, 3), (4, 2100, 8, 2, 2), (5, 900, 1, 0, 1),
         (6, 2300, 4, 0, 4)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("seed,n,d,ties,cap", CASES)
def test_capped_schedule_matches_oracle(ctx, prec, seed, n, d, ties, cap):
    w = synth.random_case(seed, n, d, ties=ties, shuffle=True)
    ell_ref, g_ref, lam = oracle.loglik_and_grad(w.t, w.X, w.params)
    gp_ref, gp_scale = oracle.grad_params_scaled(w.t, w.X, w.params, lam)
    opts = {"partial_slots": cap, "block_warps": 2}
    ell, g, gp = _with(ctx, opts, lambda: _eval(ctx, w, prec, grad_params=True))
    scale = float(np.sum(np.abs(np.log(lam))) + oracle.Lambda(w.t, w.params))
    tl, tg = (1e-12, 1e-12) if prec == "fp64" else (1e-6, 1e-5)
    assert abs(ell - ell_ref) <= tl * scale
    assert rel_l2(g, g_ref) <= tg
    assert np.max(np.abs(gp - gp_ref) / gp_scale) <= tl
    # the same call without the cap: one phase, the same results to rounding
    ell1, g1, _ = _with(ctx, {"block_warps": 2}, lambda: _eval(ctx, w, prec, grad_params=True))
    assert abs(ell - ell1) <= tl * scale
    assert rel_l2(g, g1) <= tg


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_launches_per_phase(ctx, prec):
    """Each pair pass makes ceil((nb | 1) / G) pair launches and a fold after
    each but the first."""
    w = synth.random_case(7, 2500, 2, shuffle=True)
    nb = _blocks(w.n, w.d, prec, 2)
    counts = {}
    for cap in (0, 1, 3):
        def run():
            ctx.reset_stats()
            _eval(ctx, w, prec)
            return ctx.launch_count()["own"]
        counts[cap] = _with(ctx, {"partial_slots": cap, "block_warps": 2}, run)
    nt = nb | 1
    for cap in (1, 3):
        assert counts[cap] - counts[0] == 2 * 2 * (math.ceil(nt / cap) - 1), (nb, counts)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_capped_self_excitation_probability(ctx, prec):
    import torch

    from paper_2010_02994_gb300 import hawkes_self_excitation_prob

    w = synth.random_case(71, 2200, 2, ties=2, shuffle=True)
    lam, mu, xi = oracle.rates(w.t, w.X, w.params, parts=True)
    got = _with(ctx, {"partial_slots": 2, "block_warps": 2},
                lambda: hawkes_self_excitation_prob(ctx, torch.tensor(w.t, device="cuda"),
                                                    torch.tensor(w.X, device="cuda"), w.params,
                                                    precision=prec).cpu().numpy())
    assert np.max(np.abs(got - xi / lam)) <= (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec,one_launch", [("mixed", 0), ("mixed", 1), ("fp64", 0)])
def test_capped_batch(prec, one_launch):
    """Sets of several dimensions and sizes: the phases of a launch cover
    every set that still has rounds (small sets end in the first phase)."""
    import torch

    from paper_2010_02994_gb300 import HawkesContext, hawkes_batch_loglik_grad

    sets = [synth.random_case(40 + i, n, d, shuffle=True)
            for i, (n, d) in enumerate([(300, 2), (2600, 2), (1900, 4), (700, 4), (1500, 8), (2400, 2), (90, 8)])]
    ctx = HawkesContext(device=0, max_n=sum(w.n for w in sets), max_d=8)
    ctx.set_option("one_launch", one_launch)
    ctx.set_option("partial_slots", 2)
    ctx.set_option("block_warps", 2)
    cat = lambda arrs: torch.tensor(np.concatenate([np.asarray(a).reshape(-1) for a in arrs]), device="cuda")
    ell, g = hawkes_batch_loglik_grad(ctx, [w.n for w in sets], [w.d for w in sets], cat([w.t for w in sets]),
                                      cat([w.X for w in sets]), [w.params for w in sets], precision=prec)
    ell, g = ell.cpu().numpy(), g.cpu().numpy()
    ctx.close()
    tl, tg = (1e-12, 1e-12) if prec == "fp64" else (1e-6, 1e-5)
    off = 0
    for i, w in enumerate(sets):
        e_ref, g_ref, lam = oracle.loglik_and_grad(w.t, w.X, w.params)
        scale = float(np.sum(np.abs(np.log(lam))) + oracle.Lambda(w.t, w.params))
        assert abs(ell[i] - e_ref) <= tl * scale, i
        assert rel_l2(g[off:off + w.n * w.d].reshape(w.n, w.d), g_ref) <= tg, i
        off += w.n * w.d


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_capped_hmc_trajectory(prec):
    """A 10-step trajectory through the captured leapfrog graph, whose pair
    passes are one launch per phase plus the folds, against the oracle's
    replay."""
    import torch

    from paper_2010_02994_gb300 import HawkesContext, hmc_leapfrog_trajectory

    w = synth.random_case(12, 2400, 2, shuffle=True)
    p0 = np.random.default_rng(3).standard_normal(size=w.X.shape)
    eps, L = 1e-3, 10
    ref = oracle.hmc_trajectory(w.t, w.X, p0, w.params, eps, L, -np.inf)
    ctx = HawkesContext(device=0, max_n=w.n, max_d=w.d)
    ctx.set_option("partial_slots", 3)
    ctx.set_option("block_warps", 2)
    X = torch.tensor(w.X, device="cuda")
    H0, H1, acc = hmc_leapfrog_trajectory(ctx, torch.tensor(w.t, device="cuda"), X, torch.tensor(p0, device="cuda"),
                                          w.params, eps, L, -np.inf, precision=prec)
    X = X.cpu().numpy()
    ctx.close()
    tol = 1e-10 if prec == "fp64" else 1e-6
    assert int(acc.item()) == 1
    assert abs(H0.item() - ref["H0"]) <= tol * abs(ref["H0"])
    assert abs(H1.item() - ref["H1"]) <= tol * abs(ref["H1"])
    assert np.max(np.abs(X - ref["X"])) <= tol * max(1.0, float(np.max(np.abs(ref["X"]))))


def test_capped_far_block_skipping_is_exact(ctx):
    """Skipped blocks store zero partials in a slot of phase 0 and leave a
    cleared scratch slot alone, which reproduces the dense evaluation bit
    for bit."""
    w = synth.make_c3()
    opts = {"partial_slots": 2, "block_warps": 2}
    dense = _with(ctx, opts, lambda: _eval(ctx, w, "mixed"))
    skipped = _with(ctx, dict(opts, skip_far_blocks=1), lambda: _eval(ctx, w, "mixed"))
    assert skipped[0] == dense[0] and np.array_equal(skipped[1], dense[1])


@pytest.mark.slow
def test_fp64_at_300k_runs_symmetric_in_phases():
    """N = 300,000, D = 2 (the sparse wide-domain workload at three times its
    size): the default 1 GiB budget gives G = 27 slots and 27 scratch slots
    of 19.2 MB (nb = 1,172 blocks of 256 rows, 1,173 rounds, 44 phases per
    pass).  ell and the gradient agree with a single phase to 1e-12."""
    import torch

    from paper_2010_02994_gb300 import HawkesContext, hawkes_loglik_grad_locations

    w = synth.make_c5(n=300_000)
    ctx = HawkesContext(device=0, max_n=w.n, max_d=w.d)
    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda")

    def run():
        ctx.reset_stats()
        ell, g = hawkes_loglik_grad_locations(ctx, t, X, w.params, precision="fp64")
        out = ell.item(), g.cpu().numpy()
        return out + (ctx.launch_count()["own"],)

    nb = -(-w.n // 256)
    nt = nb | 1
    per_slot = nb * 256 * (6 + w.d) * 8
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    G = max(2**30 // (2 * per_slot), math.ceil(16 * sms / ((nt + 1) // 2)))
    phases = math.ceil(nt / G)
    assert phases > 1
    ell_a, g_a, n_a = run()
    ctx.set_option("partial_slots", nt)
    ell_1, g_1, n_1 = run()
    ctx.close()
    assert n_a - n_1 == 2 * 2 * (phases - 1)
    assert abs(ell_a - ell_1) <= 1e-12 * abs(ell_1)
    assert rel_l2(g_a, g_1) <= 1e-12
    assert np.isfinite(ell_a) and np.all(np.isfinite(g_a))


@pytest.mark.slow
def test_mixed_at_1m_within_slot_budget():
    """N = 1,000,000, D = 2: the mixed slots of every round would take
    11.7 GB; under the default budget the passes run in phases and agree with
    the single-phase evaluation within the mixed tolerances."""
    import torch

    from paper_2010_02994_gb300 import HawkesContext, hawkes_loglik_grad_locations

    w = synth.make_c5(n=1_000_000)
    ctx = HawkesContext(device=0, max_n=w.n, max_d=w.d)
    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda")

    def run():
        ctx.reset_stats()
        ell, g = hawkes_loglik_grad_locations(ctx, t, X, w.params, precision="mixed")
        return ell.item(), g.cpu().numpy(), ctx.launch_count()["own"]

    ell_a, g_a, n_a = run()
    ctx.set_option("partial_slots", 1 << 20)
    ell_1, g_1, n_1 = run()
    ctx.close()
    assert n_a > n_1  # the capped evaluation ran in phases
    assert abs(ell_a - ell_1) <= 1e-6 * abs(ell_1)
    assert rel_l2(g_a, g_1) <= 1e-5


def test_hmc_graph_follows_option_changes():
    """A trajectory's CUDA graph is cached per shape; changing the slot cap
    (or the far-block skip) between two calls on the same context must run
    the new plan's launches (its phases and folds), not replay the old ones:
    both calls follow the oracle's replay."""
    import torch

    from paper_2010_02994_gb300 import HawkesContext, hmc_leapfrog_trajectory

    w = synth.random_case(13, 2400, 2, shuffle=True)
    p0 = np.random.default_rng(4).standard_normal(size=w.X.shape)
    eps, L = 1e-3, 6
    ref = oracle.hmc_trajectory(w.t, w.X, p0, w.params, eps, L, -np.inf)
    ctx = HawkesContext(device=0, max_n=20_000, max_d=2)
    ctx.set_option("block_warps", 2)
    for opts in ({}, {"partial_slots": 2}, {"partial_slots": 2, "skip_far_blocks": 1}, {}):
        for k in ("partial_slots", "skip_far_blocks"):
            ctx.set_option(k, opts.get(k, 0))
        X = torch.tensor(w.X, device="cuda")
        H0, H1, acc = hmc_leapfrog_trajectory(ctx, torch.tensor(w.t, device="cuda"), X,
                                              torch.tensor(p0, device="cuda"), w.params, eps, L, -np.inf,
                                              precision="mixed")
        assert int(acc.item()) == 1, opts
        assert abs(H1.item() - ref["H1"]) <= 1e-6 * abs(ref["H1"]), opts
        assert np.max(np.abs(X.cpu().numpy() - ref["X"])) <= 1e-6 * max(1.0, float(np.max(np.abs(ref["X"])))), opts
    ctx.close()
