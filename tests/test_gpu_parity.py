"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (fixed for this method): the FP64 path within 1e-12 (relative for
ell, relative L2 for the gradient); the mixed path within 1e-6 for ell and
1e-5 for the gradient.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-12, 1e-12), "mixed": (1e-6, 1e-5)}


@pytest.fixture(scope="module")
def ctx():
    from paper_2010_02994_gb300 import HawkesContext

    c = HawkesContext(device=0, max_n=100_000, max_d=8)
    yield c
    c.close()


def gpu_eval(ctx, w, prec, t=None, X=None):
    import torch

    from paper_2010_02994_gb300 import hawkes_loglik_grad_locations

    t = torch.tensor(w.t if t is None else t, device="cuda")
    X = torch.tensor(w.X if X is None else X, device="cuda")
    ell, g = hawkes_loglik_grad_locations(ctx, t, X, w.params, precision=prec)
    return ell.item(), g.cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def ell_scale(w, lam=None):
    """Sum of the magnitudes of the terms of ell (sum |log lambda_n| + sum Lambda_n):
    the scale a rounding error of the terms is relative to, even when ell
    itself is near zero by cancellation."""
    if lam is None:
        lam = oracle.rates(w.t, w.X, w.params)
    return float(np.sum(np.abs(np.log(lam))) + oracle.Lambda(w.t, w.params))


def assert_close(ctx, w, prec, ref=None, conditioned=True):
    """ell within TOL of the oracle relative to |ell| (paper-shaped workloads,
    conditioned=False) or to the terms' magnitude (random data); the gradient
    in relative L2."""
    ell_ref, g_ref, lam = oracle.loglik_and_grad(w.t, w.X, w.params) if ref is None else (*ref, None)
    ell, g = gpu_eval(ctx, w, prec)
    tl, tg = TOL[prec]
    assert math.isfinite(ell)
    scale = ell_scale(w, lam) if conditioned else abs(ell_ref)
    el = abs(ell - ell_ref) / scale
    eg = rel_l2(g, g_ref)
    assert el <= tl, f"{w.name} {prec}: ell {ell} vs {ell_ref} (rel {el:.2e})"
    assert eg <= tg, f"{w.name} {prec}: grad rel-L2 {eg:.2e}"
    return el, eg


CASES = [
    (1, 2, 1, 0), (2, 3, 3, 0), (3, 37, 2, 0), (4, 130, 1, 1), (5, 700, 2, 2), (6, 1100, 3, 0),
    (7, 300, 5, 1), (8, 260, 8, 0), (9, 513, 4, 2), (10, 129, 6, 0), (11, 200, 7, 0), (12, 2600, 2, 3),
]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("seed,n,d,ties", CASES)
def test_random_cases(ctx, prec, seed, n, d, ties):
    w = synth.random_case(seed, n, d, ties=ties, shuffle=True)
    assert_close(ctx, w, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("make", [synth.make_c1, synth.make_c3, synth.make_c2])
def test_paper_shaped_workloads(ctx, prec, make):
    w = make()
    assert_close(ctx, w, prec, conditioned=False)


@pytest.fixture(scope="module")
def c5_reference():
    """Oracle rates of every row of the N=1e5 workload, and ell_n, grad_n of
    2,000 seeded random rows."""
    w = synth.make_c5()
    lam = oracle.rates(w.t, w.X, w.params)
    _, Lam = oracle.Lambda(w.t, w.params, per_event=True)
    ell = float(np.sum(np.log(lam)) - np.sum(Lam))
    rows = np.sort(np.random.default_rng(5).choice(w.n, size=2000, replace=False))
    g_rows = oracle.grad_rows(w.t, w.X, w.params, lam, rows)
    return w, ell, rows, g_rows, lam


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_large_workload_sampled_rows(ctx, c5_reference, prec):
    w, ell_ref, rows, g_rows, _ = c5_reference
    ell, g = gpu_eval(ctx, w, prec)
    tl, tg = TOL[prec]
    assert abs(ell - ell_ref) / abs(ell_ref) <= tl
    assert rel_l2(g[rows], g_rows) <= tg
    # translation invariance holds at every size: sum_n grad_n = 0
    assert np.all(np.abs(g.sum(axis=0)) <= 1e-6 * np.abs(g).sum(axis=0))


@pytest.mark.slow
def test_large_workload_parameter_gradient(ctx, c5_reference):
    """The N = 100,000 workload's d ell / d Theta in both precisions against
    the oracle (all rows), each component within the precision's tolerance
    relative to the magnitude of the terms it is summed from (the score
    itself is a sum of N terms of either sign near the data-generating Theta,
    so it cancels far below that magnitude)."""
    import torch

    from paper_2010_02994_gb300 import hawkes_loglik_grad_locations

    w, ell_ref, _, _, lam = c5_reference
    gp_ref, scale = oracle.grad_params_scaled(w.t, w.X, w.params, lam)
    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda")
    for prec, tol in (("mixed", 1e-6), ("fp64", 1e-12)):
        ell, _, gp = hawkes_loglik_grad_locations(ctx, t, X, w.params, precision=prec, grad_params=True)
        err = np.abs(gp.cpu().numpy() - gp_ref) / scale
        assert np.all(err <= tol), (prec, err, gp.cpu().numpy(), gp_ref)
        assert abs(ell.item() - ell_ref) <= TOL[prec][0] * abs(ell_ref)
        print(f"c5 grad_params {prec}: max error / scale {np.max(err):.2e}")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_event_and_all_tied(ctx, prec):
    import torch

    from paper_2010_02994_gb300 import HawkesError, hawkes_loglik, hawkes_loglik_grad_locations

    P = synth.random_case(0, 2, 2).params
    for t_np, X_np in (([1.0], [[0.3, 0.2]]), ([2.0, 2.0, 2.0], [[0.0, 0.0], [0.1, 0.0], [0.0, 0.2]])):
        t = torch.tensor(t_np, dtype=torch.float64, device="cuda")
        X = torch.tensor(X_np, dtype=torch.float64, device="cuda")
        ell = hawkes_loglik(ctx, t, X, P, precision=prec)
        assert ell.item() == -math.inf
        with pytest.raises(HawkesError) as e:
            hawkes_loglik_grad_locations(ctx, t, X, P, precision=prec)
        assert "ZERO_RATE" in str(e.value)
        ctx.sync_status()  # the status is cleared once reported


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_signed_zero_times_tie(ctx, prec):
    """Times of exactly +0 and -0 are equal (a tie: neither excites the
    other), and the time sort and the tie runs must treat them so: the keys
    of the time sort compare bit patterns, with the sign cleared."""
    w = synth.random_case(61, 400, 2, shuffle=True)
    t = w.t.copy()
    t[[3, 50, 199]] = 0.0
    t[[7, 120]] = -0.0
    w = dataclasses.replace(w, t=t)
    assert np.sum(np.signbit(w.t)) == 2
    assert_close(ctx, w, prec)


def test_ragged_block_edges(ctx):
    """Sizes around the pair-block edge with the smallest block (128 rows at D=2)."""
    ctx.set_option("block_warps", 1)
    try:
        for n in (127, 128, 129, 257, 383):
            w = synth.random_case(40 + n, n, 2, ties=1, shuffle=True)
            assert_close(ctx, w, "mixed")
    finally:
        ctx.set_option("block_warps", 0)


@pytest.mark.parametrize("warps", [1, 2, 4, 8])
def test_every_block_shape(ctx, warps):
    ctx.set_option("block_warps", warps)
    try:
        for d in (2, 3, 8):
            w = synth.random_case(60 + warps * 10 + d, 1500, d, ties=2, shuffle=True)
            assert_close(ctx, w, "mixed")
    finally:
        ctx.set_option("block_warps", 0)


def test_isolated_events_take_the_fp64_fixup(ctx):
    """Events far from every other in space and time have rates far below the
    FP32 range of the kernel values; they are recomputed in FP64."""
    w = synth.random_case(77, 600, 2, shuffle=True)
    P = w.params
    t = w.t.copy()
    X = w.X.copy()
    last = int(np.argmax(t))
    # the latest event, 15 tau_t after the others and 6 km away: every kernel
    # value it sees is ~e^-140, far below FP32's range but not zero in FP64
    t[5] = t[last] + 15.0 * P["tau_t"]
    X[5] = X[last] + [6.0, 0.0]
    # an event 12 km from all others, inside the time range: ~e^-112
    X[17] = X.min(axis=0) - [12.0, 0.0]
    w2 = synth.Workload("isolated", t, X, X, None, None, P)
    lam = oracle.rates(t, X, P)
    assert 0.0 < lam[5] < 1e-40 and 0.0 < lam[17] < 1e-40
    assert_close(ctx, w2, "mixed")
    assert_close(ctx, w2, "fp64")


@pytest.mark.parametrize("n,d,extent", [(600, 8, 40.0), (2000, 6, 60.0), (400, 4, 100.0), (1000, 5, 80.0)])
def test_most_rows_take_the_fp64_fixup(ctx, n, d, extent):
    """Events spread so far apart (bandwidths small against the spacing) that
    nearly every rate underflows the FP32 kernel values: those rows are
    recomputed in FP64, their work dealt over several CTAs per segment at
    these sizes, and the location gradient takes their FP64 terms."""
    rng = np.random.default_rng(100 + d)
    t = np.sort(rng.uniform(0.0, 365.0, size=n))
    X = rng.uniform(0.0, extent, size=(n, d))
    P = {"mu0": 0.5, "tau_x": 1.0, "tau_t": 14.0, "theta": 0.5, "omega": 0.5, "h": 0.1}
    w = synth.Workload("spread_out", t, X, X, None, None, P)
    lam = oracle.rates(t, X, P)
    Pmu = P["mu0"] / (P["tau_x"] ** d * P["tau_t"] * (2 * math.pi) ** (d / 2 + 0.5))
    assert np.mean(lam / Pmu < 2.0 ** -76) > 0.9  # rows below the FP32 threshold
    assert_close(ctx, w, "mixed")
    assert_close(ctx, w, "fp64")


def test_invalid_data_is_reported(ctx):
    import torch

    from paper_2010_02994_gb300 import HawkesError, hawkes_loglik_grad_locations

    w = synth.random_case(3, 50, 2)
    for bad in ("nan_x", "neg_t", "inf_t"):
        t = torch.tensor(w.t, device="cuda")
        X = torch.tensor(w.X, device="cuda")
        if bad == "nan_x":
            X[3, 1] = float("nan")
        elif bad == "neg_t":
            t[7] = -1.0
        else:
            t[0] = float("inf")
        with pytest.raises(HawkesError) as e:
            hawkes_loglik_grad_locations(ctx, t, X, w.params)
        assert "INVALID_DATA" in str(e.value)
    # the context is usable afterwards
    assert_close(ctx, w, "mixed")


def test_invalid_arguments(ctx):
    import torch

    from paper_2010_02994_gb300 import HawkesError, hawkes_loglik

    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    X = torch.zeros(4, 9, dtype=torch.float64, device="cuda")
    with pytest.raises(HawkesError):
        hawkes_loglik(ctx, t, X, synth.random_case(0, 2, 2).params)
    with pytest.raises(HawkesError):
        hawkes_loglik(ctx, t, X[:, :2], dict(synth.random_case(0, 2, 2).params, h=-1.0))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_deterministic_and_permutation_equivariant(ctx, prec):
    w = synth.random_case(91, 1800, 2, shuffle=True)
    a = gpu_eval(ctx, w, prec)
    b = gpu_eval(ctx, w, prec)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    perm = np.random.default_rng(1).permutation(w.n)
    c = gpu_eval(ctx, w, prec, t=w.t[perm], X=w.X[perm])
    assert c[0] == a[0] and np.array_equal(c[1], a[1][perm])


def test_times_sorted_option(ctx):
    from paper_2010_02994_gb300 import HawkesError

    w = synth.random_case(5, 900, 2, shuffle=False)
    ref = gpu_eval(ctx, w, "mixed")
    ctx.set_option("times_sorted", 1)
    try:
        got = gpu_eval(ctx, w, "mixed")
        assert got[0] == ref[0] and np.array_equal(got[1], ref[1])
        ws = synth.random_case(5, 900, 2, shuffle=True)
        with pytest.raises(HawkesError):
            gpu_eval(ctx, ws, "mixed")
    finally:
        ctx.set_option("times_sorted", 0)


@pytest.mark.parametrize("make", [synth.make_c5, synth.make_c3])
def test_far_block_skipping_is_exact(ctx, make):
    """Blocks whose closest pair already underflows FP32 contribute exactly
    zero, so skipping them must reproduce the dense result bit for bit."""
    w = make()
    dense = gpu_eval(ctx, w, "mixed")
    ctx.set_option("skip_far_blocks", 1)
    try:
        skipped = gpu_eval(ctx, w, "mixed")
    finally:
        ctx.set_option("skip_far_blocks", 0)
    assert skipped[0] == dense[0]
    assert np.array_equal(skipped[1], dense[1])


def test_pipe_rate_probes():
    """The measured rates the rooflines use are finite and plausible for one
    SM (FP32 FMA up to 128 lanes per clock, MUFU ex2 and FP64 FMA far fewer)."""
    from paper_2010_02994_gb300 import probe_dfma_rate, probe_pipe_rates

    r = probe_pipe_rates(0)
    assert 32.0 <= r["fma_per_sm_clk"] <= 160.0
    assert 4.0 <= r["ex2_per_sm_clk"] <= 64.0
    assert 100.0 <= r["sm_mhz"] <= 4000.0
    dfma = probe_dfma_rate(0)
    assert 0.0 < dfma <= 64.0
