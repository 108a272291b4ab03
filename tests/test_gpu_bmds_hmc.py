"""HMC over the BMDS-Hawkes potential (hawkes_bmds_hmc_trajectory) against
the FP64 oracle's trajectory of the same potential: FP64 to 1e-10, mixed
precision to 1e-6 (relative, as for the Hawkes-only trajectory)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2010_02994_gb300 import HawkesContext

    c = HawkesContext(device=0, max_n=5000, max_d=8)
    yield c
    c.close()


def case(seed, n, d):
    """Hawkes events with latent locations near an embedding whose distances
    (plus noise) form Y, as in the influenza model."""
    w = synth.random_case(seed, n, d, shuffle=True, extent=2.0, t_end=5.0)
    rng = np.random.default_rng(seed)
    D = np.sqrt(((w.X[:, None, :] - w.X[None, :, :]) ** 2).sum(-1))
    Y = np.abs(D + 0.2 * rng.normal(size=(n, n)))
    Y = np.tril(Y, -1) + np.tril(Y, -1).T
    p0 = rng.standard_normal(size=w.X.shape)
    return w, Y, p0


def gpu(ctx, w, Y, p0, sigma2, eps, L, log_u, prec, y32=False):
    import torch

    from paper_2010_02994_gb300 import hawkes_bmds_hmc_trajectory

    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda")
    Yd = torch.tensor(Y, device="cuda")
    if y32:
        Yd = Yd.float()
    p = torch.tensor(p0, device="cuda")
    H0, H1, acc = hawkes_bmds_hmc_trajectory(ctx, t, X, p, w.params, Yd, sigma2, eps, L, log_u, precision=prec)
    return X.cpu().numpy(), H0.item(), H1.item(), int(acc.item())


@pytest.mark.parametrize("seed,n,d", [(1, 150, 2), (2, 400, 6), (3, 97, 3)])
def test_fp64_bmds_trajectory_matches_oracle(ctx, seed, n, d):
    w, Y, p0 = case(seed, n, d)
    ref = oracle.bmds_hmc_trajectory(w.t, w.X, p0, w.params, Y, 0.3, 0.002, 12, -np.inf)
    X, H0, H1, acc = gpu(ctx, w, Y, p0, 0.3, 0.002, 12, -np.inf, "fp64")
    assert acc == ref["accepted"] == 1
    assert abs(H0 - ref["H0"]) <= 1e-11 * abs(ref["H0"])
    assert abs(H1 - ref["H1"]) <= 1e-10 * abs(ref["H1"])
    assert np.max(np.abs(X - ref["X"])) <= 1e-10 * (1 + np.max(np.abs(ref["X"])))


def test_mixed_bmds_trajectory_matches_oracle(ctx):
    w, Y, p0 = case(4, 600, 6)
    ref = oracle.bmds_hmc_trajectory(w.t, w.X, p0, w.params, Y, 0.3, 0.002, 10, -np.inf)
    for y32 in (False, True):
        X, H0, H1, acc = gpu(ctx, w, Y, p0, 0.3, 0.002, 10, -np.inf, "mixed", y32=y32)
        assert acc == 1
        assert abs(H0 - ref["H0"]) <= 1e-6 * abs(ref["H0"])
        assert abs(H1 - ref["H1"]) <= 1e-6 * abs(ref["H1"])
        assert np.max(np.abs(X - ref["X"])) <= 1e-6 * np.max(np.abs(ref["X"]))


def test_bmds_trajectory_recaptures_on_new_sigma2_and_rejects(ctx):
    """The cached graph is keyed by sigma2 (and Y): a second call with another
    variance follows the oracle for that variance; a log u above H0 - H1
    rejects and leaves X unchanged."""
    w, Y, p0 = case(5, 200, 2)
    for s2 in (0.3, 0.7):
        ref = oracle.bmds_hmc_trajectory(w.t, w.X, p0, w.params, Y, s2, 0.002, 8, -np.inf)
        X, H0, H1, acc = gpu(ctx, w, Y, p0, s2, 0.002, 8, -np.inf, "fp64")
        assert abs(H1 - ref["H1"]) <= 1e-10 * abs(ref["H1"])
        dh = ref["H0"] - ref["H1"]
        X, _, _, acc = gpu(ctx, w, Y, p0, s2, 0.002, 8, dh + 1e-6, "fp64")
        assert acc == 0 and np.array_equal(X, w.X)


def _case_ties(seed, n, d, ties):
    w = synth.random_case(seed, n, d, ties=ties, shuffle=True, extent=2.0, t_end=5.0)
    rng = np.random.default_rng(seed)
    D = np.sqrt(((w.X[:, None, :] - w.X[None, :, :]) ** 2).sum(-1))
    Y = np.abs(D + 0.2 * rng.normal(size=(n, n)))
    Y = np.tril(Y, -1) + np.tril(Y, -1).T
    return w, Y, rng.standard_normal(size=w.X.shape)


DEFAULTS = {"bmds_fused": 0, "mixed_fixup_exp": -76}


def _with(ctx, opts, fn):
    for k, v in opts.items():
        ctx.set_option(k, v)
    try:
        return fn()
    finally:
        for k in opts:
            ctx.set_option(k, DEFAULTS.get(k, 0))


# (seed, n, d, ties, options): the fused gradient pass (forced on) with
# tied times, odd and even block counts, padded last blocks, rows recomputed
# in FP64 (a fixup threshold of 2^-1 flags most rows) and a slot cap that
# runs the gradient pass in phases with folds
FUSED_CASES = [(11, 600, 6, 0, {}), (12, 517, 2, 2, {}), (13, 300, 3, 1, {"block_warps": 1}),
               (14, 450, 6, 0, {"mixed_fixup_exp": -1}), (15, 700, 4, 0, {"partial_slots": 2, "block_warps": 2}),
               (16, 333, 8, 1, {"block_warps": 2})]


@pytest.mark.parametrize("seed,n,d,ties,opts", FUSED_CASES)
def test_fused_bmds_gradient_pass_matches_oracle(ctx, seed, n, d, ties, opts):
    """The BMDS term inside the Hawkes gradient pass (one pair loop, a
    time-ordered FP32 copy of Y, the BMDS kernels only for ell_B at the ends)
    follows the oracle's trajectory to 1e-6, as the two-stream form does."""
    w, Y, p0 = _case_ties(seed, n, d, ties)
    ref = oracle.bmds_hmc_trajectory(w.t, w.X, p0, w.params, Y, 0.3, 0.002, 8, -np.inf)
    for fused in (1, 0):
        X, H0, H1, acc = _with(ctx, dict(opts, bmds_fused=fused),
                               lambda: gpu(ctx, w, Y, p0, 0.3, 0.002, 8, -np.inf, "mixed"))
        assert acc == 1
        assert abs(H0 - ref["H0"]) <= 1e-6 * abs(ref["H0"]), fused
        assert abs(H1 - ref["H1"]) <= 1e-6 * abs(ref["H1"]), fused
        assert np.max(np.abs(X - ref["X"])) <= 1e-6 * np.max(np.abs(ref["X"])), fused


@pytest.mark.slow
def test_fused_bmds_influenza_like_trajectory(ctx):
    """The influenza-shaped workload (N = 4,733, D = 6, 20 leapfrog steps):
    fused and two-stream trajectories against the oracle's."""
    import torch

    from paper_2010_02994_gb300 import hawkes_bmds_hmc_trajectory

    w, b = synth.make_bmds_hawkes()
    Y, sigma2 = b.Y, b.sigma2
    p0 = np.random.default_rng(8).standard_normal(size=w.X.shape)
    eps, L = 1e-3, 20
    ref = oracle.bmds_hmc_trajectory(w.t, w.X, p0, w.params, Y, sigma2, eps, L, -np.inf)
    for fused in (1, 0):
        ctx.set_option("bmds_fused", fused)
        X = torch.tensor(w.X, device="cuda")
        H0, H1, acc = hawkes_bmds_hmc_trajectory(ctx, torch.tensor(w.t, device="cuda"), X,
                                                 torch.tensor(p0, device="cuda"), w.params,
                                                 torch.tensor(Y, device="cuda").float(), sigma2, eps, L, -np.inf,
                                                 precision="mixed")
        ctx.set_option("bmds_fused", 0)
        X = X.cpu().numpy()
        assert int(acc.item()) == ref["accepted"]
        assert abs(H0.item() - ref["H0"]) <= 1e-6 * abs(ref["H0"])
        assert abs(H1.item() - ref["H1"]) <= 1e-6 * abs(ref["H1"])
        assert np.max(np.abs(X - ref["X"])) <= 1e-6 * np.max(np.abs(ref["X"]))


def test_fused_term_does_not_leak_into_later_calls(ctx):
    """After a fused BMDS-Hawkes trajectory, a plain evaluation (with most
    rows recomputed in FP64, where the BMDS term would enter) is the same
    bit for bit as before it."""
    import torch

    from paper_2010_02994_gb300 import hawkes_loglik_grad_locations

    w, Y, p0 = _case_ties(21, 400, 6, 0)
    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda")

    def plain():
        ell, g = hawkes_loglik_grad_locations(ctx, t, X, w.params, precision="mixed")
        return ell.item(), g.cpu().numpy()

    before = _with(ctx, {"mixed_fixup_exp": -1}, plain)
    _with(ctx, {"bmds_fused": 1}, lambda: gpu(ctx, w, Y, p0, 0.3, 0.002, 4, -np.inf, "mixed"))
    after = _with(ctx, {"mixed_fixup_exp": -1}, plain)
    assert before[0] == after[0] and np.array_equal(before[1], after[1])
