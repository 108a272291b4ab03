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
