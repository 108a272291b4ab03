"""HMC trajectories and the batched entry point against the FP64 oracle."""
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


def hmc_case(seed, n, d, box=True):
    w = synth.random_case(seed, n, d, shuffle=True, extent=2.0, t_end=5.0)
    rng = np.random.default_rng(seed)
    lo = w.X - rng.uniform(0.01, 0.08, size=w.X.shape) if box else None
    hi = w.X + rng.uniform(0.01, 0.08, size=w.X.shape) if box else None
    p0 = rng.standard_normal(size=w.X.shape)
    return w, lo, hi, p0


def gpu_hmc(ctx, w, lo, hi, p0, eps, L, log_u, prec):
    import torch

    from paper_2010_02994_gb300 import hmc_leapfrog_trajectory

    dev = "cuda"
    t = torch.tensor(w.t, device=dev)
    X = torch.tensor(w.X, device=dev)
    p = torch.tensor(p0, device=dev)
    blo = None if lo is None else torch.tensor(lo, device=dev)
    bhi = None if hi is None else torch.tensor(hi, device=dev)
    H0, H1, acc = hmc_leapfrog_trajectory(ctx, t, X, p, w.params, eps, L, log_u, blo, bhi, precision=prec)
    return X.cpu().numpy(), H0.item(), H1.item(), int(acc.item())


@pytest.mark.parametrize("box", [True, False])
def test_fp64_trajectory_matches_oracle(ctx, box):
    w, lo, hi, p0 = hmc_case(3, 300, 2, box)
    ref = oracle.hmc_trajectory(w.t, w.X, p0, w.params, 0.01, 20, -np.inf, lo, hi)
    X, H0, H1, acc = gpu_hmc(ctx, w, lo, hi, p0, 0.01, 20, -np.inf, "fp64")
    assert acc == ref["accepted"] == 1
    assert abs(H0 - ref["H0"]) <= 1e-11 * abs(ref["H0"])
    assert abs(H1 - ref["H1"]) <= 1e-10 * abs(ref["H1"])
    assert np.max(np.abs(X - ref["X"])) <= 1e-10
    if box:
        assert np.all(X >= lo) and np.all(X <= hi)


def test_mixed_trajectory_matches_oracle(ctx):
    w, lo, hi, p0 = hmc_case(4, 500, 2, True)
    ref = oracle.hmc_trajectory(w.t, w.X, p0, w.params, 0.01, 20, -np.inf, lo, hi)
    X, H0, H1, acc = gpu_hmc(ctx, w, lo, hi, p0, 0.01, 20, -np.inf, "mixed")
    assert acc == 1
    assert abs(H0 - ref["H0"]) <= 1e-6 * abs(ref["H0"])
    assert abs(H1 - ref["H1"]) <= 1e-6 * abs(ref["H1"])
    assert np.max(np.abs(X - ref["X"])) <= 1e-6 * np.max(np.abs(ref["X"]))


def test_accept_and_reject_decisions(ctx):
    w, lo, hi, p0 = hmc_case(5, 200, 2, True)
    ref = oracle.hmc_trajectory(w.t, w.X, p0, w.params, 0.02, 10, -np.inf, lo, hi)
    dh = ref["H0"] - ref["H1"]
    # accepted just below the threshold, rejected just above: X unchanged
    X, _, _, acc = gpu_hmc(ctx, w, lo, hi, p0, 0.02, 10, dh - 1e-6, "fp64")
    assert acc == 1 and np.max(np.abs(X - ref["X"])) <= 1e-10
    X, _, _, acc = gpu_hmc(ctx, w, lo, hi, p0, 0.02, 10, dh + 1e-6, "fp64")
    assert acc == 0 and np.array_equal(X, w.X)


def test_graph_replay_is_reproducible(ctx):
    w, lo, hi, p0 = hmc_case(6, 400, 3, True)
    a = gpu_hmc(ctx, w, lo, hi, p0, 0.01, 5, -np.inf, "mixed")
    b = gpu_hmc(ctx, w, lo, hi, p0, 0.01, 5, -np.inf, "mixed")
    assert a[1:] == b[1:] and np.array_equal(a[0], b[0])


def test_zero_steps(ctx):
    w, lo, hi, p0 = hmc_case(7, 100, 2, True)
    X, H0, H1, acc = gpu_hmc(ctx, w, lo, hi, p0, 0.01, 0, -1e-3, "fp64")
    assert H0 == H1 and acc == 1 and np.array_equal(X, w.X)


def batch_sets(seed, specs):
    sets = []
    for i, (n, d) in enumerate(specs):
        w = synth.random_case(seed + i, n, d, ties=i % 2, shuffle=True)
        if i % 3 == 1:
            w.params = dict(w.params, h=0.2, omega=1.3)
        sets.append(w)
    return sets


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_per_set_oracle(ctx, prec):
    import torch

    from paper_2010_02994_gb300 import hawkes_batch_loglik_grad

    sets = batch_sets(100, [(300, 2), (1000, 4), (90, 8), (2500, 2), (1, 2), (640, 8), (700, 3)])
    t = torch.tensor(np.concatenate([w.t for w in sets]), device="cuda")
    X = torch.tensor(np.concatenate([w.X.reshape(-1) for w in sets]), device="cuda")
    from paper_2010_02994_gb300 import HawkesError

    with pytest.raises(HawkesError):  # the one-event set has a zero rate
        hawkes_batch_loglik_grad(ctx, [w.n for w in sets], [w.d for w in sets], t, X, [w.params for w in sets],
                                 precision=prec)
    sets = [w for w in sets if w.n > 1]
    t = torch.tensor(np.concatenate([w.t for w in sets]), device="cuda")
    X = torch.tensor(np.concatenate([w.X.reshape(-1) for w in sets]), device="cuda")
    ell, g = hawkes_batch_loglik_grad(ctx, [w.n for w in sets], [w.d for w in sets], t, X,
                                      [w.params for w in sets], precision=prec)
    ell = ell.cpu().numpy()
    g = g.cpu().numpy()
    off = 0
    tl, tg = (1e-12, 1e-12) if prec == "fp64" else (1e-6, 1e-5)
    for i, w in enumerate(sets):
        e_ref, g_ref, _ = oracle.loglik_and_grad(w.t, w.X, w.params)
        gi = g[off:off + w.n * w.d].reshape(w.n, w.d)
        off += w.n * w.d
        assert abs(ell[i] - e_ref) <= tl * abs(e_ref)
        assert np.linalg.norm(gi - g_ref) <= tg * np.linalg.norm(g_ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_hmc_matches_per_set_oracle(ctx, prec):
    import torch

    from paper_2010_02994_gb300 import hawkes_batch_hmc_trajectory

    specs = [(200, 2), (350, 4), (120, 8), (500, 2), (90, 3)]
    sets, p0s, los, his = [], [], [], []
    for i, (n, d) in enumerate(specs):
        w, lo, hi, p0 = hmc_case(300 + i, n, d, True)
        sets.append(w)
        p0s.append(p0)
        los.append(lo)
        his.append(hi)
    eps = [0.01, 0.008, 0.012, 0.01, 0.009]
    refs = [oracle.hmc_trajectory(w.t, w.X, p0, w.params, e, 12, -np.inf, lo, hi)
            for w, p0, lo, hi, e in zip(sets, p0s, los, his, eps)]
    # set 3 gets a log u above its energy gain: it must be rejected
    log_u = [-np.inf, -np.inf, -np.inf, refs[3]["H0"] - refs[3]["H1"] + 1.0, -np.inf]
    cat = lambda arrs: torch.tensor(np.concatenate([a.reshape(-1) for a in arrs]), device="cuda")
    t = torch.tensor(np.concatenate([w.t for w in sets]), device="cuda")
    X = cat([w.X for w in sets])
    H0, H1, acc = hawkes_batch_hmc_trajectory(ctx, [w.n for w in sets], [w.d for w in sets], t, X, cat(p0s),
                                              [w.params for w in sets], eps, 12,
                                              torch.tensor(log_u, dtype=torch.float64, device="cuda"), cat(los),
                                              cat(his), precision=prec)
    H0, H1, acc, X = H0.cpu().numpy(), H1.cpu().numpy(), acc.cpu().numpy(), X.cpu().numpy()
    tol = 1e-10 if prec == "fp64" else 1e-6
    off = 0
    for i, (w, ref) in enumerate(zip(sets, refs)):
        Xi = X[off:off + w.n * w.d].reshape(w.n, w.d)
        off += w.n * w.d
        assert abs(H0[i] - ref["H0"]) <= tol * abs(ref["H0"])
        assert abs(H1[i] - ref["H1"]) <= tol * abs(ref["H1"])
        if i == 3:
            assert acc[i] == 0 and np.array_equal(Xi, w.X)
        else:
            assert acc[i] == 1
            assert np.max(np.abs(Xi - ref["X"])) <= tol * max(1.0, np.max(np.abs(ref["X"])))
