"""Incremental Metropolis-within-Gibbs state (hawkes_mwg_*) against the FP64
oracle: Delta ell of a block move equals ell(X*) - ell(X) from two full oracle
evaluations, the cached rates equal the oracle's, and a sequence of steps
takes the decisions the oracle's deltas imply.

Tolerance: everything is FP64 on both sides; Delta ell is compared with an
absolute bound 1e-11 x (sum |log lambda_n| + sum Lambda_n), the magnitude of
the two full log-likelihoods whose difference the oracle forms."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def scale(w):
    lam = oracle.rates(w.t, w.X, w.params)
    return float(np.sum(np.abs(np.log(lam))) + oracle.Lambda(w.t, w.params))


def random_block(rng, w, nb, step=0.3):
    idx = rng.choice(w.n, size=nb, replace=False)
    Xn = w.X[idx] + step * rng.standard_normal(size=(nb, w.d))
    return idx, Xn


@pytest.mark.parametrize("seed,n,d,ties", [(1, 300, 2, 0), (2, 1000, 3, 2), (3, 2500, 1, 0), (4, 700, 8, 0),
                                           (5, 1500, 2, 5)])
def test_mwg_rates_and_delta_match_oracle(seed, n, d, ties):
    import torch

    from paper_2010_02994_gb300 import HawkesMwG

    w = synth.random_case(seed, n, d, ties=ties, shuffle=True)
    s = HawkesMwG(torch.tensor(w.t, device="cuda"), torch.tensor(w.X, device="cuda"), w.params, max_block=64)
    X, lam, ell = s.read()
    lam_ref = oracle.rates(w.t, w.X, w.params)
    assert np.max(np.abs(lam.cpu().numpy() - lam_ref) / lam_ref) <= 1e-12
    ell0 = oracle.loglik(w.t, w.X, w.params)
    sc = scale(w)
    assert abs(ell.item() - ell0) <= 1e-12 * sc
    rng = np.random.default_rng(seed)
    for nb in (1, 2, 7, 64):
        idx, Xn = random_block(rng, w, nb)
        X1 = w.X.copy()
        X1[idx] = Xn
        ref = oracle.loglik(w.t, X1, w.params) - ell0
        got = s.delta(idx, Xn).item()
        assert abs(got - ref) <= 1e-11 * sc, (nb, got, ref)
    s.close()


def test_mwg_steps_follow_oracle_decisions():
    import torch

    from paper_2010_02994_gb300 import HawkesMwG

    w = synth.random_case(21, 800, 2, ties=1, shuffle=True)
    s = HawkesMwG(torch.tensor(w.t, device="cuda"), torch.tensor(w.X, device="cuda"), w.params, max_block=16)
    rng = np.random.default_rng(5)
    X = w.X.copy()
    ell = oracle.loglik(w.t, X, w.params)
    sc = scale(w)
    n_acc = 0
    for k in range(40):
        nb = int(rng.integers(1, 17))
        idx = rng.choice(w.n, size=nb, replace=False)
        Xn = X[idx] + 0.3 * rng.standard_normal(size=(nb, w.d))
        log_q = float(rng.normal(scale=0.1))
        log_u = math.log(rng.uniform())
        X1 = X.copy()
        X1[idx] = Xn
        ell1 = oracle.loglik(w.t, X1, w.params)
        ref = ell1 - ell
        if abs(log_u - (ref + log_q)) < 1e-6:
            log_u -= 1e-3  # keep the decision away from the rounding boundary
        dl, acc = s.step(idx, Xn, log_u, log_q)
        assert abs(dl.item() - ref) <= 1e-11 * sc
        expect = log_u < ref + log_q
        assert bool(acc.item()) == expect
        if expect:
            X, ell = X1, ell1
            n_acc += 1
    assert 5 <= n_acc <= 35  # both outcomes occur (14 of 40 accepted for this seed)
    Xg, lam, ellg = s.read()
    assert np.array_equal(Xg.cpu().numpy(), X)
    lam_ref = oracle.rates(w.t, X, w.params)
    assert np.max(np.abs(lam.cpu().numpy() - lam_ref) / lam_ref) <= 1e-11
    assert abs(ellg.item() - ell) <= 1e-11 * sc
    s.refresh()
    _, lam2, ell2 = s.read()
    assert np.max(np.abs(lam2.cpu().numpy() - lam_ref) / lam_ref) <= 1e-12
    assert abs(ell2.item() - ell) <= 1e-12 * sc
    s.close()


def test_mwg_graph_captured_steps():
    """A run of steps captured once in a CUDA graph and replayed gives the
    same state as the same steps issued one by one."""
    import torch

    from paper_2010_02994_gb300 import HawkesMwG

    w = synth.random_case(22, 600, 3, shuffle=True)
    rng = np.random.default_rng(9)
    steps = []
    for k in range(6):
        idx = rng.choice(w.n, size=4, replace=False)
        steps.append((idx, 0.05 * rng.standard_normal(size=(4, w.d)), math.log(rng.uniform())))
    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda")
    a = HawkesMwG(t, X, w.params, max_block=4)
    b = HawkesMwG(t, X, w.params, max_block=4)
    dev_steps = []
    for idx, dx, lu in steps:
        dev_steps.append((torch.tensor(idx, device="cuda"), torch.tensor(w.X[idx] + dx, device="cuda"),
                          torch.tensor(lu, dtype=torch.float64, device="cuda")))
    outs = [(torch.empty((), dtype=torch.float64, device="cuda"), torch.empty((), dtype=torch.int32, device="cuda"))
            for _ in steps]
    for (i, xn, lu), o in zip(dev_steps, outs):
        a.step(i, xn, lu, out=o, check=False)
    a.sync_status()
    Xa, la, ea = a.read()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            for (i, xn, lu), o in zip(dev_steps, outs):
                b.step(i, xn, lu, out=o, check=False)
    g.replay()
    torch.cuda.synchronize()
    b.sync_status()
    Xb, lb, eb = b.read()
    torch.cuda.synchronize()
    assert torch.equal(Xa, Xb) and torch.equal(la, lb) and ea.item() == eb.item()
    a.close()
    b.close()


def test_mwg_edge_cases():
    import torch

    from paper_2010_02994_gb300 import HawkesError, HawkesMwG

    w = synth.random_case(23, 200, 2, shuffle=True)
    s = HawkesMwG(torch.tensor(w.t, device="cuda"), torch.tensor(w.X, device="cuda"), w.params, max_block=8)
    # empty block: no change, always accepted for log u < log q-ratio
    assert s.delta([], np.zeros((0, 2))).item() == 0.0
    # moving to the same place: zero up to rounding
    idx = np.array([3, 150])
    assert abs(s.delta(idx, w.X[idx]).item()) <= 1e-12 * scale(w)
    # repeated index, index out of range, non-finite proposal: NaN and an error
    for bad_idx, bad_x in (([5, 5], w.X[[5, 5]]), ([0, 200], w.X[[0, 1]]), ([7], np.array([[np.nan, 0.0]]))):
        out = s.delta(bad_idx, bad_x, check=False)
        torch.cuda.synchronize()
        assert math.isnan(out.item())
        with pytest.raises(HawkesError, match="INVALID_DATA"):
            s.sync_status()
    # a rejected step leaves the state unchanged
    X0, lam0, ell0 = s.read()
    dl, acc = s.step([3], w.X[[3]] + 5.0, log_u=1e9)
    assert acc.item() == 0
    X1, lam1, ell1 = s.read()
    assert torch.equal(X0, X1) and torch.equal(lam0, lam1) and ell0.item() == ell1.item()
    with pytest.raises(HawkesError, match="INVALID_ARG"):
        s.delta(np.arange(9), np.zeros((9, 2)))
    s.close()


def circle_case(seed, n):
    """Wildfire-like circle priors: centres at the observed points, radii from
    fire areas, latent points inside their circles."""
    rng = np.random.default_rng(seed)
    w = synth.random_case(seed, n, 2, shuffle=True)
    radii = rng.choice([0.05, 0.5, 5.0], size=n, p=[0.5, 0.3, 0.2])
    ang = rng.uniform(0, 2 * np.pi, size=n)
    rr = radii * np.sqrt(rng.uniform(size=n)) * 0.999
    centers = w.X - np.stack([rr * np.cos(ang), rr * np.sin(ang)], axis=1)
    return w, centers, radii


def test_mwg_circle_proposals_match_oracle():
    import torch

    from paper_2010_02994_gb300 import HawkesMwG

    w, centers, radii = circle_case(31, 500)
    s = HawkesMwG(torch.tensor(w.t, device="cuda"), torch.tensor(w.X, device="cuda"), w.params, max_block=64)
    rng = np.random.default_rng(2)
    for nb, eps, tries in ((1, 0.3, 4), (17, 1.5, 3), (64, 0.8, 8), (64, 3.0, 1)):
        idx = rng.choice(w.n, size=nb, replace=False)
        u = rng.uniform(size=(nb, tries, 2))
        Xn, lq = s.propose_circle(idx, centers, radii, eps, tries, u)
        Xr, lqr = oracle.circle_proposals(w.X[idx], centers[idx], radii[idx], eps, tries, u)
        Xn = Xn.cpu().numpy()
        assert np.max(np.abs(Xn - Xr)) <= 1e-12 * (1 + np.max(np.abs(Xr)))
        assert abs(lq.item() - lqr) <= 1e-10 * (1 + abs(lqr)), (lq.item(), lqr)
        inside = np.hypot(*(Xn - centers[idx]).T) < radii[idx]
        assert inside.all()
    s.close()


def test_mwg_box_proposals_match_oracle():
    import torch

    from paper_2010_02994_gb300 import HawkesMwG

    w = synth.make_c3()  # wildfire-like boxes of sides 0.1, 1, 10 km
    s = HawkesMwG(torch.tensor(w.t, device="cuda"), torch.tensor(w.X, device="cuda"), w.params, max_block=128)
    rng = np.random.default_rng(4)
    for nb, sd in ((1, 0.05), (33, 0.5), (128, 2.0)):
        idx = rng.choice(w.n, size=nb, replace=False)
        u = rng.uniform(size=(nb, w.d))
        Xn, lq = s.propose_box(idx, w.box_lo, w.box_hi, sd, u)
        Xr, lqr = oracle.box_proposals(w.X[idx], w.box_lo[idx], w.box_hi[idx], sd, u)
        Xn = Xn.cpu().numpy()
        assert np.max(np.abs(Xn - Xr)) <= 1e-9 * (1 + np.max(np.abs(Xr)))
        assert abs(lq.item() - lqr) <= 1e-8 * (1 + abs(lqr)), (lq.item(), lqr)
        assert np.all((Xn >= w.box_lo[idx]) & (Xn <= w.box_hi[idx]))
    s.close()


def test_mwg_circle_chain_on_device():
    """Propose on the device, step on the device: the chain's decisions match
    the oracle's deltas and ratios, and every location stays in its circle."""
    import torch

    from paper_2010_02994_gb300 import HawkesMwG

    w, centers, radii = circle_case(32, 400)
    s = HawkesMwG(torch.tensor(w.t, device="cuda"), torch.tensor(w.X, device="cuda"), w.params, max_block=8)
    rng = np.random.default_rng(6)
    X = w.X.copy()
    ell = oracle.loglik(w.t, X, w.params)
    n_acc = 0
    for k in range(25):
        idx = rng.choice(w.n, size=8, replace=False)
        u = rng.uniform(size=(8, 4, 2))
        Xn, lq = s.propose_circle(idx, centers, radii, 0.5, 4, u)
        Xr, lqr = oracle.circle_proposals(X[idx], centers[idx], radii[idx], 0.5, 4, u)
        X1 = X.copy()
        X1[idx] = Xr
        ell1 = oracle.loglik(w.t, X1, w.params)
        log_u = math.log(rng.uniform())
        if abs(log_u - (ell1 - ell + lqr)) < 1e-6:
            log_u -= 1e-3
        dl, acc = s.step(torch.as_tensor(idx, device="cuda"), Xn, log_u, lq)
        expect = log_u < ell1 - ell + lqr
        assert bool(acc.item()) == expect
        if expect:
            X, ell = X1, ell1
            n_acc += 1
    Xg, _, _ = s.read()
    Xg = Xg.cpu().numpy()
    assert np.max(np.abs(Xg - X)) <= 1e-12 * (1 + np.max(np.abs(X)))
    assert np.all(np.hypot(*(Xg - centers).T) < radii)
    assert 0 < n_acc < 25
    s.close()
