"""Mixed-precision pair terms of the incremental Metropolis-within-Gibbs state
(hawkes_mwg_set_precision(HAWKES_PREC_MIXED)) against the FP64 oracle.

Tolerance, from the arithmetic.  With u = 2^-24, a pair term k = C e^{-A}
evaluated in FP32 has relative error at most about (8 + 12 A) u: the
differences (hi - hi) + (lo - lo) carry a few u, the squared distance and the
exponent a few more, times the exponent A (natural units) because an
absolute error in the exponent becomes a relative error of the term, and
ex2.approx adds up to 4 u.  Compensated sums add u.  So the new rate of an
unmoved event m (lambda*_m = lambda_m + sum_b [k(m <- x*_b) - k(m <- x_b)])
has absolute error at most sum_b (8 + 12 A) k u over its old and new block
terms, and log lambda*_m at most that over lambda*_m; a moved event's new
rate, a sum of positive terms, has relative error sum_m (8 + 12 A) k u /
lambda*_b.  The bound T below adds these up over all events, from pair terms
computed here with numpy; |Delta ell_mixed - Delta ell_oracle| <= T.  Events
that take the FP64 path (tiny rates, near-total cancellation) are held to
the FP64 bound instead (1e-10 relative of their log ratio)."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def terms(tm, Xm, ts, Xs, p):
    """Pair terms k(m <- s) (rows m, columns s) of Eq. (1) and their error
    weights (8 + 12 A) k, for the tolerance only."""
    D = Xm.shape[1]
    dt = tm[:, None] - ts[None, :]
    r2 = ((Xm[:, None, :] - Xs[None, :, :]) ** 2).sum(-1)
    cmu = p["mu0"] / (p["tau_x"] ** D * p["tau_t"] * (2 * np.pi) ** ((D + 1) / 2))
    cxi = p["theta"] * p["omega"] / (p["h"] ** D * (2 * np.pi) ** (D / 2))
    amu = r2 / (2 * p["tau_x"] ** 2) + dt * dt / (2 * p["tau_t"] ** 2)
    axi = p["omega"] * dt + r2 / (2 * p["h"] ** 2)
    mu = np.where(dt != 0, cmu * np.exp(-amu), 0.0)
    xi = np.where(dt > 0, cxi * np.exp(-np.where(dt > 0, axi, 0.0)), 0.0)
    return mu + xi, mu * (8 + 12 * amu) + xi * (8 + 12 * np.where(dt > 0, axi, 0.0))


def bound(w, X, idx, Xn, skip=()):
    """T of the module docstring for moving events idx of X to Xn."""
    X1 = X.copy()
    X1[idx] = Xn
    lam1 = oracle.rates(w.t, X1, w.params)
    moved = np.zeros(w.n, bool)
    moved[idx] = True
    _, wo = terms(w.t, X, w.t[idx], X[idx], w.params)
    _, wn = terms(w.t, X1, w.t[idx], Xn, w.params)
    col = (wo + wn).sum(1) / lam1
    col[moved] = 0.0
    _, wr = terms(w.t[idx], Xn, w.t, X1, w.params)
    wr[np.arange(len(idx)), idx] = 0.0
    row = np.zeros(w.n)
    row[idx] = wr.sum(1) / lam1[idx]
    tot = col + row
    tot[list(skip)] = 0.0
    return U * float(tot.sum())


def mixed_state(w, max_block):
    import torch

    from paper_2010_02994_gb300 import HawkesMwG

    return HawkesMwG(torch.tensor(w.t, device="cuda"), torch.tensor(w.X, device="cuda"), w.params,
                     max_block=max_block, precision="mixed")


@pytest.mark.parametrize("seed,n,d,ties", [(1, 300, 2, 0), (2, 1000, 3, 2), (3, 2500, 1, 0), (4, 700, 8, 0),
                                           (5, 1500, 2, 5)])
def test_mixed_delta_within_bound(seed, n, d, ties):
    w = synth.random_case(seed, n, d, ties=ties, shuffle=True)
    s = mixed_state(w, 64)
    ell0 = oracle.loglik(w.t, w.X, w.params)
    rng = np.random.default_rng(seed)
    for nb, step in ((1, 0.3), (2, 0.3), (7, 0.05), (64, 0.3), (64, 1e-4)):
        idx = rng.choice(w.n, size=nb, replace=False)
        Xn = w.X[idx] + step * rng.standard_normal(size=(nb, w.d))
        X1 = w.X.copy()
        X1[idx] = Xn
        ref = oracle.loglik(w.t, X1, w.params) - ell0
        got = s.delta(idx, Xn).item()
        T = bound(w, w.X, idx, Xn)
        assert abs(got - ref) <= T, (nb, step, got, ref, T)
    s.close()


def test_mixed_steps_follow_oracle():
    """A chain of mixed steps: decisions as the oracle's (where the oracle's
    Delta ell is farther than the bound from the threshold), locations
    identical, rates and ell within the accumulated bound; a refresh restores
    FP64 rates."""
    w = synth.random_case(21, 800, 2, ties=1, shuffle=True)
    s = mixed_state(w, 16)
    rng = np.random.default_rng(5)
    X = w.X.copy()
    ell = oracle.loglik(w.t, X, w.params)
    n_acc, drift = 0, 0.0
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
        T = bound(w, X, idx, Xn)
        if abs(log_u - (ref + log_q)) <= 2 * T:
            log_u -= 1e-3  # keep the decision away from the rounding boundary
        dl, acc = s.step(idx, Xn, log_u, log_q)
        assert abs(dl.item() - ref) <= T
        expect = log_u < ref + log_q
        assert bool(acc.item()) == expect
        if expect:
            X, ell = X1, ell1
            n_acc += 1
            drift += T
    assert 5 <= n_acc <= 35
    Xg, lam, ellg = s.read()
    assert np.array_equal(Xg.cpu().numpy(), X)
    assert abs(ellg.item() - ell) <= drift
    lam_ref = oracle.rates(w.t, X, w.params)
    assert np.max(np.abs(lam.cpu().numpy() - lam_ref) / lam_ref) <= 1e-4
    s.refresh()
    _, lam2, ell2 = s.read()
    assert np.max(np.abs(lam2.cpu().numpy() - lam_ref) / lam_ref) <= 1e-12


def test_mixed_fp64_fallbacks():
    """Hand-placed events that need the FP64 path (the rest of the events
    lie in [0, 3]^2):
    - m0 sits at (15, 15), so its rate (~1e-69) is made of terms below the
      FP32 range; the moved event m1 lands next to it and raises its rate by
      68 orders of magnitude;
    - m2 sits next to m1 at (5, 5), so m1 carries all but 1.4e-4 of m2's rate;
      moving m1 away cancels nearly all of it;
    - m3 moves to (-9, -9), so its new rate (~4e-58) is below the FP32 range.
    Each such log ratio must be exact to FP64 level; the rest is held to T."""
    w = synth.random_case(41, 300, 2, shuffle=True, extent=3.0, t_end=10.0)
    t, X = w.t.copy(), w.X.copy()
    m0, m1, m2, m3 = 0, 1, 2, 3
    X[m0] = (15.0, 15.0)
    t[m0] = 5.0
    X[m1] = (5.0, 5.0)
    t[m1] = 4.0
    X[m2] = (5.05, 5.0)
    t[m2] = 4.2
    w = dataclasses.replace(w, t=t, X=X)
    lam = oracle.rates(w.t, w.X, w.params)
    assert lam[m0] < 1e-30  # below the FP32 range of the terms
    s = mixed_state(w, 4)
    ell0 = oracle.loglik(w.t, w.X, w.params)
    idx = np.array([m1, m3])
    Xn = np.array([[14.9, 15.0], [-9.0, -9.0]])
    X1 = w.X.copy()
    X1[idx] = Xn
    lam1 = oracle.rates(w.t, X1, w.params)
    assert lam1[m0] / lam[m0] > 1e60  # m0's rate grows by many orders
    assert lam1[m2] / lam[m2] < 1e-3  # m2 loses nearly all of its rate
    assert 0.0 < lam1[m3] < 1e-50  # m3 is isolated
    ref = oracle.loglik(w.t, X1, w.params) - ell0
    special = [m0, m2, m3]
    big = float(np.sum(np.abs(np.log(lam1[special]) - np.log(lam[special]))))
    T = bound(w, w.X, idx, Xn, skip=special) + 1e-10 * big
    got = s.delta(idx, Xn).item()
    assert abs(got - ref) <= T, (got, ref, T)
    s.close()


def test_mixed_graph_and_precision_switch():
    """Mixed steps captured in a CUDA graph equal the same steps issued one by
    one; switching the state back to FP64 gives FP64 deltas again."""
    import torch

    w = synth.random_case(22, 600, 3, shuffle=True)
    rng = np.random.default_rng(9)
    t = torch.tensor(w.t, device="cuda")
    Xd = torch.tensor(w.X, device="cuda")
    from paper_2010_02994_gb300 import HawkesMwG

    a = HawkesMwG(t, Xd, w.params, max_block=4, precision="mixed")
    b = HawkesMwG(t, Xd, w.params, max_block=4, precision="mixed")
    dev_steps = []
    for k in range(6):
        idx = rng.choice(w.n, size=4, replace=False)
        dev_steps.append((torch.tensor(idx, device="cuda"),
                          torch.tensor(w.X[idx] + 0.05 * rng.standard_normal(size=(4, w.d)), device="cuda"),
                          torch.tensor(math.log(rng.uniform()), dtype=torch.float64, device="cuda")))
    outs = [(torch.empty((), dtype=torch.float64, device="cuda"), torch.empty((), dtype=torch.int32, device="cuda"))
            for _ in dev_steps]
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
    # back to FP64: the delta of a further move matches the oracle to FP64 level
    a.set_precision("fp64")
    a.refresh()
    Xc = Xa.cpu().numpy()
    idx = np.array([5, 77])
    Xn = Xc[idx] + 0.2
    X1 = Xc.copy()
    X1[idx] = Xn
    ref = oracle.loglik(w.t, X1, w.params) - oracle.loglik(w.t, Xc, w.params)
    lam = oracle.rates(w.t, Xc, w.params)
    sc = float(np.sum(np.abs(np.log(lam))) + oracle.Lambda(w.t, w.params))
    assert abs(a.delta(idx, Xn).item() - ref) <= 1e-11 * sc
    a.close()
    b.close()


def test_mixed_invalid_and_out_of_range():
    import torch

    from paper_2010_02994_gb300 import HawkesError, HawkesMwG

    w = synth.random_case(23, 200, 2, shuffle=True)
    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda")
    # a scale outside [2^-100, 2^100]: mixed precision is refused
    p = dict(w.params, tau_x=1e-40)
    s = HawkesMwG(t, X, p, max_block=4)
    with pytest.raises(HawkesError, match="INVALID_ARG"):
        s.set_precision("mixed")
    s.close()
    # a proposal coordinate of 2^100 or more is a bad proposal in mixed precision
    s = HawkesMwG(t, X, w.params, max_block=4, precision="mixed")
    out = s.delta([3], np.array([[2.0 ** 101, 0.0]]), check=False)
    torch.cuda.synchronize()
    assert math.isnan(out.item())
    with pytest.raises(HawkesError, match="INVALID_DATA"):
        s.sync_status()
    # data of 2^100 or more keeps the state on FP64: the delta is FP64-exact.
    # Event 10 is then isolated (rate 0 before and after, contributing 0), so
    # the reference sums the log ratios of the other rates.
    X2 = w.X.copy()
    X2[10] = (2.0 ** 101, 0.0)
    s2 = HawkesMwG(t, torch.tensor(X2, device="cuda"), w.params, max_block=4, precision="mixed")
    idx = np.array([4])
    Xn = X2[idx] + 0.1
    X3 = X2.copy()
    X3[idx] = Xn
    lam2, lam3 = oracle.rates(w.t, X2, w.params), oracle.rates(w.t, X3, w.params)
    live = lam2 > 0
    assert not live[10] and lam3[10] == 0.0
    ref = float(np.sum(np.log(lam3[live]) - np.log(lam2[live])))
    assert abs(s2.delta(idx, Xn).item() - ref) <= 1e-11 * float(np.sum(np.abs(np.log(lam2[live]))))
    s.close()
    s2.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_largest_block_in_eight_dimensions(prec):
    """The largest block (256 events, D = 8: the most staged shared memory)
    in both precisions, against the oracle."""
    import torch

    from paper_2010_02994_gb300 import HawkesMwG

    w = synth.random_case(51, 900, 8, ties=2, shuffle=True)
    s = HawkesMwG(torch.tensor(w.t, device="cuda"), torch.tensor(w.X, device="cuda"), w.params, max_block=256,
                  precision=prec)
    rng = np.random.default_rng(51)
    idx = rng.choice(w.n, size=256, replace=False)
    Xn = w.X[idx] + 0.2 * rng.standard_normal(size=(256, w.d))
    X1 = w.X.copy()
    X1[idx] = Xn
    ref = oracle.loglik(w.t, X1, w.params) - oracle.loglik(w.t, w.X, w.params)
    got = s.delta(idx, Xn).item()
    if prec == "fp64":
        lam = oracle.rates(w.t, w.X, w.params)
        sc = float(np.sum(np.abs(np.log(lam))) + oracle.Lambda(w.t, w.params))
        assert abs(got - ref) <= 1e-11 * sc
    else:
        assert abs(got - ref) <= bound(w, w.X, idx, Xn)
    s.close()


def test_mixed_signed_zero_times():
    """In the mixed precision the tie indicators compare time bit patterns with
    the sign cleared, so +0 and -0 are tied as in the FP64 comparison."""
    w = synth.random_case(62, 300, 2, shuffle=True)
    t = w.t.copy()
    t[[3, 50]] = 0.0
    t[[7, 120]] = -0.0
    w = dataclasses.replace(w, t=t)
    s = mixed_state(w, 4)
    ell0 = oracle.loglik(w.t, w.X, w.params)
    idx = np.array([3, 7, 50])
    Xn = w.X[idx] + 0.05
    X1 = w.X.copy()
    X1[idx] = Xn
    ref = oracle.loglik(w.t, X1, w.params) - ell0
    assert abs(s.delta(idx, Xn).item() - ref) <= bound(w, w.X, idx, Xn)
    s.close()
