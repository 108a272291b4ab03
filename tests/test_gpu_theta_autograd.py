"""Parameter gradient and the autograd wrapper against the FP64 oracle and
against finite differences.

The parameter gradient is compared per component relative to the magnitude
of the terms that component is summed from (oracle.grad_params_scaled): near
the data-generating parameters each score is a sum of N terms of either sign
that cancels far below them, and a rounding error of the row sums is relative
to the terms, not to the sum.  Tolerances: 1e-12 (FP64) and 1e-6 (mixed)."""
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


def gpu_all(ctx, w, prec):
    import torch

    from paper_2010_02994_gb300 import hawkes_loglik_grad_locations

    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda")
    ell, g, gp = hawkes_loglik_grad_locations(ctx, t, X, w.params, precision=prec, grad_params=True)
    return ell.item(), g.cpu().numpy(), gp.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("seed,n,d,ties", [(1, 300, 2, 0), (2, 900, 3, 1), (3, 2000, 1, 0), (4, 700, 8, 0),
                                           (5, 1500, 2, 2)])
def test_parameter_gradient_matches_oracle(ctx, prec, seed, n, d, ties):
    w = synth.random_case(seed, n, d, ties=ties, shuffle=True)
    ell_ref, g_ref, lam = oracle.loglik_and_grad(w.t, w.X, w.params)
    gp_ref, gp_scale = oracle.grad_params_scaled(w.t, w.X, w.params, lam)
    ell, g, gp = gpu_all(ctx, w, prec)
    err = np.max(np.abs(gp - gp_ref) / gp_scale)
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert err <= tol, (gp, gp_ref, err)
    scale = float(np.sum(np.abs(np.log(lam))) + oracle.Lambda(w.t, w.params))
    assert abs(ell - ell_ref) <= (1e-12 if prec == "fp64" else 1e-6) * scale


def test_parameter_gradient_wildfire_like(ctx):
    w = synth.make_c3()
    ell_ref, g_ref, lam = oracle.loglik_and_grad(w.t, w.X, w.params)
    gp_ref, gp_scale = oracle.grad_params_scaled(w.t, w.X, w.params, lam)
    for prec, tol in (("fp64", 1e-12), ("mixed", 1e-6)):
        _, _, gp = gpu_all(ctx, w, prec)
        assert np.max(np.abs(gp - gp_ref) / gp_scale) <= tol


def test_autograd_gradcheck_fp64(ctx):
    import torch

    from paper_2010_02994_gb300 import hawkes_loglik_autograd

    w = synth.random_case(9, 25, 2, shuffle=True)
    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda", requires_grad=True)
    th = torch.tensor(w.theta_vector(), device="cuda", requires_grad=True)
    f = lambda X_, th_: hawkes_loglik_autograd(ctx, t, X_, th_, "fp64")
    assert torch.autograd.gradcheck(f, (X, th), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_autograd_backward_matches_oracle(ctx):
    import torch

    from paper_2010_02994_gb300 import hawkes_loglik_autograd

    w = synth.make_c3()
    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda", requires_grad=True)
    th = torch.tensor(w.theta_vector(), device="cuda", requires_grad=True)
    ll = hawkes_loglik_autograd(ctx, t, X, th, "mixed")
    (2.0 * ll).backward()
    ell_ref, g_ref, lam = oracle.loglik_and_grad(w.t, w.X, w.params)
    gp_ref, gp_scale = oracle.grad_params_scaled(w.t, w.X, w.params, lam)
    gx = X.grad.cpu().numpy()
    assert np.linalg.norm(gx - 2 * g_ref) <= 1e-5 * np.linalg.norm(2 * g_ref)
    assert np.max(np.abs(th.grad.cpu().numpy() - 2 * gp_ref) / (2 * gp_scale)) <= 1e-6


def test_location_gradient_against_finite_differences_of_gpu_loglik(ctx):
    """The wildfire-shaped workload's location gradient against central
    differences of the GPU FP64 log-likelihood on a few coordinates."""
    import torch

    from paper_2010_02994_gb300 import hawkes_loglik

    w = synth.make_c3()
    _, g, _ = gpu_all(ctx, w, "fp64")
    t = torch.tensor(w.t, device="cuda")
    rng = np.random.default_rng(0)
    for i in rng.choice(w.n, size=6, replace=False):
        for k in range(w.d):
            h = 1e-4 * w.params["h"]
            vals = []
            for sgn in (1, -1):
                X = w.X.copy()
                X[i, k] += sgn * h
                vals.append(hawkes_loglik(ctx, t, torch.tensor(X, device="cuda"), w.params, precision="fp64").item())
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - g[i, k]) <= 1e-5 * max(1.0, abs(g[i, k]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_self_excitation_probability(ctx, prec):
    import torch

    from paper_2010_02994_gb300 import hawkes_self_excitation_prob

    for w in (synth.random_case(71, 1200, 2, ties=2, shuffle=True), synth.make_c3()):
        lam, mu, xi = oracle.rates(w.t, w.X, w.params, parts=True)
        ref = xi / lam
        got = hawkes_self_excitation_prob(ctx, torch.tensor(w.t, device="cuda"), torch.tensor(w.X, device="cuda"),
                                          w.params, precision=prec).cpu().numpy()
        tol = 1e-12 if prec == "fp64" else 1e-5
        assert np.max(np.abs(got - ref)) <= tol
        assert np.all((got >= 0) & (got <= 1))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("d,n", [(1, 700), (3, 650), (5, 520), (8, 600)])
def test_self_excitation_probability_every_dimension(ctx, d, n, prec):
    """The rate pass that keeps the self-excitation sums apart (mixed) or the
    FP64 rate pass with the parameter-gradient sums, in the dimensions the
    D = 2 cases above do not reach (ragged last block, tied times)."""
    import torch

    from paper_2010_02994_gb300 import hawkes_self_excitation_prob

    w = synth.random_case(80 + d, n, d, ties=2, shuffle=True)
    lam, mu, xi = oracle.rates(w.t, w.X, w.params, parts=True)
    got = hawkes_self_excitation_prob(ctx, torch.tensor(w.t, device="cuda"), torch.tensor(w.X, device="cuda"),
                                      w.params, precision=prec).cpu().numpy()
    assert np.max(np.abs(got - xi / lam)) <= (1e-5 if prec == "mixed" else 1e-12)
