"""BMDS likelihood of Eq. (4) and its gradients on the GPU against the FP64
oracle (element by element), plus the invariances and error paths.

Tolerances: FP64 GPU 1e-12 relative; mixed precision 1e-6 relative on ell and
on d ell / d sigma2 and 1e-5 relative L2 on the location gradient.  The
scalars are conditioned by the magnitude of the sums they come from: ell by
|N (1 - N) / 4 log sigma2| + sum_{n>n'} |r_nn'| (bounded here by |ell| plus
twice the log-normaliser), d ell / d sigma2 by |N (1 - N) / (4 sigma2)| +
|result|, since the two parts cancel near the maximum."""
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

    c = HawkesContext(device=0, max_n=10_000, max_d=8)
    yield c
    c.close()


def gpu_bmds(ctx, Y, X, sigma2, prec, y32=False):
    import torch

    from paper_2010_02994_gb300 import hawkes_bmds_loglik_grad

    Yd = torch.tensor(Y, device="cuda")
    if y32:
        Yd = Yd.float()
    Xd = torch.tensor(X, device="cuda")
    ell, g, gs = hawkes_bmds_loglik_grad(ctx, Yd, Xd, sigma2, precision=prec)
    return ell.item(), g.cpu().numpy(), gs.item()


def assert_close(n, sigma2, got, ref, prec):
    tol_s, tol_g = TOL[prec]
    ell, g, gs = got
    ell_r, g_r, gs_r = ref
    c = n * (1 - n) / 4.0
    ell_scale = abs(ell_r) + 2 * abs(c * math.log(sigma2)) + 1e-300
    assert abs(ell - ell_r) <= tol_s * ell_scale, (ell, ell_r)
    gs_scale = abs(c / sigma2) + abs(gs_r) + 1e-300
    assert abs(gs - gs_r) <= tol_s * gs_scale, (gs, gs_r)
    gn = np.linalg.norm(g_r)
    if gn > 0:
        assert np.linalg.norm(g - g_r) <= tol_g * gn, np.linalg.norm(g - g_r) / gn
    else:
        assert np.all(g == 0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("seed,n,d", [(1, 2, 2), (2, 3, 1), (3, 31, 2), (4, 64, 3), (5, 65, 6), (6, 129, 8),
                                      (7, 200, 4), (8, 517, 5), (9, 1000, 7), (10, 333, 1)])
def test_bmds_matches_oracle(ctx, prec, seed, n, d):
    w = synth.bmds_random(seed, n, d)
    ref = oracle.bmds(w.Y, w.X, w.sigma2)
    got = gpu_bmds(ctx, w.Y, w.X, w.sigma2, prec)
    assert_close(n, w.sigma2, got, ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bmds_influenza_like(ctx, prec):
    """N = 4,733 cases, D = 6, the configuration of Section 4.3 (block-structured
    Y, zero within a country)."""
    w = synth.make_bmds()
    ref = oracle.bmds(w.Y, w.X, w.sigma2)
    got = gpu_bmds(ctx, w.Y, w.X, w.sigma2, prec)
    assert_close(w.X.shape[0], w.sigma2, got, ref, prec)


def test_bmds_large_tiles(ctx):
    """n >= 8192 takes the 128-row tiles; ragged last tile."""
    w = synth.make_bmds(seed=11, n=8300, d=2, n_countries=60)
    ref = oracle.bmds(w.Y, w.X, w.sigma2)
    for prec in ("mixed", "fp64"):
        got = gpu_bmds(ctx, w.Y, w.X, w.sigma2, prec)
        assert_close(w.X.shape[0], w.sigma2, got, ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bmds_single_event(ctx, prec):
    ell, g, gs = gpu_bmds(ctx, np.zeros((1, 1)), np.array([[0.3, -1.0]]), 0.5, prec)
    assert ell == 0.0 and gs == 0.0 and np.all(g == 0.0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bmds_reads_only_below_diagonal(ctx, prec):
    w = synth.bmds_random(12, 150, 3)
    Yg = w.Y.copy()
    Yg[np.triu_indices(150)] = np.nan  # the diagonal and above hold garbage
    a = gpu_bmds(ctx, w.Y, w.X, w.sigma2, prec)
    b = gpu_bmds(ctx, Yg, w.X, w.sigma2, prec)
    assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bmds_coincident_points(ctx, prec):
    w = synth.bmds_random(13, 90, 2)
    w.X[7] = w.X[3]
    w.X[50] = w.X[3]
    ref = oracle.bmds(w.Y, w.X, w.sigma2)
    got = gpu_bmds(ctx, w.Y, w.X, w.sigma2, prec)
    assert np.isfinite(got[0]) and np.all(np.isfinite(got[1]))
    assert_close(90, w.sigma2, got, ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bmds_deterministic_and_permutation(ctx, prec):
    w = synth.bmds_random(14, 700, 4)
    a = gpu_bmds(ctx, w.Y, w.X, w.sigma2, prec)
    b = gpu_bmds(ctx, w.Y, w.X, w.sigma2, prec)
    assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1])
    perm = np.random.default_rng(0).permutation(700)
    c = gpu_bmds(ctx, w.Y[perm][:, perm], w.X[perm], w.sigma2, prec)
    assert_close(700, w.sigma2, (c[0], c[1], c[2]), (a[0], a[1][perm], a[2]), prec)


def test_bmds_invalid_data_and_args(ctx):
    import torch

    from paper_2010_02994_gb300 import HawkesError, hawkes_bmds_loglik_grad

    w = synth.bmds_random(15, 100, 2)
    for bad in ("neg_y", "nan_x", "inf_y"):
        Y, X = w.Y.copy(), w.X.copy()
        if bad == "neg_y":
            Y[40, 3] = -0.5
        elif bad == "inf_y":
            Y[99, 98] = np.inf
        else:
            X[17, 1] = np.nan
        Yd, Xd = torch.tensor(Y, device="cuda"), torch.tensor(X, device="cuda")
        ell, g, gs = hawkes_bmds_loglik_grad(ctx, Yd, Xd, w.sigma2, precision="mixed", check=False)
        torch.cuda.synchronize()
        assert math.isnan(ell.item()) and math.isnan(gs.item()) and torch.isnan(g).all()
        with pytest.raises(HawkesError, match="INVALID_DATA"):
            ctx.sync_status()
    Yd, Xd = torch.tensor(w.Y, device="cuda"), torch.tensor(w.X, device="cuda")
    for s2 in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(HawkesError, match="INVALID_ARG"):
            hawkes_bmds_loglik_grad(ctx, Yd, Xd, s2)
    # a valid call afterwards is unaffected
    ell, g, gs = hawkes_bmds_loglik_grad(ctx, Yd, Xd, w.sigma2, precision="fp64")
    assert abs(ell.item() - oracle.bmds(w.Y, w.X, w.sigma2)[0]) <= 1e-12 * abs(ell.item())


def test_bmds_value_only(ctx):
    import torch

    from paper_2010_02994_gb300 import hawkes_bmds_loglik_grad

    w = synth.bmds_random(16, 300, 3)
    Yd, Xd = torch.tensor(w.Y, device="cuda"), torch.tensor(w.X, device="cuda")
    ell, g, gs = hawkes_bmds_loglik_grad(ctx, Yd, Xd, w.sigma2, precision="fp64", grad=False)
    assert g is None and gs is None
    assert abs(ell.item() - oracle.bmds(w.Y, w.X, w.sigma2)[0]) <= 1e-12 * abs(ell.item())


def test_bmds_float_distances(ctx):
    """Y given as float32: the mixed precision gives bit-identical results to
    FP64 Y (it rounds FP64 distances to nearest-even FP32 as it reads them);
    FP64 precision widens float distances exactly, so it matches the oracle
    run on the float-rounded matrix."""
    w = synth.make_bmds(seed=17, n=1500, d=6)
    rng = np.random.default_rng(3)
    Y = w.Y.copy()
    # entries exactly halfway between two floats, and a spread of magnitudes
    idx = rng.integers(0, 1500, size=(2000, 2))
    f = np.float32(rng.uniform(0.5, 20.0, size=2000))
    half = (np.nextafter(f, np.float32(np.inf)).astype(np.float64) - f.astype(np.float64)) / 2
    Y[idx[:, 0], idx[:, 1]] = f.astype(np.float64) + half
    Y[idx[:, 1], idx[:, 0]] = Y[idx[:, 0], idx[:, 1]]
    Y[5:40, 0:5] *= 1e6
    Y[50:90, 10:20] *= 1e-5
    a = gpu_bmds(ctx, Y, w.X, w.sigma2, "mixed")
    b = gpu_bmds(ctx, Y, w.X, w.sigma2, "mixed", y32=True)
    assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1])
    Yr = Y.astype(np.float32).astype(np.float64)
    ref = oracle.bmds(Yr, w.X, w.sigma2)
    got = gpu_bmds(ctx, Y, w.X, w.sigma2, "fp64", y32=True)
    assert_close(1500, w.sigma2, got, ref, "fp64")
    assert_close(1500, w.sigma2, b, ref, "mixed")
