"""The paper-shaped workloads at their full sizes against the FP64 oracle.

  * the 64-set batch (N log-uniform in [500, 20,000], D in {2, 4, 8}, 317,933
    events): every set's ell and location gradient in both precisions, and a
    20-step HMC proposal per set (Section 3) replayed by the oracle for the
    smallest sets of each dimension;
  * the gunfire-like HMC trajectory (N = 10,000, D = 2, 100 m boxes, 20
    leapfrog steps): the mixed path against the FP64 GPU path at rel <= 1e-6,
    and the FP64 GPU path against the oracle's replay of the same trajectory;
  * the autotuner on one set of the batch: the shape it keeps is stored in
    the context, the options it tried are put back, and a call with the
    stored shape is bit-identical to one with the shape set explicitly.

The N = 100,000 parameter gradient is in test_gpu_parity.py beside the other
N = 100,000 comparisons (it shares their all-row oracle rates).

Tolerances: mixed ell relative 1e-6 and gradient relative L2 1e-5, FP64 1e-12
(relative to |ell|: these workloads' ell is far from zero).  HMC: the FP64
GPU path replays the oracle to 1e-10 (twenty leapfrog steps of FP64 rounding
in a different summation order); mixed to 1e-6.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = {"fp64": (1e-12, 1e-12), "mixed": (1e-6, 1e-5)}


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def c4():
    sets = synth.make_c4()
    refs = [oracle.loglik_and_grad(w.t, w.X, w.params)[:2] for w in sets]
    return sets, refs


def _cat(arrs, dev="cuda"):
    import torch

    return torch.tensor(np.concatenate([np.asarray(a).reshape(-1) for a in arrs]), device=dev)


@pytest.mark.parametrize("prec,one_launch", [("mixed", 0), ("fp64", 0), ("mixed", 1)])
def test_batch_of_64_sets_matches_per_set_oracle(c4, prec, one_launch):
    """Per-dimension launches, and (one_launch) every dimension's pair blocks
    in one persistent launch per pass."""
    from paper_2010_02994_gb300 import HawkesContext, hawkes_batch_loglik_grad

    sets, refs = c4
    sizes = [w.n for w in sets]
    dims = [w.d for w in sets]
    ctx = HawkesContext(device=0, max_n=sum(sizes), max_d=8)
    ctx.set_option("one_launch", one_launch)
    ell, g = hawkes_batch_loglik_grad(ctx, sizes, dims, _cat([w.t for w in sets]), _cat([w.X for w in sets]),
                                      [w.params for w in sets], precision=prec)
    ell = ell.cpu().numpy()
    g = g.cpu().numpy()
    ctx.close()
    tl, tg = TOL[prec]
    off = 0
    worst_l = worst_g = 0.0
    for i, (w, (e_ref, g_ref)) in enumerate(zip(sets, refs)):
        gi = g[off:off + w.n * w.d].reshape(w.n, w.d)
        off += w.n * w.d
        el = abs(ell[i] - e_ref) / abs(e_ref)
        eg = rel_l2(gi, g_ref)
        worst_l, worst_g = max(worst_l, el), max(worst_g, eg)
        assert el <= tl, f"set {i} (n={w.n}, d={w.d}) {prec}: ell rel {el:.2e}"
        assert eg <= tg, f"set {i} (n={w.n}, d={w.d}) {prec}: grad rel-L2 {eg:.2e}"
    print(f"c4 {prec} one_launch={one_launch}: worst ell rel {worst_l:.2e}, worst grad rel-L2 {worst_g:.2e}")


@pytest.mark.parametrize("prec,one_launch", [("mixed", 0), ("fp64", 0), ("mixed", 1)])
def test_batched_hmc_over_64_sets_replays_oracle(c4, prec, one_launch):
    """One 20-step proposal per set for all 64 sets in one call; the two
    smallest sets of each dimension are replayed by the oracle, and one of
    them gets a log u above its energy gain, so it must be rejected."""
    import torch

    from paper_2010_02994_gb300 import HawkesContext, hawkes_batch_hmc_trajectory

    sets, _ = c4
    sizes = [w.n for w in sets]
    dims = [w.d for w in sets]
    rng = np.random.default_rng(23)
    p0s = [rng.standard_normal(size=w.X.shape) for w in sets]
    eps = [1e-3] * len(sets)
    L = 20
    check = []
    for d in (2, 4, 8):
        idx = sorted((i for i in range(len(sets)) if dims[i] == d), key=lambda i: sizes[i])[:2]
        check.extend(idx)
    refs = {i: oracle.hmc_trajectory(sets[i].t, sets[i].X, p0s[i], sets[i].params, eps[i], L, -np.inf)
            for i in check}
    reject = check[0]
    log_u = [-np.inf] * len(sets)
    log_u[reject] = refs[reject]["H0"] - refs[reject]["H1"] + 1.0
    ctx = HawkesContext(device=0, max_n=sum(sizes), max_d=8)
    ctx.set_option("one_launch", one_launch)
    X = _cat([w.X for w in sets])
    H0, H1, acc = hawkes_batch_hmc_trajectory(ctx, sizes, dims, _cat([w.t for w in sets]), X, _cat(p0s),
                                              [w.params for w in sets], eps, L,
                                              torch.tensor(log_u, dtype=torch.float64, device="cuda"),
                                              precision=prec)
    H0, H1, acc, X = H0.cpu().numpy(), H1.cpu().numpy(), acc.cpu().numpy(), X.cpu().numpy()
    ctx.close()
    tol = 1e-10 if prec == "fp64" else 1e-6
    offs = np.concatenate([[0], np.cumsum([w.n * w.d for w in sets])])
    for i in check:
        w, ref = sets[i], refs[i]
        Xi = X[offs[i]:offs[i + 1]].reshape(w.n, w.d)
        assert abs(H0[i] - ref["H0"]) <= tol * abs(ref["H0"]), (i, H0[i], ref["H0"])
        assert abs(H1[i] - ref["H1"]) <= tol * abs(ref["H1"]), (i, H1[i], ref["H1"])
        if i == reject:
            assert acc[i] == 0 and np.array_equal(Xi, w.X)
        else:
            assert acc[i] == 1
            assert np.max(np.abs(Xi - ref["X"])) <= tol * max(1.0, np.max(np.abs(ref["X"])))
    others = [i for i in range(len(sets)) if i != reject]
    assert np.all(np.isfinite(H0[others])) and np.all(np.isfinite(H1[others]))
    assert np.all(acc[others] == 1)


@pytest.fixture(scope="module")
def c2_hmc():
    w = synth.make_c2()
    rng = np.random.default_rng(11)
    p0 = rng.standard_normal(size=w.X.shape)
    return w, p0, 2e-3, w.meta["hmc_steps"]


def _gpu_hmc(w, p0, eps, L, log_u, prec):
    import torch

    from paper_2010_02994_gb300 import HawkesContext, hmc_leapfrog_trajectory

    ctx = HawkesContext(device=0, max_n=w.n, max_d=w.d)
    X = torch.tensor(w.X, device="cuda")
    H0, H1, acc = hmc_leapfrog_trajectory(ctx, torch.tensor(w.t, device="cuda"), X, torch.tensor(p0, device="cuda"),
                                          w.params, eps, L, log_u, torch.tensor(w.box_lo, device="cuda"),
                                          torch.tensor(w.box_hi, device="cuda"), precision=prec)
    out = X.cpu().numpy(), H0.item(), H1.item(), int(acc.item())
    ctx.close()
    return out


def test_gunfire_like_hmc_trajectory_mixed_vs_fp64_and_oracle(c2_hmc):
    """The N = 10,000 trajectory with reflection at the 100 m cell walls: the
    FP64 GPU path replays the oracle, and the mixed path matches the FP64
    GPU path at rel <= 1e-6 (energies, and the end state relative to the
    domain's extent)."""
    w, p0, eps, L = c2_hmc
    Xf, H0f, H1f, accf = _gpu_hmc(w, p0, eps, L, -np.inf, "fp64")
    Xm, H0m, H1m, accm = _gpu_hmc(w, p0, eps, L, -np.inf, "mixed")
    ref = oracle.hmc_trajectory(w.t, w.X, p0, w.params, eps, L, -np.inf, w.box_lo, w.box_hi)
    assert accf == accm == ref["accepted"] == 1
    assert abs(H0f - ref["H0"]) <= 1e-10 * abs(ref["H0"])
    assert abs(H1f - ref["H1"]) <= 1e-10 * abs(ref["H1"])
    ext = float(np.max(np.abs(ref["X"])))
    assert np.max(np.abs(Xf - ref["X"])) <= 1e-10 * ext
    assert abs(H0m - H0f) <= 1e-6 * abs(H0f)
    assert abs(H1m - H1f) <= 1e-6 * abs(H1f)
    assert np.max(np.abs(Xm - Xf)) <= 1e-6 * ext
    assert np.all(Xm >= w.box_lo) and np.all(Xm <= w.box_hi)
    assert float(np.max(np.abs(Xf - w.X))) > 1e-4  # the trajectory moved
    print(f"c2 HMC: fp64 vs oracle dH1 {abs(H1f - ref['H1']) / abs(ref['H1']):.2e}, "
          f"mixed vs fp64 dH1 {abs(H1m - H1f) / abs(H1f):.2e}, dX {np.max(np.abs(Xm - Xf)) / ext:.2e}")


def _rows_per_lane(d):
    return 4 if d <= 4 else 2


def test_autotuner_on_a_batch_set():
    """hawkes_autotune times every tile shape on one set of the batch and
    keeps the fastest in the context; afterwards the options it tried are
    back at their defaults, and the default shape choice follows the stored
    entry (or ignores it when it would leave fewer than three pair blocks per
    SM): a default call is bit-identical to a call with the chosen shape set
    explicitly, or else to the call made before tuning."""
    import torch

    from paper_2010_02994_gb300 import HawkesContext, hawkes_loglik_grad_locations, tuning

    sets = synth.make_c4()
    w = next(s for s in sets if s.d == 4 and 5000 <= s.n <= 12000)
    ctx = HawkesContext(device=0, max_n=w.n, max_d=w.d, tuning=False)
    t = torch.tensor(w.t, device="cuda")
    X = torch.tensor(w.X, device="cuda")

    def run():
        ell, g = hawkes_loglik_grad_locations(ctx, t, X, w.params, precision="mixed")
        return ell.item(), g.cpu().numpy()

    before = run()
    res = tuning.autotune(ctx, t, X, w.params)
    assert res["warps"] in (1, 2, 4, 8) and res["col_groups"] in (0, 1, 2, 4) and res["ctas_per_sm"] >= 0
    assert res["warps"] * max(1, res["col_groups"]) <= 8 and res["ms"] > 0
    assert ctx.get_tuning(w.d, tuning.bucket(w.n)) == {k: res[k] for k in ("warps", "col_groups", "ctas_per_sm")}
    after = run()
    ctx.set_option("block_warps", res["warps"])
    ctx.set_option("col_groups", res["col_groups"])
    ctx.set_option("ctas_per_sm", res["ctas_per_sm"])
    explicit = run()
    for name in ("block_warps", "col_groups", "ctas_per_sm"):
        ctx.set_option(name, 0)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    T = math.ceil(w.n / (32 * _rows_per_lane(w.d) * res["warps"]))
    expected = explicit if T * (T + 1) // 2 >= 3 * sm else before
    assert after[0] == expected[0] and np.array_equal(after[1], expected[1])
    ctx.close()
