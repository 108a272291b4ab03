"""Seeded synthetic workloads: determinism, sizes, and the box structure."""
import numpy as np

import synth


def test_deterministic_and_sized():
    a, b = synth.make_c1(), synth.make_c1()
    assert np.array_equal(a.t, b.t) and np.array_equal(a.X, b.X)
    assert a.n == 1000 and a.d == 2
    assert np.all(np.diff(a.t) >= 0) and a.t.min() >= 0 and a.t.max() <= 100.0


def test_boxes_contain_latent_locations():
    for w in (synth.make_c1(), synth.make_c3()):
        assert np.all(w.X >= w.box_lo) and np.all(w.X <= w.box_hi)
        assert np.all(w.box_hi - w.box_lo > 0)


def test_grid_coarsening_is_100m():
    w = synth.make_c1()
    assert np.allclose(np.round(w.X_obs / 0.1) * 0.1, w.X_obs)
    assert np.allclose(w.box_hi - w.box_lo, 0.1)


def test_batched_sets_cover_the_stated_ranges():
    sets = synth.make_c4()
    assert len(sets) == 64
    ns = np.array([w.n for w in sets])
    ds = {w.d for w in sets}
    assert ns.min() >= 500 and ns.max() <= 20_000 and ds <= {2, 4, 8}


def test_random_case_ties_and_shuffle():
    w = synth.random_case(3, 50, 2, ties=3, shuffle=True)
    assert len(np.unique(w.t)) < 50
    assert np.any(np.diff(w.t) < 0)
