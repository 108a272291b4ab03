"""The FP64 oracle against its pins (CPU only).

See ``oracle_pins.py`` for what each pin compares against; none of them
re-types the oracle's own formulas."""
import numpy as np
import pytest

import oracle
import oracle_pins as pins


@pytest.fixture(scope="module")
def o():
    return oracle.default()


@pytest.mark.parametrize("name", sorted(pins.ALL_PINS))
def test_pin(o, name):
    ok, detail = pins.ALL_PINS[name](o)
    assert ok, f"{name}: {detail}"


def test_spatial_kernel_is_a_density():
    ok, detail = pins.pin_spatial_kernel_normalised()
    assert ok, detail


def test_zero_rate_gives_minus_infinity(o):
    # a single event has no other event to excite it: lambda_1 = 0, ell = -inf
    assert o.loglik([1.0], [[0.0, 0.0]], pins.P_DEFAULT) == -np.inf
    # two tied events: both indicators vanish, both rates are zero
    assert o.loglik([1.0, 1.0], [[0.0], [0.1]], pins.P_DEFAULT) == -np.inf


def test_invalid_arguments_rejected(o):
    with pytest.raises(ValueError):
        o.loglik([1.0, 2.0], [[0.0], [1.0]], dict(pins.P_DEFAULT, h=0.0))
    with pytest.raises(ValueError):
        o.loglik([1.0, 2.0], [[0.0], [1.0]], dict(pins.P_DEFAULT, omega=-1.0))


def test_thread_count_does_not_change_results(o):
    import synth

    w = synth.random_case(31, 200, 2)
    a = o.loglik_and_grad(w.t, w.X, w.params, nthreads=1)
    b = o.loglik_and_grad(w.t, w.X, w.params, nthreads=4)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1])
