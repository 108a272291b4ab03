"""The entry point that allocates no device memory, against the FP64 oracle.

Callers hosted by a framework that owns every device allocation, or real-time
callers that may not allocate after start-up, cannot create a context (its
workspace is allocated), so they use hawkes_loglik_noalloc, which keeps its
scratch in the library's static device memory.  This file runs last (pytest
collects it after the others) so that a failure here leaves every other test
already run; it passes alone in a fresh process as well.

Tolerance: the entry point computes in FP64, so its ell is held to the FP64
path's 1e-12, relative to the magnitude of the terms of ell
(sum |log lambda_n| + sum Lambda_n), which random data can cancel to near zero.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, t, X, params, out):
    import torch

    from paper_2010_02994_gb300 import params_struct

    p = params_struct(params)
    n, d = X.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.hawkes_loglik_noalloc(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(X.data_ptr()), n, d,
                                     ctypes.byref(p), stream, ctypes.c_void_p(out.data_ptr()))


def _noalloc(lib, t_np, X_np, params):
    import torch

    from paper_2010_02994_gb300 import _lib

    t = torch.tensor(np.asarray(t_np, dtype=np.float64), device="cuda")
    X = torch.tensor(np.asarray(X_np, dtype=np.float64), device="cuda")
    out = torch.full((1,), 12345.0, dtype=torch.float64, device="cuda")
    assert _call_noalloc(lib, t, X, params, out) == _lib.HAWKES_OK
    torch.cuda.synchronize()
    return out.item()


def _scale(w):
    lam = oracle.rates(w.t, w.X, w.params)
    return float(np.sum(np.abs(np.log(lam))) + oracle.Lambda(w.t, w.params))


def test_noalloc_matches_oracle_on_consecutive_calls():
    """Two calls in a row on different data (the second must not see the
    first's scratch), then the largest size it accepts in eight dimensions,
    each against the oracle."""
    from paper_2010_02994_gb300 import _lib

    lib = _lib.load()
    cases = (synth.random_case(201, 3000, 2, ties=2, shuffle=True),
             synth.random_case(202, 1700, 3, ties=1, shuffle=True),
             synth.random_case(203, _lib.NOALLOC_MAX_N, 8, ties=3, shuffle=True))
    for w in cases:
        got = _noalloc(lib, w.t, w.X, w.params)
        ref = oracle.loglik(w.t, w.X, w.params)
        assert math.isfinite(got)
        assert abs(got - ref) <= 1e-12 * _scale(w), (w.n, w.d, got, ref)


def test_noalloc_matches_context_entry_point():
    """The same value as the context entry point in FP64, on a paper-shaped
    workload (the wildfire-like events, N = 5,000)."""
    import torch

    from paper_2010_02994_gb300 import HawkesContext, _lib, hawkes_loglik

    lib = _lib.load()
    w = synth.make_c3()
    ctx = HawkesContext(device=0, max_n=w.n, max_d=w.d)
    ref = hawkes_loglik(ctx, torch.tensor(w.t, device="cuda"), torch.tensor(w.X, device="cuda"), w.params,
                        precision="fp64").item()
    ctx.close()
    got = _noalloc(lib, w.t, w.X, w.params)
    assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)


def test_noalloc_zero_rate_and_invalid_data():
    """A rate of zero gives -inf (one event; three tied events); a negative or
    non-finite time, or a non-finite coordinate, gives NaN; a valid call
    afterwards is unaffected by the status the invalid ones left."""
    from paper_2010_02994_gb300 import _lib

    lib = _lib.load()
    P = synth.random_case(0, 2, 2).params
    assert _noalloc(lib, [1.0], [[0.3, 0.2]], P) == -math.inf
    assert _noalloc(lib, [2.0, 2.0, 2.0], [[0.0, 0.0], [0.1, 0.0], [0.0, 0.2]], P) == -math.inf
    w = synth.random_case(204, 500, 2, shuffle=True)
    for k, bad in enumerate((-1.0, math.nan, math.inf)):
        t = w.t.copy()
        t[37 * (k + 1)] = bad
        assert math.isnan(_noalloc(lib, t, w.X, w.params))
    X = w.X.copy()
    X[123, 1] = math.nan
    assert math.isnan(_noalloc(lib, w.t, X, w.params))
    ref = oracle.loglik(w.t, w.X, w.params)
    assert abs(_noalloc(lib, w.t, w.X, w.params) - ref) <= 1e-12 * _scale(w)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch

    from paper_2010_02994_gb300 import _lib

    lib = _lib.load()
    n = _lib.NOALLOC_MAX_N + 1
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    X = torch.zeros(n, 2, dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    assert _call_noalloc(lib, t, X, synth.random_case(0, 2, 2).params, out) == 1  # HAWKES_ERR_INVALID_ARG
    X9 = torch.zeros(8, 9, dtype=torch.float64, device="cuda")
    assert _call_noalloc(lib, t[:8], X9, synth.random_case(0, 2, 2).params, out) == 1
