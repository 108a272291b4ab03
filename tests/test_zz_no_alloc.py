"""The entry point that allocates no device memory, against the context entry point.

Callers hosted by a framework that owns every device allocation, or real-time
callers that may not allocate after start-up, use hawkes_loglik_noalloc: it
keeps its scratch in the library's static device memory.  This file runs last
(pytest collects it after the others) so that a failure here leaves every
other test already run; it passes alone in a fresh process as well.
"""
import ctypes
import math

import numpy as np
import pytest

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


def test_noalloc_matches_context_entry_point_on_consecutive_calls():
    import torch

    from paper_2010_02994_gb300 import HawkesContext, _lib, hawkes_loglik

    lib = _lib.load()
    ctx = HawkesContext(device=0, max_n=4096, max_d=3)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    # two calls in a row on different data: the second must not see the first's scratch
    for w in (synth.random_case(201, 3000, 2, ties=2, shuffle=True),
              synth.random_case(202, 1700, 3, ties=1, shuffle=True)):
        t = torch.tensor(w.t, device="cuda")
        X = torch.tensor(w.X, device="cuda")
        ref = hawkes_loglik(ctx, t, X, w.params, precision="fp64").item()
        out.fill_(float("nan"))
        assert _call_noalloc(lib, t, X, w.params, out) == _lib.HAWKES_OK
        torch.cuda.synchronize()
        got = out.item()
        assert math.isfinite(got)
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (got, ref)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch

    from paper_2010_02994_gb300 import _lib

    lib = _lib.load()
    n = _lib.NOALLOC_MAX_N + 1
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    X = torch.zeros(n, 2, dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    assert _call_noalloc(lib, t, X, synth.random_case(0, 2, 2).params, out) == 1  # HAWKES_ERR_INVALID_ARG
