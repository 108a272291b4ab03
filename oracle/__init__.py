"""FP64 CPU oracle for the spatiotemporal Hawkes log-likelihood (test infrastructure).

This package is the slow, obviously correct reference that the GPU library is
checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the GPU
path: the arithmetic lives in ``hawkes_oracle.c`` (plain double loops, written
from the definitions of Section 2.1, Eq. (1) and Appendix A of the paper) and
this module only marshals numpy arrays into it.

Every function here is pinned by ``tests/test_oracle_pins.py`` against
brute force from the free-point rate definition, quadrature of the integrated
rate, a symbolic two-event case, finite differences, invariances and closed
forms.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hawkes_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libhawkes_oracle.so")

_lock = threading.Lock()


class OracleParams(ctypes.Structure):
    """Theta = (mu0, tau_x, tau_t, theta, omega, h), the order of Section 2.1."""

    _fields_ = [(name, ctypes.c_double) for name in ("mu0", "tau_x", "tau_t", "theta", "omega", "h")]


def compile_command(out_path: str = _LIB_PATH, extra: list[str] | None = None) -> list[str]:
    """gcc command that builds the oracle as a shared library (no fused multiply-add)."""
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", out_path, "-lm"]
    if extra:
        cmd[1:1] = extra
    return cmd


def build(force: bool = False) -> str:
    """Compile hawkes_oracle.c if the library is missing or older than the source."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(compile_command(tmp), check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load_library(path: str) -> ctypes.CDLL:
    """Load an oracle build and declare its C signatures."""
    lib = ctypes.CDLL(path)
    i64, i32, dp = ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_int64)
    pp = ctypes.POINTER(OracleParams)
    lib.oracle_rates.argtypes = [i64, i32, dp, dp, pp, dp, dp, dp, i32]
    lib.oracle_rates_rows.argtypes = [i64, i32, dp, dp, pp, i64, lp, dp, i32]
    lib.oracle_Lambda.argtypes = [i64, dp, pp, dp]
    lib.oracle_Lambda.restype = ctypes.c_double
    lib.oracle_loglik.argtypes = [i64, i32, dp, dp, pp, dp, dp, i32]
    lib.oracle_grad_locations.argtypes = [i64, i32, dp, dp, pp, dp, dp, i32]
    lib.oracle_grad_rows.argtypes = [i64, i32, dp, dp, pp, dp, i64, lp, dp, i32]
    lib.oracle_grad_params.argtypes = [i64, i32, dp, dp, pp, dp, dp, i32]
    lib.oracle_grad_params_scaled.argtypes = [i64, i32, dp, dp, pp, dp, dp, dp, i32]
    lib.oracle_hmc_trajectory.argtypes = [i64, i32, dp, dp, dp, dp, dp, pp, ctypes.c_double, i32,
                                          ctypes.c_double, dp, dp, dp, dp,
                                          ctypes.POINTER(ctypes.c_int32), i32]
    lib.oracle_bmds_hmc_trajectory.argtypes = [i64, i32, dp, dp, dp, pp, dp, ctypes.c_double, ctypes.c_double, i32,
                                               ctypes.c_double, dp, dp, dp, dp, ctypes.POINTER(ctypes.c_int32), i32]
    lib.oracle_bmds_hmc_trajectory.restype = ctypes.c_int
    lib.oracle_bmds.argtypes = [i64, i32, dp, dp, ctypes.c_double, dp, dp, dp, i32]
    lib.oracle_bmds.restype = ctypes.c_int
    lib.oracle_lens_area.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.oracle_lens_area.restype = ctypes.c_double
    lib.oracle_circle_proposals.argtypes = [i32, dp, dp, dp, ctypes.c_double, i32, dp, dp, dp]
    lib.oracle_circle_proposals.restype = ctypes.c_int
    lib.oracle_box_proposals.argtypes = [i32, i32, dp, dp, dp, ctypes.c_double, dp, dp, dp]
    lib.oracle_box_proposals.restype = ctypes.c_int
    lib.oracle_max_threads.restype = i32
    for name in ("oracle_rates", "oracle_rates_rows", "oracle_loglik", "oracle_grad_locations",
                 "oracle_grad_rows", "oracle_grad_params", "oracle_grad_params_scaled", "oracle_hmc_trajectory"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _prep(t, X):
    t = _as_f64(t).reshape(-1)
    X = _as_f64(X)
    if X.ndim == 1:
        X = X.reshape(-1, 1)
    if X.shape[0] != t.shape[0]:
        raise ValueError("t and X disagree on the number of events")
    return t, X


def params_struct(params) -> OracleParams:
    """Accept a mapping with the six names, a sequence in Theta order, or OracleParams."""
    if isinstance(params, OracleParams):
        return params
    if isinstance(params, dict):
        return OracleParams(*(float(params[k]) for k in ("mu0", "tau_x", "tau_t", "theta", "omega", "h")))
    vals = [float(v) for v in params]
    if len(vals) != 6:
        raise ValueError("Theta has six components")
    return OracleParams(*vals)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid argument")


class Oracle:
    """Methods over one loaded oracle build (the default build, or a variant
    compiled elsewhere, e.g. a deliberately broken copy in a mutation test)."""

    def __init__(self, lib: ctypes.CDLL):
        self.lib = lib

    def rates(self, t, X, params, nthreads: int = 0, parts: bool = False):
        """lambda_n for all rows (Eq. (1)); with parts=True also (M_n, Xi_n)."""
        t, X = _prep(t, X)
        n, d = X.shape
        lam = np.empty(n)
        mu = np.empty(n) if parts else None
        xi = np.empty(n) if parts else None
        p = params_struct(params)
        _check(self.lib.oracle_rates(n, d, _dp(t), _dp(X), ctypes.byref(p), _dp(lam), _dp(mu), _dp(xi),
                                     nthreads), "rates")
        return (lam, mu, xi) if parts else lam

    def rates_rows(self, t, X, params, rows, nthreads: int = 0):
        """lambda_n for the listed rows only."""
        t, X = _prep(t, X)
        n, d = X.shape
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        lam = np.empty(rows.shape[0])
        p = params_struct(params)
        _check(self.lib.oracle_rates_rows(n, d, _dp(t), _dp(X), ctypes.byref(p), rows.shape[0],
                                          rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(lam),
                                          nthreads), "rates_rows")
        return lam

    def Lambda(self, t, params, per_event: bool = False):
        """Integrated rate of Section 2.1: sum_n Lambda_n (and the Lambda_n)."""
        t = _as_f64(t).reshape(-1)
        out = np.empty(t.shape[0]) if per_event else None
        p = params_struct(params)
        total = self.lib.oracle_Lambda(t.shape[0], _dp(t), ctypes.byref(p), _dp(out))
        return (total, out) if per_event else total

    def loglik(self, t, X, params, nthreads: int = 0, return_rates: bool = False):
        """ell of Eq. (1)."""
        t, X = _prep(t, X)
        n, d = X.shape
        out = np.empty(1)
        lam = np.empty(n)
        p = params_struct(params)
        _check(self.lib.oracle_loglik(n, d, _dp(t), _dp(X), ctypes.byref(p), _dp(out), _dp(lam), nthreads),
               "loglik")
        return (float(out[0]), lam) if return_rates else float(out[0])

    def grad_locations(self, t, X, params, lam=None, nthreads: int = 0):
        """d ell / d X (Appendix A), shape (N, D)."""
        t, X = _prep(t, X)
        n, d = X.shape
        if lam is None:
            lam = self.rates(t, X, params, nthreads)
        lam = _as_f64(lam)
        g = np.empty((n, d))
        p = params_struct(params)
        _check(self.lib.oracle_grad_locations(n, d, _dp(t), _dp(X), ctypes.byref(p), _dp(lam), _dp(g),
                                              nthreads), "grad_locations")
        return g

    def grad_rows(self, t, X, params, lam, rows, nthreads: int = 0):
        """d ell / d x_n for the listed rows; lam holds lambda for every row."""
        t, X = _prep(t, X)
        n, d = X.shape
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        lam = _as_f64(lam)
        g = np.empty((rows.shape[0], d))
        p = params_struct(params)
        _check(self.lib.oracle_grad_rows(n, d, _dp(t), _dp(X), ctypes.byref(p), _dp(lam), rows.shape[0],
                                         rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(g),
                                         nthreads), "grad_rows")
        return g

    def grad_params(self, t, X, params, lam=None, nthreads: int = 0):
        """d ell / d Theta in the order (mu0, tau_x, tau_t, theta, omega, h)."""
        t, X = _prep(t, X)
        n, d = X.shape
        if lam is None:
            lam = self.rates(t, X, params, nthreads)
        lam = _as_f64(lam)
        out = np.empty(6)
        p = params_struct(params)
        _check(self.lib.oracle_grad_params(n, d, _dp(t), _dp(X), ctypes.byref(p), _dp(lam), _dp(out),
                                           nthreads), "grad_params")
        return out

    def grad_params_scaled(self, t, X, params, lam=None, nthreads: int = 0):
        """(d ell / d Theta, scale): scale[k] sums the magnitudes of the terms
        component k is summed from (the pair-term pieces over lambda_n and the
        derivatives of Lambda_n), the size a rounding error of the row sums is
        relative to.  The gradient is the one grad_params returns."""
        t, X = _prep(t, X)
        n, d = X.shape
        if lam is None:
            lam = self.rates(t, X, params, nthreads)
        lam = _as_f64(lam)
        out = np.empty(6)
        scale = np.empty(6)
        p = params_struct(params)
        _check(self.lib.oracle_grad_params_scaled(n, d, _dp(t), _dp(X), ctypes.byref(p), _dp(lam), _dp(out),
                                                  _dp(scale), nthreads), "grad_params_scaled")
        return out, scale

    def loglik_and_grad(self, t, X, params, nthreads: int = 0):
        """(ell, d ell / d X, lambda)."""
        ell, lam = self.loglik(t, X, params, nthreads, return_rates=True)
        g = self.grad_locations(t, X, params, lam, nthreads)
        return ell, g, lam

    def hmc_trajectory(self, t, X0, p0, params, eps, n_steps, log_u, box_lo=None, box_hi=None,
                       nthreads: int = 0):
        """One HMC proposal over the locations (Section 3).  Returns a dict with
        X (accepted state), p (final momenta of the proposal), H0, H1, accepted."""
        t, X0 = _prep(t, X0)
        n, d = X0.shape
        p0 = _as_f64(p0).reshape(n, d)
        lo = None if box_lo is None else _as_f64(box_lo).reshape(n, d)
        hi = None if box_hi is None else _as_f64(box_hi).reshape(n, d)
        Xo = np.empty((n, d))
        po = np.empty((n, d))
        H0 = np.empty(1)
        H1 = np.empty(1)
        acc = ctypes.c_int32(0)
        p = params_struct(params)
        _check(self.lib.oracle_hmc_trajectory(n, d, _dp(t), _dp(X0), _dp(p0), _dp(lo), _dp(hi), ctypes.byref(p),
                                              float(eps), int(n_steps), float(log_u), _dp(Xo), _dp(po),
                                              _dp(H0), _dp(H1), ctypes.byref(acc), nthreads), "hmc_trajectory")
        return {"X": Xo, "p": po, "H0": float(H0[0]), "H1": float(H1[0]), "accepted": int(acc.value)}

    def bmds_hmc_trajectory(self, t, X0, p0, params, Y, sigma2, eps, n_steps, log_u, nthreads: int = 0):
        """One HMC proposal over the locations of the BMDS-Hawkes model
        (potential -ell_Hawkes - ell_BMDS, unconstrained); as hmc_trajectory."""
        t, X0 = _prep(t, X0)
        n, d = X0.shape
        p0 = _as_f64(p0).reshape(n, d)
        Y = _as_f64(Y).reshape(n, n)
        Xo = np.empty((n, d))
        po = np.empty((n, d))
        H0 = np.empty(1)
        H1 = np.empty(1)
        acc = ctypes.c_int32(0)
        p = params_struct(params)
        _check(self.lib.oracle_bmds_hmc_trajectory(n, d, _dp(t), _dp(X0), _dp(p0), ctypes.byref(p), _dp(Y),
                                                   float(sigma2), float(eps), int(n_steps), float(log_u), _dp(Xo),
                                                   _dp(po), _dp(H0), _dp(H1), ctypes.byref(acc), nthreads),
               "bmds_hmc_trajectory")
        return {"X": Xo, "p": po, "H0": float(H0[0]), "H1": float(H1[0]), "accepted": int(acc.value)}

    def bmds(self, Y, X, sigma2, nthreads: int = 0):
        """BMDS log-likelihood of Eq. (4) (up to a constant), its gradient in X
        and in sigma2: (ell, grad (N, D), d ell / d sigma2)."""
        X = _as_f64(X)
        if X.ndim == 1:
            X = X.reshape(-1, 1)
        n, d = X.shape
        Y = _as_f64(Y).reshape(n, n)
        out = np.empty(1)
        g = np.empty((n, d))
        gs = np.empty(1)
        _check(self.lib.oracle_bmds(n, d, _dp(Y), _dp(X), float(sigma2), _dp(out), _dp(g), _dp(gs), nthreads),
               "bmds")
        return float(out[0]), g, float(gs[0])

    def lens_area(self, R, rho, c) -> float:
        """Area of the intersection of discs of radii R and rho, centres c apart."""
        return float(self.lib.oracle_lens_area(float(R), float(rho), float(c)))

    def circle_proposals(self, X, centers, radii, eps, tries, u):
        """Lens proposals of Eq. (6) for the D = 2 rows of X: (X_new, log q-ratio).
        u has shape (nb, tries, 2)."""
        X = _as_f64(X).reshape(-1, 2)
        nb = X.shape[0]
        C = _as_f64(centers).reshape(nb, 2)
        r = _as_f64(radii).reshape(nb)
        u = _as_f64(u).reshape(nb, int(tries), 2)
        Xn = np.empty((nb, 2))
        lq = np.empty(1)
        _check(self.lib.oracle_circle_proposals(nb, _dp(X), _dp(C), _dp(r), float(eps), int(tries), _dp(u), _dp(Xn),
                                                _dp(lq)), "circle_proposals")
        return Xn, float(lq[0])

    def box_proposals(self, X, lo, hi, s, u):
        """Truncated-normal proposals inside the boxes [lo, hi]: (X_new, log q-ratio)."""
        X = _as_f64(X)
        if X.ndim == 1:
            X = X.reshape(-1, 1)
        nb, d = X.shape
        lo = _as_f64(lo).reshape(nb, d)
        hi = _as_f64(hi).reshape(nb, d)
        u = _as_f64(u).reshape(nb, d)
        Xn = np.empty((nb, d))
        lq = np.empty(1)
        _check(self.lib.oracle_box_proposals(nb, d, _dp(X), _dp(lo), _dp(hi), float(s), _dp(u), _dp(Xn), _dp(lq)),
               "box_proposals")
        return Xn, float(lq[0])

    def max_threads(self) -> int:
        """Threads an OpenMP region of the oracle uses by default."""
        return int(self.lib.oracle_max_threads())


_default = None


def default() -> Oracle:
    """The oracle built from hawkes_oracle.c in this directory."""
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(load_library(build()))
        return _default


def rates(*a, **k):
    return default().rates(*a, **k)


def rates_rows(*a, **k):
    return default().rates_rows(*a, **k)


def Lambda(*a, **k):
    return default().Lambda(*a, **k)


def loglik(*a, **k):
    return default().loglik(*a, **k)


def grad_locations(*a, **k):
    return default().grad_locations(*a, **k)


def grad_rows(*a, **k):
    return default().grad_rows(*a, **k)


def grad_params(*a, **k):
    return default().grad_params(*a, **k)


def grad_params_scaled(*a, **k):
    return default().grad_params_scaled(*a, **k)


def loglik_and_grad(*a, **k):
    return default().loglik_and_grad(*a, **k)


def hmc_trajectory(*a, **k):
    return default().hmc_trajectory(*a, **k)


def bmds(*a, **k):
    return default().bmds(*a, **k)


def bmds_hmc_trajectory(*a, **k):
    return default().bmds_hmc_trajectory(*a, **k)


def lens_area(*a, **k):
    return default().lens_area(*a, **k)


def circle_proposals(*a, **k):
    return default().circle_proposals(*a, **k)


def box_proposals(*a, **k):
    return default().box_proposals(*a, **k)


def max_threads() -> int:
    """Threads an OpenMP region of the oracle uses by default."""
    return default().max_threads()
