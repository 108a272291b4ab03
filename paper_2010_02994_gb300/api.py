"""Python binding of libhawkes: argument marshalling only.

Functions named after the C entry points take torch CUDA tensors (float64,
contiguous) and enqueue the work on the current torch stream of the tensors'
device.  Every step of the computation runs in the library's CUDA kernels.

    ctx = HawkesContext(device=0, max_n=100_000, max_d=2)
    ell, grad = hawkes_loglik_grad_locations(ctx, t, X, params)   # device tensors
    ctx.sync_status()                                             # raises on a device-side error
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import HawkesError, HawkesParams

PARAM_NAMES = ("mu0", "tau_x", "tau_t", "theta", "omega", "h")


def params_struct(params) -> HawkesParams:
    """A mapping with the six names, a sequence in Theta order, or HawkesParams."""
    if isinstance(params, HawkesParams):
        return params
    if isinstance(params, dict):
        return HawkesParams(*(float(params[k]) for k in PARAM_NAMES))
    if isinstance(params, torch.Tensor):
        params = params.detach().cpu().tolist()
    vals = [float(v) for v in params]
    if len(vals) != 6:
        raise ValueError("Theta has six components")
    return HawkesParams(*vals)


def _ptr(x: torch.Tensor | None) -> int | None:
    return None if x is None else x.data_ptr()


def _dev_f64(x: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    return x.contiguous()


def _precision(p) -> int:
    if isinstance(p, int):
        return p
    return _lib.PREC[p]


class HawkesContext:
    """Owns a libhawkes context (device workspace, cached HMC graphs)."""

    def __init__(self, device: int = 0, max_n: int = 1024, max_d: int = 8, tuning: bool = True):
        """tuning: load this GPU's entries of the tile-shape table (tuning.json)."""
        self.lib = _lib.load()
        self.device = int(device)
        h = ctypes.c_void_p()
        st = self.lib.hawkes_ctx_create(ctypes.byref(h), self.device, int(max_n), int(max_d))
        if st != _lib.HAWKES_OK:
            raise HawkesError(st, self.lib.hawkes_last_error(None).decode())
        self.handle = h
        if tuning:
            from . import tuning as _tuning

            _tuning.load_into(self)

    def get_tuning(self, d: int, bucket: int):
        w, wc, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self.check(self.lib.hawkes_ctx_get_tuning(self.handle, int(d), int(bucket), ctypes.byref(w), ctypes.byref(wc),
                                                  ctypes.byref(c)))
        return {"warps": w.value, "col_groups": wc.value, "ctas_per_sm": c.value}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.hawkes_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, status: int):
        if status != _lib.HAWKES_OK:
            raise HawkesError(status, self.lib.hawkes_last_error(self.handle).decode())

    def stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def sync_status(self):
        """Wait for the current stream and raise if a device-side error was recorded."""
        self.check(self.lib.hawkes_ctx_sync_status(self.handle, self.stream()))

    def set_option(self, name: str, value: int):
        self.check(self.lib.hawkes_ctx_set_option(self.handle, _lib.OPTIONS[name], int(value)))

    def kernel_stats(self, kernel: int):
        ms, n, pairs = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        self.check(self.lib.hawkes_ctx_kernel_stats(self.handle, int(kernel), ctypes.byref(ms), ctypes.byref(n),
                                                    ctypes.byref(pairs)))
        return {"ms": ms.value, "launches": n.value, "pairs": pairs.value}

    def launch_count(self):
        own, lib = ctypes.c_int64(), ctypes.c_int64()
        self.check(self.lib.hawkes_ctx_launch_count(self.handle, ctypes.byref(own), ctypes.byref(lib)))
        return {"own": own.value, "library": lib.value}

    def reset_stats(self):
        self.check(self.lib.hawkes_ctx_reset_stats(self.handle))


def _shape(t: torch.Tensor, X: torch.Tensor):
    n = t.numel()
    if X.dim() == 1:
        X = X.reshape(n, 1)
    if X.dim() != 2 or X.shape[0] != n:
        raise ValueError("X must be (N, D) with N = len(t)")
    return n, X.shape[1], X


def hawkes_loglik(ctx: HawkesContext, t, X, params, precision="mixed", check: bool = True) -> torch.Tensor:
    """ell of Eq. (1) as a 0-d float64 tensor on the device."""
    t = _dev_f64(t, "t")
    X = _dev_f64(X, "X")
    n, d, X = _shape(t, X)
    out = torch.empty((), dtype=torch.float64, device=t.device)
    p = params_struct(params)
    ctx.check(ctx.lib.hawkes_loglik(ctx.handle, _ptr(t), _ptr(X), n, d, ctypes.byref(p), _precision(precision),
                                    ctx.stream(), _ptr(out)))
    if check:
        ctx.sync_status()
    return out


def hawkes_self_excitation_prob(ctx: HawkesContext, t, X, params, precision="mixed", check: bool = True):
    """xi / (xi + mu) at every event (Section 4.3), as a device tensor (N,)."""
    t = _dev_f64(t, "t")
    X = _dev_f64(X, "X")
    n, d, X = _shape(t, X)
    out = torch.empty(n, dtype=torch.float64, device=t.device)
    p = params_struct(params)
    ctx.check(ctx.lib.hawkes_self_excitation_prob(ctx.handle, _ptr(t), _ptr(X), n, d, ctypes.byref(p),
                                                  _precision(precision), ctx.stream(), _ptr(out)))
    if check:
        ctx.sync_status()
    return out


def hawkes_loglik_grad_locations(ctx: HawkesContext, t, X, params, precision="mixed", grad_params: bool = False,
                                 check: bool = True, out=None):
    """(ell, d ell/d X) -- and d ell/d Theta when grad_params -- as device tensors."""
    t = _dev_f64(t, "t")
    X = _dev_f64(X, "X")
    n, d, X = _shape(t, X)
    if out is None:
        ell = torch.empty((), dtype=torch.float64, device=t.device)
        g = torch.empty((n, d), dtype=torch.float64, device=t.device)
        gp = torch.empty(6, dtype=torch.float64, device=t.device) if grad_params else None
    else:
        ell, g, gp = out
        gp = gp if grad_params else None
    p = params_struct(params)
    ctx.check(ctx.lib.hawkes_loglik_grad_locations(ctx.handle, _ptr(t), _ptr(X), n, d, ctypes.byref(p),
                                                   _precision(precision), ctx.stream(), _ptr(ell), _ptr(g),
                                                   _ptr(gp)))
    if check:
        ctx.sync_status()
    return (ell, g, gp) if grad_params else (ell, g)


def hawkes_bmds_hmc_trajectory(ctx: HawkesContext, t, X, p0, params, Y, sigma2: float, eps: float, n_steps: int,
                               log_u, precision="mixed", check: bool = True):
    """One HMC proposal over the locations of the BMDS-Hawkes model (potential
    -ell - ell_B).  X is updated in place when accepted.  Y is (N, N), float64
    or float32.  Returns (H0, H1, accepted) as device tensors."""
    t = _dev_f64(t, "t")
    if not (X.is_cuda and X.dtype == torch.float64 and X.is_contiguous()):
        raise TypeError("X must be a contiguous float64 CUDA tensor (it is updated in place)")
    n, d, _ = _shape(t, X)
    p0 = _dev_f64(p0, "p0")
    if not isinstance(Y, torch.Tensor) or not Y.is_cuda or Y.dtype not in (torch.float64, torch.float32):
        raise TypeError("Y must be a float64 or float32 CUDA tensor")
    Y = Y.contiguous()
    if Y.shape != (n, n):
        raise ValueError("Y must be (N, N)")
    if not isinstance(log_u, torch.Tensor):
        log_u = torch.tensor(float(log_u), dtype=torch.float64, device=t.device)
    log_u = _dev_f64(log_u, "log_u")
    H0 = torch.empty((), dtype=torch.float64, device=t.device)
    H1 = torch.empty((), dtype=torch.float64, device=t.device)
    acc = torch.empty((), dtype=torch.int32, device=t.device)
    p = params_struct(params)
    ctx.check(ctx.lib.hawkes_bmds_hmc_trajectory(ctx.handle, _ptr(t), _ptr(X), _ptr(p0), n, d, ctypes.byref(p),
                                                 _ptr(Y), 1 if Y.dtype == torch.float32 else 0, float(sigma2),
                                                 float(eps), int(n_steps), _ptr(log_u), _precision(precision),
                                                 ctx.stream(), _ptr(H0), _ptr(H1), _ptr(acc)))
    if check:
        ctx.sync_status()
    return H0, H1, acc


def hawkes_bmds_loglik_grad(ctx: HawkesContext, Y, X, sigma2: float, precision="mixed", grad: bool = True,
                            check: bool = True, out=None):
    """BMDS likelihood of Eq. (4) with its gradients: (ell_B, d ell_B/d X,
    d ell_B/d sigma2) as device tensors (the gradients None when grad is
    False).  Y is the (N, N) distance matrix, float64 or float32 (a float32
    copy halves the memory traffic of the mixed precision and gives the same
    results); only its entries below the diagonal are read."""
    if not isinstance(Y, torch.Tensor) or not Y.is_cuda or Y.dtype not in (torch.float64, torch.float32):
        raise TypeError("Y must be a float64 or float32 CUDA tensor")
    Y = Y.contiguous()
    y_type = 1 if Y.dtype == torch.float32 else 0
    X = _dev_f64(X, "X")
    if X.dim() == 1:
        X = X.reshape(-1, 1)
    n, d = X.shape
    if Y.shape != (n, n):
        raise ValueError("Y must be (N, N) with N = X.shape[0]")
    if out is None:
        ell = torch.empty((), dtype=torch.float64, device=X.device)
        g = torch.empty((n, d), dtype=torch.float64, device=X.device) if grad else None
        gs = torch.empty((), dtype=torch.float64, device=X.device) if grad else None
    else:
        ell, g, gs = out
    ctx.check(ctx.lib.hawkes_bmds_loglik_grad(ctx.handle, _ptr(Y), y_type, _ptr(X), n, d, float(sigma2),
                                              _precision(precision), ctx.stream(), _ptr(ell), _ptr(g), _ptr(gs)))
    if check:
        ctx.sync_status()
    return ell, g, gs


def hmc_leapfrog_trajectory(ctx: HawkesContext, t, X, p0, params, eps: float, n_steps: int, log_u,
                            box_lo=None, box_hi=None, precision="mixed", check: bool = True):
    """One HMC proposal (Section 3).  X is updated in place when accepted.
    Returns (H0, H1, accepted) as device tensors."""
    t = _dev_f64(t, "t")
    if not (X.is_cuda and X.dtype == torch.float64 and X.is_contiguous()):
        raise TypeError("X must be a contiguous float64 CUDA tensor (it is updated in place)")
    n, d, _ = _shape(t, X)
    p0 = _dev_f64(p0, "p0")
    lo = None if box_lo is None else _dev_f64(box_lo, "box_lo")
    hi = None if box_hi is None else _dev_f64(box_hi, "box_hi")
    if not isinstance(log_u, torch.Tensor):
        log_u = torch.tensor(float(log_u), dtype=torch.float64, device=t.device)
    log_u = _dev_f64(log_u, "log_u")
    H0 = torch.empty((), dtype=torch.float64, device=t.device)
    H1 = torch.empty((), dtype=torch.float64, device=t.device)
    acc = torch.empty((), dtype=torch.int32, device=t.device)
    p = params_struct(params)
    ctx.check(ctx.lib.hmc_leapfrog_trajectory(ctx.handle, _ptr(t), _ptr(X), _ptr(p0), _ptr(lo), _ptr(hi), n, d,
                                              ctypes.byref(p), float(eps), int(n_steps), _ptr(log_u),
                                              _precision(precision), ctx.stream(), _ptr(H0), _ptr(H1), _ptr(acc)))
    if check:
        ctx.sync_status()
    return H0, H1, acc


def hawkes_batch_loglik_grad(ctx: HawkesContext, sizes, dims, t, X, params_list, precision="mixed",
                             check: bool = True):
    """Log-likelihoods (n_sets,) and the packed location gradient of a batch
    of independent sets.  sizes/dims: per-set event counts and dimensions;
    t: all times back to back; X: all locations back to back, each set
    row-major with its own width."""
    t = _dev_f64(t, "t")
    X = _dev_f64(X, "X").reshape(-1)
    ns = len(sizes)
    offs = (ctypes.c_int64 * (ns + 1))()
    acc = 0
    for i, s in enumerate(sizes):
        offs[i] = acc
        acc += int(s)
    offs[ns] = acc
    dims_c = (ctypes.c_int32 * ns)(*[int(v) for v in dims])
    ps = (HawkesParams * ns)(*[params_struct(p) for p in params_list])
    ell = torch.empty(ns, dtype=torch.float64, device=t.device)
    g = torch.empty_like(X)
    ctx.check(ctx.lib.hawkes_batch_loglik_grad(ctx.handle, ns, offs, dims_c, _ptr(t), _ptr(X), ps,
                                               _precision(precision), ctx.stream(), _ptr(ell), _ptr(g)))
    if check:
        ctx.sync_status()
    return ell, g


def hawkes_loglik_noalloc(t, X, params) -> torch.Tensor:
    """ell of Eq. (1) (FP64) through the entry point that allocates no device
    memory, for up to 8192 events; runs on the tensors' device and stream.
    The returned 0-d tensor is the caller's output buffer."""
    lib = _lib.load()
    t = _dev_f64(t, "t")
    X = _dev_f64(X, "X")
    n, d, X = _shape(t, X)
    out = torch.empty((), dtype=torch.float64, device=t.device)
    p = params_struct(params)
    with torch.cuda.device(t.device):
        st = lib.hawkes_loglik_noalloc(_ptr(t), _ptr(X), n, d, ctypes.byref(p),
                                       ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream), _ptr(out))
    if st != _lib.HAWKES_OK:
        raise HawkesError(st, f"hawkes_loglik_noalloc: n must be in [1, {_lib.NOALLOC_MAX_N}], d in [1, 8], "
                              "parameters finite and positive")
    return out


def probe_pipe_rates(device: int = 0) -> dict:
    """Measured FP32 FMA and MUFU ex2 results per SM per clock (and the SM clock)."""
    lib = _lib.load()
    f, e, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = lib.hawkes_probe_pipe_rates(int(device), ctypes.byref(f), ctypes.byref(e), ctypes.byref(mhz))
    if st != _lib.HAWKES_OK:
        raise HawkesError(st, "pipe-rate probe failed")
    return {"fma_per_sm_clk": f.value, "ex2_per_sm_clk": e.value, "sm_mhz": mhz.value}


def probe_dfma_rate(device: int = 0) -> float:
    """Measured FP64 FMA results per SM per clock (the bound of the FP64 path)."""
    lib = _lib.load()
    r = ctypes.c_double()
    st = lib.hawkes_probe_dfma_rate(int(device), ctypes.byref(r))
    if st != _lib.HAWKES_OK:
        raise HawkesError(st, "DFMA probe failed")
    return r.value


def probe_exp2_fp64(y: torch.Tensor) -> torch.Tensor:
    """2^y by the FP64 pair kernels' exponential (Tang's table-driven method),
    for a CUDA float64 tensor y; y <= 0 is the meaningful range."""
    if not (y.is_cuda and y.dtype == torch.float64):
        raise ValueError("y must be a CUDA float64 tensor")
    y = y.contiguous()
    out = torch.empty_like(y)
    lib = _lib.load()
    st = lib.hawkes_probe_exp2_fp64(ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(out.data_ptr()), y.numel(),
                                    ctypes.c_void_p(torch.cuda.current_stream(y.device).cuda_stream))
    if st != _lib.HAWKES_OK:
        raise HawkesError(st, "exp2 probe failed")
    return out


def hawkes_batch_hmc_trajectory(ctx: HawkesContext, sizes, dims, t, X, p0, params_list, eps, n_steps: int, log_u,
                                box_lo=None, box_hi=None, precision="mixed", check: bool = True):
    """One HMC proposal per set (layout as in hawkes_batch_loglik_grad); X is
    updated in place for the sets that accept.  eps: one step size per set;
    log_u: (n_sets,) device tensor.  Returns (H0, H1, accepted) per set."""
    t = _dev_f64(t, "t")
    if not (X.is_cuda and X.dtype == torch.float64 and X.is_contiguous()):
        raise TypeError("X must be a contiguous float64 CUDA tensor (it is updated in place)")
    p0 = _dev_f64(p0, "p0")
    lo = None if box_lo is None else _dev_f64(box_lo, "box_lo")
    hi = None if box_hi is None else _dev_f64(box_hi, "box_hi")
    ns = len(sizes)
    offs = (ctypes.c_int64 * (ns + 1))()
    acc = 0
    for i, s_ in enumerate(sizes):
        offs[i] = acc
        acc += int(s_)
    offs[ns] = acc
    dims_c = (ctypes.c_int32 * ns)(*[int(v) for v in dims])
    ps = (HawkesParams * ns)(*[params_struct(p) for p in params_list])
    eps_c = (ctypes.c_double * ns)(*[float(v) for v in eps])
    log_u = _dev_f64(log_u, "log_u")
    H0 = torch.empty(ns, dtype=torch.float64, device=t.device)
    H1 = torch.empty(ns, dtype=torch.float64, device=t.device)
    accd = torch.empty(ns, dtype=torch.int32, device=t.device)
    ctx.check(ctx.lib.hawkes_batch_hmc_trajectory(ctx.handle, ns, offs, dims_c, _ptr(t), _ptr(X), _ptr(p0), _ptr(lo),
                                                  _ptr(hi), ps, eps_c, int(n_steps), _ptr(log_u),
                                                  _precision(precision), ctx.stream(), _ptr(H0), _ptr(H1),
                                                  _ptr(accd)))
    if check:
        ctx.sync_status()
    return H0, H1, accd


def version() -> str:
    return _lib.load().hawkes_version().decode()


class HawkesMwG:
    """Incremental Metropolis-within-Gibbs state over the event locations
    (hawkes_mwg_* in the C ABI): FP64 rates cached on the device, block moves
    evaluated in O(|B| N), accept and commit on the device.  precision
    "fp64" (default) evaluates the pair terms in FP64, "mixed" in FP32 with
    FP64 logs, rates and decisions."""

    def __init__(self, t, X, params, max_block: int = 64, device: int | None = None, precision: str = "fp64"):
        self.lib = _lib.load()
        t = _dev_f64(t, "t")
        X = _dev_f64(X, "X")
        n, d, X = _shape(t, X)
        self.n, self.d = n, d
        self.device = t.device.index if device is None else int(device)
        self.max_block = int(max_block)
        p = params_struct(params)
        h = ctypes.c_void_p()
        st = self.lib.hawkes_mwg_create(self.device, _ptr(t), _ptr(X), n, d, ctypes.byref(p), self.max_block,
                                        self.stream(), ctypes.byref(h))
        if st != 0:
            raise HawkesError(st, "hawkes_mwg_create failed")
        self.handle = h
        self._dev = t.device
        if precision != "fp64":
            self.set_precision(precision)

    def stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def check(self, status: int):
        if status != 0:
            raise HawkesError(status, self.lib.hawkes_mwg_last_error(self.handle).decode())

    def set_precision(self, precision: str):
        """Precision of the pair terms of later calls ("mixed" or "fp64")."""
        self.check(self.lib.hawkes_mwg_set_precision(self.handle, _precision(precision), self.stream()))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.hawkes_mwg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync_status(self):
        self.check(self.lib.hawkes_mwg_sync_status(self.handle, self.stream()))

    def _block(self, idx, X_new):
        idx = torch.as_tensor(idx, dtype=torch.int64, device=self._dev).contiguous()
        X_new = torch.as_tensor(X_new, dtype=torch.float64, device=self._dev).reshape(-1, self.d).contiguous()
        if X_new.shape[0] != idx.numel():
            raise ValueError("X_new must have one row per index")
        return idx, X_new

    def delta(self, idx, X_new, out=None, check: bool = True):
        """Delta ell of moving events idx to X_new (device tensor, state unchanged)."""
        idx, X_new = self._block(idx, X_new)
        out = torch.empty((), dtype=torch.float64, device=self._dev) if out is None else out
        self.check(self.lib.hawkes_mwg_delta(self.handle, idx.numel(), _ptr(idx), _ptr(X_new), self.stream(),
                                             _ptr(out)))
        if check:
            self.sync_status()
        return out

    def step(self, idx, X_new, log_u, log_q_ratio=None, out=None, check: bool = True):
        """One Metropolis-Hastings step; returns (Delta ell, accepted) as device tensors."""
        idx, X_new = self._block(idx, X_new)
        if not isinstance(log_u, torch.Tensor):
            log_u = torch.tensor(float(log_u), dtype=torch.float64, device=self._dev)
        if log_q_ratio is not None and not isinstance(log_q_ratio, torch.Tensor):
            log_q_ratio = torch.tensor(float(log_q_ratio), dtype=torch.float64, device=self._dev)
        if out is None:
            out = (torch.empty((), dtype=torch.float64, device=self._dev),
                   torch.empty((), dtype=torch.int32, device=self._dev))
        self.check(self.lib.hawkes_mwg_step(self.handle, idx.numel(), _ptr(idx), _ptr(X_new), _ptr(log_q_ratio),
                                            _ptr(log_u), self.stream(), _ptr(out[0]), _ptr(out[1])))
        if check:
            self.sync_status()
        return out

    def propose_circle(self, idx, centers, radii, eps: float, tries: int, u, out=None, check: bool = True):
        """Lens proposals of Eq. (6) (D = 2): (X_new, log q-ratio) as device tensors.
        centers (N, 2) and radii (N,) cover every event; u has nb * tries * 2 uniforms."""
        idx = torch.as_tensor(idx, dtype=torch.int64, device=self._dev).contiguous()
        centers = _dev_f64(torch.as_tensor(centers, dtype=torch.float64, device=self._dev), "centers")
        radii = _dev_f64(torch.as_tensor(radii, dtype=torch.float64, device=self._dev), "radii")
        u = _dev_f64(torch.as_tensor(u, dtype=torch.float64, device=self._dev), "u")
        nb = idx.numel()
        if out is None:
            out = (torch.empty((nb, self.d), dtype=torch.float64, device=self._dev),
                   torch.empty((), dtype=torch.float64, device=self._dev))
        self.check(self.lib.hawkes_mwg_propose_circle(self.handle, nb, _ptr(idx), _ptr(centers), _ptr(radii),
                                                      float(eps), int(tries), _ptr(u), self.stream(), _ptr(out[0]),
                                                      _ptr(out[1])))
        if check:
            self.sync_status()
        return out

    def propose_box(self, idx, lo, hi, sd: float, u, out=None, check: bool = True):
        """Truncated-normal proposals inside the boxes of Eq. (2): (X_new, log q-ratio)."""
        idx = torch.as_tensor(idx, dtype=torch.int64, device=self._dev).contiguous()
        lo = _dev_f64(torch.as_tensor(lo, dtype=torch.float64, device=self._dev), "lo")
        hi = _dev_f64(torch.as_tensor(hi, dtype=torch.float64, device=self._dev), "hi")
        u = _dev_f64(torch.as_tensor(u, dtype=torch.float64, device=self._dev), "u")
        nb = idx.numel()
        if out is None:
            out = (torch.empty((nb, self.d), dtype=torch.float64, device=self._dev),
                   torch.empty((), dtype=torch.float64, device=self._dev))
        self.check(self.lib.hawkes_mwg_propose_box(self.handle, nb, _ptr(idx), _ptr(lo), _ptr(hi), float(sd),
                                                   _ptr(u), self.stream(), _ptr(out[0]), _ptr(out[1])))
        if check:
            self.sync_status()
        return out

    def refresh(self):
        self.check(self.lib.hawkes_mwg_refresh(self.handle, self.stream()))

    def read(self):
        """(X, lambda, ell) of the current state as device tensors."""
        X = torch.empty((self.n, self.d), dtype=torch.float64, device=self._dev)
        lam = torch.empty(self.n, dtype=torch.float64, device=self._dev)
        ell = torch.empty((), dtype=torch.float64, device=self._dev)
        self.check(self.lib.hawkes_mwg_read(self.handle, self.stream(), _ptr(X), _ptr(lam), _ptr(ell)))
        return X, lam, ell
