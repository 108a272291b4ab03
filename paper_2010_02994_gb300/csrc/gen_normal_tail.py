"""Fit of the scaled normal tail used by the FP32 BMDS pair kernels.

For z >= 0 the kernels need the standard normal tail Q(z) = 1 - Phi(z), the
CDF Phi(z) and phi(z) / Phi(z).  They compute exp(-z^2 / 2) with the hardware
exp2 and the smooth, bounded factor

    g(z) = Q(z) exp(z^2 / 2)        (g(0) = 1/2, g(z) ~ 1 / (z sqrt(2 pi)))

as a rational function P(z) / B(z) with deg P = 4, deg B = 5 (so P / B keeps
the 1/z decay) and B(0) = 1.  The fit is linearised least squares
(P - g B = 0, weighted by 1 / (g B_prev), iterated as in Loeb's method) with
Lawson's reweighting towards the minimax relative error, on [0, 14]: beyond
z = 14, exp(-z^2 / 2) is below the FP32 range and the kernels evaluate P / B
at min(z, 14).  The target g comes from scipy.special.erfcx.

Run:  python gen_normal_tail.py   (prints the FP32 coefficients and the
maximum relative error in exact arithmetic and in FP32 Horner evaluation
with fused multiply-adds).
"""
import numpy as np
from scipy.special import erfcx

DEG_P = 4
Z_MAX = 14.0


def target(z):
    return 0.5 * erfcx(z / np.sqrt(2.0))


def fit(deg_p=DEG_P, z_max=Z_MAX, iters=60):
    z = np.concatenate([np.linspace(0.0, 2.0, 4000), np.linspace(2.0, z_max, 12000)])
    y = target(z)
    deg_b = deg_p + 1
    VP = np.vander(z, deg_p + 1, increasing=True)
    VB = np.vander(z, deg_b + 1, increasing=True)[:, 1:]
    A = np.hstack([VP, -(y[:, None] * VB)])
    b_prev = np.ones_like(z)
    lawson = np.ones_like(z)
    best = None
    for _ in range(iters):
        w = np.sqrt(lawson) / (y * b_prev)
        sol, *_ = np.linalg.lstsq(A * w[:, None], y * w, rcond=None)
        p = sol[:deg_p + 1]
        b = np.concatenate([[1.0], sol[deg_p + 1:]])
        P = VP @ p
        B = np.concatenate([np.ones((len(z), 1)), VB], axis=1) @ b
        rel = (P / B - y) / y
        err = float(np.max(np.abs(rel)))
        if best is None or err < best[0]:
            best = (err, p.copy(), b.copy())
        b_prev = np.abs(B)
        lawson = lawson * (np.abs(rel) + 1e-30)
        lawson /= lawson.sum()
    return best


def fp32_horner_error(p, b, z_max=Z_MAX):
    """Max relative error of P / B evaluated with FP32 coefficients and one
    rounding per Horner step (a fused multiply-add)."""
    z = np.linspace(0.0, z_max, 400001).astype(np.float32).astype(np.float64)

    def horner(c):
        acc = np.zeros_like(z)
        for ck in np.asarray(c, dtype=np.float32).astype(np.float64)[::-1]:
            acc = (acc * z + ck).astype(np.float32).astype(np.float64)
        return acc

    return float(np.max(np.abs(horner(p) / horner(b) / target(z) - 1.0)))


def main():
    err, p, b = fit()
    print(f"max relative error, exact arithmetic: {err:.3e}")
    print(f"max relative error, FP32 Horner:      {fp32_horner_error(p, b):.3e}")
    print("P:", ", ".join(repr(float(np.float32(c))) for c in p))
    print("B:", ", ".join(repr(float(np.float32(c))) for c in b))


if __name__ == "__main__":
    main()
