"""Table and coefficients of the FP64 base-2 exponential of the symmetric FP64
pair kernels (hk_pairs_fp64_sym.cu).

The kernels evaluate 2^y for y <= 0 by Tang's table-driven method
(P. T. P. Tang, "Table-driven implementation of the exponential function in
IEEE floating-point arithmetic", ACM TOMS 15(2), 1989), in base 2:

    y = (j + 2048 k) / 2048 + f,  j in [0, 2048), |f| <= 2^-12
    2^y = 2^k * T[j] * (1 + q(f)),  T[j] = 2^(j/2048),
    q(f) = 2^f - 1 = sum_{m >= 1} (f ln 2)^m / m!  cut after m = 3.

The table entries are 2^(j/2048) rounded to the nearest double; the
coefficients are (ln 2)^m / m!, also rounded to the nearest double.  Both come
from 60-digit decimal arithmetic.  The truncation error of q is below
(2^-12 ln 2)^4 / 4! < 3.5e-17, under a sixth of an ulp of T[j] (1 + q).

Run:  python gen_exp2_table.py > hk_exp2_table.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 60
TABLE = 2048
DEGREE = 3


def main() -> None:
    ln2 = Decimal(2).ln()
    lines = [
        f"// Written by gen_exp2_table.py beside this file: 2^(j/{TABLE}) for j = 0..{TABLE - 1}",
        "// and the Taylor coefficients (ln 2)^m / m! of 2^f - 1, each rounded to the",
        "// nearest double from 60-digit decimal arithmetic.",
        "#pragma once",
        "",
        "namespace hk {",
        "",
        f"constexpr int kExp2TabSize = {TABLE};",
        "// Global memory (not const, so not the constant bank): lanes read it",
        "// with different indices.",
        f"static __device__ double kExp2Tab[{TABLE}] = {{",
    ]
    for j0 in range(0, TABLE, 4):
        vals = [float((ln2 * j / TABLE).exp()).hex() for j in range(j0, j0 + 4)]
        lines.append("    " + ", ".join(vals) + ",")
    lines.append("};")
    fact = 1
    for m in range(1, DEGREE + 1):
        fact *= m
        c = float(ln2 ** m / fact)
        lines.append(f"constexpr double kExp2C{m} = {c.hex()};  // (ln 2)^{m} / {m}!")
    lines += ["", "}  // namespace hk", ""]
    print("\n".join(lines))


if __name__ == "__main__":
    main()
