"""Constants of the FP64 exponential used by the FP64 pair terms (Tang's
table-driven method in base 2): the committed table header must be what its
generator writes, every entry must be 2^(j/2048) rounded to the nearest
double, and the polynomial's coefficients and truncation bound must be those
of the Taylor series of 2^f - 1 on |f| <= 2^-12.  The checks use Python's
decimal arithmetic and read the header as text."""
import os
import re
import subprocess
import sys
from decimal import Decimal, getcontext
from fractions import Fraction

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2010_02994_gb300", "csrc")
HEADER = os.path.join(CSRC, "hk_exp2_table.h")


def header_values():
    text = open(HEADER).read()
    body = text[text.index("kExp2Tab[2048] = {"):text.index("};")]
    table = [float.fromhex(v) for v in re.findall(r"0x[0-9a-fA-F.]+p[+-]\d+", body)]
    coef = {int(m): float.fromhex(v) for m, v in re.findall(r"kExp2C(\d) = (0x[0-9a-fA-F.]+p[+-]\d+)", text)}
    return table, coef


def test_header_is_the_generators_output():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "gen_exp2_table.py")], capture_output=True, text=True,
                         check=True).stdout
    assert out == open(HEADER).read()


def test_table_entries_are_correctly_rounded():
    getcontext().prec = 50
    ln2 = Decimal(2).ln()
    table, _ = header_values()
    assert len(table) == 2048
    for j, v in enumerate(table):
        exact = (ln2 * j / 2048).exp()
        err = abs(Fraction(v) - Fraction(exact))
        ulp = Fraction(2) ** (-52)  # every entry lies in [1, 2)
        assert 1.0 <= v < 2.0
        assert err <= ulp / 2, (j, v)


def test_polynomial_coefficients_and_truncation():
    getcontext().prec = 50
    ln2 = Decimal(2).ln()
    _, coef = header_values()
    assert sorted(coef) == [1, 2, 3]
    fact = 1
    for m in range(1, 4):
        fact *= m
        exact = Fraction(ln2 ** m / fact)
        assert abs(Fraction(coef[m]) - exact) <= abs(exact) * Fraction(2) ** (-53)
    # the first omitted term bounds the truncation of q(f) = 2^f - 1 on |f| <= 2^-12
    f = Decimal(2) ** -12
    omitted = (f * ln2) ** 4 / 24
    assert omitted < Decimal("3.5e-17")
    # and q(f) itself at both ends of the range, against the exact 2^f - 1
    for x in (f, -f):
        q = sum(Decimal(coef[m]) * x ** m for m in range(1, 4))
        assert abs(q - ((x * ln2).exp() - 1)) < Decimal("3.6e-17")
