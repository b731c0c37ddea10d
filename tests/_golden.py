"""Loaders for the paper's printed values stored under tests/golden/."""
import os
from fractions import Fraction

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


def table(name):
    """Numeric rows; a leading non-numeric tag is kept as a string."""
    res = []
    for r in rows(name):
        vals = []
        for tok in r:
            try:
                vals.append(float(tok))
            except ValueError:
                vals.append(tok)
        res.append(vals)
    return res


def trace_polynomial():
    """{mu_power: (Fraction scale, {C_power: int coefficient})} of the Appendix."""
    poly = {}
    for r in rows("appendix_trace_polynomial.txt"):
        mu_pow, sign, den = int(r[0]), int(r[1]), int(r[2])
        coeffs = {}
        for tok in r[3:]:
            e, c = tok.split(":")
            coeffs[int(e)] = int(c)
        poly[mu_pow] = (Fraction(sign, den), coeffs)
    return poly


def eval_trace(C, mu):
    s = Fraction(0)
    Cf, muf = Fraction(C), Fraction(mu)
    for mp, (scale, coeffs) in trace_polynomial().items():
        s += scale * sum(Fraction(c) * Cf ** e for e, c in coeffs.items()) * muf ** mp
    return float(s)
