"""Readers of the paper-printed fixtures under tests/golden/ (each file
states the passage its values come from)."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line.split()


def legendre_polynomials():
    """{n: numpy.polynomial coefficients of P_n in ascending powers} (Appendix A)."""
    out = {}
    for row in _rows("legendre_polynomials.txt"):
        n, den = int(row[0]), float(row[1])
        num = [float(x) for x in row[2:]]
        assert len(num) == n + 1
        out[n] = np.array(num[::-1]) / den
    return out


def rk_tableaux():
    """{order: (A [s, s], b [s], c [s])} as printed in Appendix D."""
    out, cur = {}, None
    for row in _rows("ssp_rk_tableaux.txt"):
        if row[0] == "order":
            order, s = int(row[1]), int(row[3])
            cur = dict(order=order, s=s, rows=[], b=None)
            out[order] = cur
        elif row[0] == "b":
            cur["b"] = [float(Fraction(x)) for x in row[1:]]
        else:
            cur["rows"].append([float(Fraction(x)) for x in row])
    tabs = {}
    for order, t in out.items():
        s = t["s"]
        A, c = np.zeros((s, s)), np.zeros(s)
        assert len(t["rows"]) == s and len(t["b"]) == s
        for i, r in enumerate(t["rows"]):
            assert len(r) == i + 1
            c[i] = r[0]
            A[i, :i] = r[1:]
        tabs[order] = (A, np.array(t["b"]), c)
    return tabs


def validation_figures():
    """{key: value} of the figures the paper prints for its validation runs."""
    return {row[0]: float(row[1]) for row in _rows("validation_figures.txt")}


def lobatto_first_weight():
    """{k: first GLL weight} printed in Sec. 3.4."""
    return {int(row[0]): float(Fraction(row[1])) for row in _rows("lobatto_first_weight.txt")}
