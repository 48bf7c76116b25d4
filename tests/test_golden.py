"""Values the paper prints, read from tests/golden/ (each fixture cites its
passage) and checked against the oracle."""
import os

import numpy as np

from oracle import quadrature as oq

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_fixture(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                key, val = line.split(None, 1)
                vals[key] = val
    return vals


def test_sec5_1_rule_has_the_printed_node():
    """Sec. 5.1: the 45-node Gauss-Chebyshev rule after x = (1-t)/(1+t) has a
    node at 3.05e-4 (three significant digits).  A wrong node family (second
    kind, Gauss-Legendre), a wrong map or a wrong node count misses it."""
    g = read_fixture("sec5_1_quadrature_node.txt")
    t, _ = oq.rule(g["func"], int(g["ell"]), float(g["c"]))
    node = float(g["node"])
    half_ulp = 0.5 * 10.0 ** (np.floor(np.log10(node)) - (int(g["significant_digits"]) - 1))
    assert len(t) == int(g["ell"])
    assert np.min(np.abs(np.asarray(t) - node)) <= half_ulp
