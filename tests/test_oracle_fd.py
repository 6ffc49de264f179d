"""Pins for the oracle's FD weights (paper §4: nine-point central FD Laplacian)."""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

from oracle.fd import fd_weights

# Tabulated central second-derivative weights (Fornberg, Math. Comp. 51 (1988), Table 1).
TABLE = {
    2: ["-2", "1"],
    4: ["-5/2", "4/3", "-1/12"],
    6: ["-49/18", "3/2", "-3/20", "1/90"],
    8: ["-205/72", "8/5", "-1/5", "8/315", "-1/560"],
}


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_table(order):
    assert fd_weights(order) == [Fraction(s) for s in TABLE[order]]


@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12])
def test_closed_form(order):
    # c_k = 2 (-1)^{k+1} (m!)^2 / (k^2 (m-k)! (m+k)!),  c_0 = -2 sum c_k
    m = order // 2
    ck = [Fraction(2 * (-1) ** (k + 1) * factorial(m) ** 2, k * k * factorial(m - k) * factorial(m + k))
          for k in range(1, m + 1)]
    c0 = -2 * sum(ck)
    assert fd_weights(order) == [c0] + ck


@pytest.mark.parametrize("order", [4, 8])
def test_symbol(order):
    # -(c0 + 2 sum c_k cos(k t)) = t^2 + O(t^{order+2})
    c = [float(x) for x in fd_weights(order)]
    for t in (0.05, 0.1):
        sym = -(c[0] + 2 * sum(c[k] * np.cos(k * t) for k in range(1, len(c))))
        assert abs(sym - t * t) < 10 * t ** (order + 2)
