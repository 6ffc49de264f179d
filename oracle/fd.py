"""Central finite-difference weights for the second derivative (oracle).

The paper discretises the Laplacian with a "nine-point" central finite difference
(§4), i.e. order 8 with half-width m = 4.  Here the weights c_0..c_m of

    f''(0) ~ (1/h^2) [ c_0 f(0) + sum_{k=1..m} c_k (f(kh) + f(-kh)) ]

are obtained by requiring exactness on the even monomials x^0, x^2, ..., x^{2m},
solved in exact rational arithmetic (Gaussian elimination on Fractions).

Pins (tests/test_oracle_fd.py): tabulated weights for orders 2, 4, 6, 8; exactness on
x^{2j}; the symbol -(c_0 + 2 sum c_k cos(k t)) = t^2 + O(t^{2m+2}).
"""
from __future__ import annotations

from fractions import Fraction


def fd_weights(order: int) -> list[Fraction]:
    """Return [c_0, c_1, ..., c_m] for a central second-derivative of the given even order."""
    if order < 2 or order % 2:
        raise ValueError("order must be an even integer >= 2")
    m = order // 2
    # unknowns c_0..c_m; equation j (j = 0..m): sum over the stencil of c * x^{2j} / h^2
    # equals d^2/dx^2 x^{2j} at 0, which is 2 for j = 1 and 0 otherwise.
    rows = []
    for j in range(m + 1):
        row = [Fraction(1 if j == 0 else 0)]               # c_0 * 0^{2j}
        row += [Fraction(2 * k ** (2 * j)) for k in range(1, m + 1)]
        rhs = Fraction(2 if j == 1 else 0)
        rows.append(row + [rhs])
    n = m + 1
    for col in range(n):
        piv = next(r for r in range(col, n) if rows[r][col] != 0)
        rows[col], rows[piv] = rows[piv], rows[col]
        p = rows[col][col]
        rows[col] = [v / p for v in rows[col]]
        for r in range(n):
            if r != col and rows[r][col] != 0:
                f = rows[r][col]
                rows[r] = [a - f * b for a, b in zip(rows[r], rows[col])]
    return [rows[i][n] for i in range(n)]


def fd_weights_float(order: int) -> list[float]:
    return [float(c) for c in fd_weights(order)]
