"""Two-circle quadrature for the annulus lambda_min < |z| < 1/lambda_min (oracle).

Paper §3.2: the target region of Eq. (5) is a ring; the contour is the outer circle
Gamma_1 (radius 1/lambda_min) minus the inner circle Gamma_2 (radius lambda_min), each
sampled at N_int points

    z_j^(1) = lambda_min^{-1} exp(i theta_j),   z_j^(2) = lambda_min exp(i theta_j),
    theta_j = 2 pi (j - 1/2) / N_int,  j = 1..N_int.

Weights: the paper prints omega_j = exp(i theta_j)/N_int for both circles.  The
trapezoidal rule for (1/(2 pi i)) oint f(z) dz on |z| = rho, with dz = i z dtheta,
gives omega_j = z_j / N_int = rho exp(i theta_j) / N_int, i.e. the printed weight times
the radius.  Without the radius the two circles would be scaled differently and poles
inside the inner circle would leak into the moments, so this oracle uses
omega_j^(c) = z_j^(c) / N_int (the reading used throughout this project).

Pin (tests/test_oracle_ss.py): on a diagonal QEP the quadrature moments equal the
residue sum over the poles inside the ring to within the trapezoid error.
"""
from __future__ import annotations

import numpy as np


def ring_contour(lambda_min: float, n_int: int):
    """Return (z1, w1, z2, w2): points and weights of the outer and inner circles."""
    if not (0.0 < lambda_min < 1.0):
        raise ValueError("lambda_min must lie in (0, 1)")
    j = np.arange(1, n_int + 1)
    theta = 2.0 * np.pi * (j - 0.5) / n_int
    e = np.exp(1j * theta)
    z1 = e / lambda_min
    z2 = e * lambda_min
    return z1, z1 / n_int, z2, z2 / n_int
