"""Energy scans: the complex band structure k(E) over a grid of energies, joined into branches.

A complex-band-structure plot (the paper's §4 figures) is the set of Bloch factors
lambda(E) = exp(i k(E) a) in the ring lambda_min < |lambda| < 1/lambda_min over a dense list of
energies.  `scan` solves the energies in batches through `cbs.solve` (by default with the
shifted family, one Krylov sequence per quadrature point for a whole batch), and `connect`
joins the eigenvalues of neighbouring energies into branches.

Joining: k is compared in the cell-phase form a*k = arg(lambda) - i ln|lambda|, with arg
taken modulo 2 pi.  Each open branch predicts its next value by linear extrapolation of its
last two points (its last point if it has one), and the eigenvalues of the next energy are
assigned to open branches by minimum total distance to the predictions (linear assignment);
an assignment farther than `max_jump` is refused.  Unassigned eigenvalues start branches,
unassigned branches end.  Using the extrapolated value lets two branches that cross (two
propagating bands meeting on the unit circle) keep their slopes instead of swapping.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def phase_distance(ka1, ka2):
    """|a k1 - a k2| with the real part (arg lambda) compared modulo 2 pi."""
    d = np.asarray(ka1) - np.asarray(ka2)
    re = (d.real + np.pi) % (2 * np.pi) - np.pi
    return np.hypot(re, d.imag)


def cell_phase(lam):
    """a k = arg(lambda) - i ln|lambda| (the branch with arg in (-pi, pi])."""
    lam = np.asarray(lam, complex)
    return np.angle(lam) - 1j * np.log(np.abs(lam))


@dataclass
class Branch:
    """One connected branch: energy indices (increasing) and the eigenvalues there."""
    energy_index: list = field(default_factory=list)
    lam: list = field(default_factory=list)

    def ka(self):
        return cell_phase(np.array(self.lam))

    def predict(self):
        ka = cell_phase(np.array(self.lam[-2:]))
        if len(ka) == 1:
            return ka[0]
        step = ka[1] - ka[0]
        step = complex((step.real + np.pi) % (2 * np.pi) - np.pi, step.imag)
        return ka[1] + step


def connect(lams, max_jump):
    """Join per-energy eigenvalue lists (lams[e] = array of lambda at energy e, energies in
    increasing order) into branches; returns the list of Branch objects.  Every eigenvalue
    belongs to exactly one branch."""
    from scipy.optimize import linear_sum_assignment

    done, open_ = [], []
    for e, lam in enumerate(lams):
        lam = np.asarray(lam, complex)
        ka = cell_phase(lam)
        taken = np.zeros(len(lam), bool)
        keep = []
        if open_ and len(lam):
            pred = np.array([b.predict() for b in open_])
            last = np.array([cell_phase(b.lam[-1]) for b in open_])
            # distance to the extrapolated value, and no farther than max_jump from the
            # branch's last point
            cost = phase_distance(pred[:, None], ka[None, :])
            far = phase_distance(last[:, None], ka[None, :]) > max_jump
            big = 1e6 * (1 + cost.max())
            cost = np.where(far, big, cost)
            rows, cols = linear_sum_assignment(cost)
            for r, c in zip(rows, cols):
                if cost[r, c] < big:
                    open_[r].energy_index.append(e)
                    open_[r].lam.append(lam[c])
                    taken[c] = True
                    keep.append(r)
        kept = set(keep)
        for i, b in enumerate(open_):
            if i not in kept:
                done.append(b)
        open_ = [open_[i] for i in sorted(kept)]
        for c in np.nonzero(~taken)[0]:
            open_.append(Branch([e], [lam[c]]))
    return done + open_


def scan(H, energies, lambda_min, n_int, L, M, V, opts=None, batch=16):
    """Solve every energy (ascending order is assumed by `connect`) in batches of `batch`
    through cbs.solve; returns per-energy dicts with lam, k, residual (and vectors)."""
    from . import cbs

    if opts is None:
        opts = cbs.options(multi_shift=1)
    out = []
    energies = np.asarray(energies, float)
    for i in range(0, len(energies), batch):
        res = cbs.solve(H, energies[i:i + batch], lambda_min, n_int, L, M, V, opts)
        out.extend(res.energies)
    return out
