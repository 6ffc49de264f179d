"""Branch connection of an energy scan (paper_1709_09347_gb300.scan.connect) on a closed
form: the order-2 FD free electron along z, where each transverse mode of energy eps gives
cos(theta) = 1 - h^2 (E - eps) and the two Bloch factors lambda = exp(+-i nz theta(E)),
with known branch labels (mode, sign).  Propagating branches of different modes cross on the
unit circle and each mode's pair meets at its band edge, so the test checks that every
point lands in exactly one branch and that a branch changes label only where two labels
meet."""
import numpy as np

from paper_1709_09347_gb300 import scan


def _closed_form(eps_list, energies, h=0.4, nz=4, lambda_min=0.5):
    per_e = []
    for E in energies:
        pts = []
        for i, eps in enumerate(eps_list):
            th = np.arccos(complex(1 - h * h * (E - eps)))
            for sgn in (1, -1):
                lam = np.exp(1j * sgn * nz * th)
                if lambda_min < abs(lam) < 1 / lambda_min:
                    pts.append((lam, (i, sgn)))
        per_e.append(pts)
    return per_e


def test_connect_recovers_closed_form_branches():
    energies = np.arange(0.05, 4.0, 0.02)
    eps_list = [0.0, 0.9, 2.3]
    data = _closed_form(eps_list, energies)
    rng = np.random.default_rng(0)
    lams, labels = [], []
    for pts in data:
        order = rng.permutation(len(pts))
        lams.append(np.array([pts[o][0] for o in order]))
        labels.append([pts[o][1] for o in order])
    branches = scan.connect(lams, max_jump=0.6)
    # every point in exactly one branch
    seen = set()
    for b in branches:
        for e, lam in zip(b.energy_index, b.lam):
            k = int(np.argmin(np.abs(lams[e] - lam)))
            assert (e, k) not in seen
            seen.add((e, k))
    assert len(seen) == sum(len(x) for x in lams)
    # labels: a branch keeps its label except where the two labels involved meet
    pairs = changes = 0
    for b in branches:
        idx = [int(np.argmin(np.abs(lams[e] - lam))) for e, lam in zip(b.energy_index, b.lam)]
        for (e0, k0), (e1, k1) in zip(zip(b.energy_index, idx), zip(b.energy_index[1:], idx[1:])):
            assert e1 == e0 + 1
            pairs += 1
            if labels[e0][k0] != labels[e1][k1]:
                changes += 1
                # the branch's label A and the label B it moved to must meet there: within
                # one step of each other at e0 or at e1 (a crossing, or a band edge where a
                # mode's evanescent pair lambda, 1/lambda turns into the propagating pair,
                # a square-root branch point at which either pairing continues analytically)
                A, B = labels[e0][k0], labels[e1][k1]
                gap = []
                for e in (e0, e1):
                    pa = [lams[e][j] for j, lab in enumerate(labels[e]) if lab == A]
                    pb = [lams[e][j] for j, lab in enumerate(labels[e]) if lab == B]
                    if pa and pb:
                        gap.append(abs(pa[0] - pb[0]))
                assert gap and min(gap) < 0.5, (e0, A, B, gap)
    assert changes <= 0.02 * pairs


def test_phase_distance_wraps():
    a = np.pi - 0.01
    b = -np.pi + 0.01
    assert abs(scan.phase_distance(a, b) - 0.02) < 1e-12
    assert abs(scan.phase_distance(0.3 + 0.2j, 0.3 - 0.1j) - 0.3) < 1e-12
