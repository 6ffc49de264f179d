"""Write oracle eigenvalues for the 32x32x16 workload at three energies.

Runs only the CPU oracle (oracle/) on the seeded synthetic inputs and stores, per
energy, the kept eigenvalues of Algorithm 1 (BiCG to 1e-12), their residuals, the
numerical rank and the BiCG iteration counts, and the same eigenvalues refined to
rounding level by residual inverse iteration on Eq. (4) (oracle/polish.py), in
tests/golden/c2_oracle.npz.  Energy index 3 is one where the Hankel rank reaches
L*M = 256 (rank saturation), kept to check the count there.  The quadrature points are
solved in parallel worker processes (spawned); a few minutes per energy on 8 cores, plus
about a minute per kept eigenvalue for the dense LU of the refinement.

    python tests/golden/make_c2_oracle.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import polish, ss  # noqa: E402
from oracle.operator import CellOperator  # noqa: E402
from paper_1709_09347_gb300 import synth  # noqa: E402

ENERGY_INDEX = (3, 7, 12)
# BiCG tolerance of the stored run: the eigenvalue error of the method follows the solve
# error, so a 1e-10 comparison of eigenvalues needs both sides solved to 1e-12
TOL = 1e-12


def main():
    import concurrent.futures as cf
    import multiprocessing as mp
    # one BLAS thread in each spawned solver process (they read the variable when they
    # start); this process loaded its BLAS at import and keeps all threads for the dense LU
    # of the refinement, unless the calling shell limited them
    os.environ["OMP_NUM_THREADS"] = "1"
    pool = cf.ProcessPoolExecutor(max_workers=os.cpu_count(), mp_context=mp.get_context("spawn"))
    wl = synth.workload("c2")
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    out = {"energy_index": np.array(ENERGY_INDEX), "energies": wl.energies[list(ENERGY_INDEX)],
           "tol": np.array(TOL)}
    runs = {}
    for e in ENERGY_INDEX:
        E = float(wl.energies[e])
        t = time.time()
        r = ss.ss_hankel(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, delta=wl.delta, tol=TOL,
                         pool=pool)
        print(f"E={E:+.4f}: {len(r.lam)} kept, rank {r.rank}, iters {r.iters.max()}, "
              f"{time.time() - t:.0f} s", flush=True)
        runs[e] = r
        out[f"lam_{e}"] = r.lam
        out[f"res_{e}"] = r.residual
        out[f"rank_{e}"] = np.array(r.rank)
        out[f"iters_{e}"] = r.iters
    pool.shutdown()
    for e in ENERGY_INDEX:
        r = runs[e]
        E = float(wl.energies[e])
        t = time.time()
        if len(r.lam):
            lp, _, rp = polish.polish(op, E, r.lam, r.vectors)
        else:
            lp, rp = np.zeros(0, complex), np.zeros(0)
        print(f"E={E:+.4f}: polished {len(lp)}, max change "
              f"{np.max(np.abs(lp - r.lam) / np.abs(lp)) if len(lp) else 0:.2e}, "
              f"max residual {rp.max() if len(rp) else 0:.1e}, {time.time() - t:.0f} s", flush=True)
        out[f"lam_polished_{e}"] = lp
        out[f"res_polished_{e}"] = rp
    np.savez(os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_oracle.npz"), **out)


if __name__ == "__main__":
    main()
