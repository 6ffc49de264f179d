"""Write oracle results for the 64x64x24 workload (120 atoms, N_int = 64, L = 32, M = 8,
lambda_min = 0.3) at selected energies.

Runs only the CPU oracle (oracle/) on the seeded synthetic inputs: Algorithm 1 with the
paper's BiCG tolerance 1e-10 (§4.1), primal and dual solves at the 64 outer-circle points
in parallel worker processes (spawned).  Per energy it stores, in
tests/golden/c3_oracle_e<index>.npz, the kept eigenvalues, their residuals, the numerical
rank, the singular values' extremes and the BiCG iteration counts.  Cost grows steeply with
the energy (about 200 BiCG iterations per point at E = -0.5 Ha, about 2000 at +0.18 Ha, at
roughly 0.7 s per iteration and point on one core): energy index 0 takes about twenty
minutes on 8 cores, index 21 a few hours.

    python tests/golden/make_c3_oracle.py [energy_index ...]     (default: 0)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ss  # noqa: E402
from oracle.operator import CellOperator  # noqa: E402
from paper_1709_09347_gb300 import synth  # noqa: E402

TOL = 1e-10


def main(indices):
    import concurrent.futures as cf
    import multiprocessing as mp
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    pool = cf.ProcessPoolExecutor(max_workers=os.cpu_count(), mp_context=mp.get_context("spawn"))
    wl = synth.workload("c3")
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    for e in indices:
        E = float(wl.energies[e])
        t = time.time()
        r = ss.ss_hankel(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, delta=wl.delta, tol=TOL,
                         pool=pool)
        print(f"E={E:+.4f}: {len(r.lam)} kept, rank {r.rank}, iters {r.iters.max()}, "
              f"{time.time() - t:.0f} s", flush=True)
        np.savez(os.path.join(os.path.dirname(os.path.abspath(__file__)), f"c3_oracle_e{e:02d}.npz"),
                 energy_index=np.array(e), energy=np.array(E), tol=np.array(TOL), lam=r.lam,
                 res=r.residual, rank=np.array(r.rank), sigma_max=np.array(r.sigma[0]),
                 sigma_cut=np.array(r.sigma[r.rank - 1] if r.rank else 0.0), iters=r.iters)
    pool.shutdown()


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [0])
