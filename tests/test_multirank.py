"""Splitting the work across ranks (CPU, gloo, world size 2): energy shares, quadrature-point
shares, and the sum reduction of partial moments, which must equal the moments of all points
(Algorithm 1, first step, summed over the ring of §3.2)."""
import os
import socket

import numpy as np
import pytest

from paper_1709_09347_gb300 import shard


def test_block_range_covers_once():
    for n in (0, 1, 5, 16, 33):
        for world in (1, 2, 3, 8):
            got = [i for r in range(world) for i in shard.block_range(n, r, world)]
            assert got == list(range(n))
            sizes = [len(shard.block_range(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.block_range(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import scipy.sparse.linalg as spla
    import torch
    import torch.distributed as dist

    from oracle import ss
    from oracle.contour import ring_contour
    from oracle.operator import CellOperator
    from paper_1709_09347_gb300 import synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = synth.tiny_workload(nx=5, ny=4, nz=4, h=0.45, fd_order=4, n_atoms=1, r_c=0.8, sigma=0.3,
                             L=3, M=2, n_int=8, energies=(0.2,))
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    E = float(wl.energies[0])
    z1, _, _, _ = ring_contour(wl.lambda_min, wl.n_int)
    N, L = wl.V.shape
    Y1 = np.zeros((wl.n_int, N, L), complex)
    Y2 = np.zeros((wl.n_int, N, L), complex)
    for j in shard.points_for_rank(wl.n_int, rank, world):
        P = op.P_matrix(z1[j], E).tocsc()
        Y1[j] = spla.spsolve(P, wl.V)
        Y2[j] = spla.spsolve(P.conj().T.tocsc(), wl.V)     # P(z1)^dagger = P(z2)
    S, mu = ss.moments(Y1, Y2, wl.lambda_min, wl.n_int, wl.V, wl.M)
    St, mut = torch.from_numpy(S), torch.from_numpy(mu)
    shard.reduce_moments(St, mut)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), S=St.numpy(), mu=mut.numpy())
    dist.destroy_process_group()


def test_moment_reduction_two_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import scipy.sparse.linalg as spla

    from oracle import ss
    from oracle.contour import ring_contour
    from oracle.operator import CellOperator
    from paper_1709_09347_gb300 import synth

    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    wl = synth.tiny_workload(nx=5, ny=4, nz=4, h=0.45, fd_order=4, n_atoms=1, r_c=0.8, sigma=0.3,
                             L=3, M=2, n_int=8, energies=(0.2,))
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    E = float(wl.energies[0])
    z1, _, _, _ = ring_contour(wl.lambda_min, wl.n_int)
    Y1 = np.stack([spla.spsolve(op.P_matrix(z, E).tocsc(), wl.V) for z in z1])
    Y2 = np.stack([spla.spsolve(op.P_matrix(z, E).conj().T.tocsc(), wl.V) for z in z1])
    S, mu = ss.moments(Y1, Y2, wl.lambda_min, wl.n_int, wl.V, wl.M)
    for r in range(2):
        got = np.load(tmp_path / f"rank{r}.npz")
        assert np.allclose(got["S"], S, rtol=1e-12, atol=1e-12 * np.abs(S).max())
        assert np.allclose(got["mu"], mu, rtol=1e-12, atol=1e-12 * np.abs(mu).max())


def test_energy_shares():
    E = list(np.linspace(-0.5, 0.5, 16))
    parts = [shard.energies_for_rank(E, r, 3) for r in range(3)]
    assert sum(parts, []) == E
