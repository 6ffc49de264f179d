"""Seeded synthetic inputs: unit cells, potentials, projector tables, right-hand sides.

This module only *generates inputs*; it holds none of the method's arithmetic (no
operator assembly, no contour, no solver).  Both the CUDA library and the CPU oracle
consume what it produces, so that the two sides see bit-identical inputs.

Physical picture (paper §2): a crystal is cut into unit cells along z; inside one
cell the Kohn-Sham Hamiltonian lives on an ``nx x ny x nz`` real-space grid that is
periodic in x and y (Gamma point only, paper §4) and couples to the two neighbouring
cells along z.  The paper's RSPACE potentials are not public, so every input here is
a seeded stand-in with the paper's structure:

* local potential = sum of Gaussian wells ``U_a exp(-|r-R_a|^2 / (2 w^2))`` summed over
  all periodic images of the cell (bulk crystal),
* separable non-local projectors per atom: a Gaussian radial part times real
  spherical harmonics with l <= 1 (s, p_x, p_y, p_z), hard cut at ``r_c``,
  discretely normalised, with a diagonal coupling block ``h_a``,
* the block ``V`` of right-hand sides: i.i.d. real Gaussians N(0, 1).  The blocks of the
  Hamiltonian are real, so with a real ``V`` the solutions at conjugate contour points are
  complex conjugates of each other, which the library uses to solve half the points.

Projector table format (consumed as-is by both sides):

* ``sup_ptr[n_atoms+1]``  offsets of each atom's support entries,
* ``sup_idx[nnz]``        grid index ``ix + nx*(iy + ny*iz)`` of the support point,
* ``sup_wrap[nnz]``       z-image ``m`` in {-1, 0, +1}: the support point belongs to
                          the copy of atom a displaced by ``m`` cells along z,
* ``sup_val[nnz, n_proj]`` projector values times ``sqrt(dV)``,
* ``h[n_atoms, n_proj, n_proj]`` symmetric coupling blocks.

A grid point carries at most one entry per atom; this needs ``2 r_c`` smaller than
each cell edge, which the generator checks.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Grid", "Projectors", "Workload",
    "gaussian_wells", "make_projectors", "random_rhs", "random_rhs_complex",
    "workload", "tiny_workload", "CONFIG_NAMES",
]


@dataclasses.dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    fd_order: int

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def cell(self) -> tuple[float, float, float]:
        return (self.nx * self.hx, self.ny * self.hy, self.nz * self.hz)

    @property
    def a(self) -> float:
        """Cell length along the transport axis z."""
        return self.nz * self.hz


@dataclasses.dataclass
class Projectors:
    n_atoms: int
    n_proj: int
    sup_ptr: np.ndarray   # int64 [n_atoms+1]
    sup_idx: np.ndarray   # int32 [nnz]
    sup_wrap: np.ndarray  # int8  [nnz]
    sup_val: np.ndarray   # float64 [nnz, n_proj]
    h: np.ndarray         # float64 [n_atoms, n_proj, n_proj]

    @property
    def nnz(self) -> int:
        return int(self.sup_ptr[-1])


@dataclasses.dataclass
class Workload:
    name: str
    grid: Grid
    vloc: np.ndarray               # float64 [N]
    projectors: Projectors | None
    energies: np.ndarray           # float64 [n_e]
    lambda_min: float
    n_int: int
    L: int
    M: int
    V: np.ndarray                  # complex128 [N, L]
    delta: float = 1e-10
    tol: float = 1e-10
    seed: int = 0
    notes: str = ""


def _axis_window(c: float, reach: float, h: float):
    """Unwrapped grid indices k with |k*h - c| < reach (k may fall outside the cell)."""
    lo = int(math.ceil((c - reach) / h))
    hi = int(math.floor((c + reach) / h))
    return np.arange(lo, hi + 1)


def gaussian_wells(g: Grid, centres: np.ndarray, depths: np.ndarray, width: float,
                   cutoff_widths: float = 7.0) -> np.ndarray:
    """Local potential: sum over atoms and all periodic images of Gaussian wells.

    Grid points are visited through unwrapped index windows around each centre, and
    folded back into the cell by ``k mod n``; this sums every periodic image whose
    tail reaches ``cutoff_widths * width``.
    """
    reach = cutoff_widths * width
    v = np.zeros((g.nz, g.ny, g.nx))
    for c, u in zip(np.asarray(centres, float), np.asarray(depths, float)):
        kx = _axis_window(c[0], reach, g.hx)
        ky = _axis_window(c[1], reach, g.hy)
        kz = _axis_window(c[2], reach, g.hz)
        dx2 = (kx * g.hx - c[0]) ** 2
        dy2 = (ky * g.hy - c[1]) ** 2
        dz2 = (kz * g.hz - c[2]) ** 2
        d2 = dz2[:, None, None] + dy2[None, :, None] + dx2[None, None, :]
        val = np.where(d2 < reach * reach, u * np.exp(-d2 / (2.0 * width * width)), 0.0)
        np.add.at(v, np.ix_(kz % g.nz, ky % g.ny, kx % g.nx), val)
    return v.ravel()


def make_projectors(g: Grid, centres: np.ndarray, r_c: float = 2.0, sigma: float = 0.5,
                    h_s: float = 0.5, h_p: float = 0.25) -> Projectors:
    """Gaussian x real-Y_lm (l<=1) projectors, hard cut at r_c, sum(p^2 dV) = 1.

    The wrap tag of a support point is the z-image m of the atom copy that covers it:
    the point sits at ``r_i = R_a + m*a*z_hat + d`` with ``|d| < r_c``.
    """
    lx, ly, lz = g.cell
    if not (2 * r_c < lz and 2 * r_c < lx and 2 * r_c < ly):
        raise ValueError("projector support 2*r_c must be shorter than every cell edge")
    dv = g.hx * g.hy * g.hz
    n_proj = 4
    ptr = [0]
    idx_l, wrap_l, val_l = [], [], []
    for c in np.asarray(centres, float):
        kx = _axis_window(c[0], r_c, g.hx)
        ky = _axis_window(c[1], r_c, g.hy)
        kz = _axis_window(c[2], r_c, g.hz)
        KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
        d = np.stack([KX * g.hx - c[0], KY * g.hy - c[1], KZ * g.hz - c[2]], axis=-1).reshape(-1, 3)
        KX, KY, KZ = KX.ravel(), KY.ravel(), KZ.ravel()
        d2 = np.sum(d * d, axis=1)
        sel = d2 < r_c * r_c
        d, KX, KY, KZ, d2 = d[sel], KX[sel], KY[sel], KZ[sel], d2[sel]
        idx = (KX % g.nx) + g.nx * ((KY % g.ny) + g.ny * (KZ % g.nz))
        # unwrapped z index KZ = iz + nz*q  =>  r_i = KZ*h - q*a, atom copy at R_a - q*a
        wrap = -np.floor_divide(KZ, g.nz)
        order = np.argsort(idx, kind="stable")
        idx, wrap, d, d2 = idx[order], wrap[order], d[order], d2[order]
        if np.any(np.diff(idx) == 0):
            raise ValueError("grid point covered twice by one atom")
        gss = np.exp(-d2 / (2 * sigma * sigma))
        vals = np.stack([gss, d[:, 0] * gss, d[:, 1] * gss, d[:, 2] * gss], axis=1)
        norm = np.sqrt(np.sum(vals * vals, axis=0) * dv)
        vals = vals / norm * math.sqrt(dv)       # sum over the support of sup_val^2 = 1
        idx_l.append(idx.astype(np.int32))
        wrap_l.append(wrap.astype(np.int8))
        val_l.append(vals)
        ptr.append(ptr[-1] + len(idx))
    n_atoms = len(centres)
    h = np.zeros((n_atoms, n_proj, n_proj))
    h[:, 0, 0] = h_s
    for k in range(1, n_proj):
        h[:, k, k] = h_p
    return Projectors(
        n_atoms=n_atoms, n_proj=n_proj,
        sup_ptr=np.array(ptr, dtype=np.int64),
        sup_idx=np.concatenate(idx_l) if idx_l else np.zeros(0, np.int32),
        sup_wrap=np.concatenate(wrap_l) if wrap_l else np.zeros(0, np.int8),
        sup_val=np.ascontiguousarray(np.concatenate(val_l)) if val_l else np.zeros((0, n_proj)),
        h=h,
    )


def random_rhs(n: int, L: int, seed: int) -> np.ndarray:
    """Block of L real Gaussian right-hand sides, entries N(0,1), stored as complex128."""
    rng = np.random.default_rng([seed, 0x5EED])
    return rng.standard_normal((n, L)).astype(np.complex128)


def random_rhs_complex(n: int, L: int, seed: int) -> np.ndarray:
    """Block of L complex Gaussian right-hand sides, real and imaginary parts N(0,1)."""
    rng = np.random.default_rng([seed, 0xC0DE])
    return rng.standard_normal((n, L)) + 1j * rng.standard_normal((n, L))


CONFIG_NAMES = ("c1", "c2", "c3", "c4a", "c4b", "c4c", "c5")


def workload(name: str, with_rhs: bool = True) -> Workload:
    """The five synthetic workloads (c4 is three uneven cells c4a/c4b/c4c).

    c1  8x8x4,    h=0.4,  FD4,  3 wells, no projectors, E=0.3,          lmin 0.5, Nint 32, L16 M8
    c2  32x32x16, h=0.35, FD8, 40 atoms + 4 projectors each, 16 E in [-.5,.5], lmin 0.5, Nint 32, L32 M8
    c3  64x64x24, h=0.35, FD8, 120 atoms, 32 E,  lmin 0.3, Nint 64, L32 M8
    c4  48x48x12 / 64x64x16 / 96x96x20, h=0.35, 60/120/270 atoms, 64 E, lmin 0.5, Nint 48, L24 M8
    c5  160x160x32, h=0.2, 640 wells on a cylinder of radius 12, 8 E in [-.3,.3], lmin 0.5, Nint 64, L48 M8
    """
    if name == "c1":
        g = Grid(8, 8, 4, 0.4, 0.4, 0.4, 4)
        seed = 1
        rng = np.random.default_rng(seed)
        centres = rng.uniform(0.0, 1.0, (3, 3)) * np.array(g.cell)
        depths = rng.uniform(-1.0, 0.0, 3)
        vloc = gaussian_wells(g, centres, depths, 0.8)
        wl = Workload(name, g, vloc, None, np.array([0.3]), 0.5, 32, 16, 8,
                      np.zeros((0, 0)), seed=seed)
    elif name in ("c2", "c3", "c4a", "c4b", "c4c"):
        spec = {
            "c2": (Grid(32, 32, 16, 0.35, 0.35, 0.35, 8), 40, 2, np.linspace(-0.5, 0.5, 16), 0.5, 32, 32),
            "c3": (Grid(64, 64, 24, 0.35, 0.35, 0.35, 8), 120, 3, np.linspace(-0.5, 0.5, 32), 0.3, 64, 32),
            "c4a": (Grid(48, 48, 12, 0.35, 0.35, 0.35, 8), 60, 41, np.linspace(-0.5, 0.5, 64), 0.5, 48, 24),
            "c4b": (Grid(64, 64, 16, 0.35, 0.35, 0.35, 8), 120, 42, np.linspace(-0.5, 0.5, 64), 0.5, 48, 24),
            "c4c": (Grid(96, 96, 20, 0.35, 0.35, 0.35, 8), 270, 43, np.linspace(-0.5, 0.5, 64), 0.5, 48, 24),
        }[name]
        g, n_atoms, seed, energies, lmin, n_int, L = spec
        rng = np.random.default_rng(seed)
        centres = rng.uniform(0.0, 1.0, (n_atoms, 3)) * np.array(g.cell)
        depths = rng.uniform(-1.0, 0.0, n_atoms)
        vloc = gaussian_wells(g, centres, depths, 0.8)
        proj = make_projectors(g, centres)
        wl = Workload(name, g, vloc, proj, energies, lmin, n_int, L, 8, np.zeros((0, 0)), seed=seed)
    elif name == "c5":
        g = Grid(160, 160, 32, 0.2, 0.2, 0.2, 8)
        seed = 5
        rng = np.random.default_rng(seed)
        n_atoms = 640
        lx, ly, lz = g.cell
        phi = rng.uniform(0.0, 2 * math.pi, n_atoms)
        zz = rng.uniform(0.0, lz, n_atoms)
        centres = np.stack([lx / 2 + 12.0 * np.cos(phi), ly / 2 + 12.0 * np.sin(phi), zz], axis=1)
        depths = np.full(n_atoms, -0.5)
        sub = rng.uniform(0.0, 1.0, n_atoms) < 0.05
        depths[sub] = np.where(rng.uniform(0.0, 1.0, int(sub.sum())) < 0.5, -0.8, -0.2)
        vloc = gaussian_wells(g, centres, depths, 0.8)
        proj = make_projectors(g, centres)
        wl = Workload(name, g, vloc, proj, np.linspace(-0.3, 0.3, 8), 0.5, 64, 48, 8,
                      np.zeros((0, 0)), seed=seed)
    else:
        raise KeyError(name)
    if with_rhs:
        wl.V = random_rhs(wl.grid.n, wl.L, wl.seed)
    return wl


def tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, projectors=True,
                  energies=(0.2,), lambda_min=0.5, n_int=32, L=8, M=6, seed=11,
                  r_c=0.8, sigma=0.3) -> Workload:
    """Small cells for oracle pins and parity tests (odd sizes, ragged tiles)."""
    g = Grid(nx, ny, nz, h, h, h, fd_order)
    rng = np.random.default_rng([seed, 17])
    centres = rng.uniform(0.0, 1.0, (n_atoms, 3)) * np.array(g.cell)
    depths = rng.uniform(-1.0, 0.0, n_atoms)
    vloc = gaussian_wells(g, centres, depths, 0.6)
    proj = make_projectors(g, centres, r_c=r_c, sigma=sigma) if projectors and n_atoms else None
    V = random_rhs(g.n, L, seed)
    return Workload("tiny", g, vloc, proj, np.asarray(energies, float), lambda_min, n_int, L, M, V,
                    seed=seed)
