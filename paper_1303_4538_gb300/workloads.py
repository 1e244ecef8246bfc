"""Seeded synthetic 7-point systems shaped like the paper's workloads.

This module only draws inputs: coefficient arrays, a manufactured solution
x* and the right-hand side b = A x*.  It holds none of the solver's
arithmetic (no factorisation, no sweeps, no norms) and is the one module that
both the CPU oracle's tests and the CUDA path's tests and benchmark use.

The paper's test cases (forward-facing step, channel, Taylor-Green; Sec. 3)
are not available as data; only their grid sizes are given.  The generators
follow the finite-volume structure the paper describes (co-located FV on
hexahedral blocks, 7-point coupling, symmetric pressure-correction matrix,
non-symmetric convective momentum matrix; Sec. 4.1):

* diffusion: one conductance D ~ U[0.5, 2] per interior face, shared by the
  two cells of the face;
* convection (``convdiff``): one face flux F per interior face, F = g with
  g ~ N(0, 1), or F = Pe * D * g / 0.6745 so that the median cell Peclet
  number |F|/D is ``pe``; first-order upwind:
  A_E(P) = -(D + max(-F, 0)),  A_W(E) = -(D + max(F, 0)) (same for y, z);
* ``poisson``: no convection; the bottom face (k = 0) is a Dirichlet face
  whose conductance D ~ U[0.5, 2] is added to AP (boundary value 0), which
  makes the matrix nonsingular;
* AP = sum |A_nb| (+ Dirichlet conductances) (+ ``time_term``, 0.01 for
  convdiff); boundary faces otherwise carry no coefficient (zero);
* x* ~ U[-1, 1]; b = A x* in FP64.

Random draws use numpy ``Generator(PCG64(seed))`` in the fixed order
D_x, D_y, D_z, [D_dir], [g_x, g_y, g_z], x*; each generator draws only what
it uses.  Arrays are flat in the natural layout p = i + nx*(j + ny*k).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

COEF_NAMES = ("ap", "aw", "ae", "as", "an", "ab", "at")


@dataclass
class Block:
    """One hexahedral block's 7-point system A x = b (natural layout)."""

    nx: int
    ny: int
    nz: int
    coefs: Dict[str, np.ndarray]  # the seven matrix diagonals, FP64, flat
    b: np.ndarray  # FP64 right-hand side
    xstar: Optional[np.ndarray] = None  # manufactured solution
    symmetric: bool = False
    kind: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def coef_list(self) -> List[np.ndarray]:
        return [self.coefs[k] for k in COEF_NAMES]


def _shapes(nx: int, ny: int, nz: int):
    return (nz, ny, max(nx - 1, 0)), (nz, max(ny - 1, 0), nx), (max(nz - 1, 0), ny, nx)


def apply_matrix(nx: int, ny: int, nz: int, coefs: Dict[str, np.ndarray],
                 x: np.ndarray) -> np.ndarray:
    """A x for the 7-point matrix (used to manufacture b = A x*)."""
    sh = (nz, ny, nx)
    X = x.reshape(sh)
    C = {k: v.reshape(sh) for k, v in coefs.items()}
    out = C["ap"] * X
    out[:, :, 1:] += C["aw"][:, :, 1:] * X[:, :, :-1]
    out[:, :, :-1] += C["ae"][:, :, :-1] * X[:, :, 1:]
    out[:, 1:, :] += C["as"][:, 1:, :] * X[:, :-1, :]
    out[:, :-1, :] += C["an"][:, :-1, :] * X[:, 1:, :]
    out[1:, :, :] += C["ab"][1:, :, :] * X[:-1, :, :]
    out[:-1, :, :] += C["at"][:-1, :, :] * X[1:, :, :]
    return out.reshape(-1)


def make_block(nx: int, ny: int, nz: int, seed: int, kind: str = "convdiff",
               pe: Optional[float] = None, time_term: Optional[float] = None,
               dirichlet_bottom: Optional[bool] = None) -> Block:
    """Draw one block.  ``kind`` is ``convdiff`` or ``poisson``."""
    if kind not in ("convdiff", "poisson"):
        raise ValueError(f"unknown generator kind {kind!r}")
    if min(nx, ny, nz) < 1:
        raise ValueError("block dimensions must be >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    sx, sy, sz = _shapes(nx, ny, nz)
    Dx = rng.uniform(0.5, 2.0, size=sx)
    Dy = rng.uniform(0.5, 2.0, size=sy)
    Dz = rng.uniform(0.5, 2.0, size=sz)
    if dirichlet_bottom is None:
        dirichlet_bottom = kind == "poisson"
    Ddir = rng.uniform(0.5, 2.0, size=(ny, nx)) if dirichlet_bottom else None
    if kind == "convdiff":
        gx = rng.standard_normal(size=sx)
        gy = rng.standard_normal(size=sy)
        gz = rng.standard_normal(size=sz)
        if pe is None:
            Fx, Fy, Fz = gx, gy, gz
        else:
            c = pe / 0.6745
            Fx, Fy, Fz = c * Dx * gx, c * Dy * gy, c * Dz * gz
        if time_term is None:
            time_term = 0.01
    else:
        Fx = np.zeros(sx)
        Fy = np.zeros(sy)
        Fz = np.zeros(sz)
        if time_term is None:
            time_term = 0.0
    xstar = rng.uniform(-1.0, 1.0, size=nx * ny * nz)

    sh = (nz, ny, nx)
    coefs = {k: np.zeros(sh) for k in COEF_NAMES}
    # x faces: between (i, j, k) and (i+1, j, k)
    coefs["ae"][:, :, :-1] = -(Dx + np.maximum(-Fx, 0.0))
    coefs["aw"][:, :, 1:] = -(Dx + np.maximum(Fx, 0.0))
    coefs["an"][:, :-1, :] = -(Dy + np.maximum(-Fy, 0.0))
    coefs["as"][:, 1:, :] = -(Dy + np.maximum(Fy, 0.0))
    coefs["at"][:-1, :, :] = -(Dz + np.maximum(-Fz, 0.0))
    coefs["ab"][1:, :, :] = -(Dz + np.maximum(Fz, 0.0))
    ap = sum(np.abs(coefs[k]) for k in COEF_NAMES[1:]) + time_term
    if Ddir is not None:
        ap[0, :, :] += Ddir
    coefs["ap"] = ap
    coefs = {k: np.ascontiguousarray(v.reshape(-1)) for k, v in coefs.items()}
    b = apply_matrix(nx, ny, nz, coefs, xstar)
    return Block(nx, ny, nz, coefs, b, xstar, symmetric=(kind == "poisson"), kind=kind,
                 meta={"seed": seed, "pe": pe, "time_term": time_term,
                       "dirichlet_bottom": bool(dirichlet_bottom)})


# Workloads named by what they are (seed = 4538 + index of the workload).
def convdiff_32cube() -> Block:
    """32x32x32 convection-diffusion block, F ~ N(0,1), time term 0.01."""
    return make_block(32, 32, 32, seed=4539, kind="convdiff")


def poisson_256cube(n: int = 256) -> Block:
    """n^3 pressure-Poisson block with a Dirichlet bottom face (n=256 default)."""
    return make_block(n, n, n, seed=4540, kind="poisson")


def convdiff_pe10_384cube(n: int = 384) -> Block:
    """n^3 convection-diffusion block with median cell Peclet 10 (FP32 storage)."""
    return make_block(n, n, n, seed=4542, kind="convdiff", pe=10.0)


@dataclass
class Mesh:
    """Blocks of a block-structured mesh chained along x: interface q =
    (lo, hi, nj, nk) joins cell (nx_lo - 1, j, k) of block lo with cell
    (0, j, k) of block hi for j < nj, k < nk.  The coupling entries sit in
    lo's AE and hi's AW on those cells; b of every block includes the
    interface terms of the manufactured solution."""

    blocks: List[Block]
    ifaces: List[Tuple[int, int, int, int]]

    @property
    def n(self) -> int:
        return sum(b.n for b in self.blocks)


def make_mesh(dims, seed: int, kind: str = "convdiff", pe: Optional[float] = None) -> Mesh:
    """Blocks of sizes dims[b] = (nx, ny, nz), block b drawn with
    make_block(seed = seed * 1000 + b); consecutive blocks coupled across the
    overlap rectangle of their x faces, nj = min(ny), nk = min(nz).  Each
    interface face draws its conductance D ~ U[0.5, 2] (and, for convdiff, a
    flux as make_block does) from Generator(PCG64([seed, 1])) in interface
    order; the two upwind entries go to lo's AE and hi's AW and their
    magnitudes to the two cells' AP; b = A x* of the coupled system."""
    dims = [tuple(int(v) for v in d) for d in dims]
    blocks = [make_block(nx, ny, nz, seed=seed * 1000 + b, kind=kind, pe=pe) for b, (nx, ny, nz) in enumerate(dims)]
    rng = np.random.Generator(np.random.PCG64([seed, 1]))
    ifaces = []
    for lo in range(len(blocks) - 1):
        hi = lo + 1
        L, H = blocks[lo], blocks[hi]
        nj, nk = min(L.ny, H.ny), min(L.nz, H.nz)
        D = rng.uniform(0.5, 2.0, size=(nk, nj))
        if kind == "convdiff":
            g = rng.standard_normal(size=(nk, nj))
            F = g if pe is None else (pe / 0.6745) * D * g
        else:
            F = np.zeros((nk, nj))
        kk, jj = np.meshgrid(np.arange(nk), np.arange(nj), indexing="ij")
        pl = (L.nx - 1) + L.nx * (jj + L.ny * kk)
        ph = H.nx * (jj + H.ny * kk)
        e_lo = -(D + np.maximum(-F, 0.0))
        e_hi = -(D + np.maximum(F, 0.0))
        L.coefs["ae"][pl] = e_lo
        H.coefs["aw"][ph] = e_hi
        L.coefs["ap"][pl] += np.abs(e_lo)
        H.coefs["ap"][ph] += np.abs(e_hi)
        ifaces.append((lo, hi, nj, nk))
    for b, B in enumerate(blocks):
        B.b = apply_matrix(B.nx, B.ny, B.nz, B.coefs, B.xstar)
    for lo, hi, nj, nk in ifaces:
        L, H = blocks[lo], blocks[hi]
        kk, jj = np.meshgrid(np.arange(nk), np.arange(nj), indexing="ij")
        pl = ((L.nx - 1) + L.nx * (jj + L.ny * kk)).reshape(-1)
        ph = (H.nx * (jj + H.ny * kk)).reshape(-1)
        L.b[pl] += L.coefs["ae"][pl] * H.xstar[ph]
        H.b[ph] += H.coefs["aw"][ph] * L.xstar[pl]
    return Mesh(blocks, ifaces)


def random_block_dims(rng: np.random.Generator, count: int, lo: int, hi: int) -> np.ndarray:
    return rng.integers(lo, hi + 1, size=(count, 3))


def batched_mesh_dims(seed: int = 4541, nblocks: int = 64, lo: int = 24, hi: int = 128,
                      total_lo: int = 18_000_000, total_hi: int = 22_000_000
                      ) -> Tuple[np.ndarray, int]:
    """Block sizes of the multi-block mesh: nx, ny, nz i.i.d. U{lo..hi};
    the whole draw is redrawn with seed + 1000 t until the total cell count
    lies in [total_lo, total_hi].  Returns (dims[nblocks, 3], t)."""
    for t in range(10_000):
        rng = np.random.Generator(np.random.PCG64(seed + 1000 * t))
        dims = random_block_dims(rng, nblocks, lo, hi)
        tot = int(np.prod(dims, axis=1).sum())
        if total_lo <= tot <= total_hi:
            return dims, t
    raise RuntimeError("no admissible draw")


def batched_mesh(seed: int = 4541) -> Mesh:
    """The 64-block convection-diffusion mesh of ~20 M cells (x chain)."""
    dims, _ = batched_mesh_dims(seed)
    return make_mesh(dims, seed, kind="convdiff")


@dataclass
class PcorrInputs:
    """Inputs of the pressure-correction assembly on one rectilinear block:
    cell widths dx (nx), dy (ny), dz (nz); per cell the density ``rho`` and the
    momentum equation's V / a_P (``g``); face-normal velocities u* on every
    face: ``ux`` ((nx+1) ny nz, face i = west face of cell i, index
    (k ny + j)(nx+1) + i), ``uy`` (nx (ny+1) nz, index (k (ny+1) + j) nx + i),
    ``uz`` (nx ny (nz+1), index (k ny + j) nx + i)."""

    nx: int
    ny: int
    nz: int
    dx: np.ndarray
    dy: np.ndarray
    dz: np.ndarray
    rho: np.ndarray
    g: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray
    dirichlet_bottom: bool = True

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


def pcorr_inputs(nx: int, ny: int, nz: int, seed: int, dirichlet_bottom: bool = True) -> PcorrInputs:
    """Seeded inputs of the pressure-correction assembly: a stretched grid
    (widths U[0.5, 2] / n per axis), rho ~ U[0.8, 1.2], g ~ U[0.5, 2],
    interior-face velocities u* ~ N(0, 1), zero velocity on the wall faces
    (x and y boundaries, top), u* ~ N(0, 1) on the bottom (Dirichlet, open)
    face.  Draw order: dx, dy, dz, rho, g, ux, uy, uz."""
    if min(nx, ny, nz) < 1:
        raise ValueError("block dimensions must be >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = rng.uniform(0.5, 2.0, size=nx) / nx
    dy = rng.uniform(0.5, 2.0, size=ny) / ny
    dz = rng.uniform(0.5, 2.0, size=nz) / nz
    n = nx * ny * nz
    rho = rng.uniform(0.8, 1.2, size=n)
    g = rng.uniform(0.5, 2.0, size=n)
    ux = rng.standard_normal(size=(nz, ny, nx + 1))
    uy = rng.standard_normal(size=(nz, ny + 1, nx))
    uz = rng.standard_normal(size=(nz + 1, ny, nx))
    ux[:, :, 0] = 0.0
    ux[:, :, nx] = 0.0
    uy[:, 0, :] = 0.0
    uy[:, ny, :] = 0.0
    uz[nz, :, :] = 0.0
    if not dirichlet_bottom:
        uz[0, :, :] = 0.0
    return PcorrInputs(nx, ny, nz, dx, dy, dz, rho, g, ux.reshape(-1).copy(), uy.reshape(-1).copy(),
                       uz.reshape(-1).copy(), dirichlet_bottom)


def make_block_device(nx: int, ny: int, nz: int, seed: int, kind: str = "convdiff", device="cuda"):
    """The ``make_block`` recipe drawn on a device with torch's seeded
    generator (for request streams too large to draw on the host): the same
    distributions and structure (D ~ U[0.5, 2] per interior face; convdiff: F ~
    N(0, 1) per interior face, upwind, time term 0.01; poisson: a Dirichlet
    bottom face with D ~ U[0.5, 2], no convection), x* ~ U[-1, 1], b = A x*.
    The random streams differ from ``make_block``'s (torch's generator, not
    PCG64).  Returns (coefs: list of the seven FP64 tensors in COEF_NAMES
    order, b, xstar); for ``poisson`` aw, as, ab are returned too (the matrix is
    symmetric)."""
    import torch

    if kind not in ("convdiff", "poisson"):
        raise ValueError(f"unknown generator kind {kind!r}")
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = dict(dtype=torch.float64, device=device)

    def U(shape):
        return torch.rand(shape, generator=g, **f64) * 1.5 + 0.5

    sx, sy, sz = _shapes(nx, ny, nz)
    Dx, Dy, Dz = U(sx), U(sy), U(sz)
    sh = (nz, ny, nx)
    C = {k: torch.zeros(sh, **f64) for k in COEF_NAMES}
    if kind == "convdiff":
        Fx = torch.randn(sx, generator=g, **f64)
        Fy = torch.randn(sy, generator=g, **f64)
        Fz = torch.randn(sz, generator=g, **f64)
        tt = 0.01
    else:
        Fx, Fy, Fz = torch.zeros(sx, **f64), torch.zeros(sy, **f64), torch.zeros(sz, **f64)
        tt = 0.0
    C["ae"][:, :, :-1] = -(Dx + torch.clamp(-Fx, min=0.0))
    C["aw"][:, :, 1:] = -(Dx + torch.clamp(Fx, min=0.0))
    C["an"][:, :-1, :] = -(Dy + torch.clamp(-Fy, min=0.0))
    C["as"][:, 1:, :] = -(Dy + torch.clamp(Fy, min=0.0))
    C["at"][:-1, :, :] = -(Dz + torch.clamp(-Fz, min=0.0))
    C["ab"][1:, :, :] = -(Dz + torch.clamp(Fz, min=0.0))
    ap = sum(C[k].abs() for k in COEF_NAMES[1:]) + tt
    if kind == "poisson":
        ap[0] += U((ny, nx))
    C["ap"] = ap
    xs = torch.rand(sh, generator=g, **f64) * 2.0 - 1.0
    out = C["ap"] * xs
    out[:, :, 1:] += C["aw"][:, :, 1:] * xs[:, :, :-1]
    out[:, :, :-1] += C["ae"][:, :, :-1] * xs[:, :, 1:]
    out[:, 1:, :] += C["as"][:, 1:, :] * xs[:, :-1, :]
    out[:, :-1, :] += C["an"][:, :-1, :] * xs[:, 1:, :]
    out[1:, :, :] += C["ab"][1:, :, :] * xs[:-1, :, :]
    out[:-1, :, :] += C["at"][:-1, :, :] * xs[1:, :, :]
    return [C[k].reshape(-1) for k in COEF_NAMES], out.reshape(-1), xs.reshape(-1)
