"""Seeded synthetic inputs for the five workloads (shared by the library's
tests, the benchmark and the CPU oracle).

This module only draws and samples input fields; it holds none of the
method's arithmetic (no operator assembly, no interpolation) and imports
nothing but numpy/scipy.  Every generator is a pure function of its seed.

Workloads (sizes as the paper's experiments use them, Sec. III-A to III-D):
  adv_diff_2d     linear 2D advection-diffusion, D = 0.1, b = -(1, 0.5),
                  homogeneous Dirichlet on a 64 x 64 interior grid,
                  v = sum of 8 random-amplitude sine modes.
  adr_3d          3D advection-diffusion-reaction on n^3 cells (n = 256 or 512),
                  D(x) = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z),
                  b(x) a smooth random field with max |b| = 2, Neumann,
                  u_0 a sum of 4 Gaussians (sigma = 0.05) scaled into [0, 1].
  batch_2d        1024 independent 2D advection-diffusion problems with
                  log-uniform sides in [32, 512] and per-side Dirichlet/Neumann.
  combustion_3d   Sec. III-C combustion model, Table 4 step: 256^3 interior,
                  Laplacian, homogeneous Dirichlet, u0 = 1, h = tol = 1e-4.
  combustion_field  u ~ U[1, 2] on n^3 points (Table 3's evaluation).
  rgg_graph       -(graph Laplacian) of a random geometric graph in the unit
                  cube: 2^20 nodes, mean degree 12, edge weights U[0.5, 2].
  spin_bath       Hamiltonian of two central spins in a bath (Sec. III-D):
                  21 spins, n = 2^21 states, 39 XYZ bonds, 40 entries a row.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

DIRICHLET0 = 0
NEUMANN0 = 1
SEED_BASE = 1234


# --------------------------------------------------------------------------
# 2D advection-diffusion, 64 x 64
# --------------------------------------------------------------------------
@dataclass
class Stencil2D:
    n: tuple            # (nx, ny)
    dx: tuple
    D: float
    b: tuple            # constant b (the operator uses + b . grad u)
    bc: tuple           # x-lo, x-hi, y-lo, y-hi
    v: np.ndarray       # [y, x]
    h: float
    tol: float


def adv_diff_2d(seed: int = SEED_BASE + 0, n: int = 64, modes: int = 8,
                max_mode: int = 16) -> Stencil2D:
    rng = np.random.default_rng(seed)
    dx = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * dx                      # vertex-centred interior points
    v = np.zeros((n, n))
    for _ in range(modes):
        p, r = rng.integers(1, max_mode + 1, size=2)
        a = rng.standard_normal()
        v += a * np.outer(np.sin(r * math.pi * x), np.sin(p * math.pi * x))
    return Stencil2D(n=(n, n), dx=(dx, dx), D=0.1, b=(-1.0, -0.5),
                     bc=(DIRICHLET0,) * 4, v=v, h=1e-3, tol=1e-10)


# --------------------------------------------------------------------------
# 3D advection-diffusion-reaction on n^3 cells
# --------------------------------------------------------------------------
@dataclass
class Stencil3D:
    n: tuple            # (nx, ny, nz)
    dx: tuple
    D: np.ndarray       # [z, y, x]
    b: tuple            # three arrays [z, y, x]
    bc: tuple
    u0: np.ndarray      # [z, y, x]
    h: float
    tol: float
    steps: int


def _cell_centres(n):
    return (np.arange(n) + 0.5) / n


def smooth_vector_field(rng, n, n_modes=4, kmax=2, bmax=2.0, dtype=np.float64):
    """Three components, each a sum of n_modes random Fourier modes
    a sin(2 pi k.x + phase) with integer |k_i| <= kmax, rescaled so that
    max_x |b(x)|_2 = bmax on the cell centres."""
    x = _cell_centres(n)
    comps = []
    for _ in range(3):
        acc = np.zeros((n, n, n), dtype=np.float64)
        for _ in range(n_modes):
            k = rng.integers(-kmax, kmax + 1, size=3)
            a = rng.standard_normal()
            ph = rng.uniform(0.0, 2.0 * math.pi)
            ex = np.exp(2j * math.pi * k[0] * x)
            ey = np.exp(2j * math.pi * k[1] * x)
            ez = np.exp(2j * math.pi * k[2] * x) * np.exp(1j * ph)
            acc += a * (ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).imag
        comps.append(acc)
    mag = np.sqrt(comps[0] ** 2 + comps[1] ** 2 + comps[2] ** 2).max()
    scale = bmax / mag if mag > 0 else 0.0
    return tuple((c * scale).astype(dtype) for c in comps)


def gaussian_bumps(rng, n, count=4, sigma=0.05):
    x = _cell_centres(n)
    u = np.zeros((n, n, n))
    for _ in range(count):
        cx, cy, cz = rng.uniform(0.2, 0.8, size=3)
        a = rng.uniform(0.5, 1.0)
        gx = np.exp(-(x - cx) ** 2 / (2 * sigma ** 2))
        gy = np.exp(-(x - cy) ** 2 / (2 * sigma ** 2))
        gz = np.exp(-(x - cz) ** 2 / (2 * sigma ** 2))
        u += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return u / max(1.0, float(u.max()))


def diffusion_field(n):
    x = _cell_centres(n)
    s = np.sin(2 * math.pi * x)
    return 1.0 + 0.5 * s[:, None, None] * s[None, :, None] * s[None, None, :]


def adr_3d(n: int = 256, seed: int = SEED_BASE + 1, h: float = 1e-4,
           tol: float = 1e-10, steps: int = 20) -> Stencil3D:
    rng = np.random.default_rng(seed)
    b = smooth_vector_field(rng, n)
    u0 = gaussian_bumps(rng, n)
    dx = 1.0 / n
    return Stencil3D(n=(n, n, n), dx=(dx, dx, dx), D=diffusion_field(n), b=b,
                     bc=(NEUMANN0,) * 6, u0=u0, h=h, tol=tol, steps=steps)


def adr_3d_fp32(n: int = 512, seed: int = SEED_BASE + 2) -> Stencil3D:
    """The reduced-precision workload: same fields on 512^3, h = 5e-5, tol 1e-6."""
    return adr_3d(n=n, seed=seed, h=5e-5, tol=1e-6, steps=10)


def combustion_3d(n: int = 256, h: float = 1e-4, tol: float = 1e-4, steps: int = 1) -> Stencil3D:
    """The combustion model of Sec. III-C, u_t = Laplace(u) + g(u) with
    g(u) = (2 - u) e^{20 (1 - 1/u)} / 4, with the step of Table 4: n^3
    interior points of the unit cube (dx = 1/(n+1)), homogeneous Dirichlet
    boundaries, u0 = 1, h = tol = 1e-4.  D and b are constants (1 and 0),
    given as scalars."""
    dx = 1.0 / (n + 1)
    return Stencil3D(n=(n, n, n), dx=(dx, dx, dx), D=1.0, b=(0.0, 0.0, 0.0),
                     bc=(DIRICHLET0,) * 6, u0=np.ones((n, n, n)), h=h, tol=tol, steps=steps)


def combustion_field(n: int, seed: int = SEED_BASE + 5) -> np.ndarray:
    """u uniform in [1, 2] (the combustion model's range) on n^3 points: the
    input of the pointwise evaluation timed in Table 3."""
    return np.random.default_rng(seed).uniform(1.0, 2.0, (n, n, n))


# --------------------------------------------------------------------------
# Batched 2D problems
# --------------------------------------------------------------------------
@dataclass
class BatchInstance:
    n: tuple
    dx: tuple
    D: float
    b: tuple
    bc: tuple
    h: float
    v: np.ndarray


def batch_2d(count: int = 1024, seed: int = SEED_BASE + 3, nmin: int = 32,
             nmax: int = 512) -> list:
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        D = float(rng.uniform(0.01, 1.0))
        b = tuple(float(t) for t in rng.uniform(-1.0, 1.0, size=2))
        h = float(rng.uniform(1e-4, 1e-2))
        bc = tuple(int(t) for t in rng.integers(0, 2, size=4))
        dx = 1.0 / (n + 1)
        x = (np.arange(n) + 1) * dx
        v = np.zeros((n, n))
        for _ in range(3):
            kx, ky = rng.integers(1, 6, size=2)
            a = rng.standard_normal()
            px, py = rng.uniform(0.0, 2.0 * math.pi, size=2)
            v += a * np.outer(np.cos(ky * math.pi * x + py), np.cos(kx * math.pi * x + px))
        out.append(BatchInstance(n=(n, n), dx=(dx, dx), D=D, b=b, bc=bc, h=h, v=v))
    return out


# --------------------------------------------------------------------------
# Random geometric graph, CSR
# --------------------------------------------------------------------------
@dataclass
class Graph:
    n: int
    rowptr: np.ndarray      # int64, n+1
    col: np.ndarray         # int32, off-diagonal neighbours
    val: np.ndarray         # float64 edge weights (symmetric)
    deg_w: np.ndarray       # float64 weighted degree
    radius: float


def _morton3(ix, iy, iz, bits=10):
    code = np.zeros(ix.shape, dtype=np.int64)
    for bit in range(bits):
        code |= ((ix >> bit) & 1).astype(np.int64) << (3 * bit)
        code |= ((iy >> bit) & 1).astype(np.int64) << (3 * bit + 1)
        code |= ((iz >> bit) & 1).astype(np.int64) << (3 * bit + 2)
    return code


def rgg_graph(n: int = 1 << 20, mean_degree: float = 12.0, seed: int = SEED_BASE + 4,
              order: str = "morton") -> Graph:
    """Nodes uniform in [0,1]^3; the radius is the distance of the
    (n*mean_degree/2)-th closest pair, so the realised mean degree is exact;
    weights U[0.5, 2] per undirected edge; nodes sorted by the Morton code of
    their radius-sized cell ("morton") or randomly permuted ("random")."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(n, 3))
    target_pairs = int(round(n * mean_degree / 2))
    r0 = (3.0 * mean_degree / (4.0 * math.pi * n)) ** (1.0 / 3.0) * 1.15
    tree = cKDTree(pts)
    pairs = tree.query_pairs(r0, output_type="ndarray")
    while pairs.shape[0] < target_pairs:
        r0 *= 1.1
        pairs = tree.query_pairs(r0, output_type="ndarray")
    dist = np.linalg.norm(pts[pairs[:, 0]] - pts[pairs[:, 1]], axis=1)
    keep = np.argsort(dist, kind="stable")[:target_pairs]
    radius = float(dist[keep[-1]])
    pairs = pairs[np.sort(keep)]
    w = rng.uniform(0.5, 2.0, size=pairs.shape[0])
    if order == "morton":
        cell = np.minimum((pts / radius).astype(np.int64), (1 << 10) - 1)
        perm = np.argsort(_morton3(cell[:, 0], cell[:, 1], cell[:, 2]), kind="stable")
    else:
        perm = rng.permutation(n)
    newid = np.empty(n, dtype=np.int64)
    newid[perm] = np.arange(n)
    i = newid[pairs[:, 0]]
    j = newid[pairs[:, 1]]
    rows = np.concatenate([i, j])
    cols = np.concatenate([j, i])
    vals = np.concatenate([w, w])
    o = np.lexsort((cols, rows))
    rows, cols, vals = rows[o], cols[o], vals[o]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    deg_w = np.bincount(rows, weights=vals, minlength=n)
    return Graph(n=n, rowptr=rowptr, col=cols.astype(np.int32), val=vals,
                 deg_w=deg_w, radius=radius)


def random_vector(n, seed):
    return np.random.default_rng(seed).standard_normal(n)


# --------------------------------------------------------------------------
# Two central spins in a spin bath (Sec. III-D), CSR in the sigma_z basis
# --------------------------------------------------------------------------
@dataclass
class SpinBath:
    n: int
    rowptr: np.ndarray      # int64, n+1
    col: np.ndarray         # int32, off-diagonal entries (one per bond)
    val: np.ndarray         # float64
    diag: np.ndarray        # float64
    bonds: list             # (i, j, Jx, Jy, Jz)


def spin_bath(n_spins: int = 21, seed: int = SEED_BASE + 6) -> SpinBath:
    """H = sum over bonds (i, j) of Jx X_i X_j + Jy Y_i Y_j + Jz Z_i Z_j for
    spins 0 and 1 (the central pair, bonded to each other) and the bath
    spins 2..n_spins-1 (each bonded to both central spins, not to each
    other): 2 n_spins - 3 bonds, so each row holds one entry per bond plus the
    diagonal (40 for 21 spins: 2^21 x 40 = 83.9e6 entries, as in the paper).
    Couplings: central pair U[0.5, 1.5] per component, central-bath
    U[-0.5, 0.5].  In the sigma_z basis (bit i of the state = spin i down)
    X_i X_j and Y_i Y_j both flip bits i and j: the entry is Jx - Jy for
    aligned spins and Jx + Jy for opposite ones; Z_i Z_j is diagonal, +-Jz.
    H is real symmetric; columns of a row are in bond order."""
    rng = np.random.default_rng(seed)
    bonds = [(0, 1, *rng.uniform(0.5, 1.5, 3))]
    for b in range(2, n_spins):
        for c in (0, 1):
            bonds.append((c, b, *rng.uniform(-0.5, 0.5, 3)))
    n = 1 << n_spins
    st = np.arange(n, dtype=np.int64)
    nb = len(bonds)
    col = np.empty((n, nb), dtype=np.int32)
    val = np.empty((n, nb), dtype=np.float64)
    diag = np.zeros(n)
    for q, (i, j, jx, jy, jz) in enumerate(bonds):
        anti = ((st >> i) ^ (st >> j)) & 1
        col[:, q] = st ^ ((1 << i) | (1 << j))
        val[:, q] = np.where(anti == 1, jx + jy, jx - jy)
        diag += np.where(anti == 1, -jz, jz)
    rowptr = np.arange(0, n * nb + 1, nb, dtype=np.int64)
    return SpinBath(n=n, rowptr=rowptr, col=col.reshape(-1), val=val.reshape(-1), diag=diag,
                    bonds=bonds)


def spin_state(n: int, seed: int = SEED_BASE + 7) -> np.ndarray:
    """A random normalised complex state (Gaussian real and imaginary parts)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return v / np.linalg.norm(v)
