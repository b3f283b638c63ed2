"""Seeded synthetic inputs for the block-multicolor ICCG path.

This module is the only code shared by the CPU oracle (``oracle/``) and the
CUDA path (``paper_2609_00561_gb300``).  It builds sparse SPD matrices and
right-hand sides and nothing else: no blocking, coloring, factorisation or
solver arithmetic lives here.

The paper evaluates eight SuiteSparse SPD matrices (Sec. 4, Table 1) that are
not available offline; the generators below are synthetic stand-ins with the
same character (grid/stencil problems with 5-44 nonzeros per row, n up to a
few million).

Conventions (all generators):
  * CSR with ``rowptr`` int64[n+1], ``colind`` int32[nnz], ``val`` float64[nnz];
  * both triangles stored, columns sorted ascending within a row, explicit
    diagonal entry in every row;
  * every random draw comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

__all__ = [
    "CSR", "from_scipy", "poisson2d_5pt", "poisson3d_7pt", "diffusion3d_27pt",
    "rhs_uniform", "rhs_ones", "config1", "config2", "config3", "config4",
    "stencil_aniso", "rgg_laplacian", "elasticity_like", "config5_matrix",
    "config5_specs", "random_spd_small",
]


@dataclasses.dataclass
class CSR:
    """Sparse matrix in CSR form (int64 rowptr, int32 colind, float64 val)."""
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.n, self.n))


def from_scipy(a, name: str = "") -> CSR:
    """Canonicalise a scipy sparse matrix into the CSR convention above."""
    a = sp.csr_matrix(a, dtype=np.float64)
    n = a.shape[0]
    # make sure the diagonal is structurally present
    a = (a + sp.diags(np.zeros(n), 0, format="csr")).tocsr()
    a.sum_duplicates()
    a.sort_indices()
    return CSR(n=n, rowptr=a.indptr.astype(np.int64), colind=a.indices.astype(np.int32),
               val=a.data.astype(np.float64), name=name)


def _lap1d(m: int, diag: float = 2.0) -> sp.csr_matrix:
    return sp.diags([-np.ones(m - 1), np.full(m, diag), -np.ones(m - 1)], [-1, 0, 1], format="csr")


def poisson2d_5pt(nx: int, ny: int | None = None) -> CSR:
    """2D 5-point Dirichlet Laplacian (diag 4, off-diagonal -1), lexicographic order."""
    ny = nx if ny is None else ny
    ix, iy = sp.identity(nx, format="csr"), sp.identity(ny, format="csr")
    a = sp.kron(iy, _lap1d(nx)) + sp.kron(_lap1d(ny), ix)
    return from_scipy(a, name=f"poisson2d_5pt_{nx}x{ny}")


def poisson3d_7pt(nx: int, shift: float = 0.0) -> CSR:
    """3D 7-point Dirichlet Laplacian (diag 6 + shift, off-diagonal -1), x fastest."""
    i = sp.identity(nx, format="csr")
    l1 = _lap1d(nx)
    a = sp.kron(sp.kron(i, i), l1) + sp.kron(sp.kron(i, l1), i) + sp.kron(sp.kron(l1, i), i)
    if shift:
        a = a + shift * sp.identity(nx ** 3, format="csr")
    return from_scipy(a, name=f"poisson3d_7pt_{nx}^3")


def diffusion3d_27pt(nx: int, seed: int = 0, contrast: float = 1e3,
                     shift_rel: float = 1e-6) -> CSR:
    """27-point variable-coefficient diffusion on an nx^3 grid.

    Cell coefficients kappa_i = exp(sigma * clip(z_i, -3, 3)), z ~ N(0, 1),
    sigma = ln(contrast) / 6, so max/min <= contrast.  Each of the 26
    neighbours gets the harmonic-mean weight w_ij = 2 k_i k_j / (k_i + k_j);
    A is the weighted graph Laplacian plus shift_rel * max(diag) * I.
    """
    rng = np.random.default_rng(seed)
    n = nx ** 3
    z = np.clip(rng.standard_normal(n), -3.0, 3.0)
    kap = np.exp(math.log(contrast) / 6.0 * z)
    idx = np.arange(n, dtype=np.int64).reshape(nx, nx, nx)  # [z][y][x]
    rows, cols, ws = [], [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dz == 0 and dy == 0 and dx == 0:
                    continue
                sz = slice(max(0, -dz), nx - max(0, dz))
                sy = slice(max(0, -dy), nx - max(0, dy))
                sx = slice(max(0, -dx), nx - max(0, dx))
                tz = slice(max(0, dz), nx - max(0, -dz))
                ty = slice(max(0, dy), nx - max(0, -dy))
                tx = slice(max(0, dx), nx - max(0, -dx))
                a_ = idx[sz, sy, sx].ravel()
                b_ = idx[tz, ty, tx].ravel()
                ka, kb = kap[a_], kap[b_]
                rows.append(a_)
                cols.append(b_)
                ws.append(2.0 * ka * kb / (ka + kb))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    w = np.concatenate(ws)
    off = sp.csr_matrix((-w, (r, c)), shape=(n, n))
    deg = -np.asarray(off.sum(axis=1)).ravel()
    shift = shift_rel * deg.max()
    a = off + sp.diags(deg + shift, 0, format="csr")
    return from_scipy(a, name=f"diffusion3d_27pt_{nx}^3")


def rhs_uniform(n: int, seed: int = 0) -> np.ndarray:
    """b ~ U[-1, 1] from the given seed."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)


def rhs_ones(a: CSR) -> np.ndarray:
    """b = A * ones (so the exact solution is the all-ones vector)."""
    return np.asarray(a.to_scipy() @ np.ones(a.n)).ravel()


def config1():
    """2D 5-point Laplacian 64x64 (n=4096), b = A*1, ABMC block size 16."""
    a = poisson2d_5pt(64)
    return a, rhs_ones(a), {"blocking": "abmc", "block_size": 16}


def config2(nx: int = 128, seed: int = 0):
    """3D 7-point Poisson 128^3 (n=2,097,152), b ~ U[-1,1]."""
    a = poisson3d_7pt(nx)
    return a, rhs_uniform(a.n, seed), {"blocking": "abmc", "block_size": 32}


def config3(nx: int = 96, seed: int = 0):
    """3D 27-point variable-coefficient diffusion 96^3 (contrast 1e3), ABMC 32."""
    a = diffusion3d_27pt(nx, seed=seed)
    return a, rhs_uniform(a.n, seed + 1), {"blocking": "abmc", "block_size": 32}


def config4(seed: int = 0, nsys: int = 64, nrhs: int = 16, side_lo: int = 16, side_hi: int = 64):
    """Batch of nsys 3D 7-point Poisson systems with sides U{side_lo..side_hi},
    diagonal shifts U[1e-4, 1e-1] and nrhs right-hand sides U[-1, 1] each."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=nsys)
    shifts = rng.uniform(1e-4, 1e-1, size=nsys)
    systems = []
    for s, d in zip(sides, shifts):
        a = poisson3d_7pt(int(s), shift=float(d))
        b = rng.uniform(-1.0, 1.0, size=(nrhs, a.n))
        systems.append((a, b))
    return systems, {"blocking": "abmc", "block_size": 32}


# ---------------------------------------------------------------------------
# Generators for the learned-blocking training set (200 matrices).
# ---------------------------------------------------------------------------

def stencil_aniso(kind: str, n_target: int, a_ratio: float) -> CSR:
    """Anisotropic constant-coefficient stencil with axis weights (1, a, a^2)
    (2D: (1, a)); kind in {'5pt', '7pt', '27pt'}.  Dirichlet boundary."""
    if kind == "5pt":
        nx = max(4, int(round(math.sqrt(n_target))))
        w = [1.0, a_ratio]
        ix = sp.identity(nx, format="csr")
        a = w[0] * sp.kron(ix, _lap1d(nx)) + w[1] * sp.kron(_lap1d(nx), ix)
        return from_scipy(a, name=f"aniso5_{nx}")
    nx = max(4, int(round(n_target ** (1.0 / 3.0))))
    w = [1.0, a_ratio, a_ratio ** 2]
    i = sp.identity(nx, format="csr")
    l1 = _lap1d(nx)
    if kind == "7pt":
        a = (w[0] * sp.kron(sp.kron(i, i), l1) + w[1] * sp.kron(sp.kron(i, l1), i)
             + w[2] * sp.kron(sp.kron(l1, i), i))
        return from_scipy(a, name=f"aniso7_{nx}")
    # 27pt: neighbour (dx,dy,dz) weight = mean of the axis weights it moves along
    n = nx ** 3
    idx = np.arange(n, dtype=np.int64).reshape(nx, nx, nx)
    rows, cols, ws = [], [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dz == 0 and dy == 0 and dx == 0:
                    continue
                mv = [abs(dx), abs(dy), abs(dz)]
                wt = sum(wi * m for wi, m in zip(w, mv)) / sum(mv)
                sz = slice(max(0, -dz), nx - max(0, dz)); tz = slice(max(0, dz), nx - max(0, -dz))
                sy = slice(max(0, -dy), nx - max(0, dy)); ty = slice(max(0, dy), nx - max(0, -dy))
                sx = slice(max(0, -dx), nx - max(0, dx)); tx = slice(max(0, dx), nx - max(0, -dx))
                a_ = idx[sz, sy, sx].ravel(); b_ = idx[tz, ty, tx].ravel()
                rows.append(a_); cols.append(b_); ws.append(np.full(a_.size, wt))
    r = np.concatenate(rows); c = np.concatenate(cols); wv = np.concatenate(ws)
    off = sp.csr_matrix((-wv, (r, c)), shape=(n, n))
    # Dirichlet boundary: every row's diagonal is the full 26-neighbour weight
    # sum, so boundary rows are strictly diagonally dominant and A is SPD.
    full = 0.0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dz or dy or dx:
                    mv = [abs(dx), abs(dy), abs(dz)]
                    full += sum(wi * m for wi, m in zip(w, mv)) / sum(mv)
    a = off + full * sp.identity(n, format="csr")
    return from_scipy(a, name=f"aniso27_{nx}")


def rgg_laplacian(n: int, avg_degree: float, seed: int) -> CSR:
    """Random geometric graph in the unit cube with expected degree avg_degree;
    unweighted graph Laplacian + 1e-2 * I."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    r = (3.0 * avg_degree / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    i, j = pairs[:, 0], pairs[:, 1]
    adj = sp.csr_matrix((np.ones(i.size), (i, j)), shape=(n, n))
    adj = adj + adj.T
    deg = np.asarray(adj.sum(axis=1)).ravel()
    a = sp.diags(deg + 1e-2, 0, format="csr") - adj
    return from_scipy(a, name=f"rgg_{n}_{avg_degree:.1f}")


def elasticity_like(n_nodes_target: int, stencil: int, lam: float) -> CSR:
    """3 dof per node spring network on a 3D grid (7- or 27-neighbour).  Each
    edge e with unit direction u contributes K_e = mu I + lam u u^T (mu = 1)
    as [[K, -K], [-K, K]] (PSD); A gets + 1e-6 * max(diag) * I."""
    nx = max(3, int(round(n_nodes_target ** (1.0 / 3.0))))
    nn = nx ** 3
    idx = np.arange(nn, dtype=np.int64).reshape(nx, nx, nx)
    offs = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dz, dy, dx) <= (0, 0, 0):
                    continue  # half of the neighbours: each undirected edge once
                if stencil == 7 and abs(dx) + abs(dy) + abs(dz) != 1:
                    continue
                offs.append((dz, dy, dx))
    R, C, V = [], [], []
    for dz, dy, dx in offs:
        sz = slice(max(0, -dz), nx - max(0, dz)); tz = slice(max(0, dz), nx - max(0, -dz))
        sy = slice(max(0, -dy), nx - max(0, dy)); ty = slice(max(0, dy), nx - max(0, -dy))
        sx = slice(max(0, -dx), nx - max(0, dx)); tx = slice(max(0, dx), nx - max(0, -dx))
        a_ = idx[sz, sy, sx].ravel(); b_ = idx[tz, ty, tx].ravel()
        u = np.array([dx, dy, dz], dtype=np.float64); u /= np.linalg.norm(u)
        K = np.eye(3) + lam * np.outer(u, u)
        for p in range(3):
            for q in range(3):
                kv = K[p, q]
                if kv == 0.0:
                    continue
                for (ri, ci, sgn) in ((a_, a_, 1.0), (b_, b_, 1.0), (a_, b_, -1.0), (b_, a_, -1.0)):
                    R.append(3 * ri + p); C.append(3 * ci + q); V.append(np.full(ri.size, sgn * kv))
    n = 3 * nn
    a = sp.csr_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=(n, n))
    a.sum_duplicates()
    # exact symmetry: the assembly sums (i,j) and (j,i) in different orders,
    # so a cancellation could leave one of them a stored zero and not the other
    a = ((a + a.T) * 0.5).tocsr()
    a.eliminate_zeros()
    dmax = a.diagonal().max()
    a = a + 1e-6 * dmax * sp.identity(n, format="csr")
    return from_scipy(a, name=f"elast{stencil}_{nx}")


def config5_specs(count: int = 200, seed: int = 0, n_lo: float = 1e5, n_hi: float = 2e6):
    """Deterministic list of (kind, params) for the learned-blocking set."""
    rng = np.random.default_rng(seed)
    specs = []
    kinds = ["5pt", "7pt", "27pt", "rgg", "elast7", "elast27"]
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        kind = kinds[k % len(kinds)]
        a_ratio = float(math.exp(rng.uniform(0.0, math.log(1e3))))
        deg = float(rng.uniform(8.0, 30.0))
        lam = float(rng.uniform(0.0, 10.0))
        specs.append({"index": k, "kind": kind, "n": n, "a": a_ratio, "deg": deg,
                      "lam": lam, "seed": int(seed * 100003 + k)})
    return specs


def config5_matrix(spec) -> CSR:
    kind = spec["kind"]
    if kind in ("5pt", "7pt", "27pt"):
        return stencil_aniso(kind, spec["n"], spec["a"])
    if kind == "rgg":
        return rgg_laplacian(spec["n"], spec["deg"], spec["seed"])
    if kind == "elast7":
        return elasticity_like(spec["n"] // 3, 7, spec["lam"])
    if kind == "elast27":
        return elasticity_like(spec["n"] // 3, 27, spec["lam"])
    raise ValueError(kind)


def random_spd_small(n: int, density: float, seed: int) -> CSR:
    """Small random sparse SPD matrix: symmetric random pattern, weights
    U[0.1, 1], diagonal = row sum of |off| + U[0.1, 1] (strictly dominant)."""
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=density, random_state=np.random.RandomState(seed), format="csr")
    m.data[:] = rng.uniform(0.1, 1.0, size=m.data.size)
    s = sp.triu(m, 1)
    s = s + s.T
    s.data = -s.data
    d = -np.asarray(s.sum(axis=1)).ravel() + rng.uniform(0.1, 1.0, size=n)
    return from_scipy(s + sp.diags(d, 0), name=f"rspd_{n}_{seed}")
