"""CPU oracle for block-multicolor ICCG -- TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU statement of the method of Suzuki, "Comparison of Algebraic
Block Multi-Coloring and Leiden Methods for Parallel Preconditioning in the
ICCG Method".  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this package.  It shares no code with the
CUDA library; its only common dependency is the input generator package
``gen`` (matrices and right-hand sides, no method arithmetic).

Heavy loops (graph, ABMC, coloring, Leiden, IC(0), substitutions, PCG) live in
``iccg_oracle.c``, the sequential statement of the library's parallel Leiden
in ``par_leiden.c`` (single-threaded, -ffp-contract=off).  This module adds
ctypes marshalling and a few plain numpy definitions:

  * ``permute``            A_hat = P A P^T with P from perm[new] = old (Sec. 3);
  * ``quality_modularity`` Eq. (1);
  * ``quality_cpm``        Eq. (2);
  * ``block_stats``        G (Gini, Sec. 6.3), B_max, B_max/B_avg, C_max/C_avg
                           (Table 6 definitions).

Parity unpinned: the Leiden partition itself (igraph, which the paper used,
is not available; several partitions are valid).  Its invariants and planted
cases are pinned instead; see tests/test_oracle_leiden.py.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import scipy.sparse as sp

from . import build as _build

_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        c_i32, c_i64, c_d, c_u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
        L.orc_philox_stream.argtypes = [c_u64, c_i64, _u64p]
        L.orc_shuffle_stream.argtypes = [c_u64, c_i64, _i32p]
        L.orc_graph.argtypes = [c_i32, _i64p, _i32p, _i64p, ctypes.c_void_p]
        L.orc_graph.restype = c_i64
        L.orc_abmc.argtypes = [c_i32, _i64p, _i32p, c_i32, _i32p]
        L.orc_abmc.restype = c_i32
        L.orc_color_blocks.argtypes = [c_i32, _i64p, _i32p, c_i32, _i32p, _i32p]
        L.orc_color_blocks.restype = c_i32
        L.orc_leiden.argtypes = [c_i32, _i64p, _i32p, c_i32, c_d, c_i32, c_d, c_u64, _i32p]
        L.orc_leiden.restype = c_i32
        L.orc_par_leiden.argtypes = [c_i32, _i64p, _i32p, c_i32, c_d, c_i32, _i32p]
        L.orc_par_leiden.restype = c_i32
        L.orc_delta_quality.argtypes = [c_i32, _i64p, _i32p, c_i32, c_d, _i32p, c_i32, c_i32]
        L.orc_delta_quality.restype = c_d
        L.orc_sort_blocks_desc.argtypes = [c_i32, c_i32, _i32p]
        L.orc_order.argtypes = [c_i32, c_i32, c_i32, _i32p, _i32p, _i32p, _i32p, _i32p]
        L.orc_level_order.argtypes = [c_i32, _i64p, _i32p, _i32p, _i32p, _i32p, _i32p]
        L.orc_level_order.restype = c_i32
        L.orc_ic0.argtypes = [c_i32, _i64p, _i32p, _f64p, _f64p]
        L.orc_ic0.restype = c_i64
        L.orc_forward.argtypes = [c_i32, _i64p, _i32p, _f64p, _f64p, _f64p]
        L.orc_backward.argtypes = [c_i32, _i64p, _i32p, _f64p, _f64p, _f64p]
        L.orc_spmv.argtypes = [c_i32, _i64p, _i32p, _f64p, _f64p, _f64p]
        L.orc_pcg.argtypes = [c_i32, _i64p, _i32p, _f64p, _i64p, _i32p, _f64p, _f64p, _f64p,
                              c_d, c_i32, ctypes.POINTER(c_i32), ctypes.c_void_p]
        L.orc_pcg.restype = c_i32
        _lib = L
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------------------
# random numbers (Philox4x64-10, counter incremented before each block)
# ---------------------------------------------------------------------------
def philox_stream(seed: int, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint64)
    lib().orc_philox_stream(seed, count, out)
    return out


def shuffle_stream(seed: int, length: int) -> np.ndarray:
    out = np.zeros(length, dtype=np.int32)
    lib().orc_shuffle_stream(seed, length, out)
    return out


# ---------------------------------------------------------------------------
# graph, blocking, coloring, ordering
# ---------------------------------------------------------------------------
def graph(n, rowptr, colind):
    """Adjacency graph of A (Sec. 3): returns (gptr int64[n+1], gadj int32[])."""
    rowptr = _c(rowptr, np.int64)
    colind = _c(colind, np.int32)
    gptr = np.zeros(n + 1, dtype=np.int64)
    m = lib().orc_graph(n, rowptr, colind, gptr, None)
    gadj = np.zeros(max(m, 1), dtype=np.int32)
    lib().orc_graph(n, rowptr, colind, gptr, gadj.ctypes.data)
    return gptr, gadj[:m]


def abmc(n, gptr, gadj, s):
    """ABMC blocks of size s (Sec. 3).  Returns (block_of int32[n], n_b)."""
    block_of = np.zeros(n, dtype=np.int32)
    nb = lib().orc_abmc(n, _c(gptr, np.int64), _c(gadj, np.int32), int(s), block_of)
    return block_of, nb


def color_blocks(n, gptr, gadj, n_b, block_of):
    """Greedy block coloring (Sec. 3, Sec. 5.1).  Returns (color_of int32[n_b], n_c)."""
    color_of = np.zeros(max(n_b, 1), dtype=np.int32)
    nc = lib().orc_color_blocks(n, _c(gptr, np.int64), _c(gadj, np.int32), n_b,
                                _c(block_of, np.int32), color_of)
    return color_of[:n_b], nc


def leiden(n, gptr, gadj, quality: str, gamma: float, n_iter: int = 2, beta: float = 0.01,
           seed: int = 42):
    """Leiden communities (Sec. 4, Sec. 6.1).  quality in {'modularity', 'cpm'}.
    Returns (memb int32[n], number of communities)."""
    q = {"modularity": 0, "md": 0, "cpm": 1, "cp": 1}[quality.lower()]
    memb = np.zeros(max(n, 1), dtype=np.int32)
    k = lib().orc_leiden(n, _c(gptr, np.int64), _c(gadj, np.int32), q, float(gamma),
                         int(n_iter), float(beta), int(seed), memb)
    return memb[:n], k


def par_leiden(n, gptr, gadj, quality: str, gamma: float, n_iter: int = 2):
    """The parallel Leiden of the GPU library (synchronous sub-rounds, greedy
    refinement, connected blocks), stated sequentially (par_leiden.c).
    Returns (block_of int32[n], number of blocks)."""
    q = {"modularity": 0, "md": 0, "cpm": 1, "cp": 1}[quality.lower()]
    memb = np.zeros(max(n, 1), dtype=np.int32)
    k = lib().orc_par_leiden(n, _c(gptr, np.int64), _c(gadj, np.int32), q, float(gamma), int(n_iter), memb)
    return memb[:n], k


def delta_quality(n, gptr, gadj, quality: str, gamma: float, memb, v: int, target: int) -> float:
    """Q(after) - Q(before) for moving node v to community target, computed
    with the gain function of the Leiden local moving."""
    q = {"modularity": 0, "md": 0, "cpm": 1, "cp": 1}[quality.lower()]
    return lib().orc_delta_quality(n, _c(gptr, np.int64), _c(gadj, np.int32), q, float(gamma),
                                   _c(memb, np.int32), int(v), int(target))


def sort_blocks_desc(n, n_b, block_of):
    b = _c(block_of, np.int32).copy()
    lib().orc_sort_blocks_desc(n, n_b, b)
    return b


def order(n, n_b, n_c, block_of, color_of):
    """Block-multicolor ordering.  Returns (perm, block_ptr, color_ptr)."""
    perm = np.zeros(max(n, 1), dtype=np.int32)
    bptr = np.zeros(n_b + 1, dtype=np.int32)
    cptr = np.zeros(n_c + 1, dtype=np.int32)
    lib().orc_order(n, n_b, n_c, _c(block_of, np.int32), _c(color_of, np.int32), perm, bptr, cptr)
    return perm[:n], bptr, cptr


def level_order(n, gptr, gadj):
    """Level sets of the natural order (level scheduling, Sec. 2): returns
    (level [n], n_levels, perm, block_ptr [n+1], color_ptr [n_levels+1])."""
    lev = np.zeros(max(n, 1), dtype=np.int32)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    bptr = np.zeros(n + 1, dtype=np.int32)
    cptr = np.zeros(n + 1, dtype=np.int32)
    nl = lib().orc_level_order(n, _c(gptr, np.int64), _c(gadj, np.int32), lev, perm, bptr, cptr)
    return lev[:n], int(nl), perm[:n], bptr, cptr[:nl + 1]


def split_levels(a, bl, max_rows=32):
    """Intra-block level sets for oversized blocks (blocks as the unit of
    parallelism of Sec. 3, made finer for blocks too large for one warp):
    every block of more than max_rows rows is split by in-block level (the
    longest chain of earlier rows of the same block, through the pattern,
    ending at the row); each level of a color becomes a color of one-row
    blocks, after the color's small blocks.  Plain loops; returns a blocking
    dict (perm, block_ptr, color_ptr, n_b, n_c)."""
    n = a.n
    perm = np.asarray(bl["perm"])
    bptr = np.asarray(bl["block_ptr"])
    cptr = np.asarray(bl["color_ptr"])[:bl["n_c"] + 1]
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    lev = {}
    for b in range(bl["n_b"]):
        r0, r1 = int(bptr[b]), int(bptr[b + 1])
        if r1 - r0 <= max_rows:
            continue
        for i in range(r0, r1):
            o = perm[i]
            lv = 0
            for e in range(a.rowptr[o], a.rowptr[o + 1]):
                j = int(iperm[a.colind[e]])
                if r0 <= j < i:
                    lv = max(lv, lev[j] + 1)
            lev[i] = lv
    out_perm, out_bptr, out_cptr = [], [], []
    for c in range(bl["n_c"]):
        blocks = range(int(cptr[c]), int(cptr[c + 1]))
        small = [b for b in blocks if bptr[b + 1] - bptr[b] <= max_rows]
        big = [b for b in blocks if bptr[b + 1] - bptr[b] > max_rows]
        if small:
            out_cptr.append(len(out_bptr))
            for b in small:
                out_bptr.append(len(out_perm))
                out_perm.extend(int(v) for v in perm[bptr[b]:bptr[b + 1]])
        depth = max([lev[i] + 1 for b in big for i in range(bptr[b], bptr[b + 1])], default=0)
        for v in range(depth):
            out_cptr.append(len(out_bptr))
            for b in big:
                for i in range(int(bptr[b]), int(bptr[b + 1])):
                    if lev[i] == v:
                        out_bptr.append(len(out_perm))
                        out_perm.append(int(perm[i]))
    out_cptr.append(len(out_bptr))
    out_bptr.append(len(out_perm))
    return {"perm": np.array(out_perm, dtype=np.int32), "block_ptr": np.array(out_bptr, dtype=np.int32),
            "color_ptr": np.array(out_cptr, dtype=np.int32), "n_b": len(out_bptr) - 1, "n_c": len(out_cptr) - 1}


def blocking(a, method: str = "abmc", block_size: int = 32, gamma: float = 1.0,
             n_iter: int = 2, beta: float = 0.01, seed: int = 42):
    """Full blocking pipeline: graph -> blocks -> (Leiden: size sort) -> colors ->
    ordering, or the level-set ordering of the natural order ("levels").
    Returns dict(perm, block_ptr, color_ptr, n_b, n_c, block_of, color_of)."""
    n = a.n
    gptr, gadj = graph(n, a.rowptr, a.colind)
    if method == "levels":
        lev, nl, perm, bptr, cptr = level_order(n, gptr, gadj)
        return {"perm": perm, "block_ptr": bptr, "color_ptr": cptr, "n_b": n, "n_c": nl,
                "block_of": np.arange(n, dtype=np.int32), "color_of": lev}
    if method == "abmc":
        block_of, nb = abmc(n, gptr, gadj, block_size)
    elif method in ("leiden_md", "leiden_cpm"):
        q = "modularity" if method == "leiden_md" else "cpm"
        block_of, nb = leiden(n, gptr, gadj, q, gamma, n_iter, beta, seed)
        block_of = sort_blocks_desc(n, nb, block_of)
    else:
        raise ValueError(method)
    color_of, nc = color_blocks(n, gptr, gadj, nb, block_of)
    perm, bptr, cptr = order(n, nb, nc, block_of, color_of)
    return {"perm": perm, "block_ptr": bptr, "color_ptr": cptr, "n_b": nb, "n_c": nc,
            "block_of": block_of, "color_of": color_of}


# ---------------------------------------------------------------------------
# permutation, IC(0), substitutions, PCG
# ---------------------------------------------------------------------------
def permute(a, perm):
    """A_hat = P A P^T: A_hat[i, j] = A[perm[i], perm[j]]; returns scipy CSR
    with sorted indices."""
    m = a.to_scipy() if hasattr(a, "to_scipy") else sp.csr_matrix(a)
    perm = np.asarray(perm, dtype=np.int64)
    ah = m[perm, :][:, perm].tocsr()
    ah.sort_indices()
    return ah


def tril_csr(ah):
    """Lower triangle including the diagonal, as (lptr int64, lcol int32, aval)."""
    lo = sp.tril(ah, 0, format="csr")
    lo.sort_indices()
    return (lo.indptr.astype(np.int64), lo.indices.astype(np.int32), lo.data.astype(np.float64))


def ic0(lptr, lcol, aval):
    """IC(0): returns (lval, breakdown_row) with breakdown_row = -1 on success."""
    n = len(lptr) - 1
    lval = np.zeros_like(np.asarray(aval, dtype=np.float64))
    row = lib().orc_ic0(n, _c(lptr, np.int64), _c(lcol, np.int32), _c(aval, np.float64), lval)
    return lval, int(row)


def forward(lptr, lcol, lval, r):
    n = len(lptr) - 1
    y = np.zeros(n)
    lib().orc_forward(n, _c(lptr, np.int64), _c(lcol, np.int32), _c(lval, np.float64),
                      _c(r, np.float64), y)
    return y


def backward(lptr, lcol, lval, y):
    n = len(lptr) - 1
    z = np.zeros(n)
    lib().orc_backward(n, _c(lptr, np.int64), _c(lcol, np.int32), _c(lval, np.float64),
                       _c(y, np.float64), z)
    return z


def spmv(ah, x):
    n = ah.shape[0]
    y = np.zeros(n)
    lib().orc_spmv(n, _c(ah.indptr, np.int64), _c(ah.indices, np.int32), _c(ah.data, np.float64),
                   _c(x, np.float64), y)
    return y


def pcg(ah, lptr, lcol, lval, b, x0=None, tol=1e-8, maxit=10000):
    """PCG on the permuted system.  Returns (x, iterations, hist, status)."""
    n = ah.shape[0]
    x = np.zeros(n) if x0 is None else _c(x0, np.float64).copy()
    hist = np.zeros(maxit + 1)
    it = ctypes.c_int32(0)
    st = lib().orc_pcg(n, _c(ah.indptr, np.int64), _c(ah.indices, np.int32), _c(ah.data, np.float64),
                       _c(lptr, np.int64), _c(lcol, np.int32), _c(lval, np.float64),
                       _c(b, np.float64), x, float(tol), int(maxit), ctypes.byref(it),
                       hist.ctypes.data)
    return x, it.value, hist[: it.value + 1].copy(), st


def iccg(a, b, perm, x0=None, tol=1e-8, maxit=10000):
    """ICCG in the original numbering: permute, IC(0), PCG, un-permute.
    Returns dict(x, iterations, hist, status, breakdown_row, true_relres)."""
    perm = np.asarray(perm, dtype=np.int64)
    ah = permute(a, perm)
    lptr, lcol, aval = tril_csr(ah)
    lval, brow = ic0(lptr, lcol, aval)
    if brow >= 0:
        return {"x": None, "iterations": 0, "hist": None, "status": "breakdown",
                "breakdown_row": int(perm[brow]), "true_relres": None}
    bh = np.asarray(b, dtype=np.float64)[perm]
    xh0 = None if x0 is None else np.asarray(x0, dtype=np.float64)[perm]
    xh, it, hist, st = pcg(ah, lptr, lcol, lval, bh, xh0, tol, maxit)
    x = np.zeros(a.n)
    x[perm] = xh
    bn = np.linalg.norm(b)
    tr = float(np.linalg.norm(b - a.to_scipy() @ x) / bn) if bn > 0 else 0.0
    return {"x": x, "iterations": it, "hist": hist,
            "status": {0: "converged", 1: "not_converged", 2: "nonfinite"}[st],
            "breakdown_row": -1, "true_relres": tr}


# ---------------------------------------------------------------------------
# quality functions (Eqs. 1, 2) and block statistics (Sec. 6.3, Table 6)
# ---------------------------------------------------------------------------
def _edges(n, gptr, gadj):
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(gptr))
    return src, np.asarray(gadj, dtype=np.int64)


def quality_modularity(n, gptr, gadj, memb, gamma=1.0):
    """Eq. (1): Q = 1/(2m) sum_ij (A_ij - gamma k_i k_j / 2m) delta(c_i, c_j)."""
    src, dst = _edges(n, gptr, gadj)
    two_m = float(len(dst))
    memb = np.asarray(memb)
    inside = float(np.sum(memb[src] == memb[dst]))
    k = np.diff(gptr).astype(np.float64)
    K = np.bincount(memb, weights=k)
    return (inside - gamma * float(np.sum(K * K)) / two_m) / two_m


def quality_cpm(n, gptr, gadj, memb, gamma):
    """Eq. (2): Q = 1/(2m) sum_ij (A_ij - gamma) delta(c_i, c_j), the sum over
    all ordered pairs (i, j) including i = j."""
    src, dst = _edges(n, gptr, gadj)
    two_m = float(len(dst))
    memb = np.asarray(memb)
    inside = float(np.sum(memb[src] == memb[dst]))
    sizes = np.bincount(memb).astype(np.float64)
    return (inside - gamma * float(np.sum(sizes * sizes))) / two_m


def gini(sizes):
    """G = sum_i sum_j |s_i - s_j| / (2 n_b^2 mean(s))  (Sec. 6.3)."""
    s = np.sort(np.asarray(sizes, dtype=np.float64))
    nb = s.size
    if nb == 0 or s.sum() == 0:
        return 0.0
    # sum_ij |s_i - s_j| = 2 sum_k (2k - nb + 1) s_(k) for sorted s (k from 0)
    k = np.arange(nb, dtype=np.float64)
    tot = 2.0 * float(np.sum((2.0 * k - nb + 1.0) * s))
    return tot / (2.0 * nb * nb * float(s.mean()))


def block_stats(block_ptr, color_ptr):
    """n_b, n_c, G, B_max, B_max/B_avg, C_max/C_avg (Table 6 definitions)."""
    bp = np.asarray(block_ptr, dtype=np.int64)
    cp = np.asarray(color_ptr, dtype=np.int64)
    sizes = np.diff(bp)
    nb = sizes.size
    nc = cp.size - 1
    csz = np.array([sizes[cp[c]:cp[c + 1]].sum() for c in range(nc)], dtype=np.float64)
    return {"n_b": int(nb), "n_c": int(nc), "G": gini(sizes),
            "B_max": int(sizes.max()) if nb else 0,
            "B_max/B_avg": float(sizes.max() / sizes.mean()) if nb else 0.0,
            "C_max/C_avg": float(csz.max() / csz.mean()) if nc else 0.0}
