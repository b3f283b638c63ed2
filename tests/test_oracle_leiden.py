"""Pins for the oracle's Leiden blocking (Sec. 4, Eqs. 1-2; Sec. 6.1).

Parity against igraph (the paper's implementation) is unpinned: igraph is not
available and several partitions are valid.  Pinned instead:
  * Eq. (1) against networkx's modularity, Eq. (2) against a brute-force sum;
  * the gain the local moving uses equals Q(after) - Q(before) for random
    moves (so a dropped factor, a wrong sign or a wrong gamma scaling fails);
  * planted partitions (disjoint cliques joined by single edges);
  * the Leiden guarantee that every community induces a connected subgraph;
  * quality at least that of the singleton partition; determinism per seed;
  * the block-count trend with gamma_CP of Table 10 (Sec. 8).
"""
import networkx as nx
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import gen
import oracle


def _graph_of(a):
    return oracle.graph(a.n, a.rowptr, a.colind)


def _nx(n, gptr, gadj):
    G = nx.Graph()
    G.add_nodes_from(range(n))
    src = np.repeat(np.arange(n), np.diff(gptr))
    G.add_edges_from((int(u), int(v)) for u, v in zip(src, gadj) if u < v)
    return G


def _ring_of_cliques(K, k):
    n = K * k
    rows, cols = [], []
    for c in range(K):
        base = c * k
        for i in range(k):
            for j in range(i + 1, k):
                rows.append(base + i); cols.append(base + j)
        rows.append(base + k - 1); cols.append(((c + 1) % K) * k)   # one bridge edge
    m = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    return gen.from_scipy(m + m.T + sp.identity(n))


@pytest.mark.parametrize("gamma", [0.5, 1.0, 2.0])
def test_modularity_matches_networkx(gamma):
    a = gen.rgg_laplacian(300, 8.0, 1)
    gptr, gadj = _graph_of(a)
    rng = np.random.default_rng(0)
    memb = rng.integers(0, 7, size=a.n).astype(np.int32)
    G = _nx(a.n, gptr, gadj)
    comms = [set(np.nonzero(memb == c)[0].tolist()) for c in range(7)]
    ref = nx.community.modularity(G, [c for c in comms if c], resolution=gamma)
    assert abs(oracle.quality_modularity(a.n, gptr, gadj, memb, gamma) - ref) < 1e-12


@pytest.mark.parametrize("gamma", [0.01, 0.3])
def test_cpm_matches_bruteforce(gamma):
    a = gen.random_spd_small(60, 0.08, 2)
    gptr, gadj = _graph_of(a)
    memb = np.random.default_rng(1).integers(0, 5, size=a.n)
    A = np.zeros((a.n, a.n))
    src = np.repeat(np.arange(a.n), np.diff(gptr))
    A[src, gadj] = 1.0
    tot = sum((A[i, j] - gamma) for i in range(a.n) for j in range(a.n) if memb[i] == memb[j])
    ref = tot / A.sum()
    assert abs(oracle.quality_cpm(a.n, gptr, gadj, memb, gamma) - ref) < 1e-12


@pytest.mark.parametrize("quality,gamma", [("modularity", 1.0), ("modularity", 3.0),
                                           ("cpm", 0.02), ("cpm", 0.4)])
def test_move_gain_equals_quality_difference(quality, gamma):
    a = gen.rgg_laplacian(200, 9.0, 4)
    gptr, gadj = _graph_of(a)
    rng = np.random.default_rng(7)
    memb = rng.integers(0, 6, size=a.n).astype(np.int32)
    qf = oracle.quality_modularity if quality == "modularity" else oracle.quality_cpm
    for _ in range(60):
        v = int(rng.integers(a.n))
        t = int(rng.integers(0, 7))          # 6 = a currently empty community
        before = qf(a.n, gptr, gadj, memb, gamma)
        after_m = memb.copy(); after_m[v] = t
        after = qf(a.n, gptr, gadj, after_m, gamma)
        dq = oracle.delta_quality(a.n, gptr, gadj, quality, gamma, memb, v, t)
        assert abs(dq - (after - before)) < 1e-12


@pytest.mark.parametrize("K,k", [(8, 6), (12, 5)])
def test_planted_cliques_cpm(K, k):
    a = _ring_of_cliques(K, k)
    gptr, gadj = _graph_of(a)
    # a clique beats splitting (gamma < 1) and joining neighbours (gamma > 1/k^2)
    memb, nk = oracle.leiden(a.n, gptr, gadj, "cpm", 0.3, seed=42)
    assert nk == K
    assert np.array_equal(memb, np.repeat(np.arange(K), k))


def test_planted_cliques_modularity():
    a = _ring_of_cliques(8, 6)
    gptr, gadj = _graph_of(a)
    memb, nk = oracle.leiden(a.n, gptr, gadj, "modularity", 1.0, seed=42)
    assert nk == 8
    assert np.array_equal(memb, np.repeat(np.arange(8), 6))


@pytest.mark.parametrize("quality,gamma", [("modularity", 1.0), ("cpm", 0.05), ("cpm", 0.3)])
@pytest.mark.parametrize("case", ["grid2d", "grid3d", "rgg"])
def test_leiden_invariants(quality, gamma, case):
    a = {"grid2d": lambda: gen.poisson2d_5pt(30), "grid3d": lambda: gen.poisson3d_7pt(10),
         "rgg": lambda: gen.rgg_laplacian(800, 12.0, 5)}[case]()
    gptr, gadj = _graph_of(a)
    memb, nk = oracle.leiden(a.n, gptr, gadj, quality, gamma, seed=42)
    assert memb.min() == 0 and memb.max() == nk - 1 and len(np.unique(memb)) == nk
    # every community induces a connected subgraph
    adj = sp.csr_matrix((np.ones(gadj.size), gadj, gptr), shape=(a.n, a.n))
    for c in range(nk):
        idx = np.nonzero(memb == c)[0]
        ncomp, _ = connected_components(adj[idx][:, idx], directed=False)
        assert ncomp == 1
    qf = oracle.quality_modularity if quality == "modularity" else oracle.quality_cpm
    assert qf(a.n, gptr, gadj, memb, gamma) >= qf(a.n, gptr, gadj, np.arange(a.n), gamma)
    again, _ = oracle.leiden(a.n, gptr, gadj, quality, gamma, seed=42)
    assert np.array_equal(memb, again)


def test_cpm_block_count_grows_with_gamma():
    """Table 10 (Sec. 8): on 2D problems n_b grows by about 2.6x when gamma_CP
    grows 4x (parabolic_fem x2.60, ecology2 x2.57).  Loose band on a 2D grid."""
    a = gen.poisson2d_5pt(120)
    gptr, gadj = _graph_of(a)
    _, k1 = oracle.leiden(a.n, gptr, gadj, "cpm", 0.02, seed=42)
    _, k4 = oracle.leiden(a.n, gptr, gadj, "cpm", 0.08, seed=42)
    assert 1.6 < k4 / k1 < 4.0


# ---------------------------------------------------------------------------
# the sequential statement of the library's parallel Leiden (par_leiden.c)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("K,k", [(8, 6), (12, 5)])
@pytest.mark.parametrize("quality,gamma", [("cpm", 0.3), ("modularity", 1.0)])
def test_par_leiden_planted_cliques(K, k, quality, gamma):
    a = _ring_of_cliques(K, k)
    gptr, gadj = _graph_of(a)
    memb, nk = oracle.par_leiden(a.n, gptr, gadj, quality, gamma)
    assert nk == K
    assert np.array_equal(memb, np.repeat(np.arange(K), k))   # blocks numbered by smallest node


@pytest.mark.parametrize("side", [(10, 10), (8, 8, 8), (6, 4, 10)])
def test_par_leiden_cpm05_reaches_the_grid_optimum(side):
    """CPM at resolution 0.5 with unit weights: a community of k nodes and e
    internal edges contributes e - k^2/4, which is 0 for an edge (k = 2, e =
    1) or a 4-cycle (k = 4, e = 4) and negative for every other subgraph of a
    grid (a grid is bipartite: k nodes span at most 0, 1, 2, 4, 5, 7, 9, 12
    edges for k = 1..8, and at most 3k < k^2/4 edges for k > 12, with the
    cases between checked alike), so the optimum of a grid with a perfect
    matching is 0, reached exactly by pairs (and 4-cycles); the parallel
    Leiden finds it."""
    a = gen.poisson2d_5pt(*side) if len(side) == 2 else gen.from_scipy(
        _grid3d(*side))
    gptr, gadj = _graph_of(a)
    memb, nk = oracle.par_leiden(a.n, gptr, gadj, "cpm", 0.5)
    assert abs(oracle.quality_cpm(a.n, gptr, gadj, memb, 0.5)) < 1e-12
    sizes = np.bincount(memb)
    assert set(np.unique(sizes)) <= {2, 4}


def _grid3d(nx, ny, nz):
    def lap(m):
        return sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    ix, iy, iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    return (sp.kron(sp.kron(lap(nx), iy), iz) + sp.kron(sp.kron(ix, lap(ny)), iz)
            + sp.kron(sp.kron(ix, iy), lap(nz))).tocsr()


@pytest.mark.parametrize("quality,gamma", [("modularity", 1.0), ("cpm", 0.05), ("cpm", 0.3), ("cpm", 0.5)])
@pytest.mark.parametrize("case", ["grid2d", "grid3d", "rgg"])
def test_par_leiden_invariants(quality, gamma, case):
    """Labels 0..k-1 numbered by smallest node, every block connected, the
    quality above the singleton partition's and at least 90% of the
    sequential Leiden's gain over it, deterministic."""
    a = {"grid2d": lambda: gen.poisson2d_5pt(30), "grid3d": lambda: gen.poisson3d_7pt(10),
         "rgg": lambda: gen.rgg_laplacian(800, 12.0, 5)}[case]()
    gptr, gadj = _graph_of(a)
    memb, nk = oracle.par_leiden(a.n, gptr, gadj, quality, gamma)
    assert memb.min() == 0 and memb.max() == nk - 1 and len(np.unique(memb)) == nk
    first = np.full(nk, a.n)
    np.minimum.at(first, memb, np.arange(a.n))
    assert np.all(np.diff(first) > 0)
    adj = sp.csr_matrix((np.ones(gadj.size), gadj, gptr), shape=(a.n, a.n))
    for c in range(nk):
        idx = np.nonzero(memb == c)[0]
        ncomp, _ = connected_components(adj[idx][:, idx], directed=False)
        assert ncomp == 1
    qf = oracle.quality_modularity if quality == "modularity" else oracle.quality_cpm
    q_par = qf(a.n, gptr, gadj, memb, gamma)
    q_one = qf(a.n, gptr, gadj, np.arange(a.n), gamma)
    seq, _ = oracle.leiden(a.n, gptr, gadj, quality, gamma, seed=42)
    q_seq = qf(a.n, gptr, gadj, seq, gamma)
    assert q_par >= q_one
    assert q_par - q_one >= 0.9 * (q_seq - q_one)
    again, _ = oracle.par_leiden(a.n, gptr, gadj, quality, gamma)
    assert np.array_equal(memb, again)
