"""Pins for the oracle's ABMC blocking, greedy block coloring and ordering.

ABMC (Sec. 3; block size s = ceil(n/n_b), Sec. 5.1) is pinned by closed forms
(path graph, block sizes), the Table 6 ABMC rows and a hand-worked 4x4 grid;
greedy coloring (Sec. 3, Sec. 5.1) by networkx's independent greedy_color and
the invariant that same-color blocks share no edge.
"""
import math
import os

import networkx as nx
import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _path_graph(n):
    m = sp.diags([np.ones(n - 1), np.ones(n), np.ones(n - 1)], [-1, 0, 1], format="csr")
    return gen.from_scipy(m)


def _truncated_grid(n, w):
    """n nodes of a w-wide 2D grid, numbered row-major."""
    i = np.arange(n)
    right = i[(i % w != w - 1) & (i + 1 < n)]
    down = i[i + w < n]
    r = np.concatenate([right, down])
    c = np.concatenate([right + 1, down + w])
    m = sp.csr_matrix((np.ones(r.size), (r, c)), shape=(n, n))
    return gen.from_scipy(m + m.T + sp.identity(n))


@pytest.mark.parametrize("n,s", [(1, 1), (10, 3), (100, 7), (257, 16), (64, 64), (5, 10)])
def test_abmc_path_graph_is_contiguous_segments(n, s):
    a = _path_graph(n)
    gptr, gadj = oracle.graph(a.n, a.rowptr, a.colind)
    block_of, nb = oracle.abmc(n, gptr, gadj, s)
    assert nb == math.ceil(n / s)
    assert np.array_equal(block_of, np.arange(n) // s)


@pytest.mark.parametrize("seed", range(4))
def test_abmc_block_sizes_closed_form(seed):
    rng = np.random.default_rng(seed)
    a = gen.random_spd_small(int(rng.integers(50, 400)), 0.03, seed)
    s = int(rng.integers(1, 40))
    gptr, gadj = oracle.graph(a.n, a.rowptr, a.colind)
    block_of, nb = oracle.abmc(a.n, gptr, gadj, s)
    sizes = np.bincount(block_of, minlength=nb)
    assert nb == math.ceil(a.n / s)
    assert np.all(sizes[:-1] == s)
    assert sizes[-1] == a.n - (nb - 1) * s


def test_abmc_table6_rows():
    """Table 6: ABMC has B_max = ceil(n/n_b), G = 0.00, B_max/B_avg = 1.00."""
    rows = [l.split() for l in open(os.path.join(GOLD, "table6_abmc.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 8
    for name, n, nb_paper, bmax, g, ratio in rows:
        n, nb_paper, bmax = int(n), int(nb_paper), int(bmax)
        s = math.ceil(n / nb_paper)
        a = _truncated_grid(n, 1024)
        gptr, gadj = oracle.graph(a.n, a.rowptr, a.colind)
        block_of, nb = oracle.abmc(n, gptr, gadj, s)
        sizes = np.bincount(block_of)
        assert nb == nb_paper, name
        assert sizes.max() == bmax, name
        assert f"{oracle.gini(sizes):.2f}" == g, name
        assert f"{sizes.max() / sizes.mean():.2f}" == ratio, name


def _read_gold(name):
    d = {}
    for l in open(os.path.join(GOLD, name)):
        if l.strip() and not l.startswith("#"):
            k, *v = l.split()
            d[k] = np.array([int(x) for x in v])
    return d


def test_abmc_hand_worked_grid():
    g = _read_gold("grid4x4_abmc4.txt")
    a = gen.poisson2d_5pt(4)
    bl = oracle.blocking(a, "abmc", 4)
    assert np.array_equal(bl["block_of"], g["block_of"])
    assert np.array_equal(bl["color_of"], g["color_of"])
    assert np.array_equal(bl["perm"], g["perm"])
    assert np.array_equal(bl["block_ptr"], g["block_ptr"])
    assert np.array_equal(bl["color_ptr"], g["color_ptr"])


def _block_graph(n, gptr, gadj, block_of, nb):
    src = np.repeat(np.arange(n), np.diff(gptr))
    bs, bd = block_of[src], block_of[gadj]
    keep = bs != bd
    G = nx.Graph()
    G.add_nodes_from(range(nb))
    G.add_edges_from(zip(bs[keep].tolist(), bd[keep].tolist()))
    return G


@pytest.mark.parametrize("case", ["grid2d", "grid3d", "rspd", "rgg"])
@pytest.mark.parametrize("s", [1, 4, 16])
def test_greedy_coloring_matches_networkx(case, s):
    a = {"grid2d": lambda: gen.poisson2d_5pt(20), "grid3d": lambda: gen.poisson3d_7pt(8),
         "rspd": lambda: gen.random_spd_small(300, 0.02, 5),
         "rgg": lambda: gen.rgg_laplacian(500, 10.0, 3)}[case]()
    gptr, gadj = oracle.graph(a.n, a.rowptr, a.colind)
    block_of, nb = oracle.abmc(a.n, gptr, gadj, s)
    color_of, nc = oracle.color_blocks(a.n, gptr, gadj, nb, block_of)
    G = _block_graph(a.n, gptr, gadj, block_of, nb)
    ref = nx.greedy_color(G, strategy=lambda g, colors: list(range(nb)))
    assert all(color_of[b] == ref[b] for b in range(nb))
    assert nc == max(ref.values()) + 1
    # invariant: no edge joins two blocks of one color
    for u, v in G.edges():
        assert color_of[u] != color_of[v]
    maxdeg = max((d for _, d in G.degree()), default=0)
    assert nc <= maxdeg + 1


def test_path_of_blocks_needs_two_colors():
    a = _path_graph(100)
    bl = oracle.blocking(a, "abmc", 10)
    assert bl["n_c"] == 2
    assert np.array_equal(bl["color_of"], np.arange(10) % 2)


@pytest.mark.parametrize("method,kw", [("abmc", {"block_size": 8}), ("leiden_cpm", {"gamma": 0.1}),
                                       ("leiden_md", {"gamma": 1.0})])
def test_ordering_is_color_block_row_major(method, kw):
    a = gen.poisson2d_5pt(24)
    bl = oracle.blocking(a, method, **kw)
    perm, bp, cp = bl["perm"], bl["block_ptr"], bl["color_ptr"]
    assert np.array_equal(np.sort(perm), np.arange(a.n))
    assert bp[0] == 0 and bp[-1] == a.n and np.all(np.diff(bp) > 0)
    assert cp[0] == 0 and cp[-1] == bl["n_b"] and np.all(np.diff(cp) > 0)
    # rows ascending inside each block; one block id and one color per block
    for j in range(bl["n_b"]):
        rows = perm[bp[j]:bp[j + 1]]
        assert np.all(np.diff(rows) > 0)
        assert len(set(bl["block_of"][rows])) == 1
    # same-color blocks share no edge (checked on the permuted matrix)
    ah = oracle.permute(a, perm)
    blk = np.repeat(np.arange(bl["n_b"]), np.diff(bp))
    col = np.repeat(np.arange(bl["n_c"]), np.diff(cp))[blk]
    coo = ah.tocoo()
    other = blk[coo.row] != blk[coo.col]
    assert not np.any(col[coo.row][other] == col[coo.col][other])


def test_leiden_block_sort_descending():
    a = gen.poisson2d_5pt(30)
    gptr, gadj = oracle.graph(a.n, a.rowptr, a.colind)
    memb, k = oracle.leiden(a.n, gptr, gadj, "cpm", 0.05)
    b = oracle.sort_blocks_desc(a.n, k, memb)
    sizes = np.bincount(b, minlength=k)
    assert np.all(np.diff(sizes) <= 0)
    # ties broken by the smallest original row, ascending
    first = np.array([np.nonzero(b == j)[0].min() for j in range(k)])
    for j in range(k - 1):
        if sizes[j] == sizes[j + 1]:
            assert first[j] < first[j + 1]
    # same partition, relabelled
    assert len(set(zip(memb.tolist(), b.tolist()))) == k


# ---------------------------------------------------------------------------
# level-set ordering (the level-scheduling baseline of Sec. 2)
# ---------------------------------------------------------------------------
def _levels_by_relaxation(n, gptr, gadj):
    """Longest chain of preceding neighbours, by repeated relaxation until no
    level changes (an algorithm other than the oracle's single pass)."""
    lev = np.zeros(n, dtype=np.int64)
    changed = True
    while changed:
        changed = False
        for i in range(n):
            nb = gadj[gptr[i]:gptr[i + 1]]
            lower = nb[nb < i]
            want = int(lev[lower].max()) + 1 if lower.size else 0
            if want != lev[i]:
                lev[i] = want
                changed = True
    return lev


@pytest.mark.parametrize("kind", ["rspd", "rgg", "grid2d"])
def test_level_order_is_longest_chain_and_independent(kind):
    a = {"rspd": lambda: gen.random_spd_small(300, 0.02, 5), "rgg": lambda: gen.rgg_laplacian(400, 9.0, 3),
         "grid2d": lambda: gen.poisson2d_5pt(13)}[kind]()
    gptr, gadj = oracle.graph(a.n, a.rowptr, a.colind)
    lev, nl, perm, bptr, cptr = oracle.level_order(a.n, gptr, gadj)
    assert np.array_equal(lev, _levels_by_relaxation(a.n, gptr, gadj))
    assert nl == lev.max() + 1
    # rows of a level are never adjacent (a valid coloring of one-row blocks)
    src = np.repeat(np.arange(a.n), np.diff(gptr))
    assert not np.any(lev[src] == lev[gadj])
    # levels ascending, rows ascending within a level
    assert np.array_equal(perm, np.lexsort((np.arange(a.n), lev)))
    assert np.array_equal(bptr, np.arange(a.n + 1)) and np.array_equal(np.diff(cptr), np.bincount(lev))


@pytest.mark.parametrize("nx", [5, 9])
def test_level_order_grid_closed_form(nx):
    """Natural order of a 3D 7-point grid: the level of node (i, j, k) is
    i + j + k, so there are 3 nx - 2 levels."""
    a = gen.poisson3d_7pt(nx)
    gptr, gadj = oracle.graph(a.n, a.rowptr, a.colind)
    lev, nl, *_ = oracle.level_order(a.n, gptr, gadj)
    idx = np.arange(a.n)
    i, j, k = idx % nx, (idx // nx) % nx, idx // (nx * nx)
    assert np.array_equal(lev, i + j + k) and nl == 3 * nx - 2


def test_level_order_gives_the_natural_order_ic0_and_iccg():
    """Every adjacent pair keeps its relative order, so IC(0) in the level
    order is the natural-order IC(0) permuted, and ICCG converges alike."""
    a = gen.rgg_laplacian(500, 8.0, 7)
    b = gen.rhs_uniform(a.n, 2)
    gptr, gadj = oracle.graph(a.n, a.rowptr, a.colind)
    lev, nl, perm, *_ = oracle.level_order(a.n, gptr, gadj)
    ident = np.arange(a.n, dtype=np.int32)
    an = oracle.permute(a, ident)
    ap = oracle.permute(a, perm)
    ln, _ = oracle.ic0(*oracle.tril_csr(an))
    lp, _ = oracle.ic0(*oracle.tril_csr(ap))
    import scipy.sparse as sps
    Ln = sps.csr_matrix((ln, oracle.tril_csr(an)[1], oracle.tril_csr(an)[0]), shape=(a.n, a.n))
    Lp = sps.csr_matrix((lp, oracle.tril_csr(ap)[1], oracle.tril_csr(ap)[0]), shape=(a.n, a.n))
    back = Lp[np.argsort(perm)][:, np.argsort(perm)]
    assert abs(back - Ln).max() <= 1e-13 * abs(Ln).max()
    rn = oracle.iccg(a, b, ident)
    rp = oracle.iccg(a, b, perm)
    assert rn["iterations"] == rp["iterations"]
    assert np.linalg.norm(rn["x"] - rp["x"]) <= 1e-10 * np.linalg.norm(rn["x"])


# ---------------------------------------------------------------------------
# intra-block level sets for oversized blocks
# ---------------------------------------------------------------------------
def test_split_levels_keeps_the_factor_and_the_solve():
    """Splitting Leiden-modularity blocks (hundreds of rows) by in-block level
    gives a valid block-multicolor ordering whose IC(0) is the original one
    permuted (adjacent pairs keep their order) and whose ICCG converges alike."""
    a = gen.poisson2d_5pt(30)
    b = gen.rhs_uniform(a.n, 3)
    bl = oracle.blocking(a, "leiden_md", gamma=1.0)
    assert np.diff(bl["block_ptr"]).max() > 32
    sp_ = oracle.split_levels(a, bl, 32)
    assert sorted(sp_["perm"].tolist()) == list(range(a.n))
    # coloring invariant: no edge inside a color between different blocks
    n = a.n
    gptr, gadj = oracle.graph(n, a.rowptr, a.colind)
    newpos = np.empty(n, dtype=np.int64)
    newpos[sp_["perm"]] = np.arange(n)
    blk = np.repeat(np.arange(sp_["n_b"]), np.diff(sp_["block_ptr"]))
    col = np.repeat(np.arange(sp_["n_c"]), np.diff(sp_["color_ptr"]))
    src = np.repeat(np.arange(n), np.diff(gptr))
    bi, bj = blk[newpos[src]], blk[newpos[gadj]]
    assert not np.any((bi != bj) & (col[bi] == col[bj]))
    # factor: the original one, permuted
    import scipy.sparse as sps
    def lfac(perm):
        ah = oracle.permute(a, perm)
        lp, lc, av = oracle.tril_csr(ah)
        lv, br = oracle.ic0(lp, lc, av)
        assert br == -1
        m = sps.csr_matrix((lv, lc, lp), shape=(n, n))
        inv = np.argsort(perm)
        return m[inv][:, inv]
    f0, f1 = lfac(bl["perm"]), lfac(sp_["perm"])
    assert abs(f0 - f1).max() <= 1e-13 * abs(f0).max()
    r0, r1 = oracle.iccg(a, b, bl["perm"]), oracle.iccg(a, b, sp_["perm"])
    assert r0["iterations"] == r1["iterations"]
    assert np.linalg.norm(r0["x"] - r1["x"]) <= 1e-10 * np.linalg.norm(r0["x"])


def test_split_levels_leaves_small_blocks_alone():
    a = gen.poisson3d_7pt(8)
    bl = oracle.blocking(a, "abmc", 16)
    sp_ = oracle.split_levels(a, bl, 32)
    assert np.array_equal(sp_["perm"], bl["perm"]) and sp_["n_c"] == bl["n_c"]
    assert np.array_equal(sp_["block_ptr"], bl["block_ptr"])
