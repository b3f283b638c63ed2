"""Device-side blocking against the oracle.

The device graph (Sec. 3), the device greedy block coloring with the
block-multicolor ordering (Sec. 3, Sec. 5.1) and the device Leiden block
order (Sec. 6.1) must reproduce the oracle's results exactly: gptr / gadj,
color_of, n_c, perm, block_ptr, color_ptr and the relabelled block_of.
Blockings come from the oracle (ABMC of several sizes, Leiden CPM and
modularity, singleton blocks) on every matrix family of the generators, plus
the 128^3 benchmark problem with its default Leiden CPM 0.5 blocking.

The device Leiden is a parallel form of the method and does not reproduce
the host partition; it is held to the invariants (labels, connected blocks,
determinism), to planted cliques, to the oracle's quality (Eqs. 1-2: at least
90% of the oracle Leiden's gain over the singleton partition), and to the
ICCG solve its blocking gives.
"""
import time

import numpy as np
import pytest

import gen
import oracle
from paper_2609_00561_gb300 import build as libbuild
from paper_2609_00561_gb300 import iccg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def _d(a, dt):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def _h(t):
    return t.cpu().numpy()


MATRICES = {
    "grid2d_33": lambda: gen.poisson2d_5pt(33),
    "grid3d_17": lambda: gen.poisson3d_7pt(17),
    "diff27_12": lambda: gen.diffusion3d_27pt(12, seed=3),
    "rgg_3000": lambda: gen.rgg_laplacian(3000, 12.0, seed=5),
    "elast7": lambda: gen.elasticity_like(2000, 7, 3.0),
    "spd_rand": lambda: gen.random_spd_small(400, 0.02, seed=9),
    "single": lambda: gen.poisson2d_5pt(1),
}

BLOCKINGS = [("abmc", 1), ("abmc", 4), ("abmc", 32), ("leiden_cpm", 0.5), ("leiden_cpm", 0.05),
             ("leiden_md", 1.0)]


@pytest.mark.parametrize("name", sorted(MATRICES))
def test_device_graph_equals_oracle(name):
    a = MATRICES[name]()
    gp, ga = oracle.graph(a.n, a.rowptr, a.colind)
    dgp, dga = iccg.iccg_dev_graph(_d(a.rowptr, torch.int64), _d(a.colind, torch.int32))
    torch.cuda.synchronize()
    assert np.array_equal(_h(dgp), gp)
    assert np.array_equal(_h(dga), ga)


@pytest.mark.parametrize("name", sorted(MATRICES))
@pytest.mark.parametrize("method,param", BLOCKINGS)
def test_device_color_order_equals_oracle(name, method, param):
    a = MATRICES[name]()
    n = a.n
    gp, ga = oracle.graph(n, a.rowptr, a.colind)
    if method == "abmc":
        block_of, nb = oracle.abmc(n, gp, ga, param)
    else:
        q = "cpm" if method == "leiden_cpm" else "modularity"
        raw, nb = oracle.leiden(n, gp, ga, q, param)
        block_of = oracle.sort_blocks_desc(n, nb, raw)
        # the device Leiden block order on the raw communities
        dbo = _d(raw, torch.int32)
        iccg.iccg_dev_sort_blocks_desc(nb, dbo)
        assert np.array_equal(_h(dbo), block_of)
    color_of, nc = oracle.color_blocks(n, gp, ga, nb, block_of)
    perm, bptr, cptr = oracle.order(n, nb, nc, block_of, color_of)
    dgp, dga = iccg.iccg_dev_graph(_d(a.rowptr, torch.int64), _d(a.colind, torch.int32))
    dc, dnc, dperm, dbptr, dcptr = iccg.iccg_dev_color_order(dgp, dga, nb, _d(block_of, torch.int32))
    torch.cuda.synchronize()
    assert dnc == nc
    assert np.array_equal(_h(dc), color_of)
    assert np.array_equal(_h(dperm), perm)
    assert np.array_equal(_h(dbptr), bptr)
    assert np.array_equal(_h(dcptr), cptr)


def test_device_blocking_rejects_bad_input():
    a = gen.poisson2d_5pt(6)
    col = a.colind.copy()
    col[5] = a.n + 3
    with pytest.raises(iccg.IccgError) as ei:
        iccg.iccg_dev_graph(_d(a.rowptr, torch.int64), _d(col, torch.int32))
    assert ei.value.status == iccg.ICCG_ERR_ARG
    dgp, dga = iccg.iccg_dev_graph(_d(a.rowptr, torch.int64), _d(a.colind, torch.int32))
    bo = np.zeros(a.n, dtype=np.int32)
    bo[7] = 4
    with pytest.raises(iccg.IccgError) as ei:
        iccg.iccg_dev_color_order(dgp, dga, 2, _d(bo, torch.int32))
    assert ei.value.status == iccg.ICCG_ERR_ARG
    with pytest.raises(iccg.IccgError) as ei:
        iccg.iccg_dev_sort_blocks_desc(2, _d(bo, torch.int32))
    assert ei.value.status == iccg.ICCG_ERR_ARG


def test_device_blocking_full_size_cpm05():
    """128^3 7-point Poisson with the bench's Leiden CPM 0.5 blocking: the
    device graph and coloring / ordering equal the production host code's
    (itself equal to the oracle's, test_abi_host), and the times are printed."""
    a = gen.poisson3d_7pt(128)
    n = a.n
    t0 = time.perf_counter()
    gp, ga = iccg.iccg_graph(n, a.rowptr, a.colind)
    t_hg = time.perf_counter() - t0
    raw, nb = iccg.iccg_block_leiden(n, gp, ga, "cpm", 0.5)
    t0 = time.perf_counter()
    block_of = iccg.iccg_sort_blocks_desc(n, nb, raw)
    color_of, nc, perm, bptr, cptr = iccg.iccg_color_order(n, gp, ga, nb, block_of)
    t_hc = time.perf_counter() - t0
    rp, ci = _d(a.rowptr, torch.int64), _d(a.colind, torch.int32)
    draw = _d(raw, torch.int32)
    iccg.iccg_dev_graph(rp, ci)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dgp, dga = iccg.iccg_dev_graph(rp, ci)
    torch.cuda.synchronize()
    t_dg = time.perf_counter() - t0
    t0 = time.perf_counter()
    iccg.iccg_dev_sort_blocks_desc(nb, draw)
    dc, dnc, dperm, dbptr, dcptr = iccg.iccg_dev_color_order(dgp, dga, nb, draw)
    torch.cuda.synchronize()
    t_dc = time.perf_counter() - t0
    print(f"\n128^3 graph: host {t_hg * 1e3:.0f} ms, device {t_dg * 1e3:.1f} ms; "
          f"sort + coloring + ordering: host {t_hc * 1e3:.0f} ms, device {t_dc * 1e3:.1f} ms")
    assert np.array_equal(_h(dgp), gp) and np.array_equal(_h(dga), ga)
    assert np.array_equal(_h(draw), block_of)
    assert dnc == nc
    assert np.array_equal(_h(dc), color_of)
    assert np.array_equal(_h(dperm), perm)
    assert np.array_equal(_h(dbptr), bptr)
    assert np.array_equal(_h(dcptr), cptr)


# ---------------------------------------------------------------------------
# device Leiden: not the host partition (parallel moves, greedy refinement),
# so it is held to the method's invariants, to planted partitions, to the
# oracle's quality (Eqs. 1-2) and to the solve the blocking gives
# ---------------------------------------------------------------------------
def _ring_of_cliques(K, k):
    import scipy.sparse as sp
    n = K * k
    rows, cols = [], []
    for c in range(K):
        base = c * k
        for i in range(k):
            for j in range(i + 1, k):
                rows.append(base + i)
                cols.append(base + j)
        rows.append(base + k - 1)
        cols.append(((c + 1) % K) * k)
    m = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    return gen.from_scipy(m + m.T + sp.identity(n))


def _dev_leiden(a, quality, gamma):
    dgp, dga = iccg.iccg_dev_graph(_d(a.rowptr, torch.int64), _d(a.colind, torch.int32))
    bo, nb = iccg.iccg_dev_block_leiden(dgp, dga, quality, gamma)
    torch.cuda.synchronize()
    return _h(bo), nb


def _connected(a, memb, nk):
    """Every community induces a connected subgraph: the graph restricted to
    edges inside communities has exactly nk components."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    gp, ga = oracle.graph(a.n, a.rowptr, a.colind)
    src = np.repeat(np.arange(a.n), np.diff(gp))
    keep = memb[src] == memb[ga]
    adj = sp.csr_matrix((np.ones(int(keep.sum())), (src[keep], ga[keep])), shape=(a.n, a.n))
    ncomp, _ = connected_components(adj, directed=False)
    return ncomp == nk


@pytest.mark.parametrize("K,k", [(8, 6), (12, 5)])
@pytest.mark.parametrize("quality,gamma", [("cpm", 0.3), ("modularity", 1.0)])
def test_device_leiden_planted_cliques(K, k, quality, gamma):
    a = _ring_of_cliques(K, k)
    memb, nb = _dev_leiden(a, quality, gamma)
    assert nb == K
    # the cliques, whatever their labels
    lab = memb.reshape(K, k)
    assert np.all(lab == lab[:, :1]) and len(np.unique(lab[:, 0])) == K


QCASES = {
    "grid2d_40": lambda: gen.poisson2d_5pt(40),
    "grid3d_16": lambda: gen.poisson3d_7pt(16),
    "rgg_4000": lambda: gen.rgg_laplacian(4000, 12.0, 5),
    "diff27_12": lambda: gen.diffusion3d_27pt(12, seed=3),
}


@pytest.mark.parametrize("case", sorted(QCASES))
@pytest.mark.parametrize("quality,gamma", [("cpm", 0.5), ("cpm", 0.1), ("cpm", 0.02), ("modularity", 1.0)])
def test_device_leiden_invariants_and_quality(case, quality, gamma):
    """Labels 0..n_b-1, every block connected, quality above the singleton
    partition's and within 5% of the oracle Leiden's (Eq. 1 / Eq. 2 evaluated
    by the oracle); deterministic."""
    a = QCASES[case]()
    memb, nb = _dev_leiden(a, quality, gamma)
    assert memb.min() == 0 and memb.max() == nb - 1 and len(np.unique(memb)) == nb
    assert _connected(a, memb, nb)
    gp, ga = oracle.graph(a.n, a.rowptr, a.colind)
    qf = oracle.quality_modularity if quality == "modularity" else oracle.quality_cpm
    q_dev = qf(a.n, gp, ga, memb, gamma)
    ref, _ = oracle.leiden(a.n, gp, ga, quality, gamma)
    q_orc = qf(a.n, gp, ga, ref, gamma)
    q_one = qf(a.n, gp, ga, np.arange(a.n), gamma)
    print(f"\n{case} {quality} {gamma}: Q device {q_dev:.5f}, oracle {q_orc:.5f}, singletons {q_one:.5f}")
    assert q_dev >= q_one
    # the quality gained over the singleton partition, against the oracle's
    assert q_dev - q_one >= 0.9 * (q_orc - q_one)
    again, nb2 = _dev_leiden(a, quality, gamma)
    assert nb2 == nb and np.array_equal(again, memb)


@pytest.mark.parametrize("method,gamma", [("leiden_cpm", 0.5), ("leiden_md", 1.0)])
def test_device_blocking_solves_like_host_blocking(method, gamma):
    """ICCG with the device blocking reaches 1e-8, matches the oracle's solve
    in that ordering (1e-10, iterations +-1), and needs at most 10% more
    iterations than with the host blocking."""
    a = gen.poisson3d_7pt(24)
    b = gen.rhs_uniform(a.n, 2)
    bd = iccg.dev_blocking(a, method, gamma)
    bh = oracle.blocking(a, method, gamma=gamma)
    ref_d = oracle.iccg(a, b, bd["perm"], tol=1e-8, maxit=5000)
    ref_h = oracle.iccg(a, b, bh["perm"], tol=1e-8, maxit=5000)
    S = iccg.Solver(a, bd)
    x = np.zeros(a.n)
    st, it, _ = iccg.iccg_solve(S.ctx, b, x, 1e-8, 5000)
    S.close()
    assert st == iccg.ICCG_OK
    assert abs(it - ref_d["iterations"]) <= 1
    assert np.linalg.norm(x - ref_d["x"]) / np.linalg.norm(ref_d["x"]) <= 1e-10
    assert ref_d["iterations"] <= 1.1 * ref_h["iterations"] + 1


def test_device_leiden_full_size_cpm05():
    """128^3, Leiden CPM 0.5 on the device: time, quality against the host
    Leiden's, and the blocking's colors; the whole device pipeline (graph,
    Leiden, size order, coloring, ordering) printed against the host's."""
    a = gen.poisson3d_7pt(128)
    n = a.n
    rp, ci = _d(a.rowptr, torch.int64), _d(a.colind, torch.int32)
    iccg.iccg_dev_graph(rp, ci)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bd = iccg.dev_blocking(a, "leiden_cpm", 0.5)
    t_dev = time.perf_counter() - t0
    t0 = time.perf_counter()
    bh = iccg.blocking(a, "leiden_cpm", gamma=0.5)
    t_host = time.perf_counter() - t0
    gp, ga = iccg.iccg_graph(n, a.rowptr, a.colind)
    q_dev = oracle.quality_cpm(n, gp, ga, bd["block_of"], 0.5)
    q_host = oracle.quality_cpm(n, gp, ga, bh["block_of"], 0.5)
    print(f"\n128^3 CPM 0.5 blocking: device {t_dev * 1e3:.0f} ms (n_b {bd['n_b']}, n_c {bd['n_c']}, Q {q_dev:.5f}); "
          f"host {t_host * 1e3:.0f} ms (n_b {bh['n_b']}, n_c {bh['n_c']}, Q {q_host:.5f})")
    q_one = oracle.quality_cpm(n, gp, ga, np.arange(n), 0.5)
    assert q_dev - q_one >= 0.9 * (q_host - q_one)
    assert _connected(a, bd["block_of"], bd["n_b"])


@pytest.mark.parametrize("s", [1, 2, 8, 32])
def test_device_pipeline_abmc_equals_oracle(s):
    """ABMC through the device pipeline (device graph, host ABMC blocks,
    device coloring and ordering) gives the oracle's ordering exactly."""
    a = gen.diffusion3d_27pt(14, seed=2)
    bd = iccg.dev_blocking(a, "abmc", block_size=s)
    bo = oracle.blocking(a, "abmc", s)
    assert bd["n_b"] == bo["n_b"] and bd["n_c"] == bo["n_c"]
    for k in ("perm", "block_ptr", "color_ptr", "color_of"):
        assert np.array_equal(np.asarray(bd[k]), np.asarray(bo[k])), k


# ---------------------------------------------------------------------------
# the device Leiden against its sequential statement in the oracle
# (par_leiden.c): the same partition, integer for integer
# ---------------------------------------------------------------------------
PAR_CASES = {
    "grid2d_40": lambda: gen.poisson2d_5pt(40),
    "grid3d_20": lambda: gen.poisson3d_7pt(20),
    "rgg_4000": lambda: gen.rgg_laplacian(4000, 12.0, 5),
    "diff27_14": lambda: gen.diffusion3d_27pt(14, seed=3),
    "elast7": lambda: gen.elasticity_like(2000, 7, 3.0),
    "cliques": lambda: _ring_of_cliques(12, 5),
}


@pytest.mark.parametrize("case", sorted(PAR_CASES))
@pytest.mark.parametrize("quality,gamma", [("cpm", 0.5), ("cpm", 0.1), ("cpm", 0.02), ("modularity", 1.0)])
def test_device_leiden_equals_oracle_statement(case, quality, gamma):
    a = PAR_CASES[case]()
    gp, ga = oracle.graph(a.n, a.rowptr, a.colind)
    ref, nref = oracle.par_leiden(a.n, gp, ga, quality, gamma)
    memb, nb = _dev_leiden(a, quality, gamma)
    assert nb == nref
    assert np.array_equal(memb, ref)


def test_device_leiden_equals_oracle_statement_full_size():
    a = gen.poisson3d_7pt(128)
    gp, ga = oracle.graph(a.n, a.rowptr, a.colind)
    ref, nref = oracle.par_leiden(a.n, gp, ga, "cpm", 0.5)
    memb, nb = _dev_leiden(a, "cpm", 0.5)
    assert nb == nref
    assert np.array_equal(memb, ref)


@pytest.mark.parametrize("method,gamma", [("leiden_cpm", 0.5), ("leiden_cpm", 0.05), ("leiden_md", 1.0)])
def test_device_pipeline_parallel_leiden_equals_oracle(method, gamma):
    """The whole device blocking pipeline with the parallel Leiden (graph,
    Leiden, size order, coloring, ordering) gives the ordering of the
    oracle's pipeline with its sequential statement of that Leiden (the
    reference arm of bench.py for the *_par blockings)."""
    a = gen.diffusion3d_27pt(14, seed=2) if method == "leiden_md" else gen.poisson3d_7pt(24)
    bd = iccg.dev_blocking(a, method, gamma)
    gp, ga = oracle.graph(a.n, a.rowptr, a.colind)
    raw, nb = oracle.par_leiden(a.n, gp, ga, "cpm" if method == "leiden_cpm" else "modularity", gamma)
    block_of = oracle.sort_blocks_desc(a.n, nb, raw)
    color_of, nc = oracle.color_blocks(a.n, gp, ga, nb, block_of)
    perm, bptr, cptr = oracle.order(a.n, nb, nc, block_of, color_of)
    assert bd["n_b"] == nb and bd["n_c"] == nc
    assert np.array_equal(bd["perm"], perm)
    assert np.array_equal(bd["block_ptr"], bptr)
    assert np.array_equal(bd["color_ptr"], cptr)
