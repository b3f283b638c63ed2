"""CPU checks of the C-ABI library (no GPU compute calls).

  * libiccg.so loads and exports every function declared in include/iccg.h;
  * iccg_setup rejects bad inputs before touching the GPU (argument errors,
    non-permutations, the coloring invariant of Sec. 3);
  * the production host blocking (graph, ABMC, Leiden, block sort, greedy
    coloring, ordering) equals the oracle's bit for bit.
"""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle
from paper_2609_00561_gb300 import build as libbuild
from paper_2609_00561_gb300 import iccg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def _declared():
    txt = open(os.path.join(ROOT, "include", "iccg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(iccg_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert "iccg_setup" in names and "iccg_solve" in names and "iccg_factor" in names
    lib = ctypes.CDLL(iccg.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def _setup_err(a, perm, bp, cp, nb, nc):
    with pytest.raises(iccg.IccgError) as ei:
        iccg.iccg_setup(a.n, a.nnz, a.rowptr, a.colind, a.val, perm, bp, cp, nb, nc)
    return ei.value


def test_setup_rejects_bad_inputs_before_gpu():
    a = gen.poisson2d_5pt(6)
    bl = oracle.blocking(a, "abmc", 4)
    perm, bp, cp, nb, nc = bl["perm"], bl["block_ptr"], bl["color_ptr"], bl["n_b"], bl["n_c"]
    bad = perm.copy(); bad[0] = bad[1]
    assert _setup_err(a, bad, bp, cp, nb, nc).status == 1
    bbp = bp.copy(); bbp[-1] += 1
    assert _setup_err(a, perm, bbp, cp, nb, nc).status == 1
    bcp = cp.copy(); bcp[1] = bcp[0]
    assert _setup_err(a, perm, bp, bcp, nb, nc).status == 1
    # all blocks in one color: adjacent blocks share a color -> coloring error
    e = _setup_err(a, perm, bp, np.array([0, nb], dtype=np.int32), nb, 1)
    assert e.status == 2 and 0 <= e.index < nb
    # missing diagonal
    m = a.to_scipy().tolil(); m[3, 3] = 0; m = m.tocsr(); m.eliminate_zeros()
    a2 = gen.CSR(a.n, m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data)
    assert _setup_err(a2, perm, bp, cp, nb, nc).status == 1
    # unsymmetric pattern
    m = a.to_scipy().tolil(); m[0, 20] = -0.5; m = m.tocsr()
    a3 = gen.CSR(a.n, m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data)
    assert _setup_err(a3, perm, bp, cp, nb, nc).status == 1
    # out-of-range column
    a4 = gen.CSR(a.n, a.rowptr.copy(), a.colind.copy(), a.val.copy()); a4.colind[5] = a.n
    assert _setup_err(a4, perm, bp, cp, nb, nc).status == 1
    # non-finite value
    a5 = gen.CSR(a.n, a.rowptr.copy(), a.colind.copy(), a.val.copy()); a5.val[7] = np.nan
    assert _setup_err(a5, perm, bp, cp, nb, nc).status == 1
    # invalid options: solver id, warps per CTA, rows per thread, lane blocks, tile mapping
    for kw in (dict(solver=3), dict(solver=-1), dict(warps_per_cta=17), dict(rows_per_thread=3),
               dict(lane_block_max=33), dict(lane_block_max=-2), dict(tile_mapping=5), dict(tile_mapping=-1)):
        with pytest.raises(iccg.IccgError) as ei:
            iccg.iccg_setup(a.n, a.nnz, a.rowptr, a.colind, a.val, perm, bp, cp, nb, nc, iccg.make_opts(**kw))
        assert ei.value.status == 1, kw
    # batched: null contexts, bad right-hand-side counts
    import ctypes
    L = iccg.load()
    h = ctypes.c_void_p()
    for nsys, nrhs in ((0, 4), (1, 0), (1, 33)):
        assert L.iccg_batch_create(ctypes.byref(h), None, nsys, nrhs, None) == 1


CASES = {
    "grid2d": lambda: gen.poisson2d_5pt(40),
    "grid3d": lambda: gen.poisson3d_7pt(14),
    "aniso27": lambda: gen.stencil_aniso("27pt", 3000, 7.0),
    "rgg": lambda: gen.rgg_laplacian(3000, 14.0, 2),
    "elast": lambda: gen.elasticity_like(600, 7, 2.0),
    "rspd": lambda: gen.random_spd_small(500, 0.01, 1),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_graph_equals_oracle(case):
    a = CASES[case]()
    g1 = iccg.iccg_graph(a.n, a.rowptr, a.colind)
    g2 = oracle.graph(a.n, a.rowptr, a.colind)
    assert np.array_equal(g1[0], g2[0]) and np.array_equal(g1[1], g2[1])


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("s", [1, 8, 32, 100])
def test_abmc_coloring_order_equal_oracle(case, s):
    a = CASES[case]()
    p = iccg.blocking(a, "abmc", s)
    o = oracle.blocking(a, "abmc", s)
    for k in ("block_of", "color_of", "perm", "block_ptr", "color_ptr"):
        assert np.array_equal(p[k], o[k]), k
    assert p["n_b"] == o["n_b"] and p["n_c"] == o["n_c"]


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("method,gamma", [("leiden_md", 1.0), ("leiden_md", 4.0), ("leiden_cpm", 0.01),
                                          ("leiden_cpm", 0.1), ("leiden_cpm", 0.5)])
def test_leiden_equals_oracle(case, method, gamma):
    a = CASES[case]()
    for seed in (42, 9):
        p = iccg.blocking(a, method, gamma=gamma, seed=seed)
        o = oracle.blocking(a, method, gamma=gamma, seed=seed)
        for k in ("block_of", "color_of", "perm", "block_ptr", "color_ptr"):
            assert np.array_equal(p[k], o[k]), (k, seed)


def test_leiden_iteration_count_and_beta_are_honoured():
    a = CASES["grid2d"]()
    gptr, gadj = iccg.iccg_graph(a.n, a.rowptr, a.colind)
    for n_iter in (1, 3):
        for beta in (0.01, 1.0):
            m1, k1 = iccg.iccg_block_leiden(a.n, gptr, gadj, "cpm", 0.05, n_iter, beta, 7)
            m2, k2 = oracle.leiden(a.n, gptr, gadj, "cpm", 0.05, n_iter, beta, 7)
            assert k1 == k2 and np.array_equal(m1, m2)


@pytest.mark.parametrize("name", sorted(CASES))
def test_level_order_equals_oracle(name):
    a = CASES[name]()
    gptr, gadj = iccg.iccg_graph(a.n, a.rowptr, a.colind)
    lev, nl, perm, bptr, cptr = iccg.iccg_level_order(a.n, gptr, gadj)
    og, oa = oracle.graph(a.n, a.rowptr, a.colind)
    olev, onl, operm, obptr, ocptr = oracle.level_order(a.n, og, oa)
    assert nl == onl and np.array_equal(lev, olev) and np.array_equal(perm, operm)
    assert np.array_equal(bptr, obptr) and np.array_equal(cptr, ocptr)


@pytest.mark.parametrize("case", ["md2d", "md3d", "abmc100"])
def test_split_levels_equals_oracle(case):
    if case == "md2d":
        a = gen.poisson2d_5pt(30)
        bl = oracle.blocking(a, "leiden_md", gamma=1.0)
    elif case == "md3d":
        a = gen.poisson3d_7pt(12)
        bl = oracle.blocking(a, "leiden_md", gamma=1.0)
    else:
        a = gen.stencil_aniso("27pt", 2000, 5.0)
        bl = oracle.blocking(a, "abmc", 100)
    got = iccg.iccg_split_levels(a, bl, 32)
    want = oracle.split_levels(a, bl, 32)
    for k in ("perm", "block_ptr", "color_ptr"):
        assert np.array_equal(got[k], want[k]), k
    assert got["n_b"] == want["n_b"] and got["n_c"] == want["n_c"]
    st, *_ = iccg.check_layout(a, got)
    assert st == 0
