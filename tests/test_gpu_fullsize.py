"""GPU parity at the benchmark's full size: the 128^3 7-point Poisson problem
(n = 2,097,152, nnz = 14,581,760, b ~ U[-1, 1] seed 0) in the layout bench.py
times (the parallel Leiden at CPM resolution 0.5 on the device + greedy
coloring, automatic tile mapping), with the sequential Leiden CPM 0.5 blocking
and with ABMC s = 8.

  * blockings: the library's permutation, block and color pointers equal the
    oracle's bit for bit (integer work);
  * IC(0): (L L^T)_ij = a_ij on the pattern of L (the defining property of
    IC(0), any size) on sampled rows, and L_ii > 0;
  * SpMV against scipy on the whole vector;
  * preconditioner: L L^T z = r on the whole vector (two scipy products);
  * FP64 solve against the oracle's full solve (one run, ~10 s on the host):
    relative error <= 1e-10, iterations within +-1, true residual <= 1e-8;
  * FP32 preconditioner: true residual <= 1e-8 within the same iteration
    count +-2, error against the FP64 oracle <= 1e-6.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle
from paper_2609_00561_gb300 import build as libbuild
from paper_2609_00561_gb300 import iccg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LAYOUTS = {"cpm05": ("leiden_cpm", {"gamma": 0.5}), "abmc8": ("abmc", {"block_size": 8}),
           "cpm05par": ("leiden_cpm_par", {"gamma": 0.5})}


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


@pytest.fixture(scope="module")
def problem():
    a, b, _ = gen.config2()
    return a, b


_bl = {}


def _oracle_par_blocking(a, gamma):
    """The oracle's pipeline around its sequential statement of the parallel
    Leiden (the bench default's blocking)."""
    gp, ga = oracle.graph(a.n, a.rowptr, a.colind)
    raw, nb = oracle.par_leiden(a.n, gp, ga, "cpm", gamma)
    block_of = oracle.sort_blocks_desc(a.n, nb, raw)
    color_of, nc = oracle.color_blocks(a.n, gp, ga, nb, block_of)
    perm, bptr, cptr = oracle.order(a.n, nb, nc, block_of, color_of)
    return {"perm": perm, "block_ptr": bptr, "color_ptr": cptr, "n_b": nb, "n_c": nc}


def _blocking(a, name):
    if name not in _bl:
        method, kw = LAYOUTS[name]
        if method == "leiden_cpm_par":
            _bl[name] = (_oracle_par_blocking(a, kw["gamma"]), iccg.dev_blocking(a, "leiden_cpm", kw["gamma"]))
        else:
            _bl[name] = (oracle.blocking(a, method, **kw), iccg.blocking(a, method, **kw))
    return _bl[name]


_sol = {}


def _oracle_solution(a, b, name):
    if name not in _sol:
        bo, _ = _blocking(a, name)
        _sol[name] = oracle.iccg(a, b, bo["perm"], tol=1e-8, maxit=5000)
    return _sol[name]


@pytest.fixture(scope="module")
def oracle_solve(problem):
    a, b = problem
    return _oracle_solution(a, b, "cpm05")


@pytest.mark.parametrize("name", sorted(LAYOUTS))
def test_blocking_bit_exact_at_full_size(problem, name):
    a, _ = problem
    bo, bp = _blocking(a, name)
    for k in ("perm", "block_ptr", "color_ptr"):
        assert np.array_equal(np.asarray(bo[k]), np.asarray(bp[k])), k
    assert (bo["n_b"], bo["n_c"]) == (bp["n_b"], bp["n_c"])


@pytest.mark.parametrize("name", sorted(LAYOUTS))
def test_factor_spmv_precond_at_full_size(problem, name):
    a, b = problem
    _, bl = _blocking(a, name)
    S = iccg.Solver(a, bl)
    ah = oracle.permute(a, bl["perm"])
    lptr, lcol, aval = oracle.tril_csr(ah)
    lval = iccg.iccg_get_factor(S.ctx)
    n = a.n
    L = sp.csr_matrix((lval, lcol, lptr), shape=(n, n))
    assert np.all(L.diagonal() > 0)
    # (L L^T)_ij = a_ij for (i, j) in the pattern of L, on sampled rows
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([rng.choice(n, 3000, replace=False), [0, n - 1]]))
    Lr = L[rows]
    prod = (Lr @ L.T).tocsr()
    for k, i in enumerate(rows):
        for e in range(lptr[i], lptr[i + 1]):
            j = lcol[e]
            assert abs(prod[k, j] - aval[e]) <= 1e-12 * max(1.0, abs(aval[e])), (i, j)
    # SpMV on the whole vector
    p = rng.uniform(-1, 1, n)
    q = np.zeros(n)
    iccg.iccg_spmv(S.ctx, p, q)
    qref = a.to_scipy() @ p
    assert np.max(np.abs(q - qref)) <= 1e-13 * np.max(np.abs(qref))
    # preconditioner: L L^T z_hat = r_hat in the permuted order
    z = np.zeros(n)
    iccg.iccg_precond(S.ctx, p, z)
    perm = np.asarray(bl["perm"])
    zh, rh = z[perm], p[perm]
    res = L @ (L.T @ zh) - rh
    assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(rh)
    S.close()


@pytest.mark.parametrize("name", ["cpm05", "cpm05par"])
def test_solve_fp64_matches_oracle_at_full_size(problem, name):
    a, b = problem
    _, bl = _blocking(a, name)
    S = iccg.Solver(a, bl)
    x = np.zeros(a.n)
    st, it, hist = iccg.iccg_solve(S.ctx, b, x, 1e-8, 5000)
    S.close()
    ref = _oracle_solution(a, b, name)
    assert st == iccg.ICCG_OK
    assert abs(it - ref["iterations"]) <= 1, (it, ref["iterations"])
    err = float(np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]))
    assert err <= 1e-10, err
    true_rel = np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)
    assert true_rel <= 1e-8


@pytest.mark.parametrize("name", ["cpm05", "cpm05par"])
def test_solve_fp32_preconditioner_at_full_size(problem, name):
    a, b = problem
    _, bl = _blocking(a, name)
    S = iccg.Solver(a, bl, precond_fp32=True)
    x = np.zeros(a.n)
    st, it, hist = iccg.iccg_solve(S.ctx, b, x, 1e-8, 5000)
    S.close()
    ref = _oracle_solution(a, b, name)
    assert st == iccg.ICCG_OK and abs(it - ref["iterations"]) <= 2, (it, ref["iterations"])
    assert np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b) <= 1e-8
    assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-6


def test_leiden_md_split_levels_at_full_size(problem):
    """Leiden modularity on 128^3 gives tens of blocks of tens of thousands of
    rows; split into in-block levels (one color of one-row blocks per level of
    a color) the solve runs all rows of a level in parallel and matches the
    oracle's solve on the same ordering (the IC(0) of the unsplit ordering,
    pinned on the host)."""
    a, b = problem
    bo = oracle.blocking(a, "leiden_md", gamma=1.0)
    bp = iccg.blocking(a, "leiden_md", gamma=1.0)
    for k in ("perm", "block_ptr", "color_ptr"):
        assert np.array_equal(np.asarray(bo[k]), np.asarray(bp[k])), k
    assert np.diff(bp["block_ptr"]).max() > 1000
    sl = iccg.iccg_split_levels(a, bp, 32)
    ref = oracle.iccg(a, b, sl["perm"], tol=1e-8, maxit=5000)
    S = iccg.Solver(a, sl)
    x = np.zeros(a.n)
    st, it, _ = iccg.iccg_solve(S.ctx, b, x, 1e-8, 5000)
    S.close()
    assert st == iccg.ICCG_OK
    assert abs(it - ref["iterations"]) <= 1, (it, ref["iterations"])
    assert np.linalg.norm(x - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])
