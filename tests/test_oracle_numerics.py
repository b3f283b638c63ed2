"""Pins for the oracle's IC(0), substitutions, PCG and block statistics.

  * IC(0) (Sec. 3): (L L^T)_ij = a_ij on the pattern; full pattern -> equals
    numpy's Cholesky; tridiagonal -> exact factor; non-SPD -> breakdown row.
  * substitutions (Alg. 1): equal scipy's dense/sparse triangular solves, and
    the block-multicolor order of Alg. 1 (colors in sequence, blocks of one
    color in any order) gives bit-identical results to the sequential order.
  * PCG: tridiagonal with the natural order converges in exactly one
    iteration (M = A); with M = I the iterates equal scipy's CG; small dense
    systems match numpy.linalg.solve; A-norm error decreases monotonically;
    b = A*1 recovers x = 1; b = 0 gives x = 0 in 0 iterations.
  * Gini (Sec. 6.3): closed forms and brute force.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import gen
import oracle


def _factor(a, perm=None):
    perm = np.arange(a.n) if perm is None else perm
    ah = oracle.permute(a, perm)
    lptr, lcol, aval = oracle.tril_csr(ah)
    lval, brow = oracle.ic0(lptr, lcol, aval)
    return ah, lptr, lcol, aval, lval, brow


def _dense_L(lptr, lcol, lval, n):
    return sp.csr_matrix((lval, lcol, lptr), shape=(n, n)).toarray()


@pytest.mark.parametrize("case", ["grid2d", "grid3d", "rspd", "aniso27"])
def test_ic0_reproduces_a_on_pattern(case):
    a = {"grid2d": lambda: gen.poisson2d_5pt(12), "grid3d": lambda: gen.poisson3d_7pt(6),
         "rspd": lambda: gen.random_spd_small(150, 0.05, 3),
         "aniso27": lambda: gen.stencil_aniso("27pt", 300, 5.0)}[case]()
    bl = oracle.blocking(a, "abmc", 8)
    ah, lptr, lcol, aval, lval, brow = _factor(a, bl["perm"])
    assert brow == -1
    L = _dense_L(lptr, lcol, lval, a.n)
    LLt = L @ L.T
    A = ah.toarray()
    mask = np.tril(A != 0)
    rel = np.abs(LLt - A)[mask] / np.abs(A).max()
    assert rel.max() < 1e-13


def test_ic0_full_pattern_is_cholesky():
    rng = np.random.default_rng(0)
    m = rng.standard_normal((40, 40))
    A = m @ m.T + 40 * np.eye(40)
    a = gen.from_scipy(sp.csr_matrix(A))
    _, lptr, lcol, _, lval, brow = _factor(a)
    assert brow == -1
    L = _dense_L(lptr, lcol, lval, a.n)
    assert np.allclose(L, np.linalg.cholesky(A), rtol=1e-13, atol=1e-13)


def test_ic0_tridiagonal_is_exact():
    n = 50
    d = np.linspace(3.0, 5.0, n)
    e = -np.linspace(0.5, 1.5, n - 1)
    A = sp.diags([e, d, e], [-1, 0, 1], format="csr")
    a = gen.from_scipy(A)
    _, lptr, lcol, _, lval, brow = _factor(a)
    L = _dense_L(lptr, lcol, lval, n)
    assert np.allclose(L @ L.T, A.toarray(), rtol=0, atol=1e-14)
    assert np.allclose(L, np.linalg.cholesky(A.toarray()), atol=1e-14)


def test_ic0_breakdown_reports_row():
    A = sp.csr_matrix(np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]]))
    a = gen.from_scipy(A)
    _, _, _, _, _, brow = _factor(a)
    assert brow == 1
    r = oracle.iccg(a, np.ones(3), np.array([2, 0, 1]))
    assert r["status"] == "breakdown" and r["breakdown_row"] == 1


@pytest.mark.parametrize("seed", range(3))
def test_substitutions_match_dense_triangular_solve(seed):
    a = gen.random_spd_small(120, 0.06, seed)
    bl = oracle.blocking(a, "abmc", 6)
    _, lptr, lcol, _, lval, _ = _factor(a, bl["perm"])
    L = _dense_L(lptr, lcol, lval, a.n)
    r = np.random.default_rng(seed).uniform(-1, 1, a.n)
    y = oracle.forward(lptr, lcol, lval, r)
    z = oracle.backward(lptr, lcol, lval, y)
    y_ref = sla.solve_triangular(L, r, lower=True)
    z_ref = sla.solve_triangular(L.T, y_ref, lower=False)
    assert np.max(np.abs(y - y_ref)) <= 1e-13 * np.max(np.abs(y_ref))
    assert np.max(np.abs(z - z_ref)) <= 1e-13 * np.max(np.abs(z_ref))


def test_substitutions_match_sparse_solver_config1():
    a, b, opt = gen.config1()
    bl = oracle.blocking(a, "abmc", opt["block_size"])
    _, lptr, lcol, _, lval, _ = _factor(a, bl["perm"])
    L = sp.csr_matrix((lval, lcol, lptr), shape=(a.n, a.n))
    r = b[bl["perm"]]
    y = oracle.forward(lptr, lcol, lval, r)
    z = oracle.backward(lptr, lcol, lval, y)
    y_ref = spla.spsolve_triangular(L, r, lower=True)
    z_ref = spla.spsolve_triangular(L.T.tocsr(), y_ref, lower=False)
    assert np.max(np.abs(y - y_ref)) <= 1e-13 * np.max(np.abs(y_ref))
    assert np.max(np.abs(z - z_ref)) <= 1e-13 * np.max(np.abs(z_ref))


def _alg1_forward(lptr, lcol, lval, r, bp, cp, block_order_rng):
    """Alg. 1 literally: colors in sequence; the blocks of one color in a
    shuffled order (any order is a valid parallel schedule); rows ascending."""
    n = len(r)
    y = np.full(n, np.nan)
    for c in range(len(cp) - 1):
        blocks = list(range(cp[c], cp[c + 1]))
        block_order_rng.shuffle(blocks)
        for j in blocks:
            for i in range(bp[j], bp[j + 1]):
                s = r[i]
                for p in range(lptr[i], lptr[i + 1] - 1):
                    s -= lval[p] * y[lcol[p]]
                y[i] = s / lval[lptr[i + 1] - 1]
    return y


@pytest.mark.parametrize("method,kw", [("abmc", {"block_size": 5}), ("leiden_cpm", {"gamma": 0.1})])
def test_block_multicolor_order_equals_sequential(method, kw):
    a = gen.poisson2d_5pt(16)
    bl = oracle.blocking(a, method, **kw)
    _, lptr, lcol, _, lval, _ = _factor(a, bl["perm"])
    r = np.random.default_rng(3).uniform(-1, 1, a.n)
    y_seq = oracle.forward(lptr, lcol, lval, r)
    y_par = _alg1_forward(lptr, lcol, lval, r, bl["block_ptr"], bl["color_ptr"],
                          np.random.default_rng(9))
    assert np.array_equal(y_seq, y_par)   # same per-row arithmetic -> bit-identical


def test_pcg_tridiagonal_converges_in_one_iteration():
    n = 200
    A = sp.diags([-np.ones(n - 1), 2.5 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    a = gen.from_scipy(A)
    b = np.random.default_rng(0).uniform(-1, 1, n)
    r = oracle.iccg(a, b, np.arange(n), tol=1e-12)
    assert r["iterations"] == 1
    assert r["true_relres"] < 1e-13


def test_pcg_with_identity_preconditioner_matches_scipy_cg():
    a = gen.poisson2d_5pt(15)
    ah = a.to_scipy()
    n = a.n
    lptr = np.arange(n + 1, dtype=np.int64)
    lcol = np.arange(n, dtype=np.int32)
    lval = np.ones(n)
    b = np.random.default_rng(1).uniform(-1, 1, n)
    for k in (1, 3, 10, 25):
        x, it, _, _ = oracle.pcg(ah, lptr, lcol, lval, b, tol=0.0, maxit=k)
        assert it == k
        xs, _ = spla.cg(ah, b, x0=np.zeros(n), rtol=0.0, atol=0.0, maxiter=k)
        assert np.max(np.abs(x - xs)) <= 1e-10 * np.max(np.abs(xs))


def test_pcg_dense_small_matches_solve_and_a_norm_decreases():
    rng = np.random.default_rng(2)
    m = rng.standard_normal((30, 30))
    A = m @ m.T + 5 * np.eye(30)
    a = gen.from_scipy(sp.csr_matrix(A * (np.abs(A) > 2.0) + np.diag(np.diag(A))))
    Ad = a.to_scipy().toarray()
    assert np.linalg.eigvalsh(Ad).min() > 0
    b = rng.uniform(-1, 1, 30)
    xs = np.linalg.solve(Ad, b)
    perm = np.arange(30)
    ah, lptr, lcol, aval, lval, brow = _factor(a, perm)
    assert brow == -1
    errs = []
    for k in range(1, 15):
        x, it, _, _ = oracle.pcg(ah, lptr, lcol, lval, b, tol=0.0, maxit=k)
        e = x - xs
        errs.append(float(e @ Ad @ e))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) for i in range(len(errs) - 1) if errs[i] > 1e-24)
    r = oracle.iccg(a, b, perm, tol=1e-12)
    kappa = np.linalg.cond(Ad)
    assert np.linalg.norm(r["x"] - xs) / np.linalg.norm(xs) <= kappa * 1e-12 * 10


def test_pcg_config1_recovers_ones():
    a, b, opt = gen.config1()
    bl = oracle.blocking(a, "abmc", opt["block_size"])
    r = oracle.iccg(a, b, bl["perm"])
    assert r["status"] == "converged"
    assert r["hist"][-1] <= 1e-8 and r["hist"][-2] > 1e-8
    assert len(r["hist"]) == r["iterations"] + 1
    assert np.max(np.abs(r["x"] - 1.0)) < 1e-5
    assert r["true_relres"] < 1e-7


def test_pcg_zero_rhs():
    a = gen.poisson2d_5pt(8)
    r = oracle.iccg(a, np.zeros(a.n), np.arange(a.n))
    assert r["iterations"] == 0 and np.all(r["x"] == 0)


def test_gini_closed_forms_and_bruteforce():
    assert oracle.gini([5, 5, 5, 5]) == 0.0
    nb = 10
    assert abs(oracle.gini([0] * (nb - 1) + [7]) - (nb - 1) / nb) < 1e-15
    s = np.random.default_rng(0).integers(1, 100, size=37)
    brute = np.abs(s[:, None] - s[None, :]).sum() / (2 * len(s) ** 2 * s.mean())
    assert abs(oracle.gini(s) - brute) < 1e-14


def test_block_stats_definitions():
    bp = np.array([0, 4, 6, 12, 13])   # sizes 4, 2, 6, 1
    cp = np.array([0, 2, 4])           # colors: {4, 2} and {6, 1}
    st = oracle.block_stats(bp, cp)
    assert st["n_b"] == 4 and st["n_c"] == 2 and st["B_max"] == 6
    assert abs(st["B_max/B_avg"] - 6 / 3.25) < 1e-15
    assert abs(st["C_max/C_avg"] - 7 / 6.5) < 1e-15
