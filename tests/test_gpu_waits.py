"""Bounded device-side waits: a wait that runs out returns an error status.

The persistent solver and the cooperative sweep (layouts of one- and two-row
blocks) separate the colors of Alg. 1 by grid barriers, and the batched
solver separates its phases by per-system barriers.  Every barrier wait gives up after a wall-time limit,
sets an error word, and the kernel returns; the host reads ICCG_ERR_TIMEOUT.
Here the limit is set to 1 ns, so the first CTA that has to wait at all gives
up (no fault, no hang: the kernel ends normally with an error status).  The
same context then solves again with the default limit and matches the oracle.
"""
import numpy as np
import pytest

import gen
import oracle
from paper_2609_00561_gb300 import build as libbuild
from paper_2609_00561_gb300 import iccg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TIMEOUT = 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def _rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def test_persistent_wait_runs_out_then_context_solves():
    a = gen.poisson3d_7pt(20)
    b = gen.rhs_uniform(a.n, 3)
    bl = oracle.blocking(a, "abmc", 8)
    ref = oracle.iccg(a, b, bl["perm"], tol=1e-8, maxit=5000)
    S = iccg.Solver(a, bl, solver="persistent")
    iccg.iccg_set_wait_limit(S.ctx, 1)
    x = np.zeros(a.n)
    with pytest.raises(iccg.IccgError) as ei:
        iccg.iccg_solve(S.ctx, b, x, 1e-8, 5000)
    assert ei.value.status == TIMEOUT
    _, msg = iccg.iccg_last_error(S.ctx)
    assert "gave up" in msg
    # default limit again: the same context solves and matches the oracle
    iccg.iccg_set_wait_limit(S.ctx, 0)
    x = np.zeros(a.n)
    st, it, _ = iccg.iccg_solve(S.ctx, b, x, 1e-8, 5000)
    assert st == iccg.ICCG_OK
    assert abs(it - ref["iterations"]) <= 1
    assert _rel(x, ref["x"]) <= 1e-10
    S.close()


@pytest.mark.parametrize("fuse", [1, 2])
@pytest.mark.parametrize("fp32", [False, True])
def test_cooperative_sweep_wait_runs_out_then_context_solves(fp32, fuse):
    a = gen.poisson3d_7pt(40)
    b = gen.rhs_uniform(a.n, 5)
    bl = oracle.blocking(a, "leiden_cpm", gamma=0.5)
    ref = oracle.iccg(a, b, bl["perm"], tol=1e-8, maxit=5000)
    S = iccg.Solver(a, bl, precond_fp32=fp32, fuse_sweep=fuse)
    assert iccg.iccg_info(S.ctx)["fused_sweep"] == fuse
    iccg.iccg_set_wait_limit(S.ctx, 1)
    x = np.zeros(a.n)
    with pytest.raises(iccg.IccgError) as ei:
        iccg.iccg_solve(S.ctx, b, x, 1e-8, 5000)
    assert ei.value.status == TIMEOUT
    iccg.iccg_set_wait_limit(S.ctx, 0)
    x = np.zeros(a.n)
    st, it, _ = iccg.iccg_solve(S.ctx, b, x, 1e-8, 5000)
    assert st == iccg.ICCG_OK
    if not fp32:
        assert abs(it - ref["iterations"]) <= 1
        assert _rel(x, ref["x"]) <= 1e-10
    S.close()


def test_batched_wait_runs_out_then_batch_solves():
    systems = [(gen.poisson3d_7pt(s), s) for s in (10, 12)]
    nrhs = 4
    solvers, B, refs = [], [], []
    for k, (a, _) in enumerate(systems):
        bl = oracle.blocking(a, "abmc", 8)
        solvers.append(iccg.Solver(a, bl, lane_block_max=-1))
        bk = np.random.default_rng(40 + k).uniform(-1, 1, (nrhs, a.n))
        B.append(bk)
        refs.append(oracle.iccg(a, bk[0], bl["perm"], tol=1e-8, maxit=5000))
    bs = iccg.BatchSolver(solvers, nrhs)
    bs.set_wait_limit(1)
    X = [np.zeros_like(bk) for bk in B]
    with pytest.raises(iccg.IccgError) as ei:
        bs.solve(B, X, 1e-8, 5000)
    assert ei.value.status == TIMEOUT
    bs.set_wait_limit(0)
    X = [np.zeros_like(bk) for bk in B]
    st, its, stv, _ = bs.solve(B, X, 1e-8, 5000)
    assert st == iccg.ICCG_OK and np.all(stv == 0)
    for k in range(len(systems)):
        assert abs(int(its[k, 0]) - refs[k]["iterations"]) <= 1
        assert _rel(X[k][0], refs[k]["x"]) <= 1e-10
    bs.close()
    for S in solvers:
        S.close()
