"""GPU parity of the batched solve (many systems, several right-hand sides,
one launch) against the CPU oracle, system by system and right-hand side by
right-hand side.

Bars: FP64 preconditioner: ||x - x_orc|| / ||x_orc|| <= 1e-10 and iteration
counts within +-1 (the single-system bar); FP32 preconditioner: true
residual <= 1e-7, error against the FP64 oracle <= 1e-6 x (iterations / 10),
iterations within 3 + 10%.  Converged right-hand sides are frozen while the
others continue (a zero right-hand side, an exact x0), and maxit is honoured
per right-hand side.
"""
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


def _batch(sides, shifts, nrhs, block, seed):
    rng = np.random.default_rng(seed)
    out = []
    for side, d in zip(sides, shifts):
        a = gen.poisson3d_7pt(side, shift=d)
        bl = oracle.blocking(a, "abmc", block)
        b = rng.uniform(-1.0, 1.0, size=(nrhs, a.n))
        out.append((a, bl, b))
    return out


def _rel(x, y):
    return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))


_ref_cache = {}


def _refs(systems, key):
    if key not in _ref_cache:
        _ref_cache[key] = [[oracle.iccg(a, b[j], bl["perm"], tol=1e-8, maxit=5000) for j in range(b.shape[0])]
                           for a, bl, b in systems]
    return _ref_cache[key]


SMALL = dict(sides=[5, 9, 12, 7, 10], shifts=[1e-3, 1e-2, 1e-4, 5e-2, 0.0], nrhs=3, block=8, seed=3)


@pytest.mark.parametrize("shape", [dict(), dict(warps_per_cta=4, ctas_per_sm=1), dict(warps_per_cta=16),
                                   dict(rows_per_thread=2), dict(rows_per_thread=4, warps_per_cta=4)])
def test_batched_fp64_matches_oracle(shape):
    systems = _batch(**SMALL)
    refs = _refs(systems, "small")
    solvers = [iccg.Solver(a, bl, lane_block_max=-1) for a, bl, b in systems]
    bs = iccg.BatchSolver(solvers, SMALL["nrhs"], **shape)
    B = [np.ascontiguousarray(b) for _, _, b in systems]
    X = [np.zeros_like(b) for b in B]
    st, it, stv, hist = bs.solve(B, X, 1e-8, 5000, want_hist=True)
    assert st == iccg.ICCG_OK and np.all(stv == 0)
    for s, (a, bl, b) in enumerate(systems):
        for j in range(b.shape[0]):
            ref = refs[s][j]
            assert abs(int(it[s, j]) - ref["iterations"]) <= 1
            assert _rel(X[s][j], ref["x"]) <= 1e-10
            k = min(int(it[s, j]), ref["iterations"]) + 1
            assert np.allclose(hist[s][:k, j], ref["hist"][:k], rtol=1e-3, atol=0)
    bs.close()
    for S in solvers:
        S.close()


def test_batched_fp32_preconditioner():
    systems = _batch(**SMALL)
    refs = _refs(systems, "small")
    solvers = [iccg.Solver(a, bl, lane_block_max=-1, precond_fp32=True) for a, bl, b in systems]
    bs = iccg.BatchSolver(solvers, SMALL["nrhs"])
    B = [np.ascontiguousarray(b) for _, _, b in systems]
    X = [np.zeros_like(b) for b in B]
    st, it, stv, _ = bs.solve(B, X, 1e-8, 5000)
    assert st == iccg.ICCG_OK
    for s, (a, bl, b) in enumerate(systems):
        m = a.to_scipy()
        for j in range(b.shape[0]):
            ref = refs[s][j]
            assert np.linalg.norm(b[j] - m @ X[s][j]) / np.linalg.norm(b[j]) <= 1e-7
            assert _rel(X[s][j], ref["x"]) <= 1e-6 * max(1.0, ref["iterations"] / 10.0)
            assert abs(int(it[s, j]) - ref["iterations"]) <= 3 + ref["iterations"] // 10
    bs.close()
    for S in solvers:
        S.close()


def test_batched_masks_converged_and_honours_maxit():
    systems = _batch(sides=[8, 11], shifts=[1e-3, 0.0], nrhs=4, block=8, seed=5)
    refs = _refs(systems, "mask")
    solvers = [iccg.Solver(a, bl, lane_block_max=-1) for a, bl, b in systems]
    bs = iccg.BatchSolver(solvers, 4)
    B = [np.ascontiguousarray(b.copy()) for _, _, b in systems]
    B[0][1] = 0.0                                   # b = 0 -> x = 0, 0 iterations
    X = [np.zeros_like(b) for b in B]
    X[1][2] = refs[1][2]["x"]                       # x0 = the solution -> 0 iterations at tol 1e-6
    st, it, stv, _ = bs.solve(B, X, 1e-6, 5000)
    assert it[0, 1] == 0 and np.all(X[0][1] == 0.0) and stv[0, 1] == 0
    assert it[1, 2] == 0 and stv[1, 2] == 0
    r = oracle.iccg(systems[0][0], B[0][0], systems[0][1]["perm"], tol=1e-6)
    assert abs(int(it[0, 0]) - r["iterations"]) <= 1 and _rel(X[0][0], r["x"]) <= 1e-10
    # maxit = 3: every non-trivial right-hand side stops at 3, not converged
    X = [np.zeros_like(b) for b in B]
    st, it, stv, _ = bs.solve(B, X, 1e-12, 3)
    assert st == iccg.ICCG_NOT_CONVERGED
    assert it[0, 0] == 3 and stv[0, 0] == 4 and it[0, 1] == 0
    bs.close()
    for S in solvers:
        S.close()


def test_batched_device_buffers_and_autotune():
    systems = _batch(sides=[6, 9, 7], shifts=[1e-2, 1e-3, 0.0], nrhs=16, block=8, seed=7)
    solvers = [iccg.Solver(a, bl, lane_block_max=-1) for a, bl, b in systems]
    bs = iccg.BatchSolver(solvers, 16, autotune=True)
    info = bs.info()
    assert info["kp"] == 16 and info["warps_per_cta"] in (4, 8, 16) and info["grid"] >= 3
    assert info["rows_per_thread"] in (1, 2, 4)
    B = [torch.tensor(b, device="cuda") for _, _, b in systems]
    X = [torch.zeros_like(b) for b in B]
    st, it, stv, _ = bs.solve(B, X, 1e-8, 5000)
    assert st == iccg.ICCG_OK
    Xh = [np.zeros(b.shape) for _, _, b in systems]
    bs.solve([np.ascontiguousarray(b) for _, _, b in systems], Xh, 1e-8, 5000)
    for s in range(3):
        assert np.array_equal(X[s].cpu().numpy(), Xh[s])   # deterministic, host == device buffers
        for j in (0, 7, 15):
            ref = oracle.iccg(systems[s][0], systems[s][2][j], systems[s][1]["perm"])
            assert _rel(Xh[s][j], ref["x"]) <= 1e-10
    bs.close()
    for S in solvers:
        S.close()


def test_batched_rejects_lane_tile_contexts():
    a = gen.poisson3d_7pt(6)
    bl = oracle.blocking(a, "abmc", 8)
    S = iccg.Solver(a, bl)                          # warp units (default for 8-row blocks)
    with pytest.raises(iccg.IccgError) as ei:
        iccg.BatchSolver([S], 2)
    assert ei.value.status == 1
    S.close()
    S = iccg.Solver(a, bl, tile_mapping="cta")      # lane tiles
    with pytest.raises(iccg.IccgError) as ei:
        iccg.BatchSolver([S], 2)
    assert ei.value.status == 1
    S.close()
