"""The allocation-free SpMV + dot entry point (iccg_spmv_dot_noalloc).

It serves callers that cannot allocate device memory where they need the
product (latency-critical loops that must not meet the allocator's implicit
synchronisation, host frameworks that own all device memory).  Its scratch is
a fixed array in the library's device image, shared by all calls.  These
tests call it through the C ABI twice in a row on the same inputs and check
both results against the existing entry point iccg_spmv and against scipy
(same tolerance as the SpMV parity test), also at the largest size it
accepts (every CTA slot and group counter of the scratch in use), and that a
size above the maximum is rejected.  The file name makes pytest collect it
last.
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


@pytest.mark.parametrize("case", ["grid3d", "rspd"])
def test_noalloc_matches_existing_spmv_twice(case):
    a = gen.poisson3d_7pt(41) if case == "grid3d" else gen.random_spd_small(5003, 0.002, 4)
    p = np.random.default_rng(5).uniform(-1, 1, a.n)
    # existing entry point (through a context)
    bl = oracle.blocking(a, "abmc", 16)
    S = iccg.Solver(a, bl, factor=False)
    q_ref = np.zeros(a.n)
    iccg.iccg_spmv(S.ctx, p, q_ref)
    S.close()
    pq_ref = float(p @ q_ref)
    dev = torch.device("cuda")
    rp = torch.tensor(a.rowptr, dtype=torch.int64, device=dev)
    ci = torch.tensor(a.colind, dtype=torch.int32, device=dev)
    va = torch.tensor(a.val, dtype=torch.float64, device=dev)
    pd = torch.tensor(p, dtype=torch.float64, device=dev)
    results = []
    for _ in range(2):
        qd = torch.full((a.n,), np.nan, dtype=torch.float64, device=dev)
        pqd = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        st = iccg.iccg_spmv_dot_noalloc(a.n, rp, ci, va, pd, qd, pqd,
                                        torch.cuda.current_stream().cuda_stream)
        assert st == iccg.ICCG_OK
        torch.cuda.synchronize()
        q = qd.cpu().numpy()
        pq = float(pqd.cpu().item())
        assert np.max(np.abs(q - q_ref)) <= 1e-13 * np.max(np.abs(q_ref))
        assert abs(pq - pq_ref) <= 1e-12 * abs(pq_ref)
        q_sp = a.to_scipy() @ p
        assert np.max(np.abs(q - q_sp)) <= 1e-13 * np.max(np.abs(q_sp))
        assert abs(pq - float(p @ q_sp)) <= 1e-12 * abs(float(p @ q_sp))
        results.append((q, pq))
    assert np.array_equal(results[0][0], results[1][0])
    assert results[0][1] == results[1][1]


def test_noalloc_at_the_row_limit_twice():
    """n = ICCG_NOALLOC_MAX_ROWS (2D 5-point Laplacian on 2048 x 2048): all
    16,384 CTA partials and 512 group counters of the scratch are used."""
    a = gen.poisson2d_5pt(2048)
    assert a.n == iccg.NOALLOC_MAX_ROWS
    p = np.random.default_rng(9).uniform(-1, 1, a.n)
    q_sp = a.to_scipy() @ p
    pq_sp = float(p @ q_sp)
    dev = torch.device("cuda")
    rp = torch.tensor(a.rowptr, dtype=torch.int64, device=dev)
    ci = torch.tensor(a.colind, dtype=torch.int32, device=dev)
    va = torch.tensor(a.val, dtype=torch.float64, device=dev)
    pd = torch.tensor(p, dtype=torch.float64, device=dev)
    got = []
    for _ in range(2):
        qd = torch.full((a.n,), np.nan, dtype=torch.float64, device=dev)
        pqd = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        st = iccg.iccg_spmv_dot_noalloc(a.n, rp, ci, va, pd, qd, pqd, torch.cuda.current_stream().cuda_stream)
        assert st == iccg.ICCG_OK
        torch.cuda.synchronize()
        q = qd.cpu().numpy()
        pq = float(pqd.cpu().item())
        assert np.max(np.abs(q - q_sp)) <= 1e-13 * np.max(np.abs(q_sp))
        assert abs(pq - pq_sp) <= 1e-12 * abs(pq_sp)
        got.append(pq)
    assert got[0] == got[1]


def test_noalloc_rejects_oversize_and_bad_args():
    dev = torch.device("cuda")
    small = torch.zeros(4, dtype=torch.float64, device=dev)
    rp = torch.zeros(4, dtype=torch.int64, device=dev)
    ci = torch.zeros(4, dtype=torch.int32, device=dev)
    st = iccg.iccg_spmv_dot_noalloc(iccg.NOALLOC_MAX_ROWS + 1, rp, ci, small, small, small, small)
    assert st == 1   # ICCG_ERR_ARG, nothing launched
    st = iccg.iccg_spmv_dot_noalloc(-1, rp, ci, small, small, small, small)
    assert st == 1
    pq = torch.full((1,), 7.0, dtype=torch.float64, device=dev)
    st = iccg.iccg_spmv_dot_noalloc(0, rp, ci, small, small, small, pq)
    torch.cuda.synchronize()
    assert st == iccg.ICCG_OK and float(pq.item()) == 0.0
