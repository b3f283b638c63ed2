"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (element by element on the same seeded inputs):
  * IC(0) factor, SpMV, preconditioner apply: relative max difference
    <= 1e-12 (FP64; only the summation order differs);
  * FP64 ICCG solve: ||x_gpu - x_orc|| / ||x_orc|| <= 1e-10 and iteration
    counts within +-1;
  * blockings / permutations are inputs and bit-exact by construction.
Cases span several tiles, ragged tails, multi-tile blocks (ABMC s > 32R,
Leiden modularity blocks of hundreds of rows), one-color and one-row systems,
and every launch shape: warp units (one warp per block of up to 32 rows, a lane
per row), lane tiles (one block per lane) and CTA groups (level by level)
under several rows-per-thread / warps-per-CTA choices, the phased solve as a
CUDA graph or a host loop, with or without programmatic dependent launch, and
the persistent single-launch solve.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def _tri(n):
    return gen.from_scipy(sp.diags([-np.ones(n - 1), 2.5 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]))


CASES = {
    "c1_abmc16": (lambda: gen.config1(), "abmc", {"block_size": 16}),
    "grid3d_abmc8": (lambda: (gen.poisson3d_7pt(20), gen.rhs_uniform(8000, 3), None), "abmc", {"block_size": 8}),
    "grid3d_abmc32": (lambda: (gen.poisson3d_7pt(20), gen.rhs_uniform(8000, 3), None), "abmc", {"block_size": 32}),
    "grid3d_abmc100": (lambda: (gen.poisson3d_7pt(20), gen.rhs_uniform(8000, 3), None), "abmc", {"block_size": 100}),
    "grid3d_abmc2": (lambda: (gen.poisson3d_7pt(22), gen.rhs_uniform(10648, 13), None), "abmc", {"block_size": 2}),
    "grid3d_cpm_singletons": (lambda: (gen.poisson3d_7pt(21), gen.rhs_uniform(9261, 14), None), "leiden_cpm",
                              {"gamma": 1.0}),
    "grid3d_cpm_pairs": (lambda: (gen.poisson3d_7pt(23), gen.rhs_uniform(12167, 15), None), "leiden_cpm",
                         {"gamma": 0.5}),
    "grid2d_leiden_md": (lambda: (gen.poisson2d_5pt(45), gen.rhs_uniform(2025, 4), None), "leiden_md", {"gamma": 1.0}),
    "grid3d_leiden_cpm": (lambda: (gen.poisson3d_7pt(15), gen.rhs_uniform(3375, 5), None), "leiden_cpm", {"gamma": 0.1}),
    "rspd_777": (lambda: (gen.random_spd_small(777, 0.01, 7), gen.rhs_uniform(777, 6), None), "abmc", {"block_size": 13}),
    "aniso27": (lambda: (gen.stencil_aniso("27pt", 3375, 4.0), gen.rhs_uniform(3375, 8), None), "abmc", {"block_size": 32}),
    "elast27": (lambda: (gen.elasticity_like(700, 27, 3.0), gen.rhs_uniform(2187, 9), None), "abmc", {"block_size": 24}),
    "diff27": (lambda: (gen.diffusion3d_27pt(14, seed=2), gen.rhs_uniform(2744, 10), None), "abmc", {"block_size": 32}),
    # two-row blocks of a 27-point stencil: pair tiles whose steps have more
    # entries to other colors than the pair kernels stage in shared memory
    "aniso27_abmc2": (lambda: (gen.stencil_aniso("27pt", 3375, 4.0), gen.rhs_uniform(3375, 18), None), "abmc",
                      {"block_size": 2}),
    # level scheduling of the natural order: one-row blocks, a color per level
    "grid3d_levels": (lambda: (gen.poisson3d_7pt(13), gen.rhs_uniform(2197, 16), None), "levels", {}),
    "rgg_levels": (lambda: (gen.rgg_laplacian(1500, 10.0, 5), gen.rhs_uniform(1500, 17), None), "levels", {}),
    # Leiden modularity blocks of hundreds of rows split into in-block levels
    "grid2d_leiden_md_split": (lambda: (gen.poisson2d_5pt(45), gen.rhs_uniform(2025, 4), None), "leiden_md_split",
                               {"gamma": 1.0}),
}

_cache = {}


def _case(name):
    if name not in _cache:
        mk, method, kw = CASES[name]
        a, b, _ = mk()
        if method == "leiden_md_split":
            bl = oracle.split_levels(a, oracle.blocking(a, "leiden_md", **kw), 32)
        else:
            bl = oracle.blocking(a, method, **kw)
        ref = oracle.iccg(a, b, bl["perm"], tol=1e-8, maxit=20000)
        _cache[name] = (a, b, bl, ref)
    return _cache[name]


def _rel(x, y):
    return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))


SHAPES = [dict(), dict(lane_block_max=8), dict(lane_block_max=-1),
          dict(lane_block_max=-1, rows_per_thread=2, warps_per_cta=4), dict(lane_block_max=-1, warps_per_cta=1),
          dict(lane_block_max=-1, warps_per_cta=16), dict(no_graph=1), dict(no_pdl=1),
          dict(solver="persistent"), dict(solver="persistent", rows_per_thread=4, warps_per_cta=4),
          dict(solver="persistent", warps_per_cta=16), dict(tile_mapping="warp"), dict(tile_mapping="cta"),
          dict(tile_mapping="warp", warps_per_cta=3, lane_block_max=16), dict(tile_mapping="units"),
          dict(tile_mapping="units", lane_block_max=16), dict(tile_mapping="units", no_graph=1),
          dict(fuse_sweep=1), dict(fuse_sweep=1, no_graph=1), dict(fuse_sweep=1, precond_fp32=0, warps_per_cta=4),
          dict(fuse_sweep=2), dict(fuse_sweep=2, no_graph=1)]
LAYOUTS = {"lanes": dict(), "groups": dict(lane_block_max=-1), "warp_tiles": dict(tile_mapping="warp"),
           "cta_tiles": dict(tile_mapping="cta"), "pair_tiles": dict(tile_mapping="pair"),
           "units": dict(tile_mapping="units"), "units16": dict(tile_mapping="units", lane_block_max=16),
           "fused": dict(fuse_sweep=1), "tail": dict(fuse_sweep=2)}
SOLVERS = {"lanes": dict(), "groups": dict(lane_block_max=-1), "persistent": dict(solver="persistent"),
           "warp_tiles": dict(tile_mapping="warp"), "cta_tiles": dict(tile_mapping="cta"),
           "pair_tiles": dict(tile_mapping="pair"), "units": dict(tile_mapping="units"),
           "fused": dict(fuse_sweep=1), "tail": dict(fuse_sweep=2)}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("layout", sorted(LAYOUTS))
def test_factor_spmv_precond_match_oracle(name, layout):
    a, b, bl, ref = _case(name)
    S = iccg.Solver(a, bl, **LAYOUTS[layout])
    ah = oracle.permute(a, bl["perm"])
    lptr, lcol, aval = oracle.tril_csr(ah)
    lref, brow = oracle.ic0(lptr, lcol, aval)
    assert brow == -1
    lgpu = iccg.iccg_get_factor(S.ctx)
    assert np.max(np.abs(lgpu - lref)) <= 1e-12 * np.max(np.abs(lref))
    rng = np.random.default_rng(11)
    p = rng.uniform(-1, 1, a.n)
    q = np.zeros(a.n)
    iccg.iccg_spmv(S.ctx, p, q)
    qref = a.to_scipy() @ p
    assert np.max(np.abs(q - qref)) <= 1e-13 * np.max(np.abs(qref))
    z = np.zeros(a.n)
    iccg.iccg_precond(S.ctx, p, z)
    perm = bl["perm"]
    zref_h = oracle.backward(lptr, lcol, lref, oracle.forward(lptr, lcol, lref, p[perm]))
    zref = np.zeros(a.n)
    zref[perm] = zref_h
    assert np.max(np.abs(z - zref)) <= 1e-12 * np.max(np.abs(zref))
    S.close()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_solve_fp64_matches_oracle(name, shape):
    a, b, bl, ref = _case(name)
    S = iccg.Solver(a, bl, **SHAPES[shape])
    x = np.zeros(a.n)
    st, it, hist = iccg.iccg_solve(S.ctx, b, x, 1e-8, 20000)
    assert st == iccg.ICCG_OK
    assert abs(it - ref["iterations"]) <= 1
    assert _rel(x, ref["x"]) <= 1e-10
    assert hist[-1] <= 1e-8
    # the recursive residual history is a property check, not the parity bar:
    # its late entries carry rounding-order differences amplified by the
    # condition number (observed up to 6e-6 relative on the elasticity case)
    k = min(len(hist), len(ref["hist"]))
    assert np.allclose(hist[:k], ref["hist"][:k], rtol=1e-3, atol=0)
    S.close()


@pytest.mark.parametrize("name", ["c1_abmc16", "grid3d_abmc100", "grid2d_leiden_md", "diff27", "elast27"])
@pytest.mark.parametrize("solver", sorted(SOLVERS))
def test_solve_fp32_preconditioner(name, solver):
    """Extension 1: FP32 factors/substitutions, FP64 CG; reaches the same
    recursive residual; its error against the FP64 oracle is reported."""
    a, b, bl, ref = _case(name)
    S = iccg.Solver(a, bl, precond_fp32=True, **SOLVERS[solver])
    x = np.zeros(a.n)
    st, it, hist = iccg.iccg_solve(S.ctx, b, x, 1e-8, 20000)
    assert st == iccg.ICCG_OK and hist[-1] <= 1e-8
    true_rel = np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)
    assert true_rel <= 1e-7
    err = _rel(x, ref["x"])
    kappa_proxy = max(1.0, ref["iterations"] / 10.0)
    assert err <= 1e-6 * kappa_proxy, err
    # FP32 factors perturb the preconditioner; on the nearly singular
    # elasticity case this costs a few iterations (61 -> 65 observed)
    assert abs(it - ref["iterations"]) <= 3 + ref["iterations"] // 10
    S.close()


@pytest.mark.parametrize("name", ["grid3d_abmc2", "grid3d_cpm_pairs", "rgg_levels", "aniso27_abmc2"])
@pytest.mark.parametrize("shape", [dict(tile_mapping="pair"), dict(tile_mapping="pair", warps_per_cta=16),
                                   dict(tile_mapping="pair", no_graph=1)])
def test_fp32_preconditioner_on_pair_tiles(name, shape):
    """Extension 1 on the pair kernels, which in FP32 stage every color's
    entries to other colors: two-row blocks (ABMC 2), one- and two-row
    blocks mixed in a tile (CPM 0.5), and one-row blocks with up to a dozen
    entries to earlier levels (a random geometric graph by level sets, past
    the six entries per step staged in shared memory)."""
    a, b, bl, ref = _case(name)
    S = iccg.Solver(a, bl, precond_fp32=True, **shape)
    assert iccg.iccg_info(S.ctx)["pair_tile_colors"] > 0
    x = np.zeros(a.n)
    st, it, hist = iccg.iccg_solve(S.ctx, b, x, 1e-8, 20000)
    assert st == iccg.ICCG_OK and hist[-1] <= 1e-8
    true_rel = np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)
    assert true_rel <= 1e-7
    err = _rel(x, ref["x"])
    assert err <= 1e-6 * max(1.0, ref["iterations"] / 10.0), err
    assert abs(it - ref["iterations"]) <= 3 + ref["iterations"] // 10
    # the preconditioner apply alone against the oracle's FP64 substitutions:
    # FP32 factors and accumulation give a relative error of order (entries
    # per row) x 2^-24 x cond(L), well below 1e-4 for these matrices
    z = np.zeros(a.n)
    iccg.iccg_precond(S.ctx, b, z)
    ah = oracle.permute(a, bl["perm"])
    lptr, lcol, aval = oracle.tril_csr(ah)
    lref, _ = oracle.ic0(lptr, lcol, aval)
    zp = oracle.backward(lptr, lcol, lref, oracle.forward(lptr, lcol, lref, b[bl["perm"]]))
    zref = np.zeros(a.n)
    zref[bl["perm"]] = zp
    assert _rel(z, zref) <= 1e-4
    S.close()


@pytest.mark.parametrize("solver", sorted(SOLVERS))
def test_device_and_host_pointers_agree_and_are_deterministic(solver):
    a, b, bl, ref = _case("grid3d_abmc32")
    S = iccg.Solver(a, bl, **SOLVERS[solver])
    xh = np.zeros(a.n)
    iccg.iccg_solve(S.ctx, b, xh)
    bd = torch.tensor(b, device="cuda")
    xd = torch.zeros_like(bd)
    iccg.iccg_solve(S.ctx, bd, xd)
    assert np.array_equal(xd.cpu().numpy(), xh)
    xh2 = np.zeros(a.n)
    iccg.iccg_solve(S.ctx, b, xh2)
    assert np.array_equal(xh, xh2)
    S.close()


@pytest.mark.parametrize("solver", sorted(SOLVERS))
def test_edge_cases(solver):
    a, b, bl, ref = _case("c1_abmc16")
    S = iccg.Solver(a, bl, **SOLVERS[solver])
    # b = 0 -> x = 0, 0 iterations
    x = np.full(a.n, 3.0)
    st, it, hist = iccg.iccg_solve(S.ctx, np.zeros(a.n), x)
    assert st == iccg.ICCG_OK and it == 0 and np.all(x == 0)
    # x0 = exact solution (to rounding) -> converged at k = 0
    x = ref["x"].copy()
    st, it, hist = iccg.iccg_solve(S.ctx, b, x, 1e-6)
    assert st == iccg.ICCG_OK and it == 0
    # maxit = 0 and maxit reached
    x = np.zeros(a.n)
    st, it, hist = iccg.iccg_solve(S.ctx, b, x, 1e-8, 0)
    assert st == iccg.ICCG_NOT_CONVERGED and it == 0 and len(hist) == 1
    x = np.zeros(a.n)
    st, it, hist = iccg.iccg_solve(S.ctx, b, x, 1e-8, 5)
    assert st == iccg.ICCG_NOT_CONVERGED and it == 5
    xo, ito, _, sto = oracle.pcg(oracle.permute(a, bl["perm"]), *_factor_of(a, bl), b[bl["perm"]], tol=1e-8, maxit=5)
    xr = np.zeros(a.n); xr[bl["perm"]] = xo
    assert _rel(x, xr) <= 1e-12
    # a non-zero x0
    x0 = np.random.default_rng(1).uniform(-1, 1, a.n)
    x = x0.copy()
    st, it, hist = iccg.iccg_solve(S.ctx, b, x)
    r2 = oracle.iccg(a, b, bl["perm"], x0=x0)
    assert abs(it - r2["iterations"]) <= 1 and _rel(x, r2["x"]) <= 1e-10
    S.close()


def _factor_of(a, bl):
    ah = oracle.permute(a, bl["perm"])
    lptr, lcol, aval = oracle.tril_csr(ah)
    lval, _ = oracle.ic0(lptr, lcol, aval)
    return lptr, lcol, lval


@pytest.mark.parametrize("solver", sorted(SOLVERS))
def test_single_block_tridiagonal_converges_in_one_iteration(solver):
    a = _tri(300)
    bl = {"perm": np.arange(300, dtype=np.int32), "block_ptr": np.array([0, 300], dtype=np.int32),
          "color_ptr": np.array([0, 1], dtype=np.int32), "n_b": 1, "n_c": 1}
    S = iccg.Solver(a, bl, **SOLVERS[solver])
    b = gen.rhs_uniform(300, 2)
    x = np.zeros(300)
    st, it, hist = iccg.iccg_solve(S.ctx, b, x, 1e-12)
    assert st == iccg.ICCG_OK and it == 1
    assert np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b) < 1e-12
    S.close()


@pytest.mark.parametrize("solver", sorted(SOLVERS))
def test_one_row_system(solver):
    a = gen.from_scipy(sp.csr_matrix(np.array([[4.0]])))
    bl = {"perm": np.array([0], dtype=np.int32), "block_ptr": np.array([0, 1], dtype=np.int32),
          "color_ptr": np.array([0, 1], dtype=np.int32), "n_b": 1, "n_c": 1}
    S = iccg.Solver(a, bl, **SOLVERS[solver])
    x = np.zeros(1)
    st, it, hist = iccg.iccg_solve(S.ctx, np.array([2.0]), x)
    assert st == iccg.ICCG_OK and it == 1 and abs(x[0] - 0.5) < 1e-15
    S.close()


def test_breakdown_reports_oracle_row():
    m = sp.diags([np.full(39, 1.2), np.ones(40), np.full(39, 1.2)], [-1, 0, 1], format="csr")
    a = gen.from_scipy(m)
    bl = oracle.blocking(a, "abmc", 4)
    r = oracle.iccg(a, np.ones(40), bl["perm"])
    assert r["status"] == "breakdown"
    S = iccg.Solver(a, bl, factor=False)
    with pytest.raises(iccg.IccgError) as ei:
        iccg.iccg_factor(S.ctx)
    assert ei.value.status == 3 and ei.value.index == r["breakdown_row"]
    # solving without a successful factor is a state error
    with pytest.raises(iccg.IccgError) as ei2:
        iccg.iccg_solve(S.ctx, np.ones(40), np.zeros(40))
    assert ei2.value.status == 9
    S.close()


def test_production_blocking_drives_the_same_solve():
    a, b, _ = gen.config1()
    bp = iccg.blocking(a, "leiden_cpm", gamma=0.2)
    bo = oracle.blocking(a, "leiden_cpm", gamma=0.2)
    assert np.array_equal(bp["perm"], bo["perm"])
    S = iccg.Solver(a, bp)
    x = np.zeros(a.n)
    st, it, hist = iccg.iccg_solve(S.ctx, b, x)
    ref = oracle.iccg(a, b, bo["perm"])
    assert abs(it - ref["iterations"]) <= 1 and _rel(x, ref["x"]) <= 1e-10
    S.close()


def test_layout_choice_follows_block_sizes():
    """Colors of blocks of 5..32 rows run as warp units (a warp per block, a
    lane per row) by default and as lane tiles (32 blocks per tile) when asked;
    larger blocks run as CTA groups."""
    a, b, bl, ref = _case("grid3d_abmc8")
    cp = np.asarray(bl["color_ptr"])
    S = iccg.Solver(a, bl)
    info = iccg.iccg_info(S.ctx)
    assert info["unit_colors"] == bl["n_c"] and info["tile_colors"] == 0 and info["groups"] == 0
    S.close()
    S = iccg.Solver(a, bl, tile_mapping="cta")
    info = iccg.iccg_info(S.ctx)
    assert info["tile_colors"] == bl["n_c"] and info["unit_colors"] == 0
    assert info["tiles"] == sum((int(cp[c + 1] - cp[c]) + 31) // 32 for c in range(bl["n_c"]))
    assert info["groups"] == 0
    assert info["warp_tile_colors"] == 0
    assert info["pair_tile_colors"] == 0        # blocks of 8 rows: one CTA per tile
    S.close()
    S = iccg.Solver(a, bl, tile_mapping="warp")
    assert iccg.iccg_info(S.ctx)["warp_tile_colors"] == bl["n_c"]
    S.close()
    a4, b4, bl4, ref4 = _case("grid3d_abmc100")
    S = iccg.Solver(a4, bl4)
    assert iccg.iccg_info(S.ctx)["groups"] > 0     # blocks above 32 rows: CTA groups
    assert iccg.iccg_info(S.ctx)["fused_sweep"] == 0
    S.close()
    # blocks of one or two rows: each sweep one cooperative launch on request
    a5, b5, bl5, ref5 = _case("grid3d_cpm_pairs")
    S = iccg.Solver(a5, bl5, fuse_sweep=1)
    assert iccg.iccg_info(S.ctx)["fused_sweep"] == 1
    S.close()
    S = iccg.Solver(a5, bl5)
    assert iccg.iccg_info(S.ctx)["fused_sweep"] == 0
    S.close()
    a2, b2, bl2, ref2 = _case("grid3d_cpm_singletons")
    S = iccg.Solver(a2, bl2)
    info = iccg.iccg_info(S.ctx)
    assert info["tile_colors"] == bl2["n_c"] and info["pair_tile_colors"] == 0   # one-row blocks: CTA per tile
    S.close()
    S = iccg.Solver(a2, bl2, tile_mapping="pair")
    assert iccg.iccg_info(S.ctx)["pair_tile_colors"] == bl2["n_c"]
    S.close()
    a2, b2, bl2, ref2 = _case("grid3d_abmc2")
    S = iccg.Solver(a2, bl2)
    sizes = np.diff(np.asarray(bl2["block_ptr"]))
    cp2 = np.asarray(bl2["color_ptr"])
    twos = sum(int(np.all(sizes[cp2[c]:cp2[c + 1]] == 2)) for c in range(bl2["n_c"]))
    assert twos == bl2["n_c"]
    assert iccg.iccg_info(S.ctx)["pair_tile_colors"] == twos   # colors of two-row blocks only: pair kernels
    S.close()
    # tiles mixing one- and two-row blocks: pair kernels only on request
    a3, b3, bl3, ref3 = _case("grid3d_cpm_pairs")
    sizes = np.diff(np.asarray(bl3["block_ptr"]))
    assert sizes.max() <= 2 and sizes.min() == 1
    S = iccg.Solver(a3, bl3, tile_mapping="pair")
    assert iccg.iccg_info(S.ctx)["pair_tile_colors"] == bl3["n_c"]
    S.close()
    S = iccg.Solver(a3, bl3)
    assert iccg.iccg_info(S.ctx)["pair_tile_colors"] < bl3["n_c"]
    S.close()
    S = iccg.Solver(a, bl, lane_block_max=-1)
    assert iccg.iccg_info(S.ctx)["tile_colors"] == 0
    S.close()
    a, b, bl, ref = _case("grid3d_abmc100")
    S = iccg.Solver(a, bl)
    assert iccg.iccg_info(S.ctx)["tile_colors"] == 0
    S.close()


def _rgg_plus_isolated(n_rgg=20000, n_iso=37, seed=11):
    """A random geometric graph Laplacian (ABMC 32: tiles whose in-block
    entries are too many for a second staged set in the fused launch) plus
    n_iso isolated rows forming a last color of singleton blocks (no in-block
    entries at all)."""
    a = gen.rgg_laplacian(n_rgg, 29.0, seed).to_scipy()
    m = sp.block_diag([a, sp.diags(np.linspace(1.0, 2.0, n_iso))], format="csr")
    big = gen.from_scipy(m)
    bl = oracle.blocking(gen.from_scipy(a.tocsr()), "abmc", 32)
    nb, nc = bl["n_b"], bl["n_c"]
    perm = np.concatenate([bl["perm"], n_rgg + np.arange(n_iso)]).astype(np.int32)
    bptr = np.concatenate([bl["block_ptr"], n_rgg + 1 + np.arange(n_iso)]).astype(np.int32)
    cptr = np.concatenate([bl["color_ptr"][:nc + 1], [nb + n_iso]]).astype(np.int32)
    return big, {"perm": perm, "block_ptr": bptr, "color_ptr": cptr, "n_b": nb + n_iso, "n_c": nc + 1}


def test_fused_color_without_in_block_entries():
    """The fused last color's tiles have no in-block upper entries while the
    launch has no room for a second staged set: nothing may be copied."""
    a, bl = _rgg_plus_isolated()
    b = gen.rhs_uniform(a.n, 12)
    ref = oracle.iccg(a, b, bl["perm"])
    for fp32 in (False, True):
        # the lane-tile layout the regression concerns, then the default
        # (warp units for the 32-row blocks)
        for mapping in ("cta", "auto"):
            S = iccg.Solver(a, bl, precond_fp32=fp32, tile_mapping=mapping)
            info = iccg.iccg_info(S.ctx)
            if mapping == "cta":
                assert info["tile_colors"] == bl["n_c"]
            else:
                assert info["unit_colors"] + info["tile_colors"] == bl["n_c"]
            x = np.zeros(a.n)
            st, it, _ = iccg.iccg_solve(S.ctx, b, x)
            assert st == iccg.ICCG_OK
            if not fp32:
                assert abs(it - ref["iterations"]) <= 1 and _rel(x, ref["x"]) <= 1e-10
            S.close()


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("no_graph", [0, 1])
def test_tail_colors_in_one_cooperative_launch(fp32, no_graph):
    """fuse_sweep = 2: the last colors of every sweep (at most n/32 rows, blocks
    of one or two rows) run forward, fused and backward in one cooperative
    launch between the per-color launches; the solve equals the oracle's."""
    a = gen.poisson3d_7pt(40)
    b = gen.rhs_uniform(a.n, 6)
    bl = oracle.blocking(a, "leiden_cpm", gamma=0.5)
    ref = oracle.iccg(a, b, bl["perm"], tol=1e-8, maxit=5000)
    S = iccg.Solver(a, bl, fuse_sweep=2, precond_fp32=fp32, no_graph=no_graph)
    info = iccg.iccg_info(S.ctx)
    assert info["fused_sweep"] == 2
    assert info["launches_per_iteration"] < 2 + 2 * bl["n_c"] - 1
    x = np.zeros(a.n)
    st, it, hist = iccg.iccg_solve(S.ctx, b, x, 1e-8, 5000)
    S.close()
    assert st == iccg.ICCG_OK
    if fp32:
        assert np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b) <= 1e-7
        assert abs(it - ref["iterations"]) <= 3 + ref["iterations"] // 10
    else:
        assert abs(it - ref["iterations"]) <= 1
        assert _rel(x, ref["x"]) <= 1e-10
