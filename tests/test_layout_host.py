"""Host-only checks of the device layout (iccg_check_layout): for matrices of
every generated family and every blocking method, the lane tiles and CTA
groups iccg_setup builds satisfy the index invariants the kernels rely on
(step rows, active-lane prefixes, sliced-ELL ranges, in-block references to
existing earlier / later rows of the same block, level schedules)."""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle
from paper_2609_00561_gb300 import build as libbuild
from paper_2609_00561_gb300 import iccg


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


MATS = {
    "grid3d": lambda: gen.poisson3d_7pt(11),
    "aniso27": lambda: gen.stencil_aniso("27pt", 1500, 40.0),
    "rgg": lambda: gen.rgg_laplacian(3000, 25.0, 4),
    "elast27": lambda: gen.elasticity_like(300, 27, 2.0),
    "rspd": lambda: gen.random_spd_small(600, 0.015, 2),
}
BLOCKINGS = [("abmc", dict(block_size=s)) for s in (1, 2, 8, 32, 100)] + \
            [("leiden_cpm", dict(gamma=g)) for g in (0.05, 0.5, 2.0)] + [("leiden_md", dict(gamma=1.0))]


@pytest.mark.parametrize("mat", sorted(MATS))
@pytest.mark.parametrize("blk", range(len(BLOCKINGS)))
@pytest.mark.parametrize("lane_max", [32, 8, 0])
@pytest.mark.parametrize("units", [False, True])
def test_layout_invariants(mat, blk, lane_max, units):
    a = MATS[mat]()
    method, kw = BLOCKINGS[blk]
    bl = iccg.blocking(a, method, **kw)
    st, tiles, groups, failed, first, what = iccg.check_layout(a, bl, group_rows=256, lane_max=lane_max,
                                                               use_units=units)
    assert st == 0 and failed == 0, (what, first)
    sizes = np.diff(np.asarray(bl["block_ptr"]))
    if lane_max == 0 and not units:
        assert tiles == 0
    if (lane_max and sizes.max() <= lane_max) or (units and sizes.max() <= 32):
        assert groups == 0


def test_layout_of_the_fused_singleton_case():
    """Tiles too large for a second staged set plus a last color of
    singleton blocks (the layout of the fused-launch regression test)."""
    a0 = gen.rgg_laplacian(5000, 29.0, 11).to_scipy()
    m = sp.block_diag([a0, sp.diags(np.linspace(1.0, 2.0, 37))], format="csr")
    a = gen.from_scipy(m)
    bl0 = oracle.blocking(gen.from_scipy(a0.tocsr()), "abmc", 32)
    nb, nc = bl0["n_b"], bl0["n_c"]
    bl = {"perm": np.concatenate([bl0["perm"], 5000 + np.arange(37)]).astype(np.int32),
          "block_ptr": np.concatenate([bl0["block_ptr"], 5001 + np.arange(37)]).astype(np.int32),
          "color_ptr": np.concatenate([bl0["color_ptr"][:nc + 1], [nb + 37]]).astype(np.int32),
          "n_b": nb + 37, "n_c": nc + 1}
    st, tiles, groups, failed, first, what = iccg.check_layout(a, bl)
    assert st == 0 and failed == 0 and groups == 0
