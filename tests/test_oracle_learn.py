"""Pins of the learned-blocking oracle (CPU): feature closed forms, the MLP
gradient against finite differences, the loss of a zero network; and the
production feature extractor of the library against the oracle."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import gen
from oracle import learn as ol
from paper_2609_00561_gb300 import build as libbuild
from paper_2609_00561_gb300 import iccg


def _csr(m):
    m = sp.csr_matrix(m)
    return m.shape[0], m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.astype(np.float64)


def test_features_tridiagonal_closed_form():
    n = 10
    m = sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    f = ol.features(*_csr(m))
    mean = (2 * 2 + 3 * (n - 2)) / n
    var = (2 * (2 - mean) ** 2 + (n - 2) * (3 - mean) ** 2) / n
    assert f[0] == pytest.approx(1.0)
    assert f[1] == pytest.approx(mean) and f[2] == pytest.approx(var) and f[4] == 3
    assert f[5] == pytest.approx(math.log10(3 * n - 2))
    assert f[6] == pytest.approx((2 * 2.0 + (n - 2) * 1.0) / n) and f[7] == 1.0 and f[8] == 1.0
    assert f[9] == pytest.approx(1 / n) and f[10] == pytest.approx(1 / n)
    assert f[11] == 1.0 and np.all(f[12:19] == 0.0) and f[19] == 0.0


def test_features_diagonal_and_spread():
    f = ol.features(*_csr(sp.diags(np.arange(1.0, 6.0))))
    assert f[2] == 0.0 and f[3] == 0.0 and f[6] == 10.0 and f[7] == 10.0 and f[10] == 0.0 and f[19] == 0.0
    m = sp.csr_matrix(np.array([[4.0, -1e-3, 0], [-1e-3, 4.0, -10.0], [0, -10.0, 30.0]]))
    f = ol.features(*_csr(m))
    assert f[19] == pytest.approx(4.0)                      # log10(10 / 1e-3)
    assert f[7] == pytest.approx(4.0 / (1e-3 + 10.0))       # row 1


@pytest.mark.parametrize("mk", [lambda: gen.poisson3d_7pt(9), lambda: gen.stencil_aniso("27pt", 1000, 30.0),
                                lambda: gen.rgg_laplacian(800, 12.0, 3), lambda: gen.elasticity_like(200, 27, 4.0),
                                lambda: gen.random_spd_small(300, 0.02, 5)])
def test_production_features_match_oracle(mk):
    libbuild.build()
    a = mk()
    fo = ol.features(a.n, a.rowptr, a.colind, a.val)
    fp = iccg.features(a)
    assert np.allclose(fp, fo, rtol=1e-12, atol=1e-14)
    assert np.array_equal(fp[11:19], fo[11:19])


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    nf, h, c, B = 5, 7, 4, 9
    p = rng.normal(0, 0.5, ol.mlp_offsets(nf, h, c)["total"])
    X = rng.normal(size=(B, nf))
    y = rng.integers(0, c, B)
    yr = rng.normal(size=B)
    g = ol.mlp_grad(p, nf, h, c, X, y, yr, 0.7)
    eps = 1e-6
    fd = np.zeros_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = eps
        fd[k] = (ol.mlp_loss(p + e, nf, h, c, X, y, yr, 0.7) - ol.mlp_loss(p - e, nf, h, c, X, y, yr, 0.7)) / (2 * eps)
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-7)


def test_mlp_zero_network_loss():
    nf, h, c = 3, 4, 5
    p = np.zeros(ol.mlp_offsets(nf, h, c)["total"])
    X = np.ones((6, nf))
    yr = np.full(6, 2.0)
    assert ol.mlp_loss(p, nf, h, c, X, np.arange(6) % c, yr, 0.5) == pytest.approx(math.log(c) + 0.5 * 4.0)


def test_adam_first_step_is_signed_lr():
    p, g = np.array([1.0, -2.0, 3.0]), np.array([0.5, -0.1, 0.0])
    q, m, v = ol.adam(p, g, np.zeros(3), np.zeros(3), 0.01, 0.9, 0.999, 1e-12, 1)
    assert np.allclose(q, p - 0.01 * np.sign(g))
