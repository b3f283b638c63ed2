"""Pins for the oracle's random numbers and adjacency graph (CPU only).

Philox4x64-10 is checked against numpy's independent implementation; the
graph of A (Sec. 3) against a brute-force dense construction.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle


@pytest.mark.parametrize("seed", [0, 1, 42, 2**40 + 7])
def test_philox_matches_numpy(seed):
    ref = np.random.Philox(key=seed).random_raw(37)
    got = oracle.philox_stream(seed, 37)
    assert np.array_equal(ref.astype(np.uint64), got)


def test_shuffle_is_uniform_permutation():
    counts = {}
    for seed in range(3000):
        p = tuple(oracle.shuffle_stream(seed, 3))
        assert sorted(p) == [0, 1, 2]
        counts[p] = counts.get(p, 0) + 1
    assert len(counts) == 6
    # each of the 3! orders within 5 sigma of 500
    for c in counts.values():
        assert abs(c - 500) < 5 * np.sqrt(3000 * (1 / 6) * (5 / 6))


def _dense_graph(a):
    d = a.to_scipy().toarray() != 0
    d = d | d.T
    np.fill_diagonal(d, False)
    return d


@pytest.mark.parametrize("seed", range(5))
def test_graph_matches_dense_pattern(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    # deliberately unsymmetric stored pattern: the graph must symmetrise it
    m = sp.random(n, n, density=0.15, random_state=np.random.RandomState(seed), format="csr")
    m = m + sp.identity(n)
    a = gen.from_scipy(m)
    gptr, gadj = oracle.graph(a.n, a.rowptr, a.colind)
    d = _dense_graph(a)
    for i in range(n):
        nb = gadj[gptr[i]:gptr[i + 1]]
        assert list(nb) == list(np.nonzero(d[i])[0])


def test_graph_of_grid():
    a = gen.poisson2d_5pt(5)
    gptr, gadj = oracle.graph(a.n, a.rowptr, a.colind)
    assert gptr[-1] == 2 * (2 * 5 * 4)          # 2 * number of grid edges
    deg = np.diff(gptr)
    assert deg.min() == 2 and deg.max() == 4    # corners and interior
