"""Learned blocking end to end on the committed label sweep: the MLP is
trained on the GPU by the library's kernels (160 matrices) and evaluated on
the 40 held-out matrices against the exhaustive sweep: what it gains over the
method without it (fixed ABMC block size 32, fixed CPM resolution 0.05),
and its regret against the best swept setting."""
import os

import numpy as np
import pytest

from paper_2609_00561_gb300 import build as libbuild
from paper_2609_00561_gb300.learn import model as lm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SWEEP = os.path.join(os.path.dirname(lm.__file__), "blocking_sweep.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


@pytest.mark.skipif(not os.path.exists(SWEEP), reason="label sweep not committed")
def test_learned_blocking_gains_over_fixed_settings():
    data = lm.load_sweep(SWEEP)
    X, yc, yr, ta, tc = lm.labels(data)
    assert X.shape == (len(data["records"]), 20)
    tr, te = lm.split(len(yc))
    assert len(te) == 40 and len(set(tr) & set(te)) == 0
    m = lm.Model(X.shape[1], len(data["meta"]["block_sizes"]), seed=0)
    hist = m.fit(X[tr], yc[tr], yr[tr], epochs=3000)
    assert hist[-1] < hist[0]
    ev = lm.evaluate(m, X[te], ta[te], tc[te], data["meta"]["gammas"], data["meta"]["block_sizes"])
    base = lm.evaluate_fixed(ta[te], tc[te], data["meta"]["gammas"], data["meta"]["block_sizes"])
    # the model beats the method without it on held-out matrices ...
    assert ev["abmc_gain_vs_fixed32"] > 1.0
    assert ev["combined_gain_vs_fixed"] > 1.0
    # ... and is closer to the sweep's best than the fixed settings
    assert ev["abmc_regret_mean"] < base["abmc_regret_mean"]
    assert ev["combined_regret_mean"] < base["combined_regret_mean"]
