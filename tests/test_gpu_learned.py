"""Learned blocking end to end on the committed label sweep (200 generated
matrices of config 5's recipe, n in [1e5, 2e6]): the MLP ensemble is
selected (training length and CPM margin by cross-validation on the 160
training matrices) and trained on the GPU by the library's kernels, and
evaluated on the 40 held-out matrices against the exhaustive sweep: its
regret against the best constant settings chosen on the training labels and
against the method without it (fixed ABMC block size 32, fixed CPM
resolution 0.05)."""
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


@pytest.fixture(scope="module")
def report():
    data = lm.load_sweep(SWEEP)
    return data, lm.report(data)[1]


def test_sweep_is_config5_at_its_stated_size(report):
    data, _ = report
    meta = data["meta"]
    assert len(data["records"]) == 200 and meta["n_lo"] == 1e5 and meta["n_hi"] == 2e6
    ns = np.array([r["n"] for r in data["records"]])
    assert ns.min() >= 0.9e5 and ns.max() <= 2.1e6
    X, yc, yr, ta, tc = lm.labels(data)
    assert X.shape == (200, 20)
    tr, te = lm.split(len(yc))
    assert len(te) == 40 and len(set(tr) & set(te)) == 0


def test_learned_blocking_beats_the_best_constant_and_the_fixed_settings(report):
    _, rep = report
    ev, const, fixed = rep["test"], rep["test_best_constant"], rep["test_fixed"]
    # the block-size head and the combined choice beat the best constant
    # setting chosen on the training labels, on the held-out matrices
    assert ev["abmc_regret_mean"] < const["abmc_regret_mean"]
    assert ev["combined_regret_mean"] < const["combined_regret_mean"]
    # the resolution head: 1.0 is the fastest on 176 of the 200 matrices; the
    # cross-validated margin keeps the head within 1% of that constant
    assert ev["cpm_regret_mean"] <= 1.01 * const["cpm_regret_mean"]
    # both heads are far better than the method without the model
    assert ev["abmc_regret_mean"] < fixed["abmc_regret_mean"]
    assert ev["cpm_regret_mean"] < fixed["cpm_regret_mean"]
    assert ev["abmc_gain_vs_fixed32"] > 1.2 and ev["cpm_gain_vs_fixed005"] > 1.2
