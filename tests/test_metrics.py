"""AUC and NLL helpers against closed forms and a library routine."""
import math

import numpy as np
import pytest

from paper_2408_09066_gb300 import metrics


def test_auc_closed_forms():
    y = np.array([0, 0, 1, 1])
    assert metrics.auc([0.1, 0.2, 0.8, 0.9], y) == 1.0
    assert metrics.auc([0.9, 0.8, 0.2, 0.1], y) == 0.0
    assert metrics.auc([0.5, 0.5, 0.5, 0.5], y) == 0.5
    # one inverted pair of four: 3/4
    assert metrics.auc([0.1, 0.85, 0.8, 0.9], y) == 0.75
    assert math.isnan(metrics.auc([0.1, 0.2], [1, 1]))


def test_auc_matches_sklearn_with_ties():
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(0)
    y = rng.integers(0, 2, 5000)
    s = np.round(rng.normal(y * 0.7, 1.0), 1)  # many ties
    assert abs(metrics.auc(s, y) - sk.roc_auc_score(y, s)) < 1e-12


def test_nll_closed_form():
    assert abs(metrics.nll([0.5, 0.5], [0, 1]) - math.log(2)) < 1e-15
    assert abs(metrics.nll([0.9], [1]) + math.log(0.9)) < 1e-15
    assert metrics.nll([0.0], [1]) == pytest.approx(-math.log(1e-7))


def test_evaluate_looks_up_cells():
    occ = np.zeros((4, 5))
    occ[2, 3] = 0.9  # cell i = 3, j = 2
    xy = np.array([[3.5, 2.5], [0.5, 0.5], [9.0, 9.0]], np.float32)
    r = metrics.evaluate(occ, xy, np.array([1, 0, 1]), 1.0, 0.0, 0.0)
    assert r["points"] == 2 and r["auc"] == 1.0
