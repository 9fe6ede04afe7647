"""Fixtures written from the paper's text (tests/golden/, each with its
citation) against the oracle's defaults and its sorting stage."""
import json
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def test_model_constants_are_the_papers(orc):
    g = _load("paper_constants.json")
    assert orc.DEFAULTS["alpha"] == g["alpha"]
    assert orc.DEFAULTS["beta"] == g["beta"]
    assert orc.DEFAULTS["eta"] == g["eta"]
    lo, hi = g["sigma_range"]
    assert lo <= orc.DEFAULTS["sigma"] <= hi
    from paper_1807_08116_gb300 import native
    for k in ("alpha", "beta", "eta", "sigma", "gamma", "G", "eps"):
        assert native.DEFAULT_PARAMS[k] == orc.DEFAULTS[k]


def test_counting_sort_matches_the_listings(orc):
    g = _load("sorting_worked_example.json")
    key = np.array(g["cell_of_particle"], np.int32)
    count, start, perm = orc.counting_sort(key, g["M"])
    assert count.tolist() == g["CellSPH_x"]
    # the paper's inclusive CellSPH[k].y is the exclusive start of cell k + 1
    assert start[1:].tolist() == g["CellSPH_y"]
    assert start[0] == 0
    assert perm.tolist() == g["slot_order_stable"]
