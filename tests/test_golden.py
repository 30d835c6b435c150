"""Golden fixtures: the paper's scale figures and the oracle regression file."""
import json
import os

import pytest

from paper_2103_14737_gb300 import synth

G = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_geometry_matches_paper_scales(geo):
    with open(os.path.join(G, "paper_scales.json")) as f:
        p = json.load(f)
    assert geo.n_layers == p["n_layers"]["value"]
    assert geo.n_regions == p["n_regions"]["value"]
    # synthetic cell grid: within 0.5 % of the paper's element count
    assert abs(geo.n_cells - p["n_cells"]["value"]) <= 0.005 * p["n_cells"]["value"]


def test_oracle_regression():
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(G, "make_oracle_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(os.path.join(G, "oracle_regression.json")) as f:
        want = json.load(f)
    got = mk.compute()
    for k in want:
        for f_ in want[k]:
            if isinstance(want[k][f_], float):
                assert got[k][f_] == pytest.approx(want[k][f_], rel=1e-12)
            else:
                assert got[k][f_] == want[k][f_], (k, f_)
