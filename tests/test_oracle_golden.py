"""Regression pin of the oracle against its stored fixture."""
import json
import os

import numpy as np

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings

HERE = os.path.dirname(os.path.abspath(__file__))


def test_s128_matches_fixture(ob):
    ref = json.load(open(os.path.join(HERE, "golden", "s128_oracle.json")))
    w = I.workload("s128")
    out = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc)
    assert np.isclose(out["e_total"] / w.n_atoms, ref["e_per_atom"], rtol=1e-12)
    assert np.isclose(out["e_fermi"], ref["e_fermi"], atol=1e-12)
    assert np.allclose(out["mu"][0, 0, 0], ref["mu_atom0"], rtol=1e-12)
    assert np.allclose(out["forces"][:4], ref["forces_atoms0_3"], atol=1e-10)
