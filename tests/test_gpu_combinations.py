"""GPU against the oracle for combinations of the model options: the sd
model with Stoner magnetism and with the path-radius cut, the pair
repulsion with the variational SCF, and a band-width estimate with LCN in
FP32 products."""
import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bop():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_07491_gb300 import build, bop as b
    build.build()
    return b


CASES = {
    "sd_stoner": (I.MODEL_SD, dict(n_e=8.0, n_spin=2, scf="stoner", stoner_I=0.8, m_mix=1.0, eta=1.0,
                                   mix_history=8, scf_tol=1e-11, scf_max_it=300)),
    "sd_pathcut": (I.MODEL_SD, dict(n_e=8.0, r_path=5.5, scf="lcn", scf_tol=1e-11)),
    "rep_variational": (I.MODEL_D_REP, dict(n_e=6.8, scf="variational", J_ii=5.0, eta=1.0, mix_history=8,
                                            scf_tol=1e-11, scf_max_it=300)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_combination_fp64(bop, ob, case):
    model, kw = CASES[case]
    w = I.small_bcc(2, 2, 2, 0.08, 97, model=model, run=I.RunParams(**kw))
    res = bop.Context(w.model, w.run, "fp64").evaluate(w.pos, w.cell, w.pbc)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc)
    assert res.stats["scf_converged"] == 1 and ref["scf_converged"]
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < 1e-8
    assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < 1e-7
    assert np.max(np.abs(res.virial.cpu().numpy() - ref["virial"])) < 1e-6


def test_bandwidth_lcn_fp32(bop, ob):
    w = I.small_bcc(2, 2, 2, 0.08, 98, run=I.RunParams(n_e=6.8, scf="lcn", scf_tol=3e-5, bandwidth="minmax"))
    res = bop.Context(w.model, w.run, "fp32").evaluate(w.pos, w.cell, w.pbc)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(I.with_run(w, scf_tol=1e-12).run), w.pos, w.cell,
                      w.pbc)
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < 1e-3
    assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < 1e-2
