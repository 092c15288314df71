"""Pins of the oracle's pair repulsion (U_rep of Eq. U_B as
rep_A exp(-rep_p (r - r0)) fcut(r)): a dimer at distances inside, on and
beyond the taper, forces and the virial against central differences, and
the zero pressure of perfect bcc for the amplitude of MODEL_D_REP."""
from dataclasses import replace

import numpy as np

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings


def _dimer(ob, model, r):
    pos = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
    cell = np.eye(3) * 20.0
    return ob.evaluate(oracle_model(model), oracle_settings(I.RunParams(n_e=0.7)), pos, cell, (0, 0, 0))


def test_dimer_values(ob):
    """The repulsive part of a dimer's energy is one bond's phi(r): e^{-p
    (r - r0)} A below the taper, half of it mid-taper, nothing beyond rc."""
    A, p = 0.7, 3.0
    base = I.MODEL_S
    rep = replace(base, rep_A=A, rep_p=p)
    for r, f in ((2.5, 1.0), (base.rc - 0.5 * base.dc, 0.5), (base.rc + 0.05, 0.0)):
        e1, e0 = _dimer(ob, rep, r), _dimer(ob, base, r)
        d = e1["e_total"] - e0["e_total"]
        assert abs(d - f * A * np.exp(-p * (r - base.r0))) < 1e-13, (r, d)
        assert np.allclose(e1["e_atom"] - e0["e_atom"], d / 2, atol=1e-14)


def test_forces_and_virial_central_differences(ob):
    w = I.small_bcc(2, 2, 2, 0.08, 90, model=I.MODEL_D_REP)
    m, st = oracle_model(w.model), oracle_settings(w.run)
    out = ob.evaluate(m, st, w.pos, w.cell, w.pbc)
    F, V = out["forces"], out["virial"]
    assert np.allclose(F.sum(axis=0), 0, atol=1e-11)
    h = 1e-4
    for (i, c) in [(0, 0), (5, 1), (11, 2)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        fd = -(ob.evaluate(m, st, p, w.cell, w.pbc, want_forces=False)["e_total"] -
               ob.evaluate(m, st, q, w.cell, w.pbc, want_forces=False)["e_total"]) / (2 * h)
        assert abs(F[i, c] - fd) < 1e-6 + 1e-5 * abs(fd), (i, c, F[i, c], fd)
    for (a, b) in [(0, 0), (1, 2)]:
        e = np.zeros((3, 3))
        e[a, b] = e[b, a] = h / (2 if a != b else 1)
        vals = []
        for sgn in (1, -1):
            D = np.eye(3) + sgn * e
            vals.append(ob.evaluate(m, st, w.pos @ D.T, w.cell @ D.T, w.pbc, want_forces=False)["e_total"])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(0.5 * (V[a, b] + V[b, a]) - fd) < 1e-6 + 1e-5 * abs(fd)


def test_md_model_has_zero_pressure_in_perfect_bcc(ob):
    """rep_A of MODEL_D_REP cancels the trace of the bond virial of perfect
    bcc (no SCF is needed there: every atom is alike)."""
    w = I.small_bcc(2, 2, 2, 0.0, 0, model=I.MODEL_D_REP)
    out = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc)
    bond = ob.evaluate(oracle_model(I.MODEL_D), oracle_settings(w.run), w.pos, w.cell, w.pbc)
    assert abs(np.trace(out["virial"])) < 1e-9 * abs(np.trace(bond["virial"]))
    assert np.max(np.abs(out["forces"])) < 1e-10
