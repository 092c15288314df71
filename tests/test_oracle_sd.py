"""Pins of the oracle's sd-valent blocks (norb 6, s first): the bond-frame
block rotated with the paper's App. D d-orbital matrices (s is invariant),
moments against exact diagonalisation, and forces and the virial against
central differences."""
import numpy as np

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings
from test_oracle_moments import dense_periodic_H
from test_oracle_structure import paper_rotation_d


def test_sd_block_is_rotated_bond_frame_block(ob):
    """In the bond frame (bond along z) s couples only to d_{3z^2-r^2}, by
    sd sigma; the global block is R6^T H^(b) R6 with R6 = diag(1, R(theta,
    phi)) of App. D (the reading of R12)."""
    model = oracle_model(I.MODEL_SD)
    rng = np.random.default_rng(5)
    for _ in range(10):
        d = rng.normal(size=3)
        d *= rng.uniform(2.3, 3.1) / np.linalg.norm(d)
        r = np.linalg.norm(d)
        dd_s, dd_p, dd_d, ss, sd = np.array(model.b0) * np.exp(-model.lam * (r - model.r0))
        Hb = np.zeros((6, 6))
        Hb[0, 0] = ss
        Hb[0, 1] = Hb[1, 0] = sd
        Hb[1:, 1:] = np.diag([dd_s, dd_p, dd_p, dd_d, dd_d])
        R6 = np.eye(6)
        R6[1:, 1:] = paper_rotation_d(np.arccos(d[2] / r), np.arctan2(d[1], d[0]))
        B = ob.sk_block(model, d)
        assert np.allclose(B, R6.T @ Hb @ R6, atol=1e-12)
        assert np.allclose(B[1:, 1:], ob.sk_block(oracle_model(I.MODEL_D), d), atol=1e-14)


def test_sd_moments_exact_diagonalisation(ob):
    pos, cell = I.bcc_cell(5, 5, 5)
    pos = I.jittered(pos, cell, (1, 1, 1), 0.03, np.random.default_rng(32))
    p = I.ModelParams(norb=6, b0=(-0.9, 0.6, -0.15, -1.4, -0.7), r0=2.48, lam=1.8, rc=2.75, dc=0.2)
    m = oracle_model(p)
    onsite = np.random.default_rng(2).normal(0, 0.2, size=(len(pos), 6))
    onsite[:, 0] += 3.0
    D, nbr, H = dense_periodic_H(ob, m, pos, cell, (1, 1, 1), onsite)
    assert np.allclose(D, D.T, atol=1e-14)
    evals, evecs = np.linalg.eigh(D)
    sel = [0, 77, 249]
    mu = ob.moments(nbr, H, onsite, 7, sel=sel)
    for q, i in enumerate(sel):
        for al in range(6):
            wgt = evecs[i * 6 + al] ** 2
            ref = [np.sum(wgt * evals ** n) for n in range(7)]
            assert np.allclose(mu[q, al], ref, rtol=1e-9, atol=1e-10)


def test_sd_forces_and_virial_central_differences(ob):
    w = I.small_bcc(2, 2, 2, 0.08, 93, model=I.MODEL_SD)
    m, st = oracle_model(w.model), oracle_settings(w.run)
    out = ob.evaluate(m, st, w.pos, w.cell, w.pbc)
    F, V = out["forces"], out["virial"]
    assert np.allclose(F.sum(axis=0), 0, atol=1e-11)
    h = 1e-4
    for (i, c) in [(0, 0), (7, 2), (12, 1)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        fd = -(ob.evaluate(m, st, p, w.cell, w.pbc, want_forces=False)["e_total"] -
               ob.evaluate(m, st, q, w.cell, w.pbc, want_forces=False)["e_total"]) / (2 * h)
        assert abs(F[i, c] - fd) < 1e-6 + 1e-5 * abs(fd), (i, c, F[i, c], fd)
    e = np.zeros((3, 3))
    e[1, 2] = e[2, 1] = h / 2
    vals = [ob.evaluate(m, st, w.pos @ D.T, w.cell @ D.T, w.pbc, want_forces=False)["e_total"]
            for D in (np.eye(3) + e, np.eye(3) - e)]
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(0.5 * (V[1, 2] + V[2, 1]) - fd) < 1e-6 + 1e-5 * abs(fd)
    # the s level sits above the d band: the s orbitals hold few electrons
    N = out["N"][0]
    assert 2 * N[:, 0].mean() < 1.0 < 2 * N[:, 1:].sum(axis=1).mean()
