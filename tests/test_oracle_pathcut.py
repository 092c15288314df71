"""Pins of the oracle's path-radius cut ("Performance", item (iii)): moments
against powers of the dense Hamiltonian projected onto the sites inside the
radius, no change for a radius beyond every path, smaller clusters for a
smaller radius, and forces against central differences of the cut energy."""
import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings
from test_oracle_moments import dense_periodic_H


def test_moments_are_projected_hamiltonian_powers(ob):
    """mu_n(i alpha) = <i alpha|(P H P)^n|i alpha>, P the projector on the
    atoms closer than R to atom i (a 17.2 A box: within R every site is the
    nearest image)."""
    pos, cell = I.bcc_cell(6, 6, 6)
    pos = I.jittered(pos, cell, (1, 1, 1), 0.03, np.random.default_rng(31))
    p = I.ModelParams(norb=5, b0=(-0.9, 0.6, -0.15), r0=2.48, lam=1.8, rc=2.75, dc=0.2)
    m = oracle_model(p)
    onsite = np.random.default_rng(1).normal(0, 0.2, size=(len(pos), 5))
    D, nbr, H = dense_periodic_H(ob, m, pos, cell, (1, 1, 1), onsite)
    R = 5.0
    sel = [0, 101, 431]
    mu = ob.moments(nbr.with_path_radius(pos, cell, R), H, onsite, 9, sel=sel)
    mu_full = ob.moments(nbr, H, onsite, 9, sel=sel)
    for q, i in enumerate(sel):
        d = pos - pos[i]
        fr = d @ np.linalg.inv(cell)
        d = (fr - np.round(fr)) @ cell
        inside = np.repeat(np.linalg.norm(d, axis=1) < R, 5).astype(float)
        for al in range(5):
            v = np.zeros(len(pos) * 5)
            v[i * 5 + al] = 1.0
            ref = [1.0]
            w = v.copy()
            for n in range(1, 9):
                w = inside * (D @ (inside * w))
                ref.append(v @ w)
            assert np.allclose(mu[q, al], ref, rtol=1e-10, atol=1e-11)
        assert not np.allclose(mu[q], mu_full[q], rtol=1e-6)   # the cut removes paths


def test_radius_beyond_every_path_changes_nothing(ob):
    w = I.small_bcc(2, 2, 2, 0.08, 42)
    m = oracle_model(w.model)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    on = np.zeros((w.n_atoms, 5))
    a = ob.moments(nbr, H, on, 9)
    b = ob.moments(nbr.with_path_radius(w.pos, w.cell, 4 * m.rc + 1.0), H, on, 9)
    assert np.array_equal(a, b)
    sizes = [len(ob.cluster(0, 4, nbr.with_path_radius(w.pos, w.cell, R))[0]) for R in (3.0, 5.0, 7.0, 100.0)]
    assert sizes == sorted(sizes) and sizes[0] < sizes[-1] == len(ob.cluster(0, 4, nbr)[0])


def _site_distances(ob, w, m, K):
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    out = []
    for i in range(w.n_atoms):
        at, im, _ = ob.cluster(i, K, nbr)
        d = w.pos[at] + im.astype(float) @ w.cell - w.pos[i]
        out.append(np.linalg.norm(d, axis=1))
    return np.concatenate(out)


@pytest.mark.parametrize("R", [3.4, 5.5])
def test_forces_central_differences(ob, R):
    w = I.with_run(I.small_bcc(2, 2, 2, 0.08, 91), r_path=R)
    m, st = oracle_model(w.model), oracle_settings(w.run)
    # no site sits within 2e-3 A of the radius, so h = 1e-4 moves none across it
    assert np.min(np.abs(_site_distances(ob, w, m, 4) - R)) > 2e-3
    out = ob.evaluate(m, st, w.pos, w.cell, w.pbc)
    full = ob.evaluate(m, oracle_settings(I.with_run(w, r_path=0.0).run), w.pos, w.cell, w.pbc, want_forces=False)
    assert abs(out["e_total"] - full["e_total"]) > 1e-3
    F = out["forces"]
    assert np.allclose(F.sum(axis=0), 0, atol=1e-11)
    h = 1e-4
    for (i, c) in [(0, 0), (6, 1), (13, 2)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        fd = -(ob.evaluate(m, st, p, w.cell, w.pbc, want_forces=False)["e_total"] -
               ob.evaluate(m, st, q, w.cell, w.pbc, want_forces=False)["e_total"]) / (2 * h)
        assert abs(F[i, c] - fd) < 1e-6 + 1e-5 * abs(fd), (i, c, F[i, c], fd)
