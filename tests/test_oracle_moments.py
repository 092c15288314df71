"""Pins of the oracle's moments (Eq. momDOS) and their reverse sweep."""
from math import comb

import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model


def test_mu0_mu1_mu2_s(ob):
    """mu_0 = 1, mu_1 = E_i, mu_2 = E_i^2 + sum_j beta(r_ij)^2 for s orbitals."""
    w = I.small_bcc(3, 3, 3, 0.06, 21, model=I.MODEL_S)
    m = oracle_model(w.model)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    E = np.random.default_rng(0).normal(0, 0.3, size=(w.n_atoms, 1))
    mu = ob.moments(nbr, H, E, 5)
    assert np.allclose(mu[:, 0, 0], 1.0)
    assert np.allclose(mu[:, 0, 1], E[:, 0], atol=1e-14)
    b2 = np.zeros(w.n_atoms)
    np.add.at(b2, np.repeat(np.arange(w.n_atoms), np.diff(nbr.row_ptr)), H[:, 0, 0] ** 2)
    assert np.allclose(mu[:, 0, 2], E[:, 0] ** 2 + b2, rtol=1e-13)


def test_dimer_closed_form(ob):
    """Two s atoms with one bond: eigenvalues +-beta, mu_n = (beta^n + (-beta)^n)/2."""
    cell = np.diag([30.0, 30.0, 30.0])
    pos = np.array([[10.0, 10.0, 10.0], [10.0, 11.5, 12.0]])
    m = oracle_model(I.MODEL_S)
    nbr = ob.neighbors(pos, cell, (0, 0, 0), m.rc)
    assert nbr.n_edges == 2
    H = ob.blocks(m, pos, cell, nbr)
    beta = H[0, 0, 0]
    mu = ob.moments(nbr, H, np.zeros((2, 1)), 9)
    ref = [0.5 * (beta ** n + (-beta) ** n) for n in range(9)]
    assert np.allclose(mu[0, 0], ref, rtol=1e-13, atol=1e-15)
    assert np.allclose(mu[1, 0], ref, rtol=1e-13, atol=1e-15)


def test_perfect_bcc_first_shell_walks(ob):
    """1st-shell-only s bonds on perfect bcc: a closed walk of 2n hops is
    three independent +-1 walks, so mu_2n = beta^2n C(2n,n)^3, odd ones 0."""
    pos, cell = I.bcc_cell(4, 4, 4)
    p = I.ModelParams(norb=1, b0=(-1.0,), r0=2.48, lam=1.5, rc=2.7, dc=0.1)
    m = oracle_model(p)
    nbr = ob.neighbors(pos, cell, (1, 1, 1), m.rc)
    assert np.all(np.diff(nbr.row_ptr) == 8)
    H = ob.blocks(m, pos, cell, nbr)
    beta = H[0, 0, 0]
    mu = ob.moments(nbr, H, np.zeros((128, 1)), 9, sel=[0, 77])
    for n in range(9):
        ref = beta ** n * comb(n, n // 2) ** 3 if n % 2 == 0 else 0.0
        assert np.allclose(mu[:, 0, n], ref, rtol=1e-12, atol=1e-12)


def dense_periodic_H(ob, m, pos, cell, pbc, onsite):
    nbr = ob.neighbors(pos, cell, pbc, m.rc)
    H = ob.blocks(m, pos, cell, nbr)
    n, no = onsite.shape
    D = np.zeros((n * no, n * no))
    for i in range(n):
        D[i * no:(i + 1) * no, i * no:(i + 1) * no] += np.diag(onsite[i])
        for e in range(nbr.row_ptr[i], nbr.row_ptr[i + 1]):
            j = nbr.col[e]
            D[i * no:(i + 1) * no, j * no:(j + 1) * no] += H[e]
    return D, nbr, H


def test_exact_diagonalisation_d(ob):
    """mu_n(i alpha) = sum_k |<i alpha|k>|^2 E_k^n on a periodic cell whose
    shortest winding loop is longer than n hops (1st-shell bonds move at most
    ~1.5 A per axis; the box is 17.2 A), so the periodic and the
    infinite-crystal moments coincide."""
    pos, cell = I.bcc_cell(6, 6, 6)
    pos = I.jittered(pos, cell, (1, 1, 1), 0.03, np.random.default_rng(31))
    p = I.ModelParams(norb=5, b0=(-0.9, 0.6, -0.15), r0=2.48, lam=1.8, rc=2.75, dc=0.2)
    m = oracle_model(p)
    onsite = np.random.default_rng(1).normal(0, 0.2, size=(len(pos), 5))
    D, nbr, H = dense_periodic_H(ob, m, pos, cell, (1, 1, 1), onsite)
    assert np.allclose(D, D.T, atol=1e-14)
    evals, evecs = np.linalg.eigh(D)
    sel = [0, 101, 431]
    mu = ob.moments(nbr, H, onsite, 9, sel=sel)
    for q, i in enumerate(sel):
        for al in range(5):
            wgt = evecs[i * 5 + al] ** 2
            ref = [np.sum(wgt * evals ** n) for n in range(9)]
            assert np.allclose(mu[q, al], ref, rtol=1e-9, atol=1e-10)


def test_rotation_invariance_of_orbital_trace(ob):
    """sum_alpha mu_n(i alpha) = Tr_i H^n is invariant under a rigid rotation
    of the whole periodic structure."""
    w = I.small_bcc(3, 3, 3, 0.08, 17)
    m = oracle_model(w.model)
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    mu = ob.moments(nbr, H, np.zeros((w.n_atoms, 5)), 9, sel=[0, 3])
    pos2, cell2 = w.pos @ Q.T, w.cell @ Q.T
    nbr2 = ob.neighbors(pos2, cell2, w.pbc, m.rc)
    H2 = ob.blocks(m, pos2, cell2, nbr2)
    mu2 = ob.moments(nbr2, H2, np.zeros((w.n_atoms, 5)), 9, sel=[0, 3])
    assert np.allclose(mu.sum(axis=1), mu2.sum(axis=1), rtol=1e-11)


def test_adjoint_matches_finite_differences(ob):
    """The reverse sweep gives d(sum w mu)/dH_e and d(sum w mu)/dE; check
    against central differences of the forward moments."""
    w = I.small_bcc(2, 2, 2, 0.08, 5)
    m = oracle_model(w.model)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    rng = np.random.default_rng(9)
    E = rng.normal(0, 0.2, size=(w.n_atoms, 5))
    sel = np.array([1, 6], np.int32)
    wt = rng.normal(size=(2, 5, 9))
    Hbar, Ebar = ob.moments_adjoint(nbr, H, E, wt, sel=sel)

    def f(Hx, Ex):
        return np.sum(wt * ob.moments(nbr, Hx, Ex, 9, sel=sel))

    h = 1e-5
    for (e, b, g) in [(0, 0, 0), (3, 1, 4), (17, 2, 2), (40, 4, 3)]:
        Hp, Hm = H.copy(), H.copy()
        Hp[e, b, g] += h
        Hm[e, b, g] -= h
        fd = (f(Hp, E) - f(Hm, E)) / (2 * h)
        assert np.isclose(Hbar[e, b, g], fd, rtol=1e-6, atol=1e-8)
    for (a, b) in [(1, 0), (6, 3), (0, 2)]:
        Ep, Em = E.copy(), E.copy()
        Ep[a, b] += h
        Em[a, b] -= h
        fd = (f(H, Ep) - f(H, Em)) / (2 * h)
        assert np.isclose(Ebar[a, b], fd, rtol=1e-6, atol=1e-8)
