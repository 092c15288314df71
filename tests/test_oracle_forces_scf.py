"""Pins of the oracle's energy gradient (forces, virial) and of its
self-consistency loops."""
import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings


def run(ob, w, **kw):
    return ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc, **kw)


@pytest.mark.parametrize("which", ["s", "d"])
def test_forces_central_differences(ob, which):
    """F = -dE/dr against central differences, h = 1e-4 A."""
    if which == "s":
        w = I.small_bcc(3, 3, 3, 0.08, 41, model=I.MODEL_S)
    else:
        w = I.small_bcc(2, 2, 2, 0.08, 42)
    out = run(ob, w)
    F = out["forces"]
    assert np.allclose(F.sum(axis=0), 0, atol=1e-11)
    h = 1e-4
    for (i, c) in [(0, 0), (3, 2), (7, 1)]:
        p, m = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        m[i, c] -= h
        Ep = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), p, w.cell, w.pbc,
                         want_forces=False)["e_total"]
        Em = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), m, w.cell, w.pbc,
                         want_forces=False)["e_total"]
        fd = -(Ep - Em) / (2 * h)
        assert abs(F[i, c] - fd) < 1e-6 + 1e-5 * abs(fd), (i, c, F[i, c], fd)


def test_virial_is_strain_derivative(ob):
    """virial W_ab = sum_e g_e,a d_e,b = dE/dF_ab for a deformation
    r -> F r of cell and positions.  Its symmetric part is the derivative
    with respect to symmetric strain.  It is symmetric for s orbitals.  For
    d orbitals it is not, because the orbital-resolved energy is invariant
    only under the cubic group and not under every rotation."""
    ws = I.small_bcc(2, 2, 2, 0.08, 43, model=I.MODEL_S)
    Vs = run(ob, ws)["virial"]
    assert np.allclose(Vs, Vs.T, atol=1e-9)
    w = I.small_bcc(2, 2, 2, 0.08, 43)
    out = run(ob, w)
    V = out["virial"]
    h = 1e-5
    for (a, b) in [(0, 0), (1, 2), (2, 2)]:
        e = np.zeros((3, 3))
        e[a, b] = e[b, a] = h / (2 if a != b else 1)
        vals = []
        for sgn in (1, -1):
            D = np.eye(3) + sgn * e
            vals.append(ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos @ D.T,
                                    w.cell @ D.T, w.pbc, want_forces=False)["e_total"])
        fd = (vals[0] - vals[1]) / (2 * h)
        ref = 0.5 * (V[a, b] + V[b, a])
        assert abs(ref - fd) < 1e-6 + 1e-5 * abs(fd), (a, b, ref, fd)


@pytest.mark.parametrize("which", ["s", "d"])
def test_rotation_and_permutation_invariance(ob, which):
    """s: any rotation.  d: the orbital-resolved moments (Eq. momDOS per
    i alpha) only permute under the cubic group, so a 90 degree rotation
    about z (plus a translation) leaves the energy unchanged."""
    rng = np.random.default_rng(3)
    if which == "s":
        w = I.small_bcc(2, 2, 2, 0.08, 44, model=I.MODEL_S)
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1
    else:
        w = I.small_bcc(2, 2, 2, 0.08, 44)
        Q = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    out = run(ob, w)
    pos2, cell2 = w.pos @ Q.T, w.cell @ Q.T
    if which == "d":  # keep the rotated cell a right-handed box with atoms inside
        cell2 = np.abs(cell2)
        pos2 = I.wrap(pos2, cell2, w.pbc)
    o2 = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), pos2, cell2, w.pbc)
    assert np.allclose(o2["e_atom"], out["e_atom"], atol=1e-10)
    assert np.allclose(o2["forces"], out["forces"] @ Q.T, atol=1e-9)
    perm = rng.permutation(w.n_atoms)
    o3 = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos[perm], w.cell, w.pbc)
    assert np.allclose(o3["e_atom"], out["e_atom"][perm], atol=1e-10)
    assert np.allclose(o3["forces"], out["forces"][perm], atol=1e-9)


@pytest.mark.parametrize("scf", ["lcn", "stoner"])
def test_scf_forces_central_differences(ob, scf):
    """With an SCF the forces are the total derivative of the self-consistent
    energy (onsite shifts, and for Stoner the moments, follow the atoms):
    against central differences of the converged energy, h = 1e-4 A.  The
    Hellmann-Feynman form (fixed onsite levels) misses that response."""
    base = I.small_bcc(2, 2, 2, 0.08, 47)
    kw = dict(scf="lcn") if scf == "lcn" else dict(scf="stoner", n_spin=2, stoner_I=0.8)
    w = I.with_run(base, scf_tol=1e-13, scf_max_it=400, **kw)
    out = run(ob, w)
    assert out["scf_converged"] and out["forces_include_scf_response"]
    warm = dict(delta0=out["delta"], m_init=out["m"])
    hf = run(ob, I.with_run(w, scf_response=False), **warm)
    assert not hf["forces_include_scf_response"]
    F, Fhf = out["forces"], hf["forces"]
    assert np.allclose(F.sum(axis=0), 0, atol=1e-10)
    h = 1e-4
    gap = 0.0
    for (i, c) in [(0, 0), (5, 2), (11, 1)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        Ep = run(ob, I.Workload("p", p, w.cell, w.pbc, w.model, w.run), want_forces=False, **warm)["e_total"]
        Eq = run(ob, I.Workload("q", q, w.cell, w.pbc, w.model, w.run), want_forces=False, **warm)["e_total"]
        fd = -(Ep - Eq) / (2 * h)
        assert abs(F[i, c] - fd) < 1e-6 + 1e-5 * abs(fd), (i, c, F[i, c], fd)
        gap = max(gap, abs(Fhf[i, c] - fd))
    assert gap > 1e-4


def test_lcn_scf_reaches_local_neutrality(ob):
    w = I.with_run(I.small_bcc(3, 3, 3, 0.08, 45), scf="lcn")
    out = run(ob, w, want_forces=False)
    assert out["scf_converged"]
    Ni = 2 * out["N"].sum(axis=(0, 2))
    assert np.max(np.abs(Ni - 6.8)) < 1e-9
    assert abs(out["delta"].mean()) < 1e-12
    assert out["scf_iterations"] > 1


def test_stoner_without_exchange_is_two_nonmagnetic_channels(ob):
    """I = 0 and a zero starting moment: both channels equal the
    non-magnetic run, m stays 0 and the energy is the non-magnetic one."""
    base = I.small_bcc(2, 2, 2, 0.08, 46)
    nm = run(ob, I.with_run(base, scf="lcn"), want_forces=False)
    mg = run(ob, I.with_run(base, scf="stoner", n_spin=2, stoner_I=0.0, m0=0.0),
             want_forces=False)
    assert np.allclose(mg["m"], 0, atol=1e-12)
    assert np.allclose(mg["e_atom"], nm["e_atom"], atol=1e-9)
    assert abs(mg["e_fermi"] - nm["e_fermi"]) < 1e-9


def test_stoner_magnetic_solution(ob):
    """A large exchange gives a ferromagnetic solution: equal moments in a
    perfect crystal, U_X < 0, and the two spin channels split by I m."""
    pos, cell = I.bcc_cell(2, 2, 2)
    w = I.Workload("fm", pos, cell, (1, 1, 1), I.MODEL_D,
                   I.RunParams(n_e=6.8, n_spin=2, scf="stoner", stoner_I=0.8))
    out = run(ob, w, want_forces=False)
    assert out["scf_converged"]
    m = out["m"]
    assert np.all(m > 0.1) and np.ptp(m) < 1e-8
    on = out["onsite"]
    assert np.allclose(on[1] - on[0], 0.8 * m[:, None], atol=1e-12)
