"""Pins of the oracle's non-collinear magnetism (section "Magnetism", Eqs.
onsite_CM, onsite-noncollinear; section "Torques", Eq. torque): the 2x2
spin moments against dense matrix powers of the spinor Hamiltonian of a
cell too large for any walk to wrap, the collinear limit (one common
direction reproduces the collinear Stoner result), invariance under a
global spin rotation (no spin-orbit coupling), forces and torques against
central differences of the energy, and the vanishing total torque."""
import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings


def _rot(axis, ang):
    """Rotation matrix about a unit axis (Rodrigues)."""
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def _nc(w, scf="none", **kw):
    args = dict(n_spin=2, scf=scf, stoner_I=0.8, noncollinear=True, scf_response=False, eta=1.0, m_mix=1.0,
                mix_history=8, scf_tol=1e-11, scf_max_it=300)
    args.update(kw)
    return I.with_run(w, **args)


def _fixed(ob, w, sdir, m, pos=None, want_forces=True):
    """Energy at fixed moment magnitudes m and directions sdir (no SCF)."""
    return ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos if pos is None else pos, w.cell,
                       w.pbc, want_forces=want_forces, m_init=m, spin_dir=sdir)


@pytest.mark.parametrize("model", ["s", "d"])
def test_spin_moments_against_dense_powers(ob, model):
    """M_n[a][b] = <i alpha, a|H^n|i alpha, b> for n < 5 from the cluster
    recursion against powers of the dense spinor matrix of a 6x6x6x2 cell
    (17.2 A > 4 hops x 3.6 A: no closed walk of length 4 reaches a periodic
    image), random levels, field magnitudes and directions."""
    mp = I.MODEL_S if model == "s" else I.MODEL_D
    w = I.small_bcc(6, 6, 6, 0.08, 71, model=mp)
    m = oracle_model(w.model)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    n, norb = len(w.pos), m.norb
    rng = np.random.default_rng(72)
    onsite2 = rng.normal(scale=0.3, size=(2, n, norb))
    sdir = I.random_directions(n, 73)
    sel = np.array([0, 17, 300], np.int32)
    M = ob.moments_nc(nbr, H, onsite2, sdir, 5, sel=sel)
    # dense spinor Hamiltonian: H_e (x) 1 on every directed edge, onsite blocks
    D = np.zeros((n * norb * 2, n * norb * 2), np.complex128)
    src = np.repeat(np.arange(n), np.diff(nbr.row_ptr))
    for e in range(nbr.n_edges):
        i, j = src[e], nbr.col[e]
        for b in range(norb):
            for g in range(norb):
                for sp in range(2):
                    D[(i * norb + b) * 2 + sp, (j * norb + g) * 2 + sp] += H[e, b, g]
    sx = np.array([[0, 1], [1, 0]], complex)
    sy = np.array([[0, -1j], [1j, 0]])
    sz = np.diag([1.0, -1.0]).astype(complex)
    for i in range(n):
        for b in range(norb):
            eb = 0.5 * (onsite2[0, i, b] + onsite2[1, i, b])
            h = 0.5 * (onsite2[1, i, b] - onsite2[0, i, b]) * sdir[i]
            o = (i * norb + b) * 2
            D[o:o + 2, o:o + 2] += eb * np.eye(2) + h[0] * sx + h[1] * sy + h[2] * sz
    assert np.allclose(D, D.conj().T)
    for q, i in enumerate(sel):
        for al in range(norb):
            o = (i * norb + al) * 2
            V = np.zeros((D.shape[0], 2), complex)
            V[o, 0] = V[o + 1, 1] = 1.0
            X = V.copy()
            for k in range(5):
                ref = V.conj().T @ X
                assert np.allclose(M[q, al, k], ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max())), (i, al, k)
                X = D @ X


def test_common_direction_is_collinear(ob):
    """All moments along one direction: the local channels are the
    collinear spin channels, so the Stoner SCF, energies, Fermi level,
    moments and forces equal the collinear ones for any common direction."""
    w = I.small_bcc(2, 2, 2, 0.08, 74)
    m = oracle_model(w.model)
    col = I.with_run(w, n_spin=2, scf="stoner", stoner_I=0.8, scf_response=False, eta=1.0, m_mix=1.0,
                     mix_history=8, scf_tol=1e-11, scf_max_it=300)
    ref = ob.evaluate(m, oracle_settings(col.run), w.pos, w.cell, w.pbc)
    assert ref["scf_converged"] and np.min(ref["m"]) > 0.5
    wn = _nc(w, scf="stoner")
    for s in ([0.0, 0.0, 1.0], [0.3, -0.5, 0.8], [-1.0, 0.0, 0.0]):
        sdir = np.tile(np.asarray(s) / np.linalg.norm(s), (w.n_atoms, 1))
        out = ob.evaluate(m, oracle_settings(wn.run), w.pos, w.cell, w.pbc, spin_dir=sdir)
        assert out["scf_converged"]
        assert abs(out["e_total"] - ref["e_total"]) < 1e-10 * w.n_atoms
        assert abs(out["e_fermi"] - ref["e_fermi"]) < 1e-10
        assert np.max(np.abs(out["m"] - ref["m"])) < 1e-8
        assert np.max(np.abs(out["forces"] - ref["forces"])) < 1e-9
        assert np.max(np.abs(out["torques"])) < 1e-10


def test_global_spin_rotation(ob):
    """Without spin-orbit coupling a rotation R of every moment direction
    leaves energy and forces unchanged and rotates the torques."""
    w = _nc(I.small_bcc(2, 2, 2, 0.08, 75))
    sdir = I.random_directions(w.n_atoms, 76)
    mag = np.random.default_rng(77).uniform(1.0, 2.5, w.n_atoms)
    a = _fixed(ob, w, sdir, mag)
    R = _rot([0.2, -0.7, 0.4], 1.1)
    b = _fixed(ob, w, sdir @ R.T, mag)
    assert abs(a["e_total"] - b["e_total"]) < 1e-11 * w.n_atoms
    assert np.max(np.abs(a["forces"] - b["forces"])) < 1e-10
    assert np.max(np.abs(a["torques"] @ R.T - b["torques"])) < 1e-10
    assert np.max(np.abs(a["torques"])) > 1e-3


def test_forces_central_differences(ob):
    """F = -dE/dr at fixed moment magnitudes and directions."""
    w = _nc(I.small_bcc(2, 2, 2, 0.08, 78))
    sdir = I.random_directions(w.n_atoms, 79)
    mag = np.random.default_rng(80).uniform(1.0, 2.5, w.n_atoms)
    F = _fixed(ob, w, sdir, mag)["forces"]
    assert np.allclose(F.sum(axis=0), 0, atol=1e-10)
    h = 1e-4
    for (i, c) in [(0, 0), (5, 2), (13, 1)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        fd = -(_fixed(ob, w, sdir, mag, pos=p, want_forces=False)["e_total"] -
               _fixed(ob, w, sdir, mag, pos=q, want_forces=False)["e_total"]) / (2 * h)
        assert abs(F[i, c] - fd) < 1e-7 + 1e-5 * abs(fd), (i, c, F[i, c], fd)


@pytest.mark.parametrize("norb", [1, 5])
def test_torques_central_differences(ob, norb):
    """t_i = dU/ds_i x s_i (Eq. torque): rotating s_i by a small angle e
    about an axis a changes the energy by dE/de = -t_i . a."""
    mp = I.MODEL_S if norb == 1 else I.MODEL_D
    w = _nc(I.small_bcc(2, 2, 2, 0.08, 81, model=mp), stoner_I=1.5 if norb == 1 else 0.8)
    sdir = I.random_directions(w.n_atoms, 82)
    mag = np.random.default_rng(83).uniform(0.2, 0.6 if norb == 1 else 2.5, w.n_atoms)
    out = _fixed(ob, w, sdir, mag)
    t = out["torques"]
    assert np.allclose(np.sum(t * sdir, axis=1), 0, atol=1e-14)
    # no spin-orbit coupling: rotating every moment together costs nothing
    assert np.max(np.abs(t.sum(axis=0))) < 1e-10 * max(1.0, np.abs(t).max())
    h = 1e-4
    for (i, ax) in [(0, [1, 0, 0]), (6, [0, 1, 0]), (11, [0, 0, 1]), (3, [0.4, -0.2, 0.9])]:
        ax = np.asarray(ax, float) / np.linalg.norm(ax)
        E = []
        for e in (h, -h):
            sd = sdir.copy()
            sd[i] = _rot(ax, e) @ sdir[i]
            E.append(_fixed(ob, w, sd, mag, want_forces=False)["e_total"])
        fd = (E[0] - E[1]) / (2 * h)
        assert abs(-t[i] @ ax - fd) < 1e-8 + 1e-6 * abs(fd), (i, t[i] @ ax, fd)


def test_stoner_scf_at_fixed_directions(ob):
    """Stoner SCF of the magnitudes under fixed non-collinear directions:
    the converged magnitudes reproduce themselves as local moments
    sum_alpha (N_up - N_dn), and the charge is neutral per atom."""
    w = _nc(I.small_bcc(2, 2, 2, 0.08, 84), scf="stoner")
    sdir = I.spiral_directions(w.pos, w.cell[0, 0], np.pi / 3)
    out = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc, spin_dir=sdir)
    assert out["scf_converged"]
    N = out["N"]
    assert np.max(np.abs((N[0] - N[1]).sum(axis=1) - out["m"])) < 1e-9
    assert np.max(np.abs(N.sum(axis=(0, 2)) - w.run.n_e)) < 1e-10
    assert np.min(out["m"]) > 0.5


def test_local_channels_and_global_weights(ob):
    """The projections and the global weights of section "Torques": for a
    moment along +z the up channel (lower level, spin antiparallel to s) is
    the z-down spin, and W = (w_up + w_dn)/2 + (w_dn - w_up)/2 s.sigma gives
    Re Tr(W M) = sum_nu w_nu Tr(P_nu M) for any Hermitian M."""
    rng = np.random.default_rng(106)
    n, norb, nm = 7, 5, 9
    A = rng.normal(size=(n, norb, nm, 2, 2)) + 1j * rng.normal(size=(n, norb, nm, 2, 2))
    M = A + np.conj(np.swapaxes(A, -1, -2))
    z = np.tile([0.0, 0.0, 1.0], (n, 1))
    mu = ob.local_moments(M, z)
    assert np.allclose(mu[0], M[..., 1, 1].real) and np.allclose(mu[1], M[..., 0, 0].real)
    s = I.random_directions(n, 107)
    w = rng.normal(size=(2, n, norb, nm))
    W = ob.global_weights(w, s)
    assert np.allclose(W, np.conj(np.swapaxes(W, -1, -2)))
    lhs = np.real(np.einsum("iompq,iomqp->", W, M))
    assert np.isclose(lhs, np.sum(w * ob.local_moments(M, s)), rtol=1e-13)
    # Tr(sigma M) against the Pauli matrices written out
    P = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1.0, -1.0])]
    v = ob.pauli_vector(M)
    for x in range(3):
        assert np.allclose(v[..., x], np.real(np.einsum("pq,iomqp->iom", P[x], M)))
