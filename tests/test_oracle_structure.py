"""Pins of the oracle's structural part: neighbour list, clusters and
Slater-Koster blocks, each checked against an independent construction."""
import itertools

import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model

pytestmark = pytest.mark.filterwarnings("ignore")


def numpy_pairs(pos, cell, pbc, rc):
    """Independent enumeration of all (i, j, S) with 0 < |d| < rc."""
    n = len(pos)
    rng = [range(-2, 3) if p else range(0, 1) for p in pbc]
    out = set()
    for S in itertools.product(*rng):
        sh = np.asarray(S, float) @ cell
        d = pos[None, :, :] + sh[None, None, :] - pos[:, None, :]
        r = np.linalg.norm(d, axis=-1)
        ii, jj = np.nonzero((r < rc) & (r > 0))
        out |= {(int(i), int(j)) + tuple(S) for i, j in zip(ii, jj)}
    return out


def test_neighbors_match_numpy_enumeration(ob):
    w = I.small_bcc(2, 2, 3, 0.08, 11)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, 3.6)
    got = []
    for i in range(w.n_atoms):
        for e in range(nbr.row_ptr[i], nbr.row_ptr[i + 1]):
            got.append((i, int(nbr.col[e])) + tuple(int(x) for x in nbr.img[e]))
    assert set(got) == numpy_pairs(w.pos, w.cell, w.pbc, 3.6)
    # CSR rows sorted by (j, sx, sy, sz)
    for i in range(w.n_atoms):
        row = got[nbr.row_ptr[i]:nbr.row_ptr[i + 1]]
        assert row == sorted(row)


def test_neighbors_perfect_bcc_shells(ob):
    pos, cell = I.bcc_cell(4, 4, 4)
    nbr = ob.neighbors(pos, cell, (1, 1, 1), 3.6)
    assert np.all(np.diff(nbr.row_ptr) == 14)
    d = np.linalg.norm(ob.edge_vectors(pos, cell, nbr), axis=1)
    r1, r2 = I.A_BCC * np.sqrt(3) / 2, I.A_BCC
    assert np.sum(np.isclose(d, r1)) == 8 * 128 and np.sum(np.isclose(d, r2)) == 6 * 128


def test_neighbors_slab_and_symmetry(ob):
    pos, cell, pbc = I.slab_with_vacancies(3, 3, 4, 3, 0.08, 5)
    nbr = ob.neighbors(pos, cell, pbc, 3.6)
    assert set(map(tuple, nbr.img[:, 2:3].tolist())) == {(0,)}
    fwd = set()
    for i in range(len(pos)):
        for e in range(nbr.row_ptr[i], nbr.row_ptr[i + 1]):
            fwd.add((i, int(nbr.col[e])) + tuple(int(x) for x in nbr.img[e]))
    for (i, j, a, b, c) in fwd:
        assert (j, i, -a, -b, -c) in fwd
    assert fwd == numpy_pairs(pos, cell, pbc, 3.6)


def lattice_bfs_sizes(K, lattice="bcc"):
    """Hop-level sizes on the infinite bcc / fcc lattice with 1st+2nd shell
    bonds, in integer coordinates (units of a/2)."""
    if lattice == "bcc":
        vecs = [v for v in itertools.product((-1, 1), repeat=3)]
    else:  # fcc: 12 first neighbours (a/2)(+-1, +-1, 0) and permutations
        vecs = [v for v in itertools.product((-1, 0, 1), repeat=3) if sum(abs(c) for c in v) == 2]
    vecs += [(2, 0, 0), (-2, 0, 0), (0, 2, 0), (0, -2, 0), (0, 0, 2), (0, 0, -2)]
    seen = {(0, 0, 0)}
    front = [(0, 0, 0)]
    sizes = [1]
    for _ in range(K):
        new = set()
        for p in front:
            for v in vecs:
                q = (p[0] + v[0], p[1] + v[1], p[2] + v[2])
                if q not in seen:
                    new.add(q)
        seen |= new
        front = list(new)
        sizes.append(len(seen))
    return sizes


@pytest.mark.parametrize("K", [4, 6])
def test_cluster_levels_perfect_bcc(ob, K):
    pos, cell = I.bcc_cell(4, 4, 4)
    nbr = ob.neighbors(pos, cell, (1, 1, 1), 3.6)
    _, _, lev = ob.cluster(5, K, nbr)
    assert list(lev) == lattice_bfs_sizes(K)
    if K == 6:
        assert list(lev) == [1, 15, 65, 175, 369, 671, 1105]


@pytest.mark.parametrize("K", [4, 5])
def test_cluster_levels_perfect_fcc(ob, K):
    """fcc with 1st (12) + 2nd (6) shells within 3.6 A: the same hop-level
    sizes as a breadth-first search on the integer lattice."""
    pos, cell = I.fcc_cell(4, 4, 4, I.A_FCC)
    nbr = ob.neighbors(pos, cell, (1, 1, 1), 3.6)
    assert np.all(np.diff(nbr.row_ptr) == 18)
    _, _, lev = ob.cluster(9, K, nbr)
    assert list(lev) == lattice_bfs_sizes(K, "fcc")


def test_cluster_is_bfs_in_canonical_order(ob):
    w = I.small_bcc(3, 3, 3, 0.08, 12)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, 3.6)
    atom, im, lev = ob.cluster(7, 4, nbr)
    key = {(int(a),) + tuple(int(x) for x in s): t for t, (a, s) in enumerate(zip(atom, im))}
    level = np.searchsorted(lev, np.arange(len(atom)), side="right")
    assert len(key) == len(atom)
    for t, (a, s) in enumerate(zip(atom, im)):
        nb_levels = []
        for e in range(nbr.row_ptr[a], nbr.row_ptr[a + 1]):
            q = (int(nbr.col[e]),) + tuple(int(x) for x in (s + nbr.img[e]))
            if q in key:
                nb_levels.append(level[key[q]])
            else:
                assert level[t] == len(lev) - 1  # only the outer shell has outside neighbours
        if t > 0:
            assert min(nb_levels) == level[t] - 1
    for k in range(1, len(lev)):
        seg = [(int(atom[t]),) + tuple(int(x) for x in im[t]) for t in range(lev[k - 1], lev[k])]
        assert seg == sorted(seg)


def real_d_orbitals(u):
    """Coefficients of the d orbital aligned with unit vector u (the
    3z'^2-r^2 orbital along u) in the basis d_{3z^2-r^2}, d_zx, d_yz,
    d_{x^2-y^2}, d_xy (real spherical harmonics)."""
    l, m, n = u
    return np.array([(3 * n * n - 1) / 2, np.sqrt(3) * l * n, np.sqrt(3) * m * n,
                     np.sqrt(3) / 2 * (l * l - m * m), np.sqrt(3) * l * m])


def test_sk_d_block_spectrum_and_sigma_axis(ob):
    model = oracle_model(I.MODEL_D)
    rng = np.random.default_rng(3)
    for _ in range(20):
        d = rng.normal(size=3)
        d *= rng.uniform(2.3, 3.5) / np.linalg.norm(d)
        B = ob.sk_block(model, d)
        r = np.linalg.norm(d)
        f = 1.0 if r < model.rc - model.dc else 0.5 * (np.cos(np.pi * (r - model.rc + model.dc) / model.dc) + 1)
        s, p, t = (np.array(model.b0) * np.exp(-model.lam * (r - model.r0)) * f)
        assert np.allclose(B, B.T, atol=1e-14)
        assert np.allclose(np.sort(np.linalg.eigvalsh(B)), np.sort([s, p, p, t, t]), atol=1e-12)
        v = real_d_orbitals(d / r)
        assert np.allclose(np.linalg.norm(v), 1.0)
        assert np.allclose(B @ v, s * v, atol=1e-12)


def test_sk_bond_along_z_is_diagonal(ob):
    model = oracle_model(I.MODEL_D)
    B = ob.sk_block(model, np.array([0.0, 0.0, 2.48]))
    assert np.allclose(B, np.diag([-0.9, 0.6, 0.6, -0.15, -0.15]), atol=1e-14)
    ms = oracle_model(I.MODEL_S)
    r = 3.3
    Bs = ob.sk_block(ms, np.array([r, 0, 0]))
    fc = 0.5 * (np.cos(np.pi * (r - 3.2) / 0.4) + 1)
    assert np.isclose(Bs[0, 0], -1.0 * np.exp(-1.5 * (r - 2.48)) * fc, rtol=1e-14)


def paper_rotation_d(theta, phi):
    """App. D d-orbital rotation matrix R(theta, phi) as printed, entries
    R[row, col] with 1-based indices in the paper."""
    c, s, cp, sp = np.cos(theta), np.sin(theta), np.cos(phi), np.sin(phi)
    r3 = np.sqrt(3)
    R = np.zeros((5, 5))
    R[0, 0] = c * c - 0.5 * s * s
    R[1, 0] = -r3 * s * c
    R[2, 0] = 0
    R[3, 0] = np.sqrt(0.75) * s * s
    R[4, 0] = 0
    R[0, 1] = r3 * cp * s * c
    R[1, 1] = cp * (c * c - s * s)
    R[2, 1] = -sp * c
    R[3, 1] = -cp * s * c
    R[4, 1] = sp * s
    R[0, 2] = r3 * sp * s * c
    R[1, 2] = sp * (c * c - s * s)
    R[2, 2] = cp * c
    R[3, 2] = -sp * s * c
    R[4, 2] = -cp * s
    R[0, 3] = (cp * cp - sp * sp) * np.sqrt(0.75) * s * s
    R[1, 3] = (cp * cp - sp * sp) * s * c
    R[2, 3] = -2 * sp * cp * s
    R[3, 3] = (cp * cp - sp * sp) * (c * c + 0.5 * s * s)
    R[4, 3] = -2 * sp * cp * c
    R[0, 4] = r3 * sp * cp * s * s
    R[1, 4] = 2 * sp * cp * s * c
    R[2, 4] = (cp * cp - sp * sp) * s
    R[3, 4] = sp * cp * (c * c + 1)
    R[4, 4] = (cp * cp - sp * sp) * c
    return R


def test_paper_rotation_matrices_agree_with_sk_table(ob):
    """App. D: with theta read as the polar angle from +z (not the angle to
    the xy-plane) and the printed R[a, b] applied as R^T H^(b) R, the
    paper's rotation reproduces the Slater-Koster block; the other index
    reading R H^(b) R^T does not."""
    model = oracle_model(I.MODEL_D)
    rng = np.random.default_rng(4)
    ok_a = ok_b = True
    for _ in range(10):
        d = rng.normal(size=3)
        d *= 2.6 / np.linalg.norm(d)
        r = np.linalg.norm(d)
        theta, phi = np.arccos(d[2] / r), np.arctan2(d[1], d[0])
        s, p, t = np.array(model.b0) * np.exp(-model.lam * (r - model.r0))
        Hb = np.diag([s, p, p, t, t])
        R = paper_rotation_d(theta, phi)
        B = ob.sk_block(model, d)
        ok_a &= np.allclose(R @ Hb @ R.T, B, atol=1e-12)
        ok_b &= np.allclose(R.T @ Hb @ R, B, atol=1e-12)
    assert ok_b and not ok_a
    # both matrices become the identity at theta = phi = 0 (App. D)
    assert np.allclose(paper_rotation_d(0.0, 0.0), np.eye(5))


def test_block_rotation_covariance(ob):
    """Rotating the bond vector by a rotation Q transforms the d block as
    D(Q) B D(Q)^T, where D(Q) is read off the rotated d orbitals."""
    model = oracle_model(I.MODEL_D)
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    d = rng.normal(size=3)
    d *= 2.7 / np.linalg.norm(d)
    B = ob.sk_block(model, d)
    B2 = ob.sk_block(model, Q @ d)
    # invariants of the similarity transform
    assert np.allclose(np.trace(B), np.trace(B2))
    assert np.allclose(np.linalg.eigvalsh(B), np.linalg.eigvalsh(B2))
    assert np.isclose(np.linalg.norm(B), np.linalg.norm(B2))
