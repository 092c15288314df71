"""The seeded input generators: Maxwell-Boltzmann velocities (no net
momentum, equipartition temperature) and the MD workload's metadata."""
import numpy as np

from paper_1803_07491_gb300 import inputs as I


def test_maxwell_velocities():
    n, T, m = 20000, 300.0, I.MASS_FE
    v = I.maxwell_velocities(n, T, m, 3)
    assert np.allclose(v.mean(axis=0), 0.0, atol=1e-15)
    # equipartition: <m v^2 / 2> = 3 kT / 2 per atom (3n - 3 free components)
    ke = 0.5 * m * np.sum(v * v) / I.EV_PER_AMU
    T_est = 2.0 * ke / ((3 * n - 3) * I.K_B)
    assert abs(T_est - T) < 0.02 * T
    assert np.array_equal(v, I.maxwell_velocities(n, T, m, 3))


def test_velocity_unit():
    """1 eV/amu in (A/fs)^2 from the SI constants."""
    ev, amu = 1.602176634e-19, 1.66053906660e-27
    assert abs(I.EV_PER_AMU - ev / amu * 1e20 / 1e30) < 1e-12


def test_md_workload():
    w = I.workload("md2000")
    assert w.n_atoms == 2000 and w.meta["dt"] == 1.0 and w.meta["mass"] == I.MASS_FE
    assert w.meta["vel"].shape == (2000, 3)
    assert np.array_equal(w.pos, I.workload("d2000").pos)


def test_spin_directions():
    """Unit vectors; the spiral keeps its cone angle and turns once over one
    period along x; the spin-spiral workload lays it over the mag2000 cell."""
    d = I.random_directions(5000, 4)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0)
    assert np.all(np.abs(d.mean(axis=0)) < 0.05)
    assert np.array_equal(d, I.random_directions(5000, 4))
    pos = np.array([[0.0, 0, 0], [2.5, 1, 1], [5.0, 2, 0], [10.0, 0, 3]])
    s = I.spiral_directions(pos, 10.0, np.pi / 3)
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0)
    assert np.allclose(s[:, 2], 0.5)
    assert np.allclose(s[0], s[3]) and np.allclose(s[2, :2], -s[0, :2]) and np.allclose(s[1, 0], 0.0)
    w = I.workload("nc2000")
    assert w.run.noncollinear and w.run.scf == "stoner" and not w.run.scf_response
    assert np.array_equal(w.pos, I.workload("mag2000").pos) and w.meta["spin_dir"].shape == (2000, 3)
