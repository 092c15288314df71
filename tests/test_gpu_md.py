"""Molecular dynamics on the GPU forces: the velocity-Verlet update against
its formula, conservation of the total energy of an NVE run with exact
(SCF-response) forces, and the warm start of the SCF from the previous
step's shifts (fewer iterations, the same self-consistent energy)."""
import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bop():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_07491_gb300 import build, bop as b
    build.build()
    return b


def test_verlet_update_formula(bop):
    rng = np.random.default_rng(80)
    n, dt, mass = 1001, 0.7, 12.5
    x, v, f = (rng.normal(size=(n, 3)) for _ in range(3))
    xd, vd, fd = (torch.tensor(a, device="cuda") for a in (x, v, f))
    a = f / mass * I.EV_PER_AMU
    bop.bop_md_verlet(xd, vd, fd, dt, mass, 0)
    v1 = v + 0.5 * dt * a
    x1 = x + dt * v1
    assert np.max(np.abs(vd.cpu().numpy() - v1)) < 1e-14
    assert np.max(np.abs(xd.cpu().numpy() - x1)) < 1e-14
    bop.bop_md_verlet(None, vd, fd, dt, mass, 1)
    assert np.max(np.abs(vd.cpu().numpy() - (v1 + 0.5 * dt * a))) < 1e-14
    # wrapping back into a periodic cell: whole lattice vectors only
    cell = np.array([[2.0, 0.0, 0.0], [0.5, 3.0, 0.0], [0.0, 0.0, 4.0]])
    xw = rng.uniform(-1.0, 5.0, size=(n, 3))
    xd = torch.tensor(xw, device="cuda")
    vd = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    fz = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    bop.bop_md_verlet(xd, vd, fz, dt, mass, 0, cell, (1, 1, 0))
    got = xd.cpu().numpy()
    fr = np.linalg.solve(cell.T, got.T).T
    assert np.all(fr[:, :2] >= -1e-12) and np.all(fr[:, :2] < 1 + 1e-12)
    k = np.linalg.solve(cell.T, (xw - got).T).T
    assert np.max(np.abs(k - np.round(k))) < 1e-9 and np.all(np.round(k[:, 2]) == 0)
    for bad in (dict(dt=0.0), dict(mass=-1.0), dict(phase=2)):
        kw = dict(dt=dt, mass=mass, phase=0)
        kw.update(bad)
        with pytest.raises(bop.BopError):
            bop.bop_md_verlet(xd, vd, fd, kw["dt"], kw["mass"], kw["phase"])


def _run_nve(bop, w, T, dt, t_end, seed=82):
    n, mass = w.n_atoms, I.MASS_FE
    ctx = bop.Context(w.model, w.run, "fp64")
    pos = torch.tensor(w.pos, device="cuda")
    vel = torch.tensor(I.maxwell_velocities(n, T, mass, seed), device="cuda")
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    delta = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.build(pos, w.cell, w.pbc)
    _, st = ctx.energy(delta=delta)
    F.copy_(ctx.forces()[0])

    def kin():
        return 0.5 * mass * float((vel * vel).sum()) / I.EV_PER_AMU

    e0 = st["e_total"] + kin()
    pots, tots, iters = [st["e_total"]], [e0], []
    for _ in range(int(round(t_end / dt))):
        _, st = ctx.md_step(pos, vel, F, w.cell, w.pbc, dt, mass, delta)
        pots.append(st["e_total"])
        tots.append(st["e_total"] + kin())
        iters.append(st["scf_iterations"])
    ctx.close()
    return np.array(pots), np.array(tots), iters, pos


def test_repulsion_matches_oracle(bop, ob):
    from conftest import oracle_model, oracle_settings
    w = I.with_run(I.small_bcc(2, 2, 2, 0.08, 90, model=I.MODEL_D_REP), scf="lcn", scf_tol=1e-12)
    res = bop.Context(w.model, w.run, "fp64").evaluate(w.pos, w.cell, w.pbc)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc)
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < 1e-9
    assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < 1e-8
    assert np.max(np.abs(res.virial.cpu().numpy() - ref["virial"])) < 1e-7


def test_nve_energy_conservation_and_warm_start(bop):
    """54-atom d cell with the pair repulsion and LCN (FP64, SCF to 1e-11,
    exact forces), 20 fs from 600 K: the total energy fluctuates by far less
    than the potential energy swings, and by a quarter as much when the time
    step is halved (velocity Verlet is second order in dt only when the
    forces are the gradient of the energy).  Warm-started SCFs take fewer
    iterations than a cold start and land on the same energy."""
    w = I.with_run(I.small_bcc(3, 3, 3, 0.05, 81, model=I.MODEL_D_REP), scf="lcn", scf_tol=1e-11, eta=1.0,
                   mix_history=8)
    n = w.n_atoms
    p1, t1, it1, pos = _run_nve(bop, w, 600.0, 1.0, 20.0)
    p2, t2, _, _ = _run_nve(bop, w, 600.0, 0.5, 20.0)
    f1 = np.max(np.abs(t1 - t1[0])) / n
    f2 = np.max(np.abs(t2 - t2[0])) / n
    swing = (p2.max() - p2.min()) / n
    print(f"fluctuation of E_tot: dt 1 fs {f1 * 1e3:.4f} meV/atom, 0.5 fs {f2 * 1e3:.4f}; E_pot swing "
          f"{swing * 1e3:.2f} meV/atom; SCF iterations {it1}")
    assert f1 < 1e-3 and swing > 20 * f2
    assert 0.15 < f2 / f1 < 0.35
    cold = bop.Context(w.model, w.run, "fp64")
    cold.build(pos, w.cell, w.pbc)
    _, sc = cold.energy()
    assert np.mean(it1[5:]) < sc["scf_iterations"]
    assert abs(sc["e_total"] - p1[-1]) < 1e-8 * n
    cold.close()
