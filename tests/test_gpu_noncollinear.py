"""GPU parity of non-collinear magnetism (section "Magnetism", Eqs.
onsite_CM and onsite-noncollinear; section "Torques", Eq. torque) against
the oracle: local channel moments, energies, Fermi level, forces, virial
and torques at fixed moment magnitudes and under the Stoner SCF at fixed
directions, for s, d and sd models, with FP32 products; the collinear
limit on the GPU; the properties of the 2,000-atom spin-spiral workload
(total torque zero, torques normal to the moments, forces summing to
zero); and the model and state checks of the C ABI."""
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


def _nc(w, scf="none", **kw):
    args = dict(n_spin=2, scf=scf, stoner_I=0.8, noncollinear=True, scf_response=False, eta=1.0, m_mix=1.0,
                mix_history=8, scf_tol=1e-11, scf_max_it=300)
    args.update(kw)
    return I.with_run(w, **args)


def _compare(bop, ob, w, sdir, mag=None, prec="fp64", tolE=1e-9, tolF=1e-8):
    ctx = bop.Context(w.model, w.run, prec)
    res = ctx.evaluate(w.pos, w.cell, w.pbc, spin_dir=sdir, m=mag)
    mu_gpu = bop.bop_get_orbital_state(ctx.h, 2 * w.n_atoms * w.model.norb, w.run.n_mom)["mu"].cpu().numpy()
    ctx.close()
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc, m_init=mag,
                      spin_dir=sdir)
    n = w.n_atoms
    sE = max(1.0, np.abs(ref["e_atom"]).max())
    sF = max(1.0, np.abs(ref["forces"]).max())
    sT = max(1.0, np.abs(ref["torques"]).max())
    mu_ref = np.asarray(ref["mu"]).reshape(mu_gpu.shape)
    assert np.max(np.abs(mu_gpu - mu_ref) / np.maximum(1.0, np.abs(mu_ref))) < tolE
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < tolE * sE
    assert abs(res.e_fermi - ref["e_fermi"]) < tolE * sE
    assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < tolF * sF
    assert np.max(np.abs(res.virial.cpu().numpy() - ref["virial"])) < tolF * sF * n
    assert np.max(np.abs(res.torques.cpu().numpy() - ref["torques"])) < tolF * sT
    return res, ref


@pytest.mark.parametrize("model", ["s", "d", "sd"])
def test_fixed_moments_match_oracle(bop, ob, model):
    """Random directions and magnitudes, no SCF (the energy is then an exact
    function of positions and directions): everything to FP64 rounding."""
    mp = {"s": I.MODEL_S, "d": I.MODEL_D, "sd": I.MODEL_SD}[model]
    w = _nc(I.small_bcc(2, 2, 2, 0.08, 91, model=mp), stoner_I=1.5 if model == "s" else 0.8)
    sdir = I.random_directions(w.n_atoms, 92)
    mag = np.random.default_rng(93).uniform(0.2, 0.6 if model == "s" else 2.5, w.n_atoms)
    res, _ = _compare(bop, ob, w, sdir, mag)
    assert np.max(np.abs(res.torques.cpu().numpy())) > 1e-3


def test_stoner_spiral_matches_oracle(bop, ob):
    """Stoner SCF of the magnitudes under a conical spin spiral."""
    w = _nc(I.small_bcc(2, 2, 2, 0.08, 94), scf="stoner")
    sdir = I.spiral_directions(w.pos, w.cell[0, 0], np.pi / 3)
    res, ref = _compare(bop, ob, w, sdir, tolE=1e-8, tolF=1e-7)
    assert res.stats["scf_converged"] == 1 and ref["scf_converged"]
    assert res.stats["forces_scf_response"] == 0


def test_fp32_products(bop, ob):
    w = _nc(I.small_bcc(2, 2, 2, 0.08, 95))
    sdir = I.random_directions(w.n_atoms, 96)
    mag = np.random.default_rng(97).uniform(1.0, 2.5, w.n_atoms)
    _compare(bop, ob, w, sdir, mag, prec="fp32", tolE=1e-4, tolF=1e-3)


def test_three_cells_ragged_tail(bop, ob):
    """A 3x3x2 cell (36 atoms: items spread over many CTAs, clusters of
    different sizes from the jitter), 13 moments."""
    w = _nc(I.small_bcc(3, 3, 2, 0.1, 98), n_mom=13, n_exp=120)
    sdir = I.random_directions(w.n_atoms, 99)
    mag = np.random.default_rng(100).uniform(1.0, 2.5, w.n_atoms)
    _compare(bop, ob, w, sdir, mag, tolE=1e-9, tolF=1e-8)


def test_common_direction_is_collinear_on_gpu(bop):
    """One common direction: the non-collinear path gives the collinear
    Stoner energies, moments and forces, and zero torques."""
    w = I.small_bcc(3, 3, 3, 0.06, 101)
    col = I.with_run(w, n_spin=2, scf="stoner", stoner_I=0.8, scf_response=False, eta=1.0, m_mix=1.0,
                     mix_history=8, scf_tol=1e-11, scf_max_it=300)
    c1 = bop.Context(w.model, col.run)
    a = c1.evaluate(w.pos, w.cell, w.pbc)
    c1.close()
    wn = _nc(w, scf="stoner")
    s = np.array([0.3, -0.5, 0.8])
    c2 = bop.Context(wn.model, wn.run)
    b = c2.evaluate(w.pos, w.cell, w.pbc, spin_dir=np.tile(s / np.linalg.norm(s), (w.n_atoms, 1)))
    c2.close()
    assert abs(a.e_total - b.e_total) < 1e-9 * w.n_atoms
    assert np.max(np.abs(a.forces.cpu().numpy() - b.forces.cpu().numpy())) < 1e-8
    assert np.max(np.abs(b.torques.cpu().numpy())) < 1e-9


def test_spiral_workload_properties(bop):
    """The 2,000-atom spin-spiral workload as benched (FP32 products):
    converged SCF, torques normal to the moments and summing to zero (no
    spin-orbit coupling), forces summing to zero."""
    # FP32 moments put a floor of a few 1e-6 electrons under the SCF
    # residual: the tolerance the benchmark takes with FP32 products
    w = I.with_run(I.workload("nc2000"), scf_tol=3e-5)
    ctx = bop.Context(w.model, w.run, "fp32")
    res = ctx.evaluate(w.pos, w.cell, w.pbc, spin_dir=w.meta["spin_dir"])
    ctx.close()
    assert res.stats["scf_converged"] == 1
    T = res.torques.cpu().numpy()
    F = res.forces.cpu().numpy()
    s = w.meta["spin_dir"]
    assert np.max(np.abs(np.sum(T * s, axis=1))) < 1e-9 * max(1.0, np.abs(T).max())
    assert np.abs(T).max() > 1e-3
    assert np.max(np.abs(T.sum(axis=0))) < 1e-3 * np.abs(T).sum(axis=0).max()
    assert np.max(np.abs(F.sum(axis=0))) < 1e-6 * w.n_atoms


def test_model_and_state_checks(bop):
    w = _nc(I.small_bcc(2, 2, 2, 0.05, 102))
    for kw in (dict(n_spin=1, scf="none"), dict(scf="stoner", scf_response=True), dict(scf="lcn"),
               dict(terminator="mlp")):
        with pytest.raises(bop.BopError) as e:
            bop.bop_create(bop.make_model(w.model, I.with_run(w, **kw).run))
        assert e.value.status == bop.BOP_ERR_ARG
    ctx = bop.Context(w.model, w.run)
    ctx.build(w.pos, w.cell, w.pbc)
    with pytest.raises(bop.BopError) as e:
        ctx.energy()
    assert e.value.status == bop.BOP_ERR_STATE
    bad = I.random_directions(w.n_atoms, 103)
    bad[3] = 0.0
    with pytest.raises(bop.BopError) as e:
        ctx.set_spin_directions(bad)
    assert e.value.status == bop.BOP_ERR_ARG
    ctx.set_spin_directions(I.random_directions(w.n_atoms, 104))
    ctx.energy()
    with pytest.raises(bop.BopError) as e:
        ctx.torques()
    assert e.value.status == bop.BOP_ERR_STATE
    ctx.forces()
    assert ctx.torques().shape == (w.n_atoms, 3)
    ctx.close()
    col = bop.Context(w.model, I.with_run(w, noncollinear=False, scf="none").run)
    col.build(w.pos, w.cell, w.pbc)
    with pytest.raises(bop.BopError) as e:
        col.set_spin_directions(I.random_directions(w.n_atoms, 105))
    assert e.value.status == bop.BOP_ERR_ARG
    col.close()
