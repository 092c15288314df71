"""GPU variational SCF (Eq. BOP_SCF, U_B = U_bond + J_ii q^2 / 2) against
the oracle: shifts, energies, Fermi level, forces and virial of small cells
(FP64 and FP32 products); forces of the 2,000-atom cell against central
differences of the GPU's own energy; the model checks of the C ABI."""
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


def _var(w, J=2.0, **kw):
    args = dict(scf="variational", J_ii=J, eta=1.0, mix_history=8, scf_tol=1e-11, scf_max_it=300)
    args.update(kw)
    return I.with_run(w, **args)


@pytest.mark.parametrize("which", ["d", "s"])
def test_variational_matches_oracle_fp64(bop, ob, which):
    if which == "d":
        w = _var(I.small_bcc(2, 2, 2, 0.08, 44))
    else:
        w = _var(I.small_bcc(2, 2, 2, 0.08, 63, model=I.MODEL_S, run=I.RunParams(n_e=0.7)))
    ctx = bop.Context(w.model, w.run, "fp64")
    ctx.build(w.pos, w.cell, w.pbc)
    delta = torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda")
    e, st = ctx.energy(delta=delta)
    F, W, fs = bop.bop_forces_stats(ctx.h, w.n_atoms)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc)
    assert st["scf_converged"] == 1 and ref["scf_converged"]
    assert st["scf_residual"] < 1e-11
    assert fs["forces_scf_response"] == 1 and fs["response_iterations"] == 0
    assert np.max(np.abs(delta.cpu().numpy() - ref["delta"])) < 1e-9
    assert np.max(np.abs(e.cpu().numpy() - ref["e_atom"])) < 1e-9
    assert abs(st["e_fermi"] - ref["e_fermi"]) < 1e-9
    assert np.max(np.abs(F.cpu().numpy() - ref["forces"])) < 1e-8
    assert np.max(np.abs(W.cpu().numpy() - ref["virial"])) < 1e-7
    ctx.close()


def test_variational_fp32_products(bop, ob):
    w = _var(I.small_bcc(2, 2, 2, 0.08, 44), scf_tol=3e-5)
    res = bop.Context(w.model, w.run, "fp32").evaluate(w.pos, w.cell, w.pbc)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(_var(I.small_bcc(2, 2, 2, 0.08, 44)).run),
                      w.pos, w.cell, w.pbc)
    assert res.stats["scf_converged"] == 1
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < 1e-3
    assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < 1e-2


def test_d2000_variational_forces_by_finite_differences(bop):
    """The 2,000-atom cell in FP64: forces of the self-consistent U_B against
    central differences of the GPU energy, h = 1e-4 A (SCF to 1e-11,
    warm-started from the converged shifts)."""
    w = I.with_run(I.workload("d2000var"), scf_tol=1e-11, scf_max_it=300)
    ctx = bop.Context(w.model, w.run, "fp64")
    ctx.build(w.pos, w.cell, w.pbc)
    delta = torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda")
    _, st = ctx.energy(delta=delta)
    assert st["scf_converged"] == 1
    F, _, fs = bop.bop_forces_stats(ctx.h, w.n_atoms)
    assert fs["response_iterations"] == 0
    F = F.cpu().numpy()
    d0 = delta.clone()

    def energy(pos):
        ctx.build(pos, w.cell, w.pbc)
        d = d0.clone()
        _, s = ctx.energy(delta=d)
        assert s["scf_converged"] == 1
        return s["e_total"]

    h = 1e-4
    for (i, c) in [(0, 0), (1234, 2)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        fd = -(energy(p) - energy(q)) / (2 * h)
        assert abs(F[i, c] - fd) < 2e-5 + 1e-4 * abs(fd), (i, c, F[i, c], fd)
    ctx.close()


def test_model_checks(bop):
    w = I.small_bcc(2, 2, 2, 0.05, 46)
    for r in (I.with_run(w, scf="variational", J_ii=-1.0).run,
              I.with_run(w, scf="variational", n_spin=2).run):
        with pytest.raises(bop.BopError) as e:
            bop.bop_create(bop.make_model(w.model, r))
        assert e.value.status == bop.BOP_ERR_ARG
    bop.Context(w.model, I.with_run(w, scf="variational", J_ii=0.0).run).close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-4)])
def test_stored_and_recomputed_sweeps_agree(bop, prec, tol):
    """The SCF loop's reverse sweeps over the stored Psi (default) and with
    Psi recomputed (store budget 0): the same shifts, energy and forces."""
    w = _var(I.small_bcc(3, 3, 3, 0.08, 47), scf_tol=1e-10 if prec == "fp64" else 1e-3)
    out = []
    for budget in (-1, 0):
        ctx = bop.Context(w.model, w.run, prec)
        bop.bop_set_store_budget(ctx.h, budget)
        ctx.build(w.pos, w.cell, w.pbc)
        d = torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda")
        e, st = ctx.energy(delta=d)
        F, _ = ctx.forces()
        out.append((d.cpu().numpy(), st["e_total"], F.cpu().numpy(), st["scf_iterations"]))
        ctx.close()
    (d1, e1, F1, i1), (d2, e2, F2, i2) = out
    if prec == "fp64":
        assert i1 == i2
    assert np.max(np.abs(d1 - d2)) < tol
    assert abs(e1 - e2) < tol * w.n_atoms
    assert np.max(np.abs(F1 - F2)) < tol * max(1.0, np.abs(F2).max())
