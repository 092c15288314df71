"""GPU forces with the SCF response (the exact gradient of the
self-consistent energy): parity with the oracle's dense implicit-function
solve on small cells (LCN and Stoner, FP64 and FP32 products), the
Hellmann-Feynman form when the response is switched off, and central
differences of the GPU's own energy on the 2,000-atom LCN workload and a
2,662-atom Stoner cell."""
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


def _case(scf):
    base = I.small_bcc(2, 2, 2, 0.08, 47)
    kw = dict(scf="lcn") if scf == "lcn" else dict(scf="stoner", n_spin=2, stoner_I=0.8)
    return I.with_run(base, scf_tol=1e-12, scf_max_it=400, **kw)


@pytest.mark.parametrize("scf", ["lcn", "stoner"])
@pytest.mark.parametrize("response", [True, False])
def test_scf_forces_match_oracle_fp64(bop, ob, scf, response):
    w = _case(scf)
    w = I.with_run(w, scf_response=response)
    ctx = bop.Context(w.model, w.run, "fp64")
    ctx.build(w.pos, w.cell, w.pbc)
    e, st = ctx.energy()
    F, W, fs = bop.bop_forces_stats(ctx.h, w.n_atoms)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc)
    assert st["scf_converged"] == 1 and ref["scf_converged"]
    assert fs["forces_scf_response"] == (1 if response else 0)
    assert ref["forces_include_scf_response"] == response
    if response:
        assert fs["response_converged"] == 1 and fs["response_residual"] < 1e-10
        assert 0 < fs["response_iterations"] < 60
    assert np.max(np.abs(e.cpu().numpy() - ref["e_atom"])) < 1e-8
    assert np.max(np.abs(F.cpu().numpy() - ref["forces"])) < 1e-7
    assert np.max(np.abs(W.cpu().numpy() - ref["virial"])) < 1e-6
    ctx.close()


def test_scf_forces_fp32_products(bop, ob):
    w = I.with_run(_case("lcn"), scf_tol=1e-5)
    ctx = bop.Context(w.model, w.run, "fp32")
    ctx.build(w.pos, w.cell, w.pbc)
    e, st = ctx.energy()
    F, W, fs = bop.bop_forces_stats(ctx.h, w.n_atoms)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(I.with_run(w, scf_tol=1e-12).run), w.pos, w.cell,
                      w.pbc)
    assert fs["response_converged"] == 1
    assert np.max(np.abs(e.cpu().numpy() - ref["e_atom"])) < 1e-3
    assert np.max(np.abs(F.cpu().numpy() - ref["forces"])) < 1e-2
    ctx.close()


def test_d2000_lcn_forces_by_finite_differences(bop):
    """The bench workload in FP64: forces of the self-consistent energy
    against central differences of the GPU energy, h = 1e-4 A (SCF to 1e-11
    electrons, warm-started from the converged shifts)."""
    w = I.with_run(I.workload("d2000"), scf_tol=1e-11)
    ctx = bop.Context(w.model, w.run, "fp64")
    ctx.build(w.pos, w.cell, w.pbc)
    delta = torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda")
    _, st = ctx.energy(delta=delta)
    F, W, fs = bop.bop_forces_stats(ctx.h, w.n_atoms)
    assert fs["response_converged"] == 1
    F = F.cpu().numpy()
    d0 = delta.clone()

    def energy(pos):
        ctx.build(pos, w.cell, w.pbc)
        d = d0.clone()
        _, s = ctx.energy(delta=d)
        return s["e_total"]

    h = 1e-4
    for (i, c) in [(0, 0), (1234, 2)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        fd = -(energy(p) - energy(q)) / (2 * h)
        assert abs(F[i, c] - fd) < 2e-5 + 1e-4 * abs(fd), (i, c, F[i, c], fd)
    ctx.close()


def test_stoner_forces_by_finite_differences(bop):
    """A 2,662-atom Stoner cell in FP64 (5,324 unknowns of the response
    solve: shifts and moments): forces with the SCF response against
    central differences of the GPU energy, h = 1e-4 A (SCF to 1e-11,
    warm-started from the converged shifts and moments)."""
    base = I.workload("mag2000")
    pos, cell = I.bcc_jittered(11, 11, 11, 0.05, 9)
    w = I.with_run(I.Workload("mag2662", pos, cell, (1, 1, 1), base.model, base.run), scf_tol=1e-11)
    ctx = bop.Context(w.model, w.run, "fp64")
    ctx.build(w.pos, w.cell, w.pbc)
    delta = torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda")
    m = torch.full((w.n_atoms,), w.run.m0, dtype=torch.float64, device="cuda")
    _, st = ctx.energy(delta=delta, m=m)
    assert st["scf_converged"] == 1
    F, W, fs = bop.bop_forces_stats(ctx.h, w.n_atoms)
    assert fs["response_converged"] == 1 and fs["forces_scf_response"] == 1
    F = F.cpu().numpy()
    d0, m0 = delta.clone(), m.clone()

    def energy(p):
        ctx.build(p, w.cell, w.pbc)
        _, s = ctx.energy(delta=d0.clone(), m=m0.clone())
        assert s["scf_converged"] == 1
        return s["e_total"]

    h = 1e-4
    for (i, c) in [(0, 1), (2000, 0)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        fd = -(energy(p) - energy(q)) / (2 * h)
        assert abs(F[i, c] - fd) < 2e-5 + 1e-4 * abs(fd), (i, c, F[i, c], fd)
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-4)])
@pytest.mark.parametrize("which", ["d_lcn", "s", "d13"])
def test_stored_and_recomputed_reverse_sweeps_agree(bop, prec, tol, which):
    """bop_forces with Psi stored (default) and with Psi recomputed in every
    reverse sweep (store budget 0): the same forces, virial and weights."""
    if which == "d_lcn":
        w = I.with_run(I.small_bcc(3, 3, 3, 0.08, 48), scf="lcn", scf_tol=1e-10 if prec == "fp64" else 1e-5)
    elif which == "s":
        w = I.small_bcc(3, 3, 3, 0.08, 49, model=I.MODEL_S, run=I.RunParams(n_e=0.7))
    else:
        w = I.with_run(I.small_bcc(2, 2, 2, 0.08, 50), n_mom=13)
    out = []
    for budget in (-1, 0):
        ctx = bop.Context(w.model, w.run, prec)
        bop.bop_set_store_budget(ctx.h, budget)
        res = ctx.evaluate(w.pos, w.cell, w.pbc)
        orb = bop.bop_get_orbital_state(ctx.h, w.n_atoms * w.model.norb * w.run.n_spin, w.run.n_mom, weights=True)
        out.append((res.forces.cpu().numpy(), res.virial.cpu().numpy(), orb["weights"].cpu().numpy()))
        ctx.close()
    (F1, V1, W1), (F2, V2, W2) = out
    scale = max(1.0, np.abs(F2).max())
    assert np.max(np.abs(F1 - F2)) < tol * scale
    assert np.max(np.abs(V1 - V2)) < tol * max(1.0, np.abs(V2).max())
    assert np.max(np.abs(W1 - W2)) < tol * max(1.0, np.abs(W2).max())
