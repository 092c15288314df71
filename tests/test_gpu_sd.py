"""GPU sd-valent model (norb 6) against the oracle: bond blocks, moments,
energies, Fermi level, forces and virial of small cells (FP64 with and
without LCN, FP32 products), stored and recomputed reverse sweeps, and the
2,000-atom cell's forces against central differences of its energy."""
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


def test_sd_blocks_and_moments(bop, ob):
    w = I.small_bcc(2, 2, 2, 0.08, 94, model=I.MODEL_SD)
    ctx = bop.Context(w.model, w.run, "fp64")
    ctx.build(w.pos, w.cell, w.pbc)
    atoms, d, blk = bop.bop_get_bonds(ctx.h, 6)
    m = oracle_model(w.model)
    iu = np.triu_indices(6)
    for b in range(0, len(d), 7):
        B = ob.sk_block(m, d[b].cpu().numpy())
        assert np.allclose(blk[b].cpu().numpy(), B[iu], atol=1e-14)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    on = np.zeros((w.n_atoms, 6))
    on[:, 0] = w.model.onsite_s
    ref = ob.moments(nbr, H, on, 9)
    mu = bop.bop_moments(ctx.h, 1, w.n_atoms, 6, 9, onsite=torch.tensor(on, device="cuda"))
    assert np.max(np.abs(mu.cpu().numpy().reshape(ref.shape) - ref) / np.maximum(1.0, np.abs(ref))) < 1e-12
    ctx.close()


@pytest.mark.parametrize("scf,prec", [("none", "fp64"), ("lcn", "fp64"), ("none", "fp32"), ("lcn", "fp32")])
def test_sd_energy_forces_match_oracle(bop, ob, scf, prec):
    w = I.with_run(I.small_bcc(2, 2, 2, 0.08, 95, model=I.MODEL_SD), scf=scf,
                   scf_tol=1e-12 if prec == "fp64" else 3e-5)
    res = bop.Context(w.model, w.run, prec).evaluate(w.pos, w.cell, w.pbc)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(I.with_run(w, scf_tol=1e-12).run), w.pos, w.cell,
                      w.pbc)
    tolE, tolF = (1e-9, 1e-8) if prec == "fp64" else (1e-3, 1e-2)
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < tolE
    assert abs(res.e_fermi - ref["e_fermi"]) < tolE
    assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < tolF
    assert np.max(np.abs(res.virial.cpu().numpy() - ref["virial"])) < tolF * w.n_atoms


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-4)])
def test_sd_stored_and_recomputed_sweeps_agree(bop, prec, tol):
    w = I.with_run(I.small_bcc(3, 3, 3, 0.08, 96, model=I.MODEL_SD), scf="lcn",
                   scf_tol=1e-10 if prec == "fp64" else 3e-5)
    out = []
    for budget in (-1, 0):
        ctx = bop.Context(w.model, w.run, prec)
        bop.bop_set_store_budget(ctx.h, budget)
        res = ctx.evaluate(w.pos, w.cell, w.pbc)
        out.append((res.forces.cpu().numpy(), res.virial.cpu().numpy()))
        ctx.close()
    (F1, V1), (F2, V2) = out
    assert np.max(np.abs(F1 - F2)) < tol * max(1.0, np.abs(F2).max())
    assert np.max(np.abs(V1 - V2)) < tol * max(1.0, np.abs(V2).max())


def test_sd2000_forces_by_finite_differences(bop):
    w = I.with_run(I.workload("sd2000"), scf_tol=1e-11)
    ctx = bop.Context(w.model, w.run, "fp64")
    ctx.build(w.pos, w.cell, w.pbc)
    delta = torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda")
    _, st = ctx.energy(delta=delta)
    F, _, fs = bop.bop_forces_stats(ctx.h, w.n_atoms)
    assert st["scf_converged"] == 1 and fs["response_converged"] == 1
    F = F.cpu().numpy()
    d0 = delta.clone()

    def energy(pos):
        ctx.build(pos, w.cell, w.pbc)
        d = d0.clone()
        _, s = ctx.energy(delta=d)
        return s["e_total"]

    h = 1e-4
    for (i, c) in [(0, 1), (1500, 0)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        fd = -(energy(p) - energy(q)) / (2 * h)
        assert abs(F[i, c] - fd) < 2e-5 + 1e-4 * abs(fd), (i, c, F[i, c], fd)
    ctx.close()
