"""GPU-vs-oracle parity of every step of the BOP path, through the C ABI.

Tolerances (stated per test): integer arrays bit-exact; FP64 mode energies
within 1e-6 eV/atom (the achieved error is ~1e-12); FP32-products mode
within 1 meV/atom; forces within 1e-6 eV/A in FP64 mode.
"""
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


def tiny_cells():
    """Structures with degenerate features: images of the same atom in a
    2x2x2 cell (12 A wide wraps at 4 hops), a slab, vacancies."""
    out = [I.small_bcc(2, 2, 2, 0.08, 101, model=I.MODEL_S),
           I.small_bcc(3, 3, 3, 0.05, 102),
           I.workload("s128")]
    pos, cell, pbc = I.slab_with_vacancies(3, 3, 4, 3, 0.08, 103)
    out.append(I.Workload("slab", pos, cell, pbc, I.MODEL_D, I.RunParams(n_e=6.8)))
    pos, cell = I.fcc_jittered(2, 2, 2, 0.06, 104)
    out.append(I.Workload("fcc", pos, cell, (1, 1, 1), I.MODEL_D, I.RunParams(n_e=6.8)))
    return out


def oracle_nbr(ob, w):
    return ob.neighbors(w.pos, w.cell, w.pbc, w.model.rc)


@pytest.mark.parametrize("k", range(5))
def test_neighbor_list_bit_exact(bop, ob, k):
    w = tiny_cells()[k]
    ctx = bop.Context(w.model, w.run)
    ctx.build(w.pos, w.cell, w.pbc)
    row, col, img = bop.bop_get_neighbors(ctx.h)
    ref = oracle_nbr(ob, w)
    assert np.array_equal(row.cpu().numpy(), ref.row_ptr)
    assert np.array_equal(col.cpu().numpy(), ref.col)
    assert np.array_equal(img.cpu().numpy(), ref.img)


@pytest.mark.parametrize("k", range(5))
def test_clusters_bit_exact(bop, ob, k):
    w = tiny_cells()[k]
    ctx = bop.Context(w.model, w.run)
    st = ctx.build(w.pos, w.cell, w.pbc)
    ref_nbr = oracle_nbr(ob, w)
    K = (w.run.n_mom - 1) // 2
    for atom in sorted({0, w.n_atoms // 2, w.n_atoms - 1}):
        sa, si, lev = bop.bop_get_cluster(ctx.h, atom, K, st["max_cluster"])
        ra, ri, rl = ob.cluster(atom, K, ref_nbr)
        assert np.array_equal(lev.cpu().numpy(), rl)
        assert np.array_equal(sa.cpu().numpy(), ra)
        assert np.array_equal(si.cpu().numpy(), ri)


@pytest.mark.parametrize("k", [1, 3])
def test_bond_blocks(bop, ob, k):
    w = tiny_cells()[k]
    ctx = bop.Context(w.model, w.run)
    ctx.build(w.pos, w.cell, w.pbc)
    atoms, d, blk = bop.bop_get_bonds(ctx.h, w.model.norb)
    d = d.cpu().numpy()
    blk = blk.cpu().numpy()
    m = oracle_model(w.model)
    iu = np.triu_indices(5)
    for b in range(0, len(d), max(1, len(d) // 50)):
        B = ob.sk_block(m, d[b])
        assert np.allclose(blk[b], B[iu], rtol=1e-13, atol=1e-15)


def moment_case(ob, w, seed=0):
    m = oracle_model(w.model)
    nbr = oracle_nbr(ob, w)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    rng = np.random.default_rng(seed)
    on = rng.normal(0, 0.2, size=(w.n_atoms, w.model.norb))
    return nbr, H, on


@pytest.mark.parametrize("k", range(5))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_moments(bop, ob, k, prec):
    w = tiny_cells()[k]
    nbr, H, on = moment_case(ob, w)
    ref = ob.moments(nbr, H, on, w.run.n_mom)
    ctx = bop.Context(w.model, w.run, prec)
    ctx.build(w.pos, w.cell, w.pbc)
    mu = bop.bop_moments(ctx.h, 1, w.n_atoms, w.model.norb, w.run.n_mom,
                         onsite=torch.tensor(on[None], dtype=torch.float64, device="cuda").contiguous())
    mu = mu[0].cpu().numpy()
    scale = np.abs(ref).max(axis=-1, keepdims=True) + 1.0
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert np.max(np.abs(mu - ref) / scale) < tol


def test_scalar_stage_matches_oracle(bop, ob):
    w = tiny_cells()[1]
    nbr, H, on = moment_case(ob, w)
    mu = ob.moments(nbr, H, on, 9).reshape(-1, 9)
    ex = ob.scalar_stage(mu, 200)
    ctx = bop.Context(w.model, w.run)
    a, b, nlev, ai, bi, gs = bop.bop_recursion(ctx.h, torch.tensor(mu, device="cuda"), 200)
    assert np.array_equal(nlev.cpu().numpy(), ex.nlev)
    assert np.allclose(a.cpu().numpy(), ex.a, atol=1e-11)
    assert np.allclose(b.cpu().numpy(), ex.b, atol=1e-11)
    assert np.allclose(ai.cpu().numpy(), ex.a_inf, atol=1e-11)
    assert np.allclose(bi.cpu().numpy(), ex.b_inf, atol=1e-11)
    assert np.allclose(gs.cpu().numpy(), ex.gsig, atol=1e-10)


def run_both(bop, ob, w, prec="fp64", forces=True):
    ctx = bop.Context(w.model, w.run, prec)
    res = ctx.evaluate(w.pos, w.cell, w.pbc, forces=forces)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc,
                      want_forces=forces)
    return ctx, res, ref


@pytest.mark.parametrize("k", range(5))
def test_energy_and_forces_fp64(bop, ob, k):
    w = tiny_cells()[k]
    ctx, res, ref = run_both(bop, ob, w)
    assert abs(res.e_fermi - ref["e_fermi"]) < 1e-9
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < 1e-8
    assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < 1e-7
    assert np.max(np.abs(res.virial.cpu().numpy() - ref["virial"])) < 1e-6


def test_weights_match_oracle(bop, ob):
    w = tiny_cells()[1]
    ctx, res, ref = run_both(bop, ob, w)
    M = w.n_atoms * w.model.norb
    st = bop.bop_get_orbital_state(ctx.h, M, w.run.n_mom, weights=True)
    # mu_0 = <i alpha|i alpha> = 1 is not a function of the structure, so
    # w_0 never reaches a force; the two sides differ only off mu_0 = 1
    wg = st["weights"].cpu().numpy()[:, 1:]
    wr = ref["weights"].reshape(M, -1)[:, 1:]
    scale = np.abs(wr).max(axis=1, keepdims=True) + 1e-3
    assert np.max(np.abs(wg - wr) / scale) < 1e-7


@pytest.mark.parametrize("k", [0, 1])
def test_energy_fp32_products(bop, ob, k):
    w = tiny_cells()[k]
    ctx, res, ref = run_both(bop, ob, w, "fp32")
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < 1e-3
    assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < 1e-2


def test_lcn_scf(bop, ob):
    w = I.with_run(I.small_bcc(3, 3, 3, 0.08, 45), scf="lcn")
    ctx, res, ref = run_both(bop, ob, w, forces=False)
    assert res.stats["scf_converged"] == 1
    assert res.stats["scf_iterations"] == ref["scf_iterations"]
    assert abs(res.e_fermi - ref["e_fermi"]) < 1e-8
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < 1e-7


def test_stoner_scf(bop, ob):
    pos, cell = I.bcc_cell(2, 2, 2)
    pos = I.jittered(pos, cell, (1, 1, 1), 0.05, np.random.default_rng(4))
    w = I.Workload("fm", pos, cell, (1, 1, 1), I.MODEL_D,
                   I.RunParams(n_e=6.8, n_spin=2, scf="stoner", stoner_I=0.8))
    ctx = bop.Context(w.model, w.run)
    ctx.build(w.pos, w.cell, w.pbc)
    mdev = torch.full((w.n_atoms,), 2.0, dtype=torch.float64, device="cuda")
    e, st = ctx.energy(m=mdev)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc,
                      want_forces=False)
    assert st["scf_converged"] == 1
    assert np.max(np.abs(mdev.cpu().numpy() - ref["m"])) < 1e-6
    assert np.max(np.abs(e.cpu().numpy() - ref["e_atom"])) < 1e-7


def test_isolated_atoms_and_dimer(bop, ob):
    """Degenerate chains: an isolated atom (no neighbours) truncates the
    recursion at level 1, a dimer at level 2 (s orbitals)."""
    cell = np.diag([30.0, 30.0, 30.0])
    pos = np.array([[5.0, 5.0, 5.0], [20.0, 20.0, 20.0], [20.0, 21.5, 22.0]])
    w = I.Workload("iso", pos, cell, (0, 0, 0), I.MODEL_S, I.RunParams(n_e=0.7))
    ctx, res, ref = run_both(bop, ob, w)
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < 1e-8
    assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < 1e-7


def test_autograd_function(bop):
    w = tiny_cells()[0]
    ctx = bop.Context(w.model, w.run)
    pos = torch.tensor(w.pos, dtype=torch.float64, device="cuda", requires_grad=True)
    E = bop.BopEnergy.apply(pos, ctx, w.cell, w.pbc)
    E.backward()
    F, _ = ctx.forces()
    assert torch.allclose(pos.grad, -F)


def test_autograd_cell_gradient_by_finite_differences(bop):
    """The cell as a differentiable input (Eq. sigma_k): dE/dcell at fixed
    Cartesian positions against central differences of the energy (FP64,
    d-valent, 16 atoms moved away from the cell faces), and the symmetric
    strain derivative that follows from it equals the symmetric virial."""
    w = I.small_bcc(2, 2, 2, 0.05, 31)
    pos_np = I.wrap(w.pos + 0.37, w.cell, w.pbc)
    frac = np.linalg.solve(w.cell.T, pos_np.T).T
    assert frac.min() > 1e-3 and frac.max() < 1.0 - 1e-3
    ctx = bop.Context(w.model, w.run, "fp64")
    pos = torch.tensor(pos_np, dtype=torch.float64, device="cuda", requires_grad=True)
    cell = torch.tensor(w.cell, dtype=torch.float64, requires_grad=True)
    E = bop.BopEnergy.apply(pos, ctx, cell, w.pbc)
    E.backward()
    g = cell.grad.numpy()

    def energy(c):
        ctx.build(pos_np, c, w.pbc)
        _, st = ctx.energy()
        return st["e_total"]

    h = 1e-5
    for (c, a) in [(0, 0), (1, 2), (2, 1), (2, 2), (0, 1)]:
        cp, cm = w.cell.copy(), w.cell.copy()
        cp[c, a] += h
        cm[c, a] -= h
        fd = (energy(cp) - energy(cm)) / (2 * h)
        assert abs(g[c, a] - fd) < 1e-6 + 1e-6 * abs(fd), (c, a, g[c, a], fd)
    # homogeneous deformation r -> (1 + e) r of positions and cell: dE/de =
    # F^T... = (dE/dpos)^T pos + (dE/dcell)^T cell = W
    ctx.build(pos_np, w.cell, w.pbc)
    ctx.energy()
    _, W = ctx.forces()
    dEde = (-ctx.forces()[0]).cpu().numpy().T @ pos_np + g.T @ w.cell
    assert np.allclose(dEde, W.cpu().numpy(), atol=1e-9)
    ctx.close()


def test_repeated_builds_of_one_context(bop, ob):
    """One context evaluates structures of the same atom count in turn:
    small displacements (the clusters keep their sizes), large ones
    (neighbours cross r_cut, the clusters change) and the first structure
    again.  Every evaluation equals the oracle's: clusters bit-exact,
    energies and forces (no state of one build leaks into the next)."""
    base = I.small_bcc(3, 3, 3, 0.03, 61)  # 54 atoms, d orbitals, no SCF
    rng = np.random.default_rng(62)
    A = base.pos
    A2 = I.wrap(A + rng.normal(scale=0.005, size=A.shape), base.cell, base.pbc)
    B = I.wrap(A + rng.normal(scale=0.4, size=A.shape), base.cell, base.pbc)
    K = (base.run.n_mom - 1) // 2
    m = oracle_model(base.model)
    ctx = bop.Context(base.model, base.run, "fp64")
    for pos in (A, A2, B, A):
        res = ctx.evaluate(pos, base.cell, base.pbc)
        nbr = ob.neighbors(pos, base.cell, base.pbc, m.rc)
        ref = ob.evaluate(m, oracle_settings(base.run), pos, base.cell, base.pbc)
        assert abs(res.e_total - ref["e_total"]) < 1e-9 * base.n_atoms
        assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < 1e-8
        st = ctx.build(pos, base.cell, base.pbc)
        for atom in (0, 27, 53):
            sa, si, lev = bop.bop_get_cluster(ctx.h, atom, K, st["max_cluster"])
            ra, ri, rl = ob.cluster(atom, K, nbr)
            assert np.array_equal(lev.cpu().numpy(), rl)
            assert np.array_equal(sa.cpu().numpy(), ra)
            assert np.array_equal(si.cpu().numpy(), ri)
    ctx.close()
