"""GPU path-radius cut against the oracle: cluster sites bit for bit
(the same FP64 distance arithmetic decides), and energies, forces and
virial of small cells (FP64, with and without an SCF; FP32 products), plus
the gain in work on the 2,000-atom cell."""
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


@pytest.mark.parametrize("R", [3.4, 5.5])
def test_clusters_bit_exact(bop, ob, R):
    w = I.with_run(I.small_bcc(3, 3, 3, 0.08, 92), r_path=R)
    ctx = bop.Context(w.model, w.run)
    st = ctx.build(w.pos, w.cell, w.pbc)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, w.model.rc).with_path_radius(w.pos, w.cell, R)
    for atom in (0, 17, 53):
        sa, si, lev = bop.bop_get_cluster(ctx.h, atom, 4, st["max_cluster"])
        ra, ri, rl = ob.cluster(atom, 4, nbr)
        assert np.array_equal(lev.cpu().numpy(), rl)
        assert np.array_equal(sa.cpu().numpy(), ra)
        assert np.array_equal(si.cpu().numpy(), ri)
    ctx.close()


@pytest.mark.parametrize("R,scf,prec", [(3.4, "none", "fp64"), (5.5, "none", "fp64"), (5.5, "lcn", "fp64"),
                                        (5.5, "none", "fp32")])
def test_energy_forces_match_oracle(bop, ob, R, scf, prec):
    w = I.with_run(I.small_bcc(2, 2, 2, 0.08, 91), r_path=R, scf=scf, scf_tol=1e-12 if prec == "fp64" else 3e-5)
    res = bop.Context(w.model, w.run, prec).evaluate(w.pos, w.cell, w.pbc)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(I.with_run(w, scf_tol=1e-12).run), w.pos, w.cell,
                      w.pbc)
    tolE, tolF = (1e-9, 1e-8) if prec == "fp64" else (1e-3, 1e-2)
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < tolE
    assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < tolF
    assert np.max(np.abs(res.virial.cpu().numpy() - ref["virial"])) < tolF * w.n_atoms


def test_cut_reduces_work_on_d2000(bop):
    """A 5.5 A sphere (five neighbour shells) against the full 4-hop
    clusters: fewer sites and block products, and a finite energy per atom
    near the uncut one."""
    w = I.workload("d2000nscf")
    full = bop.Context(w.model, w.run)
    s_full = full.build(w.pos, w.cell, w.pbc)
    e_full = full.energy()[1]["e_total"]
    cut = bop.Context(w.model, I.with_run(w, r_path=5.5).run)
    s_cut = cut.build(w.pos, w.cell, w.pbc)
    e_cut = cut.energy()[1]["e_total"]
    assert s_cut["n_sites"] < 0.5 * s_full["n_sites"]
    assert s_cut["moment_products"] < s_full["moment_products"]
    assert abs(e_cut - e_full) / w.n_atoms < 0.5
    print(f"sites {s_full['n_sites']} -> {s_cut['n_sites']}, products {s_full['moment_products']} -> "
          f"{s_cut['moment_products']}, energy {(e_cut - e_full) / w.n_atoms * 1e3:.2f} meV/atom")
    full.close()
    cut.close()
