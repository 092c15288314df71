"""GPU parity of the band centre / width estimates (section "Band-width
estimates") and of the weighted-average terminator (Eq. weighted) against
the oracle: terminator values, energy, Fermi level, forces, virial and the
count of orbitals whose density leaves the estimated band, per estimate;
with an LCN SCF and its response; with FP32 products; and the model
checks of the C ABI."""
import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = ["gershgorin", "lowest", "highest", "average", "average_centre", "minmax", "global", "weighted"]


@pytest.fixture(scope="module")
def bop():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_07491_gb300 import build, bop as b
    build.build()
    return b


def _run(w, mode, **kw):
    return I.with_run(w, bandwidth=mode, bw_beta=1.5, bw_a=-0.5, bw_b=2.5, **kw)


def _compare(bop, ob, w, prec="fp64", tolE=1e-9, tolF=1e-8):
    ctx = bop.Context(w.model, w.run, prec)
    res = ctx.evaluate(w.pos, w.cell, w.pbc)
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc)
    n = len(w.pos)
    sE = max(1.0, np.abs(ref["e_atom"]).max())
    sF = max(1.0, np.abs(ref["forces"]).max())
    assert np.max(np.abs(res.e_atom.cpu().numpy() - ref["e_atom"])) < tolE * sE
    assert abs(res.e_fermi - ref["e_fermi"]) < tolE * sE
    assert np.max(np.abs(res.forces.cpu().numpy() - ref["forces"])) < tolF * sF
    assert np.max(np.abs(res.virial.cpu().numpy() - ref["virial"])) < tolF * sF * n
    ctx.close()
    return res, ref


@pytest.mark.parametrize("mode", MODES)
def test_estimate_matches_oracle(bop, ob, mode):
    """d orbitals, n_exp = 20: the terminator (a_inf, b_inf) of every
    orbital, energies, forces and the out-of-band count."""
    w = _run(I.small_bcc(2, 2, 2, 0.08, 42), mode, n_exp=20)
    res, ref = _compare(bop, ob, w)
    # the scalar stage alone on the oracle's moments
    mu = np.asarray(ref["mu"]).reshape(-1, w.run.n_mom)
    ctx = bop.Context(w.model, w.run)
    _, _, _, ai, bi, gs = bop.bop_recursion(ctx.h, torch.tensor(mu, device="cuda"), w.run.n_exp)
    ex = ob.scalar_stage(mu, w.run.n_exp, oracle_settings(w.run).bandwidth)
    assert np.max(np.abs(ai.cpu().numpy() - ex.a_inf)) < 1e-12
    assert np.max(np.abs(bi.cpu().numpy() - ex.b_inf)) < 1e-12
    gs = gs.cpu().numpy()
    assert np.max(np.abs(gs - ex.gsig) / np.maximum(1.0, np.abs(ex.gsig))) < 1e-9
    ctx.close()
    assert res.stats["n_unbounded"] == int(ref["unbounded"].sum())
    if mode in ("gershgorin", "minmax", "global"):
        assert res.stats["n_unbounded"] == 0
    if mode in ("lowest", "highest"):
        assert res.stats["n_unbounded"] > 0


@pytest.mark.parametrize("mode", ["minmax", "weighted", "global"])
def test_bounded_estimates_full_expansion(bop, ob, mode):
    """n_exp = 200 with the estimates whose band holds this cell's spectrum."""
    w = _run(I.small_bcc(2, 2, 2, 0.08, 43), mode)
    res, ref = _compare(bop, ob, w)
    assert res.stats["n_unbounded"] == 0 and not ref["unbounded"].any()


@pytest.mark.parametrize("mode", ["weighted", "average_centre"])
def test_estimate_with_lcn_scf_response(bop, ob, mode):
    w = _run(I.small_bcc(2, 2, 2, 0.08, 44), mode, n_exp=40, scf="lcn", scf_tol=1e-12, scf_max_it=400)
    res, ref = _compare(bop, ob, w, tolE=1e-8, tolF=1e-7)
    assert res.stats["scf_converged"] == 1 and ref["scf_converged"]


def test_estimate_fp32_products(bop, ob):
    w = _run(I.small_bcc(3, 3, 3, 0.08, 45, model=I.MODEL_S), "minmax")
    _compare(bop, ob, w, prec="fp32", tolE=1e-3, tolF=1e-2)


def test_model_checks(bop):
    w = I.small_bcc(2, 2, 2, 0.05, 46)
    for mode in MODES:
        bop.Context(w.model, I.with_run(w, bandwidth=mode).run).close()
    bad = [I.with_run(w, bandwidth="global", bw_b=0.0).run,
           I.with_run(w, bandwidth="weighted", bw_beta=-1.0).run,
           I.with_run(w, bandwidth="minmax", terminator="mlp").run]
    for r in bad:
        with pytest.raises(bop.BopError) as e:
            bop.bop_create(bop.make_model(w.model, r))
        assert e.value.status == bop.BOP_ERR_ARG
    m = bop.make_model(w.model, w.run)
    m.bandwidth = 8
    with pytest.raises(bop.BopError):
        bop.bop_create(m)
