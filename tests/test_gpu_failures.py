"""Failure paths of the C ABI on the GPU, all made on the host side: the
SCF loop stopped at its cap ("maximum number of steps" of the paper's
self-consistency loop, "Program flow"), the response solve of the exact
forces stopped at its cap, positions that are not numbers, and electron
counts no band can hold.  Every case returns a status code; none faults or
waits on the GPU, and the context stays usable afterwards."""
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


def _cell(**kw):
    base = I.small_bcc(2, 2, 2, 0.08, 47)  # 16 atoms, d orbitals
    return I.with_run(base, mixer="linear", **kw)


@pytest.mark.parametrize("scf,cap", [("lcn", 1), ("lcn", 3), ("stoner", 2)])
def test_scf_cap_returns_last_iterate(bop, ob, scf, cap):
    """scf_max_it = cap: BOP_ERR_NO_CONVERGENCE, and the outputs are the
    last iterate: energies, shifts and moments equal the oracle's run with
    the same cap (its loop stops at the same iteration)."""
    kw = dict(scf="lcn") if scf == "lcn" else dict(scf="stoner", n_spin=2, stoner_I=0.8)
    w = _cell(scf_tol=1e-12, scf_max_it=cap, **kw)
    ctx = bop.Context(w.model, w.run, "fp64")
    ctx.build(w.pos, w.cell, w.pbc)
    with pytest.raises(bop.BopError) as e:
        ctx.energy()
    assert e.value.status == bop.BOP_ERR_NO_CONVERGENCE
    delta = torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda")
    m = torch.full((w.n_atoms,), w.run.m0, dtype=torch.float64, device="cuda") if scf == "stoner" else None
    e_atom, st = ctx.energy(delta=delta, m=m, allow_noconv=True)
    assert st["scf_converged"] == 0 and st["scf_iterations"] == cap and st["scf_residual"] > 1e-12
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc, want_forces=False)
    assert not ref["scf_converged"] and ref["scf_iterations"] == cap
    assert np.max(np.abs(e_atom.cpu().numpy() - ref["e_atom"])) < 1e-8
    assert np.max(np.abs(delta.cpu().numpy() - ref["delta"])) < 1e-9
    if scf == "stoner":
        assert np.max(np.abs(m.cpu().numpy() - ref["m"])) < 1e-9
    # the context stays usable: the uncapped run converges
    ctx.close()
    w2 = I.with_run(w, scf_max_it=400)
    ctx = bop.Context(w2.model, w2.run, "fp64")
    ctx.build(w2.pos, w2.cell, w2.pbc)
    _, st = ctx.energy()
    assert st["scf_converged"] == 1
    ctx.close()


def test_response_solve_cap(bop, ob):
    """The GMRES solve of the exact SCF forces stopped after one iteration:
    BOP_ERR_NO_CONVERGENCE, its residual and iteration count in the stats,
    finite forces of the last iterate.  With the default limits restored the
    same context gives the oracle's forces."""
    w = _cell(scf="lcn", scf_tol=1e-12, scf_max_it=400)
    ctx = bop.Context(w.model, w.run, "fp64")
    ctx.build(w.pos, w.cell, w.pbc)
    ctx.energy()
    with pytest.raises(bop.BopError):
        bop.bop_set_response_limits(ctx.h, -1, 0.0)
    with pytest.raises(bop.BopError):
        bop.bop_set_response_limits(ctx.h, 1, float("nan"))
    bop.bop_set_response_limits(ctx.h, 1, 0.0)
    with pytest.raises(bop.BopError) as e:
        bop.bop_forces_stats(ctx.h, w.n_atoms)
    assert e.value.status == bop.BOP_ERR_NO_CONVERGENCE
    ctx.energy()
    F1, _, fs = bop.bop_forces_stats(ctx.h, w.n_atoms, allow_noconv=True)
    assert fs["response_converged"] == 0 and fs["response_iterations"] == 1
    assert fs["response_residual"] > 1e-10
    assert torch.isfinite(F1).all()
    bop.bop_set_response_limits(ctx.h, 0, 0.0)
    ctx.energy()
    F, W, fs = bop.bop_forces_stats(ctx.h, w.n_atoms)
    assert fs["response_converged"] == 1 and fs["response_iterations"] > 1
    ref = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc)
    assert np.max(np.abs(F.cpu().numpy() - ref["forces"])) < 1e-7
    # one iteration is not the converged answer
    assert np.max(np.abs(F1.cpu().numpy() - ref["forces"])) > 1e-7
    ctx.close()


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_non_finite_positions_are_refused(bop, bad):
    w = I.small_bcc(2, 2, 2, 0.05, 1)
    ctx = bop.Context(w.model, w.run)
    pos = w.pos.copy()
    pos[5, 1] = bad
    with pytest.raises(bop.BopError) as e:
        ctx.build(pos, w.cell, w.pbc)
    assert e.value.status == bop.BOP_ERR_ARG
    assert "non-finite" in str(e.value)
    res = ctx.evaluate(w.pos, w.cell, w.pbc)
    assert np.isfinite(res.e_total)
    ctx.close()


@pytest.mark.parametrize("n_e", [-0.5, 10.5, 11.0, float("nan")])
def test_impossible_electron_count_is_refused(bop, n_e):
    """A d band holds at most 10 electrons per atom (2 spins x 5 orbitals):
    a count outside [0, 10] has no Fermi level and is refused when the
    context is created, before any launch."""
    run = I.RunParams(n_e=n_e, scf="lcn")
    with pytest.raises(bop.BopError) as e:
        bop.bop_create(bop.make_model(I.MODEL_D, run))
    assert e.value.status == bop.BOP_ERR_ARG


def test_collective_failure_and_single_process_reduce(bop):
    """The reduce callback of a spatial decomposition: one that fails makes
    bop_energy return BOP_ERR_COLLECTIVE (the failure of a collective, made
    on the host), and the context evaluates again afterwards; one that
    leaves the sums as they are (one process) gives the run without a
    callback (the distributed Fermi search follows the same rules)."""
    w = I.small_bcc(2, 2, 2, 0.05, 48)
    ref = bop.Context(w.model, w.run, "fp64").evaluate(w.pos, w.cell, w.pbc)
    ctx = bop.Context(w.model, w.run, "fp64")
    calls = []

    def fail(values, count, op, user):
        calls.append(op)
        return 1

    def identity(values, count, op, user):
        calls.append(op)
        return 0

    bad = bop.REDUCE_FN(fail)
    bop.bop_set_reduce(ctx.h, bad)
    ctx.build(w.pos, w.cell, w.pbc)
    with pytest.raises(bop.BopError) as e:
        ctx.energy()
    assert e.value.status == bop.BOP_ERR_COLLECTIVE and calls
    calls.clear()
    good = bop.REDUCE_FN(identity)
    bop.bop_set_reduce(ctx.h, good)
    res = ctx.evaluate(w.pos, w.cell, w.pbc)
    assert calls
    assert abs(res.e_fermi - ref.e_fermi) < 1e-9
    assert abs(res.e_total - ref.e_total) < 1e-9 * w.n_atoms
    assert np.max(np.abs(res.forces.cpu().numpy() - ref.forces.cpu().numpy())) < 1e-9
    bop.bop_set_reduce(ctx.h, None)
    ctx.close()
