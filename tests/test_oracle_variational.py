"""Pins of the oracle's variational SCF (Eq. BOP_SCF with the binding energy
U_B = U_bond + sum_i J_ii q_i^2 / 2): the residual Delta_i = sum_alpha
(Theta~_ii - N_i) against central differences of U_B in the shifts, forces
of the converged energy against central differences (no response solve:
U_B is stationary in the shifts), the LCN limit of a large J_ii, the
perfect crystal, and the minimum."""
import numpy as np

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings


def _s_cell(seed, sigma=0.08):
    return I.small_bcc(2, 2, 2, sigma, seed, model=I.MODEL_S, run=I.RunParams(n_e=0.7))


def _var(w, J=2.0, **kw):
    args = dict(scf="variational", J_ii=J, eta=1.0, mix_history=8, scf_tol=1e-11, scf_max_it=300)
    args.update(kw)
    return I.with_run(w, **args)


def _energy_at(ob, w, delta):
    """U_B at given shifts (no SCF update: scf_max_it = 0)."""
    st = oracle_settings(I.with_run(w, scf_max_it=0).run)
    return ob.evaluate(oracle_model(w.model), st, w.pos, w.cell, w.pbc, want_forces=False, delta0=delta)


def test_residual_is_derivative_of_binding_energy(ob):
    """Delta_i from the reverse sweep against central differences of U_B in
    delta_i (E_F re-solved for the electron count), at shifts away from
    self-consistency."""
    w = _var(_s_cell(61), J=2.0)
    rng = np.random.default_rng(62)
    delta = rng.normal(scale=0.05, size=w.n_atoms)
    out = _energy_at(ob, w, delta)
    st = oracle_settings(w.run)
    stage = lambda m: ob.scalar_stage(m, st.n_exp)  # noqa: E731
    D, _, q = ob.variational_gradient(st, out["neighbors"], out["H"], out["onsite"], out["mu"].reshape(-1, 9),
                                      out["e_fermi"], stage, 2.0)
    assert abs(D.sum()) < 1e-12          # a uniform shift leaves U_B unchanged
    assert np.max(np.abs(q)) > 1e-3      # not self-consistent: the J term contributes
    h = 1e-5
    for i in (0, 5, 11):
        dp, dm = delta.copy(), delta.copy()
        dp[i] += h
        dm[i] -= h
        fd = (_energy_at(ob, w, dp)["e_total"] - _energy_at(ob, w, dm)["e_total"]) / (2 * h)
        assert abs(D[i] - fd) < 1e-8 + 1e-6 * abs(fd), (i, D[i], fd)


def test_fermi_derivative_of_bond_energy(ob):
    """dU/dE_F = (E_F - E_on) n(E_F) for every orbital of the expansion
    (U and N integrate the same density), the identity the GPU uses to form
    the E_F multiplier of U_B."""
    w = I.small_bcc(2, 2, 2, 0.08, 42)
    m = oracle_model(w.model)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    mu = ob.moments(nbr, H, np.full((w.n_atoms, 5), 0.3), 9).reshape(-1, 9)
    E_on = np.full(mu.shape[0], 0.3)
    _, _, _, dN_dEF, dU_dEF, _ = ob.weights(mu, E_on, 1.1, 200, 2.0)
    assert np.max(np.abs(dU_dEF - (1.1 - E_on) * dN_dEF)) < 1e-13


def test_forces_central_differences(ob):
    w = _var(_s_cell(63))
    m = oracle_model(w.model)
    out = ob.evaluate(m, oracle_settings(w.run), w.pos, w.cell, w.pbc)
    assert out["scf_converged"] and out["forces_include_scf_response"]
    F = out["forces"]
    assert np.allclose(F.sum(axis=0), 0, atol=1e-11)
    d0 = out["delta"]

    def energy(pos):
        r = ob.evaluate(m, oracle_settings(w.run), pos, w.cell, w.pbc, want_forces=False, delta0=d0)
        assert r["scf_converged"]
        return r["e_total"]

    h = 1e-4
    for (i, c) in [(0, 0), (3, 2), (9, 1)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        fd = -(energy(p) - energy(q)) / (2 * h)
        assert abs(F[i, c] - fd) < 1e-7 + 1e-5 * abs(fd), (i, c, F[i, c], fd)


def test_large_J_is_local_charge_neutrality(ob):
    """J_ii -> infinity forces q_i -> 0: energy and shifts approach LCN."""
    w = I.small_bcc(2, 2, 2, 0.08, 44)
    m = oracle_model(w.model)
    lcn = ob.evaluate(m, oracle_settings(I.with_run(w, scf="lcn", scf_tol=1e-11, eta=1.0, mix_history=8).run),
                      w.pos, w.cell, w.pbc, want_forces=False)
    var = ob.evaluate(m, oracle_settings(_var(w, J=1000.0, scf_tol=1e-9).run), w.pos, w.cell, w.pbc,
                      want_forces=False)
    assert var["scf_converged"]
    q = 2 * var["N"].sum(axis=(0, 2)) - w.run.n_e
    assert np.max(np.abs(q)) < 2e-4
    assert np.max(np.abs(var["delta"] - lcn["delta"])) < 1e-3
    assert abs(var["e_total"] - lcn["e_total"]) < 1e-4


def test_perfect_crystal_needs_no_shift(ob):
    w = _var(_s_cell(0, sigma=0.0))
    out = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc, want_forces=False)
    assert out["scf_converged"] and out["scf_iterations"] == 0
    assert np.max(np.abs(out["delta"])) == 0.0


def test_self_consistent_shifts_minimise_binding_energy(ob):
    w = _var(_s_cell(64))
    out = ob.evaluate(oracle_model(w.model), oracle_settings(w.run), w.pos, w.cell, w.pbc, want_forces=False)
    assert out["scf_converged"]
    d0, e0 = out["delta"], out["e_total"]
    rng = np.random.default_rng(65)
    for _ in range(3):
        v = rng.normal(size=w.n_atoms)
        v -= v.mean()
        v /= np.linalg.norm(v)
        ep = _energy_at(ob, w, d0 + 1e-3 * v)["e_total"]
        em = _energy_at(ob, w, d0 - 1e-3 * v)["e_total"]
        assert ep > e0 and em > e0
        assert abs(ep - em) < 1e-3 * (ep + em - 2 * e0)   # first order vanishes
