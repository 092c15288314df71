"""Pins of the oracle's band centre / width estimates (section "Band-width
estimates", items (i)-(v), (vii), (viii)) and of the weighted-average
terminator (Eq. weighted): values worked by hand on a short chain, the
semicircle for which every estimate is exact, limits of the weights, the
global mode against Gershgorin on a cell whose orbitals are all alike, the
bands of (v) and (vii) holding every Gershgorin disc, the indicator of a
density outside the band, and forces against central differences of the
energy for each estimate."""
import numpy as np
import pytest
from scipy import special

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings

# a_0..a_3, b_0..b_4 of a four-level chain (b_0 = 0 by definition)
A4 = np.array([[1.0, 2.0, -1.0, 0.5]])
B4 = np.array([[0.0, 1.0, 3.0, 2.0, 0.5]])

# (A, B) worked by hand from the definitions, L = 4
HAND = {
    "lowest": (1.0, 1.0),                                    # a_0, b_1
    "highest": (0.5, 0.5),                                   # a_3, b_4
    "average": (0.625, np.sqrt((1 + 9 + 4 + 0.25) / 4)),     # mean a, rms b
    "average_centre": (0.625, 0.5),                          # mean a, b_4
    "minmax": (0.5, (2 - (-1) + 4 * 3) / 4),                 # (2 + -1)/2, (3 + 12)/4
    # beta = 1: a weights 1/4, 1/3, 1/2, 1 (sum 25/12), sum w a = 11/12;
    #           b weights 1/4, 1/3, 1/2, 1, sum w b = 11/4
    "weighted": (11 / 25, 33 / 25),
    # Gershgorin: lo = 0, -2, -6, -2; hi = 2, 6, 4, 3 -> bot -6, top 6
    "gershgorin": (0.0, 3.0),
}


@pytest.mark.parametrize("mode", list(HAND))
def test_hand_worked_chain(ob, mode):
    A, B = ob.band_estimate(A4, B4, np.array([4]), ob.Bandwidth(mode, beta=1.0))
    assert np.allclose([A[0], B[0]], HAND[mode], rtol=0, atol=1e-15)


def test_truncated_chain_uses_computed_levels_only(ob):
    """nlev = 2: a_0, a_1 and b_1, b_2 are the computed coefficients."""
    a = np.array([[1.0, 2.0, 7.0, 9.0]])
    b = np.array([[0.0, 1.0, 3.0, 8.0, 9.0]])
    L = np.array([2])
    est = lambda m, **k: tuple(x[0] for x in ob.band_estimate(a, b, L, ob.Bandwidth(m, **k)))  # noqa: E731
    assert est("highest") == (2.0, 3.0)
    assert est("average_centre") == (1.5, 3.0)
    assert np.allclose(est("average"), (1.5, np.sqrt(5.0)))
    assert est("minmax") == (1.5, (1.0 + 12.0) / 4)
    assert np.allclose(est("weighted", beta=2.0), ((1 / 3 + 2) / (4 / 3), (1 / 3 + 3) / (4 / 3)))


def test_weighted_limits(ob):
    """beta = 0: plain means; beta -> infinity: the highest computed level."""
    L = np.array([4])
    A0, B0 = ob.band_estimate(A4, B4, L, ob.Bandwidth("weighted", beta=0.0))
    assert np.isclose(A0[0], A4.mean()) and np.isclose(B0[0], B4[0, 1:].mean())
    Ai, Bi = ob.band_estimate(A4, B4, L, ob.Bandwidth("weighted", beta=1e12))
    assert np.allclose([Ai[0], Bi[0]], HAND["highest"], atol=1e-10)


def test_floor_and_global(ob):
    a = np.zeros((1, 4))
    b = np.zeros((1, 5))
    for m in ob.BANDWIDTH_MODES:
        if m == "global":
            continue
        _, B = ob.band_estimate(a, b, np.array([1]), ob.Bandwidth(m))
        assert B[0] == ob.B_INF_MIN, m
    A, B = ob.band_estimate(A4, B4, np.array([4]), ob.Bandwidth("global", ga=-0.4, gb=2.5))
    assert (A[0], B[0]) == (-0.4, 2.5)


def _semicircle_mu(A, B, n):
    return np.array([[sum(special.comb(k, j) * A ** (k - j) * B ** j *
                          (special.comb(j, j // 2) / (j // 2 + 1) if j % 2 == 0 else 0) for j in range(k + 1))
                      for k in range(n)]])


@pytest.mark.parametrize("mode", [m for m in ("lowest", "highest", "average", "average_centre", "minmax",
                                              "weighted", "gershgorin")])
def test_semicircle_every_estimate_is_exact(ob, mode):
    """Moments of a semicircle of centre A and half-width 2B: a_n = A and
    b_n = B at every level, so every estimate returns (A, B) and the
    expansion is the bare semicircle, sigma_m = delta_m0."""
    A, B = 0.3, 1.1
    ex = ob.scalar_stage(_semicircle_mu(A, B, 9), 200, ob.Bandwidth(mode, beta=1.5))
    assert np.isclose(ex.a_inf[0], A, atol=1e-12) and np.isclose(ex.b_inf[0], B, atol=1e-12)
    assert np.allclose(ex.sigma[0, 1:], 0, atol=1e-10) and np.isclose(ex.sigma[0, 0], 1)


def test_global_equals_gershgorin_when_all_orbitals_alike(ob):
    """Perfect bcc with s orbitals: every orbital has the same chain, so the
    global (A, B) set to the Gershgorin values of one orbital reproduces the
    Gershgorin energy and Fermi level."""
    w = I.small_bcc(2, 2, 2, 0.0, 0, model=I.MODEL_S, run=I.RunParams(n_e=0.7))
    m = oracle_model(w.model)
    ref = ob.evaluate(m, oracle_settings(w.run), w.pos, w.cell, w.pbc, want_forces=False)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    mu = ob.moments(nbr, H, np.zeros((len(w.pos), 1)), 9).reshape(-1, 9)
    a, b, L = ob.recursion_coefficients(mu)
    ga, gb = ob.gershgorin(a, b, L)
    assert np.ptp(ga) < 1e-12 and np.ptp(gb) < 1e-12
    st = oracle_settings(w.run)
    st.bandwidth = ob.Bandwidth("global", ga=float(ga[0]), gb=float(gb[0]))
    out = ob.evaluate(m, st, w.pos, w.cell, w.pbc, want_forces=False)
    assert abs(out["e_total"] - ref["e_total"]) < 1e-12 * len(w.pos)
    assert abs(out["e_fermi"] - ref["e_fermi"]) < 1e-12


def test_minmax_and_gershgorin_bands_hold_every_disc(ob):
    """(v) and (vii) give bands [A - 2B, A + 2B] that contain every
    Gershgorin disc [a_n - b_n - b_n+1, a_n + b_n + b_n+1] of the computed
    levels; on random chains."""
    rng = np.random.default_rng(3)
    a = rng.normal(size=(200, 4))
    b = np.concatenate([np.zeros((200, 1)), rng.uniform(0.1, 2.0, size=(200, 4))], axis=1)
    L = rng.integers(1, 5, size=200)
    for mode in ("minmax", "gershgorin"):
        A, B = ob.band_estimate(a, b, L, ob.Bandwidth(mode))
        for i in range(200):
            for n in range(L[i]):
                assert a[i, n] - b[i, n] - b[i, n + 1] >= A[i] - 2 * B[i] - 1e-12
                assert a[i, n] + b[i, n] + b[i, n + 1] <= A[i] + 2 * B[i] + 1e-12


def test_outside_band_indicator(ob):
    """A band that holds the chain's spectrum keeps |sigma_m| <= m + 1 at
    every m; a band far narrower than the chain's spectrum does not."""
    w = I.small_bcc(2, 2, 2, 0.08, 42)
    m = oracle_model(w.model)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    mu = ob.moments(nbr, H, np.zeros((len(w.pos), 5)), 9).reshape(-1, 9)
    for mode in ("gershgorin", "minmax"):
        assert not ob.outside_band(ob.scalar_stage(mu, 200, ob.Bandwidth(mode)).sigma).any()
    # every band edge of this d band lies within 4 eV of E = 0.5
    assert not ob.outside_band(ob.scalar_stage(mu, 200, ob.Bandwidth("global", ga=0.5, gb=2.5)).sigma).any()
    assert ob.outside_band(ob.scalar_stage(mu, 200, ob.Bandwidth("global", ga=0.5, gb=0.5)).sigma).all()
    # a delta at the band edge x = 1 sits exactly on the bound: sigma_m = m + 1
    assert not ob.outside_band((np.arange(50) + 1.0)[None, :])


@pytest.mark.parametrize("mode", ["lowest", "highest", "average", "average_centre", "minmax", "global",
                                  "weighted"])
def test_forces_central_differences(ob, mode):
    """F = -dE/dr against central differences (h = 1e-4 A) with each
    estimate, d orbitals, n_exp = 20 (the energy is a smooth function of the
    positions at any finite n_exp, whether or not the band holds the
    chain's spectrum); the estimates differ, so the energies do too."""
    w = I.with_run(I.small_bcc(2, 2, 2, 0.08, 42), bandwidth=mode, bw_beta=1.5, bw_a=-0.5, bw_b=2.5, n_exp=20)
    m, st = oracle_model(w.model), oracle_settings(w.run)
    out = ob.evaluate(m, st, w.pos, w.cell, w.pbc)
    base = ob.evaluate(m, oracle_settings(I.with_run(w, bandwidth="gershgorin").run), w.pos, w.cell, w.pbc,
                       want_forces=False)
    assert abs(out["e_total"] - base["e_total"]) > 1e-4
    F = out["forces"]
    assert np.allclose(F.sum(axis=0), 0, atol=1e-9 * max(1.0, np.abs(F).max()))
    h = 1e-4
    for (i, c) in [(0, 0), (3, 2), (7, 1)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        Ep = ob.evaluate(m, st, p, w.cell, w.pbc, want_forces=False)["e_total"]
        Em = ob.evaluate(m, st, q, w.cell, w.pbc, want_forces=False)["e_total"]
        fd = -(Ep - Em) / (2 * h)
        assert abs(F[i, c] - fd) < 1e-6 + 1e-5 * abs(fd), (i, c, F[i, c], fd)
