"""Pins of the oracle's scalar stage: recursion coefficients, Gershgorin
terminator, Chebyshev expansion, zeta chain, Jackson damping, response
functions, electron count / bond energy, Fermi level and weights."""
import numpy as np
import pytest
from scipy import integrate, special

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model


def chain_moments(a, b, n_mom):
    """Moments <0|T^n|0> of the tridiagonal (Lanczos chain) matrix T."""
    L = len(a)
    T = np.diag(a) + np.diag(b[1:L], 1) + np.diag(b[1:L], -1)
    v = np.zeros(L)
    v[0] = 1.0
    out = []
    for n in range(n_mom):
        out.append(v[0])
        v = T @ v
    return np.array(out)


def test_first_four_moments_from_chain():
    """mu_0 = 1, mu_1 = a0, mu_2 = a0^2 + b1^2, mu_3 = a0^3 + 2 a0 b1^2 + a1 b1^2
    (the relations printed under Eq. xi_merge)."""
    rng = np.random.default_rng(0)
    a = rng.normal(size=6)
    b = np.concatenate([[0.0], rng.uniform(0.5, 1.5, size=6)])
    mu = chain_moments(a, b, 4)
    a0, a1, b1 = a[0], a[1], b[1]
    assert np.allclose(mu, [1, a0, a0 ** 2 + b1 ** 2, a0 ** 3 + 2 * a0 * b1 ** 2 + a1 * b1 ** 2])


@pytest.mark.parametrize("n_mom", [5, 9, 13, 17])
def test_recursion_round_trip(ob, n_mom):
    """(a, b) -> chain moments -> recursion coefficients recovers (a, b)."""
    rng = np.random.default_rng(n_mom)
    Kp = (n_mom - 1) // 2
    M = 6
    A = rng.normal(0, 0.3, size=(M, Kp + 3))
    B = np.concatenate([np.zeros((M, 1)), rng.uniform(0.6, 1.2, size=(M, Kp + 3))], axis=1)
    mu = np.stack([chain_moments(A[r], B[r], n_mom) for r in range(M)])
    a, b, nlev = ob.recursion_coefficients(mu)
    assert np.all(nlev == Kp)
    tol = 1e-10 if n_mom <= 13 else 1e-7
    assert np.allclose(a, A[:, :Kp], atol=tol)
    assert np.allclose(b[:, 1:], B[:, 1:Kp + 1], atol=tol)
    assert np.all(b[:, 0] == 0)


def test_recursion_matches_lanczos_and_momtob(ob):
    """On moments of a random symmetric matrix the recursion gives the
    Lanczos coefficients, and b_n also equals Eq. momtob's double sum."""
    rng = np.random.default_rng(5)
    n = 40
    X = rng.normal(size=(n, n))
    H = (X + X.T) / np.sqrt(4 * n)
    v = np.zeros(n)
    v[0] = 1
    mu = []
    u = v.copy()
    for k in range(9):
        mu.append(v @ u)
        u = H @ u
    mu = np.array(mu)[None, :]
    a, b, _ = ob.recursion_coefficients(mu)
    # plain Lanczos with full re-orthogonalisation
    Q = [v]
    al, be = [], [0.0]
    for k in range(4):
        w = H @ Q[-1]
        al.append(Q[-1] @ w)
        w = w - al[-1] * Q[-1] - (be[-1] * Q[-2] if k > 0 else 0)
        for q in Q:
            w -= (q @ w) * q
        be.append(np.linalg.norm(w))
        Q.append(w / be[-1])
    assert np.allclose(a[0], al, atol=1e-10)
    assert np.allclose(b[0, 1:], be[1:5], atol=1e-10)
    # Eq. momtob: b_n = sum_j sum_l c_j^n c_l^{n-1} mu_{j+l+1}; the c's are
    # the coefficients of u_n = sum_j c_j^n H^j u_0, i.e. Q[n] in the Krylov basis
    K = np.stack([np.linalg.matrix_power(H, j) @ v for j in range(5)], axis=1)
    C = [np.linalg.lstsq(K[:, :k + 1], Q[k], rcond=None)[0] for k in range(5)]
    for nn in range(1, 5):
        s = sum(C[nn][j] * C[nn - 1][l] * mu[0, j + l + 1]
                for j in range(nn + 1) for l in range(nn))
        assert np.isclose(s, b[0, nn], atol=1e-8)


def test_semicircle_moments_give_constant_chain(ob):
    """Catalan moments (semicircle of half-width 2) -> a_n = 0, b_n = 1."""
    mu = np.array([[special.comb(n, n // 2) / (n // 2 + 1) if n % 2 == 0 else 0.0
                    for n in range(13)]])
    a, b, nlev = ob.recursion_coefficients(mu)
    assert np.allclose(a, 0, atol=1e-12) and np.allclose(b[0, 1:], 1, atol=1e-12)
    a_inf, b_inf = ob.gershgorin(a, b, nlev)
    # Gershgorin: bottom = min(a_n - b_n - b_{n+1}) = -2, top = 2
    assert np.isclose(a_inf[0], 0.0) and np.isclose(b_inf[0], 1.0)


def test_gershgorin_definition(ob):
    a = np.array([[0.1, -0.3, 0.2]])
    b = np.array([[0.0, 1.0, 1.4, 0.9]])
    a_inf, b_inf = ob.gershgorin(a, b, np.array([3]))
    bot = min(0.1 - 0 - 1.0, -0.3 - 1.0 - 1.4, 0.2 - 1.4 - 0.9)
    top = max(0.1 + 0 + 1.0, -0.3 + 1.0 + 1.4, 0.2 + 1.4 + 0.9)
    assert np.isclose(a_inf[0], (top + bot) / 2) and np.isclose(b_inf[0], (top - bot) / 4)


def test_chebyshev_coefficients_and_sine_form(ob):
    p = ob.cheb_p(20)
    x = np.linspace(-0.99, 0.99, 17)
    phi = np.arccos(x)
    for m in range(21):
        Pm = np.polyval(p[m, :m + 1][::-1], x)
        assert np.allclose(Pm, special.eval_chebyu(m, x), atol=1e-9)
        assert np.allclose(Pm, np.sin((m + 1) * phi) / np.sin(phi), atol=1e-9)


def test_jackson_factors(ob):
    g = ob.jackson(200)
    assert g[0] == 1.0 and abs(g[-1]) < 1e-15
    assert np.all(np.diff(g) < 0) and np.all(g[:-1] > 0)


def test_jackson_factors_worked_by_hand(ob):
    """Eq. Jackson evaluated by hand at small N = n_exp, then g_m =
    g^J_{m+1} / g^J_1 (m = 0..N).
    N = 2: pi/(N+1) = pi/3; g^J_1 = (2 cos(pi/3) + sin(pi/3) cot(pi/3))/3
      = (1 + 1/2)/3 = 1/2, g^J_2 = (cos(2pi/3) + sin(2pi/3) cot(pi/3))/3
      = (-1/2 + 1/2)/3 = 0, g^J_3 = 0 (sin(pi) = 0, N - 3 + 1 = 0):
      g = [1, 0, 0].
    N = 3: pi/4; g^J_1 = (3/sqrt2 + 1/sqrt2)/4 = 1/sqrt2,
      g^J_2 = (2 cos(pi/2) + 1)/4 = 1/4, g^J_3 = (-1/sqrt2 + 1/sqrt2)/4 = 0:
      g = [1, sqrt2/4, 0, 0].
    N = 5: pi/6, cot(pi/6) = sqrt3; g^J_1 = (5 sqrt3/2 + sqrt3/2)/6 =
      sqrt3/2, g^J_2 = (4/2 + 3/2)/6 = 7/12, g^J_3 = (0 + sqrt3)/6,
      g^J_4 = (2 (-1/2) + 3/2)/6 = 1/12, g^J_5 = (-sqrt3/2 + sqrt3/2)/6 = 0:
      g = [1, 7/(6 sqrt3), 1/3, 1/(6 sqrt3), 0, 0]."""
    r3 = np.sqrt(3.0)
    cases = {2: [1.0, 0.0, 0.0],
             3: [1.0, np.sqrt(2.0) / 4.0, 0.0, 0.0],
             5: [1.0, 7.0 / (6.0 * r3), 1.0 / 3.0, 1.0 / (6.0 * r3), 0.0, 0.0]}
    for N, ref in cases.items():
        g = ob.jackson(N)
        assert g.shape == (N + 1,)
        assert np.allclose(g, ref, atol=1e-15, rtol=1e-14), (N, g)


@pytest.mark.parametrize("m", [0, 1, 2, 5, 12])
def test_chi_hat_is_integral_of_dos_basis(ob, m):
    """chi_{m+1}(phi_F) = int_{-1}^{eps_F} (2/pi) sqrt(1-eps^2) U_m(eps) d eps
    with eps = cos(phi) (the reading of the phase convention)."""
    for eF in [-0.7, -0.1, 0.35, 0.9]:
        ref, _ = integrate.quad(lambda e: 2 / np.pi * np.sqrt(1 - e * e) * special.eval_chebyu(m, e),
                                -1, eF, epsabs=1e-13, epsrel=1e-13)
        chi = ob.chi_hat(m + 2, np.array([np.arccos(eF)]))
        assert np.isclose(chi[0, m + 1], ref, atol=1e-12)
    assert np.all(ob.chi_hat(5, np.array([0.3, 2.0]))[:, 0] == 0)


def d_expansion(ob, sigma=0.08, seed=3, n_mom=9, sel=None):
    w = I.small_bcc(3, 3, 3, sigma, seed)
    m = oracle_model(w.model)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    mu = ob.moments(nbr, H, np.zeros((w.n_atoms, 5)), n_mom, sel=sel)
    return mu.reshape(-1, n_mom)


def test_zeta_chain_reproduces_sigma_from_moments(ob):
    mu = d_expansion(ob, sel=[0, 4])
    a, b, nlev = ob.recursion_coefficients(mu)
    a_inf, b_inf = ob.gershgorin(a, b, nlev)
    s1 = ob.sigma_from_moments(ob.normalised_moments(mu, a_inf, b_inf))
    s2 = ob.zeta_sigma(a, b, nlev, a_inf, b_inf, 30)
    assert np.allclose(s1, s2[:, :9], atol=1e-10)


def test_band_edges_and_dos_positive(ob):
    mu = d_expansion(ob, sel=[0, 4, 11])
    ex = ob.scalar_stage(mu, 200)
    z = np.zeros_like(ex.a_inf)
    N_top, _ = ob.orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, z, float(np.max(ex.a_inf + 2 * ex.b_inf)) + 0.1)
    N_bot, _ = ob.orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, z, float(np.min(ex.a_inf - 2 * ex.b_inf)) - 0.1)
    assert np.allclose(N_top, 1.0, atol=1e-12) and np.allclose(N_bot, 0.0, atol=1e-14)
    for E in np.linspace(float(np.min(ex.a_inf - 2 * ex.b_inf)), float(np.max(ex.a_inf + 2 * ex.b_inf)), 301):
        assert np.all(ob.dos_at(ex.gsig, ex.a_inf, ex.b_inf, E) > -1e-10)
    # N is the integral of the DOS
    E0 = float(ex.a_inf[0]) + 0.3
    ref = integrate.quad(lambda E: ob.dos_at(ex.gsig[:1], ex.a_inf[:1], ex.b_inf[:1], E)[0],
                         float(ex.a_inf[0] - 2 * ex.b_inf[0]), E0, limit=400, epsabs=1e-12)[0]
    N0, _ = ob.orbital_N_U(ex.gsig[:1], ex.a_inf[:1], ex.b_inf[:1], z[:1], E0)
    assert np.isclose(N0[0], ref, atol=1e-9)


def test_energy_is_first_moment_integral(ob):
    """U = int^{E_F} (E - E_ialpha) n(E) dE (Eq. TB-Ubond), which pins the
    gamma_0 reading, against quadrature of the expanded DOS."""
    mu = d_expansion(ob, sel=[2])
    ex = ob.scalar_stage(mu, 200)
    Eon = np.array([0.13] * 5)
    for EF in [-1.0, 0.4, 1.3]:
        _, U = ob.orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, Eon, EF)
        for al in range(5):
            lo = float(ex.a_inf[al] - 2 * ex.b_inf[al])
            hi = min(EF, float(ex.a_inf[al] + 2 * ex.b_inf[al]))
            ref = integrate.quad(lambda E: (E - 0.13) * ob.dos_at(ex.gsig[al:al + 1], ex.a_inf[al:al + 1],
                                                                  ex.b_inf[al:al + 1], E)[0],
                                 lo, hi, limit=400, epsabs=1e-12)[0]
            assert np.isclose(U[al], ref, atol=1e-8)


def test_continued_fraction_square_root_terminator(ob):
    """Without damping (g = 1) and with a long expansion, N(E_F) equals the
    integral of the DOS of the square-root-terminated continued fraction
    (Eq. DOS-G with the tail of Eq. abinf)."""
    mu = d_expansion(ob, sel=[0])[:1]
    a, b, nlev = ob.recursion_coefficients(mu)
    a_inf, b_inf = ob.gershgorin(a, b, nlev)
    n_exp = 600
    sig = ob.zeta_sigma(a, b, nlev, a_inf, b_inf, n_exp)
    sig[:, :9] = ob.sigma_from_moments(ob.normalised_moments(mu, a_inf, b_inf))
    A, Bv = float(a_inf[0]), float(b_inf[0])

    def dos_cf(E):
        z = E + 1e-13j
        # tail: T = G of the constant chain, T = (z - A - sqrt((z-A)^2 - 4B^2)) / (2 B^2)
        q = z - A
        sq = np.sqrt(q * q - 4 * Bv * Bv)
        if np.imag(sq) < 0:
            sq = -sq
        T = (q - sq) / (2 * Bv * Bv)
        Kp = a.shape[1]
        g = b[0, Kp] ** 2 * T
        for n in range(Kp - 1, -1, -1):
            g = 1.0 / (z - a[0, n] - g)
            if n > 0:
                g = b[0, n] ** 2 * g
        return -np.imag(g) / np.pi

    for EF in [A - 1.0, A + 0.2, A + 1.5]:
        ref = integrate.quad(dos_cf, A - 2 * Bv, EF, limit=500, epsabs=1e-12)[0]
        N, _ = ob.orbital_N_U(sig, a_inf, b_inf, np.zeros(1), EF)
        assert np.isclose(N[0], ref, atol=1e-6)


def test_semicircle_closed_form(ob):
    """A pure semicircle (all a = A, b = B) has sigma_m = delta_m0, so
    N = g_0 chi_1(phi_F), U = B [g_1 sigma_1 chi_1 ... ] reduces to
    B[chi_2 - gamma_0 chi_1] (+ chi_0 = 0)."""
    A, Bv = 0.3, 1.1
    mu = np.array([[sum(special.comb(n, k) * A ** (n - k) * Bv ** k *
                        (special.comb(k, k // 2) / (k // 2 + 1) if k % 2 == 0 else 0) for k in range(n + 1))
                    for n in range(9)]])
    ex = ob.scalar_stage(mu, 200)
    assert np.allclose(ex.sigma[0, 1:], 0, atol=1e-10) and np.isclose(ex.sigma[0, 0], 1)
    EF, Eon = 0.8, 0.05
    N, U = ob.orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, np.array([Eon]), EF)
    phi = np.arccos((EF - A) / (2 * Bv))
    chi = ob.chi_hat(3, np.array([phi]))[0]
    assert np.isclose(N[0], chi[1], atol=1e-12)
    assert np.isclose(U[0], Bv * (chi[2] - (Eon - A) / Bv * chi[1] + chi[0]), atol=1e-12)


def test_fermi_bisection_hits_electron_count(ob):
    mu = d_expansion(ob)
    ex = ob.scalar_stage(mu, 200)
    nat = mu.shape[0] // 5
    EF, _ = ob.fermi_bisect(ex, 2.0, 6.8 * nat)
    N, _ = ob.orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, np.zeros(len(mu)), EF)
    assert abs(2 * N.sum() - 6.8 * nat) < 1e-9


def test_weights_complex_step_matches_central_differences(ob):
    mu = d_expansion(ob, sel=[0, 1])
    Eon = np.zeros(len(mu))
    ex = ob.scalar_stage(mu, 200)
    EF, _ = ob.fermi_bisect(ex, 2.0, 6.8 * 2)
    w, *_ = ob.weights(mu, Eon, EF, 200, 2.0)

    def total(m):
        e = ob.scalar_stage(m, 200)
        ef, _ = ob.fermi_bisect(e, 2.0, 6.8 * 2)
        return 2.0 * ob.orbital_N_U(e.gsig, e.a_inf, e.b_inf, Eon, ef)[1].sum()

    for (r, n) in [(0, 2), (3, 4), (7, 8), (9, 5)]:
        h = 1e-6 * max(1.0, abs(mu[r, n]))
        mp, mm = mu.copy(), mu.copy()
        mp[r, n] += h
        mm[r, n] -= h
        fd = (total(mp) - total(mm)) / (2 * h)
        assert np.isclose(w[r, n], fd, rtol=1e-4, atol=1e-7)
