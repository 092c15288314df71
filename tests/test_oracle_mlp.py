"""Pins of the learned-terminator oracle (oracle/mlp.py) to things other than
itself: tabulated values of the normal distribution, torch's float64
autograd and Adam (independent implementations), central differences, the
semicircle chain in closed form, and the identity between the continued
chain built from exact 17-moment targets and the 17-moment expansion."""
import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def om(ob):
    from oracle import mlp
    return mlp


def _torch_net(om, p):
    W1, b1, W2, b2, W3, b3 = [torch.tensor(a, dtype=torch.float64) for a in om.unpack(p)]
    for t in (W1, b1, W2, b2, W3, b3):
        t.requires_grad_(True)
    f = lambda x: (torch.nn.functional.gelu(torch.nn.functional.gelu(x @ W1.T + b1) @ W2.T + b2)  # noqa: E731
                   @ W3.T + b3)
    return f, [W1, b1, W2, b2, W3, b3]


def _data(seed, B=64):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(B, 18)), rng.normal(size=(B, 10)), (rng.uniform(size=B) > 0.2).astype(float)


def test_gelu_tabulated_values_and_torch(om):
    # Phi(1) = 0.841344746068543, Phi(-1) = 0.158655253931457 (normal table)
    assert om.gelu(np.array(0.0)) == 0.0
    assert abs(om.gelu(np.array(1.0)) - 0.841344746068543) < 1e-15
    assert abs(om.gelu(np.array(-1.0)) + 0.158655253931457) < 1e-15
    x = np.linspace(-6, 6, 241)
    xt = torch.tensor(x, requires_grad=True)
    yt = torch.nn.functional.gelu(xt)
    yt.sum().backward()
    assert np.max(np.abs(om.gelu(x) - yt.detach().numpy())) < 1e-15
    assert np.max(np.abs(om.gelu_prime(x) - xt.grad.numpy())) < 1e-14
    h = 1e-5
    fd = (om.gelu_prime(x + h) - om.gelu_prime(x - h)) / (2 * h)
    assert np.max(np.abs(om.gelu_second(x) - fd)) < 1e-9
    # complex step of GELU is its derivative
    z = om.gelu(x + 1e-30j)
    assert np.max(np.abs(z.imag / 1e-30 - om.gelu_prime(x))) < 1e-15


def test_forward_loss_gradient_match_torch(om):
    p = I.mlp_init_params(3)
    xs, ts, m = _data(4)
    f, leaves = _torch_net(om, p)
    y = f(torch.tensor(xs))
    assert np.max(np.abs(om.forward(p, xs)[-1] - y.detach().numpy())) < 1e-13
    mt = torch.tensor(m)
    loss_t = (((y - torch.tensor(ts)) ** 2) * mt[:, None]).sum() / (10 * mt.sum())
    loss_t.backward()
    loss, g = om.loss_and_grad(p, xs, ts, m)
    assert abs(loss - loss_t.item()) < 1e-14
    gt = np.concatenate([t.grad.numpy().ravel() for t in leaves])
    assert np.max(np.abs(g - gt)) < 1e-14 * max(1.0, np.abs(gt).max())


def test_gradient_by_central_differences(om):
    p = I.mlp_init_params(5)
    xs, ts, m = _data(6, B=16)
    _, g = om.loss_and_grad(p, xs, ts, m)
    rng = np.random.default_rng(7)
    for k in rng.choice(om.N_PARAM, size=10, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (om.loss_and_grad(pp, xs, ts, m)[0] - om.loss_and_grad(pm, xs, ts, m)[0]) / (2 * h)
        assert abs(fd - g[k]) < 1e-8 + 1e-6 * abs(fd), (k, fd, g[k])


def test_input_gradient_matches_torch(om):
    p = I.mlp_init_params(8)
    xs, _, _ = _data(9, B=8)
    ybar = np.random.default_rng(10).normal(size=(8, 10))
    f, _ = _torch_net(om, p)
    xt = torch.tensor(xs, requires_grad=True)
    (f(xt) * torch.tensor(ybar)).sum().backward()
    assert np.max(np.abs(om.input_gradient(p, xs, ybar) - xt.grad.numpy())) < 1e-13


def test_adam_matches_torch(om):
    p = I.mlp_init_params(11)
    rng = np.random.default_rng(12)
    pt = torch.tensor(p, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    st = om.AdamState(np.zeros_like(p), np.zeros_like(p))
    q = p.copy()
    for _ in range(3):
        g = rng.normal(size=p.shape)
        pt.grad = torch.tensor(g)
        opt.step()
        q = om.adam(q, g, st, 3e-3)
    assert np.max(np.abs(q - pt.detach().numpy())) < 1e-15
    # first step moves every parameter by lr * g / (|g| + eps)
    st = om.AdamState(np.zeros(3), np.zeros(3))
    g = np.array([2.0, -0.5, 1e-3])
    step = om.adam(np.zeros(3), g, st, 0.1)
    assert np.allclose(step, -0.1 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-16)


def test_bf16_rounding_matches_torch(om):
    rng = np.random.default_rng(13)
    x = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-5, 5, size=1000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0]])  # two ties
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(om.bf16_round(x), ref)
    assert om.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0            # tie to even (down)
    assert om.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # tie to even (up)


def _semicircle_moments(ac, bc, n):
    """mu_n of the chain a_k = ac, b_k = bc: a semicircle of centre ac and
    radius 2 bc, central moments C_k bc^{2k} (Catalan numbers)."""
    from math import comb
    cm = [0.0] * n
    for k in range(0, (n + 1) // 2):
        if 2 * k < n:
            cm[2 * k] = comb(2 * k, k) / (k + 1) * bc ** (2 * k)
    return np.array([[sum(comb(m, l) * ac ** (m - l) * cm[l] for l in range(m + 1)) for m in range(n)]])


def test_semicircle_features_and_targets(om):
    from math import comb
    ac, bc = -0.3, 0.7
    mu = _semicircle_moments(ac, bc, 17)
    x, a, b, nlev, ai, bi = om.features(mu[:, :9])
    assert nlev[0] == 4 and abs(ai[0] - ac) < 1e-12 and abs(bi[0] - bc) < 1e-12
    cat = [comb(2 * k, k) / (k + 1) / 4 ** k for k in range(5)]
    mh = [0.0, cat[1], 0.0, cat[2], 0.0, cat[3], 0.0, cat[4]]
    ref = np.array([0, 0, 0, 0, 1, 1, 1, 1, ac, bc] + mh)
    assert np.max(np.abs(x[0] - ref)) < 1e-11
    t, mask = om.targets(mu)
    assert mask[0] == 1.0
    assert np.max(np.abs(t[0] - np.array([0, 1, 0, 0, 0, 0, 1, 1, 1, 1]))) < 1e-9


def test_exact_targets_reproduce_17_moment_expansion(ob, om):
    w = I.small_bcc(2, 2, 2, 0.08, 21)
    m = oracle_model(w.model)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    onsite = np.zeros((len(w.pos), 5))
    mu17 = ob.moments(nbr, H, onsite, 17).reshape(-1, 17)
    t, mask = om.targets(mu17)
    assert mask.all()
    ex = om.exact_chain_stage(mu17[:, :9], t, 200)
    ref = ob.scalar_stage(mu17, 200)
    assert np.max(np.abs(ex.a_inf - ref.a_inf)) < 1e-12
    assert np.max(np.abs(ex.b_inf - ref.b_inf)) < 1e-12
    assert np.max(np.abs(ex.gsig - ref.gsig)) < 1e-9
    for ef in (-0.5, 0.0, 0.4):
        N1, U1 = ob.orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, onsite.ravel(), ef)
        N2, U2 = ob.orbital_N_U(ref.gsig, ref.a_inf, ref.b_inf, onsite.ravel(), ef)
        assert np.max(np.abs(N1 - N2)) < 1e-10 and np.max(np.abs(U1 - U2)) < 1e-10


def _fitted_net(ob, om, seed, w):
    """A random network whose standardisation is fitted to the 17-moment
    data of structure w itself (so that its orbitals are in range)."""
    m = oracle_model(w.model)
    nbr = ob.neighbors(w.pos, w.cell, w.pbc, m.rc)
    H = ob.blocks(m, w.pos, w.cell, nbr)
    mu17 = ob.moments(nbr, H, np.zeros((len(w.pos), 5)), 17).reshape(-1, 17)
    x = om.features(mu17[:, :9])[0]
    t, mask = om.targets(mu17)
    q = om.fit_normalisation(x, t, mask)
    # widen the range so that displaced structures stay inside it
    xm, xs, lo, hi, ym, ys = om.unpack_norm(q)
    q = np.concatenate([xm, xs, lo - 0.5 * (hi - lo) - 1e-3, hi + 0.5 * (hi - lo) + 1e-3, ym, ys])
    p = I.mlp_init_params(seed, 0.3)
    return om.Net(p, q)


def test_learned_energy_forces_by_central_differences(ob, om):
    w = I.small_bcc(2, 2, 2, 0.08, 22)
    net = _fitted_net(ob, om, 23, w)
    st = oracle_settings(w.run)
    st.terminator, st.net = "mlp", net
    m = oracle_model(w.model)
    res = ob.evaluate(m, st, w.pos, w.cell, w.pbc)
    assert res["learned"].all()
    plain = ob.evaluate(m, oracle_settings(w.run), w.pos, w.cell, w.pbc, want_forces=False)
    assert abs(res["e_total"] - plain["e_total"]) > 1e-4  # the network changes the energy
    h = 1e-4
    for (i, c) in [(0, 0), (5, 2), (11, 1)]:
        p, q = w.pos.copy(), w.pos.copy()
        p[i, c] += h
        q[i, c] -= h
        ep = ob.evaluate(m, st, p, w.cell, w.pbc, want_forces=False)
        eq = ob.evaluate(m, st, q, w.cell, w.pbc, want_forces=False)
        assert ep["learned"].all() and eq["learned"].all()
        fd = -(ep["e_total"] - eq["e_total"]) / (2 * h)
        assert abs(res["forces"][i, c] - fd) < 1e-7 + 1e-6 * abs(fd), (i, c, res["forces"][i, c], fd)


def test_fallback_outside_training_range_is_constant_terminator(ob, om):
    w = I.small_bcc(2, 2, 2, 0.08, 24)
    net = _fitted_net(ob, om, 25, w)
    xm, xs, lo, hi, ym, ys = om.unpack_norm(net.norm)
    net.norm = np.concatenate([xm, xs, lo + 1e3, hi + 2e3, ym, ys])  # nothing is in range
    st = oracle_settings(w.run)
    st.terminator, st.net = "mlp", net
    m = oracle_model(w.model)
    res = ob.evaluate(m, st, w.pos, w.cell, w.pbc, want_forces=False)
    ref = ob.evaluate(m, oracle_settings(w.run), w.pos, w.cell, w.pbc, want_forces=False)
    assert not res["learned"].any()
    assert abs(res["e_total"] - ref["e_total"]) < 1e-10 * len(w.pos)
