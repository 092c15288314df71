"""FP64 oracle of the learned terminator: a small MLP that continues the
recursion chain of a 9-moment run.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper closes the recursion chain with a constant terminator (a_n = a_inf,
b_n = b_inf beyond the computed levels, Eq. abinf, with a_inf / b_inf from the
Gershgorin band edges, Eq. gershogorin).  The learned terminator keeps that
form but predicts, from the first 9 moments of an orbital, the next four
levels of its chain and the band centre / width that a 17-moment run would
give; the constant terminator then starts after level 8.

Readings taken here (the paper describes no such network):
  * inputs x (18): (a_k - a_inf)/b_inf for k = 0..3, b_k/b_inf for k = 1..4,
    a_inf, b_inf (eV), mu-hat_1 .. mu-hat_8 (Eq. sigma_i normalisation), all
    with the 9-moment Gershgorin a_inf, b_inf;
  * outputs y (10): (a*_inf - a_inf)/b_inf, b*_inf/b_inf, (a_k - a_inf)/b_inf
    for k = 4..7 and b_k/b_inf for k = 5..8, where a*_inf, b*_inf and
    a_4..a_7, b_5..b_8 belong to the 17-moment chain of the same orbital;
  * network 18 -> 128 -> 128 -> 10, GELU (x Phi(x), the exact form), on
    inputs and targets standardised by the training set's mean and standard
    deviation; loss: mean squared error over the standardised targets of the
    orbitals whose 17-moment chain has all 8 levels;
  * inference rounds the three weight matrices to bfloat16 (round to
    nearest even); biases and the standardisation stay FP32 values and the
    activations are computed at full precision, so the energy stays a smooth
    function of the moments and the forces are its exact derivative;
  * fallback to the plain constant terminator of the 9-moment chain when
    the 9-moment chain is truncated, an input lies outside the training
    range (widened by 5 % of its span on each side), a predicted b_k or
    b*_inf is not above the band-width floor, or a value is not finite.

Parity: every function here is pinned by tests/test_oracle_mlp.py (closed
forms of the normal distribution, torch's float64 autograd and Adam as
independent implementations, central differences, the semicircle chain, and
the exact-target identity with the 17-moment expansion).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.special import ndtr

from . import bop as ob

N_IN, N_H, N_OUT = 18, 128, 10
K_BASE = 4           # levels of the 9-moment chain (a_0..a_3, b_1..b_4)
K_EXT = 8            # levels of the continued chain (a_0..a_7, b_1..b_8)
RANGE_MARGIN = 0.05  # training range widened by this fraction of its span
STD_FLOOR = 1e-6

# flat parameter layout: W1 [128][18], b1 [128], W2 [128][128], b2 [128], W3 [10][128], b3 [10]
_SHAPES = [(N_H, N_IN), (N_H,), (N_H, N_H), (N_H,), (N_OUT, N_H), (N_OUT,)]
N_PARAM = sum(int(np.prod(s)) for s in _SHAPES)
# normalisation layout: x_mean [18], x_std [18], x_lo [18], x_hi [18], y_mean [10], y_std [10]
N_NORM = 4 * N_IN + 2 * N_OUT


def unpack(p):
    out, o = [], 0
    for s in _SHAPES:
        k = int(np.prod(s))
        out.append(p[o:o + k].reshape(s))
        o += k
    return out


def unpack_norm(q):
    q = np.asarray(q, np.float64)
    return (q[0:18], q[18:36], q[36:54], q[54:72], q[72:82], q[82:92])


# ---------------------------------------------------------------- GELU

def _is_c(x):
    return np.iscomplexobj(x)


def gelu(x):
    """GELU(x) = x Phi(x), Phi the standard normal CDF.  For a complex
    argument (complex-step differentiation) the first-order expansion
    f(re) + i im f'(re) is returned, which is all the complex step uses."""
    if _is_c(x):
        r, i = np.real(x), np.imag(x)
        return gelu(r) + 1j * i * gelu_prime(r)
    return x * ndtr(x)


def gelu_prime(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    if _is_c(x):
        r, i = np.real(x), np.imag(x)
        return gelu_prime(r) + 1j * i * gelu_second(r)
    return ndtr(x) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def gelu_second(x):
    """d2/dx2 [x Phi(x)] = phi(x) (2 - x^2)."""
    return np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi) * (2.0 - x * x)


# ---------------------------------------------------------------- network

def forward(params, xs):
    """Network on standardised inputs xs [B, 18]; returns the pre-activations
    and activations of both hidden layers and the standardised output."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    z1 = xs @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    y = h2 @ W3.T + b3
    return z1, h1, z2, h2, y


def loss_and_grad(params, xs, ts, mask):
    """L = sum_b mask_b sum_j (y_bj - t_bj)^2 / (10 sum_b mask_b) and its
    gradient with respect to the flat parameters (reverse mode written out
    layer by layer)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    z1, h1, z2, h2, y = forward(params, xs)
    m = np.asarray(mask, np.float64)
    den = N_OUT * max(float(m.sum()), 1.0)
    r = (y - ts) * m[:, None]
    loss = float(np.sum(r * r) / den)
    dy = 2.0 * r / den
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dz2 = (dy @ W3) * gelu_prime(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * gelu_prime(z1)
    gW1 = dz1.T @ xs
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def input_gradient(params, xs, ybar):
    """x-bar = (dy/dxs)^T ybar for every row (the reverse of ``forward``)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    z1, h1, z2, h2, _ = forward(params, xs)
    dz2 = (ybar @ W3) * gelu_prime(z2)
    dz1 = (dz2 @ W2) * gelu_prime(z1)
    return dz1 @ W1


@dataclass
class AdamState:
    m: np.ndarray
    v: np.ndarray
    t: int = 0


def adam(params, grad, st: AdamState, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, bias-corrected moments)."""
    st.t += 1
    st.m = beta1 * st.m + (1.0 - beta1) * grad
    st.v = beta2 * st.v + (1.0 - beta2) * grad * grad
    mh = st.m / (1.0 - beta1 ** st.t)
    vh = st.v / (1.0 - beta2 ** st.t)
    return params - lr * mh / (np.sqrt(vh) + eps)


def bf16_round(x):
    """Round FP32 values to the nearest bfloat16 (ties to even), returned as
    float64: keep the top 16 bits of the IEEE single after adding half an
    ulp of bfloat16 plus the parity of the kept part."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def inference_params(params):
    """The deployed network: weights rounded to bfloat16, biases FP32."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(params, np.float64))
    f32 = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    return np.concatenate([bf16_round(W1).ravel(), f32(b1), bf16_round(W2).ravel(), f32(b2),
                           bf16_round(W3).ravel(), f32(b3)])


@dataclass
class Net:
    params: np.ndarray   # FP32 master values (float64 array)
    norm: np.ndarray     # [N_NORM] standardisation and training range


def fit_normalisation(x, t, mask) -> np.ndarray:
    """Mean, population standard deviation (floored) and widened range of
    the inputs, mean and standard deviation of the targets, over the rows
    with mask = 1; returned as FP32 values in the layout of ``unpack_norm``."""
    sel = np.asarray(mask) > 0
    xv, tv = np.asarray(x, np.float64)[sel], np.asarray(t, np.float64)[sel]
    xm, xs = xv.mean(axis=0), np.maximum(xv.std(axis=0), STD_FLOOR)
    lo, hi = xv.min(axis=0), xv.max(axis=0)
    span = hi - lo
    tm, ts = tv.mean(axis=0), np.maximum(tv.std(axis=0), STD_FLOOR)
    q = np.concatenate([xm, xs, lo - RANGE_MARGIN * span, hi + RANGE_MARGIN * span, tm, ts])
    return q.astype(np.float32).astype(np.float64)


def predict(net: Net, x):
    """Raw inputs [M, 18] -> raw outputs [M, 10] through the deployed
    (bfloat16-weight) network; also returns whether each row is inside the
    training range."""
    xm, xs, lo, hi, ym, ys = unpack_norm(net.norm)
    xr = np.real(x)
    inside = np.all((xr >= lo) & (xr <= hi), axis=1)
    _, _, _, _, y = forward(inference_params(net.params), (x - xm) / xs)
    return ym + ys * y, inside


# ---------------------------------------------------------------- chain data

def features(mu9):
    """Inputs of the network from the first 9 moments of each orbital.
    Returns (x [M, 18], a [M, 4], b [M, 5], nlev [M], a_inf [M], b_inf [M])."""
    mu9 = np.asarray(mu9)[:, :2 * K_BASE + 1]
    a, b, nlev = ob.recursion_coefficients(mu9)
    ai, bi = ob.gershgorin(a, b, nlev)
    mh = ob.normalised_moments(mu9, ai, bi)
    x = np.concatenate([(a - ai[:, None]) / bi[:, None], b[:, 1:] / bi[:, None],
                        ai[:, None], bi[:, None], mh[:, 1:]], axis=1)
    return x, a, b, nlev, ai, bi


def targets(mu17):
    """Targets of the network from the 17 moments of each orbital, relative
    to the 9-moment Gershgorin centre and width.  Returns (t [M, 10],
    mask [M]: 1 where the 17-moment chain has all 8 levels)."""
    mu17 = np.asarray(mu17, np.float64)
    a, b, nlev = ob.recursion_coefficients(mu17)
    a17, b17 = ob.gershgorin(a, b, nlev)
    a9, b9 = ob.gershgorin(a[:, :K_BASE], b[:, :K_BASE + 1], np.minimum(nlev, K_BASE))
    t = np.concatenate([((a17 - a9) / b9)[:, None], (b17 / b9)[:, None],
                        (a[:, K_BASE:] - a9[:, None]) / b9[:, None],
                        b[:, K_BASE + 1:] / b9[:, None]], axis=1)
    return t, (nlev == K_EXT).astype(np.float64)


def extend_chain(a, b, nlev, ai, bi, y, inside):
    """The continued chain of every orbital: levels 0..3 computed, 4..7 and
    the terminator predicted (y raw), or the plain 9-moment chain where the
    fallback applies.  Returns (a8 [M, 8], b9 [M, 9], nlev8 [M], a_inf,
    b_inf, learned [M] bool)."""
    M = a.shape[0]
    dt = np.result_type(a, b, ai, bi, y)
    a_star = ai + bi * y[:, 0]
    b_star = bi * y[:, 1]
    a_ext = ai[:, None] + bi[:, None] * y[:, 2:6]
    b_ext = bi[:, None] * y[:, 6:10]
    yr = np.real(y)
    ok = (nlev == K_BASE) & inside & np.all(np.isfinite(yr), axis=1)
    ok &= np.all(np.real(b_ext) > ob.B_INF_MIN, axis=1) & (np.real(b_star) > ob.B_INF_MIN)
    a8 = np.zeros((M, K_EXT), dt)
    b9 = np.zeros((M, K_EXT + 1), dt)
    a8[:, :K_BASE] = a
    b9[:, :K_BASE + 1] = b
    a8[:, K_BASE:] = np.where(ok[:, None], a_ext, 0.0)
    b9[:, K_BASE + 1:] = np.where(ok[:, None], b_ext, 0.0)
    nl = np.where(ok, K_EXT, nlev)
    return a8, b9, nl, np.where(ok, a_star, ai), np.where(ok, b_star, bi), ok


def learned_stage(mu9, net: Net, n_exp: int) -> ob.Expansion:
    """Moments -> features -> network -> continued chain -> sigma_m by the
    chain recursion of Eq. aexp (all m) -> g_m sigma_m.  The Expansion's a,
    b, nlev are those of the continued chain; ``learned`` marks the orbitals
    that did not fall back."""
    x, a, b, nlev, ai, bi = features(mu9)
    y, inside = predict(net, x)
    a8, b9, nl, a_inf, b_inf, ok = extend_chain(a, b, nlev, ai, bi, y, inside)
    sig = ob.zeta_sigma(a8, b9, nl, a_inf, b_inf, n_exp)
    g = ob.jackson(n_exp)
    ex = ob.Expansion(a8, b9, nl, a_inf, b_inf, sig, sig * g[None, :])
    ex.learned = ok
    return ex


def exact_chain_stage(mu9, t, n_exp: int) -> ob.Expansion:
    """The continued chain built from given targets t (e.g. those of the
    17-moment chain) instead of the network, with no range test."""
    x, a, b, nlev, ai, bi = features(mu9)
    a8, b9, nl, a_inf, b_inf, ok = extend_chain(a, b, nlev, ai, bi, t, np.ones(len(ai), bool))
    sig = ob.zeta_sigma(a8, b9, nl, a_inf, b_inf, n_exp)
    g = ob.jackson(n_exp)
    return ob.Expansion(a8, b9, nl, a_inf, b_inf, sig, sig * g[None, :])
