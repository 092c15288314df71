"""FP64 oracle of the analytic-BOP hot path, written from arXiv:1803.07491.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The structural part
(neighbours, Slater-Koster blocks, clusters, moments and their reverse sweep)
is plain C in ``bop_oracle.c``; the per-orbital scalar stages below are
numpy, written so that every function also accepts complex input: the
weights w_n = dU/dmu_n are taken by complex-step differentiation of the
scalar stage, which is exact to rounding and independent of any hand-written
chain rule.

Readings of the paper taken here (where the text is silent, garbled or
inconsistent):
  * n moments means mu_0 .. mu_{n-1}; n is odd, K = (n-1)/2 hops.
  * the phase is eps = +cos(phi) (band bottom at phi = pi); Eq. chi and
    Eq. Fermi-phase are only consistent with that sign.
  * gamma_0 in the bond energy is (E_ialpha - a_inf)/b_inf.
  * the DOS sums run over m = 0 .. n_exp with g_0 = 1.
  * Jackson kernel with N = n_exp; g_m = g^J_{m+1}/g^J_1.
  * Gershgorin over the computed levels n = 0 .. K'-1, b_0 = 0.
  * b_inf is floored at B_INF_MIN so that an isolated atom (zero band width)
    gives a narrow band instead of a division by zero.
  * the recursion is truncated where b_{n+1}^2 <= TRUNC_REL * (mu_2 - mu_1^2).
  * local charge neutrality acts per atom (one shift per atom).
  * the SCF update is either linear mixing of the DOS-preconditioned
    residual or Anderson (type-II Broyden) mixing of it; both reach the
    same self-consistent state.
  * the variational SCF (Eq. BOP_SCF) shifts one onsite level per atom and
    drives sum_alpha (Theta~_ii - N_i) = dU_B/d delta_i to zero, with
    U_B = U_bond + sum_i J_ii q_i^2 / 2 (one species: U_prom and the
    electronegativity term sum to E^0 sum_i q_i = 0 at fixed electron count).
  * non-collinear magnetism fixes one moment direction s_i per atom; the
    onsite matrix is (E_up + E_dn)/2 + (E_dn - E_up)/2 s_i.sigma, the lower
    level E_up belonging to the spin antiparallel to s_i (the convention
    under which the paper's torque expression and its global weights hold
    with their printed signs); the local channel moments Tr(P_nu M_n) take
    the place of the collinear spin channels; torques t_i = dU/ds_i x s_i
    at fixed magnitudes.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bop_oracle.c")
_SO = os.path.join(_HERE, "_build", platform.machine(), "liborc.so")
_LIB = None

B_INF_MIN = 1e-3      # eV, floor of the band-width estimate
TRUNC_REL = 1e-10     # relative threshold of the recursion truncation
CS_H = 1e-30          # complex step


def build(force: bool = False) -> str:
    """Compile bop_oracle.c into oracle/_build/liborc.so (gcc, no FMA)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(build())
        L = _LIB
        L.orc_neighbors.restype = ctypes.c_long
        L.orc_cluster.restype = ctypes.c_int
        L.orc_moments.restype = ctypes.c_int
        L.orc_moments_adjoint.restype = ctypes.c_int
        L.orc_moments_nc.restype = ctypes.c_int
        L.orc_moments_nc_adjoint.restype = ctypes.c_int
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class _CModel(ctypes.Structure):
    _fields_ = [("norb", ctypes.c_int), ("r0", ctypes.c_double), ("lam", ctypes.c_double),
                ("rc", ctypes.c_double), ("dc", ctypes.c_double), ("b0", ctypes.c_double * 5)]


@dataclass
class Model:
    """Orthogonal two-centre TB model of one element (Eq. Hij, Eq. cutoff).

    beta_x(r) = b0[x] * exp(-lam (r - r0)) * fcut(r); b0 = (ss sigma,) for s,
    (dd sigma, dd pi, dd delta) for d, or (dd sigma, dd pi, dd delta,
    ss sigma, sd sigma) for sd (norb 6, s first), in eV at r0 (Angstrom).
    onsite_s: the reference level of the s orbital of an sd model (the d
    orbitals take onsite0)."""
    norb: int
    b0: tuple
    r0: float
    lam: float
    rc: float
    dc: float
    onsite0: float = 0.0
    rep_A: float = 0.0    # repulsive energy U_rep (Eq. U_B) as a pair form, see pair_repulsion
    rep_p: float = 0.0
    onsite_s: float = 0.0

    def c(self) -> _CModel:
        b = list(self.b0) + [0.0] * (5 - len(self.b0))
        return _CModel(self.norb, self.r0, self.lam, self.rc, self.dc, (ctypes.c_double * 5)(*b))


@dataclass
class Settings:
    """Run settings: moments, expansion length, spin, electron count, SCF."""
    n_e: float                 # electrons per atom, summed over spin
    n_mom: int = 9
    n_exp: int = 200
    n_spin: int = 1
    scf: str = "none"          # none | lcn | stoner | variational
    eta: float = 0.5           # LCN mixing
    scf_tol: float = 1e-9      # max |N_i - N_i^0| (and |dm| for Stoner: scf_tol*10)
    scf_max_it: int = 200
    stoner_I: float = 0.0
    m_mix: float = 0.3
    m0: float = 2.0
    dos_floor: float = 0.1     # states/eV, LCN preconditioner floor
    mixer: str = "linear"      # linear | anderson (type-II Broyden, "SCF" of the paper)
    mix_history: int = 6
    terminator: str = "constant"  # constant | mlp (learned continuation, oracle/mlp.py)
    net: object = None            # mlp.Net for terminator = "mlp"
    scf_response: bool = True     # forces include the response of the SCF onsite levels
    bandwidth: object = None      # Bandwidth (None: Gershgorin)
    J_ii: float = 0.0             # variational SCF: onsite charging J_ii of Eq. TB-Uion (eV / e^2)
    r_path: float = 0.0           # path-radius cut (A), 0 = none ("Performance", item (iii))
    noncollinear: bool = False    # one moment direction per atom (section "Magnetism"), n_spin = 2


@dataclass
class Neighbors:
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [E]
    img: np.ndarray      # int8  [E, 3]
    # path-radius cut ("Performance", item (iii)): (pos, cell, r_path) or None
    path: tuple | None = None

    def with_path_radius(self, pos, cell, r_path: float) -> "Neighbors":
        """The same list with the path-radius cut r_path (<= 0: none)."""
        if r_path <= 0:
            return Neighbors(self.row_ptr, self.col, self.img)
        return Neighbors(self.row_ptr, self.col, self.img,
                         (np.ascontiguousarray(pos, dtype=np.float64), np.ascontiguousarray(cell, dtype=np.float64),
                          float(r_path)))

    def _path_args(self):
        if self.path is None:
            return None, None, ctypes.c_double(0.0)
        pos, cell, r = self.path
        return _p(pos), _p(cell), ctypes.c_double(r)

    @property
    def n_edges(self):
        return int(self.row_ptr[-1])


# ---------------------------------------------------------------- structure

def neighbors(pos, cell, pbc, rcut) -> Neighbors:
    """Short-range neighbour list by brute force ("Initialisation": linked
    cells only make it O(N)); directed CSR sorted by (j, sx, sy, sz)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    pbc = np.ascontiguousarray(pbc, dtype=np.int32)
    n = len(pos)
    cap = max(64, 32 * n)
    while True:
        row = np.zeros(n + 1, np.int64)
        col = np.zeros(cap, np.int32)
        img = np.zeros((cap, 3), np.int8)
        ne = _lib().orc_neighbors(n, _p(pos), _p(cell), _p(pbc), ctypes.c_double(rcut),
                                  ctypes.c_long(cap), _p(row), _p(col), _p(img))
        if ne >= 0:
            return Neighbors(row, col[:ne].copy(), img[:ne].copy())
        cap = -ne


def sk_block(model: Model, d) -> np.ndarray:
    """Block <i b|H|j g> for bond vector d = r_j - r_i (Eq. Hij rotated by
    Eq. Hij_rot, via the Slater-Koster direction-cosine table)."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    B = np.zeros(model.norb * model.norb)
    _lib().orc_block(ctypes.byref(model.c()), _p(d), _p(B))
    return B.reshape(model.norb, model.norb)


def blocks(model: Model, pos, cell, nbr: Neighbors) -> np.ndarray:
    """H_e for every directed edge: [E, norb, norb]."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    H = np.zeros((nbr.n_edges, model.norb, model.norb))
    _lib().orc_blocks(len(pos), _p(pos), _p(cell), _p(nbr.row_ptr), _p(nbr.col), _p(nbr.img),
                      ctypes.byref(model.c()), _p(H))
    return H


def edge_vectors(pos, cell, nbr: Neighbors) -> np.ndarray:
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    d = np.zeros((nbr.n_edges, 3))
    _lib().orc_edge_vectors(len(pos), _p(pos), _p(cell), _p(nbr.row_ptr), _p(nbr.col),
                            _p(nbr.img), _p(d))
    return d


def cluster(i: int, K: int, nbr: Neighbors, max_sites: int = 200000):
    """Hop levels of (atom, image) sites around atom i (support of the
    self-returning paths, Eq. momDOS).  Returns (site_atom, site_img,
    level_end) in canonical order: level, atom, image."""
    atom = np.zeros(max_sites, np.int32)
    im = np.zeros((max_sites, 3), np.int8)
    lev = np.zeros(K + 1, np.int32)
    ns = _lib().orc_cluster(int(i), int(K), _p(nbr.row_ptr), _p(nbr.col), _p(nbr.img), *nbr._path_args(),
                            int(max_sites), _p(atom), _p(im), _p(lev))
    if ns < 0:
        raise ValueError("image index overflow in cluster")
    if ns > max_sites:
        return cluster(i, K, nbr, ns)
    return atom[:ns].copy(), im[:ns].copy(), lev


def moments(nbr: Neighbors, H, onsite, n_mom: int, sel=None) -> np.ndarray:
    """mu_n(i alpha) = <i alpha|H^n|i alpha>, n = 0..n_mom-1 (Eq. momDOS),
    for one spin channel.  onsite: [n, norb].  Returns [nsel, norb, n_mom]."""
    assert n_mom % 2 == 1 and n_mom >= 3
    onsite = np.ascontiguousarray(onsite, dtype=np.float64)
    n, norb = onsite.shape
    sel = np.arange(n, dtype=np.int32) if sel is None else np.ascontiguousarray(sel, np.int32)
    H = np.ascontiguousarray(H, dtype=np.float64)
    mu = np.zeros((len(sel), norb, n_mom))
    st = _lib().orc_moments(len(sel), _p(sel), n_mom, norb, _p(nbr.row_ptr), _p(nbr.col),
                            _p(nbr.img), *nbr._path_args(), _p(H), _p(onsite), _p(mu))
    if st != 0:
        raise ValueError("image index overflow in cluster")
    return mu


def moments_adjoint(nbr: Neighbors, H, onsite, w, sel=None):
    """Reverse sweep of ``moments``: with w = dU/dmu [nsel, norb, n_mom]
    returns (Hbar [E, norb, norb] = dU/dH_e, Ebar [n, norb] = dU/dE)."""
    onsite = np.ascontiguousarray(onsite, dtype=np.float64)
    n, norb = onsite.shape
    sel = np.arange(n, dtype=np.int32) if sel is None else np.ascontiguousarray(sel, np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n_mom = w.shape[-1]
    Hbar = np.zeros((nbr.n_edges, norb, norb))
    Ebar = np.zeros((n, norb))
    st = _lib().orc_moments_adjoint(len(sel), _p(sel), n_mom, norb, _p(nbr.row_ptr),
                                    _p(nbr.col), _p(nbr.img), *nbr._path_args(),
                                    _p(np.ascontiguousarray(H, dtype=np.float64)),
                                    _p(onsite), _p(w), _p(Hbar), _p(Ebar))
    if st != 0:
        raise ValueError("image index overflow in cluster")
    return Hbar, Ebar


def moments_nc(nbr: Neighbors, H, onsite2, sdir, n_mom: int, sel=None) -> np.ndarray:
    """Global 2x2 spin moments M_n[a][b] = <i alpha, a|H^n|i alpha, b> of
    non-collinear magnetism (section "Magnetism", Eq. onsite_CM): hopping
    H_e x 1, onsite matrix (E_up + E_dn)/2 + (E_dn - E_up)/2 s_i . sigma,
    spin basis along z.  onsite2: [2, n, norb] (E_up, E_dn), sdir: [n, 3]
    unit moment directions.  Returns [nsel, norb, n_mom, 2, 2] complex."""
    assert n_mom % 2 == 1 and n_mom >= 3
    onsite2 = np.ascontiguousarray(onsite2, dtype=np.float64)
    _, n, norb = onsite2.shape
    sdir = np.ascontiguousarray(sdir, dtype=np.float64)
    sel = np.arange(n, dtype=np.int32) if sel is None else np.ascontiguousarray(sel, np.int32)
    M = np.zeros((len(sel), norb, n_mom, 2, 2), np.complex128)
    st = _lib().orc_moments_nc(len(sel), _p(sel), n, n_mom, norb, _p(nbr.row_ptr), _p(nbr.col), _p(nbr.img),
                               *nbr._path_args(), _p(np.ascontiguousarray(H, dtype=np.float64)), _p(onsite2),
                               _p(sdir), _p(M))
    if st != 0:
        raise ValueError("image index overflow in cluster")
    return M


def moments_nc_adjoint(nbr: Neighbors, H, onsite2, sdir, W, sel=None):
    """Reverse sweep of ``moments_nc`` for L = sum_n Re Tr(W_n M_n), W
    [nsel, norb, n_mom, 2, 2] Hermitian: returns (Hbar [E, norb, norb] =
    dL/dH_e, Obar [n, norb, 4] = dL/d(Ebar, h_x, h_y, h_z) of every onsite
    matrix Ebar + h . sigma)."""
    onsite2 = np.ascontiguousarray(onsite2, dtype=np.float64)
    _, n, norb = onsite2.shape
    sel = np.arange(n, dtype=np.int32) if sel is None else np.ascontiguousarray(sel, np.int32)
    W = np.ascontiguousarray(W, dtype=np.complex128)
    n_mom = W.shape[2]
    Hbar = np.zeros((nbr.n_edges, norb, norb))
    Obar = np.zeros((n, norb, 4))
    st = _lib().orc_moments_nc_adjoint(len(sel), _p(sel), n, n_mom, norb, _p(nbr.row_ptr), _p(nbr.col),
                                       _p(nbr.img), *nbr._path_args(),
                                       _p(np.ascontiguousarray(H, dtype=np.float64)), _p(onsite2),
                                       _p(np.ascontiguousarray(sdir, dtype=np.float64)), _p(W), _p(Hbar), _p(Obar))
    if st != 0:
        raise ValueError("image index overflow in cluster")
    return Hbar, Obar


def pauli_vector(M) -> np.ndarray:
    """Tr(sigma M) of 2x2 matrices [..., 2, 2] -> [..., 3] (real part)."""
    vx = M[..., 0, 1] + M[..., 1, 0]
    vy = 1j * (M[..., 0, 1] - M[..., 1, 0])
    vz = M[..., 0, 0] - M[..., 1, 1]
    return np.real(np.stack([vx, vy, vz], axis=-1))


def local_moments(M, sdir) -> np.ndarray:
    """Moments of the local up / down channels (Eq. onsite-noncollinear),
    mu_nu = Tr(P_nu M) with the projectors P_up = (1 - s.sigma)/2 (spin
    antiparallel to the moment direction s, the lower level) and
    P_dn = (1 + s.sigma)/2.  M [n, norb, n_mom, 2, 2] -> [2, n, norb, n_mom]."""
    tr = np.real(M[..., 0, 0] + M[..., 1, 1])
    sv = np.einsum("iamx,ix->iam", pauli_vector(M), sdir)
    return np.stack([0.5 * (tr - sv), 0.5 * (tr + sv)])


def global_weights(w, sdir) -> np.ndarray:
    """Weights in the global spin frame from the local ones (section
    "Torques"): W = (w_up + w_dn)/2 1 + (w_dn - w_up)/2 s.sigma.
    w [2, n, norb, n_mom] -> [n, norb, n_mom, 2, 2] complex."""
    a = 0.5 * (w[0] + w[1])
    c = 0.5 * (w[1] - w[0])
    sx, sy, sz = (sdir[:, x][:, None, None] for x in range(3))
    W = np.zeros(a.shape + (2, 2), np.complex128)
    W[..., 0, 0] = a + c * sz
    W[..., 1, 1] = a - c * sz
    W[..., 0, 1] = c * (sx - 1j * sy)
    W[..., 1, 0] = c * (sx + 1j * sy)
    return W


def bond_gradient(model: Model, pos, cell, nbr: Neighbors, Hbar) -> np.ndarray:
    """g_e = sum Hbar_e * dH_e/dd_e for every directed edge, [E, 3]."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    g = np.zeros((nbr.n_edges, 3))
    _lib().orc_bond_gradient(len(pos), _p(pos), _p(cell), _p(nbr.row_ptr), _p(nbr.col),
                             _p(nbr.img), ctypes.byref(model.c()),
                             _p(np.ascontiguousarray(Hbar, dtype=np.float64)), _p(g))
    return g


# ---------------------------------------------------------------- scalar stage

def pair_repulsion(model: Model, r):
    """U_rep of one bond: rep_A exp(-rep_p (r - r0)) fcut(r), with the
    cosine taper of Eq. cutoff (the paper leaves U_rep to empirical
    functions).  Returns (phi, dphi/dr)."""
    r = np.asarray(r, dtype=np.float64)
    e = model.rep_A * np.exp(-model.rep_p * (r - model.r0))
    de = -model.rep_p * e
    lo = model.rc - model.dc
    x = np.clip((r - lo) / model.dc, 0.0, 1.0)
    f = np.where(r < lo, 1.0, np.where(r > model.rc, 0.0, 0.5 * (np.cos(np.pi * x) + 1.0)))
    df = np.where((r < lo) | (r > model.rc), 0.0, -0.5 * np.pi / model.dc * np.sin(np.pi * x))
    return e * f, de * f + e * df


def _re(x):
    return np.real(x)


def recursion_coefficients(mu):
    """Recursion coefficients from moments (Eqs. momtoa, momtob and the
    c_j^n recursion).  mu: [M, n_mom].  With K' = (n_mom-1)/2 returns
    a [M, K'] (a_0..a_{K'-1}), b [M, K'+1] (b_0 = 0, b_1..b_{K'}) and
    nlev [M] = number of a's computed (< K' where the chain was truncated,
    in which case b[nlev] = 0)."""
    mu = np.asarray(mu)
    M, n_mom = mu.shape
    Kp = (n_mom - 1) // 2
    dt = mu.dtype
    a = np.zeros((M, Kp), dt)
    b = np.zeros((M, Kp + 1), dt)
    nlev = np.full(M, Kp, np.int64)
    alive = np.ones(M, bool)
    width = np.maximum(_re(mu[:, 2] - mu[:, 1] ** 2), 0.0)
    c_prev = np.zeros((M, Kp + 2), dt)
    c = np.zeros((M, Kp + 2), dt)
    c[:, 0] = 1.0
    for n in range(Kp):
        # a_n = sum_{j,l} c_j^n c_l^n mu_{j+l+1}
        an = np.zeros(M, dt)
        for j in range(n + 1):
            for l in range(n + 1):
                an = an + c[:, j] * c[:, l] * mu[:, j + l + 1]
        a[:, n] = np.where(alive, an, 0.0)
        # b_{n+1} c^{n+1} = c^n shifted - a_n c^n - b_n c^{n-1}
        d = np.zeros_like(c)
        d[:, 1:] = c[:, :-1]
        d = d - an[:, None] * c - b[:, n][:, None] * c_prev
        b2 = np.zeros(M, dt)
        for j in range(n + 2):
            for l in range(n + 2):
                b2 = b2 + d[:, j] * d[:, l] * mu[:, j + l]
        trunc = alive & (_re(b2) <= TRUNC_REL * width)
        nlev = np.where(trunc, n + 1, nlev)
        keep = alive & ~trunc
        bn1 = np.sqrt(np.where(keep, b2, 1.0))
        b[:, n + 1] = np.where(keep, bn1, 0.0)
        c_new = d / bn1[:, None]
        c_prev = np.where(keep[:, None], c, c_prev)
        c = np.where(keep[:, None], c_new, c)
        alive = keep
    return a, b, nlev


def gershgorin(a, b, nlev):
    """Band edges from Gershgorin's circle theorem, Eq. gershogorin, over the
    computed levels n < nlev: E_bot = min(a_n - b_n - b_{n+1}),
    E_top = max(a_n + b_n + b_{n+1}).  Returns (a_inf, b_inf) with
    A = (top+bot)/2, B = (top-bot)/4 (constant terminator, Eq. abinf)."""
    M, Kp = a.shape
    lo = np.zeros_like(a)
    hi = np.zeros_like(a)
    for n in range(Kp):
        lo[:, n] = a[:, n] - b[:, n] - b[:, n + 1]
        hi[:, n] = a[:, n] + b[:, n] + b[:, n + 1]
    valid = np.arange(Kp)[None, :] < nlev[:, None]
    ilo = np.argmin(np.where(valid, _re(lo), np.inf), axis=1)
    ihi = np.argmax(np.where(valid, _re(hi), -np.inf), axis=1)
    bot = lo[np.arange(M), ilo]
    top = hi[np.arange(M), ihi]
    a_inf = 0.5 * (top + bot)
    b_inf = 0.25 * (top - bot)
    b_inf = np.where(_re(b_inf) < B_INF_MIN, B_INF_MIN, b_inf)
    return a_inf, b_inf


BANDWIDTH_MODES = ("gershgorin", "lowest", "highest", "average", "average_centre", "minmax", "global",
                   "weighted")


@dataclass
class Bandwidth:
    """Choice of the band centre / width estimate ("Band-width estimates"
    (i)-(v), (vii), (viii)) or of the weighted-average terminator (Eq.
    weighted, parameter beta).  ga, gb: the global values of (viii)."""
    mode: str = "gershgorin"
    beta: float = 1.0
    ga: float = 0.0
    gb: float = 1.0


def _pick(x, idx):
    return x[np.arange(x.shape[0]), idx]


def band_estimate(a, b, nlev, bw: Bandwidth):
    """(a_inf, b_inf) = (A, B) for every orbital from its computed levels
    a_0 .. a_{L-1}, b_1 .. b_L (L = nlev), by the chosen estimate.
    Readings: (i) "lowest" takes a_0 and b_1 (the lowest computed of each;
    the printed a^(1) would skip the first computed a); (ii) "highest" takes
    a_{L-1} and b_L; (iii) "average" averages a_0..a_{L-1} and takes the root
    mean square of b_1..b_L; (iv) "average_centre" the same centre with b_L;
    (v) "minmax" (max a + min a)/2 and (max a - min a + 4 max b)/4; (viii)
    "global" (ga, gb) for every orbital; "weighted" the weighted averages of
    Eq. weighted with w_m = 1/(beta (m_max - m) + 1), m_max the highest
    computed index of each sequence (L-1 for a, L for b).  B is floored at
    B_INF_MIN as for Gershgorin (complex-step safe: max / min by real part)."""
    if bw.mode == "gershgorin":
        return gershgorin(a, b, nlev)
    M, Kp = a.shape
    L = np.asarray(nlev)
    dt = np.result_type(a, b)
    ka = np.arange(Kp)[None, :]
    kb = np.arange(Kp + 1)[None, :]
    va = ka < L[:, None]                  # computed a_n
    vb = (kb >= 1) & (kb <= L[:, None])   # computed b_n
    zero = np.zeros((), dt)
    if bw.mode == "lowest":
        A, B = a[:, 0], b[:, 1]
    elif bw.mode == "highest":
        A, B = _pick(a, L - 1), _pick(b, L)
    elif bw.mode in ("average", "average_centre"):
        A = np.sum(np.where(va, a, zero), axis=1) / L
        if bw.mode == "average":
            B = np.sqrt(np.sum(np.where(vb, b * b, zero), axis=1) / L)
        else:
            B = _pick(b, L)
    elif bw.mode == "minmax":
        ar = np.real(a)
        imax = np.argmax(np.where(va, ar, -np.inf), axis=1)
        imin = np.argmin(np.where(va, ar, np.inf), axis=1)
        ib = np.argmax(np.where(vb, np.real(b), -np.inf), axis=1)
        amax, amin, bmax = _pick(a, imax), _pick(a, imin), _pick(b, ib)
        A = 0.5 * (amax + amin)
        B = 0.25 * (amax - amin + 4.0 * bmax)
    elif bw.mode == "global":
        A = np.full(M, bw.ga, dt)
        B = np.full(M, bw.gb, dt)
    elif bw.mode == "weighted":
        with np.errstate(divide="ignore"):  # levels beyond L are masked out
            wa = np.where(va, 1.0 / (bw.beta * ((L[:, None] - 1) - ka) + 1.0), 0.0)
            wb = np.where(vb, 1.0 / (bw.beta * (L[:, None] - kb) + 1.0), 0.0)
        A = np.sum(wa * a, axis=1) / np.sum(wa, axis=1)
        B = np.sum(wb * b, axis=1) / np.sum(wb, axis=1)
    else:
        raise ValueError(bw.mode)
    B = np.where(np.real(B) < B_INF_MIN, B_INF_MIN, B)
    return A, B


def outside_band(sigma):
    """Per orbital: True if some |sigma_m| > m + 1.  sigma_m integrates
    U_m(x) against a density of unit weight (section "Chebyshev
    polynomials", Eq. sigma_i), and |U_m| <= m + 1 on [-1, 1], so the
    density then has weight outside the estimated band and the series grows
    with m instead of decaying."""
    m = np.arange(sigma.shape[1])
    return np.any(np.abs(np.real(sigma)) > (m + 1) * (1.0 + 1e-9), axis=1)


def normalised_moments(mu, a_inf, b_inf):
    """mu-hat_n = (2 b_inf)^-n sum_l C(n,l) (-a_inf)^l mu_{n-l}
    (Eq. sigma_i and the normalisation beneath it)."""
    M, n_mom = mu.shape
    out = np.zeros_like(mu, dtype=np.result_type(mu, a_inf, b_inf))
    for n in range(n_mom):
        acc = 0.0
        for l in range(n + 1):
            acc = acc + comb(n, l) * (-a_inf) ** l * mu[:, n - l]
        out[:, n] = acc / (2.0 * b_inf) ** n
    return out


def cheb_p(m_max: int) -> np.ndarray:
    """Coefficients p_mn of the Chebyshev polynomials of the second kind,
    P_m(eps) = sum_n p_mn eps^n (Eq. chebyshev), from
    p_{(m+1)n} = 2 p_{m(n-1)} - p_{(m-1)n}, P_0 = 1, P_1 = 2 eps."""
    p = np.zeros((m_max + 1, m_max + 1))
    p[0, 0] = 1.0
    if m_max >= 1:
        p[1, 1] = 2.0
    for m in range(1, m_max):
        for n in range(m + 2):
            p[m + 1, n] = (2.0 * p[m, n - 1] if n >= 1 else 0.0) - p[m - 1, n]
    return p


def sigma_from_moments(mu_hat):
    """sigma_m = sum_n p_mn mu-hat_n for m < n_mom (Eq. sigma_i)."""
    n_mom = mu_hat.shape[1]
    p = cheb_p(n_mom - 1)
    return mu_hat @ p.T


def zeta_sigma(a, b, nlev, a_inf, b_inf, n_exp: int):
    """sigma_m = zeta_0^(m), m = 0..n_exp, from the semi-infinite chain
    recursion zeta^(m+1)_k = 2[a^_k z_k + b^_k z_{k-1} + b^_{k+1} z_{k+1}]
    - zeta^(m-1)_k (Eq. aexp), with a^_k = (a_k - a_inf)/(2 b_inf),
    b^_k = b_k/(2 b_inf) on the computed levels and the constant
    terminator a_k = a_inf, b_k = b_inf (a^ = 0, b^ = 1/2) beyond them."""
    M, Kp = a.shape
    L = n_exp + 2
    dt = np.result_type(a, b, a_inf, b_inf)
    ah = np.zeros((M, L + 1), dt)
    bh = np.full((M, L + 2), 0.5, dt)
    bh[:, 0] = 0.0
    for k in range(Kp):
        on = k < nlev
        ah[:, k] = np.where(on, (a[:, k] - a_inf) / (2.0 * b_inf), 0.0)
    for k in range(1, Kp + 1):
        on = k <= nlev
        bh[:, k] = np.where(on, b[:, k] / (2.0 * b_inf), 0.5)
    sig = np.zeros((M, n_exp + 1), dt)
    z_prev = np.zeros((M, L + 1), dt)
    z = np.zeros((M, L + 1), dt)
    z[:, 0] = 1.0
    sig[:, 0] = 1.0
    for m in range(n_exp):
        hz = ah * z
        hz[:, 1:] = hz[:, 1:] + bh[:, 1:L + 1] * z[:, :-1]
        hz[:, :-1] = hz[:, :-1] + bh[:, 1:L + 1] * z[:, 1:]
        z_new = 2.0 * hz - z_prev
        z_prev, z = z, z_new
        sig[:, m + 1] = z[:, 0]
    return sig


def jackson(n_exp: int) -> np.ndarray:
    """Damping factors g_m = g^J_{m+1} / g^J_1, m = 0..n_exp, from the
    Jackson kernel Eq. Jackson with N = n_exp."""
    N = n_exp
    m = np.arange(N + 2, dtype=np.float64)
    x = np.pi / (N + 1)
    gJ = ((N - m + 1) * np.cos(m * x) + np.sin(m * x) / np.tan(x)) / (N + 1)
    return gJ[1:N + 2] / gJ[1]


def chi_hat(m_max: int, phi):
    """Response functions chi-hat_m(phi), m = 0..m_max (Eq. chi and the
    two special cases above it).  phi: [M].  Returns [M, m_max+1]."""
    phi = np.asarray(phi)
    out = np.zeros(phi.shape + (m_max + 1,), dtype=phi.dtype)
    if m_max >= 1:
        out[..., 1] = 1.0 - phi / np.pi + np.sin(2.0 * phi) / (2.0 * np.pi)
    for m in range(2, m_max + 1):
        out[..., m] = (np.sin((m + 1) * phi) / (m + 1) - np.sin((m - 1) * phi) / (m - 1)) / np.pi
    return out


def fermi_phase(E_F, a_inf, b_inf):
    """phi_F from cos(phi_F) = (E_F - a_inf)/(2 b_inf) (Eq. Fermi-phase),
    the cosine clamped to [-1, 1] (E_F below / above the band)."""
    x = (E_F - a_inf) / (2.0 * b_inf)
    xr = _re(x)
    x = np.where(xr > 1.0, 1.0, np.where(xr < -1.0, -1.0, x))
    return np.arccos(x)


def orbital_N_U(gsig, a_inf, b_inf, E_on, E_F):
    """Per-orbital, per-spin electron count and bond energy:
    N = sum_m g_m sigma_m chi_{m+1}(phi_F);
    U = b_inf sum_m g_m sigma_m [chi_{m+2} - gamma_0 chi_{m+1} + chi_m],
    gamma_0 = (E_ialpha - a_inf)/b_inf (bond energy of Eq. TB-Ubond in the
    closed form given with Eq. chi)."""
    n_exp = gsig.shape[1] - 1
    phi = fermi_phase(E_F, a_inf, b_inf)
    chi = chi_hat(n_exp + 2, phi)
    N = np.sum(gsig * chi[:, 1:n_exp + 2], axis=1)
    g0 = (E_on - a_inf) / b_inf
    U = b_inf * np.sum(gsig * (chi[:, 2:n_exp + 3] - g0[:, None] * chi[:, 1:n_exp + 2]
                               + chi[:, 0:n_exp + 1]), axis=1)
    return N, U


def dos_at(gsig, a_inf, b_inf, E):
    """Local DOS per orbital and spin at energy E (Eq. nialpha, divided by
    2 b_inf for the change of variable eps -> E); zero outside the band."""
    eps = (E - a_inf) / (2.0 * b_inf)
    inside = np.abs(eps) < 1.0
    e = np.where(inside, eps, 0.0)
    n_exp = gsig.shape[1] - 1
    Um1 = np.zeros_like(e)
    Um = np.ones_like(e)
    acc = gsig[:, 0] * Um
    for m in range(1, n_exp + 1):
        Up = 2.0 * e * Um - Um1
        Um1, Um = Um, Up
        acc = acc + gsig[:, m] * Um
    val = (2.0 / np.pi) * np.sqrt(1.0 - e * e) * acc / (2.0 * b_inf)
    return np.where(inside, val, 0.0)


@dataclass
class Expansion:
    a: np.ndarray
    b: np.ndarray
    nlev: np.ndarray
    a_inf: np.ndarray
    b_inf: np.ndarray
    sigma: np.ndarray
    gsig: np.ndarray


def scalar_stage(mu, n_exp: int, bw: Bandwidth | None = None) -> Expansion:
    """Moments -> (a, b) -> (a_inf, b_inf) (Gershgorin unless bw says
    otherwise) -> mu-hat -> sigma (Eq. sigma_i below n_mom, the zeta chain
    above) -> g_m sigma_m."""
    a, b, nlev = recursion_coefficients(mu)
    a_inf, b_inf = gershgorin(a, b, nlev) if bw is None else band_estimate(a, b, nlev, bw)
    n_mom = mu.shape[1]
    sig_mom = sigma_from_moments(normalised_moments(mu, a_inf, b_inf))
    sig = zeta_sigma(a, b, nlev, a_inf, b_inf, n_exp)
    sig[:, :n_mom] = sig_mom
    g = jackson(n_exp)
    return Expansion(a, b, nlev, a_inf, b_inf, sig, sig * g[None, :])


def fermi_bisect(ex: Expansion, spin_factor: float, target: float,
                 max_it: int = 100, tol: float = 1e-13):
    """Fermi level by bisection on the total electron count
    s * sum N_ialpha(E_F) = target ("DOS and Fermi energy").  The bracket is
    [min(a_inf - 2 b_inf) - 1e-3, max(a_inf + 2 b_inf) + 1e-3]; stops after
    max_it halvings or at a width below tol; returns the midpoint."""
    lo = float(np.min(ex.a_inf - 2.0 * ex.b_inf)) - 1e-3
    hi = float(np.max(ex.a_inf + 2.0 * ex.b_inf)) + 1e-3
    zero_on = np.zeros_like(ex.a_inf)
    it = 0
    for it in range(max_it):
        if hi - lo < tol:
            break
        mid = 0.5 * (lo + hi)
        N, _ = orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, zero_on, mid)
        f = spin_factor * float(np.sum(N)) - target
        if f == 0.0:
            return mid, it + 1
        if f < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi), it


def weights(mu, E_on, E_F, n_exp: int, spin_factor: float, stage=None):
    """w_n = dU_total/dmu_n per orbital (Eq. weights), including the
    response of E_F at fixed total electron number, by complex-step
    differentiation of the scalar stage.  Returns (w [M, n_mom],
    dU_dE [M] = direct derivative of s*U_ialpha w.r.t. its onsite level,
    dN_dmu [M, n_mom], dN_dEF [M], dU_dEF [M]).  ``stage`` (mu -> Expansion)
    replaces ``scalar_stage``, e.g. by the learned continuation of the chain."""
    if stage is None:
        stage = lambda m: scalar_stage(m, n_exp)  # noqa: E731
    M, n_mom = mu.shape
    dU = np.zeros((M, n_mom))
    dN = np.zeros((M, n_mom))
    for n in range(n_mom):
        mc = mu.astype(np.complex128)
        mc[:, n] += 1j * CS_H
        ex = stage(mc)
        N, U = orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, E_on.astype(np.complex128), E_F)
        dU[:, n] = np.imag(U) / CS_H
        dN[:, n] = np.imag(N) / CS_H
    ex = stage(mu)
    N, U = orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, E_on.astype(np.complex128),
                       E_F + 1j * CS_H)
    dU_dEF = np.imag(U) / CS_H
    dN_dEF = np.imag(N) / CS_H
    N, U = orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, E_on + 1j * CS_H, E_F)
    dU_dE = spin_factor * np.imag(U) / CS_H
    lam = np.sum(dU_dEF) / np.sum(dN_dEF)
    w = spin_factor * (dU - lam * dN)
    return w, dU_dE, dN, dN_dEF, dU_dEF, dU


def variational_gradient(st: Settings, nbr: Neighbors, H, onsite, mu_f, E_F, stage, s: float):
    """Gradient of the binding energy U_B = U_bond + sum_i J_ii q_i^2 / 2
    (Eqs. U_B, TB-Ubond, TB-Uion; q_i = s sum_alpha N_i alpha - n_e) with
    respect to the per-atom onsite shifts delta_i at fixed electron count:
    Delta_i = sum_alpha dU_B/dE_i alpha = sum_alpha (Theta~_i alpha i alpha -
    N_i alpha) of Eq. BOP_SCF, Theta~_ii the derivative of U_B through the
    moments (reverse sweep of the moments with the weights below) and -N the
    explicit derivative of U_bond's (E - E_i alpha) term (n_spin = 1).

    The weights are those of U_B with E_F following the electron count:
    w = s dU/dmu + s (J_ii q_i - Lambda) dN/dmu,
    Lambda = (dU_B/dE_F) / (dN_total/dE_F).  Returns (Delta [n], w
    [1, n, norb, n_mom], q [n])."""
    S, n, norb = onsite.shape
    n_mom = mu_f.shape[1]
    _, dU_dE, dN, dN_dEF, dU_dEF, dU = weights(mu_f, onsite.reshape(-1), E_F, st.n_exp, s, stage)
    ex = stage(mu_f)
    N, _ = orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, onsite.reshape(-1), E_F)
    q = s * N.reshape(n, norb).sum(axis=1) - st.n_e
    qo = np.repeat(q, norb)                            # q of each orbital's atom
    dUB_dEF = s * np.sum(dU_dEF) + st.J_ii * s * np.sum(qo * dN_dEF)
    Lam = dUB_dEF / (s * np.sum(dN_dEF))
    w = s * dU + (s * (st.J_ii * qo - Lam))[:, None] * dN
    _, Ebar = moments_adjoint(nbr, H, onsite[0], w.reshape(n, norb, n_mom))
    Delta = (Ebar + dU_dE.reshape(n, norb)).sum(axis=1)
    return Delta, w.reshape(1, n, norb, n_mom), q


# ---------------------------------------------------------------- driver

def evaluate(model: Model, st: Settings, pos, cell, pbc, want_forces: bool = True,
             delta0=None, m_init=None, spin_dir=None):
    """Energy (and forces, virial) of the analytic BOP for one structure.

    Flow of Fig. BOP-calculation: neighbours -> H -> [moments -> recursion ->
    terminator -> E_F -> N, U -> onsite update]* -> energy -> weights ->
    reverse sweep -> forces.  Forces are the exact derivative of the energy
    with E_F following the electron count.  With an SCF the forces are the
    total derivative of the self-consistent energy (``scf_response``, the
    default; see ``scf_response_weights``), otherwise the derivative at fixed
    onsite levels (the Hellmann-Feynman form of Eq. F_k).

    Non-collinear magnetism (``st.noncollinear``, section "Magnetism"):
    spin_dir [n, 3] fixes the direction of every atom's moment; the
    moments are the 2x2 spin moments of ``moments_nc`` projected on the
    local up / down channels, which then take the place of the two
    collinear spin channels (Stoner SCF of the magnitudes m_i, or fixed
    magnitudes m_init without an SCF).  The torques of Eq. torque,
    t_i = dU/ds_i x s_i, are returned with the forces."""
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    norb = model.norb
    S = st.n_spin
    s = 2.0 if S == 1 else 1.0
    nbr = neighbors(pos, cell, pbc, model.rc).with_path_radius(pos, cell, st.r_path)
    H = blocks(model, pos, cell, nbr)
    delta = np.zeros(n) if delta0 is None else np.array(delta0, np.float64)
    m = None
    nc = st.noncollinear
    if nc:
        assert S == 2 and st.scf in ("none", "stoner") and not (st.scf == "stoner" and st.scf_response)
        assert st.terminator == "constant"
        sdir = np.array(spin_dir, np.float64)
        sdir = sdir / np.linalg.norm(sdir, axis=1)[:, None]
    magnetic = st.scf == "stoner" or nc
    if magnetic:
        m = np.full(n, st.m0) if m_init is None else np.array(m_init, np.float64)
    N0 = st.n_e
    target = st.n_e * n
    hist_x, hist_f = [], []
    if st.terminator == "mlp":
        from . import mlp as _mlp
        assert st.n_mom == 9 and st.net is not None
        stage = lambda m: _mlp.learned_stage(m, st.net, st.n_exp)  # noqa: E731
    else:
        stage = lambda m: scalar_stage(m, st.n_exp, st.bandwidth)  # noqa: E731
    it = 0
    converged = st.scf == "none"
    while True:
        onsite = np.zeros((S, n, norb))
        for v in range(S):
            onsite[v] = model.onsite0 + delta[:, None]
            if norb == 6:
                onsite[v][:, 0] = model.onsite_s + delta
            if magnetic:
                sign = -1.0 if v == 0 else 1.0
                onsite[v] += sign * 0.5 * st.stoner_I * m[:, None]
        if nc:
            Mnc = moments_nc(nbr, H, onsite, sdir, st.n_mom)
            mu = local_moments(Mnc, sdir)
        else:
            mu = np.stack([moments(nbr, H, onsite[v], st.n_mom) for v in range(S)])
        mu_f = mu.reshape(-1, st.n_mom)
        ex = stage(mu_f)
        E_F, n_bis = fermi_bisect(ex, s, target)
        N, U = orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, onsite.reshape(-1), E_F)
        Nsv = N.reshape(S, n, norb)
        if st.scf == "none" or it >= st.scf_max_it:
            break
        Ni = s * Nsv.sum(axis=(0, 2))
        res = Ni - N0
        dos = s * dos_at(ex.gsig, ex.a_inf, ex.b_inf, E_F).reshape(S, n, norb).sum(axis=(0, 2))
        if st.scf == "variational":
            # residual Delta_i = dU_B/d delta_i; Newton-like step with the
            # local estimate d Delta_i / d delta_i ~ D (1 + J_ii D), D = s n_i(E_F)
            res, _, _ = variational_gradient(st, nbr, H, onsite, mu_f, E_F, stage, s)
        done = np.max(np.abs(res)) < st.scf_tol
        if st.scf == "stoner":
            m_out = (Nsv[0] - Nsv[1]).sum(axis=1)
            done = done and np.max(np.abs(m_out - m)) < 10 * st.scf_tol
        if done:
            converged = True
            break
        # preconditioned residual F; linear mixing x += F, or Anderson mixing
        if st.scf == "variational":
            Dt = np.maximum(dos, st.dos_floor)
            F = -st.eta * res / (Dt * (1.0 + st.J_ii * Dt))
        else:
            F = st.eta * res / np.maximum(dos, st.dos_floor)
        x = delta.copy()
        if st.scf == "stoner":
            F = np.concatenate([F, st.m_mix * (m_out - m)])
            x = np.concatenate([x, m])
        if st.mixer == "anderson":
            hist_x.append(x)
            hist_f.append(F)
            del hist_x[:-(st.mix_history + 1)], hist_f[:-(st.mix_history + 1)]
            h = len(hist_f) - 1
            x_new = x + F
            if h > 0:
                dF = np.array([hist_f[j + 1] - hist_f[j] for j in range(h)])
                dX = np.array([hist_x[j + 1] - hist_x[j] for j in range(h)])
                A = dF @ dF.T
                A[np.diag_indices(h)] += 1e-12 * np.max(np.diag(A)) + 1e-300
                gamma = np.linalg.solve(A, dF @ F)
                x_new = x_new - gamma @ (dX + dF)
        else:
            x_new = x + F
        delta = x_new[:n] - x_new[:n].mean()
        if st.scf == "stoner":
            m = x_new[n:]
        it += 1
    e_atom = s * U.reshape(S, n, norb).sum(axis=(0, 2))
    if magnetic:
        e_atom = e_atom - 0.25 * st.stoner_I * m ** 2
    if st.scf == "variational":
        q = s * Nsv.sum(axis=(0, 2)) - N0
        e_atom = e_atom + 0.5 * st.J_ii * q ** 2
    if model.rep_A != 0.0:
        # half of every bond to each of its atoms: half of each directed edge
        dvec = edge_vectors(pos, cell, nbr)
        phi, _ = pair_repulsion(model, np.linalg.norm(dvec, axis=1))
        src = np.repeat(np.arange(n), np.diff(nbr.row_ptr))
        e_atom = e_atom + np.bincount(src, weights=0.5 * phi, minlength=n)
    out = dict(e_atom=e_atom, e_total=float(e_atom.sum()), e_fermi=E_F, mu=mu,
               a=ex.a, b=ex.b, a_inf=ex.a_inf, b_inf=ex.b_inf, N=Nsv, delta=delta, m=m,
               scf_iterations=it, scf_converged=converged, bisection_steps=n_bis,
               neighbors=nbr, H=H, onsite=onsite, forces_include_scf_response=st.scf == "none",
               learned=getattr(ex, "learned", None), M_nc=Mnc if nc else None,
               unbounded=outside_band(ex.sigma))
    if want_forces:
        w, dU_dE, dN, _, _, dU = weights(mu_f, onsite.reshape(-1), E_F, st.n_exp, s, stage)
        w = w.reshape(S, n, norb, st.n_mom)
        resp = st.scf in ("lcn", "stoner") and st.scf_response
        if st.scf == "variational":
            # U_B is stationary in delta: its derivative at fixed delta is exact
            _, w, _ = variational_gradient(st, nbr, H, onsite, mu_f, E_F, stage, s)
        if resp:
            w, lam_scf = scf_response_weights(st, nbr, H, onsite, m, s * dU.reshape(w.shape),
                                              dU_dE.reshape(S, n, norb), dN.reshape(w.shape))
            out.update(scf_multipliers=lam_scf)
        out["forces_include_scf_response"] = st.scf in ("none", "variational") or resp
        Hbar = np.zeros((nbr.n_edges, norb, norb))
        if nc:
            # weights in the global frame; torques (section "Torques"):
            # dU/ds = 1/2 Tr(Theta~ sigma) Delta + 1/2 sum_n (w_dn - w_up) Tr(sigma M_n)
            # per orbital, Delta = E_dn - E_up; the term -I m m_i of the same
            # equation is parallel to s_i and drops out of t = dU/ds x s
            Hbar, Obar = moments_nc_adjoint(nbr, H, onsite, sdir, global_weights(w, sdir))
            dUds = 0.5 * np.einsum("ia,iax->ix", onsite[1] - onsite[0], Obar[:, :, 1:])
            dUds += 0.5 * np.einsum("iam,iamx->ix", w[1] - w[0], pauli_vector(Mnc))
            out.update(torques=np.cross(dUds, sdir), dU_ds=dUds, Obar=Obar)
        else:
            for v in range(S):
                hb, _ = moments_adjoint(nbr, H, onsite[v], w[v])
                Hbar += hb
        g = bond_gradient(model, pos, cell, nbr, Hbar)
        if model.rep_A != 0.0:
            dvec = edge_vectors(pos, cell, nbr)
            r = np.linalg.norm(dvec, axis=1)
            _, dphi = pair_repulsion(model, r)
            g = g + (0.5 * dphi / r)[:, None] * dvec   # d(phi/2)/dd per directed edge
        F = np.zeros((n, 3))
        src = np.repeat(np.arange(n), np.diff(nbr.row_ptr))
        np.add.at(F, src, g)
        np.add.at(F, nbr.col, -g)
        dvec = edge_vectors(pos, cell, nbr)
        vir = np.einsum("ea,eb->ab", g, dvec)
        out.update(forces=F, virial=vir, weights=w, Hbar=Hbar)
    return out


def scf_response_weights(st: Settings, nbr: Neighbors, H, onsite, m, wU, dUE, wN):
    """Weights dE/dmu of the self-consistent energy including the response
    of the SCF unknowns u (the per-atom shifts delta, and for Stoner the
    moments m), by the implicit function theorem written out densely.

    SCF conditions at fixed E_F: R_i = s sum_{alpha,nu} N_i - n_e = 0 and,
    for Stoner, Q_i = sum_alpha (N_i,up - N_i,down) - m_i = 0, with the onsite
    levels E_i alpha nu = E0 + delta_i -/+ I m_i / 2.  A joint shift of all
    levels and E_F leaves N and U unchanged, so with E_F held fixed the
    partial derivatives below already satisfy the stationarity condition of
    E_F and no gauge multiplier enters.  With J = d(R, Q)/du and
    g = dE/du (both at fixed E_F and structure), J^T y = g gives the
    multipliers y = (lambda, kappa), and
        dE/dx = dE/dx|_u - lambda . dR/dx|_u - kappa . dQ/dx|_u,
    i.e. the weights w = wU - c w^N with c_i,nu = s lambda_i + sigma_nu kappa_i
    (sigma = +1 up, -1 down).  J is built row by row from the reverse sweep
    of the moments (``moments_adjoint``) and solved with numpy.linalg.solve.
    wU = s dU/dmu, wN = dN/dmu (fixed E_F), dUE = direct d(sU)/dE; all
    [S, n, norb(, n_mom)]."""
    S, n, norb, n_mom = wU.shape
    s = 2.0 if S == 1 else 1.0
    stoner = st.scf == "stoner"
    I = st.stoner_I
    sig = np.array([1.0, -1.0]) if S == 2 else np.array([1.0])
    nu = 2 * n if stoner else n

    def ebar_of(wts, atom=None):
        """d(sum wts . mu)/dE for every orbital: [S, n, norb].  With ``atom``
        the weights vanish outside that atom, so only its cluster is swept
        (the other clusters would add exact zeros)."""
        if atom is None:
            return np.stack([moments_adjoint(nbr, H, onsite[v], wts[v])[1] for v in range(S)])
        sel = np.array([atom], np.int32)
        return np.stack([moments_adjoint(nbr, H, onsite[v], wts[v][atom:atom + 1], sel)[1] for v in range(S)])

    def project(eb):
        """Derivative with respect to u of a function whose derivative with
        respect to the onsite levels is eb [S, n, norb]."""
        gd = eb.sum(axis=(0, 2))
        if not stoner:
            return gd
        gm = -0.5 * I * eb[0].sum(axis=1) + 0.5 * I * eb[1].sum(axis=1)
        return np.concatenate([gd, gm])

    g = project(ebar_of(wU) + dUE)
    if stoner:
        g[n:] += -0.5 * I * m
    J = np.zeros((nu, nu))
    for i in range(nu):
        c = np.zeros((S, n))
        if i < n:
            c[:, i] = s
        else:
            c[:, i - n] = sig
        row = project(ebar_of(c[:, :, None, None] * wN, i % n))
        if i >= n:
            row[i] -= 1.0
        J[i] = row
    y = np.linalg.solve(J.T, g)
    lam = y[:n]
    kap = y[n:] if stoner else np.zeros(n)
    cc = s * lam[None, :] + sig[:, None] * kap[None, :]
    return wU - cc[:, :, None, None] * wN, y
