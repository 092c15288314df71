"""Seeded synthetic inputs: bcc/fcc cells, jitter, vacancies, slabs, and the
model parameter sets of the benchmark workloads.

This module holds no arithmetic of the BOP method.  It is the one module
that both the CUDA path and the CPU oracle take their inputs from.

Random numbers come from ``numpy.random.default_rng(seed)``; the draws are
made in a fixed order that is stated in each function.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

A_BCC = 2.87  # Angstrom, lattice constant of all bcc workloads


def bcc_cell(n1: int, n2: int, n3: int, a: float = A_BCC):
    """Perfect bcc crystal of n1 x n2 x n3 conventional cells (2 atoms each).
    Atom order: cells in (i, j, k) row-major order, basis (0,0,0) then
    (1/2,1/2,1/2).  Returns (pos [N,3], cell [3,3] rows = lattice vectors)."""
    ii, jj, kk = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    corners = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.float64)
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    frac = (corners[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    pos = frac * a
    cell = np.diag([n1 * a, n2 * a, n3 * a]).astype(np.float64)
    return pos, cell


def fcc_cell(n1: int, n2: int, n3: int, a: float):
    """Perfect fcc crystal, 4 atoms per conventional cell, same ordering."""
    ii, jj, kk = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    corners = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.float64)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], np.float64)
    pos = (corners[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    return pos, np.diag([n1 * a, n2 * a, n3 * a]).astype(np.float64)


def wrap(pos, cell, pbc):
    """Map positions into the cell along the periodic axes (fractional
    coordinates in [0, 1))."""
    frac = np.linalg.solve(np.asarray(cell).T, np.asarray(pos).T).T
    for ax in range(3):
        if pbc[ax]:
            frac[:, ax] -= np.floor(frac[:, ax])
            frac[:, ax] = np.where(frac[:, ax] >= 1.0, 0.0, frac[:, ax])
    return frac @ np.asarray(cell)


def jittered(pos, cell, pbc, sigma: float, rng):
    """Add N(0, sigma^2) to every Cartesian component (one draw of shape
    [N, 3], atom order then x, y, z) and wrap into the cell."""
    d = rng.normal(0.0, sigma, size=pos.shape)
    return wrap(pos + d, cell, pbc)


@dataclass(frozen=True)
class ModelParams:
    """Exponential two-centre bond integrals with a cosine taper."""
    norb: int          # 1 = s, 5 = d
    b0: tuple          # eV at r0: (ss sigma,), (dd sigma, dd pi, dd delta) or, for sd,
    #                    (dd sigma, dd pi, dd delta, ss sigma, sd sigma)
    r0: float          # Angstrom
    lam: float         # 1/Angstrom
    rc: float          # cutoff radius, Angstrom
    dc: float          # taper width, Angstrom
    onsite0: float = 0.0
    rep_A: float = 0.0   # pair repulsion rep_A exp(-rep_p (r - r0)) fcut(r), eV; 0 = none
    rep_p: float = 0.0   # 1/Angstrom
    onsite_s: float = 0.0  # sd model (norb 6): reference level of the s orbital, eV


# s-valent model: ss sigma = -1.0 eV exp(-1.5 (r - 2.48)), taper 3.2-3.6 A
MODEL_S = ModelParams(norb=1, b0=(-1.0,), r0=2.48, lam=1.5, rc=3.6, dc=0.4)
# canonical d model: sigma:pi:delta = -6:4:-1 scaled to dd sigma(2.48) = -0.9 eV,
# exp decay 1.8/A, cutoff 3.6 A with a 0.4 A taper (1st + 2nd bcc shells)
MODEL_D = ModelParams(norb=5, b0=(-0.9, 0.6, -0.15), r0=2.48, lam=1.8, rc=3.6, dc=0.4)
# sd-valent model (norb 6, s first): the canonical d block plus ss sigma =
# -1.4 eV and sd sigma = -0.7 eV at r0 with the same decay, s level 3 eV
# above the d level
MODEL_SD = ModelParams(norb=6, b0=(-0.9, 0.6, -0.15, -1.4, -0.7), r0=2.48, lam=1.8, rc=3.6, dc=0.4,
                       onsite_s=3.0)
# the same with a pair repulsion decaying twice as fast as the bond integrals,
# its amplitude chosen so that perfect bcc of the cells below has zero
# pressure without SCF (a stable lattice for MD; checked by the oracle tests)
MODEL_D_REP = ModelParams(norb=5, b0=(-0.9, 0.6, -0.15), r0=2.48, lam=1.8, rc=3.6, dc=0.4,
                          rep_A=0.6218844075436114, rep_p=3.6)


@dataclass(frozen=True)
class RunParams:
    n_e: float            # electrons per atom, summed over spin
    n_mom: int = 9
    n_exp: int = 200
    n_spin: int = 1
    scf: str = "none"     # none | lcn | stoner | variational
    eta: float = 0.5
    scf_tol: float = 1e-9
    scf_max_it: int = 200
    stoner_I: float = 0.0
    m_mix: float = 0.3
    m0: float = 2.0
    dos_floor: float = 0.1
    mixer: str = "anderson"   # linear | anderson (type-II Broyden)
    mix_history: int = 6
    terminator: str = "constant"  # constant | mlp (learned continuation of the chain, n_mom = 9)
    scf_response: bool = True     # with an SCF, forces include the response of the onsite levels
    bandwidth: str = "gershgorin"  # gershgorin | lowest | highest | average | average_centre | minmax | global
    #                                | weighted: the band centre / width estimate of the constant terminator
    bw_beta: float = 1.0          # weighted: w_m = 1/(beta (m_max - m) + 1)
    bw_a: float = 0.0             # global: A (eV)
    bw_b: float = 1.0             # global: B (eV)
    J_ii: float = 0.0             # variational SCF: onsite charging energy J_ii q_i^2 / 2 (eV / e^2)
    r_path: float = 0.0           # path-radius cut (A): only sites closer than r_path to the atom; 0 = none
    noncollinear: bool = False    # one moment direction per atom (n_spin = 2, scf none | stoner)


@dataclass
class Workload:
    name: str
    pos: np.ndarray
    cell: np.ndarray
    pbc: tuple
    model: ModelParams
    run: RunParams
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self):
        return len(self.pos)


A_FCC = 3.51  # Angstrom: nearest-neighbour distance 2.482 A, the canonical model's r0


def fcc_jittered(n1, n2, n3, sigma, seed, a=A_FCC, pbc=(1, 1, 1)):
    pos, cell = fcc_cell(n1, n2, n3, a)
    rng = np.random.default_rng(seed)
    return jittered(pos, cell, pbc, sigma, rng), cell


def bcc_jittered(n1, n2, n3, sigma, seed, pbc=(1, 1, 1)):
    pos, cell = bcc_cell(n1, n2, n3)
    rng = np.random.default_rng(seed)
    return jittered(pos, cell, pbc, sigma, rng), cell


def slab_with_vacancies(n1, n2, n3, n_vac, sigma, seed, vacuum=10.0):
    """bcc slab with two free (001) surfaces: pbc (1, 1, 0); the cell's z
    vector is n3*a + vacuum and the slab is centred in it.  Draw order from
    default_rng(seed): first the vacancy indices (choice without
    replacement), then the jitter of the remaining atoms."""
    pos, cell = bcc_cell(n1, n2, n3)
    rng = np.random.default_rng(seed)
    vac = rng.choice(len(pos), size=n_vac, replace=False)
    keep = np.ones(len(pos), bool)
    keep[vac] = False
    pos = pos[keep]
    pos[:, 2] += 0.5 * vacuum
    cell = cell.copy()
    cell[2, 2] = n3 * A_BCC + vacuum
    pbc = (1, 1, 0)
    pos = jittered(pos, cell, pbc, sigma, rng)
    return pos, cell, pbc


# Anderson mixing of the workloads: unit steps on the DOS-preconditioned
# residual over 8 iterations (the SCF reaches the same state in fewer
# iterations than with the linear-mixing step 0.5: d2000 FP32 7 -> 5,
# mag65k 21 -> 13).
ANDERSON_STEP = dict(eta=1.0, mix_history=8)


MASS_FE = 55.845       # amu
K_B = 8.617333262e-5   # eV / K
EV_PER_AMU = 1.602176634e-19 / 1.66053906660e-27 * 1e-10   # (A / fs)^2 per (eV / amu)


def maxwell_velocities(n: int, T: float, mass: float, seed: int) -> np.ndarray:
    """Velocities (A/fs) drawn from the Maxwell-Boltzmann distribution at T,
    with the mean (net momentum) removed."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3)) * np.sqrt(K_B * T / mass * EV_PER_AMU)
    return v - v.mean(axis=0)


def random_directions(n: int, seed: int) -> np.ndarray:
    """n unit vectors uniform on the sphere: default_rng(seed).normal
    (n, 3), each row divided by its norm."""
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


def spiral_directions(pos: np.ndarray, period: float, cone: float) -> np.ndarray:
    """A conical spin spiral along x: s_i = (sin c cos q x_i, sin c sin q x_i,
    cos c), q = 2 pi / period (A), c = cone (radians)."""
    ph = 2.0 * np.pi * pos[:, 0] / period
    return np.stack([np.sin(cone) * np.cos(ph), np.sin(cone) * np.sin(ph), np.full(len(pos), np.cos(cone))], axis=1)


def workload(name: str) -> Workload:
    """Named workloads.

    s128      128-atom bcc (4x4x4x2), jitter 0.05 A, seed 1; s model; 9 moments;
              N_e = 0.7 per atom; no SCF.
    d2000     2,000-atom bcc (10x10x10x2), jitter 0.05 A, seed 2; canonical d;
              N_d = 6.8; local charge neutrality (Anderson, ANDERSON_STEP);
              9 moments.
    d2000nscf the same cell without SCF (fixed onsite levels).
    sd2000    the d2000 cell with the sd-valent model MODEL_SD (6 orbitals,
              8 electrons per atom), local charge neutrality.
    d2000cut  d2000 with the path-radius cut at 5.5 A (five neighbour shells;
              "Performance", item (iii)).
    d2000var  the same cell with the variational SCF (Eq. BOP_SCF), J_ii =
              20 eV / e^2 (Anderson, ANDERSON_STEP); with J_ii = 2 the minimum
              of this cell sits on a kink of the Gershgorin estimate and the
              residual stalls at 9e-5.
    slab16k   16x16x32x2 bcc slab with (001) surfaces, 64 vacancies, jitter
              0.08 A, seed 3; canonical d; 13 moments; no SCF.
    mag65k    65,536-atom bcc (32x32x32x2), jitter 0.05 A, seed 4; canonical d;
              two spin channels, Stoner I = 0.8 eV from a ferromagnetic start
              (Anderson, ANDERSON_STEP, moment step 1.0); 9 moments.
    mag2000   its 2,000-atom (10x10x10x2) counterpart, seed 4.
    fcc2048   2,048-atom fcc (8x8x8x4, a = 3.51 A: 12 + 6 neighbours within
              3.6 A), jitter 0.05 A, seed 6; canonical d; N_d = 6.8; local
              charge neutrality; 9 moments.
    md2000    the d2000 cell and settings (LCN) with the pair repulsion of
              MODEL_D_REP, as the start of an NVE run: Maxwell-Boltzmann
              velocities at 300 K (seed 7, no net momentum), iron's mass,
              time step 1 fs (meta: vel, mass, dt).
    nc2000    the mag2000 cell with non-collinear moments: a conical spin
              spiral along x (one period over the cell, cone angle 60
              degrees; meta: spin_dir), Stoner SCF of the magnitudes at fixed
              directions (forces and torques at the self-consistent onsite
              levels).
    learned131k 131,072-atom bcc (32x32x64x2), jitter 0.05 A, seed 5;
              canonical d; 9 moments; no SCF (evaluation cell of the
              learned terminator).
    """
    if name == "s128":
        pos, cell = bcc_jittered(4, 4, 4, 0.05, 1)
        return Workload(name, pos, cell, (1, 1, 1), MODEL_S, RunParams(n_e=0.7))
    if name in ("d2000", "d2000nscf", "d2000var", "d2000cut"):
        pos, cell = bcc_jittered(10, 10, 10, 0.05, 2)
        scf = {"d2000": "lcn", "d2000nscf": "none", "d2000var": "variational", "d2000cut": "lcn"}[name]
        J = 20.0 if name == "d2000var" else 0.0
        r_path = 5.5 if name == "d2000cut" else 0.0
        return Workload(name, pos, cell, (1, 1, 1), MODEL_D,
                        RunParams(n_e=6.8, scf=scf, J_ii=J, r_path=r_path, **ANDERSON_STEP))
    if name == "sd2000":
        pos, cell = bcc_jittered(10, 10, 10, 0.05, 2)
        return Workload(name, pos, cell, (1, 1, 1), MODEL_SD, RunParams(n_e=8.0, scf="lcn", **ANDERSON_STEP))
    if name == "slab16k":
        pos, cell, pbc = slab_with_vacancies(16, 16, 32, 64, 0.08, 3)
        return Workload(name, pos, cell, pbc, MODEL_D, RunParams(n_e=6.8, n_mom=13))
    if name in ("mag65k", "mag2000"):
        n = 32 if name == "mag65k" else 10
        pos, cell = bcc_jittered(n, n, n, 0.05, 4)
        return Workload(name, pos, cell, (1, 1, 1), MODEL_D,
                        RunParams(n_e=6.8, n_spin=2, scf="stoner", stoner_I=0.8, m_mix=1.0, **ANDERSON_STEP))
    if name == "nc2000":
        w = workload("mag2000")
        run = replace(w.run, noncollinear=True, scf_response=False)
        sd = spiral_directions(w.pos, w.cell[0, 0], np.pi / 3)
        return Workload(name, w.pos, w.cell, w.pbc, w.model, run, dict(spin_dir=sd))
    if name == "fcc2048":
        pos, cell = fcc_jittered(8, 8, 8, 0.05, 6)
        return Workload(name, pos, cell, (1, 1, 1), MODEL_D, RunParams(n_e=6.8, scf="lcn", **ANDERSON_STEP))
    if name == "md2000":
        w = workload("d2000")
        vel = maxwell_velocities(w.n_atoms, 300.0, MASS_FE, 7)
        return Workload(name, w.pos, w.cell, w.pbc, MODEL_D_REP, w.run, dict(vel=vel, mass=MASS_FE, dt=1.0))
    if name == "learned131k":
        pos, cell = bcc_jittered(32, 32, 64, 0.05, 5)
        return Workload(name, pos, cell, (1, 1, 1), MODEL_D, RunParams(n_e=6.8))
    raise KeyError(name)


def training_cell(k: int, n: int = 10) -> Workload:
    """Training cell k of the learned terminator: n x n x n x 2 bcc under a
    homogeneous symmetric strain, jittered.  Draw order from
    default_rng(1000 + k): sigma ~ U[0.02, 0.15] A, the strain components
    (xx, yy, zz, yz, xz, xy) ~ U[-0.03, 0.03], then the jitter.  Canonical d,
    17 moments, no SCF."""
    rng = np.random.default_rng(1000 + k)
    sigma = rng.uniform(0.02, 0.15)
    e = rng.uniform(-0.03, 0.03, size=6)
    eps = np.array([[e[0], e[5], e[4]], [e[5], e[1], e[3]], [e[4], e[3], e[2]]])
    D = np.eye(3) + eps
    pos, cell = bcc_cell(n, n, n)
    pos, cell = pos @ D.T, cell @ D.T
    pos = jittered(pos, cell, (1, 1, 1), sigma, rng)
    return Workload(f"train{k}", pos, cell, (1, 1, 1), MODEL_D, RunParams(n_e=6.8, n_mom=17),
                    {"sigma": sigma, "strain": eps})


def small_bcc(n1, n2, n3, sigma, seed, model=MODEL_D, run=None, pbc=(1, 1, 1)):
    """A small jittered bcc cell for tests."""
    pos, cell = bcc_cell(n1, n2, n3)
    rng = np.random.default_rng(seed)
    pos = jittered(pos, cell, pbc, sigma, rng)
    run = run or RunParams(n_e={1: 0.7, 5: 6.8, 6: 8.0}[model.norb])
    return Workload(f"bcc{n1}x{n2}x{n3}", pos, cell, tuple(pbc), model, run)


def with_run(w: Workload, **kw) -> Workload:
    return Workload(w.name, w.pos, w.cell, w.pbc, w.model, replace(w.run, **kw), w.meta)


# ---------------------------------------------------------------- learned terminator
MLP_SHAPES = [(128, 18), (128,), (128, 128), (128,), (10, 128), (10,)]


def mlp_init_params(seed: int, scale: float = 1.0) -> np.ndarray:
    """Initial parameters of the 18-128-128-10 network in the flat layout
    W1, b1, W2, b2, W3, b3: weights ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from
    default_rng(seed) in layout order, times scale; zero biases; FP32
    values (returned as float64)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in MLP_SHAPES:
        if len(s) == 2:
            lim = 1.0 / np.sqrt(s[1])
            parts.append(scale * rng.uniform(-lim, lim, size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts).astype(np.float32).astype(np.float64)


def mlp_fixed_norm() -> np.ndarray:
    """A fixed normalisation vector for tests of the learned path (layout
    x_mean, x_std, x_lo, x_hi, y_mean, y_std): identity standardisation of
    the inputs with an unbounded range, outputs centred on the constant
    chain (a*_inf = a_inf, b*_inf = b_inf, a_k = a_inf, b_k = b_inf / 2 in
    units of b_inf) with standard deviation 0.05."""
    x_mean, x_std = np.zeros(18), np.ones(18)
    lo, hi = np.full(18, -1e30), np.full(18, 1e30)
    y_mean = np.array([0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.5, 0.5, 0.5, 0.5])
    y_std = np.full(10, 0.05)
    return np.concatenate([x_mean, x_std, lo, hi, y_mean, y_std]).astype(np.float32).astype(np.float64)
