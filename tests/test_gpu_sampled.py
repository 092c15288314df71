"""FP32-products error at the full sizes of the large workloads, on samples
the oracle can compute atom by atom: the 16,320-atom slab (13 moments), the
65,536-atom magnetic cell (two spin channels at fixed moments m0, 9 moments)
and the 131,072-atom evaluation cell of the learned terminator (9 moments).

The GPU computes the moments of every atom of the full cell; the oracle
computes them for a compact group of 16 atoms on a cut-out of the same cell
(every atom image within K r_cut of the group, which holds the group's
clusters, as the domain tests show).  The FP32 moments are compared with the
oracle's, and their error carried into the band energy of each sampled atom
by the oracle's own scalar stage at a common Fermi level (the oracle's
bisection over the sample), so that the per-atom energy error of FP32
products is stated per configuration.
"""
import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bop():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_07491_gb300 import build, bop as b
    build.build()
    return b


def cut_out(pos, cell, pbc, centre_atoms, radius):
    """Every atom image (periodic images along the periodic axes) within
    `radius` of the centroid of centre_atoms, plus those atoms; returns
    (positions, box cell, local index of each centre atom).  The box is a
    non-periodic cube around the cut-out."""
    pos = np.asarray(pos, np.float64)
    c = pos[centre_atoms].mean(axis=0)
    rng = [range(-1, 2) if p else range(0, 1) for p in pbc]
    keep, seen = [], {}
    for sx in rng[0]:
        for sy in rng[1]:
            for sz in rng[2]:
                shift = np.array([sx, sy, sz], np.float64) @ np.asarray(cell)
                p = pos + shift
                d = np.linalg.norm(p - c, axis=1)
                for j in np.nonzero(d <= radius)[0]:
                    seen[(int(j), sx, sy, sz)] = len(keep)
                    keep.append(p[j])
    local = np.array(keep)
    lo = local.min(axis=0) - 1.0
    box = np.diag(local.max(axis=0) - lo + 1.0)
    idx = np.array([seen[(int(j), 0, 0, 0)] for j in centre_atoms])
    return local - lo, box, idx


def _group(w, n=16):
    """16 atoms closest to a seeded point inside the cell (away from a free
    surface for the slab)."""
    rng = np.random.default_rng(11)
    f = rng.uniform(0.3, 0.7, size=3)
    p = f @ w.cell
    d = np.linalg.norm(w.pos - p, axis=1)
    return np.argsort(d)[:n]


@pytest.mark.parametrize("name", ["slab16k", "mag65k", "learned131k"])
def test_fp32_moments_and_band_energy_error_on_a_sample(bop, ob, name):
    w = I.workload(name)
    run = I.with_run(w, scf="none", scf_response=False).run
    n_spin, norb, n_mom = run.n_spin, w.model.norb, run.n_mom
    K = (n_mom - 1) // 2
    grp = _group(w)
    # oracle: moments of the group on the cut-out, FP64
    m = oracle_model(w.model)
    lp, lcell, lidx = cut_out(w.pos, w.cell, w.pbc, grp, K * m.rc + 8.0)
    nl = ob.neighbors(lp, lcell, (0, 0, 0), m.rc)
    Hl = ob.blocks(m, lp, lcell, nl)
    mu_ref = []
    for v in range(n_spin):
        lev = 0.0 if n_spin == 1 else (-0.5 if v == 0 else 0.5) * run.stoner_I * run.m0
        mu_ref.append(ob.moments(nl, Hl, np.full((len(lp), norb), lev), n_mom, lidx.astype(np.int32)))
    mu_ref = np.stack(mu_ref)  # [S, 16, norb, n_mom]
    errs = {}
    for prec in ("fp64", "fp32"):
        ctx = bop.Context(w.model, run, prec)
        ctx.build(w.pos, w.cell, w.pbc)
        onsite = torch.zeros((n_spin, w.n_atoms, norb), dtype=torch.float64, device="cuda")
        if n_spin == 2:
            onsite[0] = -0.5 * run.stoner_I * run.m0
            onsite[1] = 0.5 * run.stoner_I * run.m0
        mu_all = bop.bop_moments(ctx.h, n_spin, w.n_atoms, norb, n_mom, onsite)
        mu = mu_all.reshape(n_spin, w.n_atoms, norb, n_mom)[:, torch.as_tensor(grp, device="cuda")].cpu().numpy()
        ctx.close()
        scale = np.abs(mu_ref).max(axis=-1, keepdims=True) + 1.0
        rel = float(np.max(np.abs(mu - mu_ref) / scale))
        # band energy of each sampled atom from either set of moments through
        # the oracle's scalar stage, at the oracle's Fermi level of the sample
        s = 2.0 if n_spin == 1 else 1.0
        ex_ref = ob.scalar_stage(mu_ref.reshape(-1, n_mom), run.n_exp)
        E_F, _ = ob.fermi_bisect(ex_ref, s, run.n_e * len(grp))
        on = np.zeros(mu_ref.size // n_mom)
        _, U_ref = ob.orbital_N_U(ex_ref.gsig, ex_ref.a_inf, ex_ref.b_inf, on, E_F)
        ex = ob.scalar_stage(mu.reshape(-1, n_mom), run.n_exp)
        _, U = ob.orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, on, E_F)
        e_ref = s * U_ref.reshape(n_spin, len(grp), norb).sum(axis=(0, 2))
        e = s * U.reshape(n_spin, len(grp), norb).sum(axis=(0, 2))
        errs[prec] = (rel, float(np.max(np.abs(e - e_ref))))
    print(f"\n{name}: fp64 moments {errs['fp64'][0]:.2e} energy {errs['fp64'][1]:.2e} eV/atom; "
          f"fp32 moments {errs['fp32'][0]:.2e} energy {errs['fp32'][1]:.2e} eV/atom")
    assert errs["fp64"][0] < 1e-11 and errs["fp64"][1] < 1e-8
    assert errs["fp32"][0] < 1e-5 and errs["fp32"][1] < 1e-3
