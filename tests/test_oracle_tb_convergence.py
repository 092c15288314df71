"""The oracle's energy pipeline as a whole against exact tight binding.

The BOP band energy (moments -> recursion -> constant terminator ->
Chebyshev expansion -> Fermi level -> bond energy) approximates the band
energy of the same orthogonal TB Hamiltonian; with more moments the local
DOS is resolved further and the two approach each other (Appendix A, Eq.
TB-Ubond; the moments theorem of section "Moments").  The reference here is
the TB band energy of the periodic crystal by Bloch sums H(k) over a dense
Monkhorst-Pack grid and numpy's eigvalsh (no moments, no recursion), at the
same electron count, with the onsite level 0 so that both energies are
sum_alpha int^E_F E n(E) dE.  The comparison is a trend: the expansion
length is raised to 1000 so that the Jackson broadening of the 200-term
expansion, which holds its own error of a few meV, does not mask the
convergence in the moments.
"""
import numpy as np

from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model


def tb_band_energy(ob, model, pos, cell, pbc, n_e, mk):
    """Band energy per atom of the periodic crystal (spin factor 2): Bloch
    Hamiltonian H_ij(k) = sum over the bonds i -> j (image S) of
    H_ij e^{i k . d_ij}, d_ij = r_j + S cell - r_i, on an mk^3 grid shifted
    by half a step; the lowest n_e N / 2 states per k-point on average are
    filled (the last one fractionally)."""
    nbr = ob.neighbors(pos, cell, pbc, model.rc)
    H = ob.blocks(model, pos, cell, nbr)
    n, no = len(pos), model.norb
    src = np.repeat(np.arange(n), np.diff(nbr.row_ptr))
    d = ob.edge_vectors(pos, cell, nbr)
    rec = 2.0 * np.pi * np.linalg.inv(cell).T
    g = (np.arange(mk) + 0.5) / mk
    ks = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) @ rec
    ph = np.exp(1j * (ks @ d.T))
    Hk = np.zeros((len(ks), n * no, n * no), complex)
    for e in range(len(src)):
        i, j = src[e], nbr.col[e]
        Hk[:, i * no:(i + 1) * no, j * no:(j + 1) * no] += H[e].reshape(no, no)[None] * ph[:, e, None, None]
    assert np.allclose(Hk, np.conj(np.transpose(Hk, (0, 2, 1))))
    E = np.sort(np.linalg.eigvalsh(Hk).ravel())
    nk = len(ks)
    states = n_e * n * nk / 2.0
    full = int(np.floor(states))
    return 2.0 / nk * (E[:full].sum() + (states - full) * E[full]) / n


def test_bop_band_energy_converges_to_tb(ob):
    model = oracle_model(I.MODEL_D)
    pos, cell = I.bcc_jittered(2, 2, 2, 0.05, 11)
    e_tb = tb_band_energy(ob, model, pos, cell, (1, 1, 1), 6.8, 8)
    # the k-grid is converged well below the differences tested below
    assert abs(e_tb - tb_band_energy(ob, model, pos, cell, (1, 1, 1), 6.8, 6)) < 3e-4
    err = {}
    for nm in (5, 9, 13, 17):
        st = ob.Settings(n_e=6.8, n_mom=nm, n_exp=1000)
        out = ob.evaluate(model, st, pos, cell, (1, 1, 1), want_forces=False)
        err[nm] = abs(out["e_total"] / len(pos) - e_tb)
    # measured: 8.0e-2, 1.4e-2, 1.7e-3, 1.0e-3 eV/atom
    assert err[5] > err[9] > err[13] > err[17]
    assert err[5] > 3e-2 and err[17] < 3e-3
