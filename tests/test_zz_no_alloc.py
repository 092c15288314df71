"""The allocation-free Fermi-level entry point (collected last on purpose).

Some callers cannot call cudaMalloc: code under a device-memory budget fixed
in advance, hosts that reserve all GPU memory at start-up, paths where an
allocation would synchronise the device at the wrong moment.  For them
bop_fermi_level_noalloc runs the library's Fermi-level search with its
scratch in a static device array.  This test checks, through the C ABI, that
two calls in a row give the Fermi level that bop_energy found for the same
orbitals, within the 1e-9 eV used by the other Fermi-level tests, and that a
problem too large for the static array, or an electron count no Fermi level
inside the band can hold, is refused.
"""
import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fermi_level_noalloc_matches_bop_energy():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_07491_gb300 import bop, build
    build.build()
    w = I.small_bcc(3, 3, 3, 0.05, 102)  # 54 atoms, d orbitals, 9 moments, no SCF
    ctx = bop.Context(w.model, w.run, "fp64")
    res = ctx.evaluate(w.pos, w.cell, w.pbc, forces=False)
    M = w.n_atoms * w.model.norb
    st = bop.bop_get_orbital_state(ctx.h, M, w.run.n_mom)
    _, _, _, a_inf, b_inf, gsig = bop.bop_recursion(ctx.h, st["mu"], w.run.n_exp)
    gsig_cm = gsig.t().contiguous()  # [n_exp+1][M]
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(np.nan)
        status = bop.bop_fermi_level_noalloc(gsig_cm, a_inf, b_inf, 2.0, w.run.n_e * w.n_atoms, out)
        torch.cuda.synchronize()
        assert status == bop.BOP_OK
        assert abs(float(out.item()) - res.e_fermi) < 1e-9
    # more orbitals than the static scratch holds: refused before any launch
    big = torch.zeros((w.run.n_exp + 1, 20000), dtype=torch.float64, device="cuda")
    zeros = torch.zeros(20000, dtype=torch.float64, device="cuda")
    status = bop.bop_fermi_level_noalloc(big, zeros, zeros + 1.0, 2.0, 1.0, out)
    assert status == bop.BOP_ERR_OVERFLOW
    # an electron count that no Fermi level inside the band holds: refused
    # before any launch instead of ending at a bracket edge
    for n_el in (0.0, -1.0, 2.0 * M, 2.0 * M + 5.0, float("nan")):
        status = bop.bop_fermi_level_noalloc(gsig_cm, a_inf, b_inf, 2.0, n_el, out)
        assert status == bop.BOP_ERR_BRACKET
    # the entry point still works after the refusals
    out.fill_(np.nan)
    status = bop.bop_fermi_level_noalloc(gsig_cm, a_inf, b_inf, 2.0, w.run.n_e * w.n_atoms, out)
    torch.cuda.synchronize()
    assert status == bop.BOP_OK and abs(float(out.item()) - res.e_fermi) < 1e-9
    ctx.close()
