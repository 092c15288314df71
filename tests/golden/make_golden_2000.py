"""Writes tests/golden/{d2000,mag2000}_oracle.npz from the oracle alone.

The FP64 oracle's self-consistent state of the two 2,000-atom workloads,
for the element-by-element checks of the FP32-products GPU path:

  d2000    canonical d, local charge neutrality (Eq. BOP_LCN, per atom);
  mag2000  canonical d, two spin channels, collinear Stoner exchange
           I = 0.8 eV (section "Magnetism", Eqs. onsite_NCM and TB-UX) from
           a ferromagnetic start.

Stored per workload: energy per atom, Fermi level, onsite shifts, magnetic
moments (mag2000), the forces with the response of the self-consistent
onsite levels (the exact gradient, `forces`) and without it (the
Hellmann-Feynman form of Eq. F_k, `forces_hf`), and the virial.  SCF
tolerance 1e-10 electrons.  Takes about ten minutes per workload on one
core.  Run from the repository root:
    python tests/golden/make_golden_2000.py [d2000] [mag2000]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

from oracle import bop  # noqa: E402
from paper_1803_07491_gb300 import inputs as I  # noqa: E402
from conftest import oracle_model, oracle_settings  # noqa: E402


def run(name):
    w = I.with_run(I.workload(name), scf_tol=1e-10)
    m = oracle_model(w.model)
    t0 = time.time()
    out = bop.evaluate(m, oracle_settings(w.run), w.pos, w.cell, w.pbc)
    assert out["scf_converged"] and out["forces_include_scf_response"]
    # the Hellmann-Feynman forces of the same state: restart from the
    # converged shifts (and moments), one or two SCF iterations
    hf = bop.evaluate(m, oracle_settings(I.with_run(w, scf_response=False).run), w.pos, w.cell, w.pbc,
                      delta0=out["delta"], m_init=out["m"])
    assert hf["scf_converged"] and not hf["forces_include_scf_response"]
    rec = dict(e_atom=out["e_atom"], e_fermi=np.float64(out["e_fermi"]), delta=out["delta"],
               forces=out["forces"], forces_hf=hf["forces"], virial=out["virial"],
               scf_iterations=np.int64(out["scf_iterations"]))
    if out["m"] is not None:
        rec["m"] = out["m"]
    path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle.npz")
    np.savez_compressed(path, **rec)
    print(f"{name}: {time.time() - t0:.0f} s, {out['scf_iterations']} SCF iterations, "
          f"E = {out['e_total'] / w.n_atoms:.9f} eV/atom, |E_hf - E| = "
          f"{abs(hf['e_total'] - out['e_total']):.2e} eV -> {path}")


if __name__ == "__main__":
    for name in sys.argv[1:] or ["d2000", "mag2000"]:
        run(name)
