"""Writes tests/golden/s128_oracle.json from the oracle alone.

The paper prints no numeric worked example for this path, so the stored
values are the oracle's own on the 128-atom s-valent bcc workload (9
moments, constant terminator, N_e = 0.7); they are a regression pin of the
oracle's arithmetic.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bop  # noqa: E402
from paper_1803_07491_gb300 import inputs as I  # noqa: E402


def main():
    w = I.workload("s128")
    p, r = w.model, w.run
    m = bop.Model(p.norb, tuple(p.b0), p.r0, p.lam, p.rc, p.dc, p.onsite0)
    st = bop.Settings(n_e=r.n_e, n_mom=r.n_mom, n_exp=r.n_exp)
    out = bop.evaluate(m, st, w.pos, w.cell, w.pbc)
    rec = {
        "workload": "s128",
        "source": "oracle (tests/golden/make_golden.py)",
        "e_per_atom": out["e_total"] / w.n_atoms,
        "e_fermi": out["e_fermi"],
        "mu_atom0": out["mu"][0, 0, 0].tolist(),
        "a_atom0": out["a"][0].tolist(),
        "b_atom0": out["b"][0].tolist(),
        "forces_atoms0_3": out["forces"][:4].tolist(),
        "virial": out["virial"].tolist(),
    }
    with open(os.path.join(ROOT, "tests", "golden", "s128_oracle.json"), "w") as f:
        json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main()
