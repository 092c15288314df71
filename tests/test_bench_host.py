"""Host logic of bench.py that needs no GPU: the per-atom error measure of
the learned-vs-plain comparison (errors of opposite sign must not cancel)
and the work model's scaling with the workload's sizes."""
import numpy as np
import pytest

import bench
from paper_1803_07491_gb300 import inputs as I


def test_atom_errors_do_not_cancel():
    e_ref = np.zeros(4)
    e = np.array([1e-3, -1e-3, 2e-3, -2e-3])  # eV
    err = bench.atom_errors(e, e_ref)
    assert err["mean_abs"] == pytest.approx(1.5)   # meV
    assert err["max_abs"] == pytest.approx(2.0)
    assert err["of_mean"] == pytest.approx(0.0)    # the signed mean cancels


def test_work_model_scales_with_products_and_coefficients():
    w = I.workload("d2000")
    stats = {"moment_products": 3584 * w.n_atoms, "bisection_rounds": 2}
    prof = {"adjoint": {"regions": 3}}
    mom = bench.algorithmic_flops("moments", w, stats, prof, n_spin=1)
    # 2 x 5 x 5 multiply-adds per column, 5 columns: 250 FLOP per block product
    assert mom == pytest.approx(3584 * w.n_atoms * 250.0)
    # three sweeps per step, one of them with bond cotangents (twice the work)
    adj = bench.algorithmic_flops("adjoint", w, stats, prof, n_spin=1, steps=1)
    assert adj == pytest.approx(mom * (2.0 + 1.0 + 1.0) / 3.0)
    M = w.n_atoms * 5
    fermi = bench.algorithmic_flops("fermi", w, stats, prof, n_spin=1)
    assert fermi == pytest.approx(2 * M * (w.run.n_exp + 2) * 4.0)
    K = (w.run.n_mom - 1) // 2
    assert bench.algorithmic_flops("expand", w, stats, prof, n_spin=1) == pytest.approx(
        M * (w.run.n_exp + 1) * (4.0 * K + 1.0))
    # two spin channels double every per-orbital family
    assert bench.algorithmic_flops("expand", w, stats, prof, n_spin=2) == pytest.approx(
        2 * M * (w.run.n_exp + 1) * (4.0 * K + 1.0))
