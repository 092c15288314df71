"""Spatial decomposition through the library on the GPU: two processes (gloo,
both on cuda:0; no kernel of one process waits on the other, the sums meet on
the host through bop_set_reduce) each evaluate their domain of the
2,000-atom cell with fixed onsite levels; the energies, forces, virial and
Fermi level gathered over the processes equal the single-process run of the
whole cell (FP64: 1e-9)."""
import os
import socket
from datetime import timedelta

import numpy as np
import pytest

from paper_1803_07491_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _worker(rank, size, port, out_path, prec):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=size, timeout=timedelta(seconds=120))
    try:
        torch.cuda.set_device(0)
        from paper_1803_07491_gb300 import domain
        w = I.workload("d2000nscf")
        res = domain.evaluate(w.model, w.run, prec, w.pos, w.cell, w.pbc)
        if rank == 0:
            np.savez(out_path, e_fermi=res["e_fermi"], e_total=res["e_total"], e_atom=res["e_atom"],
                     forces=res["forces"], virial=res["virial"], n_local=res["n_local"], n_own=res["n_own"])
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 2e-4)])
def test_two_domains_match_one_process(tmp_path, prec, tol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_07491_gb300 import build, bop
    build.build()
    import torch.multiprocessing as mp
    out = str(tmp_path / "dom.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out, prec), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    w = I.workload("d2000nscf")
    ctx = bop.Context(w.model, w.run, prec)
    ref = ctx.evaluate(w.pos, w.cell, w.pbc)
    ctx.close()
    assert int(got["n_own"]) < w.n_atoms < int(got["n_local"]) + int(got["n_own"])
    assert abs(float(got["e_fermi"]) - ref.e_fermi) < tol
    assert abs(float(got["e_total"]) - ref.e_total) < tol * w.n_atoms
    assert np.max(np.abs(got["e_atom"] - ref.e_atom.cpu().numpy())) < tol
    assert np.max(np.abs(got["forces"] - ref.forces.cpu().numpy())) < tol
    assert np.max(np.abs(got["virial"] - ref.virial.cpu().numpy())) < tol * w.n_atoms
