"""Spatial decomposition (section "Performance", parallelisation by spatial
domains) on the CPU: the partition and its halo, and the whole multi-process
evaluation with the oracle as each process's engine, on two gloo processes.

Each process builds its domain (own atoms, then the halo within K r_cut),
computes the moments, electrons and energies of its own atoms only, finds
the one Fermi level of the whole structure by bisection on the electron
count summed over the processes (the oracle's bisection rules), forms the
E_F multiplier of the weights from sums over the processes, and returns the
forces its own atoms' energies put on every atom of its domain.  Summed over
the processes by global atom, energies, forces, virial and E_F equal the
oracle's single-process run of the whole structure.
"""
import os
import socket

import numpy as np
import pytest

from paper_1803_07491_gb300 import domain as D
from paper_1803_07491_gb300 import inputs as I
from conftest import oracle_model, oracle_settings


def _cell(model=I.MODEL_S, n3=10, sigma=0.05, seed=21):
    pos, cell = I.bcc_cell(3, 3, n3)
    rng = np.random.default_rng(seed)
    pos = I.jittered(pos, cell, (1, 1, 1), sigma, rng)
    return pos, cell, (1, 1, 1), model


def test_partition_owns_every_atom_once_and_halo_covers_clusters(ob):
    """Own atoms of all domains are the structure's atoms, each once; the
    moments of the own atoms computed on the domain equal those of the whole
    structure (the halo holds every cluster)."""
    pos, cell, pbc, model = _cell()
    m = oracle_model(model)
    K = 4
    nbr = ob.neighbors(pos, cell, pbc, m.rc)
    H = ob.blocks(m, pos, cell, nbr)
    mu_ref = ob.moments(nbr, H, np.zeros((len(pos), m.norb)), 2 * K + 1)
    owned = []
    for size in (2, 3):
        owned.clear()
        for rank in range(size):
            dom = D.decompose(pos, cell, pbc, size, rank, K * m.rc * (1 + 1e-9) + 1e-6)
            assert dom.pbc[dom.axis] == 0
            frac = np.linalg.solve(dom.cell.T, dom.pos.T).T
            assert frac.min() >= 0.0 and frac.max() < 1.0
            owned.extend(dom.gid[:dom.n_own].tolist())
            nl = ob.neighbors(dom.pos, dom.cell, dom.pbc, m.rc)
            Hl = ob.blocks(m, dom.pos, dom.cell, nl)
            sel = np.arange(dom.n_own, dtype=np.int32)
            mu = ob.moments(nl, Hl, np.zeros((len(dom.pos), m.norb)), 2 * K + 1, sel)
            assert np.allclose(mu, mu_ref[dom.gid[:dom.n_own]], rtol=1e-12, atol=1e-12)
        assert sorted(owned) == list(range(len(pos)))


def _rank_oracle(ob, model, st, dom, n_global, allreduce):
    """One process's share of the evaluation with the oracle's pieces."""
    s = 2.0
    m = oracle_model(model)
    nl = ob.neighbors(dom.pos, dom.cell, dom.pbc, m.rc)
    Hl = ob.blocks(m, dom.pos, dom.cell, nl)
    onsite = np.zeros((len(dom.pos), m.norb))
    sel = np.arange(dom.n_own, dtype=np.int32)
    mu = ob.moments(nl, Hl, onsite, st.n_mom, sel).reshape(-1, st.n_mom)
    ex = ob.scalar_stage(mu, st.n_exp)
    # one Fermi level: the oracle's bisection on the electron count of all processes
    lo = -allreduce(np.array([-np.min(ex.a_inf - 2.0 * ex.b_inf)]), "max")[0] - 1e-3
    hi = allreduce(np.array([np.max(ex.a_inf + 2.0 * ex.b_inf)]), "max")[0] + 1e-3
    target = st.n_e * n_global
    zero = np.zeros(len(mu))
    for _ in range(100):
        if hi - lo < 1e-13:
            break
        mid = 0.5 * (lo + hi)
        N, _ = ob.orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, zero, mid)
        f = s * allreduce(np.array([np.sum(N)]), "sum")[0] - target
        if f == 0.0:
            lo = hi = mid
            break
        if f < 0.0:
            lo = mid
        else:
            hi = mid
    E_F = 0.5 * (lo + hi)
    N, U = ob.orbital_N_U(ex.gsig, ex.a_inf, ex.b_inf, zero, E_F)
    e_own = s * U.reshape(dom.n_own, m.norb).sum(axis=1)
    # weights with the E_F multiplier of the whole structure
    _, _, dN, dN_dEF, dU_dEF, dU = ob.weights(mu, zero, E_F, st.n_exp, s)
    sums = allreduce(np.array([np.sum(dU_dEF), np.sum(dN_dEF)]), "sum")
    w = s * (dU - sums[0] / sums[1] * dN)
    Hbar, _ = ob.moments_adjoint(nl, Hl, onsite, w.reshape(dom.n_own, m.norb, st.n_mom), sel)
    g = ob.bond_gradient(m, dom.pos, dom.cell, nl, Hbar)
    F = np.zeros((len(dom.pos), 3))
    src = np.repeat(np.arange(len(dom.pos)), np.diff(nl.row_ptr))
    np.add.at(F, src, g)
    np.add.at(F, nl.col, -g)
    W = np.einsum("ea,eb->ab", g, ob.edge_vectors(dom.pos, dom.cell, nl))
    return E_F, e_own, F, W


def _worker(rank, size, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=size)
    try:
        from oracle import bop as ob
        ob.build()
        pos, cell, pbc, model = _cell()
        st = oracle_settings(I.RunParams(n_e=0.7))
        K = (st.n_mom - 1) // 2
        dom = D.decompose(pos, cell, pbc, size, rank, K * model.rc * (1 + 1e-9) + 1e-6)
        import torch

        def allreduce(a, op):
            t = torch.tensor(np.asarray(a, np.float64))
            dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
            return t.numpy()

        E_F, e_own, F_loc, W = _rank_oracle(ob, model, st, dom, len(pos), allreduce)
        e_atom = D.all_reduce_sum(D.gather_by_atom(e_own, dom.gid[:dom.n_own], len(pos)))
        F = D.all_reduce_sum(D.gather_by_atom(F_loc, dom.gid, len(pos)))
        W = D.all_reduce_sum(W)
        if rank == 0:
            np.savez(out_path, e_fermi=E_F, e_atom=e_atom, forces=F, virial=W)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_process_oracle_domains_match_single_process(ob, tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "dom.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    pos, cell, pbc, model = _cell()
    ref = ob.evaluate(oracle_model(model), oracle_settings(I.RunParams(n_e=0.7)), pos, cell, pbc)
    assert abs(float(got["e_fermi"]) - ref["e_fermi"]) < 1e-10
    assert np.max(np.abs(got["e_atom"] - ref["e_atom"])) < 1e-10
    assert np.max(np.abs(got["forces"] - ref["forces"])) < 1e-10
    assert np.max(np.abs(got["virial"] - ref["virial"])) < 1e-9
