"""Spatial decomposition of one structure over several processes.

The paper parallelises BOPfox by spatial domains, one per MPI process
(section "Performance", parallelisation).  Here every process owns the atoms
of one slab of the cell and builds its domain as one structure: its own
atoms first, then a halo of every atom (with the periodic image it needs)
within K r_cut of the slab along the decomposed direction, so that the
cluster of every own atom (K = (n_mom - 1)/2 hops of at most r_cut each)
lies inside the domain.  The library computes the clusters, moments,
electrons and energies of the own atoms only (bop_set_centers) and combines
its few global sums over the processes through a reduce function
(bop_set_reduce): the band edges and Newton sums of the one Fermi level, the
total energy and the E_F multiplier of the forces.  Each process's forces are
its own atoms' contributions to the forces on every atom of its domain; the
sum over the processes by global atom (the reverse halo exchange, here one
all-reduce of an [N][3] array) gives the forces of the whole structure.

This module holds the host-side partition and the collective glue; it does
no arithmetic of the method.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np


@dataclass
class Domain:
    rank: int
    size: int
    axis: int            # decomposed lattice direction
    pos: np.ndarray      # [n_local, 3] own atoms first, then the halo
    cell: np.ndarray     # [3, 3] rows; the decomposed vector stretched to a box around the domain
    pbc: tuple           # the decomposed direction is not periodic inside a domain
    n_own: int
    gid: np.ndarray      # [n_local] global index of every local atom


def plane_spacing(cell: np.ndarray, axis: int) -> float:
    """Distance between the lattice planes spanned by the two other cell
    vectors (the thickness of the cell along the normal of those planes)."""
    cell = np.asarray(cell, np.float64)
    b, c = cell[(axis + 1) % 3], cell[(axis + 2) % 3]
    return abs(float(np.linalg.det(cell))) / float(np.linalg.norm(np.cross(b, c)))


def choose_axis(cell: np.ndarray, pbc) -> int:
    """The direction with the largest plane spacing (periodic ones first)."""
    order = sorted(range(3), key=lambda a: (not pbc[a], -plane_spacing(cell, a)))
    return order[0]


def decompose(pos, cell, pbc, size: int, rank: int, halo: float, axis: int | None = None) -> Domain:
    """Domain of `rank` among `size` slabs of equal thickness along `axis`
    (fractional coordinate in [rank/size, (rank+1)/size)), with every atom
    image whose fractional coordinate along the axis lies within `halo`
    (Angstrom, along the plane normal) of the slab as halo.  Positions must
    lie inside the cell (fractional coordinates in [0, 1))."""
    pos = np.asarray(pos, np.float64)
    cell = np.asarray(cell, np.float64)
    if axis is None:
        axis = choose_axis(cell, pbc)
    frac = np.linalg.solve(cell.T, pos.T).T
    f = frac[:, axis]
    lo, hi = rank / size, (rank + 1) / size
    own = np.nonzero((f >= lo) & (f < hi))[0]
    h = halo / plane_spacing(cell, axis)
    shifts = range(-int(np.ceil(h)) - 1, int(np.ceil(h)) + 2) if pbc[axis] else (0,)
    hidx, hshift = [], []
    for m in shifts:
        fm = f + m
        sel = (fm >= lo - h) & (fm < hi + h)
        if m == 0:
            sel &= ~((f >= lo) & (f < hi))
        idx = np.nonzero(sel)[0]
        hidx.append(idx)
        hshift.append(np.full(len(idx), m))
    hidx = np.concatenate(hidx)
    hshift = np.concatenate(hshift)
    gid = np.concatenate([own, hidx]).astype(np.int64)
    shift = np.concatenate([np.zeros(len(own)), hshift])
    fl = f[gid] + shift
    # box along the axis around [lo - h, hi + h), with a margin so that every
    # atom lies strictly inside it
    margin = 1e-6 + 1e-3 * (hi - lo + 2 * h)
    start = lo - h - margin
    length = (hi - lo) + 2 * h + 2 * margin
    local_frac = frac[gid].copy()
    local_frac[:, axis] = (fl - start) / length
    lcell = cell.copy()
    lcell[axis] = cell[axis] * length
    lpos = local_frac @ lcell
    lpbc = tuple(0 if a == axis else int(pbc[a]) for a in range(3))
    return Domain(rank, size, axis, lpos, lcell, lpbc, len(own), gid)


def gather_by_atom(local: np.ndarray, gid: np.ndarray, n_global: int) -> np.ndarray:
    """Scatter-add rows of `local` into an [n_global, ...] array by global
    atom index (one process's share, summed over the processes by the
    caller's all-reduce)."""
    out = np.zeros((n_global,) + local.shape[1:], np.float64)
    np.add.at(out, gid, local)
    return out


def torch_reduce_fn(group=None):
    """A bop_reduce_fn that all-reduces over a torch.distributed group (gloo:
    CPU tensors; NCCL: the current CUDA device)."""
    import torch
    import torch.distributed as dist

    from .bop import BOP_REDUCE_MAX, REDUCE_FN

    def fn(values, count, op, user):
        try:
            a = np.ctypeslib.as_array(values, shape=(count,))
            backend = dist.get_backend(group)
            dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
            t = torch.tensor(a, dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX if op == BOP_REDUCE_MAX else dist.ReduceOp.SUM, group=group)
            a[:] = t.cpu().numpy()
            return 0
        except Exception:  # reported to the library as BOP_ERR_COLLECTIVE
            return 1

    return REDUCE_FN(fn)


def all_reduce_sum(a: np.ndarray, group=None) -> np.ndarray:
    import torch
    import torch.distributed as dist
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor(a, dtype=torch.float64, device=dev)
    dist.all_reduce(t, group=group)
    return t.cpu().numpy()


def evaluate(params, run, precision: str, pos, cell, pbc, group=None, axis: int | None = None):
    """Energy per atom, total energy, forces and virial of the whole
    structure from this process's domain (torch.distributed initialised,
    one process per domain).  Returns numpy arrays of the whole structure on
    every process and the Fermi level."""
    import torch
    import torch.distributed as dist

    from . import bop
    size, rank = dist.get_world_size(group), dist.get_rank(group)
    n = len(pos)
    K = (run.n_mom - 1) // 2
    dom = decompose(pos, cell, pbc, size, rank, K * params.rc * (1.0 + 1e-9) + 1e-6, axis)
    ctx = bop.Context(params, run, precision)
    red = torch_reduce_fn(group)
    try:
        bop.bop_set_centers(ctx.h, dom.n_own)
        bop.bop_set_reduce(ctx.h, red)
        ctx.build(dom.pos, dom.cell, dom.pbc)
        e_loc, st = ctx.energy()
        F_loc, W_loc = ctx.forces()
        e_atom = all_reduce_sum(gather_by_atom(e_loc.cpu().numpy()[:dom.n_own], dom.gid[:dom.n_own], n), group)
        F = all_reduce_sum(gather_by_atom(F_loc.cpu().numpy(), dom.gid, n), group)
        W = all_reduce_sum(W_loc.cpu().numpy(), group)
        torch.cuda.synchronize()
        return dict(e_atom=e_atom, e_total=st["e_total"], forces=F, virial=W, e_fermi=st["e_fermi"],
                    n_local=len(dom.gid), n_own=dom.n_own)
    finally:
        bop.bop_set_reduce(ctx.h, None)
        ctx.close()
