"""Thin ctypes binding of libbopgb (include/bopgb.h).

Argument marshalling only: every step of the BOP path runs in the CUDA
kernels of libbopgb.so.  PyTorch provides device memory and the current
stream.  There is no CPU fallback: a missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

BOP_OK, BOP_ERR_ARG, BOP_ERR_CUDA, BOP_ERR_OOM, BOP_ERR_NO_CONVERGENCE = 0, 1, 2, 3, 4
BOP_ERR_BRACKET, BOP_ERR_NUMERIC, BOP_ERR_STATE, BOP_ERR_OVERFLOW = 5, 6, 7, 8
BOP_ERR_COLLECTIVE = 9
BOP_REDUCE_SUM, BOP_REDUCE_MAX = 0, 1
# bop_reduce_fn: int (*)(double* values, int count, int op, void* user)
REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                             ctypes.c_void_p)
SCF = {"none": 0, "lcn": 1, "stoner": 2, "variational": 3}
PREC = {"fp64": 0, "fp32": 1}
MIXER = {"linear": 0, "anderson": 1}
TERM = {"constant": 0, "mlp": 1}
BANDWIDTH = {"gershgorin": 0, "lowest": 1, "highest": 2, "average": 3, "average_centre": 4, "minmax": 5,
             "global": 6, "weighted": 7}
MLP_NIN, MLP_NHID, MLP_NOUT, MLP_NPARAM, MLP_NNORM = 18, 128, 10, 20234, 92


class BopError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libbopgb status {status}: {msg}")
        self.status = status


class bop_model(ctypes.Structure):
    _fields_ = [("norb", ctypes.c_int), ("b0", ctypes.c_double * 5), ("r0", ctypes.c_double),
                ("lam", ctypes.c_double), ("rc", ctypes.c_double), ("dc", ctypes.c_double),
                ("onsite0", ctypes.c_double), ("n_mom", ctypes.c_int), ("n_exp", ctypes.c_int),
                ("n_spin", ctypes.c_int), ("n_e", ctypes.c_double), ("scf", ctypes.c_int),
                ("eta", ctypes.c_double), ("scf_tol", ctypes.c_double), ("scf_max_it", ctypes.c_int),
                ("stoner_I", ctypes.c_double), ("m_mix", ctypes.c_double), ("m0", ctypes.c_double),
                ("dos_floor", ctypes.c_double), ("precision", ctypes.c_int), ("mixer", ctypes.c_int),
                ("mix_history", ctypes.c_int), ("terminator", ctypes.c_int), ("scf_response", ctypes.c_int),
                ("bandwidth", ctypes.c_int), ("bw_beta", ctypes.c_double), ("bw_a", ctypes.c_double),
                ("bw_b", ctypes.c_double), ("j_ii", ctypes.c_double), ("rep_A", ctypes.c_double),
                ("rep_p", ctypes.c_double), ("r_path", ctypes.c_double), ("onsite_s", ctypes.c_double),
                ("noncollinear", ctypes.c_int)]


class bop_stats(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("K", ctypes.c_int), ("n_edges", ctypes.c_longlong),
                ("n_bonds", ctypes.c_longlong), ("n_sites", ctypes.c_longlong), ("n_adj", ctypes.c_longlong),
                ("max_cluster", ctypes.c_int), ("scf_iterations", ctypes.c_int), ("scf_converged", ctypes.c_int),
                ("bisection_rounds", ctypes.c_int), ("scf_residual", ctypes.c_double),
                ("e_fermi", ctypes.c_double), ("e_total", ctypes.c_double),
                ("forces_scf_response", ctypes.c_int), ("n_learned", ctypes.c_int),
                ("moment_products", ctypes.c_longlong), ("response_iterations", ctypes.c_int),
                ("response_converged", ctypes.c_int), ("response_residual", ctypes.c_double),
                ("n_unbounded", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bop_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong), ("regions", ctypes.c_longlong),
                ("ms", ctypes.c_double)]


_LIB = None
_VP = ctypes.c_void_p


def lib(path: str | None = None):
    """Load libbopgb.so (built in-tree by paper_1803_07491_gb300.build)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1803_07491_gb300.build.build(); "
                           "the BOP path has no CPU fallback")
    L = ctypes.CDLL(path)
    sig = {
        "bop_version": ([], ctypes.c_int),
        "bop_create": ([ctypes.POINTER(_VP), ctypes.POINTER(bop_model)], ctypes.c_int),
        "bop_destroy": ([_VP], ctypes.c_int),
        "bop_last_error": ([_VP], ctypes.c_char_p),
        "bop_build_hamiltonian": ([_VP, ctypes.c_int, _VP, _VP, _VP, _VP], ctypes.c_int),
        "bop_get_stats": ([_VP, ctypes.POINTER(bop_stats)], ctypes.c_int),
        "bop_get_neighbors": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
        "bop_get_cluster": ([_VP, ctypes.c_int, _VP, _VP, _VP, _VP], ctypes.c_int),
        "bop_get_bonds": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
        "bop_moments": ([_VP, _VP, _VP, _VP], ctypes.c_int),
        "bop_recursion": ([_VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
        "bop_energy": ([_VP, _VP, _VP, _VP, ctypes.POINTER(bop_stats), _VP], ctypes.c_int),
        "bop_forces": ([_VP, _VP, _VP, ctypes.POINTER(bop_stats), _VP], ctypes.c_int),
        "bop_get_orbital_state": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
        "bop_evaluate_host": ([_VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                               ctypes.POINTER(bop_stats), _VP], ctypes.c_int),
        "bop_fermi_level_noalloc": ([ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, ctypes.c_double,
                                     ctypes.c_double, _VP, _VP], ctypes.c_int),
        "bop_set_profiling": ([_VP, ctypes.c_int], ctypes.c_int),
        "bop_mlp_create": ([ctypes.POINTER(_VP), _VP], ctypes.c_int),
        "bop_mlp_destroy": ([_VP], ctypes.c_int),
        "bop_mlp_last_error": ([_VP], ctypes.c_char_p),
        "bop_mlp_get": ([_VP, _VP, _VP], ctypes.c_int),
        "bop_mlp_set_norm": ([_VP, _VP], ctypes.c_int),
        "bop_mlp_dataset": ([ctypes.c_longlong, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
        "bop_mlp_fit_norm": ([_VP, ctypes.c_longlong, _VP, _VP, _VP, _VP], ctypes.c_int),
        "bop_mlp_gradient": ([_VP, ctypes.c_longlong, _VP, _VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP],
                             ctypes.c_int),
        "bop_mlp_adam": ([_VP, ctypes.c_float, _VP], ctypes.c_int),
        "bop_mlp_check": ([_VP, _VP], ctypes.c_int),
        "bop_mlp_train_step": ([_VP, ctypes.c_longlong, _VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_float, _VP,
                                _VP], ctypes.c_int),
        "bop_mlp_predict": ([_VP, ctypes.c_longlong, _VP, _VP, _VP], ctypes.c_int),
        "bop_set_mlp": ([_VP, _VP], ctypes.c_int),
        "bop_set_store_budget": ([_VP, ctypes.c_longlong], ctypes.c_int),
        "bop_set_response_limits": ([_VP, ctypes.c_int, ctypes.c_double], ctypes.c_int),
        "bop_set_centers": ([_VP, ctypes.c_int], ctypes.c_int),
        "bop_set_reduce": ([_VP, REDUCE_FN, _VP], ctypes.c_int),
        "bop_set_spin_directions": ([_VP, _VP, _VP], ctypes.c_int),
        "bop_torques": ([_VP, _VP, _VP], ctypes.c_int),
        "bop_md_verlet": ([ctypes.c_int, _VP, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                           _VP], ctypes.c_int),
        "bop_reset_profile": ([_VP], ctypes.c_int),
        "bop_get_profile": ([_VP, ctypes.POINTER(bop_kernel_time), ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
                            ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _LIB = L
    return L


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        assert t.is_contiguous(), "tensors passed to libbopgb must be contiguous"
        return _VP(t.data_ptr())
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data_as(_VP)
    raise TypeError(type(t))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _VP(s.cuda_stream)


def make_model(params, run, precision: str = "fp64") -> bop_model:
    """bop_model from inputs.ModelParams + inputs.RunParams."""
    b0 = list(params.b0) + [0.0] * (5 - len(params.b0))
    return bop_model(params.norb, (ctypes.c_double * 5)(*b0), params.r0, params.lam, params.rc, params.dc,
                     params.onsite0, run.n_mom, run.n_exp, run.n_spin, run.n_e, SCF[run.scf], run.eta,
                     run.scf_tol, run.scf_max_it, run.stoner_I, run.m_mix, run.m0, run.dos_floor,
                     PREC[precision], MIXER[run.mixer], run.mix_history, TERM[run.terminator],
                     1 if run.scf_response else 0, BANDWIDTH[run.bandwidth], run.bw_beta, run.bw_a, run.bw_b,
                     run.J_ii, params.rep_A, params.rep_p, run.r_path, params.onsite_s,
                     1 if run.noncollinear else 0)


def _check(ctx, st, allow=()):
    if st != BOP_OK and st not in allow:
        msg = lib().bop_last_error(ctx)
        raise BopError(st, msg.decode() if msg else "")
    return st


# ------------------------------------------------------------ ABI mirrors

def bop_create(model: bop_model):
    h = _VP()
    st = lib().bop_create(ctypes.byref(h), ctypes.byref(model))
    if st != BOP_OK:
        raise BopError(st, "bop_create rejected the model")
    return h


def bop_destroy(ctx):
    lib().bop_destroy(ctx)


def bop_build_hamiltonian(ctx, pos: torch.Tensor, cell, pbc, stream=None):
    cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(3, 3)
    pbc = np.ascontiguousarray(pbc, dtype=np.int32).reshape(3)
    assert pos.is_cuda and pos.dtype == torch.float64 and pos.shape[-1] == 3
    _check(ctx, lib().bop_build_hamiltonian(ctx, pos.shape[0], _ptr(pos), _ptr(cell), _ptr(pbc), _stream(stream)))


def bop_get_stats(ctx) -> dict:
    s = bop_stats()
    _check(ctx, lib().bop_get_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


def bop_get_neighbors(ctx, stream=None):
    st = bop_get_stats(ctx)
    n, E = st["n_atoms"], st["n_edges"]
    dev = torch.device("cuda")
    row = torch.empty(n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(E, 1), dtype=torch.int32, device=dev)
    img = torch.empty((max(E, 1), 3), dtype=torch.int8, device=dev)
    _check(ctx, lib().bop_get_neighbors(ctx, _ptr(row), _ptr(col), _ptr(img), _stream(stream)))
    return row, col[:E], img[:E]


def bop_get_cluster(ctx, atom: int, K: int, max_sites: int, stream=None):
    dev = torch.device("cuda")
    sa = torch.empty(max_sites, dtype=torch.int32, device=dev)
    si = torch.empty((max_sites, 3), dtype=torch.int8, device=dev)
    lev = torch.empty(K + 1, dtype=torch.int32, device=dev)
    _check(ctx, lib().bop_get_cluster(ctx, atom, _ptr(sa), _ptr(si), _ptr(lev), _stream(stream)))
    ns = int(lev[-1].item())
    return sa[:ns], si[:ns], lev


def bop_get_bonds(ctx, norb: int, stream=None):
    st = bop_get_stats(ctx)
    nb = st["n_bonds"]
    dev = torch.device("cuda")
    hs = {1: 1, 5: 15, 6: 21}[norb]
    atoms = torch.empty((max(nb, 1), 2), dtype=torch.int32, device=dev)
    d = torch.empty((max(nb, 1), 3), dtype=torch.float64, device=dev)
    blk = torch.empty((max(nb, 1), hs), dtype=torch.float64, device=dev)
    _check(ctx, lib().bop_get_bonds(ctx, _ptr(atoms), _ptr(d), _ptr(blk), _stream(stream)))
    return atoms[:nb], d[:nb], blk[:nb]


def bop_moments(ctx, n_spin: int, n: int, norb: int, n_mom: int, onsite=None, stream=None):
    mu = torch.empty((n_spin, n, norb, n_mom), dtype=torch.float64, device="cuda")
    _check(ctx, lib().bop_moments(ctx, _ptr(onsite), _ptr(mu), _stream(stream)))
    return mu


def bop_recursion(ctx, mu: torch.Tensor, n_exp: int, stream=None):
    """Scalar stage of M orbitals: returns a, b, nlev, a_inf, b_inf, gsig [M][n_exp+1]."""
    M, n_mom = mu.shape
    Kp = (n_mom - 1) // 2
    dev = mu.device
    a = torch.empty((M, Kp), dtype=torch.float64, device=dev)
    b = torch.empty((M, Kp + 1), dtype=torch.float64, device=dev)
    nlev = torch.empty(M, dtype=torch.int32, device=dev)
    ai = torch.empty(M, dtype=torch.float64, device=dev)
    bi = torch.empty(M, dtype=torch.float64, device=dev)
    gs = torch.empty((n_exp + 1, M), dtype=torch.float64, device=dev)
    _check(ctx, lib().bop_recursion(ctx, M, _ptr(mu.contiguous()), _ptr(a), _ptr(b), _ptr(nlev), _ptr(ai),
                                    _ptr(bi), _ptr(gs), _stream(stream)))
    return a, b, nlev, ai, bi, gs.t().contiguous()


def bop_energy(ctx, n: int, delta=None, m=None, stream=None, allow_noconv=False):
    e = torch.empty(n, dtype=torch.float64, device="cuda")
    s = bop_stats()
    _check(ctx, lib().bop_energy(ctx, _ptr(e), _ptr(delta), _ptr(m), ctypes.byref(s), _stream(stream)),
           allow=(BOP_ERR_NO_CONVERGENCE,) if allow_noconv else ())
    return e, s.as_dict()


def bop_forces(ctx, n: int, stream=None):
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    W = torch.empty((3, 3), dtype=torch.float64, device="cuda")
    s = bop_stats()
    _check(ctx, lib().bop_forces(ctx, _ptr(F), _ptr(W), ctypes.byref(s), _stream(stream)))
    return F, W


def bop_set_spin_directions(ctx, sdir, stream=None):
    """Moment directions [n][3] of a non-collinear model (device float64)."""
    sdir = torch.as_tensor(sdir, dtype=torch.float64, device="cuda").contiguous()
    _check(ctx, lib().bop_set_spin_directions(ctx, _ptr(sdir), _stream(stream)))


def bop_torques(ctx, n: int, stream=None):
    t = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    _check(ctx, lib().bop_torques(ctx, _ptr(t), _stream(stream)))
    return t


def bop_forces_stats(ctx, n: int, stream=None, allow_noconv=False):
    """bop_forces plus its statistics (SCF-response solve).  allow_noconv:
    a response solve stopped at its limit returns the forces of its last
    iterate instead of raising."""
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    W = torch.empty((3, 3), dtype=torch.float64, device="cuda")
    s = bop_stats()
    _check(ctx, lib().bop_forces(ctx, _ptr(F), _ptr(W), ctypes.byref(s), _stream(stream)),
           allow=(BOP_ERR_NO_CONVERGENCE,) if allow_noconv else ())
    return F, W, s.as_dict()


def bop_get_orbital_state(ctx, M: int, n_mom: int, weights=False, stream=None):
    dev = torch.device("cuda")
    out = {k: torch.empty(M, dtype=torch.float64, device=dev) for k in ("N", "U", "a_inf", "b_inf", "onsite")}
    out["mu"] = torch.empty((M, n_mom), dtype=torch.float64, device=dev)
    out["weights"] = torch.empty((M, n_mom), dtype=torch.float64, device=dev) if weights else None
    _check(ctx, lib().bop_get_orbital_state(ctx, _ptr(out["mu"]), _ptr(out["N"]), _ptr(out["U"]),
                                            _ptr(out["a_inf"]), _ptr(out["b_inf"]), _ptr(out["weights"]),
                                            _ptr(out["onsite"]), _stream(stream)))
    return out


def bop_evaluate_host(ctx, pos_host: torch.Tensor, cell, pbc, e_atom_host=None, forces_host=None,
                      virial_host=None, stream=None):
    """End-to-end E+F through host buffers (pinned tensors recommended)."""
    cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(3, 3)
    pbc = np.ascontiguousarray(pbc, dtype=np.int32).reshape(3)
    et = ctypes.c_double(0.0)
    s = bop_stats()
    _check(ctx, lib().bop_evaluate_host(ctx, pos_host.shape[0], _ptr(pos_host), _ptr(cell), _ptr(pbc),
                                        _ptr(e_atom_host), _ptr(forces_host), _ptr(virial_host),
                                        ctypes.cast(ctypes.pointer(et), _VP), ctypes.byref(s), _stream(stream)))
    return et.value, s.as_dict()


def bop_md_verlet(pos, vel: torch.Tensor, forces: torch.Tensor, dt: float, mass: float, phase: int,
                  cell=None, pbc=None, stream=None):
    """Half of a velocity-Verlet step in place (phase 0: kick + drift, 1:
    kick); with cell and pbc, atoms that left the cell are moved back."""
    c = None if cell is None else np.ascontiguousarray(cell, dtype=np.float64).reshape(3, 3)
    p = None if pbc is None else np.ascontiguousarray(pbc, dtype=np.int32).reshape(3)
    st = lib().bop_md_verlet(vel.shape[0], _ptr(pos), _ptr(vel), _ptr(forces), _ptr(c), _ptr(p), dt, mass, phase,
                             _stream(stream))
    if st != BOP_OK:
        raise BopError(st, "bop_md_verlet rejected its arguments")


def bop_fermi_level_noalloc(gsig_cm: torch.Tensor, a_inf: torch.Tensor, b_inf: torch.Tensor,
                            spin_factor: float, n_electrons: float, e_fermi: torch.Tensor, stream=None) -> int:
    """Fermi level without device allocation (scratch in a static device
    array).  gsig_cm: [n_exp+1][M] coefficient-major.  Returns the status;
    e_fermi (device, 1 element) holds the result on success."""
    n_exp = gsig_cm.shape[0] - 1
    M = gsig_cm.shape[1]
    return lib().bop_fermi_level_noalloc(M, n_exp, _ptr(gsig_cm), _ptr(a_inf), _ptr(b_inf), spin_factor,
                                         n_electrons, _ptr(e_fermi), _stream(stream))


def bop_set_profiling(ctx, on: bool):
    _check(ctx, lib().bop_set_profiling(ctx, 1 if on else 0))


def bop_reset_profile(ctx):
    _check(ctx, lib().bop_reset_profile(ctx))


def bop_get_profile(ctx) -> dict:
    """{family: {"launches", "regions", "ms"}} of the timed launch regions."""
    arr = (bop_kernel_time * 32)()
    n = ctypes.c_int(0)
    _check(ctx, lib().bop_get_profile(ctx, arr, 32, ctypes.byref(n)))
    return {arr[i].name.decode(): {"launches": arr[i].launches, "regions": arr[i].regions, "ms": arr[i].ms}
            for i in range(n.value)}


# ------------------------------------------------------------ learned terminator

def _mcheck(net, st):
    if st != BOP_OK:
        msg = lib().bop_mlp_last_error(net) if net else b""
        raise BopError(st, msg.decode() if msg else "")
    return st


def bop_mlp_create(params) -> _VP:
    p = np.ascontiguousarray(params, dtype=np.float32).reshape(MLP_NPARAM)
    h = _VP()
    st = lib().bop_mlp_create(ctypes.byref(h), _ptr(p))
    if st != BOP_OK:
        raise BopError(st, "bop_mlp_create failed")
    return h


def bop_mlp_destroy(net):
    lib().bop_mlp_destroy(net)


def bop_mlp_get(net):
    p = np.zeros(MLP_NPARAM, np.float32)
    q = np.zeros(MLP_NNORM, np.float32)
    _mcheck(net, lib().bop_mlp_get(net, _ptr(p), _ptr(q)))
    return p, q


def bop_mlp_set_norm(net, norm):
    q = np.ascontiguousarray(norm, dtype=np.float32).reshape(MLP_NNORM)
    _mcheck(net, lib().bop_mlp_set_norm(net, _ptr(q)))


def bop_mlp_dataset(mu17: torch.Tensor, stream=None):
    """Raw inputs x [M][18], targets t [M][10] and mask [M] (device FP32)
    from 17-moment runs mu17 [M][17] (device FP64)."""
    mu17 = mu17.reshape(-1, 17).contiguous()
    M = mu17.shape[0]
    x = torch.empty((M, MLP_NIN), dtype=torch.float32, device=mu17.device)
    t = torch.empty((M, MLP_NOUT), dtype=torch.float32, device=mu17.device)
    m = torch.empty(M, dtype=torch.float32, device=mu17.device)
    st = lib().bop_mlp_dataset(M, _ptr(mu17), _ptr(x), _ptr(t), _ptr(m), _stream(stream))
    if st != BOP_OK:
        raise BopError(st, "bop_mlp_dataset failed")
    return x, t, m


def bop_mlp_fit_norm(net, x, t, mask, stream=None):
    _mcheck(net, lib().bop_mlp_fit_norm(net, x.shape[0], _ptr(x), _ptr(t), _ptr(mask), _stream(stream)))


def bop_mlp_gradient(net, x, t, mask, idx: torch.Tensor, grad_out=None, loss_out=None, stream=None):
    _mcheck(net, lib().bop_mlp_gradient(net, x.shape[0], _ptr(x), _ptr(t), _ptr(mask), _ptr(idx),
                                        idx.shape[0], _ptr(grad_out), _ptr(loss_out), _stream(stream)))


def bop_mlp_adam(net, lr: float, stream=None):
    _mcheck(net, lib().bop_mlp_adam(net, lr, _stream(stream)))


def bop_mlp_train_step(net, x, t, mask, idx: torch.Tensor, lr: float, loss_out=None, stream=None):
    _mcheck(net, lib().bop_mlp_train_step(net, x.shape[0], _ptr(x), _ptr(t), _ptr(mask), _ptr(idx),
                                          idx.shape[0], lr, _ptr(loss_out), _stream(stream)))


def bop_mlp_predict(net, x: torch.Tensor, stream=None) -> torch.Tensor:
    y = torch.empty((x.shape[0], MLP_NOUT), dtype=torch.float32, device=x.device)
    _mcheck(net, lib().bop_mlp_predict(net, x.shape[0], _ptr(x), _ptr(y), _stream(stream)))
    return y


def bop_set_response_limits(ctx, max_iterations: int = 0, rtol: float = 0.0):
    _check(ctx, lib().bop_set_response_limits(ctx, int(max_iterations), float(rtol)))


def bop_set_centers(ctx, n_centers: int):
    _check(ctx, lib().bop_set_centers(ctx, int(n_centers)))


def bop_set_reduce(ctx, fn):
    """fn: a REDUCE_FN (kept alive by the caller), or None for one process."""
    _check(ctx, lib().bop_set_reduce(ctx, fn if fn is not None else REDUCE_FN(), None))


def bop_set_store_budget(ctx, nbytes: int):
    _check(ctx, lib().bop_set_store_budget(ctx, int(nbytes)))


def bop_set_mlp(ctx, net):
    _check(ctx, lib().bop_set_mlp(ctx, net))


class Network:
    """A learned-terminator network on the current device (bop_mlp)."""

    def __init__(self, params):
        self.h = bop_mlp_create(params)

    def close(self):
        if self.h:
            bop_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self):
        return bop_mlp_get(self.h)

    def set_norm(self, norm):
        bop_mlp_set_norm(self.h, norm)

    def fit_norm(self, x, t, mask):
        bop_mlp_fit_norm(self.h, x, t, mask)

    def train(self, x, t, mask, epochs: int, batch: int, lr: float, seed: int, lr_final: float | None = None,
              stream=None):
        """Mini-batch Adam over the rows with mask 1 of (x, t): each epoch a
        permutation drawn from default_rng(seed) (one draw per epoch); the
        learning rate decays geometrically from lr to lr_final.  Returns the
        mean batch loss of every epoch (one synchronisation per epoch)."""
        rows = torch.nonzero(mask > 0).flatten().to(torch.int32)
        n = rows.numel()
        rng = np.random.default_rng(seed)
        losses = torch.zeros(max(1, (n + batch - 1) // batch), dtype=torch.float32, device=x.device)
        out = []
        lr_final = lr if lr_final is None else lr_final
        for ep in range(epochs):
            perm = torch.as_tensor(rng.permutation(n), device=x.device)
            order = rows[perm].contiguous()
            f = ep / max(1, epochs - 1)
            lr_ep = lr * (lr_final / lr) ** f
            nb = 0
            for b0 in range(0, n - batch + 1, batch):
                bop_mlp_train_step(self.h, x, t, mask, order[b0:b0 + batch], lr_ep, losses[nb:nb + 1], stream)
                nb += 1
            out.append(float(losses[:nb].mean().item()))
        _mcheck(self.h, lib().bop_mlp_check(self.h, _stream(stream)))
        return out


# ------------------------------------------------------------ convenience

@dataclass
class Result:
    e_atom: torch.Tensor
    e_total: float
    e_fermi: float
    forces: torch.Tensor | None
    virial: torch.Tensor | None
    stats: dict
    torques: torch.Tensor | None = None


class Context:
    """One model on the current CUDA device; owns a libbopgb context."""

    def __init__(self, params, run, precision: str = "fp64", net: Network | None = None):
        self.params, self.run, self.precision = params, run, precision
        self.model = make_model(params, run, precision)
        self.h = bop_create(self.model)
        self.n = 0
        self.net = net
        if net is not None:
            bop_set_mlp(self.h, net.h)

    def close(self):
        if self.h:
            bop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, pos, cell, pbc, stream=None):
        pos = torch.as_tensor(pos, dtype=torch.float64, device="cuda").contiguous()
        bop_build_hamiltonian(self.h, pos, cell, pbc, stream)
        self.n = pos.shape[0]
        return bop_get_stats(self.h)

    def energy(self, delta=None, m=None, stream=None, allow_noconv=False):
        return bop_energy(self.h, self.n, delta, m, stream, allow_noconv)

    def forces(self, stream=None):
        return bop_forces(self.h, self.n, stream)

    def md_step(self, pos, vel, forces, cell, pbc, dt: float, mass: float, delta=None, stream=None):
        """One velocity-Verlet MD step on the device: kick + drift, new
        Hamiltonian, energy (warm-started from `delta`, the previous step's
        shifts, updated in place), forces into `forces`, kick.  pos, vel,
        forces: device [n][3] float64.  Returns (e_atom, stats)."""
        bop_md_verlet(pos, vel, forces, dt, mass, 0, cell, pbc, stream)
        bop_build_hamiltonian(self.h, pos, cell, pbc, stream)
        self.n = pos.shape[0]
        e, st = bop_energy(self.h, self.n, delta, None, stream)
        s = bop_stats()
        _check(self.h, lib().bop_forces(self.h, _ptr(forces), None, ctypes.byref(s), _stream(stream)))
        bop_md_verlet(None, vel, forces, dt, mass, 1, stream=stream)
        return e, st

    def set_spin_directions(self, sdir, stream=None):
        bop_set_spin_directions(self.h, sdir, stream)

    def torques(self, stream=None):
        return bop_torques(self.h, self.n, stream)

    def evaluate(self, pos, cell, pbc, forces=True, spin_dir=None, m=None) -> Result:
        """Energy (and forces, virial; torques of a non-collinear model,
        whose moment directions spin_dir [n][3] are set after the build;
        m: moment magnitudes, the start of a Stoner SCF or fixed without
        one)."""
        self.build(pos, cell, pbc)
        if spin_dir is not None:
            self.set_spin_directions(spin_dir)
        if m is not None:
            m = torch.as_tensor(m, dtype=torch.float64, device="cuda").clone()
        e, st = self.energy(m=m)
        F = W = T = None
        if forces:
            F, W = self.forces()
            if self.run.noncollinear:
                T = self.torques()
        return Result(e, st["e_total"], st["e_fermi"], F, W, st, T)


class BopEnergy(torch.autograd.Function):
    """E_total(pos, cell) with the exact gradient from the adjoint kernels.

    forward: bop_build_hamiltonian + bop_energy + bop_forces; backward:
    dE/dpos = -F, and when the cell is a tensor dE/dcell at fixed Cartesian
    positions from the virial (Eq. sigma_k): with bond vectors
    d = r_j - r_i + sum_c S_c cell[c], W_ab = sum_bonds g_a d_b =
    sum_i (dE/dr_i)_a r_ib + sum_c (dE/dcell[c])_a cell[c]_b, so
    dE/dcell = (cell^-1)^T (W + F^T pos)^T.  Both scaled by the incoming
    gradient.  cell: [3][3] rows (numpy, a list or a tensor)."""

    @staticmethod
    def forward(actx, pos, ctx: Context, cell, pbc):
        cell_is_tensor = torch.is_tensor(cell)
        cell_np = cell.detach().cpu().numpy() if cell_is_tensor else np.asarray(cell, np.float64)
        ctx.build(pos.detach(), cell_np, pbc)
        e, st = ctx.energy()
        F, W = ctx.forces()
        actx.cell_is_tensor = cell_is_tensor
        actx.cell_meta = (cell.device, cell.dtype) if cell_is_tensor else None
        actx.save_for_backward(F, W, pos.detach(), torch.as_tensor(cell_np, dtype=torch.float64, device=pos.device))
        return torch.as_tensor(st["e_total"], dtype=torch.float64, device=pos.device)

    @staticmethod
    def backward(actx, g):
        F, W, pos, cell = actx.saved_tensors
        g_cell = None
        if actx.cell_is_tensor:
            dE_dcell_T = (W + F.T @ pos) @ torch.linalg.inv(cell)
            dev, dt = actx.cell_meta
            g_cell = (dE_dcell_T.T * g).to(device=dev, dtype=dt)
        return -F * g, None, g_cell, None
