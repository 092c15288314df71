/*
 * bopgb — GB300 (sm_103a) analytic bond-order potential, C ABI.
 *
 * The library computes, for one atomic structure, the hot path of the
 * analytic BOP described in the BOPfox paper (arXiv:1803.07491):
 *   short-range neighbour list ("Initialisation")
 *   -> two-centre Slater-Koster Hamiltonian blocks (Eq. Hij, Eq. cutoff,
 *      Eq. Hij_rot)
 *   -> moments mu_n(i alpha) = <i alpha|H^n|i alpha> of every orbital
 *      (Eq. momDOS) by the iterated interference paths (Eqs. xi_rec,
 *      xi_merge) over each atom's cluster
 *   -> recursion coefficients (Eqs. momtoa, momtob), Gershgorin band edges
 *      (Eq. gershogorin), constant terminator (Eq. abinf), expansion
 *      coefficients (Eq. sigma_i, Eq. aexp) with Jackson damping
 *      (Eq. Jackson)
 *   -> Fermi level by bisection ("DOS and Fermi energy"), local charge
 *      neutrality (Eq. BOP_LCN) and collinear Stoner magnetism
 *      (Eq. onsite_NCM, Eq. TB-UX) self-consistency
 *   -> bond energy per atom (Eq. TB-Ubond in the closed form of Eq. chi)
 *   -> exact gradient: weights (Eq. weights), reverse sweep of the moments
 *      (Eqs. theta-tilde, Xi), forces (Eq. F_k) and virial (Eq. sigma_k).
 *
 * Conventions (all entry points):
 *   - Every function returns an int status (enum bop_status); 0 = success.
 *     On failure bop_last_error(ctx) describes the cause.  Outputs are
 *     valid only on success, except BOP_ERR_NO_CONVERGENCE, where they hold
 *     the last iterate.
 *   - Array arguments are DEVICE pointers unless the parameter name ends
 *     in _host.  The caller owns every array it passes; the library owns
 *     only the workspaces inside the opaque context (allocated with
 *     cudaMalloc on the current device, freed by bop_destroy).
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it; functions that must read sizes or convergence flags
 *     synchronise that stream, as stated per function.
 *   - Energies in eV, lengths in Angstrom, forces in eV/Angstrom.
 *   - Orbitals: s (1) or d (5, order d_{3z^2-r^2}, d_zx, d_yz,
 *     d_{x^2-y^2}, d_xy as in Eq. Hij).  "M" below = n_spin * n * norb.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef BOPGB_H
#define BOPGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bop_ctx bop_ctx;
typedef struct bop_mlp bop_mlp;
typedef void* bop_stream; /* cudaStream_t */

enum bop_status {
  BOP_OK = 0,
  BOP_ERR_ARG = 1,            /* invalid argument or model */
  BOP_ERR_CUDA = 2,           /* a CUDA call failed */
  BOP_ERR_OOM = 3,            /* device allocation failed */
  BOP_ERR_NO_CONVERGENCE = 4, /* SCF hit scf_max_it; outputs = last iterate */
  BOP_ERR_BRACKET = 5,        /* Fermi level could not be bracketed */
  BOP_ERR_NUMERIC = 6,        /* NaN/Inf in the scalar stages */
  BOP_ERR_STATE = 7,          /* call order violated (e.g. forces before energy) */
  BOP_ERR_OVERFLOW = 8,       /* neighbour degree / cluster / image index limit exceeded */
  BOP_ERR_COLLECTIVE = 9      /* the reduce function of bop_set_reduce reported a failure */
};

/* Reductions over the processes of a spatial decomposition (bop_set_reduce). */
enum { BOP_REDUCE_SUM = 0, BOP_REDUCE_MAX = 1 };
/* Replaces values[0..count) on every process by their sum (op
 * BOP_REDUCE_SUM) or maximum (BOP_REDUCE_MAX) over all processes, in place;
 * host memory; returns 0 on success.  Every process calls it the same number
 * of times in the same order. */
typedef int (*bop_reduce_fn)(double* values, int count, int op, void* user);

enum { BOP_SCF_NONE = 0, BOP_SCF_LCN = 1, BOP_SCF_STONER = 2, BOP_SCF_VARIATIONAL = 3 };
enum { BOP_PREC_FP64 = 0, BOP_PREC_FP32 = 1 };
enum { BOP_MIX_LINEAR = 0, BOP_MIX_ANDERSON = 1 };
enum { BOP_TERM_CONSTANT = 0, BOP_TERM_MLP = 1 };
/* Band centre / width estimate (A, B) of the constant terminator (section
 * "Band-width estimates"; L = levels computed for the orbital, a_0..a_{L-1},
 * b_1..b_L): */
enum {
  BOP_BW_GERSHGORIN = 0,  /* (vii) Eq. gershogorin band edges (default) */
  BOP_BW_LOWEST = 1,      /* (i) A = a_0, B = b_1 */
  BOP_BW_HIGHEST = 2,     /* (ii) A = a_{L-1}, B = b_L */
  BOP_BW_AVERAGE = 3,     /* (iii) A = mean of a_0..a_{L-1}, B = rms of b_1..b_L */
  BOP_BW_AVG_CENTRE = 4,  /* (iv) A as (iii), B = b_L */
  BOP_BW_MINMAX = 5,      /* (v) A = (max a + min a)/2, B = (max a - min a + 4 max b)/4 */
  BOP_BW_GLOBAL = 6,      /* (viii) A = bw_a, B = bw_b for every orbital */
  BOP_BW_WEIGHTED = 7     /* Eq. weighted: w_m = 1/(bw_beta (m_max - m) + 1), m_max = L-1 for a, L for b */
};

/* Model and run settings.
 * beta_x(r) = b0[x] * exp(-lam (r - r0)) * fcut(r), fcut the cosine taper
 * of Eq. cutoff on [rc - dc, rc]; b0 = {ss sigma} (norb 1),
 * {dd sigma, dd pi, dd delta} (norb 5) or {dd sigma, dd pi, dd delta,
 * ss sigma, sd sigma} (norb 6: sd-valent, the s orbital first, then the d
 * orbitals in the order 3z^2-r^2, zx, yz, x^2-y^2, xy) in eV at r0; unused
 * entries are ignored.  Onsite reference levels: onsite0 for every orbital,
 * except onsite_s for the s orbital of an sd model.
 * n_mom odd in [3, 17]; n_exp in [n_mom - 1, 253].
 * n_e: electrons per atom summed over spin.  n_spin 1 (non-magnetic, spin
 * factor 2) or 2 (collinear, Stoner).
 * scf: LCN shifts one onsite level per atom, delta_i += eta (N_i - n_e) /
 * max(n_i(E_F), dos_floor) then removes the mean, until max|N_i - n_e| <
 * scf_tol; STONER additionally mixes m_i with m_mix from m0 until
 * max|m_out - m| < 10 scf_tol, E_{i,up/down} = E0 + delta_i -/+ I m_i / 2.
 * VARIATIONAL (n_spin 1, Eq. BOP_SCF) minimises the binding energy
 * U_B = U_bond + sum_i j_ii q_i^2 / 2 (q_i = N_i - n_e, Eq. TB-Uion) over
 * one onsite shift per atom: Delta_i = sum_alpha (Theta~_ii - N_i) =
 * dU_B/d delta_i at fixed electron count comes from a reverse sweep of the
 * moments every iteration, delta_i -= eta Delta_i / (D (1 + j_ii D)) with
 * D = max(n_i(E_F), dos_floor) (mixed like LCN), until max|Delta_i| <
 * scf_tol.  The energy per atom includes j_ii q_i^2 / 2, and the forces
 * need no response solve (U_B is stationary in the shifts).  With j_ii = 0
 * the minimum can sit on a kink of the Gershgorin estimate, where Delta
 * jumps across zero; the loop then stops at scf_max_it.
 * precision: FP64 everywhere, or FP32 products and accumulation in the
 * moments and their reverse sweep; with one spin channel the sigma_m
 * recurrences of the expansion and of the weights, and the weights' sums
 * over the coefficients, run in FP32 as well (two spin channels keep them in
 * FP64: the exchange enhancement of the Stoner moments amplifies their
 * rounding).  In FP32 mode the forces take the bond blocks' position
 * derivatives in FP32 too.  The moments -> recursion coefficients, the band
 * width, the Fermi level and the energy's N and U sums stay FP64.
 * mixer: BOP_MIX_LINEAR (x += F, F the preconditioned residual above) or
 * BOP_MIX_ANDERSON (type-II Broyden over the last mix_history <= 8
 * iterations, one of the paper's mixers); both converge to the same
 * self-consistent state.
 * terminator: BOP_TERM_CONSTANT (Eq. abinf with the Gershgorin band edges)
 * or BOP_TERM_MLP, the learned continuation of the chain (n_mom must be 9;
 * a network must be attached with bop_set_mlp, see the learned-terminator
 * section below).
 * scf_response: with an SCF, 1 = forces and virial are the total derivative
 * of the self-consistent energy (the onsite shifts, and for STONER the
 * moments, follow the atoms; an adjoint linear solve, see bop_forces);
 * 0 = the derivative at fixed onsite levels (the Hellmann-Feynman form of
 * Eq. F_k, which the paper notes is not exact for a non-variational SCF).
 * rep_A (eV), rep_p (1/A) >= 0: the repulsive energy U_rep of Eq. U_B,
 * which the paper leaves to empirical functions, as the pair form
 * sum over bonds of rep_A exp(-rep_p (r - r0)) fcut(r) (the taper of the
 * bond integrals); each atom's energy holds half of each of its bonds.
 * r_path > 0: the path-radius cut of "Performance", item (iii): the
 * cluster of atom i keeps only the sites (atom, image) closer than r_path
 * to i, so the moments count only the self-returning paths that stay
 * inside that sphere (an extra approximation; the energy jumps where a site
 * crosses the sphere, and forces are the derivative between such jumps).
 * bandwidth: one of BOP_BW_*; B is floored at 1e-3 eV in every mode (no
 * derivative flows through a floored B).  bw_beta >= 0 (WEIGHTED), bw_a and
 * bw_b > 0 (GLOBAL, eV); ignored otherwise.  The MLP terminator takes
 * BOP_BW_GERSHGORIN only.
 * noncollinear = 1: non-collinear magnetism (section "Magnetism", Eqs.
 * onsite_CM and onsite-noncollinear) with one fixed moment direction s_i
 * per atom (bop_set_spin_directions).  The onsite matrix of orbital alpha
 * of atom i in the spin basis along z is
 *   (E_up + E_dn)/2 1 + (E_dn - E_up)/2 s_i . sigma,
 *   E_up/dn = E0 + delta_i -/+ stoner_I m_i / 2,
 * so that in the frame of s_i it is diag(E_up, E_dn), the lower level E_up
 * belonging to the spin antiparallel to s_i; the hopping is spin
 * independent.  The moments of the two local channels (starting states the
 * local spin states of the orbital) take the place of the collinear spin
 * channels; with every s_i equal the results are the collinear ones.
 * Needs n_spin = 2, scf STONER (magnitudes m_i self-consistent at fixed
 * directions, scf_response = 0: forces and torques at the self-consistent
 * onsite levels) or NONE (magnitudes fixed by m_io of bop_energy, m0 when
 * NULL), the constant terminator.  The energy per atom includes
 * -stoner_I m_i^2 / 4 in both cases. */
typedef struct {
  int norb;
  double b0[5];
  double r0, lam, rc, dc;
  double onsite0;
  int n_mom;
  int n_exp;
  int n_spin;
  double n_e;
  int scf;
  double eta, scf_tol;
  int scf_max_it;
  double stoner_I, m_mix, m0, dos_floor;
  int precision;
  int mixer;
  int mix_history;
  int terminator;
  int scf_response;
  int bandwidth;
  double bw_beta;
  double bw_a, bw_b;
  double j_ii;  /* VARIATIONAL: onsite charging J_ii >= 0 (eV / e^2) */
  double rep_A, rep_p;  /* pair repulsion (described above): rep_A = 0 for none */
  double r_path;        /* path-radius cut in A (described above): 0 for none */
  double onsite_s;      /* sd model: reference level of the s orbital (eV) */
  int noncollinear;     /* 1: non-collinear magnetism (described above), 0: collinear */
} bop_model;

typedef struct {
  int n_atoms;
  int K;                  /* hops (n_mom - 1) / 2 */
  long long n_edges;      /* directed neighbour pairs */
  long long n_bonds;      /* undirected bonds = n_edges / 2 */
  long long n_sites;      /* cluster sites summed over atoms */
  long long n_adj;        /* cluster adjacency entries */
  int max_cluster;        /* largest |C_K| */
  int scf_iterations;
  int scf_converged;
  int bisection_rounds;
  double scf_residual;    /* max |N_i - n_e| of the last iteration */
  double e_fermi;
  double e_total;
  int forces_scf_response;/* 1 if forces include the SCF response (scf == NONE) */
  int n_learned;          /* orbitals (all spins) on the learned chain in the last
                             energy; the others fell back to the constant terminator */
  long long moment_products; /* block products Psi_k(t) += H_ts Psi_k-1(s) of one
                                moments pass, summed over atoms (one spin) */
  int response_iterations;   /* GMRES iterations of the SCF-response solve (last forces) */
  int response_converged;    /* 1 if that solve reached its tolerance */
  double response_residual;  /* its final relative residual */
  int n_unbounded;           /* orbitals (all spins) of the last energy, constant
                                terminator, whose expansion has some |sigma_m| > m + 1:
                                the chain has weight outside [A - 2B, A + 2B] and the
                                Chebyshev series grows with n_exp.  Checked for the
                                estimates other than BOP_BW_GERSHGORIN (0 there) */
} bop_stats;

/* Library version (major * 10000 + minor * 100 + patch). */
int bop_version(void);

/* Creates a context for one model on the current CUDA device.
 * Errors: BOP_ERR_ARG for an invalid model, BOP_ERR_CUDA / BOP_ERR_OOM. */
int bop_create(bop_ctx** ctx, const bop_model* model);

/* Frees all device workspaces; ctx may be NULL. */
int bop_destroy(bop_ctx* ctx);

/* Text of the last error of ctx ("" if none); owned by ctx. */
const char* bop_last_error(const bop_ctx* ctx);

/* Neighbour list (linked cells, pairs with r < rc incl. periodic images),
 * canonical bonds with their blocks and bond vectors, and the cluster of
 * every atom ("Initialisation", Eq. Hij_rot, Eq. momDOS support).
 *   n         atoms (>= 1)
 *   pos       device [n][3] positions; must lie inside the cell
 *             (fractional coordinates in [0, 1)) along every axis
 *   cell_host host [3][3], rows = lattice vectors (right-handed or not)
 *   pbc_host  host [3], 1 = periodic along that lattice vector
 * Copies pos into the context.  Synchronises stream (reads back sizes).
 * Errors: BOP_ERR_ARG (atom outside the cell, a NaN or Inf coordinate,
 * singular cell),
 * BOP_ERR_OVERFLOW (> 64 neighbours of an atom, image index beyond
 * +-127, cluster scratch exhausted after retries). */
int bop_build_hamiltonian(bop_ctx* ctx, int n, const double* pos, const double* cell_host,
                          const int* pbc_host, bop_stream stream);

/* Sizes of the last build and statistics of the last energy/forces call
 * (host struct). */
int bop_get_stats(const bop_ctx* ctx, bop_stats* stats_host);

/* Copies the neighbour list of the last build: row_ptr [n+1] (int64),
 * col [E] (int32), img [E][3] (int8); rows sorted by (j, sx, sy, sz). */
int bop_get_neighbors(bop_ctx* ctx, long long* row_ptr, int* col, signed char* img, bop_stream stream);

/* Copies the cluster of one atom: site_atom [n_site], site_img
 * [n_site][3], level_end [K+1] (all device); n_site = level_end[K].
 * Order: hop level, then atom, then image.  Synchronises stream. */
int bop_get_cluster(bop_ctx* ctx, int atom, int* site_atom, signed char* site_img, int* level_end,
                    bop_stream stream);

/* Copies the bonds: atoms [nb][2] (i < j or image-ordered), bond vectors
 * d = r_j + S.cell - r_i [nb][3], unique block elements [nb][15] (d; the
 * upper triangle row by row), [nb][21] (sd, likewise, s first) or [nb][1]
 * (s). Any pointer may be NULL. */
int bop_get_bonds(bop_ctx* ctx, int* atoms, double* d, double* blocks, bop_stream stream);

/* Moments (Eq. momDOS) of every orbital for the given onsite levels.
 *   onsite  device [n_spin][n][norb] (FP64) or NULL for the reference
 *           levels (onsite0, and onsite_s on the s orbital of an sd model)
 *   mu      device [n_spin][n][norb][n_mom] output (FP64 storage; FP32
 *           arithmetic when precision = FP32)
 * For a noncollinear model onsite holds (E_up, E_dn) of every orbital and
 * mu the moments of the local up / down channels of the directions set by
 * bop_set_spin_directions (BOP_ERR_STATE without them).
 * Requires a build. */
int bop_moments(bop_ctx* ctx, const double* onsite, double* mu, bop_stream stream);

/* Scalar stage of M orbitals from their moments: recursion coefficients
 *   a [M][Kp], b [M][Kp+1] (b_0 = 0), nlev [M] (levels computed, < Kp
 *   where the chain was truncated), a_inf, b_inf [M] (Gershgorin
 *   terminator), gsig [n_exp+1][M] = g_m sigma_m (coefficient-major).
 * Kp = (n_mom - 1) / 2.  Any output except gsig may be NULL. */
int bop_recursion(bop_ctx* ctx, int M, const double* mu, double* a, double* b, int* nlev, double* a_inf,
                  double* b_inf, double* gsig, bop_stream stream);

/* Energy of the last built structure, including the SCF loop.
 *   e_atom    device [n] bond (+ exchange) energy per atom, or NULL
 *   delta_io  device [n] LCN onsite shifts: read as the starting guess
 *             (warm start) and overwritten with the result; NULL = start
 *             from 0 and keep internally.  With delta_io the first Fermi
 *             solve also starts from the previous call's Fermi level (when
 *             it lies in the new bracket)
 *   m_io      device [n] Stoner moments, same convention (NULL = m0)
 *   stats_host optional host struct
 * Synchronises stream once per SCF iteration (convergence flag) and at
 * the end. */
int bop_energy(bop_ctx* ctx, double* e_atom, double* delta_io, double* m_io, bop_stats* stats_host,
               bop_stream stream);

/* Forces (Eq. F_k) and virial W_ab = sum_bonds g_a d_b = dE/dF_ab for a
 * deformation r -> F r (Eq. sigma_k summed over atoms), as the exact
 * derivative of the energy of the last bop_energy call with E_F following
 * the electron count.  With an SCF and model.scf_response = 1 the
 * derivative includes the response of the SCF unknowns u (delta_i, and
 * m_i for STONER): with R(u) = 0 the SCF conditions at fixed E_F and
 * J = dR/du, the multipliers y of J^T y = dE/du (GMRES, right-preconditioned
 * by the inverse local DOS, each product J^T v one reverse sweep of the
 * moments) give dE/dx = dE/dx|_u - y . dR/dx|_u; stats report its
 * iterations and residual (relative tolerance 1e-10 in FP64 mode, 1e-6
 * with FP32 products, where the forces reach the FP32 noise floor).  BOP_ERR_NO_CONVERGENCE if it stops at 120
 * iterations above tolerance (outputs then use the last iterate).
 *   forces device [n][3], virial device [3][3] (row-major), either may be NULL.
 * Errors: BOP_ERR_STATE without a preceding bop_energy. */
int bop_forces(bop_ctx* ctx, double* forces, double* virial, bop_stats* stats_host, bop_stream stream);

/* Moment directions of a noncollinear model (section "Magnetism"):
 * s device [n][3], one direction per atom of the structure built last,
 * normalised by the library (copied through the host once).  Needed before
 * bop_energy; kept until the next call or the next structure of another
 * size.  Errors: BOP_ERR_ARG for a collinear model or a vector of norm
 * below 1e-12 or not finite, BOP_ERR_STATE without a built structure. */
int bop_set_spin_directions(bop_ctx* ctx, const double* s, bop_stream stream);

/* Magnetic torques of Eq. torque after bop_forces of a noncollinear model:
 * t_i = dU/ds_i x s_i, dU/ds_i the derivative of the energy of the last
 * bop_energy call with respect to the direction s_i at fixed magnitudes
 * m_i and shifts delta_i (E_F following the electron count):
 *   dU/ds_i = sum_alpha [ (E_dn - E_up)/2 Tr(Theta~_ii sigma)
 *                         + sum_n (w_dn,n - w_up,n)/2 Tr(sigma M_n) ],
 * Theta~_ii the 2x2 derivative of the energy with respect to the onsite
 * matrix (reverse sweep of the spin moments), w the weights of the local
 * channels and M_n the 2x2 spin moments of the orbital; the term of the
 * paper's expression along m_i is parallel to s_i and drops out of the
 * cross product.  Rotating s_i by a small angle e about a unit axis a
 * changes the energy by -e t_i . a.
 *   t device [n][3].
 * Errors: BOP_ERR_ARG for a collinear model, BOP_ERR_STATE without a
 * preceding bop_forces. */
int bop_torques(bop_ctx* ctx, double* t, bop_stream stream);

/* Spatial decomposition (section "Performance", parallelisation: the paper
 * decomposes the structure into spatial domains, one per process).  Each
 * process builds its domain as one structure: its own atoms first, then the
 * halo, every atom (with the periodic image it needs) within K r_cut of an
 * own atom along the decomposed directions, K = (n_mom - 1)/2, so that the
 * cluster of every own atom lies inside the domain.
 *
 * bop_set_centers(ctx, n_centers): from the next bop_build_hamiltonian on,
 * only atoms [0, n_centers) of a structure are centres: they get clusters,
 * moments, electrons and energies; atoms [n_centers, n) are environment
 * atoms, which take part in the neighbour list, the bond blocks and the
 * clusters of the centres as sites, receive the forces of the bonds they
 * take part in, and have energy 0 in e_atom.  0 (the default) makes every
 * atom a centre.  Errors: BOP_ERR_ARG for n_centers < 0; the build returns
 * BOP_ERR_ARG when n_centers exceeds the atoms of the structure.
 *
 * bop_set_reduce(ctx, fn, user): the context combines its global sums over
 * all processes with fn (NULL: one process): the band edges and the sums of
 * every Newton round of the Fermi-level search (one E_F for the whole
 * structure), the total energy in bop_stats, and the two sums of the E_F
 * multiplier of the forces.  The forces a process returns are its centres'
 * contributions to the forces on every atom of its domain (own and halo):
 * summed over the processes by global atom they give the forces of the
 * whole structure; the virial likewise.
 *
 * With centres or a reduce function the model must have scf NONE and be
 * collinear (bop_energy returns BOP_ERR_ARG otherwise). */
int bop_set_centers(bop_ctx* ctx, int n_centers);
int bop_set_reduce(bop_ctx* ctx, bop_reduce_fn fn, void* user);

/* Limits of the SCF-response solve of bop_forces (GMRES, described there):
 * max_iterations caps its Arnoldi iterations (0 = the default, 3 cycles of
 * 40), rtol its relative residual (0 = the default of the precision).  A
 * solve that stops at the cap above rtol makes bop_forces return
 * BOP_ERR_NO_CONVERGENCE with forces and virial from the last iterate and
 * the residual in bop_stats.response_residual.  The paper's SCF loop has a
 * "maximum number of steps" too ("Program flow", self-consistency); this is
 * the same guard for the linear solve of the exact forces.
 * Errors: BOP_ERR_ARG for max_iterations < 0 or rtol < 0 or not finite. */
int bop_set_response_limits(bop_ctx* ctx, int max_iterations, double rtol);

/* Memory for the reverse sweeps of bop_forces.  When several reverse sweeps
 * follow (an SCF with scf_response = 1) and all starting orbitals of an atom
 * share one work item of the moments kernel, bop_forces runs one extra
 * forward pass that stores Psi_k of every atom's cluster (rows of norb x
 * norb values per site and level, FP32 or FP64 as the precision) when it
 * fits in a third of the free device memory, and every reverse sweep then
 * reads Psi instead of recomputing it (the sweep that forms the bond
 * cotangents forms them level by level from the same store).
 * bytes >= 0 caps that store (0 = always recompute, which also frees it);
 * bytes < 0 restores the default. */
int bop_set_store_budget(bop_ctx* ctx, long long bytes);

/* Per-orbital state of the last bop_energy / bop_forces call (device
 * outputs, each may be NULL): mu [M][n_mom], N [M] and U [M] (per spin
 * channel, before the spin factor), a_inf, b_inf [M], weights [M][n_mom]
 * (dE/dmu, valid after bop_forces), onsite [M]. */
int bop_get_orbital_state(bop_ctx* ctx, double* mu, double* N, double* U, double* a_inf, double* b_inf,
                          double* weights, double* onsite, bop_stream stream);

/* End-to-end energy + forces with HOST buffers: copies pos_host in,
 * runs build, energy and forces, copies the results out and synchronises.
 *   pos_host [n][3]; e_atom_host [n]; forces_host [n][3]; virial_host [9];
 *   e_total_host [1]; outputs may be NULL. */
int bop_evaluate_host(bop_ctx* ctx, int n, const double* pos_host, const double* cell_host,
                      const int* pbc_host, double* e_atom_host, double* forces_host, double* virial_host,
                      double* e_total_host, bop_stats* stats_host, bop_stream stream);

/* One half of a velocity-Verlet step of molecular dynamics on BOP forces
 * (the MD loop that the warm start of the onsite levels, speed-up (ii) under
 * "Performance", is meant for: pass the previous step's shifts to
 * bop_energy as delta_io).  With a = F / mass:
 *   phase 0: v += a dt / 2, then x += v dt   (before the force evaluation)
 *   phase 1: v += a dt / 2                   (after it)
 * Units: positions A, velocities A/fs, forces eV/A, dt fs, mass amu (one
 * mass for all atoms).  pos, vel, forces: device [n][3], in place; pos may
 * be NULL for phase 1.  cell_host [3][3] (rows: lattice vectors) and
 * pbc_host [3], or both NULL: after the drift, an atom that left the cell
 * along a periodic axis is moved back by whole lattice vectors (atoms
 * inside are untouched), as bop_build_hamiltonian requires.
 * Stream-ordered; no synchronisation.
 * Errors: BOP_ERR_ARG for n < 0, dt <= 0, mass <= 0, a bad phase, a
 * missing pointer or a singular cell; BOP_ERR_CUDA if the launch fails. */
int bop_md_verlet(int n, double* pos, double* vel, const double* forces, const double* cell_host,
                  const int* pbc_host, double dt, double mass, int phase, bop_stream stream);

/* Per-kernel-family timing, for measurement.  While profiling is on, every
 * launch region of the context is bracketed by two CUDA events on the
 * stream it is launched on; launch counts are kept whether or not
 * profiling is on.  Families: "neighbours", "cluster", "onsite", "moments",
 * "expand", "fermi", "orbital_NU", "scf", "energy", "ef_response",
 * "weights", "adjoint", "forces".  bop_get_profile synchronises on the
 * recorded events; name points to a static string. */
typedef struct {
  const char* name;
  long long launches; /* kernels launched (all calls since the last reset) */
  long long regions;  /* event-timed launch regions */
  double ms;          /* summed device time of the timed regions */
} bop_kernel_time;

int bop_set_profiling(bop_ctx* ctx, int on);
int bop_reset_profile(bop_ctx* ctx);
/* Writes up to max entries, *n_out = number of families. */
int bop_get_profile(bop_ctx* ctx, bop_kernel_time* out_host, int max, int* n_out);

/* Fermi level of M orbitals without any device allocation.  This entry
 * point has no counterpart in the paper: it serves callers that cannot call
 * cudaMalloc, because they run under a device-memory budget fixed in
 * advance, because their host framework pre-reserves all GPU memory at
 * start-up (a new allocation would fail or bypass its accounting), or
 * because an allocation would synchronise the device at a point they do not
 * control.  It runs the library's bisection kernels (100 halvings or a
 * bracket narrower than 1e-13 eV; the root of the Newton-accelerated search
 * of bop_energy, which stops on its own rule: the two agree to 1e-9 eV in
 * the tests) with their scratch in a 16 MiB file-scope __device__ array
 * that every GPU loading the library keeps until the process exits.
 *   M            orbitals (all spins)
 *   n_exp        expansion length of gsig (2 .. 253)
 *   gsig         device [n_exp+1][M]: g_m sigma_m, as written by bop_recursion
 *   a_inf, b_inf device [M]: terminator of every orbital (bop_recursion)
 *   spin_factor  2 for non-magnetic orbitals, 1 per collinear spin channel
 *   n_electrons  total electron count the Fermi level must hold, in
 *                (0, spin_factor M); outside it BOP_ERR_BRACKET (no launch)
 *   e_fermi      device [1] output
 * Caller-owned inputs and output; nothing is allocated.  The scratch needs
 * 16896 + 8 (n_exp + 3) M bytes: larger problems (more than 10,300 orbitals
 * at n_exp = 200) are rejected with BOP_ERR_OVERFLOW and a message on
 * stderr, before anything is launched.  The first call on a device looks up
 * the array's device address (once per device), so make that first call
 * before any stream capture; the address is kept for the life of the
 * process and does not survive a cudaDeviceReset, after which this entry
 * point is not supported.  All calls share the one array, which keeps
 * the last call's contents: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller. */
int bop_fermi_level_noalloc(int M, int n_exp, const double* gsig, const double* a_inf, const double* b_inf,
                            double spin_factor, double n_electrons, double* e_fermi, bop_stream stream);

/* ------------------------------------------------------------------ learned terminator
 * The paper closes the recursion chain with a constant terminator (Eq. abinf,
 * a_inf / b_inf from Eq. gershogorin).  The learned terminator keeps that form
 * but continues the 9-moment chain of every orbital: a small network predicts
 * the next four levels (a_4..a_7, b_5..b_8) and the band centre / width
 * (a*_inf, b*_inf) that a 17-moment run of the same orbital would give, and
 * the constant terminator then starts after level 8.  The paper has no such
 * network; its constant terminator is the fallback and the reference the
 * network is compared with.
 *   inputs x (BOP_MLP_NIN = 18): (a_k - a_inf)/b_inf, k = 0..3; b_k/b_inf,
 *     k = 1..4; a_inf; b_inf; mu-hat_1 .. mu-hat_8 (Eq. sigma_i normalisation);
 *     a_inf, b_inf from the 9-moment Gershgorin bounds;
 *   outputs y (BOP_MLP_NOUT = 10): (a*_inf - a_inf)/b_inf, b*_inf/b_inf,
 *     (a_k - a_inf)/b_inf for k = 4..7, b_k/b_inf for k = 5..8;
 *   network: 18 -> 128 -> 128 -> 10, GELU (x Phi(x)), on inputs and outputs
 *     standardised by the training set (mean, standard deviation);
 *   parameters (BOP_MLP_NPARAM floats, row-major [out][in] matrices):
 *     W1 [128][18], b1 [128], W2 [128][128], b2 [128], W3 [10][128], b3 [10];
 *   normalisation (BOP_MLP_NNORM floats): x_mean [18], x_std [18], x_lo [18],
 *     x_hi [18] (training range widened by 5 % of its span), y_mean [10],
 *     y_std [10];
 *   training: FP32, mean squared error of the standardised outputs over the
 *     rows with mask 1, Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected);
 *   inference: weight matrices rounded to bfloat16 (nearest even), biases
 *     FP32, activations FP32 (precision FP32) or FP64 (precision FP64), so
 *     the energy stays smooth in the moments and the forces are its exact
 *     derivative;
 *   fallback to the constant terminator of the 9-moment chain where that
 *     chain is truncated, an input lies outside [x_lo, x_hi], a predicted
 *     b_k or b*_inf is not above 1e-3 eV, or a value is not finite.
 * A bop_mlp lives on the device that was current at bop_mlp_create. */
#define BOP_MLP_NIN 18
#define BOP_MLP_NHID 128
#define BOP_MLP_NOUT 10
#define BOP_MLP_NPARAM 20234
#define BOP_MLP_NNORM 92

/* Creates a network from params_host [BOP_MLP_NPARAM] (host FP32), with the
 * identity standardisation and an unbounded training range; Adam state 0.
 * Synchronises the device. */
int bop_mlp_create(bop_mlp** net, const float* params_host);
int bop_mlp_destroy(bop_mlp* net);
const char* bop_mlp_last_error(const bop_mlp* net);

/* Copies the FP32 master parameters and / or the normalisation to host
 * arrays (either may be NULL).  Synchronous. */
int bop_mlp_get(bop_mlp* net, float* params_host, float* norm_host);
/* Sets the normalisation from a host array; standard deviations must be > 0. */
int bop_mlp_set_norm(bop_mlp* net, const float* norm_host);

/* Training data from 17-moment runs: for M orbitals with moments mu17
 * (device [M][17], FP64, e.g. from bop_moments of a context with n_mom 17)
 * writes the raw inputs x [M][18] (from mu_0..mu_8), the raw targets
 * t [M][10] and mask [M] (1 where the 17-moment chain has all 8 levels and
 * every target is finite, else 0; t is 0 there).  Device outputs. */
int bop_mlp_dataset(long long M, const double* mu17, float* x, float* t, float* mask, bop_stream stream);

/* Fits the normalisation to the rows with mask > 0 of x [M][18], t [M][10]
 * (device): means, population standard deviations floored at 1e-6, input
 * range widened by 5 % of its span. */
int bop_mlp_fit_norm(bop_mlp* net, long long M, const float* x, const float* t, const float* mask,
                     bop_stream stream);

/* Gradient of the loss over one batch: rows idx[0..batch-1] (device int32,
 * each in [0, M)) of the raw data x, t, mask (device).  The gradient is kept
 * in the network for bop_mlp_adam and copied to grad_out (device
 * [BOP_MLP_NPARAM]) if not NULL; the batch loss goes to loss_out (device
 * [1]) if not NULL.  Deterministic (fixed reduction order). */
int bop_mlp_gradient(bop_mlp* net, long long M, const float* x, const float* t, const float* mask, const int* idx,
                     int batch, float* grad_out, float* loss_out, bop_stream stream);
/* Reads back (synchronising stream) whether any row index of the batches
 * since the last check was outside [0, M): such rows enter the gradient as
 * masked rows of zeros.  BOP_ERR_ARG if so. */
int bop_mlp_check(bop_mlp* net, bop_stream stream);
/* One Adam step with the last gradient; refreshes the bfloat16 weights. */
int bop_mlp_adam(bop_mlp* net, float lr, bop_stream stream);
/* bop_mlp_gradient followed by bop_mlp_adam. */
int bop_mlp_train_step(bop_mlp* net, long long M, const float* x, const float* t, const float* mask, const int* idx,
                       int batch, float lr, float* loss_out, bop_stream stream);

/* Inference: raw outputs y [M][10] for raw inputs x [M][18] (device) with the
 * bfloat16 weights and FP32 activations. */
int bop_mlp_predict(bop_mlp* net, long long M, const float* x, float* y, bop_stream stream);

/* Attaches a network to a context whose model has terminator = BOP_TERM_MLP
 * (NULL detaches).  The context keeps the pointer: the network must outlive
 * its use, and training steps change what the next bop_energy computes.
 * Errors: BOP_ERR_ARG if the model's terminator is not BOP_TERM_MLP. */
int bop_set_mlp(bop_ctx* ctx, bop_mlp* net);

#ifdef __cplusplus
}
#endif
#endif /* BOPGB_H */
