// C ABI of libbopgb: the context (device workspaces), the build of the
// neighbour list / bonds / clusters, and the orchestration of the energy
// (SCF loop) and force passes.  Every arithmetic step of the path runs in
// the kernels of nbr.cu, cluster.cu, moments.cu, scalar.cu and forces.cu;
// this file only sizes buffers, launches and reads back flags.
#include <cub/cub.cuh>
#include <cuda/std/functional>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/bopgb.h"
#include "kernels.h"

int moments_columns(int norb, int cap_sum, int fp64);
int adjoint_columns(int norb);

constexpr int FERMI_ROUNDS_COLD = 16;  // Newton rounds launched for a cold start
constexpr int FERMI_ROUNDS_WARM = 5;  // ... and from the previous SCF iteration's E_F
constexpr int FERMI_ROUNDS_MORE = 64;  // extra rounds if a solve has not converged
constexpr int FERMI_MAX_ROUNDS = 256;  // hard cap per solve
constexpr double FERMI_TOL = 1e-13;    // eV
constexpr int FERMI_F32_START = 65536; // orbitals from which a cold solve starts with FP32 rounds

namespace {

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

enum ProfKind {
  PK_NBR = 0, PK_CLUSTER, PK_ONSITE, PK_MOMENTS, PK_EXPAND, PK_FERMI, PK_NU, PK_SCF, PK_ENERGY, PK_EFRESP,
  PK_WEIGHTS, PK_ADJOINT, PK_FORCES, PK_MLP, PK_N
};
static const char* const PK_NAMES[PK_N] = {"neighbours", "cluster", "onsite", "moments", "expand", "fermi",
                                          "orbital_NU", "scf", "energy", "ef_response", "weights", "adjoint",
                                          "forces", "mlp"};

struct Prof {
  bool on = false;
  long long launches[PK_N] = {0};
  std::vector<cudaEvent_t> pool;  // events in recording order: pairs (begin, end)
  std::vector<int> kind;          // one entry per pair
  size_t used = 0;                // events used in the pool
};

struct bop_ctx {
  bop_model m;
  BondModel bm;
  int norb, HS, HSu, K, Kp, n_mom, n_exp, S, fp64;
  double sfac;
  int device;
  // structure: n atoms, of which the first nc have clusters (centres); the
  // others are environment (halo) atoms of a spatial domain
  int n = 0, nc = 0, nc_req = 0;
  // reductions over the processes of a spatial decomposition (NULL: one process)
  bop_reduce_fn reduce_fn = nullptr;
  void* reduce_user = nullptr;
  double ef_host = 0.0;  // E_F of the last distributed solve (its warm start)
  long long E = 0, nb = 0, nsite = 0, nadj = 0;
  Geometry g;
  int maxlev[BOP_MAX_K + 2];  // largest |C_k| per level, then the largest adjacency
  bool built = false, energized = false, weighted = false;
  // buffers
  DBuf pos, cell_of, cell_count, cell_start, cell_fill, cell_atoms, deg, row_ptr, col, img, flag, bond_scan,
      bond_of_edge, bond_atoms, bond_img, bond_d, H64, H32, frac;
  DBuf hkeys, hvals, skeys, sslot, scount;
  DBuf level_end, atom_nsite, atom_nadj, max_level, site_off, adj_base, site_atom, site_img, adj_off, adj, lvcnt;
  DBuf onsite, onsite32, delta, mval, delta_new, m_new, mu, a, b, nlev, a_inf, b_inf, gsig, D, gjack;
  DBuf N, U, dos, fstate, partials, counter, result, e_total, lam, e_atom;
  DBuf w, zscr, adjscr, Hbar, Ebar, ginv;
  DBuf hx, hf, gamma, scfred;
  // learned terminator
  bop_mlp* net = nullptr;
  DBuf lbase, lnlev, lflag, lxs, lys, lZ1, lH1, lZ2, lH2, lybar, lcot, lxbar, lcount;
  // SCF response of the forces (rjv: per-site values of one dN/dmu sweep, the
  // rows of the Jacobian)
  DBuf rwN, rwt, rdUE, rvec, rcoef, rjv, rjcnt, rjptr, rjidx, rjrow;
  // variational SCF: dU_B/d delta, q; weights in w valid for the final state
  DBuf vgrad, vq;
  bool var_w_valid = false;
  // the last bop_energy was followed by bop_forces: the next one stores Psi
  // in its SCF passes for the reverse sweeps (no extra forward pass)
  bool forces_follow = false;
  bool ef_solved = false;  // fstate holds a Fermi level of an earlier solve
  DBuf erep;  // pair repulsion per atom
  // non-collinear magnetism: unit moment directions [n][3] (sdir_n atoms),
  // Tr(sigma M_n) [n][norb][n_mom][3], onsite cotangents [n][norb][4],
  // torques [n][3], per-CTA spinor scratch
  DBuf sdir, vmom, obar, torque, ncscr;
  int sdir_n = -1;
  // stored Psi of every work item for the reverse sweeps (when it fits)
  DBuf psi_off, psis, lsum;
  DBuf fev;  // two device doubles of the distributed Fermi solve
  DBuf gs32;  // FP32 copy of gsig for the starting point of a cold Fermi solve
  DBuf cw_misc, cw_keys, cw_epack;  // warp cluster builder: max degree / failure flags, site keys per
                                    // atom, packed neighbour edges
  int cw_maxdeg = -1;  // largest degree of the centres, read back with the neighbour list's status
  long long psi_tot = 0;
  bool psi_valid = false;
  size_t store_budget = (size_t)-1;
  int resp_max_it = 0;     // cap of the SCF-response solve's iterations (0: GM_KRYLOV x GM_CYCLES)
  double resp_rtol = 0.0;  // its relative tolerance (0: the precision's default)
  DBuf status;
  // pinned host staging of the small reads taken at a synchronisation
  void* pin = nullptr;
  DBuf cub_tmp;
  DBuf nprod;
  int cl_hcap = 0, cl_maxs = 0, cl_slots = 0;
  bop_stats st;
  Prof prof;
  char err[512];
};

namespace {

int fail(bop_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(c, BOP_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                        \
  } while (0)

#define CKS(expr)            \
  do {                       \
    int s_ = (expr);         \
    if (s_ != BOP_OK) return s_; \
  } while (0)

cudaEvent_t prof_event(bop_ctx* c) {
  if (c->prof.used == c->prof.pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->prof.pool.push_back(e);
  }
  return c->prof.pool[c->prof.used++];
}

// Brackets one launch region of `nk` kernels of family k on stream s.
struct Region {
  bop_ctx* c;
  int k;
  cudaStream_t s;
  Region(bop_ctx* c_, int k_, int nk, cudaStream_t s_) : c(c_), k(k_), s(s_) {
    c->prof.launches[k] += nk;
    if (c->prof.on) {
      cudaEvent_t e = prof_event(c);
      if (e) cudaEventRecord(e, s);
      c->prof.kind.push_back(k);
    }
  }
  ~Region() {
    if (c->prof.on) {
      cudaEvent_t e = prof_event(c);
      if (e) cudaEventRecord(e, s);
    }
  }
};

int ensure(bop_ctx* c, DBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return BOP_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, BOP_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  b.bytes = bytes;
  return BOP_OK;
}

template <class T>
T* P(DBuf& b) {
  return reinterpret_cast<T*>(b.p);
}

cudaStream_t S_(bop_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// The sigma_m recurrences run in FP32 in the FP32-products mode of a single
// spin channel.  With two spin channels the Stoner moments amplify the
// error of N(E) by the exchange enhancement 1/(1 - I n(E_F)) (measured on
// the 2,000-atom Stoner cell: Hellmann-Feynman forces 9e-3 eV/A off the FP64
// oracle against < 5e-4 with FP64 recurrences), so they stay FP64 there.
bool sig32_mode(const bop_ctx* c) { return !c->fp64 && c->S == 1; }

// Stopping rule of the Fermi search: a Newton step shorter than this.  The
// root is then known to about C tol^2 (C = |N''| / 2N', of order 10 per eV
// for the Jackson-damped DOS), far inside tol, while the N and DOS stored
// per orbital are those of the last evaluation, within tol of E_F: that
// bounds the SCF residual they feed (the energy, the weights and the E_F
// response are evaluated at E_F itself).  FP64 mode: 1e-13 eV.  FP32
// products: 1e-6 eV, or 1e-2 of the SCF tolerance when that is smaller.
double fermi_tol(const bop_ctx* c) {
  if (c->fp64) return FERMI_TOL;
  double t = 1e-6;
  if (c->m.scf != BOP_SCF_NONE) t = std::fmin(t, 1e-2 * c->m.scf_tol);
  return std::fmax(t, FERMI_TOL);
}

constexpr size_t PIN_BYTES = 16384;

// The small device-to-host reads of one synchronisation point: each lands in
// the context's pinned staging area (an asynchronous copy, where a copy into
// pageable memory synchronises the stream by itself), and all of them are
// copied to their destinations once the stream has synchronised.  A read
// that does not fit goes straight to its destination.
struct Readback {
  bop_ctx* c;
  cudaStream_t s;
  int n = 0;
  size_t used = 0;
  void* dst[16];
  size_t off[16], len[16];
  Readback(bop_ctx* c_, cudaStream_t s_) : c(c_), s(s_) {}
  // an error return between add and sync: the staged copies land before the
  // staging area is used again
  ~Readback() {
    if (n > 0) cudaStreamSynchronize(s);
  }
  int add(void* h, const void* d, size_t bytes) {
    const size_t at = (used + 15) & ~(size_t)15;
    if (c->pin == nullptr || n == 16 || at + bytes > PIN_BYTES) {
      CK(cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, s));
      return BOP_OK;
    }
    CK(cudaMemcpyAsync(static_cast<char*>(c->pin) + at, d, bytes, cudaMemcpyDeviceToHost, s));
    dst[n] = h;
    off[n] = at;
    len[n++] = bytes;
    used = at + bytes;
    return BOP_OK;
  }
  // synchronises s and copies the staged reads out
  int sync() {
    CK(cudaStreamSynchronize(s));
    for (int q = 0; q < n; q++) memcpy(dst[q], static_cast<char*>(c->pin) + off[q], len[q]);
    n = 0;
    used = 0;
    return BOP_OK;
  }
  // the same, with the device status word read and decoded (check_status)
  int finish();
};

int decode_status(bop_ctx* c, unsigned h, cudaStream_t s) {
  if (h == 0) return BOP_OK;
  CK(cudaMemsetAsync(c->status.p, 0, sizeof(unsigned), s));
  if (h & BOP_DEV_ERR_DEGREE) return fail(c, BOP_ERR_OVERFLOW, "an atom has more than %d neighbours", BOP_MAX_DEG);
  if (h & BOP_DEV_ERR_IMAGE) return fail(c, BOP_ERR_OVERFLOW, "periodic image index outside [-127, 127]");
  if (h & BOP_DEV_ERR_CLUSTER) return fail(c, BOP_ERR_OVERFLOW, "cluster scratch exhausted");
  if (h & BOP_DEV_ERR_REVERSE) return fail(c, BOP_ERR_ARG, "neighbour list not symmetric");
  if (h & BOP_DEV_ERR_NONFINITE) return fail(c, BOP_ERR_NUMERIC, "non-finite value in the scalar stages");
  return fail(c, BOP_ERR_CUDA, "device status 0x%x", h);
}

int Readback::finish() {
  unsigned h = 0;
  CKS(add(&h, c->status.p, sizeof(unsigned)));
  CKS(sync());
  return decode_status(c, h, s);
}

int check_status(bop_ctx* c, cudaStream_t s) {
  Readback rb(c, s);
  return rb.finish();
}

// Exclusive prefix sum accumulated in the output type (an int count
// summed into 64-bit offsets must not wrap at 2^31).
template <class Tin, class Tout>
int exclusive_scan(bop_ctx* c, const Tin* in, Tout* out, long long n, cudaStream_t s) {
  size_t tmp = 0;
  CK(cub::DeviceScan::ExclusiveScan(nullptr, tmp, in, out, cuda::std::plus<Tout>{}, Tout(0), (int)n, s));
  CKS(ensure(c, c->cub_tmp, tmp));
  CK(cub::DeviceScan::ExclusiveScan(c->cub_tmp.p, tmp, in, out, cuda::std::plus<Tout>{}, Tout(0), (int)n, s));
  return BOP_OK;
}

int validate_model(bop_ctx* c, const bop_model* m) {
  if (!m) return fail(c, BOP_ERR_ARG, "model is NULL");
  if (m->norb != 1 && m->norb != 5 && m->norb != 6) return fail(c, BOP_ERR_ARG, "norb must be 1 (s), 5 (d) or 6 (sd)");
  if (m->n_mom < 3 || m->n_mom > BOP_MAX_NMOM || m->n_mom % 2 == 0)
    return fail(c, BOP_ERR_ARG, "n_mom must be odd in [3, %d]", BOP_MAX_NMOM);
  if (m->n_exp < m->n_mom - 1 || m->n_exp > BOP_MAX_NEXP)
    return fail(c, BOP_ERR_ARG, "n_exp must be in [n_mom-1, %d]", BOP_MAX_NEXP);
  if (m->n_spin != 1 && m->n_spin != 2) return fail(c, BOP_ERR_ARG, "n_spin must be 1 or 2");
  if (!(m->rc > 0) || !(m->dc > 0) || m->dc > m->rc) return fail(c, BOP_ERR_ARG, "need 0 < dc <= rc");
  if (m->scf < 0 || m->scf > 3) return fail(c, BOP_ERR_ARG, "scf must be NONE, LCN, STONER or VARIATIONAL");
  if (m->scf == BOP_SCF_VARIATIONAL && m->n_spin != 1) return fail(c, BOP_ERR_ARG, "VARIATIONAL needs n_spin = 1");
  if (m->scf == BOP_SCF_VARIATIONAL && !(m->j_ii >= 0 && m->j_ii < 1e300))
    return fail(c, BOP_ERR_ARG, "j_ii must be finite and >= 0");
  if (m->scf == BOP_SCF_STONER && m->n_spin != 2) return fail(c, BOP_ERR_ARG, "STONER needs n_spin = 2");
  if (m->n_spin == 2 && m->scf != BOP_SCF_STONER && m->scf != BOP_SCF_NONE)
    return fail(c, BOP_ERR_ARG, "n_spin = 2 needs scf STONER or NONE");
  if (!(m->n_e >= 0 && m->n_e <= 2.0 * m->norb)) return fail(c, BOP_ERR_ARG, "n_e must be in [0, 2 norb]");
  if (m->precision != BOP_PREC_FP64 && m->precision != BOP_PREC_FP32)
    return fail(c, BOP_ERR_ARG, "precision must be FP64 or FP32");
  if (m->scf != BOP_SCF_NONE && (m->scf_max_it < 0 || !(m->scf_tol > 0)))
    return fail(c, BOP_ERR_ARG, "scf_tol > 0 and scf_max_it >= 0 required");
  if (m->mixer != BOP_MIX_LINEAR && m->mixer != BOP_MIX_ANDERSON)
    return fail(c, BOP_ERR_ARG, "mixer must be LINEAR or ANDERSON");
  if (m->mixer == BOP_MIX_ANDERSON && (m->mix_history < 1 || m->mix_history > 8))
    return fail(c, BOP_ERR_ARG, "mix_history must be in [1, 8]");
  if (m->terminator != BOP_TERM_CONSTANT && m->terminator != BOP_TERM_MLP)
    return fail(c, BOP_ERR_ARG, "terminator must be CONSTANT or MLP");
  if (m->terminator == BOP_TERM_MLP && m->n_mom != 9) return fail(c, BOP_ERR_ARG, "the MLP terminator needs n_mom = 9");
  if (m->scf_response != 0 && m->scf_response != 1) return fail(c, BOP_ERR_ARG, "scf_response must be 0 or 1");
  if (m->bandwidth < BOP_BW_GERSHGORIN || m->bandwidth > BOP_BW_WEIGHTED)
    return fail(c, BOP_ERR_ARG, "bandwidth must be one of BOP_BW_*");
  if (m->bandwidth == BOP_BW_WEIGHTED && !(m->bw_beta >= 0 && m->bw_beta < 1e300))
    return fail(c, BOP_ERR_ARG, "bw_beta must be finite and >= 0");
  if (m->bandwidth == BOP_BW_GLOBAL && !(m->bw_b > 0 && m->bw_b < 1e300 && fabs(m->bw_a) < 1e300))
    return fail(c, BOP_ERR_ARG, "bw_a must be finite and bw_b finite and > 0");
  if (!(m->r_path >= 0 && m->r_path < 1e300)) return fail(c, BOP_ERR_ARG, "r_path must be finite and >= 0");
  if (!(m->rep_A >= 0 && m->rep_A < 1e300 && m->rep_p >= 0 && m->rep_p < 1e300))
    return fail(c, BOP_ERR_ARG, "rep_A and rep_p must be finite and >= 0");
  if (m->terminator == BOP_TERM_MLP && m->bandwidth != BOP_BW_GERSHGORIN)
    return fail(c, BOP_ERR_ARG, "the MLP terminator takes the Gershgorin band width only");
  if (m->noncollinear != 0 && m->noncollinear != 1) return fail(c, BOP_ERR_ARG, "noncollinear must be 0 or 1");
  if (m->noncollinear) {
    if (m->n_spin != 2) return fail(c, BOP_ERR_ARG, "noncollinear needs n_spin = 2");
    if (m->scf != BOP_SCF_NONE && m->scf != BOP_SCF_STONER)
      return fail(c, BOP_ERR_ARG, "noncollinear needs scf STONER or NONE");
    if (m->scf == BOP_SCF_STONER && m->scf_response)
      return fail(c, BOP_ERR_ARG, "noncollinear STONER needs scf_response = 0");
    if (m->terminator != BOP_TERM_CONSTANT) return fail(c, BOP_ERR_ARG, "noncollinear needs the constant terminator");
  }
  return BOP_OK;
}

BandSel band_sel(const bop_model& m) {
  BandSel b;
  b.mode = m.bandwidth;
  b.beta = m.bw_beta;
  b.ga = m.bw_a;
  b.gb = m.bw_b;
  return b;
}

int geometry(bop_ctx* c, const double* cell, const int* pbc, Geometry* g) {
  memcpy(g->cell, cell, 9 * sizeof(double));
  const double* a0 = cell;
  const double* a1 = cell + 3;
  const double* a2 = cell + 6;
  double c12[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]};
  double c20[3] = {a2[1] * a0[2] - a2[2] * a0[1], a2[2] * a0[0] - a2[0] * a0[2], a2[0] * a0[1] - a2[1] * a0[0]};
  double c01[3] = {a0[1] * a1[2] - a0[2] * a1[1], a0[2] * a1[0] - a0[0] * a1[2], a0[0] * a1[1] - a0[1] * a1[0]};
  double vol = a0[0] * c12[0] + a0[1] * c12[1] + a0[2] * c12[2];
  if (!(std::fabs(vol) > 1e-12)) return fail(c, BOP_ERR_ARG, "singular cell");
  // inv[r][a] such that frac_a = sum_r pos_r inv[r][a]: columns = reciprocal vectors
  for (int r = 0; r < 3; r++) {
    g->inv[r * 3 + 0] = c12[r] / vol;
    g->inv[r * 3 + 1] = c20[r] / vol;
    g->inv[r * 3 + 2] = c01[r] / vol;
  }
  const double* rec[3] = {c12, c20, c01};
  for (int a = 0; a < 3; a++) {
    double nb = std::sqrt(rec[a][0] * rec[a][0] + rec[a][1] * rec[a][1] + rec[a][2] * rec[a][2]) / std::fabs(vol);
    double width = 1.0 / nb;  // distance between the lattice planes spanned by the other two vectors
    int nc = (int)std::floor(width / (c->m.rc * (1.0 + 1e-9) + 1e-9));
    if (nc < 1) nc = 1;
    if (nc > 1024) nc = 1024;
    g->nc[a] = nc;
    g->pbc[a] = pbc[a] ? 1 : 0;
    g->nimg[a] = pbc[a] ? (int)std::ceil(c->m.rc * nb) + 1 : 0;
  }
  g->rc = c->m.rc;
  return BOP_OK;
}

// Warp-per-atom builder (clusters of at most cluster_warp_max_sites()
// sites, atoms of at most 32 neighbours); *done = false when it does not
// apply, and the block builder below runs instead.
int build_clusters_warp(bop_ctx* c, cudaStream_t s, bool* done) {
  *done = false;
  const int n = c->nc, K = c->K;  // clusters of the centres
  if (n == 0 || (c->cl_maxs && c->cl_maxs > cluster_warp_max_sites())) return BOP_OK;
  if (K > 5 && !(c->m.r_path > 0)) return BOP_OK;  // bcc has 1,105 sites within 6 hops
  int misc[4] = {0, 0, 0, 0};
  CKS(ensure(c, c->cw_misc, 4 * sizeof(int)));
  if (c->cw_maxdeg < 0) {  // not read with the neighbour list
    CK(cudaMemsetAsync(c->cw_misc.p, 0, 4 * sizeof(int), s));
    launch_max_degree(n, P<long long>(c->row_ptr), P<int>(c->cw_misc), s);
    Readback rb(c, s);
    CKS(rb.add(misc, c->cw_misc.p, 4 * sizeof(int)));
    CKS(rb.sync());
    c->cw_maxdeg = misc[0];
  }
  const int max_deg = c->cw_maxdeg;
  c->cw_maxdeg = -1;
  CK(cudaMemsetAsync(P<int>(c->cw_misc) + 1, 0, 3 * sizeof(int), s));
  if (max_deg > 32) return BOP_OK;
  int* wfail = P<int>(c->cw_misc) + 1;
  CKS(ensure(c, c->level_end, sizeof(int) * (size_t)n * (K + 1)));
  CKS(ensure(c, c->atom_nsite, sizeof(int) * (n + 1)));
  CKS(ensure(c, c->atom_nadj, sizeof(int) * (n + 1)));
  CK(cudaMemsetAsync(c->atom_nsite.p, 0, sizeof(int) * (n + 1), s));
  CK(cudaMemsetAsync(c->atom_nadj.p, 0, sizeof(int) * (n + 1), s));
  CKS(ensure(c, c->max_level, sizeof(int) * (K + 2)));
  CKS(ensure(c, c->site_off, sizeof(long long) * (n + 1)));
  CKS(ensure(c, c->adj_base, sizeof(long long) * (n + 1)));
  CKS(ensure(c, c->cw_keys, sizeof(unsigned long long) * (size_t)n * cluster_warp_max_sites()));
  CKS(ensure(c, c->cw_epack, sizeof(int2) * (size_t)(c->E > 0 ? c->E : 1)));
  launch_pack_edges(c->E, P<int>(c->col), P<signed char>(c->img), P<int2>(c->cw_epack), s);
  CK(cudaMemsetAsync(c->max_level.p, 0, sizeof(int) * (K + 2), s));
  PathCut pc;
  pc.pos = P<double>(c->pos);
  for (int q = 0; q < 9; q++) pc.cell[q] = c->g.cell[q];
  pc.r2 = c->m.r_path > 0 ? c->m.r_path * c->m.r_path : 0.0;
  ClusterOut out{};
  out.level_end = P<int>(c->level_end);
  out.atom_nsite = P<int>(c->atom_nsite);
  out.atom_nadj = P<int>(c->atom_nadj);
  out.max_level = P<int>(c->max_level);
  {
    Region R0(c, PK_CLUSTER, 1, s);
    if (launch_cluster_warp(0, n, K, max_deg, P<long long>(c->row_ptr), P<int2>(c->cw_epack),
                            P<int>(c->bond_of_edge), pc, P<unsigned long long>(c->cw_keys), out, wfail,
                            P<unsigned>(c->status), s))
      return fail(c, BOP_ERR_CUDA, "cluster pass 0 launch failed");
  }
  // the sizes and the flags of pass 0 in one synchronisation (the scans run
  // before it is known whether pass 0 succeeded; they are discarded if not)
  CKS(exclusive_scan(c, P<int>(c->atom_nsite), P<long long>(c->site_off), n + 1, s));
  CKS(exclusive_scan(c, P<int>(c->atom_nadj), P<long long>(c->adj_base), n + 1, s));
  long long tot[2];
  {
    Readback rb(c, s);
    CKS(rb.add(&tot[0], P<long long>(c->site_off) + n, sizeof(long long)));
    CKS(rb.add(&tot[1], P<long long>(c->adj_base) + n, sizeof(long long)));
    CKS(rb.add(c->maxlev, c->max_level.p, sizeof(int) * (K + 2)));
    CKS(rb.add(misc, c->cw_misc.p, 4 * sizeof(int)));
    CKS(rb.finish());  // synchronises
  }
  if (misc[1] != 0) return BOP_OK;  // too large for the warp builder
  c->nsite = tot[0];
  c->nadj = tot[1];
  CKS(ensure(c, c->site_atom, sizeof(int) * c->nsite));
  CKS(ensure(c, c->site_img, 3 * c->nsite));
  CKS(ensure(c, c->adj_off, sizeof(long long) * (c->nsite + 1)));
  CKS(ensure(c, c->adj, sizeof(int2) * c->nadj));
  CKS(ensure(c, c->lvcnt, sizeof(unsigned long long) * c->nsite));
  out.site_off = P<long long>(c->site_off);
  out.adj_base = P<long long>(c->adj_base);
  out.site_atom = P<int>(c->site_atom);
  out.site_img = P<signed char>(c->site_img);
  out.adj_off = P<long long>(c->adj_off);
  out.adj = P<int2>(c->adj);
  out.lvcnt = P<unsigned long long>(c->lvcnt);
  CKS(ensure(c, c->nprod, sizeof(unsigned long long)));
  CK(cudaMemsetAsync(c->nprod.p, 0, sizeof(unsigned long long), s));
  out.n_products = P<unsigned long long>(c->nprod);
  {
    Region R1(c, PK_CLUSTER, 1, s);
    if (launch_cluster_warp(1, n, K, max_deg, P<long long>(c->row_ptr), P<int2>(c->cw_epack),
                            P<int>(c->bond_of_edge), pc, P<unsigned long long>(c->cw_keys), out, wfail,
                            P<unsigned>(c->status), s))
      return fail(c, BOP_ERR_CUDA, "cluster pass 1 launch failed");
  }
  CK(cudaMemcpyAsync(P<long long>(c->adj_off) + c->nsite, P<long long>(c->adj_base) + n, sizeof(long long),
                     cudaMemcpyDeviceToDevice, s));
  *done = true;  // the status of pass 1 is read with the structure's last readback
  return BOP_OK;
}

int build_clusters(bop_ctx* c, cudaStream_t s) {
  const int n = c->nc, K = c->K;  // clusters of the centres
  {
    bool done = false;
    CKS(build_clusters_warp(c, s, &done));
    if (done) return BOP_OK;
  }
  int grid = n < 1216 ? n : 1216;
  int maxs = c->cl_maxs ? c->cl_maxs : (K <= 4 ? 1024 : (K <= 6 ? 2048 : 4096));
  CKS(ensure(c, c->level_end, sizeof(int) * (size_t)n * (K + 1)));
  CKS(ensure(c, c->atom_nsite, sizeof(int) * (n + 1)));
  CKS(ensure(c, c->atom_nadj, sizeof(int) * (n + 1)));
  CK(cudaMemsetAsync(c->atom_nsite.p, 0, sizeof(int) * (n + 1), s));
  CK(cudaMemsetAsync(c->atom_nadj.p, 0, sizeof(int) * (n + 1), s));
  CKS(ensure(c, c->max_level, sizeof(int) * (K + 2)));
  CKS(ensure(c, c->site_off, sizeof(long long) * (n + 1)));
  CKS(ensure(c, c->adj_base, sizeof(long long) * (n + 1)));
  for (int attempt = 0; attempt < 4; attempt++) {
    int hcap = 1;
    while (hcap < 2 * maxs) hcap <<= 1;
    int newcap = 1;
    while (newcap < maxs && newcap < 8192) newcap <<= 1;
    CKS(ensure(c, c->hkeys, sizeof(unsigned long long) * (size_t)grid * hcap));
    CKS(ensure(c, c->hvals, sizeof(int) * (size_t)grid * hcap));
    CKS(ensure(c, c->skeys, sizeof(unsigned long long) * (size_t)grid * maxs));
    CKS(ensure(c, c->sslot, sizeof(int) * (size_t)grid * maxs));
    CKS(ensure(c, c->scount, sizeof(int) * (size_t)grid * maxs));
    CK(cudaMemsetAsync(c->hkeys.p, 0xff, sizeof(unsigned long long) * (size_t)grid * hcap, s));
    CK(cudaMemsetAsync(c->max_level.p, 0, sizeof(int) * (K + 2), s));
    ClusterScratch sc{P<unsigned long long>(c->hkeys), P<int>(c->hvals), P<unsigned long long>(c->skeys),
                      P<int>(c->sslot), P<int>(c->scount), hcap, maxs, newcap};
    PathCut pc;
    pc.pos = P<double>(c->pos);
    for (int q = 0; q < 9; q++) pc.cell[q] = c->g.cell[q];
    pc.r2 = c->m.r_path > 0 ? c->m.r_path * c->m.r_path : 0.0;
    ClusterOut out{};
    out.level_end = P<int>(c->level_end);
    out.atom_nsite = P<int>(c->atom_nsite);
    out.atom_nadj = P<int>(c->atom_nadj);
    out.max_level = P<int>(c->max_level);
    {
    Region R0(c, PK_CLUSTER, 1, s);
    if (launch_cluster(0, n, K, P<long long>(c->row_ptr), P<int>(c->col), P<signed char>(c->img),
                       P<int>(c->bond_of_edge), pc, sc, out, grid, P<unsigned>(c->status), s))
      return fail(c, BOP_ERR_CUDA, "cluster pass 0 launch failed");
    }
    unsigned h = 0;
    {
      Readback rb(c, s);
      CKS(rb.add(&h, c->status.p, sizeof(unsigned)));
      CKS(rb.sync());
    }
    if (h & BOP_DEV_ERR_CLUSTER) {
      CK(cudaMemsetAsync(c->status.p, 0, sizeof(unsigned), s));
      maxs *= 2;
      continue;
    }
    CKS(check_status(c, s));
    c->cl_maxs = maxs;
    // offsets
    CKS(exclusive_scan(c, P<int>(c->atom_nsite), P<long long>(c->site_off), n + 1, s));
    CKS(exclusive_scan(c, P<int>(c->atom_nadj), P<long long>(c->adj_base), n + 1, s));
    long long tot[2];
    {
      Readback rb(c, s);
      CKS(rb.add(&tot[0], P<long long>(c->site_off) + n, sizeof(long long)));
      CKS(rb.add(&tot[1], P<long long>(c->adj_base) + n, sizeof(long long)));
      CKS(rb.add(c->maxlev, c->max_level.p, sizeof(int) * (K + 2)));
      CKS(rb.sync());
    }
    c->nsite = tot[0];
    c->nadj = tot[1];
    CKS(ensure(c, c->site_atom, sizeof(int) * c->nsite));
    CKS(ensure(c, c->site_img, 3 * c->nsite));
    CKS(ensure(c, c->adj_off, sizeof(long long) * (c->nsite + 1)));
    CKS(ensure(c, c->adj, sizeof(int2) * c->nadj));
    CKS(ensure(c, c->lvcnt, sizeof(unsigned long long) * c->nsite));
    out.site_off = P<long long>(c->site_off);
    out.adj_base = P<long long>(c->adj_base);
    out.site_atom = P<int>(c->site_atom);
    out.site_img = P<signed char>(c->site_img);
    out.adj_off = P<long long>(c->adj_off);
    out.adj = P<int2>(c->adj);
    out.lvcnt = P<unsigned long long>(c->lvcnt);
    CKS(ensure(c, c->nprod, sizeof(unsigned long long)));
    CK(cudaMemsetAsync(c->nprod.p, 0, sizeof(unsigned long long), s));
    out.n_products = P<unsigned long long>(c->nprod);
    {
    Region R1(c, PK_CLUSTER, 1, s);
    if (launch_cluster(1, n, K, P<long long>(c->row_ptr), P<int>(c->col), P<signed char>(c->img),
                       P<int>(c->bond_of_edge), pc, sc, out, grid, P<unsigned>(c->status), s))
      return fail(c, BOP_ERR_CUDA, "cluster pass 1 launch failed");
    }
    CK(cudaMemcpyAsync(P<long long>(c->adj_off) + c->nsite, P<long long>(c->adj_base) + n, sizeof(long long),
                       cudaMemcpyDeviceToDevice, s));
    return check_status(c, s);
  }
  return fail(c, BOP_ERR_OVERFLOW, "cluster larger than %d sites", maxs);
}

ClusterView cview(bop_ctx* c) {
  return ClusterView{P<long long>(c->site_off), P<int>(c->level_end), P<int>(c->site_atom),
                     P<long long>(c->adj_off), P<int2>(c->adj), P<unsigned long long>(c->lvcnt), c->K};
}

int size_state(bop_ctx* c) {
  const size_t M = (size_t)c->S * c->nc * c->norb;      // orbitals of the centres
  const size_t Mon = (size_t)c->S * c->n * c->norb;     // onsite levels of every atom
  CKS(ensure(c, c->onsite, sizeof(double) * Mon));
  CKS(ensure(c, c->onsite32, sizeof(float) * Mon));
  CKS(ensure(c, c->delta, sizeof(double) * c->n));
  CKS(ensure(c, c->mval, sizeof(double) * c->n));
  CKS(ensure(c, c->delta_new, sizeof(double) * c->n));
  CKS(ensure(c, c->m_new, sizeof(double) * c->n));
  CKS(ensure(c, c->mu, sizeof(double) * M * c->n_mom));
  CKS(ensure(c, c->a, sizeof(double) * M * c->Kp));
  CKS(ensure(c, c->b, sizeof(double) * M * (c->Kp + 1)));
  CKS(ensure(c, c->nlev, sizeof(int) * M));
  CKS(ensure(c, c->a_inf, sizeof(double) * M));
  CKS(ensure(c, c->b_inf, sizeof(double) * M));
  CKS(ensure(c, c->gsig, sizeof(double) * M * (c->n_exp + 1)));
  CKS(ensure(c, c->D, sizeof(double) * M * (c->n_exp + 3)));
  CKS(ensure(c, c->N, sizeof(double) * M));
  CKS(ensure(c, c->U, sizeof(double) * M));
  CKS(ensure(c, c->dos, sizeof(double) * M));
  CKS(ensure(c, c->e_atom, sizeof(double) * c->n));
  const int H = c->m.mixer == BOP_MIX_ANDERSON ? c->m.mix_history : 1;
  const size_t n2 = (size_t)c->n * (c->m.scf == BOP_SCF_STONER ? 2 : 1);
  CKS(ensure(c, c->hx, sizeof(double) * (H + 1) * n2));
  CKS(ensure(c, c->hf, sizeof(double) * (H + 1) * n2));
  CKS(ensure(c, c->gamma, sizeof(double) * 16));
  CKS(ensure(c, c->scfred, sizeof(double) * 64 * 1024));
  return BOP_OK;
}

// Columns per work item of the forward pass (all 5 starting orbitals when
// both stored levels fit in shared memory).
int forward_nc(bop_ctx* c) {
  int ce = 1, co = 1;
  for (int k = 0; k < c->K; k++) {
    int& cap = (k & 1) ? co : ce;
    if (c->maxlev[k] > cap) cap = c->maxlev[k];
  }
  return moments_columns(c->norb, ce + co, c->fp64);
}

// Arguments of the spinor kernel (non-collinear magnetism): per-CTA scratch
// for Psi and Psi-bar of all levels of one work item.
int nc_args(bop_ctx* c, NcArgs* a) {
  if (c->sdir_n != c->n) return fail(c, BOP_ERR_STATE, "noncollinear model: bop_set_spin_directions first");
  memset(a, 0, sizeof(*a));
  a->cv = cview(c);
  a->H = c->fp64 ? c->H64.p : c->H32.p;
  a->HS = c->HS;
  a->onsite = c->fp64 ? c->onsite.p : c->onsite32.p;
  a->sdir = P<double>(c->sdir);
  a->n = c->n;
  a->norb = c->norb;
  a->n_mom = c->n_mom;
  a->cap_even = a->cap_odd = 1;
  for (int k = 0; k < c->K; k++) {  // level K is never stored by the forward pass
    int& cap = (k & 1) ? a->cap_odd : a->cap_even;
    if (c->maxlev[k] > cap) cap = c->maxlev[k];
  }
  long long levsum = 0;
  for (int k = 0; k <= c->K; k++) levsum += c->maxlev[k];
  a->slot_elems = 2 * (size_t)levsum * c->norb * 8 + 64;
  const int nwork = c->n * c->norb;
  a->slots = nwork < 1216 ? nwork : 1216;
  const size_t esz = c->fp64 ? sizeof(double) : sizeof(float);
  CKS(ensure(c, c->ncscr, esz * a->slot_elems * (a->slots > 0 ? a->slots : 1)));
  a->scratch = c->ncscr.p;
  return BOP_OK;
}

int run_moments(bop_ctx* c, const double* onsite_dev, double* mu, cudaStream_t s, void* pstore = nullptr) {
  if (c->m.noncollinear) {  // the onsite levels are in c->onsite / c->onsite32
    NcArgs a;
    CKS(nc_args(c, &a));
    CKS(ensure(c, c->vmom, sizeof(double) * (size_t)c->n * c->norb * c->n_mom * 3));
    a.mu = mu;
    a.vmom = P<double>(c->vmom);
    Region R(c, PK_MOMENTS, 1, s);
    if (launch_nc(a, c->fp64, s)) return fail(c, BOP_ERR_CUDA, "spinor moments launch failed");
    return BOP_OK;
  }
  MomentsArgs a;
  a.cv = cview(c);
  a.H = c->fp64 ? c->H64.p : c->H32.p;
  a.HS = c->HS;
  a.onsite = c->fp64 ? (const void*)onsite_dev : (const void*)c->onsite32.p;
  a.n = c->nc;
  a.n_on = c->n;
  a.n_spin = c->S;
  a.norb = c->norb;
  a.n_mom = c->n_mom;
  a.max_sites = c->maxlev[c->K] > 0 ? c->maxlev[c->K] : 1;
  a.max_adj = c->maxlev[c->K + 1] > 0 ? c->maxlev[c->K + 1] : 1;
  a.cap_even = a.cap_odd = 1;
  for (int k = 0; k < c->K; k++) {  // level K is never stored
    int& cap = (k & 1) ? a.cap_odd : a.cap_even;
    if (c->maxlev[k] > cap) cap = c->maxlev[k];
  }
  a.mu = mu;
  a.pstore = pstore;
  a.psi_off = P<long long>(c->psi_off);
  a.psi_tot = c->psi_tot;
  Region R(c, PK_MOMENTS, 1, s);
  int r = launch_moments(a, c->fp64, s);
  if (r == -2) return fail(c, BOP_ERR_OVERFLOW, "cluster level too large for shared memory");
  if (r) return fail(c, BOP_ERR_CUDA, "moments launch: %s", cudaGetErrorString(cudaGetLastError()));
  return BOP_OK;
}

LearnedArgs learned_args(bop_ctx* c, int M, const double* mu) {
  LearnedArgs L;
  L.M = M;
  L.n_exp = c->n_exp;
  L.fp64 = c->fp64;
  L.sig32 = sig32_mode(c);
  L.mu = mu;
  L.base = P<double>(c->lbase);
  L.nlev = P<int>(c->lnlev);
  L.flag = P<unsigned char>(c->lflag);
  L.xs = c->lxs.p;
  L.ys = c->lys.p;
  L.norm = mlp_norm_dev(c->net);
  L.a_inf = P<double>(c->a_inf);
  L.b_inf = P<double>(c->b_inf);
  L.gsig = P<double>(c->gsig);
  L.g = P<double>(c->gjack);
  L.n_learned = P<unsigned>(c->lcount);
  L.status = P<unsigned>(c->status);
  L.ybar = c->lybar.p;
  L.cot = P<double>(c->lcot);
  L.xbar = c->lxbar.p;
  memset(&L.W, 0, sizeof(L.W));
  return L;
}

// Learned terminator: features -> network -> continued chain -> g_m sigma_m.
int run_learned(bop_ctx* c, int M, const double* mu, cudaStream_t s) {
  if (!c->net) return fail(c, BOP_ERR_STATE, "terminator MLP needs a network (bop_set_mlp)");
  const size_t T = c->fp64 ? sizeof(double) : sizeof(float);
  const size_t m = (size_t)M;
  CKS(ensure(c, c->lbase, sizeof(double) * m * 10));
  CKS(ensure(c, c->lnlev, sizeof(int) * m));
  CKS(ensure(c, c->lflag, m));
  CKS(ensure(c, c->lxs, T * m * BOP_MLP_NIN));
  CKS(ensure(c, c->lys, T * m * BOP_MLP_NOUT));
  CKS(ensure(c, c->lZ1, T * m * BOP_MLP_NHID));
  CKS(ensure(c, c->lH1, T * m * BOP_MLP_NHID));
  CKS(ensure(c, c->lZ2, T * m * BOP_MLP_NHID));
  CKS(ensure(c, c->lH2, T * m * BOP_MLP_NHID));
  CKS(ensure(c, c->lcount, 2 * sizeof(unsigned)));
  LearnedArgs L = learned_args(c, M, mu);
  CK(cudaMemsetAsync(c->lcount.p, 0, 2 * sizeof(unsigned), s));
  {
    Region R(c, PK_EXPAND, 1, s);
    if (launch_learned(0, L, s)) return fail(c, BOP_ERR_CUDA, "features launch failed");
  }
  {
    Region R(c, PK_MLP, 3, s);
    if (mlp_infer_forward(c->fp64, M, c->lxs.p, mlp_params_dev(c->net), mlp_wbf_dev(c->net), c->lZ1.p, c->lH1.p,
                          c->lZ2.p, c->lH2.p, c->lys.p, s))
      return fail(c, BOP_ERR_CUDA, "network launch failed");
  }
  Region R(c, PK_EXPAND, 1, s);
  if (launch_learned(1, L, s)) return fail(c, BOP_ERR_CUDA, "continued-chain expansion launch failed");
  return BOP_OK;
}

int run_scalar(bop_ctx* c, int M, const double* mu, cudaStream_t s) {
  if (c->m.terminator == BOP_TERM_MLP) return run_learned(c, M, mu, s);
  ScalarArgs a;
  a.M = M;
  a.n_mom = c->n_mom;
  a.n_exp = c->n_exp;
  a.mu = mu;
  a.a = P<double>(c->a);
  a.b = P<double>(c->b);
  a.nlev = P<int>(c->nlev);
  a.a_inf = P<double>(c->a_inf);
  a.b_inf = P<double>(c->b_inf);
  a.gsig = P<double>(c->gsig);
  a.g = P<double>(c->gjack);
  a.status = P<unsigned>(c->status);
  a.bw = band_sel(c->m);
  // lcount: [0] learned orbitals, [1] orbitals outside the estimated band
  // (checked for the estimates other than Gershgorin, whose band holds every
  // Gershgorin disc; the check costs FP64 work in every coefficient)
  CKS(ensure(c, c->lcount, 2 * sizeof(unsigned)));
  CK(cudaMemsetAsync(c->lcount.p, 0, 2 * sizeof(unsigned), s));
  a.n_unbounded = c->m.bandwidth != BOP_BW_GERSHGORIN ? P<unsigned>(c->lcount) + 1 : nullptr;
  a.sig32 = sig32_mode(c);
  Region R(c, PK_EXPAND, 1, s);
  if (launch_expand(a, s)) return fail(c, BOP_ERR_CUDA, "expand launch failed");
  return BOP_OK;
}

// Sum (or max) of v[0..n) over the processes of a spatial decomposition;
// nothing with one process.
int reduce_over_ranks(bop_ctx* c, double* v, int n, int op) {
  if (!c->reduce_fn) return BOP_OK;
  if (c->reduce_fn(v, n, op, c->reduce_user) != 0) return fail(c, BOP_ERR_COLLECTIVE, "reduce callback failed");
  return BOP_OK;
}

// Fermi level over several processes ("DOS and Fermi energy": one E_F for
// the whole structure): the bracket and the sums of every Newton round are
// this process's, reduced over the processes, and the update rules are those
// of k_fermi_newton; then N and DOS of this process's orbitals at E_F.
int fermi_distributed(bop_ctx* c, int warm, cudaStream_t s) {
  const int M = c->S * c->nc * c->norb;
  CKS(ensure(c, c->fev, 2 * sizeof(double)));
  double ncg = (double)c->nc;
  CKS(reduce_over_ranks(c, &ncg, 1, BOP_REDUCE_SUM));
  const double target = c->m.n_e * ncg;
  double v[2];
  auto eval = [&](int mode, double E) -> int {
    {
      Region R(c, PK_FERMI, 1, s);
      if (launch_fermi_eval(mode, M, P<double>(c->gsig), P<double>(c->ginv), P<double>(c->a_inf),
                            P<double>(c->b_inf), c->n_exp, E, P<double>(c->partials), P<unsigned>(c->counter),
                            P<double>(c->fev), s))
        return fail(c, BOP_ERR_CUDA, "fermi launch failed");
    }
    {
      Readback rb(c, s);
      CKS(rb.add(v, c->fev.p, 2 * sizeof(double)));
      CKS(rb.sync());
    }
    return reduce_over_ranks(c, v, 2, mode == 0 ? BOP_REDUCE_MAX : BOP_REDUCE_SUM);
  };
  CKS(eval(0, 0.0));
  double lo = -v[0] - 1e-3, hi = v[1] + 1e-3;
  double E = (warm && c->ef_solved && c->ef_host > lo && c->ef_host < hi) ? c->ef_host : 0.5 * (lo + hi);
  FermiState fs;
  memset(&fs, 0, sizeof(fs));
  double ef = 0.5 * (lo + hi);
  const double ftol = fermi_tol(c);
  bool done = hi - lo < ftol;
  while (!done) {
    CKS(eval(1, E));
    const double f = c->sfac * v[0] - target, fp = c->sfac * v[1];
    fs.iters++;
    if (f == 0.0) {
      ef = E;
      break;
    }
    if (f < 0.0) lo = E;
    else hi = E;
    double xn = fp > 0.0 ? E - f / fp : lo - 1.0;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (std::fabs(xn - E) < ftol || hi - lo < ftol || fs.iters >= FERMI_MAX_ROUNDS) {
      ef = xn;
      done = true;
    } else {
      E = xn;
    }
  }
  if (fs.iters >= FERMI_MAX_ROUNDS)
    return fail(c, BOP_ERR_BRACKET, "Fermi level not converged after %d rounds", fs.iters);
  fs.lo = lo;
  fs.hi = hi;
  fs.mid = E;
  fs.ef = ef;
  fs.done = 1;
  c->ef_host = ef;
  CK(cudaMemcpyAsync(c->fstate.p, &fs, sizeof(fs), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  Region R(c, PK_NU, 1, s);
  if (launch_orbital_N(M, c->n_exp, P<double>(c->gsig), P<double>(c->ginv), P<double>(c->a_inf),
                       P<double>(c->b_inf), P<FermiState>(c->fstate), P<double>(c->N), P<double>(c->dos), s))
    return fail(c, BOP_ERR_CUDA, "orbital N launch failed");
  return BOP_OK;
}

// Fermi level (Newton steps inside the bisection bracket) and N, DOS of every
// orbital at E_F.  warm: start from the previous solve's E_F.
int fermi_and_N(bop_ctx* c, int warm, cudaStream_t s) {
  if (c->reduce_fn) return fermi_distributed(c, warm, s);
  const int M = c->S * c->nc * c->norb;
  const double target = c->m.n_e * c->nc;
  {
    // one cooperative launch: bracket, Newton rounds to convergence, N and DOS;
    // a cold start of many orbitals takes its starting point from Newton
    // rounds on an FP32 copy of the coefficients (the FP64 rounds that follow
    // decide the root, inside the full bracket)
    const float* gs32 = nullptr;
    if (!warm && M >= FERMI_F32_START) {
      CKS(ensure(c, c->gs32, sizeof(float) * (size_t)M * (c->n_exp + 1)));
      Region R(c, PK_FERMI, 1, s);
      if (launch_gsig_f32(M, c->n_exp, P<double>(c->gsig), P<float>(c->gs32), s))
        return fail(c, BOP_ERR_CUDA, "fermi launch failed");
      gs32 = P<float>(c->gs32);
    }
    Region R(c, PK_FERMI, 1, s);
    const int r = launch_fermi_coop(M, P<double>(c->gsig), P<double>(c->ginv), P<double>(c->a_inf),
                                    P<double>(c->b_inf), c->n_exp, c->sfac, target, P<FermiState>(c->fstate),
                                    P<double>(c->partials), warm, FERMI_MAX_ROUNDS, fermi_tol(c), P<double>(c->N),
                                    P<double>(c->dos), s, gs32);
    if (r == 0) return BOP_OK;
    if (r != -2) return fail(c, BOP_ERR_CUDA, "fermi launch failed");
  }
  const int rounds = warm ? FERMI_ROUNDS_WARM : FERMI_ROUNDS_COLD;
  {
    Region R(c, PK_FERMI, 1 + rounds, s);
    if (launch_fermi_newton(M, P<double>(c->gsig), P<double>(c->ginv), P<double>(c->a_inf), P<double>(c->b_inf),
                            c->n_exp, c->sfac, target, P<FermiState>(c->fstate), P<double>(c->partials),
                            P<unsigned>(c->counter), warm, rounds, FERMI_MAX_ROUNDS, fermi_tol(c), s))
      return fail(c, BOP_ERR_CUDA, "fermi launch failed");
  }
  Region R(c, PK_NU, 1, s);
  if (launch_orbital_N(M, c->n_exp, P<double>(c->gsig), P<double>(c->ginv), P<double>(c->a_inf),
                       P<double>(c->b_inf), P<FermiState>(c->fstate), P<double>(c->N), P<double>(c->dos), s))
    return fail(c, BOP_ERR_CUDA, "orbital N launch failed");
  return BOP_OK;
}

// More Newton rounds for a solve that has not converged, then N and DOS again.
int fermi_more(bop_ctx* c, cudaStream_t s) {
  const int M = c->S * c->nc * c->norb;
  {
    Region R(c, PK_FERMI, FERMI_ROUNDS_MORE, s);
    if (launch_fermi_more(M, P<double>(c->gsig), P<double>(c->ginv), P<double>(c->a_inf), P<double>(c->b_inf),
                          c->n_exp, c->sfac, c->m.n_e * c->nc, P<FermiState>(c->fstate), P<double>(c->partials),
                          P<unsigned>(c->counter), FERMI_ROUNDS_MORE, FERMI_MAX_ROUNDS, fermi_tol(c), s))
      return fail(c, BOP_ERR_CUDA, "fermi launch failed");
  }
  Region R(c, PK_NU, 1, s);
  if (launch_orbital_N(M, c->n_exp, P<double>(c->gsig), P<double>(c->ginv), P<double>(c->a_inf),
                       P<double>(c->b_inf), P<FermiState>(c->fstate), P<double>(c->N), P<double>(c->dos), s))
    return fail(c, BOP_ERR_CUDA, "orbital N launch failed");
  return BOP_OK;
}


// Weights of L = cU U + cN N for every orbital (cN = -cU * lam[0] with a
// device lam, else cN0), through the constant- or learned-terminator path,
// into w [M][n_mom]; dUE [M] = direct dL/dE (may be NULL).
int compute_weights(bop_ctx* c, double cU, const double* lam, double cN0, double* w, double* dUE, cudaStream_t s,
                    const double* var_q = nullptr, const double* var_lam = nullptr, double var_J = 0.0) {
  const int M = c->S * c->nc * c->norb;
  WeightArgs wa;
  wa.M = M;
  wa.n_mom = c->n_mom;
  wa.n_exp = c->n_exp;
  wa.norb = c->norb;
  wa.mu = P<double>(c->mu);
  wa.onsite = P<double>(c->onsite);
  wa.st = P<FermiState>(c->fstate);
  wa.g = P<double>(c->gjack);
  wa.inv = P<double>(c->ginv);
  wa.cU = cU;
  wa.lam = lam;
  wa.cN0 = cN0;
  wa.w = w;
  wa.dU_dE = dUE;
  wa.zscratch = P<double>(c->zscr);
  wa.status = P<unsigned>(c->status);
  wa.bw = band_sel(c->m);
  wa.sig32 = sig32_mode(c);
  wa.var_q = var_q;
  wa.var_lam = var_lam;
  wa.var_J = var_J;
  if (c->m.terminator == BOP_TERM_MLP) {
    if (!c->net) return fail(c, BOP_ERR_STATE, "terminator MLP needs a network (bop_set_mlp)");
    const size_t T = c->fp64 ? sizeof(double) : sizeof(float);
    CKS(ensure(c, c->lybar, T * (size_t)M * BOP_MLP_NOUT));
    CKS(ensure(c, c->lcot, sizeof(double) * (size_t)M * 10));
    CKS(ensure(c, c->lxbar, T * (size_t)M * BOP_MLP_NIN));
    LearnedArgs L = learned_args(c, M, P<double>(c->mu));
    L.W = wa;
    {
      Region R(c, PK_WEIGHTS, 1, s);
      if (launch_learned(2, L, s)) return fail(c, BOP_ERR_CUDA, "weights launch failed");
    }
    {
      Region R(c, PK_MLP, 3, s);
      if (mlp_infer_backward(c->fp64, M, c->lybar.p, mlp_wbf_dev(c->net), c->lZ1.p, c->lZ2.p, c->lH1.p, c->lH2.p,
                             c->lxbar.p, s))
        return fail(c, BOP_ERR_CUDA, "network reverse launch failed");
    }
    Region R(c, PK_WEIGHTS, 1, s);
    if (launch_learned(3, L, s)) return fail(c, BOP_ERR_CUDA, "weights launch failed");
    return BOP_OK;
  }
  Region R(c, PK_WEIGHTS, 1, s);
  if (launch_weights(wa, s)) return fail(c, BOP_ERR_CUDA, "weights launch failed");
  return BOP_OK;
}

// Row padding of a stored Psi row (norb x nc values), as in the kernels.
int psi_row(int N, int fp64) {
  if (N == 1) return 1;
  return fp64 ? (N + 1) / 2 * 2 : (N + 3) / 4 * 4;
}

// Stores Psi of every work item (one more forward pass at the current
// onsite levels) when it fits: all starting orbitals share one work item
// (the stored-Psi sweep keeps two Psi-bar levels of all five columns in
// shared memory; with one column per item it gathers every block five times
// and is slower than recomputing), and the store fits in a third of the free
// device memory and the store budget (psi_store_alloc).  Otherwise the
// reverse sweeps recompute Psi.
int psi_store_alloc(bop_ctx* c, bool* fits) {
  *fits = false;
  const int nc = forward_nc(c);
  if (c->norb > 1 && nc != c->norb) return BOP_OK;
  const size_t esz = c->fp64 ? sizeof(double) : sizeof(float);
  const size_t bytes = (size_t)c->S * (c->norb / nc) * (size_t)c->psi_tot * psi_row(c->norb * nc, c->fp64) * esz;
  size_t freeb = 0, totalb = 0;
  CK(cudaMemGetInfo(&freeb, &totalb));
  const size_t held = c->psis.bytes;
  if (bytes > (freeb + held) / 3 || bytes > c->store_budget) return BOP_OK;
  CKS(ensure(c, c->psis, bytes));
  *fits = true;
  return BOP_OK;
}

int prepare_psi_store(bop_ctx* c, cudaStream_t s) {
  // the SCF loop may have stored Psi in its forward passes; the last one is
  // at the final onsite levels
  c->forces_follow = !c->m.noncollinear;
  if (c->m.scf == BOP_SCF_VARIATIONAL || c->psi_valid || c->m.noncollinear) return BOP_OK;
  // a forward pass that stores Psi and the stored-Psi sweeps cost less than
  // the recomputing sweep even for one sweep (131,072 atoms: 12 + 21 ms
  // against 71 ms), so store whenever it fits
  bool fits = false;
  CKS(psi_store_alloc(c, &fits));
  if (!fits) return BOP_OK;
  CKS(run_moments(c, P<double>(c->onsite), P<double>(c->mu), s, c->psis.p));
  c->psi_valid = true;
  return BOP_OK;
}

// One reverse sweep of the moments with weights w: Hbar += dL/dH (if not
// NULL), Ebar += dL/dE (if not NULL).  Over the stored Psi when present.
int adjoint_pass(bop_ctx* c, const double* w, void* Hbar, double* Ebar, cudaStream_t s,
                 double* siteval = nullptr) {
  const int n = c->nc;
  AdjointArgs aa;
  memset(&aa, 0, sizeof(aa));
  aa.n_on = c->n;
  aa.cv = cview(c);
  aa.H = c->fp64 ? c->H64.p : c->H32.p;
  aa.HS = c->HS;
  aa.onsite = c->fp64 ? c->onsite.p : c->onsite32.p;
  aa.n = n;
  aa.n_spin = c->S;
  aa.norb = c->norb;
  aa.n_mom = c->n_mom;
  aa.w = w;
  aa.Hbar = Hbar;
  aa.HSh = bond_cotangent_stride(c->norb, c->fp64);
  aa.Ebar = Ebar;
  if (c->psi_valid) {
    aa.pstore = c->psis.p;
    aa.psi_off = P<long long>(c->psi_off);
    aa.psi_tot = c->psi_tot;
    aa.nc = forward_nc(c);
    int ce = 1, co = 1;
    for (int k = 1; k <= c->K; k++) {
      int& cap = (k & 1) ? co : ce;
      if (c->maxlev[k] > cap) cap = c->maxlev[k];
    }
    aa.cap_even = ce;
    aa.cap_odd = co;
    aa.max_sites = c->maxlev[c->K] > 0 ? c->maxlev[c->K] : 1;
    aa.max_adj = c->maxlev[c->K + 1] > 0 ? c->maxlev[c->K + 1] : 1;
    aa.cap_eb = c->maxlev[c->K - 1] > 0 ? c->maxlev[c->K - 1] : 1;
    aa.siteval = siteval;
    aa.sv_stride = c->nsite;
  } else {
    if (siteval) return fail(c, BOP_ERR_STATE, "per-site cotangents need the stored Psi");
    int nc = adjoint_columns(c->norb);
    size_t per_site = (size_t)c->norb * nc;
    long long levsum = 0;
    for (int k = 0; k <= c->K; k++) levsum += c->maxlev[k];
    size_t slot_elems = (2 * (size_t)levsum) * per_site + 64;
    int nwork = n * c->S * (c->norb / nc);
    int slots = nwork < 1216 ? nwork : 1216;
    size_t esz = c->fp64 ? sizeof(double) : sizeof(float);
    CKS(ensure(c, c->adjscr, esz * slot_elems * slots));
    aa.scratch = c->adjscr.p;
    aa.slot_elems = slot_elems;
    aa.slots = slots;
  }
  Region R(c, PK_ADJOINT, 1, s);
  const int r = launch_moments_adjoint(aa, c->fp64, s);
  if (r == -2) return fail(c, BOP_ERR_OVERFLOW, "cluster level too large for shared memory");
  if (r) return fail(c, BOP_ERR_CUDA, "adjoint launch failed");
  return BOP_OK;
}

constexpr int GM_KRYLOV = 40;   // GMRES basis size per cycle
constexpr int GM_CYCLES = 3;    // cycles (restarts + 1)

// Reads nv doubles from the device (synchronises s).
int read_back(bop_ctx* c, const double* d, double* h, int nv, cudaStream_t s) {
  Readback rb(c, s);
  CKS(rb.add(h, d, sizeof(double) * nv));
  return rb.sync();
}

// SCF response of the forces: weights w = wU - c wN with the multipliers y
// of J^T y = dE/du (see bop_forces), then Hbar from one reverse sweep.
int scf_response(bop_ctx* c, cudaStream_t s) {
  const int n = c->n, S = c->S, norb = c->norb, nm = c->n_mom;
  const int M = S * n * norb;
  const bool stoner = c->m.scf == BOP_SCF_STONER;
  const int nu = stoner ? 2 * n : n;
  const double I = c->m.stoner_I;
  // FP32 products: 1e-6 reaches the FP32 noise floor of the forces (measured
  // on the 2,000-atom LCN / Stoner cells against the FP64 oracle: 1e-5 /
  // 9e-5 eV/A, against 1e-3 / 6e-3 at 1e-4) for a few more iterations
  const double rtol = c->resp_rtol > 0.0 ? c->resp_rtol : (c->fp64 ? 1e-10 : 1e-6);
  const int max_it = c->resp_max_it > 0 ? c->resp_max_it : GM_KRYLOV * GM_CYCLES;
  CKS(ensure(c, c->rwN, sizeof(double) * (size_t)M * nm));
  CKS(ensure(c, c->rwt, sizeof(double) * (size_t)M * nm));
  CKS(ensure(c, c->rdUE, sizeof(double) * (size_t)M));
  CKS(ensure(c, c->rvec, sizeof(double) * (size_t)nu * (GM_KRYLOV + 6)));
  // coef: [0, K+2) host-set coefficients; then the Gram-Schmidt passes and
  // the norm of one Arnoldi step, read back together
  CKS(ensure(c, c->rcoef, sizeof(double) * (3 * GM_KRYLOV + 8)));
  double* V = P<double>(c->rvec);                 // Krylov basis [GM_KRYLOV + 1][nu]
  double* rhs = V + (size_t)(GM_KRYLOV + 1) * nu;  // dE/du
  double* Pd = rhs + nu;                           // diagonal preconditioner
  double* tmp = Pd + nu;
  double* y = tmp + nu;                            // solution
  double* yc = y + nu;                             // one cycle's correction
  double* coef = P<double>(c->rcoef);
  double* wU = P<double>(c->w);
  double* wN = P<double>(c->rwN);
  double* Eb = P<double>(c->Ebar);
  // weights of U (fixed E_F, no multiplier) and of N
  if (c->m.terminator == BOP_TERM_MLP) {
    CKS(compute_weights(c, c->sfac, nullptr, 0.0, wU, P<double>(c->rdUE), s));
    CKS(compute_weights(c, 0.0, nullptr, 1.0, wN, nullptr, s));
  } else {  // both from one forward pass of the chain
    CKS(ensure(c, c->zscr, sizeof(double) * (size_t)M * (c->n_exp + 1) * 4));
    WeightArgs wa;
    wa.M = M;
    wa.n_mom = c->n_mom;
    wa.n_exp = c->n_exp;
    wa.norb = c->norb;
    wa.mu = P<double>(c->mu);
    wa.onsite = P<double>(c->onsite);
    wa.st = P<FermiState>(c->fstate);
    wa.g = P<double>(c->gjack);
    wa.inv = P<double>(c->ginv);
    wa.cU = 0.0;
    wa.lam = nullptr;
    wa.cN0 = 0.0;
    wa.w = wU;
    wa.dU_dE = P<double>(c->rdUE);
    wa.zscratch = P<double>(c->zscr);
    wa.status = P<unsigned>(c->status);
    wa.bw = band_sel(c->m);
    wa.var_q = wa.var_lam = nullptr;
    wa.var_J = 0.0;
    wa.sig32 = sig32_mode(c);
    Region R(c, PK_WEIGHTS, 1, s);
    if (launch_weights_pair(wa, c->sfac, 0.0, 0.0, 1.0, wN, s)) return fail(c, BOP_ERR_CUDA, "weights launch failed");
  }
  // right-hand side g = dE/du
  CK(cudaMemsetAsync(Eb, 0, sizeof(double) * M, s));
  CKS(adjoint_pass(c, wU, nullptr, Eb, s));
  if (launch_project(n, norb, S, I, Eb, P<double>(c->rdUE), stoner ? P<double>(c->mval) : nullptr, -0.5 * I,
                     nullptr, rhs, s) ||
      launch_precond_diag(n, norb, S, c->sfac, c->m.dos_floor, P<double>(c->dos), Pd, s))
    return fail(c, BOP_ERR_CUDA, "response kernels failed");
  // J^T v -> out.  With the stored Psi, one sweep with the dN/dmu weights
  // gives every row of J as per-site values (the weights of a product only
  // scale each work item's), and each product is then a sparse pass over
  // them instead of a reverse sweep.
  const bool use_rows = c->psi_valid;
  if (use_rows) {
    const size_t ns = (size_t)(c->nsite > 0 ? c->nsite : 1);
    CKS(ensure(c, c->rjv, sizeof(double) * (size_t)S * ns));
    CKS(ensure(c, c->rjcnt, sizeof(int) * (size_t)(n + 1)));
    CKS(ensure(c, c->rjptr, sizeof(long long) * (size_t)(n + 1)));
    CKS(ensure(c, c->rjidx, sizeof(long long) * ns));
    CKS(ensure(c, c->rjrow, sizeof(int) * ns));
    CK(cudaMemsetAsync(c->rjv.p, 0, sizeof(double) * (size_t)S * c->nsite, s));
    CKS(adjoint_pass(c, wN, nullptr, nullptr, s, P<double>(c->rjv)));
    // transpose of the rows (structure only)
    CK(cudaMemsetAsync(c->rjcnt.p, 0, sizeof(int) * (size_t)(n + 1), s));
    if (launch_jt_build(n, c->K, P<long long>(c->site_off), P<int>(c->level_end), P<int>(c->site_atom),
                        P<int>(c->rjcnt), 0, nullptr, nullptr, nullptr, s))
      return fail(c, BOP_ERR_CUDA, "response kernels failed");
    CKS(exclusive_scan(c, P<int>(c->rjcnt), P<long long>(c->rjptr), n + 1, s));
    CK(cudaMemsetAsync(c->rjcnt.p, 0, sizeof(int) * (size_t)(n + 1), s));
    if (launch_jt_build(n, c->K, P<long long>(c->site_off), P<int>(c->level_end), P<int>(c->site_atom),
                        P<int>(c->rjcnt), 1, P<long long>(c->rjptr), P<long long>(c->rjidx), P<int>(c->rjrow), s))
      return fail(c, BOP_ERR_CUDA, "response kernels failed");
  }
  auto matvec = [&](const double* v, double* out) -> int {
    if (use_rows) {
      if (launch_jt_gather(n, S, P<long long>(c->rjptr), P<long long>(c->rjidx), P<int>(c->rjrow),
                           P<double>(c->rjv), c->nsite, v, c->sfac, stoner ? 1 : 0, Eb, s) ||
          launch_project(n, 1, S, I, Eb, nullptr, nullptr, 0.0, stoner ? v + n : nullptr, out, s))
        return fail(c, BOP_ERR_CUDA, "response kernels failed");
      return BOP_OK;
    }
    if (launch_scale_weights(n, norb, S, nm, c->sfac, stoner ? 1 : 0, v, 1.0, wN, nullptr, P<double>(c->rwt), s))
      return fail(c, BOP_ERR_CUDA, "response kernels failed");
    CK(cudaMemsetAsync(Eb, 0, sizeof(double) * M, s));
    CKS(adjoint_pass(c, P<double>(c->rwt), nullptr, Eb, s));
    if (launch_project(n, norb, S, I, Eb, nullptr, nullptr, 0.0, stoner ? v + n : nullptr, out, s))
      return fail(c, BOP_ERR_CUDA, "response kernels failed");
    return BOP_OK;
  };
  auto dot = [&](const double* a, const double* b, double* h) -> int {
    if (launch_dots(nu, 1, a, b, coef, s)) return fail(c, BOP_ERR_CUDA, "response kernels failed");
    return read_back(c, coef, h, 1, s);
  };
  CK(cudaMemsetAsync(y, 0, sizeof(double) * nu, s));
  double bnorm = 0.0;
  CKS(dot(rhs, rhs, &bnorm));
  bnorm = std::sqrt(bnorm);
  int iters = 0;
  double rel = 0.0;
  bool conv = bnorm == 0.0;
  const double one = 1.0, minus_one = -1.0;
  for (int cyc = 0; cyc < GM_CYCLES && !conv && iters < max_it; cyc++) {
    // residual r = g - J^T y into V_0
    CK(cudaMemcpyAsync(V, rhs, sizeof(double) * nu, cudaMemcpyDeviceToDevice, s));
    if (cyc > 0) {
      CKS(matvec(y, tmp));
      CK(cudaMemcpyAsync(coef, &one, sizeof(double), cudaMemcpyHostToDevice, s));
      if (launch_axpy_multi(nu, 1, tmp, coef, V, s)) return fail(c, BOP_ERR_CUDA, "response kernels failed");
    }
    double beta = bnorm;  // y = 0 in the first cycle: the residual is g
    if (cyc > 0) {
      CKS(dot(V, V, &beta));
      beta = std::sqrt(beta);
    }
    if (beta <= rtol * bnorm) {
      conv = true;
      rel = beta / bnorm;
      break;
    }
    if (launch_scale_vec(nu, V, nullptr, 1.0 / beta, V, s)) return fail(c, BOP_ERR_CUDA, "response kernels failed");
    double Hh[GM_KRYLOV + 1][GM_KRYLOV], cs[GM_KRYLOV], sn[GM_KRYLOV], gv[GM_KRYLOV + 1];
    for (int q = 0; q <= GM_KRYLOV; q++) gv[q] = 0.0;
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < GM_KRYLOV; j++) {
      double* vj = V + (size_t)j * nu;
      double* u = V + (size_t)(j + 1) * nu;
      if (launch_scale_vec(nu, vj, Pd, 1.0, tmp, s)) return fail(c, BOP_ERR_CUDA, "response kernels failed");
      CKS(matvec(tmp, u));
      // classical Gram-Schmidt, twice, with the coefficients kept on the
      // device; then |u|^2 and u / |u| (device norm): one readback per step
      double* gs1 = coef + GM_KRYLOV + 2;
      double* gs2 = gs1 + GM_KRYLOV + 1;
      double* nrm = gs2 + GM_KRYLOV + 1;
      if (launch_dots(nu, j + 1, V, u, gs1, s) || launch_axpy_multi(nu, j + 1, V, gs1, u, s) ||
          launch_dots(nu, j + 1, V, u, gs2, s) || launch_axpy_multi(nu, j + 1, V, gs2, u, s) ||
          launch_dots(nu, 1, u, u, nrm, s) || launch_scale_by_inv_norm(nu, u, nrm, s))
        return fail(c, BOP_ERR_CUDA, "response kernels failed");
      double hb[3 * GM_KRYLOV + 4];
      CKS(read_back(c, gs1, hb, 2 * (GM_KRYLOV + 1) + 1, s));
      double h[GM_KRYLOV + 1];
      for (int q = 0; q <= j; q++) h[q] = hb[q] + hb[GM_KRYLOV + 1 + q];
      const double hn = std::sqrt(hb[2 * (GM_KRYLOV + 1)]);
      // Givens rotations on the new Hessenberg column
      for (int q = 0; q < j; q++) {
        const double t0 = cs[q] * h[q] + sn[q] * h[q + 1];
        h[q + 1] = -sn[q] * h[q] + cs[q] * h[q + 1];
        h[q] = t0;
      }
      const double rr = std::hypot(h[j], hn);
      cs[j] = rr > 0.0 ? h[j] / rr : 1.0;
      sn[j] = rr > 0.0 ? hn / rr : 0.0;
      h[j] = rr;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      for (int q = 0; q <= j; q++) Hh[q][j] = h[q];
      k = j + 1;
      iters++;
      rel = std::fabs(gv[j + 1]) / bnorm;
      if (rel <= rtol || hn == 0.0 || iters >= max_it) break;
    }
    // z = H^-1 g (upper triangular), y += P sum z_q V_q
    double z[GM_KRYLOV];
    for (int q = k - 1; q >= 0; q--) {
      double a = gv[q];
      for (int r = q + 1; r < k; r++) a -= Hh[q][r] * z[r];
      z[q] = a / Hh[q][q];
    }
    CK(cudaMemcpyAsync(coef, z, sizeof(double) * k, cudaMemcpyHostToDevice, s));
    if (launch_lincomb(nu, k, V, coef, Pd, 1.0, yc, s)) return fail(c, BOP_ERR_CUDA, "response kernels failed");
    CK(cudaMemcpyAsync(coef, &minus_one, sizeof(double), cudaMemcpyHostToDevice, s));
    if (launch_axpy_multi(nu, 1, yc, coef, y, s)) return fail(c, BOP_ERR_CUDA, "response kernels failed");
    conv = rel <= rtol;
  }
  c->st.response_iterations = iters;
  c->st.response_converged = conv ? 1 : 0;
  c->st.response_residual = rel;
  // final weights w = wU - c wN, then Hbar
  if (launch_scale_weights(n, norb, S, nm, c->sfac, stoner ? 1 : 0, y, -1.0, wN, wU, wU, s))
    return fail(c, BOP_ERR_CUDA, "response kernels failed");
  CKS(adjoint_pass(c, wU, c->Hbar.p, nullptr, s));
  return conv ? BOP_OK : BOP_ERR_NO_CONVERGENCE;
}

// Variational SCF: the weights of U_B = U_bond + J sum q^2 / 2 with E_F
// following the electron count, L = s U + s (J q_i - Lambda) N per orbital,
// into c->w (one pass of the chain); rdUE = the explicit d(s U)/dE.
int var_weights(bop_ctx* c, cudaStream_t s) {
  const int n = c->n, norb = c->norb, nm = c->n_mom, M = n * norb;
  CKS(ensure(c, c->w, sizeof(double) * (size_t)M * nm));
  CKS(ensure(c, c->rdUE, sizeof(double) * (size_t)M));
  CKS(ensure(c, c->vq, sizeof(double) * (size_t)n));
  CKS(ensure(c, c->zscr, sizeof(double) * (size_t)M * (c->n_exp + 1) * 2));
  {
    Region R(c, PK_SCF, 1, s);
    if (launch_var_lambda(n, norb, c->sfac, c->m.j_ii, c->m.n_e, P<double>(c->N), P<double>(c->dos),
                          P<double>(c->onsite), P<FermiState>(c->fstate), P<double>(c->vq), P<double>(c->lam),
                          P<double>(c->scfred), P<unsigned>(c->counter), s))
      return fail(c, BOP_ERR_CUDA, "variational multiplier launch failed");
  }
  return compute_weights(c, c->sfac, nullptr, 0.0, P<double>(c->w), P<double>(c->rdUE), s, P<double>(c->vq),
                         P<double>(c->lam), c->m.j_ii);
}

// Delta_i = dU_B/d delta_i = sum_alpha (Theta~_ii + explicit dU_B/dE) into
// c->vgrad: the weights above, one reverse sweep for the onsite cotangents,
// and their per-atom sums.
int var_gradient(bop_ctx* c, cudaStream_t s) {
  const int n = c->n, M = n * c->norb;
  CKS(var_weights(c, s));
  CKS(ensure(c, c->Ebar, sizeof(double) * (size_t)M));
  CKS(ensure(c, c->vgrad, sizeof(double) * (size_t)n));
  CK(cudaMemsetAsync(c->Ebar.p, 0, sizeof(double) * (size_t)M, s));
  CKS(adjoint_pass(c, P<double>(c->w), nullptr, P<double>(c->Ebar), s));
  Region R(c, PK_SCF, 1, s);
  if (launch_project(n, c->norb, 1, 0.0, P<double>(c->Ebar), P<double>(c->rdUE), nullptr, 0.0, nullptr,
                     P<double>(c->vgrad), s))
    return fail(c, BOP_ERR_CUDA, "variational gradient launch failed");
  return BOP_OK;
}

}  // namespace

extern "C" {

int bop_version(void) { return 100; }

int bop_create(bop_ctx** out, const bop_model* model) {
  if (!out) return BOP_ERR_ARG;
  *out = nullptr;
  bop_ctx* c = new (std::nothrow) bop_ctx();
  if (!c) return BOP_ERR_OOM;
  c->err[0] = 0;
  int r = validate_model(c, model);
  if (r) {
    fprintf(stderr, "bop_create: %s\n", c->err);
    delete c;
    return r;
  }
  c->m = *model;
  c->norb = model->norb;
  c->HS = block_store(model->norb);
  c->HSu = block_unique(model->norb);
  c->n_mom = model->n_mom;
  c->K = (model->n_mom - 1) / 2;
  c->Kp = c->K;
  c->n_exp = model->n_exp;
  c->S = model->n_spin;
  c->fp64 = model->precision == BOP_PREC_FP64;
  c->sfac = model->n_spin == 1 ? 2.0 : 1.0;
  c->bm.norb = model->norb;
  for (int q = 0; q < 5; q++) c->bm.b0[q] = model->b0[q];
  c->bm.r0 = model->r0;
  c->bm.lam = model->lam;
  c->bm.rc = model->rc;
  c->bm.dc = model->dc;
  c->bm.rep_A = model->rep_A;
  c->bm.rep_p = model->rep_p;
  cudaGetDevice(&c->device);
  memset(&c->st, 0, sizeof(c->st));
  if ((r = ensure(c, c->status, sizeof(unsigned))) || (r = ensure(c, c->gjack, sizeof(double) * (c->n_exp + 1))) ||
      (r = ensure(c, c->fstate, sizeof(FermiState))) || (r = ensure(c, c->partials, sizeof(double) * 3 * 4096)) ||
      (r = ensure(c, c->counter, sizeof(unsigned))) || (r = ensure(c, c->result, sizeof(double) * 4)) ||
      (r = ensure(c, c->e_total, sizeof(double))) || (r = ensure(c, c->lam, sizeof(double) * 4)) ||
      (r = ensure(c, c->ginv, sizeof(double) * (c->n_exp + 8)))) {
    bop_destroy(c);
    return r;
  }
  cudaMemset(c->status.p, 0, sizeof(unsigned));
  cudaMemset(c->counter.p, 0, sizeof(unsigned));
  if (cudaHostAlloc(&c->pin, PIN_BYTES, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    c->pin = nullptr;  // reads go straight to their destinations
  }
  launch_jackson(P<double>(c->gjack), c->n_exp, 0);
  launch_inverse_table(P<double>(c->ginv), c->n_exp + 8, 0);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    bop_destroy(c);
    return BOP_ERR_CUDA;
  }
  *out = c;
  return BOP_OK;
}

int bop_destroy(bop_ctx* c) {
  if (!c) return BOP_OK;
  DBuf* bufs[] = {&c->pos, &c->cell_of, &c->cell_count, &c->cell_start, &c->cell_fill, &c->cell_atoms, &c->deg,
                  &c->row_ptr, &c->col, &c->img, &c->flag, &c->bond_scan, &c->bond_of_edge, &c->bond_atoms,
                  &c->bond_img, &c->bond_d, &c->H64, &c->H32, &c->frac, &c->hkeys, &c->hvals, &c->skeys,
                  &c->sslot, &c->scount, &c->level_end, &c->atom_nsite, &c->atom_nadj, &c->max_level,
                  &c->site_off, &c->adj_base, &c->site_atom, &c->site_img, &c->adj_off, &c->adj, &c->lvcnt, &c->onsite,
                  &c->onsite32, &c->delta, &c->mval, &c->delta_new, &c->m_new, &c->mu, &c->a, &c->b, &c->nlev,
                  &c->a_inf, &c->b_inf, &c->gsig, &c->D, &c->gjack, &c->N, &c->U, &c->dos, &c->fstate,
                  &c->partials, &c->counter, &c->result, &c->e_total, &c->lam, &c->e_atom, &c->w, &c->zscr,
                  &c->adjscr, &c->Hbar, &c->Ebar, &c->status, &c->cub_tmp, &c->nprod,
                  &c->ginv, &c->hx, &c->hf, &c->gamma, &c->scfred, &c->lbase, &c->lnlev, &c->lflag, &c->lxs,
                  &c->lys, &c->lZ1, &c->lH1, &c->lZ2, &c->lH2, &c->lybar, &c->lcot, &c->lxbar, &c->lcount,
                  &c->rwN, &c->rwt, &c->rdUE, &c->rvec, &c->rcoef, &c->rjv, &c->rjcnt, &c->rjptr, &c->rjidx, &c->rjrow, &c->vgrad, &c->vq, &c->erep,
                  &c->psi_off, &c->psis, &c->lsum, &c->sdir, &c->vmom, &c->obar, &c->torque,
                  &c->ncscr, &c->cw_misc, &c->cw_keys, &c->cw_epack, &c->fev, &c->gs32};
  for (DBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (c->pin) cudaFreeHost(c->pin);
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  delete c;
  return BOP_OK;
}

const char* bop_last_error(const bop_ctx* c) { return c ? c->err : "null context"; }

int bop_get_stats(const bop_ctx* c, bop_stats* st) {
  if (!c || !st) return BOP_ERR_ARG;
  *st = c->st;
  return BOP_OK;
}

int bop_build_hamiltonian(bop_ctx* c, int n, const double* pos, const double* cell, const int* pbc,
                          bop_stream stream) {
  if (!c) return BOP_ERR_ARG;
  if (n < 1 || !pos || !cell || !pbc) return fail(c, BOP_ERR_ARG, "need n >= 1, pos, cell and pbc");
  cudaStream_t s = S_(stream);
  c->built = c->energized = c->weighted = false;
  if (c->nc_req > n) return fail(c, BOP_ERR_ARG, "%d centres requested for %d atoms", c->nc_req, n);
  c->n = n;
  c->nc = c->nc_req > 0 ? c->nc_req : n;
  CKS(geometry(c, cell, pbc, &c->g));
  const Geometry& g = c->g;
  CKS(ensure(c, c->pos, sizeof(double) * 3 * n));
  CK(cudaMemcpyAsync(c->pos.p, pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
  const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
  CKS(ensure(c, c->cell_of, sizeof(int) * n));
  CKS(ensure(c, c->cell_count, sizeof(int) * (ncell + 1)));
  CKS(ensure(c, c->cell_start, sizeof(int) * (ncell + 1)));
  CKS(ensure(c, c->cell_fill, sizeof(int) * ncell));
  CKS(ensure(c, c->cell_atoms, sizeof(int) * n));
  CKS(ensure(c, c->deg, sizeof(int) * (n + 1)));
  CKS(ensure(c, c->row_ptr, sizeof(long long) * (n + 1)));
  CKS(ensure(c, c->frac, sizeof(double) * 6 * 64));
  const int TB = 256, gb = (n + TB - 1) / TB;
  {
  Region Rn(c, PK_NBR, 5, s);
  bopk::k_frac_range<<<64, 256, 0, s>>>(n, P<double>(c->pos), g, P<double>(c->frac));
  CK(cudaMemsetAsync(c->cell_count.p, 0, sizeof(int) * (ncell + 1), s));
  CK(cudaMemsetAsync(c->cell_fill.p, 0, sizeof(int) * ncell, s));
  bopk::k_bin_atoms<<<gb, TB, 0, s>>>(n, P<double>(c->pos), g, P<int>(c->cell_of), P<int>(c->cell_count));
  CKS(exclusive_scan(c, P<int>(c->cell_count), P<int>(c->cell_start), ncell + 1, s));
  bopk::k_fill_cells<<<gb, TB, 0, s>>>(n, P<int>(c->cell_of), P<int>(c->cell_start), P<int>(c->cell_fill),
                                       P<int>(c->cell_atoms));
  CK(cudaMemsetAsync(c->deg.p, 0, sizeof(int) * (n + 1), s));
  launch_neighbors(0, n, P<double>(c->pos), g, P<int>(c->cell_of), P<int>(c->cell_start), P<int>(c->cell_atoms),
                   P<int>(c->deg), nullptr, nullptr, nullptr, P<unsigned>(c->status), s);
  CK(cudaGetLastError());
  CKS(exclusive_scan(c, P<int>(c->deg), P<long long>(c->row_ptr), n + 1, s));
  }
  double fr[6 * 64];
  long long E = 0;
  {
    Readback rb(c, s);
    CKS(rb.add(fr, c->frac.p, sizeof(double) * 6 * 64));
    CKS(rb.add(&E, P<long long>(c->row_ptr) + n, sizeof(long long)));
    CKS(rb.finish());
  }
  for (int a = 0; a < 3; a++) {
    double mn = 1e300, mx = -1e300;
    for (int q = 0; q < 64; q++) {
      mn = fmin(mn, fr[6 * q + a]);
      mx = fmax(mx, fr[6 * q + 3 + a]);
    }
    if (std::isinf(mn) || std::isinf(mx))
      return fail(c, BOP_ERR_ARG, "non-finite atom positions (NaN or Inf)");
    if (mn < -1e-9 || mx >= 1.0 + 1e-9)
      return fail(c, BOP_ERR_ARG, "atoms outside the cell along axis %d (fractional range [%g, %g])", a, mn, mx);
  }
  if (E % 2) return fail(c, BOP_ERR_ARG, "odd number of directed neighbour pairs");
  c->E = E;
  c->nb = E / 2;
  const long long nb = c->nb;
  CKS(ensure(c, c->col, sizeof(int) * E));
  CKS(ensure(c, c->img, 3 * E));
  CKS(ensure(c, c->flag, sizeof(int) * (E + 1)));
  CKS(ensure(c, c->bond_scan, sizeof(int) * (E + 1)));
  CKS(ensure(c, c->bond_of_edge, sizeof(int) * E));
  CKS(ensure(c, c->bond_atoms, sizeof(int) * 2 * nb));
  CKS(ensure(c, c->bond_img, 3 * nb));
  CKS(ensure(c, c->bond_d, sizeof(double) * 3 * nb));
  CKS(ensure(c, c->H64, sizeof(double) * c->HS * nb));
  CKS(ensure(c, c->H32, sizeof(float) * c->HS * nb));
  {
  Region Rn2(c, PK_NBR, E > 0 ? 4 : 2, s);
  launch_neighbors(1, n, P<double>(c->pos), g, P<int>(c->cell_of), P<int>(c->cell_start), P<int>(c->cell_atoms),
                   nullptr, P<long long>(c->row_ptr), P<int>(c->col), P<signed char>(c->img),
                   P<unsigned>(c->status), s);
  bopk::k_edge_flags<<<gb, TB, 0, s>>>(n, P<long long>(c->row_ptr), P<int>(c->col), P<signed char>(c->img),
                                       P<int>(c->flag));
  if (E > 0) {
    CKS(exclusive_scan(c, P<int>(c->flag), P<int>(c->bond_scan), E, s));
    bopk::k_bonds<<<gb, TB, 0, s>>>(n, P<long long>(c->row_ptr), P<int>(c->col), P<signed char>(c->img),
                                    P<int>(c->flag), P<int>(c->bond_scan), P<int>(c->bond_of_edge),
                                    P<int>(c->bond_atoms), P<signed char>(c->bond_img), P<unsigned>(c->status));
    bopk::k_bond_blocks<<<(int)((nb + TB - 1) / TB), TB, 0, s>>>(
        (int)nb, P<double>(c->pos), g, c->bm, P<int>(c->bond_atoms), P<signed char>(c->bond_img),
        P<double>(c->bond_d), P<double>(c->H64), P<float>(c->H32), c->HS);
  }
  }
  CK(cudaGetLastError());
  // the centres' largest degree (the cluster builder's variant) read back
  // with the neighbour list's status
  int md[4] = {0, 0, 0, 0};
  CKS(ensure(c, c->cw_misc, 4 * sizeof(int)));
  CK(cudaMemsetAsync(c->cw_misc.p, 0, 4 * sizeof(int), s));
  launch_max_degree(c->nc, P<long long>(c->row_ptr), P<int>(c->cw_misc), s);
  {
    Readback rb(c, s);
    CKS(rb.add(md, c->cw_misc.p, 4 * sizeof(int)));
    CKS(rb.finish());
  }
  c->cw_maxdeg = md[0];
  CKS(build_clusters(c, s));
  CKS(size_state(c));
  // per-atom row offsets of a stored Psi sweep
  const int nc = c->nc;
  CKS(ensure(c, c->lsum, sizeof(long long) * (nc + 1)));
  CKS(ensure(c, c->psi_off, sizeof(long long) * (nc + 1)));
  CK(cudaMemsetAsync(c->lsum.p, 0, sizeof(long long) * (nc + 1), s));
  launch_level_sums(nc, c->K, P<int>(c->level_end), P<long long>(c->lsum), s);
  CKS(exclusive_scan(c, P<long long>(c->lsum), P<long long>(c->psi_off), nc + 1, s));
  unsigned long long np = 0;
  {
    Readback rb(c, s);
    CKS(rb.add(&c->psi_tot, P<long long>(c->psi_off) + nc, sizeof(long long)));
    CKS(rb.add(&np, c->nprod.p, sizeof(np)));
    CKS(rb.finish());  // synchronises; also the status of the cluster writes
  }
  c->psi_valid = false;
  c->built = true;
  memset(&c->st, 0, sizeof(c->st));
  c->st.n_atoms = n;
  c->st.K = c->K;
  c->st.n_edges = E;
  c->st.n_bonds = nb;
  c->st.n_sites = c->nsite;
  c->st.n_adj = c->nadj;
  c->st.max_cluster = c->maxlev[c->K];
  c->st.moment_products = (long long)np;
  return BOP_OK;
}

int bop_get_neighbors(bop_ctx* c, long long* row_ptr, int* col, signed char* img, bop_stream stream) {
  if (!c || !c->built) return fail(c, BOP_ERR_STATE, "no structure built");
  cudaStream_t s = S_(stream);
  if (row_ptr) CK(cudaMemcpyAsync(row_ptr, c->row_ptr.p, sizeof(long long) * (c->n + 1), cudaMemcpyDeviceToDevice, s));
  if (col && c->E) CK(cudaMemcpyAsync(col, c->col.p, sizeof(int) * c->E, cudaMemcpyDeviceToDevice, s));
  if (img && c->E) CK(cudaMemcpyAsync(img, c->img.p, 3 * c->E, cudaMemcpyDeviceToDevice, s));
  return BOP_OK;
}

int bop_get_cluster(bop_ctx* c, int atom, int* site_atom, signed char* site_img, int* level_end, bop_stream stream) {
  if (!c || !c->built) return fail(c, BOP_ERR_STATE, "no structure built");
  if (atom < 0 || atom >= c->nc) return fail(c, BOP_ERR_ARG, "atom index out of range (clusters of the centres)");
  cudaStream_t s = S_(stream);
  long long s0 = 0;
  int lev[BOP_MAX_K + 1];
  CK(cudaMemcpyAsync(&s0, P<long long>(c->site_off) + atom, sizeof(long long), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(lev, P<int>(c->level_end) + (size_t)atom * (c->K + 1), sizeof(int) * (c->K + 1),
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int ns = lev[c->K];
  if (level_end) CK(cudaMemcpyAsync(level_end, lev, sizeof(int) * (c->K + 1), cudaMemcpyHostToDevice, s));
  if (site_atom) CK(cudaMemcpyAsync(site_atom, P<int>(c->site_atom) + s0, sizeof(int) * ns, cudaMemcpyDeviceToDevice, s));
  if (site_img) CK(cudaMemcpyAsync(site_img, P<signed char>(c->site_img) + 3 * s0, 3 * ns, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  return BOP_OK;
}

int bop_get_bonds(bop_ctx* c, int* atoms, double* d, double* blocks, bop_stream stream) {
  if (!c || !c->built) return fail(c, BOP_ERR_STATE, "no structure built");
  cudaStream_t s = S_(stream);
  if (c->nb == 0) return BOP_OK;
  if (atoms) CK(cudaMemcpyAsync(atoms, c->bond_atoms.p, sizeof(int) * 2 * c->nb, cudaMemcpyDeviceToDevice, s));
  if (d) CK(cudaMemcpyAsync(d, c->bond_d.p, sizeof(double) * 3 * c->nb, cudaMemcpyDeviceToDevice, s));
  if (blocks)
    CK(cudaMemcpy2DAsync(blocks, sizeof(double) * c->HSu, c->H64.p, sizeof(double) * c->HS, sizeof(double) * c->HSu,
                         c->nb, cudaMemcpyDeviceToDevice, s));
  return BOP_OK;
}

int bop_moments(bop_ctx* c, const double* onsite, double* mu, bop_stream stream) {
  if (!c || !c->built) return fail(c, BOP_ERR_STATE, "no structure built");
  if (!mu) return fail(c, BOP_ERR_ARG, "mu is NULL");
  cudaStream_t s = S_(stream);
  const size_t M = (size_t)c->S * c->n * c->norb;  // onsite levels of every atom
  if (onsite) {
    CK(cudaMemcpyAsync(c->onsite.p, onsite, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
    Region R(c, PK_ONSITE, 1, s);
    launch_to_float(P<double>(c->onsite), P<float>(c->onsite32), M, s);
  } else {
    Region R(c, PK_ONSITE, 1, s);
    launch_build_onsite(c->n, c->norb, c->S, c->m.onsite0, c->m.onsite_s, 0.0, nullptr, nullptr, P<double>(c->onsite),
                        P<float>(c->onsite32), s);
  }
  CKS(run_moments(c, P<double>(c->onsite), mu, s));
  CK(cudaGetLastError());
  return BOP_OK;
}

int bop_recursion(bop_ctx* c, int M, const double* mu, double* a, double* b, int* nlev, double* a_inf,
                  double* b_inf, double* gsig, bop_stream stream) {
  if (!c) return BOP_ERR_ARG;
  if (M < 1 || !mu || !gsig) return fail(c, BOP_ERR_ARG, "need M >= 1, mu and gsig");
  cudaStream_t s = S_(stream);
  DBuf ta, tb, tn, tai, tbi;
  auto cleanup = [&]() {
    for (DBuf* q : {&ta, &tb, &tn, &tai, &tbi})
      if (q->p) cudaFree(q->p);
  };
  int r;
  if ((r = ensure(c, ta, sizeof(double) * M * c->Kp)) || (r = ensure(c, tb, sizeof(double) * M * (c->Kp + 1))) ||
      (r = ensure(c, tn, sizeof(int) * M)) || (r = ensure(c, tai, sizeof(double) * M)) ||
      (r = ensure(c, tbi, sizeof(double) * M))) {
    cleanup();
    return r;
  }
  ScalarArgs A;
  A.M = M;
  A.n_mom = c->n_mom;
  A.n_exp = c->n_exp;
  A.mu = mu;
  A.a = a ? a : P<double>(ta);
  A.b = b ? b : P<double>(tb);
  A.nlev = nlev ? nlev : P<int>(tn);
  A.a_inf = a_inf ? a_inf : P<double>(tai);
  A.b_inf = b_inf ? b_inf : P<double>(tbi);
  A.gsig = gsig;
  A.g = P<double>(c->gjack);
  A.status = P<unsigned>(c->status);
  A.bw = band_sel(c->m);
  A.n_unbounded = nullptr;
  r = launch_expand(A, s) ? fail(c, BOP_ERR_CUDA, "expand launch failed") : BOP_OK;
  if (r == BOP_OK) r = check_status(c, s);
  cleanup();
  return r;
}

int bop_energy(bop_ctx* c, double* e_atom, double* delta_io, double* m_io, bop_stats* st, bop_stream stream) {
  if (!c || !c->built) return fail(c, BOP_ERR_STATE, "no structure built");
  if ((c->reduce_fn || c->nc < c->n) && (c->m.scf != BOP_SCF_NONE || c->m.noncollinear))
    return fail(c, BOP_ERR_ARG, "a spatial domain (centres or a reduce function) needs scf NONE, collinear");
  cudaStream_t s = S_(stream);
  const int n = c->n, nc = c->nc, M = c->S * nc * c->norb;
  c->energized = c->weighted = false;
  c->psi_valid = false;
  c->var_w_valid = false;
  const bool variational = c->m.scf == BOP_SCF_VARIATIONAL;
  if (delta_io) CK(cudaMemcpyAsync(c->delta.p, delta_io, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  else CK(cudaMemsetAsync(c->delta.p, 0, sizeof(double) * n, s));
  const bool stoner = c->m.scf == BOP_SCF_STONER;
  // moment magnitudes: Stoner SCF, or fixed for a non-collinear model without SCF
  const bool magnetic = stoner || c->m.noncollinear;
  if (c->m.noncollinear && c->sdir_n != n)
    return fail(c, BOP_ERR_STATE, "noncollinear model: bop_set_spin_directions first");
  if (magnetic) {
    CKS(ensure(c, c->mval, sizeof(double) * n));
    if (m_io) CK(cudaMemcpyAsync(c->mval.p, m_io, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    else {
      std::vector<double> h(n, c->m.m0);
      CK(cudaMemcpyAsync(c->mval.p, h.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
      CK(cudaStreamSynchronize(s));
    }
  }
  int it = 0, converged = c->m.scf == BOP_SCF_NONE;
  double res[4] = {0, 0, 0, 0};
  FermiState fs;
  ScfArgs a;
  a.n = n;
  a.norb = c->norb;
  a.n_spin = c->S;
  a.mode = c->m.scf;
  a.spin_factor = c->sfac;
  a.n0 = c->m.n_e;
  a.eta = c->m.eta;
  a.tol = c->m.scf_tol;
  a.dos_floor = c->m.dos_floor;
  a.stoner_I = c->m.stoner_I;
  a.m_mix = c->m.m_mix;
  a.onsite0 = c->m.onsite0;
  a.N = P<double>(c->N);
  a.dos = P<double>(c->dos);
  a.delta = P<double>(c->delta);
  a.m = P<double>(c->mval);
  a.delta_new = P<double>(c->delta_new);
  a.m_new = P<double>(c->m_new);
  a.onsite = P<double>(c->onsite);
  a.onsite32 = P<float>(c->onsite32);
  a.red = P<double>(c->scfred);
  a.counter = P<unsigned>(c->counter);
  a.result = P<double>(c->result);
  a.mixer = c->m.mixer;
  a.hist = c->m.mixer == BOP_MIX_ANDERSON ? c->m.mix_history : 1;
  a.hx = P<double>(c->hx);
  a.hf = P<double>(c->hf);
  a.gamma = P<double>(c->gamma);
  a.grad = nullptr;
  a.J = c->m.j_ii;
  // SCF residual of this iteration (for VARIATIONAL after the gradient sweep)
  // the variational SCF sweeps back once per iteration, and the response
  // solve of forces that are expected to follow sweeps back several times:
  // store Psi in each forward pass when it fits (the last pass is at the
  // final onsite levels)
  bool var_store = false;
  // (without an SCF the one forward pass stores Psi for the single reverse
  // sweep of the forces, which then needs no recomputation)
  const bool resp_store = c->forces_follow && (c->m.scf == BOP_SCF_NONE || ((c->m.scf == BOP_SCF_LCN ||
                                                                            c->m.scf == BOP_SCF_STONER) &&
                                                                           c->m.scf_response));
  if (variational || resp_store) CKS(psi_store_alloc(c, &var_store));
  c->forces_follow = false;
  auto residual = [&]() -> int {
    if (variational) {
      CKS(var_gradient(c, s));
      a.grad = P<double>(c->vgrad);
    }
    Region R(c, PK_SCF, 1, s);
    if (launch_scf_residual(a, s)) return fail(c, BOP_ERR_CUDA, "scf residual launch failed");
    return BOP_OK;
  };
  for (;;) {
    a.it = it;
    {
      Region R(c, PK_ONSITE, 1, s);
      launch_build_onsite(n, c->norb, c->S, c->m.onsite0, c->m.onsite_s, c->m.stoner_I, P<double>(c->delta),
                          magnetic ? P<double>(c->mval) : nullptr, P<double>(c->onsite), P<float>(c->onsite32), s);
    }
    CKS(run_moments(c, P<double>(c->onsite), P<double>(c->mu), s, var_store ? c->psis.p : nullptr));
    c->psi_valid = var_store;
    CKS(run_scalar(c, M, P<double>(c->mu), s));
    // warm Fermi start: later SCF iterations, and the first one of a
    // warm-started call after a previous solve
    CKS(fermi_and_N(c, it > 0 || (delta_io != nullptr && c->ef_solved), s));
    const bool last_it = c->m.scf == BOP_SCF_NONE || it >= c->m.scf_max_it;
    if (!last_it) CKS(residual());
    // one synchronisation per iteration: Fermi solve converged?  SCF converged?
    for (int extra = 0;; extra++) {
      Readback rb(c, s);
      CKS(rb.add(&fs, c->fstate.p, sizeof(FermiState)));
      if (!last_it) CKS(rb.add(res, c->result.p, sizeof(double) * 4));
      CKS(rb.finish());
      if (fs.done) break;
      if (fs.iters >= FERMI_MAX_ROUNDS || extra >= 4)
        return fail(c, BOP_ERR_BRACKET, "Fermi level not converged after %d rounds", fs.iters);
      CKS(fermi_more(c, s));
      if (!last_it) CKS(residual());
    }
    if (last_it) break;
    if (res[2] != 0.0) {
      converged = 1;
      c->var_w_valid = variational;  // c->w holds the weights of this final state
      break;
    }
    {
      Region R(c, PK_SCF, 1, s);
      if (launch_scf_apply(a, s)) return fail(c, BOP_ERR_CUDA, "scf apply launch failed");
    }
    it++;
  }
  {
    Region R(c, PK_NU, 1, s);
    if (launch_orbital_NU(M, c->n_exp, P<double>(c->gsig), P<double>(c->ginv), P<double>(c->a_inf),
                          P<double>(c->b_inf), P<double>(c->onsite), P<FermiState>(c->fstate), P<double>(c->N),
                          P<double>(c->U), P<double>(c->dos), s))
      return fail(c, BOP_ERR_CUDA, "orbital N/U launch failed");
  }
  const bool rep = c->m.rep_A != 0.0;
  if (rep) {
    CKS(ensure(c, c->erep, sizeof(double) * (size_t)(n > 0 ? n : 1)));
    Region Rr(c, PK_ENERGY, 1, s);
    if (launch_rep_energy(n, c->bm, P<long long>(c->row_ptr), P<int>(c->bond_of_edge), P<double>(c->bond_d),
                          P<double>(c->erep), s))
      return fail(c, BOP_ERR_CUDA, "repulsion launch failed");
  }
  {
  Region Re(c, PK_ENERGY, 1, s);
  double* ea = e_atom ? e_atom : P<double>(c->e_atom);
  if (launch_energy(nc, c->norb, c->S, c->sfac, c->m.stoner_I, P<double>(c->U), magnetic ? P<double>(c->mval) : nullptr,
                    c->m.j_ii, variational ? P<double>(c->N) : nullptr, c->m.n_e, rep ? P<double>(c->erep) : nullptr,
                    ea, P<double>(c->partials), P<unsigned>(c->counter), P<double>(c->e_total), s))
    return fail(c, BOP_ERR_CUDA, "energy launch failed");
  // environment atoms of a spatial domain carry no energy of their own
  if (nc < n) CK(cudaMemsetAsync(ea + nc, 0, sizeof(double) * (size_t)(n - nc), s));
  }
  if (delta_io) CK(cudaMemcpyAsync(delta_io, c->delta.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  if (m_io && magnetic) CK(cudaMemcpyAsync(m_io, c->mval.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  double et = 0.0;
  unsigned nl[2] = {0, 0};
  {
    Readback rb(c, s);
    CKS(rb.add(&et, c->e_total.p, sizeof(double)));
    CKS(rb.add(nl, c->lcount.p, 2 * sizeof(unsigned)));
    CKS(rb.finish());
  }
  CKS(reduce_over_ranks(c, &et, 1, BOP_REDUCE_SUM));  // the whole structure's energy
  c->ef_solved = true;
  c->st.n_learned = (int)nl[0];
  c->st.n_unbounded = (int)nl[1];
  c->st.scf_iterations = it;
  c->st.scf_converged = converged;
  c->st.bisection_rounds = fs.iters;
  c->st.scf_residual = res[0];
  c->st.e_fermi = fs.ef;
  c->st.e_total = et;
  c->st.forces_scf_response =
      (c->m.scf == BOP_SCF_NONE || c->m.scf == BOP_SCF_VARIATIONAL || c->m.scf_response) ? 1 : 0;
  if (st) *st = c->st;
  c->energized = true;
  if (!converged) return fail(c, BOP_ERR_NO_CONVERGENCE, "SCF not converged after %d iterations (residual %g)",
                              it, res[0]);
  return BOP_OK;
}

int bop_forces(bop_ctx* c, double* forces, double* virial, bop_stats* st, bop_stream stream) {
  if (!c || !c->built || !c->energized) return fail(c, BOP_ERR_STATE, "bop_forces needs a preceding bop_energy");
  cudaStream_t s = S_(stream);
  const int n = c->n, M = c->S * c->nc * c->norb;
  CKS(ensure(c, c->w, sizeof(double) * (size_t)M * c->n_mom));
  CKS(ensure(c, c->zscr, sizeof(double) * (size_t)M * (c->n_exp + 1) * 2));
  // bond cotangents in the product type (FP32: float4 reductions)
  const size_t hbar_bytes = (c->fp64 ? sizeof(double) : sizeof(float)) * (size_t)(c->nb > 0 ? c->nb : 1) *
                            bond_cotangent_stride(c->norb, c->fp64);
  CKS(ensure(c, c->Hbar, hbar_bytes));
  CKS(ensure(c, c->Ebar, sizeof(double) * (size_t)c->S * n * c->norb));  // onsite cotangents of every atom
  CK(cudaMemsetAsync(c->Hbar.p, 0, hbar_bytes, s));
  CKS(prepare_psi_store(c, s));
  int solve_status = BOP_OK;
  c->st.response_iterations = 0;
  c->st.response_converged = 1;
  c->st.response_residual = 0.0;
  if (c->m.scf == BOP_SCF_VARIATIONAL) {
    // U_B is stationary in the shifts: its weights at fixed shifts give the
    // exact derivative (no response solve)
    if (!c->var_w_valid) CKS(var_weights(c, s));
    CKS(adjoint_pass(c, P<double>(c->w), c->Hbar.p, nullptr, s));
  } else if (c->m.scf != BOP_SCF_NONE && c->m.scf_response) {
    solve_status = scf_response(c, s);
    if (solve_status != BOP_OK && solve_status != BOP_ERR_NO_CONVERGENCE) return solve_status;
  } else {
    // E_F response (global multiplier), weights, reverse sweep
    {
      Region R(c, PK_EFRESP, 1, s);
      if (launch_ef_response(M, c->n_exp, P<double>(c->gsig), P<double>(c->ginv), P<double>(c->a_inf),
                             P<double>(c->b_inf), P<double>(c->onsite), P<FermiState>(c->fstate),
                             P<double>(c->partials), P<unsigned>(c->counter), P<double>(c->lam), s))
        return fail(c, BOP_ERR_CUDA, "E_F response launch failed");
    }
    if (c->reduce_fn) {
      // one E_F for all processes: its multiplier from the sums of all of them
      double l[3];
      {
        Readback rb(c, s);
        CKS(rb.add(l, c->lam.p, 3 * sizeof(double)));
        CKS(rb.sync());
      }
      CKS(reduce_over_ranks(c, l + 1, 2, BOP_REDUCE_SUM));
      l[0] = l[2] > 0.0 ? l[1] / l[2] : 0.0;
      CK(cudaMemcpyAsync(c->lam.p, l, 3 * sizeof(double), cudaMemcpyHostToDevice, s));
      CK(cudaStreamSynchronize(s));
    }
    CKS(compute_weights(c, c->sfac, P<double>(c->lam), 0.0, P<double>(c->w), nullptr, s));
    if (c->m.noncollinear) {
      // reverse sweep of the spinor moments: bond and onsite-matrix
      // cotangents, then the torques of Eq. torque
      NcArgs a;
      CKS(nc_args(c, &a));
      CKS(ensure(c, c->obar, sizeof(double) * (size_t)n * c->norb * 4));
      CKS(ensure(c, c->torque, sizeof(double) * 3 * (size_t)n));
      CK(cudaMemsetAsync(c->obar.p, 0, sizeof(double) * (size_t)n * c->norb * 4, s));
      a.w = P<double>(c->w);
      a.Hbar = c->Hbar.p;
      a.HSh = bond_cotangent_stride(c->norb, c->fp64);
      a.obar = P<double>(c->obar);
      {
        Region R(c, PK_ADJOINT, 1, s);
        if (launch_nc(a, c->fp64, s)) return fail(c, BOP_ERR_CUDA, "spinor reverse sweep launch failed");
      }
      Region R(c, PK_FORCES, 1, s);
      if (launch_torques(n, c->norb, c->n_mom, P<double>(c->onsite), P<double>(c->sdir), P<double>(c->w),
                         P<double>(c->vmom), P<double>(c->obar), P<double>(c->torque), s))
        return fail(c, BOP_ERR_CUDA, "torques launch failed");
    } else {
      CK(cudaMemsetAsync(c->Ebar.p, 0, sizeof(double) * (size_t)c->S * n * c->norb, s));
      CKS(adjoint_pass(c, P<double>(c->w), c->Hbar.p, P<double>(c->Ebar), s));
    }
  }
  DBuf* fb = nullptr;
  DBuf tf, tv;
  double* F = forces;
  double* W = virial;
  if (!F) {
    CKS(ensure(c, tf, sizeof(double) * 3 * n));
    F = P<double>(tf);
    fb = &tf;
  }
  if (!W) {
    CKS(ensure(c, tv, sizeof(double) * 9));
    W = P<double>(tv);
  }
  CK(cudaMemsetAsync(F, 0, sizeof(double) * 3 * n, s));
  CK(cudaMemsetAsync(W, 0, sizeof(double) * 9, s));
  {
    Region Rf(c, PK_FORCES, c->nb > 0 ? 1 : 0, s);
    if (c->nb > 0 && launch_forces((int)c->nb, c->bm, P<double>(c->bond_d), P<int>(c->bond_atoms),
                                   c->Hbar.p, bond_cotangent_stride(c->norb, c->fp64), c->fp64, F, W, s))
      return fail(c, BOP_ERR_CUDA, "forces launch failed");
  }
  int r = check_status(c, s);
  if (fb && tf.p) cudaFree(tf.p);
  if (tv.p) cudaFree(tv.p);
  if (r) return r;
  c->weighted = true;
  c->st.forces_scf_response =
      (c->m.scf == BOP_SCF_NONE || c->m.scf == BOP_SCF_VARIATIONAL || c->m.scf_response) ? 1 : 0;
  if (st) *st = c->st;
  if (solve_status != BOP_OK)
    return fail(c, solve_status, "SCF-response solve stopped at relative residual %g after %d iterations",
                c->st.response_residual, c->st.response_iterations);
  return BOP_OK;
}

int bop_set_spin_directions(bop_ctx* c, const double* sd, bop_stream stream) {
  if (!c) return BOP_ERR_ARG;
  if (!c->m.noncollinear) return fail(c, BOP_ERR_ARG, "spin directions need a noncollinear model");
  if (!c->built) return fail(c, BOP_ERR_STATE, "no structure built");
  if (!sd) return fail(c, BOP_ERR_ARG, "directions are NULL");
  cudaStream_t s = S_(stream);
  const int n = c->n;
  std::vector<double> h(3 * (size_t)n);
  CK(cudaMemcpyAsync(h.data(), sd, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < n; i++) {
    double* v = h.data() + 3 * (size_t)i;
    const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(r >= 1e-12 && r < 1e300)) return fail(c, BOP_ERR_ARG, "direction of atom %d has norm %g", i, r);
    for (int x = 0; x < 3; x++) v[x] /= r;
  }
  CKS(ensure(c, c->sdir, sizeof(double) * 3 * (size_t)n));
  CK(cudaMemcpyAsync(c->sdir.p, h.data(), sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  c->sdir_n = n;
  c->energized = c->weighted = false;
  return BOP_OK;
}

int bop_torques(bop_ctx* c, double* t, bop_stream stream) {
  if (!c) return BOP_ERR_ARG;
  if (!c->m.noncollinear) return fail(c, BOP_ERR_ARG, "torques need a noncollinear model");
  if (!c->weighted) return fail(c, BOP_ERR_STATE, "bop_torques needs a preceding bop_forces");
  if (!t) return fail(c, BOP_ERR_ARG, "t is NULL");
  CK(cudaMemcpyAsync(t, c->torque.p, sizeof(double) * 3 * (size_t)c->n, cudaMemcpyDeviceToDevice, S_(stream)));
  return BOP_OK;
}

int bop_get_orbital_state(bop_ctx* c, double* mu, double* N, double* U, double* a_inf, double* b_inf,
                          double* weights, double* onsite, bop_stream stream) {
  if (!c || !c->energized) return fail(c, BOP_ERR_STATE, "no energy computed");
  cudaStream_t s = S_(stream);
  const size_t M = (size_t)c->S * c->nc * c->norb;
  if (mu) CK(cudaMemcpyAsync(mu, c->mu.p, sizeof(double) * M * c->n_mom, cudaMemcpyDeviceToDevice, s));
  if (N) CK(cudaMemcpyAsync(N, c->N.p, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
  if (U) CK(cudaMemcpyAsync(U, c->U.p, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
  if (a_inf) CK(cudaMemcpyAsync(a_inf, c->a_inf.p, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
  if (b_inf) CK(cudaMemcpyAsync(b_inf, c->b_inf.p, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
  if (onsite) CK(cudaMemcpyAsync(onsite, c->onsite.p, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
  if (weights) {
    if (!c->weighted) return fail(c, BOP_ERR_STATE, "weights need bop_forces");
    CK(cudaMemcpyAsync(weights, c->w.p, sizeof(double) * M * c->n_mom, cudaMemcpyDeviceToDevice, s));
  }
  return BOP_OK;
}

int bop_evaluate_host(bop_ctx* c, int n, const double* pos_host, const double* cell_host, const int* pbc_host,
                      double* e_atom_host, double* forces_host, double* virial_host, double* e_total_host,
                      bop_stats* st, bop_stream stream) {
  if (!c) return BOP_ERR_ARG;
  if (n < 1 || !pos_host) return fail(c, BOP_ERR_ARG, "need n >= 1 and pos_host");
  cudaStream_t s = S_(stream);
  DBuf dpos, dF, dW;
  int r = ensure(c, dpos, sizeof(double) * 3 * n);
  if (!r) r = ensure(c, dF, sizeof(double) * 3 * n);
  if (!r) r = ensure(c, dW, sizeof(double) * 9);
  if (!r && cudaMemcpyAsync(dpos.p, pos_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
    r = fail(c, BOP_ERR_CUDA, "H2D copy of positions failed");
  if (!r) r = bop_build_hamiltonian(c, n, P<double>(dpos), cell_host, pbc_host, stream);
  if (!r) r = bop_energy(c, nullptr, nullptr, nullptr, nullptr, stream);
  if (!r) r = bop_forces(c, P<double>(dF), P<double>(dW), nullptr, stream);
  if (!r && e_atom_host &&
      cudaMemcpyAsync(e_atom_host, c->e_atom.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    r = fail(c, BOP_ERR_CUDA, "D2H copy failed");
  if (!r && forces_host &&
      cudaMemcpyAsync(forces_host, dF.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    r = fail(c, BOP_ERR_CUDA, "D2H copy failed");
  if (!r && virial_host &&
      cudaMemcpyAsync(virial_host, dW.p, sizeof(double) * 9, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    r = fail(c, BOP_ERR_CUDA, "D2H copy failed");
  if (!r && cudaStreamSynchronize(s) != cudaSuccess) r = fail(c, BOP_ERR_CUDA, "synchronise failed");
  if (!r && e_total_host) *e_total_host = c->st.e_total;
  if (!r && st) *st = c->st;
  for (DBuf* q : {&dpos, &dF, &dW})
    if (q->p) cudaFree(q->p);
  return r;
}

int bop_set_centers(bop_ctx* c, int n_centers) {
  if (!c) return BOP_ERR_ARG;
  if (n_centers < 0) return fail(c, BOP_ERR_ARG, "n_centers must be >= 0");
  c->nc_req = n_centers;
  return BOP_OK;
}

int bop_set_reduce(bop_ctx* c, bop_reduce_fn fn, void* user) {
  if (!c) return BOP_ERR_ARG;
  c->reduce_fn = fn;
  c->reduce_user = user;
  return BOP_OK;
}

int bop_set_response_limits(bop_ctx* c, int max_iterations, double rtol) {
  if (!c) return BOP_ERR_ARG;
  if (max_iterations < 0 || !(rtol >= 0.0) || !std::isfinite(rtol))
    return fail(c, BOP_ERR_ARG, "response limits: max_iterations >= 0 and a finite rtol >= 0");
  c->resp_max_it = max_iterations;
  c->resp_rtol = rtol;
  return BOP_OK;
}

int bop_set_store_budget(bop_ctx* c, long long bytes) {
  if (!c) return BOP_ERR_ARG;
  c->store_budget = bytes < 0 ? (size_t)-1 : (size_t)bytes;
  if (c->store_budget == 0) {
    for (DBuf* b : {&c->psis})
      if (b->p) {
        cudaFree(b->p);
        b->p = nullptr;
        b->bytes = 0;
      }
  }
  return BOP_OK;
}

int bop_set_mlp(bop_ctx* c, bop_mlp* net) {
  if (!c) return BOP_ERR_ARG;
  if (c->m.terminator != BOP_TERM_MLP) return fail(c, BOP_ERR_ARG, "the model's terminator is not MLP");
  c->net = net;
  c->energized = c->weighted = false;
  return BOP_OK;
}

int bop_mlp_dataset(long long M, const double* mu17, float* x, float* t, float* mask, bop_stream stream) {
  if (M < 1 || !mu17 || !x || !t || !mask) return BOP_ERR_ARG;
  if (launch_mlp_dataset(M, mu17, x, t, mask, S_(stream))) return BOP_ERR_CUDA;
  return BOP_OK;
}

int bop_set_profiling(bop_ctx* c, int on) {
  if (!c) return BOP_ERR_ARG;
  c->prof.on = on != 0;
  return BOP_OK;
}

int bop_reset_profile(bop_ctx* c) {
  if (!c) return BOP_ERR_ARG;
  if (c->prof.used) CK(cudaEventSynchronize(c->prof.pool[c->prof.used - 1]));
  for (int k = 0; k < PK_N; k++) c->prof.launches[k] = 0;
  c->prof.kind.clear();
  c->prof.used = 0;
  return BOP_OK;
}

int bop_get_profile(bop_ctx* c, bop_kernel_time* out, int max, int* n_out) {
  if (!c || !out) return BOP_ERR_ARG;
  double ms[PK_N] = {0};
  long long reg[PK_N] = {0};
  if (c->prof.used) CK(cudaEventSynchronize(c->prof.pool[c->prof.used - 1]));
  for (size_t q = 0; q < c->prof.kind.size() && 2 * q + 1 < c->prof.used; q++) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->prof.pool[2 * q], c->prof.pool[2 * q + 1]));
    ms[c->prof.kind[q]] += t;
    reg[c->prof.kind[q]]++;
  }
  for (int k = 0; k < PK_N && k < max; k++) {
    out[k].name = PK_NAMES[k];
    out[k].launches = c->prof.launches[k];
    out[k].regions = reg[k];
    out[k].ms = ms[k];
  }
  if (n_out) *n_out = PK_N;
  return BOP_OK;
}

}  // extern "C"
