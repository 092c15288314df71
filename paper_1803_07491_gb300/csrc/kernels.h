// Internal interface between the C-ABI layer (api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bopgb.h"
#include "common.cuh"

// Cell, its inverse and the linked-cell grid of one structure.
struct Geometry {
  double cell[9];  // rows = lattice vectors
  double inv[9];   // inverse matrix: frac = pos * inv
  int nc[3];       // linked cells per axis (cell width >= rc)
  int nimg[3];     // image search range for axes with fewer than 3 cells
  int pbc[3];
  double rc;
};

// Per-CTA scratch of the cluster builder (global memory).
struct ClusterScratch {
  unsigned long long* hkeys;  // [slots][hcap]
  int* hvals;                 // [slots][hcap]
  unsigned long long* skeys;  // [slots][maxs] site keys in cluster order
  int* sslot;                 // [slots][maxs] hash slot of every site
  int* scount;                // [slots][maxs] adjacency count / offset per site
  int hcap, maxs, newcap;
};

// Outputs of the cluster builder.
struct ClusterOut {
  int* level_end;        // [n][K+1]
  int* atom_nsite;       // [n]  (pass 1)
  int* atom_nadj;        // [n]  (pass 1)
  int* max_level;        // [K+2] largest |C_k| over atoms, then the largest adjacency (pass 1)
  const long long* site_off;  // [n+1] (pass 2 input)
  const long long* adj_base;  // [n+1] (pass 2 input)
  int* site_atom;        // [S]
  signed char* site_img; // [S][3]
  long long* adj_off;    // [S+1]
  int2* adj;             // [A]
  unsigned long long* n_products;  // block products of one moments pass (pass 2)
  unsigned long long* lvcnt;       // [S] per-level entry counts (pass 2)
};

namespace bopk {
// nbr.cu
__global__ void k_bin_atoms(int n, const double* pos, Geometry g, int* cell_of, int* cell_count);
__global__ void k_fill_cells(int n, const int* cell_of, const int* cell_start, int* cell_fill, int* cell_atoms);
__global__ void k_edge_flags(int n, const long long* row_ptr, const int* col, const signed char* img, int* flag);
__global__ void k_bonds(int n, const long long* row_ptr, const int* col, const signed char* img, const int* flag,
                        const int* bond_scan, int* bond_of_edge, int* bond_atoms, signed char* bond_img,
                        unsigned* status);
__global__ void k_bond_blocks(int nb, const double* pos, Geometry g, BondModel m, const int* bond_atoms,
                              const signed char* bond_img, double* bond_d, double* H64, float* H32, int HS);
__global__ void k_frac_range(int n, const double* pos, Geometry g, double* out);
}  // namespace bopk

// Host launchers (defined in the .cu files that hold the templates).
void launch_neighbors(int mode, int n, const double* pos, Geometry g, const int* cell_of, const int* cell_start,
                      const int* cell_atoms, int* deg, const long long* row_ptr, int* col, signed char* img,
                      unsigned* status, cudaStream_t s);
// Path-radius cut: with r2 > 0 only sites closer than sqrt(r2) to the
// cluster's atom (bond_vector arithmetic) join its cluster.
struct PathCut {
  const double* pos;  // [n][3] device
  double cell[9];
  double r2;
};
int launch_cluster(int pass, int n, int K, const long long* row_ptr, const int* col, const signed char* img,
                   const int* bond_of_edge, PathCut pc, ClusterScratch sc, ClusterOut out, int grid,
                   unsigned* status, cudaStream_t s);

void launch_level_sums(int n, int K, const int* level_end, long long* out, cudaStream_t s);
// Warp-per-atom cluster builder (cluster.cu): the same outputs as
// launch_cluster for clusters of at most cluster_warp_max_sites() sites and
// atoms of at most 32 neighbours; pass 0 keeps every atom's site keys in
// gkeys [n][cluster_warp_max_sites()].  *wfail != 0 after a pass: fall back
// to launch_cluster.
int launch_cluster_warp(int pass, int n, int K, int max_deg, const long long* row_ptr, const int2* epack,
                        const int* bond_of_edge, PathCut pc, unsigned long long* gkeys,
                        ClusterOut out, int* wfail, unsigned* status, cudaStream_t s);
// epack[e] = {col[e], image bytes + 128} of every directed neighbour edge.
void launch_pack_edges(long long E, const int* col, const signed char* img, int2* epack, cudaStream_t s);
int cluster_warp_max_sites();
void launch_max_degree(int n, const long long* row_ptr, int* out, cudaStream_t s);

struct MomentsArgs {
  ClusterView cv;
  const void* H;       // float or double [nb][HS]
  int HS;
  const void* onsite;  // float or double [S][n_on][norb]
  int n, n_spin, norb, n_mom;  // n: atoms with clusters (centers), the first n of the structure
  int n_on;            // atoms of the structure (stride of the onsite levels)
  int cap_even;        // largest stored even level |C_k| (k < K) over atoms
  int cap_odd;         // largest stored odd level |C_k| (k < K) over atoms
  int max_sites;       // largest cluster |C_K|
  int max_adj;         // largest adjacency of one cluster
  double* mu;          // [S][n][norb][n_mom]
  // optional store of every Psi_k (NULL = none): rows of the item
  // (spin, atom[, alpha]) at ((spin (norb/nc) + alpha) psi_tot + psi_off[atom]) rows,
  // level k at row offset sum_{j<k} |C_j|; row = norb x nc values padded
  void* pstore;
  const long long* psi_off;  // [n+1] prefix sums of sum_k |C_k| over atoms
  long long psi_tot;
};
int launch_moments(const MomentsArgs& a, int fp64, cudaStream_t s);

struct AdjointArgs {
  ClusterView cv;
  const void* H;
  int HS;
  const void* onsite;  // [S][n_on][norb]
  int n, n_spin, norb, n_mom;  // n: centers, as MomentsArgs
  int n_on;            // atoms of the structure (stride of onsite and Ebar)
  const double* w;     // [S][n][norb][n_mom]
  void* scratch;       // per-CTA Psi / Psi-bar storage
  size_t slot_elems;   // elements of T per CTA
  int slots;
  void* Hbar;          // [nb][HSh] (+=), the product type T (bond_cotangent_stride)
  int HSh;
  double* Ebar;        // [S][n_on][norb] (+=), may be null
  // reverse sweep over stored Psi (pstore != NULL; layout of MomentsArgs.pstore)
  const void* pstore;
  const long long* psi_off;
  long long psi_tot;
  int nc;              // columns per work item used by the forward pass that stored Psi
  int cap_even, cap_odd;  // largest even / odd level |C_k|, k = 1..K
  int max_sites, max_adj, cap_eb;  // cap_eb: largest |C_K-1|
  // stored-Psi sweep only: per cluster site t of work item (spin, atom i),
  // sum over the orbitals of dL/dE_t (+=), at siteval[spin * sv_stride +
  // site_off[i] + t] (t < |C_K-1|); may be null
  double* siteval;
  long long sv_stride;
};
int launch_moments_adjoint(const AdjointArgs& a, int fp64, cudaStream_t s);
// Elements per bond of the cotangent array Hbar: the unique block elements
// (1, 15, 21), padded to a multiple of four in FP32 (float4 reductions).
int bond_cotangent_stride(int norb, int fp64);

// Non-collinear spin moments (moments.cu): work item (atom, orbital), the
// two local spin states of the atom as starting spinors.
struct NcArgs {
  ClusterView cv;
  const void* H;       // float or double [nb][HS]
  int HS;
  const void* onsite;  // float or double [2][n][norb]: E_up, E_dn
  const double* sdir;  // [n][3] unit moment directions
  int n, norb, n_mom;
  int cap_even, cap_odd;  // largest even / odd level |C_k| (k < K) over atoms (forward in shared memory)
  void* scratch;       // per-CTA Psi / Psi-bar storage
  size_t slot_elems;   // elements of T per CTA: 2 sum_k max |C_k| norb 8
  int slots;
  // forward (w == NULL): local channel moments and Tr(sigma M_n)
  double* mu;          // [2][n][norb][n_mom]
  double* vmom;        // [n][norb][n_mom][3]
  // reverse (w != NULL): cotangents of sum w mu
  const double* w;     // [2][n][norb][n_mom]
  void* Hbar;          // [nb][HSh] (+=), the product type T (bond_cotangent_stride)
  int HSh;
  double* obar;        // [n][norb][4] (+=): d/d(Ebar, h_x, h_y, h_z)
};
int launch_nc(const NcArgs& a, int fp64, cudaStream_t s);
int launch_torques(int n, int norb, int n_mom, const double* onsite, const double* sdir, const double* w,
                   const double* vmom, const double* obar, double* t, cudaStream_t s);

// Band centre / width estimate of the constant terminator (BOP_BW_* of
// bopgb.h): mode, beta of the weighted average, (A, B) of the global mode.
struct BandSel {
  int mode;
  double beta, ga, gb;
};

// scalar.cu
struct ScalarArgs {
  int M;               // orbitals (all spins)
  int n_mom, n_exp;
  const double* mu;    // [M][n_mom]
  double* a;           // [M][Kp]
  double* b;           // [M][Kp+1]
  int* nlev;           // [M]
  double* a_inf;       // [M]
  double* b_inf;       // [M]
  double* gsig;        // [n_exp+1][M]   (coefficient-major)
  const double* g;     // [n_exp+1] damping
  unsigned* status;
  BandSel bw;
  unsigned* n_unbounded;  // may be null: orbitals with some |sigma_m| > m + 1
  int sig32 = 0;          // 1: the sigma_m recurrence in FP32 (FP32-products mode)
};
int launch_expand(const ScalarArgs& a, cudaStream_t s);
void launch_jackson(double* g, int n_exp, cudaStream_t s);

struct FermiState {
  double lo, hi, mid, ef;
  int done, iters, pad0, pad1;
};
int launch_fermi(int M, const double* D, const double* gsig, const double* a_inf, const double* b_inf, int n_exp,
                 double spin_factor, double target, FermiState* st, double* partials, unsigned* counter,
                 int max_rounds, double tol, cudaStream_t s);

// One piece of a Fermi-level solve spread over several processes (chain.cu):
// mode 0: out = {-min(a_inf - 2 b_inf), max(a_inf + 2 b_inf)}; mode 1: out =
// {sum N_o(E), sum n_o(E)} over this process's M orbitals (out device [2]).
int launch_fermi_eval(int mode, int M, const double* gsig, const double* inv, const double* a_inf,
                      const double* b_inf, int n_exp, double E, double* partials, unsigned* counter, double* out,
                      cudaStream_t s);
int launch_orbital_NU(int M, int n_exp, const double* gsig, const double* inv, const double* a_inf,
                      const double* b_inf, const double* onsite, const FermiState* st, double* N, double* U,
                      double* dos, cudaStream_t s);
int launch_orbital_N(int M, int n_exp, const double* gsig, const double* inv, const double* a_inf,
                     const double* b_inf, const FermiState* st, double* N, double* dos, cudaStream_t s);
// Newton steps inside the bisection bracket (chain.cu); warm: start from st->ef
int launch_fermi_newton(int M, const double* gsig, const double* inv, const double* a_inf, const double* b_inf,
                        int n_exp, double spin_factor, double target, FermiState* st, double* partials,
                        unsigned* counter, int warm, int rounds, int max_rounds, double tol, cudaStream_t s);
int launch_fermi_more(int M, const double* gsig, const double* inv, const double* a_inf, const double* b_inf,
                      int n_exp, double spin_factor, double target, FermiState* st, double* partials,
                      unsigned* counter, int rounds, int max_rounds, double tol, cudaStream_t s);
void launch_inverse_table(double* inv, int n, cudaStream_t s);
// The whole Fermi solve (bracket, Newton rounds, N and DOS at E_F) in one
// cooperative launch; partials: >= 4 x (grid) doubles.  -2: cooperative
// launch unavailable.
int launch_fermi_coop(int M, const double* gsig, const double* inv, const double* a_inf, const double* b_inf,
                      int n_exp, double spin_factor, double target, FermiState* st, double* partials, int warm,
                      int max_rounds, double tol, double* N, double* dos, cudaStream_t s,
                      const float* gs32 = nullptr);
// FP32 copy of gsig [n_exp+1][M] (the starting point of a cold Fermi search).
int launch_gsig_f32(int M, int n_exp, const double* gsig, float* gs32, cudaStream_t s);

struct ScfArgs {
  int n, norb, n_spin, mode;  // mode 1 = LCN, 2 = Stoner
  double spin_factor, n0, eta, tol, dos_floor, stoner_I, m_mix, onsite0;
  const double* N;     // [S][n][norb]
  const double* dos;   // [S][n][norb]
  double* delta;       // [n]
  double* m;           // [n]
  double* delta_new;   // [n]
  double* m_new;       // [n]
  double* onsite;      // [S][n][norb] (rebuilt)
  float* onsite32;
  double* red;         // partials [grid][64]
  unsigned* counter;
  double* result;      // [4]: max|res|, max|dm|, converged, mean
  int mixer;           // 0 linear, 1 Anderson
  int hist;            // Anderson history depth (<= 8)
  int it;              // iteration index of this update (0-based)
  double* hx;          // [(hist+1)][ncomp*n] iterates
  double* hf;          // [(hist+1)][ncomp*n] preconditioned residuals
  double* gamma;       // [hist] least-squares coefficients
  const double* grad;  // mode 3 (variational): dU_B/d delta_i [n]
  double J;            // mode 3: onsite charging J_ii
};
int launch_scf_residual(const ScfArgs& a, cudaStream_t s);
int launch_scf_apply(const ScfArgs& a, cudaStream_t s);
void launch_to_float(const double* in, float* out, size_t n, cudaStream_t s);
void launch_build_onsite(int n, int norb, int n_spin, double onsite0, double onsite_s, double stoner_I,
                         const double* delta,
                         const double* m, double* onsite, float* onsite32, cudaStream_t s);

// e_i = s sum U (- I m_i^2 / 4 with m) (+ J q_i^2 / 2, q_i = s sum N - n0, with N)
//       (+ erep_i with erep)
int launch_energy(int n, int norb, int n_spin, double spin_factor, double stoner_I, const double* U,
                  const double* m, double J, const double* N, double n0, const double* erep, double* e_atom,
                  double* red, unsigned* counter, double* e_total, cudaStream_t s);

struct WeightArgs {
  int M, n_mom, n_exp, norb;
  const double* mu;
  const double* onsite;  // [M]
  const FermiState* st;
  const double* g;
  const double* inv;     // [n_exp+8] 1/k
  double cU;             // L = cU*U + cN*N
  const double* lam;     // device scalar: cN = -cU * (*lam)  (E_F response); NULL: cN = cN0
  double cN0;
  double* w;             // [M][n_mom]
  double* dU_dE;         // [M] direct derivative of L w.r.t. the onsite level, may be null
  double* zscratch;      // [2][n_exp+1][M]: sigma_m and its cotangent
  unsigned* status;
  BandSel bw;
  // n_spin 1 only: per-atom cN = cU (var_J var_q[i] - var_lam[0]) when var_q
  // is set (the variational SCF's binding energy U_B); else lam / cN0 above
  const double* var_q;
  const double* var_lam;
  double var_J;
  int sig32 = 0;  // 1: the sigma_m recurrences (forward and reverse) in FP32 (FP32-products mode)
};
int launch_weights(const WeightArgs& a, cudaStream_t s);
// Weights of L1 = cU1 U + cN1 N into a.w and of L2 = cU2 U + cN2 N into w2 at
// fixed E_F (a.lam unused), one lane per seed; a.zscratch: [4][n_exp+1][M].
int launch_weights_pair(const WeightArgs& a, double cU1, double cN1, double cU2, double cN2, double* w2,
                        cudaStream_t s);
int launch_ef_response(int M, int n_exp, const double* gsig, const double* inv, const double* a_inf,
                       const double* b_inf, const double* onsite, const FermiState* st, double* red,
                       unsigned* counter, double* lam, cudaStream_t s);

// learned.cu: the learned terminator (n_mom = 9, continued to 8 levels)
struct LearnedArgs {
  int M, n_exp, fp64;
  int sig32;             // 1: the sigma_m recurrences in FP32
  const double* mu;      // [M][9]
  double* base;          // [M][10]: a_0..a_3, b_1..b_4, a_inf, b_inf of the 9-moment chain
  int* nlev;             // [M] levels of the 9-moment chain
  unsigned char* flag;   // [M]: 1 = inputs inside the training range, 2 = continued chain used
  void* xs;              // T [M][18] standardised inputs (T = double if fp64 else float)
  const void* ys;        // T [M][10] standardised outputs
  const float* norm;     // [BOP_MLP_NNORM] standardisation and training range
  double* a_inf;         // [M] terminator of the chain used
  double* b_inf;
  double* gsig;          // [n_exp+1][M]
  const double* g;       // [n_exp+1] damping
  unsigned* n_learned;   // += orbitals on the continued chain
  unsigned* status;
  void* ybar;            // T [M][10] cotangent of the standardised outputs
  double* cot;           // [M][10] cotangent of the base record
  const void* xbar;      // T [M][18] cotangent of the standardised inputs
  WeightArgs W;          // E_F, onsite, damping, 1/k table, cU, lam, w, zscratch
};
// stage 0: features, 1: continued chain + expansion, 2: reverse of the chain
// part, 3: reverse of features / Gershgorin / recursion -> W.w
int launch_learned(int stage, const LearnedArgs& a, cudaStream_t s);
int launch_mlp_dataset(long long M, const double* mu17, float* x, float* t, float* mask, cudaStream_t s);

// mlp.cu: network on M rows with the bfloat16 inference weights
int mlp_infer_forward(int fp64, int M, const void* xs, const float* params, const void* wbf, void* Z1, void* H1,
                      void* Z2, void* H2, void* ys, cudaStream_t s);
int mlp_infer_backward(int fp64, int M, const void* ybar, const void* wbf, void* Z1, void* Z2, void* dZ1, void* dZ2,
                       void* xbar, cudaStream_t s);
const float* mlp_params_dev(const bop_mlp* net);
const void* mlp_wbf_dev(const bop_mlp* net);
const float* mlp_norm_dev(const bop_mlp* net);

// scf_adjoint.cu: vector kernels of the SCF-response solve (nu = n or 2n unknowns)
// w_out = (wU or 0) + sign * c_{atom,spin} * wN, c = s v[atom] + sigma_spin v[n + atom] (Stoner)
// Variational SCF: q_i = s sum_alpha N - n0 into q, and the E_F multiplier
// of U_B = U_bond + J sum q^2 / 2 into lam[0]:
// Lambda = sum_i D_i (E_F - E_i + J q_i) / sum_i D_i, D_i = s sum_alpha dos.
int launch_var_lambda(int n, int norb, double s, double J, double n0, const double* N, const double* dos,
                      const double* onsite, const FermiState* st, double* q, double* lam, double* red,
                      unsigned* counter, cudaStream_t stream);
int launch_scale_by_inv_norm(int nu, double* u, const double* nsq, cudaStream_t stream);
// J^T v of the SCF response from the per-site values of one sweep with the
// dN/dmu weights (AdjointArgs.siteval).  The transpose of the rows: for
// every atom j the global sites of other atoms' clusters (first |C_K-1|
// sites) whose atom is j, with the owning atom (stage 0: counts into cnt;
// stage 1 after the scan of cnt into ptr: fill, cnt zeroed first).  Then
// Eb[spin][j] = sum over the entries of c_{i,spin} val[spin][site], c =
// s v[i] (+ sigma_spin v[n + i] for Stoner).  Eb: [S][n].
int launch_jt_build(int n, int K, const long long* site_off, const int* level_end, const int* site_atom,
                    int* cnt, int stage, const long long* ptr, long long* idx, int* row, cudaStream_t stream);
int launch_jt_gather(int n, int S, const long long* ptr, const long long* idx, const int* row, const double* val,
                     long long stride, const double* v, double s, int stoner, double* Eb, cudaStream_t stream);
int launch_scale_weights(int n, int norb, int S, int n_mom, double s, int stoner, const double* v, double sign,
                         const double* wN, const double* wU, double* w_out, cudaStream_t st);
// out_u = derivative w.r.t. u of a function whose onsite-level derivative is Eb (+ dUE):
//   delta part sum_{alpha,nu}; Stoner moment part sum_alpha (-I/2 up + I/2 down),
//   plus mcoef * m[i] (energy: -I/2 m) and minus v_m[i] if v_m (the -m_i of Q_i)
int launch_project(int n, int norb, int S, double I, const double* Eb, const double* dUE, const double* m,
                   double mcoef, const double* v_m, double* out, cudaStream_t st);
// P = diagonal preconditioner: -1/max(s sum n_i, floor) for delta, -1 for m
int launch_precond_diag(int n, int norb, int S, double s, double floor_, const double* dos, double* P,
                        cudaStream_t st);
int launch_dots(int nu, int nvec, const double* V, const double* w, double* out, cudaStream_t st);
// w -= sum_k coef[k] V[k]  (coef device)
int launch_axpy_multi(int nu, int nvec, const double* V, const double* coef, double* w, cudaStream_t st);
// out = scale * (sum_k coef[k] V[k]) * (P if P else 1)
int launch_lincomb(int nu, int nvec, const double* V, const double* coef, const double* P, double scale,
                   double* out, cudaStream_t st);
// out = a * x * (P if P else 1)
int launch_scale_vec(int nu, const double* x, const double* P, double a, double* out, cudaStream_t st);

// forces.cu
// Pair repulsion per atom (half of each of its bonds) into erep [n].
int launch_rep_energy(int n, BondModel m, const long long* row_ptr, const int* bond_of_edge, const double* bond_d,
                      double* erep, cudaStream_t s);
int launch_forces(int nb, BondModel m, const double* bond_d, const int* bond_atoms, const void* Hbar, int HSh, int fp64,
                  double* forces, double* virial, cudaStream_t s);
