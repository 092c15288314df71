// Shared device definitions of libbopgb: limits, views of the context's
// device arrays, forward-mode dual numbers and the two-centre block.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define BOP_MAX_NMOM 17            // n moments: odd, 3..17
#define BOP_MAX_K 8                // hops K = (n_mom-1)/2
#define BOP_MAX_NEXP 253           // expansion length n_exp
#define BOP_MAX_DEG 64             // neighbours per atom
#define BOP_HS_D 16                // stored elements of a d block (15 unique + pad)
#define BOP_HS_SD 24               // stored elements of an sd block (21 unique + pad)

// Error bits raised by kernels into the context's device status word.
#define BOP_DEV_ERR_DEGREE 1u      // more than BOP_MAX_DEG neighbours
#define BOP_DEV_ERR_CLUSTER 2u     // cluster larger than its scratch capacity
#define BOP_DEV_ERR_IMAGE 4u       // periodic image index outside [-127, 127]
#define BOP_DEV_ERR_NONFINITE 8u   // NaN/Inf in a scalar stage
#define BOP_DEV_ERR_REVERSE 16u    // reverse edge not found (asymmetric list)

// Parameters of the exponential two-centre model (beta = b0 e^{-lam(r-r0)} fcut).
struct BondModel {
  int norb;     // 1 (s), 5 (d) or 6 (sd: s first)
  double b0[5];  // s: ss sigma; d: dd sigma, pi, delta; sd: dd sigma, pi, delta, ss sigma, sd sigma
  double r0, lam, rc, dc;
  double rep_A, rep_p;  // pair repulsion A e^{-p(r-r0)} fcut(r); A = 0: none
};

// Cluster of (atom, image) sites around every atom, hop levels in order.
struct ClusterView {
  const long long* site_off;  // [n+1] first site of each atom
  const int* level_end;       // [n][K+1] sites [0, level_end[k]) form C_k
  const int* site_atom;       // [S] atom of every site
  const long long* adj_off;   // [S+1] adjacency of every site
  const int2* adj;            // {neighbour site (local index), bond}, ascending site
  const unsigned long long* lvcnt;  // [S] byte k = entries with site < level_end[k]
  int K;
};

// ---------------------------------------------------------------- duals
// Value plus its gradient with respect to the three bond-vector components,
// in FP64 (D3) or FP32 (D3f, the forces of the FP32-products mode).
template <class T>
struct D3T {
  T v, g0, g1, g2;
};
using D3 = D3T<double>;
using D3f = D3T<float>;
__device__ __forceinline__ D3 dmk(double v) { return {v, 0.0, 0.0, 0.0}; }
template <class T>
__device__ __forceinline__ D3T<T> operator+(D3T<T> a, D3T<T> b) {
  return {a.v + b.v, a.g0 + b.g0, a.g1 + b.g1, a.g2 + b.g2};
}
template <class T>
__device__ __forceinline__ D3T<T> operator-(D3T<T> a, D3T<T> b) {
  return {a.v - b.v, a.g0 - b.g0, a.g1 - b.g1, a.g2 - b.g2};
}
template <class T>
__device__ __forceinline__ D3T<T> operator*(D3T<T> a, D3T<T> b) {
  return {a.v * b.v, a.g0 * b.v + a.v * b.g0, a.g1 * b.v + a.v * b.g1, a.g2 * b.v + a.v * b.g2};
}
// a constant of the model (FP64) taken in the dual's type
template <class T>
__device__ __forceinline__ D3T<T> operator*(double s, D3T<T> a) {
  const T t = (T)s;
  return {t * a.v, t * a.g0, t * a.g1, t * a.g2};
}
template <class T>
__device__ __forceinline__ D3T<T> operator*(D3T<T> a, double s) { return s * a; }
template <class T>
__device__ __forceinline__ D3T<T> operator+(D3T<T> a, double s) { return {a.v + (T)s, a.g0, a.g1, a.g2}; }
template <class T>
__device__ __forceinline__ D3T<T> operator+(double s, D3T<T> a) { return a + s; }
template <class T>
__device__ __forceinline__ D3T<T> operator-(D3T<T> a, double s) { return {a.v - (T)s, a.g0, a.g1, a.g2}; }
template <class T>
__device__ __forceinline__ D3T<T> operator-(double s, D3T<T> a) { return {(T)s - a.v, -a.g0, -a.g1, -a.g2}; }
template <class T>
__device__ __forceinline__ D3T<T> operator/(D3T<T> a, D3T<T> b) {
  const T q = a.v / b.v, ib = T(1) / b.v;
  return {q, (a.g0 - q * b.g0) * ib, (a.g1 - q * b.g1) * ib, (a.g2 - q * b.g2) * ib};
}
template <class T>
__device__ __forceinline__ D3T<T> dsqrt(D3T<T> a) {
  const T r = sqrt(a.v), h = T(0.5) / r;
  return {r, a.g0 * h, a.g1 * h, a.g2 * h};
}
template <class T>
__device__ __forceinline__ D3T<T> dexp(D3T<T> a) {
  const T e = exp(a.v);
  return {e, a.g0 * e, a.g1 * e, a.g2 * e};
}
template <class T>
__device__ __forceinline__ D3T<T> dcos(D3T<T> a) {
  T s, c;
  sincos(a.v, &s, &c);
  return {c, -s * a.g0, -s * a.g1, -s * a.g2};
}
template <class T>
__device__ __forceinline__ double dval(D3T<T> x) { return (double)x.v; }
__device__ __forceinline__ double dval(double x) { return x; }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ double dcos(double x) { return cos(x); }

// ---------------------------------------------------------------- blocks
// Cosine taper (Eq. cutoff) times the exponential bond integral.
template <class S>
__device__ __forceinline__ S bond_integral(const BondModel& m, int x, S r) {
  const double PI = 3.14159265358979323846;
  double rv = dval(r);
  S e = m.b0[x] * dexp(-m.lam * (r - m.r0));
  if (rv < m.rc - m.dc) return e;
  if (rv > m.rc) return 0.0 * e;
  S f = 0.5 * (dcos((PI / m.dc) * (r - (m.rc - m.dc))) + 1.0);
  return e * f;
}

// Pair repulsion of one bond, A e^{-p (r - r0)} fcut(r), with the taper of
// the bond integrals.
template <class S>
__device__ __forceinline__ S pair_repulsion(const BondModel& m, S r) {
  const double PI = 3.14159265358979323846;
  double rv = dval(r);
  S e = m.rep_A * dexp(-m.rep_p * (r - m.r0));
  if (rv < m.rc - m.dc) return e;
  if (rv > m.rc) return 0.0 * e;
  S f = 0.5 * (dcos((PI / m.dc) * (r - (m.rc - m.dc))) + 1.0);
  return e * f;
}

// Unique elements of the symmetric two-centre block for bond vector d
// (Eq. Hij rotated as in Eq. Hij_rot), from the Slater-Koster
// direction-cosine table.  s: u[0] = ss sigma.  d: orbital order
// 0 = 3z^2-r^2, 1 = zx, 2 = yz, 3 = x^2-y^2, 4 = xy; u[] holds the upper
// triangle row by row: (0,0) (0,1) (0,2) (0,3) (0,4) (1,1) (1,2) (1,3)
// (1,4) (2,2) (2,3) (2,4) (3,3) (3,4) (4,4).
// sd (norb 6): u[] holds the 21-element upper triangle of the 6x6 block,
// s first: (s,s) (s,d0..d4), then the d rows as above; the s-d elements are
// even in the direction cosines, so the block is symmetric.
template <class S>
__device__ void sk_unique_d(const BondModel& m, const S d[3], S r, S u[15]);

template <class S>
__device__ void sk_unique(const BondModel& m, const S d[3], S u[21]) {
  S r = dsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (m.norb == 1) {
    u[0] = bond_integral(m, 0, r);
    return;
  }
  if (m.norb == 5) {
    sk_unique_d(m, d, r, u);
    return;
  }
  S ud[15];
  sk_unique_d(m, d, r, ud);
  const S ss = bond_integral(m, 3, r), sd = bond_integral(m, 4, r);
  const S l = d[0] / r, mm = d[1] / r, n = d[2] / r;
  const double r3 = 1.7320508075688772;
  u[0] = ss;
  u[1] = (n * n - 0.5 * (l * l + mm * mm)) * sd;  // 3z^2 - r^2
  u[2] = r3 * n * l * sd;                          // zx
  u[3] = r3 * mm * n * sd;                         // yz
  u[4] = 0.5 * r3 * (l * l - mm * mm) * sd;        // x^2 - y^2
  u[5] = r3 * l * mm * sd;                         // xy
#pragma unroll
  for (int q = 0; q < 15; q++) u[6 + q] = ud[q];   // the d rows keep their order
}

template <class S>
__device__ void sk_unique_d(const BondModel& m, const S d[3], S r, S u[15]) {
  const S vs = bond_integral(m, 0, r), vp = bond_integral(m, 1, r), vd = bond_integral(m, 2, r);
  const S l = d[0] / r, mm = d[1] / r, n = d[2] / r;
  const S L = l * l, M = mm * mm, N = n * n;
  const S LM = L - M, LpM = L + M;
  const S q = N - 0.5 * LpM;  // n^2 - (l^2+m^2)/2
  const double r3 = 1.7320508075688772;
  // 3z^2-r^2 row
  u[0] = q * q * vs + 3.0 * N * LpM * vp + 0.75 * LpM * LpM * vd;
  u[1] = r3 * l * n * q * vs + r3 * l * n * (LpM - N) * vp - 0.5 * r3 * l * n * LpM * vd;
  u[2] = r3 * mm * n * q * vs + r3 * mm * n * (LpM - N) * vp - 0.5 * r3 * mm * n * LpM * vd;
  u[3] = 0.5 * r3 * LM * q * vs - r3 * N * LM * vp + 0.25 * r3 * (1.0 + N) * LM * vd;
  u[4] = r3 * l * mm * q * vs - 2.0 * r3 * l * mm * N * vp + 0.5 * r3 * l * mm * (1.0 + N) * vd;
  // zx row
  u[5] = 3.0 * N * L * vs + (N + L - 4.0 * N * L) * vp + (M + N * L) * vd;
  u[6] = 3.0 * l * mm * N * vs + l * mm * (1.0 - 4.0 * N) * vp + l * mm * (N - 1.0) * vd;
  u[7] = 1.5 * n * l * LM * vs + n * l * (1.0 - 2.0 * LM) * vp - n * l * (1.0 - 0.5 * LM) * vd;
  u[8] = 3.0 * L * mm * n * vs + mm * n * (1.0 - 4.0 * L) * vp + mm * n * (L - 1.0) * vd;
  // yz row
  u[9] = 3.0 * M * N * vs + (M + N - 4.0 * M * N) * vp + (L + M * N) * vd;
  u[10] = 1.5 * mm * n * LM * vs - mm * n * (1.0 + 2.0 * LM) * vp + mm * n * (1.0 + 0.5 * LM) * vd;
  u[11] = 3.0 * l * M * n * vs + l * n * (1.0 - 4.0 * M) * vp + l * n * (M - 1.0) * vd;
  // x^2-y^2 row
  u[12] = 0.75 * LM * LM * vs + (LpM - LM * LM) * vp + (N + 0.25 * LM * LM) * vd;
  u[13] = 1.5 * l * mm * LM * vs - 2.0 * l * mm * LM * vp + 0.5 * l * mm * LM * vd;
  // xy row
  u[14] = 3.0 * L * M * vs + (LpM - 4.0 * L * M) * vp + (N + L * M) * vd;
}

// Position of element (b, g) of an NO x NO symmetric block in the unique
// list (upper triangle, row by row).
__host__ __device__ __forceinline__ constexpr int sym_index_n(int b, int g, int no) {
  return b <= g ? b * no - (b * (b - 1)) / 2 + (g - b) : g * no - (g * (g - 1)) / 2 + (b - g);
}
__host__ __device__ __forceinline__ int sym_index(int b, int g) { return sym_index_n(b, g, 5); }
// stored / unique elements of a block
__host__ __device__ __forceinline__ constexpr int block_store(int norb) {
  return norb == 1 ? 1 : (norb == 5 ? BOP_HS_D : BOP_HS_SD);
}
__host__ __device__ __forceinline__ constexpr int block_unique(int norb) {
  return norb == 1 ? 1 : (norb == 5 ? 15 : 21);
}

// The FP64 bond-vector arithmetic of the neighbour test, one rounding per
// operation (no contraction into FMA):
//   shift_c = (sx*c0c + sy*c1c) + sz*c2c,  d_c = (p_j,c + shift_c) - p_i,c
__device__ __forceinline__ void bond_vector(const double* __restrict__ pi, const double* __restrict__ pj,
                                            const double cell[9], int sx, int sy, int sz, double d[3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double sh = __dadd_rn(__dmul_rn((double)sx, cell[c]), __dmul_rn((double)sy, cell[3 + c]));
    sh = __dadd_rn(sh, __dmul_rn((double)sz, cell[6 + c]));
    d[c] = __dsub_rn(__dadd_rn(pj[c], sh), pi[c]);
  }
}
__device__ __forceinline__ double norm2_rn(const double d[3]) {
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__device__ __forceinline__ void raise_error(unsigned* status, unsigned bit) { atomicOr(status, bit); }
