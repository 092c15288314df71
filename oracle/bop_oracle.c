/*
 * Plain FP64 CPU oracle for the analytic-BOP moments path (BOPfox paper,
 * arXiv:1803.07491).  TEST INFRASTRUCTURE ONLY: it is loaded by the tests,
 * by __graft_entry__.smoke() and by bench.py's cpu_baseline / reference
 * arm.  The product path never calls it and shares no code with it.
 *
 * Written for obviousness, not speed: every loop follows the definition it
 * cites.  Compile with -ffp-contract=off so that no multiply-add is fused
 * (the neighbour-list distance test must be reproducible bit for bit).
 *
 * Contents
 *   orc_neighbors   short-range neighbour list by brute force over all atoms
 *                   and periodic images ("Initialisation", the linked-cell
 *                   list only makes this O(N)); sorted by (j, sx, sy, sz).
 *   orc_block       two-centre Slater-Koster block of one bond (Eq. Hij,
 *                   Eq. cutoff, Eq. Hij_rot), complex-capable for
 *                   complex-step derivatives.  The rotation to the global
 *                   frame is taken from the Slater-Koster direction-cosine
 *                   table (Phys. Rev. 94, 1498 (1954), Table I).
 *   orc_cluster     hop levels C_0 c C_1 c ... c C_K of (atom, image) sites
 *                   reachable from atom i -- the support of the
 *                   self-returning paths of Eq. momDOS; canonical order:
 *                   level, then atom, then image (sx, sy, sz).
 *   orc_moments     mu_n(i alpha) = <i alpha|H^n|i alpha> (Eq. momDOS) with
 *                   Psi_k = H Psi_{k-1} (Eq. xi_rec) and the merge property
 *                   (Eq. xi_merge): mu_2k = <Psi_k|Psi_k>,
 *                   mu_2k+1 = <Psi_k|Psi_k+1>.
 *   orc_moments_adjoint
 *                   reverse sweep of orc_moments: given w_n = dU/dmu_n
 *                   (Eq. weights) it accumulates dU/dH for every directed
 *                   edge and dU/dE for every onsite level -- the bond-order
 *                   like term Theta-tilde of Eq. theta-tilde, obtained here by
 *                   plain reverse-mode differentiation of the forward loop.
 *   orc_bond_gradient
 *                   g_e = sum_{beta gamma} Hbar_e dH_e/dd_e by complex-step
 *                   differentiation of orc_block (exact to rounding).
 *   orc_moments_nc  non-collinear magnetism (section "Magnetism"): the 2x2
 *                   spin moments <i alpha, a|H^n|i alpha, b> of the spinor
 *                   Hamiltonian H_e x 1 + onsite Ebar + h.sigma, by the same
 *                   recursion with complex 2-spinor amplitudes.
 *   orc_moments_nc_adjoint
 *                   its reverse sweep for sum_n Re Tr(W_n M_n): bond
 *                   cotangents and those of every onsite matrix.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double PI = 3.14159265358979323846;

/* Model of one element.  norb = 1 (s), 5 (d) or 6 (sd: s first, then the
 * five d orbitals).  b0[] holds the bond integrals at r0: s -> {ss sigma},
 * d -> {dd sigma, dd pi, dd delta}, sd -> {dd sigma, dd pi, dd delta,
 * ss sigma, sd sigma}.  beta(r) = b0 * exp(-lam (r - r0)) * fcut(r)
 * (exponential form). */
typedef struct {
  int norb;
  double r0, lam, rc, dc;
  double b0[5];
} orc_model;

/* ------------------------------------------------------------------ */
/* Neighbour list                                                       */
/* ------------------------------------------------------------------ */

/* Reciprocal vectors b_a (without 2 pi): rows of inv(cell)^T, where the
 * rows of cell are the lattice vectors. */
static void recip(const double *cell, double *b) {
  const double *a0 = cell, *a1 = cell + 3, *a2 = cell + 6;
  double c12[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2],
                   a1[0] * a2[1] - a1[1] * a2[0]};
  double c20[3] = {a2[1] * a0[2] - a2[2] * a0[1], a2[2] * a0[0] - a2[0] * a0[2],
                   a2[0] * a0[1] - a2[1] * a0[0]};
  double c01[3] = {a0[1] * a1[2] - a0[2] * a1[1], a0[2] * a1[0] - a0[0] * a1[2],
                   a0[0] * a1[1] - a0[1] * a1[0]};
  double vol = a0[0] * c12[0] + a0[1] * c12[1] + a0[2] * c12[2];
  for (int c = 0; c < 3; c++) {
    b[0 * 3 + c] = c12[c] / vol;
    b[1 * 3 + c] = c20[c] / vol;
    b[2 * 3 + c] = c01[c] / vol;
  }
}

/* Image search range along each axis: positions lie inside the cell, so
 * fractional differences are in (-1, 1); ceil(rcut |b_a|) + 1 images cover
 * every pair closer than rcut. */
void orc_image_range(const double *cell, const int *pbc, double rcut, int *nimg) {
  double b[9];
  recip(cell, b);
  for (int a = 0; a < 3; a++) {
    double nb = sqrt(b[a * 3] * b[a * 3] + b[a * 3 + 1] * b[a * 3 + 1] +
                     b[a * 3 + 2] * b[a * 3 + 2]);
    nimg[a] = pbc[a] ? (int)ceil(rcut * nb) + 1 : 0;
  }
}

/* The distance test, spelled out operation by operation:
 *   shift_c = (sx*cell[0][c] + sy*cell[1][c]) + sz*cell[2][c]
 *   d_c     = (pos_j_c + shift_c) - pos_i_c
 *   r2      = (dx*dx + dy*dy) + dz*dz,   pair kept iff r2 < rcut*rcut. */
static int pair_in_range(const double *pi, const double *pj, const double *cell,
                         int sx, int sy, int sz, double rc2, double *d) {
  double r2 = 0.0;
  for (int c = 0; c < 3; c++) {
    double sh = (double)sx * cell[c] + (double)sy * cell[3 + c];
    sh = sh + (double)sz * cell[6 + c];
    double x = pj[c] + sh;
    d[c] = x - pi[c];
  }
  r2 = d[0] * d[0] + d[1] * d[1];
  r2 = r2 + d[2] * d[2];
  return r2 < rc2;
}

/* Directed neighbour list in CSR form for the atoms 0..n-1.
 * Returns the number of edges, or -(needed) when max_e is too small
 * (row_ptr is then still filled with the counts' prefix sums). */
long orc_neighbors(int n, const double *pos, const double *cell, const int *pbc,
                   double rcut, long max_e, long *row_ptr, int *col,
                   signed char *img) {
  int ni[3];
  orc_image_range(cell, pbc, rcut, ni);
  double rc2 = rcut * rcut;
  long e = 0;
  row_ptr[0] = 0;
  for (int i = 0; i < n; i++) {
    for (int j = 0; j < n; j++)
      for (int sx = -ni[0]; sx <= ni[0]; sx++)
        for (int sy = -ni[1]; sy <= ni[1]; sy++)
          for (int sz = -ni[2]; sz <= ni[2]; sz++) {
            if (i == j && sx == 0 && sy == 0 && sz == 0) continue;
            double d[3];
            if (!pair_in_range(pos + 3 * i, pos + 3 * j, cell, sx, sy, sz, rc2, d))
              continue;
            if (e < max_e) {
              col[e] = j;
              img[3 * e] = (signed char)sx;
              img[3 * e + 1] = (signed char)sy;
              img[3 * e + 2] = (signed char)sz;
            }
            e++;
          }
    row_ptr[i + 1] = e;
  }
  return e <= max_e ? e : -e;
}

/* Bond vector of directed edge (i -> j, image S), same arithmetic as the
 * distance test. */
static void edge_vector(const double *pos, const double *cell, int i, int j,
                        const signed char *s, double *d) {
  (void)pair_in_range(pos + 3 * i, pos + 3 * j, cell, s[0], s[1], s[2], 0.0, d);
}

/* ------------------------------------------------------------------ */
/* Slater-Koster blocks                                                 */
/* ------------------------------------------------------------------ */

/* Cosine cutoff, Eq. cutoff: 1 below rc - dc, the cosine taper on
 * [rc - dc, rc], 0 beyond.  Branches use the real part (complex step). */
static cplx fcut(const orc_model *m, cplx r) {
  double rr = creal(r);
  if (rr < m->rc - m->dc) return 1.0;
  if (rr > m->rc) return 0.0;
  return 0.5 * (ccos(PI * (r - (m->rc - m->dc)) / m->dc) + 1.0);
}

/* Bond integral beta_x(r) = b0_x exp(-lam (r - r0)) fcut(r). */
static cplx bond_integral(const orc_model *m, int x, cplx r) {
  return m->b0[x] * cexp(-m->lam * (r - m->r0)) * fcut(m, r);
}

static void d_block(const orc_model *m, const cplx *d, cplx r, cplx E[5][5]);

/* Block <i beta|H|j gamma> for the bond vector d = r_j - r_i.
 * d orbitals ordered d_{3z^2-r^2}, d_zx, d_yz, d_{x^2-y^2}, d_xy (the order
 * stated under Eq. Hij); sd blocks put s first.  Output row-major
 * [beta][gamma]. */
void orc_block_c(const orc_model *m, const cplx *d, cplx *B) {
  cplx r = csqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (m->norb == 1) {
    B[0] = bond_integral(m, 0, r);
    return;
  }
  cplx E[5][5];
  d_block(m, d, r, E);
  if (m->norb == 5) {
    for (int b = 0; b < 5; b++)
      for (int g = 0; g < 5; g++) B[b * 5 + g] = E[b][g];
    return;
  }
  /* sd: the s-d elements of the Slater-Koster table, each an even function
   * of the direction cosines, so <s|H|d> = <d|H|s> and the block is
   * symmetric. */
  cplx ss = bond_integral(m, 3, r), sd = bond_integral(m, 4, r);
  cplx l = d[0] / r, mm = d[1] / r, n = d[2] / r;
  const double r3 = sqrt(3.0);
  cplx f[5];
  f[0] = (n * n - 0.5 * (l * l + mm * mm)) * sd; /* 3z^2 - r^2 */
  f[1] = r3 * n * l * sd;                         /* zx */
  f[2] = r3 * mm * n * sd;                        /* yz */
  f[3] = 0.5 * r3 * (l * l - mm * mm) * sd;       /* x^2 - y^2 */
  f[4] = r3 * l * mm * sd;                        /* xy */
  B[0] = ss;
  for (int g = 0; g < 5; g++) {
    B[1 + g] = f[g];
    B[(1 + g) * 6] = f[g];
    for (int b = 0; b < 5; b++) B[(1 + b) * 6 + 1 + g] = E[b][g];
  }
}

/* The 5x5 d-d block (dd sigma, pi, delta = b0[0..2]). */
static void d_block(const orc_model *m, const cplx *d, cplx r, cplx E[5][5]) {
  cplx s = bond_integral(m, 0, r), p = bond_integral(m, 1, r),
       t = bond_integral(m, 2, r); /* sigma, pi, delta */
  cplx l = d[0] / r, mm = d[1] / r, n = d[2] / r;
  cplx L = l * l, M = mm * mm, N = n * n;
  const double r3 = sqrt(3.0);
  enum { Z2 = 0, ZX = 1, YZ = 2, X2Y2 = 3, XY = 4 };
  E[XY][XY] = 3.0 * L * M * s + (L + M - 4.0 * L * M) * p + (N + L * M) * t;
  E[YZ][YZ] = 3.0 * M * N * s + (M + N - 4.0 * M * N) * p + (L + M * N) * t;
  E[ZX][ZX] = 3.0 * N * L * s + (N + L - 4.0 * N * L) * p + (M + N * L) * t;
  E[XY][YZ] = 3.0 * l * M * n * s + l * n * (1.0 - 4.0 * M) * p + l * n * (M - 1.0) * t;
  E[YZ][ZX] = 3.0 * mm * N * l * s + mm * l * (1.0 - 4.0 * N) * p + mm * l * (N - 1.0) * t;
  E[ZX][XY] = 3.0 * n * L * mm * s + n * mm * (1.0 - 4.0 * L) * p + n * mm * (L - 1.0) * t;
  E[XY][X2Y2] = 1.5 * l * mm * (L - M) * s + 2.0 * l * mm * (M - L) * p +
                0.5 * l * mm * (L - M) * t;
  E[YZ][X2Y2] = 1.5 * mm * n * (L - M) * s - mm * n * (1.0 + 2.0 * (L - M)) * p +
                mm * n * (1.0 + 0.5 * (L - M)) * t;
  E[ZX][X2Y2] = 1.5 * n * l * (L - M) * s + n * l * (1.0 - 2.0 * (L - M)) * p -
                n * l * (1.0 - 0.5 * (L - M)) * t;
  E[XY][Z2] = r3 * l * mm * (N - 0.5 * (L + M)) * s - 2.0 * r3 * l * mm * N * p +
              0.5 * r3 * l * mm * (1.0 + N) * t;
  E[YZ][Z2] = r3 * mm * n * (N - 0.5 * (L + M)) * s + r3 * mm * n * (L + M - N) * p -
              0.5 * r3 * mm * n * (L + M) * t;
  E[ZX][Z2] = r3 * l * n * (N - 0.5 * (L + M)) * s + r3 * l * n * (L + M - N) * p -
              0.5 * r3 * l * n * (L + M) * t;
  E[X2Y2][X2Y2] = 0.75 * (L - M) * (L - M) * s + (L + M - (L - M) * (L - M)) * p +
                  (N + 0.25 * (L - M) * (L - M)) * t;
  E[X2Y2][Z2] = 0.5 * r3 * (L - M) * (N - 0.5 * (L + M)) * s + r3 * N * (M - L) * p +
                0.25 * r3 * (1.0 + N) * (L - M) * t;
  E[Z2][Z2] = (N - 0.5 * (L + M)) * (N - 0.5 * (L + M)) * s + 3.0 * N * (L + M) * p +
              0.75 * (L + M) * (L + M) * t;
  /* the table lists each unordered pair once; the block is symmetric */
  const int pairs[10][2] = {{XY, YZ}, {YZ, ZX}, {ZX, XY}, {XY, X2Y2}, {YZ, X2Y2},
                            {ZX, X2Y2}, {XY, Z2}, {YZ, Z2}, {ZX, Z2}, {X2Y2, Z2}};
  for (int q = 0; q < 10; q++) E[pairs[q][1]][pairs[q][0]] = E[pairs[q][0]][pairs[q][1]];
}

/* Real-valued block for a bond vector d (used by the tests directly). */
void orc_block(const orc_model *m, const double *d, double *B) {
  cplx dc[3] = {d[0], d[1], d[2]}, Bc[36];
  orc_block_c(m, dc, Bc);
  for (int q = 0; q < m->norb * m->norb; q++) B[q] = creal(Bc[q]);
}

/* Blocks of all directed edges: H[e] = block(d_e), d_e = r_j + S.cell - r_i. */
void orc_blocks(int n, const double *pos, const double *cell, const long *row_ptr,
                const int *col, const signed char *img, const orc_model *m,
                double *H) {
  int nb = m->norb * m->norb;
  for (int i = 0; i < n; i++)
    for (long e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
      double d[3];
      edge_vector(pos, cell, i, col[e], img + 3 * e, d);
      orc_block(m, d, H + e * nb);
    }
}

/* ------------------------------------------------------------------ */
/* Cluster of (atom, image) sites                                       */
/* ------------------------------------------------------------------ */

typedef struct {
  uint64_t *keys;
  int *vals;
  long cap;
} hmap;

static uint64_t site_key(int atom, int sx, int sy, int sz) {
  return ((uint64_t)(uint32_t)atom << 24) | ((uint64_t)(sx + 128) << 16) |
         ((uint64_t)(sy + 128) << 8) | (uint64_t)(sz + 128);
}

static void hm_init(hmap *h, long cap) {
  h->cap = 1;
  while (h->cap < 2 * cap) h->cap <<= 1;
  h->keys = (uint64_t *)malloc(sizeof(uint64_t) * h->cap);
  h->vals = (int *)malloc(sizeof(int) * h->cap);
  for (long q = 0; q < h->cap; q++) h->keys[q] = UINT64_MAX;
}
static void hm_free(hmap *h) {
  free(h->keys);
  free(h->vals);
}
static long hm_slot(const hmap *h, uint64_t k) {
  uint64_t x = k * 0x9E3779B97F4A7C15ull;
  long q = (long)(x >> 20) & (h->cap - 1);
  while (h->keys[q] != UINT64_MAX && h->keys[q] != k) q = (q + 1) & (h->cap - 1);
  return q;
}
static int hm_get(const hmap *h, uint64_t k) {
  long q = hm_slot(h, k);
  return h->keys[q] == k ? h->vals[q] : -1;
}
static void hm_put(hmap *h, uint64_t k, int v) {
  long q = hm_slot(h, k);
  h->keys[q] = k;
  h->vals[q] = v;
}

typedef struct {
  int nsite;
  int K;
  int *level_end; /* [K+1]: sites [0, level_end[k]) form C_k */
  int *atom;      /* [nsite] */
  signed char *im; /* [nsite][3] */
  hmap map;
} cluster;

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y);
}

/* Path-radius cut ("Performance", item (iii)): with rpath > 0 only sites
 * closer than rpath to atom i (distance by the arithmetic of the neighbour
 * test) join the cluster, so paths that leave that sphere are dropped.
 * pos, cell may be NULL when rpath <= 0. */
typedef struct {
  const double *pos, *cell;
  double r2; /* rpath^2, or <= 0 for no cut */
} pathcut;

/* C_0 = {(i,0)}; C_k = C_{k-1} plus every neighbour of a site of C_{k-1}
 * (inside the path radius when one is set).  Only the frontier
 * C_{k-1} \ C_{k-2} can add new sites.  New sites of a level are appended
 * in ascending (atom, sx, sy, sz) order.
 * Returns 0, or -1 if an image index leaves [-127, 127]. */
static int build_cluster(cluster *c, int i, int K, const long *row_ptr,
                         const int *col, const signed char *img, pathcut pc) {
  long cap = 64, nsite = 1;
  c->K = K;
  c->level_end = (int *)malloc(sizeof(int) * (K + 1));
  c->atom = (int *)malloc(sizeof(int) * cap);
  c->im = (signed char *)malloc(3 * cap);
  hm_init(&c->map, 2048);
  c->atom[0] = i;
  c->im[0] = c->im[1] = c->im[2] = 0;
  hm_put(&c->map, site_key(i, 0, 0, 0), 0);
  c->level_end[0] = 1;
  int ok = 0;
  for (int k = 1; k <= K; k++) {
    int f0 = k >= 2 ? c->level_end[k - 2] : 0, f1 = c->level_end[k - 1];
    long nnew = 0, newcap = 256;
    uint64_t *nk = (uint64_t *)malloc(sizeof(uint64_t) * newcap);
    hmap seen; /* keys already queued for this level */
    hm_init(&seen, 1024);
    for (int t = f0; t < f1; t++) {
      int a = c->atom[t];
      for (long e = row_ptr[a]; e < row_ptr[a + 1]; e++) {
        int sx = c->im[3 * t] + img[3 * e], sy = c->im[3 * t + 1] + img[3 * e + 1],
            sz = c->im[3 * t + 2] + img[3 * e + 2];
        if (sx < -127 || sx > 127 || sy < -127 || sy > 127 || sz < -127 || sz > 127) {
          ok = -1;
          continue;
        }
        uint64_t key = site_key(col[e], sx, sy, sz);
        if (hm_get(&c->map, key) >= 0 || hm_get(&seen, key) >= 0) continue;
        if (pc.r2 > 0.0) {
          double d[3];
          if (!pair_in_range(pc.pos + 3 * i, pc.pos + 3 * col[e], pc.cell, sx, sy, sz, pc.r2, d)) continue;
        }
        if (nnew == newcap) {
          newcap *= 2;
          nk = (uint64_t *)realloc(nk, sizeof(uint64_t) * newcap);
        }
        if (2 * (nnew + 1) > seen.cap) {
          hmap h2;
          hm_init(&h2, 2 * (nnew + 1));
          for (long q = 0; q < nnew; q++) hm_put(&h2, nk[q], 0);
          hm_free(&seen);
          seen = h2;
        }
        hm_put(&seen, key, 0);
        nk[nnew++] = key;
      }
    }
    hm_free(&seen);
    qsort(nk, nnew, sizeof(uint64_t), cmp_u64);
    if (nsite + nnew > cap) {
      while (nsite + nnew > cap) cap *= 2;
      c->atom = (int *)realloc(c->atom, sizeof(int) * cap);
      c->im = (signed char *)realloc(c->im, 3 * cap);
    }
    if (2 * (nsite + nnew) > c->map.cap) { /* grow the map */
      hmap h2;
      hm_init(&h2, 2 * (nsite + nnew));
      for (long q = 0; q < nsite; q++)
        hm_put(&h2, site_key(c->atom[q], c->im[3 * q], c->im[3 * q + 1], c->im[3 * q + 2]),
               (int)q);
      hm_free(&c->map);
      c->map = h2;
    }
    for (long q = 0; q < nnew; q++) {
      uint64_t key = nk[q];
      c->atom[nsite] = (int)(key >> 24);
      c->im[3 * nsite] = (signed char)((int)((key >> 16) & 0xff) - 128);
      c->im[3 * nsite + 1] = (signed char)((int)((key >> 8) & 0xff) - 128);
      c->im[3 * nsite + 2] = (signed char)((int)(key & 0xff) - 128);
      hm_put(&c->map, key, (int)nsite);
      nsite++;
    }
    free(nk);
    c->level_end[k] = (int)nsite;
  }
  c->nsite = (int)nsite;
  return ok;
}

static void free_cluster(cluster *c) {
  free(c->level_end);
  free(c->atom);
  free(c->im);
  hm_free(&c->map);
}

/* Local index of the neighbour of site t across edge e, or -1. */
static int neighbour_site(const cluster *c, int t, long e, const int *col,
                          const signed char *img) {
  int sx = c->im[3 * t] + img[3 * e], sy = c->im[3 * t + 1] + img[3 * e + 1],
      sz = c->im[3 * t + 2] + img[3 * e + 2];
  if (sx < -127 || sx > 127 || sy < -127 || sy > 127 || sz < -127 || sz > 127) return -1;
  return hm_get(&c->map, site_key(col[e], sx, sy, sz));
}

/* Exported cluster enumeration for the bit-exact tests: writes up to
 * max_sites sites (atom, image) and the K+1 level ends.  Returns the number
 * of sites, or -1 on an image overflow. */
int orc_cluster(int i, int K, const long *row_ptr, const int *col,
                const signed char *img, const double *pos, const double *cell, double rpath,
                int max_sites, int *site_atom, signed char *site_img, int *level_end) {
  cluster c;
  pathcut pc = {pos, cell, rpath > 0.0 ? rpath * rpath : 0.0};
  if (build_cluster(&c, i, K, row_ptr, col, img, pc) < 0) {
    free_cluster(&c);
    return -1;
  }
  for (int k = 0; k <= K; k++) level_end[k] = c.level_end[k];
  for (int t = 0; t < c.nsite && t < max_sites; t++) {
    site_atom[t] = c.atom[t];
    site_img[3 * t] = c.im[3 * t];
    site_img[3 * t + 1] = c.im[3 * t + 1];
    site_img[3 * t + 2] = c.im[3 * t + 2];
  }
  int ns = c.nsite;
  free_cluster(&c);
  return ns;
}

/* ------------------------------------------------------------------ */
/* Moments and their reverse sweep                                      */
/* ------------------------------------------------------------------ */

/* out[t] += (H Psi_in)[t] restricted to rows t < rows and columns
 * s < cols: onsite term E_t Psi_in[t] plus sum over edges t->s of
 * H_e Psi_in[s] (Eq. xi_rec). */
static void apply_H(const cluster *c, int rows, int cols, int norb, const long *row_ptr,
                    const int *col, const signed char *img, const double *H,
                    const double *onsite, const double *in, double *out) {
  int nb = norb * norb;
  for (int t = 0; t < rows; t++) {
    int a = c->atom[t];
    if (t < cols)
      for (int b = 0; b < norb; b++) out[t * norb + b] += onsite[a * norb + b] * in[t * norb + b];
    for (long e = row_ptr[a]; e < row_ptr[a + 1]; e++) {
      int s = neighbour_site(c, t, e, col, img);
      if (s < 0 || s >= cols) continue;
      const double *B = H + e * nb;
      for (int b = 0; b < norb; b++)
        for (int g = 0; g < norb; g++) out[t * norb + b] += B[b * norb + g] * in[s * norb + g];
    }
  }
}

static double dot(const double *x, const double *y, long n) {
  double acc = 0.0;
  for (long q = 0; q < n; q++) acc += x[q] * y[q];
  return acc;
}

/* Moments of the atoms listed in sel[0..nsel-1] for n_mom = 2K+1 moments.
 * onsite: [n][norb] for one spin channel.  mu: [nsel][norb][n_mom].
 * Returns 0, or -1 on an image overflow. */
int orc_moments(int nsel, const int *sel, int n_mom, int norb, const long *row_ptr,
                const int *col, const signed char *img, const double *pos, const double *cell,
                double rpath, const double *H, const double *onsite, double *mu) {
  int K = (n_mom - 1) / 2, status = 0;
  pathcut pc = {pos, cell, rpath > 0.0 ? rpath * rpath : 0.0};
  for (int q = 0; q < nsel; q++) {
    int i = sel[q];
    cluster c;
    if (build_cluster(&c, i, K, row_ptr, col, img, pc) < 0) status = -1;
    long len = (long)c.nsite * norb;
    double *prev = (double *)calloc(len, sizeof(double));
    double *cur = (double *)calloc(len, sizeof(double));
    for (int al = 0; al < norb; al++) {
      double *m = mu + ((long)q * norb + al) * n_mom;
      memset(prev, 0, sizeof(double) * len);
      prev[al] = 1.0; /* Psi_0 = |i alpha>, site 0 is atom i itself */
      m[0] = 1.0;
      for (int k = 1; k <= K; k++) {
        memset(cur, 0, sizeof(double) * len);
        apply_H(&c, c.level_end[k], c.level_end[k - 1], norb, row_ptr, col, img, H, onsite,
                prev, cur);
        m[2 * k - 1] = dot(prev, cur, (long)c.level_end[k - 1] * norb);
        m[2 * k] = dot(cur, cur, (long)c.level_end[k] * norb);
        double *sw = prev; prev = cur; cur = sw;
      }
    }
    free(prev);
    free(cur);
    free_cluster(&c);
  }
  return status;
}

/* Reverse sweep.  w: [nsel][norb][n_mom] = dU/dmu.  Accumulates (+=)
 *   Hbar[e][b][g] = dU/dH_e[b][g]   for every directed edge e (entries of H
 *                                  treated as independent variables),
 *   Ebar[a][b]    = dU/dE_{a b}    for every onsite level. */
int orc_moments_adjoint(int nsel, const int *sel, int n_mom, int norb,
                        const long *row_ptr, const int *col, const signed char *img,
                        const double *pos, const double *cell, double rpath,
                        const double *H, const double *onsite, const double *w,
                        double *Hbar, double *Ebar) {
  int K = (n_mom - 1) / 2, nb = norb * norb, status = 0;
  pathcut pc = {pos, cell, rpath > 0.0 ? rpath * rpath : 0.0};
  for (int q = 0; q < nsel; q++) {
    int i = sel[q];
    cluster c;
    if (build_cluster(&c, i, K, row_ptr, col, img, pc) < 0) status = -1;
    long len = (long)c.nsite * norb;
    double *psi = (double *)calloc(len * (K + 1), sizeof(double)); /* Psi_0..Psi_K */
    double *bar = (double *)calloc(len, sizeof(double));
    double *nbar = (double *)calloc(len, sizeof(double));
    for (int al = 0; al < norb; al++) {
      const double *wm = w + ((long)q * norb + al) * n_mom;
      memset(psi, 0, sizeof(double) * len * (K + 1));
      psi[al] = 1.0;
      for (int k = 1; k <= K; k++)
        apply_H(&c, c.level_end[k], c.level_end[k - 1], norb, row_ptr, col, img, H, onsite,
                psi + (k - 1) * len, psi + k * len);
      /* cotangent of Psi_K: from mu_2K = <Psi_K|Psi_K> and
       * mu_2K-1 = <Psi_K-1|Psi_K> */
      for (long x = 0; x < len; x++)
        bar[x] = 2.0 * wm[2 * K] * psi[K * len + x] + wm[2 * K - 1] * psi[(K - 1) * len + x];
      for (int k = K; k >= 1; k--) {
        const double *pin = psi + (k - 1) * len;
        int rows = c.level_end[k], cols = c.level_end[k - 1];
        memset(nbar, 0, sizeof(double) * len);
        for (int t = 0; t < rows; t++) {
          int a = c.atom[t];
          if (t < cols)
            for (int b = 0; b < norb; b++) {
              Ebar[a * norb + b] += bar[t * norb + b] * pin[t * norb + b];
              nbar[t * norb + b] += onsite[a * norb + b] * bar[t * norb + b];
            }
          for (long e = row_ptr[a]; e < row_ptr[a + 1]; e++) {
            int s = neighbour_site(&c, t, e, col, img);
            if (s < 0 || s >= cols) continue;
            const double *B = H + e * nb;
            double *Bb = Hbar + e * nb;
            for (int b = 0; b < norb; b++)
              for (int g = 0; g < norb; g++) {
                Bb[b * norb + g] += bar[t * norb + b] * pin[s * norb + g];
                nbar[s * norb + g] += B[b * norb + g] * bar[t * norb + b];
              }
          }
        }
        if (k == 1) break;
        /* dot-product cotangents of Psi_{k-1}: mu_2(k-1), mu_2k-1, mu_2k-3 */
        for (long x = 0; x < (long)cols * norb; x++) {
          double v = nbar[x] + 2.0 * wm[2 * (k - 1)] * pin[x] + wm[2 * k - 1] * psi[k * len + x];
          v += wm[2 * k - 3] * psi[(k - 2) * len + x];
          bar[x] = v;
        }
        for (long x = (long)cols * norb; x < len; x++) bar[x] = 0.0;
      }
    }
    free(psi);
    free(bar);
    free(nbar);
    free_cluster(&c);
  }
  return status;
}

/* g[e] = sum_{b,g} Hbar[e][b][g] dH_e[b][g]/dd_e, d_e = r_j + S.cell - r_i,
 * by complex-step differentiation (step 1e-30i). */
void orc_bond_gradient(int n, const double *pos, const double *cell, const long *row_ptr,
                       const int *col, const signed char *img, const orc_model *m,
                       const double *Hbar, double *g) {
  int nb = m->norb * m->norb;
  const double h = 1e-30;
  for (int i = 0; i < n; i++)
    for (long e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
      double d[3];
      edge_vector(pos, cell, i, col[e], img + 3 * e, d);
      for (int c = 0; c < 3; c++) {
        cplx dc[3] = {d[0], d[1], d[2]}, B[36];
        dc[c] += h * I;
        orc_block_c(m, dc, B);
        double acc = 0.0;
        for (int q = 0; q < nb; q++) acc += Hbar[e * nb + q] * cimag(B[q]) / h;
        g[3 * e + c] = acc;
      }
    }
}

/* Bond vectors of all directed edges (for the virial). */
void orc_edge_vectors(int n, const double *pos, const double *cell, const long *row_ptr,
                      const int *col, const signed char *img, double *dvec) {
  for (int i = 0; i < n; i++)
    for (long e = row_ptr[i]; e < row_ptr[i + 1]; e++)
      edge_vector(pos, cell, i, col[e], img + 3 * e, dvec + 3 * e);
}

/* ------------------------------------------------------------------ */
/* Non-collinear magnetism: spinor moments and their reverse sweep      */
/* ------------------------------------------------------------------ */

/* Section "Magnetism", Eq. onsite_CM and Eq. onsite-noncollinear: the
 * hopping is spin independent (H_e x 1), the onsite matrix of orbital b of
 * atom a is
 *     O_ab = Ebar 1 + h . sigma,   Ebar = (E_up + E_dn)/2,
 *                                  h = (E_dn - E_up)/2 s_a,
 * s_a the unit direction of the atom's moment; in the frame along s_a it is
 * diag(E_up, E_dn), the lower level E_up belonging to the spin antiparallel
 * to s_a.  onsite2: [2][n][norb] (E_up, E_dn), sdir: [n][3].  Amplitudes
 * are [site][orbital][spin] complex, spin the basis along z. */
static void onsite_field(const double *onsite2, const double *sdir, int n, int norb, int a, int b,
                         double *eb, double h[3]) {
  double eu = onsite2[(long)a * norb + b], ed = onsite2[((long)n + a) * norb + b];
  *eb = 0.5 * (eu + ed);
  for (int x = 0; x < 3; x++) h[x] = 0.5 * (ed - eu) * sdir[3 * a + x];
}

/* out += H in for one starting column, rows t < rows, columns s < cols */
static void apply_H_nc(const cluster *c, int rows, int cols, int norb, int n, const long *row_ptr,
                       const int *col, const signed char *img, const double *H,
                       const double *onsite2, const double *sdir, const cplx *in, cplx *out) {
  int nb = norb * norb;
  for (int t = 0; t < rows; t++) {
    int a = c->atom[t];
    if (t < cols)
      for (int b = 0; b < norb; b++) {
        double eb, h[3];
        onsite_field(onsite2, sdir, n, norb, a, b, &eb, h);
        cplx u = in[(t * norb + b) * 2], d = in[(t * norb + b) * 2 + 1];
        /* (Ebar + h.sigma)(u, d), sigma_x = [[0,1],[1,0]],
         * sigma_y = [[0,-i],[i,0]], sigma_z = diag(1,-1) */
        out[(t * norb + b) * 2] += (eb + h[2]) * u + (h[0] - I * h[1]) * d;
        out[(t * norb + b) * 2 + 1] += (h[0] + I * h[1]) * u + (eb - h[2]) * d;
      }
    for (long e = row_ptr[a]; e < row_ptr[a + 1]; e++) {
      int s = neighbour_site(c, t, e, col, img);
      if (s < 0 || s >= cols) continue;
      const double *B = H + e * nb;
      for (int b = 0; b < norb; b++)
        for (int g = 0; g < norb; g++)
          for (int sp = 0; sp < 2; sp++)
            out[(t * norb + b) * 2 + sp] += B[b * norb + g] * in[(s * norb + g) * 2 + sp];
    }
  }
}

/* <x|y> = sum conj(x) y */
static cplx cdot(const cplx *x, const cplx *y, long len) {
  cplx acc = 0.0;
  for (long q = 0; q < len; q++) acc += conj(x[q]) * y[q];
  return acc;
}

/* Psi_0..Psi_K of both starting columns |i alpha, z-up>, |i alpha, z-down>
 * into psi[col][k][len] (len = nsite * norb * 2). */
static void spinor_levels(const cluster *c, int K, int al, int norb, int n, const long *row_ptr,
                          const int *col, const signed char *img, const double *H,
                          const double *onsite2, const double *sdir, cplx *psi, long len) {
  memset(psi, 0, sizeof(cplx) * 2 * (K + 1) * len);
  for (int a = 0; a < 2; a++) {
    cplx *p = psi + (long)a * (K + 1) * len;
    p[al * 2 + a] = 1.0;
    for (int k = 1; k <= K; k++)
      apply_H_nc(c, c->level_end[k], c->level_end[k - 1], norb, n, row_ptr, col, img, H, onsite2, sdir,
                 p + (k - 1) * len, p + k * len);
  }
}

/* Global 2x2 moments M_n[a][b] = <i alpha, a|H^n|i alpha, b>, n < n_mom,
 * by the merge property (Eq. xi_merge) for both starting spin states:
 * M_2k = <Psi_k^a|Psi_k^b>, M_2k-1 = <Psi_k-1^a|Psi_k^b>.
 * M: [nsel][norb][n_mom][2][2] complex.  Returns 0, or -1 on an image
 * overflow. */
int orc_moments_nc(int nsel, const int *sel, int n, int n_mom, int norb, const long *row_ptr,
                   const int *col, const signed char *img, const double *pos, const double *cell,
                   double rpath, const double *H, const double *onsite2, const double *sdir, cplx *M) {
  int K = (n_mom - 1) / 2, status = 0;
  pathcut pc = {pos, cell, rpath > 0.0 ? rpath * rpath : 0.0};
  for (int q = 0; q < nsel; q++) {
    cluster c;
    if (build_cluster(&c, sel[q], K, row_ptr, col, img, pc) < 0) status = -1;
    long len = (long)c.nsite * norb * 2;
    cplx *psi = (cplx *)calloc(2 * (K + 1) * len, sizeof(cplx));
    for (int al = 0; al < norb; al++) {
      spinor_levels(&c, K, al, norb, n, row_ptr, col, img, H, onsite2, sdir, psi, len);
      cplx *m = M + ((long)q * norb + al) * n_mom * 4;
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
          const cplx *pa = psi + (long)a * (K + 1) * len, *pb = psi + (long)b * (K + 1) * len;
          m[a * 2 + b] = a == b ? 1.0 : 0.0;
          for (int k = 1; k <= K; k++) {
            m[(2 * k - 1) * 4 + a * 2 + b] =
                cdot(pa + (k - 1) * len, pb + k * len, (long)c.level_end[k - 1] * norb * 2);
            m[(2 * k) * 4 + a * 2 + b] = cdot(pa + k * len, pb + k * len, (long)c.level_end[k] * norb * 2);
          }
        }
    }
    free(psi);
    free_cluster(&c);
  }
  return status;
}

/* Reverse sweep of orc_moments_nc for L = sum_n Re Tr(W_n M_n) with
 * Hermitian 2x2 weights W: [nsel][norb][n_mom][2][2] complex (Eq.
 * dUdLambda-noncollinear).  A term Re sum_ab W_ba <p^a|q^b> gives the
 * cotangents (d/dRe + i d/dIm) p-bar^c += sum_b W_bc q^b and
 * q-bar^c += sum_a W_ac p^a.  Accumulates (+=)
 *   Hbar[e][b][g] = dL/dH_e[b][g] for every directed edge,
 *   Obar[a][b][0..3] = dL/d(Ebar, h_x, h_y, h_z) of orbital b of atom a. */
int orc_moments_nc_adjoint(int nsel, const int *sel, int n, int n_mom, int norb, const long *row_ptr,
                           const int *col, const signed char *img, const double *pos,
                           const double *cell, double rpath, const double *H, const double *onsite2,
                           const double *sdir, const cplx *W, double *Hbar, double *Obar) {
  int K = (n_mom - 1) / 2, nb = norb * norb, status = 0;
  pathcut pc = {pos, cell, rpath > 0.0 ? rpath * rpath : 0.0};
  for (int q = 0; q < nsel; q++) {
    cluster c;
    if (build_cluster(&c, sel[q], K, row_ptr, col, img, pc) < 0) status = -1;
    long len = (long)c.nsite * norb * 2;
    cplx *psi = (cplx *)calloc(2 * (K + 1) * len, sizeof(cplx));
    cplx *bar = (cplx *)calloc(2 * len, sizeof(cplx));
    cplx *nbar = (cplx *)calloc(2 * len, sizeof(cplx));
    for (int al = 0; al < norb; al++) {
      const cplx *w = W + ((long)q * norb + al) * n_mom * 4; /* w[m*4 + a*2 + b] */
      spinor_levels(&c, K, al, norb, n, row_ptr, col, img, H, onsite2, sdir, psi, len);
#define PSI(a, k) (psi + ((long)(a) * (K + 1) + (k)) * len)
      /* Psi-bar_K: 2 W_2K (self product) and W_2K-1 (q = Psi_K) */
      for (int cc = 0; cc < 2; cc++)
        for (long x = 0; x < len; x++) {
          cplx v = 0.0;
          for (int b = 0; b < 2; b++) {
            v += 2.0 * w[(2 * K) * 4 + b * 2 + cc] * PSI(b, K)[x];
            v += w[(2 * K - 1) * 4 + b * 2 + cc] * PSI(b, K - 1)[x];
          }
          bar[cc * len + x] = v;
        }
      for (int k = K; k >= 1; k--) {
        int rows = c.level_end[k], cols = c.level_end[k - 1];
        memset(nbar, 0, sizeof(cplx) * 2 * len);
        for (int cc = 0; cc < 2; cc++) {
          const cplx *pin = PSI(cc, k - 1), *bk = bar + cc * len;
          cplx *nb_ = nbar + cc * len;
          for (int t = 0; t < rows; t++) {
            int a = c.atom[t];
            if (t < cols)
              for (int b = 0; b < norb; b++) {
                double eb, h[3];
                onsite_field(onsite2, sdir, n, norb, a, b, &eb, h);
                cplx bu = bk[(t * norb + b) * 2], bd = bk[(t * norb + b) * 2 + 1];
                cplx pu = pin[(t * norb + b) * 2], pd = pin[(t * norb + b) * 2 + 1];
                double *ob = Obar + ((long)a * norb + b) * 4;
                ob[0] += creal(conj(bu) * pu + conj(bd) * pd);
                ob[1] += creal(conj(bu) * pd + conj(bd) * pu);
                ob[2] += creal(conj(bu) * (-I * pd) + conj(bd) * (I * pu));
                ob[3] += creal(conj(bu) * pu - conj(bd) * pd);
                /* O is Hermitian: the cotangent goes back through O itself */
                nb_[(t * norb + b) * 2] += (eb + h[2]) * bu + (h[0] - I * h[1]) * bd;
                nb_[(t * norb + b) * 2 + 1] += (h[0] + I * h[1]) * bu + (eb - h[2]) * bd;
              }
            for (long e = row_ptr[a]; e < row_ptr[a + 1]; e++) {
              int s = neighbour_site(&c, t, e, col, img);
              if (s < 0 || s >= cols) continue;
              const double *B = H + e * nb;
              double *Bb = Hbar + e * nb;
              for (int b = 0; b < norb; b++)
                for (int g = 0; g < norb; g++)
                  for (int sp = 0; sp < 2; sp++) {
                    Bb[b * norb + g] += creal(conj(bk[(t * norb + b) * 2 + sp]) * pin[(s * norb + g) * 2 + sp]);
                    nb_[(s * norb + g) * 2 + sp] += B[b * norb + g] * bk[(t * norb + b) * 2 + sp];
                  }
            }
          }
        }
        if (k == 1) break;
        /* dot-product cotangents of Psi_k-1: M_2(k-1) (self), M_2k-1 (as
         * p, partner Psi_k), M_2k-3 (as q, partner Psi_k-2) */
        for (int cc = 0; cc < 2; cc++)
          for (long x = 0; x < len; x++) {
            cplx v = 0.0;
            if (x < (long)cols * norb * 2) {
              v = nbar[cc * len + x];
              for (int b = 0; b < 2; b++) {
                v += 2.0 * w[(2 * k - 2) * 4 + b * 2 + cc] * PSI(b, k - 1)[x];
                v += w[(2 * k - 1) * 4 + b * 2 + cc] * PSI(b, k)[x];
                v += w[(2 * k - 3) * 4 + b * 2 + cc] * PSI(b, k - 2)[x];
              }
            }
            bar[cc * len + x] = v;
          }
#undef PSI
      }
    }
    free(psi);
    free(bar);
    free(nbar);
    free_cluster(&c);
  }
  return status;
}
