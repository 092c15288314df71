// Device helpers shared by the FP64 scalar-stage kernels (scalar.cu,
// chain.cu): moments -> recursion coefficients (Eqs. momtoa, momtob and the
// c_j^n recursion), Gershgorin band edges (Eq. gershogorin), the constant
// terminator (Eq. abinf) and the normalised chain parameters (Eq. aexp).
#pragma once
#include "kernels.h"

namespace scal {

constexpr double PI = 3.14159265358979323846;
constexpr double B_INF_MIN = 1e-3;   // eV, floor of the band-width estimate
constexpr double TRUNC_REL = 1e-10;  // recursion truncation threshold
constexpr int KPMAX = (BOP_MAX_NMOM - 1) / 2;

// ------------------------------------------------------------ recursion
struct Rec {
  double a[KPMAX];
  double b[KPMAX + 1];
  int nlev;
  bool trunc;
};

// a_n = sum c_j c_l mu_{j+l+1};  b_{n+1} c^{n+1} = c^n shifted - a_n c^n - b_n c^{n-1}
__device__ inline void recursion(const double* mu, int Kp, Rec& r) {
  double c[KPMAX + 2], cp[KPMAX + 2], d[KPMAX + 2];
  for (int j = 0; j < KPMAX + 2; j++) c[j] = cp[j] = 0.0;
  c[0] = 1.0;
  r.b[0] = 0.0;
  r.nlev = Kp;
  r.trunc = false;
  double width = fmax(mu[2] - mu[1] * mu[1], 0.0);
  for (int n = 0; n < Kp; n++) {
    double an = 0.0;
    for (int j = 0; j <= n; j++)
      for (int l = 0; l <= n; l++) an += c[j] * c[l] * mu[j + l + 1];
    r.a[n] = an;
    for (int j = 0; j <= n + 1; j++) d[j] = (j >= 1 ? c[j - 1] : 0.0) - an * c[j] - r.b[n] * cp[j];
    double b2 = 0.0;
    for (int j = 0; j <= n + 1; j++)
      for (int l = 0; l <= n + 1; l++) b2 += d[j] * d[l] * mu[j + l];
    if (b2 <= TRUNC_REL * width) {
      r.b[n + 1] = 0.0;
      r.nlev = n + 1;
      r.trunc = true;
      for (int q = n + 1; q < Kp; q++) {
        r.a[q] = 0.0;
        r.b[q + 1] = 0.0;
      }
      return;
    }
    double bn = sqrt(b2);
    r.b[n + 1] = bn;
    for (int j = 0; j <= n + 1; j++) {
      cp[j] = c[j];
      c[j] = d[j] / bn;
    }
  }
}

struct Term {
  double a_inf, b_inf;
  int ilo, ihi;  // Gershgorin: bottom / top level; MINMAX: argmin / argmax of a
  int ib;        // MINMAX: argmax of b
  double bsum;   // AVERAGE: rms b before the floor; WEIGHTED: sum of the a weights
  double wsum_b; // WEIGHTED: sum of the b weights
  bool floored;
};

// Gershgorin over the computed levels n < nlev (b_0 = 0); first index wins ties.
__device__ inline Term gershgorin(const Rec& r) {
  Term t;
  double bot = 0.0, top = 0.0;
  t.ilo = t.ihi = t.ib = 0;
  t.bsum = t.wsum_b = 0.0;
  for (int n = 0; n < r.nlev; n++) {
    double lo = r.a[n] - r.b[n] - r.b[n + 1];
    double hi = r.a[n] + r.b[n] + r.b[n + 1];
    if (n == 0 || lo < bot) { bot = lo; t.ilo = n; }
    if (n == 0 || hi > top) { top = hi; t.ihi = n; }
  }
  t.a_inf = 0.5 * (top + bot);
  t.b_inf = 0.25 * (top - bot);
  t.floored = t.b_inf < B_INF_MIN;
  if (t.floored) t.b_inf = B_INF_MIN;
  return t;
}

// The other estimates of the band centre A and width B (section "Band-width
// estimates", items (i)-(v), (viii), and the weighted averages of Eq.
// weighted) over the computed levels a_0..a_{L-1}, b_1..b_L, L = nlev.
// Ties in max / min go to the first index.  B is floored like Gershgorin's.
__device__ inline Term bandwidth(const Rec& r, const BandSel& p) {
  if (p.mode == BOP_BW_GERSHGORIN) return gershgorin(r);
  Term t;
  const int L = r.nlev;
  t.ilo = t.ihi = t.ib = 0;
  t.bsum = t.wsum_b = 0.0;
  double A = 0.0, B = 0.0;
  switch (p.mode) {
    case BOP_BW_LOWEST:
      A = r.a[0];
      B = r.b[1];
      break;
    case BOP_BW_HIGHEST:
      A = r.a[L - 1];
      B = r.b[L];
      break;
    case BOP_BW_AVERAGE:
    case BOP_BW_AVG_CENTRE: {
      double sa = 0.0, sb = 0.0;
      for (int n = 0; n < L; n++) sa += r.a[n];
      for (int n = 1; n <= L; n++) sb += r.b[n] * r.b[n];
      A = sa / L;
      B = p.mode == BOP_BW_AVERAGE ? sqrt(sb / L) : r.b[L];
      t.bsum = B;
      break;
    }
    case BOP_BW_MINMAX: {
      double amax = r.a[0], amin = r.a[0], bmax = r.b[1];
      for (int n = 1; n < L; n++) {
        if (r.a[n] > amax) { amax = r.a[n]; t.ihi = n; }
        if (r.a[n] < amin) { amin = r.a[n]; t.ilo = n; }
      }
      t.ib = 1;
      for (int n = 2; n <= L; n++)
        if (r.b[n] > bmax) { bmax = r.b[n]; t.ib = n; }
      A = 0.5 * (amax + amin);
      B = 0.25 * (amax - amin + 4.0 * bmax);
      break;
    }
    case BOP_BW_GLOBAL:
      A = p.ga;
      B = p.gb;
      break;
    default: {  // BOP_BW_WEIGHTED
      double wa = 0.0, wb = 0.0, sa = 0.0, sb = 0.0;
      for (int m = 0; m < L; m++) {
        const double w = 1.0 / (p.beta * (L - 1 - m) + 1.0);
        wa += w;
        sa += w * r.a[m];
      }
      for (int m = 1; m <= L; m++) {
        const double w = 1.0 / (p.beta * (L - m) + 1.0);
        wb += w;
        sb += w * r.b[m];
      }
      A = sa / wa;
      B = sb / wb;
      t.bsum = wa;
      t.wsum_b = wb;
    }
  }
  t.a_inf = A;
  t.b_inf = B;
  t.floored = B < B_INF_MIN;
  if (t.floored) t.b_inf = B_INF_MIN;
  return t;
}

// Chain parameters: a^_k (k < nlev) and b^_k (1 <= k <= Kp, k <= nlev);
// the constant terminator a^ = 0, b^ = 1/2 elsewhere.
struct Chain {
  double ah[KPMAX + 1];
  double bh[KPMAX + 2];
};
__device__ inline void chain_params(const Rec& r, const Term& t, int Kp, Chain& ch) {
  for (int k = 0; k <= KPMAX; k++) ch.ah[k] = 0.0;
  for (int k = 0; k <= KPMAX + 1; k++) ch.bh[k] = 0.5;
  ch.bh[0] = 0.0;
  for (int k = 0; k < r.nlev; k++) ch.ah[k] = (r.a[k] - t.a_inf) / (2.0 * t.b_inf);
  for (int k = 1; k <= Kp; k++)
    if (k <= r.nlev) ch.bh[k] = r.b[k] / (2.0 * t.b_inf);
}
__device__ __forceinline__ double AH(const Chain& ch, int k) { return k <= KPMAX ? ch.ah[k] : 0.0; }
__device__ __forceinline__ double BH(const Chain& ch, int k) { return k <= KPMAX + 1 ? ch.bh[k] : 0.5; }


__device__ __forceinline__ double clamp1(double x) { return x > 1.0 ? 1.0 : (x < -1.0 ? -1.0 : x); }

template <int NT>
__device__ inline double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < NT / 32; q++) t += sh[q];
  __syncthreads();
  return t;  // valid on thread 0
}

constexpr int RT = 256;
// Reduction of per-block partials by the last block of a grid: every thread
// of that block reads a strided share of the partials (L2 loads), then a
// fixed shuffle tree and a fixed cross-warp order.  Deterministic for a
// given grid size.  All threads of the block must call it; every thread
// receives the result.  sh: >= NT/32 + 1 doubles of shared memory.
template <int NT>
__device__ inline double final_reduce(const double* part, size_t stride, int q, int nblk, bool take_max,
                                      double* sh) {
  double v = take_max ? -1.0e300 : 0.0;
  for (int b = threadIdx.x; b < nblk; b += NT) {
    const double x = __ldcg(part + (size_t)b * stride + q);
    v = take_max ? fmax(v, x) : v + x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = take_max ? fmax(v, w) : v + w;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = sh[0];
    for (int w = 1; w < NT / 32; w++) t = take_max ? fmax(t, sh[w]) : t + sh[w];
    sh[NT / 32] = t;
  }
  __syncthreads();
  return sh[NT / 32];
}

}  // namespace scal
