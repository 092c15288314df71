// Per-orbital pieces of the expansion and of its reverse mode, shared by
// the constant-terminator kernels (chain.cu) and the learned-terminator
// kernels (learned.cu): the generating polynomials of the Chebyshev chain
// (Eq. aexp as a rational generating function), the sigma_m recurrence,
// and the reverse of each stage (chain -> sigma -> N, P; chain parameters;
// Gershgorin; moment recursion).
#pragma once
#include "scalar_common.cuh"

namespace scal {

// Polynomial coefficients D_0 (Q) and D_1 (P) of sum_m sigma_m t^m = D_1/D_0
// for a chain of L levels (D_L = D_{L+1} = 1).
template <int KP>
__device__ __forceinline__ void gen_polys(const Chain& ch, int L, double Q[2 * KP + 1], double P[2 * KP + 1]) {
  constexpr int NP = 2 * KP + 1;
  double d2[NP], d1[NP];
#pragma unroll
  for (int j = 0; j < NP; j++) d2[j] = d1[j] = (j == 0) ? 1.0 : 0.0;
  for (int k = L - 1; k >= 0; k--) {
    const double a2 = 2.0 * ch.ah[k];
    const double bb = 4.0 * ch.bh[k + 1] * ch.bh[k + 1];
    double dn[NP];
#pragma unroll
    for (int j = 0; j < NP; j++) {
      double v = d1[j];
      if (j >= 1) v -= a2 * d1[j - 1];
      if (j >= 2) v += d1[j - 2] - bb * d2[j - 2];
      dn[j] = v;
    }
#pragma unroll
    for (int j = 0; j < NP; j++) {
      d2[j] = d1[j];
      d1[j] = dn[j];
    }
  }
#pragma unroll
  for (int j = 0; j < NP; j++) {
    Q[j] = d1[j];
    P[j] = d2[j];
  }
}

// g_m sigma_m, m = 0..ne, into gsig[m][M] from the recurrence
// sigma_m = [D_1]_m - sum_{j>=1} [D_0]_j sigma_{m-j}.  Returns sigma_ne.
// With CHECK, *outside becomes true if some |sigma_m| > m + 1: sigma_m is
// the integral of U_m(x) times a density of unit weight, and |U_m| <= m + 1
// on [-1, 1], so the density then has weight outside the estimated band (a
// bound state of the terminated chain) and the series grows with m.  (A
// separate instantiation: the check is FP64 work in every coefficient.)
//
// With F32 the recurrence runs in FP32 (the FP32-products mode): its
// coefficients are O(1) for a chain scaled to the terminator's band, so that
// the rounding of each step is not amplified; the relative error of sigma_m
// stays below 1e-6 at 9 and 1e-5 at 17 moments (200 coefficients), a band
// energy error below 1e-6 eV per orbital.
template <int KP, bool CHECK = false, bool F32 = false>
__device__ __forceinline__ double sigma_series(double Q[2 * KP + 1], double P[2 * KP + 1], int ne,
                                               const double* __restrict__ g, double* __restrict__ gsig, int M,
                                               int o, bool* outside = nullptr) {
  constexpr int NP = 2 * KP + 1;
  if constexpr (F32) {
    float qf[NP], pf[NP], hf[NP - 1];
#pragma unroll
    for (int j = 0; j < NP; j++) {
      qf[j] = (float)Q[j];
      pf[j] = (float)P[j];
    }
#pragma unroll
    for (int j = 0; j < NP - 1; j++) hf[j] = 0.f;
    for (int m = 0; m <= ne; m++) {
      float v = pf[0];
#pragma unroll
      for (int j = 0; j < NP - 1; j++) pf[j] = pf[j + 1];
      pf[NP - 1] = 0.f;
#pragma unroll
      for (int j = 1; j < NP; j++) v -= qf[j] * hf[j - 1];
#pragma unroll
      for (int j = NP - 2; j >= 1; j--) hf[j] = hf[j - 1];
      hf[0] = v;
      gsig[(size_t)m * M + o] = g[m] * (double)v;
      if (CHECK && fabsf(v) > (m + 1) * (1.0f + 1e-6f)) *outside = true;
    }
    return (double)hf[0];
  } else {
    double h[NP - 1];  // h[j] = sigma_{m-1-j}
#pragma unroll
    for (int j = 0; j < NP - 1; j++) h[j] = 0.0;
    for (int m = 0; m <= ne; m++) {
      double v = P[0];
#pragma unroll
      for (int j = 0; j < NP - 1; j++) P[j] = P[j + 1];
      P[NP - 1] = 0.0;
#pragma unroll
      for (int j = 1; j < NP; j++) v -= Q[j] * h[j - 1];
#pragma unroll
      for (int j = NP - 2; j >= 1; j--) h[j] = h[j - 1];
      h[0] = v;
      gsig[(size_t)m * M + o] = g[m] * v;
      if (CHECK && fabs(v) > (m + 1) * (1.0 + 1e-9)) *outside = true;
    }
    return h[0];
  }
}

// ------------------------------------------------------------ recursion with tape
// The moment recursion of ``recursion`` keeping what its reverse needs: the
// normalised coefficient vectors c^n (C) and the unnormalised d^n (Dv).
template <int KP>
struct RecTape {
  double C[KP + 1][KP + 2];
  double Dv[KP][KP + 2];
};

template <int KP>
__device__ inline void recursion_taped(const double* mu, Rec& r, RecTape<KP>& tp) {
  double c[KP + 2], cp[KP + 2], d[KP + 2];
  for (int j = 0; j < KP + 2; j++) c[j] = cp[j] = 0.0;
  c[0] = 1.0;
  r.b[0] = 0.0;
  r.nlev = KP;
  r.trunc = false;
  for (int q = 0; q <= KP; q++)
    for (int j = 0; j < KP + 2; j++) tp.C[q][j] = 0.0;
  tp.C[0][0] = 1.0;
  const double width = fmax(mu[2] - mu[1] * mu[1], 0.0);
  for (int n = 0; n < KP; n++) {
    double an = 0.0;
    for (int j = 0; j <= n; j++)
      for (int l = 0; l <= n; l++) an += c[j] * c[l] * mu[j + l + 1];
    r.a[n] = an;
    for (int j = 0; j < KP + 2; j++) d[j] = 0.0;
    for (int j = 0; j <= n + 1; j++) d[j] = (j >= 1 ? c[j - 1] : 0.0) - an * c[j] - r.b[n] * cp[j];
    for (int j = 0; j < KP + 2; j++) tp.Dv[n][j] = d[j];
    double b2 = 0.0;
    for (int j = 0; j <= n + 1; j++)
      for (int l = 0; l <= n + 1; l++) b2 += d[j] * d[l] * mu[j + l];
    if (b2 <= TRUNC_REL * width) {
      r.b[n + 1] = 0.0;
      r.nlev = n + 1;
      r.trunc = true;
      for (int q = n + 1; q < KP; q++) {
        r.a[q] = 0.0;
        r.b[q + 1] = 0.0;
      }
      break;
    }
    const double bn = sqrt(b2);
    r.b[n + 1] = bn;
    for (int j = 0; j < KP + 2; j++) {
      cp[j] = c[j];
      c[j] = d[j] / bn;
      tp.C[n + 1][j] = c[j];
    }
  }
}

// ------------------------------------------------------------ reverse of the chain
// Reverse of chain -> sigma_m -> (N, P) -> L = cU U + cN N for one orbital
// (fixed E_F and onsite level E), U = b_inf P - (E - a_inf) N, for NS seeds
// (cU[q], cN[q]) at once: the forward part (generating polynomials, sigma_m,
// the sums N, P) is shared and everything after it is linear in the seed.
// The chain (ch, L levels, b^_k set for k <= Kb) has terminator (ai, bi).
// Adds the cotangents of the raw chain coefficients to abar[q][k] (k < L)
// and bbar[q][k] (1 <= k <= min(Kb, L)) and of the terminator to
// abar_inf[q], bbar_inf[q]; dE[q] = dL/dE.  zs: sigma_m [ne+1][M]; zb[q]:
// its cotangent for seed q, [ne+1][M] each.
template <int KP, int NS>
__device__ inline void chain_reverse_ns(const Chain& ch, int L, int Kb, double ai, double bi, double E, double ef,
                                        const double* __restrict__ g, const double* __restrict__ inv, int ne, int M,
                                        int o, const double* cU, const double* cN, double* zs, double* const* zb,
                                        double (*abar)[KPMAX + 1], double (*bbar)[KPMAX + 2], double* abar_inf,
                                        double* bbar_inf, double* dE, bool f32 = false) {
  constexpr int NP = 2 * KP + 1;
  // ---- generating polynomials D_0 .. D_{L+1}, all kept
  double Dk[KP + 2][NP];
  for (int k = 0; k < KP + 2; k++)
    for (int j = 0; j < NP; j++) Dk[k][j] = 0.0;
  Dk[L + 1][0] = 1.0;
  Dk[L][0] = 1.0;
  for (int k = L - 1; k >= 0; k--) {
    const double a2 = 2.0 * ch.ah[k], bb = 4.0 * ch.bh[k + 1] * ch.bh[k + 1];
    for (int j = 0; j < NP; j++) {
      double v = Dk[k + 1][j];
      if (j >= 1) v -= a2 * Dk[k + 1][j - 1];
      if (j >= 2) v += Dk[k + 1][j - 2] - bb * Dk[k + 2][j - 2];
      Dk[k][j] = v;
    }
  }
  // ---- sigma_m and the sums N, P, dN/deps, dP/deps (with f32 the two
  // recurrences over m, forward and reverse, in FP32 as in sigma_series; the
  // sums and the chi_m stay FP64)
  if (f32) {
    float qf[NP], hf[NP - 1];
#pragma unroll
    for (int j = 0; j < NP; j++) qf[j] = (float)Dk[0][j];
#pragma unroll
    for (int j = 0; j < NP - 1; j++) hf[j] = 0.f;
    for (int m = 0; m <= ne; m++) {
      float v = m < NP ? (float)Dk[1][m] : 0.f;
#pragma unroll
      for (int j = 1; j < NP; j++) v -= qf[j] * hf[j - 1];
#pragma unroll
      for (int j = NP - 2; j >= 1; j--) hf[j] = hf[j - 1];
      hf[0] = v;
      reinterpret_cast<float*>(zs)[(size_t)m * M + o] = v;  // FP32 scratch with f32
    }
  } else {
    double h[NP - 1];
    for (int j = 0; j < NP - 1; j++) h[j] = 0.0;
    for (int m = 0; m <= ne; m++) {
      double v = m < NP ? Dk[1][m] : 0.0;
#pragma unroll
      for (int j = 1; j < NP; j++) v -= Dk[0][j] * h[j - 1];
#pragma unroll
      for (int j = NP - 2; j >= 1; j--) h[j] = h[j - 1];
      h[0] = v;
      zs[(size_t)m * M + o] = v;
    }
  }
  const double xr = (ef - ai) / (2.0 * bi);
  const bool inside = xr > -1.0 && xr < 1.0;
  const double x = clamp1(xr);
  const double phi = acos(x), s1 = sqrt(fmax(0.0, 1.0 - x * x));
  double Nbar[NS], Pbar[NS];
#pragma unroll
  for (int q = 0; q < NS; q++) {
    Nbar[q] = cN[q] - cU[q] * (E - ai);
    Pbar[q] = cU[q] * bi;
  }
  double Nv = 0.0, Pv = 0.0, dN = 0.0, dP = 0.0;
  if (f32) {
    // the same sums in FP32 (sigma_m and its cotangent in FP32 scratch): the
    // sines s_j = sin(j phi) = sinpi(j phi/pi) directly (no recurrence, so no
    // growth near the band edges), chi_j carried from step to step
    const float* zsf = reinterpret_cast<const float*>(zs);
    float* zbf[NS];
    float Nbf[NS], Pbf[NS];
#pragma unroll
    for (int q = 0; q < NS; q++) {
      zbf[q] = reinterpret_cast<float*>(zb[q]);
      Nbf[q] = (float)Nbar[q];
      Pbf[q] = (float)Pbar[q];
    }
    const float theta = (float)(phi / PI), phim = (float)(phi - PI);
    constexpr float INV_PI_F = 0.318309886183790672f;
    auto chi = [&](int j, float sjm1, float sjp1) -> float {
      if (j == 0) return 0.f;
      const float lo = (j == 1) ? phim : __fdividef(sjm1, (float)(j - 1));  // s~_{j-1}
      return (__fdividef(sjp1, (float)(j + 1)) - lo) * INV_PI_F;
    };
    float s0 = 0.f, sp1 = sinpif(theta), sp2 = sinpif(2.f * theta), sp3 = sinpif(3.f * theta);
    float c_m = 0.f, c_m1 = chi(1, s0, sp2);
    float Nf = 0.f, Pf = 0.f, dNf = 0.f, dPf = 0.f;
    for (int m = 0; m <= ne; m++) {
      const float c_m2 = chi(m + 2, sp1, sp3);
      const float gm = (float)g[m];
      const float gsm = gm * zsf[(size_t)m * M + o];
      Nf += gsm * c_m1;
      Pf += gsm * (c_m2 + c_m);
      dNf += gsm * sp1;
      dPf += gsm * (sp2 + s0);
#pragma unroll
      for (int q = 0; q < NS; q++) zbf[q][(size_t)m * M + o] = gm * (Nbf[q] * c_m1 + Pbf[q] * (c_m2 + c_m));
      c_m = c_m1;
      c_m1 = c_m2;
      s0 = sp1;
      sp1 = sp2;
      sp2 = sp3;
      sp3 = sinpif((float)(m + 4) * theta);
    }
    Nv = Nf;
    Pv = Pf;
    dN = dNf * (2.0 / PI);
    dP = dPf * (2.0 / PI);
  } else {
    // sines s_j = sin(j phi) by the recurrence; chi_j = (s~_{j+1} - s~_{j-1})/pi,
    // s~_k = sin(k phi)/k, s~_0 = phi - pi
    double s0 = 0.0, sp1 = s1, sp2 = 2.0 * x * s1, sp3 = 2.0 * x * sp2 - s1;  // s_m..s_{m+3}
    // chi_j needs s_{j-1} and s_{j+1}; each step forms chi_{m+2} only and
    // carries chi_m, chi_{m+1} over from the steps before
    constexpr double INV_PI = 1.0 / PI;
    auto chi = [&](int j, double sjm1, double sjp1) -> double {
      if (j == 0) return 0.0;
      const double lo = (j == 1) ? (phi - PI) : sjm1 * inv[j - 1];  // s~_{j-1}
      return (sjp1 * inv[j + 1] - lo) * INV_PI;
    };
    double c_m = 0.0, c_m1 = chi(1, s0, sp2);
    for (int m = 0; m <= ne; m++) {
      const double c_m2 = chi(m + 2, sp1, sp3);
      const double gsm = g[m] * zs[(size_t)m * M + o];
      Nv += gsm * c_m1;
      Pv += gsm * (c_m2 + c_m);
      dN += gsm * sp1;
      dP += gsm * (sp2 + s0);
#pragma unroll
      for (int q = 0; q < NS; q++) zb[q][(size_t)m * M + o] = g[m] * (Nbar[q] * c_m1 + Pbar[q] * (c_m2 + c_m));
      c_m = c_m1;
      c_m1 = c_m2;
      s0 = sp1;
      sp1 = sp2;
      sp2 = sp3;
      sp3 = 2.0 * x * sp2 - sp1;
    }
    dN *= 2.0 / PI;
    dP *= 2.0 / PI;
  }
#pragma unroll
  for (int q = 0; q < NS; q++) {
    abar_inf[q] += cU[q] * Nv;
    bbar_inf[q] += cU[q] * Pv;
    if (inside) {
      const double ebar = Nbar[q] * dN + Pbar[q] * dP;
      abar_inf[q] += -ebar / (2.0 * bi);
      bbar_inf[q] += -ebar * xr / bi;
    }
    dE[q] = -cU[q] * Nv;
  }
  // ---- reverse of the recurrence: lambda_m, Pb = dL/d[D_1], Qb = dL/d[D_0]
  double Pb[NS][NP], Qb[NS][NP];
  for (int q = 0; q < NS; q++)
    for (int j = 0; j < NP; j++) Pb[q][j] = Qb[q][j] = 0.0;
  if (f32) {
    float qf[NP];
#pragma unroll
    for (int j = 0; j < NP; j++) qf[j] = (float)Dk[0][j];
    float lf[NS][NP - 1], qb[NS][NP], sw[NP - 1];
    const float* zsf = reinterpret_cast<const float*>(zs);
#pragma unroll
    for (int j = 0; j < NP - 1; j++) {
#pragma unroll
      for (int q = 0; q < NS; q++) lf[q][j] = 0.f;
      const int mm = ne - 1 - j;
      sw[j] = mm >= 0 ? zsf[(size_t)mm * M + o] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < NS; q++)
#pragma unroll
      for (int j = 0; j < NP; j++) qb[q][j] = 0.f;
    for (int m = ne; m >= 0; m--) {
#pragma unroll
      for (int q = 0; q < NS; q++) {
        float lam = reinterpret_cast<const float*>(zb[q])[(size_t)m * M + o];
#pragma unroll
        for (int j = 1; j < NP; j++) lam -= qf[j] * lf[q][j - 1];
        if (m < NP) Pb[q][m] += (double)lam;
#pragma unroll
        for (int j = 1; j < NP; j++) qb[q][j] -= lam * sw[j - 1];
#pragma unroll
        for (int j = NP - 2; j >= 1; j--) lf[q][j] = lf[q][j - 1];
        lf[q][0] = lam;
      }
#pragma unroll
      for (int j = 0; j < NP - 2; j++) sw[j] = sw[j + 1];
      const int mm = m - NP;
      sw[NP - 2] = mm >= 0 ? zsf[(size_t)mm * M + o] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < NS; q++)
#pragma unroll
      for (int j = 1; j < NP; j++) Qb[q][j] = (double)qb[q][j];
  } else {
    double lf[NS][NP - 1];  // lf[q][j] = lambda_{m+1+j}
    double sw[NP - 1];      // sw[j] = sigma_{m-1-j}
    for (int j = 0; j < NP - 1; j++) {
#pragma unroll
      for (int q = 0; q < NS; q++) lf[q][j] = 0.0;
      const int mm = ne - 1 - j;
      sw[j] = mm >= 0 ? zs[(size_t)mm * M + o] : 0.0;
    }
    for (int m = ne; m >= 0; m--) {
#pragma unroll
      for (int q = 0; q < NS; q++) {
        double lam = zb[q][(size_t)m * M + o];
#pragma unroll
        for (int j = 1; j < NP; j++) lam -= Dk[0][j] * lf[q][j - 1];
        if (m < NP) Pb[q][m] += lam;
#pragma unroll
        for (int j = 1; j < NP; j++) Qb[q][j] -= lam * sw[j - 1];
#pragma unroll
        for (int j = NP - 2; j >= 1; j--) lf[q][j] = lf[q][j - 1];
        lf[q][0] = lam;
      }
#pragma unroll
      for (int j = 0; j < NP - 2; j++) sw[j] = sw[j + 1];
      const int mm = m - NP;  // sigma_{m-1-(NP-2)} for the next step
      sw[NP - 2] = mm >= 0 ? zs[(size_t)mm * M + o] : 0.0;
    }
  }
  // ---- reverse of the polynomial recursion -> a^bar, b^bar; chain parameters
  for (int q = 0; q < NS; q++) {
    double ahb[KP + 1], bhb[KP + 2];
    for (int k = 0; k <= KP; k++) ahb[k] = 0.0;
    for (int k = 0; k <= KP + 1; k++) bhb[k] = 0.0;
    {
      double Db[KP + 2][NP];
      for (int k = 0; k < KP + 2; k++)
        for (int j = 0; j < NP; j++) Db[k][j] = 0.0;
      for (int j = 0; j < NP; j++) {
        Db[0][j] = Qb[q][j];
        Db[1][j] = Pb[q][j];
      }
      for (int k = 0; k < L; k++) {
        const double a2 = 2.0 * ch.ah[k], bb = 4.0 * ch.bh[k + 1] * ch.bh[k + 1];
        double ga = 0.0, gb = 0.0;
        for (int j = 0; j < NP; j++) {
          const double gg = Db[k][j];
          Db[k + 1][j] += gg;
          if (j >= 1) {
            Db[k + 1][j - 1] -= a2 * gg;
            ga -= 2.0 * gg * Dk[k + 1][j - 1];
          }
          if (j >= 2) {
            Db[k + 1][j - 2] += gg;
            Db[k + 2][j - 2] -= bb * gg;
            gb -= 8.0 * ch.bh[k + 1] * gg * Dk[k + 2][j - 2];
          }
        }
        ahb[k] += ga;
        bhb[k + 1] += gb;
      }
    }
    // chain parameters a^_k = (a_k - a_inf)/(2 b_inf), b^_k = b_k/(2 b_inf)
    for (int k = 0; k < L; k++) {
      abar[q][k] += ahb[k] / (2.0 * bi);
      abar_inf[q] += -ahb[k] / (2.0 * bi);
      bbar_inf[q] += -ahb[k] * ch.ah[k] / bi;
    }
    for (int k = 1; k <= Kb; k++)
      if (k <= L) {
        bbar[q][k] += bhb[k] / (2.0 * bi);
        bbar_inf[q] += -bhb[k] * ch.bh[k] / bi;
      }
  }
}

// One seed (cU, cN); returns dL/dE.
template <int KP>
__device__ inline double chain_reverse(const Chain& ch, int L, int Kb, double ai, double bi, double E, double ef,
                                       const double* __restrict__ g, const double* __restrict__ inv, int ne,
                                       int M, int o, double cU, double cN, double* zs, double* zb, double* abar,
                                       double* bbar, double& abar_inf, double& bbar_inf, bool f32 = false) {
  double* zbs[1] = {zb};
  double ab[1][KPMAX + 1], bb_[1][KPMAX + 2];
  for (int k = 0; k <= KPMAX; k++) ab[0][k] = abar[k];
  for (int k = 0; k <= KPMAX + 1; k++) bb_[0][k] = bbar[k];
  double ai_[1] = {abar_inf}, bi_[1] = {bbar_inf}, dE[1];
  chain_reverse_ns<KP, 1>(ch, L, Kb, ai, bi, E, ef, g, inv, ne, M, o, &cU, &cN, zs, zbs, ab, bb_, ai_, bi_, dE, f32);
  for (int k = 0; k <= KPMAX; k++) abar[k] = ab[0][k];
  for (int k = 0; k <= KPMAX + 1; k++) bbar[k] = bb_[0][k];
  abar_inf = ai_[0];
  bbar_inf = bi_[0];
  return dE[0];
}

// Reverse of Gershgorin: a_inf = (top+bot)/2, b_inf = (top-bot)/4 with
// top = a_ihi + b_ihi + b_ihi+1, bot = a_ilo - b_ilo - b_ilo+1 (no
// b_inf cotangent where the floor is active).
__device__ inline void gershgorin_reverse(const Term& t, double abar_inf, double bbar_inf, double* abar,
                                          double* bbar) {
  const double topb = 0.5 * abar_inf + (t.floored ? 0.0 : 0.25 * bbar_inf);
  const double botb = 0.5 * abar_inf - (t.floored ? 0.0 : 0.25 * bbar_inf);
  abar[t.ihi] += topb;
  bbar[t.ihi] += topb;
  bbar[t.ihi + 1] += topb;
  abar[t.ilo] += botb;
  bbar[t.ilo] -= botb;
  bbar[t.ilo + 1] -= botb;
}

// Reverse of bandwidth(): adds the cotangents of a_inf, b_inf onto those of
// the computed a_n, b_n (nothing through a floored B or the global mode).
__device__ inline void bandwidth_reverse(const Rec& r, const Term& t, const BandSel& p, double abar_inf,
                                         double bbar_inf, double* abar, double* bbar) {
  const int L = r.nlev;
  const double Bb = t.floored ? 0.0 : bbar_inf;
  switch (p.mode) {
    case BOP_BW_GERSHGORIN:
      gershgorin_reverse(t, abar_inf, bbar_inf, abar, bbar);
      return;
    case BOP_BW_LOWEST:
      abar[0] += abar_inf;
      bbar[1] += Bb;
      return;
    case BOP_BW_HIGHEST:
      abar[L - 1] += abar_inf;
      bbar[L] += Bb;
      return;
    case BOP_BW_AVERAGE:
    case BOP_BW_AVG_CENTRE:
      for (int n = 0; n < L; n++) abar[n] += abar_inf / L;
      if (p.mode == BOP_BW_AVG_CENTRE) {
        bbar[L] += Bb;
      } else if (Bb != 0.0) {  // B = sqrt(sum b^2 / L) >= the floor here
        for (int n = 1; n <= L; n++) bbar[n] += Bb * r.b[n] / (L * t.bsum);
      }
      return;
    case BOP_BW_MINMAX:
      abar[t.ihi] += 0.5 * abar_inf + 0.25 * Bb;
      abar[t.ilo] += 0.5 * abar_inf - 0.25 * Bb;
      bbar[t.ib] += Bb;
      return;
    case BOP_BW_GLOBAL:
      return;
    default:  // BOP_BW_WEIGHTED
      for (int m = 0; m < L; m++) abar[m] += abar_inf / ((p.beta * (L - 1 - m) + 1.0) * t.bsum);
      for (int m = 1; m <= L; m++) bbar[m] += Bb / ((p.beta * (L - m) + 1.0) * t.wsum_b);
  }
}

// Reverse of the moment recursion: adds d/dmu of (abar . a + bbar . b) to mub.
template <int KP>
__device__ inline void recursion_reverse(const double* mu, const Rec& r, const RecTape<KP>& tp, double* abar,
                                         double* bbar, double* mub) {
  const int L = r.nlev;
  double cb[KP + 1][KP + 2];
  for (int q = 0; q <= KP; q++)
    for (int j = 0; j < KP + 2; j++) cb[q][j] = 0.0;
  for (int n = L - 1; n >= 0; n--) {
    double db[KP + 2];
    for (int j = 0; j < KP + 2; j++) db[j] = 0.0;
    const bool made_next = !(r.trunc && n == L - 1);
    if (made_next) {
      const double bn = r.b[n + 1];
      double dotc = 0.0;
      for (int j = 0; j <= n + 1; j++) {
        db[j] = cb[n + 1][j] / bn;
        dotc += cb[n + 1][j] * tp.Dv[n][j];
      }
      const double bnb = bbar[n + 1] - dotc / (bn * bn);
      const double b2b = bnb / (2.0 * bn);
      for (int j = 0; j <= n + 1; j++) {
        double acc = 0.0;
        for (int l = 0; l <= n + 1; l++) {
          acc += mu[j + l] * tp.Dv[n][l];
          mub[j + l] += b2b * tp.Dv[n][j] * tp.Dv[n][l];
        }
        db[j] += 2.0 * b2b * acc;
      }
    }
    double an_b = abar[n];
    for (int j = 0; j <= n + 1; j++) {
      if (j >= 1) cb[n][j - 1] += db[j];
      cb[n][j] += -r.a[n] * db[j];
      an_b += -db[j] * tp.C[n][j];
      if (n >= 1) {
        bbar[n] += -db[j] * tp.C[n - 1][j];
        cb[n - 1][j] += -r.b[n] * db[j];
      }
    }
    for (int j = 0; j <= n; j++) {
      double acc = 0.0;
      for (int l = 0; l <= n; l++) {
        acc += mu[j + l + 1] * tp.C[n][l];
        mub[j + l + 1] += an_b * tp.C[n][j] * tp.C[n][l];
      }
      cb[n][j] += 2.0 * an_b * acc;
    }
  }
}

}  // namespace scal
