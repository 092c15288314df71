// Expansion coefficients sigma_m of the local DOS (Eq. sigma_i, Eq. aexp)
// through the generating function of the Chebyshev chain, the Fermi level
// (Newton steps inside the bisection bracket), the electron count / bond
// energy / DOS of every orbital (Eq. chi, Eq. Fermi-phase) and the weights
// dU/dmu (Eq. weights) by reverse-mode differentiation, in FP64.
//
// Generating function.  The paper obtains sigma_m = zeta_0^(m) from the
// semi-infinite chain recursion zeta^(m+1) = 2 h zeta^(m) - zeta^(m-1),
// i.e. sigma_m = [U_m(h)]_00 with the normalised chain matrix h (a^_k,
// b^_k on the computed levels, a^ = 0 and b^ = 1/2 in the constant
// terminator).  Since sum_m U_m(x) t^m = 1 / (1 - 2 x t + t^2),
//     sum_m sigma_m t^m = [(1 - 2 t h + t^2)^{-1}]_00 = D_1(t) / D_0(t),
// where D_{L+1} = D_L = 1 and, down the L computed levels,
//     D_k(t) = (1 - 2 a^_k t + t^2) D_{k+1}(t) - 4 b^_{k+1}^2 t^2 D_{k+2}(t)
// (the terminator tail contributes the factor 2t of a free chain, which
// the recursion absorbs).  D_0(0) = 1, so the sigma_m follow from the
// linear recurrence  sigma_m = [D_1]_m - sum_{j>=1} [D_0]_j sigma_{m-j}:
// 2L multiply-adds per coefficient instead of a sweep over the chain.  The
// numbers are the same as the chain's (the tests compare with the oracle,
// which runs the chain as printed).
#include "scalar_common.cuh"

using namespace scal;

namespace {

constexpr int CT = 32;  // threads per block: one orbital per thread, small blocks so that
                         // a few thousand orbitals still spread over all SMs (FP64-bound)

// polynomial coefficients D_0 (Q) and D_1 (P) of the generating function
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

// moments -> (a, b, a_inf, b_inf) -> g_m sigma_m, m = 0..n_exp, stored
// coefficient-major gsig[m][M].
template <int KP>
__global__ void __launch_bounds__(CT) k_expand(ScalarArgs A) {
  const int o = blockIdx.x * CT + threadIdx.x;
  if (o >= A.M) return;
  constexpr int NP = 2 * KP + 1;
  const int M = A.M, ne = A.n_exp, nm = 2 * KP + 1;
  double mu[BOP_MAX_NMOM];
  for (int n = 0; n < nm; n++) mu[n] = A.mu[(size_t)o * nm + n];
  Rec r;
  recursion(mu, KP, r);
  Term t = gershgorin(r);
  Chain ch;
  chain_params(r, t, KP, ch);
  for (int k = 0; k < KP; k++) A.a[(size_t)o * KP + k] = r.a[k];
  for (int k = 0; k <= KP; k++) A.b[(size_t)o * (KP + 1) + k] = r.b[k];
  A.nlev[o] = r.nlev;
  A.a_inf[o] = t.a_inf;
  A.b_inf[o] = t.b_inf;
  double Q[NP], P[NP];
  gen_polys<KP>(ch, r.nlev, Q, P);
  double h[NP - 1];  // h[j] = sigma_{m-1-j}
#pragma unroll
  for (int j = 0; j < NP - 1; j++) h[j] = 0.0;
  double last = 0.0;
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
    last = A.g[m] * v;
    A.gsig[(size_t)m * M + o] = last;
  }
  if (!isfinite(t.a_inf) || !isfinite(t.b_inf) || !isfinite(h[0])) raise_error(A.status, BOP_DEV_ERR_NONFINITE);
}

// Sums over the sine series of one orbital at x = cos(phi) (Clenshaw):
//   N    = gs_0 (1 - phi/pi) + sum_k (gs_{k-2} - gs_k)/(pi k) sin(k phi)
//   dNde = (2/pi) sum_m gs_m sin((m+1) phi)            (= dN/d eps)
// gs_j = 0 outside 0..ne; inv[k] = 1/k.
__device__ __forceinline__ void count_and_dos(const double* __restrict__ gsig, const double* __restrict__ inv,
                                              int M, int o, int ne, double x, double* N, double* dNde) {
  auto G = [&](int j) -> double { return (j >= 0 && j <= ne) ? gsig[(size_t)j * M + o] : 0.0; };
  const double phi = acos(x), s = sqrt(fmax(0.0, 1.0 - x * x));
  const double x2 = 2.0 * x;
  double b1 = 0.0, b2 = 0.0, c1 = 0.0, c2 = 0.0;
  for (int k = ne + 2; k >= 1; k--) {  // coefficient of U_{k-1}
    const double b0 = (G(k - 2) - G(k)) * inv[k] + x2 * b1 - b2;
    b2 = b1;
    b1 = b0;
    const double c0 = G(k - 1) + x2 * c1 - c2;
    c2 = c1;
    c1 = c0;
  }
  *N = G(0) * (1.0 - phi / PI) + s * b1 / PI;
  *dNde = (2.0 / PI) * s * c1;
}

constexpr int RT2 = 32;  // threads per block of the per-orbital FP64 kernels (see CT)

// Bracket [min(a_inf - 2 b_inf) - 1e-3, max(a_inf + 2 b_inf) + 1e-3]; the
// first iterate is the previous Fermi level when warm and inside, else the
// midpoint.
__global__ void __launch_bounds__(RT2) k_bracket_warm(int M, const double* __restrict__ a_inf,
                                                      const double* __restrict__ b_inf, FermiState* st,
                                                      double* partials, unsigned* counter, double tol, int warm) {
  __shared__ double smn[RT2], smx[RT2];
  __shared__ bool last;
  double mn = 1e300, mx = -1e300;
  for (int o = blockIdx.x * RT2 + threadIdx.x; o < M; o += gridDim.x * RT2) {
    mn = fmin(mn, a_inf[o] - 2.0 * b_inf[o]);
    mx = fmax(mx, a_inf[o] + 2.0 * b_inf[o]);
  }
  smn[threadIdx.x] = mn;
  smx[threadIdx.x] = mx;
  __syncthreads();
  for (int w = RT2 / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + w]);
      smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = -smn[0];  // negated: both halves reduce with max
    partials[2 * blockIdx.x + 1] = smx[0];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __shared__ double fr[RT2 / 32 + 1];
  double lo = -final_reduce<RT2>(partials, 2, 0, gridDim.x, true, fr);  // stored as -min below
  double hi = final_reduce<RT2>(partials, 2, 1, gridDim.x, true, fr);
  if (threadIdx.x == 0) {
    lo -= 1e-3;
    hi += 1e-3;
    const double prev = st->ef;
    st->lo = lo;
    st->hi = hi;
    st->mid = (warm && prev > lo && prev < hi) ? prev : 0.5 * (lo + hi);
    st->iters = 0;
    st->done = (hi - lo < tol) ? 1 : 0;
    if (st->done) st->ef = 0.5 * (lo + hi);
    *counter = 0;
  }
}

// One safeguarded Newton step on f(E) = s sum_o N_o(E) - target: the sign of
// f shrinks the bracket as in bisection; the next iterate is E - f/f' when it
// falls strictly inside the bracket, else the bracket midpoint.  Converged
// when the step or the bracket is below tol, or f = 0.
__global__ void __launch_bounds__(RT2) k_fermi_newton(int M, const double* __restrict__ gsig,
                                                      const double* __restrict__ inv, const double* __restrict__ a_inf,
                                                      const double* __restrict__ b_inf, int ne, double sfac,
                                                      double target, FermiState* st, double* partials,
                                                      unsigned* counter, int max_rounds, double tol) {
  __shared__ double sh[RT2 / 32];
  __shared__ bool last;
  if (*(volatile int*)&st->done) return;
  const double E = st->mid;
  double aN = 0.0, aD = 0.0;
  for (int o = blockIdx.x * RT2 + threadIdx.x; o < M; o += gridDim.x * RT2) {
    const double bi = b_inf[o];
    const double xr = (E - a_inf[o]) / (2.0 * bi);
    double N, dN;
    count_and_dos(gsig, inv, M, o, ne, clamp1(xr), &N, &dN);
    aN += N;
    if (xr > -1.0 && xr < 1.0) aD += dN / (2.0 * bi);
  }
  const double bN = block_sum<RT2>(aN, sh);
  const double bD = block_sum<RT2>(aD, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = bN;
    partials[2 * blockIdx.x + 1] = bD;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __shared__ double fr[RT2 / 32 + 1];
  const double tN = final_reduce<RT2>(partials, 2, 0, gridDim.x, false, fr);
  const double tD = final_reduce<RT2>(partials, 2, 1, gridDim.x, false, fr);
  if (threadIdx.x == 0) {
    const double f = sfac * tN - target, fp = sfac * tD;
    st->iters += 1;
    if (f == 0.0) {
      st->ef = E;
      st->done = 1;
    } else {
      if (f < 0.0) st->lo = E; else st->hi = E;
      double xn = fp > 0.0 ? E - f / fp : st->lo - 1.0;
      if (!(xn > st->lo && xn < st->hi)) xn = 0.5 * (st->lo + st->hi);
      if (fabs(xn - E) < tol || st->hi - st->lo < tol || st->iters >= max_rounds) {
        st->ef = xn;
        st->done = 1;
      } else {
        st->mid = xn;
      }
    }
    *counter = 0;
  }
}

// N and DOS (per energy) of every orbital at E_F.
__global__ void __launch_bounds__(RT2) k_orbital_N(int M, int ne, const double* __restrict__ gsig,
                                                   const double* __restrict__ inv, const double* __restrict__ a_inf,
                                                   const double* __restrict__ b_inf, const FermiState* st,
                                                   double* __restrict__ N, double* __restrict__ dos) {
  const int o = blockIdx.x * RT2 + threadIdx.x;
  if (o >= M) return;
  const double bi = b_inf[o];
  const double xr = (st->ef - a_inf[o]) / (2.0 * bi);
  double n, d;
  count_and_dos(gsig, inv, M, o, ne, clamp1(xr), &n, &d);
  N[o] = n;
  dos[o] = (xr > -1.0 && xr < 1.0) ? d / (2.0 * bi) : 0.0;
}

// Bond energy U = b_inf P - (E_ialpha - a_inf) N with
//   P = sum_m gs_m (chi_{m+2} + chi_m)
//     = (1/pi)[-gs_1 (phi - pi) - (gs_0 + gs_2) sin(phi)
//              + sum_{k>=2} (gs_{k-3} - gs_{k+1}) sin(k phi)/k],
// together with N and the DOS.
__global__ void __launch_bounds__(RT2) k_orbital_NU2(int M, int ne, const double* __restrict__ gsig,
                                                     const double* __restrict__ inv,
                                                     const double* __restrict__ a_inf,
                                                     const double* __restrict__ b_inf,
                                                     const double* __restrict__ onsite, const FermiState* st,
                                                     double* __restrict__ N, double* __restrict__ U,
                                                     double* __restrict__ dos) {
  const int o = blockIdx.x * RT2 + threadIdx.x;
  if (o >= M) return;
  const double ai = a_inf[o], bi = b_inf[o];
  const double xr = (st->ef - ai) / (2.0 * bi);
  const double x = clamp1(xr);
  double n, d;
  count_and_dos(gsig, inv, M, o, ne, x, &n, &d);
  auto G = [&](int j) -> double { return (j >= 0 && j <= ne) ? gsig[(size_t)j * M + o] : 0.0; };
  const double phi = acos(x), s = sqrt(fmax(0.0, 1.0 - x * x)), x2 = 2.0 * x;
  double b1 = 0.0, b2 = 0.0;
  for (int k = ne + 3; k >= 2; k--) {  // sum_{k>=2} e_k sin(k phi) = s sum e_k U_{k-1}
    const double e = (G(k - 3) - G(k + 1)) * inv[k];
    const double b0 = e + x2 * b1 - b2;
    b2 = b1;
    b1 = b0;
  }
  // b1 now holds sum_{k>=2} e_k U_{k-1} minus the k = 1 step: finish with e_1
  const double e1 = -(G(0) + G(2));
  const double b0 = e1 + x2 * b1 - b2;
  const double Pv = (-G(1) * (phi - PI) + s * b0) / PI;
  N[o] = n;
  U[o] = bi * Pv - (onsite[o] - ai) * n;
  dos[o] = (xr > -1.0 && xr < 1.0) ? d / (2.0 * bi) : 0.0;
}

// sum over orbitals of dU/dE_F and dN/dE_F -> lam = sum dU / sum dN (the
// response of E_F at fixed electron count).
__global__ void __launch_bounds__(RT2) k_ef_response2(int M, int ne, const double* __restrict__ gsig,
                                                      const double* __restrict__ inv,
                                                      const double* __restrict__ a_inf,
                                                      const double* __restrict__ b_inf,
                                                      const double* __restrict__ onsite, const FermiState* st,
                                                      double* partials, unsigned* counter, double* lam) {
  __shared__ double sh[RT2 / 32];
  __shared__ bool last;
  double aU = 0.0, aN = 0.0;
  for (int o = blockIdx.x * RT2 + threadIdx.x; o < M; o += gridDim.x * RT2) {
    const double ai = a_inf[o], bi = b_inf[o];
    const double xr = (st->ef - ai) / (2.0 * bi);
    if (!(xr > -1.0 && xr < 1.0)) continue;
    // dN/deps = (2/pi) sum gs_m sin((m+1) phi), dP/deps = (2/pi) sum gs_m (sin((m+2) phi) + sin(m phi))
    const double x2 = 2.0 * xr, s = sqrt(1.0 - xr * xr);
    double c1 = 0.0, c2 = 0.0, p1 = 0.0, p2 = 0.0;
    auto G = [&](int j) -> double { return (j >= 0 && j <= ne) ? gsig[(size_t)j * M + o] : 0.0; };
    for (int k = ne + 2; k >= 1; k--) {  // coefficients of sin(k phi): g_{k-1} (N), g_{k-2} + g_k (P)
      const double c0 = G(k - 1) + x2 * c1 - c2;
      c2 = c1;
      c1 = c0;
      const double q0 = (G(k - 2) + G(k)) + x2 * p1 - p2;
      p2 = p1;
      p1 = q0;
    }
    const double dN = (2.0 / PI) * s * c1, dP = (2.0 / PI) * s * p1;
    const double dU = bi * dP - (onsite[o] - ai) * dN;
    aU += dU / (2.0 * bi);
    aN += dN / (2.0 * bi);
  }
  const double bU = block_sum<RT2>(aU, sh);
  const double bN = block_sum<RT2>(aN, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = bU;
    partials[2 * blockIdx.x + 1] = bN;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __shared__ double fr[RT2 / 32 + 1];
  const double tU = final_reduce<RT2>(partials, 2, 0, gridDim.x, false, fr);
  const double tN = final_reduce<RT2>(partials, 2, 1, gridDim.x, false, fr);
  if (threadIdx.x == 0) {
    lam[0] = tN > 0.0 ? tU / tN : 0.0;
    lam[1] = tU;
    lam[2] = tN;
    *counter = 0;
  }
}

__global__ void k_inverse_table(double* inv, int n) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) inv[k] = k == 0 ? 0.0 : 1.0 / (double)k;
}

// ------------------------------------------------------------ weights
// Reverse-mode derivative of L = cU U + cN N (fixed E_F and onsite level)
// with respect to the moments of one orbital.  Forward: recursion,
// Gershgorin, chain parameters, generating polynomials D_k, sigma_m (kept in
// zscratch[m][M]), N, P and their derivatives.  Reverse: sbar_m, the
// recurrence adjoint lambda_m = sbar_m - sum_j [D_0]_j lambda_{m+j}, then
// the polynomial recursion, the chain parameters, Gershgorin and the
// moment recursion.
template <int KP>
__global__ void __launch_bounds__(CT) k_weights(WeightArgs A) {
  const int o = blockIdx.x * CT + threadIdx.x;
  if (o >= A.M) return;
  constexpr int NP = 2 * KP + 1;
  const int M = A.M, ne = A.n_exp, nm = 2 * KP + 1;
  const double cU = A.cU, cN = -A.cU * A.lam[0];
  double mu[BOP_MAX_NMOM];
  for (int n = 0; n < nm; n++) mu[n] = A.mu[(size_t)o * nm + n];

  // ---- recursion, storing what the reverse needs
  double C[KP + 1][KP + 2], Dv[KP][KP + 2];
  Rec r;
  {
    double c[KP + 2], cp[KP + 2], d[KP + 2];
    for (int j = 0; j < KP + 2; j++) c[j] = cp[j] = 0.0;
    c[0] = 1.0;
    r.b[0] = 0.0;
    r.nlev = KP;
    r.trunc = false;
    for (int q = 0; q <= KP; q++)
      for (int j = 0; j < KP + 2; j++) C[q][j] = 0.0;
    C[0][0] = 1.0;
    const double width = fmax(mu[2] - mu[1] * mu[1], 0.0);
    for (int n = 0; n < KP; n++) {
      double an = 0.0;
      for (int j = 0; j <= n; j++)
        for (int l = 0; l <= n; l++) an += c[j] * c[l] * mu[j + l + 1];
      r.a[n] = an;
      for (int j = 0; j < KP + 2; j++) d[j] = 0.0;
      for (int j = 0; j <= n + 1; j++) d[j] = (j >= 1 ? c[j - 1] : 0.0) - an * c[j] - r.b[n] * cp[j];
      for (int j = 0; j < KP + 2; j++) Dv[n][j] = d[j];
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
        C[n + 1][j] = c[j];
      }
    }
  }
  const Term t = gershgorin(r);
  Chain ch;
  chain_params(r, t, KP, ch);
  const double ai = t.a_inf, bi = t.b_inf;
  const int L = r.nlev;

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
  // ---- sigma_m (zs[m][M]) and the sums N, P, dN/deps, dP/deps
  double* zs = A.zscratch;                          // sigma_m
  double* zb = A.zscratch + (size_t)(ne + 1) * M;   // sbar_m
  {
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
  const double E = A.onsite[o];
  const double xr = (A.st->ef - ai) / (2.0 * bi);
  const bool inside = xr > -1.0 && xr < 1.0;
  const double x = clamp1(xr);
  const double phi = acos(x), s1 = sqrt(fmax(0.0, 1.0 - x * x));
  const double Nbar = cN - cU * (E - ai), Pbar = cU * bi;
  double Nv = 0.0, Pv = 0.0, dN = 0.0, dP = 0.0;
  {
    // sines s_j = sin(j phi) by the recurrence; chi_j = (s~_{j+1} - s~_{j-1})/pi,
    // s~_k = sin(k phi)/k, s~_0 = phi - pi
    const double* inv = A.inv;
    double sm1 = 0.0, s0 = 0.0, sp1 = s1, sp2 = 2.0 * x * s1, sp3 = 2.0 * x * sp2 - s1;  // s_{m-1}..s_{m+3}
    auto chi = [&](int j, double sjm1, double sjp1) -> double {
      if (j == 0) return 0.0;
      const double lo = (j == 1) ? (phi - PI) : sjm1 * inv[j - 1];  // s~_{j-1}
      return (sjp1 * inv[j + 1] - lo) / PI;
    };
    for (int m = 0; m <= ne; m++) {
      const double c_m = chi(m, sm1, sp1), c_m1 = chi(m + 1, s0, sp2), c_m2 = chi(m + 2, sp1, sp3);
      const double gsm = A.g[m] * zs[(size_t)m * M + o];
      Nv += gsm * c_m1;
      Pv += gsm * (c_m2 + c_m);
      dN += gsm * sp1;
      dP += gsm * (sp2 + s0);
      zb[(size_t)m * M + o] = A.g[m] * (Nbar * c_m1 + Pbar * (c_m2 + c_m));
      sm1 = s0;
      s0 = sp1;
      sp1 = sp2;
      sp2 = sp3;
      sp3 = 2.0 * x * sp2 - sp1;
    }
    dN *= 2.0 / PI;
    dP *= 2.0 / PI;
  }
  double abar_inf = cU * Nv, bbar_inf = cU * Pv;
  if (inside) {
    const double ebar = Nbar * dN + Pbar * dP;
    abar_inf += -ebar / (2.0 * bi);
    bbar_inf += -ebar * xr / bi;
  }
  if (A.dU_dE) A.dU_dE[o] = -cU * Nv;

  // ---- reverse of the recurrence: lambda_m, Pbar = dL/d[D_1], Qbar = dL/d[D_0]
  double Pb[NP], Qb[NP];
  for (int j = 0; j < NP; j++) Pb[j] = Qb[j] = 0.0;
  {
    double lf[NP - 1];  // lf[j] = lambda_{m+1+j}
    double sw[NP - 1];  // sw[j] = sigma_{m-1-j}
    for (int j = 0; j < NP - 1; j++) {
      lf[j] = 0.0;
      const int mm = ne - 1 - j;
      sw[j] = mm >= 0 ? zs[(size_t)mm * M + o] : 0.0;
    }
    for (int m = ne; m >= 0; m--) {
      double lam = zb[(size_t)m * M + o];
#pragma unroll
      for (int j = 1; j < NP; j++) lam -= Dk[0][j] * lf[j - 1];
      if (m < NP) Pb[m] += lam;
#pragma unroll
      for (int j = 1; j < NP; j++) Qb[j] -= lam * sw[j - 1];
#pragma unroll
      for (int j = NP - 2; j >= 1; j--) lf[j] = lf[j - 1];
      lf[0] = lam;
#pragma unroll
      for (int j = 0; j < NP - 2; j++) sw[j] = sw[j + 1];
      const int mm = m - NP;  // sigma_{m-1-(NP-2)} for the next step
      sw[NP - 2] = mm >= 0 ? zs[(size_t)mm * M + o] : 0.0;
    }
  }
  // ---- reverse of the polynomial recursion -> a^bar, b^bar
  double ahb[KP + 1], bhb[KP + 2];
  for (int k = 0; k <= KP; k++) ahb[k] = 0.0;
  for (int k = 0; k <= KP + 1; k++) bhb[k] = 0.0;
  {
    double Db[KP + 2][NP];
    for (int k = 0; k < KP + 2; k++)
      for (int j = 0; j < NP; j++) Db[k][j] = 0.0;
    for (int j = 0; j < NP; j++) {
      Db[0][j] = Qb[j];
      Db[1][j] = Pb[j];
    }
    for (int k = 0; k < L; k++) {
      const double a2 = 2.0 * ch.ah[k], bb = 4.0 * ch.bh[k + 1] * ch.bh[k + 1];
      double ga = 0.0, gb = 0.0;
      for (int j = 0; j < NP; j++) {
        const double g = Db[k][j];
        Db[k + 1][j] += g;
        if (j >= 1) {
          Db[k + 1][j - 1] -= a2 * g;
          ga -= 2.0 * g * Dk[k + 1][j - 1];
        }
        if (j >= 2) {
          Db[k + 1][j - 2] += g;
          Db[k + 2][j - 2] -= bb * g;
          gb -= 8.0 * ch.bh[k + 1] * g * Dk[k + 2][j - 2];
        }
      }
      ahb[k] += ga;
      bhb[k + 1] += gb;
    }
  }
  // ---- chain parameters -> (a, b, a_inf, b_inf)
  double abar[KPMAX + 1], bbar[KPMAX + 2];
  for (int k = 0; k <= KPMAX; k++) abar[k] = 0.0;
  for (int k = 0; k <= KPMAX + 1; k++) bbar[k] = 0.0;
  for (int k = 0; k < L; k++) {
    abar[k] += ahb[k] / (2.0 * bi);
    abar_inf += -ahb[k] / (2.0 * bi);
    bbar_inf += -ahb[k] * ch.ah[k] / bi;
  }
  for (int k = 1; k <= KP; k++)
    if (k <= L) {
      bbar[k] += bhb[k] / (2.0 * bi);
      bbar_inf += -bhb[k] * ch.bh[k] / bi;
    }
  {  // Gershgorin: a_inf = (top+bot)/2, b_inf = (top-bot)/4
    const double topb = 0.5 * abar_inf + (t.floored ? 0.0 : 0.25 * bbar_inf);
    const double botb = 0.5 * abar_inf - (t.floored ? 0.0 : 0.25 * bbar_inf);
    abar[t.ihi] += topb;
    bbar[t.ihi] += topb;
    bbar[t.ihi + 1] += topb;
    abar[t.ilo] += botb;
    bbar[t.ilo] -= botb;
    bbar[t.ilo + 1] -= botb;
  }
  // ---- reverse of the moment recursion
  double mub[BOP_MAX_NMOM];
  for (int n = 0; n < nm; n++) mub[n] = 0.0;
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
        dotc += cb[n + 1][j] * Dv[n][j];
      }
      const double bnb = bbar[n + 1] - dotc / (bn * bn);
      const double b2b = bnb / (2.0 * bn);
      for (int j = 0; j <= n + 1; j++) {
        double acc = 0.0;
        for (int l = 0; l <= n + 1; l++) {
          acc += mu[j + l] * Dv[n][l];
          mub[j + l] += b2b * Dv[n][j] * Dv[n][l];
        }
        db[j] += 2.0 * b2b * acc;
      }
    }
    double an_b = abar[n];
    for (int j = 0; j <= n + 1; j++) {
      if (j >= 1) cb[n][j - 1] += db[j];
      cb[n][j] += -r.a[n] * db[j];
      an_b += -db[j] * C[n][j];
      if (n >= 1) {
        bbar[n] += -db[j] * C[n - 1][j];
        cb[n - 1][j] += -r.b[n] * db[j];
      }
    }
    for (int j = 0; j <= n; j++) {
      double acc = 0.0;
      for (int l = 0; l <= n; l++) {
        acc += mu[j + l + 1] * C[n][l];
        mub[j + l + 1] += an_b * C[n][j] * C[n][l];
      }
      cb[n][j] += 2.0 * an_b * acc;
    }
  }
  bool bad = false;
  for (int n = 0; n < nm; n++) {
    A.w[(size_t)o * nm + n] = mub[n];
    bad |= !isfinite(mub[n]);
  }
  if (bad) raise_error(A.status, BOP_DEV_ERR_NONFINITE);
}

int red_grid2(int M) {
  int g = (M + RT2 - 1) / RT2;
  return g < 1 ? 1 : (g > 4096 ? 4096 : g);  // the context's partials hold 2 x 4096 values
}

}  // namespace

void launch_inverse_table(double* inv, int n, cudaStream_t s) {
  k_inverse_table<<<(n + 127) / 128, 128, 0, s>>>(inv, n);
}

int launch_expand(const ScalarArgs& a, cudaStream_t s) {
  const int g = (a.M + CT - 1) / CT, Kp = (a.n_mom - 1) / 2;
  switch (Kp) {
    case 1: k_expand<1><<<g, CT, 0, s>>>(a); break;
    case 2: k_expand<2><<<g, CT, 0, s>>>(a); break;
    case 3: k_expand<3><<<g, CT, 0, s>>>(a); break;
    case 4: k_expand<4><<<g, CT, 0, s>>>(a); break;
    case 5: k_expand<5><<<g, CT, 0, s>>>(a); break;
    case 6: k_expand<6><<<g, CT, 0, s>>>(a); break;
    case 7: k_expand<7><<<g, CT, 0, s>>>(a); break;
    case 8: k_expand<8><<<g, CT, 0, s>>>(a); break;
    default: return -1;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_weights(const WeightArgs& a, cudaStream_t s) {
  const int g = (a.M + CT - 1) / CT, Kp = (a.n_mom - 1) / 2;
  switch (Kp) {
    case 1: k_weights<1><<<g, CT, 0, s>>>(a); break;
    case 2: k_weights<2><<<g, CT, 0, s>>>(a); break;
    case 3: k_weights<3><<<g, CT, 0, s>>>(a); break;
    case 4: k_weights<4><<<g, CT, 0, s>>>(a); break;
    case 5: k_weights<5><<<g, CT, 0, s>>>(a); break;
    case 6: k_weights<6><<<g, CT, 0, s>>>(a); break;
    case 7: k_weights<7><<<g, CT, 0, s>>>(a); break;
    case 8: k_weights<8><<<g, CT, 0, s>>>(a); break;
    default: return -1;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_fermi_newton(int M, const double* gsig, const double* inv, const double* a_inf, const double* b_inf,
                        int n_exp, double spin_factor, double target, FermiState* st, double* partials,
                        unsigned* counter, int warm, int rounds, int max_rounds, double tol, cudaStream_t s) {
  const int g = red_grid2(M);
  k_bracket_warm<<<g, RT2, 0, s>>>(M, a_inf, b_inf, st, partials, counter, tol, warm);
  for (int r = 0; r < rounds; r++)
    k_fermi_newton<<<g, RT2, 0, s>>>(M, gsig, inv, a_inf, b_inf, n_exp, spin_factor, target, st, partials, counter,
                                     max_rounds, tol);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_fermi_more(int M, const double* gsig, const double* inv, const double* a_inf, const double* b_inf,
                      int n_exp, double spin_factor, double target, FermiState* st, double* partials,
                      unsigned* counter, int rounds, int max_rounds, double tol, cudaStream_t s) {
  const int g = red_grid2(M);
  for (int r = 0; r < rounds; r++)
    k_fermi_newton<<<g, RT2, 0, s>>>(M, gsig, inv, a_inf, b_inf, n_exp, spin_factor, target, st, partials, counter,
                                     max_rounds, tol);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_orbital_N(int M, int n_exp, const double* gsig, const double* inv, const double* a_inf,
                     const double* b_inf, const FermiState* st, double* N, double* dos, cudaStream_t s) {
  k_orbital_N<<<(M + RT2 - 1) / RT2, RT2, 0, s>>>(M, n_exp, gsig, inv, a_inf, b_inf, st, N, dos);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_orbital_NU(int M, int n_exp, const double* gsig, const double* inv, const double* a_inf,
                      const double* b_inf, const double* onsite, const FermiState* st, double* N, double* U,
                      double* dos, cudaStream_t s) {
  k_orbital_NU2<<<(M + RT2 - 1) / RT2, RT2, 0, s>>>(M, n_exp, gsig, inv, a_inf, b_inf, onsite, st, N, U, dos);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_ef_response(int M, int n_exp, const double* gsig, const double* inv, const double* a_inf,
                       const double* b_inf, const double* onsite, const FermiState* st, double* red,
                       unsigned* counter, double* lam, cudaStream_t s) {
  k_ef_response2<<<red_grid2(M), RT2, 0, s>>>(M, n_exp, gsig, inv, a_inf, b_inf, onsite, st, red, counter, lam);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
