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
#include <cooperative_groups.h>

#include "chain_common.cuh"

using namespace scal;

namespace {

constexpr int CT = 32;  // threads per block: one orbital per thread, small blocks so that
                         // a few thousand orbitals still spread over all SMs (FP64-bound)

// Fewer orbitals than one warp per SM sub-partition: the FP64 kernels then
// give each orbital two lanes (the Fermi sums, the two seeds of the response
// weights) so that every sub-partition's FP64 unit has work; with more
// orbitals one lane per orbital avoids duplicating the per-orbital setup.
int few_orbitals(int M) {
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cap = (sms > 0 ? sms : 1) * 4 * 32;
  }
  return M < cap;
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
  Term t = bandwidth(r, A.bw);
  Chain ch;
  chain_params(r, t, KP, ch);
  for (int k = 0; k < KP; k++) A.a[(size_t)o * KP + k] = r.a[k];
  for (int k = 0; k <= KP; k++) A.b[(size_t)o * (KP + 1) + k] = r.b[k];
  A.nlev[o] = r.nlev;
  A.a_inf[o] = t.a_inf;
  A.b_inf[o] = t.b_inf;
  double Q[NP], P[NP];
  gen_polys<KP>(ch, r.nlev, Q, P);
  bool outside = false;
  double last;
  if (A.sig32)
    last = A.n_unbounded ? sigma_series<KP, true, true>(Q, P, ne, A.g, A.gsig, M, o, &outside)
                         : sigma_series<KP, false, true>(Q, P, ne, A.g, A.gsig, M, o);
  else
    last = A.n_unbounded ? sigma_series<KP, true>(Q, P, ne, A.g, A.gsig, M, o, &outside)
                         : sigma_series<KP, false>(Q, P, ne, A.g, A.gsig, M, o);
  if (outside) atomicAdd(A.n_unbounded, 1u);
  if (!isfinite(t.a_inf) || !isfinite(t.b_inf) || !isfinite(last)) raise_error(A.status, BOP_DEV_ERR_NONFINITE);
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

// count_and_dos in FP32 on an FP32 copy of the coefficients: only for the
// starting point of the FP64 Newton search (its sums carry errors of ~1e-6
// of the electron count, far above the FP64 tolerance).
__device__ __forceinline__ void count_and_dos_f32(const float* __restrict__ gs32, int M, int o, int ne, float x,
                                                  float* N, float* dNde) {
  auto G = [&](int j) -> float { return (j >= 0 && j <= ne) ? gs32[(size_t)j * M + o] : 0.f; };
  const float phi = acosf(x), s = sqrtf(fmaxf(0.f, 1.f - x * x));
  const float x2 = 2.f * x;
  float b1 = 0.f, b2 = 0.f, c1 = 0.f, c2 = 0.f;
  for (int k = ne + 2; k >= 1; k--) {
    const float b0 = (G(k - 2) - G(k)) / (float)k + x2 * b1 - b2;
    b2 = b1;
    b1 = b0;
    const float c0 = G(k - 1) + x2 * c1 - c2;
    c2 = c1;
    c1 = c0;
  }
  const float pi = 3.14159265358979f;
  *N = G(0) * (1.f - phi / pi) + s * b1 / pi;
  *dNde = (2.f / pi) * s * c1;
}

// The same sums by a pair of adjacent lanes (par = lane & 1): with
// sin(k phi) = s U_{k-1}(x), each sum over U_j splits into its even and odd
// terms, which obey U_{j+2} = y U_j - U_{j-2} with y = 4x^2 - 2; lane 0 runs
// the even Clenshaw chains (U_0 = 1, U_2 - y U_0 = 1), lane 1 the odd ones
// (U_1 = 2x, U_3 - y U_1 = 0), exchanged at the end.  An orbital's FP64
// work thus runs on two lanes (twice the warps for the same orbitals;
// measured faster than one lane and than four lanes per orbital when there
// are fewer orbitals than one warp per SM sub-partition).
// pm: the pair's lane mask.  Both lanes return N and dNde.
__device__ __forceinline__ void count_and_dos2(const double* __restrict__ gsig, const double* __restrict__ inv,
                                               int M, int o, int ne, double x, int par, unsigned pm, double* N,
                                               double* dNde) {
  auto G = [&](int j) -> double { return (j >= 0 && j <= ne) ? gsig[(size_t)j * M + o] : 0.0; };
  const double y = 4.0 * x * x - 2.0;
  // lane par sums the terms U_j with j = 2i + par:
  //   S_par = sum_i a_{j+1} U_j, a_k = (gs_{k-2} - gs_k)/k;  C_par = sum_i gs_j U_j
  double b1 = 0.0, b2 = 0.0, c1 = 0.0, c2 = 0.0;
  const int top = (ne + 2) / 2;
  double gp = G(2 * top + par + 1);  // gs_{j+1}
  for (int i = top; i >= 0; i--) {
    const int j = 2 * i + par;
    const double gm = G(j - 1), g0 = G(j);
    const double a = (gm - gp) * inv[j + 1];
    const double b0 = a + y * b1 - b2;
    const double c0 = g0 + y * c1 - c2;
    b2 = b1;
    b1 = b0;
    c2 = c1;
    c1 = c0;
    gp = gm;
  }
  // even: U_0 = 1, U_2 - y U_0 = 1;  odd: U_1 = 2x, U_3 - y U_1 = 0
  const double Sp = par == 0 ? b1 + b2 : 2.0 * x * b1;
  const double Cp = par == 0 ? c1 + c2 : 2.0 * x * c1;
  const double S = Sp + __shfl_xor_sync(pm, Sp, 1);
  const double C = Cp + __shfl_xor_sync(pm, Cp, 1);
  const double phi = acos(x), s = sqrt(fmax(0.0, 1.0 - x * x));
  *N = G(0) * (1.0 - phi / PI) + s * S / PI;
  *dNde = (2.0 / PI) * s * C;
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

// Pieces of a Fermi-level solve whose sums span several processes (a
// spatial domain per rank): mode 0 writes out = {-min(a_inf - 2 b_inf),
// max(a_inf + 2 b_inf)} over the orbitals, mode 1 writes out = {sum_o N_o(E),
// sum_o n_o(E)} (the DOS per energy, as k_fermi_newton), both for this
// process's orbitals; the caller reduces them over the processes.
__global__ void __launch_bounds__(RT2) k_fermi_eval(int mode, int M, int ne, const double* __restrict__ gsig,
                                                    const double* __restrict__ inv, const double* __restrict__ a_inf,
                                                    const double* __restrict__ b_inf, double E, double* partials,
                                                    unsigned* counter, double* out) {
  __shared__ double sh[RT2 / 32];
  __shared__ bool last;
  double v0 = mode == 0 ? -1e300 : 0.0, v1 = mode == 0 ? -1e300 : 0.0;
  for (int o = blockIdx.x * RT2 + threadIdx.x; o < M; o += gridDim.x * RT2) {
    const double ai = a_inf[o], bi = b_inf[o];
    if (mode == 0) {
      v0 = fmax(v0, -(ai - 2.0 * bi));
      v1 = fmax(v1, ai + 2.0 * bi);
    } else {
      const double xr = (E - ai) / (2.0 * bi);
      double N, dN;
      count_and_dos(gsig, inv, M, o, ne, clamp1(xr), &N, &dN);
      v0 += N;
      if (xr > -1.0 && xr < 1.0) v1 += dN / (2.0 * bi);
    }
  }
  double b0, b1;
  if (mode == 0) {
    __shared__ double smx[2][RT2];
    smx[0][threadIdx.x] = v0;
    smx[1][threadIdx.x] = v1;
    __syncthreads();
    for (int w = RT2 / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        smx[0][threadIdx.x] = fmax(smx[0][threadIdx.x], smx[0][threadIdx.x + w]);
        smx[1][threadIdx.x] = fmax(smx[1][threadIdx.x], smx[1][threadIdx.x + w]);
      }
      __syncthreads();
    }
    b0 = smx[0][0];
    b1 = smx[1][0];
  } else {
    b0 = block_sum<RT2>(v0, sh);
    b1 = block_sum<RT2>(v1, sh);
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = b0;
    partials[2 * blockIdx.x + 1] = b1;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __shared__ double fr[RT2 / 32 + 1];
  const double t0 = final_reduce<RT2>(partials, 2, 0, gridDim.x, mode == 0, fr);
  const double t1 = final_reduce<RT2>(partials, 2, 1, gridDim.x, mode == 0, fr);
  if (threadIdx.x == 0) {
    out[0] = t0;
    out[1] = t1;
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


// The whole Fermi-level solve in one cooperative launch: the bracket, the
// safeguarded Newton rounds of k_fermi_newton (same update rules) until
// convergence or max_rounds, then N and the DOS of every orbital at E_F.
// Per round every block writes its partial sums, the grid synchronises once,
// and every block reduces all partials in the same fixed order, so all
// blocks take the same decision without a second synchronisation.  The
// partial buffers alternate between rounds (a block can only overwrite a
// buffer after every block has passed the next grid barrier).
// Threads per block of the cooperative solve: 64 for few orbitals (more
// blocks), 256 for many (the sums walk each orbital's coefficients one cache
// line per term, so the rounds wait on memory unless many warps are resident).
constexpr int FC_SMALL = 64, FC_LARGE = 256;

template <int FC>
__device__ __forceinline__ double coop_block_reduce(double v, double* sh, bool take_max) {
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = take_max ? fmax(v, w) : v + w;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = sh[0];
  for (int w = 1; w < FC / 32; w++) t = take_max ? fmax(t, sh[w]) : t + sh[w];
  return t;  // every thread
}

// Rounds evaluate N and the DOS of every orbital at the current iterate and
// store them; the stored values are those of the last iterate E, within
// tol of E_F (the SCF residual uses them; the energy is evaluated at E_F).
template <int FC>
__global__ void __launch_bounds__(FC) k_fermi_coop(int M, const double* __restrict__ gsig,
                                                   const double* __restrict__ inv, const double* __restrict__ a_inf,
                                                   const double* __restrict__ b_inf, int ne, double sfac,
                                                   double target, FermiState* st, double* part, int warm,
                                                   int max_rounds, double tol, double* __restrict__ Nout,
                                                   double* __restrict__ dos, int lanes,
                                                   const float* __restrict__ gs32) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  __shared__ double sh[FC / 32 + 1];
  __shared__ double fr[FC / 32 + 1];
  const int nb = gridDim.x, b = blockIdx.x;
  const int stride = nb * FC;
  // bracket [min(a - 2b) - 1e-3, max(a + 2b) + 1e-3]
  double mn = 1e300, mx = -1e300;
  for (int o = b * FC + threadIdx.x; o < M; o += stride) {
    mn = fmin(mn, a_inf[o] - 2.0 * b_inf[o]);
    mx = fmax(mx, a_inf[o] + 2.0 * b_inf[o]);
  }
  mn = coop_block_reduce<FC>(-mn, sh, true);
  mx = coop_block_reduce<FC>(mx, sh, true);
  if (threadIdx.x == 0) {
    part[2 * b] = mn;
    part[2 * b + 1] = mx;
  }
  grid.sync();
  double lo = -final_reduce<FC>(part, 2, 0, nb, true, fr) - 1e-3;
  double hi = final_reduce<FC>(part, 2, 1, nb, true, fr) + 1e-3;
  const double prev = st->ef;
  double E = (warm && prev > lo && prev < hi) ? prev : 0.5 * (lo + hi);
  if (gs32 != nullptr && !(warm && prev > lo && prev < hi)) {
    // cold start: safeguarded Newton rounds on FP32 sums (their own bracket,
    // which the FP64 rounds below do not inherit) give the starting point
    double l32 = lo, h32 = hi;
    for (int r = 0; r < 16; r++) {
      double aN = 0.0, aD = 0.0;
      for (int o = b * FC + threadIdx.x; o < M; o += stride) {
        const float bi = (float)b_inf[o];
        const float xr = (float)((E - a_inf[o]) / (2.0 * b_inf[o]));
        float Nv, dN;
        count_and_dos_f32(gs32, M, o, ne, fminf(1.f, fmaxf(-1.f, xr)), &Nv, &dN);
        aN += Nv;
        if (xr > -1.f && xr < 1.f) aD += dN / (2.f * bi);
      }
      aN = coop_block_reduce<FC>(aN, sh, false);
      aD = coop_block_reduce<FC>(aD, sh, false);
      double* pr = part + (size_t)((r + 1) & 1) * 2 * nb;
      if (threadIdx.x == 0) {
        pr[2 * b] = aN;
        pr[2 * b + 1] = aD;
      }
      grid.sync();
      const double f = sfac * final_reduce<FC>(pr, 2, 0, nb, false, fr) - target;
      const double fp = sfac * final_reduce<FC>(pr, 2, 1, nb, false, fr);
      if (f < 0.0) l32 = E; else h32 = E;
      double xn = fp > 0.0 ? E - f / fp : l32 - 1.0;
      if (!(xn > l32 && xn < h32)) xn = 0.5 * (l32 + h32);
      const double step = fabs(xn - E);
      E = xn;
      if (step < 1e-5 || h32 - l32 < 1e-5) break;
    }
    if (!(E > lo && E < hi)) E = 0.5 * (lo + hi);
    grid.sync();  // every block has read the last FP32 partials before they are reused
  }
  double ef = E;
  int iters = 0;
  bool done = hi - lo < tol;
  if (done) ef = 0.5 * (lo + hi);
  bool evaluated = false;
  // lanes (1 or 2) per orbital: thread t takes orbital t / lanes; with two,
  // the pair shares the sums (count_and_dos2)
  const int sh_l = lanes == 2 ? 1 : 0;
  const int par = lanes == 2 ? (threadIdx.x & 1) : 0;
  const unsigned pm = 3u << ((threadIdx.x & 31) & ~1);
  for (int r = 0; !done && r < max_rounds; r++) {
    double aN = 0.0, aD = 0.0;
    for (int t = b * FC + threadIdx.x; (t >> sh_l) < M; t += stride) {
      const int o = t >> sh_l;
      const double bi = b_inf[o];
      const double xr = (E - a_inf[o]) / (2.0 * bi);
      double Nv, dN;
      if (sh_l) count_and_dos2(gsig, inv, M, o, ne, clamp1(xr), par, pm, &Nv, &dN);
      else count_and_dos(gsig, inv, M, o, ne, clamp1(xr), &Nv, &dN);
      const double d = (xr > -1.0 && xr < 1.0) ? dN / (2.0 * bi) : 0.0;
      if (par == 0) {
        aN += Nv;
        aD += d;
        Nout[o] = Nv;
        dos[o] = d;
      }
    }
    evaluated = true;
    aN = coop_block_reduce<FC>(aN, sh, false);
    aD = coop_block_reduce<FC>(aD, sh, false);
    double* pr = part + (size_t)((r + 1) & 1) * 2 * nb;
    if (threadIdx.x == 0) {
      pr[2 * b] = aN;
      pr[2 * b + 1] = aD;
    }
    grid.sync();
    const double tN = final_reduce<FC>(pr, 2, 0, nb, false, fr);
    const double tD = final_reduce<FC>(pr, 2, 1, nb, false, fr);
    const double f = sfac * tN - target, fp = sfac * tD;
    iters++;
    if (f == 0.0) {
      ef = E;
      done = true;
    } else {
      if (f < 0.0) lo = E; else hi = E;
      double xn = fp > 0.0 ? E - f / fp : lo - 1.0;
      if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
      if (fabs(xn - E) < tol || hi - lo < tol || iters >= max_rounds) {
        ef = xn;
        done = true;
      } else {
        E = xn;
      }
    }
  }
  if (b == 0 && threadIdx.x == 0) {
    st->lo = lo;
    st->hi = hi;
    st->mid = E;
    st->ef = ef;
    st->iters = iters;
    st->done = done ? 1 : 0;
  }
  if (!evaluated) {  // bracket narrower than tol: N and DOS at its midpoint
    for (int t = b * FC + threadIdx.x; (t >> sh_l) < M; t += stride) {
      const int o = t >> sh_l;
      const double bi = b_inf[o];
      const double xr = (ef - a_inf[o]) / (2.0 * bi);
      double Nv, dN;
      if (sh_l) count_and_dos2(gsig, inv, M, o, ne, clamp1(xr), par, pm, &Nv, &dN);
      else count_and_dos(gsig, inv, M, o, ne, clamp1(xr), &Nv, &dN);
      if (par == 0) {
        Nout[o] = Nv;
        dos[o] = (xr > -1.0 && xr < 1.0) ? dN / (2.0 * bi) : 0.0;
      }
    }
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
  const int M = A.M, nm = 2 * KP + 1;
  const double cU = A.cU;
  const double cN = A.var_q ? cU * (A.var_J * A.var_q[o / A.norb] - A.var_lam[0])
                            : (A.lam ? -A.cU * A.lam[0] : A.cN0);
  double mu[BOP_MAX_NMOM];
  for (int n = 0; n < nm; n++) mu[n] = A.mu[(size_t)o * nm + n];
  Rec r;
  RecTape<KP> tp;
  recursion_taped<KP>(mu, r, tp);
  const Term t = bandwidth(r, A.bw);
  Chain ch;
  chain_params(r, t, KP, ch);
  double abar[KPMAX + 1], bbar[KPMAX + 2];
  for (int k = 0; k <= KPMAX; k++) abar[k] = 0.0;
  for (int k = 0; k <= KPMAX + 1; k++) bbar[k] = 0.0;
  double abar_inf = 0.0, bbar_inf = 0.0;
  const double dE = chain_reverse<KP>(ch, r.nlev, KP, t.a_inf, t.b_inf, A.onsite[o], A.st->ef, A.g, A.inv, A.n_exp,
                                      M, o, cU, cN, A.zscratch, A.zscratch + (size_t)(A.n_exp + 1) * M, abar, bbar,
                                      abar_inf, bbar_inf, A.sig32 != 0);
  if (A.dU_dE) A.dU_dE[o] = dE;
  bandwidth_reverse(r, t, A.bw, abar_inf, bbar_inf, abar, bbar);
  double mub[BOP_MAX_NMOM];
  for (int n = 0; n < nm; n++) mub[n] = 0.0;
  recursion_reverse<KP>(mu, r, tp, abar, bbar, mub);
  bool bad = false;
  for (int n = 0; n < nm; n++) {
    A.w[(size_t)o * nm + n] = mub[n];
    bad |= !isfinite(mub[n]);
  }
  if (bad) raise_error(A.status, BOP_DEV_ERR_NONFINITE);
}

// Two weight sets at once, w1 for (cU1, cN1) and w2 for (cU2, cN2), both
// at fixed E_F (no E_F multiplier): the SCF-response solve needs dU/dmu and
// dN/dmu.  The forward part of the chain runs once.  zscratch holds sigma_m
// and the two cotangents ([3][n_exp+1][M]).
template <int KP>
__global__ void __launch_bounds__(CT) k_weights_pair(WeightArgs A, double cU1, double cN1, double cU2, double cN2,
                                                     double* __restrict__ w2) {
  const int o = blockIdx.x * CT + threadIdx.x;
  if (o >= A.M) return;
  const int M = A.M, nm = 2 * KP + 1;
  double mu[BOP_MAX_NMOM];
  for (int n = 0; n < nm; n++) mu[n] = A.mu[(size_t)o * nm + n];
  Rec r;
  RecTape<KP> tp;
  recursion_taped<KP>(mu, r, tp);
  const Term t = bandwidth(r, A.bw);
  Chain ch;
  chain_params(r, t, KP, ch);
  double abar[2][KPMAX + 1], bbar[2][KPMAX + 2];
  for (int q = 0; q < 2; q++) {
    for (int k = 0; k <= KPMAX; k++) abar[q][k] = 0.0;
    for (int k = 0; k <= KPMAX + 1; k++) bbar[q][k] = 0.0;
  }
  double abar_inf[2] = {0.0, 0.0}, bbar_inf[2] = {0.0, 0.0}, dE[2];
  const double cU[2] = {cU1, cU2}, cN[2] = {cN1, cN2};
  const size_t zl = (size_t)(A.n_exp + 1) * M;
  double* zb[2] = {A.zscratch + zl, A.zscratch + 2 * zl};
  chain_reverse_ns<KP, 2>(ch, r.nlev, KP, t.a_inf, t.b_inf, A.onsite[o], A.st->ef, A.g, A.inv, A.n_exp, M, o, cU,
                          cN, A.zscratch, zb, abar, bbar, abar_inf, bbar_inf, dE, A.sig32 != 0);
  if (A.dU_dE) A.dU_dE[o] = dE[0];
  bool bad = false;
  for (int q = 0; q < 2; q++) {
    bandwidth_reverse(r, t, A.bw, abar_inf[q], bbar_inf[q], abar[q], bbar[q]);
    double mub[BOP_MAX_NMOM];
    for (int n = 0; n < nm; n++) mub[n] = 0.0;
    recursion_reverse<KP>(mu, r, tp, abar[q], bbar[q], mub);
    double* w = q == 0 ? A.w : w2;
    for (int n = 0; n < nm; n++) {
      w[(size_t)o * nm + n] = mub[n];
      bad |= !isfinite(mub[n]);
    }
  }
  if (bad) raise_error(A.status, BOP_DEV_ERR_NONFINITE);
}

// Two weight sets, w1 for (cU1, cN1) and w2 for (cU2, cN2), both at fixed
// E_F, on two lanes per orbital (t = 2 o + q, q the seed): each lane runs the
// forward part of the chain and the reverse for its own seed, so that the
// FP64 work spreads over twice the warps.  zscratch: [4][n_exp+1][M] (sigma
// and its cotangent per seed).
template <int KP>
__global__ void __launch_bounds__(CT) k_weights_split(WeightArgs A, double cU1, double cN1, double cU2, double cN2,
                                                      double* __restrict__ w2) {
  const int t = blockIdx.x * CT + threadIdx.x;
  const int o = t >> 1, q = t & 1;
  if (o >= A.M) return;
  const int M = A.M, nm = 2 * KP + 1;
  const double cU = q ? cU2 : cU1, cN = q ? cN2 : cN1;
  double mu[BOP_MAX_NMOM];
  for (int n = 0; n < nm; n++) mu[n] = A.mu[(size_t)o * nm + n];
  Rec r;
  RecTape<KP> tp;
  recursion_taped<KP>(mu, r, tp);
  const Term tm = bandwidth(r, A.bw);
  Chain ch;
  chain_params(r, tm, KP, ch);
  double abar[KPMAX + 1], bbar[KPMAX + 2];
  for (int k = 0; k <= KPMAX; k++) abar[k] = 0.0;
  for (int k = 0; k <= KPMAX + 1; k++) bbar[k] = 0.0;
  double abar_inf = 0.0, bbar_inf = 0.0;
  const size_t zl = (size_t)(A.n_exp + 1) * M;
  double* zs = A.zscratch + (size_t)q * 2 * zl;
  const double dE = chain_reverse<KP>(ch, r.nlev, KP, tm.a_inf, tm.b_inf, A.onsite[o], A.st->ef, A.g, A.inv,
                                      A.n_exp, M, o, cU, cN, zs, zs + zl, abar, bbar, abar_inf, bbar_inf,
                                      A.sig32 != 0);
  if (q == 0 && A.dU_dE) A.dU_dE[o] = dE;
  bandwidth_reverse(r, tm, A.bw, abar_inf, bbar_inf, abar, bbar);
  double mub[BOP_MAX_NMOM];
  for (int n = 0; n < nm; n++) mub[n] = 0.0;
  recursion_reverse<KP>(mu, r, tp, abar, bbar, mub);
  double* w = q ? w2 : A.w;
  bool bad = false;
  for (int n = 0; n < nm; n++) {
    w[(size_t)o * nm + n] = mub[n];
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

int launch_weights_pair(const WeightArgs& a, double cU1, double cN1, double cU2, double cN2, double* w2,
                        cudaStream_t s) {
  const int Kp = (a.n_mom - 1) / 2;
  if (!few_orbitals(a.M)) {  // enough warps already: one lane, one forward pass for both seeds
    const int g = (a.M + CT - 1) / CT;
    switch (Kp) {
      case 1: k_weights_pair<1><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
      case 2: k_weights_pair<2><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
      case 3: k_weights_pair<3><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
      case 4: k_weights_pair<4><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
      case 5: k_weights_pair<5><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
      case 6: k_weights_pair<6><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
      case 7: k_weights_pair<7><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
      case 8: k_weights_pair<8><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
      default: return -1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
  }
  const int g = (2 * a.M + CT - 1) / CT;
  switch (Kp) {
    case 1: k_weights_split<1><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
    case 2: k_weights_split<2><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
    case 3: k_weights_split<3><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
    case 4: k_weights_split<4><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
    case 5: k_weights_split<5><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
    case 6: k_weights_split<6><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
    case 7: k_weights_split<7><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
    case 8: k_weights_split<8><<<g, CT, 0, s>>>(a, cU1, cN1, cU2, cN2, w2); break;
    default: return -1;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_fermi_eval(int mode, int M, const double* gsig, const double* inv, const double* a_inf,
                      const double* b_inf, int n_exp, double E, double* partials, unsigned* counter, double* out,
                      cudaStream_t s) {
  k_fermi_eval<<<red_grid2(M), RT2, 0, s>>>(mode, M, n_exp, gsig, inv, a_inf, b_inf, E, partials, counter, out);
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

template <int FC>
int fermi_coop_grid() {
  static int g = 0;
  if (g == 0) {
    int dev = 0, sms = 0, per = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fermi_coop<FC>, FC, 0);
    g = coop && per > 0 ? sms * (per < 4 ? per : 4) : -1;
  }
  return g;
}

int launch_fermi_coop(int M, const double* gsig, const double* inv, const double* a_inf, const double* b_inf,
                      int n_exp, double spin_factor, double target, FermiState* st, double* partials, int warm,
                      int max_rounds, double tol, double* N, double* dos, cudaStream_t s, const float* gs32) {
  const bool few = few_orbitals(M);
  const int fc = few ? FC_SMALL : FC_LARGE;
  const int gmax = few ? fermi_coop_grid<FC_SMALL>() : fermi_coop_grid<FC_LARGE>();
  if (gmax <= 0) return -2;
  int lanes = few ? 2 : 1;
  int g = (lanes * M + fc - 1) / fc;
  if (g > gmax) g = gmax;
  if (g < 1) g = 1;
  void* args[] = {&M, &gsig, &inv, &a_inf, &b_inf, &n_exp, &spin_factor, &target, &st, &partials, &warm,
                  &max_rounds, &tol, &N, &dos, &lanes, &gs32};
  const void* fn = few ? (const void*)k_fermi_coop<FC_SMALL> : (const void*)k_fermi_coop<FC_LARGE>;
  if (cudaLaunchCooperativeKernel(fn, g, fc, args, 0, s) != cudaSuccess) return -1;
  return 0;
}

__global__ void k_to_f32(long long n, const double* __restrict__ in, float* __restrict__ out) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    out[q] = (float)in[q];
}

int launch_gsig_f32(int M, int n_exp, const double* gsig, float* gs32, cudaStream_t s) {
  const long long n = (long long)M * (n_exp + 1);
  const long long g = (n + 255) / 256;
  k_to_f32<<<(int)(g < 65536 ? g : 65536), 256, 0, s>>>(n, gsig, gs32);
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
