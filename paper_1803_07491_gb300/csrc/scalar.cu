// FP64 scalar stages of the analytic BOP, one thread per orbital (and spin):
//   moments -> recursion coefficients (Eqs. momtoa, momtob, c_j^n recursion)
//   -> Gershgorin band edges (Eq. gershogorin) -> constant terminator
//   (Eq. abinf) -> expansion coefficients sigma_m from the semi-infinite
//   chain (Eq. aexp) -> Jackson damping (Eq. Jackson) -> electron count and
//   bond energy from the response functions (Eq. chi, Eq. Fermi-phase),
//   the Fermi level by bisection on the total electron count, the local
//   charge-neutrality / Stoner updates (Eqs. BOP_LCN, onsite_NCM) and the
//   weights w_n = dU/dmu_n (Eq. weights) by reverse-mode differentiation of
//   all of the above.
//
// Phase convention: eps = cos(phi), the band bottom at phi = pi.
#include "kernels.h"

namespace {

constexpr double PI = 3.14159265358979323846;
constexpr double B_INF_MIN = 1e-3;   // eV, floor of the band-width estimate
constexpr double TRUNC_REL = 1e-10;  // recursion truncation threshold
constexpr int ZB = 32;               // threads per block of the chain kernels
constexpr int KPMAX = (BOP_MAX_NMOM - 1) / 2;

// ------------------------------------------------------------ recursion
struct Rec {
  double a[KPMAX];
  double b[KPMAX + 1];
  int nlev;
  bool trunc;
};

// a_n = sum c_j c_l mu_{j+l+1};  b_{n+1} c^{n+1} = c^n shifted - a_n c^n - b_n c^{n-1}
__device__ void recursion(const double* mu, int Kp, Rec& r) {
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
  int ilo, ihi;
  bool floored;
};

// Gershgorin over the computed levels n < nlev (b_0 = 0); first index wins ties.
__device__ Term gershgorin(const Rec& r) {
  Term t;
  double bot = 0.0, top = 0.0;
  t.ilo = t.ihi = 0;
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

// Chain parameters: a^_k (k < nlev) and b^_k (1 <= k <= Kp, k <= nlev);
// the constant terminator a^ = 0, b^ = 1/2 elsewhere.
struct Chain {
  double ah[KPMAX + 1];
  double bh[KPMAX + 2];
};
__device__ void chain_params(const Rec& r, const Term& t, int Kp, Chain& ch) {
  for (int k = 0; k <= KPMAX; k++) ch.ah[k] = 0.0;
  for (int k = 0; k <= KPMAX + 1; k++) ch.bh[k] = 0.5;
  ch.bh[0] = 0.0;
  for (int k = 0; k < r.nlev; k++) ch.ah[k] = (r.a[k] - t.a_inf) / (2.0 * t.b_inf);
  for (int k = 1; k <= Kp; k++)
    if (k <= r.nlev) ch.bh[k] = r.b[k] / (2.0 * t.b_inf);
}
__device__ __forceinline__ double AH(const Chain& ch, int k) { return k <= KPMAX ? ch.ah[k] : 0.0; }
__device__ __forceinline__ double BH(const Chain& ch, int k) { return k <= KPMAX + 1 ? ch.bh[k] : 0.5; }

// one step of the chain recursion at level k: 2 (h z)_k - zp_k
__device__ __forceinline__ double chain_step(const Chain& ch, const double* z, const double* zp, int k) {
  double hz = AH(ch, k) * z[k * ZB] + BH(ch, k + 1) * z[(k + 1) * ZB];
  if (k >= 1) hz += BH(ch, k) * z[(k - 1) * ZB];
  return 2.0 * hz - zp[k * ZB];
}

__global__ void k_jackson(double* g, int n_exp) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > n_exp) return;
  const double N = n_exp, x = PI / (N + 1.0);
  auto gJ = [&](double mm) { return ((N - mm + 1.0) * cos(mm * x) + sin(mm * x) / tan(x)) / (N + 1.0); };
  g[m] = gJ(m + 1.0) / gJ(1.0);
}

// moments -> (a, b, a_inf, b_inf) -> g_m sigma_m (m = 0..n_exp) and the
// sine-series coefficients D_k of N(phi) = D_0 (1 - phi/pi) + sum_k D_k sin(k phi).
__global__ void __launch_bounds__(ZB) k_expand(ScalarArgs A) {
  extern __shared__ double zs[];
  const int L = A.n_exp + 3;
  const int o = blockIdx.x * ZB + threadIdx.x;
  double* z = zs + threadIdx.x;
  double* zp = zs + (size_t)L * ZB + threadIdx.x;
  for (int k = 0; k < L; k++) z[k * ZB] = zp[k * ZB] = 0.0;
  if (o >= A.M) return;
  const int Kp = (A.n_mom - 1) / 2;
  double mu[BOP_MAX_NMOM];
  for (int n = 0; n < A.n_mom; n++) mu[n] = A.mu[(size_t)o * A.n_mom + n];
  Rec r;
  recursion(mu, Kp, r);
  Term t = gershgorin(r);
  Chain ch;
  chain_params(r, t, Kp, ch);
  for (int k = 0; k < Kp; k++) A.a[(size_t)o * Kp + k] = r.a[k];
  for (int k = 0; k <= Kp; k++) A.b[(size_t)o * (Kp + 1) + k] = r.b[k];
  A.nlev[o] = r.nlev;
  A.a_inf[o] = t.a_inf;
  A.b_inf[o] = t.b_inf;
  const int M = A.M, ne = A.n_exp;
  z[0] = 1.0;
  double gs_m2 = 0.0, gs_m1 = 0.0;  // g sigma at m-2, m-1
  bool bad = !isfinite(t.a_inf) || !isfinite(t.b_inf);
  for (int m = 0; m <= ne; m++) {
    double sig = z[0];
    double gs = A.g[m] * sig;
    A.gsig[(size_t)m * M + o] = gs;
    // D_m = (gs_{m-2} - gs_m) / (pi m), D_0 = gs_0
    A.D[(size_t)m * M + o] = m == 0 ? gs : (gs_m2 - gs) / (PI * m);
    gs_m2 = gs_m1;
    gs_m1 = gs;
    if (m == ne) break;
    const int kmax = min(m + 1, ne - m - 1);
    for (int k = 0; k <= kmax; k++) zp[k * ZB] = chain_step(ch, z, zp, k);
    double* sw = z;
    z = zp;
    zp = sw;
  }
  A.D[(size_t)(ne + 1) * M + o] = gs_m2 / (PI * (ne + 1));
  A.D[(size_t)(ne + 2) * M + o] = gs_m1 / (PI * (ne + 2));
  if (bad || !isfinite(gs_m1)) raise_error(A.status, BOP_DEV_ERR_NONFINITE);
}

// N(phi) per orbital from the sine series by Clenshaw's recurrence.
__device__ __forceinline__ double count_from_D(const double* __restrict__ D, int M, int o, int ne, double x) {
  double phi = acos(x);
  double s = sqrt(fmax(0.0, 1.0 - x * x));
  double b1 = 0.0, b2 = 0.0;
  for (int j = ne + 1; j >= 0; j--) {  // sum_j D_{j+1} U_j(x)
    double b0 = D[(size_t)(j + 1) * M + o] + 2.0 * x * b1 - b2;
    b2 = b1;
    b1 = b0;
  }
  return D[o] * (1.0 - phi / PI) + s * b1;
}

__device__ __forceinline__ double clamp1(double x) { return x > 1.0 ? 1.0 : (x < -1.0 ? -1.0 : x); }

template <int NT>
__device__ double block_sum(double v, double* sh) {
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

// Bracket of the bisection: [min(a_inf - 2 b_inf) - 1e-3, max(a_inf + 2 b_inf) + 1e-3].
__global__ void __launch_bounds__(RT) k_bracket(int M, const double* __restrict__ a_inf,
                                                const double* __restrict__ b_inf, FermiState* st,
                                                double* partials, unsigned* counter, double tol) {
  __shared__ double smn[RT], smx[RT];
  __shared__ bool last;
  double mn = 1e300, mx = -1e300;
  for (int o = blockIdx.x * RT + threadIdx.x; o < M; o += gridDim.x * RT) {
    mn = fmin(mn, a_inf[o] - 2.0 * b_inf[o]);
    mx = fmax(mx, a_inf[o] + 2.0 * b_inf[o]);
  }
  smn[threadIdx.x] = mn;
  smx[threadIdx.x] = mx;
  __syncthreads();
  for (int w = RT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + w]);
      smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = smn[0];
    partials[2 * blockIdx.x + 1] = smx[0];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    volatile double* p = partials;
    double lo = 1e300, hi = -1e300;
    for (unsigned q = 0; q < gridDim.x; q++) {
      lo = fmin(lo, p[2 * q]);
      hi = fmax(hi, p[2 * q + 1]);
    }
    st->lo = lo - 1e-3;
    st->hi = hi + 1e-3;
    st->mid = 0.5 * (st->lo + st->hi);
    st->iters = 0;
    st->done = (st->hi - st->lo < tol) ? 1 : 0;
    st->ef = st->mid;
    *counter = 0;
  }
}

// One bisection step: s * sum N(mid) - target decides the half.
__global__ void __launch_bounds__(RT) k_fermi_round(int M, const double* __restrict__ D,
                                                    const double* __restrict__ a_inf,
                                                    const double* __restrict__ b_inf, int ne, double sfac,
                                                    double target, FermiState* st, double* partials,
                                                    unsigned* counter, int max_rounds, double tol) {
  __shared__ double sh[RT / 32];
  __shared__ bool last;
  if (*(volatile int*)&st->done) return;
  const double E = st->mid;
  double acc = 0.0;
  for (int o = blockIdx.x * RT + threadIdx.x; o < M; o += gridDim.x * RT) {
    double x = clamp1((E - a_inf[o]) / (2.0 * b_inf[o]));
    acc += count_from_D(D, M, o, ne, x);
  }
  double bs = block_sum<RT>(acc, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    volatile double* p = partials;
    double tot = 0.0;
    for (unsigned q = 0; q < gridDim.x; q++) tot += p[q];
    double f = sfac * tot - target;
    double mid = st->mid;
    st->iters += 1;
    if (f == 0.0) {
      st->ef = mid;
      st->done = 1;
    } else {
      if (f < 0.0) st->lo = mid; else st->hi = mid;
      if (st->hi - st->lo < tol || st->iters >= max_rounds) {
        st->ef = 0.5 * (st->lo + st->hi);
        st->done = 1;
      } else {
        st->mid = 0.5 * (st->lo + st->hi);
      }
    }
    *counter = 0;
  }
}

// chi-hat_j(phi) for j = 0 .. ne+2 on the fly: sin(k phi) by the recurrence
// s_{k+1} = 2 x s_k - s_{k-1}.
struct ChiIter {
  double x, phi, s_prev, s_cur;  // s_{k-1}, s_k
  int k;
};

// Electron count, bond energy and DOS at E_F of every orbital:
//   N = sum g_m sigma_m chi_{m+1};  U = b_inf P - (E_ialpha - a_inf) N with
//   P = sum g_m sigma_m (chi_{m+2} + chi_m);  n(E_F) = (1/(2 b_inf)) dN/deps.
__global__ void __launch_bounds__(RT) k_orbital_NU(int M, int ne, const double* __restrict__ gsig,
                                                   const double* __restrict__ a_inf,
                                                   const double* __restrict__ b_inf,
                                                   const double* __restrict__ onsite, const FermiState* st,
                                                   double* __restrict__ N, double* __restrict__ U,
                                                   double* __restrict__ dos) {
  int o = blockIdx.x * RT + threadIdx.x;
  if (o >= M) return;
  const double ai = a_inf[o], bi = b_inf[o];
  const double xr = (st->ef - ai) / (2.0 * bi);
  const double x = clamp1(xr);
  const double phi = acos(x), s1 = sqrt(fmax(0.0, 1.0 - x * x));
  // sines s_j = sin(j phi), j = 0..ne+3
  double sj[4];                         // s_{m}, s_{m+1}, s_{m+2}, s_{m+3}
  sj[0] = 0.0;
  sj[1] = s1;
  sj[2] = 2.0 * x * s1;
  sj[3] = 2.0 * x * sj[2] - s1;
  auto chi = [&](int j, double sjm1, double sjp1) -> double {
    if (j == 0) return 0.0;
    if (j == 1) return 1.0 - phi / PI + sjp1 / (2.0 * PI);
    return (sjp1 / (j + 1) - sjm1 / (j - 1)) / PI;
  };
  // chi_m needs s_{m-1}, s_{m+1}; keep s_{m-1} .. s_{m+3}
  double s_mm1 = 0.0;  // s_{-1} = -s_1, but chi_0 = 0 does not use it
  double Nv = 0.0, Pv = 0.0, dv = 0.0;
  for (int m = 0; m <= ne; m++) {
    // s_{m-1}=s_mm1, s_m=sj[0], s_{m+1}=sj[1], s_{m+2}=sj[2], s_{m+3}=sj[3]
    double c_m = chi(m, s_mm1, sj[1]);
    double c_m1 = chi(m + 1, sj[0], sj[2]);
    double c_m2 = chi(m + 2, sj[1], sj[3]);
    double gs = gsig[(size_t)m * M + o];
    Nv += gs * c_m1;
    Pv += gs * (c_m2 + c_m);
    dv += gs * sj[1];
    s_mm1 = sj[0];
    sj[0] = sj[1];
    sj[1] = sj[2];
    sj[2] = sj[3];
    sj[3] = 2.0 * x * sj[2] - sj[1];
  }
  const double E = onsite[o];
  N[o] = Nv;
  U[o] = bi * Pv - (E - ai) * Nv;
  dos[o] = (xr > -1.0 && xr < 1.0) ? (2.0 / PI) * dv / (2.0 * bi) : 0.0;
}

// dN/dE_F and dU/dE_F summed over all orbitals -> lam = sum dU / sum dN.
__global__ void __launch_bounds__(RT) k_ef_response(int M, int ne, const double* __restrict__ gsig,
                                                    const double* __restrict__ a_inf,
                                                    const double* __restrict__ b_inf,
                                                    const double* __restrict__ onsite, const FermiState* st,
                                                    double* partials, unsigned* counter, double* lam) {
  __shared__ double sh[RT / 32];
  __shared__ bool last;
  double aU = 0.0, aN = 0.0;
  for (int o = blockIdx.x * RT + threadIdx.x; o < M; o += gridDim.x * RT) {
    const double ai = a_inf[o], bi = b_inf[o];
    const double xr = (st->ef - ai) / (2.0 * bi);
    if (!(xr > -1.0 && xr < 1.0)) continue;
    const double x = xr, s1 = sqrt(1.0 - x * x);
    double dN = 0.0, dP = 0.0;
    double s_m = 0.0, s_m1 = s1, s_m2 = 2.0 * x * s1;
    for (int m = 0; m <= ne; m++) {
      double gs = gsig[(size_t)m * M + o];
      dN += gs * s_m1;
      dP += gs * (s_m2 + s_m);
      s_m = s_m1;
      s_m1 = s_m2;
      s_m2 = 2.0 * x * s_m1 - s_m;
    }
    dN *= 2.0 / PI;
    dP *= 2.0 / PI;
    const double dU = bi * dP - (onsite[o] - ai) * dN;
    aU += dU / (2.0 * bi);
    aN += dN / (2.0 * bi);
  }
  double bU = block_sum<RT>(aU, sh);
  double bN = block_sum<RT>(aN, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = bU;
    partials[2 * blockIdx.x + 1] = bN;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    volatile double* p = partials;
    double tU = 0.0, tN = 0.0;
    for (unsigned q = 0; q < gridDim.x; q++) {
      tU += p[2 * q];
      tN += p[2 * q + 1];
    }
    lam[0] = tN > 0.0 ? tU / tN : 0.0;
    lam[1] = tU;
    lam[2] = tN;
    *counter = 0;
  }
}

// ------------------------------------------------------------ weights
// Reverse-mode derivative of L = cU U + cN N (fixed E_F and onsite level)
// with respect to the moments of one orbital.  The forward chain is
// recomputed; zeta^(m)_k (k <= Kp) is kept in zscr for the reverse sweep,
// which runs the adjoint chain lambda^(m) = sbar_m e_0 + 2 h lambda^(m+1)
// - lambda^(m+2) and accumulates dL/dh.
__global__ void __launch_bounds__(ZB) k_weights(WeightArgs A) {
  extern __shared__ double zs[];
  const int L = A.n_exp + 3;
  const int o = blockIdx.x * ZB + threadIdx.x;
  double* z = zs + threadIdx.x;
  double* zp = zs + (size_t)L * ZB + threadIdx.x;
  for (int k = 0; k < L; k++) z[k * ZB] = zp[k * ZB] = 0.0;
  if (o >= A.M) return;
  const int M = A.M, ne = A.n_exp, nm = A.n_mom, Kp = (nm - 1) / 2;
  const double cU = A.cU, cN = -A.cU * A.lam[0];
  double mu[BOP_MAX_NMOM];
  for (int n = 0; n < nm; n++) mu[n] = A.mu[(size_t)o * nm + n];

  // ---- forward, keeping what the reverse needs
  double C[KPMAX + 1][KPMAX + 2], Dv[KPMAX][KPMAX + 2];
  Rec r;
  {
    double c[KPMAX + 2], cp[KPMAX + 2], d[KPMAX + 2];
    for (int j = 0; j < KPMAX + 2; j++) c[j] = cp[j] = 0.0;
    c[0] = 1.0;
    r.b[0] = 0.0;
    r.nlev = Kp;
    r.trunc = false;
    for (int q = 0; q <= KPMAX; q++)
      for (int j = 0; j < KPMAX + 2; j++) C[q][j] = 0.0;
    C[0][0] = 1.0;
    double width = fmax(mu[2] - mu[1] * mu[1], 0.0);
    for (int n = 0; n < Kp; n++) {
      double an = 0.0;
      for (int j = 0; j <= n; j++)
        for (int l = 0; l <= n; l++) an += c[j] * c[l] * mu[j + l + 1];
      r.a[n] = an;
      for (int j = 0; j < KPMAX + 2; j++) d[j] = 0.0;
      for (int j = 0; j <= n + 1; j++) d[j] = (j >= 1 ? c[j - 1] : 0.0) - an * c[j] - r.b[n] * cp[j];
      for (int j = 0; j < KPMAX + 2; j++) Dv[n][j] = d[j];
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
        break;
      }
      double bn = sqrt(b2);
      r.b[n + 1] = bn;
      for (int j = 0; j < KPMAX + 2; j++) {
        cp[j] = c[j];
        c[j] = d[j] / bn;
        C[n + 1][j] = c[j];
      }
    }
  }
  const Term t = gershgorin(r);
  Chain ch;
  chain_params(r, t, Kp, ch);
  const double ai = t.a_inf, bi = t.b_inf;
  double* zsave = A.zscratch;  // [(m*(Kp+1)+k)*M + o], then sbar at [(ne+1)*(Kp+1) + m]*M + o
  z[0] = 1.0;
  for (int m = 0; m <= ne; m++) {
    if (m < ne)
      for (int k = 0; k <= Kp; k++) zsave[((size_t)m * (Kp + 1) + k) * M + o] = z[k * ZB];
    double sig = z[0];
    zsave[((size_t)(ne + 1) * (Kp + 1) + m) * M + o] = sig;  // sigma_m, replaced by sbar_m below
    if (m == ne) break;
    const int kmax = min(m + 1, ne - m - 1 + Kp);
    for (int k = 0; k <= kmax; k++) zp[k * ZB] = chain_step(ch, z, zp, k);
    double* sw = z;
    z = zp;
    zp = sw;
  }
  // ---- N, P and their cotangents
  const double E = A.onsite[o];
  const double xr = (A.st->ef - ai) / (2.0 * bi);
  const bool inside = xr > -1.0 && xr < 1.0;
  const double x = clamp1(xr);
  const double phi = acos(x), s1 = sqrt(fmax(0.0, 1.0 - x * x));
  double Nv = 0.0, Pv = 0.0, dN = 0.0, dP = 0.0;
  {
    double s_mm1 = 0.0, sj0 = 0.0, sj1 = s1, sj2 = 2.0 * x * s1, sj3 = 2.0 * x * sj2 - s1;
    auto chi = [&](int j, double a, double b) -> double {
      if (j == 0) return 0.0;
      if (j == 1) return 1.0 - phi / PI + b / (2.0 * PI);
      return (b / (j + 1) - a / (j - 1)) / PI;
    };
    for (int m = 0; m <= ne; m++) {
      double c_m = chi(m, s_mm1, sj1), c_m1 = chi(m + 1, sj0, sj2), c_m2 = chi(m + 2, sj1, sj3);
      size_t ix = ((size_t)(ne + 1) * (Kp + 1) + m) * M + o;
      double gs = A.g[m] * zsave[ix];
      Nv += gs * c_m1;
      Pv += gs * (c_m2 + c_m);
      dN += gs * sj1;
      dP += gs * (sj2 + sj0);
      s_mm1 = sj0;
      sj0 = sj1;
      sj1 = sj2;
      sj2 = sj3;
      sj3 = 2.0 * x * sj2 - sj1;
    }
    const double Nbar = cN - cU * (E - ai), Pbar = cU * bi;
    // sbar_m = g_m (Nbar chi_{m+1} + Pbar (chi_{m+2} + chi_m))
    s_mm1 = 0.0; sj0 = 0.0; sj1 = s1; sj2 = 2.0 * x * s1; sj3 = 2.0 * x * sj2 - s1;
    for (int m = 0; m <= ne; m++) {
      double c_m = chi(m, s_mm1, sj1), c_m1 = chi(m + 1, sj0, sj2), c_m2 = chi(m + 2, sj1, sj3);
      size_t ix = ((size_t)(ne + 1) * (Kp + 1) + m) * M + o;
      zsave[ix] = A.g[m] * (Nbar * c_m1 + Pbar * (c_m2 + c_m));
      s_mm1 = sj0;
      sj0 = sj1;
      sj1 = sj2;
      sj2 = sj3;
      sj3 = 2.0 * x * sj2 - sj1;
    }
    dN *= 2.0 / PI;
    dP *= 2.0 / PI;
  }
  const double Nbar = cN - cU * (E - ai), Pbar = cU * bi;
  double abar_inf = cU * Nv, bbar_inf = cU * Pv;
  if (inside) {
    const double ebar = Nbar * dN + Pbar * dP;
    abar_inf += -ebar / (2.0 * bi);
    bbar_inf += -ebar * xr / bi;
  }
  if (A.dU_dE) A.dU_dE[o] = -cU * Nv;

  // ---- reverse of the chain: lambda in the (now free) z buffers
  for (int k = 0; k < L; k++) z[k * ZB] = zp[k * ZB] = 0.0;
  double ahb[KPMAX + 1], bhb[KPMAX + 2];
  for (int k = 0; k <= KPMAX; k++) ahb[k] = 0.0;
  for (int k = 0; k <= KPMAX + 1; k++) bhb[k] = 0.0;
  // lam holds lambda^(m+1), lamp holds lambda^(m+2)
  double* lam = z;
  double* lamp = zp;
  lam[0] = zsave[((size_t)(ne + 1) * (Kp + 1) + ne) * M + o];  // lambda^(ne) = sbar_ne e_0
  for (int m = ne - 1; m >= 0; m--) {
    // accumulate with lambda^(m+1) and zeta^(m)
    const double* zm = zsave + (size_t)m * (Kp + 1) * M + o;
    for (int k = 0; k <= Kp; k++) {
      double zk = zm[(size_t)k * M];
      ahb[k] += 2.0 * lam[k * ZB] * zk;
      if (k >= 1) {
        double zk1 = zm[(size_t)(k - 1) * M];
        bhb[k] += 2.0 * (lam[(k - 1) * ZB] * zk + lam[k * ZB] * zk1);
      }
    }
    if (m == 0) break;
    // lambda^(m) = sbar_m e_0 + 2 h lambda^(m+1) - lambda^(m+2), into lamp
    const int kmax = min(ne - m, m + Kp);
    for (int k = 0; k <= kmax; k++) lamp[k * ZB] = chain_step(ch, lam, lamp, k);
    lamp[0] += zsave[((size_t)(ne + 1) * (Kp + 1) + m) * M + o];
    double* sw = lam;
    lam = lamp;
    lamp = sw;
  }
  // ---- chain parameters -> (a, b, a_inf, b_inf)
  double abar[KPMAX + 1], bbar[KPMAX + 2];
  for (int k = 0; k <= KPMAX; k++) abar[k] = 0.0;
  for (int k = 0; k <= KPMAX + 1; k++) bbar[k] = 0.0;
  for (int k = 0; k < r.nlev; k++) {
    abar[k] += ahb[k] / (2.0 * bi);
    abar_inf += -ahb[k] / (2.0 * bi);
    bbar_inf += -ahb[k] * ch.ah[k] / bi;
  }
  for (int k = 1; k <= Kp; k++)
    if (k <= r.nlev) {
      bbar[k] += bhb[k] / (2.0 * bi);
      bbar_inf += -bhb[k] * ch.bh[k] / bi;
    }
  // ---- Gershgorin: a_inf = (top+bot)/2, b_inf = (top-bot)/4
  {
    double topb = 0.5 * abar_inf + (t.floored ? 0.0 : 0.25 * bbar_inf);
    double botb = 0.5 * abar_inf - (t.floored ? 0.0 : 0.25 * bbar_inf);
    abar[t.ihi] += topb;
    bbar[t.ihi] += topb;
    bbar[t.ihi + 1] += topb;
    abar[t.ilo] += botb;
    bbar[t.ilo] -= botb;
    bbar[t.ilo + 1] -= botb;
  }
  // ---- reverse of the recursion
  double mub[BOP_MAX_NMOM];
  for (int n = 0; n < nm; n++) mub[n] = 0.0;
  double cb[KPMAX + 1][KPMAX + 2];
  for (int q = 0; q <= KPMAX; q++)
    for (int j = 0; j < KPMAX + 2; j++) cb[q][j] = 0.0;
  const int nsteps = r.nlev;  // steps executed (the last may be the truncating one)
  for (int n = nsteps - 1; n >= 0; n--) {
    double db[KPMAX + 2];
    for (int j = 0; j < KPMAX + 2; j++) db[j] = 0.0;
    const bool made_next = !(r.trunc && n == nsteps - 1);
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
    // d_j = c_{j-1} - a_n c_j - b_n c^{n-1}_j
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
    // a_n = sum c_j c_l mu_{j+l+1}
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

// ------------------------------------------------------------ SCF
__global__ void __launch_bounds__(RT) k_scf_residual(ScfArgs A) {
  __shared__ double sh[RT / 32];
  __shared__ bool last;
  double mres = 0.0, mdm = 0.0, sd = 0.0;
  for (int i = blockIdx.x * RT + threadIdx.x; i < A.n; i += gridDim.x * RT) {
    double Ni = 0.0, di = 0.0;
    for (int v = 0; v < A.n_spin; v++)
      for (int a = 0; a < A.norb; a++) {
        size_t q = ((size_t)v * A.n + i) * A.norb + a;
        Ni += A.N[q];
        di += A.dos[q];
      }
    Ni *= A.spin_factor;
    di *= A.spin_factor;
    double res = Ni - A.n0;
    double dn = A.delta[i] + A.eta * res / fmax(di, A.dos_floor);
    A.delta_new[i] = dn;
    sd += dn;
    mres = fmax(mres, fabs(res));
    if (A.mode == 2) {
      double mo = 0.0;
      for (int a = 0; a < A.norb; a++)
        mo += A.N[(size_t)i * A.norb + a] - A.N[((size_t)A.n + i) * A.norb + a];
      mdm = fmax(mdm, fabs(mo - A.m[i]));
      A.m_new[i] = (1.0 - A.m_mix) * A.m[i] + A.m_mix * mo;
    }
  }
  // max reductions via the same shuffle tree
  for (int o = 16; o > 0; o >>= 1) {
    mres = fmax(mres, __shfl_xor_sync(0xffffffffu, mres, o));
    mdm = fmax(mdm, __shfl_xor_sync(0xffffffffu, mdm, o));
  }
  __shared__ double shm[2][RT / 32];
  if ((threadIdx.x & 31) == 0) {
    shm[0][threadIdx.x >> 5] = mres;
    shm[1][threadIdx.x >> 5] = mdm;
  }
  double bs = block_sum<RT>(sd, sh);
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < RT / 32; q++) {
      a = fmax(a, shm[0][q]);
      b = fmax(b, shm[1][q]);
    }
    A.red[3 * blockIdx.x] = a;
    A.red[3 * blockIdx.x + 1] = b;
    A.red[3 * blockIdx.x + 2] = bs;
    __threadfence();
    last = atomicAdd(A.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    volatile double* p = A.red;
    double a = 0.0, b = 0.0, s = 0.0;
    for (unsigned q = 0; q < gridDim.x; q++) {
      a = fmax(a, p[3 * q]);
      b = fmax(b, p[3 * q + 1]);
      s += p[3 * q + 2];
    }
    bool conv = a < A.tol && (A.mode != 2 || b < 10.0 * A.tol);
    A.result[0] = a;
    A.result[1] = b;
    A.result[2] = conv ? 1.0 : 0.0;
    A.result[3] = s / A.n;
    *A.counter = 0;
  }
}

__global__ void __launch_bounds__(RT) k_scf_apply(ScfArgs A) {
  if (A.result[2] != 0.0) return;
  const double mean = A.result[3];
  for (int i = blockIdx.x * RT + threadIdx.x; i < A.n; i += gridDim.x * RT) {
    A.delta[i] = A.delta_new[i] - mean;
    if (A.mode == 2) A.m[i] = A.m_new[i];
  }
}

// E_ialpha,nu = E^0 + delta_i -/+ I m_i / 2 (spin up lower).
__global__ void __launch_bounds__(RT) k_build_onsite(int n, int norb, int n_spin, double e0, double I,
                                                     const double* __restrict__ delta,
                                                     const double* __restrict__ m, double* __restrict__ on,
                                                     float* __restrict__ on32) {
  int q = blockIdx.x * RT + threadIdx.x;
  int tot = n_spin * n * norb;
  if (q >= tot) return;
  int i = (q / norb) % n, v = q / (n * norb);
  double e = e0 + (delta ? delta[i] : 0.0);
  if (m && n_spin == 2) e += (v == 0 ? -0.5 : 0.5) * I * m[i];
  on[q] = e;
  if (on32) on32[q] = (float)e;
}

__global__ void __launch_bounds__(RT) k_energy(int n, int norb, int n_spin, double sfac, double I,
                                               const double* __restrict__ U, const double* __restrict__ m,
                                               double* __restrict__ e_atom, double* red, unsigned* counter,
                                               double* e_total) {
  __shared__ double sh[RT / 32];
  __shared__ bool last;
  double acc = 0.0;
  for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT) {
    double e = 0.0;
    for (int v = 0; v < n_spin; v++)
      for (int a = 0; a < norb; a++) e += U[((size_t)v * n + i) * norb + a];
    e *= sfac;
    if (m && n_spin == 2) e -= 0.25 * I * m[i] * m[i];
    e_atom[i] = e;
    acc += e;
  }
  double bs = block_sum<RT>(acc, sh);
  if (threadIdx.x == 0) {
    red[blockIdx.x] = bs;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    volatile double* p = red;
    double s = 0.0;
    for (unsigned q = 0; q < gridDim.x; q++) s += p[q];
    *e_total = s;
    *counter = 0;
  }
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  size_t q = (size_t)blockIdx.x * RT + threadIdx.x;
  if (q < n) out[q] = (float)in[q];
}

int red_grid(int M) {
  int g = (M + RT - 1) / RT;
  return g < 1 ? 1 : (g > 1024 ? 1024 : g);
}

}  // namespace

void launch_jackson(double* g, int n_exp, cudaStream_t s) {
  k_jackson<<<(n_exp + 1 + 127) / 128, 128, 0, s>>>(g, n_exp);
}

int launch_expand(const ScalarArgs& a, cudaStream_t s) {
  size_t smem = (size_t)2 * (a.n_exp + 3) * ZB * sizeof(double);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_expand, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_expand<<<(a.M + ZB - 1) / ZB, ZB, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_fermi(int M, const double* D, const double* gsig, const double* a_inf, const double* b_inf, int n_exp,
                 double spin_factor, double target, FermiState* st, double* partials, unsigned* counter,
                 int max_rounds, double tol, cudaStream_t s) {
  (void)gsig;
  int g = red_grid(M);
  k_bracket<<<g, RT, 0, s>>>(M, a_inf, b_inf, st, partials, counter, tol);
  for (int r = 0; r < max_rounds; r++)
    k_fermi_round<<<g, RT, 0, s>>>(M, D, a_inf, b_inf, n_exp, spin_factor, target, st, partials, counter,
                                   max_rounds, tol);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_orbital_NU(int M, int n_exp, const double* gsig, const double* a_inf, const double* b_inf,
                      const double* onsite, const FermiState* st, double* N, double* U, double* dos,
                      cudaStream_t s) {
  k_orbital_NU<<<(M + RT - 1) / RT, RT, 0, s>>>(M, n_exp, gsig, a_inf, b_inf, onsite, st, N, U, dos);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_ef_response(int M, int n_exp, const double* gsig, const double* a_inf, const double* b_inf,
                       const double* onsite, const FermiState* st, double* red, unsigned* counter, double* lam,
                       cudaStream_t s) {
  k_ef_response<<<red_grid(M), RT, 0, s>>>(M, n_exp, gsig, a_inf, b_inf, onsite, st, red, counter, lam);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_weights(const WeightArgs& a, cudaStream_t s) {
  size_t smem = (size_t)2 * (a.n_exp + 3) * ZB * sizeof(double);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_weights, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_weights<<<(a.M + ZB - 1) / ZB, ZB, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_scf_update(const ScfArgs& a, cudaStream_t s) {
  int g = red_grid(a.n);
  k_scf_residual<<<g, RT, 0, s>>>(a);
  k_scf_apply<<<g, RT, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void launch_to_float(const double* in, float* out, size_t n, cudaStream_t s) {
  if (n) k_to_float<<<(unsigned)((n + RT - 1) / RT), RT, 0, s>>>(in, out, n);
}

void launch_build_onsite(int n, int norb, int n_spin, double onsite0, double stoner_I, const double* delta,
                         const double* m, double* onsite, float* onsite32, cudaStream_t s) {
  int tot = n_spin * n * norb;
  k_build_onsite<<<(tot + RT - 1) / RT, RT, 0, s>>>(n, norb, n_spin, onsite0, stoner_I, delta, m, onsite,
                                                   onsite32);
}

int launch_energy(int n, int norb, int n_spin, double spin_factor, double stoner_I, const double* U,
                  const double* m, double* e_atom, double* red, unsigned* counter, double* e_total,
                  cudaStream_t s) {
  k_energy<<<red_grid(n), RT, 0, s>>>(n, norb, n_spin, spin_factor, stoner_I, U, m, e_atom, red, counter,
                                      e_total);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
