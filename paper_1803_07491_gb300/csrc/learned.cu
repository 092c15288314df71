// Per-orbital kernels of the learned terminator: the network's inputs from
// the first 9 moments, its training data from 17-moment runs, the continued
// chain (4 computed levels, 4 predicted levels and a predicted band centre
// and width, then the constant terminator of Eq. abinf) with its expansion
// (Eq. aexp through the generating function), and the reverse mode of all
// of it around the network's own reverse pass (mlp.cu).
//
// Inputs x (18): (a_k - a_inf)/b_inf (k = 0..3), b_k/b_inf (k = 1..4),
// a_inf, b_inf, mu-hat_1 .. mu-hat_8 (Eq. sigma_i normalisation), with the
// 9-moment Gershgorin a_inf, b_inf (Eq. gershogorin).  Outputs y (10):
// (a*_inf - a_inf)/b_inf, b*_inf/b_inf, (a_k - a_inf)/b_inf (k = 4..7),
// b_k/b_inf (k = 5..8) of the 17-moment chain.  The constant terminator of
// the 9-moment chain is kept where that chain is truncated, an input is
// outside the training range, a predicted b is not above the band-width
// floor, or a value is not finite.
#include "chain_common.cuh"

using namespace scal;

namespace {

constexpr int CT = 32;  // one orbital per thread, small blocks (FP64-bound)
constexpr int NI = BOP_MLP_NIN, NO = BOP_MLP_NOUT;
constexpr int NORM_XM = 0, NORM_XS = NI, NORM_LO = 2 * NI, NORM_HI = 3 * NI, NORM_YM = 4 * NI,
              NORM_YS = 4 * NI + NO;
constexpr int KB = 4, KX = 8;  // levels of the 9-moment and of the continued chain
constexpr int NB = 10;         // base record: a_0..a_3, b_1..b_4, a_inf, b_inf

__device__ __forceinline__ double ldv(const float* p, size_t i) { return p[i]; }
__device__ __forceinline__ double ldv(const double* p, size_t i) { return p[i]; }

// Inputs of the network for one orbital (9-moment chain r, terminator t).
__device__ inline void features9(const double* mu, const Rec& r, const Term& t, double x[NI]) {
  const double ai = t.a_inf, bi = t.b_inf;
  for (int k = 0; k < KB; k++) x[k] = (r.a[k] - ai) / bi;
  for (int k = 1; k <= KB; k++) x[KB + k - 1] = r.b[k] / bi;
  x[8] = ai;
  x[9] = bi;
  // mu-hat_n = (2 b_inf)^-n sum_l C(n,l) (-a_inf)^l mu_{n-l}
  double s = 1.0;
  for (int n = 1; n <= 8; n++) {
    s /= (2.0 * bi);
    double acc = 0.0, c = 1.0, p = 1.0;  // C(n,l), (-a_inf)^l
    for (int l = 0; l <= n; l++) {
      acc += c * p * mu[n - l];
      c = c * (double)(n - l) / (double)(l + 1);
      p *= -ai;
    }
    x[9 + n] = acc * s;
  }
}

// The continued chain from the base record and the de-standardised outputs
// yh; false where the fallback applies.
__device__ inline bool continue_chain(const double* base, int nlev, const double yh[NO], Rec& r, Term& t) {
  const double ai = base[8], bi = base[9];
  bool ok = nlev == KB;
  for (int j = 0; j < NO; j++) ok &= isfinite(yh[j]);
  const double as = ai + bi * yh[0], bs = bi * yh[1];
  ok &= bs > B_INF_MIN;
  for (int k = KB + 1; k <= KX; k++) ok &= bi * yh[k + 1] > B_INF_MIN;
  r.b[0] = 0.0;
  for (int k = 0; k < KB; k++) r.a[k] = base[k];
  for (int k = 1; k <= KB; k++) r.b[k] = base[KB + k - 1];
  for (int k = KB; k < KPMAX; k++) r.a[k] = 0.0;
  for (int k = KB + 1; k <= KPMAX; k++) r.b[k] = 0.0;
  r.trunc = nlev < KB;
  t.ilo = t.ihi = 0;
  t.floored = false;
  if (ok) {
    for (int k = KB; k < KX; k++) r.a[k] = ai + bi * yh[k - 2];
    for (int k = KB + 1; k <= KX; k++) r.b[k] = bi * yh[k + 1];
    r.nlev = KX;
    t.a_inf = as;
    t.b_inf = bs;
  } else {
    r.nlev = nlev;
    t.a_inf = ai;
    t.b_inf = bi;
  }
  return ok;
}

// The plain 9-moment chain with its Gershgorin terminator.
__device__ inline void base_chain(const double* base, int nlev, Rec& r, Term& t) {
  r.b[0] = 0.0;
  for (int k = 0; k < KPMAX; k++) r.a[k] = k < KB ? base[k] : 0.0;
  for (int k = 1; k <= KPMAX; k++) r.b[k] = k <= KB ? base[KB + k - 1] : 0.0;
  r.nlev = nlev;
  r.trunc = nlev < KB;
  t.a_inf = base[8];
  t.b_inf = base[9];
  t.ilo = t.ihi = 0;
  t.floored = false;
}

template <class T>
__device__ inline void destandardise(const LearnedArgs& A, int o, double yh[NO]) {
  const T* ys = static_cast<const T*>(A.ys);
  for (int j = 0; j < NO; j++)
    yh[j] = (double)A.norm[NORM_YM + j] + (double)A.norm[NORM_YS + j] * ldv(ys, (size_t)o * NO + j);
}

// mu[9] -> base record, nlev, standardised inputs, in-range flag.
template <class T>
__global__ void __launch_bounds__(CT) k_features(LearnedArgs A) {
  const int o = blockIdx.x * CT + threadIdx.x;
  if (o >= A.M) return;
  double mu[9];
  for (int n = 0; n < 9; n++) mu[n] = A.mu[(size_t)o * 9 + n];
  Rec r;
  recursion(mu, KB, r);
  const Term t = gershgorin(r);
  double x[NI];
  features9(mu, r, t, x);
  double* base = A.base + (size_t)o * NB;
  for (int k = 0; k < KB; k++) base[k] = r.a[k];
  for (int k = 1; k <= KB; k++) base[KB + k - 1] = r.b[k];
  base[8] = t.a_inf;
  base[9] = t.b_inf;
  A.nlev[o] = r.nlev;
  bool inside = r.nlev == KB;
  T* xs = static_cast<T*>(A.xs);
  for (int j = 0; j < NI; j++) {
    inside &= x[j] >= (double)A.norm[NORM_LO + j] && x[j] <= (double)A.norm[NORM_HI + j];
    xs[(size_t)o * NI + j] = (T)((x[j] - (double)A.norm[NORM_XM + j]) / (double)A.norm[NORM_XS + j]);
  }
  A.flag[o] = inside ? 1 : 0;
}

// Continued chain -> a*_inf, b*_inf, g_m sigma_m (n_exp + 1 terms).
template <class T>
__global__ void __launch_bounds__(CT) k_expand_learned(LearnedArgs A) {
  const int o = blockIdx.x * CT + threadIdx.x;
  bool ok = false;
  if (o < A.M) {
    double yh[NO];
    destandardise<T>(A, o, yh);
    const double* base = A.base + (size_t)o * NB;
    Rec r;
    Term t;
    ok = (A.flag[o] & 1) && continue_chain(base, A.nlev[o], yh, r, t);
    if (!ok) base_chain(base, A.nlev[o], r, t);
    Chain ch;
    chain_params(r, t, ok ? KX : KB, ch);
    double Q[2 * KX + 1], P[2 * KX + 1];
    gen_polys<KX>(ch, r.nlev, Q, P);
    const double last = A.sig32 ? sigma_series<KX, false, true>(Q, P, A.n_exp, A.g, A.gsig, A.M, o)
                                : sigma_series<KX>(Q, P, A.n_exp, A.g, A.gsig, A.M, o);
    A.a_inf[o] = t.a_inf;
    A.b_inf[o] = t.b_inf;
    A.flag[o] = (A.flag[o] & 1) | (ok ? 2 : 0);
    if (!isfinite(t.a_inf) || !isfinite(t.b_inf) || !isfinite(last)) raise_error(A.status, BOP_DEV_ERR_NONFINITE);
  }
  const unsigned bal = __ballot_sync(0xffffffffu, ok);
  if (threadIdx.x == 0 && bal) atomicAdd(A.n_learned, (unsigned)__popc(bal));
}

// Reverse of the chain part: cotangents of the network outputs (ybar,
// standardised) and of the base record (cot).
template <class T>
__global__ void __launch_bounds__(CT) k_weights_learned_a(LearnedArgs A) {
  const int o = blockIdx.x * CT + threadIdx.x;
  if (o >= A.M) return;
  const WeightArgs& W = A.W;
  const int M = A.M;
  const double cU = W.cU;
  const double cN = W.var_q ? cU * (W.var_J * W.var_q[o / W.norb] - W.var_lam[0])
                            : (W.lam ? -W.cU * W.lam[0] : W.cN0);
  double yh[NO];
  destandardise<T>(A, o, yh);
  const double* base = A.base + (size_t)o * NB;
  const bool learned = (A.flag[o] & 2) != 0;
  Rec r;
  Term t;
  if (learned) continue_chain(base, KB, yh, r, t);
  else base_chain(base, A.nlev[o], r, t);
  Chain ch;
  chain_params(r, t, learned ? KX : KB, ch);
  double abar[KPMAX + 1], bbar[KPMAX + 2];
  for (int k = 0; k <= KPMAX; k++) abar[k] = 0.0;
  for (int k = 0; k <= KPMAX + 1; k++) bbar[k] = 0.0;
  double abar_inf = 0.0, bbar_inf = 0.0;
  const double dE = chain_reverse<KX>(ch, r.nlev, learned ? KX : KB, t.a_inf, t.b_inf, W.onsite[o], W.st->ef, W.g,
                                      W.inv, W.n_exp, M, o, cU, cN, W.zscratch,
                                      W.zscratch + (size_t)(W.n_exp + 1) * M, abar, bbar, abar_inf, bbar_inf,
                                      A.sig32 != 0);
  if (W.dU_dE) W.dU_dE[o] = dE;
  double yb[NO];
  for (int j = 0; j < NO; j++) yb[j] = 0.0;
  double aib = 0.0, bib = 0.0;  // cotangents of the 9-moment a_inf, b_inf
  if (learned) {
    const double bi = base[9];
    // a*_inf = a_inf + b_inf yh_0, b*_inf = b_inf yh_1
    yb[0] += abar_inf * bi;
    aib += abar_inf;
    bib += abar_inf * yh[0];
    yb[1] += bbar_inf * bi;
    bib += bbar_inf * yh[1];
    for (int k = KB; k < KX; k++) {  // a_k = a_inf + b_inf yh_{k-2}
      yb[k - 2] += abar[k] * bi;
      aib += abar[k];
      bib += abar[k] * yh[k - 2];
    }
    for (int k = KB + 1; k <= KX; k++) {  // b_k = b_inf yh_{k+1}
      yb[k + 1] += bbar[k] * bi;
      bib += bbar[k] * yh[k + 1];
    }
  } else {
    aib = abar_inf;
    bib = bbar_inf;
  }
  T* ybar = static_cast<T*>(A.ybar);
  for (int j = 0; j < NO; j++) ybar[(size_t)o * NO + j] = (T)(yb[j] * (double)A.norm[NORM_YS + j]);
  double* cot = A.cot + (size_t)o * NB;
  for (int k = 0; k < KB; k++) cot[k] = abar[k];
  for (int k = 1; k <= KB; k++) cot[KB + k - 1] = bbar[k];
  cot[8] = aib;
  cot[9] = bib;
}

// Reverse of the features, Gershgorin and the moment recursion -> w.
template <class T>
__global__ void __launch_bounds__(CT) k_weights_learned_b(LearnedArgs A) {
  const int o = blockIdx.x * CT + threadIdx.x;
  if (o >= A.M) return;
  double mu[9];
  for (int n = 0; n < 9; n++) mu[n] = A.mu[(size_t)o * 9 + n];
  Rec r;
  RecTape<KB> tp;
  recursion_taped<KB>(mu, r, tp);
  const Term t = gershgorin(r);
  const double* cot = A.cot + (size_t)o * NB;
  double abar[KPMAX + 1], bbar[KPMAX + 2];
  for (int k = 0; k <= KPMAX; k++) abar[k] = 0.0;
  for (int k = 0; k <= KPMAX + 1; k++) bbar[k] = 0.0;
  for (int k = 0; k < KB; k++) abar[k] = cot[k];
  for (int k = 1; k <= KB; k++) bbar[k] = cot[KB + k - 1];
  double abar_inf = cot[8], bbar_inf = cot[9];
  double mub[9];
  for (int n = 0; n < 9; n++) mub[n] = 0.0;
  if (A.flag[o] & 2) {
    const T* xbar = static_cast<const T*>(A.xbar);
    double xb[NI];
    for (int j = 0; j < NI; j++) xb[j] = ldv(xbar, (size_t)o * NI + j) / (double)A.norm[NORM_XS + j];
    const double ai = t.a_inf, bi = t.b_inf;
    for (int k = 0; k < KB; k++) {  // x_k = (a_k - a_inf)/b_inf
      const double xk = (r.a[k] - ai) / bi;
      abar[k] += xb[k] / bi;
      abar_inf -= xb[k] / bi;
      bbar_inf -= xb[k] * xk / bi;
    }
    for (int k = 1; k <= KB; k++) {  // x = b_k/b_inf
      const double xk = r.b[k] / bi;
      bbar[k] += xb[KB + k - 1] / bi;
      bbar_inf -= xb[KB + k - 1] * xk / bi;
    }
    abar_inf += xb[8];
    bbar_inf += xb[9];
    double s = 1.0;
    for (int n = 1; n <= 8; n++) {  // mu-hat_n
      s /= (2.0 * bi);
      const double g = xb[9 + n];
      double acc = 0.0, dacc = 0.0, c = 1.0, p = 1.0, pm = 0.0;  // pm = (-a_inf)^(l-1)
      for (int l = 0; l <= n; l++) {
        acc += c * p * mu[n - l];
        mub[n - l] += g * s * c * p;
        if (l >= 1) dacc += c * (double)l * pm * mu[n - l];  // d/d(-a_inf) of (-a_inf)^l
        c = c * (double)(n - l) / (double)(l + 1);
        pm = p;
        p *= -ai;
      }
      abar_inf += -g * s * dacc;
      bbar_inf += -g * (double)n / bi * acc * s;
    }
  }
  gershgorin_reverse(t, abar_inf, bbar_inf, abar, bbar);
  recursion_reverse<KB>(mu, r, tp, abar, bbar, mub);
  bool bad = false;
  for (int n = 0; n < 9; n++) {
    A.W.w[(size_t)o * 9 + n] = mub[n];
    bad |= !isfinite(mub[n]);
  }
  if (bad) raise_error(A.W.status, BOP_DEV_ERR_NONFINITE);
}

// Training data from 17 moments: x (18, raw), t (10, raw), mask (1 where
// the 17-moment chain has all 8 levels).
__global__ void __launch_bounds__(CT) k_mlp_dataset(long long M, const double* __restrict__ mu17,
                                                    float* __restrict__ x, float* __restrict__ t,
                                                    float* __restrict__ mask) {
  const long long o = (long long)blockIdx.x * CT + threadIdx.x;
  if (o >= M) return;
  double mu[17];
  for (int n = 0; n < 17; n++) mu[n] = mu17[o * 17 + n];
  Rec r9, r17;
  recursion(mu, KB, r9);
  const Term t9 = gershgorin(r9);
  recursion(mu, KX, r17);
  const Term t17 = gershgorin(r17);
  double xf[NI];
  features9(mu, r9, t9, xf);
  for (int j = 0; j < NI; j++) x[o * NI + j] = (float)xf[j];
  const double ai = t9.a_inf, bi = t9.b_inf;
  double tv[NO];
  tv[0] = (t17.a_inf - ai) / bi;
  tv[1] = t17.b_inf / bi;
  for (int k = KB; k < KX; k++) tv[k - 2] = (r17.a[k] - ai) / bi;
  for (int k = KB + 1; k <= KX; k++) tv[k + 1] = r17.b[k] / bi;
  bool ok = r17.nlev == KX;
  for (int j = 0; j < NO; j++) {
    ok &= isfinite(tv[j]);
    t[o * NO + j] = (float)(isfinite(tv[j]) ? tv[j] : 0.0);
  }
  mask[o] = ok ? 1.f : 0.f;
}

}  // namespace

int launch_learned(int stage, const LearnedArgs& a, cudaStream_t s) {
  const int g = (a.M + CT - 1) / CT;
  if (a.M <= 0) return 0;
  switch (stage * 2 + (a.fp64 ? 1 : 0)) {
    case 0: k_features<float><<<g, CT, 0, s>>>(a); break;
    case 1: k_features<double><<<g, CT, 0, s>>>(a); break;
    case 2: k_expand_learned<float><<<g, CT, 0, s>>>(a); break;
    case 3: k_expand_learned<double><<<g, CT, 0, s>>>(a); break;
    case 4: k_weights_learned_a<float><<<g, CT, 0, s>>>(a); break;
    case 5: k_weights_learned_a<double><<<g, CT, 0, s>>>(a); break;
    case 6: k_weights_learned_b<float><<<g, CT, 0, s>>>(a); break;
    case 7: k_weights_learned_b<double><<<g, CT, 0, s>>>(a); break;
    default: return -1;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_mlp_dataset(long long M, const double* mu17, float* x, float* t, float* mask, cudaStream_t s) {
  if (M <= 0) return 0;
  k_mlp_dataset<<<(unsigned)((M + CT - 1) / CT), CT, 0, s>>>(M, mu17, x, t, mask);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
