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
#include "scalar_common.cuh"

namespace {
using namespace scal;

__global__ void k_jackson(double* g, int n_exp) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > n_exp) return;
  const double N = n_exp, x = PI / (N + 1.0);
  auto gJ = [&](double mm) { return ((N - mm + 1.0) * cos(mm * x) + sin(mm * x) / tan(x)) / (N + 1.0); };
  g[m] = gJ(m + 1.0) / gJ(1.0);
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




int launch_scf_residual(const ScfArgs& a, cudaStream_t s) {
  k_scf_residual<<<red_grid(a.n), RT, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_scf_apply(const ScfArgs& a, cudaStream_t s) {
  k_scf_apply<<<red_grid(a.n), RT, 0, s>>>(a);
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
