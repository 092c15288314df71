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
// Self-consistency of the onsite levels (local charge neutrality, Eq.
// BOP_LCN, per atom; collinear Stoner moments, Eq. onsite_NCM).  With the
// preconditioned residual of atom i
//   F_delta = eta (N_i - N0) / max(n_i(E_F), dos_floor),   F_m = m_mix (m_out - m),
// linear mixing is x_{k+1} = x_k + F_k.  Anderson mixing (type-II Broyden)
// over the last h iterations uses dF_j = F_{j+1} - F_j, dX_j = x_{j+1} - x_j:
//   gamma = argmin | F_k - sum_j gamma_j dF_j |,
//   x_{k+1} = x_k + F_k - sum_j gamma_j (dX_j + dF_j).
// The onsite shifts keep zero mean (the gauge fixed by E_F).
constexpr int NPAR = 64;  // partial sums per block: 3 + h(h+1)/2 + 2h + 1 <= 64 for h <= 8

__device__ __forceinline__ int hslot(int it, int S1) { return ((it % S1) + S1) % S1; }

// HH: the history depth of this update (min(it, hist) for Anderson, 0 for
// linear mixing), a template argument so that the per-thread sums, the
// history differences and the normal equations stay in registers.
template <int HH>
__global__ void __launch_bounds__(RT) k_scf_residual(ScfArgs A) {
  constexpr int h = HH;
  constexpr int nA = h * (h + 1) / 2;  // A_jl, j <= l
  // acc: [0] max|res| [1] max|dm| [2] sum F_delta (or sum delta_new) [3..3+nA) A
  //      [3+nA .. 3+nA+h) b_j   [3+nA+h .. 3+nA+2h) sum dF_j (delta part)
  constexpr int nv = 3 + nA + 2 * h;
  static_assert(nv <= NPAR, "partials per block");
  __shared__ double sh[nv][RT / 32];
  __shared__ double tot_s[nv];
  __shared__ bool last;
  const int S1 = A.hist + 1;
  const int slot = hslot(A.it, S1);
  double acc[nv];
#pragma unroll
  for (int q = 0; q < nv; q++) acc[q] = 0.0;
  const int ncomp = A.mode == 2 ? 2 : 1;
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
    double res, Fd;
    if (A.mode == 3) {  // variational: Newton-like step on dU_B/d delta_i
      res = A.grad[i];
      const double Dt = fmax(di, A.dos_floor);
      Fd = -A.eta * res / (Dt * (1.0 + A.J * Dt));
    } else {
      res = Ni - A.n0;
      Fd = A.eta * res / fmax(di, A.dos_floor);
    }
    acc[0] = fmax(acc[0], fabs(res));
    double Fm = 0.0;
    if (A.mode == 2) {
      double mo = 0.0;
      for (int a = 0; a < A.norb; a++) mo += A.N[(size_t)i * A.norb + a] - A.N[((size_t)A.n + i) * A.norb + a];
      acc[1] = fmax(acc[1], fabs(mo - A.m[i]));
      Fm = A.m_mix * (mo - A.m[i]);
    }
    if (A.mixer == 0) {
      const double dn = A.delta[i] + Fd;
      A.delta_new[i] = dn;
      acc[2] += dn;
      if (A.mode == 2) A.m_new[i] = A.m[i] + Fm;
      continue;
    }
    const size_t n2 = (size_t)A.n * ncomp;
    for (int c = 0; c < ncomp; c++) {
      const size_t idx = (size_t)c * A.n + i;
      const double fk = c == 0 ? Fd : Fm;
      A.hx[(size_t)slot * n2 + idx] = c == 0 ? A.delta[i] : A.m[i];
      A.hf[(size_t)slot * n2 + idx] = fk;
      double df[h > 0 ? h : 1];
#pragma unroll
      for (int j = 0; j < h; j++) {
        const int s0 = hslot(A.it - h + j, S1), s1 = hslot(A.it - h + j + 1, S1);
        const double f1 = (j == h - 1) ? fk : A.hf[(size_t)s1 * n2 + idx];
        df[j] = f1 - A.hf[(size_t)s0 * n2 + idx];
      }
#pragma unroll
      for (int j = 0; j < h; j++)
#pragma unroll
        for (int l = j; l < h; l++) acc[3 + j * h - j * (j - 1) / 2 + (l - j)] += df[j] * df[l];
#pragma unroll
      for (int j = 0; j < h; j++) acc[3 + nA + j] += df[j] * fk;
      if (c == 0) {
        acc[2] += fk;
#pragma unroll
        for (int j = 0; j < h; j++) acc[3 + nA + h + j] += df[j];
      }
    }
  }
  // block reduction: max for [0], [1], sums for the rest (a fixed shuffle
  // tree per quantity, then one thread per quantity over the warps in order)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < nv; q++) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v, o);
      v = q < 2 ? fmax(v, w) : v + w;
    }
    if (lane == 0) sh[q][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    const int q = threadIdx.x;
    double v = 0.0;
    for (int w = 0; w < RT / 32; w++) v = q < 2 ? fmax(v, sh[q][w]) : v + sh[q][w];
    A.red[(size_t)NPAR * blockIdx.x + q] = v;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(A.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  // one thread per reduced quantity, blocks in ascending order (fixed order)
  if (threadIdx.x < nv) {
    const int q = threadIdx.x;
    double v = 0.0;
    for (int b = 0; b < (int)gridDim.x; b++) {
      const double x = __ldcg(A.red + (size_t)NPAR * b + q);
      v = q < 2 ? fmax(v, x) : v + x;
    }
    tot_s[q] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const bool conv = tot_s[0] < A.tol && (A.mode != 2 || tot_s[1] < 10.0 * A.tol);
  A.result[0] = tot_s[0];
  A.result[1] = tot_s[1];
  A.result[2] = conv ? 1.0 : 0.0;
  if (A.mixer == 0 || h == 0) {
    A.result[3] = tot_s[2] / A.n;  // mean of delta_new (linear) or of x + F (no history yet)
  } else {
    // normal equations of the least-squares problem, Gaussian elimination
    // with partial pivoting (row exchanges as predicated swaps of fixed rows)
    double G[h > 0 ? h : 1][h + 1];
    double dmax = 0.0;
#pragma unroll
    for (int j = 0; j < h; j++)
#pragma unroll
      for (int l = j; l < h; l++) {
        const double g = tot_s[3 + j * h - j * (j - 1) / 2 + (l - j)];
        G[j][l] = g;
        G[l][j] = g;
        if (j == l) dmax = fmax(dmax, g);
      }
#pragma unroll
    for (int j = 0; j < h; j++) {
      G[j][h] = tot_s[3 + nA + j];
      G[j][j] += 1e-12 * dmax + 1e-300;
    }
    bool ok = true;
#pragma unroll
    for (int c = 0; c < h; c++) {
      int pr = c;
      double best = fabs(G[c][c]);
#pragma unroll
      for (int r = c + 1; r < h; r++)
        if (fabs(G[r][c]) > best) {
          best = fabs(G[r][c]);
          pr = r;
        }
      if (!(best > 0.0)) ok = false;
#pragma unroll
      for (int r = c + 1; r < h; r++)
        if (r == pr)
#pragma unroll
          for (int k = 0; k <= h; k++) {
            const double t = G[c][k];
            G[c][k] = G[r][k];
            G[r][k] = t;
          }
      if (ok) {
#pragma unroll
        for (int r = c + 1; r < h; r++) {
          const double f = G[r][c] / G[c][c];
#pragma unroll
          for (int k = c; k <= h; k++) G[r][k] -= f * G[c][k];
        }
      }
    }
    double gam[h > 0 ? h : 1];
#pragma unroll
    for (int j = h - 1; j >= 0; j--) {
      double v = ok ? G[j][h] : 0.0;
      if (ok) {
#pragma unroll
        for (int k = j + 1; k < h; k++) v -= G[j][k] * gam[k];
        v /= G[j][j];
      }
      gam[j] = isfinite(v) ? v : 0.0;
    }
    double mean = tot_s[2];
#pragma unroll
    for (int j = 0; j < h; j++) {
      A.gamma[j] = gam[j];
      mean -= gam[j] * tot_s[3 + nA + h + j];
    }
    A.result[3] = mean / A.n;  // mean of the updated delta before the gauge shift
  }
  *A.counter = 0;
}

__global__ void __launch_bounds__(RT) k_scf_apply(ScfArgs A) {
  if (A.result[2] != 0.0) return;
  const double mean = A.result[3];
  const int H = A.hist, S1 = H + 1;
  const int h = A.mixer == 1 ? (A.it < H ? A.it : H) : 0;
  const int ncomp = A.mode == 2 ? 2 : 1;
  const size_t n2 = (size_t)A.n * ncomp;
  for (int i = blockIdx.x * RT + threadIdx.x; i < A.n; i += gridDim.x * RT) {
    if (A.mixer == 0) {
      A.delta[i] = A.delta_new[i] - mean;
      if (A.mode == 2) A.m[i] = A.m_new[i];
      continue;
    }
    for (int c = 0; c < ncomp; c++) {
      const size_t idx = (size_t)c * A.n + i;
      const int sk = hslot(A.it, S1);
      double x = A.hx[(size_t)sk * n2 + idx] + A.hf[(size_t)sk * n2 + idx];
      for (int j = 0; j < h; j++) {
        const int s0 = hslot(A.it - h + j, S1), s1 = hslot(A.it - h + j + 1, S1);
        const double dX = A.hx[(size_t)s1 * n2 + idx] - A.hx[(size_t)s0 * n2 + idx];
        const double dF = A.hf[(size_t)s1 * n2 + idx] - A.hf[(size_t)s0 * n2 + idx];
        x -= A.gamma[j] * (dX + dF);
      }
      if (c == 0) A.delta[i] = x - mean;
      else A.m[i] = x;
    }
  }
}

// E_ialpha,nu = E^0_alpha + delta_i -/+ I m_i / 2 (spin up lower); E^0 is
// es for the s orbital of an sd model (orbital 0), e0 otherwise.
__global__ void __launch_bounds__(RT) k_build_onsite(int n, int norb, int n_spin, double e0, double es, double I,
                                                     const double* __restrict__ delta,
                                                     const double* __restrict__ m, double* __restrict__ on,
                                                     float* __restrict__ on32) {
  int q = blockIdx.x * RT + threadIdx.x;
  int tot = n_spin * n * norb;
  if (q >= tot) return;
  int i = (q / norb) % n, v = q / (n * norb);
  double e = (norb == 6 && q % norb == 0 ? es : e0) + (delta ? delta[i] : 0.0);
  if (m && n_spin == 2) e += (v == 0 ? -0.5 : 0.5) * I * m[i];
  on[q] = e;
  if (on32) on32[q] = (float)e;
}

__global__ void __launch_bounds__(RT) k_energy(int n, int norb, int n_spin, double sfac, double I,
                                               const double* __restrict__ U, const double* __restrict__ m,
                                               double J, const double* __restrict__ N, double n0,
                                               const double* __restrict__ erep, double* __restrict__ e_atom,
                                               double* red, unsigned* counter, double* e_total) {
  __shared__ double sh[RT / 32];
  __shared__ bool last;
  double acc = 0.0;
  for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT) {
    double e = 0.0;
    for (int v = 0; v < n_spin; v++)
      for (int a = 0; a < norb; a++) e += U[((size_t)v * n + i) * norb + a];
    e *= sfac;
    if (m && n_spin == 2) e -= 0.25 * I * m[i] * m[i];
    if (N) {
      double q = 0.0;
      for (int v = 0; v < n_spin; v++)
        for (int a = 0; a < norb; a++) q += N[((size_t)v * n + i) * norb + a];
      q = sfac * q - n0;
      e += 0.5 * J * q * q;
    }
    if (erep) e += erep[i];
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
  if (!last) return;
  __shared__ double fr[RT / 32 + 1];
  const double s = final_reduce<RT>(red, 1, 0, gridDim.x, false, fr);
  if (threadIdx.x == 0) {
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
  const int h = a.mixer == 1 ? (a.it < a.hist ? a.it : a.hist) : 0;
  const int g = red_grid(a.n);
  switch (h) {
    case 0: k_scf_residual<0><<<g, RT, 0, s>>>(a); break;
    case 1: k_scf_residual<1><<<g, RT, 0, s>>>(a); break;
    case 2: k_scf_residual<2><<<g, RT, 0, s>>>(a); break;
    case 3: k_scf_residual<3><<<g, RT, 0, s>>>(a); break;
    case 4: k_scf_residual<4><<<g, RT, 0, s>>>(a); break;
    case 5: k_scf_residual<5><<<g, RT, 0, s>>>(a); break;
    case 6: k_scf_residual<6><<<g, RT, 0, s>>>(a); break;
    case 7: k_scf_residual<7><<<g, RT, 0, s>>>(a); break;
    case 8: k_scf_residual<8><<<g, RT, 0, s>>>(a); break;
    default: return -1;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_scf_apply(const ScfArgs& a, cudaStream_t s) {
  k_scf_apply<<<red_grid(a.n), RT, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void launch_to_float(const double* in, float* out, size_t n, cudaStream_t s) {
  if (n) k_to_float<<<(unsigned)((n + RT - 1) / RT), RT, 0, s>>>(in, out, n);
}

void launch_build_onsite(int n, int norb, int n_spin, double onsite0, double onsite_s, double stoner_I,
                         const double* delta,
                         const double* m, double* onsite, float* onsite32, cudaStream_t s) {
  int tot = n_spin * n * norb;
  k_build_onsite<<<(tot + RT - 1) / RT, RT, 0, s>>>(n, norb, n_spin, onsite0, onsite_s, stoner_I, delta, m, onsite,
                                                   onsite32);
}

int launch_energy(int n, int norb, int n_spin, double spin_factor, double stoner_I, const double* U,
                  const double* m, double J, const double* N, double n0, const double* erep, double* e_atom,
                  double* red, unsigned* counter, double* e_total, cudaStream_t s) {
  k_energy<<<red_grid(n), RT, 0, s>>>(n, norb, n_spin, spin_factor, stoner_I, U, m, J, N, n0, erep, e_atom, red,
                                      counter, e_total);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
