// Vector kernels of the SCF-response solve (bop_forces with an SCF): the
// multipliers y of J^T y = dE/du, with u the SCF unknowns (one onsite shift
// per atom, and for Stoner one moment per atom) and J the derivative of the
// SCF conditions at fixed E_F.  Products J^T v come from a reverse sweep of
// the moments (moments.cu) with weights c_{i,nu} dN/dmu; these kernels form
// those weights, project onsite-level cotangents onto u, and carry out the
// Gram-Schmidt and combination steps of GMRES.  Every reduction has a fixed
// order.
#include "kernels.h"

namespace {

constexpr int VT = 256;

// c_{i,nu} = s v[i] (+ sigma_nu v[n + i] for Stoner, sigma = +1 up, -1 down)
__global__ void k_scale_weights(int n, int norb, int S, int n_mom, double s, int stoner,
                                const double* __restrict__ v, double sign, const double* __restrict__ wN,
                                const double* __restrict__ wU, double* __restrict__ w) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)S * n * norb * n_mom;
  if (q >= tot) return;
  const long long o = q / n_mom;                // orbital (spin-major)
  const int atom = (int)((o / norb) % n);
  const int spin = (int)(o / ((long long)norb * n));
  double c = s * v[atom];
  if (stoner) c += (spin == 0 ? 1.0 : -1.0) * v[n + atom];
  w[q] = (wU ? wU[q] : 0.0) + sign * c * wN[q];
}

__global__ void k_project(int n, int norb, int S, double I, const double* __restrict__ Eb,
                          const double* __restrict__ dUE, const double* __restrict__ m, double mcoef,
                          const double* __restrict__ v_m, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double gd = 0.0, gm = 0.0;
  for (int sp = 0; sp < S; sp++) {
    double a = 0.0;
    for (int al = 0; al < norb; al++) {
      const size_t o = ((size_t)sp * n + i) * norb + al;
      a += Eb[o] + (dUE ? dUE[o] : 0.0);
    }
    gd += a;
    gm += (sp == 0 ? -0.5 : 0.5) * I * a;
  }
  out[i] = gd;
  if (S == 2) {
    if (m) gm += mcoef * m[i];
    if (v_m) gm -= v_m[i];
    out[n + i] = gm;
  }
}

__global__ void k_precond_diag(int n, int norb, int S, double s, double floor_, const double* __restrict__ dos,
                               double* __restrict__ P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int sp = 0; sp < S; sp++)
    for (int al = 0; al < norb; al++) d += dos[((size_t)sp * n + i) * norb + al];
  d *= s;
  P[i] = -1.0 / (d > floor_ ? d : floor_);
  if (S == 2) P[n + i] = -1.0;
}

// out[k] = V[k] . w, one block per vector: strided partial sums, a fixed
// shuffle tree and a fixed cross-warp order.
__global__ void __launch_bounds__(VT) k_dots(int nu, const double* __restrict__ V, const double* __restrict__ w,
                                             double* __restrict__ out) {
  __shared__ double sh[VT / 32];
  const int k = blockIdx.x;
  const double* vk = V + (size_t)k * nu;
  double a = 0.0;
  for (int i = threadIdx.x; i < nu; i += VT) a += vk[i] * w[i];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < VT / 32; q++) t += sh[q];
    out[k] = t;
  }
}

__global__ void k_axpy_multi(int nu, int nvec, const double* __restrict__ V, const double* __restrict__ coef,
                             double* __restrict__ w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nu) return;
  double a = w[i];
  for (int k = 0; k < nvec; k++) a -= coef[k] * V[(size_t)k * nu + i];
  w[i] = a;
}

__global__ void k_lincomb(int nu, int nvec, const double* __restrict__ V, const double* __restrict__ coef,
                          const double* __restrict__ P, double scale, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nu) return;
  double a = 0.0;
  for (int k = 0; k < nvec; k++) a += coef[k] * V[(size_t)k * nu + i];
  out[i] = scale * a * (P ? P[i] : 1.0);
}

__global__ void k_scale_vec(int nu, const double* __restrict__ x, const double* __restrict__ P, double a,
                            double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nu) return;
  out[i] = a * x[i] * (P ? P[i] : 1.0);
}

// Variational SCF: q_i and the E_F multiplier of U_B (see kernels.h).  Block
// partial sums in red[2 b], red[2 b + 1]; the last block adds them in block
// order (deterministic for a given grid).
__global__ void __launch_bounds__(VT) k_var_lambda(int n, int norb, double s, double J, double n0,
                                                   const double* __restrict__ N, const double* __restrict__ dos,
                                                   const double* __restrict__ onsite,
                                                   const FermiState* __restrict__ st, double* __restrict__ q,
                                                   double* __restrict__ lam, double* red, unsigned* counter) {
  __shared__ double sh[2][VT / 32];
  __shared__ bool last;
  const double ef = st->ef;
  double a = 0.0, b = 0.0;
  for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT) {
    double Ni = 0.0, Di = 0.0;
    for (int al = 0; al < norb; al++) {
      Ni += N[(size_t)i * norb + al];
      Di += dos[(size_t)i * norb + al];
    }
    const double qi = s * Ni - n0;
    Di *= s;
    q[i] = qi;
    a += Di * (ef - onsite[(size_t)i * norb] + J * qi);
    b += Di;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = a;
    sh[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < VT / 32; w++) {
      ta += sh[0][w];
      tb += sh[1][w];
    }
    red[2 * blockIdx.x] = ta;
    red[2 * blockIdx.x + 1] = tb;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  double ta = 0.0, tb = 0.0;
  for (int k = 0; k < (int)gridDim.x; k++) {
    ta += __ldcg(red + 2 * k);
    tb += __ldcg(red + 2 * k + 1);
  }
  lam[0] = tb > 0.0 ? ta / tb : 0.0;
  *counter = 0;
}

// u /= sqrt(*nsq) when *nsq > 0 (the norm stays on the device)
__global__ void k_scale_by_inv_norm(int nu, double* __restrict__ u, const double* __restrict__ nsq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double q = *nsq;
  if (i >= nu || !(q > 0.0)) return;
  u[i] = u[i] * (1.0 / sqrt(q));
}

// Transpose of the Jacobian rows: for every atom j the entries (i, site)
// with site_atom[site] = j among the first |C_K-1| sites of i's cluster.
// Count, then fill (rows in arbitrary order within an atom).
__global__ void k_jt_count(int n, int K, const long long* __restrict__ site_off, const int* __restrict__ level_end,
                           const int* __restrict__ site_atom, int* __restrict__ cnt) {
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const long long s0 = site_off[i];
  const int neb = level_end[(size_t)i * (K + 1) + K - 1];
  for (int t = lane; t < neb; t += 32) atomicAdd(cnt + site_atom[s0 + t], 1);
}

__global__ void k_jt_fill(int n, int K, const long long* __restrict__ site_off, const int* __restrict__ level_end,
                          const int* __restrict__ site_atom, const long long* __restrict__ ptr,
                          int* __restrict__ fill, long long* __restrict__ idx, int* __restrict__ row) {
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const long long s0 = site_off[i];
  const int neb = level_end[(size_t)i * (K + 1) + K - 1];
  for (int t = lane; t < neb; t += 32) {
    const int j = site_atom[s0 + t];
    const long long q = ptr[j] + atomicAdd(fill + j, 1);
    idx[q] = s0 + t;
    row[q] = i;
  }
}

// One warp per (spin, atom j): Eb[spin][j] = sum over j's entries of
// c_{i,spin} val[spin][site], c = s v[i] (+ sigma_spin v[n + i] for Stoner).
__global__ void k_jt_gather(int n, int S, const long long* __restrict__ ptr, const long long* __restrict__ idx,
                            const int* __restrict__ row, const double* __restrict__ val, long long stride,
                            const double* __restrict__ v, double s, int stoner, double* __restrict__ Eb) {
  const int wg = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (wg >= S * n) return;
  const int spin = wg / n, j = wg % n;
  const double sg = spin == 0 ? 1.0 : -1.0;
  const double* vs = val + (size_t)spin * stride;
  double a = 0.0;
  for (long long q = ptr[j] + lane; q < ptr[j + 1]; q += 32) {
    const int i = row[q];
    double c = s * v[i];
    if (stoner) c += sg * v[n + i];
    a += c * vs[idx[q]];
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) Eb[(size_t)spin * n + j] = a;
}

unsigned grid(long long n) { return (unsigned)((n + VT - 1) / VT); }
int ok() { return cudaGetLastError() == cudaSuccess ? 0 : -1; }

}  // namespace

int launch_scale_weights(int n, int norb, int S, int n_mom, double s, int stoner, const double* v, double sign,
                         const double* wN, const double* wU, double* w_out, cudaStream_t st) {
  const long long tot = (long long)S * n * norb * n_mom;
  k_scale_weights<<<grid(tot), VT, 0, st>>>(n, norb, S, n_mom, s, stoner, v, sign, wN, wU, w_out);
  return ok();
}

int launch_project(int n, int norb, int S, double I, const double* Eb, const double* dUE, const double* m,
                   double mcoef, const double* v_m, double* out, cudaStream_t st) {
  k_project<<<grid(n), VT, 0, st>>>(n, norb, S, I, Eb, dUE, m, mcoef, v_m, out);
  return ok();
}

int launch_precond_diag(int n, int norb, int S, double s, double floor_, const double* dos, double* P,
                        cudaStream_t st) {
  k_precond_diag<<<grid(n), VT, 0, st>>>(n, norb, S, s, floor_, dos, P);
  return ok();
}

int launch_dots(int nu, int nvec, const double* V, const double* w, double* out, cudaStream_t st) {
  if (nvec <= 0) return 0;
  k_dots<<<nvec, VT, 0, st>>>(nu, V, w, out);
  return ok();
}

int launch_axpy_multi(int nu, int nvec, const double* V, const double* coef, double* w, cudaStream_t st) {
  if (nvec <= 0) return 0;
  k_axpy_multi<<<grid(nu), VT, 0, st>>>(nu, nvec, V, coef, w);
  return ok();
}

int launch_lincomb(int nu, int nvec, const double* V, const double* coef, const double* P, double scale,
                   double* out, cudaStream_t st) {
  k_lincomb<<<grid(nu), VT, 0, st>>>(nu, nvec, V, coef, P, scale, out);
  return ok();
}

int launch_scale_vec(int nu, const double* x, const double* P, double a, double* out, cudaStream_t st) {
  k_scale_vec<<<grid(nu), VT, 0, st>>>(nu, x, P, a, out);
  return ok();
}

int launch_var_lambda(int n, int norb, double s, double J, double n0, const double* N, const double* dos,
                      const double* onsite, const FermiState* st, double* q, double* lam, double* red,
                      unsigned* counter, cudaStream_t stream) {
  unsigned g = grid(n);
  if (g < 1) g = 1;
  if (g > 1024) g = 1024;
  k_var_lambda<<<g, VT, 0, stream>>>(n, norb, s, J, n0, N, dos, onsite, st, q, lam, red, counter);
  return ok();
}

int launch_scale_by_inv_norm(int nu, double* u, const double* nsq, cudaStream_t stream) {
  k_scale_by_inv_norm<<<grid(nu), VT, 0, stream>>>(nu, u, nsq);
  return ok();
}

int launch_jt_build(int n, int K, const long long* site_off, const int* level_end, const int* site_atom,
                    int* cnt, int stage, const long long* ptr, long long* idx, int* row, cudaStream_t stream) {
  const long long threads = (long long)n * 32;
  if (stage == 0) k_jt_count<<<grid(threads), VT, 0, stream>>>(n, K, site_off, level_end, site_atom, cnt);
  else k_jt_fill<<<grid(threads), VT, 0, stream>>>(n, K, site_off, level_end, site_atom, ptr, cnt, idx, row);
  return ok();
}

int launch_jt_gather(int n, int S, const long long* ptr, const long long* idx, const int* row, const double* val,
                     long long stride, const double* v, double s, int stoner, double* Eb, cudaStream_t stream) {
  const long long threads = (long long)S * n * 32;
  k_jt_gather<<<grid(threads), VT, 0, stream>>>(n, S, ptr, idx, row, val, stride, v, s, stoner, Eb);
  return ok();
}
