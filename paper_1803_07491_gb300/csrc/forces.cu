// Forces and virial from the bond cotangents (Eq. F_k, Eq. sigma_k): for
// every bond b with vector d_b = r_j + S.cell - r_i,
//   g_b = sum_u Hbar_b,u  dH_b,u / dd_b      (u = unique block elements;
//                                             Hbar in the product type)
//         + d phi(|d_b|) / dd_b              (pair repulsion, when present)
//   F_i += g_b,  F_j -= g_b,  W += g_b (x) d_b.
// dH/dd is exact: the two-centre block is evaluated in forward-mode dual
// numbers.
#include "kernels.h"

namespace {

constexpr int FT = 256;

template <typename HT>
__global__ void __launch_bounds__(FT) k_forces(int nb, BondModel m, const double* __restrict__ bond_d,
                                               const int* __restrict__ bond_atoms, const HT* __restrict__ Hbar,
                                               int HSh, double* __restrict__ F, double* __restrict__ W) {
  __shared__ double sw[9][FT / 32];
  double w9[9];
  for (int q = 0; q < 9; q++) w9[q] = 0.0;
  // block derivatives in the cotangents' type: FP32 duals in the
  // FP32-products mode (relative error ~1e-6 of dH/dd), FP64 otherwise
  using DT = typename std::conditional<sizeof(HT) == 4, D3f, D3>::type;
  using ST = decltype(DT{}.v);
  for (int b = blockIdx.x * FT + threadIdx.x; b < nb; b += gridDim.x * FT) {
    DT d[3];
    double dv[3] = {bond_d[3 * b], bond_d[3 * b + 1], bond_d[3 * b + 2]};
    d[0] = {(ST)dv[0], ST(1), ST(0), ST(0)};
    d[1] = {(ST)dv[1], ST(0), ST(1), ST(0)};
    d[2] = {(ST)dv[2], ST(0), ST(0), ST(1)};
    DT u[21];
    sk_unique<DT>(m, d, u);
    const int nu = block_unique(m.norb);
    ST a0 = ST(0), a1 = ST(0), a2 = ST(0);
    for (int q = 0; q < nu; q++) {
      const ST hb = (ST)Hbar[(size_t)b * HSh + q];
      a0 += hb * u[q].g0;
      a1 += hb * u[q].g1;
      a2 += hb * u[q].g2;
    }
    double g0 = a0, g1 = a1, g2 = a2;
    if (m.rep_A != 0.0) {  // pair repulsion of the bond
      const DT ph = pair_repulsion(m, dsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
      g0 += ph.g0;
      g1 += ph.g1;
      g2 += ph.g2;
    }
    int i = bond_atoms[2 * b], j = bond_atoms[2 * b + 1];
    atomicAdd(F + 3 * i, g0);
    atomicAdd(F + 3 * i + 1, g1);
    atomicAdd(F + 3 * i + 2, g2);
    atomicAdd(F + 3 * j, -g0);
    atomicAdd(F + 3 * j + 1, -g1);
    atomicAdd(F + 3 * j + 2, -g2);
    double g[3] = {g0, g1, g2};
    for (int a = 0; a < 3; a++)
      for (int c = 0; c < 3; c++) w9[3 * a + c] += g[a] * dv[c];
  }
  for (int q = 0; q < 9; q++) {
    double v = w9[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sw[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    double v = 0.0;
    for (int q = 0; q < FT / 32; q++) v += sw[threadIdx.x][q];
    atomicAdd(W + threadIdx.x, v);
  }
}

// Per-atom pair repulsion: half of every bond of the atom (its directed
// edges), in edge order.
__global__ void __launch_bounds__(FT) k_rep_energy(int n, BondModel m, const long long* __restrict__ row_ptr,
                                                   const int* __restrict__ bond_of_edge,
                                                   const double* __restrict__ bond_d, double* __restrict__ erep) {
  const int i = blockIdx.x * FT + threadIdx.x;
  if (i >= n) return;
  double e = 0.0;
  for (long long q = row_ptr[i]; q < row_ptr[i + 1]; q++) {
    const double* d = bond_d + 3 * (size_t)bond_of_edge[q];
    e += 0.5 * pair_repulsion(m, sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
  }
  erep[i] = e;
}

}  // namespace

int launch_rep_energy(int n, BondModel m, const long long* row_ptr, const int* bond_of_edge, const double* bond_d,
                      double* erep, cudaStream_t s) {
  if (n <= 0) return 0;
  k_rep_energy<<<(n + FT - 1) / FT, FT, 0, s>>>(n, m, row_ptr, bond_of_edge, bond_d, erep);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_forces(int nb, BondModel m, const double* bond_d, const int* bond_atoms, const void* Hbar, int HSh,
                  int fp64, double* forces, double* virial, cudaStream_t s) {
  int g = (nb + FT - 1) / FT;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  if (fp64)
    k_forces<double><<<g, FT, 0, s>>>(nb, m, bond_d, bond_atoms, (const double*)Hbar, HSh, forces, virial);
  else
    k_forces<float><<<g, FT, 0, s>>>(nb, m, bond_d, bond_atoms, (const float*)Hbar, HSh, forces, virial);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
