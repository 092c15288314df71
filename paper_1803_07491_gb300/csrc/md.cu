// Velocity-Verlet update for molecular dynamics on the BOP forces: the
// driver of the warm-started MD loop (speed-up (ii) under "Performance":
// the self-consistent onsite levels of one step start the SCF of the next).
// Positions and velocities stay on the device between steps.
#include <cmath>

#include "kernels.h"

namespace {

// eV / (A amu) in A / fs^2
constexpr double ACC_UNIT = 1.602176634e-19 / (1.66053906660e-27 * 1e-10) * 1e-20;

struct Wrap {
  double cell[9];  // rows: lattice vectors
  double inv[9];   // frac_a = sum_r pos_r inv[r][a]
  int pbc[3];
  int on;
};

__global__ void k_verlet(int n, double* __restrict__ pos, double* __restrict__ vel, const double* __restrict__ f,
                         double half_dt_a, double dt, int drift, Wrap w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[3];
  for (int d = 0; d < 3; d++) {
    const double v = vel[3 * i + d] + half_dt_a * f[3 * i + d];
    vel[3 * i + d] = v;
    if (drift) x[d] = pos[3 * i + d] + dt * v;
  }
  if (!drift) return;
  if (w.on) {  // back into the cell along periodic axes: subtract whole lattice vectors
    for (int a = 0; a < 3; a++) {
      if (!w.pbc[a]) continue;
      const double fa = x[0] * w.inv[a] + x[1] * w.inv[3 + a] + x[2] * w.inv[6 + a];
      const double k = floor(fa);
      if (k != 0.0)
        for (int d = 0; d < 3; d++) x[d] -= k * w.cell[3 * a + d];
    }
  }
  for (int d = 0; d < 3; d++) pos[3 * i + d] = x[d];
}

}  // namespace

extern "C" int bop_md_verlet(int n, double* pos, double* vel, const double* forces, const double* cell,
                             const int* pbc, double dt, double mass, int phase, bop_stream stream) {
  if (n < 0 || !vel || !forces || !(dt > 0) || !(mass > 0) || (phase != 0 && phase != 1) ||
      (phase == 0 && !pos) || (cell && !pbc))
    return BOP_ERR_ARG;
  Wrap w;
  w.on = cell ? 1 : 0;
  for (int q = 0; q < 9; q++) w.cell[q] = cell ? cell[q] : 0.0;
  for (int a = 0; a < 3; a++) w.pbc[a] = pbc ? (pbc[a] ? 1 : 0) : 0;
  if (cell) {
    const double* a0 = cell;
    const double* a1 = cell + 3;
    const double* a2 = cell + 6;
    const double c12[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]};
    const double c20[3] = {a2[1] * a0[2] - a2[2] * a0[1], a2[2] * a0[0] - a2[0] * a0[2], a2[0] * a0[1] - a2[1] * a0[0]};
    const double c01[3] = {a0[1] * a1[2] - a0[2] * a1[1], a0[2] * a1[0] - a0[0] * a1[2], a0[0] * a1[1] - a0[1] * a1[0]};
    const double vol = a0[0] * c12[0] + a0[1] * c12[1] + a0[2] * c12[2];
    if (!(std::fabs(vol) > 1e-12)) return BOP_ERR_ARG;
    for (int r = 0; r < 3; r++) {
      w.inv[r * 3 + 0] = c12[r] / vol;
      w.inv[r * 3 + 1] = c20[r] / vol;
      w.inv[r * 3 + 2] = c01[r] / vol;
    }
  } else {
    for (int q = 0; q < 9; q++) w.inv[q] = 0.0;
  }
  if (n == 0) return BOP_OK;
  const double half_dt_a = 0.5 * dt * ACC_UNIT / mass;
  k_verlet<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(n, pos, vel, forces, half_dt_a, dt,
                                                                phase == 0 ? 1 : 0, w);
  return cudaGetLastError() == cudaSuccess ? BOP_OK : BOP_ERR_CUDA;
}
