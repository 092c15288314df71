// Short-range neighbour list (linked cells, "Initialisation" of the paper's
// program flow) and the canonical undirected bond list with its two-centre
// blocks (Eq. Hij, Eq. cutoff, Eq. Hij_rot).
//
// Output order is fixed so that the integer arrays are reproducible bit for
// bit: each CSR row of atom i lists (j, sx, sy, sz) in ascending
// lexicographic order; a pair is kept iff r2 < rc*rc with the FP64
// arithmetic of bond_vector()/norm2_rn().
#include "kernels.h"

namespace bopk {

// Fractional coordinates f = pos * inv(cell) (rows of cell = lattice vectors)
// and the linked-cell index of every atom.
__global__ void k_bin_atoms(int n, const double* __restrict__ pos, Geometry g, int* __restrict__ cell_of,
                            int* __restrict__ cell_count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c3[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    double f = pos[3 * i] * g.inv[0 * 3 + a] + pos[3 * i + 1] * g.inv[1 * 3 + a] + pos[3 * i + 2] * g.inv[2 * 3 + a];
    int c = (int)floor(f * g.nc[a]);
    c = c < 0 ? 0 : (c >= g.nc[a] ? g.nc[a] - 1 : c);
    c3[a] = c;
  }
  int c = (c3[0] * g.nc[1] + c3[1]) * g.nc[2] + c3[2];
  cell_of[i] = c;
  atomicAdd(&cell_count[c], 1);
}

__global__ void k_fill_cells(int n, const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                             int* __restrict__ cell_fill, int* __restrict__ cell_atoms) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cell_of[i];
  int slot = atomicAdd(&cell_fill[c], 1);
  cell_atoms[cell_start[c] + slot] = i;
}

// Candidate ranges along one axis: with nc >= 3 the three adjacent cells
// (wrapped, image = floor division); with fewer cells, every cell with
// every image in [-nimg, nimg].
struct AxisIter {
  int count;
  __device__ void get(const Geometry& g, int a, int c, int q, int* cell, int* img) const {
    if (g.nc[a] >= 3) {
      int cc = c + q - 1;
      int im = 0;
      if (cc < 0) { cc += g.nc[a]; im = -1; }
      if (cc >= g.nc[a]) { cc -= g.nc[a]; im = 1; }
      *cell = cc;
      *img = im;
    } else {
      *cell = q % g.nc[a];
      *img = q / g.nc[a] - g.nimg[a];
    }
  }
};

__device__ __forceinline__ int axis_count(const Geometry& g, int a) {
  return g.nc[a] >= 3 ? 3 : g.nc[a] * (2 * g.nimg[a] + 1);
}

__device__ __forceinline__ bool axis_valid(const Geometry& g, int a, int c, int q) {
  // non-periodic axes: no wrap, no images
  if (g.pbc[a]) return true;
  if (g.nc[a] >= 3) {
    int cc = c + q - 1;
    return cc >= 0 && cc < g.nc[a];
  }
  return q / g.nc[a] - g.nimg[a] == 0;
}

__device__ __forceinline__ uint64_t nbr_key(int j, int sx, int sy, int sz) {
  return ((uint64_t)(uint32_t)j << 24) | ((uint64_t)(sx + 128) << 16) | ((uint64_t)(sy + 128) << 8) |
         (uint64_t)(sz + 128);
}

// One warp per atom.  The candidate cells (27, or more along axes with
// fewer than three cells) are enumerated 32 at a time, one per lane, with
// their atom ranges; a warp scan of the range lengths flattens their atoms
// into one candidate list that the lanes test 32 at a time, so a warp waits
// on a few rounds of loads instead of one round per cell.  Hits go to a
// per-warp list in shared memory in ballot order.  mode 0: count
// neighbours; mode 1: every entry's rank among the keys (j, sx, sy, sz)
// gives its slot in the sorted row.
constexpr int NBR_WARPS = 4;

template <int MODE>
__global__ void __launch_bounds__(32 * NBR_WARPS)
k_neighbors(int n, const double* __restrict__ pos, Geometry g, const int* __restrict__ cell_of,
            const int* __restrict__ cell_start, const int* __restrict__ cell_atoms, int* __restrict__ deg,
            const long long* __restrict__ row_ptr, int* __restrict__ col, signed char* __restrict__ img,
            unsigned* __restrict__ status) {
  __shared__ uint64_t skeys[NBR_WARPS][BOP_MAX_DEG];
  __shared__ int s_start[NBR_WARPS][32], s_pre[NBR_WARPS][33], s_img[NBR_WARPS][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int i = blockIdx.x * NBR_WARPS + wib;
  if (i >= n) return;  // whole warp
  const double rc2 = g.rc * g.rc;
  const double pi[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
  const int ci = cell_of[i];
  const int c3[3] = {ci / (g.nc[1] * g.nc[2]), (ci / g.nc[2]) % g.nc[1], ci % g.nc[2]};
  const unsigned lt_mask = (1u << lane) - 1u;
  int cnt = 0;
  const int n0 = axis_count(g, 0), n1 = axis_count(g, 1), n2 = axis_count(g, 2);
  const int ncand = n0 * n1 * n2;
  if (lane == 0) s_pre[wib][0] = 0;
  for (int cb = 0; cb < ncand; cb += 32) {
    const int q = cb + lane;
    int len = 0, start = 0, im = 0;
    if (q < ncand) {
      const int q0 = q / (n1 * n2), q1 = (q / n2) % n1, q2 = q % n2;
      if (axis_valid(g, 0, c3[0], q0) && axis_valid(g, 1, c3[1], q1) && axis_valid(g, 2, c3[2], q2)) {
        int cx, cy, cz, sx, sy, sz;
        AxisIter it;
        it.get(g, 0, c3[0], q0, &cx, &sx);
        it.get(g, 1, c3[1], q1, &cy, &sy);
        it.get(g, 2, c3[2], q2, &cz, &sz);
        const int cc = (cx * g.nc[1] + cy) * g.nc[2] + cz;
        start = cell_start[cc];
        len = cell_start[cc + 1] - start;
        im = ((sx + 128) << 16) | ((sy + 128) << 8) | (sz + 128);
      }
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    s_start[wib][lane] = start;
    s_pre[wib][lane + 1] = incl;
    s_img[wib][lane] = im;
    __syncwarp();
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    for (int base = 0; base < tot; base += 32) {
      const int p = base + lane;
      bool hit = false;
      uint64_t key = 0;
      if (p < tot) {
        int lo = 0, hi = 31;  // the candidate cell c with s_pre[c] <= p < s_pre[c + 1]
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_pre[wib][mid] <= p) lo = mid;
          else hi = mid - 1;
        }
        const int j = cell_atoms[s_start[wib][lo] + (p - s_pre[wib][lo])];
        const int code = s_img[wib][lo];
        const int sx = ((code >> 16) & 0xff) - 128, sy = ((code >> 8) & 0xff) - 128, sz = (code & 0xff) - 128;
        if (!(j == i && sx == 0 && sy == 0 && sz == 0)) {
          double d[3];
          bond_vector(pi, pos + 3 * j, g.cell, sx, sy, sz, d);
          hit = norm2_rn(d) < rc2;
          key = nbr_key(j, sx, sy, sz);
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const int slot = cnt + __popc(bal & lt_mask);
        if (slot < BOP_MAX_DEG) skeys[wib][slot] = key;
      }
      cnt += __popc(bal);
    }
    __syncwarp();
  }
  if (MODE == 0) {
    if (lane == 0) {
      deg[i] = cnt;
      if (cnt > BOP_MAX_DEG) raise_error(status, BOP_DEV_ERR_DEGREE);
    }
    return;
  }
  if (cnt > BOP_MAX_DEG) return;
  __syncwarp();
  const long long e0 = row_ptr[i];
  for (int a = lane; a < cnt; a += 32) {
    const uint64_t k = skeys[wib][a];
    int rank = 0;
    for (int b = 0; b < cnt; b++) rank += skeys[wib][b] < k ? 1 : 0;
    const long long e = e0 + rank;
    col[e] = (int)(k >> 24);
    img[3 * e] = (signed char)((int)((k >> 16) & 0xff) - 128);
    img[3 * e + 1] = (signed char)((int)((k >> 8) & 0xff) - 128);
    img[3 * e + 2] = (signed char)((int)(k & 0xff) - 128);
  }
}

// Canonical orientation of a directed edge i->(j,S): i < j, or i == j and
// S > 0 lexicographically.
__device__ __forceinline__ bool canonical(int i, int j, const signed char* s) {
  if (i != j) return i < j;
  if (s[0] != 0) return s[0] > 0;
  if (s[1] != 0) return s[1] > 0;
  return s[2] > 0;
}

__global__ void k_edge_flags(int n, const long long* __restrict__ row_ptr, const int* __restrict__ col,
                             const signed char* __restrict__ img, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (long long e = row_ptr[i]; e < row_ptr[i + 1]; e++) flag[e] = canonical(i, col[e], img + 3 * e) ? 1 : 0;
}

// bond_of_edge for every directed edge (the reverse edge of a
// non-canonical one is found by binary search in row j), and the bond's
// end atoms and image.
__global__ void k_bonds(int n, const long long* __restrict__ row_ptr, const int* __restrict__ col,
                        const signed char* __restrict__ img, const int* __restrict__ flag,
                        const int* __restrict__ bond_scan, int* __restrict__ bond_of_edge,
                        int* __restrict__ bond_atoms, signed char* __restrict__ bond_img,
                        unsigned* __restrict__ status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (long long e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
    int j = col[e];
    const signed char* s = img + 3 * e;
    if (flag[e]) {
      int b = bond_scan[e];
      bond_of_edge[e] = b;
      bond_atoms[2 * b] = i;
      bond_atoms[2 * b + 1] = j;
      bond_img[3 * b] = s[0];
      bond_img[3 * b + 1] = s[1];
      bond_img[3 * b + 2] = s[2];
    } else {
      uint64_t want = nbr_key(i, -s[0], -s[1], -s[2]);
      long long lo = row_ptr[j], hi = row_ptr[j + 1] - 1, found = -1;
      while (lo <= hi) {
        long long mid = (lo + hi) >> 1;
        const signed char* t = img + 3 * mid;
        uint64_t k = nbr_key(col[mid], t[0], t[1], t[2]);
        if (k == want) { found = mid; break; }
        if (k < want) lo = mid + 1; else hi = mid - 1;
      }
      if (found < 0) {
        raise_error(status, BOP_DEV_ERR_REVERSE);
        bond_of_edge[e] = 0;
      } else {
        bond_of_edge[e] = bond_scan[found];
      }
    }
  }
}

// Bond vectors and unique block elements of every canonical bond.
__global__ void k_bond_blocks(int nb, const double* __restrict__ pos, Geometry g, BondModel m,
                              const int* __restrict__ bond_atoms, const signed char* __restrict__ bond_img,
                              double* __restrict__ bond_d, double* __restrict__ H64, float* __restrict__ H32,
                              int HS) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  int i = bond_atoms[2 * b], j = bond_atoms[2 * b + 1];
  const signed char* s = bond_img + 3 * b;
  double d[3];
  bond_vector(pos + 3 * i, pos + 3 * j, g.cell, s[0], s[1], s[2], d);
  bond_d[3 * b] = d[0];
  bond_d[3 * b + 1] = d[1];
  bond_d[3 * b + 2] = d[2];
  double u[21];
  sk_unique<double>(m, d, u);
  const int nu = block_unique(m.norb);
  for (int q = 0; q < HS; q++) {
    double v = q < nu ? u[q] : 0.0;
    H64[(size_t)b * HS + q] = v;
    H32[(size_t)b * HS + q] = (float)v;
  }
}

// Largest / smallest fractional coordinate along each axis (validation that
// all atoms lie inside the cell; a non-finite coordinate makes the range
// infinite, which fmin / fmax alone would skip).
__global__ void k_frac_range(int n, const double* __restrict__ pos, Geometry g, double* __restrict__ out) {
  __shared__ double smin[3][256], smax[3][256];
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int a = 0; a < 3; a++) {
      double f = pos[3 * i] * g.inv[a] + pos[3 * i + 1] * g.inv[3 + a] + pos[3 * i + 2] * g.inv[6 + a];
      if (!isfinite(f)) {  // a NaN / Inf position: both ends of the range become infinite
        mn[a] = -INFINITY;
        mx[a] = INFINITY;
      }
      mn[a] = fmin(mn[a], f);
      mx[a] = fmax(mx[a], f);
    }
  }
  for (int a = 0; a < 3; a++) {
    smin[a][threadIdx.x] = mn[a];
    smax[a][threadIdx.x] = mx[a];
  }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int a = 0; a < 3; a++) {
        smin[a][threadIdx.x] = fmin(smin[a][threadIdx.x], smin[a][threadIdx.x + w]);
        smax[a][threadIdx.x] = fmax(smax[a][threadIdx.x], smax[a][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; a++) {
      out[6 * blockIdx.x + a] = smin[a][0];
      out[6 * blockIdx.x + 3 + a] = smax[a][0];
    }
}

}  // namespace bopk

void launch_neighbors(int mode, int n, const double* pos, Geometry g, const int* cell_of, const int* cell_start,
                      const int* cell_atoms, int* deg, const long long* row_ptr, int* col, signed char* img,
                      unsigned* status, cudaStream_t s) {
  const int TB = 32 * bopk::NBR_WARPS, gb = (n + bopk::NBR_WARPS - 1) / bopk::NBR_WARPS;
  if (mode == 0)
    bopk::k_neighbors<0><<<gb, TB, 0, s>>>(n, pos, g, cell_of, cell_start, cell_atoms, deg, row_ptr, col, img,
                                           status);
  else
    bopk::k_neighbors<1><<<gb, TB, 0, s>>>(n, pos, g, cell_of, cell_start, cell_atoms, deg, row_ptr, col, img,
                                           status);
}
