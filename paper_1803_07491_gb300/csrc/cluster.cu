// Hop levels of (atom, image) sites around every atom: the support of the
// self-returning paths of Eq. momDOS (C_0 = {i}, C_k = C_{k-1} plus all
// neighbours of C_{k-1}, inside the path radius when one is set:
// "Performance", item (iii)), with the adjacency between cluster sites that
// the moments kernels walk.
//
// Canonical order (reproducible bit for bit): level, then atom, then image
// (sx, sy, sz).  Each site's adjacency lists every neighbour inside the
// cluster as {local index, bond}, ascending local index.
//
// One CTA per atom (grid-stride), a hash table of site keys in per-CTA
// global scratch, the new sites of a level sorted in shared memory.
#include "kernels.h"

namespace {

constexpr unsigned long long EMPTY = ~0ull;
constexpr int CL_THREADS = 256;

__device__ __forceinline__ unsigned long long site_key(int atom, int sx, int sy, int sz) {
  return ((unsigned long long)(unsigned)atom << 24) | ((unsigned long long)(sx + 128) << 16) |
         ((unsigned long long)(sy + 128) << 8) | (unsigned long long)(sz + 128);
}
__device__ __forceinline__ int key_atom(unsigned long long k) { return (int)(k >> 24); }
__device__ __forceinline__ int key_img(unsigned long long k, int c) {
  return (int)((k >> (16 - 8 * c)) & 0xff) - 128;
}
__device__ __forceinline__ unsigned hash_slot(unsigned long long k, int mask) {
  unsigned long long x = k * 0x9E3779B97F4A7C15ull;
  return (unsigned)(x >> 32) & (unsigned)mask;
}

// Find key; returns slot or -1.  Bounded by the table size.
__device__ int h_find(const unsigned long long* __restrict__ hk, int hcap, unsigned long long key) {
  unsigned s = hash_slot(key, hcap - 1);
  for (int probe = 0; probe < hcap; probe++) {
    unsigned long long c = hk[s];
    if (c == key) return (int)s;
    if (c == EMPTY) return -1;
    s = (s + 1) & (hcap - 1);
  }
  return -1;
}

// Insert key if absent.  Returns 1 if this call inserted it, 0 if present,
// -1 if the table is full.
__device__ int h_insert(unsigned long long* hk, int hcap, unsigned long long key) {
  unsigned s = hash_slot(key, hcap - 1);
  for (int probe = 0; probe < hcap; probe++) {
    unsigned long long c = hk[s];
    if (c == key) return 0;
    if (c == EMPTY) {
      unsigned long long prev = atomicCAS(&hk[s], EMPTY, key);
      if (prev == EMPTY) return 1;
      if (prev == key) return 0;
    }
    s = (s + 1) & (hcap - 1);
  }
  return -1;
}

__device__ void block_sort_u64(unsigned long long* a, int cnt) {
  int P = 1;
  while (P < cnt) P <<= 1;
  for (int i = cnt + threadIdx.x; i < P; i += blockDim.x) a[i] = EMPTY;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          bool up = (i & k) == 0;
          unsigned long long x = a[i], y = a[ixj];
          if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
}

// Exclusive scan of v[0..cnt) in place (chunks of blockDim), returns total.
__device__ int block_exclusive_scan(int* v, int cnt, int* warp_tmp) {
  int carry = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < cnt; base += blockDim.x) {
    int i = base + threadIdx.x;
    int x = i < cnt ? v[i] : 0;
    int incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tmp[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int q = 0; q < nw; q++) {
        int t = warp_tmp[q];
        warp_tmp[q] = acc;
        acc += t;
      }
      warp_tmp[nw] = acc;
    }
    __syncthreads();
    if (i < cnt) v[i] = carry + warp_tmp[wid] + incl - x;
    carry += warp_tmp[nw];
    __syncthreads();
  }
  return carry;
}

template <int PASS, bool CUT>
__global__ void __launch_bounds__(CL_THREADS)
k_cluster(int n, int K, const long long* __restrict__ row_ptr, const int* __restrict__ col,
          const signed char* __restrict__ img, const int* __restrict__ bond_of_edge, PathCut pc, ClusterScratch sc,
          ClusterOut out, unsigned* __restrict__ status) {
  extern __shared__ unsigned long long newkeys[];  // [newcap], a power of two
  __shared__ int s_count, s_fail;
  __shared__ int s_lev[BOP_MAX_K + 1];
  __shared__ int warp_tmp[CL_THREADS / 32 + 1];
  unsigned long long* hk = sc.hkeys + (size_t)blockIdx.x * sc.hcap;
  int* hv = sc.hvals + (size_t)blockIdx.x * sc.hcap;
  unsigned long long* sk = sc.skeys + (size_t)blockIdx.x * sc.maxs;
  int* ss = sc.sslot + (size_t)blockIdx.x * sc.maxs;
  int* scnt = sc.scount + (size_t)blockIdx.x * sc.maxs;

  for (int atom = blockIdx.x; atom < n; atom += gridDim.x) {
    if (threadIdx.x == 0) {
      unsigned long long k0 = site_key(atom, 0, 0, 0);
      h_insert(hk, sc.hcap, k0);
      int sl = h_find(hk, sc.hcap, k0);
      s_fail = 0;
      if (sl < 0) {
        s_fail = 1;
        raise_error(status, BOP_DEV_ERR_CLUSTER);
        sl = 0;
      }
      hv[sl] = 0;
      sk[0] = k0;
      ss[0] = sl;
      s_lev[0] = 1;
    }
    __syncthreads();
    int nsite = 1;
    for (int k = 1; k <= K; k++) {
      if (threadIdx.x == 0) s_count = 0;
      __syncthreads();
      int f0 = k >= 2 ? s_lev[k - 2] : 0, f1 = s_lev[k - 1];
      for (int t = f0 + threadIdx.x; t < f1; t += blockDim.x) {
        unsigned long long kt = sk[t];
        int a = key_atom(kt);
        int ix = key_img(kt, 0), iy = key_img(kt, 1), iz = key_img(kt, 2);
        for (long long e = row_ptr[a]; e < row_ptr[a + 1]; e++) {
          int sx = ix + img[3 * e], sy = iy + img[3 * e + 1], sz = iz + img[3 * e + 2];
          if (sx < -127 || sx > 127 || sy < -127 || sy > 127 || sz < -127 || sz > 127) {
            s_fail = 1;
            raise_error(status, BOP_DEV_ERR_IMAGE);
            continue;
          }
          if (CUT) {  // path-radius cut: only sites closer than r_path to the atom
            double d[3];
            bond_vector(pc.pos + 3 * (size_t)atom, pc.pos + 3 * (size_t)col[e], pc.cell, sx, sy, sz, d);
            if (!(norm2_rn(d) < pc.r2)) continue;
          }
          unsigned long long key = site_key(col[e], sx, sy, sz);
          int r = h_insert(hk, sc.hcap, key);
          if (r == 1) {
            int q = atomicAdd(&s_count, 1);
            if (q < sc.newcap) newkeys[q] = key;
          } else if (r < 0) {
            s_fail = 1;
            raise_error(status, BOP_DEV_ERR_CLUSTER);
          }
        }
      }
      __syncthreads();
      int cnt = s_count;
      if (cnt > sc.newcap || nsite + cnt > sc.maxs) {
        if (threadIdx.x == 0) {
          s_fail = 1;
          raise_error(status, BOP_DEV_ERR_CLUSTER);
        }
        __syncthreads();
        cnt = 0;
      }
      if (s_fail) break;
      block_sort_u64(newkeys, cnt);
      for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        unsigned long long key = newkeys[q];
        int sl = h_find(hk, sc.hcap, key);
        if (sl < 0) {  // cannot happen for a key this level inserted; never index with it
          raise_error(status, BOP_DEV_ERR_CLUSTER);
          sl = 0;
        }
        hv[sl] = nsite + q;
        sk[nsite + q] = key;
        ss[nsite + q] = sl;
      }
      nsite += cnt;
      if (threadIdx.x == 0) s_lev[k] = nsite;
      __syncthreads();
    }
    __syncthreads();
    const bool ok = !s_fail;
    if (ok) {
      // adjacency: every neighbour inside the cluster (counts first)
      for (int t = threadIdx.x; t < nsite; t += blockDim.x) {
        unsigned long long kt = sk[t];
        int a = key_atom(kt);
        int ix = key_img(kt, 0), iy = key_img(kt, 1), iz = key_img(kt, 2);
        int c = 0;
        for (long long e = row_ptr[a]; e < row_ptr[a + 1]; e++) {
          int sx = ix + img[3 * e], sy = iy + img[3 * e + 1], sz = iz + img[3 * e + 2];
          if (sx < -127 || sx > 127 || sy < -127 || sy > 127 || sz < -127 || sz > 127) continue;
          if (h_find(hk, sc.hcap, site_key(col[e], sx, sy, sz)) >= 0) c++;
        }
        scnt[t] = c < BOP_MAX_DEG ? c : BOP_MAX_DEG;
      }
      __syncthreads();
      if (PASS == 0) {
        int tot = block_exclusive_scan(scnt, nsite, warp_tmp);
        if (threadIdx.x == 0) {
          out.atom_nsite[atom] = nsite;
          out.atom_nadj[atom] = tot;
          atomicMax(&out.max_level[K + 1], tot);  // largest adjacency
        }
        for (int k = threadIdx.x; k <= K; k += blockDim.x) {
          out.level_end[(size_t)atom * (K + 1) + k] = s_lev[k];
          atomicMax(&out.max_level[k], s_lev[k]);
        }
      } else {
        block_exclusive_scan(scnt, nsite, warp_tmp);
        long long s0 = out.site_off[atom], a0 = out.adj_base[atom];
        unsigned long long prod = 0;
        for (int t = threadIdx.x; t < nsite; t += blockDim.x) {
          unsigned long long kt = sk[t];
          out.site_atom[s0 + t] = key_atom(kt);
          out.site_img[3 * (s0 + t)] = (signed char)key_img(kt, 0);
          out.site_img[3 * (s0 + t) + 1] = (signed char)key_img(kt, 1);
          out.site_img[3 * (s0 + t) + 2] = (signed char)key_img(kt, 2);
          out.adj_off[s0 + t] = a0 + scnt[t];
          // recompute and write the sorted entries
          int a = key_atom(kt);
          int ix = key_img(kt, 0), iy = key_img(kt, 1), iz = key_img(kt, 2);
          int2 ent[BOP_MAX_DEG];
          int c = 0;
          for (long long e = row_ptr[a]; e < row_ptr[a + 1]; e++) {
            int sx = ix + img[3 * e], sy = iy + img[3 * e + 1], sz = iz + img[3 * e + 2];
            if (sx < -127 || sx > 127 || sy < -127 || sy > 127 || sz < -127 || sz > 127) continue;
            int sl = h_find(hk, sc.hcap, site_key(col[e], sx, sy, sz));
            if (sl < 0) continue;
            if (c < BOP_MAX_DEG) ent[c] = make_int2(hv[sl], bond_of_edge[e]);
            c++;
          }
          if (c > BOP_MAX_DEG) c = BOP_MAX_DEG;
          for (int x = 1; x < c; x++) {
            int2 v = ent[x];
            int y = x - 1;
            while (y >= 0 && ent[y].x > v.x) {
              ent[y + 1] = ent[y];
              y--;
            }
            ent[y + 1] = v;
          }
          long long o = a0 + scnt[t];
          for (int x = 0; x < c; x++) out.adj[o + x] = ent[x];
          // byte k: entries whose site lies in C_k (the gather of level k+1)
          unsigned long long lc = 0;
          for (int k = 0; k < K; k++) {
            unsigned cnt = 0;
            while ((int)cnt < c && ent[cnt].x < s_lev[k]) cnt++;
            lc |= (unsigned long long)cnt << (8 * k);
          }
          out.lvcnt[s0 + t] = lc;
          // forward levels k = max(lt, ls+1) .. K use the pair (t, s)
          int lt = 0;
          while (lt < K && t >= s_lev[lt]) lt++;
          for (int x = 0; x < c; x++) {
            int ls = 0;
            while (ls < K && ent[x].x >= s_lev[ls]) ls++;
            int k0 = lt > ls + 1 ? lt : ls + 1;
            if (k0 <= K) prod += (unsigned long long)(K - k0 + 1);
          }
        }
        if (prod) atomicAdd(out.n_products, prod);
      }
    } else if (PASS == 0 && threadIdx.x == 0) {
      out.atom_nsite[atom] = 0;
      out.atom_nadj[atom] = 0;
    }
    __syncthreads();
    // clear the hash table: every inserted key became a site (or the atom failed)
    for (int t = threadIdx.x; t < nsite; t += blockDim.x) {
      hk[ss[t]] = EMPTY;
    }
    if (!ok) {  // a failed atom may have left keys that never became sites
      for (int q = threadIdx.x; q < sc.hcap; q += blockDim.x) hk[q] = EMPTY;
    }
    __syncthreads();
  }
}

}  // namespace

int launch_cluster(int pass, int n, int K, const long long* row_ptr, const int* col, const signed char* img,
                   const int* bond_of_edge, PathCut pc, ClusterScratch sc, ClusterOut out, int grid,
                   unsigned* status, cudaStream_t s) {
  size_t smem = (size_t)sc.newcap * sizeof(unsigned long long);  // newcap is a power of two
  // the path cut is a separate instantiation: its distance arithmetic costs
  // registers that the uncut BFS does not need
  const bool cut = pc.r2 > 0.0;
  auto fn = pass == 0 ? (cut ? k_cluster<0, true> : k_cluster<0, false>)
                      : (cut ? k_cluster<1, true> : k_cluster<1, false>);
  if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  fn<<<grid, CL_THREADS, smem, s>>>(n, K, row_ptr, col, img, bond_of_edge, pc, sc, out, status);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Rows of one stored Psi sweep per atom: sum_{k=0..K} |C_k|.
__global__ void k_level_sums(int n, int K, const int* __restrict__ level_end, long long* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long a = 0;
  for (int k = 0; k <= K; k++) a += level_end[(size_t)i * (K + 1) + k];
  out[i] = a;
}

void launch_level_sums(int n, int K, const int* level_end, long long* out, cudaStream_t s) {
  k_level_sums<<<(n + 255) / 256, 256, 0, s>>>(n, K, level_end, out);
}
