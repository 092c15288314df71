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

// ---------------------------------------------------------------- warp builder
// The same clusters (same canonical order, same adjacency and level counts)
// with one warp per atom: a cluster of a few hundred sites has levels of
// 1, 14, 50, 110, ... new sites, which a warp covers without block-wide
// barriers, and every hash probe stays in shared memory.  Pass 0 runs the
// breadth-first search, counts the adjacency and keeps each atom's site
// keys in global scratch; pass 1 reloads them, fills the hash table and
// writes the sites, the sorted adjacency and the level counts.  Clusters of
// more than CW_MAXS sites, or atoms with more than MAXD neighbours, raise
// *wfail and the caller falls back to the block builder above.
constexpr int CW_WARPS = 3;   // warps per CTA (five CTAs of 14 KB per warp fit an SM)
constexpr int CW_MAXS = 512;  // sites of one cluster
constexpr int CW_NB = 256;    // new sites of one level
constexpr int CW_HC = 1024;   // hash slots per warp (a power of two, 2 CW_MAXS)
// A hash entry is the 48-bit site key with the site's local index + 1 in
// the top 16 bits (0 while the index is not yet assigned).
constexpr unsigned long long CW_KEY = (1ull << 48) - 1;

struct CwSmem {
  unsigned long long hk[CW_HC];
  unsigned long long sk[CW_MAXS];  // site keys in canonical order
  unsigned long long nb[CW_NB];    // new keys of one level
  int lev[BOP_MAX_K + 1];
  int cnt, fail;
};

__device__ __forceinline__ int cw_find(const unsigned long long* hk, unsigned long long key) {
  unsigned s = hash_slot(key, CW_HC - 1);
  for (int probe = 0; probe < CW_HC; probe++) {
    const unsigned long long c = hk[s];
    if (c == EMPTY) return -1;
    if ((c & CW_KEY) == key) return (int)s;
    s = (s + 1) & (CW_HC - 1);
  }
  return -1;
}

__device__ __forceinline__ int cw_index(const unsigned long long* hk, int slot) {
  return (int)(hk[slot] >> 48) - 1;
}

// 1: inserted (index unassigned), 0: present, -1: full.  slot receives the
// key's slot.
__device__ __forceinline__ int cw_insert(unsigned long long* hk, unsigned long long key, int* slot) {
  unsigned s = hash_slot(key, CW_HC - 1);
  for (int probe = 0; probe < CW_HC; probe++) {
    const unsigned long long c = hk[s];
    if (c != EMPTY && (c & CW_KEY) == key) {
      *slot = (int)s;
      return 0;
    }
    if (c == EMPTY) {
      const unsigned long long prev = atomicCAS(&hk[s], EMPTY, key);
      if (prev == EMPTY) {
        *slot = (int)s;
        return 1;
      }
      if ((prev & CW_KEY) == key) {
        *slot = (int)s;
        return 0;
      }
    }
    s = (s + 1) & (CW_HC - 1);
  }
  return -1;
}

// Ascending bitonic sort of a[0..cnt) by one warp, padded with EMPTY to the
// next power of two (at most CW_NB).
__device__ __forceinline__ void cw_sort(unsigned long long* a, int cnt, int lane) {
  int P = 1;
  while (P < cnt) P <<= 1;
  for (int i = cnt + lane; i < P; i += 32) a[i] = EMPTY;
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long x = a[i], y = a[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncwarp();
    }
}

// Image of a packed edge record: byte c of y holds image component c + 128.
__device__ __forceinline__ int epk_img(int y, int c) { return (int)(((unsigned)y >> (8 * c)) & 0xffu) - 128; }

template <int PASS, bool CUT, int MAXD>
__global__ void __launch_bounds__(32 * CW_WARPS, MAXD <= 16 ? 5 : 2)
k_cluster_warp(int n, int K, const long long* __restrict__ row_ptr, const int2* __restrict__ epack,
               const int* __restrict__ bond_of_edge, PathCut pc,
               unsigned long long* __restrict__ gkeys, ClusterOut out, int* __restrict__ wfail,
               unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char cw_raw[];
  CwSmem& sm = reinterpret_cast<CwSmem*>(cw_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * CW_WARPS;
  for (int atom = blockIdx.x * CW_WARPS + (threadIdx.x >> 5); atom < n; atom += nwarps) {
    for (int q = lane; q < CW_HC; q += 32) sm.hk[q] = EMPTY;
    if (lane == 0) {
      sm.fail = 0;
      sm.cnt = 0;
    }
    __syncwarp();
    unsigned long long* gk = gkeys + (size_t)atom * CW_MAXS;
    int nsite;
    if (PASS == 0) {
      // breadth-first search over hop levels
      if (lane == 0) {
        const unsigned long long k0 = site_key(atom, 0, 0, 0);
        int sl = 0;
        cw_insert(sm.hk, k0, &sl);
        sm.hk[sl] = k0 | (1ull << 48);
        sm.sk[0] = k0;
        sm.lev[0] = 1;
      }
      __syncwarp();
      nsite = 1;
      for (int k = 1; k <= K; k++) {
        const int f0 = k >= 2 ? sm.lev[k - 2] : 0, f1 = sm.lev[k - 1];
        for (int t = f0 + lane; t < f1; t += 32) {
          const unsigned long long kt = sm.sk[t];
          const int a = key_atom(kt);
          const int ix = key_img(kt, 0), iy = key_img(kt, 1), iz = key_img(kt, 2);
          const long long e0 = row_ptr[a];
          int deg = (int)(row_ptr[a + 1] - e0);
          if (deg > MAXD) {
            atomicOr(wfail, 2);
            deg = MAXD;
          }
          int2 pe[MAXD];  // the atom's edges, all loads in flight together
#pragma unroll
          for (int j = 0; j < MAXD; j++)
            if (j < deg) pe[j] = __ldg(epack + e0 + j);
#pragma unroll
          for (int j = 0; j < MAXD; j++) {
            if (j >= deg) continue;
            const int sx = ix + epk_img(pe[j].y, 0), sy = iy + epk_img(pe[j].y, 1), sz = iz + epk_img(pe[j].y, 2);
            if (sx < -127 || sx > 127 || sy < -127 || sy > 127 || sz < -127 || sz > 127) {
              sm.fail = 1;
              raise_error(status, BOP_DEV_ERR_IMAGE);
              continue;
            }
            if (CUT) {
              double d[3];
              bond_vector(pc.pos + 3 * (size_t)atom, pc.pos + 3 * (size_t)pe[j].x, pc.cell, sx, sy, sz, d);
              if (!(norm2_rn(d) < pc.r2)) continue;
            }
            const unsigned long long key = site_key(pe[j].x, sx, sy, sz);
            int sl = 0;
            const int r = cw_insert(sm.hk, key, &sl);
            if (r == 1) {
              const int q = atomicAdd(&sm.cnt, 1);
              if (q < CW_NB) sm.nb[q] = key;
            } else if (r < 0) {
              sm.fail = 1;
            }
          }
        }
        __syncwarp();
        const int cnt = sm.cnt;
        if (cnt > CW_NB || cnt > CW_MAXS - nsite) sm.fail = 1;
        __syncwarp();
        if (sm.fail) break;
        // canonical order inside the level: the new keys sorted
        cw_sort(sm.nb, cnt, lane);
        for (int q = lane; q < cnt; q += 32) {
          const unsigned long long key = sm.nb[q];
          sm.sk[nsite + q] = key;
          const int sl = cw_find(sm.hk, key);
          if (sl >= 0) sm.hk[sl] = key | ((unsigned long long)(nsite + q + 1) << 48);
        }
        __syncwarp();
        nsite += cnt;
        if (lane == 0) {
          sm.lev[k] = nsite;
          sm.cnt = 0;
        }
        __syncwarp();
      }
      if (sm.fail) {
        if (lane == 0) {
          atomicOr(wfail, 1);
          out.atom_nsite[atom] = 0;
          out.atom_nadj[atom] = 0;
        }
        __syncwarp();
        continue;
      }
      for (int t = lane; t < nsite; t += 32) gk[t] = sm.sk[t];
    } else {
      // pass 1: the keys of pass 0 (canonical order) and the level ends
      for (int k = lane; k <= K; k += 32) sm.lev[k] = out.level_end[(size_t)atom * (K + 1) + k];
      __syncwarp();
      nsite = sm.lev[K];
      for (int t = lane; t < nsite; t += 32) {
        const unsigned long long key = gk[t];
        sm.sk[t] = key;
        int sl = 0;
        cw_insert(sm.hk, key, &sl);
        sm.hk[sl] = key | ((unsigned long long)(t + 1) << 48);
      }
      __syncwarp();
    }
    // adjacency of every site: the neighbours inside the cluster, by local index
    const long long s0 = PASS == 1 ? out.site_off[atom] : 0;
    const long long a0 = PASS == 1 ? out.adj_base[atom] : 0;
    int run = 0;
    unsigned long long prod = 0;
    for (int tb = 0; tb < nsite; tb += 32) {
      const int t = tb + lane;
      unsigned long long ent[MAXD];
      int deg = 0, c = 0;
      int lt = 0;
      if (t < nsite) {
        const unsigned long long kt = sm.sk[t];
        const int a = key_atom(kt);
        const int ix = key_img(kt, 0), iy = key_img(kt, 1), iz = key_img(kt, 2);
        const long long e0 = row_ptr[a];
        deg = (int)(row_ptr[a + 1] - e0);
        if (deg > MAXD) {
          atomicOr(wfail, 2);
          deg = MAXD;
        }
        // without a path cut every neighbour of a site within K-1 hops is in
        // the cluster: pass 0 counts those without looking them up
        const bool inner = !CUT && PASS == 0 && t < sm.lev[K > 0 ? K - 1 : 0] && K > 0;
        if (inner) {
          c = deg;
#pragma unroll
          for (int j = 0; j < MAXD; j++) ent[j] = ~0ull;
        } else {
          int2 pe[MAXD];
          int bnd[MAXD];
#pragma unroll
          for (int j = 0; j < MAXD; j++) {
            if (j < deg) {
              pe[j] = __ldg(epack + e0 + j);
              bnd[j] = PASS == 1 ? __ldg(bond_of_edge + e0 + j) : 0;
            }
          }
#pragma unroll
          for (int j = 0; j < MAXD; j++) {
            ent[j] = ~0ull;
            if (j < deg) {
              const int sx = ix + epk_img(pe[j].y, 0), sy = iy + epk_img(pe[j].y, 1), sz = iz + epk_img(pe[j].y, 2);
              if (sx >= -127 && sx <= 127 && sy >= -127 && sy <= 127 && sz >= -127 && sz <= 127) {
                const int sl = cw_find(sm.hk, site_key(pe[j].x, sx, sy, sz));
                if (sl >= 0) {
                  ent[j] = ((unsigned long long)cw_index(sm.hk, sl) << 32) | (unsigned)bnd[j];
                  c++;
                }
              }
            }
          }
        }
        while (lt < K && t >= sm.lev[lt]) lt++;
      }
      // offsets of this chunk's rows
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int off = run + incl - c;
      run += __shfl_sync(0xffffffffu, incl, 31);
      if (PASS == 1 && t < nsite) {
        const unsigned long long kt = sm.sk[t];
        out.site_atom[s0 + t] = key_atom(kt);
        out.site_img[3 * (s0 + t)] = (signed char)key_img(kt, 0);
        out.site_img[3 * (s0 + t) + 1] = (signed char)key_img(kt, 1);
        out.site_img[3 * (s0 + t) + 2] = (signed char)key_img(kt, 2);
        out.adj_off[s0 + t] = a0 + off;
        // level ends in registers (levels above K never match)
        int lv[BOP_MAX_K];
#pragma unroll
        for (int k = 0; k < BOP_MAX_K; k++) lv[k] = k < K ? sm.lev[k] : 0x7fffffff;
        // the entries' local indices (distinct within a site; unused entries
        // 0xffffffff): the rank of an entry by its local index is its rank
        unsigned hi[MAXD];
#pragma unroll
        for (int j = 0; j < MAXD; j++) hi[j] = (unsigned)(ent[j] >> 32);
        // per-level entry counts, one byte per level (at most MAXD each)
        unsigned long long per_level = 0;
#pragma unroll
        for (int j = 0; j < MAXD; j++) {
          if (ent[j] == ~0ull) continue;
          int rank = 0;
#pragma unroll
          for (int i = 0; i < MAXD; i++) rank += hi[i] < hi[j] ? 1 : 0;
          const int sidx = (int)hi[j];
          out.adj[a0 + off + rank] = make_int2(sidx, (int)(unsigned)(ent[j] & 0xffffffffu));
          int ls = 0;  // level of the entry's site
#pragma unroll
          for (int k = 0; k < BOP_MAX_K; k++) ls += sidx >= lv[k] ? 1 : 0;
          if (ls < K) per_level += 1ull << (8 * ls);
          const int k0 = lt > ls + 1 ? lt : ls + 1;
          if (k0 <= K) prod += (unsigned long long)(K - k0 + 1);
        }
        // byte k of lvcnt: entries of level <= k, k < K (the byte-wise prefix
        // sum of per_level: every partial sum is at most MAXD <= 32 < 256)
        unsigned long long lc = per_level * 0x0101010101010101ull;
        if (K < 8) lc &= (1ull << (8 * K)) - 1ull;
        out.lvcnt[s0 + t] = lc;
      }
    }
    if (PASS == 0) {
      if (lane == 0) {
        out.atom_nsite[atom] = nsite;
        out.atom_nadj[atom] = run;
        atomicMax(&out.max_level[K + 1], run);
      }
      for (int k = lane; k <= K; k += 32) {
        out.level_end[(size_t)atom * (K + 1) + k] = sm.lev[k];
        atomicMax(&out.max_level[k], sm.lev[k]);
      }
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) prod += __shfl_xor_sync(0xffffffffu, prod, o);
      if (lane == 0 && prod) atomicAdd(out.n_products, prod);
    }
    __syncwarp();
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

// Neighbour edges packed as {col, image bytes + 128} for the warp builder.
__global__ void k_pack_edges(long long E, const int* __restrict__ col, const signed char* __restrict__ img,
                             int2* __restrict__ out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
    const unsigned b = (unsigned)(img[3 * e] + 128) | ((unsigned)(img[3 * e + 1] + 128) << 8) |
                       ((unsigned)(img[3 * e + 2] + 128) << 16);
    out[e] = make_int2(col[e], (int)b);
  }
}

void launch_pack_edges(long long E, const int* col, const signed char* img, int2* out, cudaStream_t s) {
  if (E > 0) k_pack_edges<<<(int)((E + 255) / 256 < 8192 ? (E + 255) / 256 : 8192), 256, 0, s>>>(E, col, img, out);
}

int launch_cluster_warp(int pass, int n, int K, int max_deg, const long long* row_ptr, const int2* epack,
                        const int* bond_of_edge, PathCut pc, unsigned long long* gkeys,
                        ClusterOut out, int* wfail, unsigned* status, cudaStream_t s) {
  if (n == 0) return 0;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int need = (n + CW_WARPS - 1) / CW_WARPS;
  const int grid = need < sms * 5 ? need : sms * 5;
  const bool cut = pc.r2 > 0.0;
  const size_t smem = sizeof(CwSmem) * CW_WARPS;
#define CW_LAUNCH(P, C, D)                                                                                       \
  do {                                                                                                           \
    cudaFuncSetAttribute(k_cluster_warp<P, C, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
    k_cluster_warp<P, C, D><<<grid, 32 * CW_WARPS, smem, s>>>(n, K, row_ptr, epack, bond_of_edge, pc, gkeys, out,  \
                                                              wfail, status);                                    \
  } while (0)
  if (max_deg <= 16) {
    if (pass == 0) {
      if (cut) CW_LAUNCH(0, true, 16); else CW_LAUNCH(0, false, 16);
    } else {
      if (cut) CW_LAUNCH(1, true, 16); else CW_LAUNCH(1, false, 16);
    }
  } else {
    if (pass == 0) {
      if (cut) CW_LAUNCH(0, true, 32); else CW_LAUNCH(0, false, 32);
    } else {
      if (cut) CW_LAUNCH(1, true, 32); else CW_LAUNCH(1, false, 32);
    }
  }
#undef CW_LAUNCH
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int cluster_warp_max_sites() { return CW_MAXS; }

// Largest row_ptr[i+1] - row_ptr[i] into *out (atomic max; *out starts at 0).
__global__ void k_max_degree(int n, const long long* __restrict__ row_ptr, int* __restrict__ out) {
  int m = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = max(m, (int)(row_ptr[i + 1] - row_ptr[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

void launch_max_degree(int n, const long long* row_ptr, int* out, cudaStream_t s) {
  if (n > 0) k_max_degree<<<64, 256, 0, s>>>(n, row_ptr, out);
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
