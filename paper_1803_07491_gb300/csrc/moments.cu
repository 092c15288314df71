// Moments mu_n(i alpha) = <i alpha|H^n|i alpha> (Eq. momDOS) by the
// iterated interference paths Psi_k = H Psi_{k-1} (Eq. xi_rec) over every
// atom's cluster, with the merge property (Eq. xi_merge):
//   mu_2k = <Psi_k|Psi_k>,   mu_2k-1 = <Psi_k-1|Psi_k>,
// and the reverse sweep of the same recursion, which gives dU/dH for every
// bond and dU/dE for every onsite level from the weights w_n = dU/dmu_n
// (the Theta-tilde / transfer-path sums of Eqs. theta-tilde, Xi).
//
// Forward: one CTA per (spin, atom[, alpha]).  Psi_{k-1} and Psi_k live in
// shared memory (ping-pong); the last level Psi_K is never stored, only its
// inner products.  Each thread owns one cluster site per pass and gathers
// the 5x5 blocks of its bonds (15 unique elements, 16-element records) from
// L2 (for sd blocks 21 unique elements in 24-element records).  Products in
// T (float or double), moments written as double.
//
// Adjoint: one CTA per work item as well, Psi_0..Psi_K and the cotangents
// Psi-bar_1..Psi-bar_K kept in the CTA's slot of global scratch; the bond
// cotangents are summed over levels per cluster edge and added to the
// bond's unique elements with FP64 atomics.
#include "kernels.h"

namespace {

constexpr int MOM_THREADS = 256;

// stored elements of one bond block (unique upper triangle + pad to 16 bytes)
template <int NO>
__host__ __device__ constexpr int hb_count() {
  return NO == 1 ? 1 : (NO == 5 ? 16 : 24);
}

template <typename T>
struct Blk;
// Block records are 32-byte multiples on 32-byte boundaries (16 or 24 FP32
// values, 16 FP64 values): they are read with 256-bit loads, half as many
// L1 accesses per block as 128-bit loads.
__device__ __forceinline__ void ld256(const float* p, float* v) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "l"(p));
}
template <>
struct Blk<float> {
  template <int HB>
  __device__ static void load(const float* __restrict__ h, float u[HB]) {
    static_assert(HB % 8 == 0, "block records of 32-byte multiples");
#pragma unroll
    for (int q = 0; q < HB / 8; q++) ld256(h + 8 * q, u + 8 * q);
  }
};
template <>
struct Blk<double> {
  template <int HB>
  __device__ static void load(const double* __restrict__ h, double u[HB]) {
    const double2* p = reinterpret_cast<const double2*>(h);
#pragma unroll
    for (int q = 0; q < HB / 2; q++) {
      double2 v = __ldg(p + q);
      u[2 * q] = v.x; u[2 * q + 1] = v.y;
    }
  }
};

// unique element of (row, col) in the upper triangle of an NO x NO block
template <int NO>
__device__ __forceinline__ constexpr int UI(int b, int g) {
  return b <= g ? b * NO - (b * (b - 1)) / 2 + (g - b) : g * NO - (g * (g - 1)) / 2 + (b - g);
}

// Stride of one bond's cotangents: the unique block elements, padded to a
// multiple of four for FP32 (vector atomics), unpadded for FP64.
template <typename T, int NO>
__host__ __device__ constexpr int hbar_stride() {
  return (NO == 1 || sizeof(T) == 8) ? NO * (NO + 1) / 2 : (NO * (NO + 1) / 2 + 3) / 4 * 4;
}

// Adds dL/dB (G[b][g] = dL/dB_bg of one orientation of a symmetric block)
// to the bond's unique elements: u(b, g) collects G[b][g] + G[g][b].  FP32
// cotangents go out as float4 reductions (four per d block instead of 15
// scalar ones), FP64 as scalar FP64 atomics.
template <typename T, int NO>
__device__ __forceinline__ void add_bond_cotangent(T* __restrict__ hbp, const T G[NO][NO]) {
  if constexpr (NO == 1) {
    atomicAdd(hbp, G[0][0]);
  } else if constexpr (sizeof(T) == 4) {
    constexpr int HV = hbar_stride<T, NO>();
    float v[HV];
#pragma unroll
    for (int q = 0; q < HV; q++) v[q] = 0.f;
#pragma unroll
    for (int b = 0; b < NO; b++)
#pragma unroll
      for (int g = b; g < NO; g++) v[UI<NO>(b, g)] = G[b][g] + (b != g ? G[g][b] : 0.f);
    float4* dst = reinterpret_cast<float4*>(hbp);
#pragma unroll
    for (int q = 0; q < HV / 4; q++) atomicAdd(dst + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
  } else {
#pragma unroll
    for (int b = 0; b < NO; b++)
#pragma unroll
      for (int g = b; g < NO; g++) atomicAdd(hbp + UI<NO>(b, g), G[b][g] + (b != g ? G[g][b] : T(0)));
  }
}

// acc[r][c] += B[r][g] * x[g][c] for the symmetric block B given by u[].
template <typename T, int NO, int NC>
__device__ __forceinline__ void block_apply(const T* __restrict__ hrec, const T* __restrict__ x,
                                            T acc[NO][NC]) {
  if constexpr (NO == 1) {
    T h = hrec[0];
#pragma unroll
    for (int c = 0; c < NC; c++) acc[0][c] += h * x[c];
  } else {
    T u[hb_count<NO>()];
    Blk<T>::template load<hb_count<NO>()>(hrec, u);
    T xs[NO][NC];
#pragma unroll
    for (int g = 0; g < NO; g++)
#pragma unroll
      for (int c = 0; c < NC; c++) xs[g][c] = x[g * NC + c];
#pragma unroll
    for (int r = 0; r < NO; r++)
#pragma unroll
      for (int g = 0; g < NO; g++) {
        T h = u[UI<NO>(r, g)];
#pragma unroll
        for (int c = 0; c < NC; c++) acc[r][c] += h * xs[g][c];
      }
  }
}

// next 16-byte boundary (the staged adjacency holds int2 / u64 records); the
// launchers reserve 16 bytes of slack for it
__device__ __forceinline__ unsigned char* align16(unsigned char* p) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
}

// Hint to bring the 128-byte lines of a stored row into L2 before it is read.
template <typename T, int PS>
__device__ __forceinline__ void prefetch_row_l2(const T* p) {
  constexpr int BYTES = PS * (int)sizeof(T);
#pragma unroll
  for (int o = 0; o < BYTES; o += 128)
    asm volatile("{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %0;\n\tprefetch.global.L2 [ga];\n\t}" ::"l"(
        reinterpret_cast<const char*>(p) + o));
  asm volatile("{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %0;\n\tprefetch.global.L2 [ga];\n\t}" ::"l"(
      reinterpret_cast<const char*>(p) + BYTES - 1));
}

// Asynchronous copies global -> shared (cp.async, no register round trip),
// so that all of a thread's staging copies of a work item are in flight at
// once; cp_async_wait_all() waits for the thread's own copies, a barrier
// then publishes them to the CTA.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Extent of one atom's cluster in the cluster arrays: first site, number of
// sites, adjacency range.  Read in two steps (sites, then adjacency) one work
// item ahead, so that the next item's staging starts without waiting on
// dependent loads.
struct ItemExt {
  long long s0, abase, aend;
  int nsite;
};
__device__ __forceinline__ void ext_sites(const ClusterView& cv, int atom, ItemExt& x) {
  x.s0 = cv.site_off[atom];
  x.nsite = cv.level_end[(size_t)atom * (cv.K + 1) + cv.K];
}
__device__ __forceinline__ void ext_adj(const ClusterView& cv, ItemExt& x) {
  x.abase = cv.adj_off[x.s0];
  x.aend = cv.adj_off[x.s0 + x.nsite];
}

// One work item's cluster data in shared memory: the adjacency entries of its
// sites, their adjacency offsets (absolute, as in the cluster arrays), level
// counts and atoms.
__device__ __forceinline__ void stage_item(const ClusterView& cv, const ItemExt& x, int2* s_adj, long long* s_aoff,
                                           unsigned long long* s_lvc, int* s_atom, int tid, int nthr) {
  const long long s0 = x.s0, abase = x.abase;
  const int nsite = x.nsite, nadj = (int)(x.aend - x.abase);
  for (int q = tid; q < nadj; q += nthr) cp_async8(s_adj + q, cv.adj + abase + q);
  for (int q = tid; q <= nsite; q += nthr) cp_async8(s_aoff + q, cv.adj_off + s0 + q);
  for (int q = tid; q < nsite; q += nthr) {
    cp_async8(s_lvc + q, cv.lvcnt + s0 + q);
    cp_async4(s_atom + q, cv.site_atom + s0 + q);
  }
  cp_async_wait_all();
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y[t] = E_t * x[t] (t < ncol) + sum_{adjacent s < ncol} B_ts x[s], t < nrow.
// One thread per site; returns nothing, the caller consumes acc.
template <typename T, int NO, int NC>
__device__ __forceinline__ void gather_row(const ClusterView& cv, const T* __restrict__ H, int HS,
                                           const T* __restrict__ E, const int* __restrict__ satom,
                                           const long long* __restrict__ aoff, int t, int ncol,
                                           const T* __restrict__ x, T acc[NO][NC]) {
#pragma unroll
  for (int r = 0; r < NO; r++)
#pragma unroll
    for (int c = 0; c < NC; c++) acc[r][c] = T(0);
  if (t < ncol) {
    const T* e = E + (size_t)satom[t] * NO;
#pragma unroll
    for (int r = 0; r < NO; r++) {
      T er = e[r];
#pragma unroll
      for (int c = 0; c < NC; c++) acc[r][c] = er * x[(t * NO + r) * NC + c];
    }
  }
  const long long q1 = aoff[t + 1];
  for (long long q = aoff[t]; q < q1; q++) {
    int2 en = cv.adj[q];
    if (en.x >= ncol) break;
    block_apply<T, NO, NC>(H + (size_t)en.y * HS, x + (size_t)en.x * NO * NC, acc);
  }
}

// ------------------------------------------------------------------ forward
// Shared-memory row of one site: NO x NC values padded to 16-byte multiples
// so that a row is read with vector loads.
template <typename T, int N>
struct Row {
  static constexpr int PS = (sizeof(T) == 4) ? ((N + 3) / 4) * 4 : ((N + 1) / 2) * 2;
};
template <typename T, int N, int PS>
__device__ __forceinline__ void load_row(const T* __restrict__ p, T x[N]) {
  if constexpr (N == 1) {
    x[0] = p[0];
  } else if constexpr (sizeof(T) == 4) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int v = 0; v < PS / 4; v++) {
      float4 w = q[v];
      if (4 * v + 0 < N) x[4 * v + 0] = w.x;
      if (4 * v + 1 < N) x[4 * v + 1] = w.y;
      if (4 * v + 2 < N) x[4 * v + 2] = w.z;
      if (4 * v + 3 < N) x[4 * v + 3] = w.w;
    }
  } else {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int v = 0; v < PS / 2; v++) {
      double2 w = q[v];
      if (2 * v + 0 < N) x[2 * v + 0] = w.x;
      if (2 * v + 1 < N) x[2 * v + 1] = w.y;
    }
  }
}

template <typename T, int N, int PS>
__device__ __forceinline__ void store_row(T* __restrict__ p, const T x[N]) {
  if constexpr (N == 1) {
    p[0] = x[0];
  } else if constexpr (sizeof(T) == 4) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int v = 0; v < PS / 4; v++) {
      float4 w;
      w.x = 4 * v + 0 < N ? x[4 * v + 0] : 0.f;
      w.y = 4 * v + 1 < N ? x[4 * v + 1] : 0.f;
      w.z = 4 * v + 2 < N ? x[4 * v + 2] : 0.f;
      w.w = 4 * v + 3 < N ? x[4 * v + 3] : 0.f;
      q[v] = w;
    }
  } else {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int v = 0; v < PS / 2; v++) {
      double2 w;
      w.x = 2 * v + 0 < N ? x[2 * v + 0] : 0.0;
      w.y = 2 * v + 1 < N ? x[2 * v + 1] : 0.0;
      q[v] = w;
    }
  }
}

template <typename T, int NO>
__device__ __forceinline__ void load_bond(const T* __restrict__ h, T u[hb_count<NO>()]) {
  if constexpr (NO == 1) {
    u[0] = __ldg(h);
  } else {
    Blk<T>::template load<hb_count<NO>()>(h, u);
  }
}

// acc += B x for one symmetric block (unique elements u) and a site row x
template <typename T, int NO, int NC>
__device__ __forceinline__ void block_fma(const T* u, const T* x, T acc[NO][NC]) {
  if constexpr (NO == 1) {
#pragma unroll
    for (int c = 0; c < NC; c++) acc[0][c] += u[0] * x[c];
  } else {
#pragma unroll
    for (int r = 0; r < NO; r++)
#pragma unroll
      for (int g = 0; g < NO; g++) {
        const T h = u[UI<NO>(r, g)];
#pragma unroll
        for (int c = 0; c < NC; c++) acc[r][c] += h * x[g * NC + c];
      }
  }
}

// acc += sum over the first cnt adjacency entries of t of B_ts x[s]; the
// next entry and its block are fetched while the current one is applied.
template <typename T, int NO, int NC, int PS>
__device__ __forceinline__ void gather_pf(const int2* __restrict__ adj, long long q0, int cnt,
                                          const T* __restrict__ H, int HS, const T* __restrict__ x,
                                          T acc[NO][NC]) {
  if (cnt <= 0) return;
  constexpr int HB = hb_count<NO>();
  int2 en = __ldg(adj + q0);
  T hb[HB];
  load_bond<T, NO>(H + (size_t)en.y * HS, hb);
  for (int e = 0; e < cnt; e++) {
    const int s = en.x;
    T hc[HB];
#pragma unroll
    for (int q = 0; q < HB; q++) hc[q] = hb[q];
    if (e + 1 < cnt) {
      en = __ldg(adj + q0 + e + 1);
      load_bond<T, NO>(H + (size_t)en.y * HS, hb);
    }
    T xs[NO * NC];
    load_row<T, NO * NC, PS>(x + (size_t)s * PS, xs);
    block_fma<T, NO, NC>(hc, xs, acc);
  }
}

// acc += sum over cnt adjacency entries of B_ts x[s], with the blocks of
// the next two entries in flight while the current one is applied.
template <typename T, int NO, int NC, int PS>
__device__ __forceinline__ void gather_pf2(const int2* __restrict__ ent, int cnt, const T* __restrict__ H, int HS,
                                           const T* __restrict__ x, T acc[NO][NC]) {
  constexpr int HB = hb_count<NO>();
  constexpr int N = NO * NC;
  if (cnt <= 0) return;
  int2 e0 = ent[0];
  int2 e1 = cnt > 1 ? ent[1] : e0;
  T h0[HB], h1[HB];
  load_bond<T, NO>(H + (size_t)e0.y * HS, h0);
  if (cnt > 1) load_bond<T, NO>(H + (size_t)e1.y * HS, h1);
  for (int e = 0; e < cnt; e++) {
    const int s = e0.x;
    T hc[HB];
#pragma unroll
    for (int q = 0; q < HB; q++) hc[q] = h0[q];
    e0 = e1;
#pragma unroll
    for (int q = 0; q < HB; q++) h0[q] = h1[q];
    if (e + 2 < cnt) {
      e1 = ent[e + 2];
      load_bond<T, NO>(H + (size_t)e1.y * HS, h1);
    }
    T xs[N];
    load_row<T, N, PS>(x + (size_t)s * PS, xs);
    block_fma<T, NO, NC>(hc, xs, acc);
  }
}

// The reverse sweep's gather with the bond cotangents of the same pairs:
// for each entry s of row t (t in C_{k-1}, s in C_k), acc += B_ts x[s]
// (when gather is set) and dL/dB of the forward pair (s, t), x[s] pt^T
// summed over the columns (x = Psi-bar_k, pt = Psi_k-1(t)), goes to the
// bond's unique elements; the blocks of the next two entries are in flight.
template <typename T, int NO, int NC, int PS>
__device__ __forceinline__ void gather_cot(const int2* __restrict__ ent, int cnt, const T* __restrict__ H, int HS,
                                           const T* __restrict__ x, T acc[NO][NC], bool gather, const T pt[NO * NC],
                                           T* __restrict__ Hbar, int HSh) {
  constexpr int HB = hb_count<NO>();
  constexpr int N = NO * NC;
  if (cnt <= 0) return;
  int2 e0 = ent[0];
  int2 e1 = cnt > 1 ? ent[1] : e0;
  T h0[HB], h1[HB];
  if (gather) {
    load_bond<T, NO>(H + (size_t)e0.y * HS, h0);
    if (cnt > 1) load_bond<T, NO>(H + (size_t)e1.y * HS, h1);
  }
  for (int e = 0; e < cnt; e++) {
    const int sidx = e0.x, bond = e0.y;
    T hc[HB];
#pragma unroll
    for (int q = 0; q < HB; q++) hc[q] = h0[q];
    e0 = e1;
#pragma unroll
    for (int q = 0; q < HB; q++) h0[q] = h1[q];
    if (e + 2 < cnt) {
      e1 = ent[e + 2];
      if (gather) load_bond<T, NO>(H + (size_t)e1.y * HS, h1);
    }
    T xs[N];
    load_row<T, N, PS>(x + (size_t)sidx * PS, xs);
    if (gather) block_fma<T, NO, NC>(hc, xs, acc);
    T G[NO][NO];
#pragma unroll
    for (int b = 0; b < NO; b++)
#pragma unroll
      for (int g = 0; g < NO; g++) {
        T a = T(0);
#pragma unroll
        for (int c = 0; c < NC; c++) a += xs[b * NC + c] * pt[g * NC + c];
        G[b][g] = a;
      }
    add_bond_cotangent<T, NO>(Hbar + (size_t)bond * HSh, G);
  }
}

// Forward kernel.  A persistent CTA takes a run of consecutive work items
// (spin, atom[, alpha]); neighbouring atoms share most of their clusters'
// blocks, which then come from L1.  For each item the atom's adjacency,
// per-site offsets, level counts and site atoms are staged in shared memory
// (one coalesced copy) when they fit, so that the edge loop only waits for
// the bond blocks, which are fetched one edge ahead.  Each thread computes
// all NC columns of one site (NO x NO x NC multiply-adds per edge); Psi
// rows are padded to 16-byte multiples and kept in two exactly sized
// buffers (even and odd levels).
constexpr int FWD_THREADS = 192;

struct FwdSmem {
  int cap_even, cap_odd, max_sites, max_adj;
  bool stage;
};

template <typename T, int NO, int NC>
__global__ void __launch_bounds__(FWD_THREADS, sizeof(T) == 4 ? 2 : 1)
k_moments(ClusterView cv, const T* __restrict__ H, int HS, const T* __restrict__ onsite, int n, int n_on,
          int n_mom, FwdSmem L, int n_items, int chunk, double* __restrict__ mu, T* __restrict__ pstore,
          const long long* __restrict__ psi_off, long long psi_tot) {
  constexpr int N = NO * NC;
  constexpr int PS = (N == 1) ? 1 : Row<T, N>::PS;
  constexpr int HB = hb_count<NO>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* buf[2];
  buf[0] = reinterpret_cast<T*>(smem_raw);
  buf[1] = buf[0] + (size_t)L.cap_even * PS;
  unsigned char* tail = align16(reinterpret_cast<unsigned char*>(buf[1] + (size_t)L.cap_odd * PS));
  int2* s_adj = reinterpret_cast<int2*>(tail);
  unsigned long long* s_lvc = reinterpret_cast<unsigned long long*>(s_adj + (L.stage ? L.max_adj : 0));
  long long* s_aoff = reinterpret_cast<long long*>(s_lvc + (L.stage ? L.max_sites : 0));
  int* s_atom = reinterpret_cast<int*>(s_aoff + (L.stage ? L.max_sites + 1 : 0));
  // per-warp partial sums of the two moments of a level, in two buffers
  // (level parity): the reads of level k's partials need no barrier before
  // level k + 1 starts writing its own
  __shared__ T red[2][2 * NC][FWD_THREADS / 32];
  const int K = cv.K;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int w0 = blockIdx.x * chunk, w1 = min(n_items, w0 + chunk);
  ItemExt nx{};
  if (w0 < w1) {
    ext_sites(cv, ((NC == NO) ? w0 : (w0 / NO)) % n, nx);
    ext_adj(cv, nx);
  }
  for (int w = w0; w < w1; w++) {
    const int grp = (NC == NO) ? 0 : (w % NO);
    const int sa = (NC == NO) ? w : (w / NO);
    const int spin = sa / n, atom = sa % n;
    const ItemExt cur = nx;
    const long long s0 = cur.s0, abase = cur.abase;
    const int* lev = cv.level_end + (size_t)atom * (K + 1);
    const int2* adj = cv.adj + abase;
    const unsigned long long* lvc = cv.lvcnt + s0;
    const int* satom = cv.site_atom + s0;
    const T* E = onsite + (size_t)spin * n_on * NO;
    if (L.stage) stage_item(cv, cur, s_adj, s_aoff, s_lvc, s_atom, tid, FWD_THREADS);
    const bool more = w + 1 < w1;
    if (more) ext_sites(cv, ((NC == NO) ? w + 1 : ((w + 1) / NO)) % n, nx);
    for (int q = tid; q < N; q += FWD_THREADS) {
      const int r = q / NC, c = q % NC;
      buf[0][q] = (NC == NO) ? T(r == c ? 1 : 0) : T(r == grp ? 1 : 0);
    }
    // stored Psi: item rows start at ib, level k at row lo_k = sum_{j<k} |C_j|
    T* pitem = nullptr;
    if (pstore != nullptr) {
      pitem = pstore + ((size_t)(spin * (NO / NC) + grp) * psi_tot + psi_off[atom]) * PS;
      for (int q = tid; q < PS; q += FWD_THREADS) {
        const int r = q / NC, c = q % NC;
        pitem[q] = q < N ? ((NC == NO) ? T(r == c ? 1 : 0) : T(r == grp ? 1 : 0)) : T(0);
      }
    }
    long long lo_k = 0;
    __syncthreads();
    double* out = mu + ((size_t)sa * NO + grp) * n_mom;
    if (tid < NC) out[(size_t)tid * n_mom] = 1.0;
    for (int k = 1; k <= K; k++) {
      lo_k += lev[k - 1];
      const int nrow = lev[k], ncol = lev[k - 1];
      const T* prev = buf[(k - 1) & 1];
      T* cur = buf[k & 1];
      T d1[NC], d2[NC];
#pragma unroll
      for (int c = 0; c < NC; c++) d1[c] = d2[c] = T(0);
      for (int t = tid; t < nrow; t += FWD_THREADS) {
        T acc[NO][NC];
        const bool in_prev = t < ncol;
        if (in_prev) {
          T pt[N];
          load_row<T, N, PS>(prev + (size_t)t * PS, pt);
          const T* e = E + (size_t)(L.stage ? s_atom[t] : satom[t]) * NO;
#pragma unroll
          for (int r = 0; r < NO; r++) {
            const T er = e[r];
#pragma unroll
            for (int c = 0; c < NC; c++) acc[r][c] = er * pt[r * NC + c];
          }
        } else {
#pragma unroll
          for (int r = 0; r < NO; r++)
#pragma unroll
            for (int c = 0; c < NC; c++) acc[r][c] = T(0);
        }
        const unsigned long long lc = L.stage ? s_lvc[t] : lvc[t];
        const int cnt = (int)((lc >> (8 * (k - 1))) & 0xff);
        if (cnt > 0) {
          const int q0 = (int)((L.stage ? s_aoff[t] : cv.adj_off[s0 + t]) - abase);
          gather_pf2<T, NO, NC, PS>(L.stage ? s_adj + q0 : adj + q0, cnt, H, HS, prev, acc);
        }
        if (in_prev) {  // row t of Psi_k-1 again (shared memory), rather than kept live over the gather
          T pt[N];
          load_row<T, N, PS>(prev + (size_t)t * PS, pt);
#pragma unroll
          for (int r = 0; r < NO; r++)
#pragma unroll
            for (int c = 0; c < NC; c++) d1[c] += pt[r * NC + c] * acc[r][c];
        }
#pragma unroll
        for (int r = 0; r < NO; r++)
#pragma unroll
          for (int c = 0; c < NC; c++) d2[c] += acc[r][c] * acc[r][c];
        if (k < K) {
          T* dst = cur + (size_t)t * PS;
#pragma unroll
          for (int r = 0; r < NO; r++)
#pragma unroll
            for (int c = 0; c < NC; c++) dst[r * NC + c] = acc[r][c];
        }
        if (pitem != nullptr) {
          T row[N];
#pragma unroll
          for (int r = 0; r < NO; r++)
#pragma unroll
            for (int c = 0; c < NC; c++) row[r * NC + c] = acc[r][c];
          store_row<T, N, PS>(pitem + (size_t)(lo_k + t) * PS, row);
        }
      }
#pragma unroll
      for (int c = 0; c < NC; c++) {
        T a = warp_sum(d1[c]), b = warp_sum(d2[c]);
        if (lane == 0) {
          red[k & 1][c][wid] = a;
          red[k & 1][NC + c][wid] = b;
        }
      }
      // level k's rows and partials are complete; level k + 1 writes the
      // other Psi buffer (read last at level k - 1) and the other partials
      __syncthreads();
      if (tid < 2 * NC) {
        T acc = T(0);
        for (int q = 0; q < FWD_THREADS / 32; q++) acc += red[k & 1][tid][q];
        const int c = tid % NC;
        const int m = tid < NC ? 2 * k - 1 : 2 * k;
        out[(size_t)c * n_mom + m] = (double)acc;
      }
    }
    if (more) ext_adj(cv, nx);
  }
}


// ------------------------------------------------------------------ reverse sweep over stored Psi
// With every Psi_k of every work item stored in global memory (rows of the
// forward kernel, level k at rows lo_k .. lo_k + |C_k|), the reverse sweep
//   Psi-bar_K     = 2 w_2K Psi_K + w_2K-1 Psi_K-1
//   Psi-bar_k-1   = H Psi-bar_k (rows < |C_k-1|, columns < |C_k|)
//                   + 2 w_2k-2 Psi_k-1 + w_2k-1 Psi_k + w_2k-3 Psi_k-2
// runs like the forward kernel: Psi-bar_k and Psi-bar_k-1 in two shared
// buffers (even / odd levels), the adjacency staged, one site row per
// thread.  The onsite cotangents dL/dE_t = sum_k Psi-bar_k[t] . Psi_k-1[t]
// are accumulated per site in shared memory and added once per item.
// With HBAR the gather of level k also forms the bond cotangents of its
// pairs, Psi-bar_k(s) Psi_k-1(t)^T for the forward pair (s in C_k, t in
// C_{k-1}) (Psi-bar_k(s) is the gather's operand, Psi_k-1(t) one stored row
// per site), and adds them to the bond's unique elements (gather_cot); at
// k = 1 only these products run.
struct RevSmem {
  int cap_even, cap_odd, max_sites, max_adj, cap_eb;
  bool stage;
};

template <typename T, int NO>
__host__ __device__ constexpr size_t eb_elems(int cap_eb) {
  return ((size_t)cap_eb * NO * sizeof(T) + 15) / 16 * 16 / sizeof(T);
}

template <typename T, int NO, int NC, bool HBAR>
__global__ void __launch_bounds__(FWD_THREADS, sizeof(T) == 4 ? 2 : 1)
k_adj_rev(ClusterView cv, const T* __restrict__ H, int HS, const T* __restrict__ onsite, int n, int n_on,
          int n_mom,
          RevSmem L, int n_items, int chunk, const T* __restrict__ pstore,
          const long long* __restrict__ psi_off, long long psi_tot, const double* __restrict__ wts,
          T* __restrict__ Hbar, int HSh, double* __restrict__ Ebar, double* __restrict__ siteval,
          long long sv_stride) {
  constexpr int N = NO * NC;
  constexpr int PS = (N == 1) ? 1 : Row<T, N>::PS;
  constexpr int HB = hb_count<NO>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* buf[2];
  buf[0] = reinterpret_cast<T*>(smem_raw);
  buf[1] = buf[0] + (size_t)L.cap_even * PS;
  T* eb = buf[1] + (size_t)L.cap_odd * PS;  // [cap_eb][NO], padded to 16 bytes
  unsigned char* tail = align16(reinterpret_cast<unsigned char*>(eb + eb_elems<T, NO>(L.cap_eb)));
  int2* s_adj = reinterpret_cast<int2*>(tail);
  unsigned long long* s_lvc = reinterpret_cast<unsigned long long*>(s_adj + (L.stage ? L.max_adj : 0));
  long long* s_aoff = reinterpret_cast<long long*>(s_lvc + (L.stage ? L.max_sites : 0));
  int* s_atom = reinterpret_cast<int*>(s_aoff + (L.stage ? L.max_sites + 1 : 0));
  __shared__ T ws[NC][BOP_MAX_NMOM];
  __shared__ int s_lev[BOP_MAX_K + 1];
  __shared__ long long s_lo[BOP_MAX_K + 1];
  const int K = cv.K;
  const int tid = threadIdx.x;
  const int w0 = blockIdx.x * chunk, w1 = min(n_items, w0 + chunk);
  ItemExt nx{};
  if (w0 < w1) {
    ext_sites(cv, ((NC == NO) ? w0 : (w0 / NO)) % n, nx);
    ext_adj(cv, nx);
  }
  for (int w = w0; w < w1; w++) {
    const int grp = (NC == NO) ? 0 : (w % NO);
    const int sa = (NC == NO) ? w : (w / NO);
    const int spin = sa / n, atom = sa % n;
    const ItemExt cur = nx;
    const long long s0 = cur.s0, abase = cur.abase;
    const int* lev = cv.level_end + (size_t)atom * (K + 1);
    const int2* adj = cv.adj + abase;
    const unsigned long long* lvc = cv.lvcnt + s0;
    const int* satom = cv.site_atom + s0;
    const T* E = onsite + (size_t)spin * n_on * NO;
    const size_t ib = ((size_t)(spin * (NO / NC) + grp) * psi_tot + psi_off[atom]) * PS;
    const T* P = pstore + ib;
    if (L.stage) stage_item(cv, cur, s_adj, s_aoff, s_lvc, s_atom, tid, FWD_THREADS);
    const bool more = w + 1 < w1;
    if (more) ext_sites(cv, ((NC == NO) ? w + 1 : ((w + 1) / NO)) % n, nx);
    if (tid <= K) s_lev[tid] = lev[tid];
    if (tid == 0) {
      long long o = 0;
      for (int k = 0; k <= K; k++) {
        s_lo[k] = o;
        o += lev[k];
      }
    }
    for (int q = tid; q < NC * n_mom; q += FWD_THREADS) {
      const int c = q / n_mom, m = q % n_mom;
      ws[c][m] = (T)wts[((size_t)sa * NO + grp + c) * n_mom + m];
    }
    __syncthreads();
    const int neb = s_lev[K - 1];
    for (int q = tid; q < neb * NO; q += FWD_THREADS) eb[q] = T(0);
    // Psi-bar_K
    {
      T* xb = buf[K & 1];
      for (int t = tid; t < s_lev[K]; t += FWD_THREADS) {
        T pk[N], row[N];
        load_row<T, N, PS>(P + (size_t)(s_lo[K] + t) * PS, pk);
#pragma unroll
        for (int q = 0; q < N; q++) row[q] = T(2) * ws[q % NC][2 * K] * pk[q];
        if (t < s_lev[K - 1]) {
          T pk1[N];
          load_row<T, N, PS>(P + (size_t)(s_lo[K - 1] + t) * PS, pk1);
#pragma unroll
          for (int q = 0; q < N; q++) row[q] += ws[q % NC][2 * K - 1] * pk1[q];
        }
        store_row<T, N, PS>(xb + (size_t)t * PS, row);
      }
    }
    __syncthreads();
    for (int k = K; k >= 1; k--) {
      const T* xb = buf[k & 1];
      T* yb = buf[(k - 1) & 1];
      const int nrow = s_lev[k - 1];
      for (int t = tid; t < nrow; t += FWD_THREADS) {
        // the stored rows this site needs, towards L2 while the gather runs
        const T* r1 = P + (size_t)(s_lo[k - 1] + t) * PS;
        prefetch_row_l2<T, PS>(r1);
        if (k >= 2) {
          prefetch_row_l2<T, PS>(P + (size_t)(s_lo[k] + t) * PS);
          if (t < s_lev[k - 2]) prefetch_row_l2<T, PS>(P + (size_t)(s_lo[k - 2] + t) * PS);
        }
        T acc[NO][NC];
        if (k >= 2) {
          T xt[N];
          load_row<T, N, PS>(xb + (size_t)t * PS, xt);
          const T* e = E + (size_t)(L.stage ? s_atom[t] : satom[t]) * NO;
#pragma unroll
          for (int r = 0; r < NO; r++) {
            const T er = e[r];
#pragma unroll
            for (int c = 0; c < NC; c++) acc[r][c] = er * xt[r * NC + c];
          }
        }
        if (k >= 2 || HBAR) {
          int cnt;
          if (k < K) {
            const unsigned long long lc = L.stage ? s_lvc[t] : lvc[t];
            cnt = (int)((lc >> (8 * k)) & 0xff);
          } else {
            cnt = L.stage ? (int)(s_aoff[t + 1] - s_aoff[t]) : (int)(cv.adj_off[s0 + t + 1] - cv.adj_off[s0 + t]);
          }
          if (cnt > 0) {
            const int q0 = (int)((L.stage ? s_aoff[t] : cv.adj_off[s0 + t]) - abase);
            const int2* ents = L.stage ? s_adj + q0 : adj + q0;
            if constexpr (HBAR) {
              // with the bond cotangents of the forward pairs (s, t) of level k
              T pt[N];
              load_row<T, N, PS>(r1, pt);
              gather_cot<T, NO, NC, PS>(ents, cnt, H, HS, xb, acc, k >= 2, pt, Hbar, HSh);
            } else {
              gather_pf2<T, NO, NC, PS>(ents, cnt, H, HS, xb, acc);
            }
          }
        }
        // onsite cotangent of level k: Psi-bar_k[t] . Psi_k-1[t] (rows read after the gather)
        T p1[N];
        {
          T xt[N];
          load_row<T, N, PS>(xb + (size_t)t * PS, xt);
          load_row<T, N, PS>(r1, p1);
#pragma unroll
          for (int r = 0; r < NO; r++) {
            T a = T(0);
#pragma unroll
            for (int c = 0; c < NC; c++) a += xt[r * NC + c] * p1[r * NC + c];
            eb[t * NO + r] += a;
          }
        }
        if (k >= 2) {
          T pk[N];
          load_row<T, N, PS>(P + (size_t)(s_lo[k] + t) * PS, pk);
          T row[N];
#pragma unroll
          for (int r = 0; r < NO; r++)
#pragma unroll
            for (int c = 0; c < NC; c++) {
              const int q = r * NC + c;
              row[q] = acc[r][c] + T(2) * ws[c][2 * k - 2] * p1[q] + ws[c][2 * k - 1] * pk[q];
            }
          if (t < s_lev[k - 2]) {
            T p2[N];
            load_row<T, N, PS>(P + (size_t)(s_lo[k - 2] + t) * PS, p2);
#pragma unroll
            for (int q = 0; q < N; q++) row[q] += ws[q % NC][2 * k - 3] * p2[q];
          }
          store_row<T, N, PS>(yb + (size_t)t * PS, row);
        }
      }
      __syncthreads();
    }
    if (Ebar != nullptr) {
      for (int q = tid; q < neb * NO; q += FWD_THREADS) {
        const int t = q / NO, r = q % NO;
        atomicAdd(Ebar + ((size_t)spin * n_on + (L.stage ? s_atom[t] : satom[t])) * NO + r, (double)eb[q]);
      }
    }
    if (siteval != nullptr) {  // per-site sums over the orbitals (one row of the SCF Jacobian)
      for (int t = tid; t < neb; t += FWD_THREADS) {
        double a = 0.0;
#pragma unroll
        for (int r = 0; r < NO; r++) a += (double)eb[t * NO + r];
        atomicAdd(siteval + (size_t)spin * sv_stride + s0 + t, a);
      }
    }
    if (more) ext_adj(cv, nx);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ adjoint (recompute)
__device__ __forceinline__ int site_level(const int* lev, int K, int t) {
  int k = 0;
  while (k < K && t >= lev[k]) k++;
  return k;
}

template <typename T, int NO, int NC>
__global__ void __launch_bounds__(MOM_THREADS)
k_moments_adj(ClusterView cv, const T* __restrict__ H, int HS, const T* __restrict__ onsite, int n, int n_on, int n_mom,
              int nwork, const double* __restrict__ wts, T* __restrict__ scratch, size_t slot_elems,
              T* __restrict__ Hbar, int HSh, double* __restrict__ Ebar) {
  __shared__ T ws[NC][BOP_MAX_NMOM];
  __shared__ int s_lev[BOP_MAX_K + 1];
  __shared__ long long s_off[BOP_MAX_K + 2];
  const int K = cv.K;
  const int tid = threadIdx.x;
  T* psi = scratch + (size_t)blockIdx.x * slot_elems;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int grp = (NC == NO) ? 0 : (w % NO);
    const int sa = (NC == NO) ? w : (w / NO);
    const int spin = sa / n, atom = sa % n;
    const long long s0 = cv.site_off[atom];
    const int* lev = cv.level_end + (size_t)atom * (K + 1);
    const int* satom = cv.site_atom + s0;
    const long long* aoff = cv.adj_off + s0;
    const T* E = onsite + (size_t)spin * n_on * NO;
    if (tid <= K) s_lev[tid] = lev[tid];
    if (tid == 0) {  // Psi_k at s_off[k], Psi-bar_k at s_off[K+1] + (s_off[k] - s_off[1])
      long long o = 0;
      for (int k = 0; k <= K; k++) {
        s_off[k] = o;
        o += (long long)lev[k] * NO * NC;
      }
      s_off[K + 1] = o;
    }
    for (int q = tid; q < NC * n_mom; q += blockDim.x) {
      int c = q / n_mom, m = q % n_mom;
      ws[c][m] = (T)wts[((size_t)sa * NO + grp + c) * n_mom + m];
    }
    __syncthreads();
    T* P = psi;
    T* Pb = psi + s_off[K + 1] - s_off[1];  // Pb + s_off[k] is Psi-bar_k (k >= 1)
    // forward: all levels
    for (int q = tid; q < NO * NC; q += blockDim.x) {
      int r = q / NC, c = q % NC;
      P[q] = (NC == NO) ? T(r == c ? 1 : 0) : T(r == grp ? 1 : 0);
    }
    __syncthreads();
    for (int k = 1; k <= K; k++) {
      const T* x = P + s_off[k - 1];
      T* y = P + s_off[k];
      for (int t = tid; t < s_lev[k]; t += blockDim.x) {
        T acc[NO][NC];
        gather_row<T, NO, NC>(cv, H, HS, E, satom, aoff, t, s_lev[k - 1], x, acc);
#pragma unroll
        for (int r = 0; r < NO; r++)
#pragma unroll
          for (int c = 0; c < NC; c++) y[(t * NO + r) * NC + c] = acc[r][c];
      }
      __syncthreads();
    }
    // Psi-bar_K = 2 w_2K Psi_K + w_2K-1 Psi_K-1
    {
      const T* PK = P + s_off[K];
      const T* PK1 = P + s_off[K - 1];
      T* B = Pb + s_off[K];
      for (int q = tid; q < s_lev[K] * NO * NC; q += blockDim.x) {
        int t = q / (NO * NC), c = q % NC;
        T v = T(2) * ws[c][2 * K] * PK[q];
        if (t < s_lev[K - 1]) v += ws[c][2 * K - 1] * PK1[q];
        B[q] = v;
      }
    }
    __syncthreads();
    // Psi-bar_{k-1} = H^T Psi-bar_k (rows < |C_k-1|, cols < |C_k|) + dot-product terms
    for (int k = K; k >= 2; k--) {
      const T* xb = Pb + s_off[k];
      T* yb = Pb + s_off[k - 1];
      const T* Pk = P + s_off[k];
      const T* Pk1 = P + s_off[k - 1];
      const T* Pk2 = P + s_off[k - 2];
      for (int t = tid; t < s_lev[k - 1]; t += blockDim.x) {
        T acc[NO][NC];
        gather_row<T, NO, NC>(cv, H, HS, E, satom, aoff, t, s_lev[k], xb, acc);
#pragma unroll
        for (int r = 0; r < NO; r++)
#pragma unroll
          for (int c = 0; c < NC; c++) {
            int q = (t * NO + r) * NC + c;
            T v = acc[r][c] + T(2) * ws[c][2 * k - 2] * Pk1[q] + ws[c][2 * k - 1] * Pk[q];
            if (t < s_lev[k - 2]) v += ws[c][2 * k - 3] * Pk2[q];
            yb[q] = v;
          }
      }
      __syncthreads();
    }
    // bond and onsite cotangents: dU/dH_ts = sum_k Psi-bar_k[t] Psi_k-1[s]^T
    for (int t = tid; t < s_lev[K]; t += blockDim.x) {
      const int lt = site_level(s_lev, K, t);
      const long long q1 = Hbar != nullptr ? aoff[t + 1] : aoff[t];  // no bond cotangents wanted
      for (long long q = aoff[t]; q < q1; q++) {
        int2 en = cv.adj[q];
        const int s = en.x;
        if (s >= s_lev[K - 1]) break;
        const int ls = site_level(s_lev, K, s);
        const int kmin = lt > ls + 1 ? lt : ls + 1;
        T G[NO][NO];
#pragma unroll
        for (int b = 0; b < NO; b++)
#pragma unroll
          for (int g = 0; g < NO; g++) G[b][g] = T(0);
        for (int k = kmin; k <= K; k++) {
          const T* pb = Pb + s_off[k] + (size_t)t * NO * NC;
          const T* ps = P + s_off[k - 1] + (size_t)s * NO * NC;
#pragma unroll
          for (int b = 0; b < NO; b++)
#pragma unroll
            for (int g = 0; g < NO; g++) {
              T a = T(0);
#pragma unroll
              for (int c = 0; c < NC; c++) a += pb[b * NC + c] * ps[g * NC + c];
              G[b][g] += a;
            }
        }
        add_bond_cotangent<T, NO>(Hbar + (size_t)en.y * HSh, G);
      }
      if (Ebar != nullptr) {
        double eb[NO];
#pragma unroll
        for (int b = 0; b < NO; b++) eb[b] = 0.0;
        for (int k = lt + 1; k <= K; k++) {
          const T* pb = Pb + s_off[k] + (size_t)t * NO * NC;
          const T* pt = P + s_off[k - 1] + (size_t)t * NO * NC;
#pragma unroll
          for (int b = 0; b < NO; b++) {
            T a = T(0);
#pragma unroll
            for (int c = 0; c < NC; c++) a += pb[b * NC + c] * pt[b * NC + c];
            eb[b] += (double)a;
          }
        }
        if (lt + 1 <= K) {
          double* ep = Ebar + ((size_t)spin * n_on + satom[t]) * NO;
#pragma unroll
          for (int b = 0; b < NO; b++) atomicAdd(ep + b, eb[b]);
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ non-collinear spin moments
// Non-collinear magnetism (section "Magnetism", Eqs. onsite_CM and
// onsite-noncollinear).  Work item (atom i, orbital alpha); its two
// starting states are the local spin states of atom i, chi_up antiparallel
// to the moment direction s_i (eigenvalue -1 of s_i.sigma, the lower level)
// and chi_dn parallel, complex 2-spinors in the spin basis along z.  A site
// row holds NO x 8 reals, column c = nu * 4 + sp * 2 + ri (starting spinor
// nu, spin component sp, real / imaginary part).  The hopping H_e x 1 acts
// on the orbital index (block_apply with 8 columns); the onsite matrix
// Ebar + h.sigma, Ebar = (E_up + E_dn)/2, h = (E_dn - E_up)/2 s_j, mixes
// the four reals of each spinor.  In this real form every operator is
// symmetric, so the reverse sweep gathers with the same rows.
//   forward (wts == NULL): local channel moments mu_nu,n = <chi_nu|H^n|chi_nu>
//   into mu[nu] and Tr(sigma M_n) of the global 2x2 moments M_n into vmom;
//   reverse (wts != NULL): cotangents of L = sum w_nu,n mu_nu,n for every
//   bond block (Hbar, in the product type: float4 reductions in FP32) and
//   every onsite matrix
//   (obar = dL/d(Ebar, h_x, h_y, h_z)).
// Psi_0..Psi_K (and Psi-bar_1..Psi-bar_K) of the item live in the CTA's
// slot of global scratch, as in k_moments_adj.
constexpr int NCS = 8;

// chi_up = (-(x - i y), 1 + z) r, chi_dn = (1 + z, x + i y) r for z >= 0,
// chi_up = (1 - z, -(x + i y)) r, chi_dn = (x - i y, 1 - z) r otherwise
// (r normalises; the second form avoids the zero of 1 + z at s = -z).
__device__ __forceinline__ void start_spinors(const double* s, double* out) {
  const double x = s[0], y = s[1], z = s[2];
  if (z >= 0.0) {
    const double r = 1.0 / sqrt(2.0 * (1.0 + z));
    out[0] = -x * r; out[1] = y * r; out[2] = (1.0 + z) * r; out[3] = 0.0;
    out[4] = (1.0 + z) * r; out[5] = 0.0; out[6] = x * r; out[7] = y * r;
  } else {
    const double r = 1.0 / sqrt(2.0 * (1.0 - z));
    out[0] = (1.0 - z) * r; out[1] = 0.0; out[2] = -x * r; out[3] = -y * r;
    out[4] = x * r; out[5] = -y * r; out[6] = (1.0 - z) * r; out[7] = 0.0;
  }
}

// y = (Ebar + h.sigma) x for both spinors of one orbital row
template <typename T>
__device__ __forceinline__ void spin_onsite(T eb, T hx, T hy, T hz, const T* __restrict__ x, T* y) {
#pragma unroll
  for (int nu = 0; nu < 2; nu++) {
    const T ur = x[4 * nu], ui = x[4 * nu + 1], dr = x[4 * nu + 2], di = x[4 * nu + 3];
    y[4 * nu] = (eb + hz) * ur + hx * dr + hy * di;
    y[4 * nu + 1] = (eb + hz) * ui + hx * di - hy * dr;
    y[4 * nu + 2] = (eb - hz) * dr + hx * ur - hy * ui;
    y[4 * nu + 3] = (eb - hz) * di + hx * ui + hy * ur;
  }
}

// acc = (H x)[t] over columns s < ncol (onsite term when t < ncol)
template <typename T, int NO>
__device__ __forceinline__ void gather_row_nc(const ClusterView& cv, const T* __restrict__ H, int HS,
                                              const T* __restrict__ E, const double* __restrict__ sdir, int n,
                                              const int* __restrict__ satom, const long long* __restrict__ aoff,
                                              int t, int ncol, const T* __restrict__ x, T acc[NO][NCS]) {
#pragma unroll
  for (int r = 0; r < NO; r++)
#pragma unroll
    for (int c = 0; c < NCS; c++) acc[r][c] = T(0);
  if (t < ncol) {
    const int j = satom[t];
    const T sx = (T)sdir[3 * (size_t)j], sy = (T)sdir[3 * (size_t)j + 1], sz = (T)sdir[3 * (size_t)j + 2];
#pragma unroll
    for (int r = 0; r < NO; r++) {
      const T eu = E[(size_t)j * NO + r], ed = E[((size_t)n + j) * NO + r];
      const T f = T(0.5) * (ed - eu);
      spin_onsite<T>(T(0.5) * (eu + ed), f * sx, f * sy, f * sz, x + ((size_t)t * NO + r) * NCS, acc[r]);
    }
  }
  const long long q1 = aoff[t + 1];
  for (long long q = aoff[t]; q < q1; q++) {
    const int2 en = cv.adj[q];
    if (en.x >= ncol) break;
    block_apply<T, NO, NCS>(H + (size_t)en.y * HS, x + (size_t)en.x * NO * NCS, acc);
  }
}

// Tr(sigma M) of M = C L C^dagger, C = (chi_up chi_dn), L = [[Luu, Lud],
// [conj(Lud), Ldd]] the moments between the local states.
__device__ __forceinline__ void pauli_from_local(const double* chi, double Luu, double Ldd, double Lr, double Li,
                                                 double v[3]) {
  // C_a,nu = chi[nu * 4 + a * 2] + i chi[nu * 4 + a * 2 + 1]
  double M00 = 0.0, M11 = 0.0, M01r = 0.0, M01i = 0.0;
  const double L[2][2][2] = {{{Luu, 0.0}, {Lr, Li}}, {{Lr, -Li}, {Ldd, 0.0}}};  // [nu][nu'][re/im]
#pragma unroll
  for (int nu = 0; nu < 2; nu++)
#pragma unroll
    for (int mu_ = 0; mu_ < 2; mu_++) {
      const double lr = L[nu][mu_][0], li = L[nu][mu_][1];
      // M_ab += C_a,nu L_nu,mu conj(C_b,mu)
      const double c0r = chi[nu * 4], c0i = chi[nu * 4 + 1], c1r = chi[nu * 4 + 2], c1i = chi[nu * 4 + 3];
      const double d0r = chi[mu_ * 4], d0i = chi[mu_ * 4 + 1], d1r = chi[mu_ * 4 + 2], d1i = chi[mu_ * 4 + 3];
      // x = C_a,nu L
      const double x0r = c0r * lr - c0i * li, x0i = c0r * li + c0i * lr;
      const double x1r = c1r * lr - c1i * li, x1i = c1r * li + c1i * lr;
      M00 += x0r * d0r + x0i * d0i;
      M11 += x1r * d1r + x1i * d1i;
      M01r += x0r * d1r + x0i * d1i;
      M01i += x0i * d1r - x0r * d1i;
    }
  v[0] = 2.0 * M01r;
  v[1] = -2.0 * M01i;
  v[2] = M00 - M11;
}

template <typename T, int NO>
__global__ void __launch_bounds__(MOM_THREADS)
k_nc(ClusterView cv, const T* __restrict__ H, int HS, const T* __restrict__ onsite, const double* __restrict__ sdir,
     int n, int n_mom, int nwork, T* __restrict__ scratch, size_t slot_elems, double* __restrict__ mu,
     double* __restrict__ vmom, const double* __restrict__ wts, T* __restrict__ Hbar, int HSh,
     double* __restrict__ obar) {
  constexpr int RW = NO * NCS;
  __shared__ T ws[2][BOP_MAX_NMOM];
  __shared__ int s_lev[BOP_MAX_K + 1];
  __shared__ long long s_off[BOP_MAX_K + 2];
  __shared__ T red[8][MOM_THREADS / 32];
  __shared__ double chi[NCS];
  const bool rev = wts != nullptr;
  const int K = cv.K;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  T* psi = scratch + (size_t)blockIdx.x * slot_elems;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int atom = w / NO, al = w % NO;
    const long long s0 = cv.site_off[atom];
    const int* lev = cv.level_end + (size_t)atom * (K + 1);
    const int* satom = cv.site_atom + s0;
    const long long* aoff = cv.adj_off + s0;
    if (tid <= K) s_lev[tid] = lev[tid];
    if (tid == 0) {  // Psi_k at s_off[k], Psi-bar_k at s_off[K+1] + (s_off[k] - s_off[1])
      long long o = 0;
      for (int k = 0; k <= K; k++) {
        s_off[k] = o;
        o += (long long)lev[k] * RW;
      }
      s_off[K + 1] = o;
      start_spinors(sdir + 3 * (size_t)atom, chi);
    }
    if (rev)
      for (int q = tid; q < 2 * n_mom; q += blockDim.x) {
        const int nu = q / n_mom, m = q % n_mom;
        ws[nu][m] = (T)wts[(((size_t)nu * n + atom) * NO + al) * n_mom + m];
      }
    __syncthreads();
    T* P = psi;
    T* Pb = psi + s_off[K + 1] - s_off[1];
    for (int q = tid; q < RW; q += blockDim.x) P[q] = (q / NCS == al) ? (T)chi[q % NCS] : T(0);
    if (!rev && tid < 2) {
      mu[(((size_t)tid * n + atom) * NO + al) * n_mom] = 1.0;
      vmom[(((size_t)atom * NO + al) * n_mom) * 3 + tid] = 0.0;
      if (tid == 0) vmom[(((size_t)atom * NO + al) * n_mom) * 3 + 2] = 0.0;
    }
    __syncthreads();
    for (int k = 1; k <= K; k++) {
      const T* x = P + s_off[k - 1];
      T* y = P + s_off[k];
      T d[8];
#pragma unroll
      for (int v = 0; v < 8; v++) d[v] = T(0);
      for (int t = tid; t < s_lev[k]; t += blockDim.x) {
        T acc[NO][NCS];
        gather_row_nc<T, NO>(cv, H, HS, onsite, sdir, n, satom, aoff, t, s_lev[k - 1], x, acc);
#pragma unroll
        for (int r = 0; r < NO; r++)
#pragma unroll
          for (int c = 0; c < NCS; c++) y[((size_t)t * NO + r) * NCS + c] = acc[r][c];
        if (!rev) {
          // <Psi^nu|Psi^nu'>: up-up, dn-dn, and Re / Im of up-dn
#pragma unroll
          for (int r = 0; r < NO; r++) {
            const T* a = acc[r];
            d[4] += a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3];
            d[5] += a[4] * a[4] + a[5] * a[5] + a[6] * a[6] + a[7] * a[7];
            d[6] += a[0] * a[4] + a[1] * a[5] + a[2] * a[6] + a[3] * a[7];
            d[7] += a[0] * a[5] - a[1] * a[4] + a[2] * a[7] - a[3] * a[6];
            if (t < s_lev[k - 1]) {
              const T* p = x + ((size_t)t * NO + r) * NCS;
              d[0] += p[0] * a[0] + p[1] * a[1] + p[2] * a[2] + p[3] * a[3];
              d[1] += p[4] * a[4] + p[5] * a[5] + p[6] * a[6] + p[7] * a[7];
              d[2] += p[0] * a[4] + p[1] * a[5] + p[2] * a[6] + p[3] * a[7];
              d[3] += p[0] * a[5] - p[1] * a[4] + p[2] * a[7] - p[3] * a[6];
            }
          }
        }
      }
      if (!rev) {
#pragma unroll
        for (int v = 0; v < 8; v++) {
          const T r_ = warp_sum(d[v]);
          if (lane == 0) red[v][wid] = r_;
        }
        __syncthreads();
        if (tid < 2) {  // moment 2k-1 (tid 0) and 2k (tid 1)
          double L[4];
          for (int v = 0; v < 4; v++) {
            T a = T(0);
            for (int q = 0; q < MOM_THREADS / 32; q++) a += red[4 * tid + v][q];
            L[v] = (double)a;
          }
          const int m = 2 * k - 1 + tid;
          mu[((size_t)atom * NO + al) * n_mom + m] = L[0];
          mu[(((size_t)n + atom) * NO + al) * n_mom + m] = L[1];
          double v3[3];
          pauli_from_local(chi, L[0], L[1], L[2], L[3], v3);
          for (int xx = 0; xx < 3; xx++) vmom[(((size_t)atom * NO + al) * n_mom + m) * 3 + xx] = v3[xx];
        }
      }
      __syncthreads();
    }
    if (rev) {
      // Psi-bar_K = 2 w_2K Psi_K + w_2K-1 Psi_K-1 (weights of each spinor's columns)
      {
        const T* PK = P + s_off[K];
        const T* PK1 = P + s_off[K - 1];
        T* B = Pb + s_off[K];
        for (int q = tid; q < s_lev[K] * RW; q += blockDim.x) {
          const int t = q / RW, nu = (q % NCS) >> 2;
          T v = T(2) * ws[nu][2 * K] * PK[q];
          if (t < s_lev[K - 1]) v += ws[nu][2 * K - 1] * PK1[q];
          B[q] = v;
        }
      }
      __syncthreads();
      for (int k = K; k >= 2; k--) {
        const T* xb = Pb + s_off[k];
        T* yb = Pb + s_off[k - 1];
        const T* Pk = P + s_off[k];
        const T* Pk1 = P + s_off[k - 1];
        const T* Pk2 = P + s_off[k - 2];
        for (int t = tid; t < s_lev[k - 1]; t += blockDim.x) {
          T acc[NO][NCS];
          gather_row_nc<T, NO>(cv, H, HS, onsite, sdir, n, satom, aoff, t, s_lev[k], xb, acc);
#pragma unroll
          for (int r = 0; r < NO; r++)
#pragma unroll
            for (int c = 0; c < NCS; c++) {
              const size_t q = ((size_t)t * NO + r) * NCS + c;
              const int nu = c >> 2;
              T v = acc[r][c] + T(2) * ws[nu][2 * k - 2] * Pk1[q] + ws[nu][2 * k - 1] * Pk[q];
              if (t < s_lev[k - 2]) v += ws[nu][2 * k - 3] * Pk2[q];
              yb[q] = v;
            }
        }
        __syncthreads();
      }
      for (int t = tid; t < s_lev[K]; t += blockDim.x) {
        const int lt = site_level(s_lev, K, t);
        for (long long q = aoff[t]; q < aoff[t + 1]; q++) {
          const int2 en = cv.adj[q];
          const int sidx = en.x;
          if (sidx >= s_lev[K - 1]) break;
          const int ls = site_level(s_lev, K, sidx);
          const int kmin = lt > ls + 1 ? lt : ls + 1;
          T G[NO][NO];
#pragma unroll
          for (int b = 0; b < NO; b++)
#pragma unroll
            for (int g = 0; g < NO; g++) G[b][g] = T(0);
          for (int k = kmin; k <= K; k++) {
            const T* pb = Pb + s_off[k] + (size_t)t * RW;
            const T* ps = P + s_off[k - 1] + (size_t)sidx * RW;
#pragma unroll
            for (int b = 0; b < NO; b++)
#pragma unroll
              for (int g = 0; g < NO; g++) {
                T a = T(0);
#pragma unroll
                for (int c = 0; c < NCS; c++) a += pb[b * NCS + c] * ps[g * NCS + c];
                G[b][g] += a;
              }
          }
          add_bond_cotangent<T, NO>(Hbar + (size_t)en.y * HSh, G);
        }
        if (lt + 1 <= K) {
          // dL/d(Ebar, h) of the onsite matrix of (atom of t, b): the
          // derivatives of Ebar + h.sigma in the real form
          double* op = obar + (size_t)satom[t] * NO * 4;
#pragma unroll
          for (int b = 0; b < NO; b++) {
            T o0 = T(0), ox = T(0), oy = T(0), oz = T(0);
            for (int k = lt + 1; k <= K; k++) {
              const T* pb = Pb + s_off[k] + (size_t)t * RW + b * NCS;
              const T* pt = P + s_off[k - 1] + (size_t)t * RW + b * NCS;
#pragma unroll
              for (int nu = 0; nu < 2; nu++) {
                const T bur = pb[4 * nu], bui = pb[4 * nu + 1], bdr = pb[4 * nu + 2], bdi = pb[4 * nu + 3];
                const T pur = pt[4 * nu], pui = pt[4 * nu + 1], pdr = pt[4 * nu + 2], pdi = pt[4 * nu + 3];
                o0 += bur * pur + bui * pui + bdr * pdr + bdi * pdi;
                ox += bur * pdr + bui * pdi + bdr * pur + bdi * pui;
                oy += bur * pdi - bui * pdr - bdr * pui + bdi * pur;
                oz += bur * pur + bui * pui - bdr * pdr - bdi * pdi;
              }
            }
            atomicAdd(op + 4 * b, (double)o0);
            atomicAdd(op + 4 * b + 1, (double)ox);
            atomicAdd(op + 4 * b + 2, (double)oy);
            atomicAdd(op + 4 * b + 3, (double)oz);
          }
        }
      }
    }
    __syncthreads();
  }
}

// Forward-only form of k_nc: Psi_k-1 and Psi_k in two shared-memory
// buffers (even and odd levels, each sized for the largest such level
// below K over all atoms; Psi_K is never stored, only its inner products).
template <typename T, int NO>
__global__ void __launch_bounds__(MOM_THREADS)
k_nc_fwd(ClusterView cv, const T* __restrict__ H, int HS, const T* __restrict__ onsite,
         const double* __restrict__ sdir, int n, int n_mom, int nwork, int cap_even, double* __restrict__ mu,
         double* __restrict__ vmom) {
  constexpr int RW = NO * NCS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const buf0 = reinterpret_cast<T*>(smem_raw);
  T* const buf1 = buf0 + (size_t)cap_even * RW;
  __shared__ int s_lev[BOP_MAX_K + 1];
  __shared__ T red[8][MOM_THREADS / 32];
  __shared__ double chi[NCS];
  const int K = cv.K;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int atom = w / NO, al = w % NO;
    const long long s0 = cv.site_off[atom];
    const int* lev = cv.level_end + (size_t)atom * (K + 1);
    const int* satom = cv.site_atom + s0;
    const long long* aoff = cv.adj_off + s0;
    if (tid <= K) s_lev[tid] = lev[tid];
    if (tid == 0) start_spinors(sdir + 3 * (size_t)atom, chi);
    __syncthreads();
    for (int q = tid; q < RW; q += blockDim.x) buf0[q] = (q / NCS == al) ? (T)chi[q % NCS] : T(0);
    if (tid < 2) {
      mu[(((size_t)tid * n + atom) * NO + al) * n_mom] = 1.0;
      vmom[(((size_t)atom * NO + al) * n_mom) * 3 + tid] = 0.0;
      if (tid == 0) vmom[(((size_t)atom * NO + al) * n_mom) * 3 + 2] = 0.0;
    }
    __syncthreads();
    for (int k = 1; k <= K; k++) {
      const T* x = (k & 1) ? buf0 : buf1;  // level k-1
      T* y = (k & 1) ? buf1 : buf0;        // level k
      T d[8];
#pragma unroll
      for (int v = 0; v < 8; v++) d[v] = T(0);
      for (int t = tid; t < s_lev[k]; t += blockDim.x) {
        T acc[NO][NCS];
        gather_row_nc<T, NO>(cv, H, HS, onsite, sdir, n, satom, aoff, t, s_lev[k - 1], x, acc);
#pragma unroll
        for (int r = 0; r < NO; r++) {
          const T* a = acc[r];
          d[4] += a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3];
          d[5] += a[4] * a[4] + a[5] * a[5] + a[6] * a[6] + a[7] * a[7];
          d[6] += a[0] * a[4] + a[1] * a[5] + a[2] * a[6] + a[3] * a[7];
          d[7] += a[0] * a[5] - a[1] * a[4] + a[2] * a[7] - a[3] * a[6];
          if (t < s_lev[k - 1]) {
            const T* p = x + ((size_t)t * NO + r) * NCS;
            d[0] += p[0] * a[0] + p[1] * a[1] + p[2] * a[2] + p[3] * a[3];
            d[1] += p[4] * a[4] + p[5] * a[5] + p[6] * a[6] + p[7] * a[7];
            d[2] += p[0] * a[4] + p[1] * a[5] + p[2] * a[6] + p[3] * a[7];
            d[3] += p[0] * a[5] - p[1] * a[4] + p[2] * a[7] - p[3] * a[6];
          }
        }
        if (k < K) {
#pragma unroll
          for (int r = 0; r < NO; r++)
#pragma unroll
            for (int c = 0; c < NCS; c++) y[((size_t)t * NO + r) * NCS + c] = acc[r][c];
        }
      }
#pragma unroll
      for (int v = 0; v < 8; v++) {
        const T r_ = warp_sum(d[v]);
        if (lane == 0) red[v][wid] = r_;
      }
      __syncthreads();
      if (tid < 2) {  // moment 2k-1 (tid 0) and 2k (tid 1)
        double L[4];
        for (int v = 0; v < 4; v++) {
          T a = T(0);
          for (int q = 0; q < MOM_THREADS / 32; q++) a += red[4 * tid + v][q];
          L[v] = (double)a;
        }
        const int m = 2 * k - 1 + tid;
        mu[((size_t)atom * NO + al) * n_mom + m] = L[0];
        mu[(((size_t)n + atom) * NO + al) * n_mom + m] = L[1];
        double v3[3];
        pauli_from_local(chi, L[0], L[1], L[2], L[3], v3);
        for (int xx = 0; xx < 3; xx++) vmom[(((size_t)atom * NO + al) * n_mom + m) * 3 + xx] = v3[xx];
      }
      __syncthreads();
    }
  }
}

// Torques of Eq. torque, one thread per atom: dU/ds_i = sum_alpha
// [ (E_dn - E_up)/2 dU/dh_i alpha + sum_n (w_dn - w_up)/2 Tr(sigma M_n) ],
// t_i = dU/ds_i x s_i.
__global__ void k_torques(int n, int norb, int n_mom, const double* __restrict__ onsite,
                          const double* __restrict__ sdir, const double* __restrict__ w,
                          const double* __restrict__ vmom, const double* __restrict__ obar, double* __restrict__ t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double g[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < norb; a++) {
    const size_t o = (size_t)i * norb + a;
    const double half_delta = 0.5 * (onsite[(size_t)n * norb + o] - onsite[o]);
    for (int x = 0; x < 3; x++) g[x] += half_delta * obar[o * 4 + 1 + x];
    for (int m = 0; m < n_mom; m++) {
      const double c = 0.5 * (w[((size_t)n * norb + o) * n_mom + m] - w[o * n_mom + m]);
      for (int x = 0; x < 3; x++) g[x] += c * vmom[(o * n_mom + m) * 3 + x];
    }
  }
  const double sx = sdir[3 * (size_t)i], sy = sdir[3 * (size_t)i + 1], sz = sdir[3 * (size_t)i + 2];
  t[3 * (size_t)i] = g[1] * sz - g[2] * sy;
  t[3 * (size_t)i + 1] = g[2] * sx - g[0] * sz;
  t[3 * (size_t)i + 2] = g[0] * sy - g[1] * sx;
}

template <typename T, int NO>
int run_nc(const NcArgs& a, cudaStream_t s) {
  const int nwork = a.n * NO;
  if (nwork == 0) return 0;
  const int grid = nwork < a.slots ? nwork : a.slots;
  // forward only: both stored levels in shared memory when they fit
  const size_t smem = (size_t)(a.cap_even + a.cap_odd) * NO * NCS * sizeof(T);
  if (a.w == nullptr && a.cap_even >= 1 && a.cap_odd >= 1 && smem <= 200 * 1024) {
    auto fn = k_nc_fwd<T, NO>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return -1;
    fn<<<grid, MOM_THREADS, smem, s>>>(a.cv, (const T*)a.H, a.HS, (const T*)a.onsite, a.sdir, a.n, a.n_mom, nwork,
                                       a.cap_even, a.mu, a.vmom);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
  }
  k_nc<T, NO><<<grid, MOM_THREADS, 0, s>>>(a.cv, (const T*)a.H, a.HS, (const T*)a.onsite, a.sdir, a.n, a.n_mom,
                                           nwork, (T*)a.scratch, a.slot_elems, a.mu, a.vmom, a.w, (T*)a.Hbar, a.HSh,
                                           a.obar);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T, int NO, int NC>
int run_forward(const MomentsArgs& a, cudaStream_t s) {
  constexpr int N = NO * NC;
  constexpr int PS = (N == 1) ? 1 : Row<T, N>::PS;
  FwdSmem L{a.cap_even, a.cap_odd, a.max_sites, a.max_adj, true};
  size_t psi = (size_t)(a.cap_even + a.cap_odd) * PS * sizeof(T);
  size_t stage = (size_t)a.max_adj * 8 + (size_t)a.max_sites * 8 + (size_t)(a.max_sites + 1) * 8 +
                 (size_t)a.max_sites * 4 + 16;
  size_t smem = psi + stage;
  // stage the adjacency only while two CTAs (FP32) still fit on an SM
  const size_t budget = sizeof(T) == 4 ? 110 * 1024 : 200 * 1024;
  if (smem > budget) {
    L.stage = false;
    smem = psi;
  }
  if (smem > 227 * 1024) return -2;
  auto fn = k_moments<T, NO, NC>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int n_items = a.n * a.n_spin * (NO / NC);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, FWD_THREADS, smem);
  if (per_sm < 1) per_sm = 1;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int slots = sms * per_sm;
  const int chunk = (n_items + slots - 1) / slots;
  const int grid = (n_items + chunk - 1) / chunk;
  fn<<<grid, FWD_THREADS, smem, s>>>(a.cv, (const T*)a.H, a.HS, (const T*)a.onsite, a.n, a.n_on, a.n_mom, L,
                                      n_items, chunk, a.mu, (T*)a.pstore, a.psi_off, a.psi_tot);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T, int NO, int NC>
int run_adjoint(const AdjointArgs& a, cudaStream_t s) {
  int nwork = a.n * a.n_spin * (NO / NC);
  int grid = nwork < a.slots ? nwork : a.slots;
  k_moments_adj<T, NO, NC><<<grid, MOM_THREADS, 0, s>>>(a.cv, (const T*)a.H, a.HS, (const T*)a.onsite, a.n, a.n_on,
                                                       a.n_mom, nwork, a.w, (T*)a.scratch, a.slot_elems,
                                                       (T*)a.Hbar, a.HSh, a.Ebar);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T, int NO, int NC, bool HBAR>
int run_reverse(const AdjointArgs& a, cudaStream_t s) {
  constexpr int N = NO * NC;
  constexpr int PS = (N == 1) ? 1 : Row<T, N>::PS;
  RevSmem L{a.cap_even, a.cap_odd, a.max_sites, a.max_adj, a.cap_eb, true};
  const size_t psi = (size_t)(a.cap_even + a.cap_odd) * PS * sizeof(T) + eb_elems<T, NO>(a.cap_eb) * sizeof(T);
  const size_t stage = (size_t)a.max_adj * 8 + (size_t)a.max_sites * 8 + (size_t)(a.max_sites + 1) * 8 +
                       (size_t)a.max_sites * 4 + 16;
  auto fn = k_adj_rev<T, NO, NC, HBAR>;
  size_t smem = psi + stage;
  int per_sm = 0, per_sm_unstaged = 0;
  if (smem <= 227 * 1024) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, FWD_THREADS, smem);
  }
  if (psi > 227 * 1024) return -2;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psi);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_unstaged, fn, FWD_THREADS, psi);
  if (per_sm < per_sm_unstaged) {  // staging the adjacency would cost a resident CTA
    L.stage = false;
    smem = psi;
    per_sm = per_sm_unstaged;
  } else {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (per_sm < 1) per_sm = 1;
  const int n_items = a.n * a.n_spin * (NO / NC);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int slots = sms * per_sm;
  const int chunk = (n_items + slots - 1) / slots;
  const int grid = (n_items + chunk - 1) / chunk;
  fn<<<grid, FWD_THREADS, smem, s>>>(a.cv, (const T*)a.H, a.HS, (const T*)a.onsite, a.n, a.n_on, a.n_mom, L, n_items,
                                      chunk,
                                      (const T*)a.pstore, a.psi_off, a.psi_tot, a.w, (T*)a.Hbar, a.HSh,
                                      a.Ebar, a.siteval, a.sv_stride);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T, int NO, int NC>
int run_reverse_mode(const AdjointArgs& a, cudaStream_t s) {
  return a.Hbar ? run_reverse<T, NO, NC, true>(a, s) : run_reverse<T, NO, NC, false>(a, s);
}

}  // namespace

// Column grouping: all starting orbitals of an atom in one CTA when both Psi
// levels fit in shared memory, one CTA per starting orbital otherwise.
int moments_columns(int norb, int cap_sum, int fp64) {
  if (norb == 1) return 1;
  size_t bytes = (size_t)cap_sum * norb * norb * (fp64 ? 8 : 4);
  return bytes <= 100 * 1024 ? norb : 1;
}

int launch_moments(const MomentsArgs& a, int fp64, cudaStream_t s) {
  int nc = moments_columns(a.norb, a.cap_even + a.cap_odd, fp64);
  if (a.norb == 1) return fp64 ? run_forward<double, 1, 1>(a, s) : run_forward<float, 1, 1>(a, s);
  if (a.norb == 6) {
    if (nc == 6) return fp64 ? run_forward<double, 6, 6>(a, s) : run_forward<float, 6, 6>(a, s);
    return fp64 ? run_forward<double, 6, 1>(a, s) : run_forward<float, 6, 1>(a, s);
  }
  if (nc == 5) return fp64 ? run_forward<double, 5, 5>(a, s) : run_forward<float, 5, 5>(a, s);
  return fp64 ? run_forward<double, 5, 1>(a, s) : run_forward<float, 5, 1>(a, s);
}

int adjoint_columns(int norb) { return norb; }

int bond_cotangent_stride(int norb, int fp64) {
  if (norb == 1) return 1;
  if (norb == 5) return fp64 ? hbar_stride<double, 5>() : hbar_stride<float, 5>();
  return fp64 ? hbar_stride<double, 6>() : hbar_stride<float, 6>();
}

int launch_moments_adjoint(const AdjointArgs& a, int fp64, cudaStream_t s) {
  if (a.pstore != nullptr) {  // reverse sweep over stored Psi
    if (a.norb == 1) return fp64 ? run_reverse_mode<double, 1, 1>(a, s) : run_reverse_mode<float, 1, 1>(a, s);
    if (a.norb == 6) {
      if (a.nc == 6) return fp64 ? run_reverse_mode<double, 6, 6>(a, s) : run_reverse_mode<float, 6, 6>(a, s);
      return fp64 ? run_reverse_mode<double, 6, 1>(a, s) : run_reverse_mode<float, 6, 1>(a, s);
    }
    if (a.nc == 5) return fp64 ? run_reverse_mode<double, 5, 5>(a, s) : run_reverse_mode<float, 5, 5>(a, s);
    return fp64 ? run_reverse_mode<double, 5, 1>(a, s) : run_reverse_mode<float, 5, 1>(a, s);
  }
  if (a.norb == 1) return fp64 ? run_adjoint<double, 1, 1>(a, s) : run_adjoint<float, 1, 1>(a, s);
  if (a.norb == 6) return fp64 ? run_adjoint<double, 6, 6>(a, s) : run_adjoint<float, 6, 6>(a, s);
  return fp64 ? run_adjoint<double, 5, 5>(a, s) : run_adjoint<float, 5, 5>(a, s);
}

int launch_nc(const NcArgs& a, int fp64, cudaStream_t s) {
  if (a.norb == 1) return fp64 ? run_nc<double, 1>(a, s) : run_nc<float, 1>(a, s);
  if (a.norb == 6) return fp64 ? run_nc<double, 6>(a, s) : run_nc<float, 6>(a, s);
  return fp64 ? run_nc<double, 5>(a, s) : run_nc<float, 5>(a, s);
}

int launch_torques(int n, int norb, int n_mom, const double* onsite, const double* sdir, const double* w,
                   const double* vmom, const double* obar, double* t, cudaStream_t s) {
  if (n == 0) return 0;
  k_torques<<<(n + 127) / 128, 128, 0, s>>>(n, norb, n_mom, onsite, sdir, w, vmom, obar, t);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
