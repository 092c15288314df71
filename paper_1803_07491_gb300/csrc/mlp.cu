// The learned-terminator network 18 -> 128 -> 128 -> 10 (GELU): training
// (FP32 forward, reverse mode, Adam) and inference (bfloat16 weights,
// FP32 or FP64 activations) as tiled GEMMs with fused bias / GELU /
// GELU-derivative epilogues (the FP32 inference on the tensor pipe, the rest
// as SIMT tiles), plus the bop_mlp object of the C ABI.
//
// The layers are small dense contractions (K = 18, 128, 10) applied to
// every orbital of a structure (hundreds of thousands of rows); the MLP is
// a few per cent of an energy + force evaluation, so the kernels are plain
// 64 x 64 register-blocked tiles.  Every reduction (weight gradients over a
// batch, the loss, the bias gradients, the normalisation statistics) runs
// in a fixed order, so training is deterministic.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/bopgb.h"
#include "kernels.h"

namespace {

constexpr int NI = BOP_MLP_NIN, NH = BOP_MLP_NHID, NO = BOP_MLP_NOUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NPAR = OFF_B3 + NO;
static_assert(NPAR == BOP_MLP_NPARAM, "parameter layout");
constexpr int NORM_XM = 0, NORM_XS = NI, NORM_LO = 2 * NI, NORM_HI = 3 * NI, NORM_YM = 4 * NI,
              NORM_YS = 4 * NI + NO;
static_assert(NORM_YS + NO == BOP_MLP_NNORM, "normalisation layout");

constexpr int GBM = 64, GBN = 64, GBK = 16, GT = 256;
constexpr int KCHUNK = 512;  // batch rows per split of a weight-gradient GEMM
constexpr int RT = 256;

__device__ __forceinline__ float ld(const float* p, size_t i) { return p[i]; }
__device__ __forceinline__ double ld(const double* p, size_t i) { return p[i]; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p, size_t i) { return __bfloat162float(p[i]); }

__device__ __forceinline__ float ncdf(float x) { return normcdff(x); }
__device__ __forceinline__ double ncdf(double x) { return normcdf(x); }
__device__ __forceinline__ float nexp(float x) { return expf(x); }
__device__ __forceinline__ double nexp(double x) { return exp(x); }

// GELU(z) = z Phi(z); GELU'(z) = Phi(z) + z phi(z)
template <class T>
__device__ __forceinline__ T gelu(T z) {
  return z * ncdf(z);
}
template <class T>
__device__ __forceinline__ T gelu_d(T z) {
  return ncdf(z) + z * nexp(T(-0.5) * z * z) * T(0.39894228040143267794);
}

enum { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_DGELU = 3 };

struct GemmArgs {
  int M, N, K, lda, ldb, ldc, kchunk;
  const void* A;
  const void* B;
  void* C;
  const float* bias;  // EPI_BIAS, EPI_BIAS_GELU: [N]
  void* Z;            // EPI_BIAS_GELU: pre-activation out [M][ldc]; EPI_DGELU: pre-activation in
};

// C[m][n] = sum_k opA(m,k) opB(k,n) with
//   opA(m,k) = TA ? A[k lda + m] : A[m lda + k],
//   opB(k,n) = TB ? B[n ldb + k] : B[k ldb + n],
// over k in [z kchunk, min(K, (z+1) kchunk)) for split z = blockIdx.z (the
// output of split z starts at C + z M ldc).  Tiles of 64 x 64, 16-deep
// slabs in shared memory, 4 x 4 outputs per thread; ragged edges guarded.
template <class T, class TAe, class TBe, bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(GT) k_gemm(GemmArgs g) {
  __shared__ T As[GBK][GBM + 4];
  __shared__ T Bs[GBK][GBN + 4];
  const TAe* A = static_cast<const TAe*>(g.A);
  const TBe* B = static_cast<const TBe*>(g.B);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
  const int kb = blockIdx.z * g.kchunk;
  const int ke = min(g.K, kb + g.kchunk);
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = T(0);
  for (int k0 = kb; k0 < ke; k0 += GBK) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int e = tid + q * GT;
      int ml, kl;
      if (TA) { ml = e % GBM; kl = e / GBM; } else { ml = e / GBK; kl = e % GBK; }
      const int m = m0 + ml, k = k0 + kl;
      T v = T(0);
      if (m < g.M && k < ke) v = (T)ld(A, TA ? (size_t)k * g.lda + m : (size_t)m * g.lda + k);
      As[kl][ml] = v;
      int nl, kl2;
      if (TB) { kl2 = e % GBK; nl = e / GBK; } else { nl = e % GBN; kl2 = e / GBN; }
      const int n = n0 + nl, k2 = k0 + kl2;
      T w = T(0);
      if (n < g.N && k2 < ke) w = (T)ld(B, TB ? (size_t)n * g.ldb + k2 : (size_t)k2 * g.ldb + n);
      Bs[kl2][nl] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; kk++) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  T* C = static_cast<T*>(g.C) + (size_t)blockIdx.z * g.M * g.ldc;
  T* Z = static_cast<T*>(g.Z);
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int n = n0 + tx * 4 + j;
      if (n >= g.N) continue;
      const size_t o = (size_t)m * g.ldc + n;
      T v = acc[i][j];
      if (EPI == EPI_BIAS) {
        v += (T)g.bias[n];
      } else if (EPI == EPI_BIAS_GELU) {
        v += (T)g.bias[n];
        Z[o] = v;
        v = gelu(v);
      } else if (EPI == EPI_DGELU) {
        v *= gelu_d(Z[o]);
      }
      C[o] = v;
    }
  }
}

template <class T, class TAe, class TBe, bool TA, bool TB, int EPI>
int gemm(int M, int N, int K, const void* A, int lda, const void* B, int ldb, void* C, int ldc, const float* bias,
         void* Z, int kchunk, cudaStream_t s) {
  if (M <= 0 || N <= 0) return 0;
  GemmArgs g{M, N, K, lda, ldb, ldc, kchunk > 0 ? kchunk : K, A, B, C, bias, Z};
  const int splits = kchunk > 0 ? (K + kchunk - 1) / kchunk : 1;
  dim3 grid((M + GBM - 1) / GBM, (N + GBN - 1) / GBN, splits < 1 ? 1 : splits);
  k_gemm<T, TAe, TBe, TA, TB, EPI><<<grid, GT, 0, s>>>(g);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------- inference on the tensor pipe
// The FP32-activation inference GEMMs with bfloat16 weights on the tensor
// cores (mma.sync m16n8k16, bfloat16 operands, FP32 accumulation).  Every
// activation is split into three bfloat16 parts, a = a1 + a2 + a3 (a1 the
// rounding of a, a2 of the remainder, a3 of what is left: 24 significant
// bits, the FP32 value to within its last bits); the weights are exactly
// bfloat16, every product of parts is exact in FP32, and the three products
// accumulate in FP32, so that the result is the FP32 product of the FP32
// activations with the bfloat16 weights up to the order of the sums.
//
// C[m][n] = sum_k A[m][k] W(k, n) (+ epilogue), A float [M][lda] (k < K),
// W(k, n) = TB ? B[n ldb + k] : B[k ldb + n] (bfloat16), n < N.  KP, NP: K
// and N padded to the MMA tile (16, 8).  Persistent blocks of four warps,
// each warp 16 rows of a 64-row tile; the weights are staged once per block
// as Ws[n][k] (k contiguous: the B fragment's pairs are one 32-bit load).
constexpr int TC_WARPS = 4, TC_ROWS = 16 * TC_WARPS;

__device__ __forceinline__ unsigned pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// a = p[0] + p[1] + p[2] in bfloat16 parts
__device__ __forceinline__ void split3(float a, __nv_bfloat16 p[3]) {
  p[0] = __float2bfloat16_rn(a);
  float r = a - __bfloat162float(p[0]);
  p[1] = __float2bfloat16_rn(r);
  r = r - __bfloat162float(p[1]);
  p[2] = __float2bfloat16_rn(r);
}

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int KP, int NP, bool TB, int EPI>
__global__ void __launch_bounds__(32 * TC_WARPS) k_gemm_tc(GemmArgs g) {
  static_assert(KP % 16 == 0 && NP % 8 == 0, "tile padding");
  constexpr int WS = KP + 8;  // bfloat16 per weight row (conflict-free fragment loads)
  constexpr int AS = KP + 8;  // floats per staged activation row
  extern __shared__ __align__(16) unsigned char tc_raw[];
  __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(tc_raw);
  float* As = reinterpret_cast<float*>(tc_raw + (size_t)NP * WS * sizeof(__nv_bfloat16));
  const float* A = static_cast<const float*>(g.A);
  const __nv_bfloat16* B = static_cast<const __nv_bfloat16*>(g.B);
  float* C = static_cast<float*>(g.C);
  float* Z = static_cast<float*>(g.Z);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, tq = lane & 3;
  for (int q = tid; q < NP * KP; q += 32 * TC_WARPS) {
    const int n = q / KP, k = q % KP;
    __nv_bfloat16 w = __float2bfloat16_rn(0.f);
    if (n < g.N && k < g.K) w = TB ? B[(size_t)n * g.ldb + k] : B[(size_t)k * g.ldb + n];
    Ws[n * WS + k] = w;
  }
  float* Aw = As + (size_t)warp * 16 * AS;
  for (int m0 = blockIdx.x * TC_ROWS; m0 < g.M; m0 += gridDim.x * TC_ROWS) {
    __syncthreads();  // the weights (first tile) and the previous tile's reads are done
    const int r0 = m0 + warp * 16;
    for (int q = lane; q < 16 * KP; q += 32) {
      const int r = q / KP, k = q % KP;
      const int m = r0 + r;
      Aw[r * AS + k] = (m < g.M && k < g.K) ? A[(size_t)m * g.lda + k] : 0.f;
    }
    __syncwarp();
    float acc[NP / 8][4];
#pragma unroll
    for (int t = 0; t < NP / 8; t++)
#pragma unroll
      for (int j = 0; j < 4; j++) acc[t][j] = 0.f;
#pragma unroll
    for (int kk = 0; kk < KP; kk += 16) {
      // A fragments of the three parts: rows gq, gq + 8; columns 2tq, 2tq + 1 (+8)
      unsigned af[3][4];
      const int rr[4] = {gq, gq + 8, gq, gq + 8};
      const int cc[4] = {kk + 2 * tq, kk + 2 * tq, kk + 2 * tq + 8, kk + 2 * tq + 8};
#pragma unroll
      for (int f = 0; f < 4; f++) {
        const float2 v = *reinterpret_cast<const float2*>(Aw + rr[f] * AS + cc[f]);
        __nv_bfloat16 p0[3], p1[3];
        split3(v.x, p0);
        split3(v.y, p1);
#pragma unroll
        for (int sp = 0; sp < 3; sp++) af[sp][f] = pack_bf16x2(p0[sp], p1[sp]);
      }
#pragma unroll
      for (int t = 0; t < NP / 8; t++) {
        const __nv_bfloat16* wr = Ws + (t * 8 + gq) * WS + kk + 2 * tq;
        const unsigned b0 = *reinterpret_cast<const unsigned*>(wr);
        const unsigned b1 = *reinterpret_cast<const unsigned*>(wr + 8);
#pragma unroll
        for (int sp = 2; sp >= 0; sp--) mma_bf16(acc[t], af[sp], b0, b1);
      }
    }
    // epilogue: acc[t] = rows gq, gq + 8; columns t*8 + 2tq, + 1
#pragma unroll
    for (int t = 0; t < NP / 8; t++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int m = r0 + gq + 8 * h;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 2; j++) {
          const int n = t * 8 + 2 * tq + j;
          if (n >= g.N) continue;
          const size_t o = (size_t)m * g.ldc + n;
          float v = acc[t][2 * h + j];
          if (EPI == EPI_BIAS) {
            v += g.bias[n];
          } else if (EPI == EPI_BIAS_GELU) {
            v += g.bias[n];
            Z[o] = v;
            v = gelu(v);
          } else if (EPI == EPI_DGELU) {
            v *= gelu_d(Z[o]);
          }
          C[o] = v;
        }
      }
  }
}

template <int KP, int NP, bool TB, int EPI>
int gemm_tc(int M, int N, int K, const float* A, int lda, const __nv_bfloat16* B, int ldb, float* C, int ldc,
            const float* bias, float* Z, cudaStream_t s) {
  if (M <= 0 || N <= 0) return 0;
  if (K > KP || N > NP) return -1;
  GemmArgs g{M, N, K, lda, ldb, ldc, K, A, B, C, bias, Z};
  constexpr size_t smem = (size_t)NP * (KP + 8) * sizeof(__nv_bfloat16) + (size_t)TC_ROWS * (KP + 8) * sizeof(float);
  auto fn = k_gemm_tc<KP, NP, TB, EPI>;
  static int per_sm = 0, sms = 0;
  if (per_sm == 0) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * TC_WARPS, smem);
    if (per_sm < 1) per_sm = 1;
  }
  const int tiles = (M + TC_ROWS - 1) / TC_ROWS;
  const int grid = tiles < sms * per_sm ? tiles : sms * per_sm;
  fn<<<grid, 32 * TC_WARPS, smem, s>>>(g);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------- training kernels
// Batch rows idx[b] of the raw data, standardised; den = 10 sum mask by the
// last block (fixed order).  A row index outside [0, M) is read as a masked
// row of zeros and flagged in bad[0].
__global__ void __launch_bounds__(RT) k_gather(int B, long long M, unsigned* bad, const int* __restrict__ idx,
                                               const float* __restrict__ x,
                                               const float* __restrict__ t, const float* __restrict__ mask,
                                               const float* __restrict__ norm, float* xs, float* ts, float* mb,
                                               double* part, unsigned* counter, float* den) {
  __shared__ double sh[RT / 32 + 1];
  __shared__ bool last;
  const int b = blockIdx.x * RT + threadIdx.x;
  double mv = 0.0;
  if (b < B) {
    const long long r = idx[b];
    if (r >= 0 && r < M) {
      for (int j = 0; j < NI; j++)
        xs[(size_t)b * NI + j] = (x[r * NI + j] - norm[NORM_XM + j]) / norm[NORM_XS + j];
      for (int j = 0; j < NO; j++)
        ts[(size_t)b * NO + j] = (t[r * NO + j] - norm[NORM_YM + j]) / norm[NORM_YS + j];
      mb[b] = mask[r];
      mv = mask[r];
    } else {
      for (int j = 0; j < NI; j++) xs[(size_t)b * NI + j] = 0.f;
      for (int j = 0; j < NO; j++) ts[(size_t)b * NO + j] = 0.f;
      mb[b] = 0.f;
      atomicOr(bad, 1u);
    }
  }
  for (int o = 16; o > 0; o >>= 1) mv += __shfl_xor_sync(0xffffffffu, mv, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mv;
  __syncthreads();
  if (threadIdx.x == 0) {
    double q = 0.0;
    for (int w = 0; w < RT / 32; w++) q += sh[w];
    part[blockIdx.x] = q;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  double q = 0.0;
  for (int k = 0; k < (int)gridDim.x; k++) q += __ldcg(part + k);
  den[0] = (float)(NO * (q > 1.0 ? q : 1.0));
  *counter = 0;
}

// dY = 2 (Y - T) m / den; loss = sum m (Y - T)^2 / den (last block).
__global__ void __launch_bounds__(RT) k_mse(int B, const float* __restrict__ y, const float* __restrict__ ts,
                                            const float* __restrict__ mb, const float* __restrict__ den, float* dy,
                                            double* part, unsigned* counter, float* loss) {
  __shared__ double sh[RT / 32 + 1];
  __shared__ bool last;
  const int b = blockIdx.x * RT + threadIdx.x;
  const float d = den[0];
  double acc = 0.0;
  if (b < B) {
    const float m = mb[b];
    for (int j = 0; j < NO; j++) {
      const float r = (y[(size_t)b * NO + j] - ts[(size_t)b * NO + j]) * m;
      dy[(size_t)b * NO + j] = 2.0f * r / d;
      acc += (double)r * r;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double q = 0.0;
    for (int w = 0; w < RT / 32; w++) q += sh[w];
    part[blockIdx.x] = q;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  double q = 0.0;
  for (int k = 0; k < (int)gridDim.x; k++) q += __ldcg(part + k);
  if (loss) loss[0] = (float)(q / d);
  *counter = 0;
}

// out[i] = sum_s parts[s][i], s ascending.
__global__ void k_sum_splits(int n, int S, const float* __restrict__ parts, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v = 0.f;
  for (int s = 0; s < S; s++) v += parts[(size_t)s * n + i];
  out[i] = v;
}

// out[n] = sum_b X[b][n]: one block per column, strided partial sums and a
// fixed shuffle tree.
__global__ void __launch_bounds__(RT) k_colsum(int B, int N, const float* __restrict__ X, float* out) {
  __shared__ float sh[RT / 32];
  const int n = blockIdx.x;
  float v = 0.f;
  for (int b = threadIdx.x; b < B; b += RT) v += X[(size_t)b * N + n];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float q = 0.f;
    for (int w = 0; w < RT / 32; w++) q += sh[w];
    out[n] = q;
  }
}

// Adam (bias-corrected), then the bfloat16 copy used for inference.
__global__ void k_adam(int n, float* p, const float* __restrict__ g, float* m, float* v, float lr, float b1, float b2,
                       float eps, float c1, float c2, __nv_bfloat16* wbf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / c1, vh = vi / c2;
  const float pi = p[i] - lr * mh / (sqrtf(vh) + eps);
  p[i] = pi;
  wbf[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(int n, const float* __restrict__ p, __nv_bfloat16* wbf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wbf[i] = __float2bfloat16_rn(p[i]);
}

// Normalisation statistics, one block per column (18 inputs, then 10
// targets) over the rows with mask > 0: mean, population standard deviation
// (floored at 1e-6), and for inputs the range widened by 5 % of its span.
__global__ void __launch_bounds__(RT) k_norm_stats(long long M, const float* __restrict__ x,
                                                   const float* __restrict__ t, const float* __restrict__ mask,
                                                   float* norm) {
  __shared__ double sa[RT / 32], sb[RT / 32], smn[RT / 32], smx[RT / 32];
  __shared__ double mean_s;
  const int c = blockIdx.x;
  const bool isx = c < NI;
  const int j = isx ? c : c - NI;
  const float* src = isx ? x : t;
  const int ld_ = isx ? NI : NO;
  double s = 0.0, w = 0.0, mn = 1e300, mx = -1e300;
  for (long long r = threadIdx.x; r < M; r += RT) {
    if (!(mask[r] > 0.f)) continue;
    const double v = src[r * ld_ + j];
    s += v;
    w += 1.0;
    mn = fmin(mn, v);
    mx = fmax(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    w += __shfl_xor_sync(0xffffffffu, w, o);
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = s;
    sb[threadIdx.x >> 5] = w;
    smn[threadIdx.x >> 5] = mn;
    smx[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, W = 0.0, MN = 1e300, MX = -1e300;
    for (int q = 0; q < RT / 32; q++) {
      S += sa[q];
      W += sb[q];
      MN = fmin(MN, smn[q]);
      MX = fmax(MX, smx[q]);
    }
    mean_s = W > 0.0 ? S / W : 0.0;
    sa[0] = W;
    smn[0] = MN;
    smx[0] = MX;
  }
  __syncthreads();
  const double mean = mean_s, W = sa[0], MN = smn[0], MX = smx[0];
  double q2 = 0.0;
  for (long long r = threadIdx.x; r < M; r += RT) {
    if (!(mask[r] > 0.f)) continue;
    const double d = src[r * ld_ + j] - mean;
    q2 += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) q2 += __shfl_xor_sync(0xffffffffu, q2, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = q2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double Q = 0.0;
    for (int q = 0; q < RT / 32; q++) Q += sb[q];
    double sd = W > 0.0 ? sqrt(Q / W) : 1.0;
    if (sd < 1e-6) sd = 1e-6;
    if (isx) {
      const double span = MX - MN;
      norm[NORM_XM + j] = (float)mean;
      norm[NORM_XS + j] = (float)sd;
      norm[NORM_LO + j] = (float)(MN - 0.05 * span);
      norm[NORM_HI + j] = (float)(MX + 0.05 * span);
    } else {
      norm[NORM_YM + j] = (float)mean;
      norm[NORM_YS + j] = (float)sd;
    }
  }
}

// Standardise raw inputs / de-standardise outputs (prediction entry point).
__global__ void k_standardise(long long M, const float* __restrict__ x, const float* __restrict__ norm, float* xs) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * NI) return;
  const int j = (int)(i % NI);
  xs[i] = (x[i] - norm[NORM_XM + j]) / norm[NORM_XS + j];
}
__global__ void k_destandardise(long long M, const float* __restrict__ ys, const float* __restrict__ norm,
                                float* y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * NO) return;
  const int j = (int)(i % NO);
  y[i] = norm[NORM_YM + j] + norm[NORM_YS + j] * ys[i];
}

int grid1(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------- inference (energy path)
// ys = net(xs) for M rows; Z1, Z2 keep the pre-activations for the reverse.
int mlp_infer_forward(int fp64, int M, const void* xs, const float* params, const void* wbf, void* Z1, void* H1,
                      void* Z2, void* H2, void* ys, cudaStream_t s) {
  const __nv_bfloat16* w = static_cast<const __nv_bfloat16*>(wbf);
  int r = 0;
  if (fp64) {
    r |= gemm<double, double, __nv_bfloat16, false, true, EPI_BIAS_GELU>(M, NH, NI, xs, NI, w + OFF_W1, NI, H1, NH,
                                                                         params + OFF_B1, Z1, 0, s);
    r |= gemm<double, double, __nv_bfloat16, false, true, EPI_BIAS_GELU>(M, NH, NH, H1, NH, w + OFF_W2, NH, H2, NH,
                                                                         params + OFF_B2, Z2, 0, s);
    r |= gemm<double, double, __nv_bfloat16, false, true, EPI_BIAS>(M, NO, NH, H2, NH, w + OFF_W3, NH, ys, NO,
                                                                    params + OFF_B3, nullptr, 0, s);
  } else {  // tensor pipe (three bfloat16 parts per FP32 activation)
    r |= gemm_tc<32, 128, true, EPI_BIAS_GELU>(M, NH, NI, (const float*)xs, NI, w + OFF_W1, NI, (float*)H1, NH,
                                               params + OFF_B1, (float*)Z1, s);
    r |= gemm_tc<128, 128, true, EPI_BIAS_GELU>(M, NH, NH, (const float*)H1, NH, w + OFF_W2, NH, (float*)H2, NH,
                                                params + OFF_B2, (float*)Z2, s);
    r |= gemm_tc<128, 16, true, EPI_BIAS>(M, NO, NH, (const float*)H2, NH, w + OFF_W3, NH, (float*)ys, NO,
                                          params + OFF_B3, nullptr, s);
  }
  return r;
}

// xbar = (d ys / d xs)^T ybar for M rows; dZ1, dZ2 are scratch [M][128].
int mlp_infer_backward(int fp64, int M, const void* ybar, const void* wbf, void* Z1, void* Z2, void* dZ1, void* dZ2,
                       void* xbar, cudaStream_t s) {
  const __nv_bfloat16* w = static_cast<const __nv_bfloat16*>(wbf);
  int r = 0;
  if (fp64) {
    r |= gemm<double, double, __nv_bfloat16, false, false, EPI_DGELU>(M, NH, NO, ybar, NO, w + OFF_W3, NH, dZ2, NH,
                                                                      nullptr, Z2, 0, s);
    r |= gemm<double, double, __nv_bfloat16, false, false, EPI_DGELU>(M, NH, NH, dZ2, NH, w + OFF_W2, NH, dZ1, NH,
                                                                      nullptr, Z1, 0, s);
    r |= gemm<double, double, __nv_bfloat16, false, false, EPI_NONE>(M, NI, NH, dZ1, NH, w + OFF_W1, NI, xbar, NI,
                                                                     nullptr, nullptr, 0, s);
  } else {  // tensor pipe (three bfloat16 parts per FP32 cotangent)
    r |= gemm_tc<16, 128, false, EPI_DGELU>(M, NH, NO, (const float*)ybar, NO, w + OFF_W3, NH, (float*)dZ2, NH,
                                            nullptr, (float*)Z2, s);
    r |= gemm_tc<128, 128, false, EPI_DGELU>(M, NH, NH, (const float*)dZ2, NH, w + OFF_W2, NH, (float*)dZ1, NH,
                                             nullptr, (float*)Z1, s);
    r |= gemm_tc<128, 24, false, EPI_NONE>(M, NI, NH, (const float*)dZ1, NH, w + OFF_W1, NI, (float*)xbar, NI,
                                           nullptr, nullptr, s);
  }
  return r;
}

// ---------------------------------------------------------------- the bop_mlp object
struct MBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct bop_mlp {
  MBuf params, grad, am, av, wbf, norm;
  MBuf xs, ts, mb, Z1, H1, Z2, H2, y, dy, parts, red, counter, den, loss, bad;
  int adam_t = 0;
  int batch_cap = 0;
  char err[256];
};

namespace {

int mfail(bop_mlp* n, int code, const char* fmt, ...) {
  if (n) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(n->err, sizeof(n->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

int mensure(bop_mlp* n, MBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return BOP_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return mfail(n, BOP_ERR_OOM, "cudaMalloc(%zu) failed", bytes);
  }
  b.bytes = bytes;
  return BOP_OK;
}

template <class T>
T* MP(MBuf& b) {
  return reinterpret_cast<T*>(b.p);
}

#define MCK(call)                                                                                        \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) return mfail(net, BOP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

int size_batch(bop_mlp* net, int B) {
  if (B <= net->batch_cap) return BOP_OK;
  int r;
  const size_t b = (size_t)B;
  const int S = (B + KCHUNK - 1) / KCHUNK;
  if ((r = mensure(net, net->xs, sizeof(float) * b * NI)) || (r = mensure(net, net->ts, sizeof(float) * b * NO)) ||
      (r = mensure(net, net->mb, sizeof(float) * b)) || (r = mensure(net, net->Z1, sizeof(float) * b * NH)) ||
      (r = mensure(net, net->H1, sizeof(float) * b * NH)) || (r = mensure(net, net->Z2, sizeof(float) * b * NH)) ||
      (r = mensure(net, net->H2, sizeof(float) * b * NH)) || (r = mensure(net, net->y, sizeof(float) * b * NO)) ||
      (r = mensure(net, net->dy, sizeof(float) * b * NO)) ||
      (r = mensure(net, net->parts, sizeof(float) * (size_t)S * NH * NH)) ||
      (r = mensure(net, net->red, sizeof(double) * (b / RT + 2))))
    return r;
  net->batch_cap = B;
  return BOP_OK;
}

}  // namespace

const float* mlp_params_dev(const bop_mlp* net) { return static_cast<const float*>(net->params.p); }
const void* mlp_wbf_dev(const bop_mlp* net) { return net->wbf.p; }
const float* mlp_norm_dev(const bop_mlp* net) { return static_cast<const float*>(net->norm.p); }

extern "C" {

int bop_mlp_create(bop_mlp** out, const float* params_host) {
  if (!out || !params_host) return BOP_ERR_ARG;
  *out = nullptr;
  bop_mlp* net = new (std::nothrow) bop_mlp();
  if (!net) return BOP_ERR_OOM;
  net->err[0] = 0;
  int r;
  if ((r = mensure(net, net->params, sizeof(float) * NPAR)) || (r = mensure(net, net->grad, sizeof(float) * NPAR)) ||
      (r = mensure(net, net->am, sizeof(float) * NPAR)) || (r = mensure(net, net->av, sizeof(float) * NPAR)) ||
      (r = mensure(net, net->wbf, sizeof(__nv_bfloat16) * NPAR)) ||
      (r = mensure(net, net->norm, sizeof(float) * BOP_MLP_NNORM)) || (r = mensure(net, net->counter, 16)) ||
      (r = mensure(net, net->den, 16)) || (r = mensure(net, net->loss, 16)) || (r = mensure(net, net->bad, 16))) {
    bop_mlp_destroy(net);
    return r;
  }
  float norm0[BOP_MLP_NNORM];
  for (int j = 0; j < BOP_MLP_NNORM; j++) norm0[j] = 0.f;
  for (int j = 0; j < NI; j++) {
    norm0[NORM_XS + j] = 1.f;
    norm0[NORM_LO + j] = -3.0e38f;
    norm0[NORM_HI + j] = 3.0e38f;
  }
  for (int j = 0; j < NO; j++) norm0[NORM_YS + j] = 1.f;
  if (cudaMemcpy(net->params.p, params_host, sizeof(float) * NPAR, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(net->norm.p, norm0, sizeof(norm0), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(net->am.p, 0, sizeof(float) * NPAR) != cudaSuccess ||
      cudaMemset(net->av.p, 0, sizeof(float) * NPAR) != cudaSuccess ||
      cudaMemset(net->counter.p, 0, 16) != cudaSuccess || cudaMemset(net->bad.p, 0, 16) != cudaSuccess) {
    bop_mlp_destroy(net);
    return BOP_ERR_CUDA;
  }
  k_to_bf16<<<grid1(NPAR, 256), 256>>>(NPAR, MP<float>(net->params), MP<__nv_bfloat16>(net->wbf));
  if (cudaDeviceSynchronize() != cudaSuccess) {
    bop_mlp_destroy(net);
    return BOP_ERR_CUDA;
  }
  *out = net;
  return BOP_OK;
}

int bop_mlp_destroy(bop_mlp* net) {
  if (!net) return BOP_OK;
  for (MBuf* b : {&net->params, &net->grad, &net->am, &net->av, &net->wbf, &net->norm, &net->xs, &net->ts, &net->mb,
                  &net->Z1, &net->H1, &net->Z2, &net->H2, &net->y, &net->dy, &net->parts, &net->red, &net->counter,
                  &net->den, &net->loss, &net->bad})
    if (b->p) cudaFree(b->p);
  delete net;
  return BOP_OK;
}

const char* bop_mlp_last_error(const bop_mlp* net) { return net ? net->err : "net is NULL"; }

int bop_mlp_get(bop_mlp* net, float* params_host, float* norm_host) {
  if (!net) return BOP_ERR_ARG;
  if (params_host) MCK(cudaMemcpy(params_host, net->params.p, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
  if (norm_host) MCK(cudaMemcpy(norm_host, net->norm.p, sizeof(float) * BOP_MLP_NNORM, cudaMemcpyDeviceToHost));
  return BOP_OK;
}

int bop_mlp_set_norm(bop_mlp* net, const float* norm_host) {
  if (!net || !norm_host) return BOP_ERR_ARG;
  for (int j = 0; j < NI; j++)
    if (!(norm_host[NORM_XS + j] > 0.f)) return mfail(net, BOP_ERR_ARG, "input standard deviation %d not > 0", j);
  for (int j = 0; j < NO; j++)
    if (!(norm_host[NORM_YS + j] > 0.f)) return mfail(net, BOP_ERR_ARG, "target standard deviation %d not > 0", j);
  MCK(cudaMemcpy(net->norm.p, norm_host, sizeof(float) * BOP_MLP_NNORM, cudaMemcpyHostToDevice));
  return BOP_OK;
}

int bop_mlp_fit_norm(bop_mlp* net, long long M, const float* x, const float* t, const float* mask,
                     bop_stream stream) {
  if (!net || M < 1 || !x || !t || !mask) return mfail(net, BOP_ERR_ARG, "need M >= 1, x, t and mask");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_norm_stats<<<NI + NO, RT, 0, s>>>(M, x, t, mask, MP<float>(net->norm));
  MCK(cudaGetLastError());
  return BOP_OK;
}

int bop_mlp_gradient(bop_mlp* net, long long M, const float* x, const float* t, const float* mask, const int* idx,
                     int batch, float* grad_out, float* loss_out, bop_stream stream) {
  if (!net || M < 1 || !x || !t || !mask || !idx || batch < 1)
    return mfail(net, BOP_ERR_ARG, "need M >= 1, x, t, mask, idx and batch >= 1");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int r = size_batch(net, batch);
  if (r) return r;
  const int B = batch;
  const int nb = grid1(B, RT);
  float* P = MP<float>(net->params);
  float* G = MP<float>(net->grad);
  float* xs = MP<float>(net->xs);
  float* Z1 = MP<float>(net->Z1);
  float* H1 = MP<float>(net->H1);
  float* Z2 = MP<float>(net->Z2);
  float* H2 = MP<float>(net->H2);
  float* y = MP<float>(net->y);
  float* dy = MP<float>(net->dy);
  float* parts = MP<float>(net->parts);
  k_gather<<<nb, RT, 0, s>>>(B, M, MP<unsigned>(net->bad), idx, x, t, mask, MP<float>(net->norm), xs, MP<float>(net->ts), MP<float>(net->mb),
                             MP<double>(net->red), MP<unsigned>(net->counter), MP<float>(net->den));
  int e = 0;
  // forward (FP32 master weights)
  e |= gemm<float, float, float, false, true, EPI_BIAS_GELU>(B, NH, NI, xs, NI, P + OFF_W1, NI, H1, NH, P + OFF_B1,
                                                             Z1, 0, s);
  e |= gemm<float, float, float, false, true, EPI_BIAS_GELU>(B, NH, NH, H1, NH, P + OFF_W2, NH, H2, NH, P + OFF_B2,
                                                             Z2, 0, s);
  e |= gemm<float, float, float, false, true, EPI_BIAS>(B, NO, NH, H2, NH, P + OFF_W3, NH, y, NO, P + OFF_B3, nullptr,
                                                        0, s);
  k_mse<<<nb, RT, 0, s>>>(B, y, MP<float>(net->ts), MP<float>(net->mb), MP<float>(net->den), dy,
                          MP<double>(net->red), MP<unsigned>(net->counter), loss_out ? loss_out : MP<float>(net->loss));
  const int S = (B + KCHUNK - 1) / KCHUNK;
  // layer 3: dW3 = dy^T H2, db3 = sum dy
  e |= gemm<float, float, float, true, false, EPI_NONE>(NO, NH, B, dy, NO, H2, NH, parts, NH, nullptr, nullptr,
                                                        KCHUNK, s);
  k_sum_splits<<<grid1(NO * NH, 256), 256, 0, s>>>(NO * NH, S, parts, G + OFF_W3);
  k_colsum<<<NO, RT, 0, s>>>(B, NO, dy, G + OFF_B3);
  // dZ2 = (dy W3) * gelu'(Z2), in place of Z2
  e |= gemm<float, float, float, false, false, EPI_DGELU>(B, NH, NO, dy, NO, P + OFF_W3, NH, Z2, NH, nullptr, Z2, 0,
                                                          s);
  e |= gemm<float, float, float, true, false, EPI_NONE>(NH, NH, B, Z2, NH, H1, NH, parts, NH, nullptr, nullptr,
                                                        KCHUNK, s);
  k_sum_splits<<<grid1(NH * NH, 256), 256, 0, s>>>(NH * NH, S, parts, G + OFF_W2);
  k_colsum<<<NH, RT, 0, s>>>(B, NH, Z2, G + OFF_B2);
  // dZ1 = (dZ2 W2) * gelu'(Z1), in place of Z1
  e |= gemm<float, float, float, false, false, EPI_DGELU>(B, NH, NH, Z2, NH, P + OFF_W2, NH, Z1, NH, nullptr, Z1, 0,
                                                          s);
  e |= gemm<float, float, float, true, false, EPI_NONE>(NH, NI, B, Z1, NH, xs, NI, parts, NI, nullptr, nullptr,
                                                        KCHUNK, s);
  k_sum_splits<<<grid1(NH * NI, 256), 256, 0, s>>>(NH * NI, S, parts, G + OFF_W1);
  k_colsum<<<NH, RT, 0, s>>>(B, NH, Z1, G + OFF_B1);
  if (e) return mfail(net, BOP_ERR_CUDA, "gemm launch failed");
  if (grad_out) MCK(cudaMemcpyAsync(grad_out, G, sizeof(float) * NPAR, cudaMemcpyDeviceToDevice, s));
  MCK(cudaGetLastError());
  return BOP_OK;
}

int bop_mlp_check(bop_mlp* net, bop_stream stream) {
  if (!net) return BOP_ERR_ARG;
  unsigned h = 0;
  MCK(cudaMemcpyAsync(&h, net->bad.p, sizeof(unsigned), cudaMemcpyDeviceToHost, reinterpret_cast<cudaStream_t>(stream)));
  MCK(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  if (!h) return BOP_OK;
  MCK(cudaMemset(net->bad.p, 0, sizeof(unsigned)));
  return mfail(net, BOP_ERR_ARG, "a batch row index was outside [0, M)");
  return BOP_OK;
}

int bop_mlp_adam(bop_mlp* net, float lr, bop_stream stream) {
  if (!net || !(lr > 0.f)) return mfail(net, BOP_ERR_ARG, "need lr > 0");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  net->adam_t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, net->adam_t)), c2 = (float)(1.0 - std::pow(b2, net->adam_t));
  k_adam<<<grid1(NPAR, 256), 256, 0, s>>>(NPAR, MP<float>(net->params), MP<float>(net->grad), MP<float>(net->am),
                                          MP<float>(net->av), lr, (float)b1, (float)b2, 1e-8f, c1, c2,
                                          MP<__nv_bfloat16>(net->wbf));
  MCK(cudaGetLastError());
  return BOP_OK;
}

int bop_mlp_train_step(bop_mlp* net, long long M, const float* x, const float* t, const float* mask, const int* idx,
                       int batch, float lr, float* loss_out, bop_stream stream) {
  int r = bop_mlp_gradient(net, M, x, t, mask, idx, batch, nullptr, loss_out, stream);
  if (r) return r;
  return bop_mlp_adam(net, lr, stream);
}

int bop_mlp_predict(bop_mlp* net, long long M, const float* x, float* y, bop_stream stream) {
  if (!net || M < 1 || !x || !y) return mfail(net, BOP_ERR_ARG, "need M >= 1, x and y");
  if (M > 0x7fffffffLL / NH) return mfail(net, BOP_ERR_ARG, "M too large");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int r = size_batch(net, (int)M);
  if (r) return r;
  k_standardise<<<grid1(M * NI, 256), 256, 0, s>>>(M, x, MP<float>(net->norm), MP<float>(net->xs));
  if (mlp_infer_forward(0, (int)M, net->xs.p, MP<float>(net->params), net->wbf.p, net->Z1.p, net->H1.p, net->Z2.p,
                        net->H2.p, net->y.p, s))
    return mfail(net, BOP_ERR_CUDA, "gemm launch failed");
  k_destandardise<<<grid1(M * NO, 256), 256, 0, s>>>(M, MP<float>(net->y), MP<float>(net->norm), y);
  MCK(cudaGetLastError());
  return BOP_OK;
}

}  // extern "C"
