// bop_fermi_level_noalloc: the Fermi-level search of the library for callers
// that cannot allocate device memory.  Such callers include code that runs
// under a memory budget fixed in advance, hosts that pre-reserve all GPU
// memory at start-up (so a later cudaMalloc would fail or break their
// accounting), and paths where an allocation would synchronise the device
// at the wrong moment.
//
// The search runs the library's bisection kernels (k_bracket, k_fermi_round
// in scalar.cu; bop_energy finds the same root with Newton steps inside the
// bisection bracket).  Their scratch (the sine-series coefficients
// of N(phi), the per-block partial sums, the completion counter and the
// bracket state) lives in one file-scope __device__ array instead of
// context buffers.  Every GPU that loads the library holds that array until
// the process exits.
#include <cstdio>
#include <mutex>

#include "../../include/bopgb.h"
#include "kernels.h"

namespace {

constexpr size_t NOALLOC_BYTES = (size_t)16 << 20;  // 16 MiB
constexpr size_t OFF_STATE = 0;                     // FermiState
constexpr size_t OFF_COUNTER = 256;                 // unsigned completion counter
constexpr size_t OFF_PARTIALS = 512;                // 2 x 1024 doubles of block partials
constexpr size_t OFF_D = OFF_PARTIALS + 2 * 1024 * sizeof(double);
constexpr int MAX_DEVICES = 64;
constexpr double PI = 3.14159265358979323846;

}  // namespace

// The scratch.  In host code this name is only a stand-in for the device
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_fermi_scratch[NOALLOC_BYTES];

namespace {

std::mutex g_mutex;
unsigned char* g_addr[MAX_DEVICES] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and kept for the life of the process:
// it does not survive a cudaDeviceReset (or any other reset of the primary
// context), after which calls of this entry point are not supported.
int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return BOP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_fermi_scratch);
    if (e != cudaSuccess) {
      fprintf(stderr, "bop_fermi_level_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
      return BOP_ERR_CUDA;
    }
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return BOP_OK;
}

// D_0 = g_0 s_0, D_k = (g s_{k-2} - g s_k) / (pi k) for k = 1 .. n_exp + 2
// (g s_j = 0 outside 0 .. n_exp): N(phi) = D_0 (1 - phi/pi) + sum_k D_k sin(k phi).
__global__ void k_gsig_to_D(int M, int ne, const double* __restrict__ gsig, double* __restrict__ D) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long tot = (long long)(ne + 3) * M;
  if (q >= tot) return;
  int k = (int)(q / M), o = (int)(q % M);
  if (k == 0) {
    D[q] = gsig[o];
    return;
  }
  double lo = (k - 2 >= 0 && k - 2 <= ne) ? gsig[(size_t)(k - 2) * M + o] : 0.0;
  double hi = (k <= ne) ? gsig[(size_t)k * M + o] : 0.0;
  D[q] = (lo - hi) / (PI * k);
}

__global__ void k_copy_ef(const FermiState* st, double* out) { *out = st->ef; }

}  // namespace

extern "C" int bop_fermi_level_noalloc(int M, int n_exp, const double* gsig, const double* a_inf,
                                       const double* b_inf, double spin_factor, double n_electrons,
                                       double* e_fermi, bop_stream stream) {
  if (M < 1 || n_exp < 2 || n_exp > BOP_MAX_NEXP || !gsig || !a_inf || !b_inf || !e_fermi ||
      !(spin_factor > 0.0)) {
    fprintf(stderr, "bop_fermi_level_noalloc: invalid argument (need M >= 1, 2 <= n_exp <= %d, pointers)\n",
            BOP_MAX_NEXP);
    return BOP_ERR_ARG;
  }
  // a count outside (0, s M) has no Fermi level inside the band: the search
  // would end at a bracket edge with a meaningless E_F
  if (!(n_electrons > 0.0 && n_electrons < spin_factor * (double)M)) {
    fprintf(stderr, "bop_fermi_level_noalloc: n_electrons = %g outside (0, %g) (spin_factor x M)\n", n_electrons,
            spin_factor * (double)M);
    return BOP_ERR_BRACKET;
  }
  const size_t need = OFF_D + (size_t)(n_exp + 3) * (size_t)M * sizeof(double);
  if (need > NOALLOC_BYTES) {
    fprintf(stderr,
            "bop_fermi_level_noalloc: %d orbitals x %d coefficients need %zu bytes of scratch, more than the "
            "%zu-byte static array (at most %zu orbitals at this n_exp)\n",
            M, n_exp + 3, need, NOALLOC_BYTES,
            (NOALLOC_BYTES - OFF_D) / ((size_t)(n_exp + 3) * sizeof(double)));
    return BOP_ERR_OVERFLOW;
  }
  unsigned char* base = nullptr;
  int r = scratch_address(&base);
  if (r != BOP_OK) return r;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FermiState* st = reinterpret_cast<FermiState*>(base + OFF_STATE);
  unsigned* counter = reinterpret_cast<unsigned*>(base + OFF_COUNTER);
  double* partials = reinterpret_cast<double*>(base + OFF_PARTIALS);
  double* D = reinterpret_cast<double*>(base + OFF_D);
  // the completion counter must start at zero; everything else is written before it is read
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), s) != cudaSuccess) return BOP_ERR_CUDA;
  long long tot = (long long)(n_exp + 3) * M;
  k_gsig_to_D<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, n_exp, gsig, D);
  if (launch_fermi(M, D, gsig, a_inf, b_inf, n_exp, spin_factor, n_electrons, st, partials, counter, 100, 1e-13,
                   s))
    return BOP_ERR_CUDA;
  k_copy_ef<<<1, 1, 0, s>>>(st, e_fermi);
  return cudaGetLastError() == cudaSuccess ? BOP_OK : BOP_ERR_CUDA;
}
