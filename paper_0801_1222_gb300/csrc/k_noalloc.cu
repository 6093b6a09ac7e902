// Green-function entry point that allocates no device memory.
//
// hfqmc_green_noalloc() computes, for one HS field s, the FP64 Green matrices
// of both spins, G^sigma = [1 + (1 - M)(e^{sigma lambda s} - 1)]^{-1} M, with
// M the antiperiodic bath matrix built from G0(tau_k) -- the same arithmetic
// that hfqmc_set_G0 runs for every chain of a context -- for callers that
// cannot allocate device memory (a host runtime that owns every device
// buffer through its own pool, a plugin that is not allowed to touch the
// CUDA allocator, code that runs where cudaMalloc is forbidden).  They pass
// their own device buffers for the inputs and outputs; the bath matrix and
// the Gauss-Jordan workspace live in the file-scope array below.
#include <cmath>

#include <cuda_runtime.h>

#include "../../include/hfqmc.h"
#include "hfq_device.cuh"
#include "hfq_gj.cuh"

namespace hfq {

// Scratch of the entry point: M (L x L) then [A | M] (L x 2L), FP64, for
// L <= HFQMC_NOALLOC_MAX_L; 1.5 MiB held by every GPU that loads the library
// until the process exits.  Followed by one status word.
constexpr int kNoAllocMaxL = HFQMC_NOALLOC_MAX_L;
constexpr size_t kNoAllocScratchDoubles = 3 * (size_t)kNoAllocMaxL * kNoAllocMaxL + 32;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kNoAllocNT = 256;

__global__ void __launch_bounds__(kNoAllocNT) k_green_noalloc(GridConst gc, const double* G0_tau,
                                                              const int8_t* s, double* Gup,
                                                              double* Gdn, double* scratch) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red[kNoAllocNT / 32];
  __shared__ int redi[kNoAllocNT / 32];
  __shared__ double s_inv;
  __shared__ int s_piv;
  const int L = gc.L;
  double* M = scratch;
  double* W = scratch + (size_t)L * L;
  int* status = reinterpret_cast<int*>(scratch + 3 * (size_t)kNoAllocMaxL * kNoAllocMaxL);
  double* colk = reinterpret_cast<double*>(dsm);
  if (threadIdx.x == 0) *status = 0;  // the array keeps the previous call's word
  for (int e = threadIdx.x; e < L * L; e += kNoAllocNT) {
    const int i = e / L, j = e - i * L;
    M[e] = (i >= j) ? -G0_tau[i - j] : G0_tau[i - j + L];
  }
  __syncthreads();
  gc.M = M;
  recompute_green<double, kNoAllocNT>(gc, s, Gup, Gdn, L, W, red, redi, &s_inv, &s_piv, colk,
                                      false, status);
}

}  // namespace hfq

extern "C" int hfqmc_green_noalloc(const double* G0_tau, const int8_t* s, int L, double dtau,
                                   double U, double* G_up, double* G_dn, void* cuda_stream,
                                   int* status_out) {
  using namespace hfq;
  if (L < 1 || L > kNoAllocMaxL) return HFQMC_EINVAL;
  if (!G0_tau || !s || !G_up || !G_dn) return HFQMC_EINVAL;
  if (!(dtau > 0.0) || !(U >= 0.0)) return HFQMC_EINVAL;
  // The host-side name of the array is not a device address: ask the runtime
  // for the array's address on the current device, on every call (a cached
  // address would outlive the context it belongs to after a device reset;
  // the lookup costs little next to the L^3 elimination).
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    (void)cudaGetLastError();
    return HFQMC_ECUDA;
  }
  double* scratch = static_cast<double*>(p);
  GridConst gc = {};
  gc.L = L;
  gc.lambda = std::acosh(std::exp(0.5 * dtau * U));
  gc.dV[0] = std::exp(gc.lambda) - 1.0;
  gc.dV[1] = std::exp(-gc.lambda) - 1.0;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  k_green_noalloc<<<1, kNoAllocNT, (size_t)L * sizeof(double), st>>>(gc, G0_tau, s, G_up, G_dn,
                                                                     scratch);
  if (cudaGetLastError() != cudaSuccess) return HFQMC_ECUDA;
  int word = 0;
  const double* status_addr = scratch + 3 * (size_t)kNoAllocMaxL * kNoAllocMaxL;
  if (cudaMemcpyAsync(&word, status_addr, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return HFQMC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HFQMC_ECUDA;
  if (status_out) *status_out = word;
  return (word & (kStatusSingular | kStatusNonFinite)) ? HFQMC_ENUMERIC : HFQMC_OK;
}
