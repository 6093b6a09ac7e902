// Test probe (not part of the library): Philox4x32-10 from cuRAND's
// header-only device function next to the generator the sweep kernels use
// (hfq::philox4x32_10 and the 53-bit uniform hfq::u53 of hfq_device.cuh), on
// the same counters and keys, so that a test can hold both -- and the CPU
// oracle's independent Philox -- to one implementation from outside this
// repository.
#include <cstdint>

#include <cuda_runtime.h>
#include <curand_kernel.h>

#include "hfq_device.cuh"

__global__ void k_philox_probe(const uint4* ctr, const unsigned long long* key, int n, uint4* out_lib,
                               uint4* out_hfq, double* u_hfq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = ctr[i];
  const unsigned long long k = key[i];
  out_lib[i] = curand_Philox4x32_10(c, make_uint2((unsigned)(k & 0xffffffffull), (unsigned)(k >> 32)));
  const uint4 h = hfq::philox4x32_10(c, k);
  out_hfq[i] = h;
  u_hfq[i] = hfq::u53(h.x, h.y);
}

// ctr: n x 4 words, key: n keys (word 0 = low 32 bits); out_lib, out_hfq:
// n x 4 words; u_hfq: n doubles.  Host arrays; returns a cudaError_t code.
extern "C" int philox_probe(const uint32_t* ctr, const uint64_t* key, int n, uint32_t* out_lib,
                            uint32_t* out_hfq, double* u_hfq) {
  if (n <= 0) return 0;
  uint4 *dc = nullptr, *dl = nullptr, *dh = nullptr;
  unsigned long long* dk = nullptr;
  double* du = nullptr;
  cudaError_t e = cudaMalloc(&dc, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dl, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dh, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(unsigned long long) * n);
  if (e == cudaSuccess) e = cudaMalloc(&du, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dk, key, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_philox_probe<<<(n + 255) / 256, 256>>>(dc, dk, n, dl, dh, du);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out_lib, dl, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(out_hfq, dh, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(u_hfq, du, sizeof(double) * n, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(dl);
  cudaFree(dh);
  cudaFree(dk);
  cudaFree(du);
  return (int)e;
}
