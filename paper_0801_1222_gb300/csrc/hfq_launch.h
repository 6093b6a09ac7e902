// Host-side launchers of the sweep library's kernels (C++ linkage, internal).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "hfq_device.cuh"

namespace hfq {

// Raises a kernel's dynamic shared-memory limit on the current device to at
// least smem bytes and never lowers it: the limit belongs to the function,
// while every context of the process launches the same sweep kernels with its
// own size, set once and launched later (a lower size set by one context
// would make another's launches fail).
template <typename F>
inline cudaError_t raise_smem_limit(F* f, size_t smem) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, f);
  if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < smem)
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}

// bath matrix M of one grid from G0(tau_k), and its FP64 inverse
int launch_bath_matrix(int L, const double* G0_tau, double* M, cudaStream_t st);
int launch_bath_inverse(int L, const double* M, double* Minv, int* status, cudaStream_t st);
// slices of A = M^{-1} - diag(...) for the Newton refinement of G (FP32 delayed path)
int launch_refine_prep(int L, const double* Minv, double lambda, RefineConst* rc, uint16_t* aslc,
                       cudaStream_t st);
// initial (or refreshed) field and Green matrices of the chains of one grid
int launch_init_chains(const SweepArgs& a, const GridConst* d_grid_ptr, int item0, int n_chains,
                       int L, bool f64, bool first_time, bool gj_smem, cudaStream_t st);
// measured-sweep bookkeeping of every grid for one hfqmc_sweep call
int launch_account(GridAccount* acc, int n_grids, long long n_meas, cudaStream_t st);
// per-grid mean over chains and error bars
int launch_reduce(const GridConst* grids, const ItemPtrs* items, const GridAccount* acc,
                  GridOut* gout, double* outG, double* outErr, const long long* out_off,
                  int n_grids, cudaStream_t st);

// rank-1 sweep (FP64 baseline / FP32)
size_t rank1_smem(int L, bool resident, bool f64, bool gj_smem);
int rank1_config(bool f64, size_t smem, int* threads, int* ctas_per_sm);
int launch_sweep_rank1(bool f64, const SweepArgs& a, int ctas, size_t smem, cudaStream_t st);

// delayed rank-k sweep (FP32); kDelayedTile: edge of the flush's output tiles
// (the TMA reduce moves half a tile, kDelayedTile x kDelayedTile/2, at a time)
constexpr int kDelayedTile = 128;
// ns: spins the sweep keeps (1 for the G_up-only sweep of a particle-hole
// symmetric bath)
size_t delayed_smem(int L, int k, bool resident, bool gj_smem, bool gtile = false, int ub = 2,
                    bool refine = false, int ns = 2);
int delayed_config(size_t smem, int* threads, int* ctas_per_sm);
int launch_sweep_delayed(const SweepArgs& a, int ctas, size_t smem, cudaStream_t st);

}  // namespace hfq
