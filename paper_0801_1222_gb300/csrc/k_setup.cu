// Set-up and reduction kernels of the sweep library:
//  * bath matrix M of a grid from its G0(tau_k) samples (antiperiodic Toeplitz);
//  * per-chain initial field (Philox) and FP64 Gauss-Jordan Green matrices;
//  * per-call measured-sweep bookkeeping;
//  * per-grid mean over chains and error bars (the paper averages each grid's
//    Green function over 10 to 20 impurity solutions, "Multigrid HF-QMC method").
#include <cuda_fp16.h>

#include "hfq_device.cuh"
#include "hfq_gj.cuh"
#include "hfq_launch.h"

namespace hfq {

__global__ void k_bath_matrix(int L, const double* __restrict__ G0, double* __restrict__ M) {
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < L; j += blockDim.x)
    M[(size_t)i * L + j] = (i >= j) ? -G0[i - j] : G0[i - j + L];
}

int launch_bath_matrix(int L, const double* G0_tau, double* M, cudaStream_t st) {
  k_bath_matrix<<<L, 128, 0, st>>>(L, G0_tau, M);
  return (int)cudaGetLastError();
}

// colk (L doubles), perm (L ints) and the field (L int8), 16-byte aligned,
// before the workspace
__host__ __device__ inline size_t init_head_bytes(int L) {
  return ((size_t)L * sizeof(double) + (size_t)L * sizeof(int) + (size_t)L + 15) / 16 * 16;
}
// with the workspace in HBM: whether the blocked inversion's panel scratch
// fits after the head
__host__ __device__ inline bool init_blocked(int L) {
  return init_head_bytes(L) + gj_blocked_bytes(L) <= kSmemCap;
}

// M^{-1} of one grid's bath matrix.  M is skew-circulant: M_{ll'} = c(l - l')
// with c(d) = -G0(tau_d) and c(d - L) = -c(d) (the antiperiodic wrap).  The
// plane waves e^{i theta_n l}, theta_n = (2n+1) pi / L (the fermionic
// Matsubara phases of the grid), diagonalise it with eigenvalues
//   mu_n = sum_{d<L} c(d) e^{-i theta_n d},
// so M^{-1} is skew-circulant too, with
//   c'(d) = (1/L) sum_{n<L} Re[e^{i theta_n d} / mu_n]     (real: mu_{L-1-n} = conj mu_n).
// One CTA, O(L^2) FP64 work with a table of e^{i pi m / L}, m < 2L.
__global__ void __launch_bounds__(256) k_bath_inverse(int L, const double* __restrict__ M,
                                                      double* __restrict__ Minv, int* status) {
  extern __shared__ __align__(16) unsigned char dsm[];
  double* twc = reinterpret_cast<double*>(dsm);  // cos(pi m / L), m < 2L
  double* tws = twc + 2 * L;                     // sin(pi m / L)
  double* cc = tws + 2 * L;                      // c(d), d < L
  double* ir = cc + L;                           // Re 1/mu_n
  double* ii = ir + L;                           // Im 1/mu_n
  double* cp = ii + L;                           // c'(d), d < L
  __shared__ int s_bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_bad = 0;
  for (int m = tid; m < 2 * L; m += nt) sincospi((double)m / (double)L, &tws[m], &twc[m]);
  for (int d = tid; d < L; d += nt) cc[d] = M[(size_t)d * L];  // first column
  __syncthreads();
  for (int n = tid; n < L; n += nt) {
    const int step = 2 * n + 1;  // phase index (2n+1) d mod 2L, advanced per d
    double re = 0.0, im = 0.0;
    int ph = 0;
    for (int d = 0; d < L; ++d) {
      re = fma(cc[d], twc[ph], re);
      im = fma(-cc[d], tws[ph], im);
      ph += step;
      if (ph >= 2 * L) ph -= 2 * L;
    }
    const double den = re * re + im * im;
    if (!(den > 0.0) || !isfinite(den)) atomicOr(&s_bad, 1);
    ir[n] = re / den;
    ii[n] = -im / den;
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) atomicOr(status, kStatusSingular);
    return;
  }
  for (int d = tid; d < L; d += nt) {
    const int step = (2 * d) % (2 * L);  // phase index (2n+1) d mod 2L, advanced per n
    double acc = 0.0;
    int ph = d;
    for (int n = 0; n < L; ++n) {
      acc = fma(ir[n], twc[ph], acc);
      acc = fma(-ii[n], tws[ph], acc);
      ph += step;
      if (ph >= 2 * L) ph -= 2 * L;
    }
    cp[d] = acc / (double)L;
  }
  __syncthreads();
  for (int e = tid; e < L * L; e += nt) {
    const int i = e / L, j = e - i * L;
    Minv[e] = i >= j ? cp[i - j] : -cp[i - j + L];
  }
}

int launch_bath_inverse(int L, const double* M, double* Minv, int* status, cudaStream_t st) {
  const size_t smem = 8 * (size_t)L * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024)
    e = cudaFuncSetAttribute(k_bath_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  k_bath_inverse<<<1, 256, smem, st>>>(L, M, Minv, status);
  return (int)cudaGetLastError();
}

// Slices of A = M^{-1} - diag(1 - e^{-sigma lambda s_j}) for the Newton
// refinement (hfq_refine.cuh): every entry x of M^{-1} (padded with zeros to
// whole 128-row blocks and 64-column chunks) is written as
//   x = 2^ea sum_{p<6} s_p 2^{-7(p+1)} + (remainder below 2^{ea-43}),
// s_p = rint of the running remainder times 2^7 (|s_0| <= 128, |s_p| <= 64),
// each an integer held exactly in FP16, stored in the K-major core-matrix
// layout the tensor-core operand wants (rows of A = M dimension, columns =
// K).  A_jj depends on the chain's field: its two values are sliced into
// rc->dslc and patched in per chain; ea covers both.  One block per (row
// block, K chunk); every block finds the same ea.
__device__ __forceinline__ uint32_t rf_core_offset(int r, int m) {
  return (uint32_t)((r >> 3) * (kRfKC / 8) * 128 + (m >> 3) * 128 + (r & 7) * 16 + (m & 7) * 2);
}

__device__ __forceinline__ void rf_slice6(double x, int ea, float* q) {
  double y = ldexp(x, kRfBits - ea);
#pragma unroll
  for (int p = 0; p < kRfSlicesA; ++p) {
    const double r = rint(y);
    q[p] = (float)r;
    y = (y - r) * (double)(1 << kRfBits);
  }
}

__global__ void __launch_bounds__(256) k_refine_prep(int L, const double* __restrict__ Minv, double lambda,
                                                     RefineConst* rc, uint16_t* __restrict__ aslc, int nkc) {
  __shared__ double red[8];
  const int tid = threadIdx.x;
  const double a0 = Minv[0] - (1.0 - exp(-lambda)), a1 = Minv[0] - (1.0 - exp(lambda));
  double m = fmax(fabs(a0), fabs(a1));
  for (int d = tid; d < L; d += 256) m = fmax(m, fabs(Minv[(size_t)d * L]));  // c'(d), all d
  m = block_max<256>(m, red);
  int ea = 0;
  if (m > 0.0) (void)frexp(m, &ea);  // m < 2^ea
  if (blockIdx.x == 0 && tid == 0) {
    rc->ea = ea;
    float q[kRfSlicesA];
    rf_slice6(a0, ea, q);
    for (int p = 0; p < kRfSlicesA; ++p) rc->dslc[0][p] = __half_as_ushort(__float2half_rn(q[p]));
    rf_slice6(a1, ea, q);
    for (int p = 0; p < kRfSlicesA; ++p) rc->dslc[1][p] = __half_as_ushort(__float2half_rn(q[p]));
  }
  const int rb = blockIdx.x / nkc, kc = blockIdx.x - rb * nkc;
  uint16_t* tile = aslc + (size_t)blockIdx.x * kRfSlicesA * (kRfTileA / 2);
  for (int c = tid; c < 128 * (kRfKC / 8); c += 256) {
    const int r = c / (kRfKC / 8), m0 = (c - r * (kRfKC / 8)) * 8;
    const int i = rb * 128 + r;
    uint32_t w[kRfSlicesA][4];
#pragma unroll
    for (int t = 0; t < 8; t += 2) {
      const int j = kc * kRfKC + m0 + t;
      float q0[kRfSlicesA], q1[kRfSlicesA];
      rf_slice6(i < L && j < L ? Minv[(size_t)i * L + j] : 0.0, ea, q0);
      rf_slice6(i < L && j + 1 < L ? Minv[(size_t)i * L + j + 1] : 0.0, ea, q1);
#pragma unroll
      for (int p = 0; p < kRfSlicesA; ++p)
        w[p][t / 2] = (uint32_t)__half_as_ushort(__float2half_rn(q0[p])) |
                      ((uint32_t)__half_as_ushort(__float2half_rn(q1[p])) << 16);
    }
    const uint32_t off = rf_core_offset(r, m0) / 2;
#pragma unroll
    for (int p = 0; p < kRfSlicesA; ++p)
      *reinterpret_cast<uint4*>(tile + (size_t)p * (kRfTileA / 2) + off) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
  }
}

int launch_refine_prep(int L, const double* Minv, double lambda, RefineConst* rc, uint16_t* aslc,
                       cudaStream_t st) {
  const int nrb = rf_pad(L, 128) / 128, nkc = rf_pad(L, kRfKC) / kRfKC;
  k_refine_prep<<<nrb * nkc, 256, 0, st>>>(L, Minv, lambda, rc, aslc, nkc);
  return (int)cudaGetLastError();
}

// Initial (or, after a new bath, rebuilt) Green matrices of every chain of a
// grid: block (chain, spin), so the two spins of a chain are inverted by two
// CTAs at once.  The spin-up block also resets the chain's accumulators.
template <typename T>
__global__ void __launch_bounds__(256) k_init_chains(SweepArgs a, const GridConst* gptr, int item0,
                                                     int first_time) {
  constexpr int NT = 256;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red[NT / 32];
  __shared__ int redi[NT / 32];
  __shared__ double s_inv;
  __shared__ int s_piv;
  const int tid = threadIdx.x, sp = blockIdx.y;
  const ItemPtrs ip = a.items[item0 + blockIdx.x];
  const GridConst gc = *gptr;
  const int L = gc.L;
  double* colk = reinterpret_cast<double*>(dsm);
  int* perm = reinterpret_cast<int*>(colk + L);
  int8_t* sf = reinterpret_cast<int8_t*>(perm + L);
  double* W = gc.gj_smem ? reinterpret_cast<double*>(dsm + init_head_bytes(L)) : ip.ws + (size_t)sp * L * L;
  // workspace in HBM: inverted by panels when their scratch fits after the head
  double* pan = !gc.gj_smem && init_blocked(L) ? reinterpret_cast<double*>(dsm + init_head_bytes(L)) : nullptr;
  // the field: drawn afresh (both blocks draw the same values; the spin-up
  // block stores it) or the chain's current one
  for (int l = tid; l < L; l += NT) {
    const int8_t v = first_time ? initial_spin(l, ip.chain, ip.grid, a.seed) : ip.s[l];
    sf[l] = v;
    if (first_time && sp == 0) ip.s[l] = v;
  }
  __syncthreads();
  T* G = reinterpret_cast<T*>(ip.G);
  if (pan)
    recompute_green_inv<T, NT, true>(gc, sf, G, G + (size_t)L * L, L, W, red, redi, &s_inv, &s_piv, colk,
                                     perm, false, a.status, sp, sp + 1, pan);
  else
    recompute_green_inv<T, NT>(gc, sf, G, G + (size_t)L * L, L, W, red, redi, &s_inv, &s_piv, colk, perm,
                               false, a.status, sp, sp + 1);
  if (sp != 0) return;
  for (int k = tid; k < 2 * L; k += NT) ip.acc[k] = 0.0;
  for (int k = tid; k < kBins * L; k += NT) ip.bins[k] = 0.0;
  for (int k = tid; k < 1 + kBins; k += NT) ip.accD[k] = 0.0;
  if (tid == 0) {
    ChainCounters c;
    if (first_time) {
      c.t = 0;
      c.proposals = 0;
      c.accepted = 0;
      c.recomputes = 0;
      c.hash = kFnvOffset;
      c.bad = 0;
      c.status = 0;
      c.fallbacks = 0;
    } else {
      c = *ip.cnt;
    }
    c.drift = 0.0;
    *ip.cnt = c;
  }
}

size_t init_smem(int L, bool gj_smem) {
  return init_head_bytes(L) + (gj_smem ? gj_smem_bytes(L) : (init_blocked(L) ? gj_blocked_bytes(L) : 0));
}

int launch_init_chains(const SweepArgs& a, const GridConst* d_grid_ptr, int item0, int n_chains,
                       int L, bool f64, bool first_time, bool gj_smem, cudaStream_t st) {
  const size_t sm = init_smem(L, gj_smem);
  cudaError_t e;
  if (f64) {
    e = cudaFuncSetAttribute(k_init_chains<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    k_init_chains<double><<<dim3(n_chains, 2), 256, sm, st>>>(a, d_grid_ptr, item0, first_time ? 1 : 0);
  } else {
    e = cudaFuncSetAttribute(k_init_chains<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    k_init_chains<float><<<dim3(n_chains, 2), 256, sm, st>>>(a, d_grid_ptr, item0, first_time ? 1 : 0);
  }
  return (int)cudaGetLastError();
}

// Measured sweep m (0-based within one call of n_meas) goes to bin floor(32 m / n_meas);
// bin b therefore receives ceil((b+1) n / 32) - ceil(b n / 32) sweeps.
__global__ void k_account(GridAccount* acc, int n_grids, long long n_meas) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_grids || n_meas <= 0) return;
  acc[g].n_meas += n_meas;
  for (int b = 0; b < kBins; ++b) {
    const long long lo = ((long long)b * n_meas + kBins - 1) / kBins;
    const long long hi = ((long long)(b + 1) * n_meas + kBins - 1) / kBins;
    acc[g].bin_count[b] += hi - lo;
  }
}

int launch_account(GridAccount* acc, int n_grids, long long n_meas, cudaStream_t st) {
  k_account<<<(n_grids + 127) / 128, 128, 0, st>>>(acc, n_grids, n_meas);
  return (int)cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_reduce(const GridConst* grids, const ItemPtrs* items,
                                                const GridAccount* acc, GridOut* gout,
                                                double* outG, double* outErr,
                                                const long long* out_off) {
  const int g = blockIdx.x, tid = threadIdx.x;
  const GridConst gc = grids[g];
  const int L = gc.L, nc = gc.chains, i0 = gc.item0;
  const GridAccount& A = acc[g];
  const double N = (double)A.n_meas;
  double* oG = outG + out_off[g];
  double* oE = outErr + out_off[g];
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  for (int k = tid; k < L; k += blockDim.x) {
    double mean = nan, err = nan;
    if (A.n_meas > 0) {
      if (nc >= 2) {
        double s = 0.0;
        for (int c = 0; c < nc; ++c) {
          const double* ac = items[i0 + c].acc;
          s += -(ac[k] + ac[L + k]) / (2.0 * N);
        }
        mean = s / nc;
        double v = 0.0;
        for (int c = 0; c < nc; ++c) {
          const double* ac = items[i0 + c].acc;
          const double d = -(ac[k] + ac[L + k]) / (2.0 * N) - mean;
          v += d * d;
        }
        err = sqrt(v / (nc - 1) / nc);
      } else {
        const ItemPtrs ip = items[i0];
        mean = -(ip.acc[k] + ip.acc[L + k]) / (2.0 * N);
        int nb = 0;
        double s = 0.0;
        for (int b = 0; b < kBins; ++b)
          if (A.bin_count[b] > 0) {
            s += -ip.bins[(size_t)b * L + k] / (double)A.bin_count[b];
            ++nb;
          }
        if (nb >= 2) {
          const double bm = s / nb;
          double v = 0.0;
          for (int b = 0; b < kBins; ++b)
            if (A.bin_count[b] > 0) {
              const double d = -ip.bins[(size_t)b * L + k] / (double)A.bin_count[b] - bm;
              v += d * d;
            }
          err = sqrt(v / (nb - 1) / nb);
        }
      }
    }
    oG[k] = mean;
    oE[k] = err;
  }
  __syncthreads();
  if (tid == 0) {
    oG[L] = -1.0 - oG[0];
    oE[L] = oE[0];
    GridOut o;
    o.proposals = o.accepted = o.recomputes = o.bad = o.fallbacks = 0;
    o.drift = 0.0;
    for (int c = 0; c < nc; ++c) {
      const ChainCounters cc = *items[i0 + c].cnt;
      o.proposals += cc.proposals;
      o.accepted += cc.accepted;
      o.recomputes += cc.recomputes;
      o.bad += cc.bad;
      o.fallbacks += cc.fallbacks;
      o.drift = fmax(o.drift, cc.drift);
    }
    o.D = nan;
    o.D_err = nan;
    if (A.n_meas > 0) {
      if (nc >= 2) {
        double s = 0.0, v = 0.0;
        for (int c = 0; c < nc; ++c) s += items[i0 + c].accD[0] / N;
        const double m = s / nc;
        for (int c = 0; c < nc; ++c) {
          const double d = items[i0 + c].accD[0] / N - m;
          v += d * d;
        }
        o.D = m;
        o.D_err = sqrt(v / (nc - 1) / nc);
      } else {
        o.D = items[i0].accD[0] / N;
        int nb = 0;
        double s = 0.0, v = 0.0;
        for (int b = 0; b < kBins; ++b)
          if (A.bin_count[b] > 0) {
            s += items[i0].accD[1 + b] / (double)A.bin_count[b];
            ++nb;
          }
        if (nb >= 2) {
          const double m = s / nb;
          for (int b = 0; b < kBins; ++b)
            if (A.bin_count[b] > 0) {
              const double d = items[i0].accD[1 + b] / (double)A.bin_count[b] - m;
              v += d * d;
            }
          o.D_err = sqrt(v / (nb - 1) / nb);
        }
      }
    }
    gout[g] = o;
  }
}

int launch_reduce(const GridConst* grids, const ItemPtrs* items, const GridAccount* acc,
                  GridOut* gout, double* outG, double* outErr, const long long* out_off,
                  int n_grids, cudaStream_t st) {
  k_reduce<<<n_grids, 256, 0, st>>>(grids, items, acc, gout, outG, outErr, out_off);
  return (int)cudaGetLastError();
}

}  // namespace hfq
