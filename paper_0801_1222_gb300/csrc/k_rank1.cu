// Rank-1 Hirsch-Fye sweep: one CTA per Markov chain, persistent over a
// longest-Lambda-first work queue.  T = double is the plain FP64 baseline
// (decision-for-decision identical to the FP64 oracle); T = float is the
// FP32 rank-1 path.
//
// Per sweep (introduction of the paper: single-slice flips of the binary HS
// field; Hirsch-Fye equations):
//   1. u_l = Philox(l, sweep, chain, grid) for all slices, in parallel.
//   2. Scan l = l0, l0+1, ... 32 at a time: R = R^up R^dn from the current
//      diagonals, accept iff u_l < R (or heat bath).  Rejections change
//      nothing, so a warp evaluates 32 consecutive proposals at once and a
//      ballot finds the first accepted one.
//   3. Accepted slice l: u^sigma = G^sigma_{:,l} - e_l, w^sigma = (Delta/R^sigma) G^sigma_{l,:}
//      are staged in shared memory and G^sigma += u w^T (both spins), s_l -> -s_l.
//      Every n_wrap accepted flips: FP64 recompute + drift.
//   4. Measured sweeps: g^sigma(tau_k) and D accumulated per chain in FP64.
// G is staged in shared memory for the whole chain when 2 L (L|1) sizeof(T)
// fits, else it stays in HBM/L2 and is updated there.
#include "hfq_device.cuh"
#include "hfq_gj.cuh"
#include "hfq_launch.h"

#include <type_traits>

namespace hfq {

template <typename T>
struct R1Traits;
template <>
struct R1Traits<double> {
  static constexpr int NT = 256;
};
template <>
struct R1Traits<float> {
  static constexpr int NT = 512;
};

__host__ __device__ inline int r1_ld_smem(int L) { return L | 1; }

__host__ __device__ inline size_t r1_align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Dynamic shared-memory layout:
//   head: colk[L] (double, recompute scratch), u[L] (double), perm[L] (int, pivot order of a
//   recompute), s[L] (int8)
//   body: [G^up G^dn (if resident)] diag[2L] col[2L] row[2L]
// During an FP64 recompute with gj_smem the body is overlaid by its workspace.
__host__ __device__ inline size_t r1_head_bytes(int L) {
  return r1_align16((size_t)L * sizeof(double)) * 2 + r1_align16((size_t)L * sizeof(int)) +
         r1_align16((size_t)L);
}
__host__ __device__ inline size_t r1_smem_bytes(int L, bool resident, size_t elem, bool gj_smem) {
  size_t b = 0;
  if (resident) b += r1_align16(2 * (size_t)L * r1_ld_smem(L) * elem);
  b += 3 * r1_align16(2 * (size_t)L * elem);
  if (gj_smem && gj_smem_bytes(L) > b) b = gj_smem_bytes(L);
  return r1_head_bytes(L) + b;
}

template <typename T>
__device__ __forceinline__ T tfma(T a, T b, T c);
template <>
__device__ __forceinline__ double tfma<double>(double a, double b, double c) {
  return __fma_rn(a, b, c);
}
template <>
__device__ __forceinline__ float tfma<float>(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}

// Flip ratio and decision.  FP64: evaluated exactly in the written order
// (no contraction), as in the oracle.  FP32: the ratio is FP32.
template <typename T>
__device__ __forceinline__ bool decide(const GridConst& gc, T gu, T gd, int sl, double u, int rule,
                                       bool* bad) {
  if constexpr (std::is_same<T, double>::value) {
    const double du = sl > 0 ? gc.delta[0] : gc.delta[1];
    const double dd = sl > 0 ? gc.delta[1] : gc.delta[0];
    const double Ru = __dadd_rn(1.0, __dmul_rn(__dsub_rn(1.0, gu), du));
    const double Rd = __dadd_rn(1.0, __dmul_rn(__dsub_rn(1.0, gd), dd));
    const double R = __dmul_rn(Ru, Rd);
    *bad = !(R > 0.0) || !isfinite(R);
    return rule == 0 ? (u < R) : (__dmul_rn(u, __dadd_rn(1.0, R)) < R);
  } else {
    const float du = (sl > 0 ? gc.deltaf[0] : gc.deltaf[1]);
    const float dd = (sl > 0 ? gc.deltaf[1] : gc.deltaf[0]);
    const float Ru = __fadd_rn(1.f, __fmul_rn(__fsub_rn(1.f, gu), du));
    const float Rd = __fadd_rn(1.f, __fmul_rn(__fsub_rn(1.f, gd), dd));
    const float R = __fmul_rn(Ru, Rd);
    *bad = !(R > 0.f) || !isfinite(R);
    const float uf = (float)u;
    return rule == 0 ? (u < (double)R) : (__fmul_rn(uf, __fadd_rn(1.f, R)) < R);
  }
}

template <typename T>
__device__ __forceinline__ void flip_factors(const GridConst& gc, T gu, T gd, int sl, T* fu,
                                             T* fd) {
  if constexpr (std::is_same<T, double>::value) {
    const double du = sl > 0 ? gc.delta[0] : gc.delta[1];
    const double dd = sl > 0 ? gc.delta[1] : gc.delta[0];
    const double Ru = __dadd_rn(1.0, __dmul_rn(__dsub_rn(1.0, gu), du));
    const double Rd = __dadd_rn(1.0, __dmul_rn(__dsub_rn(1.0, gd), dd));
    *fu = du / Ru;
    *fd = dd / Rd;
  } else {
    const float du = (sl > 0 ? gc.deltaf[0] : gc.deltaf[1]);
    const float dd = (sl > 0 ? gc.deltaf[1] : gc.deltaf[0]);
    const float Ru = __fadd_rn(1.f, __fmul_rn(__fsub_rn(1.f, gu), du));
    const float Rd = __fadd_rn(1.f, __fmul_rn(__fsub_rn(1.f, gd), dd));
    *fu = du / Ru;
    *fd = dd / Rd;
  }
}

// kTrace: kTraceRecord sets the bit of every accepted flip in the chain's
// decision trace; kTraceReplay takes the decisions from the trace instead of
// u < R (the flip ratios, flip factors and updates are computed as usual), so
// that an FP64 run follows the trajectory another run recorded.
template <typename T, int kTrace>
__global__ void __launch_bounds__(R1Traits<T>::NT, 1) k_sweep_rank1(SweepArgs a) {
  constexpr int NT = R1Traits<T>::NT;
  constexpr int NW = NT / 32;
  constexpr bool kF64 = std::is_same<T, double>::value;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[NW];
  __shared__ int redi[NW];
  __shared__ double s_inv;
  __shared__ int s_piv, s_item, s_first;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.queue_head, 1);
    __syncthreads();
    const int q = s_item;
    __syncthreads();
    if (q >= a.n_items) break;
    const ItemPtrs ip = a.items[a.order[q]];
    const GridConst gc = a.grids[ip.grid];
    const int L = gc.L;
    const bool resident = gc.resident != 0;

    // carve shared memory
    unsigned char* p = smem;
    double* colk = reinterpret_cast<double*>(p);
    p += r1_align16((size_t)L * sizeof(double));
    double* us = reinterpret_cast<double*>(p);
    p += r1_align16((size_t)L * sizeof(double));
    int* perm = reinterpret_cast<int*>(p);
    p += r1_align16((size_t)L * sizeof(int));
    int8_t* ss = reinterpret_cast<int8_t*>(p);
    p += r1_align16((size_t)L);
    unsigned char* body = p;
    T* Gu;
    T* Gd;
    int ld;
    T* Ggl = reinterpret_cast<T*>(ip.G);
    if (resident) {
      ld = r1_ld_smem(L);
      Gu = reinterpret_cast<T*>(p);
      Gd = Gu + (size_t)L * ld;
      p += r1_align16(2 * (size_t)L * ld * sizeof(T));
    } else {
      ld = L;
      Gu = Ggl;
      Gd = Ggl + (size_t)L * L;
    }
    T* diag = reinterpret_cast<T*>(p);  // [0,L) up, [L,2L) dn
    p += r1_align16(2 * (size_t)L * sizeof(T));
    T* col = reinterpret_cast<T*>(p);
    p += r1_align16(2 * (size_t)L * sizeof(T));
    T* row = reinterpret_cast<T*>(p);

    if (resident) {
      for (int i = warp; i < 2 * L; i += NW)
        for (int j = lane; j < L; j += 32) Gu[(size_t)i * ld + j] = Ggl[(size_t)i * L + j];
    }
    for (int l = tid; l < L; l += NT) ss[l] = ip.s[l];
    __syncthreads();
    for (int i = tid; i < L; i += NT) {
      diag[i] = Gu[(size_t)i * ld + i];
      diag[L + i] = Gd[(size_t)i * ld + i];
    }
    const ChainCounters c0 = *ip.cnt;
    long long n_acc = c0.accepted;
    // accepted flips until the next recompute (the cumulative count reaches a
    // multiple of n_wrap); counted down so the hot loop needs no 64-bit modulo
    int until_rec = gc.n_wrap > 0 ? (int)(gc.n_wrap - n_acc % gc.n_wrap) : 0;
    long long n_rec = 0, n_bad = 0;
    unsigned long long hash = c0.hash;
    double drift = c0.drift;
    const long long n_sweeps = a.n_warm + a.n_meas;
    __syncthreads();

    for (long long sw = 0; sw < n_sweeps; ++sw) {
      const long long t = c0.t + sw;
      for (int l = tid; l < L; l += NT) us[l] = proposal_uniform(l, t, ip.chain, ip.grid, a.seed);
      __syncthreads();
      int l0 = 0;
      while (l0 < L) {
        int first = L;
        if (!kF64 || warp == 0) {
          for (int w = l0; w < L; w += 32) {
            const int l = w + lane;
            bool acc = false, bad = false;
            if (l < L) acc = decide<T>(gc, diag[l], diag[L + l], ss[l], us[l], a.accept_rule, &bad);
            if constexpr (kTrace == kTraceReplay)
              acc = l < L && ((ip.trace[(size_t)sw * trace_words(L) + (l >> 5)] >> (l & 31)) & 1u);
            const unsigned b = __ballot_sync(0xffffffffu, acc);
            const unsigned bb = __ballot_sync(0xffffffffu, bad);
            if (b) {
              first = w + __ffs(b) - 1;
              const int upto = first - w;  // lanes 0..upto evaluated
              const unsigned valid = upto >= 31 ? 0xffffffffu : ((2u << upto) - 1u);
              n_bad += __popc(bb & valid);
              break;
            }
            n_bad += __popc(bb);
          }
        }
        if constexpr (kF64) {
          if (tid == 0) s_first = first;
          __syncthreads();
          first = s_first;
        }
        if (first >= L) break;
        const int sl = ss[first];
        T fu, fd;
        flip_factors<T>(gc, diag[first], diag[L + first], sl, &fu, &fd);
        for (int i = tid; i < L; i += NT) {
          const T e = (i == first) ? T(1) : T(0);
          col[i] = Gu[(size_t)i * ld + first] - e;
          col[L + i] = Gd[(size_t)i * ld + first] - e;
          row[i] = Gu[(size_t)first * ld + i] * fu;
          row[L + i] = Gd[(size_t)first * ld + i] * fd;
        }
        __syncthreads();
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) {
          T* G = sp ? Gd : Gu;
          const T* cs = col + sp * L;
          const T* rs = row + sp * L;
          for (int i = warp; i < L; i += NW) {
            const T ci = cs[i];
            T* gi = G + (size_t)i * ld;
            for (int j = lane; j < L; j += 32) gi[j] = tfma<T>(ci, rs[j], gi[j]);
          }
        }
        for (int i = tid; i < L; i += NT) {
          diag[i] = tfma<T>(col[i], row[i], diag[i]);
          diag[L + i] = tfma<T>(col[L + i], row[L + i], diag[L + i]);
        }
        if (tid == 0) ss[first] = (int8_t)(-sl);
        hash = (hash ^ (unsigned long long)(t * (long long)L + first)) * kFnvPrime;
        if constexpr (kTrace == kTraceRecord) {
          if (tid == 0) ip.trace[(size_t)sw * trace_words(L) + (first >> 5)] |= 1u << (first & 31);
        }
        ++n_acc;
        __syncthreads();
        if (gc.n_wrap > 0 && --until_rec == 0) {
          until_rec = gc.n_wrap;
          double d;
          if (gc.gj_smem) {
            // the FP64 workspace overlays the body of shared memory: G goes home to HBM first
            if (resident) {
              for (int i = warp; i < 2 * L; i += NW)
                for (int j = lane; j < L; j += 32) Ggl[(size_t)i * L + j] = Gu[(size_t)i * ld + j];
              __syncthreads();
            }
            d = recompute_green_inv<T, NT>(gc, ss, Ggl, Ggl + (size_t)L * L, L,
                                           reinterpret_cast<double*>(body), red, redi, &s_inv, &s_piv,
                                           colk, perm, true, a.status);
            if (resident) {
              for (int i = warp; i < 2 * L; i += NW)
                for (int j = lane; j < L; j += 32) Gu[(size_t)i * ld + j] = Ggl[(size_t)i * L + j];
              __syncthreads();
            }
          } else {
            d = recompute_green_inv<T, NT>(gc, ss, Gu, Gd, ld, ip.ws, red, redi, &s_inv, &s_piv, colk,
                                           perm, true, a.status);
          }
          drift = fmax(drift, d);
          ++n_rec;
          for (int i = tid; i < L; i += NT) {
            diag[i] = Gu[(size_t)i * ld + i];
            diag[L + i] = Gd[(size_t)i * ld + i];
          }
          __syncthreads();
        }
        l0 = first + 1;
      }
      if (sw >= a.n_warm) {
        const long long m = sw - a.n_warm;
        const int b = (int)((kBins * m) / a.n_meas);
        const double invL = 1.0 / (double)L;
        for (int k = tid; k < L; k += NT) {
          double su = 0.0, sd = 0.0;
          for (int l = 0; l < L; ++l) {
            const int r = l + k;
            if (r >= L) {
              su -= (double)Gu[(size_t)(r - L) * ld + l];
              sd -= (double)Gd[(size_t)(r - L) * ld + l];
            } else {
              su += (double)Gu[(size_t)r * ld + l];
              sd += (double)Gd[(size_t)r * ld + l];
            }
          }
          const double gu = su / (double)L, gd = sd / (double)L;
          ip.acc[k] += gu;
          ip.acc[L + k] += gd;
          ip.bins[(size_t)b * L + k] += 0.5 * (gu + gd);
        }
        double v = 0.0;
        for (int l = tid; l < L; l += NT) v += (1.0 - (double)diag[l]) * (1.0 - (double)diag[L + l]);
        v = block_sum<NT>(v, red);
        if (tid == 0) {
          ip.accD[0] += v * invL;
          ip.accD[1 + b] += v * invL;
        }
      }
      __syncthreads();
    }

    // write back the chain state
    if (resident) {
      for (int i = warp; i < 2 * L; i += NW)
        for (int j = lane; j < L; j += 32) Ggl[(size_t)i * L + j] = Gu[(size_t)i * ld + j];
    }
    for (int l = tid; l < L; l += NT) ip.s[l] = ss[l];
    // n_bad is warp-uniform; thread 0 holds warp 0's count, which covers every proposal once
    if (tid == 0) {
      ChainCounters c = c0;
      c.t = c0.t + n_sweeps;
      c.proposals = c0.proposals + n_sweeps * (long long)L;
      c.accepted = n_acc;
      c.recomputes = c0.recomputes + n_rec;
      c.hash = hash;
      c.bad = c0.bad + n_bad;
      c.drift = drift;
      *ip.cnt = c;
    }
    __syncthreads();
  }
}

template <typename T>
static void launch_rank1_t(const SweepArgs& a, int ctas, size_t smem, cudaStream_t st) {
  constexpr int NT = R1Traits<T>::NT;
  if (a.trace_mode == kTraceRecord)
    k_sweep_rank1<T, kTraceRecord><<<ctas, NT, smem, st>>>(a);
  else if (a.trace_mode == kTraceReplay)
    k_sweep_rank1<T, kTraceReplay><<<ctas, NT, smem, st>>>(a);
  else
    k_sweep_rank1<T, kTraceOff><<<ctas, NT, smem, st>>>(a);
}

int launch_sweep_rank1(bool f64, const SweepArgs& a, int ctas, size_t smem, cudaStream_t st) {
  if (f64)
    launch_rank1_t<double>(a, ctas, smem, st);
  else
    launch_rank1_t<float>(a, ctas, smem, st);
  return (int)cudaGetLastError();
}

template <typename T>
static cudaError_t config_rank1_t(size_t smem, int* occ) {
  cudaError_t e = raise_smem_limit(k_sweep_rank1<T, kTraceOff>, smem);
  if (e == cudaSuccess) e = raise_smem_limit(k_sweep_rank1<T, kTraceRecord>, smem);
  if (e == cudaSuccess) e = raise_smem_limit(k_sweep_rank1<T, kTraceReplay>, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_sweep_rank1<T, kTraceOff>, R1Traits<T>::NT,
                                                      smem);
  return e;
}

int rank1_config(bool f64, size_t smem, int* threads, int* ctas_per_sm) {
  int occ = 0;
  const cudaError_t e = f64 ? config_rank1_t<double>(smem, &occ) : config_rank1_t<float>(smem, &occ);
  *threads = f64 ? R1Traits<double>::NT : R1Traits<float>::NT;
  *ctas_per_sm = occ;
  return (int)e;
}

size_t rank1_smem(int L, bool resident, bool f64, bool gj_smem) {
  return r1_smem_bytes(L, resident, f64 ? sizeof(double) : sizeof(float), gj_smem);
}

}  // namespace hfq
