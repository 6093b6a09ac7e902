// FP64 recomputation of the Green matrices from the field:
//   G^sigma = A^{-1} M,  A^sigma = 1 + (1 - M) diag(e^{sigma lambda s} - 1),
// the Dyson equation that links the interacting G to the bath G0 (= M) in
// Hirsch-Fye QMC.  It is the only FP64 step of the FP32 sweep paths and is
// followed by the drift check max |G_fast - G_fresh|.
//
// Two algorithms, both Gauss-Jordan elimination with partial pivoting by one
// CTA, with per pivot column three barriers (pivot search, row swap + scale,
// elimination), bound by the FP64 pipe (about 2 DFMA/clk/SM on GB300):
//  * recompute_green: on the augmented L x 2L matrix [A | M], 1.5 L^3 DFMA
//    per spin.  Used by the entry point that allocates nothing.
//  * recompute_green_inv: G = B^{-1} with B = M^{-1}(1 + D) - D inverted in
//    place, L^3 DFMA per spin on an L x L workspace -- shared memory when it
//    fits (Lambda <= 168), the chain's HBM workspace otherwise (L2-resident
//    for the sizes used).  Used by every sweep kernel and the initialisation.
#pragma once
#include "hfq_device.cuh"

namespace hfq {

// In-place Gauss-Jordan on W = [A | B] (L rows, 2L columns, row-major), in
// shared or global memory.  colk: L doubles of shared scratch (the pivot
// column of the current step, so the elimination reads it once per row).
// The elimination keeps the pivot row in registers and updates two rows per
// warp iteration, loading 2 x kGjChunk values before any store, so each warp
// has that many independent loads and DFMAs in flight (the FP64 pipe's
// latency is long on this part) whether W lives in shared memory or in L2.
// On return the right half holds A^{-1} B.  Returns -1 on a zero pivot
// (uniformly in all threads), 0 otherwise.
// columns per lane and chunk: 8 with 8 warps; 4 with 16 warps, whose register
// budget is half as large (and twice the warps keep as many loads in flight)
template <int NT>
__host__ __device__ constexpr int gj_chunk() { return NT >= 512 ? 4 : 8; }

template <int NT>
__device__ int gj_eliminate(double* W, int L, double* red, int* redi, double* s_inv, int* s_piv,
                            double* colk) {
  constexpr int kGjChunk = gj_chunk<NT>();
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ld = 2 * L;
  for (int k = 0; k < L; ++k) {
    double best = -1.0;
    int bi = L;
    for (int i = k + tid; i < L; i += NT) {
      const double v = fabs(W[(size_t)i * ld + k]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      red[warp] = best;
      redi[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double b = red[0];
      int p = redi[0];
      for (int w = 1; w < NW; ++w)
        if (red[w] > b || (red[w] == b && redi[w] < p)) {
          b = red[w];
          p = redi[w];
        }
      if (!(b > 0.0) || p >= L) {
        *s_piv = -1;
      } else {
        *s_piv = p;
        *s_inv = 1.0 / W[(size_t)p * ld + k];
      }
    }
    __syncthreads();
    const int p = *s_piv;
    if (p < 0) return -1;
    const double inv = *s_inv;
    // swap rows k and p (columns >= k), scale the new row k; record column k
    for (int j = k + tid; j < ld; j += NT) {
      const double a = W[(size_t)k * ld + j];
      const double b = W[(size_t)p * ld + j];
      W[(size_t)p * ld + j] = a;
      W[(size_t)k * ld + j] = b * inv;
      if (j == k) colk[p] = a;
    }
    for (int i = tid; i < L; i += NT)
      if (i != k && i != p) colk[i] = W[(size_t)i * ld + k];
    __syncthreads();
    // eliminate column k from every other row
    const int j0 = k + 1;
    const double* wk = W + (size_t)k * ld;
    for (int c0 = j0; c0 < ld; c0 += 32 * kGjChunk) {
      double rk[kGjChunk];
#pragma unroll
      for (int c = 0; c < kGjChunk; ++c) {
        const int j = c0 + lane + 32 * c;
        rk[c] = j < ld ? wk[j] : 0.0;
      }
      // two rows per warp iteration: 2 x kGjChunk independent DFMAs between
      // the loads and the stores, enough to cover the FP64 pipe's latency
      for (int i = warp; i < L; i += 2 * NW) {
        const int i2 = i + NW;
        const bool has2 = i2 < L;
        double v1[kGjChunk], v2[kGjChunk];
#pragma unroll
        for (int c = 0; c < kGjChunk; ++c) {
          const int j = c0 + lane + 32 * c;
          v1[c] = j < ld ? W[(size_t)i * ld + j] : 0.0;
          v2[c] = (has2 && j < ld) ? W[(size_t)i2 * ld + j] : 0.0;
        }
        const double f1 = (i != k) ? colk[i] : 0.0;
        const double f2 = (has2 && i2 != k) ? colk[i2] : 0.0;
#pragma unroll
        for (int c = 0; c < kGjChunk; ++c) {
          v1[c] = fma(-f1, rk[c], v1[c]);
          v2[c] = fma(-f2, rk[c], v2[c]);
        }
#pragma unroll
        for (int c = 0; c < kGjChunk; ++c) {
          const int j = c0 + lane + 32 * c;
          if (j < ld) {
            if (i != k) W[(size_t)i * ld + j] = v1[c];
            if (has2 && i2 != k) W[(size_t)i2 * ld + j] = v2[c];
          }
        }
      }
    }
    __syncthreads();
  }
  return 0;
}

// Recomputes G^up and G^dn (working precision T, leading dimension ldG) for
// the field s.  Returns max |G_old - G_new| over both spins when with_drift,
// 0 otherwise, and -1 after a zero pivot (status bit set).
template <typename T, int NT>
__device__ double recompute_green(const GridConst& gc, const int8_t* s, T* Gup, T* Gdn, int ldG,
                                  double* W, double* red, int* redi, double* s_inv, int* s_piv,
                                  double* colk, bool with_drift, int* status_word) {
  constexpr int NW = NT / 32;
  const int L = gc.L, ld = 2 * L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double dmax = 0.0;
  bool finite = true;
  for (int sp = 0; sp < 2; ++sp) {
    T* G = sp ? Gdn : Gup;
    const int sig = sp ? -1 : 1;
    for (int i = warp; i < L; i += NW) {
      const double* Mi = gc.M + (size_t)i * L;
      double* Wi = W + (size_t)i * ld;
      for (int j = lane; j < L; j += 32) {
        const double m = Mi[j];
        const double d = (sig * (int)s[j] > 0) ? gc.dV[0] : gc.dV[1];
        const double e = (i == j) ? 1.0 : 0.0;
        Wi[j] = e + (e - m) * d;
        Wi[L + j] = m;
      }
    }
    __syncthreads();
    if (gj_eliminate<NT>(W, L, red, redi, s_inv, s_piv, colk) != 0) {
      if (tid == 0) atomicOr(status_word, kStatusSingular);
      return -1.0;
    }
    for (int i = warp; i < L; i += NW) {
      const double* Wi = W + (size_t)i * ld + L;
      T* Gi = G + (size_t)i * ldG;
      for (int j = lane; j < L; j += 32) {
        const double gn = Wi[j];
        if (with_drift) dmax = fmax(dmax, fabs((double)Gi[j] - gn));
        finite = finite && isfinite(gn);
        Gi[j] = (T)gn;
      }
    }
    __syncthreads();
  }
  if (!finite) atomicOr(status_word, kStatusNonFinite);
  return with_drift ? block_max<NT>(dmax, red) : 0.0;
}

// ---------------------------------------------------------------------------
// Cheaper recompute through the inverse: since G^{-1} = M^{-1} A,
//   G^{-1} = B = M^{-1} (1 + D) - D,   D = diag(e^{sigma lambda s} - 1),
// built in O(L^2) from the bath's FP64 inverse M^{-1} (one per grid), and G is
// B inverted in place by Gauss-Jordan with partial pivoting (row swaps
// recorded, undone as column swaps at the end): L^3 DFMA per spin instead of
// 1.5 L^3, on an L x L workspace.  For lambda = 0 (U = 0) D = 0 and G = M is
// copied exactly.
// ---------------------------------------------------------------------------
template <int NT>
__device__ int gj_invert_inplace(double* B, int L, double* red, int* redi, double* s_inv, int* s_piv,
                                 double* colk, int* perm) {
  constexpr int kGjChunk = gj_chunk<NT>();
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ld = L;
  for (int k = 0; k < L; ++k) {
    double best = -1.0;
    int bi = L;
    for (int i = k + tid; i < L; i += NT) {
      const double v = fabs(B[(size_t)i * ld + k]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      red[warp] = best;
      redi[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double b = red[0];
      int p = redi[0];
      for (int w = 1; w < NW; ++w)
        if (red[w] > b || (red[w] == b && redi[w] < p)) {
          b = red[w];
          p = redi[w];
        }
      if (!(b > 0.0) || p >= L) {
        *s_piv = -1;
      } else {
        *s_piv = p;
        *s_inv = 1.0 / B[(size_t)p * ld + k];
        perm[k] = p;
      }
    }
    __syncthreads();
    const int p = *s_piv;
    if (p < 0) return -1;
    const double inv = *s_inv;
    // swap rows k and p, scale the new row k (its column-k entry becomes
    // 1/pivot: the identity column folded in); record column k of the rest
    for (int j = tid; j < ld; j += NT) {
      const double a = B[(size_t)k * ld + j];
      const double b = B[(size_t)p * ld + j];
      B[(size_t)p * ld + j] = a;
      B[(size_t)k * ld + j] = (j == k) ? inv : b * inv;
      if (j == k) colk[p] = a;
    }
    for (int i = tid; i < L; i += NT)
      if (i != k && i != p) colk[i] = B[(size_t)i * ld + k];
    __syncthreads();
    // eliminate: row i -= f_i * row k over all columns (column k of row i
    // starts from 0, the identity column)
    const double* bk = B + (size_t)k * ld;
    for (int c0 = 0; c0 < ld; c0 += 32 * kGjChunk) {
      double rk[kGjChunk];
#pragma unroll
      for (int c = 0; c < kGjChunk; ++c) {
        const int j = c0 + lane + 32 * c;
        rk[c] = j < ld ? bk[j] : 0.0;
      }
      for (int i = warp; i < L; i += 2 * NW) {
        const int i2 = i + NW;
        const bool has2 = i2 < L;
        double v1[kGjChunk], v2[kGjChunk];
#pragma unroll
        for (int c = 0; c < kGjChunk; ++c) {
          const int j = c0 + lane + 32 * c;
          v1[c] = (j < ld && j != k) ? B[(size_t)i * ld + j] : 0.0;
          v2[c] = (has2 && j < ld && j != k) ? B[(size_t)i2 * ld + j] : 0.0;
        }
        const double f1 = (i != k) ? colk[i] : 0.0;
        const double f2 = (has2 && i2 != k) ? colk[i2] : 0.0;
#pragma unroll
        for (int c = 0; c < kGjChunk; ++c) {
          v1[c] = fma(-f1, rk[c], v1[c]);
          v2[c] = fma(-f2, rk[c], v2[c]);
        }
#pragma unroll
        for (int c = 0; c < kGjChunk; ++c) {
          const int j = c0 + lane + 32 * c;
          if (j < ld) {
            if (i != k) B[(size_t)i * ld + j] = v1[c];
            if (has2 && i2 != k) B[(size_t)i2 * ld + j] = v2[c];
          }
        }
      }
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first; a thread
  // owns whole rows here, so the swaps need no barrier between them
  for (int i = tid; i < L; i += NT) {
    double* Bi = B + (size_t)i * ld;
    for (int k = L - 1; k >= 0; --k) {
      const int p = perm[k];
      if (p != k) {
        const double t = Bi[k];
        Bi[k] = Bi[p];
        Bi[p] = t;
      }
    }
  }
  __syncthreads();
  return 0;
}

// Recomputes G^up and G^dn through the inverse (see above); [sp_lo, sp_hi)
// selects the spins (0: up, 1: down).  W: L x L FP64
// workspace; colk: L doubles and perm: L ints of shared scratch.  Returns the
// drift max |G_old - G_new| when with_drift, 0 otherwise, -1 after a zero pivot.
template <typename T, int NT>
__device__ double recompute_green_inv(const GridConst& gc, const int8_t* s, T* Gup, T* Gdn, int ldG,
                                      double* W, double* red, int* redi, double* s_inv, int* s_piv,
                                      double* colk, int* perm, bool with_drift, int* status_word,
                                      int sp_lo = 0, int sp_hi = 2) {
  constexpr int NW = NT / 32;
  const int L = gc.L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double dmax = 0.0;
  bool finite = true;
  const bool free_bath = gc.lambda == 0.0;
  for (int sp = sp_lo; sp < sp_hi; ++sp) {
    T* G = sp ? Gdn : Gup;
    const int sig = sp ? -1 : 1;
    const double* src = gc.M;
    if (!free_bath) {
      for (int i = warp; i < L; i += NW) {
        const double* Mi = gc.Minv + (size_t)i * L;
        double* Wi = W + (size_t)i * L;
        for (int j = lane; j < L; j += 32) {
          const double d = (sig * (int)s[j] > 0) ? gc.dV[0] : gc.dV[1];
          Wi[j] = Mi[j] * (1.0 + d) - ((i == j) ? d : 0.0);
        }
      }
      __syncthreads();
      if (gj_invert_inplace<NT>(W, L, red, redi, s_inv, s_piv, colk, perm) != 0) {
        if (tid == 0) atomicOr(status_word, kStatusSingular);
        return -1.0;
      }
      src = W;
    }
    for (int i = warp; i < L; i += NW) {
      const double* Si = src + (size_t)i * L;
      T* Gi = G + (size_t)i * ldG;
      for (int j = lane; j < L; j += 32) {
        const double gn = Si[j];
        if (with_drift) dmax = fmax(dmax, fabs((double)Gi[j] - gn));
        finite = finite && isfinite(gn);
        Gi[j] = (T)gn;
      }
    }
    __syncthreads();
  }
  if (!finite) atomicOr(status_word, kStatusNonFinite);
  return with_drift ? block_max<NT>(dmax, red) : 0.0;
}

}  // namespace hfq
