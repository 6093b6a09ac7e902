// FP64 recomputation of the Green matrices from the field:
//   G^sigma = A^{-1} M,  A^sigma = 1 + (1 - M) diag(e^{sigma lambda s} - 1),
// the Dyson equation that links the interacting G to the bath G0 (= M) in
// Hirsch-Fye QMC.  It is the only FP64 step of the FP32 sweep paths and is
// followed by the drift check max |G_fast - G_fresh|.
//
// Two algorithms, both Gauss-Jordan elimination with partial pivoting by one
// CTA, bound by the FP64 pipe (about 2 DFMA/clk/SM on GB300):
//  * recompute_green: on the augmented L x 2L matrix [A | M], 1.5 L^3 DFMA
//    per spin.  Used by the entry point that allocates nothing.
//  * recompute_green_inv: G = B^{-1} with B = M^{-1}(1 + D) - D inverted in
//    place, L^3 DFMA per spin on an L x L workspace.  Used by every sweep
//    kernel and the initialisation.  Two forms of the inversion:
//    gj_invert_inplace (row interchanges; three barriers per pivot column:
//    search, swap + scale, elimination) on a workspace in shared memory
//    (rank-1 paths and initialisation, Lambda <= 168) or in HBM when nothing
//    else fits; gj_invert_blocked (implicit pivoting, kGjPanel columns per
//    panel in shared memory, two barriers per pivot column) on the chain's
//    HBM workspace, which it reads and writes once per panel instead of once
//    per pivot column -- the FP32 delayed path always, the initialisation
//    whenever the panel fits.
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

// ---------------------------------------------------------------------------
// Blocked form of the same inversion for a workspace in HBM.  Rows are never
// interchanged (implicit pivoting): step k takes as pivot p_k the row of
// largest |B_ik| among the rows not yet used (ties: lowest index), scales row
// p_k and eliminates column k from every other row, the identity column
// folded in as above.  Relabelling row p_k as row k makes this the unpivoted
// in-place inversion of P B, whose result is (P B)^{-1} = B^{-1} P^T; with
// pos(p_k) = k the inverse is
//   (B^{-1})_{km} = B'_{p_k, pos(m)}           (B' the array on return),
// applied by the caller while it copies the result out.
//
// The pivot columns are taken kGjPanel at a time.  A panel (all L rows of
// columns k0 .. k0 + b - 1) is reduced in shared memory by the b steps; for
// every other column x the b steps compose to
//   x <- x + (V - E) x_P,
// V the reduced panel, P the panel's pivot rows and E their unit rows (a
// product of the steps' rank-1 maps, each x <- x + (v_k - e_{p_k}) x_{p_k}),
// so the rest of B takes one rank-b update per panel: its rows p in P are
// replaced by V_p x_P and the other rows i get x_i + V_i x_P.  B is read and
// written once per panel (L^3 / b words in all) instead of once per pivot
// column (L^3), and the update runs from registers at the FP64 pipe's rate.
// pan: gj_blocked_bytes(L) of shared scratch (the panel, pitch kGjPanel + 1,
// then the pivot rows' slab, pitch L); perm, pos: L ints each of shared
// memory (pivot row of step k; step of row i).  Returns -1 on a zero pivot
// (uniformly in all threads), 0 otherwise.
// ---------------------------------------------------------------------------

template <int NT>
__device__ int gj_invert_blocked(double* B, int L, double* red, int* redi, double* s_inv, int* s_piv,
                                 int* perm, int* pos, double* pan) {
  constexpr int NW = NT / 32;
  constexpr int KB = kGjPanel, PP = KB + 1;  // odd pitch: a column of the panel is conflict-free
  constexpr int TR = 8;                      // rows of an update item (one warp, 32 columns)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* slab = pan + (size_t)L * PP;
  for (int i = tid; i < L; i += NT) pos[i] = -1;
  __syncthreads();
  for (int k0 = 0; k0 < L; k0 += KB) {
    const int bb = min(KB, L - k0);
    for (int i = warp; i < L; i += NW)
      if (lane < bb) pan[i * PP + lane] = B[(size_t)i * L + k0 + lane];
    __syncthreads();
    // the largest |pivot| (then the lowest row) among the unused rows,
    // compared as the magnitudes' bit patterns: for non-negative doubles
    // their order is that of unsigned integers, and the integer compares
    // keep the search off this part's slow FP64 pipe.  Each warp's best
    // candidate goes to red / redi: for the panel's first column from a
    // search here, for every later column from the rows just updated.
    auto offer = [&](unsigned long long best, int bi) {
      for (int o = 16; o; o >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        reinterpret_cast<unsigned long long*>(red)[warp] = best;
        redi[warp] = bi;
      }
    };
    {
      unsigned long long best = 0ull;
      int bi = L;
      for (int i = tid; i < L; i += NT)
        if (pos[i] < 0) {
          const unsigned long long v = __double_as_longlong(pan[i * PP]) & 0x7fffffffffffffffull;
          if (v > best) {
            best = v;
            bi = i;
          }
        }
      offer(best, bi);
    }
    __syncthreads();
    for (int t = 0; t < bb; ++t) {
      const int k = k0 + t;
      if (warp == 0) {
        // the warps' candidates, the reciprocal, and the pivot row scaled
        // (its column-t entry becomes the reciprocal) into the slab's first
        // KB words, which the update overwrites later; the panel's copy is
        // replaced after the barrier
        unsigned long long best = lane < NW ? reinterpret_cast<const unsigned long long*>(red)[lane] : 0ull;
        int bi = lane < NW ? redi[lane] : L;
        for (int o = 16; o; o >>= 1) {
          const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ov > best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
          }
        }
        const bool ok = best > 0ull && bi < L;
        const double inv = ok ? 1.0 / pan[bi * PP + t] : 0.0;
        if (ok && lane < bb) slab[lane] = (lane == t) ? inv : pan[bi * PP + lane] * inv;
        if (lane == 0) {
          *s_piv = ok ? bi : -1;
          *s_inv = inv;
          if (ok) {
            perm[k] = bi;
            pos[bi] = k;
          }
        }
      }
      // warp 0 has read every candidate before this barrier, so the
      // candidates of column t + 1 may overwrite them after it
      __syncthreads();
      const int p = *s_piv;
      if (p < 0) return -1;
      const double inv = *s_inv;
      unsigned long long best = 0ull;
      int bi = L;
      for (int i = tid; i < L; i += NT) {
        double* pr = pan + i * PP;
        if (i == p) {
#pragma unroll
          for (int u = 0; u < KB; ++u)
            if (u < bb) pr[u] = slab[u];
          continue;
        }
        const double c = pr[t];
#pragma unroll
        for (int u = 0; u < KB; ++u)
          if (u < bb && u != t) pr[u] = fma(-c, slab[u], pr[u]);
        pr[t] = -c * inv;
        if (t + 1 < bb && pos[i] < 0) {
          const unsigned long long v = __double_as_longlong(pr[t + 1]) & 0x7fffffffffffffffull;
          if (v > best) {
            best = v;
            bi = i;
          }
        }
      }
      if (t + 1 < bb) offer(best, bi);
      __syncthreads();
    }
    // the pivot rows of the other columns, then their rank-b update, in
    // items of TR rows x 32 columns spread over the warps; the nR other
    // columns are numbered c = 0 .. nR - 1 around the panel
    const int* pk = perm + k0;
    for (int e = tid; e < bb * L; e += NT) {
      const int t = e / L, j = e - t * L;
      slab[e] = B[(size_t)pk[t] * L + j];
    }
    __syncthreads();
    const int nR = L - bb;
    const int ncg = (nR + 31) / 32, nrb = (L + TR - 1) / TR;
    for (int it = warp; it < ncg * nrb; it += NW) {
      const int cg = it % ncg, r0 = (it / ncg) * TR;
      const int c = cg * 32 + lane;
      const bool jin = c < nR;
      const int j = c < k0 ? c : c + bb;
      double acc[TR];
#pragma unroll
      for (int q = 0; q < TR; ++q) {
        const int i = r0 + q;
        const bool piv = i < L && pos[i] >= k0 && pos[i] < k0 + bb;
        acc[q] = (jin && i < L && !piv) ? B[(size_t)i * L + j] : 0.0;
      }
#pragma unroll
      for (int t = 0; t < KB; ++t) {
        if (t < bb) {
          const double sv = jin ? slab[t * L + j] : 0.0;
#pragma unroll
          for (int q = 0; q < TR; ++q)
            if (r0 + q < L) acc[q] = fma(pan[(r0 + q) * PP + t], sv, acc[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < TR; ++q)
        if (jin && r0 + q < L) B[(size_t)(r0 + q) * L + j] = acc[q];
    }
    for (int i = warp; i < L; i += NW)
      if (lane < bb) B[(size_t)i * L + k0 + lane] = pan[i * PP + lane];
    __syncthreads();
  }
  return 0;
}

// Recomputes G^up and G^dn through the inverse (see above); [sp_lo, sp_hi)
// selects the spins (0: up, 1: down).  W: L x L FP64
// workspace; colk: L doubles and perm: L ints of shared scratch.  kBlocked:
// inverted by panels, pan being gj_blocked_bytes(L) of shared scratch (colk
// then holds the row positions).  Returns the drift max |G_old - G_new| when
// with_drift, 0 otherwise, -1 after a zero pivot.
template <typename T, int NT, bool kBlocked = false>
__device__ double recompute_green_inv(const GridConst& gc, const int8_t* s, T* Gup, T* Gdn, int ldG,
                                      double* W, double* red, int* redi, double* s_inv, int* s_piv,
                                      double* colk, int* perm, bool with_drift, int* status_word,
                                      int sp_lo = 0, int sp_hi = 2, double* pan = nullptr) {
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
      int rc;
      if constexpr (kBlocked)
        rc = gj_invert_blocked<NT>(W, L, red, redi, s_inv, s_piv, perm, reinterpret_cast<int*>(colk), pan);
      else
        rc = gj_invert_inplace<NT>(W, L, red, redi, s_inv, s_piv, colk, perm);
      if (rc != 0) {
        if (tid == 0) atomicOr(status_word, kStatusSingular);
        return -1.0;
      }
      src = W;
    }
    // the blocked inversion leaves row p_k of the inverse at row perm[k] and
    // its column m at column pos[m]
    const bool implicit = kBlocked && !free_bath;
    const int* pos = reinterpret_cast<const int*>(colk);
    for (int i = warp; i < L; i += NW) {
      const double* Si = src + (size_t)(implicit ? perm[i] : i) * L;
      T* Gi = G + (size_t)i * ldG;
      for (int j = lane; j < L; j += 32) {
        const double gn = Si[implicit ? pos[j] : j];
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
