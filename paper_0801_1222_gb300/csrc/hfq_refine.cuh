// Recompute of the FP32 delayed path by one or two Newton steps from the
// current G, with the residual formed exactly enough on the tensor cores.
//
// The Hirsch-Fye Dyson equation G = [1 + (1 - M)(e^V - 1)]^{-1} M, with
// D = diag(e^{sigma lambda s} - 1), reads G^{-1} = B = M^{-1}(1 + D) - D =
// A (1 + D), A = M^{-1} - diag(1 - e^{-sigma lambda s_j}).  For an FP32 G
// that has drifted by rounding since the last recompute, Newton's iteration
// for the inverse
//     E = 1 - B G',      G_new = G' + G' E,      1 - B G_new = E^2,
// brings G back to the inverse of B for the current field in one step when
// |E| is small (the drift of N_wrap = 64 flips gives |E| ~ 1e-4).  Written
// with H' = (1 + D) G' (rows of G' scaled):
//     E = 1 - A H',      G_new = (1 + D)^{-1} (H' + H' E).
//
// E needs FP64-level accuracy where G' nearly inverts B, which FP32 products
// cannot give; the residual product A H' is therefore formed from integer
// slices (the splitting idea of Ozaki, Ogita, Oishi and Rump, written here
// for FP16 tensor-core operands):
//   * A (one table per grid, hfq_setup's k_refine_prep) = 2^ea sum_p a_p 2^{-7(p+1)},
//     6 signed 7-bit slices; the field-dependent diagonal is patched in per chain;
//   * H' = the FP32 H = fl32((1 + d_j) G_jn) rounded to the grid 2^{eh-28}
//     (eh: |H| < 2^eh) = 2^eh sum_q h_q 2^{-7(q+1)}, 4 slices, cut straight
//     into shared memory chunk by chunk while A's slices arrive.  G' =
//     (1 + D)^{-1} H' differs from G by at most half that grid step; E and
//     the update both use this same G', so Newton's identity holds for it;
//   * a_p, h_q are integers with |.| <= 128 (first slice) or <= 64, exact in
//     FP16.  The products with p + q = l go to one FP32 TMEM accumulator per
//     level l = 0..5 (at most four pairs, each K term <= 6 * 2^12 in all, so
//     every partial sum is an integer below 2^24 for Lambda <= 512: the
//     accumulation is exact).  Dropped levels and the slices' remainders
//     leave |E - E_exact| ~ 1e-10 of |A||H'|.
//   * The six level sums are combined exactly in 64-bit integers,
//     V = sum_l S_l 2^{7 (5 - l)}, so A H' = V 2^{ea + eh - 49}, and
//     E = delta - V 2^{ea+eh-49} is formed as an integer before it is
//     rounded to FP32: the cancellation costs nothing.
// The update H' E only needs FP32 accuracy (|E| is small): split FP16
// hi/lo parts with power-of-two scales, three products, FP32 accumulation.
//
// max |E| over the matrix decides: above rc.emax_step (2^-8 by default) the
// step is not taken and the caller recomputes G from scratch (Gauss-Jordan);
// above 2^-13 a second step follows.  The drift reported is the largest
// change of an entry over the steps.
#pragma once
#include <cuda_fp16.h>

#include "hfq_delayed.cuh"
#include "hfq_device.cuh"

namespace hfq {

static_assert(kDelNT == 512, "the refinement's TMEM read-out assumes 16 warps");

// The thread that issues (and commits) the residual product's MMAs: lane 0
// of the last warp, which cuts no H' slices, so the issue overlaps the
// slicing of the next chunk (threads 0 .. 255).
constexpr int kRfIssuer = kDelNT - 32;
static_assert(kRfIssuer >= kRfNMax * (kRfKC / 8), "the MMA issuer must not slice");
static_assert(kTmemCols >= kRfLevels * kRfNMax, "level accumulators must fit the TMEM allocation");

// K-major core-matrix layout (8 rows x 16 bytes per core matrix, contiguous
// along K): element (r, m) of a tile with K extent kRfKC (the residual
// product's chunks) or kRf2KC (the update's)
__device__ __forceinline__ uint32_t rf_off(int r, int m) {
  return (uint32_t)((r >> 3) * (kRfKC / 8) * 128 + (m >> 3) * 128 + (r & 7) * 16 + (m & 7) * 2);
}
__device__ __forceinline__ uint32_t rf_off2(int r, int m) {
  return (uint32_t)((r >> 3) * (kRf2KC / 8) * 128 + (m >> 3) * 128 + (r & 7) * 16 + (m & 7) * 2);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// bulk copy global -> this CTA's shared memory, completion counted on mbar
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// 2^k as an FP32 number, -126 <= k <= 127 (scalings by it are exact while
// the result stays normal)
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// 32 lanes x 32 bit, 8 consecutive columns per thread
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Block-wide max of non-negative floats, NaN counted as infinity; every
// thread gets the result.  red: kDelNT / 32 floats.  Contains barriers.
__device__ __forceinline__ float rf_block_max(float v, float* red) {
  v = (v == v) ? v : __int_as_float(0x7f800000);
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = 0.f;
#pragma unroll
  for (int w = 0; w < kDelNT / 32; ++w) r = fmaxf(r, red[w]);
  __syncthreads();
  return r;
}

// x[0..7] = p[0..7], entries t >= n read as 0.  vec: p is 16-byte aligned
// and n is a multiple of four (or <= 0), so two float4 loads serve.
__device__ __forceinline__ void rf_ld8(const float* p, int n, bool vec, float* x) {
  if (vec) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (n >= 4) a = *reinterpret_cast<const float4*>(p);
    if (n >= 8) b = *reinterpret_cast<const float4*>(p + 4);
    x[0] = a.x, x[1] = a.y, x[2] = a.z, x[3] = a.w, x[4] = b.x, x[5] = b.y, x[6] = b.z, x[7] = b.w;
  } else {
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = t < n ? p[t] : 0.f;
  }
}

// p[0..7] = x[0..7] for t < n (same vec contract as rf_ld8)
__device__ __forceinline__ void rf_st8(float* p, int n, bool vec, const float* x) {
  if (vec) {
    if (n >= 4) *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    if (n >= 8) *reinterpret_cast<float4*>(p + 4) = make_float4(x[4], x[5], x[6], x[7]);
  } else {
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (t < n) p[t] = x[t];
  }
}

// The nearest integers ra, rb of a, b (|a|, |b| <= 2^7; ties to even, as
// rintf) and both as FP16, packed (a in the low half), with full-rate FP32,
// integer and FP16x2 arithmetic only: adding 1.5 * 2^23 rounds to an integer
// (the FP32 spacing there is 1), whose bits give v; the FP16 bits of 1536 + v
// are 0x6600 + v (spacing 1 in [1024, 2048)), and 1536 subtracted in FP16
// leaves v exactly.
__device__ __forceinline__ uint32_t rf_round_h2(float a, float b, float* ra, float* rb) {
  const float ta = a + 12582912.f, tb = b + 12582912.f;
  *ra = ta - 12582912.f;
  *rb = tb - 12582912.f;
  const uint32_t pk = ((0x6600u + (uint32_t)(__float_as_int(ta) - 0x4B400000)) & 0xffffu) |
                      ((0x6600u + (uint32_t)(__float_as_int(tb) - 0x4B400000)) << 16);
  const uint32_t c1536 = 0x66006600u;
  __half2 hv, hc;
  memcpy(&hv, &pk, 4);
  memcpy(&hc, &c1536, 4);
  hv = __hsub2(hv, hc);
  uint32_t r;
  memcpy(&r, &hv, 4);
  return r;
}

// One spin: G (L x L, row-major, FP32, in global memory) is replaced by its
// Newton-refined value.  s: the field (shared memory); sig: +1 / -1; ws: the
// chain's workspace (E^T: L rows of rf_pad(L, 4) floats); sm: rf_smem_need(L) of 1024-byte aligned
// shared memory; tc: the CTA's TMEM allocation and mbarriers (tc->cbar: bulk
// copies into the two stage buffers, then their MMA completions).
// Returns the largest change of an entry (>= 0), or -1 if the caller must
// recompute from scratch (|E| too large, scale out of range, or a wait gave
// up, which also sets kStatusTimeout).  All threads call it.
__device__ inline float refine_spin(const GridConst& gc, const RefineConst& rc, const int8_t* s, int sig,
                                    float* G, float* ws, unsigned char* sm, TcState* tc, float* red, int* status,
                                    int* steps) {
  const int L = gc.L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kDelNT / 32;
  const int q4 = warp & 3, g4 = warp >> 2;  // TMEM lane quarter, column group (the update's epilogue)
  const int nkc = rc.nkc, nrb = rc.nrb;
  const int nN = rc.nN, nnb = rf_pad(L, nN) / nN;
  float* wsE = ws;
  const int ldE = rf_pad(L, 4);     // row stride of E^T in ws
  const bool vec = (L & 3) == 0;    // rows of G 16-byte aligned: float4 accesses
  const uint32_t sm0 = smem_u32(sm);
  // the row factors in registers: (1 + d_j) and its inverse as an FP32 pair,
  // selected by sigma s_j (index 0: +1, 1: -1)
  const float cpl0 = rc.cplus[0], cpl1 = rc.cplus[1];
  const float cmh0 = rc.cminus_hi[0], cmh1 = rc.cminus_hi[1], cml0 = rc.cminus_lo[0], cml1 = rc.cminus_lo[1];
  float drift = 0.f;
  uint32_t ph = tc->cphase;  // parity bits of the four barriers: copy 0, copy 1, MMA 0, MMA 1
  for (int step = 0; step < 2; ++step) {
    // ---- H = (1 + d_j) G_jn: its scale ------------------------------------
    float hmax = 0.f;
    for (int j = warp; j < L; j += NW) {
      const float cp = sig * s[j] > 0 ? cpl0 : cpl1;
      const float* Gj = G + (size_t)j * L;
      for (int n0 = 0; n0 < L; n0 += 32 * 8) {
        float g[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) g[u] = (n0 + 32 * u + lane < L) ? Gj[n0 + 32 * u + lane] : 0.f;  // loads first
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float H = g[u] * cp;
          hmax = (H == H) ? fmaxf(hmax, fabsf(H)) : __int_as_float(0x7f800000);
        }
      }
    }
    hmax = rf_block_max(hmax, red);
    int eh = 0;
    if (!(hmax < 1e30f)) {
      tc->cphase = ph;
      return -1.f;
    }
    if (hmax > 0.f) (void)frexpf(hmax, &eh);  // hmax < 2^eh
    const int sh = 49 - rc.ea - eh;           // delta in units of the integer sums
    if (sh < 0 || sh > 61 || eh < -60 || eh > 100) {  // keeps every scale below normal
      tc->cphase = ph;
      return -1.f;
    }
    const float s7 = pow2f(kRfBits - eh);  // H 2^{7-eh}: below 2^7 in magnitude

    // ---- GEMM1: E = 1 - A H', tile by tile (128 rows x nN columns) ---------
    // K goes in chunks of 32 through two stage buffers (A's six slices, 48
    // KiB, by one bulk copy; H''s four, up to 20 KiB, cut by nN * 4 threads from G):
    // chunk kc + 1 is brought in while the tensor cores multiply chunk kc.
    // Every commit of a chunk's MMAs is waited for exactly once, in order,
    // so each barrier's parity stays in step.
    float emax = 0.f;
    const uint32_t idesc1 = make_idesc_f16(nN);
    bool bad = false;  // a bounded wait gave up
    auto stage_in = [&](int nb, int rb, int kc, int b) {
      const uint32_t bar = tc->cbar + 8u * (uint32_t)b;
      if (tid == 0) {
        mbar_expect_tx(bar, (uint32_t)(kRfSlicesA * kRfTileA));
        bulk_g2s(sm0 + (uint32_t)(b * kRfStage), rc.aslc + (size_t)(rb * nkc + kc) * kRfSlicesA * (kRfTileA / 2),
                 (uint32_t)(kRfSlicesA * kRfTileA), bar);
      }
      if (tid < nN * (kRfKC / 8)) {
        // a column and eight rows of H' per thread, sliced into the buffer
        const int j8 = tid / nN, nl = tid - j8 * nN;
        const int n = nb * nN + nl, j0 = kc * kRfKC + j8 * 8;
        float y[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int j = j0 + t;
          y[t] = (j < L && n < L) ? G[(size_t)j * L + n] : 0.f;  // all loads first
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int j = j0 + t;
          y[t] = y[t] * (j < L && sig * s[j] > 0 ? cpl0 : cpl1) * s7;
        }
        unsigned char* dst = sm + b * kRfStage + kRfSlicesA * kRfTileA + rf_off(nl, j8 * 8);
#pragma unroll
        for (int q = 0; q < kRfSlicesH; ++q) {
          // slice q: the nearest integer v of the running remainder (below
          // 2^7 in magnitude), which then moves up 7 bits
          uint32_t w[4];
#pragma unroll
          for (int t = 0; t < 8; t += 2) {
            float ra, rb2;
            w[t / 2] = rf_round_h2(y[t], y[t + 1], &ra, &rb2);
            y[t] = (y[t] - ra) * (float)(1 << kRfBits);
            y[t + 1] = (y[t + 1] - rb2) * (float)(1 << kRfBits);
          }
          *reinterpret_cast<uint4*>(dst + q * kRfTileH) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
    };
    auto wait_mma = [&](int b) {  // chunk MMAs of buffer b complete (every thread)
      const uint32_t bit = 4u << b;
      if (!mbar_wait_bounded(tc->cbar + 16u + 8u * (uint32_t)b, (ph & bit) ? 1u : 0u)) bad = true;
      ph ^= bit;
    };
    for (int nb = 0; nb < nnb; ++nb) {
      for (int rb = 0; rb < nrb; ++rb) {
        stage_in(nb, rb, 0, 0);
        for (int kc = 0; kc < nkc; ++kc) {
          const int b = kc & 1;
          const uint32_t cbit = 1u << b;
          const bool got = mbar_wait_bounded(tc->cbar + 8u * (uint32_t)b, (ph & cbit) ? 1u : 0u);
          ph ^= cbit;
          // the field-dependent diagonal of A
          if (tid < kRfKC) {
            const int j = kc * kRfKC + tid;
            if (j >= rb * 128 && j < rb * 128 + 128 && j < L) {
              const int v = sig * s[j] > 0 ? 0 : 1;
              const uint32_t off = rf_off(j - rb * 128, tid);
#pragma unroll
              for (int p = 0; p < kRfSlicesA; ++p)
                *reinterpret_cast<uint16_t*>(sm + b * kRfStage + p * kRfTileA + off) = rc.dslc[v][p];
            }
          }
          fence_async_smem();
          tc_fence_before();
          if (!__syncthreads_and((got && !bad) ? 1 : 0)) {
            if (tid == 0) atomicOr(status, kStatusTimeout);
            tc->failed = 1;
            tc->cphase = ph;
            return -1.f;
          }
          if (tid == kRfIssuer) {
            tc_fence_after();
            // descriptors of slice p / q at K step kk: the base one plus the
            // byte offset >> 4 in the start-address field (no carry out of it:
            // shared addresses stay below 256 KiB); the first product of a
            // level in a tile starts its accumulator
            const uint32_t aB = sm0 + (uint32_t)(b * kRfStage), hB = aB + (uint32_t)(kRfSlicesA * kRfTileA);
#pragma unroll
            for (int kk = 0; kk < kRfKC / 16; ++kk) {
              const uint64_t da = make_smem_desc(aB + (uint32_t)(kk * 256), 128u, (kRfKC / 8) * 128u);
              const uint64_t db = make_smem_desc(hB + (uint32_t)(kk * 256), 128u, (kRfKC / 8) * 128u);
#pragma unroll
              for (int p = 0; p < kRfSlicesA; ++p)
#pragma unroll
                for (int q = 0; q < kRfSlicesH; ++q) {
                  const int lv = p + q;
                  if (lv >= kRfLevels) continue;
                  const int first_p = lv > kRfSlicesH - 1 ? lv - (kRfSlicesH - 1) : 0;
                  const int acc = (kc > 0 || kk > 0 || p != first_p) ? 1 : 0;
                  tc_mma_f16(tc->tmem + (uint32_t)(lv * nN), da + (uint64_t)(p * (kRfTileA >> 4)),
                             db + (uint64_t)(q * (kRfTileH >> 4)), idesc1, acc);
                }
            }
            tc_commit(tc->cbar + 16u + 8u * (uint32_t)b);
          }
          if (kc >= 1) wait_mma(b ^ 1);  // chunk kc - 1 done: its buffer is free
          if (kc + 1 < nkc) stage_in(nb, rb, kc + 1, b ^ 1);
        }
        wait_mma((nkc - 1) & 1);
        if (!__syncthreads_and(bad ? 0 : 1)) {
          if (tid == 0) atomicOr(status, kStatusTimeout);
          tc->failed = 1;
          tc->cphase = ph;
          return -1.f;
        }
        tc_fence_after();
        // the six level sums of a row and 16 columns per task (TMEM lane
        // quarter warp % 4, columns 16 g ..), 8 at a time, combined in 64-bit
        // integers, then E = delta - V 2^{ea+eh-49}
        const long long one = 1ll << sh;
#pragma unroll 1
        for (int task = warp; task < 4 * (nN / 16); task += NW) {
          const int g16 = task >> 2;
          const int i = rb * 128 + 32 * q4 + lane;
#pragma unroll 1
          for (int h8 = 0; h8 < 2; ++h8) {
            long long V[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) V[c] = 0;
#pragma unroll
            for (int lv = 0; lv < kRfLevels; ++lv) {
              float v[8];
              tmem_ld8(tc->tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(lv * nN + 16 * g16 + 8 * h8), v);
#pragma unroll
              for (int c = 0; c < 8; ++c) V[c] = V[c] * (1ll << kRfBits) + (long long)__float2int_rn(v[c]);
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const int n = nb * nN + 16 * g16 + 8 * h8 + c;
              const long long Ei = (i == n ? one : 0ll) - V[c];
              float E;
              if (Ei > (1ll << 54) || Ei < -(1ll << 54)) {
                E = __int_as_float(0x7f800000);  // far beyond the step's range
              } else {
                const float hi = (float)(int)(Ei >> 24), lo = (float)(int)(Ei & 0xffffffll);
                E = fmaf(hi, 16777216.f, lo) * pow2f(-sh);
              }
              // E^T: lanes (rows i) write consecutive words; rows i >= L of E
              // are exactly 0 (A's table is zero there), which fills the
              // padding of E^T's rows
              if (i < ldE && n < L) wsE[(size_t)n * ldE + i] = E;
              if (i < L && n < L) emax = fmaxf(emax, fabsf(E));
            }
          }
        }
        tc_fence_before();
        __syncthreads();
      }
    }
    emax = rf_block_max(emax, red);
    if (!(emax <= rc.emax_step)) {  // too far for Newton steps (default 2^-8)
      tc->cphase = ph;
      return -1.f;
    }
    int ee = 0;
    if (emax > 0.f) (void)frexpf(emax, &ee);  // emax < 2^ee
    // E 2^se below 2^15 (FP16 range); for |E| < 2^-25 the scale stops at
    // 2^40, where those corrections are far below G's FP32 rounding anyway
    const int se = emax > 0.f ? min(15 - ee, 40) : 0;

    // ---- GEMM2: G_new = (1 + D)^{-1} (H' + H' E), 128 rows x all columns ----
    const int Lp = rf_pad(L, 16), nkc2 = rf_pad(L, kRf2KC) / kRf2KC;
    const uint32_t bl = (uint32_t)Lp * kRf2KC * 2u;  // bytes of one E^T part (hi or lo)
    constexpr uint32_t kAbuf = 2u * 128u * kRf2KC * 2u;  // one row block's H' hi and lo
    const float sH = pow2f(28 - eh);                // H' = rint(H 2^{28-eh}) 2^{eh-28}
    const float sE = pow2f(se), sHi = pow2f(eh - 28), sQ = pow2f(eh - 14 - se);
    // two row blocks of 128 and at most 256 columns: both blocks' products at
    // once (accumulators at TMEM columns 0 and 256), so each E^T chunk is
    // staged once; else one row block at a time
    const int nr = (nrb == 2 && Lp <= 256) ? 2 : 1;
    const uint32_t b2 = sm0 + (uint32_t)nr * kAbuf;
    for (int rb0 = 0; rb0 < nrb; rb0 += nr) {
      for (int kc = 0; kc < nkc2; ++kc) {
#pragma unroll 1
        for (int ur = 0; ur < nr; ++ur) {
        const int rb = rb0 + ur;
        unsigned char* sa = sm + ur * kAbuf;
        // A: H' of rows rb*128.. (x 2^{14-eh}, below 2^14), hi / lo: 1024
        // chunks of eight K values, two per thread, the loads of both first.
        // chunk c: row ((c >> 6) << 3) | (c & 7), K offset ((c >> 3) & 7) * 8, so
        // eight lanes write one 128-byte core-matrix row group (no bank conflict)
        {
          static_assert(128 * (kRf2KC / 8) == 2 * kDelNT, "two H' chunks per thread");
          float x[2][8];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int c = tid + u * kDelNT;
            const int i = rb * 128 + (((c >> 6) << 3) | (c & 7)), k0 = kc * kRf2KC + (((c >> 3) & 7) << 3);
            rf_ld8(G + (size_t)(i < L ? i : 0) * L + k0, i < L ? L - k0 : 0, vec, x[u]);
          }
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int c = tid + u * kDelNT;
            const int r = ((c >> 6) << 3) | (c & 7), m0 = ((c >> 3) & 7) << 3;
            const int i = rb * 128 + r;
            const float cp = (i < L && sig * s[i] > 0) ? cpl0 : cpl1;
            uint32_t h[4], l[4];
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
              const float xa = rintf(x[u][t] * cp * sH) * 0x1p-14f, xb = rintf(x[u][t + 1] * cp * sH) * 0x1p-14f;
              h[t / 2] = f32x2_to_f16x2(xa, xb);
              l[t / 2] = f32x2_to_f16x2(xa - f16_lo_to_f32(h[t / 2]), xb - f16_hi_to_f32(h[t / 2]));
            }
            const uint32_t off = rf_off2(r, m0);
            *reinterpret_cast<uint4*>(sa + off) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(sa + 128 * kRf2KC * 2 + off) = make_uint4(l[0], l[1], l[2], l[3]);
          }
        }
        }
        // B: E^T (row n = column n of E, K = rows of E) x 2^se, hi / lo;
        // wsE holds E^T, so a chunk is eight consecutive words of row n (two
        // float4 loads: ldE and the offsets are multiples of four); two
        // chunks per thread in flight
        const int nc2 = Lp * (kRf2KC / 8);
        for (int c0 = tid; c0 < nc2; c0 += 2 * kDelNT) {
          float x[2][8];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int c = c0 + u * kDelNT;
            const int n = ((c >> 6) << 3) | (c & 7), k0 = kc * kRf2KC + (((c >> 3) & 7) << 3);
            const bool ok = c < nc2 && n < L;
            rf_ld8(wsE + (size_t)(ok ? n : 0) * ldE + k0, ok ? ldE - k0 : 0, true, x[u]);
          }
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int c = c0 + u * kDelNT;
            if (c < nc2) {
              const int n = ((c >> 6) << 3) | (c & 7), m0 = ((c >> 3) & 7) << 3;
              uint32_t h[4], l[4];
#pragma unroll
              for (int t = 0; t < 8; t += 2) {
                const float xa = x[u][t] * sE, xb = x[u][t + 1] * sE;
                h[t / 2] = f32x2_to_f16x2(xa, xb);
                l[t / 2] = f32x2_to_f16x2(xa - f16_lo_to_f32(h[t / 2]), xb - f16_hi_to_f32(h[t / 2]));
              }
              const uint32_t off = rf_off2(n, m0);
              unsigned char* bp = sm + nr * kAbuf;
              *reinterpret_cast<uint4*>(bp + off) = make_uint4(h[0], h[1], h[2], h[3]);
              *reinterpret_cast<uint4*>(bp + bl + off) = make_uint4(l[0], l[1], l[2], l[3]);
            }
          }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
          tc_fence_after();
#pragma unroll 1
          for (int ur = 0; ur < nr; ++ur)
#pragma unroll 1
          for (int half = 0; half * 256 < Lp; ++half) {
            const int Nh = Lp - half * 256 < 256 ? Lp - half * 256 : 256;
            const uint32_t idesc2 = make_idesc_f16(Nh);
            const uint32_t bo = (uint32_t)half * 32u * 1024u;  // 256 rows of B: 32 groups of 8 x 1024 B
            const uint32_t a2 = sm0 + (uint32_t)ur * kAbuf;
#pragma unroll 1
            for (int kk = 0; kk < kRf2KC / 16; ++kk) {
              const uint32_t ko = (uint32_t)kk * 256u;
              const uint32_t d = tc->tmem + (uint32_t)((ur + half) * 256);
              const uint64_t ahi = make_smem_desc(a2 + ko, 128u, (kRf2KC / 8) * 128u);
              const uint64_t bhi = make_smem_desc(b2 + bo + ko, 128u, (kRf2KC / 8) * 128u);
              tc_mma_f16(d, ahi, bhi, idesc2, (kc > 0 || kk > 0) ? 1 : 0);
              tc_mma_f16(d, ahi, bhi + (uint64_t)(bl >> 4), idesc2, 1);
              tc_mma_f16(d, ahi + (uint64_t)((128u * kRf2KC * 2u) >> 4), bhi, idesc2, 1);
            }
          }
        }
        if (!tc_commit_wait(tc)) {
          if (tid == 0) atomicOr(status, kStatusTimeout);
          tc->failed = 1;
          tc->cphase = ph;
          return -1.f;
        }
      }
      // epilogue: rows rb*128 + 32 q4 + lane of each row block of the group
      // (its accumulator at TMEM column 256 ur); columns in groups of eight
      // (one TMEM load each), two groups 32 apart per pass, loads first
#pragma unroll 1
      for (int ur = 0; ur < nr; ++ur) {
      const int rb = rb0 + ur;
      const int i = rb * 128 + 32 * q4 + lane;
      const bool up = i < L && sig * s[i] > 0;
      const float cp = up ? cpl0 : cpl1, cmh = up ? cmh0 : cmh1, cml = up ? cml0 : cml1;
      float* Gi = G + (size_t)(i < L ? i : 0) * L;
#pragma unroll 1
      for (int col0 = 8 * g4; col0 < Lp; col0 += 64) {
        float q[2][8], go[2][8];
#pragma unroll
        for (int u = 0; u < 2; ++u) rf_ld8(Gi + col0 + 32 * u, i < L ? L - col0 - 32 * u : 0, vec, go[u]);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (col0 + 32 * u < Lp) {  // warp-uniform
            tmem_ld8(tc->tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(256 * ur + col0 + 32 * u), q[u]);
          } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) q[u][c] = 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int nv = i < L ? L - col0 - 32 * u : 0;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float Hp = rintf(go[u][c] * cp * sH) * sHi;
            const float y = Hp + q[u][c] * sQ;
            q[u][c] = fmaf(y, cmh, y * cml);
            if (c < nv) drift = fmaxf(drift, fabsf(go[u][c] - q[u][c]));
          }
          rf_st8(Gi + col0 + 32 * u, nv, vec, q[u]);
        }
      }
      }
      tc_fence_before();
      __syncthreads();
    }
    *steps += 1;
    if (emax <= 0x1p-13f) break;
  }
  tc->cphase = ph;
  return rf_block_max(drift, red);
}

// G_dn = 1 - G_up^T for a particle-hole symmetric bath (both L x L FP32 in
// global memory), through per-warp 32 x 33 shared-memory tiles (tile: 16
// warps x 32 x 33 floats) so that reads and writes are both coalesced.  The
// rows of a tile go in batches of 16 with every load of a batch (G_up, and
// the old G_dn for the drift) issued before its stores.
// Returns max |G_dn(old) - G_dn(new)| (block-wide).  All threads call it.
__device__ inline float ph_mirror(const float* Gu, float* Gd, int L, float* tile, float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kDelNT / 32;
  float* tw = tile + warp * 32 * 33;
  const int nt = (L + 31) / 32;
  float drift = 0.f;
  for (int t = warp; t < nt * nt; t += NW) {
    const int ti = t / nt, tj = t - ti * nt;  // source tile rows ti*32.., columns tj*32..
    const int c = tj * 32 + lane;   // source column
    const int cc = ti * 32 + lane;  // destination column = source row
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
      float v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int i = ti * 32 + h + r;
        v[r] = (i < L && c < L) ? Gu[(size_t)i * L + c] : 0.f;
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) tw[(h + r) * 33 + lane] = v[r];
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
      float o[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int i = tj * 32 + h + r;  // destination row = source column
        o[r] = (i < L && cc < L) ? Gd[(size_t)i * L + cc] : 0.f;
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int i = tj * 32 + h + r;
        if (i < L && cc < L) {
          const float gn = (i == cc ? 1.f : 0.f) - tw[lane * 33 + h + r];
          drift = fmaxf(drift, fabsf(o[r] - gn));
          Gd[(size_t)i * L + cc] = gn;
        }
      }
    }
    __syncwarp();
  }
  return rf_block_max(drift, red);
}

}  // namespace hfq
