// Support of the delayed (rank-k) FP32 sweep: shared-memory layout, FP32
// flip ratio, and the two flush engines for G += U W^T:
//   * flush_tcgen05 -- 5th-generation tensor cores.  Per spin the panels are
//     scaled by powers of two (each panel's largest magnitude to [2^14, 2^15))
//     and split into FP16 hi/lo parts in shared memory (K-major, no swizzle,
//     8-row x 16-byte core matrices); per 128 x 128 output tile one thread
//     issues tcgen05.mma kind::f16 (M=128, N<=128, K=16 per instruction, FP32
//     accumulation) for hi*hi + hi*lo + lo*hi into a TMEM accumulator,
//     commits to an mbarrier, and all warps read the tile back with
//     tcgen05.ld and undo the scaling (exact).  With G in HBM the tile goes to
//     a shared-memory buffer and one TMA tensor reduce-add sends it to G (the
//     addition happens in L2; the SM never loads G); with G in shared memory
//     the warps add it in place.  hi and lo carry 11 significant bits each, as
//     TF32 would, so the dropped lo*lo term and the rounding of lo leave a
//     relative error ~2^-21 per product; the scaling keeps every part but
//     those below 2^-29 of the panel's largest entry out of the FP16
//     subnormal range, at the FP16 tensor rate (twice TF32's).
//   * flush_ffma -- FP32 FMA on the CUDA cores (4 x 4 register tiles).
#pragma once
#include <cstdint>

#include "hfq_device.cuh"

namespace hfq {

constexpr int kDelNT = 512;          // threads per CTA (16 warps)
constexpr int kUBlk = 2;             // U blocks of 128 rows staged (and multiplied) together
// TMEM columns per CTA: the flush takes one 128-column accumulator per staged
// U block, the recompute by Newton refinement (hfq_refine.cuh) up to 512
constexpr int kTmemCols = 512;
constexpr int kTileN = 128;          // output tile: 128 rows x 128 columns

struct DelLayout {
  int ldS;      // row pitch of shared-memory G (floats)
  int KP;       // row pitch of the FP32 panels (floats)
  int KS;       // k rounded up to 16 (FP16 MMA K step): K extent of a staged tile
  // head: s (and, when the recompute works in shared memory, its scratch colk
  // and perm, which must survive the workspace overlaying the body; otherwise
  // they live in the idle staging area); body: stage, G, panels, diag
  // (byte offsets in dynamic shared memory, below 227 KiB: 32 bits, which
  // keeps the kernel's copy of the layout at one register per field)
  uint32_t off_colk, off_perm, off_s, off_body;
  int ub;       // U blocks staged (and multiplied) together by the flush
  uint32_t off_stage, off_G, off_U, off_W, off_diag, off_gtile;
  size_t bytes;
  uint32_t off_gjb;  // the recompute's panel scratch (workspace in HBM), overlaying all but G
  uint32_t off_rf;   // the Newton refinement's staging (1024-aligned; overlays the whole body,
                     // a resident G included: G is kept in HBM while it runs)
};

// product buffers of the TMA reduce flush: two halves of a tile, 64 rows x
// 128 floats each, used in turn
constexpr size_t kGTileBytes = (size_t)kTileN * kTileN * 4;

__host__ __device__ inline size_t del_align(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Offset (floats) from a panel's spin-up block to its spin-down block: L KP
// rounded up to 16 (mod 32) floats.  The 8 lanes of a 16-byte access in the
// append read rows i..i+3 of both spins; with KP/4 odd those rows fill four
// of the eight 16-byte bank groups and the half-bank shift of the other spin
// fills the remaining four, so the access is conflict-free.
__host__ __device__ inline int del_spin_stride(int L, int KP) {
  return L * KP + ((16 - (L * KP) % 32) + 32) % 32;
}

// Floats of one panel (U or W): both spins at the padded stride, or, when the
// sweep keeps G_up only (ns = 1), one spin plus 16 floats (the G_up-only sweep
// starts W 16 floats into its region, off U's bank alignment).  A multiple of
// 4 (KP is), so the panels are zeroed by 16-byte stores.
__host__ __device__ inline int del_panel_floats(int L, int KP, int ns) {
  return ns == 1 ? L * KP + 16 : del_spin_stride(L, KP) + L * KP;
}

// stage: W hi, W lo (one block of 128 rows), then U hi, U lo for ub U blocks
// (at most kUBlk and at most as many as L has), FP16 in core-matrix layout,
// 128 x KS each
__host__ __device__ inline int del_ublocks(int L, int ub) {
  const int lb = (L + 127) / 128;
  const int u = ub < kUBlk ? ub : kUBlk;
  return lb < u ? lb : u;
}
__host__ __device__ inline size_t del_stage_bytes(int K, int L, int ub) {
  const int KS = (K + 15) / 16 * 16;
  return (size_t)(2 + 2 * del_ublocks(L, ub)) * kTileN * KS * 2;
}

__host__ __device__ inline size_t rf_smem_need(int L) {
  // the Newton refinement (hfq_refine.cuh): the larger of its two stage buffers of the residual product (A and H'
  // slices) and GEMM2's (H' and E^T hi / lo parts)
  const size_t g2 = (size_t)2 * 128 * kRf2KC * 2 + (size_t)2 * ((L + 15) / 16 * 16) * kRf2KC * 2;
  return g2 > (size_t)kRfSmem ? g2 : (size_t)kRfSmem;
}

// ns: spins the sweep keeps (2, or 1 for the G_up-only sweep): the panels and
// the measurement's partial sums are sized for them; a resident G keeps both.
__host__ __device__ inline DelLayout del_layout(int L, int K, bool resident, bool gj_smem,
                                                bool gtile = false, int ub = kUBlk, bool refine = false,
                                                int ns = 2) {
  DelLayout d;
  d.ldS = L | 1;
  d.KP = K + 4;  // 16-byte rows; (K+4) mod 32 spreads 8 rows of a 16-byte load over all banks
  d.KS = (K + 15) / 16 * 16;
  d.ub = del_ublocks(L, ub);
  size_t o = 0;  // offsets are computed in size_t and stored in 32 bits
  if (gj_smem) {
    d.off_colk = o;
    o += del_align((size_t)L * 8, 128);
    d.off_perm = o;
    o += del_align((size_t)L * 4, 128);
  }
  d.off_s = o;
  o += del_align((size_t)L, 128);
  o = del_align(o, 1024);
  d.off_body = o;
  d.off_stage = o;
  if (!gj_smem) {  // the recompute's scratch in the (then idle) staging area
    d.off_colk = o;
    d.off_perm = o + del_align((size_t)L * 8, 128);
  }
  // the staging area doubles as the measurement's per-warp partial sums and
  // holds the recompute's scratch when that is not in the head
  const size_t part = (size_t)ns * (kDelNT / 32) * L * 4;
  const size_t scratch = del_align((size_t)L * 8, 128) + del_align((size_t)L * 4, 128);
  size_t st = del_stage_bytes(K, L, ub);
  if (part > st) st = part;
  if (scratch > st) st = scratch;
  o += del_align(st, 1024);
  d.off_G = o;
  if (resident) o += del_align(2 * (size_t)L * d.ldS * 4, 128);
  d.off_U = o;
  o += del_align((size_t)del_panel_floats(L, d.KP, ns) * 4, 128);
  d.off_W = o;
  o += del_align((size_t)del_panel_floats(L, d.KP, ns) * 4, 128);
  d.off_diag = o;
  o += del_align(2 * (size_t)L * 4, 128);
  d.off_gtile = 0;
  if (gtile) {
    o = del_align(o, 1024);
    d.off_gtile = o;
    o += kGTileBytes;
  }
  if (gj_smem && d.off_body + gj_smem_bytes(L) > o) o = d.off_body + gj_smem_bytes(L);
  // the blocked recompute's scratch: after colk and perm, or after G when
  // G is resident (with the workspace in shared memory it is not used)
  d.off_gjb = resident ? del_align(d.off_U, 128) : del_align(d.off_body + scratch, 128);
  if (!gj_smem && d.off_gjb + gj_blocked_bytes(L) > o) o = d.off_gjb + gj_blocked_bytes(L);
  d.off_rf = d.off_body;
  if (refine && d.off_rf + rf_smem_need(L) > o) o = d.off_rf + rf_smem_need(L);
  d.bytes = o;
  return d;
}

__device__ __forceinline__ bool del_decide(float d0, float d1, float gu, float gd, int sl, float u,
                                           int rule, bool* bad) {
  const float du = sl > 0 ? d0 : d1;
  const float dd = sl > 0 ? d1 : d0;
  const float Ru = __fadd_rn(1.f, __fmul_rn(__fsub_rn(1.f, gu), du));
  const float Rd = __fadd_rn(1.f, __fmul_rn(__fsub_rn(1.f, gd), dd));
  const float R = __fmul_rn(Ru, Rd);
  *bad = !(R > 0.f) || !isfinite(R);
  return rule == 0 ? (u < R) : (__fmul_rn(u, __fadd_rn(1.f, R)) < R);
}

__device__ __forceinline__ void del_factors(float d0, float d1, float gu, float gd, int sl, float* fu,
                                            float* fd) {
  const float du = sl > 0 ? d0 : d1;
  const float dd = sl > 0 ? d1 : d0;
  const float Ru = __fadd_rn(1.f, __fmul_rn(__fsub_rn(1.f, gu), du));
  const float Rd = __fadd_rn(1.f, __fmul_rn(__fsub_rn(1.f, gd), dd));
  *fu = du / Ru;
  *fd = dd / Rd;
}

// ---------------------------------------------------------------------------
// FP32 FMA flush: G^sigma[i][c] += sum_{m<j} U^sigma[i][m] W^sigma[c][m]
// ---------------------------------------------------------------------------
// NSP = 1: spin up only (G_dn = 1 - G_up^T is not kept during the sweep).
template <int NSP = 2>
__device__ inline void flush_ffma(float* Gu, float* Gd, int ld, const float* Pu, const float* Pw,
                                  int KP, int L, int j) {
  const int T4 = (L + 3) / 4;
  const int tiles = T4 * T4;
  for (int sp = 0; sp < NSP; ++sp) {
    float* G = sp ? Gd : Gu;
    const float* U = Pu + (size_t)sp * del_spin_stride(L, KP);
    const float* W = Pw + (size_t)sp * del_spin_stride(L, KP);
    for (int t = threadIdx.x; t < tiles; t += kDelNT) {
      const int i0 = (t / T4) * 4, c0 = (t % T4) * 4;
      float acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
      for (int m = 0; m < j; ++m) {
        float av[4], bv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) av[r] = (i0 + r < L) ? U[(size_t)(i0 + r) * KP + m] : 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = (c0 + c < L) ? W[(size_t)(c0 + c) * KP + m] : 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = __fmaf_rn(av[r], bv[c], acc[r][c]);
      }
      float gv[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          gv[r][c] = (i0 + r < L && c0 + c < L) ? G[(size_t)(i0 + r) * ld + c0 + c] : 0.f;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (i0 + r < L && c0 + c < L) G[(size_t)(i0 + r) * ld + c0 + c] = gv[r][c] + acc[r][c];
    }
  }
}

// ---------------------------------------------------------------------------
// tcgen05 (5th-gen tensor core) helpers, inline PTX for sm_100a / sm_103a
// ---------------------------------------------------------------------------
struct TcState {
  uint32_t tmem;       // TMEM base address of this CTA's allocation
  uint32_t mbar;       // shared address of the MMA completion mbarrier
  uint32_t phase;      // parity of the next MMA completion
  int failed;          // a wait gave up: the tensor path is not used again
  uint32_t cbar;       // shared address of the refinement's mbarriers: bulk copy into
                       // stage buffer 0, 1, then MMA completion of buffer 0, 1 (8 bytes apart)
  uint32_t cphase;     // their parities (bit b of the barrier at cbar + 8 b)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Two FP32 values -> FP16 (round to nearest even) packed, x0 in the low half
// (the lower address), and the two halves back to FP32
__device__ __forceinline__ uint32_t f32x2_to_f16x2(float x0, float x1) {
  uint32_t h;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(x1), "f"(x0));
  return h;
}
__device__ __forceinline__ float f16_lo_to_f32(uint32_t h) {
  float x;
  asm("cvt.f32.f16 %0, %1;" : "=f"(x) : "h"((unsigned short)(h & 0xffffu)));
  return x;
}
__device__ __forceinline__ float f16_hi_to_f32(uint32_t h) {
  float x;
  asm("cvt.f32.f16 %0, %1;" : "=f"(x) : "h"((unsigned short)(h >> 16)));
  return x;
}

// K-major, no-swizzle canonical layout: element (r, m) of a rows x KS FP16
// tile lives at (r/8)*SBO + (m/8)*LBO + (r%8)*16 + (m%8)*2 bytes, with the
// 8-row x 16-byte core matrices contiguous along K (LBO = 128 B) and the
// 8-row groups SBO = (KS/8)*128 B apart.
__device__ __forceinline__ uint32_t core_offset(int r, int m, int KS) {
  return (uint32_t)((r >> 3) * (KS / 8) * 128 + (m >> 3) * 128 + (r & 7) * 16 + (m & 7) * 2);
}

__device__ __forceinline__ uint64_t make_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for sm_100-class parts
  // base offset 0, absolute LBO mode off, layout type 0 = no swizzle
  return d;
}

// Instruction descriptor: kind::f16, D = F32, A = B = F16, both K-major, M = 128.
__device__ __forceinline__ uint32_t make_idesc_f16(int N) {
  uint32_t d = 0;
  d |= 1u << 4;                       // D format F32
  // A and B format F16 (0 in bits 7-9 and 10-12), no negation, K-major
  d |= (uint32_t)(N >> 3) << 17;      // N / 8
  d |= (uint32_t)(128 >> 4) << 24;    // M / 16
  return d;
}

__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                           uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// One bounded poll of the mbarrier phase; the thread may be suspended for up
// to ~0.1 ms inside try_wait (hint), which frees issue slots while it waits.
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(mbar), "r"(phase), "r"(100000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the mbarrier phase with a one-second limit; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t phase) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(mbar, phase)) return true;
    if (global_ns() - t0 > 1000000000ull) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 lanes x 32 bit, 16 consecutive columns per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Allocates kTmemCols TMEM columns (warp 0) and initialises the MMA
// completion mbarrier s_mbar[0] and the refinement's four, s_mbar[1..4].
__device__ inline void tc_setup(TcState* tc, uint32_t* s_tmem, unsigned long long* s_mbar,
                                int* status) {
  (void)status;
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int b = 0; b < 5; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(s_mbar + b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tc->tmem = *s_tmem;
  tc->mbar = smem_u32(s_mbar);
  tc->phase = 0;
  tc->failed = 0;
  tc->cbar = smem_u32(s_mbar + 1);
  tc->cphase = 0;
}

__device__ inline void tc_teardown(TcState* tc) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc->tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// TMA tensor reduce-add (shared -> global, FP32 add performed in L2) through
// a 4-D tensor map over the G matrices of all chains of a grid, coordinates
// {column, row, spin, chain}; completion tracked by bulk async-groups.
// Boxes that reach past Lambda in a coordinate are clipped by the TMA unit.
__device__ __forceinline__ void tma_reduce_add_4d(const void* tmap, uint32_t src_smem, int x, int y,
                                                  int z, int w) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.4d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3, %4}], "
      "[%5];" ::"l"(tmap),
      "r"(x), "r"(y), "r"(z), "r"(w), "r"(src_smem)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Writes the tiles of one flush group in one pass: W block rows
// [nb, nb + nN) when doW (to W hi / lo at stage, stage + tile_bytes) and U
// blocks mg .. mg + ub - 1 when doU (to stage + (2 + 2u) tile_bytes), each
// row of a panel (pitch KP floats, j valid columns) times the power of two
// sw or su, as FP16 hi and lo parts (hi = fp16(x s), lo = fp16(x s - hi),
// both rounded to nearest) in 128-row core-matrix tiles of KS columns; rows
// and columns outside the valid range are zero.
__device__ __forceinline__ void stage_group(const float* W, int nb, int nN, bool doW, const float* U, int mg,
                                            int ub, bool doU, int L, int KP, int j, int KS, float sw, float su,
                                            unsigned char* stage, size_t tile_bytes) {
  const int cpt = kTileN * (KS / 8);  // 16-byte chunks per tile
  const int nt = (doW ? 1 : 0) + (doU ? ub : 0);
  for (int c = threadIdx.x; c < nt * cpt; c += kDelNT) {
    const int t = c / cpt, cc = c - t * cpt;
    const bool isW = doW && t == 0;
    const int u = t - (doW ? 1 : 0);
    const float* P = isW ? W : U;
    const int row0 = isW ? nb : (mg + u) * kTileN;
    const int nrows = isW ? nN : min(kTileN, L - row0);
    const float sc = isW ? sw : su;
    unsigned char* hi = isW ? stage : stage + (size_t)(2 + 2 * u) * tile_bytes;
    // cc = ((row group * KS/8) + k chunk) * 8 + row within group: eight lanes
    // write one 128-byte core matrix, conflict-free
    const int r8 = cc & 7, rest = cc >> 3;
    const int kc = rest % (KS / 8), grp = rest / (KS / 8);
    const int r = grp * 8 + r8, m0 = kc * 8;
    // two 16-byte loads per chunk (rows are 16-byte aligned: KP % 4 == 0);
    // the second only below j <= KP - 4, so never past the row
    float4 xa = make_float4(0.f, 0.f, 0.f, 0.f), xb = xa;
    if (r < nrows && m0 < j) xa = *reinterpret_cast<const float4*>(P + (row0 + r) * KP + m0);
    if (r < nrows && m0 + 4 < j) xb = *reinterpret_cast<const float4*>(P + (row0 + r) * KP + m0 + 4);
    const float xs[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float x0 = (m0 + 2 * q < j) ? xs[2 * q] * sc : 0.f;
      const float x1 = (m0 + 2 * q + 1 < j) ? xs[2 * q + 1] * sc : 0.f;
      h[q] = f32x2_to_f16x2(x0, x1);
      l[q] = f32x2_to_f16x2(x0 - f16_lo_to_f32(h[q]), x1 - f16_hi_to_f32(h[q]));
    }
    const uint32_t off = core_offset(r, m0, KS);
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(hi + tile_bytes + off) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// Per panel (U up, W up, U down, W down) the exponent a of the scale 2^a
// that brings its largest magnitude over the j valid columns (zeros beyond)
// into [2^14, 2^15): a = 141 - E for the largest biased exponent E (0 for an
// all-zero panel), from the byte-wise maxima each thread kept while
// appending: exq holds the biased exponents of its largest |u| (byte 0) and
// |w| (byte 1) for its spin sp (thread parity).  The four bytes of a warp
// travel in one word of wred (kDelNT / 32 words, one barrier).  kMirror:
// only spin up's panels, whose |u| exponents the even threads keep (byte 0)
// and |w| exponents the odd ones (byte 1).
template <bool kMirror = false>
__device__ __forceinline__ void panel_scales(uint32_t exq, uint32_t* wred, int* ea) {
  uint32_t v = (!kMirror && (threadIdx.x & 1)) ? (exq << 16) : exq;  // bytes: U up, W up, U down, W down
#pragma unroll
  for (int o = 16; o; o >>= 1) v = __vmaxu4(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t E = 0u;
#pragma unroll
  for (int w = 0; w < kDelNT / 32; ++w) E = __vmaxu4(E, wred[w]);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const uint32_t e = (E >> (8 * a)) & 255u;
    ea[a] = e == 0u ? 0 : min(141 - (int)e, 127);
  }
}

// Thread 0: issues the 3-pass split-FP16 product of one 128 x N16 tile over
// KS into the TMEM accumulator at column col (the caller has fenced and
// synchronised the staged operands).
__device__ __forceinline__ void tc_issue_product(const TcState* tc, uint32_t col, const unsigned char* Ahi,
                                                 const unsigned char* Alo, const unsigned char* Bhi,
                                                 const unsigned char* Blo, int KS, int N16) {
  const uint32_t sbo = (uint32_t)(KS / 8) * 128u, lbo = 128u;
  const uint32_t idesc = make_idesc_f16(N16);
  const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo);
  const uint32_t b_hi = smem_u32(Bhi), b_lo = smem_u32(Blo);
  const uint32_t d = tc->tmem + col;
  int acc = 0;
  for (int kb = 0; kb < KS / 16; ++kb) {
    const uint32_t koff = (uint32_t)kb * 256u;  // two core matrices of 8 FP16 along K
    tc_mma_f16(d, make_smem_desc(a_hi + koff, lbo, sbo), make_smem_desc(b_hi + koff, lbo, sbo), idesc, acc);
    acc = 1;
    tc_mma_f16(d, make_smem_desc(a_hi + koff, lbo, sbo), make_smem_desc(b_lo + koff, lbo, sbo), idesc, 1);
    tc_mma_f16(d, make_smem_desc(a_lo + koff, lbo, sbo), make_smem_desc(b_hi + koff, lbo, sbo), idesc, 1);
  }
}

// All threads: thread 0 commits the products it issued, warp 0 waits for
// their completion (the other warps wait at the barrier, which costs no issue
// slots).  Returns false, in every thread, if the wait gave up.
__device__ inline bool tc_commit_wait(TcState* tc) {
  if (threadIdx.x == 0) tc_commit(tc->mbar);
  bool ok_here = true;
  if (threadIdx.x < 32) ok_here = mbar_wait_bounded(tc->mbar, tc->phase);
  const bool ok = !__syncthreads_or(ok_here ? 0 : 1);
  tc->phase ^= 1u;
  tc_fence_after();
  return ok;
}

// G^sigma += U^sigma W^sigma^T via tcgen05, one 128 x 128 output tile at a
// time.  The product is formed transposed, D = W U^T (A = 128 rows of W, B =
// up to 128 rows of U), so TMEM lane m holds column nb+m of the G tile and
// the 32 threads of a warp touch 32 consecutive columns of one G row per
// access (coalesced in HBM, conflict-free in shared memory).
// kTR (G in HBM): the warps write the product tile, 64 rows at a time, to
// one of two shared-memory buffers (dtile) and thread 0 hands each half to a
// TMA tensor reduce-add (tensor map tmap, coordinates {nb, row, spin, chain});
// G is never loaded by the SM, a reduce streams while the next half is
// written, and the flush returns once every reduce is complete and visible.  Otherwise (G in shared
// memory, or the fallback for G in HBM) every thread adds its 64 entries of
// the tile in place.
template <bool kTR, int NSP = 2>
__device__ __forceinline__ void flush_tiles(TcState* tc, float* Gu, float* Gd, int ld, const float* Pu,
                                            const float* Pw, int KP, int L, int j, unsigned char* stage,
                                            const DelLayout& lay, int* status, uint32_t* wred,
                                            uint32_t exq, float* dtile, const void* tmap, int chain) {
  const int KS = (j + 15) / 16 * 16;
  const size_t tile_bytes = (size_t)kTileN * lay.KS * 2;
  const int LB = (L + kTileN - 1) / kTileN;  // blocks of 128 rows / columns
  const int UB = lay.ub;                     // U blocks staged together
  unsigned char* Whi = stage;
  unsigned char* Wlo = stage + tile_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // TMEM lanes 32*quarter.. (the lanes a warp may read); the kDelNT/128 warps of a
  // quarter split the tile's columns (G rows) into groups, group index `half`
  const int quarter = warp & 3, half = warp >> 2;
  const int m = 32 * quarter + lane;               // G column nb + m of a tile
  int nhalf = 0;                                   // half tiles handed to the TMA unit
  int ea[4];
  panel_scales<NSP == 1>(exq, wred, ea);
  for (int sp = 0; sp < NSP; ++sp) {
    float* G = sp ? Gd : Gu;
    const float* U = Pu + (size_t)sp * del_spin_stride(L, KP);
    const float* W = Pw + (size_t)sp * del_spin_stride(L, KP);
    const float su = ldexpf(1.f, sp ? ea[2] : ea[0]), sw = ldexpf(1.f, sp ? ea[3] : ea[1]);
    // the product comes back scaled by su sw: undone exactly in the epilogue
    const float ds = ldexpf(1.f, -(sp ? ea[2] + ea[3] : ea[0] + ea[1]));
    for (int nbi = 0; nbi < LB; ++nbi) {  // block of G columns = rows of W
      const int nb = nbi * kTileN, nN = min(kTileN, L - nb);
      for (int mg = 0; mg < LB; mg += UB) {  // group of U blocks = blocks of G rows
        const int ub = min(UB, LB - mg);
        // W's block once per block, all of U once per spin when it fits
        stage_group(W, nb, nN, mg == 0, U, mg, ub, !(UB == LB && nbi > 0), L, KP, j, KS, sw, su, stage,
                    tile_bytes);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
          tc_fence_after();
          for (int u = 0; u < ub; ++u) {
            const int nM = min(kTileN, L - (mg + u) * kTileN);
            tc_issue_product(tc, (uint32_t)(u * kTileN), Whi, Wlo, stage + (2 + 2 * u) * tile_bytes,
                             stage + (3 + 2 * u) * tile_bytes, KS, (nM + 15) / 16 * 16);
          }
        }
        if (!tc_commit_wait(tc)) {
          // a completion wait gave up: flag the context (the host returns
          // HFQMC_ETIMEOUT) and use the CUDA cores for every later flush
          if (threadIdx.x == 0) {
            atomicOr(status, kStatusTimeout);
            if constexpr (kTR) bulk_wait0();
          }
          tc->failed = 1;
          __syncthreads();
          return;
        }
        for (int u = 0; u < ub; ++u) {
          const int mb = (mg + u) * kTileN, nM = min(kTileN, L - mb);
          const int N16 = (nM + 15) / 16 * 16;
          if constexpr (kTR) {
            // two 64-row halves, each through its own buffer and TMA reduce;
            // a buffer is rewritten once the reduce issued two halves before
            // has read it, so one reduce streams while the next half is written
            for (int r0 = 0; r0 < N16; r0 += kTileN / 2) {
              float* dbuf = dtile + (size_t)(nhalf & 1) * (kTileN / 2) * kTileN;
              ++nhalf;
              if (threadIdx.x == 0) bulk_wait_read1();
              __syncthreads();
#pragma unroll
              for (int c = 0; c < 4 / (kDelNT / 128); ++c) {
                const int cb = r0 + (64 / (kDelNT / 128)) * half + 16 * c;
                if (cb < N16) {  // warp-uniform
                  float v[16];
                  tmem_ld16(tc->tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(u * kTileN + cb), v);
                  // rows >= nM and columns >= nN lie outside G and are clipped
                  float* dt = dbuf + (cb - r0) * kTileN + m;
#pragma unroll
                  for (int q = 0; q < 16; ++q) dt[q * kTileN] = v[q] * ds;
                }
              }
              tc_fence_before();
              fence_async_smem();  // the half's generic stores, seen by the TMA unit
              __syncthreads();
              if (threadIdx.x == 0) {
                tma_reduce_add_4d(tmap, smem_u32(dbuf), nb, mb + r0, sp, chain);
                bulk_commit();
              }
            }
          } else {
#pragma unroll
            for (int c = 0; c < 8 / (kDelNT / 128); ++c) {
              const int cb = (128 / (kDelNT / 128)) * half + 16 * c;
              if (cb < N16) {  // warp-uniform: tcgen05.ld is issued by whole warps
                float v[16];
                tmem_ld16(tc->tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(u * kTileN + cb), v);
                if (m < nN) {
                  float* g = G + (size_t)(mb + cb) * ld + nb + m;
#pragma unroll
                  for (int q = 0; q < 16; ++q)
                    if (cb + q < nM) g[(size_t)q * ld] += v[q] * ds;
                }
              }
            }
            tc_fence_before();
            __syncthreads();
          }
        }
      }
    }
  }
  if constexpr (kTR) {
    // every reduce complete and visible before G is read again
    if (threadIdx.x == 0) {
      bulk_wait0();
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();
  }
}

template <int NSP = 2>
__device__ inline void flush_tcgen05(TcState* tc, float* Gu, float* Gd, int ld, const float* Pu,
                                     const float* Pw, int KP, int L, int j, unsigned char* stage,
                                     const DelLayout& lay, int* status, uint32_t* wred, uint32_t exq,
                                     float* dtile = nullptr, const void* tmap = nullptr, int chain = 0) {
  if (tc->failed) {
    flush_ffma<NSP>(Gu, Gd, ld, Pu, Pw, KP, L, j);
    return;
  }
  if (dtile)
    flush_tiles<true, NSP>(tc, Gu, Gd, ld, Pu, Pw, KP, L, j, stage, lay, status, wred, exq, dtile, tmap, chain);
  else
    flush_tiles<false, NSP>(tc, Gu, Gd, ld, Pu, Pw, KP, L, j, stage, lay, status, wred, exq, nullptr, nullptr, 0);
}

// One pass of both spins with RB rows per warp in flight and CPL columns per
// lane (L <= 32 CPL): the RB x CPL loads of a batch are issued before any of
// them is used; the partial sums are then updated row after row (entries of
// one row go to distinct k, entries of different rows may share one), so the
// order of the additions is that of the plain row walk.
// G is read with plain (coherent) loads: the same kernel writes it through
// the flush's TMA reduce-adds, so the non-coherent read-only path that
// const __restrict__ would allow is not valid here.
template <int RB, int CPL, int NSP = 2>
__device__ __forceinline__ void measure_rows_batched(const float* Gu, const float* Gd, int ld, int L,
                                                     float* part) {
  constexpr int NW = kDelNT / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int sp = 0; sp < NSP; ++sp) {
    const float* G = sp ? Gd : Gu;
    float* pw = part + (size_t)(sp * NW + warp) * L;
    for (int r0 = warp; r0 < L; r0 += NW * RB) {
      float v[RB][CPL];
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const int r = r0 + NW * b;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int l = lane + 32 * c;
          v[b][c] = (r < L && l < L) ? G[(size_t)r * ld + l] : 0.f;
        }
      }
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const int r = r0 + NW * b;
        if (r < L) {  // warp-uniform
          float acc[CPL];
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int l = lane + 32 * c;
            acc[c] = l < L ? pw[r >= l ? r - l : r - l + L] : 0.f;
          }
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int l = lane + 32 * c;
            if (l < L) pw[r >= l ? r - l : r - l + L] = r >= l ? acc[c] + v[b][c] : acc[c] - v[b][c];
          }
        }
        __syncwarp();
      }
    }
  }
}

// The same sums with the bins in registers (L <= 256, L and ld multiples of
// 4, G 16-byte aligned).  A warp walks a contiguous range of rows of one spin;
// lane t holds the slots j = 128 c + 4 t + q (c < 2, q < 4) and loads
// G[r][j .. j + 3] with one 16-byte load per c.  After row r slot j holds the
// running sum of bin (r - j) mod L; from one row to the next every bin moves
// from slot j to slot j + 1 (from L - 1 to 0), so a lane's four slots shift
// by one register and the first takes the last of the lane below (lane 0:
// slot 127 of lane 31, or slot L - 1) by shuffles, and no bin is read or
// written in shared memory until the warp's range ends: one store per bin
// into the warp's partial sums (part, pitch L).
template <int RB, int NSP = 2>
__device__ __forceinline__ void measure_rows_reg(const float* Gu, const float* Gd, int ld, int L,
                                                 float* part) {
  constexpr int NW = kDelNT / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool two = L > 128;                    // slots of the second block of 128 columns in use
  const int lastc = (L - 1) >> 7, lastl = ((L - 1) & 127) >> 2;  // slot L - 1 (its q is 3)
  const int below = (lane + 31) & 31;
  for (int sp = 0; sp < NSP; ++sp) {
    const float* G = sp ? Gd : Gu;
    const int rb = (warp * L) / NW, re = ((warp + 1) * L) / NW;
    float acc[2][4];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[c][q] = 0.f;
    for (int r0 = rb; r0 < re; r0 += RB) {
      float4 v[RB][2];
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const int r = r0 + b;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int j = 128 * c + 4 * lane;
          v[b][c] = (r < re && j < L) ? *reinterpret_cast<const float4*>(G + (size_t)r * ld + j)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const int r = r0 + b;
        if (r >= re) break;  // warp-uniform
        if (r > rb) {
          // every bin one slot up
          const float t0 = __shfl_sync(0xffffffffu, acc[0][3], below);
          const float t1 = __shfl_sync(0xffffffffu, acc[1][3], below);
          const float t2 = __shfl_sync(0xffffffffu, lastc ? acc[1][3] : acc[0][3], lastl);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            acc[c][3] = acc[c][2];
            acc[c][2] = acc[c][1];
            acc[c][1] = acc[c][0];
          }
          acc[0][0] = lane ? t0 : t2;
          acc[1][0] = lane ? t1 : t0;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (c == 1 && !two) break;  // uniform
          const int j = 128 * c + 4 * lane;
          const float x[4] = {v[b][c].x, v[b][c].y, v[b][c].z, v[b][c].w};
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[c][q] += (r >= j + q) ? x[q] : -x[q];
        }
      }
    }
    // slot j holds bin (re - 1 - j) mod L of this warp's rows
    float* pw = part + (size_t)(sp * NW + warp) * L;
    if (re > rb) {
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 128 * c + 4 * lane + q;
          if (j < L) {
            int k = re - 1 - j;
            k += k < 0 ? L : 0;
            pw[k] = acc[c][q];
          }
        }
    }
  }
}

// Measurement g^sigma(tau_k) = (1/L) sum_l sgn G^sigma_{(l+k) mod L, l} for G
// in HBM, walked row by row: element (r, l) belongs to k = r - l (sign +) or
// r - l + L (sign -, antiperiodic wrap).  Each warp takes rows, lanes take
// columns (coalesced), and every warp's sums end in its own shared-memory row
// of FP32 partial sums; the warps' partials are added in a fixed order.
// Three walks, by Lambda and alignment:
//  * measure_rows_reg (L <= 256, L and ld multiples of 4, G 16-byte aligned):
//    a contiguous range of rows per warp with the bins in registers, one
//    store per bin at the end;
//  * measure_rows_batched (other L <= 512): batched loads, a shared-memory
//    read-modify-write of the warp's partial row per element;
//  * the plain row walk beyond.
// Everything stays on the FP32 pipe: the caller folds the per-sweep totals
// into FP64 accumulators.
// part: NSP * NW * L floats of shared scratch; out[k], out[L+k] receive the
// sums (not yet divided by L).  NSP = 1: spin up only (out[k]).
template <int NSP = 2>
__device__ inline void measure_rows(const float* Gu, const float* Gd, int ld, int L, float* part,
                                    float* out) {
  constexpr int NW = kDelNT / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < NSP * NW * L; e += kDelNT) part[e] = 0.f;
  __syncthreads();
  if (L <= 256 && L % 4 == 0 && ld % 4 == 0 &&
      ((reinterpret_cast<uintptr_t>(Gu) | reinterpret_cast<uintptr_t>(Gd)) & 15) == 0) {
    measure_rows_reg<4, NSP>(Gu, Gd, ld, L, part);
  } else if (L <= 256) {
    measure_rows_batched<4, 8, NSP>(Gu, Gd, ld, L, part);
  } else if (L <= 512) {
    measure_rows_batched<2, 16, NSP>(Gu, Gd, ld, L, part);
  } else {
    for (int sp = 0; sp < NSP; ++sp) {
      const float* G = sp ? Gd : Gu;
      float* pw = part + (size_t)(sp * NW + warp) * L;
      for (int r = warp; r < L; r += NW) {
        const float* gr = G + (size_t)r * ld;
        for (int l = lane; l < L; l += 32) {
          const float v = gr[l];
          if (r >= l)
            pw[r - l] += v;
          else
            pw[r - l + L] -= v;
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NSP * L; e += kDelNT) {
    const int sp = e >= L, k = e - sp * L;
    float acc = 0.f;
    for (int w = 0; w < NW; ++w) acc += part[(size_t)(sp * NW + w) * L + k];
    out[e] = acc;
  }
  __syncthreads();
}

// The same sums for G in shared memory (odd row pitch ld): thread k walks the
// wrapped diagonal k of both spins in registers; for a fixed l the threads
// of a warp read rows l+k at stride ld, i.e. 32 different banks.
template <int NSP = 2>
__device__ inline void measure_diagonals(const float* Gu, const float* Gd, int ld, int L, float* out) {
  for (int k = threadIdx.x; k < L; k += kDelNT) {
    float su = 0.f, sd = 0.f;
    int l = 0;
    for (; l + k < L; ++l) {
      const int o = (l + k) * ld + l;
      su += Gu[o];
      if (NSP == 2) sd += Gd[o];
    }
    for (; l < L; ++l) {
      const int o = (l + k - L) * ld + l;
      su -= Gu[o];
      if (NSP == 2) sd -= Gd[o];
    }
    out[k] = su;
    if (NSP == 2) out[L + k] = sd;
  }
  __syncthreads();
}

__device__ __forceinline__ float block_sum_f(float v, float* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float r = 0.f;
#pragma unroll
  for (int w = 0; w < kDelNT / 32; ++w) r += red[w];
  return r;
}

}  // namespace hfq
