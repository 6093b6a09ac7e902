// Delayed (rank-k) FP32 Hirsch-Fye sweep: one CTA per Markov chain,
// persistent over the longest-Lambda-first work queue.
//
// The accepted flips of a chain are not applied one by one.  After j accepted
// flips since the last flush the current Green matrix is
//     G_cur = G + U W^T,   U, W: L x j panels (per spin),
// and an accepted flip at slice l appends
//     u = G_cur[:, l] - e_l,           w = (Delta / R) G_cur[l, :],
// whose entries cost O(j) each (the base column / row entry plus a length-j
// dot product with the panels).  Every k accepted flips the panels are
// flushed, G += U W^T -- a dense L x L x k contraction per spin (tcgen05
// tensor cores with scaled split FP16, or FP32 FMA).  In exact arithmetic this is
// the Hirsch-Fye rank-1 update applied k times; only the rounding differs.
// The panels are also flushed before every measurement and every FP64
// recompute (every n_wrap accepted flips).
//
// Work split (16 warps): thread t owns spin (t & 1) of rows r = t/2 + 256 q.  For its
// rows it appends the panel entries, keeps the current diagonal G_cur[r][r]
// in registers, swaps it with its partner thread (the other spin) by one
// shuffle, and right away evaluates slice r as the next proposal (flip ratio
// from the new diagonals, Philox uniform drawn at the start of the sweep).
// Rejections change nothing, so the next accepted slice is the lowest r > l
// that accepts: a warp ballot and a shared-memory atomicMin find it, and one
// barrier per accepted flip publishes it with its flip factors.
#include "hfq_delayed.cuh"
#include "hfq_device.cuh"
#include "hfq_gj.cuh"
#include "hfq_launch.h"
#include "hfq_refine.cuh"

namespace hfq {

static_assert(kTileN == kDelayedTile, "tensor-map box and flush tile must agree");

constexpr int kRowsPerThread = 2;  // rows t/2 + 256 q, q < 2: L <= 512
constexpr int kRowStride = kDelNT / 2;
constexpr int kNoSlice = 0x7fffffff;

// kRecord: every accepted flip also sets its bit in the chain's decision
// trace (a.trace_mode == kTraceRecord), for replay by an FP64 run.
// kRefine: the recompute tries the Newton refinement (grids with a
// RefineConst) before Gauss-Jordan; without it the kernel carries only the
// Gauss-Jordan recompute (the refinement's code costs the accept loop some
// registers, so contexts that never refine launch the variant without it).
// kMirror (every grid's bath particle-hole symmetric, so G_dn = 1 - G_up^T
// for every field): the sweep keeps G_up only.  A thread pair owns a row of
// G_up: the even thread appends its column entry u_i, the odd one its row
// entry w_i, and they swap them by one shuffle; G_dn's diagonal is 1 minus
// G_up's, its measured sums follow from G_up's (diagonal L - k for k > 0),
// and the chain's G_dn is written as 1 - G_up^T when the chain ends.
template <bool kRecord, bool kRefine, bool kMirror = false>
__global__ void __launch_bounds__(kDelNT, 1) k_sweep_delayed(SweepArgs a) {
  constexpr int NT = kDelNT;
  constexpr int NW = NT / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[NW];
  __shared__ int redi[NW];
  __shared__ double s_inv;
  __shared__ int s_piv, s_item;
  __shared__ int s_next[3];  // next accepted slice, triple-buffered (see take_next)
  __shared__ int s_bad;
  __shared__ uint32_t s_tmem_base;
  __shared__ __align__(8) unsigned long long s_mbar[5];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool use_tc = a.flush != 2;
  TcState tc;
  if (use_tc) tc_setup(&tc, &s_tmem_base, s_mbar, a.status);

  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.queue_head, 1);
    __syncthreads();
    const int q = s_item;
    __syncthreads();
    if (q >= a.n_items) break;
    const ItemPtrs ip = a.items[a.order[q]];
    const GridConst gc = a.grids[ip.grid];
    const int L = gc.L, K = gc.k;
    const bool resident = gc.resident != 0;
    const DelLayout lay =
        del_layout(L, K, resident, gc.gj_smem != 0, gc.gtile != 0, gc.ub, gc.rc != nullptr, kMirror ? 1 : 2);
    // product tile buffer of the TMA reduce flush (G in HBM, tensor map set)
    float* dtile = gc.gtile ? reinterpret_cast<float*>(smem + lay.off_gtile) : nullptr;

    float* Ggl = reinterpret_cast<float*>(ip.G);
    float* Gu;
    float* Gd;
    int ld;
    if (resident) {
      ld = lay.ldS;
      Gu = reinterpret_cast<float*>(smem + lay.off_G);
      Gd = Gu + (size_t)L * ld;
    } else {
      ld = L;
      Gu = Ggl;
      Gd = Ggl + (size_t)L * L;
    }
    float* Pu = reinterpret_cast<float*>(smem + lay.off_U);  // [2][L][KP] (spin stride padded): U panels
    float* Pw = reinterpret_cast<float*>(smem + lay.off_W);  // [2][L][KP]: W panels
    float* fac = reinterpret_cast<float*>(smem + lay.off_diag);  // [L][2]: flip factors of candidates
    double* colk = reinterpret_cast<double*>(smem + lay.off_colk);
    int* perm = reinterpret_cast<int*>(smem + lay.off_perm);
    int8_t* ss = reinterpret_cast<int8_t*>(smem + lay.off_s);
    unsigned char* stage = smem + lay.off_stage;
    const int KP = lay.KP;
    const int panel_floats4 = del_panel_floats(L, KP, kMirror ? 1 : 2) / 4;  // one panel, the kept spins
    auto zero_panels = [&]() {
      for (int e = tid; e < 2 * panel_floats4; e += NT)
        reinterpret_cast<float4*>(e < panel_floats4 ? Pu : Pw)[e < panel_floats4 ? e : e - panel_floats4] =
            make_float4(0.f, 0.f, 0.f, 0.f);
    };
    const float d0 = gc.deltaf[0], d1 = gc.deltaf[1];
    const int rule = a.accept_rule;

    if (resident) {
      for (int i = warp; i < 2 * L; i += NW)
        for (int jj = lane; jj < L; jj += 32) Gu[(size_t)i * ld + jj] = Ggl[(size_t)i * L + jj];
    }
    for (int l = tid; l < L; l += NT) ss[l] = ip.s[l];
    if (tid < 3) s_next[tid] = kNoSlice;
    if (tid == 0) s_bad = 0;
    __syncthreads();

    // per-thread row state: this spin's current diagonal, field, this sweep's uniform
    const int sp = tid & 1;
    const int row0 = tid >> 1;
    float dg[kRowsPerThread], uv[kRowsPerThread];
    int sv[kRowsPerThread];
    bool lastbad[kRowsPerThread];
    float* Gs = (sp && !kMirror) ? Gd : Gu;
    // G_up only: W starts 16 floats into its region (sized one spin plus 16
    // floats), so row r of U and row r of W lie in different shared-memory
    // banks (see the append)
    float* const Pw1 = kMirror ? Pw + 16 : Pw;
    float* Us = Pu + (size_t)(kMirror ? 0 : sp) * del_spin_stride(L, KP);
    float* Ws = Pw1 + (size_t)(kMirror ? 0 : sp) * del_spin_stride(L, KP);
    auto load_diag = [&]() {
#pragma unroll
      for (int qq = 0; qq < kRowsPerThread; ++qq) {
        if (qq * kRowStride >= L) break;  // uniform: rows beyond the grid
        const int r = row0 + qq * kRowStride;
        if (r < L) dg[qq] = Gs[(size_t)r * ld + r];
      }
    };
#pragma unroll
    for (int qq = 0; qq < kRowsPerThread; ++qq) {
      if (qq * kRowStride >= L) break;  // uniform: rows beyond the grid
      const int r = row0 + qq * kRowStride;
      sv[qq] = r < L ? ss[r] : 1;
      uv[qq] = 0.f;
      lastbad[qq] = false;
      dg[qq] = 0.f;
    }
    load_diag();
    zero_panels();

    const ChainCounters c0 = *ip.cnt;
    long long n_acc = c0.accepted;
    // accepted flips until the next recompute (the cumulative count reaches a
    // multiple of n_wrap); counted down so the hot loop needs no 64-bit modulo
    int until_rec = gc.n_wrap > 0 ? (int)(gc.n_wrap - n_acc % gc.n_wrap) : 0;
    long long n_rec = 0, n_bad = 0;
    int n_fb = 0;  // recomputes the refinement handed to Gauss-Jordan
    unsigned long long hash = c0.hash;
    double drift = c0.drift;
    const long long n_sweeps = a.n_warm + a.n_meas;
    int j = 0;     // pending flips in the panels
    uint32_t exq = 0u;  // biased exponents of this thread's largest appended |u| (byte 0), |w| (byte 1)
    int par = 0;   // s_next buffer of the current round
    __syncthreads();

    // G += U W^T for both spins, then the diagonals are re-read from G.
    auto flush = [&]() {
      if (j == 0) return;
      if (use_tc)
        flush_tcgen05<kMirror ? 1 : 2>(&tc, Gu, Gd, ld, Pu, Pw1, KP, L, j, stage, lay, a.status,
                                       reinterpret_cast<uint32_t*>(red), exq, dtile, gc.tmapG, ip.chain);
      else
        flush_ffma<kMirror ? 1 : 2>(Gu, Gd, ld, Pu, Pw1, KP, L, j);
      __syncthreads();
      load_diag();
      j = 0;
      exq = 0u;
      // the panels restart from zeros, so the dot products may run over whole
      // 16-byte chunks past column j
      zero_panels();
      __syncthreads();
    };

    // Evaluates the owned slices r >= lo as proposals with the current
    // diagonals of both spins (partner threads swap theirs); the lowest
    // accepting slice of the CTA lands in s_next[par] (read after the next
    // barrier), its flip factors in fac[2r], fac[2r+1].
    auto propose = [&](int lo) {
      int cand = kNoSlice;
#pragma unroll
      for (int qq = 0; qq < kRowsPerThread; ++qq) {
        if (qq * kRowStride >= L) break;  // uniform: rows beyond the grid
        const int r = row0 + qq * kRowStride;
        float gu, gd;
        if constexpr (kMirror) {
          gu = dg[qq];  // both threads of the pair hold G_up's diagonal
          gd = 1.f - gu;
        } else {
          const float other = __shfl_xor_sync(0xffffffffu, dg[qq], 1);
          gu = sp ? other : dg[qq];
          gd = sp ? dg[qq] : other;
        }
        bool acc = false, bad = false;
        if (r < L && r >= lo) {
          acc = del_decide(d0, d1, gu, gd, sv[qq], uv[qq], rule, &bad);
          if (acc && sp == 0) {
            float fu, fd;
            del_factors(d0, d1, gu, gd, sv[qq], &fu, &fd);
            fac[2 * r] = fu;
            fac[2 * r + 1] = fd;
          }
        }
        lastbad[qq] = bad && sp == 0;
        const unsigned b = __ballot_sync(0xffffffffu, acc) & 0x55555555u;
        if (b && cand == kNoSlice) cand = qq * kRowStride + warp * 16 + ((__ffs(b) - 1) >> 1);
      }
      if (lane == 0 && cand != kNoSlice) atomicMin(&s_next[par], cand);
    };

    // After the barrier of a round: read the decision and reset the buffer
    // that the round before used (every thread has read it before reaching
    // this round's barrier, and it is written again only two rounds later).
    // Also counts the bad ratios among the proposals this round decided,
    // i.e. the owned slices in [lo, next].
    auto take_next = [&](int lo) -> int {
      const int nxt = s_next[par];
      if (tid == 0) s_next[(par + 2) % 3] = kNoSlice;
      par = (par + 1) % 3;
      const int hi = nxt < L ? nxt : L - 1;
#pragma unroll
      for (int qq = 0; qq < kRowsPerThread; ++qq) {
        if (qq * kRowStride >= L) break;  // uniform: rows beyond the grid
        const int r = row0 + qq * kRowStride;
        if (r >= lo && r <= hi && lastbad[qq]) ++n_bad;
      }
      return nxt;
    };

    for (long long sw = 0; sw < n_sweeps; ++sw) {
      const long long t = c0.t + sw;
#pragma unroll
      for (int qq = 0; qq < kRowsPerThread; ++qq) {
        if (qq * kRowStride >= L) break;  // uniform: rows beyond the grid
        const int r = row0 + qq * kRowStride;
        if (r < L) uv[qq] = proposal_uniform_f32(r, t, ip.chain, ip.grid, a.seed);
      }
      propose(0);
      __syncthreads();
      int l = take_next(0);
      // flip factors of the accepted slice; read before any flush or
      // recompute, whose shared-memory workspace may overlay fac[]
      float fu = 0.f, fd = 0.f;
      if (l < L) {
        fu = fac[2 * l];
        fd = fac[2 * l + 1];
      }
      while (l < L) {
        if constexpr (kMirror) {
          // spin up only: the even thread of a pair appends u_i (column l),
          // the odd one w_i (row l); one shuffle gives both the pair's values
          float gq[kRowsPerThread];
#pragma unroll
          for (int qq = 0; qq < kRowsPerThread; ++qq) {
            if (qq * kRowStride >= L) break;  // uniform: rows beyond the grid
            const int i = row0 + qq * kRowStride;
            gq[qq] = i < L ? (sp ? Gs[l * ld + i] : Gs[i * ld + l]) : 0.f;
          }
#pragma unroll
          for (int qq = 0; qq < kRowsPerThread; ++qq) {
            if (qq * kRowStride >= L) break;  // uniform: rows beyond the grid
            const int i = row0 + qq * kRowStride;
            const int oi = i * KP, ol = l * KP;  // 32-bit shared-memory offsets
            float c4[4] = {0.f, 0.f, 0.f, 0.f};
            if (i < L) {
              // even lane: U row i . W row l; odd lane: W row i . U row l.  The
              // first load reads a distinct row in every lane (U or W, whose
              // rows of one index sit 16 banks apart), the second the pair's
              // two shared rows: both conflict-free
              const float4* Ar = reinterpret_cast<const float4*>((sp ? Ws : Us) + oi);
              const float4* Br = reinterpret_cast<const float4*>((sp ? Us : Ws) + ol);
              const int j4 = (j + 3) >> 2;
              for (int m4 = 0; m4 < j4; ++m4) {
                const float4 a1 = Ar[m4], b1 = Br[m4];
                c4[0] = __fmaf_rn(a1.x, b1.x, c4[0]);
                c4[1] = __fmaf_rn(a1.y, b1.y, c4[1]);
                c4[2] = __fmaf_rn(a1.z, b1.z, c4[2]);
                c4[3] = __fmaf_rn(a1.w, b1.w, c4[3]);
              }
            }
            const float dot = gq[qq] + ((c4[0] + c4[1]) + (c4[2] + c4[3]));
            const float mine = i >= L ? 0.f : sp ? dot * fu : dot - ((i == l) ? 1.f : 0.f);
            const float theirs = __shfl_xor_sync(0xffffffffu, mine, 1);
            if (i < L) {
              const float uu = sp ? theirs : mine, ww = sp ? mine : theirs;
              if (sp) {
                exq = __vmaxu4(exq, ((__float_as_uint(ww) << 1) >> 24) << 8);
                Ws[oi + j] = ww;
              } else {
                exq = __vmaxu4(exq, (__float_as_uint(uu) << 1) >> 24);
                Us[oi + j] = uu;
              }
              dg[qq] = __fmaf_rn(uu, ww, dg[qq]);
              if (i == l) {
                sv[qq] = -sv[qq];
                if (sp == 0) ss[i] = (int8_t)sv[qq];
              }
            }
          }
        } else {
        // append column j of the panels for the owned rows of this thread's spin
        const float f = sp ? fd : fu;
        // base G entries of every owned row first (before any panel store), so
        // their latency -- L2 when G lives in HBM -- overlaps the dot products
        float gil_q[kRowsPerThread], gli_q[kRowsPerThread];
#pragma unroll
        for (int qq = 0; qq < kRowsPerThread; ++qq) {
          if (qq * kRowStride >= L) break;  // uniform: rows beyond the grid
          const int i = row0 + qq * kRowStride;
          gil_q[qq] = i < L ? Gs[i * ld + l] : 0.f;  // 2 L^2 < 2^31: 32-bit offsets
          gli_q[qq] = i < L ? Gs[l * ld + i] : 0.f;
        }
#pragma unroll
        for (int qq = 0; qq < kRowsPerThread; ++qq) {
          if (qq * kRowStride >= L) break;  // uniform: rows beyond the grid
          const int i = row0 + qq * kRowStride;
          if (i >= L) continue;
          const float gil = gil_q[qq], gli = gli_q[qq];
          float c4[4] = {0.f, 0.f, 0.f, 0.f}, r4[4] = {0.f, 0.f, 0.f, 0.f};
          const int oi = i * KP, ol = l * KP;  // 32-bit shared-memory offsets
          const float4* Ui = reinterpret_cast<const float4*>(Us + oi);
          const float4* Wl = reinterpret_cast<const float4*>(Ws + ol);
          const float4* Ul = reinterpret_cast<const float4*>(Us + ol);
          const float4* Wi = reinterpret_cast<const float4*>(Ws + oi);
          const int j4 = (j + 3) >> 2;
          for (int m4 = 0; m4 < j4; ++m4) {
            const float4 a1 = Ui[m4], b1 = Wl[m4], a2 = Ul[m4], b2 = Wi[m4];
            c4[0] = __fmaf_rn(a1.x, b1.x, c4[0]);
            c4[1] = __fmaf_rn(a1.y, b1.y, c4[1]);
            c4[2] = __fmaf_rn(a1.z, b1.z, c4[2]);
            c4[3] = __fmaf_rn(a1.w, b1.w, c4[3]);
            r4[0] = __fmaf_rn(a2.x, b2.x, r4[0]);
            r4[1] = __fmaf_rn(a2.y, b2.y, r4[1]);
            r4[2] = __fmaf_rn(a2.z, b2.z, r4[2]);
            r4[3] = __fmaf_rn(a2.w, b2.w, r4[3]);
          }
          const float uu = gil + ((c4[0] + c4[1]) + (c4[2] + c4[3])) - ((i == l) ? 1.f : 0.f);
          const float ww = (gli + ((r4[0] + r4[1]) + (r4[2] + r4[3]))) * f;
          exq = __vmaxu4(exq, ((__float_as_uint(uu) << 1) >> 24) | (((__float_as_uint(ww) << 1) >> 24) << 8));
          Us[oi + j] = uu;
          Ws[oi + j] = ww;
          dg[qq] = __fmaf_rn(uu, ww, dg[qq]);
          if (i == l) {
            sv[qq] = -sv[qq];
            if (sp == 0) ss[i] = (int8_t)sv[qq];
          }
        }
        }
        hash = (hash ^ (unsigned long long)(t * (long long)L + l)) * kFnvPrime;
        if constexpr (kRecord) {
          if (tid == 0) ip.trace[(size_t)sw * trace_words(L) + (l >> 5)] |= 1u << (l & 31);
        }
        ++n_acc;
        ++j;
        propose(l + 1);
        __syncthreads();
        const int lnext = take_next(l + 1);
        float fu_next = 0.f, fd_next = 0.f;
        if (lnext < L) {
          fu_next = fac[2 * lnext];
          fd_next = fac[2 * lnext + 1];
        }
        if (j == K) flush();
        if (gc.n_wrap > 0 && --until_rec == 0) {
          until_rec = gc.n_wrap;
          flush();
          double d = -1.0;
          // G in HBM while the refinement runs (its staging overlays the whole
          // body of shared memory, a resident G included)
          bool in_hbm = false;
          if (kRefine && gc.rc && use_tc && !tc.failed && gc.lambda != 0.0) {
            if (resident) {
              for (int i = warp; i < 2 * L; i += NW)
                for (int jj = lane; jj < L; jj += 32) Ggl[(size_t)i * L + jj] = Gu[(size_t)i * ld + jj];
              __syncthreads();
              in_hbm = true;
            }
            int steps = 0;
            float* rws = reinterpret_cast<float*>(ip.ws);
            float* rred = reinterpret_cast<float*>(red);
            const float d0 = refine_spin(gc, *gc.rc, ss, 1, Ggl, rws, smem + lay.off_rf, &tc, rred, a.status, &steps);
            // spin down: not kept during a mirrored sweep; mirrored for a
            // particle-hole symmetric bath, else refined too
            const float d1 = d0 < 0.f ? -1.f
                             : kMirror ? 0.f
                             : gc.ph   ? ph_mirror(Ggl, Ggl + (size_t)L * L, L,
                                                   reinterpret_cast<float*>(smem + lay.off_rf), rred)
                                       : refine_spin(gc, *gc.rc, ss, -1, Ggl + (size_t)L * L, rws, smem + lay.off_rf,
                                                     &tc, rred, a.status, &steps);
            if (d0 >= 0.f && d1 >= 0.f)
              d = fmax((double)d0, (double)d1);
            else
              ++n_fb;
          }
          if (d < 0.0) {
            // from scratch: FP64 workspace in HBM, inverted by panels whose
            // scratch overlays the idle part of shared memory (never G)
            d = recompute_green_inv<float, NT, true>(
                gc, ss, in_hbm ? Ggl : Gu, in_hbm ? Ggl + (size_t)L * L : Gd, in_hbm ? L : ld, ip.ws, red, redi,
                &s_inv, &s_piv, colk, perm, true, a.status, 0, kMirror ? 1 : 2,
                reinterpret_cast<double*>(smem + lay.off_gjb));
          }
          if (in_hbm) {
            for (int i = warp; i < 2 * L; i += NW)
              for (int jj = lane; jj < L; jj += 32) Gu[(size_t)i * ld + jj] = Ggl[(size_t)i * L + jj];
            __syncthreads();
          }
          drift = fmax(drift, d);
          ++n_rec;
          zero_panels();  // the recompute's workspace may have overlaid them
          load_diag();
          __syncthreads();
        }
        l = lnext;
        fu = fu_next;
        fd = fd_next;
      }
      if (sw >= a.n_warm) {
        flush();
        const long long m = sw - a.n_warm;
        const int b = (int)((kBins * m) / a.n_meas);
        // partial sums in the (idle) staging area, totals in the panels' space
        float* part = reinterpret_cast<float*>(smem + lay.off_stage);
        float* gsum = reinterpret_cast<float*>(smem + lay.off_U);
        if (resident)
          measure_diagonals<kMirror ? 1 : 2>(Gu, Gd, ld, L, gsum);
        else
          measure_rows<kMirror ? 1 : 2>(Gu, Gd, ld, L, part, gsum);
        for (int k = tid; k < L; k += NT) {
          const double gu = (double)gsum[k] / (double)L;
          // G_dn = 1 - G_up^T: its sum of diagonal k > 0 is G_up's sum of
          // diagonal L - k, of diagonal 0 it is L minus G_up's
          const double gd = kMirror ? (k == 0 ? (double)L - (double)gsum[0] : (double)gsum[L - k]) / (double)L
                                    : (double)gsum[L + k] / (double)L;
          // the three accumulators loaded before any is stored: one L2 round trip
          double* bk = ip.bins + (size_t)b * L;
          const double a0 = ip.acc[k], a1 = ip.acc[L + k], b0 = bk[k];
          ip.acc[k] = a0 + gu;
          ip.acc[L + k] = a1 + gd;
          bk[k] = b0 + 0.5 * (gu + gd);
        }
        float v = 0.f;
#pragma unroll
        for (int qq = 0; qq < kRowsPerThread; ++qq) {
          if (qq * kRowStride >= L) break;  // uniform: rows beyond the grid
          const float other = __shfl_xor_sync(0xffffffffu, dg[qq], 1);
          const float dn = kMirror ? dg[qq] : 1.f - other;  // 1 - G_dn,ii
          if (sp == 0 && row0 + qq * kRowStride < L) v += (1.f - dg[qq]) * dn;
        }
        __syncthreads();  // every thread has read its totals
        for (int e = tid; e < 2 * L; e += NT) gsum[e] = 0.f;
        v = block_sum_f(v, reinterpret_cast<float*>(red));
        if (tid == 0) {
          const double d0 = ip.accD[0], d1 = ip.accD[1 + b];
          ip.accD[0] = d0 + (double)v / (double)L;
          ip.accD[1 + b] = d1 + (double)v / (double)L;
        }
      }
      __syncthreads();
    }
    flush();

    if (resident) {
      for (int i = warp; i < 2 * L; i += NW)
        for (int jj = lane; jj < L; jj += 32) Ggl[(size_t)i * L + jj] = Gu[(size_t)i * ld + jj];
    }
    if constexpr (kMirror) {
      // the chain's G_dn for the host and the next call: 1 - G_up^T
      __syncthreads();
      (void)ph_mirror(Ggl, Ggl + (size_t)L * L, L, reinterpret_cast<float*>(smem + lay.off_rf),
                      reinterpret_cast<float*>(red));
    }
    for (int l = tid; l < L; l += NT) ip.s[l] = ss[l];
    // bad ratios were counted per owned row: sum over the CTA
    {
      const int nb = __reduce_add_sync(0xffffffffu, (int)n_bad);
      if (lane == 0 && nb) atomicAdd(&s_bad, nb);
      __syncthreads();
      n_bad = s_bad;
    }
    if (tid == 0) {
      ChainCounters c = c0;
      c.t = c0.t + n_sweeps;
      c.proposals = c0.proposals + n_sweeps * (long long)L;
      c.accepted = n_acc;
      c.recomputes = c0.recomputes + n_rec;
      c.hash = hash;
      c.bad = c0.bad + n_bad;
      c.drift = drift;
      c.fallbacks = c0.fallbacks + n_fb;
      *ip.cnt = c;
    }
    __syncthreads();
  }
  if (use_tc) tc_teardown(&tc);
}

size_t delayed_smem(int L, int k, bool resident, bool gj_smem, bool gtile, int ub, bool refine, int ns) {
  return del_layout(L, k, resident, gj_smem, gtile, ub, refine, ns).bytes;
}

int delayed_config(size_t smem, int* threads, int* ctas_per_sm) {
  cudaError_t e = cudaSuccess;
  for (auto* f : {k_sweep_delayed<false, false>, k_sweep_delayed<true, false>, k_sweep_delayed<false, true>,
                  k_sweep_delayed<true, true>, k_sweep_delayed<false, true, true>, k_sweep_delayed<true, true, true>})
    if (e == cudaSuccess) e = raise_smem_limit(f, smem);
  int occ = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep_delayed<false, true>, kDelNT, smem);
  *threads = kDelNT;
  // each CTA holds kTmemCols of the SM's 512 TMEM columns for its lifetime
  *ctas_per_sm = occ < 512 / kTmemCols ? occ : 512 / kTmemCols;
  return (int)e;
}

int launch_sweep_delayed(const SweepArgs& a, int ctas, size_t smem, cudaStream_t st) {
  const bool rec = a.trace_mode == kTraceRecord;
  if (a.refine && a.mirror)
    (rec ? k_sweep_delayed<true, true, true> : k_sweep_delayed<false, true, true>)<<<ctas, kDelNT, smem, st>>>(a);
  else if (a.refine)
    (rec ? k_sweep_delayed<true, true> : k_sweep_delayed<false, true>)<<<ctas, kDelNT, smem, st>>>(a);
  else
    (rec ? k_sweep_delayed<true, false> : k_sweep_delayed<false, false>)<<<ctas, kDelNT, smem, st>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace hfq
