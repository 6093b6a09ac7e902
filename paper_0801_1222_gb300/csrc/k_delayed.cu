// Delayed (rank-k) FP32 Hirsch-Fye sweep: one CTA per Markov chain,
// persistent over the longest-Lambda-first work queue.
//
// The accepted flips of a chain are not applied one by one.  After j accepted
// flips since the last flush the current Green matrix is
//     G_cur = G + U W^T,   U, W: L x j panels (per spin),
// so a proposal needs only the current diagonal (kept incrementally), and an
// accepted flip at slice l appends
//     u = G_cur[:, l] - e_l,           w = (Delta / R) G_cur[l, :],
// whose entries cost O(j) each (the base column / row plus a length-j dot
// product with the panels).  Every k accepted flips the panels are flushed,
// G += U W^T -- a dense L x L x k contraction per spin (tcgen05 tensor cores
// with split TF32, or FP32 FMA).  The rank-1 formula of the Hirsch-Fye update
// is recovered exactly in exact arithmetic; only the rounding differs.
// The panels are also flushed before every measurement and every FP64
// recompute (every n_wrap accepted flips).
#include "hfq_delayed.cuh"
#include "hfq_device.cuh"
#include "hfq_gj.cuh"
#include "hfq_launch.h"

namespace hfq {

__global__ void __launch_bounds__(kDelNT, 2) k_sweep_delayed(SweepArgs a) {
  constexpr int NT = kDelNT;
  constexpr int NW = NT / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[NW];
  __shared__ int redi[NW];
  __shared__ double s_inv;
  __shared__ int s_piv, s_item;
  __shared__ uint32_t s_tmem_base;
  __shared__ __align__(8) unsigned long long s_mbar;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool use_tc = a.flush != 2;
  TcState tc;
  if (use_tc) tc_setup(&tc, &s_tmem_base, &s_mbar, a.status);

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
    const DelLayout lay = del_layout(L, K, resident, gc.gj_smem != 0);

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
    float* Pu = reinterpret_cast<float*>(smem + lay.off_U);  // [2][L][KP]: spin-major U panels
    float* Pw = reinterpret_cast<float*>(smem + lay.off_W);  // [2][L][KP]: W panels
    float* diag = reinterpret_cast<float*>(smem + lay.off_diag);
    float* us = reinterpret_cast<float*>(smem + lay.off_u);  // uniforms rounded to FP32
    double* colk = reinterpret_cast<double*>(smem + lay.off_colk);
    int8_t* ss = reinterpret_cast<int8_t*>(smem + lay.off_s);
    unsigned char* stage = smem + lay.off_stage;
    const int KP = lay.KP;
    const float d0 = gc.deltaf[0], d1 = gc.deltaf[1];
    const int rule = a.accept_rule;

    if (resident) {
      for (int i = warp; i < 2 * L; i += NW)
        for (int jj = lane; jj < L; jj += 32) Gu[(size_t)i * ld + jj] = Ggl[(size_t)i * L + jj];
    }
    for (int l = tid; l < L; l += NT) ss[l] = ip.s[l];
    __syncthreads();
    for (int i = tid; i < L; i += NT) {
      diag[i] = Gu[(size_t)i * ld + i];
      diag[L + i] = Gd[(size_t)i * ld + i];
    }
    const ChainCounters c0 = *ip.cnt;
    long long n_acc = c0.accepted;
    long long n_rec = 0, n_bad = 0;
    unsigned long long hash = c0.hash;
    double drift = c0.drift;
    const long long n_sweeps = a.n_warm + a.n_meas;
    int j = 0;  // pending flips in the panels
    __syncthreads();

    // G += U W^T for both spins, then the diagonal is re-read from G.
    auto flush = [&]() {
      if (j == 0) return;
      if (use_tc)
        flush_tcgen05(&tc, Gu, Gd, ld, Pu, Pw, KP, L, j, stage, lay, a.status);
      else
        flush_ffma(Gu, Gd, ld, Pu, Pw, KP, L, j);
      __syncthreads();
      for (int i = tid; i < L; i += NT) {
        diag[i] = Gu[(size_t)i * ld + i];
        diag[L + i] = Gd[(size_t)i * ld + i];
      }
      j = 0;
      __syncthreads();
    };

    for (long long sw = 0; sw < n_sweeps; ++sw) {
      const long long t = c0.t + sw;
      for (int l = tid; l < L; l += NT)
        us[l] = (float)proposal_uniform(l, t, ip.chain, ip.grid, a.seed);
      __syncthreads();
      int l0 = 0;
      while (l0 < L) {
        // first accepted proposal at or after l0 (every warp evaluates the same window)
        int first = L;
        for (int w = l0; w < L; w += 32) {
          const int l = w + lane;
          bool acc = false, bad = false;
          if (l < L) acc = del_decide(d0, d1, diag[l], diag[L + l], ss[l], us[l], rule, &bad);
          const unsigned b = __ballot_sync(0xffffffffu, acc);
          const unsigned bb = __ballot_sync(0xffffffffu, bad);
          if (b) {
            first = w + __ffs(b) - 1;
            const int upto = first - w;
            const unsigned valid = upto >= 31 ? 0xffffffffu : ((2u << upto) - 1u);
            n_bad += __popc(bb & valid);
            break;
          }
          n_bad += __popc(bb);
        }
        if (first >= L) break;
        const int l = first;
        const int sl = ss[l];
        float fu, fd;
        del_factors(d0, d1, diag[l], diag[L + l], sl, &fu, &fd);
        // append column j of the panels: item (sp, i) -> u_i, w_i and the diagonal.
        // Current column / row entries are the base G entry plus a length-j dot
        // product with the panels (16-byte loads, four partial sums).
        for (int it = tid; it < 2 * L; it += NT) {
          const int sp = it >= L;
          const int i = it - sp * L;
          const float* G = sp ? Gd : Gu;
          float* U = Pu + (size_t)sp * L * KP;
          float* W = Pw + (size_t)sp * L * KP;
          const float g_il = G[(size_t)i * ld + l];
          const float g_li = G[(size_t)l * ld + i];
          const float4* Ui = reinterpret_cast<const float4*>(U + (size_t)i * KP);
          const float4* Ul = reinterpret_cast<const float4*>(U + (size_t)l * KP);
          const float4* Wi = reinterpret_cast<const float4*>(W + (size_t)i * KP);
          const float4* Wl = reinterpret_cast<const float4*>(W + (size_t)l * KP);
          float c4[4] = {0.f, 0.f, 0.f, 0.f}, r4[4] = {0.f, 0.f, 0.f, 0.f};
          const int j4 = j >> 2;
          for (int q = 0; q < j4; ++q) {
            const float4 ui = Ui[q], wl = Wl[q], ul = Ul[q], wi = Wi[q];
            c4[0] = __fmaf_rn(ui.x, wl.x, c4[0]);
            c4[1] = __fmaf_rn(ui.y, wl.y, c4[1]);
            c4[2] = __fmaf_rn(ui.z, wl.z, c4[2]);
            c4[3] = __fmaf_rn(ui.w, wl.w, c4[3]);
            r4[0] = __fmaf_rn(ul.x, wi.x, r4[0]);
            r4[1] = __fmaf_rn(ul.y, wi.y, r4[1]);
            r4[2] = __fmaf_rn(ul.z, wi.z, r4[2]);
            r4[3] = __fmaf_rn(ul.w, wi.w, r4[3]);
          }
          const float* Uis = U + (size_t)i * KP;
          const float* Uls = U + (size_t)l * KP;
          const float* Wis = W + (size_t)i * KP;
          const float* Wls = W + (size_t)l * KP;
          for (int m = 4 * j4; m < j; ++m) {
            c4[0] = __fmaf_rn(Uis[m], Wls[m], c4[0]);
            r4[0] = __fmaf_rn(Uls[m], Wis[m], r4[0]);
          }
          const float cc = g_il + ((c4[0] + c4[1]) + (c4[2] + c4[3]));
          const float rr = g_li + ((r4[0] + r4[1]) + (r4[2] + r4[3]));
          const float uu = cc - (i == l ? 1.f : 0.f);
          const float ww = rr * (sp ? fd : fu);
          U[(size_t)i * KP + j] = uu;
          W[(size_t)i * KP + j] = ww;
          diag[sp * L + i] = __fmaf_rn(uu, ww, diag[sp * L + i]);
        }
        if (tid == 0) ss[l] = (int8_t)(-sl);
        hash = (hash ^ (unsigned long long)(t * (long long)L + l)) * kFnvPrime;
        ++n_acc;
        ++j;
        __syncthreads();
        if (j == K) flush();
        if (gc.n_wrap > 0 && n_acc % gc.n_wrap == 0) {
          flush();
          double d;
          if (gc.gj_smem) {
            // [A | M] overlays the body of shared memory: G goes home to HBM first
            if (resident) {
              for (int i = warp; i < 2 * L; i += NW)
                for (int jj = lane; jj < L; jj += 32) Ggl[(size_t)i * L + jj] = Gu[(size_t)i * ld + jj];
              __syncthreads();
            }
            d = recompute_green<float, NT>(gc, ss, Ggl, Ggl + (size_t)L * L, L,
                                           reinterpret_cast<double*>(smem + lay.off_body), red, redi,
                                           &s_inv, &s_piv, colk, true, a.status);
            if (resident) {
              for (int i = warp; i < 2 * L; i += NW)
                for (int jj = lane; jj < L; jj += 32) Gu[(size_t)i * ld + jj] = Ggl[(size_t)i * L + jj];
              __syncthreads();
            }
          } else {
            d = recompute_green<float, NT>(gc, ss, Gu, Gd, ld, ip.ws, red, redi, &s_inv, &s_piv, colk,
                                           true, a.status);
          }
          drift = fmax(drift, d);
          ++n_rec;
          for (int i = tid; i < L; i += NT) {
            diag[i] = Gu[(size_t)i * ld + i];
            diag[L + i] = Gd[(size_t)i * ld + i];
          }
          __syncthreads();
        }
        l0 = l + 1;
      }
      if (sw >= a.n_warm) {
        flush();
        const long long m = sw - a.n_warm;
        const int b = (int)((kBins * m) / a.n_meas);
        // partial sums in the (idle) staging area, totals in the panels' space
        float* part = reinterpret_cast<float*>(smem + lay.off_stage);
        float* gsum = reinterpret_cast<float*>(smem + lay.off_U);
        measure_rows(Gu, Gd, ld, L, part, gsum);
        for (int k = tid; k < L; k += NT) {
          const double gu = (double)gsum[k] / (double)L, gd = (double)gsum[L + k] / (double)L;
          ip.acc[k] += gu;
          ip.acc[L + k] += gd;
          ip.bins[(size_t)b * L + k] += 0.5 * (gu + gd);
        }
        float v = 0.f;
        for (int l = tid; l < L; l += NT) v += (1.f - diag[l]) * (1.f - diag[L + l]);
        v = block_sum_f(v, reinterpret_cast<float*>(red));
        if (tid == 0) {
          ip.accD[0] += (double)v / (double)L;
          ip.accD[1 + b] += (double)v / (double)L;
        }
      }
      __syncthreads();
    }
    flush();

    if (resident) {
      for (int i = warp; i < 2 * L; i += NW)
        for (int jj = lane; jj < L; jj += 32) Ggl[(size_t)i * L + jj] = Gu[(size_t)i * ld + jj];
    }
    for (int l = tid; l < L; l += NT) ip.s[l] = ss[l];
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
  if (use_tc) tc_teardown(&tc);
}

size_t delayed_smem(int L, int k, bool resident, bool gj_smem) {
  return del_layout(L, k, resident, gj_smem).bytes;
}

int delayed_config(size_t smem, int* threads, int* ctas_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_sweep_delayed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  int occ = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep_delayed, kDelNT, smem);
  *threads = kDelNT;
  // each CTA holds kTmemCols of the SM's 512 TMEM columns for its lifetime
  *ctas_per_sm = occ < 512 / kTmemCols ? occ : 512 / kTmemCols;
  return (int)e;
}

int launch_sweep_delayed(const SweepArgs& a, int ctas, size_t smem, cudaStream_t st) {
  k_sweep_delayed<<<ctas, kDelNT, smem, st>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace hfq
