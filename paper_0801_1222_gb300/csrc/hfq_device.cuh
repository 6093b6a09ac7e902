// Device-side data layout of the HF-QMC sweep library (GB300, sm_103a).
//
// HBM layout (all per context, allocated once at create):
//   per grid  : GridConst (Lambda, lambda, the two flip factors Delta and the
//               two bath factors e^{+-lambda}-1), the FP64 bath matrix M
//               and its inverse (Lambda x Lambda row-major), GridAccount (measured-sweep
//               counts, 32 bin counts), GridOut (reduced G(tau), errors, D).
//   per chain : HS field s (int8[Lambda]), G^up and G^dn back to back
//               (2 x Lambda x Lambda, row-major, FP64 or FP32), the FP64
//               Gauss-Jordan workspace (Lambda x 2 Lambda; Lambda x Lambda per spin), the
//               measurement sums (2 Lambda spin-major, 32 x Lambda bins,
//               1 + 32 D sums) and ChainCounters.
// Every chain is one work item; items are processed longest-Lambda-first
// from an atomic queue by a persistent grid of CTAs.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hfq {

constexpr int kBins = 32;
constexpr unsigned long long kFnvOffset = 0xcbf29ce484222325ull;
constexpr unsigned long long kFnvPrime = 0x100000001b3ull;

// Status bits of the context-wide error word.
constexpr int kStatusSingular = 1;   // zero pivot in a Gauss-Jordan recompute
constexpr int kStatusNonFinite = 2;  // non-finite G after a recompute
constexpr int kStatusTimeout = 4;    // a bounded wait gave up

// ---------------------------------------------------------------------------
// Newton refinement of G by exact sliced tensor-core products (the FP32
// delayed path's recompute; see hfq_refine.cuh).  With D = diag(e^{sigma
// lambda s} - 1), G^{-1} = B = M^{-1}(1 + D) - D = A (1 + D) with
// A = M^{-1} - diag(1 - e^{-sigma lambda s_j}); the residual of G' is
// E = 1 - B G' = 1 - A H', H' = (1 + D) G', and one step gives
// G' + G' E = (1 + D)^{-1} (H' + H' E).  A and H' are cut into signed 7-bit
// integer slices held exactly in FP16, so every slice product accumulates
// exactly in the tensor cores' FP32 accumulators.
// ---------------------------------------------------------------------------
constexpr int kRfBits = 7;        // bits per slice
constexpr int kRfSlicesA = 6;     // slices of A (42 bits)
constexpr int kRfSlicesH = 4;     // slices of H' (28 bits)
constexpr int kRfLevels = 6;      // products p + q = 0 .. 5 kept, one FP32 accumulator per level
constexpr int kRfNMax = 80;       // columns of G per product tile: 64 or 80 per grid (rc.nN)
constexpr int kRfKC = 32;         // K (contraction) extent of one staged chunk of the residual product
constexpr int kRf2KC = 64;        // the same for the update product
constexpr int kRfTileA = 128 * kRfKC * 2;        // bytes of one A slice of a (row block, K chunk)
constexpr int kRfTileH = kRfNMax * kRfKC * 2;    // bytes of one H' slice of a (column block, K chunk)
constexpr int kRfStage = kRfSlicesA * kRfTileA + kRfSlicesH * kRfTileH;  // 68 KiB: one chunk
constexpr int kRfSmem = 2 * kRfStage;            // two stage buffers

struct RefineConst {
  const uint16_t* aslc;  // A's slices: [row block of 128][K chunk of 64][slice][128 x 64 FP16,
                         // K-major core-matrix layout], padded with zeros
  int ea;                // |A| < 2^ea (the slices' common scale)
  int nrb, nkc;          // row blocks of 128, K chunks of 64 (Lambda padded)
  float emax_step;       // Newton steps only while max |E| <= emax_step (else from scratch)
  int nN;                // columns of G per product tile: 64 or 80, whichever pads Lambda less
  float cplus[2];        // e^{+lambda}, e^{-lambda} in FP32: (1 + d_j) for sigma s_j = +1, -1
  float cminus_hi[2];    // e^{-sigma lambda s_j} = 1 / (1 + d_j) as an FP32 pair (hi + lo)
  float cminus_lo[2];
  uint16_t dslc[2][kRfSlicesA];  // slices (FP16 bits) of A_jj for sigma s_j = +1, -1
};

__host__ __device__ inline int rf_pad(int L, int m) { return (L + m - 1) / m * m; }
// Bytes of A's slice table of one grid, and of the per-chain workspace the
// refinement needs (E^T in FP32, rows padded to a multiple of four floats;
// the chain's FP64 Gauss-Jordan workspace has room).
__host__ __device__ inline size_t rf_aslc_bytes(int L) {
  return (size_t)(rf_pad(L, 128) / 128) * (rf_pad(L, kRfKC) / kRfKC) * kRfSlicesA * kRfTileA;
}
__host__ __device__ inline size_t rf_ws_bytes(int L) { return (size_t)L * rf_pad(L, 4) * 4; }

struct GridConst {
  int L;           // Lambda
  int chains;
  int item0;       // first item (chain 0) of this grid
  int resident;    // 1: G staged in shared memory for the whole chain
  int k;           // delay depth (delayed path)
  int n_wrap;      // recompute interval in accepted flips (<= 0: never)
  int gj_smem;     // 1: the FP64 recompute works in shared memory
  int gtile;       // 1: the delayed flush adds its tiles to G by TMA reduce (tmapG)
  int ub;          // U blocks staged together by the delayed flush (1 or 2)
  double lambda;   // cosh(lambda) = exp(dtau U / 2)
  double delta[2]; // Delta for sigma*s = +1: e^{-2 lambda} - 1; sigma*s = -1: e^{2 lambda} - 1
  double dV[2];    // e^{sigma lambda s} - 1 for sigma*s = +1 / -1
  float deltaf[2]; // delta[] rounded to FP32 (the FP32 paths' flip factors)
  const double* M;    // bath matrix (FP64, L x L)
  const double* Minv; // its inverse (FP64, L x L), for the recompute through G^{-1}
  const void* tmapG;  // TMA tensor map (CUtensorMap, global memory) over the FP32 G of
                      // all chains: dims {column, row, spin, chain}; null unless gtile
  const RefineConst* rc;  // recompute by Newton refinement (FP32 delayed path); null: Gauss-Jordan
  int ph;                 // the bath is particle-hole symmetric (M + M^T = 1): every field has
                          // G_dn = 1 - G_up^T, so a recompute rebuilds G_up and mirrors it
  int pad2;
};

struct ChainCounters {
  long long t;               // global index of the next sweep
  long long proposals;
  long long accepted;        // cumulative since the first set_G0 (drives n_wrap)
  long long recomputes;
  unsigned long long hash;   // FNV-1a over sweep*L + l of accepted flips
  long long bad;             // proposals with R <= 0 or non-finite R
  double drift;              // max |G_fast - G_fresh| since the last set_G0
  int status;
  int fallbacks;             // recomputes that the refinement handed to Gauss-Jordan
};

struct ItemPtrs {
  int grid, chain, L, pad;
  int8_t* s;
  void* G;        // G^up then G^dn, L x L each, row-major
  double* ws;     // L x 2L Gauss-Jordan workspace
  double* acc;    // 2L
  double* bins;   // 32 L
  double* accD;   // 1 + 32
  ChainCounters* cnt;
  uint32_t* trace;  // decision trace of this chain: [sweep][ceil(L/32) words], bit l of a
                    // sweep's words set iff slice l was flipped (null: no trace)
};

struct GridAccount {
  long long n_meas;          // measured sweeps since set_G0
  long long bin_count[kBins];
};

struct GridOut {
  long long proposals, accepted, recomputes, bad;
  double drift;
  double D, D_err;
  long long fallbacks;
};

struct SweepArgs {
  const GridConst* grids;
  const ItemPtrs* items;
  const int* order;          // LPT order of items
  int n_items;
  int* queue_head;
  int* status;               // context-wide error word (bit flags)
  unsigned long long seed;
  long long n_warm, n_meas;
  int accept_rule;           // 0 Metropolis, 1 heat bath
  int flush;                 // delayed path: 1 tcgen05, 2 FFMA
  int trace_mode;            // 0 none, 1 record the accepted flips, 2 replay them (rank-1 paths)
  int refine;                // delayed path: some grid recomputes by Newton refinement
  int mirror;                // delayed path: every grid refines and its bath is particle-hole
                             // symmetric, and the sweep keeps G_up only
};

constexpr int kTraceOff = 0, kTraceRecord = 1, kTraceReplay = 2;

// Words of one sweep's decision trace.
__host__ __device__ inline int trace_words(int L) { return (L + 31) >> 5; }

// Bytes of shared memory the FP64 recompute needs for its L x L workspace.
__host__ __device__ inline size_t gj_smem_bytes(int L) { return (size_t)L * L * sizeof(double); }

// Pivot columns per panel of the blocked FP64 inversion (workspace in HBM)
// and the shared scratch it needs: the L x kGjPanel panel (pitch kGjPanel + 1)
// and the panel's pivot rows (kGjPanel x L).
constexpr int kGjPanel = 16;
__host__ __device__ inline size_t gj_blocked_bytes(int L) {
  return ((size_t)L * (kGjPanel + 1) + (size_t)kGjPanel * L) * sizeof(double);
}

// Dynamic shared memory a kernel may request (the rest of the SM's 227 KB
// holds the static shared memory).
constexpr size_t kSmemCap = 227 * 1024 - 512;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products of counter words 0 and 2 with the round
// multipliers, combined with the other words and the key by XOR; the key is
// bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned long long seed) {
  unsigned k0 = (unsigned)(seed & 0xffffffffull);
  unsigned k1 = (unsigned)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// 53-bit uniform in [0,1) from words 0 and 1 (all steps exact in FP64).
__device__ __forceinline__ double u53(unsigned x0, unsigned x1) {
  return __dmul_rn(__dadd_rn(__dmul_rn((double)(x0 >> 5), 67108864.0), (double)(x1 >> 6)),
                   1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double proposal_uniform(int l, long long t, int chain, int grid,
                                                   unsigned long long seed) {
  const uint4 x = philox4x32_10(make_uint4((unsigned)l, (unsigned)t, (unsigned)chain,
                                           (unsigned)grid), seed);
  return u53(x.x, x.y);
}

// 24-bit uniform in [0,1) from word 0 of the same Philox output that gives
// the 53-bit uniform (the FP32 paths' proposal threshold; no FP64 involved).
__device__ __forceinline__ float proposal_uniform_f32(int l, long long t, int chain, int grid,
                                                      unsigned long long seed) {
  const uint4 x = philox4x32_10(make_uint4((unsigned)l, (unsigned)t, (unsigned)chain,
                                           (unsigned)grid), seed);
  return (float)(x.x >> 8) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ int8_t initial_spin(int l, int chain, int grid,
                                               unsigned long long seed) {
  const uint4 x = philox4x32_10(make_uint4((unsigned)l | (1u << 16), 0u, (unsigned)chain,
                                           (unsigned)grid), seed);
  return (x.x & 1u) ? (int8_t)1 : (int8_t)-1;
}

// Block-wide max of a non-negative double; every thread gets the result.
// red: NT/32 doubles of shared scratch.  Contains barriers.
template <int NT>
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) r = fmax(r, red[w]);
  return r;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) r += red[w];
  return r;
}

}  // namespace hfq
