// Host runtime of the C ABI declared in include/hfqmc.h.
//
// A context owns all device state of one batch of (U, dtau) grids x chains,
// laid out grid-major so that every per-grid reset is one contiguous memset.
// hfqmc_sweep enqueues, on the context stream, the whole hot path as four
// launches -- queue reset, measured-sweep bookkeeping, the persistent sweep
// kernel over all chains of all grids, the per-grid reduction -- plus one
// small device-to-host copy of the per-grid counters; with use_graph these
// are captured once per (n_warm, n_meas) and replayed as a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>
#include <cudaTypedefs.h>  // CUtensorMap and the cuTensorMapEncodeTiled prototype

#include "../../include/hfqmc.h"
#include "hfq_device.cuh"
#include "hfq_launch.h"

using namespace hfq;

namespace {

thread_local std::string g_create_error;

struct GridHost {
  double U, dtau, lambda;
  int L, chains, item0, k, n_wrap, resident, gj_smem, gtile = 0, ub = 2;
  int k_req = 0;        // the delay depth asked for (option or table), before fitting
  int k1 = 0, ub1 = 2;  // k and U blocks of the G_up-only sweep's layout (one spin's panels)
  bool refine = false;  // recompute by Newton refinement (FP32 delayed path)
  uint16_t* d_aslc = nullptr;  // its slice table of A (device)
  bool g0_set = false, ever_set = false;
  long long out_off;
};

// Per-Lambda defaults of the delay depth and recompute interval, measured
// on GB300 (paper_0801_1222_gb300/autotune.py): k by the sweep rate at each
// Lambda with the recompute every 64 accepted flips (k is lowered further
// when the panels or the TMA flush buffers would not fit); N_wrap = 64, the
// longest of the multigrid configuration's intervals {16, 32, 64} and the
// fastest, its FP32 G(tau) within 1e-9 of FP64 on the same trajectory.
struct TuneEntry {
  int L_max, k, n_wrap;
};
const TuneEntry kTuneTable[] = {
    {64, 24, 64}, {128, 24, 64}, {144, 32, 64}, {176, 24, 64}, {1024, 16, 64},
};

// k and N_wrap for Lambda from a table (the caller's if non-empty, else the
// built-in one); beyond its last entry the last entry applies
void tune_lookup(int L, const std::vector<TuneEntry>& user, int* k, int* n_wrap) {
  const TuneEntry* t = user.empty() ? kTuneTable : user.data();
  const size_t n = user.empty() ? sizeof(kTuneTable) / sizeof(kTuneTable[0]) : user.size();
  for (size_t i = 0; i < n; ++i)
    if (L <= t[i].L_max) {
      *k = t[i].k;
      *n_wrap = t[i].n_wrap;
      return;
    }
  *k = t[n - 1].k;
  *n_wrap = t[n - 1].n_wrap;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (the library does not link the driver API).  Null when unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      (void)cudaGetLastError();
  });
  return fn;
}

}  // namespace

struct hfqmc_ctx {
  int device = 0, n_sm = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  hfqmc_opts opts;
  double beta = 0.0;
  uint64_t seed = 0;
  int n_grids = 0, n_items = 0;
  std::vector<GridHost> gh;
  std::vector<GridConst> gc;
  std::vector<ItemPtrs> items;
  std::vector<void*> allocs;
  // device
  GridConst* d_grids = nullptr;
  ItemPtrs* d_items = nullptr;
  int* d_order = nullptr;
  int* d_queue = nullptr;
  int* d_status = nullptr;
  double* d_G0 = nullptr;
  GridAccount* d_account = nullptr;
  GridOut* d_gout = nullptr;
  double* d_outG = nullptr;
  double* d_outErr = nullptr;
  long long* d_out_off = nullptr;
  unsigned char* d_pool = nullptr;
  CUtensorMap* d_tmaps = nullptr;  // per grid (used where gh[g].gtile)
  // pinned host mirrors
  GridOut* h_gout = nullptr;
  int* h_status = nullptr;
  // sweep launch shape
  size_t sweep_smem = 0;
  int sweep_ctas = 0;
  int layout_ns = 2;  // spins the current shared-memory layout (gc[].k, ub, sweep_smem) is fitted for
  // instantiated graphs of hfqmc_sweep per (n_warm, n_meas), with the call
  // stamp of their last use (at most kMaxGraphs kept; the least recently used
  // one is destroyed first)
  struct CachedGraph {
    cudaGraphExec_t exec;
    unsigned long long used;
  };
  std::map<std::pair<long long, long long>, CachedGraph> graphs;
  unsigned long long graph_clock = 0;
  // decision trace (hfqmc_set_trace): mode, sweeps per chain, device buffer
  // and each grid's offset in it (words)
  int trace_mode = 0;
  long long trace_cap = 0;
  uint32_t* d_trace = nullptr;
  size_t trace_bytes = 0;
  std::vector<size_t> trace_off;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double last_ms = 0.0;
  long long sweeps_done = 0;
  std::string err;
};

namespace {

int fail(hfqmc_ctx* c, int code, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_error = msg;
  return code;
}

int cuda_fail(hfqmc_ctx* c, cudaError_t e, const char* where) {
  return fail(c, HFQMC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

void* dev_alloc(hfqmc_ctx* c, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 256;
  if (c->opts.alloc) {
    p = c->opts.alloc(bytes, c->opts.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    p = nullptr;
  }
  if (p) c->allocs.push_back(p);
  return p;
}

void dev_free(hfqmc_ctx* c, void* p) {
  if (!p) return;
  for (size_t i = 0; i < c->allocs.size(); ++i)
    if (c->allocs[i] == p) {
      c->allocs.erase(c->allocs.begin() + (long)i);
      break;
    }
  if (c->opts.alloc) {
    if (c->opts.free) c->opts.free(p, c->opts.alloc_user);
  } else {
    cudaFree(p);
  }
}

constexpr size_t kMaxGraphs = 8;

// The delayed sweep keeps G_up only when every grid refines and its bath is
// particle-hole symmetric (and opts.ph_symmetry is 0).
static int sweep_mirrors(const hfqmc_ctx* c) {
  if (c->opts.precision != HFQMC_F32_DELAYED || c->opts.ph_symmetry != 0) return 0;
  for (int g = 0; g < c->n_grids; ++g)
    if (!c->gh[g].refine || !c->gc[g].ph) return 0;
  return 1;
}

// The sweep launch runs the refining kernel when some grid refines with
// lambda != 0, and its G_up-only variant only then (a context whose grids
// all have lambda = 0 runs the plain two-spin kernel).
static int launch_refines(const hfqmc_ctx* c) {
  for (int g = 0; g < c->n_grids; ++g)
    if (c->gh[g].refine && c->gh[g].lambda != 0.0) return 1;
  return 0;
}
static int launch_mirrors(const hfqmc_ctx* c) { return launch_refines(c) ? sweep_mirrors(c) : 0; }

void drop_graphs(hfqmc_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
  c->graphs.clear();
}

bool f64_path(const hfqmc_ctx* c) { return c->opts.precision == HFQMC_F64_RANK1; }
size_t elem_size(const hfqmc_ctx* c) { return f64_path(c) ? sizeof(double) : sizeof(float); }

int launch_sweep_kernel(hfqmc_ctx* c, long long n_warm, long long n_meas) {
  SweepArgs a;
  a.grids = c->d_grids;
  a.items = c->d_items;
  a.order = c->d_order;
  a.n_items = c->n_items;
  a.queue_head = c->d_queue;
  a.status = c->d_status;
  a.seed = c->seed;
  a.n_warm = n_warm;
  a.n_meas = n_meas;
  a.accept_rule = c->opts.accept_rule;
  a.flush = c->opts.flush;
  a.trace_mode = c->trace_mode;
  a.refine = launch_refines(c);
  a.mirror = launch_mirrors(c);
  if (c->opts.precision == HFQMC_F32_DELAYED)
    return launch_sweep_delayed(a, c->sweep_ctas, c->sweep_smem, c->stream);
  return launch_sweep_rank1(f64_path(c), a, c->sweep_ctas, c->sweep_smem, c->stream);
}

// The whole hot path of one hfqmc_sweep call, enqueued on the context stream.
int enqueue_sweep(hfqmc_ctx* c, long long n_warm, long long n_meas) {
  cudaError_t e = cudaMemsetAsync(c->d_queue, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync(queue)");
  if (c->trace_mode == kTraceRecord) {
    e = cudaMemsetAsync(c->d_trace, 0, c->trace_bytes, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync(trace)");
  }
  int r = launch_account(c->d_account, c->n_grids, n_meas, c->stream);
  if (r) return cuda_fail(c, (cudaError_t)r, "launch_account");
  r = launch_sweep_kernel(c, n_warm, n_meas);
  if (r) return cuda_fail(c, (cudaError_t)r, "sweep kernel launch");
  r = launch_reduce(c->d_grids, c->d_items, c->d_account, c->d_gout, c->d_outG, c->d_outErr,
                    c->d_out_off, c->n_grids, c->stream);
  if (r) return cuda_fail(c, (cudaError_t)r, "launch_reduce");
  e = cudaMemcpyAsync(c->h_gout, c->d_gout, sizeof(GridOut) * c->n_grids,
                      cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync(gout)");
  e = cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync(status)");
  return HFQMC_OK;
}

int create_impl(hfqmc_ctx** out, double beta, const double* U, bool per_grid_U,
                const double* dtau, int n_grids, const int* chains, uint64_t seed,
                const hfqmc_opts* opts) {
  hfqmc_ctx* c = nullptr;
  if (!out) return fail(nullptr, HFQMC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!(beta > 0.0) || !std::isfinite(beta)) return fail(nullptr, HFQMC_EINVAL, "beta must be > 0");
  if (n_grids < 1 || n_grids > 4096) return fail(nullptr, HFQMC_EINVAL, "n_grids out of range");
  if (!dtau || !chains || !U) return fail(nullptr, HFQMC_EINVAL, "NULL array argument");
  hfqmc_opts o;
  if (opts)
    o = *opts;
  else
    hfqmc_default_opts(&o);
  if (o.precision < HFQMC_F64_RANK1 || o.precision > HFQMC_F32_DELAYED)
    return fail(nullptr, HFQMC_EINVAL, "unknown precision");
  if (o.accept_rule != HFQMC_METROPOLIS && o.accept_rule != HFQMC_HEAT_BATH)
    return fail(nullptr, HFQMC_EINVAL, "unknown accept_rule");
  if (o.recompute < HFQMC_RECOMPUTE_AUTO || o.recompute > HFQMC_RECOMPUTE_REFINE)
    return fail(nullptr, HFQMC_EINVAL, "unknown recompute method");
  if (o.recompute == HFQMC_RECOMPUTE_REFINE && o.precision != HFQMC_F32_DELAYED)
    return fail(nullptr, HFQMC_EINVAL, "the Newton refinement recompute belongs to the F32_DELAYED path");
  if (o.k != 0 && (o.k < 8 || o.k > 64 || o.k % 8 != 0))
    return fail(nullptr, HFQMC_EINVAL, "k must be 0 or a multiple of 8 in [8, 64]");
  std::vector<TuneEntry> user_table;
  if (o.tune_entries < 0 || (o.tune_entries > 0 && !o.tune_table))
    return fail(nullptr, HFQMC_EINVAL, "tune_table is NULL or tune_entries < 0");
  for (int i = 0; i < o.tune_entries; ++i) {
    const TuneEntry e{o.tune_table[3 * i], o.tune_table[3 * i + 1], o.tune_table[3 * i + 2]};
    if (e.L_max < 1 || e.k < 8 || e.k > 64 || e.k % 8 != 0 || e.n_wrap == 0 ||
        (i > 0 && e.L_max <= user_table.back().L_max))
      return fail(nullptr, HFQMC_EINVAL,
                  "tune_table entry " + std::to_string(i) +
                      ": needs Lambda_max >= 1 increasing, k a multiple of 8 in [8, 64], n_wrap != 0");
    user_table.push_back(e);
  }

  std::vector<GridHost> gh(n_grids);
  long long items = 0;
  for (int g = 0; g < n_grids; ++g) {
    const double Ug = per_grid_U ? U[g] : U[0];
    if (!(dtau[g] > 0.0) || !std::isfinite(dtau[g]))
      return fail(nullptr, HFQMC_EINVAL, "dtau must be > 0");
    if (!(Ug >= 0.0) || !std::isfinite(Ug)) return fail(nullptr, HFQMC_EINVAL, "U must be >= 0");
    const double Lr = beta / dtau[g];
    const long long L = std::llround(Lr);
    if (std::fabs(Lr - (double)L) > 1e-9 || L < 1 || L > 1024)
      return fail(nullptr, HFQMC_EINVAL,
                  "beta/dtau must be an integer Lambda in [1, 1024] (grid " + std::to_string(g) + ")");
    if (chains[g] < 1 || chains[g] > (1 << 20))
      return fail(nullptr, HFQMC_EINVAL, "chains_per_grid must be in [1, 2^20]");
    gh[g].U = Ug;
    gh[g].L = (int)L;
    gh[g].dtau = beta / (double)L;
    gh[g].lambda = std::acosh(std::exp(0.5 * gh[g].dtau * Ug));
    gh[g].chains = chains[g];
    gh[g].item0 = (int)items;
    items += chains[g];
  }
  if (items > (1 << 22)) return fail(nullptr, HFQMC_EINVAL, "too many chains");

  c = new (std::nothrow) hfqmc_ctx();
  if (!c) return fail(nullptr, HFQMC_ENOMEM, "host allocation failed");
  c->opts = o;
  c->beta = beta;
  c->seed = seed;
  c->n_grids = n_grids;
  c->n_items = (int)items;
  c->gh = gh;

  auto bail = [&](int code) {
    g_create_error = c->err;
    hfqmc_destroy(c);
    return code;
  };

  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaGetDevice"));
  e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaDeviceGetAttribute"));
  if (o.cuda_stream) {
    c->stream = (cudaStream_t)o.cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamCreate"));
    c->own_stream = true;
  }
  if ((e = cudaEventCreate(&c->ev0)) != cudaSuccess || (e = cudaEventCreate(&c->ev1)) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaEventCreate"));

  // per-grid constants, delay depth, recompute interval, residency
  const bool f64 = f64_path(c);
  const size_t es = elem_size(c);
  size_t smem_max = 0;
  const size_t kResidentBudget =
      o.resident_kb == 0 ? 200 * 1024 : (o.resident_kb < 0 ? 0 : (size_t)o.resident_kb * 1024);
  const size_t kSmemMax = kSmemCap;
  c->gc.resize(n_grids);
  long long out_off = 0;
  for (int g = 0; g < n_grids; ++g) {
    GridHost& h = c->gh[g];
    int k_t = 16, nw_t = 1024;
    if (o.autotune) {
      tune_lookup(h.L, user_table, &k_t, &nw_t);
      // the built-in table is the delayed path's; the rank-1 paths recompute
      // from scratch at a long interval (FP64: the drift of 16384 flips is
      // ~1e-12; FP32 rank-1: the interval validated for its G(tau))
      if (o.precision != HFQMC_F32_DELAYED && user_table.empty())
        nw_t = (o.precision == HFQMC_F64_RANK1 || h.L > 128) ? 16384 : 8192;
    }
    h.k = (o.precision == HFQMC_F32_DELAYED) ? (o.k ? o.k : k_t) : 1;
    h.k_req = h.k;
    h.n_wrap = o.n_wrap ? o.n_wrap : nw_t;
    size_t sm;
    // the FP64 recompute works in shared memory when its workspace fits next to the head;
    // the delayed path always inverts its HBM workspace by panels
    h.gj_smem = o.precision != HFQMC_F32_DELAYED && o.gj_smem >= 0 &&
                gj_smem_bytes(h.L) + 4 * (size_t)h.L * 8 + 1024 <= kSmemMax;
    h.refine = o.precision == HFQMC_F32_DELAYED && o.recompute != HFQMC_RECOMPUTE_GJ;
    if (o.precision == HFQMC_F32_DELAYED) {
      if (h.L > 512) {
        g_create_error = "the delayed path handles Lambda <= 512 (two rows per thread)";
        hfqmc_destroy(c);
        return HFQMC_EINVAL;
      }
      // the panels of both spins must fit in shared memory: lower k if needed
      while (h.k > 8 && delayed_smem(h.L, h.k, false, h.gj_smem, false, 1, h.refine) > kSmemMax) h.k -= 8;
      if (delayed_smem(h.L, h.k, false, h.gj_smem, false, 1, h.refine) > kSmemMax) {
        g_create_error = "Lambda too large for the delayed path's shared-memory panels";
        hfqmc_destroy(c);
        return HFQMC_EINVAL;
      }
      // staging two U blocks per flush group when it fits, else one
      h.ub = delayed_smem(h.L, h.k, false, h.gj_smem, false, 2, h.refine) <= kSmemMax ? 2 : 1;
      // residency is decided on the sweep's own layout; the refinement's
      // staging overlays it and may extend it up to the cap
      sm = delayed_smem(h.L, h.k, true, h.gj_smem, false, h.ub, h.refine);
      h.resident = delayed_smem(h.L, h.k, true, h.gj_smem, false, h.ub, false) <= kResidentBudget && sm <= kSmemMax;
      h.gtile = 0;
      if (!h.resident) {
        // flush by TMA reduce-add: G rows must be 16-byte aligned (Lambda % 4
        // == 0), the 64 KiB product buffers must fit (k is lowered for them
        // down to 8; at each k two staged U blocks are preferred, one
        // accepted), the driver must encode the tensor map
        if (o.flush != HFQMC_FLUSH_FFMA && h.L % 4 == 0 && o.gtile >= 0 &&
            tensor_map_encoder() != nullptr) {
          for (int kt = h.k; kt >= 8 && !h.gtile; kt -= 8)
            for (int ub = 2; ub >= 1 && !h.gtile; --ub)
              if (delayed_smem(h.L, kt, false, h.gj_smem, true, ub, h.refine) <= kSmemMax) {
                h.k = kt;
                h.ub = ub;
                h.gtile = 1;
              }
        }
        if (!h.gtile)
          h.ub = delayed_smem(h.L, h.k, false, h.gj_smem, false, 2, h.refine) <= kSmemMax ? 2 : 1;
        sm = delayed_smem(h.L, h.k, false, h.gj_smem, h.gtile != 0, h.ub, h.refine);
      }
    } else {
      sm = rank1_smem(h.L, true, f64, h.gj_smem);
      h.resident = sm <= kResidentBudget;
      if (!h.resident) sm = rank1_smem(h.L, false, f64, h.gj_smem);
    }
    smem_max = std::max(smem_max, sm);
    h.out_off = out_off;
    out_off += h.L + 1;
    GridConst& q = c->gc[g];
    q.L = h.L;
    q.chains = h.chains;
    q.item0 = h.item0;
    q.resident = h.resident;
    q.k = h.k;
    q.n_wrap = h.n_wrap;
    q.gj_smem = h.gj_smem;
    q.gtile = h.gtile;
    q.ub = h.ub;
    q.lambda = h.lambda;
    q.delta[0] = std::exp(-2.0 * h.lambda) - 1.0;
    q.delta[1] = std::exp(2.0 * h.lambda) - 1.0;
    q.dV[0] = std::exp(h.lambda) - 1.0;
    q.dV[1] = std::exp(-h.lambda) - 1.0;
    q.deltaf[0] = (float)q.delta[0];
    q.deltaf[1] = (float)q.delta[1];
    q.M = nullptr;
    q.Minv = nullptr;
    q.tmapG = nullptr;
    q.rc = nullptr;
    q.ph = 0;
    q.pad2 = 0;
  }

  // device memory: one pool, grid-major per category
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o2 = off;
    off += align256(bytes);
    return o2;
  };
  std::vector<size_t> offM(n_grids), offG0(n_grids), offMinv(n_grids), offRc(n_grids), offAsl(n_grids);
  for (int g = 0; g < n_grids; ++g) {
    offM[g] = take(sizeof(double) * (size_t)c->gh[g].L * c->gh[g].L);
    offG0[g] = take(sizeof(double) * (size_t)c->gh[g].L);
  }
  for (int g = 0; g < n_grids; ++g) offMinv[g] = take(sizeof(double) * (size_t)c->gh[g].L * c->gh[g].L);
  for (int g = 0; g < n_grids; ++g)
    if (c->gh[g].refine) {
      offRc[g] = take(sizeof(RefineConst));
      offAsl[g] = take(rf_aslc_bytes(c->gh[g].L));
    }
  struct ItemOff {
    size_t s, G, ws, acc, bins, accD, cnt;
  };
  std::vector<ItemOff> io(c->n_items);
  for (int g = 0; g < n_grids; ++g) {
    const size_t L = c->gh[g].L;
    for (int ch = 0; ch < c->gh[g].chains; ++ch) {
      ItemOff& x = io[c->gh[g].item0 + ch];
      x.G = take(2 * L * L * es);
    }
  }
  // workspace, accumulators and counters after the matrices, grid-major
  for (int i = 0; i < c->n_items; ++i) {
    int g = 0;
    while (g + 1 < n_grids && c->gh[g + 1].item0 <= i) ++g;
    const size_t L = c->gh[g].L;
    const size_t ws = sizeof(double) * 2 * L * L;
    io[i].ws = take(c->gh[g].refine && rf_ws_bytes((int)L) > ws ? rf_ws_bytes((int)L) : ws);
  }
  const size_t acc_begin = off;
  std::vector<size_t> acc_grid_begin(n_grids + 1);
  for (int g = 0; g < n_grids; ++g) {
    acc_grid_begin[g] = off;
    const size_t L = c->gh[g].L;
    for (int ch = 0; ch < c->gh[g].chains; ++ch) {
      ItemOff& x = io[c->gh[g].item0 + ch];
      x.s = take(L);
      x.acc = take(sizeof(double) * 2 * L);
      x.bins = take(sizeof(double) * kBins * L);
      x.accD = take(sizeof(double) * (1 + kBins));
      x.cnt = take(sizeof(ChainCounters));
    }
  }
  acc_grid_begin[n_grids] = off;
  const size_t pool_bytes = off;
  c->d_pool = (unsigned char*)dev_alloc(c, pool_bytes);
  c->d_grids = (GridConst*)dev_alloc(c, sizeof(GridConst) * n_grids);
  c->d_items = (ItemPtrs*)dev_alloc(c, sizeof(ItemPtrs) * c->n_items);
  c->d_order = (int*)dev_alloc(c, sizeof(int) * c->n_items);
  c->d_queue = (int*)dev_alloc(c, sizeof(int));
  c->d_status = (int*)dev_alloc(c, sizeof(int));
  c->d_account = (GridAccount*)dev_alloc(c, sizeof(GridAccount) * n_grids);
  c->d_gout = (GridOut*)dev_alloc(c, sizeof(GridOut) * n_grids);
  c->d_outG = (double*)dev_alloc(c, sizeof(double) * out_off);
  c->d_outErr = (double*)dev_alloc(c, sizeof(double) * out_off);
  c->d_out_off = (long long*)dev_alloc(c, sizeof(long long) * n_grids);
  c->d_tmaps = (CUtensorMap*)dev_alloc(c, sizeof(CUtensorMap) * n_grids);
  if (!c->d_tmaps || !c->d_pool || !c->d_grids || !c->d_items || !c->d_order || !c->d_queue || !c->d_status ||
      !c->d_account || !c->d_gout || !c->d_outG || !c->d_outErr || !c->d_out_off)
    return bail(fail(c, HFQMC_ENOMEM, "device allocation failed (" +
                                          std::to_string(pool_bytes >> 20) + " MiB pool)"));
  if ((e = cudaMallocHost(&c->h_gout, sizeof(GridOut) * n_grids)) != cudaSuccess ||
      (e = cudaMallocHost(&c->h_status, sizeof(int))) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMallocHost"));
  (void)acc_begin;

  std::vector<RefineConst> rcs;
  for (int g = 0; g < n_grids; ++g) {
    c->gc[g].M = (const double*)(c->d_pool + offM[g]);
    c->gc[g].Minv = (const double*)(c->d_pool + offMinv[g]);
    c->gc[g].rc = nullptr;
    if (c->gh[g].refine) {
      // the field-independent parts; ea and the slices come with each bath (set_G0)
      const int L = c->gh[g].L;
      const double lam = c->gh[g].lambda;
      RefineConst r;
      std::memset(&r, 0, sizeof(r));
      c->gh[g].d_aslc = (uint16_t*)(c->d_pool + offAsl[g]);
      r.aslc = c->gh[g].d_aslc;
      r.nrb = (L + 127) / 128;
      r.nkc = (L + kRfKC - 1) / kRfKC;
      r.emax_step = o.refine_max == 0.0 ? 0.00390625f : (o.refine_max < 0.0 ? -1.f : (float)o.refine_max);
      r.nN = (L + 79) / 80 * 80 < (L + 63) / 64 * 64 ? 80 : 64;
      r.cplus[0] = (float)std::exp(lam);
      r.cplus[1] = (float)std::exp(-lam);
      for (int v = 0; v < 2; ++v) {
        const double cm = std::exp(v == 0 ? -lam : lam);
        r.cminus_hi[v] = (float)cm;
        r.cminus_lo[v] = (float)(cm - (double)r.cminus_hi[v]);
      }
      RefineConst* dr = (RefineConst*)(c->d_pool + offRc[g]);
      if ((e = cudaMemcpyAsync(dr, &r, sizeof(r), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
        return bail(cuda_fail(c, e, "cudaMemcpyAsync"));
      c->gc[g].rc = dr;
    }
  }
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamSynchronize"));
  // tensor maps of the TMA reduce flush: the FP32 G of all chains of a grid,
  // dims {column, row, spin, chain} (the chains' G blocks are consecutive
  // takes of the pool, a constant stride apart), box 128 x 64 x 1 x 1 (half a
  // flush tile)
  std::vector<CUtensorMap> tmaps(n_grids);
  std::memset(tmaps.data(), 0, sizeof(CUtensorMap) * n_grids);
  for (int g = 0; g < n_grids; ++g) {
    GridHost& h = c->gh[g];
    if (!h.gtile) continue;
    const cuuint64_t L = (cuuint64_t)h.L;
    const cuuint64_t dims[4] = {L, L, 2, (cuuint64_t)h.chains};
    const cuuint64_t strides[3] = {L * 4, L * L * 4, (cuuint64_t)align256(2 * L * L * 4)};
    const cuuint32_t box[4] = {(cuuint32_t)kDelayedTile, (cuuint32_t)kDelayedTile / 2, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    void* base = c->d_pool + io[h.item0].G;
    if (h.chains > 1 && io[h.item0 + 1].G - io[h.item0].G != strides[2]) h.gtile = 0;
    if (h.gtile &&
        tensor_map_encoder()(&tmaps[g], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      h.gtile = 0;
    c->gc[g].gtile = h.gtile;
    c->gc[g].tmapG = h.gtile ? (const void*)(c->d_tmaps + g) : nullptr;
  }
  // the G_up-only sweep's layout: one spin's panels and partial sums leave
  // room for a deeper delay (up to the k asked for) on grids whose G stays in
  // HBM; residency and the flush kind stay those of the two-spin layout
  for (int g = 0; g < n_grids; ++g) {
    GridHost& h = c->gh[g];
    h.k1 = h.k;
    h.ub1 = h.ub;
    if (o.precision != HFQMC_F32_DELAYED || h.resident) continue;
    for (int kt = h.k_req; kt > h.k && h.k1 == h.k; kt -= 8)
      for (int ub = 2; ub >= 1 && h.k1 == h.k; --ub)
        if (delayed_smem(h.L, kt, false, h.gj_smem, h.gtile != 0, ub, h.refine, 1) <= kSmemMax) {
          h.k1 = kt;
          h.ub1 = ub;
        }
  }
  if ((e = cudaMemcpyAsync(c->d_tmaps, tmaps.data(), sizeof(CUtensorMap) * n_grids, cudaMemcpyHostToDevice,
                           c->stream)) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMemcpyAsync"));
  c->items.resize(c->n_items);
  for (int g = 0; g < n_grids; ++g)
    for (int ch = 0; ch < c->gh[g].chains; ++ch) {
      const int i = c->gh[g].item0 + ch;
      ItemPtrs& p = c->items[i];
      p.grid = g;
      p.chain = ch;
      p.L = c->gh[g].L;
      p.pad = 0;
      p.s = (int8_t*)(c->d_pool + io[i].s);
      p.G = (void*)(c->d_pool + io[i].G);
      p.ws = (double*)(c->d_pool + io[i].ws);
      p.acc = (double*)(c->d_pool + io[i].acc);
      p.bins = (double*)(c->d_pool + io[i].bins);
      p.accD = (double*)(c->d_pool + io[i].accD);
      p.cnt = (ChainCounters*)(c->d_pool + io[i].cnt);
      p.trace = nullptr;
    }
  // longest-Lambda-first order (stable)
  std::vector<int> order(c->n_items);
  for (int i = 0; i < c->n_items; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return c->items[x].L > c->items[y].L; });
  std::vector<long long> offs(n_grids);
  for (int g = 0; g < n_grids; ++g) offs[g] = c->gh[g].out_off;

  if ((e = cudaMemcpyAsync(c->d_grids, c->gc.data(), sizeof(GridConst) * n_grids, cudaMemcpyHostToDevice,
                     c->stream)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemcpyAsync"));
  if ((e = cudaMemcpyAsync(c->d_items, c->items.data(), sizeof(ItemPtrs) * c->n_items,
                     cudaMemcpyHostToDevice, c->stream)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemcpyAsync"));
  if ((e = cudaMemcpyAsync(c->d_order, order.data(), sizeof(int) * c->n_items, cudaMemcpyHostToDevice,
                     c->stream)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemcpyAsync"));
  if ((e = cudaMemcpyAsync(c->d_out_off, offs.data(), sizeof(long long) * n_grids,
                     cudaMemcpyHostToDevice, c->stream)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemcpyAsync"));
  if ((e = cudaMemsetAsync(c->d_pool + acc_grid_begin[0], 0, acc_grid_begin[n_grids] - acc_grid_begin[0],
                     c->stream)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemsetAsync"));
  if ((e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemsetAsync"));
  if ((e = cudaMemsetAsync(c->d_account, 0, sizeof(GridAccount) * n_grids, c->stream)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemsetAsync"));
  if ((e = cudaMemsetAsync(c->d_gout, 0, sizeof(GridOut) * n_grids, c->stream)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemsetAsync"));
  for (int g = 0; g < n_grids; ++g) c->gh[g].out_off = offs[g];

  // launch shape of the persistent sweep kernel
  int threads = 0, occ = 0, r;
  c->sweep_smem = smem_max;
  if (o.precision == HFQMC_F32_DELAYED)
    r = delayed_config(smem_max, &threads, &occ);
  else
    r = rank1_config(f64, smem_max, &threads, &occ);
  if (r) return bail(cuda_fail(c, (cudaError_t)r, "sweep kernel configuration"));
  if (occ < 1) return bail(fail(c, HFQMC_EINVAL, "sweep kernel does not fit on an SM"));
  c->sweep_ctas = std::min(c->n_items, occ * c->n_sm);
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamSynchronize(create)"));
  *out = c;
  return HFQMC_OK;
}

// Fits every grid's k and U blocks, and the sweep's shared memory, to the
// layout of the delayed kernel variant about to run (ns = 1: the G_up-only
// sweep, ns = 2: both spins), uploads the grids' constants and drops the
// cached graphs (their launches carry the old size).  Runs on the host before
// a sweep whose variant differs from the last one; a chain's panels are empty
// between calls, so its delay depth may change there.
int apply_layout(hfqmc_ctx* c, int ns) {
  size_t sm = 0;
  for (int g = 0; g < c->n_grids; ++g) {
    const GridHost& h = c->gh[g];
    sm = std::max(sm, delayed_smem(h.L, ns == 1 ? h.k1 : h.k, h.resident != 0, h.gj_smem != 0, h.gtile != 0,
                                   ns == 1 ? h.ub1 : h.ub, h.refine, ns));
  }
  int threads = 0, occ = 0;
  const int r = delayed_config(sm, &threads, &occ);
  if (r) return cuda_fail(c, (cudaError_t)r, "sweep kernel configuration");
  if (occ < 1) return fail(c, HFQMC_EINVAL, "sweep kernel does not fit on an SM");
  // the grids' constants change only once the new size is in place
  for (int g = 0; g < c->n_grids; ++g) {
    c->gc[g].k = ns == 1 ? c->gh[g].k1 : c->gh[g].k;
    c->gc[g].ub = ns == 1 ? c->gh[g].ub1 : c->gh[g].ub;
  }
  CK(cudaMemcpyAsync(c->d_grids, c->gc.data(), sizeof(GridConst) * c->n_grids, cudaMemcpyHostToDevice,
                     c->stream));
  c->sweep_smem = sm;
  c->sweep_ctas = std::min(c->n_items, occ * c->n_sm);
  drop_graphs(c);
  c->layout_ns = ns;
  return HFQMC_OK;
}

int check_status(hfqmc_ctx* c) {
  if (*c->h_status & kStatusSingular)
    return fail(c, HFQMC_ENUMERIC, "zero pivot in an FP64 Gauss-Jordan recompute");
  if (*c->h_status & kStatusNonFinite)
    return fail(c, HFQMC_ENUMERIC, "non-finite Green matrix after a recompute");
  if (*c->h_status & kStatusTimeout)
    return fail(c, HFQMC_ETIMEOUT, "a bounded device wait gave up");
  return HFQMC_OK;
}

}  // namespace

extern "C" {

void hfqmc_default_opts(hfqmc_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = HFQMC_F32_DELAYED;
  o->k = 0;
  o->n_wrap = 0;
  o->accept_rule = HFQMC_METROPOLIS;
  o->drift_warn = 1e-6;
  o->drift_fail = 1e-1;  // a guard: the FP32 drift at the table's N_wrap reaches a few 1e-2
  o->cuda_stream = nullptr;
  o->autotune = 1;
  o->flush = HFQMC_FLUSH_AUTO;
  o->use_graph = 1;
  o->recompute = HFQMC_RECOMPUTE_AUTO;
}

int hfqmc_create(hfqmc_ctx** out, double beta, double U, const double* dtau, int n_grids,
                 const int* chains_per_grid, uint64_t seed, const hfqmc_opts* opts) {
  return create_impl(out, beta, &U, false, dtau, n_grids, chains_per_grid, seed, opts);
}

int hfqmc_create_ex(hfqmc_ctx** out, double beta, const double* U, const double* dtau,
                    int n_grids, const int* chains_per_grid, uint64_t seed,
                    const hfqmc_opts* opts) {
  return create_impl(out, beta, U, true, dtau, n_grids, chains_per_grid, seed, opts);
}

int hfqmc_set_G0(hfqmc_ctx* c, int grid, const double* G0_tau) {
  if (!c) return fail(nullptr, HFQMC_EINVAL, "ctx is NULL");
  if (grid < 0 || grid >= c->n_grids) return fail(c, HFQMC_EINVAL, "grid out of range");
  if (!G0_tau) return fail(c, HFQMC_EINVAL, "G0_tau is NULL");
  GridHost& h = c->gh[grid];
  for (int k = 0; k < h.L; ++k)
    if (!std::isfinite(G0_tau[k])) return fail(c, HFQMC_EINVAL, "G0_tau holds a non-finite value");
  // particle-hole symmetric bath (M + M^T = 1): G0(tau_k) = G0(beta - tau_k) and
  // G0(0+) = -1/2, to 1e-12 (a Matsubara sum gives ~1e-13; the mirrored G_dn
  // then differs from the exact one by ~1e-12 x the condition of G^{-1},
  // far below FP32 rounding)
  int ph = 0;
  if (c->opts.ph_symmetry >= 0 && c->opts.precision == HFQMC_F32_DELAYED) {
    double dev = std::fabs(G0_tau[0] + 0.5);
    for (int k = 1; k < h.L; ++k) dev = std::max(dev, std::fabs(G0_tau[k] - G0_tau[h.L - k]));
    ph = dev <= 1e-12;
  }
  if (ph != c->gc[grid].ph) {
    const int was = sweep_mirrors(c);
    c->gc[grid].ph = ph;
    if (sweep_mirrors(c) != was) drop_graphs(c);  // the sweep's kernel variant changes
    CK(cudaMemcpyAsync(c->d_grids + grid, &c->gc[grid], sizeof(GridConst), cudaMemcpyHostToDevice, c->stream));
  }
  double* dM = const_cast<double*>(c->gc[grid].M);
  double* dG0 = (double*)((unsigned char*)dM + align256(sizeof(double) * (size_t)h.L * h.L));
  CK(cudaMemcpyAsync(dG0, G0_tau, sizeof(double) * h.L, cudaMemcpyHostToDevice, c->stream));
  int r = launch_bath_matrix(h.L, dG0, dM, c->stream);
  if (r) return cuda_fail(c, (cudaError_t)r, "bath matrix kernel");
  // M^{-1} (closed form of a skew-circulant matrix) for the recompute through G^{-1}
  r = launch_bath_inverse(h.L, dM, const_cast<double*>(c->gc[grid].Minv), c->d_status, c->stream);
  if (r) return cuda_fail(c, (cudaError_t)r, "bath inverse kernel");
  if (c->gc[grid].rc) {
    // the refinement's slices of A = M^{-1} - diag(...) for this bath
    RefineConst* rc = const_cast<RefineConst*>(c->gc[grid].rc);
    r = launch_refine_prep(h.L, c->gc[grid].Minv, h.lambda, rc, h.d_aslc, c->stream);
    if (r) return cuda_fail(c, (cudaError_t)r, "refinement slice kernel");
  }
  SweepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.grids = c->d_grids;
  a.items = c->d_items;
  a.status = c->d_status;
  a.seed = c->seed;
  r = launch_init_chains(a, c->d_grids + grid, h.item0, h.chains, h.L, f64_path(c), !h.ever_set,
                         h.gj_smem != 0, c->stream);
  if (r) return cuda_fail(c, (cudaError_t)r, "init kernel");
  CK(cudaMemsetAsync(c->d_account + grid, 0, sizeof(GridAccount), c->stream));
  CK(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  r = check_status(c);
  if (r) return r;
  h.g0_set = true;
  h.ever_set = true;
  return HFQMC_OK;
}

int hfqmc_sweep(hfqmc_ctx* c, int64_t n_warm, int64_t n_meas) {
  if (!c) return fail(nullptr, HFQMC_EINVAL, "ctx is NULL");
  if (n_warm < 0 || n_meas < 0) return fail(c, HFQMC_EINVAL, "negative sweep count");
  if (n_warm + n_meas > (1ll << 31)) return fail(c, HFQMC_EINVAL, "too many sweeps in one call");
  for (int g = 0; g < c->n_grids; ++g)
    if (!c->gh[g].g0_set)
      return fail(c, HFQMC_ESTATE, "hfqmc_set_G0 has not been called for grid " + std::to_string(g));
  if (c->trace_mode != kTraceOff && n_warm + n_meas > c->trace_cap)
    return fail(c, HFQMC_EINVAL, "more sweeps than the decision trace holds (hfqmc_set_trace)");
  if (c->opts.precision == HFQMC_F32_DELAYED) {
    const int ns = launch_mirrors(c) ? 1 : 2;
    if (ns != c->layout_ns) {
      const int r = apply_layout(c, ns);
      if (r) return r;
    }
  }
  CK(cudaEventRecord(c->ev0, c->stream));
  if (c->opts.use_graph) {
    auto key = std::make_pair((long long)n_warm, (long long)n_meas);
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
      if (c->graphs.size() >= kMaxGraphs) {
        auto lru = c->graphs.begin();
        for (auto g = c->graphs.begin(); g != c->graphs.end(); ++g)
          if (g->second.used < lru->second.used) lru = g;
        cudaGraphExecDestroy(lru->second.exec);
        c->graphs.erase(lru);
      }
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      int r = enqueue_sweep(c, n_warm, n_meas);
      cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
      if (r) return r;
      if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
      cudaGraphExec_t ex;
      cudaError_t e3 = cudaGraphInstantiate(&ex, graph, 0);
      cudaGraphDestroy(graph);
      if (e3 != cudaSuccess) return cuda_fail(c, e3, "cudaGraphInstantiate");
      it = c->graphs.emplace(key, hfqmc_ctx::CachedGraph{ex, 0}).first;
    }
    it->second.used = ++c->graph_clock;
    CK(cudaGraphLaunch(it->second.exec, c->stream));
  } else {
    int r = enqueue_sweep(c, n_warm, n_meas);
    if (r) return r;
  }
  CK(cudaEventRecord(c->ev1, c->stream));
  CK(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  c->last_ms = ms;
  c->sweeps_done += n_warm + n_meas;
  int r = check_status(c);
  if (r) return r;
  if (c->opts.drift_fail > 0.0)
    for (int g = 0; g < c->n_grids; ++g)
      if (c->h_gout[g].drift > c->opts.drift_fail) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "drift %.3e exceeds drift_fail %.3e on grid %d",
                      c->h_gout[g].drift, c->opts.drift_fail, g);
        return fail(c, HFQMC_EDRIFT, buf);
      }
  return HFQMC_OK;
}

int hfqmc_get_G(hfqmc_ctx* c, int grid, double* G_tau, double* G_err) {
  if (!c) return fail(nullptr, HFQMC_EINVAL, "ctx is NULL");
  if (grid < 0 || grid >= c->n_grids) return fail(c, HFQMC_EINVAL, "grid out of range");
  if (!G_tau) return fail(c, HFQMC_EINVAL, "G_tau is NULL");
  const GridHost& h = c->gh[grid];
  if (!h.g0_set) return fail(c, HFQMC_ESTATE, "no G0 set for this grid");
  CK(cudaMemcpyAsync(G_tau, c->d_outG + h.out_off, sizeof(double) * (h.L + 1),
                     cudaMemcpyDeviceToHost, c->stream));
  if (G_err)
    CK(cudaMemcpyAsync(G_err, c->d_outErr + h.out_off, sizeof(double) * (h.L + 1),
                       cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return HFQMC_OK;
}

int hfqmc_get_D(hfqmc_ctx* c, int grid, double* D, double* D_err) {
  if (!c) return fail(nullptr, HFQMC_EINVAL, "ctx is NULL");
  if (grid < 0 || grid >= c->n_grids) return fail(c, HFQMC_EINVAL, "grid out of range");
  GridOut o;
  CK(cudaMemcpyAsync(&o, c->d_gout + grid, sizeof(GridOut), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (D) *D = o.D;
  if (D_err) *D_err = o.D_err;
  return HFQMC_OK;
}

int hfqmc_get_stats(hfqmc_ctx* c, int grid, hfqmc_stats* out) {
  if (!c) return fail(nullptr, HFQMC_EINVAL, "ctx is NULL");
  if (grid < 0 || grid >= c->n_grids || !out) return fail(c, HFQMC_EINVAL, "bad argument");
  GridOut o;
  CK(cudaMemcpyAsync(&o, c->d_gout + grid, sizeof(GridOut), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const GridHost& h = c->gh[grid];
  out->L = h.L;
  out->chains = h.chains;
  out->k = c->gc[grid].k;  // the layout of the last sweep's kernel variant
  out->n_wrap = h.n_wrap;
  out->sweeps = c->sweeps_done;
  out->proposals = o.proposals;
  out->accepted = o.accepted;
  out->recomputes = o.recomputes;
  out->numeric_errors = o.bad;
  out->accept_rate = o.proposals ? (double)o.accepted / (double)o.proposals : 0.0;
  out->drift_max = o.drift;
  out->last_sweep_ms = c->last_ms;
  out->recompute_fallbacks = o.fallbacks;
  out->ph_symmetric = c->gc[grid].ph;
  return HFQMC_OK;
}

int hfqmc_grid_size(hfqmc_ctx* c, int grid, int* L) {
  if (!c) return fail(nullptr, HFQMC_EINVAL, "ctx is NULL");
  if (grid < 0 || grid >= c->n_grids || !L) return fail(c, HFQMC_EINVAL, "bad argument");
  *L = c->gh[grid].L;
  return HFQMC_OK;
}

int hfqmc_get_chain(hfqmc_ctx* c, int grid, int chain, int8_t* s, double* G_up, double* G_dn,
                    int64_t* counters, double* acc) {
  if (!c) return fail(nullptr, HFQMC_EINVAL, "ctx is NULL");
  if (grid < 0 || grid >= c->n_grids) return fail(c, HFQMC_EINVAL, "grid out of range");
  const GridHost& h = c->gh[grid];
  if (chain < 0 || chain >= h.chains) return fail(c, HFQMC_EINVAL, "chain out of range");
  const ItemPtrs& p = c->items[h.item0 + chain];
  const size_t L = h.L, LL = L * L;
  if (s) CK(cudaMemcpyAsync(s, p.s, L, cudaMemcpyDeviceToHost, c->stream));
  std::vector<float> tmp;
  if (G_up || G_dn) {
    if (f64_path(c)) {
      if (G_up) CK(cudaMemcpyAsync(G_up, p.G, LL * 8, cudaMemcpyDeviceToHost, c->stream));
      if (G_dn)
        CK(cudaMemcpyAsync(G_dn, (double*)p.G + LL, LL * 8, cudaMemcpyDeviceToHost, c->stream));
    } else {
      tmp.resize(2 * LL);
      CK(cudaMemcpyAsync(tmp.data(), p.G, 2 * LL * 4, cudaMemcpyDeviceToHost, c->stream));
    }
  }
  ChainCounters cc;
  CK(cudaMemcpyAsync(&cc, p.cnt, sizeof(cc), cudaMemcpyDeviceToHost, c->stream));
  if (acc) CK(cudaMemcpyAsync(acc, p.acc, 2 * L * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (!tmp.empty()) {
    if (G_up)
      for (size_t e = 0; e < LL; ++e) G_up[e] = tmp[e];
    if (G_dn)
      for (size_t e = 0; e < LL; ++e) G_dn[e] = tmp[LL + e];
  }
  if (counters) {
    counters[0] = cc.proposals;
    counters[1] = cc.accepted;
    counters[2] = cc.recomputes;
    counters[3] = (int64_t)cc.hash;
    counters[4] = cc.bad;
    counters[5] = cc.t;
  }
  return HFQMC_OK;
}

int hfqmc_get_chain_D(hfqmc_ctx* c, int grid, int chain, double* D_sum, double* D_bins) {
  if (!c) return fail(nullptr, HFQMC_EINVAL, "ctx is NULL");
  if (grid < 0 || grid >= c->n_grids) return fail(c, HFQMC_EINVAL, "grid out of range");
  const GridHost& h = c->gh[grid];
  if (chain < 0 || chain >= h.chains) return fail(c, HFQMC_EINVAL, "chain out of range");
  const ItemPtrs& p = c->items[h.item0 + chain];
  double buf[1 + kBins];
  CK(cudaMemcpyAsync(buf, p.accD, sizeof(buf), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (D_sum) *D_sum = buf[0];
  if (D_bins) std::memcpy(D_bins, buf + 1, sizeof(double) * kBins);
  return HFQMC_OK;
}

int hfqmc_set_trace(hfqmc_ctx* c, int mode, int64_t max_sweeps) {
  if (!c) return fail(nullptr, HFQMC_EINVAL, "ctx is NULL");
  if (mode != HFQMC_TRACE_OFF && mode != HFQMC_TRACE_RECORD && mode != HFQMC_TRACE_REPLAY)
    return fail(c, HFQMC_EINVAL, "unknown trace mode");
  if (mode == HFQMC_TRACE_REPLAY && c->opts.precision == HFQMC_F32_DELAYED)
    return fail(c, HFQMC_EINVAL, "replay runs on the rank-1 paths (F64_RANK1, F32_RANK1)");
  if (mode != HFQMC_TRACE_OFF && (max_sweeps < 1 || max_sweeps > (1ll << 31)))
    return fail(c, HFQMC_EINVAL, "max_sweeps must be in [1, 2^31]");
  drop_graphs(c);  // the launch (kernel variant and its arguments) changes
  if (mode == HFQMC_TRACE_OFF) {
    for (auto& p : c->items) p.trace = nullptr;
    c->trace_mode = kTraceOff;
  } else {
    std::vector<size_t> off(c->n_grids);
    size_t words = 0;
    for (int g = 0; g < c->n_grids; ++g) {
      off[g] = words;
      words += (size_t)c->gh[g].chains * (size_t)max_sweeps * trace_words(c->gh[g].L);
    }
    const size_t bytes = words * sizeof(uint32_t);
    if (bytes > c->trace_bytes) {
      CK(cudaStreamSynchronize(c->stream));
      dev_free(c, c->d_trace);
      c->d_trace = nullptr;
      c->trace_bytes = 0;
      c->d_trace = (uint32_t*)dev_alloc(c, bytes);
      if (!c->d_trace) return fail(c, HFQMC_ENOMEM, "device allocation of the decision trace failed");
      c->trace_bytes = bytes;
    }
    CK(cudaMemsetAsync(c->d_trace, 0, c->trace_bytes, c->stream));
    c->trace_off = off;
    c->trace_cap = max_sweeps;
    for (int g = 0; g < c->n_grids; ++g)
      for (int ch = 0; ch < c->gh[g].chains; ++ch)
        c->items[c->gh[g].item0 + ch].trace =
            c->d_trace + off[g] + (size_t)ch * (size_t)max_sweeps * trace_words(c->gh[g].L);
    c->trace_mode = mode == HFQMC_TRACE_RECORD ? kTraceRecord : kTraceReplay;
  }
  CK(cudaMemcpyAsync(c->d_items, c->items.data(), sizeof(ItemPtrs) * c->n_items, cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return HFQMC_OK;
}

// Shared checks of hfqmc_get_trace / hfqmc_put_trace; the grid's trace bytes
// and device address on success.
static int trace_span(hfqmc_ctx* c, int grid, int64_t n_words, size_t* bytes, uint32_t** dev) {
  if (!c) return fail(nullptr, HFQMC_EINVAL, "ctx is NULL");
  if (grid < 0 || grid >= c->n_grids) return fail(c, HFQMC_EINVAL, "grid out of range");
  if (c->trace_mode == kTraceOff) return fail(c, HFQMC_ESTATE, "no decision trace (hfqmc_set_trace)");
  const size_t w = (size_t)c->gh[grid].chains * (size_t)c->trace_cap * trace_words(c->gh[grid].L);
  if (n_words < 0 || (size_t)n_words != w)
    return fail(c, HFQMC_EINVAL, "n_words must be chains x max_sweeps x ceil(Lambda/32) = " + std::to_string(w));
  *bytes = w * sizeof(uint32_t);
  *dev = c->d_trace + c->trace_off[grid];
  return HFQMC_OK;
}

int hfqmc_get_trace(hfqmc_ctx* c, int grid, uint32_t* bits, int64_t n_words) {
  size_t bytes = 0;
  uint32_t* dev = nullptr;
  int r = trace_span(c, grid, n_words, &bytes, &dev);
  if (r) return r;
  if (!bits) return fail(c, HFQMC_EINVAL, "bits is NULL");
  CK(cudaMemcpyAsync(bits, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return HFQMC_OK;
}

int hfqmc_put_trace(hfqmc_ctx* c, int grid, const uint32_t* bits, int64_t n_words) {
  size_t bytes = 0;
  uint32_t* dev = nullptr;
  int r = trace_span(c, grid, n_words, &bytes, &dev);
  if (r) return r;
  if (!bits) return fail(c, HFQMC_EINVAL, "bits is NULL");
  CK(cudaMemcpyAsync(dev, bits, bytes, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return HFQMC_OK;
}

const char* hfqmc_last_error(const hfqmc_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

void hfqmc_destroy(hfqmc_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  for (void* p : c->allocs) {
    if (c->opts.alloc && c->opts.free)
      c->opts.free(p, c->opts.alloc_user);
    else if (!c->opts.alloc)
      cudaFree(p);
  }
  if (c->h_gout) cudaFreeHost(c->h_gout);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
