/*
 * hfqmc.h -- C ABI of the GB300 Hirsch-Fye QMC sweep library (libhfqmc.so).
 *
 * The library solves the fixed-bath impurity problem of the paper's
 * "Multigrid HF-QMC method" section: for one bath Green function G0 it runs
 * Hirsch-Fye QMC on several imaginary-time grids dtau_i at once, with many
 * independent Markov chains per grid (the paper averages each grid's Green
 * function over 10 to 20 independent impurity solutions), and returns the
 * measured G(tau) with error bars per grid.  The dtau -> 0 extrapolation, Fourier transforms
 * and the DMFT self-consistency are host-side glue above this ABI.
 *
 * Method (introduction of the paper: Trotter slicing into Lambda = beta/dtau
 * slices, binary Hubbard-Stratonovich field s_l = +-1, Monte Carlo sampling;
 * equations of Hirsch & Fye 1986, which the paper cites for the method):
 *   cosh(lambda) = exp(dtau U / 2),  V^sigma_l = sigma lambda s_l,
 *   G^sigma = [1 + (1 - G0)(e^{V^sigma} - 1)]^{-1} G0,
 *   flip ratio R = R^up R^dn,  R^sigma = 1 + (1 - G^sigma_ll) Delta^sigma_l,
 *   Delta^sigma_l = e^{-2 sigma lambda s_l} - 1,
 *   accepted flip: G'_ij = G_ij + (G_il - delta_il) Delta G_lj / R^sigma.
 * Matrices use the positive convention g_ll' = <T c(tau_l) c^+(tau_l')> with
 * g_ll = 1 - n; the returned physical G(tau) = -g(tau).
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter
 * (l, sweep, chain, grid) for the proposal at slice l; u = 53-bit uniform from
 * output words 0 and 1.  Initial field: s_l = +1 iff bit 0 of word 0 of the
 * counter (l | 2^16, 0, chain, grid) is set.
 *
 * Conventions for every call:
 *  - Return value: HFQMC_OK (0) or a negative HFQMC_E* code; the message is
 *    then available from hfqmc_last_error(ctx).
 *  - Host arrays are owned by the caller and only read/written during the
 *    call; the library copies what it keeps.  Device memory belongs to the
 *    context (optionally obtained through caller-supplied allocator hooks).
 *  - One context per host thread; calls on one context must not overlap.
 *  - All device work is ordered on the context's CUDA stream.
 */
#ifndef HFQMC_H
#define HFQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HFQMC_OK        0
#define HFQMC_EINVAL   (-1) /* bad argument (beta/dtau not integral, grid out of range, ...) */
#define HFQMC_ENOMEM   (-2) /* device or host allocation failed */
#define HFQMC_ECUDA    (-3) /* a CUDA call failed (message holds the CUDA error string) */
#define HFQMC_ESTATE   (-4) /* call out of order (e.g. sweep before every grid has a G0) */
#define HFQMC_EDRIFT   (-5) /* max |G_fast - G_fresh| exceeded opts.drift_fail */
#define HFQMC_ENUMERIC (-6) /* non-finite or non-positive weight ratio, singular pivot */
#define HFQMC_ETIMEOUT (-7) /* a bounded device wait gave up */

/* ---- options ------------------------------------------------------------ */
enum {
    HFQMC_F64_RANK1 = 0,   /* FP64 G, rank-1 update per accepted flip (baseline) */
    HFQMC_F32_RANK1 = 1,   /* FP32 G, rank-1 update per accepted flip            */
    HFQMC_F32_DELAYED = 2  /* FP32 G, k accepted flips gathered into one rank-k
                              update (split-FP16 tensor-core GEMM)                */
};
enum { HFQMC_METROPOLIS = 0, HFQMC_HEAT_BATH = 1 };
enum {
    HFQMC_FLUSH_AUTO = 0,    /* tensor cores where available                    */
    HFQMC_FLUSH_TCGEN05 = 1, /* rank-k flush on tcgen05 (kind::f16, 3 passes)   */
    HFQMC_FLUSH_FFMA = 2     /* rank-k flush on FP32 FMA (CUDA cores)           */
};

typedef void *(*hfqmc_alloc_fn)(size_t bytes, void *user);
typedef void (*hfqmc_free_fn)(void *ptr, void *user);

typedef struct {
    int precision;      /* HFQMC_F64_RANK1 | HFQMC_F32_RANK1 | HFQMC_F32_DELAYED    */
    int k;              /* delay depth for F32_DELAYED (8..64, multiple of 8); 0 = per-Lambda table.
                           Lowered in steps of 8 where the panels do not fit in shared memory:
                           the two-spin sweep holds both spins' panels, the G_up-only sweep of a
                           particle-hole symmetric bath one spin's (Lambda = 500: k <= 8 and
                           <= 24); hfqmc_stats.k reports the value the last sweep ran with */
    int n_wrap;         /* FP64 recompute every n_wrap accepted flips; <0 = never; 0 = per-Lambda table
                           (F32_DELAYED: 64, the multigrid configuration's interval; rank-1 paths
                           without a tune_table: 16384 for F64_RANK1, 8192 / 16384 (Lambda > 128)
                           for F32_RANK1) */
    int accept_rule;    /* HFQMC_METROPOLIS (accept iff u < R) | HFQMC_HEAT_BATH (u (1+R) < R) */
    double drift_warn;  /* recorded only */
    double drift_fail;  /* hfqmc_sweep returns HFQMC_EDRIFT above this (<= 0: never; default 1e-1) */
    void *cuda_stream;  /* cudaStream_t to order all work on; NULL = library-owned stream */
    int autotune;       /* 1: k / n_wrap left 0 come from the per-Lambda table (the caller's
                           tune_table if given, else the built-in one measured on GB300);
                           0: they default to k = 16 and n_wrap = 1024 */
    int flush;          /* HFQMC_FLUSH_* (F32_DELAYED only) */
    int use_graph;      /* 1: replay hfqmc_sweep's launches as a captured CUDA graph */
    hfqmc_alloc_fn alloc; /* optional device allocator hook (e.g. PyTorch's caching allocator) */
    hfqmc_free_fn free;
    void *alloc_user;
    int resident_kb;    /* shared-memory budget (KiB per CTA) for keeping a chain's G on chip:
                           0 = default (200), < 0 = never (G stays in HBM/L2) */
    int gj_smem;        /* rank-1 paths and initialisation: FP64 recompute in shared memory when its
                           Lambda x Lambda workspace fits (Lambda <= 168): 0 = yes, < 0 = never (HBM
                           workspace, inverted by 16-column panels when their scratch fits).  The FP32
                           delayed path always inverts its HBM workspace by panels. */
    int gtile;          /* delayed flush with G in HBM: >= 0 = add each 128x128 product tile to G
                           by one TMA tensor reduce-add when Lambda % 4 == 0 and the 64 KiB tile
                           buffer fits (default); < 0 = per-thread adds in place */
    const int *tune_table; /* optional per-Lambda table, tune_entries triples (Lambda_max, k,
                              n_wrap) with increasing Lambda_max: a grid takes the first entry
                              with Lambda <= Lambda_max (k as for opts.k; n_wrap != 0); the
                              library copies it.  NULL / 0 entries: the built-in table.  An
                              autotuner that measures one is paper_0801_1222_gb300/autotune.py */
    int tune_entries;
    int recompute;      /* F32_DELAYED: how G is rebuilt every n_wrap accepted flips.
                           HFQMC_RECOMPUTE_AUTO (default) = REFINE for F32_DELAYED, GJ otherwise;
                           HFQMC_RECOMPUTE_GJ: from the field, FP64 Gauss-Jordan inversion of
                           G^{-1} = M^{-1}(1 + D) - D (by 16-column panels);
                           HFQMC_RECOMPUTE_REFINE: one or two Newton steps G <- G + G (1 - G^{-1} G)
                           from the current FP32 G, the residual formed from exact 7-bit integer
                           slices of M^{-1} and G on the tensor cores (FP64-level accuracy of the
                           residual), falling back to GJ when max |1 - G^{-1} G| > 2^-8 or for U = 0;
                           the result is G to FP32 rounding.  EINVAL on the rank-1 paths. */
    double refine_max;  /* REFINE: the largest max |1 - G^{-1} G| for which Newton steps are taken
                           (0 = the default 2^-8; < 0 = never, every recompute from scratch);
                           above 2^-13 a second step follows */
    int ph_symmetry;    /* F32_DELAYED, REFINE: a bath that hfqmc_set_G0 finds particle-hole
                           symmetric (G0(tau_k) = G0(beta - tau_k), G0(0+) = -1/2, to 1e-12: half
                           filling) makes G_dn = 1 - G_up^T for every field configuration.
                           0 = when every grid's bath is symmetric, the sweep keeps G_up only (G_dn's
                           diagonal, its measured G(tau) and the chain's G_dn at the end of each call
                           follow from G_up); a grid whose bath is symmetric otherwise refines G_up at
                           a recompute and sets G_dn = 1 - G_up^T;
                           1 = only the recompute uses the symmetry (the sweep updates both spins);
                           < 0 = never */
} hfqmc_opts;

enum { HFQMC_RECOMPUTE_AUTO = 0, HFQMC_RECOMPUTE_GJ = 1, HFQMC_RECOMPUTE_REFINE = 2 };

/* Per-grid statistics (hfqmc_get_stats). */
typedef struct {
    int L;                  /* Lambda = beta/dtau */
    int chains;
    int k;                  /* delay depth of the last sweep's layout (before any sweep: the
                               two-spin one; 1 for rank-1 paths) */
    int n_wrap;             /* recompute interval in use */
    int64_t sweeps;         /* sweeps done per chain since the first set_G0 */
    int64_t proposals;      /* summed over chains */
    int64_t accepted;
    int64_t recomputes;
    int64_t numeric_errors; /* proposals with R <= 0 or non-finite R */
    double accept_rate;
    double drift_max;       /* max |G_fast - G_fresh| over recomputes since set_G0 */
    double last_sweep_ms;   /* device time of the last hfqmc_sweep (whole batch) */
    int64_t recompute_fallbacks; /* recomputes the Newton refinement handed to Gauss-Jordan */
    int ph_symmetric;       /* 1: the grid's bath is particle-hole symmetric (see opts.ph_symmetry) */
} hfqmc_stats;

typedef struct hfqmc_ctx hfqmc_ctx;

/* Fills *opts with defaults: F32_DELAYED, k = 0, n_wrap = 0 (table), Metropolis,
 * drift_warn 1e-6, drift_fail 1e-1, own stream, autotune on, flush auto,
 * graphs on, no allocator hooks, recompute auto (Newton refinement on the
 * delayed path).  drift_fail guards against a broken chain: at the table's
 * N_wrap = 64 the FP32 matrix drift max|G_fast - G_fresh| stays below 1e-2
 * (maximum over chains; a few 1e-2 at intervals of 8192 or more) while G(tau)
 * stays within its 1e-5 criterion, so the default sits above that. */
void hfqmc_default_opts(hfqmc_opts *opts);

/* Creates a context for one beta and one U over n_grids dtau grids.
 * Paper: "Multigrid HF-QMC method" section -- the impurity problem for one
 * bath is solved on several grids dtau_i at once (Lambda_i = beta/dtau_i
 * slices each, the Trotter discretisation of the introduction), with 10-20
 * independent impurity solutions per grid that are averaged; here each
 * solution is one Markov chain and all chains of all grids share one launch.
 * dtau[i]: grid spacing; Lambda_i = beta/dtau_i must be an integer
 *          (|beta/dtau_i - Lambda_i| < 1e-9), 1 <= Lambda_i <= 1024.
 * chains_per_grid[i] >= 1 independent chains on grid i.
 * seed: Philox key.  opts may be NULL (defaults).
 * Allocates all device state; no kernel runs until hfqmc_set_G0.
 * On error *out is NULL and the code is returned (message via hfqmc_last_error(NULL)). */
int hfqmc_create(hfqmc_ctx **out, double beta, double U, const double *dtau, int n_grids,
                 const int *chains_per_grid, uint64_t seed, const hfqmc_opts *opts);

/* As hfqmc_create, but grid i has its own interaction U[i] (several U values
 * batched in one launch); "grid" in every other call indexes these pairs.
 * Paper: the same section, applied to the several U values of the
 * "Benchmark results" runs (U = 4 ... 5.2) at once. */
int hfqmc_create_ex(hfqmc_ctx **out, double beta, const double *U, const double *dtau,
                    int n_grids, const int *chains_per_grid, uint64_t seed,
                    const hfqmc_opts *opts);

/* Paper: the bath Green function G0 that the DMFT cycle hands to the impurity
 * solver (Fig. 1, "Multigrid HF-QMC method": the same G0 for every grid),
 * sampled on the grid, and the Hirsch-Fye Dyson equation that builds each
 * chain's G from it.
 * Sets the bath of grid `grid` from Lambda samples G0_tau[k] = G0(k dtau),
 * k = 0..Lambda-1, physical sign, G0_tau[0] = G0(0+) (host array, copied).
 * Builds the antiperiodic bath matrix M_ll' = -G0(tau_{l-l'}) (l >= l'),
 * +G0(tau_{l-l'+Lambda}) (l < l'), then for every chain of the grid computes
 * G^sigma = [1 + (1 - M)(e^V - 1)]^{-1} M by FP64 Gauss-Jordan elimination.
 * First call for a grid: the field is drawn from Philox.  Later calls keep
 * each chain's field, sweep counter and flip counters, rebuild G from the new
 * bath and zero the measurement accumulators. */
int hfqmc_set_G0(hfqmc_ctx *ctx, int grid, const double *G0_tau);

/* Paper: the Monte Carlo sampling of the binary Hubbard-Stratonovich field
 * (introduction: flips of single slices s_l, cost proportional to dtau^-3),
 * the hot path of the method; the measured G_dtau(tau) is the per-grid
 * result that the multigrid section averages and extrapolates.
 * Runs n_warm unmeasured then n_meas measured sweeps (one proposal per slice
 * l = 0..Lambda-1 in order per sweep) on every chain of every grid, as one
 * persistent launch over a longest-Lambda-first work queue.  Measured sweeps
 * accumulate g^sigma(tau_k) = (1/Lambda) sum_l sgn G^sigma_{(l+k) mod Lambda, l}
 * (sgn = -1 when l + k >= Lambda) and D = (1/Lambda) sum_l n^up_l n^dn_l.
 * Then reduces chains per grid.  Blocks until the stream is done.
 * Requires hfqmc_set_G0 on every grid (HFQMC_ESTATE otherwise). */
int hfqmc_sweep(hfqmc_ctx *ctx, int64_t n_warm, int64_t n_meas);

/* Paper: the per-grid result G_dtau_i(tau) averaged over the impurity
 * solutions ("Multigrid HF-QMC method"), the input of the dtau -> 0
 * extrapolation.
 * Measured G(tau_k), k = 0..Lambda-1, and G(beta-) = -1 - G(0+) at index Lambda
 * (caller arrays of Lambda+1 doubles; G_err may be NULL).  Error: sample
 * standard deviation (n-1) of the chain means over sqrt(n_chains); for one
 * chain the measured sweeps of each hfqmc_sweep call are cut into 32
 * consecutive bins and the same estimator is applied to the bin means. */
int hfqmc_get_G(hfqmc_ctx *ctx, int grid, double *G_tau, double *G_err);

/* Paper: the double occupancy D, the benchmark observable of the "Benchmark
 * results" section (D versus dtau^2, Figs. 3-4), at fixed dtau.
 * Double occupancy D = <n_up n_dn> and its error bar (same estimator). */
int hfqmc_get_D(hfqmc_ctx *ctx, int grid, double *D, double *D_err);

/* Per-grid counters of the sweeps (hfqmc_stats above): acceptance rate, flips,
 * recomputes, drift, device time.  The paper quotes no such figure; the
 * accept rate sets the work per proposal (the rank-1 update of the
 * introduction's dtau^-3 cost runs once per accepted flip). */
int hfqmc_get_stats(hfqmc_ctx *ctx, int grid, hfqmc_stats *out);

/* Lambda = beta/dtau of a grid (the number of imaginary-time slices). */
int hfqmc_grid_size(hfqmc_ctx *ctx, int grid, int *L);

/* One chain's state, for parity tests: field s (Lambda int8), G^up and G^dn
 * (Lambda x Lambda row-major doubles, converted from the working precision),
 * counters[6] = {proposals, accepted, recomputes, decision hash, bad-ratio
 * proposals, sweep index} and acc (2 Lambda sums of g^sigma(tau_k), spin-major).
 * The decision hash is FNV-1a 64 (offset 0xcbf29ce484222325, prime
 * 0x100000001b3) over sweep*Lambda + l of every accepted flip, in order.
 * Any output pointer may be NULL. */
int hfqmc_get_chain(hfqmc_ctx *ctx, int grid, int chain, int8_t *s, double *G_up,
                    double *G_dn, int64_t *counters, double *acc);

/* One chain's double-occupancy sums, for parity tests: *D_sum = sum over the
 * measured sweeps since the last hfqmc_set_G0 of (1/Lambda) sum_l n^up_l n^dn_l
 * with n^sigma_l = 1 - G^sigma_ll ("Benchmark results": D at fixed dtau), and
 * D_bins[32] the same sums per bin of each hfqmc_sweep call (as for G_err).
 * Either pointer may be NULL. */
int hfqmc_get_chain_D(hfqmc_ctx *ctx, int grid, int chain, double *D_sum, double *D_bins);

/* ---- decision trace: FP32 against FP64 on the same trajectory ------------
 * The paper has no counterpart; these calls state the error of the FP32
 * paths' G(tau) against FP64 along one Markov trajectory.  Two runs with the
 * same seed part ways at the first proposal whose FP32 and FP64 ratios fall
 * on different sides of its uniform, after which their chains are
 * independent; a trace fixes the trajectory instead.
 * hfqmc_set_trace(ctx, mode, max_sweeps):
 *   HFQMC_TRACE_RECORD: each later hfqmc_sweep (at most max_sweeps sweeps)
 *     records, per chain and sweep, which slices it flipped (any precision);
 *   HFQMC_TRACE_REPLAY: each later hfqmc_sweep takes its accept/reject
 *     decisions from the trace (bit set = flip) instead of u < R; ratios,
 *     flip factors, updates, recomputes and measurements run as usual (rank-1
 *     paths only: HFQMC_EINVAL for F32_DELAYED);
 *   HFQMC_TRACE_OFF: back to u < R.
 *   The trace buffer (device memory of the context) holds, per grid, chains x
 *   max_sweeps x ceil(Lambda/32) words: [chain][sweep][word], bit l % 32 of
 *   word l / 32 for slice l, sweeps counted from the start of each
 *   hfqmc_sweep call.  A call with more sweeps returns HFQMC_EINVAL.
 * hfqmc_get_trace / hfqmc_put_trace copy one grid's words out of / into that
 *   buffer (host arrays of exactly that many words, else HFQMC_EINVAL;
 *   HFQMC_ESTATE without a trace).  Replaying a trace recorded by a context
 *   with the same grids, chains, seed and bath reproduces its trajectory. */
enum { HFQMC_TRACE_OFF = 0, HFQMC_TRACE_RECORD = 1, HFQMC_TRACE_REPLAY = 2 };
int hfqmc_set_trace(hfqmc_ctx *ctx, int mode, int64_t max_sweeps);
int hfqmc_get_trace(hfqmc_ctx *ctx, int grid, uint32_t *bits, int64_t n_words);
int hfqmc_put_trace(hfqmc_ctx *ctx, int grid, const uint32_t *bits, int64_t n_words);

/* ---- entry point that allocates nothing --------------------------------
 * The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory themselves or through this library -- a host
 * runtime that hands out every device buffer from its own pool, a plugin
 * barred from the CUDA allocator, code running where cudaMalloc is not
 * allowed.  It computes what hfqmc_set_G0 computes for each chain: for one
 * HS field s the FP64 Green matrices of both spins,
 *   G^sigma = [1 + (1 - M)(e^{sigma lambda s} - 1)]^{-1} M,
 *   cosh(lambda) = exp(dtau U / 2), sigma = +1 (G_up), -1 (G_dn),
 * with M the antiperiodic bath matrix built from G0_tau as in hfqmc_set_G0,
 * by Gauss-Jordan elimination with partial pivoting.
 *
 * Arguments (all pointers are DEVICE memory owned by the caller):
 *   G0_tau  L doubles, G0(k dtau), k = 0..L-1, physical sign, G0_tau[0] = G0(0+)
 *   s       L int8 values, each +1 or -1
 *   G_up, G_dn  L x L doubles each, row-major, written
 *   cuda_stream  cudaStream_t to run on (NULL: the legacy default stream)
 *   status_out   optional host int: the device status bits of this call
 * 1 <= L <= HFQMC_NOALLOC_MAX_L; larger L returns HFQMC_EINVAL before any
 * device work.  The call returns after its work on cuda_stream is done:
 * HFQMC_OK, HFQMC_ENUMERIC (zero pivot or non-finite G), HFQMC_ECUDA.
 *
 * Memory: the bath matrix and the [A | M] workspace live in one file-scope
 * device array of 3 * HFQMC_NOALLOC_MAX_L^2 doubles (1.5 MiB) that every GPU
 * which loads the library holds until the process exits.  The call allocates
 * nothing (no cudaMalloc, no allocating library routine).  Each call looks up
 * the array's device address on the current device (cudaGetSymbolAddress),
 * copies the status word back and synchronises cuda_stream before it returns,
 * so no call of it can be captured in a CUDA graph.  Every call uses the same
 * array and leaves its contents behind (each call overwrites what it reads);
 * calls that overlap on the GPU -- from several streams or threads at once --
 * race on it and must be serialised by the caller. */
#define HFQMC_NOALLOC_MAX_L 256
int hfqmc_green_noalloc(const double *G0_tau, const int8_t *s, int L, double dtau, double U,
                        double *G_up, double *G_dn, void *cuda_stream, int *status_out);

/* Message of the last failed call on ctx (or of the last failed create when ctx is NULL). */
const char *hfqmc_last_error(const hfqmc_ctx *ctx);

/* Frees all device and host state.  NULL is ignored. */
void hfqmc_destroy(hfqmc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* HFQMC_H */
