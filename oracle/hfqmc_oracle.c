/*
 * Plain FP64 CPU oracle for the Hirsch-Fye QMC sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * only tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
 * bench.py load it.  It shares no code, header or constant table with the CUDA
 * library; both sides receive the same G0(tau) samples and seed, nothing else.
 *
 * What it computes (the paper's "Multigrid HF-QMC method" section and its
 * introduction): the impurity problem at fixed bath G0 is sliced into
 * Lambda = beta/dtau imaginary-time slices, the interaction is Trotter-decoupled
 * by a binary Hubbard-Stratonovich (HS) field s_l = +-1, and the field is
 * sampled by Monte Carlo.  The equations are the standard Hirsch-Fye ones of
 * the work the paper cites for the method (Hirsch & Fye 1986):
 *
 *   cosh(lambda) = exp(dtau U / 2),          V^sigma_l = sigma lambda s_l
 *   A^sigma      = 1 + (1 - G0)(exp(V^sigma) - 1),  G^sigma = (A^sigma)^{-1} G0
 *   flip of s_l:  Delta^sigma = exp(-2 sigma lambda s_l) - 1
 *                 R^sigma = 1 + (1 - G^sigma_ll) Delta^sigma,  R = R^up R^dn
 *   accept:       G'_ij = G_ij + (G_il - delta_il) Delta G_lj / R   (each spin)
 *
 * Matrices are in the positive convention g_ll' = <T c(tau_l) c^+(tau_l')>,
 * with the diagonal equal to g(0+) = 1 - n.  The physical Green function is
 * G(tau) = -g(tau).
 *
 * Rounding: this file must be compiled with -ffp-contract=off so that the
 * ratio R and the comparison u < R are evaluated exactly in the written order.
 *
 * Parity pins (tests/test_oracle_*.py): U = 0 gives G = G0; the atomic limit
 * reproduces its closed form; R equals the determinant ratio; a rank-1 update
 * equals a fresh inversion; G_dn = 1 - G_up^T at half filling; MC agrees with
 * brute-force enumeration of all 2^Lambda fields; detailed balance at Lambda=4.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator, written from its published        */
/* definition (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two        */
/* 32x32->64 multiplies with the Weyl key schedule.                         */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], uint64_t seed, uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu);
    uint32_t k1 = (uint32_t)(seed >> 32);
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox_many(int64_t n, const uint32_t *ctrs, uint64_t seed, uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctrs + 4 * i, seed, out + 4 * i);
}

/* 53-bit uniform in [0,1) from the first two output words. */
static double orc_u53(uint32_t x0, uint32_t x1)
{
    double hi = (double)(x0 >> 5);
    double lo = (double)(x1 >> 6);
    return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0);
}

double orc_uniform(uint32_t l, uint32_t sweep, uint32_t chain, uint32_t grid, uint64_t seed)
{
    uint32_t ctr[4] = {l, sweep, chain, grid}, x[4];
    orc_philox4x32_10(ctr, seed, x);
    return orc_u53(x[0], x[1]);
}

/* Initial HS field: s_l = +1 iff bit 0 of word 0 of Philox(l | 2^16, 0, chain, grid). */
void orc_init_field(int L, uint64_t seed, uint32_t chain, uint32_t grid, int8_t *s)
{
    for (int l = 0; l < L; ++l) {
        uint32_t ctr[4] = {(uint32_t)l | (1u << 16), 0u, chain, grid}, x[4];
        orc_philox4x32_10(ctr, seed, x);
        s[l] = (x[0] & 1u) ? (int8_t)1 : (int8_t)-1;
    }
}

/* ------------------------------------------------------------------------ */
/* Grid constants and the bath matrix                                        */
/* ------------------------------------------------------------------------ */
double orc_lambda(double dtau, double U) { return acosh(exp(0.5 * dtau * U)); }

/* M_ll' = -G0(tau_{l-l'}) for l >= l', +G0(tau_{l-l'+L}) for l < l'
 * (antiperiodic in tau; G0_tau[k] = G0(k dtau), G0_tau[0] = G0(0+)). */
void orc_bath_matrix(int L, const double *G0_tau, double *M)
{
    for (int l = 0; l < L; ++l)
        for (int lp = 0; lp < L; ++lp)
            M[(size_t)l * L + lp] = (l >= lp) ? -G0_tau[l - lp] : G0_tau[l - lp + L];
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra: textbook Doolittle LU with partial pivoting.        */
/* ------------------------------------------------------------------------ */
/* In place; returns 0 on success, -1 if a zero pivot is met.  *det_out gets
 * the determinant (sign from the row swaps times the product of pivots). */
static int orc_lu(int n, double *A, int *piv, double *det_out)
{
    double det = 1.0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = fabs(A[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (best == 0.0) { *det_out = 0.0; return -1; }
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[(size_t)k * n + j];
                A[(size_t)k * n + j] = A[(size_t)p * n + j];
                A[(size_t)p * n + j] = t;
            }
            det = -det;
        }
        double akk = A[(size_t)k * n + k];
        det *= akk;
        for (int i = k + 1; i < n; ++i) {
            double f = A[(size_t)i * n + k] / akk;
            A[(size_t)i * n + k] = f;
            for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
        }
    }
    *det_out = det;
    return 0;
}

/* Solve (LU) X = B for an n x m right-hand side, B overwritten by X. */
static void orc_lu_solve(int n, const double *LU, const int *piv, double *B, int m)
{
    for (int k = 0; k < n; ++k) {
        int p = piv[k];
        if (p != k)
            for (int j = 0; j < m; ++j) {
                double t = B[(size_t)k * m + j];
                B[(size_t)k * m + j] = B[(size_t)p * m + j];
                B[(size_t)p * m + j] = t;
            }
    }
    for (int i = 0; i < n; ++i)               /* unit lower triangle */
        for (int k = 0; k < i; ++k) {
            double f = LU[(size_t)i * n + k];
            for (int j = 0; j < m; ++j) B[(size_t)i * m + j] -= f * B[(size_t)k * m + j];
        }
    for (int i = n - 1; i >= 0; --i) {        /* upper triangle */
        for (int k = i + 1; k < n; ++k) {
            double f = LU[(size_t)i * n + k];
            for (int j = 0; j < m; ++j) B[(size_t)i * m + j] -= f * B[(size_t)k * m + j];
        }
        double d = LU[(size_t)i * n + i];
        for (int j = 0; j < m; ++j) B[(size_t)i * m + j] /= d;
    }
}

/* A^sigma(s) = 1 + (1 - M) diag(exp(sigma lambda s) - 1). */
void orc_build_A(int L, const double *M, const int8_t *s, double lambda, int sigma, double *A)
{
    for (int j = 0; j < L; ++j) {
        double dj = exp((double)sigma * lambda * (double)s[j]) - 1.0;
        for (int i = 0; i < L; ++i) {
            double one_minus_m = ((i == j) ? 1.0 : 0.0) - M[(size_t)i * L + j];
            A[(size_t)i * L + j] = ((i == j) ? 1.0 : 0.0) + one_minus_m * dj;
        }
    }
}

/* G^sigma(s) = A^{-1} M by LU; det A returned in *detA (may be NULL).
 * Returns 0 on success, -1 on a singular A. */
int orc_green(int L, const double *M, const int8_t *s, double lambda, int sigma,
              double *G, double *detA)
{
    double *A = (double *)malloc(sizeof(double) * (size_t)L * L);
    int *piv = (int *)malloc(sizeof(int) * (size_t)L);
    double det = 0.0;
    orc_build_A(L, M, s, lambda, sigma, A);
    int rc = orc_lu(L, A, piv, &det);
    if (rc == 0) {
        memcpy(G, M, sizeof(double) * (size_t)L * L);
        orc_lu_solve(L, A, piv, G, L);
    }
    if (detA) *detA = det;
    free(A);
    free(piv);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Measurement: g^sigma(tau_k) = (1/L) sum_l sgn G^sigma_{(l+k) mod L, l},  */
/* with sgn = -1 when l + k wraps past L (antiperiodicity).                 */
/* ------------------------------------------------------------------------ */
void orc_measure_g(int L, const double *G, double *g)
{
    for (int k = 0; k < L; ++k) {
        double acc = 0.0;
        for (int l = 0; l < L; ++l) {
            int r = l + k;
            double v;
            if (r >= L) v = -G[(size_t)(r - L) * L + l];
            else v = G[(size_t)r * L + l];
            acc += v;
        }
        g[k] = acc / (double)L;
    }
}

/* Double occupancy of one field configuration: (1/L) sum_l n^up_l n^dn_l,
 * n^sigma_l = 1 - G^sigma_ll (spins decouple for a fixed HS field). */
double orc_measure_D(int L, const double *Gup, const double *Gdn)
{
    double acc = 0.0;
    for (int l = 0; l < L; ++l)
        acc += (1.0 - Gup[(size_t)l * L + l]) * (1.0 - Gdn[(size_t)l * L + l]);
    return acc / (double)L;
}

/* ------------------------------------------------------------------------ */
/* One Markov chain                                                          */
/* ------------------------------------------------------------------------ */
#define ORC_FNV_PRIME 0x100000001b3ull

/* stats layout (int64 in/out):
 *   [0] proposals  [1] accepted flips (cumulative, drives N_wrap)
 *   [2] recomputes [3] decision hash (FNV-1a over t*L+l of accepted flips)
 *   [4] proposals with R <= 0 or non-finite R
 * acc   : 2*L  += g^sigma(tau_k) per measured sweep (spin-major)
 * accD  : 1    += D per measured sweep
 * bins  : 32*L += (g^up + g^dn)/2, measured sweep m of this call goes to bin
 *         floor(32 m / n_meas); may be NULL
 * hist  : 2^L  += 1 per measured sweep at index sum_l [s_l = +1] 2^l; may be NULL
 * drift : max |G_fast - G_fresh| over the recomputes of this call (in/out max)
 * Returns 0, or -1 if a recompute met a singular matrix. */
int orc_run_chain(int L, double lambda, const double *M, uint64_t seed,
                  uint32_t chain, uint32_t grid, int64_t t0, int64_t n_warm,
                  int64_t n_meas, int n_wrap, int accept_rule, int8_t *s,
                  double *Gup, double *Gdn, int64_t *stats, double *acc,
                  double *accD, double *bins, int64_t *hist, double *drift)
{
    const size_t LL = (size_t)L * L;
    double *col = (double *)malloc(sizeof(double) * (size_t)L);
    double *row = (double *)malloc(sizeof(double) * (size_t)L);
    double *gtmp = (double *)malloc(sizeof(double) * (size_t)L * 2);
    double *Gfresh = (double *)malloc(sizeof(double) * LL);
    int rc = 0;
    uint64_t hash = (uint64_t)stats[3];
    const int64_t n_sweeps = n_warm + n_meas;

    for (int64_t it = 0; it < n_sweeps && rc == 0; ++it) {
        const int64_t t = t0 + it;
        for (int l = 0; l < L; ++l) {
            double Rs[2], Ds[2];
            for (int sp = 0; sp < 2; ++sp) {
                const int sigma = sp == 0 ? 1 : -1;
                const double *G = sp == 0 ? Gup : Gdn;
                double delta = exp(-2.0 * (double)sigma * lambda * (double)s[l]) - 1.0;
                double one_minus_g = 1.0 - G[(size_t)l * L + l];
                double p = one_minus_g * delta;
                Rs[sp] = 1.0 + p;
                Ds[sp] = delta;
            }
            double R = Rs[0] * Rs[1];
            double u = orc_uniform((uint32_t)l, (uint32_t)t, chain, grid, seed);
            stats[0] += 1;
            if (!(R > 0.0) || !isfinite(R)) stats[4] += 1;
            int accept;
            if (accept_rule == 1) {
                double onep = 1.0 + R;
                double lhs = u * onep;
                accept = lhs < R;
            } else {
                accept = u < R;
            }
            if (!accept) continue;

            for (int sp = 0; sp < 2; ++sp) {
                double *G = sp == 0 ? Gup : Gdn;
                double f = Ds[sp] / Rs[sp];
                for (int i = 0; i < L; ++i) {
                    col[i] = G[(size_t)i * L + l] - (i == l ? 1.0 : 0.0);
                    row[i] = G[(size_t)l * L + i];
                }
                for (int i = 0; i < L; ++i) {
                    double ci = col[i] * f;
                    for (int j = 0; j < L; ++j) G[(size_t)i * L + j] += ci * row[j];
                }
            }
            s[l] = (int8_t)-s[l];
            stats[1] += 1;
            hash ^= (uint64_t)(t * (int64_t)L + l);
            hash *= ORC_FNV_PRIME;

            if (n_wrap > 0 && stats[1] % n_wrap == 0) {
                stats[2] += 1;
                for (int sp = 0; sp < 2 && rc == 0; ++sp) {
                    double *G = sp == 0 ? Gup : Gdn;
                    rc = orc_green(L, M, s, lambda, sp == 0 ? 1 : -1, Gfresh, NULL);
                    if (rc != 0) break;
                    double dmax = 0.0;
                    for (size_t e = 0; e < LL; ++e) {
                        double d = fabs(G[e] - Gfresh[e]);
                        if (d > dmax) dmax = d;
                    }
                    if (dmax > *drift) *drift = dmax;
                    memcpy(G, Gfresh, sizeof(double) * LL);
                }
            }
        }
        if (it >= n_warm && rc == 0) {
            const int64_t m = it - n_warm;
            orc_measure_g(L, Gup, gtmp);
            orc_measure_g(L, Gdn, gtmp + L);
            for (int k = 0; k < 2 * L; ++k) acc[k] += gtmp[k];
            *accD += orc_measure_D(L, Gup, Gdn);
            if (bins) {
                int64_t b = (32 * m) / n_meas;
                for (int k = 0; k < L; ++k) bins[b * L + k] += 0.5 * (gtmp[k] + gtmp[L + k]);
            }
            if (hist) {
                int64_t idx = 0;
                for (int l = 0; l < L; ++l) if (s[l] > 0) idx |= (int64_t)1 << l;
                hist[idx] += 1;
            }
        }
    }
    stats[3] = (int64_t)hash;
    free(col);
    free(row);
    free(gtmp);
    free(Gfresh);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Brute force over all 2^L fields (L <= 20)                                  */
/* ------------------------------------------------------------------------ */
/* w(s) = det A^up(s) det A^dn(s)  (proportional to prod_sigma det G^sigma(s)^{-1});
 * g_exact[k] = sum_s w(s) meas_k(s) / sum_s w(s), meas spin-averaged (positive
 * convention); D_exact likewise.  weights (2^L) may be NULL.
 * Returns the number of configurations with w <= 0, or -1 on a singular A. */
int64_t orc_brute_force(int L, double lambda, const double *M, double *g_exact,
                        double *D_exact, double *Z_out, double *weights)
{
    const size_t LL = (size_t)L * L;
    double *Gu = (double *)malloc(sizeof(double) * LL);
    double *Gd = (double *)malloc(sizeof(double) * LL);
    double *gu = (double *)malloc(sizeof(double) * (size_t)L);
    double *gd = (double *)malloc(sizeof(double) * (size_t)L);
    int8_t *s = (int8_t *)malloc((size_t)L);
    double Z = 0.0, Dsum = 0.0;
    int64_t n_bad = 0;
    for (int k = 0; k < L; ++k) g_exact[k] = 0.0;
    const int64_t nconf = (int64_t)1 << L;
    for (int64_t c = 0; c < nconf; ++c) {
        for (int l = 0; l < L; ++l) s[l] = ((c >> l) & 1) ? (int8_t)1 : (int8_t)-1;
        double du = 0.0, dd = 0.0;
        if (orc_green(L, M, s, lambda, 1, Gu, &du) != 0 ||
            orc_green(L, M, s, lambda, -1, Gd, &dd) != 0) {
            n_bad = -1;
            break;
        }
        double w = du * dd;
        if (weights) weights[c] = w;
        if (!(w > 0.0)) n_bad += 1;
        orc_measure_g(L, Gu, gu);
        orc_measure_g(L, Gd, gd);
        for (int k = 0; k < L; ++k) g_exact[k] += w * 0.5 * (gu[k] + gd[k]);
        Dsum += w * orc_measure_D(L, Gu, Gd);
        Z += w;
    }
    if (n_bad >= 0) {
        for (int k = 0; k < L; ++k) g_exact[k] /= Z;
        *D_exact = Dsum / Z;
        *Z_out = Z;
    }
    free(Gu);
    free(Gd);
    free(gu);
    free(gd);
    free(s);
    return n_bad;
}
