/*
 * rewl_oracle.c -- plain CPU oracle of replica-exchange Wang-Landau (REWL)
 * sampling for the 2D Ising and 2D q-state Potts models.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path must compute.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it.  It shares
 * no code with the CUDA library: it has its own Philox, its own acceptance
 * threshold routine, its own window arithmetic and its own bookkeeping.
 *
 * Paper: Vogel, Li, Wuest, Landau, "Scalable replica-exchange framework for
 * Wang-Landau sampling" (arXiv:1407.5140).
 *   - WL update, ln f schedule, flatness:        Sec. II A (first paragraph)
 *   - overlapping windows, o = overlap with the next-lower window:
 *                                                 Sec. II A, Fig. 1, notation list
 *   - exchange acceptance:                        Eq. (1)
 *   - neighbour-only exchange, alternating pairs: Sec. II A, Fig. 2
 *   - m independent walkers, own g and H, merge after each WL iteration,
 *     run-past-convergence:                       Sec. II A
 *   - Potts Hamiltonian, single-spin update:      Sec. III A, Eq. (2)
 *
 * Readings where the paper is silent:
 *   - ln g is FP64; every value it takes is a multiple of 2^-32 below 2^21
 *     in magnitude, so differences are exact.  The oracle checks the bound.
 *   - ln g of a window is defined up to a constant (the pieces are joined
 *     by their differences, Sec. II B; acceptance and exchange, Eq. (1), use
 *     differences within one window), so a running window whose ln g has
 *     reached 2^s on every realisable bin of every walker has 2^s taken off
 *     those bins at the next flatness test (s = 20 unless set): on large
 *     lattices the first stages add far more than 2^21 per bin.  The
 *     trajectory is unchanged, and H is kept separately.
 *   - accept iff (ln g(E') - ln g(E)) * 2^32 < lam_fix, where
 *     lam_fix = max(1, trunc(2^32 * lam)) and lam = -ln u is evaluated in
 *     binary32 by the routine lam_spec below (u = (k+1) 2^-24, k = r >> 8).
 *     This is min(1, g(E)/g(E')) in log form (u < g(E)/g(E') <=> -ln u >
 *     ln g(E') - ln g(E)); the fixed binary32 operation sequence makes the
 *     decision reproducible on any IEEE-754 machine.
 *   - a move that leaves the walker's window is rejected and the current
 *     bin is updated.
 *   - flatness is tested after every sweep (N attempts) on the reachable
 *     bins of the window: flat iff min(H) * n_reach >= p * sum(H) (FP64).
 *     With the Zhou-Bhatt rule (Sec. IV B, Eq. (8)) the same parameter is a
 *     and a walker is flat iff min(H) >= a / sqrt(ln f); with ln f = 2^-k
 *     that is min(H) >= sqrt(2^k a^2), evaluated as sqrt(ldexp(a * a, k))
 *     (each step a correctly rounded IEEE-754 double operation).
 *     A flat walker latches and keeps walking with the same ln f.
 *   - when all m walkers of a window are latched, their ln g are replaced by
 *     the mean, rounded to the nearest multiple of 2^-32 (ties to even);
 *     H is reset; ln f -> ln f / 2, or the window converges if
 *     ln f <= ln_f_final.  Converged windows stop updating ln g and H
 *     (the histogram has no role once the window is done) and keep walking
 *     and exchanging (Sec. II A).  Sampling with given, frozen weights
 *     (oracle_set_lng with stage0 < 0) does count H.
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), key =
 *     (seed_lo, seed_hi ^ instance), counter = (draw_lo, draw_hi,
 *     window << 16 | walker, stream); stream 0 = sweep, 1 = init,
 *     2 = exchange.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_ISING 0
#define OR_POTTS 1

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from its definition in Salmon, Moraes, Dror, Shaw, */
/* "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two  */
/* 32x32->64 multiplications with a Weyl-sequence key schedule.              */
/* ------------------------------------------------------------------------ */
static void philox4x32_10(uint32_t k0, uint32_t k1, const uint32_t ctr[4], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod_b >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod_b;
        uint32_t y2 = (uint32_t)(prod_a >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform integer in [0, n): the high word of r * n */
static uint32_t scale_u32(uint32_t r, uint32_t n)
{
    return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* lam_spec: lam = -ln(u), u = (k + 1) * 2^-24, k in [0, 2^24), in binary32. */
/*                                                                          */
/* Method: split u = 2^e * m with m in [sqrt(1/2), sqrt(2)); ln m from the  */
/* series ln m = 2 atanh(s) = 2 s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9),      */
/* s = (m - 1)/(m + 1), |s| < 0.172; e * ln 2 with the Cody-Waite split     */
/* ln 2 = 355/512 + c2 (Cody & Waite, "Software Manual for the Elementary   */
/* Functions", 1980), so that e * 355/512 is exact.  Every operation is an  */
/* IEEE-754 binary32 operation rounded to nearest; products feeding a sum   */
/* are fused only where fmaf is written.                                    */
/* ------------------------------------------------------------------------ */
static int64_t lam_spec(uint32_t k)
{
    const float ln2_hi = 0.693359375f;              /* 355/512, exact       */
    const float ln2_lo = -2.12194440e-4f;           /* ln 2 - 355/512       */
    float x = (float)(k + 1u);                      /* exact: k + 1 <= 2^24 */
    uint32_t bits;
    memcpy(&bits, &x, 4);
    int e = (int)(bits >> 23) - 127;
    uint32_t mbits = (bits & 0x007FFFFFu) | 0x3F800000u;
    float m;
    memcpy(&m, &mbits, 4);                          /* m in [1, 2)          */
    if (m > 1.41421356f) {                          /* centre m on 1        */
        m = m * 0.5f;
        e = e + 1;
    }
    float a = m - 1.0f;
    float b = m + 1.0f;
    float s = a / b;
    float z = s * s;
    float p = fmaf(z, 1.0f / 9.0f, 1.0f / 7.0f);
    p = fmaf(p, z, 1.0f / 5.0f);
    p = fmaf(p, z, 1.0f / 3.0f);
    p = fmaf(p, z, 1.0f);
    float ln_m = (s + s) * p;
    float ef = (float)(e - 24);
    float t = fmaf(ef, ln2_lo, ln_m);
    float ln_u = fmaf(ef, ln2_hi, t);
    float lam = -ln_u;
    int64_t fix = (int64_t)(lam * 4294967296.0f);   /* truncation           */
    return fix < 1 ? 1 : fix;
}

/* ------------------------------------------------------------------------ */
/* Oracle state                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    int model, L, q, N;
    long e_min, e_max;
    int step;                 /* energy units per bin: 4 (Ising), 1 (Potts) */
    int B;                    /* number of bins in [e_min, e_max]            */
    int h, m, w;              /* windows, walkers per window, bins/window    */
    int *lo;                  /* first global bin of each window             */
    int *ww;                  /* bins of each window (w is the widest: the
                                 row length of ln g and H)                    */
    unsigned char *reach;     /* reach[b]: energy of bin b is realisable     */
    int *n_reach;             /* reachable bins in each window               */
    double p_flat, ln_f_final;
    int flat_rule;            /* 0: min H >= p <H>;  1: min H >= a/sqrt(ln f)  */
    long check_every;         /* sweeps between flatness tests               */
    int shift_exp;            /* ln g of a window is lowered by 2^shift_exp
                                 once all its values reach it               */
    uint32_t key0, key1;
    int n_walkers;            /* h * m, walker id = window * m + j           */
    signed char **spin;       /* per walker slot: its current configuration  */
    long *E;                  /* energy of the configuration in each slot    */
    int *bin;                 /* global bin of that energy                   */
    long *replica;            /* id of the configuration (follows exchanges) */
    double *lng;              /* [walker][w], window-local bins              */
    uint64_t *H;              /* [walker][w]                                 */
    uint64_t *draw;           /* sweep-stream Philox block counter           */
    unsigned char *latch;     /* walker has been flat in the current stage   */
    int *stage;               /* per window: ln f = 2^-stage                 */
    unsigned char *conv;      /* per window: 0 running; 1 converged (ln g
                                 frozen, H no longer counted); 2 frozen
                                 sampling from given weights (H counted)      */
    long *conv_sweep;         /* per window: sweep count at convergence      */
    long sweeps;              /* sweeps done by every walker                 */
    uint64_t t_exch;          /* exchange phases done                        */
    uint64_t *ex_prop, *ex_acc; /* per window pair (i, i+1)                  */
    uint64_t *n_acc;          /* per walker: accepted moves                  */
    int error;                /* sticky: 1 = ln g left the exact range,     */
                              /*         2 = init did not reach the window  */
} rewl_oracle;

static long model_energy(const rewl_oracle *o, const signed char *s)
{
    /* Ising: E = -sum_<ij> s_i s_j.  Potts, Eq. (2): E = -sum_<ij> delta(q_i,q_j).
     * Each site contributes its right and down bond (periodic boundaries). */
    long E = 0;
    int L = o->L;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int i = y * L + x;
            int r = y * L + (x + 1) % L;
            int d = ((y + 1) % L) * L + x;
            if (o->model == OR_ISING)
                E -= (long)s[i] * s[r] + (long)s[i] * s[d];
            else
                E -= (long)(s[i] == s[r]) + (long)(s[i] == s[d]);
        }
    return E;
}

/* energy change of proposing value `nv` at `site` */
static long delta_energy(const rewl_oracle *o, const signed char *s, int site, int nv)
{
    int L = o->L, x = site % L, y = site / L;
    int nb[4] = {y * L + (x + 1) % L, y * L + (x + L - 1) % L,
                 ((y + 1) % L) * L + x, ((y + L - 1) % L) * L + x};
    long dE = 0;
    for (int t = 0; t < 4; ++t) {
        int sj = s[nb[t]];
        if (o->model == OR_ISING)
            dE += -(long)nv * sj + (long)s[site] * sj;
        else
            dE += -(long)(nv == sj) + (long)(s[site] == sj);
    }
    return dE;
}

static int energy_to_bin(const rewl_oracle *o, long E)
{
    return (int)((E - o->e_min) / o->step);
}

static int bin_in_window(const rewl_oracle *o, int win, long E)
{
    if (E < o->e_min || E > o->e_max) return 0;
    int b = energy_to_bin(o, E);
    return b >= o->lo[win] && b <= o->lo[win] + o->ww[win] - 1;
}

/* Realisable energies on an even L x L periodic lattice (L >= 4):
 * Ising: E = -2N + 4u for u in 0..N except u = 1 and u = N - 1
 *        (no configuration has exactly two or 2N - 2 unsatisfied bonds).
 * Potts q >= 3: -2N <= E <= 0 except E + 2N in {1, 2, 3, 5}.
 * Potts q = 2: E + 2N even, except E + 2N = 2 and E = -2 (Ising images). */
static int energy_reachable(const rewl_oracle *o, long E)
{
    long N = o->N, off = E + 2 * N;
    if (o->model == OR_ISING) {
        if (off < 0 || off > 4 * N || off % 4) return 0;
        long u = off / 4;
        return !(u == 1 || u == N - 1);
    }
    if (off < 0 || off > 2 * N) return 0;
    if (o->q == 2) return off % 2 == 0 && off != 2 && off != 2 * N - 2;
    return !(off == 1 || off == 2 || off == 3 || off == 5);
}

static int check_exact(rewl_oracle *o, double v)
{
    /* every ln g value must be a multiple of 2^-32 below 2^21 so that FP64
     * holds it exactly; outside that range the oracle stops being exact */
    if (!(fabs(v) < 2097152.0)) { o->error = 1; return 0; }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* creation and windows                                                     */
/* ------------------------------------------------------------------------ */

/* Window partition (Sec. II A, Fig. 1, notation list; widths checked against
 * Sec. IV A): h windows of equal width w bins, each overlapping the next-lower
 * one by a fraction o.  Consecutive windows start (1 - o) w apart, so
 * w (1 + (h - 1)(1 - o)) covers the B bins:
 *   w = ceil(B / (1 + (h - 1)(1 - o))),  lo_i = floor(i (B - w) / (h - 1)). */
int oracle_windows(int B, int h, double o, int *lo_out, int *w_out)
{
    if (B < 1 || h < 1 || !(o >= 0.0 && o < 1.0)) return -1;
    double denom = 1.0 + (double)(h - 1) * (1.0 - o);
    int w = (int)ceil((double)B / denom);
    if (w > B) w = B;
    if (w < 1) return -1;
    *w_out = w;
    for (int i = 0; i < h; ++i)
        lo_out[i] = (h == 1) ? 0 : (int)(((long)i * (long)(B - w)) / (long)(h - 1));
    return 0;
}

void oracle_destroy(rewl_oracle *o);

rewl_oracle *oracle_create(int model, int L, int q, long e_min, long e_max,
                           int h, double overlap, int m, double p_flat,
                           double ln_f_final, uint64_t seed, uint32_t instance)
{
    if (L < 4 || L % 2 || h < 1 || m < 1 || h > 65535 || m > 65535) return NULL;
    if (model == OR_POTTS && (q < 2 || q > 127)) return NULL;
    rewl_oracle *o = (rewl_oracle *)calloc(1, sizeof(rewl_oracle));
    o->model = model; o->L = L; o->q = (model == OR_ISING) ? 2 : q; o->N = L * L;
    o->step = (model == OR_ISING) ? 4 : 1;
    long Emin_model = -2L * o->N;
    long Emax_model = (model == OR_ISING) ? 2L * o->N : 0;
    if (e_min < Emin_model || e_max > Emax_model || e_min >= e_max ||
        (e_min - Emin_model) % o->step || (e_max - Emin_model) % o->step) {
        free(o); return NULL;
    }
    o->e_min = e_min; o->e_max = e_max;
    o->B = (int)((e_max - e_min) / o->step) + 1;
    o->h = h; o->m = m;
    o->lo = (int *)calloc(h, sizeof(int));
    o->ww = (int *)calloc(h, sizeof(int));
    if (oracle_windows(o->B, h, overlap, o->lo, &o->w)) { oracle_destroy(o); return NULL; }
    o->reach = (unsigned char *)calloc(o->B, 1);
    for (int b = 0; b < o->B; ++b) o->reach[b] = (unsigned char)energy_reachable(o, e_min + (long)b * o->step);
    o->n_reach = (int *)calloc(h, sizeof(int));
    for (int i = 0; i < h; ++i)
    {
        for (int b = o->lo[i]; b < o->lo[i] + o->w; ++b) o->n_reach[i] += o->reach[b];
        o->ww[i] = o->w;
    }
    o->p_flat = p_flat; o->ln_f_final = ln_f_final;
    o->check_every = 1;
    o->shift_exp = 20;
    o->key0 = (uint32_t)seed;
    o->key1 = (uint32_t)(seed >> 32) ^ instance;
    o->n_walkers = h * m;
    int nw = o->n_walkers;
    o->spin = (signed char **)calloc(nw, sizeof(signed char *));
    for (int k = 0; k < nw; ++k) o->spin[k] = (signed char *)calloc(o->N, 1);
    o->E = (long *)calloc(nw, sizeof(long));
    o->bin = (int *)calloc(nw, sizeof(int));
    o->replica = (long *)calloc(nw, sizeof(long));
    o->lng = (double *)calloc((size_t)nw * o->w, sizeof(double));
    o->H = (uint64_t *)calloc((size_t)nw * o->w, sizeof(uint64_t));
    o->draw = (uint64_t *)calloc(nw, sizeof(uint64_t));
    o->latch = (unsigned char *)calloc(nw, 1);
    o->stage = (int *)calloc(h, sizeof(int));
    o->conv = (unsigned char *)calloc(h, 1);
    o->conv_sweep = (long *)calloc(h, sizeof(long));
    o->ex_prop = (uint64_t *)calloc(h, sizeof(uint64_t));
    o->ex_acc = (uint64_t *)calloc(h, sizeof(uint64_t));
    o->n_acc = (uint64_t *)calloc(nw, sizeof(uint64_t));
    for (int k = 0; k < nw; ++k) o->replica[k] = k;
    for (int i = 0; i < h; ++i) o->conv_sweep[i] = -1;
    return o;
}

void oracle_destroy(rewl_oracle *o)
{
    if (!o) return;
    if (o->spin) for (int k = 0; k < o->n_walkers; ++k) free(o->spin[k]);
    free(o->spin); free(o->E); free(o->bin); free(o->replica); free(o->lng); free(o->H);
    free(o->draw); free(o->latch); free(o->stage); free(o->conv); free(o->conv_sweep);
    free(o->ex_prop); free(o->ex_acc); free(o->n_acc); free(o->lo); free(o->ww); free(o->reach);
    free(o->n_reach); free(o);
}

/* ------------------------------------------------------------------------ */
/* walker initialisation (paper silent): start from the ground state when   */
/* the window lies below the infinite-temperature mean energy (0 for Ising, */
/* -2N/q for Potts), else from the two-colour checkerboard (maximum energy),*/
/* then apply unconditional random single-spin updates (stream 1) until the */
/* energy lies in the window.                                               */
/* ------------------------------------------------------------------------ */
static void init_walker(rewl_oracle *o, int k)
{
    int win = k / o->m, j = k % o->m, L = o->L, N = o->N;
    signed char *s = o->spin[k];
    long E_lo = o->e_min + (long)o->lo[win] * o->step;
    int below_mean = (o->model == OR_ISING) ? (E_lo < 0) : ((long)o->q * E_lo < -2L * N);
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int odd = (x + y) & 1;
            if (o->model == OR_ISING) s[y * L + x] = below_mean ? 1 : (odd ? -1 : 1);
            else s[y * L + x] = below_mean ? 0 : (signed char)odd;
        }
    long E = model_energy(o, s);
    uint32_t ctr[4] = {0, 0, ((uint32_t)win << 16) | (uint32_t)j, 1};
    uint64_t blk = 0;
    while (!bin_in_window(o, win, E)) {
        if (blk >= (1ull << 28)) { o->error = 2; break; }
        ctr[0] = (uint32_t)blk; ctr[1] = (uint32_t)(blk >> 32);
        uint32_t r[4];
        philox4x32_10(o->key0, o->key1, ctr, r);
        ++blk;
        if (o->model == OR_ISING) {
            for (int t = 0; t < 2 && !bin_in_window(o, win, E); ++t) {
                int site = (int)scale_u32(r[2 * t], (uint32_t)N);
                int nv = -s[site];
                E += delta_energy(o, s, site, nv);
                s[site] = (signed char)nv;
            }
        } else {
            int site = (int)scale_u32(r[0], (uint32_t)N);
            int nv = (s[site] + 1 + (int)scale_u32(r[1], (uint32_t)(o->q - 1))) % o->q;
            E += delta_energy(o, s, site, nv);
            s[site] = (signed char)nv;
        }
    }
    o->E[k] = E;
    o->bin[k] = energy_to_bin(o, E);
}

int oracle_init(rewl_oracle *o)
{
    for (int k = 0; k < o->n_walkers; ++k) init_walker(o, k);
    return o->error;
}

/* ------------------------------------------------------------------------ */
/* one Wang-Landau trial (Sec. II A): propose, accept with                  */
/* min(1, g(E)/g(E')), then ln g(E_now) += ln f and H(E_now) += 1.          */
/* ------------------------------------------------------------------------ */
static void wl_trial(rewl_oracle *o, int k, int site, int nv, uint32_t r_u, double ln_f, int conv)
{
    int win = k / o->m, lo = o->lo[win];
    signed char *s = o->spin[k];
    double *lng = o->lng + (size_t)k * o->w;
    uint64_t *H = o->H + (size_t)k * o->w;
    long dE = delta_energy(o, s, site, nv);
    long En = o->E[k] + dE;
    int accept = 0;
    if (bin_in_window(o, win, En)) {
        int bn = energy_to_bin(o, En);
        double dl = (lng[bn - lo] - lng[o->bin[k] - lo]) * 4294967296.0;
        accept = dl < (double)lam_spec(r_u >> 8);
    }
    if (accept) {
        s[site] = (signed char)nv;
        o->E[k] = En;
        o->bin[k] = energy_to_bin(o, En);
        o->n_acc[k] += 1;
    }
    if (!conv) {
        lng[o->bin[k] - lo] += ln_f;
        check_exact(o, lng[o->bin[k] - lo]);
    }
    if (conv != 1) H[o->bin[k] - lo] += 1;      /* no histogram after convergence */
}

/* one sweep = N trials (Sec. IV A: one MC sweep equals N MC steps) */
static void walker_sweep(rewl_oracle *o, int k)
{
    int win = k / o->m, j = k % o->m, N = o->N;
    double ln_f = ldexp(1.0, -o->stage[win]);
    int conv = o->conv[win];
    uint32_t ctr[4] = {0, 0, ((uint32_t)win << 16) | (uint32_t)j, 0};
    int per_block = (o->model == OR_ISING) ? 2 : 1;
    for (int t = 0; t < N; t += per_block) {
        uint64_t blk = o->draw[k]++;
        ctr[0] = (uint32_t)blk; ctr[1] = (uint32_t)(blk >> 32);
        uint32_t r[4];
        philox4x32_10(o->key0, o->key1, ctr, r);
        if (o->model == OR_ISING) {
            for (int a = 0; a < 2; ++a) {
                int site = (int)scale_u32(r[2 * a], (uint32_t)N);
                wl_trial(o, k, site, -o->spin[k][site], r[2 * a + 1], ln_f, conv);
            }
        } else {
            int site = (int)scale_u32(r[0], (uint32_t)N);
            int nv = (o->spin[k][site] + 1 + (int)scale_u32(r[1], (uint32_t)(o->q - 1))) % o->q;
            wl_trial(o, k, site, nv, r[2], ln_f, conv);
        }
    }
}

/* Zhou-Bhatt test (Eq. (8)): min H >= a / sqrt(ln f) with ln f = 2^-stage */
int oracle_zb_flat(uint64_t min_h, double a, int stage)
{
    return (double)min_h >= sqrt(ldexp(a * a, stage));
}

/* the 80 % rule (Sec. II A): min H >= p <H> over the n_reach reachable
 * bins, as min * n_reach >= p * sum in IEEE doubles */
int oracle_pct_flat(uint64_t min_h, uint64_t sum_h, int n_reach, double p)
{
    return (double)min_h * (double)n_reach >= p * (double)sum_h;
}

/* flatness test (Sec. II A): no H(E) below p times the mean of H over the
 * reachable bins of the walker's window (or the Zhou-Bhatt minimum) */
static int walker_flat(const rewl_oracle *o, int k)
{
    int win = k / o->m, lo = o->lo[win];
    const uint64_t *H = o->H + (size_t)k * o->w;
    uint64_t mn = UINT64_MAX, sum = 0;
    for (int b = 0; b < o->ww[win]; ++b) {
        if (!o->reach[lo + b]) continue;
        if (H[b] < mn) mn = H[b];
        sum += H[b];
    }
    if (o->flat_rule == 1) return oracle_zb_flat(mn, o->p_flat, o->stage[win]);
    return oracle_pct_flat(mn, sum, o->n_reach[win], o->p_flat);
}

/* nearest integer to num/den, ties to even (den > 0) */
static int64_t div_round_even(int64_t num, int64_t den)
{
    int64_t q = num / den, r = num % den;
    if (r < 0) { r += den; q -= 1; }          /* floor division */
    if (2 * r > den || (2 * r == den && (q & 1))) q += 1;
    return q;
}

/* the merge (Sec. II A): every walker of the window takes the mean of the
 * m walkers' ln g, bin by bin, rounded to the nearest multiple of 2^-32 with
 * ties to even */
void oracle_average_window(rewl_oracle *o, int win)
{
    int m = o->m;
    for (int b = 0; b < o->ww[win]; ++b) {
        int64_t units = 0;
        for (int j = 0; j < m; ++j) {
            double v = o->lng[(size_t)(win * m + j) * o->w + b];
            units += (int64_t)(v * 4294967296.0);   /* exact: v on the 2^-32 grid */
        }
        double mean = (double)div_round_even(units, m) / 4294967296.0;
        for (int j = 0; j < m; ++j) o->lng[(size_t)(win * m + j) * o->w + b] = mean;
    }
}

/* end-of-sweep bookkeeping for one window: latch flat walkers; when all m
 * walkers are latched, average their ln g (Sec. II A), reset H, and halve
 * ln f or declare the window converged */
static void window_boundary(rewl_oracle *o, int win)
{
    if (o->conv[win]) return;
    int m = o->m, all = 1;
    /* ln g is defined up to a constant per window: lower it by 2^s once every
     * realisable bin of every walker has reached 2^s */
    double lmin = INFINITY, s = ldexp(1.0, o->shift_exp);
    for (int j = 0; j < m; ++j)
        for (int b = 0; b < o->ww[win]; ++b)
            if (o->reach[o->lo[win] + b]) {
                double v = o->lng[(size_t)(win * m + j) * o->w + b];
                if (v < lmin) lmin = v;
            }
    if (lmin >= s)
        for (int j = 0; j < m; ++j)
            for (int b = 0; b < o->ww[win]; ++b)
                if (o->reach[o->lo[win] + b]) o->lng[(size_t)(win * m + j) * o->w + b] -= s;
    for (int j = 0; j < m; ++j) {
        int k = win * m + j;
        if (!o->latch[k] && walker_flat(o, k)) o->latch[k] = 1;
        all &= o->latch[k];
    }
    if (!all) return;
    oracle_average_window(o, win);
    for (int j = 0; j < m; ++j) {
        int k = win * m + j;
        memset(o->H + (size_t)k * o->w, 0, sizeof(uint64_t) * o->w);
        o->latch[k] = 0;
    }
    if (ldexp(1.0, -o->stage[win]) <= o->ln_f_final) {
        o->conv[win] = 1;
        o->conv_sweep[win] = o->sweeps;
    } else {
        o->stage[win] += 1;
    }
}

int oracle_run(rewl_oracle *o, long n_sweeps, int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    /* walkers are independent within a sweep; small instances run serially
     * (a team's barrier per sweep costs more than the sweep itself) */
    const long work = (long)o->n_walkers * o->N;
    for (long sw = 0; sw < n_sweeps; ++sw) {
        #pragma omp parallel for schedule(dynamic, 1) if (work >= 65536 && o->n_walkers >= 4)
        for (int k = 0; k < o->n_walkers; ++k) walker_sweep(o, k);
        o->sweeps += 1;
        if (o->sweeps % o->check_every == 0)
            for (int win = 0; win < o->h; ++win) window_boundary(o, win);
        if (o->error) break;
    }
    return o->error;
}

/* ------------------------------------------------------------------------ */
/* replica exchange (Eq. (1), Fig. 2): windows (i, i+1) with i of the       */
/* current parity; walker j of window i proposes a swap with walker         */
/* (j + s) mod m of window i+1, s drawn once per window pair.               */
/* ------------------------------------------------------------------------ */
int oracle_exchange(rewl_oracle *o)
{
    uint64_t t = o->t_exch;
    int m = o->m, w = o->w;
    for (int i = (int)(t & 1); i + 1 < o->h; i += 2) {
        uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), ((uint32_t)i << 16) | 0xFFFFu, 2};
        uint32_t r[4];
        philox4x32_10(o->key0, o->key1, ctr, r);
        int shift = (int)scale_u32(r[0], (uint32_t)m);
        for (int j = 0; j < m; ++j) {
            int a = i * m + j, b = (i + 1) * m + (j + shift) % m;
            ctr[2] = ((uint32_t)i << 16) | (uint32_t)j;
            philox4x32_10(o->key0, o->key1, ctr, r);
            o->ex_prop[i] += 1;
            /* both configurations must fall inside the other walker's window */
            if (!bin_in_window(o, i + 1, o->E[a]) || !bin_in_window(o, i, o->E[b])) continue;
            const double *ga = o->lng + (size_t)a * w, *gb = o->lng + (size_t)b * w;
            int lo_a = o->lo[i], lo_b = o->lo[i + 1];
            int bx = o->bin[a], by = o->bin[b];
            /* -ln of the Eq. (1) ratio: [ln g_a(Y) - ln g_a(X)] + [ln g_b(X) - ln g_b(Y)] */
            double cost = ((ga[by - lo_a] - ga[bx - lo_a]) + (gb[bx - lo_b] - gb[by - lo_b])) * 4294967296.0;
            if (cost < (double)lam_spec(r[0] >> 8)) {
                signed char *tmp = o->spin[a]; o->spin[a] = o->spin[b]; o->spin[b] = tmp;
                long te = o->E[a]; o->E[a] = o->E[b]; o->E[b] = te;
                int tb = o->bin[a]; o->bin[a] = o->bin[b]; o->bin[b] = tb;
                long tr = o->replica[a]; o->replica[a] = o->replica[b]; o->replica[b] = tr;
                o->ex_acc[i] += 1;
            }
        }
    }
    o->t_exch = t + 1;
    return 0;
}

/* warm start / fixed-weight sampling: set every walker's ln g from a global
 * table (rounded to the 2^-32 grid) and start at ln f = 2^-stage0;
 * stage0 < 0 freezes ln g from the start (pure sampling with weights 1/g). */
int oracle_set_lng(rewl_oracle *o, const double *ln_g_global, int stage0)
{
    for (int win = 0; win < o->h; ++win) {
        for (int j = 0; j < o->m; ++j) {
            double *lng = o->lng + (size_t)(win * o->m + j) * o->w;
            for (int b = 0; b < o->ww[win]; ++b) {
                double v = nearbyint(ln_g_global[o->lo[win] + b] * 4294967296.0) / 4294967296.0;
                if (!check_exact(o, v)) return o->error;
                lng[b] = v;
            }
        }
        if (stage0 < 0) { o->conv[win] = 2; o->stage[win] = 0; }
        else { o->conv[win] = 0; o->stage[win] = stage0; }
    }
    return 0;
}

/* set one walker's window-local ln g (used by the Eq. (1) pin) */
int oracle_set_walker_lng(rewl_oracle *o, int k, const double *local)
{
    for (int b = 0; b < o->w; ++b) {
        double v = nearbyint(local[b] * 4294967296.0) / 4294967296.0;
        if (!check_exact(o, v)) return o->error;
        o->lng[(size_t)k * o->w + b] = v;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* read-out                                                                 */
/* ------------------------------------------------------------------------ */
void oracle_geometry(const rewl_oracle *o, int *B, int *w, int *lo, unsigned char *reach)
{
    *B = o->B; *w = o->w;
    if (lo) memcpy(lo, o->lo, sizeof(int) * o->h);
    if (reach) memcpy(reach, o->reach, o->B);
}

/* Windows of any widths (the run-time-balanced windows of Sec. V): window i
 * covers bins lo[i]..hi[i].  They must start at bin 0, end at bin B-1, have
 * increasing lower and upper ends and overlap their neighbour by at least one
 * bin.  Call before oracle_init.  Returns 0, or -1 for an invalid set. */
int oracle_set_windows(rewl_oracle *o, const int *lo, const int *hi)
{
    int h = o->h, wmax = 0;
    if (lo[0] != 0 || hi[h - 1] != o->B - 1) return -1;
    for (int i = 0; i < h; ++i) {
        if (hi[i] < lo[i] || hi[i] >= o->B) return -1;
        if (i + 1 < h && (lo[i + 1] <= lo[i] || hi[i + 1] <= hi[i] || lo[i + 1] > hi[i])) return -1;
        if (hi[i] - lo[i] + 1 > wmax) wmax = hi[i] - lo[i] + 1;
    }
    if (wmax != o->w) {
        free(o->lng); free(o->H);
        o->w = wmax;
        o->lng = (double *)calloc((size_t)o->n_walkers * o->w, sizeof(double));
        o->H = (uint64_t *)calloc((size_t)o->n_walkers * o->w, sizeof(uint64_t));
    }
    for (int i = 0; i < h; ++i) {
        o->lo[i] = lo[i];
        o->ww[i] = hi[i] - lo[i] + 1;
        o->n_reach[i] = 0;
        for (int b = lo[i]; b <= hi[i]; ++b) o->n_reach[i] += o->reach[b];
    }
    return 0;
}

void oracle_window_widths(const rewl_oracle *o, int *ww) { memcpy(ww, o->ww, sizeof(int) * (size_t)o->h); }

/* spins_out: [n_walkers][N] as stored (Ising +-1, Potts 0..q-1) */
void oracle_get_state(const rewl_oracle *o, signed char *spins_out, long *E_out, int *bin_out,
                      double *lng_out, uint64_t *H_out, int *stage_out, unsigned char *conv_out,
                      unsigned char *latch_out, long *replica_out)
{
    for (int k = 0; k < o->n_walkers; ++k) {
        if (spins_out) memcpy(spins_out + (size_t)k * o->N, o->spin[k], o->N);
        if (E_out) E_out[k] = o->E[k];
        if (bin_out) bin_out[k] = o->bin[k];
        if (latch_out) latch_out[k] = o->latch[k];
        if (replica_out) replica_out[k] = o->replica[k];
    }
    if (lng_out) memcpy(lng_out, o->lng, sizeof(double) * (size_t)o->n_walkers * o->w);
    if (H_out) memcpy(H_out, o->H, sizeof(uint64_t) * (size_t)o->n_walkers * o->w);
    if (stage_out) memcpy(stage_out, o->stage, sizeof(int) * o->h);
    if (conv_out) memcpy(conv_out, o->conv, o->h);
}

void oracle_get_counters(const rewl_oracle *o, long *sweeps, uint64_t *t_exch, uint64_t *ex_prop,
                         uint64_t *ex_acc, uint64_t *n_acc, long *conv_sweep)
{
    if (sweeps) *sweeps = o->sweeps;
    if (t_exch) *t_exch = o->t_exch;
    if (ex_prop) memcpy(ex_prop, o->ex_prop, sizeof(uint64_t) * o->h);
    if (ex_acc) memcpy(ex_acc, o->ex_acc, sizeof(uint64_t) * o->h);
    if (n_acc) memcpy(n_acc, o->n_acc, sizeof(uint64_t) * o->n_walkers);
    if (conv_sweep) memcpy(conv_sweep, o->conv_sweep, sizeof(long) * o->h);
}

void oracle_set_check_every(rewl_oracle *o, long c) { o->check_every = c > 0 ? c : 1; }
void oracle_set_shift_exp(rewl_oracle *o, int e) { o->shift_exp = e >= 1 && e <= 20 ? e : 20; }

/* 0: fraction-of-mean flatness (Sec. II A); 1: Zhou-Bhatt minimum (Eq. (8)) */
void oracle_set_flat_rule(rewl_oracle *o, int rule) { o->flat_rule = rule == 1 ? 1 : 0; }

int oracle_all_converged(const rewl_oracle *o)
{
    for (int i = 0; i < o->h; ++i) if (!o->conv[i]) return 0;
    return 1;
}

int oracle_error(const rewl_oracle *o) { return o->error; }

long oracle_energy_of(const rewl_oracle *o, int k) { return model_energy(o, o->spin[k]); }

/* ------------------------------------------------------------------------ */
/* exported primitives for the pins                                         */
/* ------------------------------------------------------------------------ */
void oracle_philox(uint32_t k0, uint32_t k1, const uint32_t *ctr, long n, uint32_t *out)
{
    for (long i = 0; i < n; ++i) philox4x32_10(k0, k1, ctr + 4 * i, out + 4 * i);
}

void oracle_lam(const uint32_t *k, long n, int64_t *out)
{
    for (long i = 0; i < n; ++i) out[i] = lam_spec(k[i]);
}
