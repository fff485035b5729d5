/*
 * qieo_oracle.c -- reference oracle for the QIEO generation loop on the 0/1 knapsack.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only the test-suite, the package smoke
 * check and the benchmark's CPU-baseline leg load this file. It is the plain, slow,
 * single-threaded statement of what the GPU library computes; it shares no code, header,
 * table or constant with the GPU path, and the GPU path never loads it.
 *
 * Method (arxiv 2609.30862, "Portable QIEO on the GPU ecosystem"):
 *   - Sec. I and Sec. III-A: a chromosome holds Ng qubits; a qubit is an amplitude pair
 *     (alpha, beta) with alpha^2 + beta^2 = 1 that collapses to a binary allele.
 *   - Sec. III-B and Fig. 1: one generation = QIP (observe every qubit), Evaluation
 *     (eq. 1), DetermineElite (generation-best chromosome), CIP (rotate every qubit one
 *     table step toward the elite's allele), then terminate or loop.
 *   - Eq. (1): f = sum(v x) if sum(w x) <= W, else -lambda (sum(w x) - W).
 *
 * Readings where the paper is silent (labelled S1 .. S15 in this file):
 *   S1  dtheta = pi / D (D = 100 for all named workloads); start angle pi/4.
 *   S2  theta stays in [0, pi/2]; a step that would leave it is not taken.
 *   S3  rule R1: every qubit moves one step toward the elite's allele (+ if it is 1,
 *       - if it is 0); rule R2: only qubits whose allele differs from the elite's move.
 *   S5  P(x = 1) = beta^2 = sin^2(theta).
 *   S6  observation compares a 32-bit uniform draw u with the 32-bit fixed-point
 *       threshold T[n] = round(sin^2(n pi / D) 2^32) (n = k + K), mirrored so that
 *       T[2K - n] = 2^32 - T[n]; x = 1 iff u < T[n].
 *   S7  u = word (j mod 4) of Philox4x32-10(counter = (j div 4, c, t, 0),
 *       key = (seed, instance)); t is the absolute generation number.
 *   S8/S9 the elite is the lowest-index maximum of f; the best-so-far record is replaced
 *       only by a strictly larger fitness.
 *   S14 CIP also follows the last generation of a run.
 *   S15 convergence (Sec. IV, off unless asked for): stop once the elite fitness has been
 *       the same for 20 consecutive generations; the fitness values are integers, so the
 *       "within 1e-6 of their mean" clause means equal. The generation count is the cap.
 *
 * Pins (tests): Philox against PyTorch's independent header implementation; the
 * threshold table against a 60-digit evaluation; eq. (1) against a dynamic-programming
 * knapsack optimum and closed-form special cases; observation frequencies against
 * sin^2; the angle-index form (qo_run) against the amplitude form (qo_run_fp64); the
 * loop's fixed points at the bounds (qubits at theta = 0 or pi/2 on the elite's side keep
 * their angle and observe the elite's allele).
 * The exact trajectory of the heuristic has no printed values in the paper: beyond the
 * agreement of the two forms it is parity unpinned.
 *
 * Build: gcc -O2 -shared -fPIC (serial) and the same file with -fopenmp (chromosome
 * loops in parallel; results are identical because chromosomes are independent within a
 * phase).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC 2011). One round maps counter (c0, c1, c2, c3) with key (k0, k1) to
 * (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key is bumped by
 * the Weyl constants between rounds. Ten rounds.
 * ---------------------------------------------------------------------------------- */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

void qo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The draw of gene j of chromosome c at generation t (reading S7). */
static uint32_t draw(uint32_t seed, uint32_t inst, int32_t t, int32_t c, int32_t j)
{
    uint32_t ctr[4] = {(uint32_t)j >> 2, (uint32_t)c, (uint32_t)t, 0u};
    uint32_t key[2] = {seed, inst};
    uint32_t out[4];
    qo_philox4x32_10(ctr, key, out);
    return out[j & 3];
}

/* ------------------------------------------------------------------------------------
 * Fixed-point observation thresholds (reading S6): T[n] for n = 0 .. 2K, K = D / 4.
 * ---------------------------------------------------------------------------------- */
int qo_threshold_table(int32_t D, uint64_t *T)
{
    if (D < 4 || D % 4 != 0) return 1;
    const int32_t K = D / 4;
    const double two32 = 4294967296.0;
    for (int32_t n = 0; n <= K; ++n) {
        double s = sin((double)n * M_PI / (double)D);
        T[n] = (uint64_t)llround(s * s * two32);
    }
    for (int32_t n = K + 1; n <= 2 * K; ++n)
        T[n] = (1ull << 32) - T[2 * K - n];
    return 0;
}

/* Observation of one qubit with angle index n (0 .. 2K) under draw u (reading S6). */
int qo_observe(int32_t n, uint32_t u, const uint64_t *T)
{
    return (uint64_t)u < T[n] ? 1 : 0;
}

/* ------------------------------------------------------------------------------------
 * Evaluation, eq. (1).
 * ---------------------------------------------------------------------------------- */
int64_t qo_fitness(int32_t ng, const int32_t *w, const int32_t *v, int64_t W,
                   int64_t lambda, const uint8_t *x)
{
    int64_t sw = 0, sv = 0;
    for (int32_t j = 0; j < ng; ++j) {
        if (x[j]) {
            sw += w[j];
            sv += v[j];
        }
    }
    if (sw <= W) return sv;
    return -lambda * (sw - W);
}

/* DetermineElite: the lowest chromosome index among those of largest fitness (S8, S9). */
int32_t qo_determine_elite(int32_t np, const int64_t *f)
{
    int32_t e = 0;
    for (int32_t c = 1; c < np; ++c)
        if (f[c] > f[e]) e = c;
    return e;
}

/* Largest eq. (1) value over all 2^ng subsets; ng <= 24. Returns the optimal subset in
 * best_x (lowest subset index among ties). */
int64_t qo_bruteforce(int32_t ng, const int32_t *w, const int32_t *v, int64_t W,
                      int64_t lambda, uint8_t *best_x)
{
    if (ng < 1 || ng > 24) return INT64_MIN;
    uint8_t *x = (uint8_t *)calloc((size_t)ng, 1);
    int64_t best = INT64_MIN;
    for (uint32_t s = 0; s < (1u << ng); ++s) {
        for (int32_t j = 0; j < ng; ++j) x[j] = (uint8_t)((s >> j) & 1u);
        int64_t f = qo_fitness(ng, w, v, W, lambda, x);
        if (f > best) {
            best = f;
            if (best_x) memcpy(best_x, x, (size_t)ng);
        }
    }
    free(x);
    return best;
}

static int check_args(int32_t ng, const int32_t *w, int32_t np, int32_t D, int64_t lambda,
                      int32_t rule)
{
    if (ng < 1 || np < 1 || D < 4 || D % 4 != 0 || lambda <= 0) return 1;
    if (rule != 0 && rule != 1) return 1;
    for (int32_t j = 0; j < ng; ++j)
        if (w[j] < 0) return 1;
    return 0;
}

/* ------------------------------------------------------------------------------------
 * The generation loop in the angle-index form: a qubit is stored as the integer k in
 * [-K, K] with theta = pi/4 + k pi/D, so alpha = cos(theta), beta = sin(theta).
 *
 * In/out: k[np*ng] (row c is chromosome c, gene-fastest), *t (absolute generation of
 * the next generation), best[3] = {best fitness, generation (-1 = none), chromosome},
 * best_x[ng]. Out: x[np*ng] and f[np] of the last generation run, hist_e[G] and
 * hist_f[G] the elite index and fitness of each generation run.
 * Runs G generations; each is QIP, Evaluation, DetermineElite, CIP (Fig. 1).
 *
 * Convergence (Sec. IV, Workload): the run stops once the elite fitness has been the same
 * for `window` consecutive generations (reading S15: the fitness values are integers, so
 * "within 1e-6 of their mean" means equal); the generation cap is G. window = 0 turns the
 * test off. conv[3] carries the test across calls: {length of the run of equal elite
 * fitness values ending at the last generation, 1 once stopped, that fitness}. A stopped
 * instance runs no further generation. Returns the number of generations run in *done.
 * ---------------------------------------------------------------------------------- */
static int run_loop(int32_t ng, const int32_t *w, const int32_t *v, int64_t W,
                    int32_t np, int32_t D, int64_t lambda, uint32_t seed, uint32_t inst,
                    int32_t rule, int32_t G, int16_t *k, int32_t *t, int64_t *best,
                    uint8_t *best_x, uint8_t *x, int64_t *f, int32_t *hist_e, int64_t *hist_f,
                    int32_t window, int64_t *conv, int32_t *done)
{
    if (check_args(ng, w, np, D, lambda, rule) || G < 0 || window < 0) return 1;
    const int32_t K = D / 4;
    uint64_t *T = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * K + 1));
    qo_threshold_table(D, T);
    *done = 0;

    for (int32_t g = 0; g < G; ++g) {
        if (window > 0 && conv[1]) break;
        const int32_t gen = *t;

        /* QIP: observe every qubit; Evaluation: eq. (1) per chromosome. */
#pragma omp parallel for schedule(static)
        for (int32_t c = 0; c < np; ++c) {
            int16_t *kc = k + (size_t)c * ng;
            uint8_t *xc = x + (size_t)c * ng;
            for (int32_t j = 0; j < ng; ++j) {
                uint32_t u = draw(seed, inst, gen, c, j);
                xc[j] = (uint8_t)qo_observe(kc[j] + K, u, T);
            }
            f[c] = qo_fitness(ng, w, v, W, lambda, xc);
        }

        /* DetermineElite. */
        const int32_t e = qo_determine_elite(np, f);
        hist_e[g] = e;
        hist_f[g] = f[e];
        if (best[1] < 0 || f[e] > best[0]) {
            best[0] = f[e];
            best[1] = gen;
            best[2] = e;
            memcpy(best_x, x + (size_t)e * ng, (size_t)ng);
        }

        /* CIP: one step toward the elite's allele, saturating at theta in {0, pi/2}. */
        const uint8_t *xe = x + (size_t)e * ng;
#pragma omp parallel for schedule(static)
        for (int32_t c = 0; c < np; ++c) {
            int16_t *kc = k + (size_t)c * ng;
            const uint8_t *xc = x + (size_t)c * ng;
            for (int32_t j = 0; j < ng; ++j) {
                if (rule == 1 && xc[j] == xe[j]) continue;
                int32_t step = xe[j] ? 1 : -1;
                int32_t kn = kc[j] + step;
                if (kn >= -K && kn <= K) kc[j] = (int16_t)kn;
            }
        }
        *t = gen + 1;
        *done = g + 1;

        /* Convergence test on the elite fitness of the generations so far. */
        if (window > 0) {
            conv[0] = (gen > 0 && conv[0] > 0 && f[e] == conv[2]) ? conv[0] + 1 : 1;
            conv[2] = f[e];
            if (conv[0] >= window) conv[1] = 1;
        }
    }
    free(T);
    return 0;
}

int qo_run(int32_t ng, const int32_t *w, const int32_t *v, int64_t W,
           int32_t np, int32_t D, int64_t lambda, uint32_t seed, uint32_t inst, int32_t rule,
           int32_t G, int16_t *k, int32_t *t, int64_t *best, uint8_t *best_x,
           uint8_t *x, int64_t *f, int32_t *hist_e, int64_t *hist_f)
{
    int32_t done = 0;
    return run_loop(ng, w, v, W, np, D, lambda, seed, inst, rule, G, k, t, best, best_x, x, f,
                    hist_e, hist_f, 0, NULL, &done);
}

int qo_run_converge(int32_t ng, const int32_t *w, const int32_t *v, int64_t W,
                    int32_t np, int32_t D, int64_t lambda, uint32_t seed, uint32_t inst,
                    int32_t rule, int32_t G, int16_t *k, int32_t *t, int64_t *best,
                    uint8_t *best_x, uint8_t *x, int64_t *f, int32_t *hist_e, int64_t *hist_f,
                    int32_t window, int64_t *conv, int32_t *done)
{
    return run_loop(ng, w, v, W, np, D, lambda, seed, inst, rule, G, k, t, best, best_x, x, f,
                    hist_e, hist_f, window, conv, done);
}

/* ------------------------------------------------------------------------------------
 * The same generation split by rows, for an instance whose population is divided into
 * row blocks (one per process): the QIP and Evaluation bullets of Sec. III-B on rows
 * [c0, c0 + nr) only, and the CIP bullet on a block toward an elite row that the caller
 * found over all blocks. Draws stay keyed by the global chromosome index (reading S7), so
 * the blocks together compute exactly what qo_run computes for the whole population.
 *
 * qo_rows_observe: in k[nr*ng] (the block's angle indices); out x[nr*ng], f[nr].
 * qo_rows_rotate:  in/out k[nr*ng]; in x[nr*ng] (the block's alleles of the same
 *                  generation) and xe[ng] (the elite's alleles).
 * ---------------------------------------------------------------------------------- */
int qo_rows_observe(int32_t ng, const int32_t *w, const int32_t *v, int64_t W, int32_t D,
                    int64_t lambda, uint32_t seed, uint32_t inst, int32_t gen, int32_t c0,
                    int32_t nr, const int16_t *k, uint8_t *x, int64_t *f)
{
    if (check_args(ng, w, 1, D, lambda, 0) || c0 < 0 || nr < 0) return 1;
    const int32_t K = D / 4;
    uint64_t *T = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * K + 1));
    qo_threshold_table(D, T);
    for (int32_t i = 0; i < nr; ++i) {
        const int16_t *ki = k + (size_t)i * ng;
        uint8_t *xi = x + (size_t)i * ng;
        for (int32_t j = 0; j < ng; ++j)
            xi[j] = (uint8_t)qo_observe(ki[j] + K, draw(seed, inst, gen, c0 + i, j), T);
        f[i] = qo_fitness(ng, w, v, W, lambda, xi);
    }
    free(T);
    return 0;
}

int qo_rows_rotate(int32_t ng, int32_t D, int32_t rule, int32_t nr, int16_t *k,
                   const uint8_t *x, const uint8_t *xe)
{
    if (ng < 1 || D < 4 || D % 4 != 0 || (rule != 0 && rule != 1) || nr < 0) return 1;
    const int32_t K = D / 4;
    for (int32_t i = 0; i < nr; ++i) {
        int16_t *ki = k + (size_t)i * ng;
        const uint8_t *xi = x + (size_t)i * ng;
        for (int32_t j = 0; j < ng; ++j) {
            if (rule == 1 && xi[j] == xe[j]) continue;
            const int32_t kn = ki[j] + (xe[j] ? 1 : -1);
            if (kn >= -K && kn <= K) ki[j] = (int16_t)kn;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------
 * The same loop in the amplitude form: each qubit is the pair (alpha, beta), started at
 * (1/sqrt2, 1/sqrt2) and turned by the rotation matrix [[cos d, -sin d], [sin d, cos d]]
 * with d = +pi/D toward allele 1 and -pi/D toward allele 0; a turn that would take
 * atan2(beta, alpha) out of [0, pi/2] is not made. Observation uses the 32-bit
 * fixed point of beta^2 directly: x = 1 iff u < round(beta^2 2^32).
 *
 * Extra outputs: stats[0] = number of observations whose beta^2 2^32 lay within 2^-10
 * of a rounding boundary (near ties, where the two forms may legitimately differ),
 * stats_d[0] = max |alpha^2 + beta^2 - 1| seen.
 * ---------------------------------------------------------------------------------- */
int qo_run_fp64(int32_t ng, const int32_t *w, const int32_t *v, int64_t W,
                int32_t np, int32_t D, int64_t lambda, uint32_t seed, uint32_t inst,
                int32_t rule, int32_t G, double *alpha, double *beta, int32_t *t,
                int64_t *best, uint8_t *best_x, uint8_t *x, int64_t *f,
                int32_t *hist_e, int64_t *hist_f, int64_t *stats, double *stats_d)
{
    if (check_args(ng, w, np, D, lambda, rule) || G < 0) return 1;
    const double d = M_PI / (double)D;
    const double cd = cos(d), sd = sin(d);
    const double two32 = 4294967296.0;
    const double lo = -1e-9, hi = M_PI / 2.0 + 1e-9;
    int64_t near = 0;
    double norm_err = 0.0;

    for (int32_t g = 0; g < G; ++g) {
        const int32_t gen = *t;
        for (int32_t c = 0; c < np; ++c) {
            for (int32_t j = 0; j < ng; ++j) {
                size_t i = (size_t)c * ng + j;
                double p = beta[i] * beta[i] * two32;
                double frac = p - floor(p);
                if (fabs(frac - 0.5) < 1.0 / 1024.0) ++near;
                uint64_t thr = (uint64_t)llround(p);
                uint32_t u = draw(seed, inst, gen, c, j);
                x[i] = (uint8_t)((uint64_t)u < thr ? 1 : 0);
            }
            f[c] = qo_fitness(ng, w, v, W, lambda, x + (size_t)c * ng);
        }
        const int32_t e = qo_determine_elite(np, f);
        hist_e[g] = e;
        hist_f[g] = f[e];
        if (best[1] < 0 || f[e] > best[0]) {
            best[0] = f[e];
            best[1] = gen;
            best[2] = e;
            memcpy(best_x, x + (size_t)e * ng, (size_t)ng);
        }
        const uint8_t *xe = x + (size_t)e * ng;
        for (int32_t c = 0; c < np; ++c) {
            for (int32_t j = 0; j < ng; ++j) {
                size_t i = (size_t)c * ng + j;
                if (rule == 1 && x[i] == xe[j]) continue;
                double s = xe[j] ? sd : -sd;
                double a2 = cd * alpha[i] - s * beta[i];
                double b2 = s * alpha[i] + cd * beta[i];
                double th = atan2(b2, a2);
                if (th < lo || th > hi) continue;
                alpha[i] = a2;
                beta[i] = b2;
                double ne = fabs(a2 * a2 + b2 * b2 - 1.0);
                if (ne > norm_err) norm_err = ne;
            }
        }
        *t = gen + 1;
    }
    stats[0] += near;
    if (norm_err > stats_d[0]) stats_d[0] = norm_err;
    return 0;
}

/* Thread control of the OpenMP build (no effect in the serial build). */
int qo_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int qo_is_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
