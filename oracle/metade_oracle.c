/*
 * metade_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the MetaDE hot path: the
 * parameterised DE (PDE) generation step of Alg. 2, its mutation (Eq. of
 * Sec. III-A-2, "DE/bl-to-br/dn"), the three crossover schemes of Sec. II-A
 * (binomial, exponential, arithmetic), greedy selection (Alg. 1/2), the
 * best-fitness reduction that becomes the meta-fitness (Sec. III-B), the
 * evolver's rand/1/bin step with floor decoding (Alg. 3), the PSO, CSO and
 * NES evolvers of the supplement's comparison of evolvers, and the synthetic shifted-rotated
 * objectives used as the CEC2022 stand-in.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this file.  It shares no code, header or table with the CUDA path;
 * the random numbers it draws come from its own Philox4x32-10, written from
 * the published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11).
 *
 * Readings of points the paper leaves open (each one also has a test):
 *  - generational ("tensorised", Alg. 2): every trial of a generation is
 *    built from the population as it was at the start of that generation;
 *  - "rand <= CR" is taken as the strict integer compare (w >> 8) < ceil(CR 2^24)
 *    with CR held as a float32 value, so CR = 0 never and CR = 1 always passes;
 *  - j_rand, the exponential start n and the pbest pick are 0-based;
 *  - exponential length L: L = 1, then L grows while L < D and the L-th
 *    uniform (0-based L-1) is below CR;
 *  - K_i is one uniform per individual; it is drawn but unused unless the
 *    crossover scheme is arithmetic;
 *  - all rand indices of one individual are mutually distinct and differ from
 *    i; best, pbest and current are not constrained (JADE convention);
 *  - pbest: top k_p = max(1, ceil(NP * pct / 100)) by stored fitness, ties by
 *    lower index; best is the first of that order;
 *  - trial vectors are clipped to the box [lo, hi];
 *  - NaN fitness counts as +inf; a tie accepts the trial (f(u) <= f(x)).
 *
 * Draw layout (both implementations follow it independently):
 *   key     = (seed_lo32, seed_hi32 ^ TAG)          TAG_INNER / TAG_OUTER
 *   counter = (stream, generation, individual, (epoch << 16) | slot)
 *   inner slot 0      : [j_rand, exp start n, K_i, pbest pick]
 *   inner slots 1..3  : rand index draws t = 0..8 (word t % 4 of slot 1 + t/4)
 *   inner slot 4+j/4  : crossover uniform of coordinate j (word j % 4)
 *   initialisation    : generation 0xFFFFFFFF, slot j/4 word j%4 -> coordinate j
 *   outer slot 0      : [j_rand]; slot 1: three rand draws; slots 2,3: genes 0..5
 *   uniform           : (w >> 8) * 2^-24;   integer in [0, m): floor(w m / 2^32)
 *   t-th distinct draw: s = floor(w_t (NP-1-t) / 2^32); the s-th smallest
 *                       member of {0..NP-1} \ ({i} U {r_0..r_{t-1}})
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TAG_INNER 0x4D455441u
#define OR_TAG_OUTER 0x4F555445u
#define OR_INIT_GEN 0xFFFFFFFFu
#define OR_REC 18 /* int32 record fields per individual, see or_pde_step */

static const double OR_PI = 3.14159265358979323846;
static const double OR_E = 2.71828182845904523536;

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds (SC'11, Sec. 3.2/Table 2): each round multiplies
 * counter words 0 and 2 by the two round constants, swaps the halves and
 * mixes in the key; the key is bumped by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
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

static void or_slot(uint64_t seed, uint32_t tag, uint32_t stream, uint32_t gen,
                    uint32_t indiv, uint32_t epoch, uint32_t slot, uint32_t w[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ tag};
    uint32_t ctr[4] = {stream, gen, indiv, (epoch << 16) | slot};
    or_philox4x32_10(ctr, key, w);
}

/* word t of the stream that starts at slot `first` */
static uint32_t or_word(uint64_t seed, uint32_t tag, uint32_t stream, uint32_t gen,
                        uint32_t indiv, uint32_t epoch, uint32_t first, uint32_t t)
{
    uint32_t w[4];
    or_slot(seed, tag, stream, gen, indiv, epoch, first + t / 4, w);
    return w[t % 4];
}

static double or_uniform(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

static uint32_t or_below(uint32_t w, uint32_t m) { return (uint32_t)(((uint64_t)w * m) >> 32); }

/* probability threshold: U < p  <=>  (w >> 8) < ceil(p * 2^24), p taken as float32 */
static uint32_t or_threshold(double p)
{
    float pf = (float)p;
    if (!(pf > 0.0f)) return 0u;
    if (pf >= 1.0f) return 16777216u;
    return (uint32_t)ceil((double)pf * 16777216.0);
}

/* The t-th distinct draw, written as the plain definition: list the
 * admissible indices in increasing order and take the s-th one. */
int or_distinct_draws(int np, int i, int m, const uint32_t *w, int32_t *r)
{
    if (m > np - 1) return -1;
    int *cand = (int *)malloc(sizeof(int) * (size_t)np);
    for (int t = 0; t < m; t++) {
        int n = 0;
        for (int c = 0; c < np; c++) {
            int taken = (c == i);
            for (int q = 0; q < t; q++) taken |= (c == r[q]);
            if (!taken) cand[n++] = c;
        }
        uint32_t s = or_below(w[t], (uint32_t)(np - 1 - t));
        r[t] = cand[s];
    }
    free(cand);
    return 0;
}

/* ------------------------------------------------------------ objectives */

/* z = R (x - o), R row-major */
static void or_rotate(int dim, const double *x, const double *o, const double *R, double *z)
{
    for (int r = 0; r < dim; r++) {
        double acc = 0.0;
        for (int c = 0; c < dim; c++) acc += R[(size_t)r * dim + c] * (x[c] - o[c]);
        z[r] = acc;
    }
}

/* Textbook objective definitions on the rotated vector z. */
double or_objective(int obj, int dim, const double *z)
{
    double f = 0.0;
    switch (obj) {
    case 0: /* sphere */
        for (int j = 0; j < dim; j++) f += z[j] * z[j];
        return f;
    case 1: /* Rosenbrock evaluated on y = z + 1, so that the optimum sits at z = 0 */
        for (int j = 0; j + 1 < dim; j++) {
            double y0 = z[j] + 1.0, y1 = z[j + 1] + 1.0;
            f += 100.0 * (y1 - y0 * y0) * (y1 - y0 * y0) + (y0 - 1.0) * (y0 - 1.0);
        }
        return f;
    case 2: /* Rastrigin */
        for (int j = 0; j < dim; j++) f += z[j] * z[j] - 10.0 * cos(2.0 * OR_PI * z[j]) + 10.0;
        return f;
    case 3: { /* Griewank */
        double s = 0.0, p = 1.0;
        for (int j = 0; j < dim; j++) {
            s += z[j] * z[j] / 4000.0;
            p *= cos(z[j] / sqrt((double)(j + 1)));
        }
        return s - p + 1.0;
    }
    case 4: { /* Ackley */
        double s = 0.0, c = 0.0;
        for (int j = 0; j < dim; j++) {
            s += z[j] * z[j];
            c += cos(2.0 * OR_PI * z[j]);
        }
        return -20.0 * exp(-0.2 * sqrt(s / dim)) - exp(c / dim) + 20.0 + OR_E;
    }
    case 5: { /* Schwefel 1.2 (6, the MLP objective, is evaluated by or_eval on the parameters) */
        double pre = 0.0;
        for (int j = 0; j < dim; j++) {
            pre += z[j];
            f += pre * pre;
        }
        return f;
    }
    default:
        return NAN;
    }
}

/* ------------------------------------------- MLP regression objective (6)
 * A neuroevolution-like large-D objective: theta holds the parameters of a
 * 16-h-2 perceptron with one tanh hidden layer, laid out as W1 [16][h]
 * (index k h + j), b1 [h], W2 [h][2] (index j 2 + o), b2 [2], so D = 19 h + 2.
 * The teacher is the problem's shift vector o, so f(o) = 0 like every other
 * objective here.  f(theta) is the mean over N = 256 inputs and the two
 * outputs of (y_theta - y_o)^2.  The inputs are uniform in [-1, 1]: input n,
 * coordinate k is 2 U - 1 with U from Philox key (0, 0 ^ TAG_DATA), counter
 * (0, 0, n, k / 4), word k % 4 (the same counter-based generator as every
 * other draw). */
#define OR_TAG_DATA 0x4D4C5044u
#define OR_MLP_IN 16
#define OR_MLP_OUT 2
#define OR_MLP_N 256

int or_mlp_hidden(int dim) { return (dim >= 21 && (dim - 2) % 19 == 0) ? (dim - 2) / 19 : 0; }

void or_mlp_inputs(double *X)
{
    for (int n = 0; n < OR_MLP_N; n++)
        for (int k = 0; k < OR_MLP_IN; k++)
            X[n * OR_MLP_IN + k] = 2.0 * or_uniform(or_word(0, OR_TAG_DATA, 0, 0, (uint32_t)n, 0, 0, (uint32_t)k)) - 1.0;
}

static void or_mlp_forward(int h, const double *th, const double *x, double *y)
{
    const double *W1 = th, *b1 = th + OR_MLP_IN * h, *W2 = b1 + h, *b2 = W2 + h * OR_MLP_OUT;
    for (int o = 0; o < OR_MLP_OUT; o++) y[o] = b2[o];
    for (int j = 0; j < h; j++) {
        double a = b1[j];
        for (int k = 0; k < OR_MLP_IN; k++) a += x[k] * W1[k * h + j];
        double t = tanh(a);
        for (int o = 0; o < OR_MLP_OUT; o++) y[o] += t * W2[j * OR_MLP_OUT + o];
    }
}

double or_mlp(int dim, const double *theta, const double *teacher)
{
    static double X[OR_MLP_N * OR_MLP_IN];
    static int have_x = 0;
    int h = or_mlp_hidden(dim);
    if (!h) return NAN;
    if (!have_x) {
        or_mlp_inputs(X);
        have_x = 1;
    }
    double s = 0.0;
    for (int n = 0; n < OR_MLP_N; n++) {
        double yt[OR_MLP_OUT], y[OR_MLP_OUT];
        or_mlp_forward(h, teacher, X + n * OR_MLP_IN, yt);
        or_mlp_forward(h, theta, X + n * OR_MLP_IN, y);
        for (int o = 0; o < OR_MLP_OUT; o++) s += (y[o] - yt[o]) * (y[o] - yt[o]);
    }
    return s / (OR_MLP_N * OR_MLP_OUT);
}

double or_eval(int obj, int dim, const double *x, const double *o, const double *R)
{
    if (obj == 6) return or_mlp(dim, x, o);  /* no rotation: f of the parameters themselves */
    double *z = (double *)malloc(sizeof(double) * (size_t)(dim > 0 ? dim : 1));
    or_rotate(dim, x, o, R, z);
    double f = or_objective(obj, dim, z);
    free(z);
    return f;
}

static double or_fitness(int obj, int dim, const double *x, const double *o, const double *R)
{
    double f = or_eval(obj, dim, x, o, R);
    return isnan(f) ? INFINITY : f;
}

/* ------------------------------------------------------- initialisation */

/* Alg. 2 and Alg. 1, initialisation: uniform in the box. */
void or_init_pop(int np, int dim, uint64_t seed, uint32_t stream, uint32_t epoch,
                 double lo, double hi, double *pop)
{
    for (int i = 0; i < np; i++)
        for (int j = 0; j < dim; j++) {
            uint32_t w = or_word(seed, OR_TAG_INNER, stream, OR_INIT_GEN, (uint32_t)i, epoch, 0, (uint32_t)j);
            pop[(size_t)i * dim + j] = lo + (hi - lo) * or_uniform(w);
        }
}

/* Alg. 2, evaluation of the initial population */
void or_eval_pop(int np, int dim, int obj, const double *o, const double *R,
                 const double *pop, double *fit)
{
    for (int i = 0; i < np; i++) fit[i] = or_fitness(obj, dim, pop + (size_t)i * dim, o, R);
}

/* ------------------------------------------------------------ PDE step */

static int or_kp(int np, int pct)
{
    int k = (np * pct + 99) / 100;
    return k < 1 ? 1 : k;
}

/* indices sorted by (fitness, index) ascending: insertion sort, plain */
static void or_order(int np, const double *fit, int *order)
{
    for (int i = 0; i < np; i++) {
        int j = i;
        while (j > 0) {
            int a = order[j - 1];
            if (fit[a] > fit[i] || (fit[a] == fit[i] && a > i)) {
                order[j] = order[j - 1];
                j--;
            } else break;
        }
        order[j] = i;
    }
}

int or_required_np(int bl, int br, int dn)
{
    int a = (bl == 1 || br == 1) ? 1 : 0;
    return a + 2 * dn + 1;
}

/*
 * One generation of PDE (Alg. 2) on one instance, in place.
 *
 * pop [np*dim], fit [np]: the generation-start state (in), the next state (out).
 * theta = (F, CR, bl, br, dn, cs), categorical entries integral.
 * Optional outputs (NULL to skip):
 *   trial [np*dim], ftrial [np], accept [np],
 *   mask [np*dim] (1 where the trial coordinate came from the mutant; all 1
 *        for arithmetic recombination),
 *   rec [np*OR_REC]: base-left index, base-right index, j_rand, exp start n,
 *        exp length L (0 unless exponential), K_i raw 24-bit value, pbest
 *        index, best index, m, r_0..r_8 (-1 when unused).
 * Returns 0, or -1 when np is too small for the strategy, -2 on bad theta.
 */
int or_pde_step(int np, int dim, int obj, const double *o, const double *R,
                double lo, double hi, uint64_t seed, uint32_t stream, uint32_t epoch, uint32_t gen,
                int p_best_pct, const double *theta, double *pop, double *fit,
                double *trial, double *ftrial, int32_t *accept, uint8_t *mask, int32_t *rec)
{
    double F = theta[0], CR = theta[1];
    int bl = (int)theta[2], br = (int)theta[3], dn = (int)theta[4], cs = (int)theta[5];
    if (bl < 1 || bl > 4 || br < 1 || br > 4 || dn < 1 || dn > 4 || cs < 1 || cs > 3) return -2;
    if (np < or_required_np(bl, br, dn) || dim < 1) return -1;

    int a = (bl == 1 || br == 1) ? 1 : 0;
    int m = a + 2 * dn;
    int kp = or_kp(np, p_best_pct);
    uint32_t cri = or_threshold(CR);

    int *order = (int *)malloc(sizeof(int) * (size_t)np);
    or_order(np, fit, order);
    int best = order[0];

    double *U = (double *)malloc(sizeof(double) * (size_t)np * dim);
    double *fU = (double *)malloc(sizeof(double) * (size_t)np);
    uint8_t *M = (uint8_t *)malloc((size_t)np * dim);
    double *v = (double *)malloc(sizeof(double) * (size_t)dim);

    for (int i = 0; i < np; i++) {
        uint32_t w0[4];
        or_slot(seed, OR_TAG_INNER, stream, gen, (uint32_t)i, epoch, 0, w0);
        int jrand = (int)or_below(w0[0], (uint32_t)dim);
        int nstart = (int)or_below(w0[1], (uint32_t)dim);
        uint32_t kraw = w0[2] >> 8;
        double K = or_uniform(w0[2]);
        int pbest = order[or_below(w0[3], (uint32_t)kp)];

        uint32_t wr[9];
        int32_t r[9];
        for (int t = 0; t < 9; t++) r[t] = -1;
        for (int t = 0; t < m; t++) wr[t] = or_word(seed, OR_TAG_INNER, stream, gen, (uint32_t)i, epoch, 1, (uint32_t)t);
        or_distinct_draws(np, i, m, wr, r);

        int ib[5];
        ib[1] = r[0]; /* meaningful only when a rand base is used */
        ib[2] = best;
        ib[3] = pbest;
        ib[4] = i;
        const double *xl = pop + (size_t)ib[bl] * dim;
        const double *xr = pop + (size_t)ib[br] * dim;
        const double *xi = pop + (size_t)i * dim;

        /* Eq. (PDE mutation): v = x_bl + F (x_br - x_bl) + F (D_1 + ... + D_dn) */
        for (int j = 0; j < dim; j++) {
            double sum = 0.0;
            for (int q = 0; q < dn; q++)
                sum += pop[(size_t)r[a + 2 * q] * dim + j] - pop[(size_t)r[a + 2 * q + 1] * dim + j];
            double dir = (bl != br) ? F * (xr[j] - xl[j]) : 0.0;
            v[j] = xl[j] + dir + F * sum;
        }

        /* crossover, Sec. II-A */
        double *u = U + (size_t)i * dim;
        uint8_t *mk = M + (size_t)i * dim;
        int L = 0;
        if (cs == 1) { /* binomial */
            for (int j = 0; j < dim; j++) {
                uint32_t w = or_word(seed, OR_TAG_INNER, stream, gen, (uint32_t)i, epoch, 4, (uint32_t)j);
                int take = ((w >> 8) < cri) || (j == jrand);
                mk[j] = (uint8_t)take;
                u[j] = take ? v[j] : xi[j];
            }
        } else if (cs == 2) { /* exponential: a cyclic run of L coordinates from n */
            L = 1;
            while (L < dim) {
                uint32_t w = or_word(seed, OR_TAG_INNER, stream, gen, (uint32_t)i, epoch, 4, (uint32_t)(L - 1));
                if ((w >> 8) < cri) L++;
                else break;
            }
            for (int j = 0; j < dim; j++) mk[j] = 0;
            for (int l = 0; l < L; l++) mk[(nstart + l) % dim] = 1;
            for (int j = 0; j < dim; j++) u[j] = mk[j] ? v[j] : xi[j];
        } else { /* arithmetic recombination */
            for (int j = 0; j < dim; j++) {
                mk[j] = 1;
                u[j] = xi[j] + K * (v[j] - xi[j]);
            }
        }
        for (int j = 0; j < dim; j++) {
            if (u[j] < lo) u[j] = lo;
            if (u[j] > hi) u[j] = hi;
        }
        fU[i] = or_fitness(obj, dim, u, o, R);

        if (rec) {
            int32_t *q = rec + (size_t)i * OR_REC;
            q[0] = ib[bl];
            q[1] = ib[br];
            q[2] = jrand;
            q[3] = nstart;
            q[4] = L;
            q[5] = (int32_t)kraw;
            q[6] = pbest;
            q[7] = best;
            q[8] = m;
            for (int t = 0; t < 9; t++) q[9 + t] = r[t];
        }
    }

    /* Alg. 2, selection: greedy selection, all trials against the start population */
    for (int i = 0; i < np; i++) {
        int acc = fU[i] <= fit[i];
        if (accept) accept[i] = acc;
        if (trial) memcpy(trial + (size_t)i * dim, U + (size_t)i * dim, sizeof(double) * (size_t)dim);
        if (ftrial) ftrial[i] = fU[i];
        if (mask) memcpy(mask + (size_t)i * dim, M + (size_t)i * dim, (size_t)dim);
        if (acc) {
            memcpy(pop + (size_t)i * dim, U + (size_t)i * dim, sizeof(double) * (size_t)dim);
            fit[i] = fU[i];
        }
    }
    free(order); free(U); free(fU); free(M); free(v);
    return 0;
}

/* Best fitness and its index (lowest index on ties): the executor's y*. */
double or_best(int np, const double *fit, int32_t *best_index)
{
    int b = 0;
    for (int i = 1; i < np; i++)
        if (fit[i] < fit[b]) b = i;
    if (best_index) *best_index = b;
    return fit[b];
}

/* A whole PDE run (Alg. 2): initialise, evaluate, `gens` generations; returns y*. */
double or_pde_run(int np, int dim, int obj, const double *o, const double *R,
                  double lo, double hi, uint64_t seed, uint32_t stream, uint32_t epoch,
                  int p_best_pct, const double *theta, int gens, double *pop, double *fit)
{
    or_init_pop(np, dim, seed, stream, epoch, lo, hi, pop);
    or_eval_pop(np, dim, obj, o, R, pop, fit);
    for (int g = 0; g < gens; g++)
        if (or_pde_step(np, dim, obj, o, R, lo, hi, seed, stream, epoch, (uint32_t)g,
                        p_best_pct, theta, pop, fit, NULL, NULL, NULL, NULL, NULL) != 0)
            return NAN;
    return or_best(np, fit, NULL);
}

/* ------------------------------------------------------------- evolver */

static const double OR_LB[6] = {0.0, 0.0, 1.0, 1.0, 1.0, 1.0};
static const double OR_UB[6] = {1.0, 1.0, 5.0, 5.0, 5.0, 4.0};

/* Alg. 3, initialisation: evolver population uniform in [lb, ub], fitness +inf. */
void or_outer_init(int n_out, uint64_t seed, uint32_t group, double *pop, double *fit)
{
    for (int i = 0; i < n_out; i++) {
        for (int j = 0; j < 6; j++) {
            uint32_t w = or_word(seed, OR_TAG_OUTER, group, OR_INIT_GEN, (uint32_t)i, 0, 0, (uint32_t)j);
            pop[i * 6 + j] = OR_LB[j] + (OR_UB[j] - OR_LB[j]) * or_uniform(w);
        }
        fit[i] = INFINITY;
    }
}

/* Alg. 3, trial generation: rand/1/bin trials with F = 0.5, CR = 0.9 (Sec. IV-A),
 * clipped to [lb, ub].  Returns -1 when n_out < 4. */
int or_outer_trial(int n_out, uint64_t seed, uint32_t group, uint32_t gen,
                   const double *pop, double *trial)
{
    if (n_out < 4) return -1;
    const double F = 0.5;
    uint32_t cri = or_threshold(0.9);
    for (int i = 0; i < n_out; i++) {
        uint32_t w0[4], w1[4];
        or_slot(seed, OR_TAG_OUTER, group, gen, (uint32_t)i, 0, 0, w0);
        or_slot(seed, OR_TAG_OUTER, group, gen, (uint32_t)i, 0, 1, w1);
        int jrand = (int)or_below(w0[0], 6u);
        int32_t r[3];
        or_distinct_draws(n_out, i, 3, w1, r);
        for (int j = 0; j < 6; j++) {
            double v = pop[r[0] * 6 + j] + F * (pop[r[1] * 6 + j] - pop[r[2] * 6 + j]);
            uint32_t w = or_word(seed, OR_TAG_OUTER, group, gen, (uint32_t)i, 0, 2, (uint32_t)j);
            int take = ((w >> 8) < cri) || (j == jrand);
            double u = take ? v : pop[i * 6 + j];
            if (u < OR_LB[j]) u = OR_LB[j];
            if (u > OR_UB[j]) u = OR_UB[j];
            trial[i * 6 + j] = u;
        }
    }
    return 0;
}

/* Alg. 3, decoding: F = u1, CR = u2, bl/br/dn/cs = floor of u3..u6, clamped to
 * their domains so that the upper bound decodes to the top category. */
void or_decode(const double *u, double *theta)
{
    static const int top[6] = {0, 0, 4, 4, 4, 3};
    theta[0] = u[0];
    theta[1] = u[1];
    for (int j = 2; j < 6; j++) {
        double c = floor(u[j]);
        if (c < 1.0) c = 1.0;
        if (c > top[j]) c = top[j];
        theta[j] = c;
    }
}

/* Alg. 3, selection: a trial replaces its parent when its meta-fitness is <=. */
void or_outer_select(int n_out, double *pop, double *fit, const double *trial,
                     const double *meta_fit, int32_t *accept)
{
    for (int i = 0; i < n_out; i++) {
        double y = isnan(meta_fit[i]) ? INFINITY : meta_fit[i];
        int acc = y <= fit[i];
        if (accept) accept[i] = acc;
        if (acc) {
            for (int j = 0; j < 6; j++) pop[i * 6 + j] = trial[i * 6 + j];
            fit[i] = y;
        }
    }
}

/*
 * PSO as the evolver (the supplement's comparison of evolvers: inertia
 * weight w and acceleration coefficients c1, c2; the paper sets w = 0.729,
 * c1 = c2 = 1.49).  Particle i has a position x (the vector evaluated this
 * generation), a velocity v, and a personal best pbest with fitness pfit,
 * which play the evolver population and fitness of Alg. 3.  Generation 0
 * evaluates the initial swarm: x = pbest (from or_outer_init), v = 0.  From
 * generation 1 every particle moves toward its own best and the run's best
 * gbest (the personal best of lowest fitness, ties to the lower index):
 *   v_j <- w v_j + c1 r1_j (pbest_j - x_j) + c2 r2_j (gbest_j - x_j)
 *   x_j <- x_j + v_j, clipped to [lb_j, ub_j] (v is kept as computed)
 * with r1_j, r2_j uniform in [0, 1): evolver draw slots 0-2, r1 = words
 * 0..5 and r2 = words 6..11 (slot = word / 4).  Selection is that of Alg. 3
 * (or_outer_select: x replaces pbest when its meta-fitness is <=).
 */
void or_pso_move(int n_out, uint64_t seed, uint32_t group, uint32_t gen, double w, double c1, double c2,
                 const double *pbest, const double *pfit, double *x, double *v)
{
    if (gen == 0) {
        for (int i = 0; i < n_out * 6; i++) {
            x[i] = pbest[i];
            v[i] = 0.0;
        }
        return;
    }
    int gb = 0;
    for (int i = 1; i < n_out; i++)
        if (pfit[i] < pfit[gb]) gb = i;
    for (int i = 0; i < n_out; i++) {
        for (int j = 0; j < 6; j++) {
            uint32_t a = or_word(seed, OR_TAG_OUTER, group, gen, (uint32_t)i, 0, (uint32_t)(j / 4), (uint32_t)(j % 4));
            uint32_t b = or_word(seed, OR_TAG_OUTER, group, gen, (uint32_t)i, 0, (uint32_t)((6 + j) / 4),
                                 (uint32_t)((6 + j) % 4));
            double r1 = (double)(a >> 8) / 16777216.0, r2 = (double)(b >> 8) / 16777216.0;
            double xi = x[i * 6 + j];
            double vi = w * v[i * 6 + j] + c1 * r1 * (pbest[i * 6 + j] - xi) + c2 * r2 * (pbest[gb * 6 + j] - xi);
            double xn = xi + vi;
            if (xn < OR_LB[j]) xn = OR_LB[j];
            if (xn > OR_UB[j]) xn = OR_UB[j];
            v[i * 6 + j] = vi;
            x[i * 6 + j] = xn;
        }
    }
}

/*
 * CSO as the evolver (Competitive Swarm Optimizer, Cheng and Jin, IEEE Trans.
 * Cybernetics 45(2), 2015; the supplement's comparison of evolvers uses it
 * without tuning).  Particle i has a position x_i (the evolver population
 * `pop`, fitness `fit`) and a velocity v_i.  Generation 0 evaluates the
 * initial swarm: x'_i = x_i, v_i = 0, every particle flagged.  From
 * generation 1 the swarm is paired at random: pi = a permutation of 0..m-1
 * by Fisher-Yates (pi = identity; for t = m-1 down to 1, j = int[0, t+1)
 * from evolver draw slot 3 word 0 of individual t, swap pi[t] and pi[j]);
 * pair p is (pi[2p], pi[2p+1]) and an odd last particle sits the generation
 * out.  In a pair the particle of lower fitness (ties to the lower index)
 * wins and is kept as it is; the loser l learns from the winner w:
 *   v_l,j <- r1_j v_l,j + r2_j (x_w,j - x_l,j)
 *   x'_l,j = x_l,j + v_l,j, clipped to [lb_j, ub_j]   (v is kept as computed)
 * with r1 = words 0..5 and r2 = words 6..11 of individual l (slots 0-2), as
 * in PSO.  The swarm-mean term of CSO is taken with its factor phi = 0 (the
 * setting Cheng and Jin give for small swarms; the supplement tunes nothing).
 * Selection (or_cso_select): a flagged particle (a loser, or any particle at
 * generation 0) takes x' and its meta-fitness unconditionally; a winner keeps
 * its position and stored fitness.
 */
void or_cso_move(int n_out, uint64_t seed, uint32_t group, uint32_t gen, const double *pop, const double *fit,
                 double *xn, double *v, int32_t *flag)
{
    for (int i = 0; i < n_out * 6; i++) xn[i] = pop[i];
    if (gen == 0) {
        for (int i = 0; i < n_out; i++) {
            flag[i] = 1;
            for (int j = 0; j < 6; j++) v[i * 6 + j] = 0.0;
        }
        return;
    }
    int32_t *pi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_out > 0 ? n_out : 1));
    for (int i = 0; i < n_out; i++) {
        pi[i] = i;
        flag[i] = 0;
    }
    for (int t = n_out - 1; t >= 1; t--) {
        uint32_t w = or_word(seed, OR_TAG_OUTER, group, gen, (uint32_t)t, 0, 3, 0);
        int j = (int)or_below(w, (uint32_t)(t + 1));
        int32_t tmp = pi[t];
        pi[t] = pi[j];
        pi[j] = tmp;
    }
    for (int q = 0; q + 1 < n_out; q += 2) {
        int a = pi[q], b = pi[q + 1];
        int a_wins = fit[a] < fit[b] || (fit[a] == fit[b] && a < b);
        int w = a_wins ? a : b, l = a_wins ? b : a;
        flag[l] = 1;
        for (int j = 0; j < 6; j++) {
            uint32_t wa = or_word(seed, OR_TAG_OUTER, group, gen, (uint32_t)l, 0, (uint32_t)(j / 4), (uint32_t)(j % 4));
            uint32_t wb = or_word(seed, OR_TAG_OUTER, group, gen, (uint32_t)l, 0, (uint32_t)((6 + j) / 4),
                                  (uint32_t)((6 + j) % 4));
            double r1 = or_uniform(wa), r2 = or_uniform(wb);
            double vj = r1 * v[l * 6 + j] + r2 * (pop[w * 6 + j] - pop[l * 6 + j]);
            double x = pop[l * 6 + j] + vj;
            if (x < OR_LB[j]) x = OR_LB[j];
            if (x > OR_UB[j]) x = OR_UB[j];
            v[l * 6 + j] = vj;
            xn[l * 6 + j] = x;
        }
    }
    free(pi);
}

void or_cso_select(int n_out, double *pop, double *fit, const double *xn, const int32_t *flag, const double *meta_fit)
{
    for (int i = 0; i < n_out; i++) {
        if (!flag[i]) continue;
        for (int j = 0; j < 6; j++) pop[i * 6 + j] = xn[i * 6 + j];
        fit[i] = isnan(meta_fit[i]) ? INFINITY : meta_fit[i];
    }
}

/*
 * NES as the evolver: exponential natural evolution strategies (xNES,
 * Wierstra, Schaul, Glasmachers, Sun, Peters, Schmidhuber, "Natural
 * Evolution Strategies", JMLR 15, 2014), whose learning rates have fixed
 * defaults (the supplement tunes nothing).  The search distribution over
 * the d = 6 genes is N(mu, sigma^2 B B^T) with det B = 1.  Generation t
 * draws lambda = n_out samples
 *   s_k ~ N(0, I): Box-Muller on evolver draw words 2q, 2q+1 (slot = word / 4)
 *       of individual k: u1 = ((w >> 8) + 1) 2^-24, u2 = (w >> 8) 2^-24,
 *       s_2q = sqrt(-2 ln u1) cos(2 pi u2), s_2q+1 = sqrt(-2 ln u1) sin(2 pi u2)
 *   z_k = mu + sigma B s_k, evaluated at clip(z_k, lb, ub) (floor-decoded).
 * With the samples ranked by meta-fitness (ascending, NaN as +inf, ties to
 * the lower index) and the utilities of rank r = 0..lambda-1
 *   u_r = max(0, ln(lambda/2 + 1) - ln(r + 1)) / sum_r' max(0, ...) - 1/lambda,
 * the natural-gradient step is
 *   G_delta = sum_k u_k s_k,  G_M = sum_k u_k (s_k s_k^T - I),
 *   G_sigma = tr(G_M) / d,    G_B = G_M - G_sigma I,
 *   mu <- mu + eta_mu sigma B G_delta,  sigma <- sigma exp(eta_sigma G_sigma / 2),
 *   B <- B expm(eta_B G_B / 2),
 * eta_mu = 1, eta_sigma = eta_B = 3 (3 + ln d) / (5 d sqrt d).  The initial
 * distribution is centred in the box, mu = (lb + ub) / 2, with
 * sigma B = diag((ub - lb) / 4): sigma = the geometric mean of (ub - lb) / 4
 * and B = diag((ub - lb) / 4) / sigma.  The evolver population and fitness
 * of Alg. 3 hold the latest samples clip(z_k) and their meta-fitness.
 * expm of the symmetric G_B here goes through a cyclic Jacobi
 * eigendecomposition, Q diag(exp(lambda_i)) Q^T.
 * State layout: st[0..5] = mu, st[6] = sigma, st[7..42] = B row-major.
 */
static const double OR_NES_D = 6.0;

void or_nes_init(double *st)
{
    double lg = 0.0;
    for (int j = 0; j < 6; j++) lg += log((OR_UB[j] - OR_LB[j]) / 4.0);
    double sigma = exp(lg / OR_NES_D);
    for (int j = 0; j < 6; j++) st[j] = 0.5 * (OR_LB[j] + OR_UB[j]);
    st[6] = sigma;
    for (int r = 0; r < 6; r++)
        for (int c = 0; c < 6; c++) st[7 + r * 6 + c] = (r == c) ? ((OR_UB[r] - OR_LB[r]) / 4.0) / sigma : 0.0;
}

/* Samples of generation `gen`: s [n_out][6], z [n_out][6] (unclipped), zc = clip(z). */
void or_nes_sample(int n_out, uint64_t seed, uint32_t group, uint32_t gen, const double *st, double *s, double *z,
                   double *zc)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < n_out; k++) {
        for (int q = 0; q < 3; q++) {
            uint32_t wa = or_word(seed, OR_TAG_OUTER, group, gen, (uint32_t)k, 0, (uint32_t)((2 * q) / 4),
                                  (uint32_t)((2 * q) % 4));
            uint32_t wb = or_word(seed, OR_TAG_OUTER, group, gen, (uint32_t)k, 0, (uint32_t)((2 * q + 1) / 4),
                                  (uint32_t)((2 * q + 1) % 4));
            double u1 = (double)((wa >> 8) + 1u) * (1.0 / 16777216.0);
            double u2 = (double)(wb >> 8) * (1.0 / 16777216.0);
            double rad = sqrt(-2.0 * log(u1));
            s[k * 6 + 2 * q] = rad * cos(two_pi * u2);
            s[k * 6 + 2 * q + 1] = rad * sin(two_pi * u2);
        }
        for (int r = 0; r < 6; r++) {
            double a = 0.0;
            for (int c = 0; c < 6; c++) a += st[7 + r * 6 + c] * s[k * 6 + c];
            double x = st[r] + st[6] * a;
            z[k * 6 + r] = x;
            if (x < OR_LB[r]) x = OR_LB[r];
            if (x > OR_UB[r]) x = OR_UB[r];
            zc[k * 6 + r] = x;
        }
    }
}

/* exp of a symmetric n x n matrix S (row-major) by cyclic Jacobi rotations. */
void or_expm_sym(int n, const double *S, double *E)
{
    double A[64], V[64];
    for (int i = 0; i < n * n; i++) A[i] = S[i];
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) off += A[p * n + q] * A[p * n + q];
        if (off < 1e-300) break;
        for (int p = 0; p < n; p++) {
            for (int q = p + 1; q < n; q++) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                /* rotation angle that zeroes A[p][q] (Golub and Van Loan, Sec. 8.5) */
                double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                for (int k = 0; k < n; k++) { /* A <- A J */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - sn * akq;
                    A[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; k++) { /* A <- J^T A */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - sn * aqk;
                    A[q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) { /* V <- V J */
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - sn * vkq;
                    V[k * n + q] = sn * vkp + c * vkq;
                }
            }
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double a = 0.0;
            for (int k = 0; k < n; k++) a += V[i * n + k] * exp(A[k * n + k]) * V[j * n + k];
            E[i * n + j] = a;
        }
}

/* The xNES update from one generation's samples s and meta-fitness y. */
void or_nes_update(int n_out, double *st, const double *s, const double *meta_fit)
{
    const int d = 6, lam = n_out;
    const double eta_mu = 1.0, eta = 3.0 * (3.0 + log(OR_NES_D)) / (5.0 * OR_NES_D * sqrt(OR_NES_D));
    double *u = (double *)malloc(sizeof(double) * (size_t)(lam > 0 ? lam : 1));
    double den = 0.0;
    for (int r = 0; r < lam; r++) {
        double a = log(lam / 2.0 + 1.0) - log(r + 1.0);
        den += a > 0.0 ? a : 0.0;
    }
    for (int k = 0; k < lam; k++) {
        double yk = isnan(meta_fit[k]) ? INFINITY : meta_fit[k];
        int rank = 0;
        for (int j = 0; j < lam; j++) {
            double yj = isnan(meta_fit[j]) ? INFINITY : meta_fit[j];
            if (yj < yk || (yj == yk && j < k)) rank++;
        }
        double a = log(lam / 2.0 + 1.0) - log(rank + 1.0);
        u[k] = (a > 0.0 ? a : 0.0) / den - 1.0 / lam;
    }
    double gd[6] = {0}, gm[36] = {0};
    for (int k = 0; k < lam; k++) {
        for (int i = 0; i < d; i++) {
            gd[i] += u[k] * s[k * 6 + i];
            for (int j = 0; j < d; j++) gm[i * 6 + j] += u[k] * (s[k * 6 + i] * s[k * 6 + j] - (i == j ? 1.0 : 0.0));
        }
    }
    double gs = 0.0;
    for (int i = 0; i < d; i++) gs += gm[i * 6 + i];
    gs /= d;
    double half[36], E[36], Bn[36];
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) half[i * 6 + j] = 0.5 * eta * (gm[i * 6 + j] - (i == j ? gs : 0.0));
    or_expm_sym(d, half, E);
    const double sigma = st[6];
    for (int i = 0; i < d; i++) {
        double a = 0.0;
        for (int j = 0; j < d; j++) a += st[7 + i * 6 + j] * gd[j];
        st[i] += eta_mu * sigma * a;
    }
    st[6] = sigma * exp(0.5 * eta * gs);
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) {
            double a = 0.0;
            for (int k = 0; k < d; k++) a += st[7 + i * 6 + k] * E[k * 6 + j];
            Bn[i * 6 + j] = a;
        }
    for (int i = 0; i < 36; i++) st[7 + i] = Bn[i];
    free(u);
}

/*
 * A whole MetaDE run (Alg. 3) for one problem, one-shot evaluation: every
 * executor starts from the same seed (stream = group, epoch 0).  `power_up`
 * gives the last evolver generation 5x the inner generations (Sec. III-D).
 * evolver: 0 DE/rand/1/bin (Alg. 3), 1 PSO, 2 CSO, 3 NES (xNES).
 * Writes the final evolver population/fitness; returns the best meta-fitness.
 */
double or_metade_run(int n_out, int np, int dim, int obj, const double *o, const double *R,
                     double lo, double hi, uint64_t seed, uint32_t group, int p_best_pct,
                     int inner_gens, int outer_gens, int power_up, int evolver,
                     double *opop, double *ofit)
{
    double *trial = (double *)malloc(sizeof(double) * (size_t)n_out * 6);
    double *vel = (double *)malloc(sizeof(double) * (size_t)n_out * 6);
    double *ns = (double *)malloc(sizeof(double) * (size_t)n_out * 6);
    int32_t *flag = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_out);
    double *yf = (double *)malloc(sizeof(double) * (size_t)n_out);
    double *pop = (double *)malloc(sizeof(double) * (size_t)np * dim);
    double *fit = (double *)malloc(sizeof(double) * (size_t)np);
    double nes[43];
    or_outer_init(n_out, seed, group, opop, ofit);
    if (evolver == 3) or_nes_init(nes);
    for (int g = 0; g < outer_gens; g++) {
        if (evolver == 1)
            or_pso_move(n_out, seed, group, (uint32_t)g, 0.729, 1.49, 1.49, opop, ofit, trial, vel);
        else if (evolver == 2)
            or_cso_move(n_out, seed, group, (uint32_t)g, opop, ofit, trial, vel, flag);
        else if (evolver == 3)
            or_nes_sample(n_out, seed, group, (uint32_t)g, nes, ns, vel, trial);
        else
            or_outer_trial(n_out, seed, group, (uint32_t)g, opop, trial);
        int gens = (power_up && g == outer_gens - 1) ? 5 * inner_gens : inner_gens;
        for (int k = 0; k < n_out; k++) {
            double th[6];
            or_decode(trial + k * 6, th);
            yf[k] = or_pde_run(np, dim, obj, o, R, lo, hi, seed, group, 0, p_best_pct, th, gens, pop, fit);
        }
        if (evolver == 2) {
            or_cso_select(n_out, opop, ofit, trial, flag, yf);
        } else if (evolver == 3) {
            or_nes_update(n_out, nes, ns, yf);
            for (int k = 0; k < n_out; k++) {
                for (int j = 0; j < 6; j++) opop[k * 6 + j] = trial[k * 6 + j];
                ofit[k] = isnan(yf[k]) ? INFINITY : yf[k];
            }
        } else {
            or_outer_select(n_out, opop, ofit, trial, yf, NULL);
        }
    }
    double b = ofit[0];
    for (int k = 1; k < n_out; k++)
        if (ofit[k] < b) b = ofit[k];
    free(trial); free(vel); free(ns); free(flag); free(yf); free(pop); free(fit);
    return b;
}
