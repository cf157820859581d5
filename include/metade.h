/*
 * metade.h -- C-ABI of the GB300 (sm_103a) MetaDE hot path.
 *
 * MetaDE (arXiv 2502.10470) evolves the hyperparameters of a parameterised
 * DE ("PDE", Sec. III-A) with an outer DE (the "evolver", Alg. 3).  Every
 * evolver vector u decodes into theta = (F, CR, bl, br, dn, cs) and drives its
 * own inner DE (an "executor", Alg. 2) on the target objective; the best
 * fitness an executor reaches is the meta-fitness the evolver selects on
 * (Sec. III-B).  This library runs the executors' generations -- index
 * draws, mutation, crossover, objective evaluation, greedy selection and the
 * best-fitness reduction -- for hundreds of executors at once, plus the
 * evolver's trial/decode/selection steps.
 *
 * Conventions shared by every entry point:
 *  - All state is caller-owned DEVICE memory (e.g. torch tensors); the
 *    library owns only its context: descriptor table, padded copies of the
 *    problem data, scratch, the tuned plan and captured CUDA graphs.
 *  - Calls are asynchronous on the context's stream.  Host-detectable errors
 *    are returned at once; errors found on the device (an invalid theta, a
 *    population too small for the strategy) are latched in a sticky status
 *    word that metade_sync() returns and clears.  Nothing is thrown across
 *    the ABI.  On error no output is guaranteed to be written.
 *  - A problem p has dimension D_p, an objective id, a shift o_p and a
 *    rotation R_p; its objective is f(x) = obj(z), z = R_p (x - o_p).
 *    Objective ids: 0 sphere, 1 Rosenbrock on z + 1, 2 Rastrigin,
 *    3 Griewank, 4 Ackley, 5 Schwefel 1.2 (all with minimum 0 at x = o_p).
 *    Id 6 is a neuroevolution-like regression problem (the paper's policy
 *    search, made synthetic): x holds the parameters of a 16-h-2 perceptron
 *    with one tanh hidden layer, laid out W1 [16][h] (k h + j), b1 [h],
 *    W2 [h][2] (2 j + o), b2 [2], so D_p = 19 h + 2 (other D_p: EINVAL).  f is
 *    the mean over 256 fixed inputs (uniform in [-1, 1], Philox key tag
 *    0x4D4C5044, counter (0, 0, input, coordinate / 4)) and both outputs of
 *    the squared difference to the outputs of the teacher network o_p, so the
 *    minimum is again 0 at x = o_p.  R_p is not used (pass any D_p^2 array).
 *    Id 6 runs on the batched path only (plain path: EUNSUPPORTED), in FP32
 *    whatever cfg.prec is, and its selection compares the FP32 values: it has
 *    no difference form for near ties.
 *  - Population layout: instance-major, row-major, each row padded to
 *    Dpad = round_up(D, 4) floats (16-byte rows); the pad columns are zero.
 *    Instance k's rows start at float offset pop_off[k]; its fitness values
 *    at fit_off[k] (see metade_offsets).
 *  - theta is float32 [n_inst][6] = (F, CR, bl, br, dn, cs) with the four
 *    categorical genes as integral values: bl, br in {1 rand, 2 best,
 *    3 pbest, 4 current}, dn in {1..4}, cs in {1 bin, 2 exp, 3 arith}.
 *  - Random numbers come from Philox4x32-10 (Salmon et al., SC'11) keyed by
 *    (seed, stream, generation, individual, draw slot), so every draw is
 *    reproducible and independent of launch shape.
 */
#ifndef METADE_H
#define METADE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define METADE_API __attribute__((visibility("default")))
#else
#define METADE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    METADE_OK = 0,
    METADE_EINVAL = 1,      /* bad argument, or (device) invalid theta / NP too small */
    METADE_ENOMEM = 2,      /* device allocation of the context failed */
    METADE_ECUDA = 3,       /* a CUDA runtime call failed */
    METADE_ETIMEOUT = 4,    /* a bounded device wait gave up */
    METADE_ESTATE = 5,      /* call out of order (e.g. evolver calls without n_out) */
    METADE_EUNSUPPORTED = 6 /* configuration not supported by this build */
} metade_status;

/* Precision of the rotation z = R (u - o).  FP32: CUDA cores.  BF16, BF16X3
 * and FP8E4M3 apply to executors with D >= metade_config.tc_min_dim (129
 * unless set or autotuned), which run on the tensor cores
 * (tcgen05) with FP32 accumulation: BF16 operands; split BF16 (hi*hi + hi*lo +
 * lo*hi, about FP32 accuracy); or e4m3 operands with a per-row scale of u - o
 * and a per-problem scale of R (each maps the largest magnitude to 448),
 * undone in the GEMM epilogue.  Executors of the MLP objective (6) never join
 * the rotation GEMM: with BF16 or BF16X3 their network's first layer runs on
 * the tensor cores in that precision (the rest in FP32; BF16 with the
 * hardware tanh approximation), with FP32 or FP8E4M3 all of it in FP32 on
 * the CUDA cores.  FP64 is only for metade_eval. */
typedef enum {
    METADE_FP32 = 0,
    METADE_BF16 = 1,
    METADE_FP8E4M3 = 2,
    METADE_BF16X3 = 3,
    METADE_FP64 = 4
} metade_prec;

typedef enum {
    METADE_PATH_BATCHED = 0, /* all executors per launch, generations fused, tuned plan */
    METADE_PATH_PLAIN = 1    /* one executor per launch per generation: FP32 baseline */
} metade_path;

typedef struct {
    /* problem table (host arrays, device data) */
    int32_t n_prob;
    const int32_t *prob_dim;  /* host [n_prob], D_p >= 1 */
    const int32_t *prob_obj;  /* host [n_prob], objective id 0..6 (6: MLP regression, see below) */
    const float *shift;       /* device [sum_p D_p]: o_p concatenated */
    const float *rot;         /* device [sum_p D_p^2]: R_p row-major, concatenated */
    /* executors */
    int32_t n_inst;
    const int32_t *inst_np;    /* host [n_inst], population sizes, 4 <= NP <= 1024 */
    const int32_t *inst_prob;  /* host [n_inst], problem index of each executor */
    const int32_t *inst_group; /* host [n_inst] or NULL: the MetaDE run of each executor */
    float lo, hi;              /* search box [lo, hi]^D */
    uint64_t seed;
    int32_t one_shot;          /* 1: executors of a run share one random stream (Sec. III-C) */
    int32_t p_best_pct;        /* pbest pool, percent of NP (0 -> 10, Sec. II-A) */
    int32_t n_out;             /* evolver population per run; 0 = no evolver */
    metade_prec prec;          /* rotation precision for D >= tc_min_dim (FP32 below): FP32, BF16, BF16X3, FP8E4M3 */
    metade_path path;
    int32_t tie_fp64;          /* selection ties: 0 = FP32 difference form, 1 = FP64 re-evaluation */
    void *stream;              /* cudaStream_t all calls are issued on (NULL = legacy) */
    int32_t evolver;           /* 0 = DE/rand/1/bin (Alg. 3); 1 = PSO (w = 0.729, c1 = c2 = 1.49);
                                  2 = CSO (n_out <= 4096); 3 = NES (xNES) */
    int32_t tc_min_dim;        /* prec BF16 / BF16X3 / FP8E4M3: executors with D >= tc_min_dim run on
                                  the tensor cores, the others in FP32 on the CUDA cores.  0 = let
                                  metade_autotune choose among 33, 129 and 256 by speed (129 until it
                                  runs); > 0 fixes it.  FP32: executors with D >= tc_min_dim (and every
                                  one with D > 256) run the same per-generation pipeline with its GEMM
                                  in FP32 on the CUDA cores, the others in the fused kernels; 0 = let
                                  metade_autotune choose among 33, 129 and 257 (257 until it runs).
                                  Negative: EINVAL */
    int32_t tc_unfused;        /* 0: BF16 tensor-core executors with D <= 256 (and FP32 difference-form
                                  ties) run four kernels per generation: ranking, trial rows, one
                                  kernel for the tcgen05 GEMM with objective, selection and the commit
                                  of accepted rows, and one for the near ties, batched per problem;
                                  1: the five-kernel pipeline every other tensor-core configuration
                                  uses (prologue, trial, GEMM, selection, ties), with bit-identical
                                  results -- for comparison */
} metade_config;

typedef struct metade_ctx metade_ctx;

/* Validate the configuration, build the descriptor table and padded problem
 * copies, allocate scratch and pick the launch plan (autotuned on first
 * batched step).  shift/rot are copied; the caller may free them after.
 * Returns EINVAL for a malformed config (sizes out of range, n_out > 0 with
 * n_inst not a multiple of n_out, n_out < 4), ENOMEM/ECUDA on device
 * failure.  *out is NULL on error. */
METADE_API metade_status metade_create(const metade_config *cfg, metade_ctx **out);

/* Release the context (synchronises its stream first).  NULL is a no-op. */
METADE_API void metade_destroy(metade_ctx *ctx);

/* Sizes: floats of the padded population, total individuals (fitness
 * length), number of runs (groups).  Any pointer may be NULL. */
METADE_API metade_status metade_layout(const metade_ctx *ctx, int64_t *pop_floats, int64_t *n_indiv,
                            int32_t *n_groups);

/* Host arrays [n_inst] of per-executor float offset, fitness offset and
 * padded row length.  Any pointer may be NULL. */
METADE_API metade_status metade_offsets(const metade_ctx *ctx, int64_t *pop_off, int64_t *fit_off,
                             int32_t *dpad);

/* Change the stream later calls are issued on. */
METADE_API metade_status metade_set_stream(metade_ctx *ctx, void *stream);

/* Alg. 2, initialisation: fill every executor's population uniformly in the box
 * (x = lo + (hi - lo) U, rounded once to float32) and evaluate it (NaN
 * fitness stored as +inf): in FP32, except executors on the tensor-core path
 * (cfg.prec BF16 / BF16X3 / FP8E4M3, D >= 256), which are evaluated by the
 * rotation GEMM in that precision like all their later evaluations, and
 * executors of the MLP objective, evaluated by that objective's kernel.  `epoch` enters
 * the draw counter: with
 * one-shot evaluation the caller passes 0 every time, so every evaluation of
 * a theta starts from the same population. */
METADE_API metade_status metade_init(metade_ctx *ctx, float *pop, float *fit, uint32_t epoch);

/* Alg. 2's generation loop, `n_gens` times, generations gen0 .. gen0 + n_gens - 1,
 * for every executor: rand/best/pbest/current base vectors and dn difference
 * vectors of distinct random individuals (Eq. of Sec. III-A-2), binomial /
 * exponential / arithmetic crossover (Sec. II-A), clip to the box, FP32
 * shifted-rotated evaluation, and generational greedy selection f(u) <= f(x).
 * Selection ties, |f(u) - f(x)| <= band |f(x)| with both values positive and
 * finite and band = max(1e-6, 2^-21 sqrt(D)) (the 1e-6 band, widened where the
 * FP32 error of f grows with D), are decided on the difference f(u) - f(x)
 * evaluated directly in FP32 from z = R(x - o) and dz = R(u - x) (error
 * proportional to the difference, not to f), or, with cfg.tie_fp64, by
 * re-evaluating both vectors in FP64; an accepted tie stores f(x) + difference
 * (resp. the FP64 value), never above f(x).  A trial identical to its target
 * is accepted without re-evaluation.  pop/fit are updated in place.  If
 * best_f / best_i are non-NULL they receive each executor's best fitness and
 * its index after the last generation (Sec. III-B: the executor's y*).
 * theta: device [n_inst][6].  n_gens == 0 only writes best_f/best_i. */
METADE_API metade_status metade_inner_step(metade_ctx *ctx, float *pop, float *fit, const float *theta,
                                uint32_t epoch, uint32_t gen0, int32_t n_gens, float *best_f,
                                int32_t *best_i);

/* Evaluate caller-given points (Sec. IV-A reports the final error
 * f(x_best) - f*; with f* = 0 that is f(x_best) in FP64):
 *   x      device float32 [n][ldx], point r at x + r * ldx, its first D
 *          coordinates used, D the dimension of executor inst[r]'s problem;
 *          16-byte aligned, ldx a multiple of 4 (>= 4)
 *   inst   device int32 [n], the executor whose problem evaluates point r
 *   f_out  device [n]: float for prec FP32, double for FP64 (the objective
 *          evaluated entirely in FP64 from the float32 coordinates)
 * n = 0 is a no-op.  Host errors (NULL pointers, ldx, alignment, n < 0, no
 * executors) return EINVAL; other precisions EUNSUPPORTED.  An executor id
 * outside [0, n_inst) or a dimension above ldx, found on the device, latches
 * EINVAL in the sticky status and writes NaN for that point.  MLP problems
 * are evaluated with their own objective. */
METADE_API metade_status metade_eval(metade_ctx *ctx, const float *x, int64_t n, const int32_t *inst, int32_t ldx,
                                     metade_prec prec, void *f_out);

/* Evaluate every population row: prec FP32 writes float f_out[n_indiv],
 * FP64 writes double f_out[n_indiv].  Other precisions return EUNSUPPORTED. */
METADE_API metade_status metade_eval_pop(metade_ctx *ctx, const float *pop, metade_prec prec, void *f_out);

/* Evolver (Alg. 3).  Its population is float32 [n_groups][n_out][6] with
 * fitness [n_groups][n_out]; executor k = g * n_out + j evaluates vector j
 * of run g.  ESTATE if the context has no evolver (n_out == 0).
 * With cfg.evolver = 1 (PSO, the supplement's comparison of evolvers) the
 * population and fitness are the particles' personal bests, and `trial` is
 * float32 [n_groups][n_out][12]: position (the vector evaluated) then
 * velocity.  Phase 0 of generation 0 evaluates the initial swarm (position =
 * personal best, velocity 0); later generations move every particle by
 * v <- w v + c1 r1 (pbest - x) + c2 r2 (gbest - x), x <- clip(x + v), gbest the
 * run's best personal best (ties to the lower index).  Phase 1 is Alg. 3's
 * selection applied to the positions.  ofit is read by phase 0.
 * With cfg.evolver = 2 (CSO, Cheng and Jin 2015) the population holds the
 * particles' positions and `trial` is float32 [n_groups][n_out][13]: the
 * position to evaluate, the velocity, a flag.  Phase 0 of generation 0
 * evaluates the initial swarm (all flagged, velocity 0); later generations
 * pair the swarm at random (Fisher-Yates on evolver draws), keep the fitter
 * particle of each pair (ties to the lower index) and move the other:
 * v <- r1 v + r2 (x_winner - x), x <- clip(x + v), flagged.  Phase 1 gives
 * every flagged particle its new position and meta-fitness unconditionally.
 * With cfg.evolver = 3 (NES: xNES, Wierstra et al. 2014) `trial` is float32
 * [n_groups][12 n_out + 96]: per run, the n_out samples [clip(z) 6 | s 6],
 * then the search distribution as doubles (mu[6], sigma, B[6][6] row-major),
 * set by phase 0 of generation 0 to mu = (lb + ub)/2, sigma B =
 * diag((ub - lb)/4).  Phase 0 draws z = mu + sigma B s, s ~ N(0, I)
 * (Box-Muller), decoded from clip(z); phase 1 ranks the samples by
 * meta-fitness and takes the xNES natural-gradient step (utilities, default
 * learning rates), then writes the samples and their meta-fitness (NaN as
 * +inf) to the population and fitness. */
/* Alg. 3, initialisation: uniform in [lb, ub] = [(0,0,1,1,1,1), (1,1,5,5,5,4)], y = +inf. */
METADE_API metade_status metade_outer_init(metade_ctx *ctx, float *opop, float *ofit);

/* phase 0 (Alg. 3, trials and decoding): rand/1/bin trials (F = 0.5, CR = 0.9) clipped to
 *   [lb, ub] into trial[n_groups][n_out][6], decoded (F = u1, CR = u2, the
 *   rest floor(u) clamped to their domain) into theta[n_inst][6].
 * phase 1 (Alg. 3, selection): where meta_fit[k] <= ofit[k] (NaN as +inf) the
 *   trial replaces the parent and ofit[k] = meta_fit[k]. */
METADE_API metade_status metade_outer_step(metade_ctx *ctx, float *opop, float *ofit, float *trial,
                                float *theta, const float *meta_fit, uint32_t outer_gen,
                                int32_t phase);

/* One whole evolver generation (Alg. 3): phase 0, executor
 * initialisation (epoch 0 under one-shot evaluation, else outer_gen),
 * n_inner_gens executor generations, the best-fitness reduction into
 * best_f/best_i, phase 1.  With use_graph != 0 the sequence is captured
 * once as a CUDA graph (per argument set) and replayed; on the plain path
 * (the no-graph baseline) it is always launched directly. */
METADE_API metade_status metade_outer_generation(metade_ctx *ctx, float *opop, float *ofit, float *trial,
                                      float *theta, float *pop, float *fit, float *best_f,
                                      int32_t *best_i, uint32_t outer_gen, int32_t n_inner_gens,
                                      int32_t use_graph);

/* Parity/debug: the draw record of generation `gen` for every individual,
 * int32 rec[n_indiv][18]: base-left index, base-right index, j_rand,
 * exponential start n, exponential length L (0 unless cs = exp), K_i as a
 * 24-bit integer, pbest index, best index, m, r_0..r_8 (-1 unused).  Uses
 * the generation-start fitness `fit`. */
METADE_API metade_status metade_draw_record(metade_ctx *ctx, const float *fit, const float *theta,
                                 uint32_t epoch, uint32_t gen, int32_t *rec);

/* One plain FP32 generation of a single executor (the computation of
 * metade_inner_step on the plain path, with one executor and n_gens = 1) that
 * allocates nothing and needs no context.  The paper has no counterpart: this
 * exists for callers that cannot allocate device memory themselves (their
 * device heap belongs to a host framework or allocator, or they must not grow
 * the process's device footprint).  The caller passes every input and output:
 *   pop [np][round_up(dim,4)] float32 (pad columns zero), 16-byte aligned
 *   (rows are accessed as float4; an unaligned pop returns METADE_EINVAL),
 *   fit [np] -- updated in place; theta [6] decoded (F, CR, bl, br, dn, cs); shift [dim];
 *   rot [dim][dim] row-major; stream_id is Philox counter word 0; p_best_pct
 *   as in metade_config (0 -> 10); stream is a cudaStream_t (NULL = legacy).
 * Scratch (trial rows, trial fitness, pbest pool) lives in one file-scope
 * device array of 2^20 floats (4 MiB) that every GPU loading the library holds
 * until the process exits; sizes with round_up(np*round_up(dim,4), 64) +
 * round_up(np, 64) + np > 2^20 floats are rejected with METADE_EINVAL, as are
 * np outside 4..1024, dim outside 1..1536 and bad objective ids.  The first
 * call made on a device (with that device current) looks up the array's
 * device address with cudaGetSymbolAddress; make that first call before any
 * stream capture.  The address is cached for the process's life: after
 * cudaDeviceReset on a device, do not call this entry point on it again.  All calls share the array and it keeps the last call's
 * contents (every element a call reads is written earlier in that call, so
 * nothing is cleared); calls that overlap on the GPU race on it.  An invalid
 * theta, or np too small for the strategy, leaves pop and fit unchanged; the
 * call's first kernel records which in a device word that
 * metade_plain_step_noalloc_status reads.
 * Asynchronous on `stream`; returns METADE_ECUDA if a launch fails (checked
 * with cudaPeekAtLastError, so an error left pending by earlier work is
 * reported too, and not cleared). */
METADE_API metade_status metade_plain_step_noalloc(float *pop, float *fit, const float *theta,
                                                   const float *shift, const float *rot, int32_t np,
                                                   int32_t dim, int32_t obj, float lo, float hi,
                                                   uint64_t seed, uint32_t stream_id, uint32_t epoch,
                                                   uint32_t gen, int32_t p_best_pct, void *stream);

/* The outcome of the last metade_plain_step_noalloc on the current device, once
 * it has run: *status = 0 for a real generation, 1 for one skipped because
 * theta was invalid or np too small for its strategy.  Waits for the device
 * (a synchronous copy from the library's device word).  The word is shared by
 * every call, like the scratch array. */
METADE_API metade_status metade_plain_step_noalloc_status(int32_t *status);

/* Wait for the context's stream; return and clear the sticky device status. */
METADE_API metade_status metade_sync(metade_ctx *ctx);

/* Autotuner: with cfg.tc_min_dim = 0, first the width of the per-generation
 * GEMM pipeline (33, 129 or 256 with BF16 / BF16X3 / FP8E4M3; 33, 129 or 257
 * with FP32): one untimed and n_gens timed generations of every executor per
 * width, on copies, keeping the fastest; in reduced precision this changes
 * which executors are evaluated in reduced precision, in FP32 only the order
 * of the FP32 sums.  Then,
 * for every bucket of the batched path, time each candidate block
 * shape (small-D kernel: 32, 64, 128, 256 threads; tile kernel: 128 or 256
 * threads with R^T resident, 256 with R^T streamed; general kernel: 128, 256,
 * 512 threads) on device copies of (pop, fit) for n_gens generations with the
 * given theta, and keep the fastest.  The caller's pop/fit are not modified;
 * the copies are allocated and freed inside the call, which synchronises the
 * stream.  The measured times are reported by metade_plan_info.  No-op on
 * the plain path. */
METADE_API metade_status metade_autotune(metade_ctx *ctx, const float *pop, const float *fit, const float *theta,
                                         int32_t n_gens);

/* Write a one-line JSON description of the launch plan into buf. */
METADE_API metade_status metade_plan_info(const metade_ctx *ctx, char *buf, size_t len);

/* Timing of the context's own kernels: with profiling enabled, calls made
 * outside stream capture record CUDA events on the context's stream around
 * each launch of the fused kernels and the tensor-core stage.  enable = n > 1
 * samples the tensor-core generations: one in n (counted over the context's
 * life) records its events, so the events perturb fewer kernel boundaries;
 * the counts are then those of the sampled launches, and ms / count is still
 * the mean launch time.  enable 1: every launch; 0: off.  Reading waits
 * for the stream and returns, per kind, the summed milliseconds and the number
 * of launches since the last read -- kinds: 0 fused small-D kernel, 1 fused
 * general kernel, 2 tensor-core rotation GEMM, 3 whole tensor-core generation,
 * 4 fused tile kernel with R^T streamed (128 < D_pad <= 256), 5 fused tile
 * kernel with R^T resident (D_pad <= 128), 6 MLP-objective generations, and
 * the other kernels of a tensor-core generation: 7 prologue (best, pbest
 * pool, and the rows' index draws where the trial kernel reads them from
 * it), 8 trial rows and GEMM operands, 9 selection, 10 near ties, 11 the
 * GEMM with objective, selection and commit of the BF16 four-kernel
 * generation -- then clears them.  Kind 12 counts selections of tensor-core
 * executors decided by the near-tie path (ms 0; counted whether or not
 * profiling is on).  ms and count are host arrays of 13 (may be NULL). */
METADE_API metade_status metade_profile(metade_ctx *ctx, int32_t enable);
METADE_API metade_status metade_profile_read(metade_ctx *ctx, double *ms, int64_t *count);

/* Check of the bounded device wait that every mbarrier wait of the
 * tensor-core pipeline uses (no context needed; runs on the current device,
 * legacy default stream, synchronously).  One thread initialises an mbarrier
 * in shared memory for one arrival and waits on its first phase for at most
 * `rounds` try_wait rounds (0: the pipeline's own limit).  arrive = 1: the
 * thread arrives first, so the wait completes; arrive = 0: nothing arrives,
 * so the wait gives up.  *completed (may be NULL) = 1 if the phase completed;
 * *seconds (may be NULL) = the wait's length in SM clock cycles over the
 * device's nominal clock rate.  Returns METADE_OK when the wait completed,
 * METADE_ETIMEOUT when it gave up (the device context stays usable),
 * METADE_EINVAL for arrive outside {0, 1}, METADE_ENOMEM / METADE_ECUDA on
 * allocation or runtime failures. */
METADE_API metade_status metade_wait_check(int32_t arrive, uint32_t rounds, int32_t *completed, double *seconds);

/* Number of kernel launches this context has issued (graph replays count the
 * kernels they contain). */
METADE_API int64_t metade_launch_count(const metade_ctx *ctx);

METADE_API const char *metade_strerror(metade_status s);

/* Name of the CUDA error behind the last METADE_ECUDA a call returned on this
 * host thread ("cudaSuccess" if none was recorded). */
METADE_API const char *metade_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* METADE_H */
