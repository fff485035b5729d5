/*
 * qieo.h -- C ABI of the GB300 QIEO library (quantum-inspired evolutionary optimisation
 * of the 0/1 knapsack, arxiv 2609.30862).
 *
 * One QIEO instance holds a population of np chromosomes of ng qubits (Sec. I, Sec. III-A)
 * for one knapsack problem. Each generation (Sec. III-B, Fig. 1) observes every qubit
 * (QIP), evaluates eq. (1) for every chromosome (Evaluation), picks the generation-best
 * chromosome (DetermineElite) and rotates every qubit one step toward the elite's allele
 * (CIP). All four steps of a generation run in one fused CUDA kernel on the GPU.
 *
 * Conventions shared by every entry point:
 *   - Return value: a qieo_status; QIEO_OK (0) on success. No entry point aborts the
 *     process; on failure the reason is available from qieo_last_error() on the calling
 *     thread and the instance is left as it was before the call unless stated otherwise.
 *   - Host pointers are caller-owned. Input arrays are copied before the call returns;
 *     output arrays must hold the stated number of elements.
 *   - The library owns the device memory of an instance from qieo_create_instance to
 *     qieo_destroy_instance.
 *   - An instance may be used from one host thread at a time.
 *
 * Qubit representation: the amplitude pair (alpha, beta) = (cos theta, sin theta) is held
 * as the angle index k in [-K, K] with theta = pi/4 + k pi/D, K = D/4 (so theta stays in
 * [0, pi/2]). Observation draws u = Philox4x32-10 word (j mod 4) of counter
 * (j div 4, c, t, 0) under key (seed, instance_id) and sets x = 1 iff
 * u < T[k + K], T[n] = round(sin^2(n pi/D) 2^32) (mirrored: T[2K-n] = 2^32 - T[n]).
 * Every result is therefore exact and reproducible bit for bit.
 */
#ifndef QIEO_H
#define QIEO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QIEO_OK = 0,
    QIEO_ERR_INVALID = 1,   /* an argument is out of range; nothing was changed */
    QIEO_ERR_OOM = 2,       /* device memory could not be obtained */
    QIEO_ERR_CUDA = 3,      /* a CUDA runtime call or kernel launch failed */
    QIEO_ERR_TIMEOUT = 4,   /* a bounded wait for the device ran out */
    QIEO_ERR_BUSY = 5       /* the instance is in use by an unfinished operation */
} qieo_status;

/* Opaque, library-owned. */
typedef struct qieo_instance qieo_instance;

/* One 0/1 knapsack problem (Sec. III-A): item j has weight weights[j] >= 0 and value
 * values[j]; capacity W >= 0. Both arrays are host memory of ng int32 entries and are
 * copied by qieo_create_instance. */
typedef struct {
    int32_t ng;
    const int32_t *weights;
    const int32_t *values;
    int64_t capacity;
} qieo_problem;

/* Rotation rules of CIP (Sec. III-B "lookup-table rotation toward the elite"):
 * R1 moves every qubit one step toward the elite's allele; R2 moves only the qubits
 * whose observed allele differs from the elite's. */
#define QIEO_RULE_R1 0
#define QIEO_RULE_R2 1

/* flags */
#define QIEO_FLAG_NO_GRAPH      0x1   /* launch generations one by one, no CUDA graph */
#define QIEO_FLAG_SYNC_RUN      0x2   /* qieo_run waits (bounded) for the device */
#define QIEO_FLAG_FORCE_WIDE    0x4   /* use 64-bit item sums even for small items */
#define QIEO_FLAG_TIME_KERNELS  0x8   /* time the generation kernels with CUDA events */
#define QIEO_FLAG_COOPERATIVE   0x10  /* one cooperative launch per run (a bounded grid
                                         barrier between generations) instead of one launch
                                         per generation. The library also picks it by itself
                                         for instances of at most 2^22 genes whose fitness
                                         fits the packed elite key (there it is faster) */
#define QIEO_FLAG_REGISTER_PREFETCH 0x20 /* stream the state with register prefetch instead
                                            of asynchronous copies into shared memory */
#define QIEO_FLAG_UNFUSED       0x40  /* run each generation as four launches, one per step
                                         of Sec. III-B (CIP, QIP, Evaluation,
                                         DetermineElite), the way the paper offloads them;
                                         same results, for the per-step time breakdown.
                                         Not with elite_on_host or QIEO_FLAG_COOPERATIVE */
#define QIEO_FLAG_CONVERGE      0x80  /* stop once the elite fitness has been the same for
                                         QIEO_CONVERGE_WINDOW consecutive generations
                                         (Sec. IV, Workload); the generations asked of a run
                                         are then a cap. The generation that meets the test
                                         still gets its CIP. Default path, batches and the
                                         server only: not with elite_on_host,
                                         QIEO_FLAG_COOPERATIVE or QIEO_FLAG_UNFUSED */
#define QIEO_CONVERGE_WINDOW    20
#define QIEO_FLAG_PER_GENERATION 0x200 /* always one launch per generation (never the
                                          cooperative form picked for small instances) */
#define QIEO_FLAG_STATE_I8      0x100 /* store each angle index in one byte instead of two
                                         (k in [-K, K] fits when dtheta_den <= 120), halving
                                         the state's memory traffic; identical results.
                                         Needs items in [0, 255]; not with
                                         QIEO_FLAG_REGISTER_PREFETCH, QIEO_FLAG_COOPERATIVE,
                                         QIEO_FLAG_UNFUSED or QIEO_FLAG_FORCE_WIDE, and not in
                                         batches */
#define QIEO_FLAG_STREAMED      0x800 /* never keep the state resident in shared memory
                                         (see qieo_launch_shape.resident): stream it from
                                         device memory every generation */
#define QIEO_FLAG_SIXTEEN       0x1000 /* one-launch-per-generation runs process 16 genes per
                                          thread and pass instead of 8 (rule R1, items of at
                                          most 127, 16-bit state, the default tile; otherwise
                                          ignored); identical results. Faster while every
                                          qubit still draws, slower once many saturate
                                          (4,096 x 100,000 genes: 406 vs 422 us per spread
                                          generation, 241 vs 184 us per collapsed one) */
#define QIEO_FLAG_NO_FIXED_WORDS 0x2000 /* keep no fixed-vector words: every generation of
                                          the one-launch-per-generation form runs the dense
                                          pass over all qubits (see qieo_launch_shape.
                                          fixed_words) */
#define QIEO_FLAG_SPARSE_ALWAYS 0x4000 /* with fixed-vector words, take the sparse form in
                                          every generation that rotates (all but a run's
                                          first), however few vectors are fixed (identical
                                          results; for tests and measurement) */
#define QIEO_FLAG_TIME_GENERATIONS 0x400 /* time every generation of a run for
                                            qieo_get_generation_times. In the resident form
                                            (qieo_launch_shape.resident) one thread reads the
                                            device clock at the start of each generation
                                            (after the grid barrier) and at the run's end;
                                            otherwise a CUDA event is recorded before every
                                            generation launch and after the last one (one
                                            launch per generation, no CUDA graph; the events
                                            keep consecutive launches from overlapping, so
                                            each time is the launch alone). Not with
                                            elite_on_host, QIEO_FLAG_COOPERATIVE or
                                            QIEO_FLAG_UNFUSED */

typedef struct {
    int32_t np;              /* chromosomes, >= 1 */
    int32_t dtheta_den;      /* D: rotation step pi/D; multiple of 4 in [4, 4000]; default 100 */
    int64_t penalty_lambda;  /* lambda of eq. (1), >= 1; default 1 */
    uint32_t seed;           /* Philox key word 0 */
    uint32_t instance_id;    /* Philox key word 1 */
    int32_t rotate_rule;     /* QIEO_RULE_R1 (default) or QIEO_RULE_R2 */
    int32_t elite_on_host;   /* 0: DetermineElite on the device, fused (default);
                                1: host variant (device->host fitness copy + host argmax) */
    int32_t flags;           /* QIEO_FLAG_* */
    void *stream;            /* cudaStream_t to run on; NULL: the instance makes its own */
} qieo_params;

/* Fills *p with the defaults above (np = 64, seed = 1, instance_id = 0). */
void qieo_default_params(qieo_params *p);

/* Creates an instance in the state before generation 0 (Sec. III-B: every qubit at
 * theta = pi/4, i.e. k = 0; no best record). Validates: ng >= 1, np >= 1,
 * weights >= 0, D a multiple of 4 in [4, 4000], lambda >= 1, lambda * sum(w) and
 * sum(|v|) below 2^62. Returns QIEO_ERR_INVALID, QIEO_ERR_OOM or QIEO_ERR_CUDA on
 * failure, with *out set to NULL. */
qieo_status qieo_create_instance(const qieo_problem *problem, const qieo_params *params,
                                 qieo_instance **out);

/* Waits for the instance's work and frees it. NULL is accepted. */
qieo_status qieo_destroy_instance(qieo_instance *inst);

/* Returns the instance to its state before generation 0 (same problem and params). */
qieo_status qieo_reset(qieo_instance *inst);

/* Runs `generations` >= 0 generations from the current one (Fig. 1: QIP, Evaluation,
 * DetermineElite, CIP, per generation; the CIP of the last generation is applied before
 * returning, so run(a) followed by run(b) equals run(a + b)). Each generation is one kernel
 * launch, chained to the next by programmatic dependent launch and replayed from a CUDA
 * graph when a run length repeats; instances of at most 2^22 genes (or any instance with
 * QIEO_FLAG_COOPERATIVE) run the whole run as one cooperative launch whose blocks meet at
 * a bounded grid barrier after each generation (qieo_launch_shape.persistent tells which).
 * Stream-ordered: returns after enqueueing unless QIEO_FLAG_SYNC_RUN is set or
 * elite_on_host is 1. A barrier wait that runs out is reported as QIEO_ERR_TIMEOUT by the
 * next call that waits for the device; the state is then undefined until qieo_reset. */
qieo_status qieo_run(qieo_instance *inst, int32_t generations);

/* Bound of one grid-barrier wait inside a cooperative run, in nanoseconds (default 10 s;
 * >= 1). */
qieo_status qieo_set_wait_timeout(qieo_instance *inst, int64_t ns);

/* Waits (bounded) until every operation enqueued for the instance has finished; reports
 * a device-side wait that ran out as QIEO_ERR_TIMEOUT. */
qieo_status qieo_synchronize(qieo_instance *inst);

/* The best-so-far record (the first generation elite of largest fitness): its alleles as
 * ng bytes of 0/1 into bits_out (may be NULL), fitness, generation and chromosome. Before
 * any generation has run, generation and chromosome are -1 and fitness is 0. Waits for
 * the instance's work. */
qieo_status qieo_get_best(qieo_instance *inst, uint8_t *bits_out, int64_t *fitness,
                          int32_t *generation, int32_t *chromosome);

/* The angle indices k (np*ng int16, row c = chromosome c) and the next generation t. */
qieo_status qieo_get_state(qieo_instance *inst, int16_t *k_out, int32_t *t_out);

/* Eq. (1) fitness of every chromosome in the last generation run (np int64). */
qieo_status qieo_get_fitness(qieo_instance *inst, int64_t *f_out);

/* Alleles observed in the last generation run (np*ng bytes of 0/1). */
qieo_status qieo_get_alleles(qieo_instance *inst, uint8_t *x_out);

/* The same for one chromosome c in [0, np) (ng bytes of 0/1); QIEO_ERR_INVALID otherwise. */
qieo_status qieo_get_allele_row(qieo_instance *inst, int32_t c, uint8_t *x_out);

/* Elite index and fitness of generations first .. first+n-1 (all < t). */
qieo_status qieo_get_elite_history(qieo_instance *inst, int32_t first, int32_t n,
                                   int32_t *idx_out, int64_t *fit_out);

/* Work of generations first .. first+n-1 (all < t) of an instance that keeps fixed-vector
 * words (qieo_launch_shape.fixed_words): out[i] = the 8-gene vectors of generation first+i
 * that drew (ran QIP, Sec. III-B, with a Philox draw per qubit, after their CIP); the rest
 * were fixed (every qubit at theta = 0 or pi/2, |alpha|^2 or |beta|^2 = 1, Sec. I), so
 * their alleles were known without a draw (the fixed-allele pass of the dense form, the
 * stable vectors of the sparse form). np * ceil(ng / 8) means every vector drew; generations
 * run in a batch, or restored by a checkpoint load, report that value (they are not counted).
 * QIEO_ERR_INVALID for an instance without the words, out NULL or a range outside [0, t). */
qieo_status qieo_get_drawn_vectors(qieo_instance *inst, int32_t first, int32_t n, int64_t *out);

/* The observation thresholds T[0 .. 2K] the device uses (2K+1 uint64). */
qieo_status qieo_get_threshold_table(qieo_instance *inst, uint64_t *t_out);

/* Launch shape of the fused generation kernel. Results do not depend on it (all sums are
 * exact integers and every draw is keyed by gene, chromosome and generation). A row is cut
 * into tiles of lanes_per_row * warps_per_row vectors of 8 genes; a persistent grid of
 * grid_ctas blocks covers the ntile * np tile-rows, in equal contiguous shares when a share
 * is below 64 tile-rows, otherwise (runs with the packed elite key) by taking segments of
 * decreasing size from a queue. */
typedef struct {
    int32_t lanes_per_row;   /* 1, 2, 4, 8, 16 or 32 threads of a warp on one row tile */
    int32_t warps_per_row;   /* 1, 2, 4 or 8 warps on one row tile (lanes_per_row 32 only) */
    int32_t grid_ctas;       /* thread blocks; 0 = three per SM (or fewer if fewer fit) */
    int32_t narrow;          /* out: 1 when 16-bit packed item sums are in use */
    int32_t tiles;           /* out: gene tiles per row */
    int32_t rows_per_cta;    /* out: most tile-rows one block sums in shared memory at once */
    int32_t persistent;      /* out: 1 when a run is one cooperative launch (see
                                QIEO_FLAG_COOPERATIVE), 0 when it is one launch per
                                generation */
    int32_t resident;        /* out: 1 when a run keeps the state in shared memory: each
                                block holds its share of the angle indices on chip from the
                                start of a run to its end (one cooperative launch; chosen
                                whenever the shares fit, e.g. up to about 20-30 MB of state on
                                a GB300, unless QIEO_FLAG_STREAMED, QIEO_FLAG_COOPERATIVE,
                                QIEO_FLAG_PER_GENERATION, QIEO_FLAG_TIME_GENERATIONS,
                                QIEO_FLAG_CONVERGE, elite_on_host or byte state) */
    int32_t fixed_words;     /* out: 1 when the instance keeps a fixed-vector bit per 8 genes
                                (set when all eight qubits sit at theta = 0 or pi/2; their
                                sides are the vector's previous alleles), so that a
                                generation in which most vectors are fixed
                                takes the sparse form: only the vectors that are not fixed, or
                                that the previous elite turns away from their bound, run CIP,
                                QIP and Evaluation in full; the rest contribute their sides.
                                Kept by the one-launch-per-generation runs with the packed
                                elite key, items in [0, 255] whose weights and values each sum
                                below 2^25, 16-bit state and the default tile, unless
                                QIEO_FLAG_NO_FIXED_WORDS, QIEO_FLAG_SIXTEEN or
                                QIEO_FLAG_CONVERGE */
} qieo_launch_shape;

qieo_status qieo_get_launch_shape(qieo_instance *inst, qieo_launch_shape *shape);
qieo_status qieo_set_launch_shape(qieo_instance *inst, const qieo_launch_shape *shape);

/* Accumulated device time of the generation kernels (QIEO_FLAG_TIME_KERNELS) and the
 * number of generation-kernel launches it covers; qieo_reset clears neither. */
qieo_status qieo_get_kernel_time(qieo_instance *inst, double *ms, int64_t *launches);

/* Device time of each generation of the last run of an instance created with
 * QIEO_FLAG_TIME_GENERATIONS: ms_out[i] = the time (ms) from the start of the run's
 * generation i to the start of the next one (for the last generation: to the end of the
 * run's last generation, before its final rotation), for i < min(n, generations of that run);
 * *count = that number. Waits (bounded) for the run to finish. The times cover one fused
 * generation kernel each (CIP of the generation before, QIP, Evaluation, DetermineElite);
 * the run's final CIP launch is not included. QIEO_ERR_INVALID without the flag. */
qieo_status qieo_get_generation_times(qieo_instance *inst, int32_t n, float *ms_out, int32_t *count);

/* Row blocks: one population sharded by chromosome rows (for example one block per GPU).
 * A generation's QIP and Evaluation (Sec. III-B) are independent per chromosome, and every
 * draw is keyed by the global chromosome index, so a block computes its rows exactly as
 * the whole population would. DetermineElite (the lowest-index best chromosome) and CIP
 * (toward the elite's alleles) need the whole population: the caller combines the blocks'
 * best rows (for example an all-reduce MAX of a key ordering (fitness, -row), then a
 * broadcast of the elite's alleles from the block that holds it) and passes the elite row
 * to every block.
 *
 * qieo_create_row_block: params->np is the number of rows of this block, which holds the
 * population's chromosomes row0 .. row0 + np - 1; the other params and the problem are
 * those of the whole population. Same validation and errors as qieo_create_instance, and
 * QIEO_ERR_INVALID for row0 < 0, elite_on_host, QIEO_FLAG_UNFUSED, QIEO_FLAG_COOPERATIVE,
 * QIEO_FLAG_CONVERGE, or a problem whose fitness does not fit the packed elite key
 * (lambda * sum(w) or sum(|v|) >= 2^39). A row block is destroyed, reset and read
 * (qieo_get_state, _fitness, _alleles) like an instance; qieo_run and batches reject it.
 *
 * qieo_rows_observe: QIP and Evaluation of generation t (absolute; it keys the draws) on the
 * block's current angle indices, without a rotation first; *best_fitness and *best_row
 * receive the block's lowest-index maximum of eq. (1) (best_row is a global chromosome
 * index). qieo_get_state then reports t + 1 as the next generation. Waits (bounded) for
 * the device. Either output may be NULL.
 *
 * qieo_rows_rotate: CIP of the block's rows after the generation last observed, toward the
 * elite alleles elite_bits (host memory, ng bytes, each 0 or 1; copied before the call
 * returns), by the instance's rotation rule (R2 compares each row's alleles of that
 * generation). QIEO_ERR_INVALID when no generation was observed since creation or reset, or
 * for a byte other than 0 or 1. Waits (bounded) for the device.
 *
 * Observing generations t0, t0 + 1, ... with a rotation toward the population's elite after
 * each one reproduces qieo_run on the whole population bit for bit. */
qieo_status qieo_create_row_block(const qieo_problem *problem, const qieo_params *params, int32_t row0,
                                  qieo_instance **out);
qieo_status qieo_rows_observe(qieo_instance *block, int32_t t, int64_t *best_fitness, int32_t *best_row);
qieo_status qieo_rows_rotate(qieo_instance *block, const uint8_t *elite_bits);

/* Measured integer ceiling of the generation kernel's per-gene work (a roofline bound
 * next to the state's 4 bytes of memory traffic per gene-update). Runs, on the current
 * device, (a) the per-gene arithmetic of the kernel's drawn pass -- CIP of the angle
 * indices, two Philox4x32-10 calls per 8 genes, the threshold compares, the allele bits and
 * the packed item sums, with the kernel's own device helpers, D = 100 -- with the state in
 * registers and nothing streamed, and (b) Philox4x32-10 alone, each in the generation
 * kernel's launch shape (256 threads, three blocks per SM), reps timed launches after one
 * warm-up launch (CUDA events; the best is kept). Allocates and frees a small device
 * buffer and a stream of its own; synchronous. QIEO_ERR_INVALID for reps outside
 * [1, 1000]. */
typedef struct {
    double drawn_genes_per_s;    /* (a): gene-updates per second */
    double philox_genes_per_s;   /* (b): genes per second at a quarter call per gene */
    int64_t genes_per_launch;
    int32_t grid_ctas;
    int32_t reps;
} qieo_integer_ceiling;

qieo_status qieo_measure_integer_ceiling(int32_t reps, qieo_integer_ceiling *out);

/* Accumulated time per step of a generation, ms[4] = {CIP, QIP, Evaluation,
 * DetermineElite}, and the number of generations it covers. Filled by runs with
 * QIEO_FLAG_TIME_KERNELS and QIEO_FLAG_UNFUSED (device time of each step's launch, CUDA
 * events), and, for the DetermineElite entry only, by runs with QIEO_FLAG_TIME_KERNELS and
 * elite_on_host = 1 (host wall time of the fitness copy to the host, the host argmax and
 * the launch that records the elite, measured after the generation kernel finished).
 * qieo_reset clears neither. */
qieo_status qieo_get_phase_times(qieo_instance *inst, double ms[4], int64_t *generations);

/* Checkpoint / resume (the paper has none). A checkpoint holds everything a later run of
 * the instance reads: the angle indices, the generation counter, the best-so-far record
 * and row, the elite history and the convergence words. Loading it into an instance
 * created with the same problem and params (ng, np, D, rule, seed, instance_id, capacity,
 * lambda, byte state or not) makes every later run bit-identical to the uninterrupted
 * instance's, because all draws are keyed by the absolute generation. The buffer is host
 * memory owned by the caller; qieo_checkpoint_size gives its size for the current
 * generation. QIEO_ERR_INVALID for a short buffer, another instance's checkpoint or a
 * corrupt header. Loading resets the instance first. */
qieo_status qieo_checkpoint_size(qieo_instance *inst, size_t *bytes);
qieo_status qieo_checkpoint_save(qieo_instance *inst, void *buffer, size_t bytes);
qieo_status qieo_checkpoint_load(qieo_instance *inst, const void *buffer, size_t bytes);

/* Convergence test of an instance created with QIEO_FLAG_CONVERGE: *stopped = 1 once it
 * stopped (no later generation runs; qieo_get_state's t is one past the generation that
 * met the test), *stable = the number of consecutive generations, ending at the last one
 * run, whose elite fitness is the same. Either pointer may be NULL. */
qieo_status qieo_get_convergence(qieo_instance *inst, int32_t *stopped, int32_t *stable);

/* A batch: many instances advanced together (batching of independent QIEO solves; the
 * paper runs one problem at a time). The instances keep their own state, records and
 * generation counters; qieo_batch_run(b, G) is equivalent to qieo_run(inst, G) on every
 * member, bit for bit. The work of a generation (every member's tiles of rows) is cut into
 * segments balanced over a grid of one block per resident slot; members are grouped by
 * item-sum form and rotation rule. By default a run is one persistent cooperative launch
 * per group for all its generations: blocks take (generation, segment) items from one queue
 * in order, and a segment of an instance's next generation waits (bounded) only for that
 * instance's previous generation to close, not for the other members. When a member uses
 * QIEO_FLAG_CONVERGE or QIEO_FLAG_PER_GENERATION, a run is instead one launch per group and
 * generation (replayed from a CUDA graph when a run length repeats). A wait that runs out
 * sets the member's error word (QIEO_ERR_TIMEOUT from its next checked call). Members must
 * live on one device, must not use elite_on_host and must not be destroyed while the batch
 * exists. */
typedef struct qieo_batch qieo_batch;

/* Creates a batch over instances[0 .. n-1] (n >= 1, distinct). The batch runs on the stream
 * of instances[0]; it waits for work already enqueued on the members' streams and the
 * members' streams wait for the batch's work. Uses each member's current launch shape. */
qieo_status qieo_create_batch(qieo_instance *const *instances, int32_t n, qieo_batch **out);

/* Runs `generations` >= 0 generations of every member (each from its own current
 * generation, including the final CIP of the run). Stream-ordered. */
qieo_status qieo_batch_run(qieo_batch *batch, int32_t generations);

/* Frees the batch (not its members). NULL is accepted. */
qieo_status qieo_destroy_batch(qieo_batch *batch);

/* One call: qieo_create_batch, qieo_batch_run(generations), qieo_destroy_batch. Returns
 * when the generations have run. For repeated runs of the same members keep a batch (its
 * work list and graphs are built once). */
qieo_status qieo_run_batch(qieo_instance *const *instances, int32_t n, int32_t generations);

/* Picks the launch shape (tile of lanes x warps vectors) of an instance at generation 0 by
 * timing `trial_generations` generations of each candidate shape, keeps the fastest, and
 * records it in a process-wide table keyed by (ng, np, D, rule, sum form) so that
 * instances created later with the same key start with it. The instance is left at
 * generation 0 (qieo_reset). Results never depend on the shape. *shape_out may be NULL. */
qieo_status qieo_autotune(qieo_instance *inst, int32_t trial_generations,
                          qieo_launch_shape *shape_out);

/* Serving (continuous batching of solve requests; the paper solves one problem per run).
 * A server reserves one device arena for resident populations and runs a worker thread:
 * submitted requests queue in arrival order and are admitted, as arena memory and the
 * active-solve limit allow, into the set of resident solves; every scheduling step runs
 * gens_per_step generations of all resident solves with the batched kernel (one launch per
 * generation), and a solve that reaches its generation count leaves, freeing its memory
 * for the next arrivals. Each result is bit-identical to qieo_run on the same problem and
 * params alone. */
typedef struct qieo_server qieo_server;

typedef struct {
    int64_t memory_bytes;     /* device arena for resident solves; 0: half of the free memory */
    int32_t max_active;       /* most resident solves at once; 0: 1024 */
    int32_t gens_per_step;    /* generations per scheduling step; 0: 25 */
} qieo_server_config;

#define QIEO_SOLVE_QUEUED 0
#define QIEO_SOLVE_RUNNING 1
#define QIEO_SOLVE_DONE 2
#define QIEO_SOLVE_CANCELLED 3
#define QIEO_SOLVE_FAILED 4

typedef struct {
    int32_t state;            /* QIEO_SOLVE_* */
    int32_t status;           /* qieo_status of a failed solve */
    int64_t fitness;          /* best-so-far record of the solve (see qieo_get_best) */
    int32_t generation, chromosome;
    double submit_s, admit_s, done_s;   /* seconds on the server's clock */
    int32_t generations_run;  /* generations the solve ran (fewer than asked if it converged) */
    int32_t converged;        /* 1: stopped by the convergence test (QIEO_FLAG_CONVERGE) */
} qieo_solve_result;

/* Creates a server on the current device. QIEO_ERR_OOM if the arena cannot be reserved. */
qieo_status qieo_server_create(const qieo_server_config *config, qieo_server **out);

/* Queues one solve: `generations` generations of problem (host arrays, copied) with params
 * (np, D, lambda, seed, instance_id, rotate_rule, and of the flags QIEO_FLAG_CONVERGE, with
 * which `generations` is a cap and the solve leaves as soon as it converged; stream, the
 * other flags and elite_on_host are ignored). *id_out receives the request id.
 * QIEO_ERR_OOM when the solve needs more device memory than the whole arena (it could
 * never be admitted); QIEO_ERR_INVALID for bad arguments. Thread-safe. */
qieo_status qieo_server_submit(qieo_server *server, const qieo_problem *problem,
                               const qieo_params *params, int32_t generations, int64_t *id_out);

/* Result of request `id`; waits up to wait_ms milliseconds for it to finish (0: do not
 * wait). bits_out (ng bytes, may be NULL) receives the best alleles once done. */
qieo_status qieo_server_poll(qieo_server *server, int64_t id, int32_t wait_ms, uint8_t *bits_out,
                             qieo_solve_result *result);

/* Counters of a server since its creation. kernel_launches counts every kernel the server
 * put on the GPU (one initialisation per admitted solve; per step and group of members,
 * one batched launch per generation plus the final rotation). */
typedef struct {
    int64_t submitted, admitted, completed, steps, kernel_launches;
    int32_t queued, active;   /* now */
    int32_t max_active;       /* most resident solves seen at once */
    int32_t reserved;
} qieo_server_stats;

qieo_status qieo_server_get_stats(qieo_server *server, qieo_server_stats *out);

/* Cancels a request that is still queued (QIEO_ERR_BUSY once it runs). */
qieo_status qieo_server_cancel(qieo_server *server, int64_t id);

/* Cancels queued requests, waits (bounded) for running ones, stops the worker, frees the
 * arena. NULL is accepted. */
qieo_status qieo_server_destroy(qieo_server *server);

/* Philox4x32-10 on the device for n (counter, key) pairs: ctr_key is n*6 host uint32
 * (c0 c1 c2 c3 k0 k1), out is n*4 host uint32. Uses the library's default stream. */
qieo_status qieo_philox(const uint32_t *ctr_key, uint32_t *out, int32_t n);

/* Largest population qieo_generation_noalloc accepts (the size of its static array). */
#define QIEO_NOALLOC_MAX_NP 65536

/* One generation (observe, evaluate, pick the elite, rotate toward it) on buffers the
 * caller already owns in device memory, allocating nothing. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc where they need a
 * generation -- code that runs while its memory pool is locked or being torn down,
 * latency-critical loops in which an allocation may stall, and hosts whose own allocator
 * owns all of device memory.
 *
 * Arguments: problem->weights and problem->values are DEVICE pointers (ng int32 each);
 * params supplies np (1 .. QIEO_NOALLOC_MAX_NP), dtheta_den, penalty_lambda, seed,
 * instance_id, rotate_rule and stream (elite_on_host and flags are ignored); t is the
 * absolute generation number (it keys the Philox draws). k (np*ng int16, in/out) holds
 * the angle indices before the generation and receives them after its rotation; x
 * (np*ng uint8) receives the alleles, fitness (np int64) the fitness values (penalised
 * as in qieo_run) and elite (one int32) the lowest-index best chromosome. All four are
 * device pointers, row c = chromosome c. Called with t = 0, 1, 2, ... on k starting at 0
 * it produces what qieo_run(inst, 1) produces for each generation. Angle indices outside
 * [-K, K] are invalid input: such an index is observed as the nearest bound, and its
 * rotation step is taken only when the step lands inside [-K, K].
 *
 * Working memory: the per-chromosome sums and a block counter live in one file-scope
 * device array of 256 + 16 * QIEO_NOALLOC_MAX_NP bytes (about 1 MB) that every GPU which
 * loads the library holds until the process exits. Every call uses that same array and
 * clears what it needs at its start, so calls whose GPU work overlaps (two streams, or two
 * host threads) race and give wrong results: serialise them. The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture. Sizes beyond the limits return QIEO_ERR_INVALID with a message; no
 * cudaMalloc, cudaFree or other allocating call is made. Stream-ordered: returns after
 * enqueueing. */
qieo_status qieo_generation_noalloc(const qieo_problem *problem, const qieo_params *params,
                                    int32_t t, int16_t *k, uint8_t *x, int64_t *fitness,
                                    int32_t *elite);

/* Message of the last failure on this thread ("" if none). */
const char *qieo_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QIEO_H */
