/*
 * cupso.h -- C ABI of the GB300 particle swarm optimizer (libcupso.so).
 *
 * The library runs the Standard PSO of Alg. 1 (Sec. 2.1 of "cuPSO: GPU
 * Parallelization for Particle Swarm Optimization Algorithms") on one GPU:
 * velocity update (Eq. 1) and position update (Eq. 2) with the clamps of
 * Alg. 1, fitness of every particle, personal-best update, and the global-best
 * aggregation of Sec. 3 (conditional atomic update instead of a tree
 * reduction; synchronous and asynchronous lock-protected forms). The
 * parameters are those of Table 1 (w, c1, c2, min/max_pos, max_v, particle
 * count); min_v = -max_v.
 *
 * Conventions for every function:
 *  - Return value: CUPSO_OK (0) or a negative cupso_status. No exception or
 *    abort crosses the ABI. Arguments are checked on the host before any GPU
 *    work; an invalid argument changes nothing.
 *  - Host pointers are host memory owned by the caller. The library owns all
 *    device memory of a handle and frees it in cupso_destroy.
 *  - Work is queued on the handle's stream (cupso_set_stream; default: a
 *    non-blocking stream the handle creates). Only cupso_get_gbest,
 *    cupso_get_state, cupso_set_state, cupso_create and cupso_destroy wait
 *    for it. A device-side error (timeout of a bounded wait, NaN fitness)
 *    sets a sticky status that the next waiting call returns.
 *  - One handle must not be used from two host threads at once.
 *  - Random numbers: Philox4x32-10 keyed by the 64-bit seed with the counter
 *    (d >> 1, particle, iteration, swarm id), so results are reproducible
 *    and independent of how the work is scheduled (Sec. 4.4 draws r1, r2
 *    uniformly; here they lie in (0, 1]).
 *  - The optimizer minimises. CUPSO_CUBIC_MAX is the paper's Eq. 3, which the
 *    paper maximises, minimised as its negation; its reported fitness is -f.
 */
#ifndef CUPSO_H
#define CUPSO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CUPSO_VERSION 1

/* Symbols of the library's ABI (everything else in libcupso.so is hidden). */
#if defined(__GNUC__)
#define CUPSO_API __attribute__((visibility("default")))
#else
#define CUPSO_API
#endif

typedef struct cupso_swarm* cupso_handle; /* opaque, owned by the library */

/* Search box, the same for every dimension (Table 1): positions are clamped
 * to [min_pos, max_pos], velocities to [-max_v, max_v]. Requires
 * min_pos < max_pos and max_v > 0, all finite. */
typedef struct {
    float min_pos;
    float max_pos;
    float max_v;
} cupso_bounds;

/* The same search box in double precision (double-precision swarms). */
typedef struct {
    double min_pos;
    double max_pos;
    double max_v;
} cupso_bounds_f64;

typedef enum {
    CUPSO_SPHERE = 0,     /* sum x^2                                   */
    CUPSO_RASTRIGIN = 1,  /* 10 D + sum (x^2 - 10 cos 2 pi x)          */
    CUPSO_ACKLEY = 2,     /* -20 e^{-0.2 sqrt(mean x^2)} - e^{mean cos 2 pi x} + 20 + e */
    CUPSO_ROSENBROCK = 3, /* sum 100 (x_{d+1} - x_d^2)^2 + (1 - x_d)^2 */
    CUPSO_CUBIC_MAX = 4,  /* Eq. 3: maximise sum x^3 - 0.8 x^2 - 1000 x + 8000 */
    CUPSO_LSQ = 5         /* ||A x - b||^2 with A, b given by cupso_set_lsq */
} cupso_fitness;

/* Arithmetic of the least-squares fitness. */
typedef enum {
    CUPSO_LSQ_FP32 = 0,   /* CUDA cores, fixed FP32 order (bit-exact with the oracle)          */
    CUPSO_LSQ_BF16 = 1,   /* tensor cores, BF16 operands, FP32 accumulation                    */
    CUPSO_LSQ_FP8 = 2,    /* tensor cores, FP8 e4m3 operands (A scaled per row), FP32 accumulation */
    CUPSO_LSQ_FP64 = 3    /* CUDA cores, FP64 in a fixed order, rounded once to FP32 (bit-exact with
                             the oracle): the exact-fitness reference of the precision comparison */
} cupso_lsq_precision;

typedef enum {
    CUPSO_OK = 0,
    CUPSO_ERR_INVALID_ARG = -1,
    CUPSO_ERR_OOM = -2,
    CUPSO_ERR_CUDA = -3,
    CUPSO_ERR_DEVICE_TIMEOUT = -4, /* a bounded device-side wait expired */
    CUPSO_ERR_NAN = -5,            /* a fitness evaluated to NaN          */
    CUPSO_ERR_UNSUPPORTED = -6
} cupso_status;

/* How the global best is aggregated (cupso_set_option(CUPSO_OPT_MODE)). */
typedef enum {
    CUPSO_MODE_AUTO = 0,   /* ONCHIP when the swarm fits, else SYNC                        */
    CUPSO_MODE_SYNC = 1,   /* fused kernel, conditional atomicMin + last-CTA gather (Sec. 3.1) */
    CUPSO_MODE_TREE = 2,   /* parallel-reduction baseline: two kernels per iteration (Sec. 2.2) */
    CUPSO_MODE_TREE_UNROLLED = 3, /* the same with the unrolled reduction (Sec. 2.2)       */
    CUPSO_MODE_ASYNC = 4,  /* persistent CTAs, no grid barrier, lock-protected gbest (Sec. 3.2) */
    CUPSO_MODE_ONCHIP = 5, /* whole swarm in one CTA cluster's shared memory, many iterations per launch */
    CUPSO_MODE_QUEUE = 6,  /* the paper's queue design (Alg. 2): one particle per thread, a
                              shared-memory queue of the particles that beat gbest, a second kernel */
    CUPSO_MODE_QUEUE_LOCK = 7, /* the paper's queue-lock design (Alg. 3): the queue, then thread 0 of
                              each block updates gbest in place under a global lock; one kernel. Blocks
                              later in the same launch may see an earlier block's update, so with more
                              than one block (N > 256) the trajectory depends on timing. */
    CUPSO_MODE_PERSISTENT = 8 /* double-precision swarms: one cooperative launch runs all iterations of a
                              cupso_step call, a grid-wide barrier per iteration in place of the kernel
                              boundary (synchronous PSO, one particle per thread) */
} cupso_mode;

typedef enum {
    CUPSO_OPT_MODE = 1,           /* value: cupso_mode                                         */
    CUPSO_OPT_GRAPH_CHUNK = 2,    /* iterations per captured CUDA graph (SYNC/TREE); 0 = none  */
    CUPSO_OPT_WAIT_LIMIT_NS = 3,  /* bound of every device-side wait (default 2e9 ns)          */
    CUPSO_OPT_CLEAR_STATUS = 4,   /* any value: clear the sticky device status                 */
    CUPSO_OPT_GRID = 5,           /* CTAs of the persistent kernels (SYNC/ASYNC); 0 = automatic */
    CUPSO_OPT_SYNC_KERNEL = 6,    /* value: cupso_sync_kernel (which SYNC kernel runs)         */
    CUPSO_OPT_PARTICLES_PER_THREAD = 8, /* pipelined SYNC kernel: 4, 2, 1, or 0 = automatic (fewer
                                           for small swarms, so that their units fill the GPU) */
    CUPSO_OPT_TIME_FITNESS = 7,   /* 1: time the fitness phase of least-squares iterations with
                                     CUDA events (no graph capture); 0: off. Read in cupso_info.
                                     BF16/FP8: the tensor-core product alone (the move kernel
                                     before it writes the operand; the selection after it adds the
                                     product's partial sums) */
    CUPSO_OPT_ITERS_PER_LAUNCH = 9, /* SYNC step on the panel layout: iterations per launch of a
                                       cupso_step call. 1: one kernel per iteration (graphs per
                                       CUPSO_OPT_GRAPH_CHUNK); n > 1: up to n per cooperative launch,
                                       all CTAs resident, a grid barrier between iterations (each
                                       wait bounded by CUPSO_OPT_WAIT_LIMIT_NS); 0 (default): up to
                                       4096. Same results either way. */
    CUPSO_OPT_LSQ_RESCORE = 10,   /* BF16 / FP8 least-squares swarm with D <= M: arithmetic of
                                     the Gram-form rescoring of its gbest candidates. 0 (default):
                                     the off-diagonal part of x^T (A^T A) x in float-float (pairs
                                     of binary32 values, about 2^-44 of the terms' magnitudes);
                                     1: binary64 throughout. The diagonal, linear and constant
                                     terms are binary64 either way. */
    CUPSO_OPT_FAULT_HOLD_LOCK = 100, /* test hook: ASYNC starts with the gbest lock held, so every
                                        lock wait must expire and report CUPSO_ERR_DEVICE_TIMEOUT */
    CUPSO_OPT_FAULT_STALL_BARRIER = 101 /* test hook: a multi-iteration panel launch waits for one CTA
                                           more than it has, so its first barrier wait expires and
                                           reports CUPSO_ERR_DEVICE_TIMEOUT; the swarm's state is then
                                           undefined (CUPSO_OPT_CLEAR_STATUS resets the counters) */
} cupso_option;

/* The implementations of the SYNC step; all compute the same bits. */
typedef enum {
    CUPSO_SYNC_KERNEL_AUTO = 0,       /* tiled for small swarms, else the panel kernel where D
                                         allows, else the deepest pipelined ring supported, else
                                         register                                           */
    CUPSO_SYNC_KERNEL_REGISTER = 1,   /* loads straight into registers, 1024-particle tiles */
    CUPSO_SYNC_KERNEL_PIPELINED3 = 2, /* rows staged through shared memory, 2 pairs ahead   */
    CUPSO_SYNC_KERNEL_PIPELINED4 = 3, /* the same, 3 pairs ahead                            */
    CUPSO_SYNC_KERNEL_TILED = 4,      /* a tile of particles with all their dimensions per block,
                                         the (dimension pair, particle) items spread over threads;
                                         AUTO uses it for D >= 8 up to about 896 particles per SM
                                         (224 for D > 64 without cos(2 pi x) in the fitness)     */
    CUPSO_SYNC_KERNEL_PANEL8 = 5,     /* the state in panels of 8 dimensions (each particle's 8 values
                                         of a panel contiguous), two threads per particle, rows staged
                                         through shared memory; D % 8 == 0, D >= 16. A particle whose
                                         pbest is pending skips its pbest load and writes the row
                                         instead: 20 bytes per particle-dimension whatever fraction of
                                         the swarm improves                                       */
    CUPSO_SYNC_KERNEL_PANEL16 = 6     /* the same with panels of 16 dimensions (64 bytes per particle,
                                         the granularity of HBM reads), four threads per particle;
                                         D % 16 == 0, D >= 32. AUTO, for D % 8 == 0: the tiled kernel
                                         below 2^17 particle-dimensions, above that 16-dimension
                                         panels for D >= 128 or N <= 8192, else 8                  */
} cupso_sync_kernel;

typedef struct {
    int N, D;             /* particles, dimensions                   */
    int Np;               /* N rounded up to 128 (device row stride) */
    int mode;             /* cupso_mode the next cupso_step will use */
    uint32_t t;           /* iterations completed                    */
    int sync_grid;        /* CTAs of the persistent SYNC launch      */
    int async_grid;       /* CTAs of the ASYNC launch                */
    int onchip_cluster;   /* CTAs per cluster if ONCHIP fits, else 0 */
    int sync_stages;      /* ring depth of the SYNC kernel in use, 0 = register kernel */
    int sync_ppt;         /* particles per thread of the pipelined SYNC kernel (0: not in use) */
    int sync_tile;        /* particles per tile of the tiled SYNC kernel (0: not in use) */
    float fitness_ms;     /* mean fitness-phase time of the timed LSQ iterations, 0 if none */
    int fitness_timed;    /* how many iterations that mean covers */
    uint64_t device_bytes;/* device memory held by the handle        */
    int sync_panel;       /* panel width (8 or 16) when the SYNC step runs the panel kernel, else 0 */
    int sync_iters_per_launch; /* most iterations one SYNC launch runs (CUPSO_OPT_ITERS_PER_LAUNCH) */
} cupso_info;

/* Create a swarm and run Step 1 of Alg. 1 (iteration t = 0) on the device:
 * pos ~ U(min_pos, max_pos], v ~ U(-max_v, max_v], pbest = pos, gbest =
 * lowest-index argmin of the fitness. D >= 1, N >= 1, N * D < 2^31 and
 * N < 2^31 - 128. Waits for the initialisation. On success *out is a new
 * handle; on error *out is set to NULL. */
CUPSO_API int cupso_create(int D, int N, const cupso_bounds* bounds, float w, float c1, float c2,
                 int fitness_id, uint64_t seed, cupso_handle* out);

/* Queue this handle's work on `cuda_stream` (a cudaStream_t; NULL selects
 * the handle's own non-blocking stream). Work already queued is not moved. */
CUPSO_API int cupso_set_stream(cupso_handle h, void* cuda_stream);

/* Set an option (cupso_option). Unknown keys: CUPSO_ERR_INVALID_ARG. */
CUPSO_API int cupso_set_option(cupso_handle h, int key, long long value);

/* Queue `iters` >= 0 iterations of Steps 2-5 (Alg. 1). SYNC, TREE,
 * TREE_UNROLLED, QUEUE and ONCHIP are synchronous PSO: every particle of
 * iteration t uses the gbest from the end of iteration t-1 (Sec. 2.2,
 * "PPSO"), and the result does not depend on the mode or the launch shape.
 * ASYNC lets CTAs run ahead of each other, and QUEUE_LOCK updates gbest in
 * place during an iteration, so their trajectories depend on timing
 * (Sec. 3.2). Does not wait. */
CUPSO_API int cupso_step(cupso_handle h, int iters);

/* Wait for the handle's stream, then return gbest: *fit_out = gbest_fit,
 * pos_out[0..D-1] = gbest_pos, *idx_out = index of the particle whose pbest
 * it is. Any output pointer may be NULL. Returns the sticky device status
 * (CUPSO_ERR_DEVICE_TIMEOUT or CUPSO_ERR_NAN) when one is set; the outputs
 * are filled in that case too. */
CUPSO_API int cupso_get_gbest(cupso_handle h, float* fit_out, float* pos_out, int64_t* idx_out);

/* The same result without waiting, for a loop that reads every step's gbest
 * while the next steps run. cupso_gbest_post queues, on the handle's stream
 * after the work queued so far, a snapshot of gbest (fitness key, index,
 * position, sticky status) into result slot `slot` (0 or 1) and its copy to
 * host memory on a second stream; it does not wait. cupso_gbest_wait waits for
 * the copy of `slot` and returns it as cupso_get_gbest does (outputs may be
 * NULL; the sticky status as the return value). A slot holds one result:
 * wait for it before posting to it again (posting again first is
 * CUPSO_ERR_INVALID_ARG; so is waiting on a slot with nothing posted).
 * Single-precision swarms only. */
CUPSO_API int cupso_gbest_post(cupso_handle h, int slot);
CUPSO_API int cupso_gbest_wait(cupso_handle h, int slot, float* fit_out, float* pos_out, int64_t* idx_out);

/* Wait, then copy the swarm state to host arrays in particle-major layout:
 * pos, v, pbest_pos are [N][D] (element i*D + d), pbest_fit is [N]; *t_out =
 * iterations completed. Any pointer may be NULL. */
CUPSO_API int cupso_get_state(cupso_handle h, float* pos, float* v, float* pbest_pos, float* pbest_fit,
                    uint32_t* t_out);

/* Load a swarm state (layout as cupso_get_state; all four arrays required)
 * and set the iteration counter to t; gbest is recomputed on the device as
 * the lowest-index argmin of pbest_fit. Waits for the upload. Together with
 * cupso_get_state this is checkpoint and resume: the random draws depend only
 * on (seed, swarm, t, particle, dimension). */
CUPSO_API int cupso_set_state(cupso_handle h, const float* pos, const float* v, const float* pbest_pos,
                    const float* pbest_fit, uint32_t t);

/* Least-squares fitness ||A x - b||^2 for a swarm created with CUPSO_LSQ:
 * A device [M][D] row-major float32, b device [M] float32, both borrowed (they
 * must stay valid until the handle is destroyed or they are replaced).
 * precision (cupso_lsq_precision) selects how the swarm's fitness -- one
 * matrix product X A^T per iteration -- is computed: FP32 or FP64 on the CUDA
 * cores in a fixed order (the synchronous trajectory is then exactly the
 * oracle's), or BF16 / FP8 e4m3 on the tensor cores with FP32 accumulation.
 * The tensor-core product takes each particle's displacement from the current
 * gbest_pos g, x - g, as its operand, and adds the residual offsets A g - b
 * (computed once per change of g with a compensated FP32 dot product) in its
 * epilogue: the same function ||A x - b||^2, with the operand rounding scaled
 * by |x - g|, which shrinks as the swarm converges, instead of by |x|. In the
 * BF16 and FP8 modes the pbest decisions use the approximate fitness, while a
 * global best is accepted only after the (up to) 16 improved particles with
 * the lowest approximate fitness are rescored in extended precision; gbest_fit
 * is then that value (rounded to float). For D <= M (and D <= 6144) the
 * rescoring takes the Gram form x^T G x - 2 c^T x + b^T b with G = A^T A and
 * c = A^T b formed once here in FP64, its off-diagonal part in float-float
 * or FP64 arithmetic (CUPSO_OPT_LSQ_RESCORE); otherwise it sums the residuals
 * (A x - b)_m^2 in FP64 directly. This call evaluates the fitness of every
 * particle's pbest_pos (the end of Step 1 for such a swarm) and the gbest, and
 * waits. Steps of a CUPSO_LSQ swarm fail until it has been called. */
CUPSO_API int cupso_set_lsq(cupso_handle h, const float* A_dev, const float* b_dev, int M, int precision);

/* Fitness ||A g - b||^2 of the current gbest_pos g of a least-squares swarm
 * (the residual by which the precision modes are compared), as a double: FP32
 * and FP64 swarms rescore g in FP64; BF16 and FP8 swarms return the value
 * their rescoring accepted g with (see cupso_set_lsq). Waits. */
CUPSO_API int cupso_get_gbest_f64(cupso_handle h, double* fit_out);

/* Double-precision swarm: the paper's own precision (Sec. 5.1 runs FP64).
 * Same algorithm, arguments and conventions as cupso_create, with binary64
 * state and arithmetic, and 53-bit uniforms: one Philox4x32-10 call per
 * (dimension, particle, iteration) with counter (d, particle, t, swarm id 0);
 * words 0,1 give r1 (pos0 at t = 0) and words 2,3 give r2 (v0), each as
 * (m + 1) 2^-53 with m = w_hi 2^21 + (w_lo >> 11). fitness_id: CUPSO_SPHERE,
 * CUPSO_ROSENBROCK or CUPSO_CUBIC_MAX (others: CUPSO_ERR_UNSUPPORTED). Modes:
 * SYNC (one fused launch per iteration: block argmin, a candidate list, the
 * last block gathers gbest), TREE, TREE_UNROLLED, QUEUE, QUEUE_LOCK (the
 * paper's four designs, one particle per thread), ONCHIP (one CTA holds the
 * swarm in shared memory; only when it fits), PERSISTENT (one cooperative
 * launch per cupso_step call); AUTO picks ONCHIP when it fits, else SYNC.
 * ASYNC is not available. Use cupso_step, cupso_set_option,
 * cupso_get_info and cupso_destroy as for any handle, and the _fp64 accessors
 * below: the float accessors return CUPSO_ERR_UNSUPPORTED on such a handle. */
CUPSO_API int cupso_create_fp64(int D, int N, const cupso_bounds_f64* bounds, double w, double c1, double c2,
                                int fitness_id, uint64_t seed, cupso_handle* out);

/* cupso_get_gbest for a double-precision swarm. */
CUPSO_API int cupso_get_gbest_fp64(cupso_handle h, double* fit_out, double* pos_out, int64_t* idx_out);

/* cupso_get_state / cupso_set_state for a double-precision swarm. */
CUPSO_API int cupso_get_state_fp64(cupso_handle h, double* pos, double* v, double* pbest_pos, double* pbest_fit,
                                   uint32_t* t_out);
CUPSO_API int cupso_set_state_fp64(cupso_handle h, const double* pos, const double* v, const double* pbest_pos,
                                   const double* pbest_fit, uint32_t t);

/* Fill *info. */
CUPSO_API int cupso_get_info(cupso_handle h, cupso_info* info);

/* One problem of a batch: an independent swarm with its own parameters.
 * swarm_id is the fourth word of the Philox counter. */
typedef struct {
    int D, N;
    cupso_bounds bounds;
    float w, c1, c2;
    int fitness_id;
    uint64_t seed;
    uint32_t swarm_id;
} cupso_problem;

typedef struct {
    float fit;        /* gbest_fit after `iters` iterations        */
    int64_t idx;      /* its particle                              */
    float* pos;       /* caller-allocated D floats, or NULL        */
    int status;       /* cupso_status of this swarm                */
} cupso_result;

/* Solve n_swarms independent problems for `iters` iterations each (Step 1
 * included) on `cuda_stream` (NULL: an internal stream) and wait. Each
 * swarm's result equals what cupso_create with seed and swarm_id, then
 * cupso_step(iters), would give. Returns CUPSO_OK if every swarm succeeded,
 * else the first failing status; results[k].status holds each swarm's.
 * Every iteration of all swarms is one launch; the kernel and launch shape
 * are tuned on the first iterations (the environment variable
 * CUPSO_BATCH_KERNEL=tiled or =streaming fixes the kernel instead).
 * CUPSO_ERR_INVALID_ARG (before any device work) for a bad argument in any
 * problem, and for CUPSO_LSQ, which needs the matrices of cupso_set_lsq. */
CUPSO_API int cupso_solve_batch(int n_swarms, const cupso_problem* problems, int iters,
                      cupso_result* results, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Allocation-free iteration. The paper has no counterpart: this entry point
 * serves callers that must not allocate device memory themselves -- typically
 * a process whose GPU memory belongs to another allocator (a serving
 * framework's caching pool, or a budget an embedding application enforces),
 * where a private cudaMalloc would escape that allocator's accounting or fail
 * against its reservation. The caller keeps the swarm in its own device
 * buffers; this call allocates nothing (no cudaMalloc, no cudaFree, no
 * allocating library routine).
 *
 * Computes iteration t (t >= 1) of synchronous PSO -- Steps 2-5 with the
 * tree-reduction aggregation, i.e. what cupso_step gives in CUPSO_MODE_TREE
 * for the same seed and swarm_id -- in place on:
 *   pos, v, pbest_pos : device, [D][ld] floats (element d*ld + i), 16-byte aligned
 *   pbest_fit         : device, [ld] floats, 16-byte aligned
 *   ld                : row stride, a multiple of 128, >= N; columns N..ld-1
 *                       are moved too but never win the global best
 *   gbest_pos         : device, [D]: in = gbest after iteration t-1, out = after t
 *   gbest_fit, gbest_idx, status_out : device, one element each, or NULL;
 *                       status_out receives the device status bits (1 = NaN fitness)
 * Work is queued on `cuda_stream` (a cudaStream_t, NULL = legacy default
 * stream); the call does not wait.
 *
 * Working storage: a fixed device array of about 41 KB inside the library
 * (static, one per GPU that loads the library, held until the process exits)
 * holds the per-block keys, the double-buffered gbest position, the iteration
 * counter and the status word. Limits: N <= CUPSO_NOALLOC_MAX_N, D <=
 * CUPSO_NOALLOC_MAX_D and also ld <= CUPSO_NOALLOC_MAX_N (every column of the
 * stride is moved and reduced, one scratch key per 1024 columns); larger sizes
 * return CUPSO_ERR_INVALID_ARG with a message in cupso_last_error(), before
 * anything is queued. The first call on each device looks up that array's
 * device address (with the device current); make that first call before any
 * stream capture. The address is remembered together with the context it was
 * taken in; after cudaDeviceReset the next call looks it up again, and that
 * call, too, must come before any stream capture. Every call on a device shares the one array and
 * clears the counters it needs at its start: calls that overlap on the GPU
 * (several streams, several host threads) race and give wrong results, so
 * serialise them.
 * ------------------------------------------------------------------------- */
#define CUPSO_NOALLOC_MAX_N 4194304
#define CUPSO_NOALLOC_MAX_D 1024
CUPSO_API int cupso_tree_step_noalloc(int D, int N, const cupso_bounds* bounds, float w, float c1, float c2,
                                      int fitness_id, uint64_t seed, uint32_t swarm_id, uint32_t t,
                                      float* pos, float* v, float* pbest_pos, float* pbest_fit, int ld,
                                      float* gbest_pos, float* gbest_fit, int64_t* gbest_idx,
                                      unsigned int* status_out, void* cuda_stream);

/* Least-squares fitness of N given positions: f_out[i] = ||A x_i - b||^2 with
 * A device [M][D] row-major, b device [M], X device [N][D] row-major, f_out
 * device [N], all float32 (caller-owned). precision selects the arithmetic:
 * FP32 follows a fixed order (per row m, r = -b_m then r = fma(A_md, x_d, r)
 * for d in order; f = sum over m in order of fma(r, r, .)); FP64 the same
 * order in binary64 (acc = acc + r * r, the square rounded first), rounded
 * once to float at the end; BF16 and FP8 form X A^T on the tensor cores from
 * the positions themselves (the fitness of the dense-fitness extension of the
 * method; the paper's own fitness is analytic, Sec. 5.1). Allocates temporary
 * device memory, queues on `cuda_stream` and waits. */
CUPSO_API int cupso_lsq_eval(const float* A_dev, const float* b_dev, int M, int D, const float* X_dev, int N,
                             int precision, float* f_out_dev, void* cuda_stream);

/* Wait for the handle's work and free everything it holds. NULL is a no-op. */
CUPSO_API int cupso_destroy(cupso_handle h);

/* Static description of a status code. */
CUPSO_API const char* cupso_status_string(int status);

/* Detail of the last error on the calling host thread (static storage). */
CUPSO_API const char* cupso_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CUPSO_H */
