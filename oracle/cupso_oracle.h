/*
 * cupso_oracle.h -- plain, slow, single-threaded CPU oracle of one PSO run.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls
 * this code: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do. It shares no source, header, table or constant with the CUDA
 * library; every constant below is derived at run time from its mathematical
 * definition.
 *
 * What it computes: the Standard PSO of Alg. 1 (Sec. 2.1) with the velocity
 * update of Eq. 1 and the position update of Eq. 2, parameters as in Table 1,
 * in FP32 with every operation rounded to nearest and in a fixed order, so that
 * a GPU implementation of the same reading can match it bit for bit. The
 * library minimises; the paper's maximised cubic (Eq. 3) is minimised as -f.
 *
 * State layout (oracle-private): particle-major, pos[i*D + d].
 */
#ifndef CUPSO_ORACLE_H
#define CUPSO_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORA_SPHERE = 0,
    ORA_RASTRIGIN = 1,
    ORA_ACKLEY = 2,
    ORA_ROSENBROCK = 3,
    ORA_CUBIC_MAX = 4,
    ORA_LSQ = 5
};

typedef struct {
    int N;          /* particle_cnt */
    int D;          /* dimensions */
    float min_pos;  /* Table 1 */
    float max_pos;
    float max_v;    /* min_v = -max_v */
    float w, c1, c2;
    int fitness;    /* ORA_* */
    uint64_t seed;  /* Philox key */
    uint32_t swarm; /* fourth Philox counter word */
    /* least squares ||A x - b||^2 (ORA_LSQ only): A is [lsq_M][D] row-major */
    const float* lsq_A;
    const float* lsq_b;
    int lsq_M;
    /* nonzero: the least-squares fitness is computed in binary64 in the order
     * of ora_lsq_f64 and rounded once to binary32 (the reference "FP64
     * fitness" swarm); zero: ora_lsq_f32 */
    int lsq_fp64;
} ora_params;

typedef struct {
    float *pos;        /* [N][D] */
    float *v;          /* [N][D] */
    float *pbest_pos;  /* [N][D] */
    float *pbest_fit;  /* [N]    */
    float *fit;        /* [N]    fitness of the current position */
    float *gbest_pos;  /* [D]    */
    float gbest_fit;
    int64_t gbest_idx;
    uint32_t t;        /* iterations completed */
} ora_state;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): 10 rounds of the 4x32 bijection keyed by key[2]. */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* One 32-bit word -> uniform in (0,1]: ((w >> 8) + 1) * 2^-24. */
float ora_u01(uint32_t w);

/* The two uniforms (r1, r2) of particle i, dimension d, iteration t. */
void ora_draw_r(const ora_params* p, uint32_t t, int i, int d, float* r1, float* r2);

/* Own cos(2*pi*x) and exp(y) in FP32 (range reduction + Taylor polynomial). */
float ora_cos2pi(float x);
float ora_exp(float y);
/* The polynomial coefficients those use, as computed here (for the pins). */
void ora_cos2pi_coeffs(float out[8]);
void ora_exp_coeffs(float out[9], float* log2e, float* ln2_hi, float* ln2_lo);

/* Fitness of one position (D contiguous floats); lower is better. */
float ora_fitness(int fitness, const float* x, int D);

/* Least-squares fitness in FP32 with a fixed order: per m, r = -b_m, then
 * r = fma(A_md, x_d, r) for d = 0..D-1; acc = fma(r, r, acc) for m = 0..M-1. */
float ora_lsq_f32(const float* A, const float* b, int M, int D, const float* x);
/* The same sum in double precision (the FP64 reference of the rescoring and
 * of the FP64-fitness swarm): per m, r = -b_m, then r = r + A_md * x_d for
 * d = 0..D-1 (each product of two binary32 values is exact in binary64, so
 * one rounding per term); acc = acc + r * r for m = 0..M-1 (the square
 * rounded, then the sum). */
double ora_lsq_f64(const float* A, const float* b, int M, int D, const float* x);
/* Rounding of binary32 values to the tensor-core operand formats: bfloat16
 * (round to nearest even) and FP8 e4m3 (round to nearest even, saturated to
 * +-448); the _n forms round an array. */
float ora_round_bf16(float x);
float ora_round_e4m3(float x);
void ora_round_bf16_n(const float* in, float* out, size_t n);
void ora_round_e4m3_n(const float* in, float* out, size_t n);
/* The least-squares fitness as the tensor-core modes of the swarm compute it:
 * ||A (x - g) + (A g - b)||^2 around the reference point g, from rounded
 * operands (fmt 1 = BF16, 2 = FP8 with row scales of A and the scale sx of the
 * displacement), evaluated in binary64. */
double ora_lsq_disp(const float* A, const float* b, int M, int D, const float* x, const float* g, int fmt,
                    float sx);
/* Fitness with the swarm's parameters (LSQ needs p->lsq_*). */
float ora_fitness_p(const ora_params* p, const float* x);

/* Order-preserving 32-bit key of a fitness value (NaN -> 0xFFFFFFFF). */
uint32_t ora_fit_key(float f);

/* Step 1 of Alg. 1 (t = 0). Arrays must be allocated by the caller. */
int ora_init(const ora_params* p, ora_state* s);

/* `iters` iterations of Steps 2-5 with synchronous gbest: every particle of
 * iteration t uses the gbest from the end of iteration t-1. If r_override is
 * non-null it holds r1,r2 for every (iteration, particle, dim):
 * r_override[((k*N + i)*D + d)*2 + {0,1}] for k < iters. */
int ora_step_sync(const ora_params* p, ora_state* s, int iters, const float* r_override);
/* ora_step_sync with Steps 2-4 on `threads` host threads (OpenMP over the
 * independent particles; Step 5 serial): the same result for any count. */
int ora_step_sync_threads(const ora_params* p, ora_state* s, int iters, int threads);

/* The same, but with gbest updated inside the particle loop exactly as the
 * sequential Alg. 1 writes it (a later particle sees an earlier one's gbest). */
int ora_step_serial(const ora_params* p, ora_state* s, int iters, const float* r_override);

/* Steps 2-4 of Alg. 1 for ONE particle with global index i at iteration t:
 * Eq. 1 and Eq. 2 with their clamps, the fitness, and the strict pbest
 * update, in place; gbest_pos is read only. r_particle (nullable) overrides
 * the draws: r_particle[2d], r_particle[2d+1] = r1, r2 of dimension d.
 * Returns the new fitness. */
float ora_move_one(const ora_params* p, uint32_t t, int i, float* pos, float* v, float* pbest_pos,
                   float* pbest_fit, const float* gbest_pos, const float* r_particle);

/* Lexicographic argmin over (pbest_fit[i], i); NaN ranks last. */
int64_t ora_argmin_pbest(const ora_params* p, const ora_state* s);


/* ------------------------------------------------------------------------- */
/* Double precision (the paper's own precision, Sec. 5.1: FP64 state and     */
/* uniforms). Same algorithm as above with every operation in binary64.      */
/* Fitness: ORA_SPHERE, ORA_ROSENBROCK and ORA_CUBIC_MAX.                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int N, D;
    double min_pos, max_pos, max_v;
    double w, c1, c2;
    int fitness;
    uint64_t seed;
    uint32_t swarm;
} ora_params_d;

typedef struct {
    double *pos, *v, *pbest_pos;  /* [N][D] */
    double *pbest_fit, *fit;      /* [N]    */
    double *gbest_pos;            /* [D]    */
    double gbest_fit;
    int64_t gbest_idx;
    uint32_t t;
} ora_state_d;

/* Two 32-bit words -> uniform in (0,1] with 53 significant bits:
 * m = hi * 2^21 + (lo >> 11), u = (m + 1) * 2^-53. */
double ora_u53(uint32_t hi, uint32_t lo);

/* (r1, r2) of particle i, dimension d, iteration t: one Philox4x32-10 call
 * with counter (d, i, t, swarm); r1 from words 0,1 and r2 from words 2,3
 * (at t = 0 the same words give pos0 and v0). */
void ora_draw_r_d(const ora_params_d* p, uint32_t t, int i, int d, double* r1, double* r2);

/* Fitness of one position in binary64 (same order as the FP32 versions). */
double ora_fitness_d(int fitness, const double* x, int D);

/* Order-preserving 64-bit key of a binary64 fitness (NaN -> all ones). */
uint64_t ora_fit_key_d(double f);

int ora_init_d(const ora_params_d* p, ora_state_d* s);
int ora_step_sync_d(const ora_params_d* p, ora_state_d* s, int iters);
int64_t ora_argmin_pbest_d(const ora_params_d* p, const ora_state_d* s);

/* Steps 2-4 for ONE particle (global index i, iteration t), in place. */
double ora_move_one_d(const ora_params_d* p, uint32_t t, int i, double* pos, double* v, double* pbest_pos,
                      double* pbest_fit, const double* gbest_pos);

#ifdef __cplusplus
}
#endif
#endif
