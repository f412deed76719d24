/*
 * cupso_oracle.c -- CPU oracle for the PSO iteration (TEST INFRASTRUCTURE ONLY).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
 * file. It follows the paper step by step:
 *   Step 1 (init)          Alg. 1, Sec. 2.1, "initialize ... uniformly distributed"
 *   Step 2 (v and pos)     Eq. 1 and Eq. 2, clamps of Alg. 1 ("keep in range")
 *   Step 3 (fitness)       Sec. 2.1 step (3); Eq. 3 for the paper's cubic
 *   Step 4 (pbest)         Alg. 1, "if fit_i better than pbest_fit_i"
 *   Step 5 (gbest)         Alg. 1, "if pbest_fit_i better than gbest_fit"
 * Random numbers (Sec. 4.4: r1, r2 uniform, cuRAND's (0,1] range) come from a
 * counter-based Philox4x32-10 written from its published definition.
 *
 * Readings where the paper is silent (each also recorded in the design notes):
 *  - minimisation (the paper maximises its cubic; we minimise -f);
 *  - r1, r2 drawn fresh per (iteration, particle, dimension);
 *  - v0 ~ U(-max_v, max_v], pos0 ~ U(min_pos, max_pos];
 *  - closed clamps; a NaN is clamped to the lower bound (IEEE maxNum/minNum);
 *  - synchronous gbest: iteration t uses the gbest at the end of t-1;
 *  - ties: strict "<" for pbest, lowest index among equal pbest_fit for gbest.
 *
 * Compile with -O2 -ffp-contract=off and no fast-math: every float operation
 * below is one IEEE-754 binary32 operation rounded to nearest.
 */
#include "cupso_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11)                                      */
/* ------------------------------------------------------------------------- */

/* Multipliers and Weyl key increments as published with the generator. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

float ora_u01(uint32_t w)
{
    /* (w >> 8) + 1 is an integer in [1, 2^24]: exact in binary32, and so is
     * its product with 2^-24. */
    return (float)((w >> 8) + 1u) * 0x1p-24f;
}

/* Counter of one draw: (dimension pair, particle, iteration, swarm). One
 * Philox call serves dimensions 2g and 2g+1 of one particle: words 0,1 are
 * (r1, r2) of dimension 2g, words 2,3 those of dimension 2g+1. At t = 0 the
 * same words give the initial (pos, v). */
static void draw_words(const ora_params* p, uint32_t t, int i, int d, uint32_t* wa, uint32_t* wb)
{
    uint32_t ctr[4] = {(uint32_t)(d >> 1), (uint32_t)i, t, p->swarm};
    uint32_t key[2] = {(uint32_t)(p->seed & 0xFFFFFFFFu), (uint32_t)(p->seed >> 32)};
    uint32_t out[4];
    ora_philox4x32_10(ctr, key, out);
    if ((d & 1) == 0) {
        *wa = out[0];
        *wb = out[1];
    } else {
        *wa = out[2];
        *wb = out[3];
    }
}

void ora_draw_r(const ora_params* p, uint32_t t, int i, int d, float* r1, float* r2)
{
    uint32_t a, b;
    draw_words(p, t, i, d, &a, &b);
    *r1 = ora_u01(a);
    *r2 = ora_u01(b);
}

/* ------------------------------------------------------------------------- */
/* Own cos(2*pi*x) and exp(y)                                                */
/* ------------------------------------------------------------------------- */
/* cos(2*pi*a) = sum_j (-1)^j (2*pi)^(2j) / (2j)! * a^(2j): Taylor series of
 * cosine, truncated after j = 7 (the j = 8 term is below 7e-11 for |a| <= 1/4).
 * exp(r) = sum_k r^k / k!, k <= 8, after Cody-Waite reduction y = n*ln2 + r.
 * The coefficients are computed here, in double, and rounded once to float. */

static float g_cos_c[8];
static float g_exp_c[9];
static float g_log2e, g_ln2_hi, g_ln2_lo;
static int g_consts_ready = 0;

static void init_consts(void)
{
    if (g_consts_ready) return;
    const double two_pi = 2.0 * M_PI;
    double term = 1.0; /* (2*pi)^(2j) / (2j)! */
    for (int j = 0; j < 8; ++j) {
        if (j > 0) term *= (two_pi * two_pi) / ((double)(2 * j - 1) * (double)(2 * j));
        g_cos_c[j] = (float)((j & 1) ? -term : term);
    }
    double fact = 1.0;
    for (int k = 0; k < 9; ++k) {
        if (k > 0) fact *= (double)k;
        g_exp_c[k] = (float)(1.0 / fact);
    }
    g_log2e = (float)(1.0 / M_LN2);
    /* ln2 cut to 16 significant bits, so n * ln2_hi is exact for |n| < 2^8. */
    double hi = ldexp(floor(ldexp(M_LN2, 16)), -16);
    g_ln2_hi = (float)hi;
    g_ln2_lo = (float)(M_LN2 - hi);
    g_consts_ready = 1;
}

void ora_cos2pi_coeffs(float out[8])
{
    init_consts();
    memcpy(out, g_cos_c, sizeof(g_cos_c));
}

void ora_exp_coeffs(float out[9], float* log2e, float* ln2_hi, float* ln2_lo)
{
    init_consts();
    memcpy(out, g_exp_c, sizeof(g_exp_c));
    *log2e = g_log2e;
    *ln2_hi = g_ln2_hi;
    *ln2_lo = g_ln2_lo;
}

/* cos(2*pi*a), 0 <= a <= 1/4, as the polynomial in z = a*a (Horner, fmaf). */
static float cos2pi_poly(float a)
{
    float z = a * a;
    float q = g_cos_c[7];
    for (int j = 6; j >= 0; --j) q = fmaf(q, z, g_cos_c[j]);
    return q;
}

float ora_cos2pi(float x)
{
    init_consts();
    if (isnan(x) || isinf(x)) return NAN;
    /* x - rint(x) is exact: for |x| >= 2^23 x is an integer (r = 0); below
     * that, x and rint(x) share the binade bounds and r fits in x's bits. */
    float r = x - rintf(x);
    float a = fabsf(r);                 /* cosine is even: 0 <= a <= 1/2 */
    if (a > 0.25f) {
        float b = 0.5f - a;             /* exact (Sterbenz): 0 <= b < 1/4 */
        return -cos2pi_poly(b);         /* cos(pi - t) = -cos(t) */
    }
    return cos2pi_poly(a);
}

float ora_exp(float y)
{
    init_consts();
    if (isnan(y)) return y;
    if (y > 88.8f) return INFINITY;
    if (y < -104.0f) return 0.0f;
    float n = rintf(y * g_log2e);
    float r = fmaf(-n, g_ln2_hi, y);
    r = fmaf(-n, g_ln2_lo, r);
    float q = g_exp_c[8];
    for (int k = 7; k >= 0; --k) q = fmaf(q, r, g_exp_c[k]);
    /* q * 2^n, in two factors so that each power of two is a normal float. */
    int ni = (int)n;
    int n1 = ni / 2;
    int n2 = ni - n1;
    return (q * ldexpf(1.0f, n1)) * ldexpf(1.0f, n2);
}

/* ------------------------------------------------------------------------- */
/* Fitness functions (Step 3). Sequential over d, accumulator starts at 0.  */
/* ------------------------------------------------------------------------- */

float ora_fitness(int fitness, const float* x, int D)
{
    init_consts();
    float acc = 0.0f;
    switch (fitness) {
    case ORA_SPHERE: /* sum x_d^2 */
        for (int d = 0; d < D; ++d) acc = fmaf(x[d], x[d], acc);
        return acc;
    case ORA_RASTRIGIN: /* sum (x_d^2 + 10 - 10 cos(2 pi x_d)) = 10 D + sum(...) */
        for (int d = 0; d < D; ++d) {
            float ten_minus = fmaf(-10.0f, ora_cos2pi(x[d]), 10.0f);
            acc = acc + fmaf(x[d], x[d], ten_minus);
        }
        return acc;
    case ORA_ACKLEY: { /* -20 exp(-0.2 sqrt(mean x^2)) - exp(mean cos 2 pi x) + 20 + e */
        float s1 = 0.0f, s2 = 0.0f;
        for (int d = 0; d < D; ++d) {
            s1 = fmaf(x[d], x[d], s1);
            s2 = s2 + ora_cos2pi(x[d]);
        }
        float m1 = s1 / (float)D;
        float m2 = s2 / (float)D;
        float e1 = ora_exp(-0.2f * sqrtf(m1));
        float part1 = 20.0f - 20.0f * e1;
        float part2 = ora_exp(1.0f) - ora_exp(m2);
        return part1 + part2;
    }
    case ORA_ROSENBROCK: /* sum_{d<D-1} 100 (x_{d+1} - x_d^2)^2 + (1 - x_d)^2 */
        for (int d = 0; d + 1 < D; ++d) {
            float p = fmaf(-x[d], x[d], x[d + 1]);
            float q = 1.0f - x[d];
            acc = acc + fmaf(100.0f * p, p, q * q);
        }
        return acc;
    case ORA_CUBIC_MAX: /* Eq. 3, maximised: return -sum (x^3 - 0.8 x^2 - 1000 x + 8000) */
        for (int d = 0; d < D; ++d) {
            float h = fmaf(fmaf(x[d] - 0.8f, x[d], -1000.0f), x[d], 8000.0f);
            acc = acc + h;
        }
        return -acc;
    default:
        return NAN;
    }
}

/* Least squares ||A x - b||^2 (the dense fitness of the precision study). */
float ora_lsq_f32(const float* A, const float* b, int M, int D, const float* x)
{
    float acc = 0.0f;
    for (int m = 0; m < M; ++m) {
        const float* row = A + (size_t)m * D;
        float r = -b[m];
        for (int d = 0; d < D; ++d) r = fmaf(row[d], x[d], r);
        acc = fmaf(r, r, acc);
    }
    return acc;
}

double ora_lsq_f64(const float* A, const float* b, int M, int D, const float* x)
{
    double acc = 0.0;
    for (int m = 0; m < M; ++m) {
        const float* row = A + (size_t)m * D;
        double r = -(double)b[m];
        for (int d = 0; d < D; ++d) r += (double)row[d] * (double)x[d];
        acc += r * r;
    }
    return acc;
}

/* ------------------------------------------------------------------------- */
/* The tensor-core fitness of the least-squares swarm, on rounded operands    */
/* ------------------------------------------------------------------------- */

/* bfloat16 keeps the upper 16 bits of the binary32 encoding: 8 significant
 * bits. Round to nearest, ties to even, by adding 0x7FFF plus the lowest kept
 * bit and truncating; a carry into the exponent gives the next binade (or
 * infinity). NaN is returned unchanged. */
float ora_round_bf16(float x)
{
    uint32_t u;
    memcpy(&u, &x, sizeof u);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) return x;
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    float r;
    memcpy(&r, &u, sizeof r);
    return r;
}

/* FP8 e4m3 (the OCP "E4M3FN" format): 3 mantissa bits, exponent bias 7, no
 * infinities, largest finite 448 = 1.75 * 2^8, normals from 2^-6, subnormals
 * k * 2^-9. Round to nearest, ties to even, on the grid of the value's binade
 * (spacing 2^(e - 3) for 2^e <= |x| < 2^(e + 1), 2^-9 below 2^-6), then
 * saturate to +-448 (the conversion the tensor-core operands use). */
float ora_round_e4m3(float x)
{
    if (isnan(x)) return x;
    const double a = fabs((double)x);
    double q = 0x1p-9;
    if (a >= 0x1p-6) {
        int e;
        frexp(a, &e);              /* a = f 2^e, 0.5 <= f < 1: the binade is 2^(e-1) */
        q = ldexp(1.0, e - 1 - 3);
    }
    double r = nearbyint(a / q) * q;   /* a / q is exact (q a power of two); default mode: ties to even */
    if (r > 448.0) r = 448.0;
    return (float)copysign(r, (double)x);
}

void ora_round_bf16_n(const float* in, float* out, size_t n)
{
    for (size_t k = 0; k < n; ++k) out[k] = ora_round_bf16(in[k]);
}

void ora_round_e4m3_n(const float* in, float* out, size_t n)
{
    for (size_t k = 0; k < n; ++k) out[k] = ora_round_e4m3(in[k]);
}

/* ||A x - b||^2 written as ||A (x - g) + (A g - b)||^2 around a reference
 * point g, with the operands the tensor cores see: per row m the offset
 * o_m = A_m g - b_m in binary64, rounded once to binary32; per dimension the
 * displacement x_d - g_d in binary32, then rounded -- BF16: A_md and the
 * displacement to bfloat16; FP8: A_md * sa_m and the displacement * sx to e4m3,
 * with sa_m = 448 / max_d |A_md| (1 for a zero row) and the product scaled back
 * by inv_m = 1 / (sx sa_m), all three in binary32. The products of the rounded
 * operands, their sum over d, the offset and the sum of squares over m are
 * then exact up to binary64 rounding: this is the value the FP32-accumulating
 * tensor-core product approximates. fmt: 1 = BF16, 2 = FP8. */
double ora_lsq_disp(const float* A, const float* b, int M, int D, const float* x, const float* g, int fmt,
                    float sx)
{
    double acc = 0.0;
    for (int m = 0; m < M; ++m) {
        const float* row = A + (size_t)m * D;
        double o = -(double)b[m];
        for (int d = 0; d < D; ++d) o += (double)row[d] * (double)g[d];
        const float off = (float)o;
        float sa = 1.0f, inv = 1.0f;
        if (fmt == 2) {
            float amax = 0.0f;
            for (int d = 0; d < D; ++d) amax = fmaxf(amax, fabsf(row[d]));
            sa = amax > 0.0f ? 448.0f / amax : 1.0f;
            inv = 1.0f / (sx * sa);
        }
        double y = 0.0;
        for (int d = 0; d < D; ++d) {
            const float dd = x[d] - g[d];
            float aq, dq;
            if (fmt == 2) {
                aq = ora_round_e4m3(row[d] * sa);
                dq = ora_round_e4m3(dd * sx);
            } else {
                aq = ora_round_bf16(row[d]);
                dq = ora_round_bf16(dd);
            }
            y += (double)aq * (double)dq;
        }
        if (fmt == 2) y *= (double)inv;
        const double r = y + (double)off;
        acc += r * r;
    }
    return acc;
}

float ora_fitness_p(const ora_params* p, const float* x)
{
    if (p->fitness == ORA_LSQ) {
        if (p->lsq_fp64) return (float)ora_lsq_f64(p->lsq_A, p->lsq_b, p->lsq_M, p->D, x);
        return ora_lsq_f32(p->lsq_A, p->lsq_b, p->lsq_M, p->D, x);
    }
    return ora_fitness(p->fitness, x, p->D);
}

/* ------------------------------------------------------------------------- */
/* Ordering of fitness values                                                */
/* ------------------------------------------------------------------------- */

uint32_t ora_fit_key(float f)
{
    if (isnan(f)) return 0xFFFFFFFFu;
    if (f == 0.0f) f = 0.0f; /* -0 and +0 are the same fitness */
    uint32_t b;
    memcpy(&b, &f, 4);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

/* a ranks strictly before b: by fitness (NaN last), then by index. */
static int better(float fa, int64_t ia, float fb, int64_t ib)
{
    uint32_t ka = ora_fit_key(fa), kb = ora_fit_key(fb);
    if (ka != kb) return ka < kb;
    return ia < ib;
}

int64_t ora_argmin_pbest(const ora_params* p, const ora_state* s)
{
    int64_t g = 0;
    for (int64_t i = 1; i < p->N; ++i)
        if (better(s->pbest_fit[i], i, s->pbest_fit[g], g)) g = i;
    return g;
}

static void take_gbest(const ora_params* p, ora_state* s, int64_t g)
{
    s->gbest_idx = g;
    s->gbest_fit = s->pbest_fit[g];
    memcpy(s->gbest_pos, s->pbest_pos + (size_t)g * p->D, sizeof(float) * (size_t)p->D);
}

/* ------------------------------------------------------------------------- */
/* Step 1: initialisation                                                    */
/* ------------------------------------------------------------------------- */

/* Closed clamp to [lo, hi] (Alg. 1, "keep in range"). A NaN is clamped to the
 * lower bound, as IEEE-754 maxNum/minNum do (fmin(fmax(a, lo), hi)); written
 * with comparisons so that no platform's handling of fmax(-0, +0) enters. */
static float clampf(float a, float lo, float hi)
{
    if (isnan(a)) return lo;
    return a < lo ? lo : (a > hi ? hi : a);
}

static int check_params(const ora_params* p)
{
    if (p->N <= 0 || p->D <= 0) return -1;
    if (!(p->min_pos < p->max_pos) || !(p->max_v > 0.0f)) return -1;
    if (p->fitness < ORA_SPHERE || p->fitness > ORA_LSQ) return -1;
    if (p->fitness == ORA_LSQ && (!p->lsq_A || !p->lsq_b || p->lsq_M <= 0)) return -1;
    return 0;
}

int ora_init(const ora_params* p, ora_state* s)
{
    if (check_params(p)) return -1;
    const int N = p->N, D = p->D;
    const float span = p->max_pos - p->min_pos;
    const float vspan = 2.0f * p->max_v;
    for (int i = 0; i < N; ++i) {
        float* pos = s->pos + (size_t)i * D;
        float* v = s->v + (size_t)i * D;
        for (int d = 0; d < D; ++d) {
            uint32_t wx, wv;
            draw_words(p, 0u, i, d, &wx, &wv);
            pos[d] = clampf(fmaf(ora_u01(wx), span, p->min_pos), p->min_pos, p->max_pos);
            v[d] = clampf(fmaf(ora_u01(wv), vspan, -p->max_v), -p->max_v, p->max_v);
        }
        s->fit[i] = ora_fitness_p(p, pos);
        s->pbest_fit[i] = s->fit[i];
        memcpy(s->pbest_pos + (size_t)i * D, pos, sizeof(float) * (size_t)D);
    }
    s->t = 0;
    take_gbest(p, s, ora_argmin_pbest(p, s));
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Steps 2-5                                                                 */
/* ------------------------------------------------------------------------- */

float ora_move_one(const ora_params* p, uint32_t t, int i, float* pos, float* v, float* pbest,
                   float* pbest_fit, const float* gbest_pos, const float* r_particle)
{
    const int D = p->D;
    for (int d = 0; d < D; ++d) {
        float r1, r2;
        if (r_particle) {
            r1 = r_particle[2 * d + 0];
            r2 = r_particle[2 * d + 1];
        } else {
            ora_draw_r(p, t, i, d, &r1, &r2);
        }
        /* Eq. 1: v <- w v + c1 r1 (pbest - pos) + c2 r2 (gbest - pos) */
        float cognitive = pbest[d] - pos[d];
        float social = gbest_pos[d] - pos[d];
        float vel = p->w * v[d];
        vel = fmaf(p->c1 * r1, cognitive, vel);
        vel = fmaf(p->c2 * r2, social, vel);
        v[d] = clampf(vel, -p->max_v, p->max_v);
        /* Eq. 2: pos <- pos + v */
        pos[d] = clampf(pos[d] + v[d], p->min_pos, p->max_pos);
    }
    float fit = ora_fitness_p(p, pos);                        /* Step 3 */
    if (fit < *pbest_fit) {                                   /* Step 4 */
        *pbest_fit = fit;
        memcpy(pbest, pos, sizeof(float) * (size_t)D);
    }
    return fit;
}

/* Steps 2-4 for particle i of the swarm at iteration t (gbest_pos is read). */
static void move_particle(const ora_params* p, ora_state* s, uint32_t t, int i,
                          const float* r_iter /* null or [N][D][2] */)
{
    const size_t D = (size_t)p->D;
    s->fit[i] = ora_move_one(p, t, i, s->pos + i * D, s->v + i * D, s->pbest_pos + i * D,
                             &s->pbest_fit[i], s->gbest_pos, r_iter ? r_iter + (size_t)i * D * 2 : NULL);
}

int ora_step_sync(const ora_params* p, ora_state* s, int iters, const float* r_override)
{
    if (check_params(p) || iters < 0) return -1;
    for (int k = 0; k < iters; ++k) {
        uint32_t t = s->t + 1;
        const float* r_iter = r_override ? r_override + (size_t)k * p->N * p->D * 2 : NULL;
        for (int i = 0; i < p->N; ++i) move_particle(p, s, t, i, r_iter);
        take_gbest(p, s, ora_argmin_pbest(p, s));           /* Step 5 */
        s->t = t;
    }
    return 0;
}

/* The same synchronous iterations with Steps 2-4 spread over `threads` host
 * threads (OpenMP): particles are independent within an iteration (each reads
 * only its own state and the gbest of the previous iteration), and Step 5 runs
 * after all of them on one thread, so the result is identical to
 * ora_step_sync's for any thread count. Used only to time the baseline on all
 * host cores. */
int ora_step_sync_threads(const ora_params* p, ora_state* s, int iters, int threads)
{
    if (check_params(p) || iters < 0 || threads < 1) return -1;
    for (int k = 0; k < iters; ++k) {
        uint32_t t = s->t + 1;
#pragma omp parallel for num_threads(threads) schedule(static)
        for (int i = 0; i < p->N; ++i) move_particle(p, s, t, i, NULL);
        take_gbest(p, s, ora_argmin_pbest(p, s));           /* Step 5 */
        s->t = t;
    }
    return 0;
}

int ora_step_serial(const ora_params* p, ora_state* s, int iters, const float* r_override)
{
    if (check_params(p) || iters < 0) return -1;
    for (int k = 0; k < iters; ++k) {
        uint32_t t = s->t + 1;
        const float* r_iter = r_override ? r_override + (size_t)k * p->N * p->D * 2 : NULL;
        for (int i = 0; i < p->N; ++i) {
            move_particle(p, s, t, i, r_iter);
            if (better(s->pbest_fit[i], i, s->gbest_fit, s->gbest_idx)) /* Step 5 in-loop */
                take_gbest(p, s, i);
        }
        s->t = t;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Double precision: the paper's own precision (Sec. 5.1 runs its GPU and    */
/* CPU versions in FP64). The same steps as above, each one binary64         */
/* operation rounded to nearest; fma() is the correctly rounded C99 fma.     */
/* ------------------------------------------------------------------------- */

double ora_u53(uint32_t hi, uint32_t lo)
{
    /* 53 random bits: all of hi, the top 21 of lo; (m + 1) 2^-53 is exact. */
    uint64_t m = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
    return ldexp((double)(m + 1u), -53);
}

static void draw_words_d(const ora_params_d* p, uint32_t t, int i, int d, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)d, (uint32_t)i, t, p->swarm};
    uint32_t key[2] = {(uint32_t)(p->seed & 0xFFFFFFFFu), (uint32_t)(p->seed >> 32)};
    ora_philox4x32_10(ctr, key, out);
}

void ora_draw_r_d(const ora_params_d* p, uint32_t t, int i, int d, double* r1, double* r2)
{
    uint32_t w[4];
    draw_words_d(p, t, i, d, w);
    *r1 = ora_u53(w[0], w[1]);
    *r2 = ora_u53(w[2], w[3]);
}

double ora_fitness_d(int fitness, const double* x, int D)
{
    double acc = 0.0;
    switch (fitness) {
    case ORA_SPHERE:
        for (int d = 0; d < D; ++d) acc = fma(x[d], x[d], acc);
        return acc;
    case ORA_ROSENBROCK:
        for (int d = 0; d + 1 < D; ++d) {
            double p = fma(-x[d], x[d], x[d + 1]);
            double q = 1.0 - x[d];
            acc = acc + fma(100.0 * p, p, q * q);
        }
        return acc;
    case ORA_CUBIC_MAX: /* Eq. 3, maximised: -sum (x^3 - 0.8 x^2 - 1000 x + 8000) */
        for (int d = 0; d < D; ++d) {
            double h = fma(fma(x[d] - 0.8, x[d], -1000.0), x[d], 8000.0);
            acc = acc + h;
        }
        return -acc;
    default:
        return NAN;
    }
}

uint64_t ora_fit_key_d(double f)
{
    if (isnan(f)) return ~(uint64_t)0;
    if (f == 0.0) f = 0.0;
    uint64_t b;
    memcpy(&b, &f, 8);
    return (b >> 63) ? ~b : (b | ((uint64_t)1 << 63));
}

static double clampd(double a, double lo, double hi)
{
    if (isnan(a)) return lo;
    return a < lo ? lo : (a > hi ? hi : a);
}

static int check_params_d(const ora_params_d* p)
{
    if (p->N <= 0 || p->D <= 0) return -1;
    if (!(p->min_pos < p->max_pos) || !(p->max_v > 0.0)) return -1;
    if (p->fitness != ORA_SPHERE && p->fitness != ORA_ROSENBROCK && p->fitness != ORA_CUBIC_MAX) return -1;
    return 0;
}

static int better_d(double fa, int64_t ia, double fb, int64_t ib)
{
    uint64_t ka = ora_fit_key_d(fa), kb = ora_fit_key_d(fb);
    if (ka != kb) return ka < kb;
    return ia < ib;
}

int64_t ora_argmin_pbest_d(const ora_params_d* p, const ora_state_d* s)
{
    int64_t g = 0;
    for (int64_t i = 1; i < p->N; ++i)
        if (better_d(s->pbest_fit[i], i, s->pbest_fit[g], g)) g = i;
    return g;
}

static void take_gbest_d(const ora_params_d* p, ora_state_d* s, int64_t g)
{
    s->gbest_idx = g;
    s->gbest_fit = s->pbest_fit[g];
    memcpy(s->gbest_pos, s->pbest_pos + (size_t)g * p->D, sizeof(double) * (size_t)p->D);
}

int ora_init_d(const ora_params_d* p, ora_state_d* s)
{
    if (check_params_d(p)) return -1;
    const int N = p->N, D = p->D;
    const double span = p->max_pos - p->min_pos;
    const double vspan = 2.0 * p->max_v;
    for (int i = 0; i < N; ++i) {
        double* pos = s->pos + (size_t)i * D;
        double* v = s->v + (size_t)i * D;
        for (int d = 0; d < D; ++d) {
            uint32_t w[4];
            draw_words_d(p, 0u, i, d, w);
            pos[d] = clampd(fma(ora_u53(w[0], w[1]), span, p->min_pos), p->min_pos, p->max_pos);
            v[d] = clampd(fma(ora_u53(w[2], w[3]), vspan, -p->max_v), -p->max_v, p->max_v);
        }
        s->fit[i] = ora_fitness_d(p->fitness, pos, D);
        s->pbest_fit[i] = s->fit[i];
        memcpy(s->pbest_pos + (size_t)i * D, pos, sizeof(double) * (size_t)D);
    }
    s->t = 0;
    take_gbest_d(p, s, ora_argmin_pbest_d(p, s));
    return 0;
}

double ora_move_one_d(const ora_params_d* p, uint32_t t, int i, double* pos, double* v, double* pbest,
                      double* pbest_fit, const double* gbest_pos)
{
    const int D = p->D;
    for (int d = 0; d < D; ++d) {
        double r1, r2;
        ora_draw_r_d(p, t, i, d, &r1, &r2);
        /* Eq. 1 */
        double cognitive = pbest[d] - pos[d];
        double social = gbest_pos[d] - pos[d];
        double vel = p->w * v[d];
        vel = fma(p->c1 * r1, cognitive, vel);
        vel = fma(p->c2 * r2, social, vel);
        v[d] = clampd(vel, -p->max_v, p->max_v);
        /* Eq. 2 */
        pos[d] = clampd(pos[d] + v[d], p->min_pos, p->max_pos);
    }
    double fit = ora_fitness_d(p->fitness, pos, D);  /* Step 3 */
    if (fit < *pbest_fit) {                          /* Step 4 */
        *pbest_fit = fit;
        memcpy(pbest, pos, sizeof(double) * (size_t)D);
    }
    return fit;
}

int ora_step_sync_d(const ora_params_d* p, ora_state_d* s, int iters)
{
    if (check_params_d(p) || iters < 0) return -1;
    const size_t D = (size_t)p->D;
    for (int k = 0; k < iters; ++k) {
        uint32_t t = s->t + 1;
        for (int i = 0; i < p->N; ++i)
            s->fit[i] = ora_move_one_d(p, t, i, s->pos + i * D, s->v + i * D, s->pbest_pos + i * D,
                                       &s->pbest_fit[i], s->gbest_pos);
        take_gbest_d(p, s, ora_argmin_pbest_d(p, s));  /* Step 5 */
        s->t = t;
    }
    return 0;
}
