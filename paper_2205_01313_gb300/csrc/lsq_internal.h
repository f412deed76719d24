// lsq_internal.h -- host-side interfaces of the least-squares fitness: the
// tensor-core product (kernels_lsq.cu, cupso_lsq.cu) and the least-squares
// swarm iteration (kernels_lsq_swarm.cu), used by the C-ABI layer.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "cupso_internal.h"

namespace cupso {

// Least-squares fitness (kernels_lsq.cu).
struct LsqTcPlan {
    alignas(64) unsigned char tmX[128];   // CUtensorMap of the position operand [Np][Kp]
    alignas(64) unsigned char tmA[128];   // CUtensorMap of A [Mp][Kp]
    bool fp8;
    int Np, Mp, Kp;                       // Np % 128 == 0, Mp % 256 == 0, Kp * elem % 128 == 0
    int num_sms;                          // grid of the persistent product kernel
};
bool lsq_tc_available();
cudaError_t lsq_prepare();
// dst[i][k] = round(src[i * si + k * sk] * (fp8 ? scale : 1)), zero-padded to [Np][Kp].
cudaError_t lsq_convert(const float* src, size_t si, size_t sk, int N, int D, int Np, int Kp, bool fp8, float scale,
                        void* dst, cudaStream_t st);
bool lsq_tc_plan(LsqTcPlan* p, void* Xq, void* Aq, bool fp8, int Np, int Mp, int Kp);
// The three tensor maps of the TMA-fed move over arrays [D][Np] of FP32 (Np a
// multiple of 64): boxes of 64 particles x 64 dimensions, zeros past D.
bool lsq_make_move_maps(unsigned char (*maps)[128], const float* x, const float* v, const float* pb, int Np, int D);
// part[k][i] (k < lsq_tc_partials) = sum of squared residuals y + off[m] of
// particle i over residual rows 128 k .. 128 k + 127 (off = -b: the positions'
// residuals; off = A c - b: residuals of displacements from c).
cudaError_t lsq_tc_launch(const LsqTcPlan& p, const float* off, const float* inv_scale, float* part,
                          unsigned int* status, long long limit_ns, cudaStream_t st);
int lsq_tc_partials(const LsqTcPlan& p);
// Tensor-core fitness state for fixed (A, b): operand copies, scales, plan.
struct LsqTcState {
    void* arena = nullptr;
    bool fp8 = false;
    int M = 0, D = 0, Np = 0, Mp = 0, Kp = 0;
    float sx = 1.0f;                 // FP8 scale of the positions
    void* Aq = nullptr;              // [Mp][Kp] operand copy of A
    void* Xq = nullptr;              // [Np][Kp] operand copy of the positions
    float* negb = nullptr;           // [Mp] -b, zero past M: the offsets of the positions' residuals
    float* roff = nullptr;           // [Mp] A c - b for the swarm's reference point c (gbest), zero past M
    int* roff_stale = nullptr;       // nonzero: roff must be recomputed (the reference point moved)
    float* inv = nullptr;            // [Mp] 1 / (sx * row scale of A) (FP8)
    float* part = nullptr;           // [Mp / 128][Np] partial sums
    unsigned int* status = nullptr;
    LsqTcPlan plan;
    // CUtensorMaps of the swarm's pos, v and pbest_pos ([D][Np] FP32, boxes of
    // 64 particles x 64 dimensions) for the TMA-fed move (lsq_make_move_maps)
    alignas(64) unsigned char tmMove[3][128];
};
int lsq_setup_tc(LsqTcState* st, const float* A, const float* b, int M, int D, int Np, bool fp8, float sx,
                 cudaStream_t stream);
void lsq_free_tc(LsqTcState* st);
// f[i] for positions X(i, k) = src[i * si + k * sk], i < N (asynchronous).
int lsq_eval_tc(LsqTcState* st, const float* src, size_t si, size_t sk, int N, float* f, cudaStream_t stream);
// f[i], i < N, for the operand already in st->Xq (asynchronous).
int lsq_eval_tc_operand(LsqTcState* st, int N, float* f, cudaStream_t stream);
// The same product for the displacement operand of the swarm (offsets
// st->roff), leaving f[i] as lsq_tc_partials(st->plan) partial sums
// st->part[k][i] (f[i] = their sum in k order).
int lsq_eval_tc_partials(LsqTcState* st, cudaStream_t stream);

// f[i] = plain FP32 fitness of X(i, d) = x[d * ldx + i], i < N.
cudaError_t lsq_fp32_launch(const float* x, int ldx, int N, int D, const float* A, const float* b, int M, float* f,
                            cudaStream_t st);
// f[i] = FP64 fitness of the same positions in the reference order, rounded to float.
cudaError_t lsq_fp64_launch(const float* x, int ldx, int N, int D, const float* A, const float* b, int M, float* f,
                            cudaStream_t st);

// Least-squares swarm iteration (kernels_lsq_swarm.cu); all read t from t_dev.
cudaError_t lsq_launch_move(const SwarmDev& s, int grid, cudaStream_t st);
// The same moves, writing the new positions also as the tensor-core operand
// Xq ([Np][Kp], BF16, or FP8 e4m3 of x * sx), zero for i >= N and k >= D.
// Tiles of pos, v, pbest_pos arrive by TMA through the maps of
// lsq_make_move_maps (maps: 3 x 128 bytes). Requires Np and Kp multiples of
// 64 and Kp >= D.
cudaError_t lsq_launch_move_q(const SwarmDev& s, const unsigned char (*maps)[128], void* Xq, int Kp, bool fp8,
                              float sx, int num_sms, cudaStream_t st);
cudaError_t lsq_launch_select_exact(const SwarmDev& s, const float* fit, unsigned int* flags, int grid,
                                    cudaStream_t st);
// Candidate lists of the selection (one of 16 keys per warp of 32 particles):
// the candidate buffer holds lists x 16 keys, the merged 16 and a ticket.
int lsq_cand_lists(int Np);
// Gram data of the rescoring (Gm = A^T A, cvec = A^T b, bb = b^T b, all FP64);
// Gm null: direct form. Gff: Gm as pairs (hi, lo) of binary32 values, ldf x ldf
// with ldf = D rounded up to kFfTile and zeros outside D x D, for the
// float-float rescoring (ff true); ff false rescores with FP64 arithmetic, whose
// kernel keeps 4 candidates x D doubles in shared memory per block.
constexpr int kGramMaxD = 6144;
constexpr int kFfTile = 64;
struct LsqGram {
    double* Gm = nullptr;
    double* cvec = nullptr;
    double bb = 0.0;
    float2* Gff = nullptr;
    int ldf = 0;
    bool ff = true;
};
// Tiles of the float-float rescoring (the upper triangle of Gm in kFfTile
// squares): four blocks each (4 candidates apiece), one partial sum per
// candidate and tile.
inline int lsq_ff_tiles(int D) {
    const int nt = (D + kFfTile - 1) / kFfTile;
    return nt * (nt + 1) / 2;
}
// Gm, cvec and Gff (ldf = D rounded up to kFfTile, zero-filled here) from A
// and b; raises the FP64 rescoring kernel's shared-memory limit for D
// (D <= kGramMaxD).
cudaError_t lsq_launch_gram(const float* A, const float* b, int M, int D, double* Gm, double* cvec, float2* Gff,
                            int ldf, cudaStream_t st);
// Steps 4-5 with an approximate fitness. lazy: flags is s.pflag and the
// improved particles' pbest_pos rows are left to the next move (and to the
// materialize kernel); otherwise they are copied here.
// fit: the approximate fitness, or null with part/nparts: its partial sums
// part[k][i] (Np apart), added in k order.
// When it accepts a new gbest it sets stale[0]; with `off` set it then
// recomputes the residual offsets of the new reference point (off[m] = A g - b,
// compensated) for the next iteration's product. stale: two ints (flag and the
// offset kernel's block counter), zero-initialised.
cudaError_t lsq_launch_gbest_approx(const SwarmDev& s, const float* fit, const float* part, int nparts, int all,
                                    bool lazy, const float* A, const float* b, int M, unsigned long long* cand,
                                    double* partial, int chunks, double* g64, unsigned int* flags, int grid,
                                    const LsqGram& gram, float* off, int* stale, int num_sms, cudaStream_t st);
// off[m] = A g - b for the current gbest_pos g (slot t & 1), if stale[0] is set.
cudaError_t lsq_launch_offsets(const SwarmDev& s, const float* A, const float* b, int M, float* off, int* stale,
                               int num_sms, cudaStream_t st);
cudaError_t lsq_launch_set_pf(const SwarmDev& s, const float* fit, cudaStream_t st);
// FP64 fitness of the pbest_pos of the particle in `key`, into *g64; waits.
cudaError_t lsq_rescore_one(const SwarmDev& s, const float* A, const float* b, int M, unsigned long long key,
                            unsigned long long* scratch, double* partial, int chunks, double* g64, cudaStream_t st);
cudaError_t lsq_launch_set_t(const SwarmDev& s, uint32_t t, cudaStream_t st);

}  // namespace cupso
