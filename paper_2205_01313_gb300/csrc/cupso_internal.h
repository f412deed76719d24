// cupso_internal.h -- host-side launch wrappers shared by the C-ABI layer.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cupso.h"
#include "cupso_device.cuh"

namespace cupso {

constexpr int kBlock = 256;             // threads per CTA of the streaming kernels
constexpr int kPerThread = 4;           // particles per thread (one float4)
constexpr int kTile = kBlock * kPerThread;
constexpr int kPad = 128;               // Np = N rounded up to a multiple of this

__host__ __device__ inline int tiles_of(int Np) { return (Np + kTile - 1) / kTile; }

// All wrappers return a cudaError_t of the launch.
cudaError_t launch_init(const SwarmDev& s, int fid, int grid, cudaStream_t st);
cudaError_t launch_sync_step(const SwarmDev& s, int fid, int grid, cudaStream_t st);
cudaError_t launch_tree_step(const SwarmDev& s, int fid, bool unrolled, cudaStream_t st);
// ASYNC: `block` threads per CTA (a multiple of 32, <= kBlock), each CTA a
// tile of 4 * block particles per pass.
cudaError_t launch_async(const SwarmDev& s, int fid, int grid, int block, uint32_t t_first, int iters,
                         int hold_lock, cudaStream_t st);
cudaError_t launch_recompute(const SwarmDev& s, uint32_t t, cudaStream_t st);

// Pipelined fused step (kernels_pipelined.cu): `stages`-deep cp.async ring.
bool pipelined_supported(int stages, int D);
cudaError_t prepare_pipelined(int D);   // raise the dynamic shared-memory limit; call outside capture
// ppt: particles per thread (4, 2 or 1); a warp takes units of 32 * ppt particles.
int pipelined_blocks_per_sm(int stages, int fid, int D, int ppt);
cudaError_t launch_sync_pipelined(const SwarmDev& s, int fid, int stages, int ppt, int grid, cudaStream_t st);
// Write back the pbest rows the pipelined step left pending (lazy pbest) and clear the flags.
cudaError_t launch_materialize(const SwarmDev& s, int grid, cudaStream_t st);

// Batched step (kernels_batch.cu): one iteration of every swarm of a batch.
cudaError_t prepare_batch();
// Shapes: (stages, minb) in {(3, 2), (3, 3), (4, 2)}; minb = CTAs per SM the
// register budget is sized for.
int batch_blocks_per_sm(int stages, int minb);
cudaError_t launch_batch_step(const BatchDev& b, int stages, int minb, int grid, cudaStream_t st);
// Step 1 (t = 0) of every swarm of a batch in one launch, over the same units;
// per swarm the same bits as launch_init. Needs gkey = all ones, done and
// pflag zero.
cudaError_t launch_batch_init(const BatchDev& b, int grid, cudaStream_t st);

// Fused SYNC step on the panel layout (kernels_panel.cu): element (d, i) of
// x, v, pb at ((d / W) * Np + i) * W + d % W, panel width W = 8 or 16, ring
// depth 3 or 5 panels.
bool panel_supported(int width, int stages, int D);
cudaError_t prepare_panel(int D);
int panel_blocks_per_sm(int width, int stages, int fid, int D);
// Iterations of one panel launch; more than one is a cooperative launch with a
// grid barrier per iteration (every CTA resident; see kernels_panel.cu).
constexpr int kPanelMaxIters = 4096;
cudaError_t launch_sync_panel(const SwarmDev& s, int fid, int width, int stages, int grid, int iters,
                              bool stall_barrier, cudaStream_t st);
cudaError_t launch_materialize_panel(const SwarmDev& s, int width, int grid, cudaStream_t st);
// dst = src in the other layout (dimension-major <-> panel of width W); D % W == 0.
cudaError_t launch_relayout(const float* src, float* dst, int D, int Np, int width, bool to_panel, int grid,
                            cudaStream_t st);

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

// Resident CTAs per SM of the persistent kernels (for grid sizing).
int sync_blocks_per_sm(int fid, int D);
int async_blocks_per_sm(int fid, int D);

// Record an error message for cupso_last_error() on the calling thread.
void set_last_error(const char* msg);
void set_cuda_error(cudaError_t e, const char* where);

// Host-side argument check of one problem (CUPSO_OK or CUPSO_ERR_INVALID_ARG).
int check_problem_args(int D, int N, const cupso_bounds* b, float w, float c1, float c2, int fid);
// Solve one problem through its own handle (create, iters steps, gbest, destroy).
int solve_one_plain(const cupso_problem& p, int iters, cupso_result& r, cudaStream_t stream);

// On-chip variant: whole swarm in the shared memory of one thread-block
// cluster, many iterations per launch.
bool onchip_fits(int N, int D, int* cluster_out, int* per_cta_out);
cudaError_t launch_onchip(const SwarmDev& s, int fid, int iters, cudaStream_t st);

}  // namespace cupso
