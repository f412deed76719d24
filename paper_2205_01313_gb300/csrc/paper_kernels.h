// paper_kernels.h -- host interface of kernels_paper.cu: the paper's own
// kernel designs (one particle per thread; the reduction of Sec. 2.2, the
// shared-memory queue of Alg. 2 and the queue with a global lock of Alg. 3)
// and the double-precision swarm that runs the paper's workload in its own
// precision (Sec. 5.1: FP64 throughout).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "cupso_device.cuh"

namespace cupso {

// A global-best candidate: order-preserving key of its fitness (FP32 keys
// zero-extended, FP64 keys full width; NaN ranks last) and its index.
// Lexicographic order, so ties go to the lowest index.
struct PKey {
    unsigned long long k;
    uint32_t i;
    uint32_t pad;
};

constexpr uint32_t kNoIdx = 0xFFFFFFFFu;

// Working storage of the one-particle-per-thread kernels (both precisions).
struct PaperBufs {
    PKey* aux;             // [blocks]   best of each block (Sec. 2.2, Alg. 2)
    PKey* list;            // [list_cap] candidates of the fused FP64 steps (one per block at most)
    unsigned int* lock;    // Alg. 3 global lock
    unsigned int* ticket;  // last-block counter of the one-kernel variants
    unsigned int* list_n;  // entries in `list`
    unsigned int list_cap; // capacity of `list`: no launch may have more blocks
    unsigned int* bar_count;  // grid barrier of the persistent kernel: arrivals
    unsigned int* bar_gen;    // and generation
};

// Device state of a double-precision swarm. Same layouts as SwarmDev:
// [D][Np] dimension-major state, gbest double-buffered by iteration parity.
struct SwarmDev64 {
    double* x;            // [D][Np]
    double* v;            // [D][Np]
    double* pb;           // [D][Np]
    double* pf;           // [Np]
    double* G;            // [2][D]
    PKey* gkey;           // [2]
    unsigned int* t_dev;  // iterations completed
    unsigned int* status; // sticky kStatus* bits
    int N, D, Np;
    double lo, hi, vmax, w, c1, c2;
    uint32_t key0, key1, swarm;
    long long wait_limit_ns;
    // Exact shortcuts (each gives the bits of the plain operation):
    int w_one;                   // w == 1: w v is v
    int c1_exp, c2_exp;          // c == 2^k: c r is r with k added to its exponent; else kNoExp
    long long k_lo, k_hi;        // order keys of min_pos, max_pos (clamps as integer compares)
    long long k_vlo, k_vhi;      // order keys of -max_v, max_v
};

constexpr int kNoExp = 0x7FFF;

// IEEE-754 order of a binary64 value as a signed integer (-0 and +0 equal);
// meaningful for non-NaN values.
__host__ __device__ inline long long order_key64(double a) {
    long long b;
    static_assert(sizeof(b) == sizeof(a), "binary64");
    __builtin_memcpy(&b, &a, 8);
    return b >= 0 ? b : -(b & 0x7FFFFFFFFFFFFFFFll);
}

constexpr int kPaperBlock = 256;   // threads (= particles) per block

enum PaperAgg : int {
    kAggReduce = 0,          // block tree reduction + second kernel (Sec. 2.2, Fig. 1)
    kAggReduceUnrolled = 1,  // the same with the unrolled reduction (Sec. 2.2)
    kAggQueue = 2,           // shared-memory queue + second kernel (Alg. 2)
    kAggQueueLock = 3,       // shared-memory queue + global lock, one kernel (Alg. 3)
    kAggSyncList = 4         // FP64 fused step: block argmin, candidate list, last block gathers
};

inline int paper_blocks(int n) { return (n + kPaperBlock - 1) / kPaperBlock; }

// Bytes of PaperBufs storage for a swarm of Np particles whose candidate list
// holds list_cap entries (256-byte aligned parts).
size_t paper_bufs_bytes(int Np, int list_cap);
// Carves PaperBufs out of `base` (paper_bufs_bytes(Np, list_cap) bytes, zeroed by the caller).
PaperBufs paper_bufs_at(void* base, int Np, int list_cap);

// FP32 swarm: one iteration of Alg. 2 (two kernels) or Alg. 3 (one kernel).
cudaError_t launch_queue_step(const SwarmDev& s, const PaperBufs& b, int fid, bool lock, cudaStream_t st);

// FP64 swarm (fitness: sphere, Rosenbrock, cubic).
bool fp64_fitness_supported(int fid);
cudaError_t launch_init64(const SwarmDev64& s, const PaperBufs& b, int fid, cudaStream_t st);
// SYNC (kAggSyncList) with D >= 16 runs the tiled kernel, which spreads a
// particle's dimensions over threads; num_sms sizes its tiles.
cudaError_t launch_step64(const SwarmDev64& s, const PaperBufs& b, int fid, int agg, int num_sms, cudaStream_t st);
cudaError_t launch_recompute64(const SwarmDev64& s, const PaperBufs& b, cudaStream_t st);
// Persistent FP64 swarm: one cooperative launch runs `iters` synchronous
// iterations, one particle per thread (looping when N exceeds the resident
// threads), with a bounded grid barrier per iteration in place of the kernel
// boundary.
cudaError_t launch_persist64(const SwarmDev64& s, const PaperBufs& b, int fid, int iters, int num_sms,
                             cudaStream_t st);
int persist64_grid(int fid, int N, int D, int num_sms);

// On-chip FP64 swarm: the whole swarm in the shared memory of one CTA cluster
// (1 to 16 CTAs, chosen from (N, D) by onchip64_cluster), `iters` iterations
// per launch. onchip64_fits says whether (N, D) fits at all.
bool onchip64_fits(int N, int D);
int onchip64_cluster(int N, int D);
cudaError_t launch_onchip64(const SwarmDev64& s, int fid, int iters, cudaStream_t st);

}  // namespace cupso
