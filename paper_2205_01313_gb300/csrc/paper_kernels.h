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
    PKey* aux;             // [blocks]  best of each block (Sec. 2.2, Alg. 2)
    PKey* list;            // [blocks]  candidates of the fused FP64 step
    unsigned int* lock;    // Alg. 3 global lock
    unsigned int* ticket;  // last-block counter of the one-kernel variants
    unsigned int* list_n;  // entries in `list`
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
};

constexpr int kPaperBlock = 256;   // threads (= particles) per block

enum PaperAgg : int {
    kAggReduce = 0,          // block tree reduction + second kernel (Sec. 2.2, Fig. 1)
    kAggReduceUnrolled = 1,  // the same with the unrolled reduction (Sec. 2.2)
    kAggQueue = 2,           // shared-memory queue + second kernel (Alg. 2)
    kAggQueueLock = 3,       // shared-memory queue + global lock, one kernel (Alg. 3)
    kAggSyncList = 4         // FP64 fused step: block argmin, candidate list, last block gathers
};

inline int paper_blocks(int n) { return (n + kPaperBlock - 1) / kPaperBlock; }

// Bytes of PaperBufs storage for a swarm of Np particles (256-byte aligned parts).
size_t paper_bufs_bytes(int Np);
// Carves PaperBufs out of `base` (paper_bufs_bytes(Np) bytes, zeroed by the caller).
PaperBufs paper_bufs_at(void* base, int Np);

// FP32 swarm: one iteration of Alg. 2 (two kernels) or Alg. 3 (one kernel).
cudaError_t launch_queue_step(const SwarmDev& s, const PaperBufs& b, int fid, bool lock, cudaStream_t st);

// FP64 swarm (fitness: sphere, Rosenbrock, cubic).
bool fp64_fitness_supported(int fid);
cudaError_t launch_init64(const SwarmDev64& s, const PaperBufs& b, int fid, cudaStream_t st);
cudaError_t launch_step64(const SwarmDev64& s, const PaperBufs& b, int fid, int agg, cudaStream_t st);
cudaError_t launch_recompute64(const SwarmDev64& s, const PaperBufs& b, cudaStream_t st);
// On-chip FP64 swarm: the whole swarm in one CTA's shared memory, `iters`
// iterations per launch. onchip64_fits says whether (N, D) fits.
bool onchip64_fits(int N, int D);
cudaError_t prepare_onchip64();
cudaError_t launch_onchip64(const SwarmDev64& s, int fid, int iters, cudaStream_t st);

}  // namespace cupso
