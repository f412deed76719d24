// async_common.cuh -- the lock-protected global-best record of the
// asynchronous kernels (Sec. 3.2, Alg. 3 taken to its asynchronous end): a
// CTA reads the record under a sequence lock and publishes an improvement by
// claiming it with atomicMin, then writing it while holding the lock. Every
// wait is bounded by s.wait_limit_ns.
#pragma once

#include <cuda_runtime.h>

#include "cupso_device.cuh"

namespace cupso {
namespace {

// Consistent snapshot of (Grec, reckey) into shared memory (sequence lock:
// the writer makes seq odd while it writes). Returns false on timeout.
__device__ bool read_record(const SwarmDev& s, float* Gs) {
    __shared__ unsigned s_seq;
    __shared__ int s_state;  // 0 retry, 1 ok, 2 timeout
    const long long deadline = global_ns() + s.wait_limit_ns;
    for (;;) {
        if (threadIdx.x == 0) {
            unsigned q = *(volatile unsigned*)s.seq;
            int state = 0;
            while (q & 1u) {
                if (global_ns() > deadline) { state = 2; break; }
                __nanosleep(64);
                q = *(volatile unsigned*)s.seq;
            }
            __threadfence();
            s_seq = q;
            s_state = state;
        }
        __syncthreads();
        if (s_state == 2) return false;
        for (int d = threadIdx.x; d < s.D; d += blockDim.x) Gs[d] = __ldcg(s.Grec + d);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned q2 = *(volatile unsigned*)s.seq;
            s_state = (q2 == s_seq) ? 1 : (global_ns() > deadline ? 2 : 0);
        }
        __syncthreads();
        const int st = s_state;
        __syncthreads();
        if (st == 1) return true;
        if (st == 2) return false;
    }
}

// Publish a CTA's best (Alg. 3): claim with atomicMin, then, holding the lock,
// write the record if the claim is still the lowest. Run by warp 0 only.
__device__ bool publish(const SwarmDev& s, unsigned long long best) {
    const int lane_id = threadIdx.x & 31;
    int ok = 1, won = 0;
    if (lane_id == 0) {
        const unsigned long long old = atomicMin(s.claim, best);
        won = old > best;
        if (won) {
            const long long deadline = global_ns() + s.wait_limit_ns;
            while (atomicCAS(s.lock, 0u, 1u) != 0u) {
                if (global_ns() > deadline) { ok = 0; break; }
                __nanosleep(64);
            }
            __threadfence();
            if (ok) won = (__ldcg(s.claim) == best);
            else won = 0;
            if (won) {
                atomicAdd(s.seq, 1u);  // odd: record being written
                __threadfence();
            } else if (ok) {
                atomicExch(s.lock, 0u);
            }
        }
    }
    won = __shfl_sync(0xFFFFFFFFu, won, 0);
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
    if (won) {
        const uint32_t g = (uint32_t)(best & 0xFFFFFFFFull);
        for (int d = lane_id; d < s.D; d += 32) __stcg(s.Grec + d, __ldcg(s.pb + (size_t)d * s.Np + g));
        __syncwarp();
        if (lane_id == 0) {
            *s.reckey = best;
            __threadfence();
            atomicAdd(s.seq, 1u);  // even: record stable
            atomicExch(s.lock, 0u);
        }
    }
    return ok != 0;
}

}  // namespace
}  // namespace cupso
