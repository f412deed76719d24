// cupso_lsq.cu -- host side of the least-squares fitness.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/cupso.h"
#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "lsq_internal.h"

using namespace cupso;

namespace {

size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// A in the tensor-core operand format ([Mp][Kp], zero rows and columns past
// M, D), per-row FP8 scales folded into inv_scale (m) = 1 / (sx * sa_m).
__global__ void row_absmax_kernel(const float* __restrict__ A, int M, int D, float* __restrict__ amax) {
    const int m = blockIdx.x;
    float v = 0.0f;
    for (int d = threadIdx.x; d < D; d += blockDim.x) v = fmaxf(v, fabsf(A[(size_t)m * D + d]));
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float w = 0.0f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) w = fmaxf(w, red[k]);
        amax[m] = w;
    }
}

// Scale each row of A in place into a scratch copy: As[m][d] = A[m][d] * sa_m,
// with sa_m = 448 / amax_m (1 for an all-zero row); inv[m] = 1 / (sx * sa_m).
__global__ void scale_rows_kernel(const float* __restrict__ A, int M, int D, const float* __restrict__ amax, float sx,
                                  float* __restrict__ As, float* __restrict__ inv, int Mp) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)M * D; e += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / D);
        const float sa = amax[m] > 0.0f ? 448.0f / amax[m] : 1.0f;
        As[e] = A[e] * sa;
    }
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < Mp; m += gridDim.x * blockDim.x) {
        if (m < M) {
            const float sa = amax[m] > 0.0f ? 448.0f / amax[m] : 1.0f;
            inv[m] = 1.0f / (sx * sa);
        } else {
            inv[m] = 0.0f;
        }
    }
}

// negb[m] = -b[m] for m < M, 0 up to Mp (negation is exact, so y + negb[m]
// rounds exactly as y - b[m]); roff starts as the same offsets (reference
// point 0) until the swarm sets its own.
__global__ void neg_pad_kernel(const float* __restrict__ b, int M, int Mp, float* __restrict__ negb,
                               float* __restrict__ roff) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < Mp; m += gridDim.x * blockDim.x) {
        const float v = m < M ? -b[m] : 0.0f;
        negb[m] = v;
        roff[m] = v;
    }
}

// out[d][i] = in[i][d] for an N x D row-major matrix.
__global__ void transpose_kernel(const float* __restrict__ in, int N, int D, float* __restrict__ out) {
    __shared__ float t[32][33];
    const int d0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int i = i0 + k, d = d0 + threadIdx.x;
        if (i < N && d < D) t[k][threadIdx.x] = in[(size_t)i * D + d];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int d = d0 + k, i = i0 + threadIdx.x;
        if (i < N && d < D) out[(size_t)d * N + i] = t[threadIdx.x][k];
    }
}

__global__ void sum_parts_kernel(const float* __restrict__ part, int nparts, int Np, int N, float* __restrict__ f) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < nparts; ++k) s = __fadd_rn(s, part[(size_t)k * Np + i]);
        f[i] = s;
    }
}

}  // namespace

// Everything the tensor-core fitness needs for fixed A, b: operand copies,
// scales, padded b, and the TMA descriptors (built for a given X buffer).
int cupso::lsq_setup_tc(LsqTcState* st, const float* A, const float* b, int M, int D, int Np, bool fp8, float sx,
                        cudaStream_t stream) {
    st->fp8 = fp8;
    st->M = M;
    st->D = D;
    st->Np = Np;
    st->Mp = (int)up((size_t)M, 256);
    st->Kp = (int)up((size_t)D, fp8 ? 128 : 64);
    st->sx = fp8 ? sx : 1.0f;
    const size_t esz = fp8 ? 1 : 2;
    const size_t bytes_A = (size_t)st->Mp * st->Kp * esz, bytes_X = (size_t)Np * st->Kp * esz;
    const size_t nparts = (size_t)st->Mp / 128;   // one partial sum per 128 residual rows
    const size_t bytes = up(bytes_A, 256) + up(bytes_X, 256) + up(sizeof(float) * st->Mp, 256) * 3 +
                         up(sizeof(float) * nparts * Np, 256) + up(sizeof(float) * (size_t)M * D, 256) +
                         up(sizeof(float) * M, 256) + 512;
    cudaError_t e = cudaMalloc(&st->arena, bytes);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaMalloc (lsq)"), e == cudaErrorMemoryAllocation ? CUPSO_ERR_OOM : CUPSO_ERR_CUDA;
    char* p = static_cast<char*>(st->arena);
    st->Aq = p; p += up(bytes_A, 256);
    st->Xq = p; p += up(bytes_X, 256);
    st->negb = reinterpret_cast<float*>(p); p += up(sizeof(float) * st->Mp, 256);
    st->roff = reinterpret_cast<float*>(p); p += up(sizeof(float) * st->Mp, 256);
    st->inv = reinterpret_cast<float*>(p); p += up(sizeof(float) * st->Mp, 256);
    st->part = reinterpret_cast<float*>(p); p += up(sizeof(float) * nparts * Np, 256);
    float* Ascaled = reinterpret_cast<float*>(p); p += up(sizeof(float) * (size_t)M * D, 256);
    float* amax = reinterpret_cast<float*>(p); p += up(sizeof(float) * M, 256);
    st->status = reinterpret_cast<unsigned int*>(p); p += 256;
    st->roff_stale = reinterpret_cast<int*>(p);
    e = cudaMemsetAsync(st->status, 0, 512, stream);
    if (e == cudaSuccess) e = lsq_prepare();
    if (e != cudaSuccess) return set_cuda_error(e, "lsq setup"), CUPSO_ERR_CUDA;
    neg_pad_kernel<<<(st->Mp + 255) / 256, 256, 0, stream>>>(b, M, st->Mp, st->negb, st->roff);
    const float* Asrc = A;
    if (fp8) {
        row_absmax_kernel<<<M, 256, 0, stream>>>(A, M, D, amax);
        scale_rows_kernel<<<1024, 256, 0, stream>>>(A, M, D, amax, st->sx, Ascaled, st->inv, st->Mp);
        Asrc = Ascaled;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = lsq_convert(Asrc, (size_t)D, 1, M, D, st->Mp, st->Kp, fp8, 1.0f, st->Aq, stream);
    if (e != cudaSuccess) return set_cuda_error(e, "lsq operand A"), CUPSO_ERR_CUDA;
    if (!lsq_tc_plan(&st->plan, st->Xq, st->Aq, fp8, Np, st->Mp, st->Kp)) {
        set_last_error("cuTensorMapEncodeTiled unavailable or rejected the operand layout");
        return CUPSO_ERR_UNSUPPORTED;
    }
    return CUPSO_OK;
}

void cupso::lsq_free_tc(LsqTcState* st) {
    if (st->arena) cudaFree(st->arena);
    st->arena = nullptr;
}

// f[i] for the positions X(i, k) = src[i * si + k * sk], i < N.
int cupso::lsq_eval_tc(LsqTcState* st, const float* src, size_t si, size_t sk, int N, float* f, cudaStream_t stream) {
    cudaError_t e = lsq_convert(src, si, sk, N, st->D, st->Np, st->Kp, st->fp8, st->sx, st->Xq, stream);
    if (e != cudaSuccess) return set_cuda_error(e, "lsq operand conversion"), CUPSO_ERR_CUDA;
    return lsq_eval_tc_operand(st, N, f, stream);
}

int cupso::lsq_eval_tc_partials(LsqTcState* st, cudaStream_t stream) {
    cudaError_t e = lsq_tc_launch(st->plan, st->roff, st->fp8 ? st->inv : nullptr, st->part, st->status,
                                  2000000000ll, stream);
    if (e != cudaSuccess) return set_cuda_error(e, "lsq tensor-core launch"), CUPSO_ERR_CUDA;
    return CUPSO_OK;
}

int cupso::lsq_eval_tc_operand(LsqTcState* st, int N, float* f, cudaStream_t stream) {
    cudaError_t e = lsq_tc_launch(st->plan, st->negb, st->fp8 ? st->inv : nullptr, st->part, st->status,
                                  2000000000ll, stream);
    const int used = lsq_tc_partials(st->plan);
    if (e == cudaSuccess) {
        sum_parts_kernel<<<std::max(1, std::min(1024, (N + 255) / 256)), 256, 0, stream>>>(st->part, used, st->Np, N, f);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_cuda_error(e, "lsq tensor-core launch"), CUPSO_ERR_CUDA;
    return CUPSO_OK;
}

extern "C" int cupso_lsq_eval(const float* A_dev, const float* b_dev, int M, int D, const float* X_dev, int N,
                              int precision, float* f_out_dev, void* cuda_stream) {
    if (!A_dev || !b_dev || !X_dev || !f_out_dev || M < 1 || D < 1 || N < 1 ||
        precision < CUPSO_LSQ_FP32 || precision > CUPSO_LSQ_FP64) {
        set_last_error("cupso_lsq_eval: invalid argument");
        return CUPSO_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == CUPSO_LSQ_FP32 || precision == CUPSO_LSQ_FP64) {
        // the FP32 and FP64 kernels read X(i, d) = x[d * ldx + i]: transpose into a temporary
        float* xd = nullptr;
        cudaError_t e = cudaMalloc(&xd, sizeof(float) * (size_t)N * D);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaMalloc"), CUPSO_ERR_OOM;
        transpose_kernel<<<dim3((D + 31) / 32, (N + 31) / 32), dim3(32, 8), 0, st>>>(X_dev, N, D, xd);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = precision == CUPSO_LSQ_FP32 ? lsq_fp32_launch(xd, N, N, D, A_dev, b_dev, M, f_out_dev, st)
                                            : lsq_fp64_launch(xd, N, N, D, A_dev, b_dev, M, f_out_dev, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(xd);
        if (e != cudaSuccess) return set_cuda_error(e, "lsq fp32/fp64"), CUPSO_ERR_CUDA;
        return CUPSO_OK;
    }
    if (!lsq_tc_available()) {
        set_last_error("tensor-core least squares needs cuTensorMapEncodeTiled from the driver");
        return CUPSO_ERR_UNSUPPORTED;
    }
    LsqTcState s{};
    const int Np = (N + 127) / 128 * 128;
    const bool fp8 = precision == CUPSO_LSQ_FP8;
    float xmax = 0.0f;
    {
        // FP8 scale of X from its largest magnitude
        std::vector<float> h((size_t)N * D);
        cudaError_t e = cudaMemcpyAsync(h.data(), X_dev, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaMemcpy"), CUPSO_ERR_CUDA;
        for (float v : h) xmax = std::max(xmax, std::fabs(v));
    }
    const float sx = xmax > 0.0f ? 448.0f / xmax : 1.0f;
    int rc = lsq_setup_tc(&s, A_dev, b_dev, M, D, Np, fp8, sx, st);
    if (rc == CUPSO_OK) rc = lsq_eval_tc(&s, X_dev, (size_t)D, 1, N, f_out_dev, st);
    cudaError_t e = cudaStreamSynchronize(st);
    unsigned int status = 0;
    if (e == cudaSuccess && s.status) e = cudaMemcpy(&status, s.status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    lsq_free_tc(&s);
    if (rc != CUPSO_OK) return rc;
    if (e != cudaSuccess) return set_cuda_error(e, "lsq eval"), CUPSO_ERR_CUDA;
    if (status & kStatusTimeout) return CUPSO_ERR_DEVICE_TIMEOUT;
    return CUPSO_OK;
}
