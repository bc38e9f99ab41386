// peaks.cu -- issue-rate probes of the instruction classes the matching kernels are built
// from, the denominators of their rooflines (measurement support; the paper has no
// counterpart).  Each probe runs `iters` iterations of a loop body of PROBE_CHAINS
// independent dependency chains x PROBE_UNROLL instructions of one class per thread, on
// `blocks` CTAs of PROBE_THREADS threads, and reports the elapsed time (CUDA events on the
// caller's stream) and the lane operations executed.  Operands come from kernel arguments
// and every chain's result is stored, so nothing folds away; the loop's own counter and
// branch add about 2 % instructions.  Nothing here changes clocks or any device setting:
// the caller samples the SM clock beside the run.
#include <cuda_runtime.h>
#include <stdint.h>

#include "msbm.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 16;

struct ProbeArgs {
    uint32_t a, b, c;        // runtime operands
    float fa, fb;
    int iters;
    uint32_t *sink;          // one word per thread
};

__global__ void __launch_bounds__(PROBE_THREADS) probe_dp4a(const ProbeArgs p) {
    uint32_t acc[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) acc[k] = threadIdx.x + k;
    for (int it = 0; it < p.iters; ++it) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) acc[k] = __dp4a(p.a, p.b + k, acc[k]);
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s ^= acc[k];
    p.sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) probe_shf(const ProbeArgs p) {
    uint32_t x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = threadIdx.x * 7 + k;
    const int sh = static_cast<int>(p.c & 31);
    for (int it = 0; it < p.iters; ++it) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = __funnelshift_r(x[k], p.a + k, sh);
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s ^= x[k];
    p.sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) probe_ffma(const ProbeArgs p) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = static_cast<float>(threadIdx.x + k);
    for (int it = 0; it < p.iters; ++it) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fmaf(x[k], p.fa, p.fb);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    p.sink[blockIdx.x * blockDim.x + threadIdx.x] = __float_as_uint(s);
}

// integer adds whose chains alternate add and xor with runtime operands, so that no two
// consecutive operations of a chain merge into one three-input instruction
__global__ void __launch_bounds__(PROBE_THREADS) probe_iadd(const ProbeArgs p) {
    uint32_t x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = threadIdx.x * 3 + k;
    for (int it = 0; it < p.iters; ++it) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = (u & 1) ? (x[k] ^ (p.b + k)) : (x[k] + p.a);
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s ^= x[k];
    p.sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 32-bit shared loads: PROBE_CHAINS independent loads per step at addresses that follow the
// previous value (conflict-free across a warp: lane-consecutive words)
__global__ void __launch_bounds__(PROBE_THREADS) probe_lds(const ProbeArgs p) {
    __shared__ uint32_t buf[PROBE_CHAINS * PROBE_THREADS];
    for (int i = threadIdx.x; i < PROBE_CHAINS * PROBE_THREADS; i += PROBE_THREADS) buf[i] = (p.a & 0) + i;
    __syncthreads();
    uint32_t x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = k * PROBE_THREADS + threadIdx.x;
    for (int it = 0; it < p.iters; ++it) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = buf[x[k]];   // buf[i] == i: stays in place
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s ^= x[k];
    p.sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" msbm_status msbm_pipe_probe(int32_t kind, int32_t blocks, int32_t iters, void *cuda_stream,
                                       float *ms, double *lane_ops) {
    if (kind < 0 || kind > 4 || blocks < 1 || blocks > 65536 || iters < 1 || iters > (1 << 24) || !ms || !lane_ops)
        return MSBM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    ProbeArgs p;
    p.a = 0x01020304u;
    p.b = 0x05060708u;
    p.c = 3u;
    p.fa = 0.999f;
    p.fb = 0.5f;
    p.iters = iters;
    p.sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&p.sink, (size_t)blocks * PROBE_THREADS * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        switch (kind) {
            case 0: probe_dp4a<<<blocks, PROBE_THREADS, 0, st>>>(p); break;
            case 1: probe_shf<<<blocks, PROBE_THREADS, 0, st>>>(p); break;
            case 2: probe_ffma<<<blocks, PROBE_THREADS, 0, st>>>(p); break;
            case 3: probe_iadd<<<blocks, PROBE_THREADS, 0, st>>>(p); break;
            default: probe_lds<<<blocks, PROBE_THREADS, 0, st>>>(p); break;
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    *lane_ops = (double)blocks * PROBE_THREADS * (double)iters * PROBE_CHAINS * PROBE_UNROLL;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (p.sink) cudaFree(p.sink);
    return e == cudaSuccess ? MSBM_OK : (e == cudaErrorMemoryAllocation ? MSBM_ERR_OOM : MSBM_ERR_CUDA);
}
