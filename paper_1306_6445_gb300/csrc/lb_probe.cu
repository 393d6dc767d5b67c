// FP64 fused multiply-add throughput of the device: the ALU roof of the FP64 update, whose
// arithmetic (about 300 dependent FP64 operations per site, Eqs. 3-8 and 17-19) outweighs
// its 144 bytes of population traffic on a GPU with a reduced FP64 rate.
#include <cuda_runtime.h>

#include "lb.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;        // independent FMA chains per thread (latency hiding)
constexpr int PROBE_BLOCKS_PER_SM = 8; // 2048 resident threads per SM

// Every thread runs PROBE_CHAINS independent chains x <- x a + b of `iters` links.
// a, b are runtime values, so nothing folds; the sum is stored only when it equals
// `never`, a value the host chooses out of reach, so nothing is dead either.
__global__ void __launch_bounds__(PROBE_THREADS)
k_dfma_chains(double *out, int iters, double a, double b, double never) {
    double x[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = 1e-3 * threadIdx.x + i;
#pragma unroll 4
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = __fma_rn(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += x[i];
    if (s == never) out[blockIdx.x] = s;
}

}  // namespace

extern "C" lb_status lb_probe_fp64_fma_rate(void *cuda_stream, int iters, double *fma_per_s) {
    if (iters < 1 || !fma_per_s) return LB_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LB_ECUDA;
    const int blocks = sms * PROBE_BLOCKS_PER_SM;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks) != cudaSuccess) return LB_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // x <- 0.999999 x + 1e-6 contracts towards 1 from its start in [0, 7.3]
    const double a = 0.999999, b = 1e-6, never = -1.0;
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_dfma_chains<<<blocks, PROBE_THREADS, 0, st>>>(out, iters, a, b, never);   // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        k_dfma_chains<<<blocks, PROBE_THREADS, 0, st>>>(out, iters, a, b, never);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || !(ms > 0.f)) return LB_ECUDA;
    *fma_per_s = (double)blocks * PROBE_THREADS * PROBE_CHAINS * (double)iters / (ms * 1e-3);
    return LB_OK;
}
