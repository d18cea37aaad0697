// Arithmetic-throughput probe: the denominator of the solve's ALU roofline.
// Every thread runs 8 independent fused multiply-add chains; the grid fills
// every SM.  The chains' results are stored so the work cannot be dropped.
#include <cuda_runtime.h>

#include "camp.h"

namespace {
template <typename T>
__global__ void k_fma_chains(T *out, int iters, T b, T c) {
    T a0 = (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    for (int i = 0; i < iters; i++) {
        a0 = a0 * b + c; a1 = a1 * b + c; a2 = a2 * b + c; a3 = a3 * b + c;
        a4 = a4 * b + c; a5 = a5 * b + c; a6 = a6 * b + c; a7 = a7 * b + c;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

template <typename T>
int run(double *gflops, int iters, cudaStream_t s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CAMP_E_CUDA;
    const int threads = 256, blocks = sms * 8;
    T *out = nullptr;
    if (cudaMallocAsync((void **)&out, sizeof(T) * threads * blocks, s) != cudaSuccess) return CAMP_E_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_chains<T><<<blocks, threads, 0, s>>>(out, iters / 10, (T)0.999999, (T)1e-7);  // warm-up
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<blocks, threads, 0, s>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaFreeAsync(out, s);
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0.f) return CAMP_E_CUDA;
    *gflops = 2.0 * 8.0 * (double)iters * threads * blocks / (ms * 1e-3) / 1e9;
    return CAMP_OK;
}
}  // namespace

extern "C" int camp_probe_fma_rate(int32_t fp64, double *gflops, void *stream) {
    if (!gflops) return CAMP_E_INVAL;
    return fp64 ? run<double>(gflops, 20000, (cudaStream_t)stream)
                : run<float>(gflops, 200000, (cudaStream_t)stream);
}
