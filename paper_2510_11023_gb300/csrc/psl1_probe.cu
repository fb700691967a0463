// psl1_probe.cu -- measured FP64 / FP32 FMA throughput of the current device.
// GB300 publishes no FP64 / FP32 figure beside its tensor rates, so the
// roofline denominators of the ALU-bound kernels are measured here: eight
// independent FMA chains per thread, 8 CTAs of 256 threads per SM, timed
// with CUDA events after a warm-up launch (best of three).
#include <cuda_runtime.h>
#include "psl1.h"

namespace {

template <typename T>
__global__ void k_fma_chains(T* out, int iters, T a, T b)
{
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
double measure(int blocks, int threads, int iters, T* buf, cudaStream_t s)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        k_fma_chains<T><<<blocks, threads, 0, s>>>(buf, iters, (T)1.0000001, (T)1e-7);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        double tf = 2.0 * blocks * threads * (double)iters * 16 * 8 / (ms * 1e-3) / 1e12;
        if (rep > 0 && tf > best) best = tf;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// FP64 tensor-core throughput: four independent accumulators per warp of
// mma.sync m8n8k4 f64 (512 FLOP per instruction and warp)
__global__ void k_dmma_chains(double* out, int iters)
{
    const double a = 1.0 + threadIdx.x * 1e-9, b = 1.0 - threadIdx.x * 1e-9;
    double c[4][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[j][0]), "+d"(c[j][1])
                         : "d"(a), "d"(b));
    }
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) t += c[j][0] + c[j][1];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace

extern "C" psl1_status psl1_probe_dmma(double* fp64_tensor_tflops)
{
    if (!fp64_tensor_tflops) return PSL1_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSL1_ERR_CUDA;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = nsm * 8, threads = 256, iters = 2000;
    void* buf = nullptr;
    if (cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return PSL1_ERR_NOMEM;
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        k_dmma_chains<<<blocks, threads, 0, s>>>((double*)buf, iters);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double tf = 512.0 * 4 * blocks * (threads / 32) * (double)iters / (ms * 1e-3) / 1e12;
        if (rep > 0 && tf > best) best = tf;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    cudaFree(buf);
    *fp64_tensor_tflops = best;
    return e == cudaSuccess ? PSL1_OK : PSL1_ERR_CUDA;
}

extern "C" psl1_status psl1_probe_peaks(double* fp64_tflops, double* fp32_tflops)
{
    if (!fp64_tflops || !fp32_tflops) return PSL1_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSL1_ERR_CUDA;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int blocks = nsm * 8, threads = 256;
    void* buf = nullptr;
    if (cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return PSL1_ERR_NOMEM;
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    *fp64_tflops = measure<double>(blocks, threads, 100, (double*)buf, s);
    *fp32_tflops = measure<float>(blocks, threads, 3000, (float*)buf, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    cudaFree(buf);
    return e == cudaSuccess ? PSL1_OK : PSL1_ERR_CUDA;
}
