// Peak microbenchmarks for the roofline denominators: dependent-FMA chains in
// FP64 and FP32 on every SM, and the FP64 tensor-core MMA (mma.sync m8n8k4
// f64). Each kernel runs a fixed, bounded number of iterations; the result is
// written to memory so that the work is not eliminated.
#include <cuda_runtime.h>

#include "../../include/pimdgb.h"

namespace {

template <typename T, int CHAINS>
__global__ void fma_chain(T* out, int iters, T a, T b)
{
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) x[c] = x[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dmma_chain(double* out, int iters)
{
    double a = 1.0 + 1e-9 * threadIdx.x, b = 1.0 - 1e-9 * threadIdx.x;
    double c0[2] = {0.0, 0.0}, c1[2] = {0.0, 0.0}, c2[2] = {0.0, 0.0}, c3[2] = {0.0, 0.0};
    for (int i = 0; i < iters; i++) {
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(c0[0]), "+d"(c0[1]) : "d"(a), "d"(b));
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(c1[0]), "+d"(c1[1]) : "d"(a), "d"(b));
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(c2[0]), "+d"(c2[1]) : "d"(a), "d"(b));
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(c3[0]), "+d"(c3[1]) : "d"(a), "d"(b));
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = c0[0] + c0[1] + c1[0] + c1[1] + c2[0] + c2[1] + c3[0] + c3[1];
}

template <typename K>
static float time_kernel(K launch)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();  // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace

// FP64 / FP32 FMA and FP64 MMA throughput (TFLOP/s, 2 flops per FMA) on `device`.
extern "C" int pimd_peak_bench(int device, double* fp64_tflops, double* fp32_tflops, double* dmma_tflops)
{
    if (cudaSetDevice(device) != cudaSuccess) return PIMD_ECUDA;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    const int threads = 256, blocks = nsm * 8;
    void* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * threads * blocks) != cudaSuccess) return PIMD_ENOMEM;
    const int it64 = 4096, it32 = 65536, itm = 8192;
    constexpr int CH = 8;
    float ms = time_kernel([&] { fma_chain<double, CH><<<blocks, threads>>>((double*)buf, it64, 0.999999, 1e-7); });
    if (fp64_tflops) *fp64_tflops = 2.0 * CH * (double)it64 * threads * blocks / (ms * 1e-3) / 1e12;
    ms = time_kernel([&] { fma_chain<float, CH><<<blocks, threads>>>((float*)buf, it32, 0.9999f, 1e-5f); });
    if (fp32_tflops) *fp32_tflops = 2.0 * CH * (double)it32 * threads * blocks / (ms * 1e-3) / 1e12;
    ms = time_kernel([&] { dmma_chain<<<blocks, threads>>>((double*)buf, itm); });
    // per warp per mma: 8 x 8 x 4 FMA
    if (dmma_tflops) *dmma_tflops = 2.0 * 256.0 * 4.0 * (double)itm * (threads / 32) * blocks / (ms * 1e-3) / 1e12;
    const cudaError_t e = cudaGetLastError();
    cudaFree(buf);
    return e == cudaSuccess ? PIMD_OK : PIMD_ECUDA;
}
