// FP64 throughput of the GPU the library runs on: FP64 FMA (DFMA) and FP64
// tensor-core MMA (mma.sync m8n8k4 f64).  These are the denominators of the
// roofline fractions reported for the FP64 path; nothing on the hot path uses them.
#include "dclno_internal.cuh"

#define PK_ITERS 2048

__global__ void k_peak_dfma(double* out, double a, double b) {
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
           x7 = x0 + 7;
    for (int i = 0; i < PK_ITERS; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void k_peak_dmma(double* out, double a) {
    double c[8][2];
#pragma unroll
    for (int t = 0; t < 8; ++t) c[t][0] = c[t][1] = 0.0;
    const double A = a * threadIdx.x, B = a;
    for (int i = 0; i < PK_ITERS / 2; ++i) {
#pragma unroll
        for (int t = 0; t < 8; ++t) dmma_8x8x4(c[t][0], c[t][1], A, B);
    }
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < 8; ++t) s += c[t][0] + c[t][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" dclno_status dclno_measure_fp64_peaks(double* dfma_tflops, double* dmma_tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DCLNO_ERR_CUDA;
    const int grid = sms * 8, block = 256;
    const size_t n = (size_t)grid * block;
    double* buf = nullptr;
    if (cudaMalloc(&buf, n * sizeof(double)) != cudaSuccess) return DCLNO_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_f = 1e30f, best_m = 1e30f, ms = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        k_peak_dfma<<<grid, block>>>(buf, 0.999, 1e-3);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        best_f = fminf(best_f, ms);
        cudaEventRecord(e0);
        k_peak_dmma<<<grid, block>>>(buf, 0.5);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        best_m = fminf(best_m, ms);
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess) return DCLNO_ERR_CUDA;
    if (dfma_tflops) *dfma_tflops = 2.0 * 8.0 * PK_ITERS * (double)n / (best_f * 1e-3) / 1e12;
    if (dmma_tflops) *dmma_tflops = 8.0 * (PK_ITERS / 2) * (double)(n / 32) * 512.0 / (best_m * 1e-3) / 1e12;
    return DCLNO_OK;
}
