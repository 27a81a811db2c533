// Diagnostics: accuracy probe of the hardware exp2 the FP32 tracer uses, and a
// micro-benchmark of the MUFU and FP32 pipes that bound it (the roofline
// denominators of the tracer are measured, not assumed).
#include "rt_internal.cuh"

namespace {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void k_probe_ex2(const float *x, float *y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = ex2_approx(x[i]);
}

constexpr int kChains = 8;

// Eight independent chains y <- 2^-y per thread: bounded (the map contracts to a
// fixed point near 0.64) and latency-hidden, so the MUFU issue rate is measured.
__global__ void k_bench_ex2(int iters, float seed, float *sink, long long *cycles)
{
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + 0.01f * c + 1e-3f * threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = ex2_approx(-v[c]);
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 12345.0f) sink[0] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void k_bench_ffma(int iters, float seed, float *sink, long long *cycles)
{
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + 0.01f * c + 1e-3f * threadIdx.x;
    const float m = 0.999f, b = 0.001f;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], m, b);
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 12345.0f) sink[0] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" {

int rt_probe_ex2(const float *x, float *y, long long n, void *cuda_stream)
{
    if (!x || !y || n < 0) return RT_ERR_INVALID_ARG;
    if (n == 0) return RT_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    long long blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_probe_ex2<<<(unsigned)blocks, 256, 0, s>>>(x, y, n);
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

int rt_probe_alu_rates(double *ex2_per_sm_clk, double *ffma_per_sm_clk, double *sm_mhz)
{
    if (!ex2_per_sm_clk || !ffma_per_sm_clk || !sm_mhz) return RT_ERR_INVALID_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RT_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RT_ERR_CUDA;
    const int threads = 512, per_sm = 2;  // 32 warps per SM, all resident in one wave
    const int blocks = nsm * per_sm;
    float *sink = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return RT_ERR_CUDA;
    if (cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess) { cudaFree(sink); return RT_ERR_CUDA; }
    long long *cyc_h = new long long[blocks];
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int status = RT_OK;
    for (int which = 0; which < 2 && status == RT_OK; ++which) {
        const int iters = which == 0 ? 4096 : 16384;
        for (int rep = 0; rep < 2; ++rep) {  // first run warms clocks and caches
            cudaEventRecord(e0);
            if (which == 0) k_bench_ex2<<<blocks, threads>>>(iters, 0.5f, sink, cyc);
            else k_bench_ffma<<<blocks, threads>>>(iters, 0.5f, sink, cyc);
            cudaEventRecord(e1);
        }
        if (cudaEventSynchronize(e1) != cudaSuccess) { status = RT_ERR_CUDA; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaMemcpy(cyc_h, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
        long long cmax = 0;
        for (int b = 0; b < blocks; ++b) cmax = cyc_h[b] > cmax ? cyc_h[b] : cmax;
        const double ops_per_sm = (double)iters * kChains * threads * per_sm;
        const double rate = ops_per_sm / (double)cmax;
        if (which == 0) {
            *ex2_per_sm_clk = rate;
            *sm_mhz = (double)cmax / (ms * 1e3);
        } else {
            *ffma_per_sm_clk = rate;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    delete[] cyc_h;
    cudaFree(sink);
    cudaFree(cyc);
    if (cudaGetLastError() != cudaSuccess) status = RT_ERR_CUDA;
    return status;
}

}  // extern "C"
