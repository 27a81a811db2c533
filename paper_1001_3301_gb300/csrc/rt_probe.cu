// Diagnostics: accuracy probes of the hardware exp2 and tanh the FP32 kernels use,
// micro-benchmarks of the MUFU, FP32 and tensor pipes that bound them (the roofline
// denominators are measured, not assumed), and a self-check of one tcgen05 product
// through the operand layout and descriptors of the surrogate's inference kernel.
#include <cuda_bf16.h>

#include "rt_internal.cuh"
#include "rt_umma.cuh"

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

__device__ __forceinline__ float tanh_f32(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ uint32_t tanh_bf16x2(uint32_t x)
{
    uint32_t y;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

__global__ void k_probe_tanh(const float *x, float *y, long long n, int packed)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (packed) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x[i], x[i]);
            const uint32_t r = tanh_bf16x2(*reinterpret_cast<const uint32_t *>(&h));
            y[i] = __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(&r));
        } else {
            y[i] = tanh_f32(x[i]);
        }
    }
}

__device__ __forceinline__ float rcp_f32(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Chains v <- tanh(v) (contracting towards 0, so bounded), eight per thread;
// packed == 2: v <- 1 / (1 + v) instead (reciprocal; bounded in (0.5, 1)).
__global__ void k_bench_tanh(int iters, int packed, float seed, float *sink, long long *cycles)
{
    float v[kChains];
    uint32_t w[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        v[c] = seed + 0.01f * c + 1e-3f * threadIdx.x;
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[c], 0.5f * v[c]);
        w[c] = *reinterpret_cast<const uint32_t *>(&h);
    }
    __syncthreads();
    const long long t0 = clock64();
    if (packed == 2) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = rcp_f32(1.0f + v[c]);
        }
    } else if (packed) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) w[c] = tanh_bf16x2(w[c]);
        }
    } else {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = tanh_f32(v[c]);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c] + __uint_as_float(w[c]);
    if (s == 12345.0f) sink[0] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Legacy warp-level tensor path: eight independent m16n8k16 BF16 products per warp.
__global__ void k_bench_mma_sync(int iters, float *sink, long long *cycles)
{
    float acc[kChains][4];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0.0f;
    const uint32_t a = 0x3c003c00u + threadIdx.x, b = 0x3c003c00u;  // small BF16 values
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(acc[c][0]), "+f"(acc[c][1]), "+f"(acc[c][2]), "+f"(acc[c][3])
                : "r"(a), "r"(a ^ 1u), "r"(a ^ 2u), "r"(a ^ 3u), "r"(b), "r"(b ^ 1u));
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
    if (s == 12345.0f) sink[0] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

constexpr uint32_t kMaxPolls = 1u << 24;
constexpr int kUmmaBenchPad = 160 * 1024;

// One D = A B^T with M = N = 128 on the tensor core; thread t reads back row t.
// status bit 0: the MMA did not complete within the bounded wait.
__global__ void __launch_bounds__(128) k_probe_umma(const uint16_t *A, const uint16_t *B, int K, float *D,
                                                    unsigned *status)
{
    using namespace rt::umma;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_bar;
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *sA = smem, *sB = smem + (K / 16) * 4096;
    for (int k = 0; k < K; ++k) {
        *reinterpret_cast<uint16_t *>(sA + kmajor_offset(tid, k, 128)) = A[tid * K + k];
        *reinterpret_cast<uint16_t *>(sB + kmajor_offset(tid, k, 128)) = B[tid * K + k];
    }
    if (warp == 0) {
        tmem_alloc(&s_taddr, 128);
        tmem_relinquish();
    }
    if (tid == 0) mbar_init(&s_bar, 1);
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t taddr = s_taddr;
    if (tid == 0) {
        const uint32_t idesc = idesc_bf16_f32(128, 128);
        for (int s = 0; s < K / 16; ++s)
            mma_bf16(taddr, desc_kmajor(smem_u32(sA + s * 4096)), desc_kmajor(smem_u32(sB + s * 4096)), idesc,
                     s > 0 ? 1u : 0u);
        mma_commit(&s_bar);
    }
    bool ok = mbar_wait_bounded(&s_bar, 0, kMaxPolls);
    if (!ok) {
        atomicOr(status, 1u);
        ok = mbar_wait_bounded(&s_bar, 0, kMaxPolls);
    }
    fence_after_sync();
    if (ok) {
        for (int c = 0; c < 4; ++c) {
            float v[32];
            tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
            for (int j = 0; j < 32; ++j) D[tid * 128 + c * 32 + j] = v[j];
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, 128);
}

// tcgen05 issue rate: one CTA per SM, thread 0 issues `iters` M=128 x N x K=16
// products into one accumulator and waits for their commit.
__global__ void __launch_bounds__(128) k_bench_umma(int iters, int n, long long *cycles, unsigned *status)
{
    using namespace rt::umma;
    __shared__ __align__(1024) unsigned char sA[4096];
    __shared__ __align__(1024) unsigned char sB[8192];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_bar;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < 4096 / 4; i += 128) reinterpret_cast<uint32_t *>(sA)[i] = 0x3c003c00u;
    for (int i = tid; i < 8192 / 4; i += 128) reinterpret_cast<uint32_t *>(sB)[i] = 0x3c003c00u;
    if (warp == 0) {
        tmem_alloc(&s_taddr, 256);
        tmem_relinquish();
    }
    if (tid == 0) mbar_init(&s_bar, 1);
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t taddr = s_taddr;
    if (tid == 0) {
        const uint32_t idesc = idesc_bf16_f32(128, (uint32_t)n);
        const uint64_t ad = desc_kmajor(smem_u32(sA)), bd = desc_kmajor(smem_u32(sB));
        const long long t0 = clock64();
        for (int i = 0; i < iters; ++i) mma_bf16(taddr, ad, bd, idesc, i > 0 ? 1u : 0u);
        mma_commit(&s_bar);
        bool ok = mbar_wait_bounded(&s_bar, 0, kMaxPolls);
        if (!ok) {
            atomicOr(status, 1u);
            ok = mbar_wait_bounded(&s_bar, 0, kMaxPolls);
        }
        cycles[blockIdx.x] = clock64() - t0;
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, 256);
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

int rt_probe_tanh(const float *x, float *y, long long n, int packed_bf16, void *cuda_stream)
{
    if (!x || !y || n < 0) return RT_ERR_INVALID_ARG;
    if (n == 0) return RT_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    long long blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_probe_tanh<<<(unsigned)blocks, 256, 0, s>>>(x, y, n, packed_bf16 ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

int rt_probe_umma(const unsigned short *a, const unsigned short *b, int k, float *d, void *cuda_stream)
{
    if (!a || !b || !d || k < 16 || k > 128 || k % 16 != 0) return RT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int smem = 2 * (k / 16) * 4096;
    if (cudaFuncSetAttribute(k_probe_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return RT_ERR_CUDA;
    unsigned *st = nullptr;
    if (cudaMalloc(&st, sizeof(unsigned)) != cudaSuccess) return RT_ERR_CUDA;
    unsigned st_h = 0;
    int status = RT_OK;
    if (cudaMemsetAsync(st, 0, sizeof(unsigned), s) != cudaSuccess) status = RT_ERR_CUDA;
    if (status == RT_OK) {
        k_probe_umma<<<1, 128, smem, s>>>(a, b, k, d, st);
        if (cudaGetLastError() != cudaSuccess) status = RT_ERR_CUDA;
    }
    if (status == RT_OK && cudaMemcpyAsync(&st_h, st, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        status = RT_ERR_CUDA;
    if (status == RT_OK && cudaStreamSynchronize(s) != cudaSuccess) status = RT_ERR_CUDA;
    cudaFree(st);
    if (status == RT_OK && st_h != 0) status = RT_ERR_TIMEOUT;
    return status;
}

int rt_probe_tensor_rates(double *mma_sync_mac, double *umma_n128_mac, double *umma_n256_mac,
                          double *tanh_f32, double *tanh_bf16x2, double *rcp_f32_rate)
{
    if (!mma_sync_mac || !umma_n128_mac || !umma_n256_mac || !tanh_f32 || !tanh_bf16x2 || !rcp_f32_rate)
        return RT_ERR_INVALID_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RT_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RT_ERR_CUDA;
    const int threads = 512, per_sm = 2;
    const int blocks = nsm * per_sm;
    float *sink = nullptr;
    long long *cyc = nullptr;
    unsigned *st = nullptr;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return RT_ERR_CUDA;
    if (cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess) { cudaFree(sink); return RT_ERR_CUDA; }
    if (cudaMalloc(&st, sizeof(unsigned)) != cudaSuccess) { cudaFree(sink); cudaFree(cyc); return RT_ERR_CUDA; }
    cudaMemset(st, 0, sizeof(unsigned));
    long long *cyc_h = new long long[blocks];
    int status = RT_OK;
    auto max_cycles = [&](int nb) {
        cudaMemcpy(cyc_h, cyc, sizeof(long long) * nb, cudaMemcpyDeviceToHost);
        long long cmax = 1;
        for (int i = 0; i < nb; ++i) cmax = cyc_h[i] > cmax ? cyc_h[i] : cmax;
        return (double)cmax;
    };
    // unused dynamic shared memory keeps the tcgen05 benchmark at one CTA per SM
    if (cudaFuncSetAttribute(k_bench_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaBenchPad) != cudaSuccess)
        status = RT_ERR_CUDA;
    // which: 0 mma.sync, 1 tanh f32, 2 tanh bf16x2, 3 umma N=128, 4 umma N=256, 5 rcp f32
    for (int which = 0; which < 6 && status == RT_OK; ++which) {
        for (int rep = 0; rep < 2; ++rep) {
            if (which == 0) k_bench_mma_sync<<<blocks, threads>>>(1024, sink, cyc);
            else if (which <= 2) k_bench_tanh<<<blocks, threads>>>(4096, which == 2, 0.5f, sink, cyc);
            else if (which == 5) k_bench_tanh<<<blocks, threads>>>(4096, 2, 0.5f, sink, cyc);
            else k_bench_umma<<<nsm, 128, kUmmaBenchPad>>>(which == 3 ? 8192 : 4096, which == 3 ? 128 : 256, cyc, st);
        }
        if (cudaDeviceSynchronize() != cudaSuccess) { status = RT_ERR_CUDA; break; }
        if (which == 0) *mma_sync_mac = 1024.0 * kChains * 2048.0 * (threads / 32) * per_sm / max_cycles(blocks);
        else if (which == 1) *tanh_f32 = 4096.0 * kChains * threads * per_sm / max_cycles(blocks);
        else if (which == 2) *tanh_bf16x2 = 4096.0 * kChains * threads * per_sm / max_cycles(blocks);
        else if (which == 3) *umma_n128_mac = 8192.0 * 128 * 128 * 16 / max_cycles(nsm);
        else if (which == 4) *umma_n256_mac = 4096.0 * 128 * 256 * 16 / max_cycles(nsm);
        else *rcp_f32_rate = 4096.0 * kChains * threads * per_sm / max_cycles(blocks);
    }
    unsigned st_h = 0;
    cudaMemcpy(&st_h, st, sizeof(unsigned), cudaMemcpyDeviceToHost);
    delete[] cyc_h;
    cudaFree(sink);
    cudaFree(cyc);
    cudaFree(st);
    if (cudaGetLastError() != cudaSuccess) status = RT_ERR_CUDA;
    if (status == RT_OK && st_h != 0) status = RT_ERR_TIMEOUT;
    return status;
}

}  // extern "C"
