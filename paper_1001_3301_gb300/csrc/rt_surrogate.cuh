// Device arithmetic shared by the learned surrogate's training and inference
// kernels, so that the network is trained with exactly the activation, feature
// encoding and operand rounding it is evaluated with.
//
// The surrogate replaces the per-bin loop of the tracer (Sect. 2.3, Eqs. 17,
// 28-32, 36) for one cell by an 8 -> 128 -> 128 -> 1 SiLU network of
//   x = (log2(tau_in at six reference frequencies + 2^-20) / 16,  T / 1000 - 0.8,
//        log2(dtau_550 + 2^-30) / 16)
// whose output y gives g = acc / (kappa_550 dN) through ln g = mu + sigma y; then
// q_abs = Gq g kappa_550 dN and a_rad = Ga0 g kappa_550.
//
// Precision: BF16 tensor-core operands with FP32 accumulation. Every continuous
// operand the tensor core reads is split into BF16 parts that sum to it (the
// features into three, the first hidden layer into two) against tied copies of the
// weights, so the inputs and activations keep FP32-like precision while the weights
// are BF16. Activations are SiLU from the hardware exp2 and reciprocal (relative
// error near 2^-22), the last layer in FP32.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace rt {
namespace sur {

constexpr int kNF = 8;        // input features
constexpr int kH = 128;       // hidden width
constexpr int kK1 = 32;       // first-layer K: features x3 (hi, mid, lo), bias column, zeros
constexpr int kBiasCol = 24;  // the constant-1 column of the first layer
constexpr int kNParams = kNF * kH + kH + kH * kH + kH + kH + 1;  // public flat layout

// offsets of the public flat parameter vector: W1 [8][128], b1, W2 [128][128], b2, w3, b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kNF * kH;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH;
constexpr int kOffB3 = kOffW3 + kH;

constexpr float kTauFloor = 9.5367431640625e-07f;    // 2^-20
constexpr float kDtauFloor = 9.3132257461547852e-10f; // 2^-30

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcpf(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2f(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sigmoid(z) = 1 / (1 + e^-z); SiLU(z) = z sigmoid(z); exact to ~2^-21 relative.
__device__ __forceinline__ float sigmoidf_(float z) { return rcpf(1.0f + ex2f(-1.4426950408889634f * z)); }
__device__ __forceinline__ float silu(float z) { return z * sigmoidf_(z); }
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = sigmoidf_(z);
    return s * fmaf(z, 1.0f - s, 1.0f);
}

// The eight features of one cell (see the file comment).
struct FeatConst {
    float kref[6];
    float k550;
};
__device__ __forceinline__ void features(float n_in, float dn, float t, const FeatConst &c, float (&x)[kNF])
{
#pragma unroll
    for (int m = 0; m < 6; ++m) x[m] = 0.0625f * lg2f(fmaf(c.kref[m], n_in, kTauFloor));
    x[6] = fmaf(t, 1e-3f, -0.8f);
    x[7] = 0.0625f * lg2f(fmaf(c.k550, dn, kDtauFloor));
}

// BF16 parts: v ~= hi + mid + lo (round to nearest each time)
__device__ __forceinline__ void split3(float v, __nv_bfloat16 &hi, __nv_bfloat16 &mid, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(hi);
    mid = __float2bfloat16_rn(r1);
    lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}
__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}
// SiLU of two first-layer pre-activations, as (hi, lo) BF16 pairs
__device__ __forceinline__ void act1_pair(float z0, float z1, uint32_t &hi, uint32_t &lo)
{
    const float h0 = silu(z0), h1 = silu(z1);
    const __nv_bfloat16 a0 = __float2bfloat16_rn(h0), a1 = __float2bfloat16_rn(h1);
    hi = pack_bf16(a0, a1);
    lo = pack_bf16(__float2bfloat16_rn(h0 - __bfloat162float(a0)), __float2bfloat16_rn(h1 - __bfloat162float(a1)));
}

// The first-layer operand row of one cell: K = 32 BF16 values as four 16-byte
// groups (k 0-7 hi parts, 8-15 mid, 16-23 lo, 24 = 1, 25-31 = 0).
__device__ __forceinline__ void feature_row(const float (&x)[kNF], uint4 (&g)[4])
{
    __nv_bfloat16 hi[kNF], mid[kNF], lo[kNF];
#pragma unroll
    for (int m = 0; m < kNF; ++m) split3(x[m], hi[m], mid[m], lo[m]);
    g[0] = make_uint4(pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]), pack_bf16(hi[4], hi[5]), pack_bf16(hi[6], hi[7]));
    g[1] = make_uint4(pack_bf16(mid[0], mid[1]), pack_bf16(mid[2], mid[3]), pack_bf16(mid[4], mid[5]),
                      pack_bf16(mid[6], mid[7]));
    g[2] = make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]), pack_bf16(lo[4], lo[5]), pack_bf16(lo[6], lo[7]));
    g[3] = make_uint4(0x3F80u, 0u, 0u, 0u);  // BF16 1.0 in the bias column, then zeros
}

// SplitMix64 finaliser (Steele, Lea & Flood 2014), for counter-based sampling
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ float u01(uint64_t seed, uint64_t stream, uint64_t i)
{
    const uint64_t h = mix64(seed * 0x9E3779B97F4A7C15ULL + mix64(stream + 0xD1B54A32D192ED03ULL * (i + 1)));
    return (float)(h >> 40) * (1.0f / 16777216.0f);
}

}  // namespace sur
}  // namespace rt
