// Learned surrogate of the per-bin absorption sum (rt_surrogate.cuh): training on
// cells the exact tracer has traced, with the library's own forward, backward and
// Adam kernels on the tensor cores (warp-level BF16 MMA), and inference with the
// fifth-generation tensor cores (tcgen05, accumulators in TMEM) fused with the ray
// scan, a trust-map gate and the exact per-bin sum as fallback.
//
// Training step (minibatch B, rows padded to a multiple of 64):
//   Xb [B][32]   BF16 feature rows (three parts of each feature, bias column)
//   Z1 = Xb W1b           [B][128] FP32;  H1 = SiLU(Z1) as (hi, lo) BF16 [B][256]
//   Z2 = H1 [W2; W2] + b2 [B][128] FP32
//   head: y = SiLU(Z2) w3 + b3, r = y - t, dZ2 = (2 r / n) w3 SiLU'(Z2)   BF16
//   dZ1 = (dZ2 W2^T) SiLU'(Z1)                                            BF16
//   dW2 = H1^T dZ2 (both halves), dW1 = Xb^T dZ1 (all three parts), split over K
//   Adam on the FP32 masters; tied copies receive the sum of their gradients.
// Every reduction runs in a fixed order, so training is deterministic.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "rt_device.cuh"
#include "rt_surrogate.cuh"
#include "rt_umma.cuh"

namespace rt {

constexpr int kHid = sur::kH;  // hidden width (rt::kH is Planck's constant)
using sur::kK1;
using sur::kNF;
using sur::kNParams;
typedef __nv_bfloat16 bf16;

namespace {

constexpr uint32_t kMaxPolls = 1u << 24;  // bounded mbarrier waits (each poll may sleep)

// trust map: 64 x 64 bins over u = log2(tau_550 in front of the cell) and
// v = log2(dtau_550 of the cell); bin 0 also takes everything below the range
constexpr int kTrustBins = 64;
constexpr float kTrustU0 = -24.0f, kTrustDU = 36.0f / kTrustBins;
constexpr float kTrustV0 = -32.0f, kTrustDV = 40.0f / kTrustBins;
constexpr int kTrustWords = kTrustBins * kTrustBins / 32;
constexpr int kTrustSamples = 32;  // judged points per bin

// ---------------------------------------------------------------------------
// warp-level MMA (training)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(umma::smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(umma::smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

enum { kEpiZ1 = 0, kEpiZ2 = 1, kEpiDZ1 = 2, kEpiPart = 3 };

struct GemmArgs {
    const bf16 *A;  // [M][K] (AT = false) or [K][M] (AT = true), row stride lda
    int lda;
    const bf16 *B;  // [K][128] (BT = false) or [128][K] (BT = true), row stride ldb
    int ldb;
    int M, K, kchunk;  // blockIdx.y covers K range [y kchunk, (y + 1) kchunk)
    float *C;          // Z1, Z2 [M][128], or partials [gridDim.y][M][128]
    bf16 *Cb;          // H1 [M][256] (Z1 epilogue) or dZ1 [M][128]
    const float *aux;  // Z1 (dZ1 epilogue)
    const float *bias; // b2 (Z2 epilogue)
};

// C[M][128] = op(A) op(B) on a 64 x 128 CTA tile (four warps of 16 rows), K staged
// 32 at a time through padded shared memory (conflict-free ldmatrix rows).
template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(128) k_gemm(const GemmArgs g)
{
    constexpr int SA = AT ? 72 : 40;
    constexpr int SB = BT ? 40 : 136;
    __shared__ __align__(16) bf16 sA[AT ? 32 * 72 : 64 * 40];
    __shared__ __align__(16) bf16 sB[BT ? 128 * 40 : 32 * 136];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.x * 64;
    const int kb = blockIdx.y * g.kchunk;
    const int ke = min(g.K, kb + g.kchunk);
    float acc[16][4];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;

    for (int k0 = kb; k0 < ke; k0 += 32) {
        for (int v = tid; v < 256; v += 128) {
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (!AT) {
                const int r = v >> 2, kv = v & 3, m = m0 + r, k = k0 + kv * 8;
                if (m < g.M && k < ke) val = *reinterpret_cast<const uint4 *>(g.A + (size_t)m * g.lda + k);
                *reinterpret_cast<uint4 *>(sA + r * SA + kv * 8) = val;
            } else {
                const int r = v >> 3, mv = v & 7, k = k0 + r, m = m0 + mv * 8;
                if (k < ke && m < g.M) val = *reinterpret_cast<const uint4 *>(g.A + (size_t)k * g.lda + m);
                *reinterpret_cast<uint4 *>(sA + r * SA + mv * 8) = val;
            }
        }
        for (int v = tid; v < 512; v += 128) {
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (!BT) {
                const int r = v >> 4, nv = v & 15, k = k0 + r;
                if (k < ke) val = *reinterpret_cast<const uint4 *>(g.B + (size_t)k * g.ldb + nv * 8);
                *reinterpret_cast<uint4 *>(sB + r * SB + nv * 8) = val;
            } else {
                const int n = v >> 2, kv = v & 3, k = k0 + kv * 8;
                if (k < ke) val = *reinterpret_cast<const uint4 *>(g.B + (size_t)n * g.ldb + k);
                *reinterpret_cast<uint4 *>(sB + n * SB + kv * 8) = val;
            }
        }
        __syncthreads();
        const int q = lane >> 3, r = lane & 7;
#pragma unroll
        for (int kc = 0; kc < 2; ++kc) {
            uint32_t a[4];
            if (!AT) ldsm_x4(a, sA + (16 * warp + (lane & 15)) * SA + kc * 16 + (lane >> 4) * 8);
            else ldsm_x4_t(a, sA + (kc * 16 + r + (q >> 1) * 8) * SA + 16 * warp + (q & 1) * 8);
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                uint32_t b[4];
                if (BT) ldsm_x4(b, sB + (16 * p + r + (q >> 1) * 8) * SB + kc * 16 + (q & 1) * 8);
                else ldsm_x4_t(b, sB + (kc * 16 + r + (q & 1) * 8) * SB + 16 * p + (q >> 1) * 8);
                mma16816(acc[2 * p], a, b[0], b[1]);
                mma16816(acc[2 * p + 1], a, b[2], b[3]);
            }
        }
        __syncthreads();
    }

    const int gq = lane >> 2, t = lane & 3;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int row = m0 + 16 * warp + gq + 8 * half;
        if (row >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = 8 * j + 2 * t;
            float v0 = acc[j][2 * half], v1 = acc[j][2 * half + 1];
            if constexpr (EPI == kEpiZ1) {
                *reinterpret_cast<float2 *>(g.C + (size_t)row * kHid + col) = make_float2(v0, v1);
                uint32_t hi, lo;
                sur::act1_pair(v0, v1, hi, lo);
                *reinterpret_cast<uint32_t *>(g.Cb + (size_t)row * 2 * kHid + col) = hi;
                *reinterpret_cast<uint32_t *>(g.Cb + (size_t)row * 2 * kHid + kHid + col) = lo;
            } else if constexpr (EPI == kEpiZ2) {
                v0 += g.bias[col];
                v1 += g.bias[col + 1];
                *reinterpret_cast<float2 *>(g.C + (size_t)row * kHid + col) = make_float2(v0, v1);
            } else if constexpr (EPI == kEpiDZ1) {
                const float2 z = *reinterpret_cast<const float2 *>(g.aux + (size_t)row * kHid + col);
                *reinterpret_cast<uint32_t *>(g.Cb + (size_t)row * kHid + col) =
                    sur::pack_bf16(__float2bfloat16_rn(v0 * sur::silu_grad(z.x)),
                                   __float2bfloat16_rn(v1 * sur::silu_grad(z.y)));
            } else {
                *reinterpret_cast<float2 *>(g.C + ((size_t)blockIdx.y * g.M + row) * kHid + col) = make_float2(v0, v1);
            }
        }
    }
}

constexpr int kHeadWarps = 8;
constexpr int kHeadPart = 2 * kHid + 2;  // db2 [128], dw3 [128], sum r^2, db3

// Output layer, loss and its gradient: one warp per row, lane l owns columns
// 4l..4l+3. Per-CTA column partials are reduced across warps in a fixed order.
__global__ void __launch_bounds__(kHeadWarps * 32) k_head(const float *Z2, const float *T, const float *master,
                                                          int n_valid, int M, float two_over_n, bf16 *dZ2,
                                                          float *part, float *y_out)
{
    __shared__ float s_c[kHeadWarps][2][kHid];
    __shared__ float s_s[kHeadWarps][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4 w = *reinterpret_cast<const float4 *>(master + sur::kOffW3 + 4 * lane);
    const float b3 = master[sur::kOffB3];
    float pdb2[4] = {0, 0, 0, 0}, pdw3[4] = {0, 0, 0, 0}, ploss = 0.0f, pdb3 = 0.0f;
    for (int row = blockIdx.x * kHeadWarps + warp; row < M; row += gridDim.x * kHeadWarps) {
        const float4 z = *reinterpret_cast<const float4 *>(Z2 + (size_t)row * kHid + 4 * lane);
        const float zz[4] = {z.x, z.y, z.z, z.w}, ww[4] = {w.x, w.y, w.z, w.w};
        float h[4], s = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            h[i] = sur::silu(zz[i]);
            s = fmaf(h[i], ww[i], s);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float y = s + b3;
        const bool valid = row < n_valid;
        const float res = valid ? y - T[row] : 0.0f;
        const float dy = res * two_over_n;
        float dz[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            dz[i] = dy * ww[i] * sur::silu_grad(zz[i]);
            pdb2[i] += dz[i];
            pdw3[i] = fmaf(dy, h[i], pdw3[i]);
        }
        *reinterpret_cast<uint2 *>(dZ2 + (size_t)row * kHid + 4 * lane) =
            make_uint2(sur::pack_bf16(__float2bfloat16_rn(dz[0]), __float2bfloat16_rn(dz[1])),
                       sur::pack_bf16(__float2bfloat16_rn(dz[2]), __float2bfloat16_rn(dz[3])));
        if (lane == 0) {
            ploss = fmaf(res, res, ploss);
            pdb3 += dy;
            if (y_out) y_out[row] = y;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        s_c[warp][0][4 * lane + i] = pdb2[i];
        s_c[warp][1][4 * lane + i] = pdw3[i];
    }
    if (lane == 0) {
        s_s[warp][0] = ploss;
        s_s[warp][1] = pdb3;
    }
    __syncthreads();
    float *out = part + (size_t)blockIdx.x * kHeadPart;
    for (int c = threadIdx.x; c < 2 * kHid; c += blockDim.x) {
        float s = 0.0f;
        for (int w2 = 0; w2 < kHeadWarps; ++w2) s += s_c[w2][c / kHid][c % kHid];
        out[c] = s;
    }
    if (threadIdx.x < 2) {
        float s = 0.0f;
        for (int w2 = 0; w2 < kHeadWarps; ++w2) s += s_s[w2][threadIdx.x];
        out[2 * kHid + threadIdx.x] = s;
    }
}

// BF16 operand copies of the masters for the training GEMMs:
// W1b [32][128] (rows 0-7, 8-15, 16-23 = W1, row 24 = b1, rest 0), W2b [256][128] = [W2; W2].
__device__ __forceinline__ void write_copies(int p, float w, bf16 *W1b, bf16 *W2b)
{
    const bf16 b = __float2bfloat16_rn(w);
    if (p < sur::kOffB1) {
        const int k = p / kHid, n = p % kHid;
        W1b[k * kHid + n] = b;
        W1b[(k + 8) * kHid + n] = b;
        W1b[(k + 16) * kHid + n] = b;
    } else if (p < sur::kOffW2) {
        W1b[sur::kBiasCol * kHid + (p - sur::kOffB1)] = b;
    } else if (p < sur::kOffB2) {
        const int q = p - sur::kOffW2;
        W2b[q] = b;
        W2b[kHid * kHid + q] = b;
    }
}

// Gradient of parameter p (public flat order) from the split-K and head partials,
// summed in a fixed order; tied copies add up.
__device__ float param_grad(int p, const float *dW1p, const float *dW2p, int S, const float *hp, int G)
{
    float g = 0.0f;
    if (p < sur::kOffB1) {
        const int k = p / kHid, n = p % kHid;
        for (int s = 0; s < S; ++s) {
            const float *b = dW1p + (size_t)s * kK1 * kHid;
            g += b[k * kHid + n] + b[(k + 8) * kHid + n] + b[(k + 16) * kHid + n];
        }
    } else if (p < sur::kOffW2) {
        const int n = p - sur::kOffB1;
        for (int s = 0; s < S; ++s) g += dW1p[(size_t)s * kK1 * kHid + sur::kBiasCol * kHid + n];
    } else if (p < sur::kOffB2) {
        const int q = p - sur::kOffW2;
        for (int s = 0; s < S; ++s) {
            const float *b = dW2p + (size_t)s * 2 * kHid * kHid;
            g += b[q] + b[kHid * kHid + q];
        }
    } else if (p < sur::kOffW3) {
        for (int i = 0; i < G; ++i) g += hp[(size_t)i * kHeadPart + (p - sur::kOffB2)];
    } else if (p < sur::kOffB3) {
        for (int i = 0; i < G; ++i) g += hp[(size_t)i * kHeadPart + kHid + (p - sur::kOffW3)];
    } else {
        for (int i = 0; i < G; ++i) g += hp[(size_t)i * kHeadPart + 2 * kHid + 1];
    }
    return g;
}

struct UpdateArgs {
    int mode;  // 0: write the gradient; 1: Adam step; 2: only refresh the BF16 copies
    float *master, *m, *v;
    const float *dW1p, *dW2p, *hp;
    int S, G;
    float lr, c1, c2;  // learning rate, 1 - beta1^t, 1 - beta2^t
    float *grad_out;
    float *loss_out;   // [1]: sum of r^2 / n
    float inv_n;
    bf16 *W1b, *W2b;
};

__global__ void k_update(const UpdateArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && a.mode != 2 && a.loss_out) {
        float s = 0.0f;
        for (int i = 0; i < a.G; ++i) s += a.hp[(size_t)i * kHeadPart + 2 * kHid];
        *a.loss_out = s * a.inv_n;
    }
    if (p >= kNParams) return;
    if (a.mode == 2) {
        write_copies(p, a.master[p], a.W1b, a.W2b);
        return;
    }
    const float g = param_grad(p, a.dW1p, a.dW2p, a.S, a.hp, a.G);
    if (a.mode == 0) {
        a.grad_out[p] = g;
        return;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float m = b1 * a.m[p] + (1.0f - b1) * g;
    const float v = b2 * a.v[p] + (1.0f - b2) * g * g;
    a.m[p] = m;
    a.v[p] = v;
    const float w = a.master[p] - a.lr * (m / a.c1) / (sqrtf(v / a.c2) + eps);
    a.master[p] = w;
    write_copies(p, w, a.W1b, a.W2b);
}

// Minibatch rows: sample i of the training set for row b, drawn by a counter hash
// of (seed, step, b); rows >= n get zero features (their loss weight is zero).
__global__ void k_gather(const float *X, const float *Y, long long n_train, float mu, float inv_sigma,
                         unsigned long long seed, long long step, int B, int n_valid, bf16 *Xb, float *Tb)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    uint4 *dst = reinterpret_cast<uint4 *>(Xb + (size_t)b * kK1);
    if (b >= n_valid) {
        dst[0] = dst[1] = dst[2] = dst[3] = make_uint4(0u, 0u, 0u, 0u);
        Tb[b] = 0.0f;
        return;
    }
    const uint64_t h = sur::mix64(seed * 0x9E3779B97F4A7C15ULL + sur::mix64((uint64_t)step * 1000003ULL + (uint64_t)b));
    const long long i = (long long)(h % (uint64_t)n_train);
    float x[kNF];
#pragma unroll
    for (int m = 0; m < kNF; ++m) x[m] = X[i * kNF + m];
    uint4 gr[4];
    sur::feature_row(x, gr);
    dst[0] = gr[0];
    dst[1] = gr[1];
    dst[2] = gr[2];
    dst[3] = gr[3];
    Tb[b] = (Y[i] - mu) * inv_sigma;
}

// Rows given directly (gradient and evaluation entry points): identity gather.
__global__ void k_rows(const float *X, const float *T, int n, int B, bf16 *Xb, float *Tb)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    uint4 *dst = reinterpret_cast<uint4 *>(Xb + (size_t)b * kK1);
    if (b >= n) {
        dst[0] = dst[1] = dst[2] = dst[3] = make_uint4(0u, 0u, 0u, 0u);
        Tb[b] = 0.0f;
        return;
    }
    float x[kNF];
#pragma unroll
    for (int m = 0; m < kNF; ++m) x[m] = X[(size_t)b * kNF + m];
    uint4 gr[4];
    sur::feature_row(x, gr);
    dst[0] = gr[0];
    dst[1] = gr[1];
    dst[2] = gr[2];
    dst[3] = gr[3];
    Tb[b] = T ? T[b] : 0.0f;
}

// ---------------------------------------------------------------------------
// training samples from traced grids
// ---------------------------------------------------------------------------
struct CollectArgs {
    int pass;  // 0: count eligible cells; 1: count selected; 2: write selected
    const float *rho, *tdust, *q;
    const float4 *rtab;
    const float *domega32;
    int nr;
    long long nrays;
    float t_sub, acc_mask;
    sur::FeatConst fc;
    unsigned long long seed;
    long long cell_base;  // global index of this grid's first cell (sampling counter)
    float p_keep, p_val;
    unsigned *cnt;              // [2 nrays]
    const long long *off;       // [2 nrays] exclusive offsets (pass 2)
    float *X, *Y, *Xv, *Yv;
    long long cap_train, cap_val;  // rows allocated in X / Xv (pass 2 writes stay below)
};

// One thread per ray walks it outward with a compensated column (Eq. 19).
__global__ void k_collect(const CollectArgs a)
{
    const long long ray = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (ray >= a.nrays) return;
    const float dom = a.domega32[ray];
    KahanSum N;
    N.zero();
    unsigned c0 = 0, c1 = 0;
    long long o0 = 0, o1 = 0;
    if (a.pass == 2) {
        o0 = a.off[2 * ray];
        o1 = a.off[2 * ray + 1];
    }
    for (int k = 0; k < a.nr; ++k) {
        const size_t cell = (size_t)ray * a.nr + k;
        const float4 g = __ldg(a.rtab + k);
        const float t = a.tdust[cell];
        const bool dust = t <= a.t_sub;
        const float d = dust ? a.rho[cell] * g.x : 0.0f;
        const float n_in = N.value();
        const float acc = a.q[cell] / g.y;
        const bool elig = dust && d > 0.0f && acc * dom > a.acc_mask;
        if (a.pass == 0) {
            c0 += elig;
        } else if (elig) {
            const float u = sur::u01(a.seed, 77, (uint64_t)(a.cell_base + (long long)cell));
            const bool tr = u < a.p_keep;
            const bool va = !tr && u < a.p_keep + a.p_val;
            if (a.pass == 1) {
                c0 += tr;
                c1 += va;
            } else if ((tr && o0 < a.cap_train) || (va && o1 < a.cap_val)) {
                float x[kNF];
                sur::features(n_in, d, t, a.fc, x);
                float *X = tr ? a.X + o0 * kNF : a.Xv + o1 * kNF;
#pragma unroll
                for (int m = 0; m < kNF; ++m) X[m] = x[m];
                const float lng = logf(acc) - logf(a.fc.k550 * d);
                if (tr) a.Y[o0++] = lng;
                else a.Yv[o1++] = lng;
            }
        }
        N.add(d);
    }
    if (a.pass != 2) {
        a.cnt[2 * ray] = c0;
        a.cnt[2 * ray + 1] = c1;
    }
}

// Exclusive scan of the per-ray counts (two interleaved streams) in one block;
// base[2] carries the running totals across grids and receives the new totals.
__global__ void k_scan_counts(const unsigned *cnt, long long nrays, long long *off, long long *base)
{
    __shared__ long long s[2][1024];
    const int t = threadIdx.x;
    const long long per = (nrays + 1023) / 1024;
    const long long b0 = t * per, b1 = min(nrays, b0 + per);
    long long sum0 = 0, sum1 = 0;
    for (long long i = b0; i < b1; ++i) {
        sum0 += cnt[2 * i];
        sum1 += cnt[2 * i + 1];
    }
    s[0][t] = sum0;
    s[1][t] = sum1;
    __syncthreads();
    if (t < 2) {  // serial exclusive scan of the 1024 block sums (fixed order)
        long long run = base[t];
        for (int i = 0; i < 1024; ++i) {
            const long long v = s[t][i];
            s[t][i] = run;
            run += v;
        }
        base[t] = run;
    }
    __syncthreads();
    long long r0 = s[0][t], r1 = s[1][t];
    for (long long i = b0; i < b1; ++i) {
        off[2 * i] = r0;
        off[2 * i + 1] = r1;
        r0 += cnt[2 * i];
        r1 += cnt[2 * i + 1];
    }
}

// mean and standard deviation of the targets (FP64, one block, fixed order)
__global__ void k_moments(const float *Y, long long n, double *out)
{
    __shared__ double s1[1024], s2[1024];
    const int t = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (long long i = t; i < n; i += 1024) {
        const double y = Y[i];
        a += y;
        b += y * y;
    }
    s1[t] = a;
    s2[t] = b;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (t < o) {
            s1[t] += s1[t + o];
            s2[t] += s2[t + o];
        }
        __syncthreads();
    }
    if (t == 0) {
        const double mu = s1[0] / n;
        out[0] = mu;
        out[1] = sqrt(fmax(s2[0] / n - mu * mu, 1e-30));
    }
}

// ---------------------------------------------------------------------------
// inference: the network on the fifth-generation tensor cores
// ---------------------------------------------------------------------------
constexpr int kInfThreads = 256;
constexpr uint32_t kSmW2 = 0, kSmH1hi = 32768, kSmH1lo = 65536, kSmW1 = 98304;
constexpr uint32_t kSmDyn = 106496;  // the feature rows (8 KB) alias the start of H1lo

struct SurNet {
    const uint4 *w1t;  // [512] 16-byte groups: W1b^T in the K-major tensor-core layout (128 x 32)
    const uint4 *w2t;  // [2048]: W2^T (128 x 128)
    const float *master;  // b2, w3, b3 in FP32
    float mu, sigma;
    sur::FeatConst fc;
};

struct MlpSmem {
    float b2[kHid], w3[kHid];
    float part[2][kHid];
    uint64_t bar;
    uint32_t taddr;
};

__device__ void mlp_load(unsigned char *dsm, MlpSmem &S, const SurNet &net)
{
    const int tid = threadIdx.x;
    for (int i = tid; i < 2048; i += kInfThreads) reinterpret_cast<uint4 *>(dsm + kSmW2)[i] = net.w2t[i];
    for (int i = tid; i < 512; i += kInfThreads) reinterpret_cast<uint4 *>(dsm + kSmW1)[i] = net.w1t[i];
    if (tid < kHid) {
        S.b2[tid] = net.master[sur::kOffB2 + tid];
        S.w3[tid] = net.master[sur::kOffW3 + tid];
    }
    if ((tid >> 5) == 0) {
        umma::tmem_alloc(&S.taddr, 128);
        umma::tmem_relinquish();
    }
    if (tid == 0) umma::mbar_init(&S.bar, 1);
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
}

__device__ void mlp_release(MlpSmem &S)
{
    umma::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) umma::tmem_dealloc(S.taddr, 128);
}

// The network on 128 rows: threads 0..127 supply row r = tid's features; y is
// returned to them. 256 threads: warp w reads TMEM lanes 32 (w % 4).. and columns
// 64 (w / 4)..+63 in the epilogues. Returns false (in every thread) if an MMA did
// not complete within the bounded wait.
__device__ bool mlp_tile(unsigned char *dsm, MlpSmem &S, uint32_t &phase, const float (&x)[kNF], bool have_x,
                         float b3, float &y)
{
    using namespace umma;
    const int tid = threadIdx.x, warp = tid >> 5, r = tid & 127, half = tid >> 7;
    unsigned char *sA1 = dsm + kSmH1lo;
    const uint32_t taddr = S.taddr;
    const uint32_t idesc = idesc_bf16_f32(128, 128);
    if (tid < 128) {
        uint4 gr[4] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u),
                       make_uint4(0u, 0u, 0u, 0u)};
        if (have_x) sur::feature_row(x, gr);
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8)
            *reinterpret_cast<uint4 *>(sA1 + kmajor_offset(r, 8 * g8, 128)) = gr[g8];
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
        fence_after_sync();
        mma_bf16(taddr, desc_kmajor(smem_u32(sA1)), desc_kmajor(smem_u32(dsm + kSmW1)), idesc, 0u);
        mma_bf16(taddr, desc_kmajor(smem_u32(sA1 + 4096)), desc_kmajor(smem_u32(dsm + kSmW1 + 4096)), idesc, 1u);
        mma_commit(&S.bar);
    }
    bool ok = mbar_wait_bounded(&S.bar, phase, kMaxPolls);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) return false;
    fence_after_sync();

    const uint32_t lane_addr = taddr + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
        const int col0 = 64 * half + 32 * c2;
        float v[32];
        tmem_ld32(lane_addr + (uint32_t)col0, v);
#pragma unroll
        for (int j8 = 0; j8 < 4; ++j8) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) sur::act1_pair(v[8 * j8 + 2 * p], v[8 * j8 + 2 * p + 1], hi[p], lo[p]);
            const uint32_t off = kmajor_offset(r, col0 + 8 * j8, 128);
            *reinterpret_cast<uint4 *>(dsm + kSmH1hi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(dsm + kSmH1lo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
        fence_after_sync();
        for (int s = 0; s < 8; ++s)
            mma_bf16(taddr, desc_kmajor(smem_u32(dsm + kSmH1hi + s * 4096)),
                     desc_kmajor(smem_u32(dsm + kSmW2 + s * 4096)), idesc, s > 0 ? 1u : 0u);
        for (int s = 0; s < 8; ++s)
            mma_bf16(taddr, desc_kmajor(smem_u32(dsm + kSmH1lo + s * 4096)),
                     desc_kmajor(smem_u32(dsm + kSmW2 + s * 4096)), idesc, 1u);
        mma_commit(&S.bar);
    }
    ok = mbar_wait_bounded(&S.bar, phase, kMaxPolls);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) return false;
    fence_after_sync();

    float part = 0.0f;
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
        const int col0 = 64 * half + 32 * c2;
        float v[32];
        tmem_ld32(lane_addr + (uint32_t)col0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) part = fmaf(sur::silu(v[j] + S.b2[col0 + j]), S.w3[col0 + j], part);
    }
    S.part[half][r] = part;
    fence_before_sync();
    __syncthreads();
    y = S.part[0][r] + S.part[1][r] + b3;
    return true;
}

// On an MMA timeout: give the tensor core a second bounded wait for the work in
// flight, then the caller frees TMEM and returns.
__device__ void mlp_drain(MlpSmem &S, uint32_t phase, unsigned *timeout)
{
    if (threadIdx.x == 0) {
        atomicOr(timeout, 1u);
        umma::mbar_wait_bounded(&S.bar, phase ^ 1u, kMaxPolls);
    }
}

// Features rows -> standardised outputs y (test entry point and trust map).
__global__ void __launch_bounds__(kInfThreads, 1) k_sur_eval(const SurNet net, const float *X, int n, float *y,
                                                            unsigned *timeout)
{
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ MlpSmem S;
    mlp_load(dsm, S, net);
    const float b3 = net.master[sur::kOffB3];
    uint32_t phase = 0;
    const int ntiles = (n + 127) / 128;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row = tile * 128 + (threadIdx.x & 127);
        float x[kNF];
        const bool have = threadIdx.x < 128 && row < n;
#pragma unroll
        for (int m = 0; m < kNF; ++m) x[m] = have ? X[(size_t)row * kNF + m] : 0.0f;
        float yy = 0.0f;
        if (!mlp_tile(dsm, S, phase, x, have, b3, yy)) {
            mlp_drain(S, phase, timeout);
            break;
        }
        if (have) y[row] = yy;
    }
    mlp_release(S);
}

// exact per-bin sum of one cell (Eqs. 17, 31-32; the rho -> 0 limit for dN == 0):
// acc = sum_i 2^(nk_i N + lf_i) (1 - e^{-kappa_i dN}), and sum_i kappa_i 2^(...)
__device__ __forceinline__ void exact_cell(const float2 *s_nu, const float *s_kap, int na, float n_in, float dn,
                                           float &acc, float &acc0)
{
    acc = 0.0f;
    acc0 = 0.0f;
    for (int i = 0; i < na; ++i) {
        const float e = sur::ex2f(fmaf(s_nu[i].x, n_in, s_nu[i].y));
        if (dn > 0.0f) acc = fmaf(e, -expm1f(s_nu[i].x * dn * (float)kLn2), acc);
        else acc0 = fmaf(e, s_kap[i], acc0);
    }
}

struct SurRayArgs {
    const float *rho, *tdust;
    float *q, *a;
    const float *q_ref, *a_ref;  // validate mode: the exact tracer's outputs
    const float4 *rtab;
    const float *domega32;
    const NuEntry *nu;
    const float *kap;
    int n_active, nnu_pad;
    const uint32_t *trust;
    SurNet net;
    float tol, acc_mask, t_sub;
    int mode;  // 0: gate by the trust map; 1: judge by the exact outputs; 2: network everywhere
    double2 *partials;  // [grid] (absorbed, escaped) / (R*^2 F_max)
    double *stats;      // [grid][5]
    unsigned *bad_input;
    unsigned seq;
    unsigned *timeout;
    unsigned ncells, nr, ntiles;
    FastDiv nrdiv;
};

// Persistent: CTA c takes tiles [c T / G, (c + 1) T / G) of 128 consecutive cells
// of the ray-major field, in order, carrying the column density of a ray that
// continues into the next tile. Per tile: masked column dN (Eq. 19), segmented
// compensated scan -> N_in, features, the network, gate or judge, outputs.
__global__ void __launch_bounds__(kInfThreads, 2) k_sur_ray(const __grid_constant__ SurRayArgs p)
{
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ MlpSmem S;
    __shared__ float2 s_nu[RT_MAX_NU + kNuPad];
    __shared__ float s_kap[RT_MAX_NU + kNuPad];
    __shared__ uint32_t s_trust[kTrustWords];
    __shared__ KahanSum s_wv[4], s_next, s_red[8];
    __shared__ int s_wf[4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, r = tid & 127;
    for (int i = tid; i < p.nnu_pad; i += kInfThreads) {
        s_nu[i] = make_float2(p.nu[i].nk, p.nu[i].lf);
        s_kap[i] = p.kap[i];
    }
    for (int i = tid; i < kTrustWords; i += kInfThreads) s_trust[i] = p.trust ? p.trust[i] : 0u;
    mlp_load(dsm, S, p.net);
    const float b3 = p.net.master[sur::kOffB3];
    const float k550 = p.net.fc.k550;
    uint32_t phase = 0;

    const unsigned t_begin = (unsigned)(((unsigned long long)p.ntiles * blockIdx.x) / gridDim.x);
    const unsigned t_end = (unsigned)(((unsigned long long)p.ntiles * (blockIdx.x + 1)) / gridDim.x);

    // column in front of the first tile when it starts inside a ray
    KahanSum carry;
    carry.zero();
    if (t_begin < t_end) {
        const unsigned first = t_begin * 128u;
        const unsigned ray0 = p.nrdiv.div(first);
        const unsigned start = ray0 * p.nr;
        KahanSum s;
        s.zero();
        if (tid < 128)
            for (unsigned c = start + tid; c < first; c += 128) {
                const unsigned k = c - start;
                const float t = p.tdust[c];
                s.add(t <= p.t_sub ? p.rho[c] * __ldg(p.rtab + k).x : 0.0f);
            }
        for (int o = 16; o > 0; o >>= 1) s.add(s.shfl_xor(o));
        if (lane == 0) s_red[warp] = s;
        __syncthreads();
        carry = s_red[0];
        carry.add(s_red[1]);
        carry.add(s_red[2]);
        carry.add(s_red[3]);
        __syncthreads();
    }

    KahanSum eabs, eesc;
    eabs.zero();
    eesc.zero();
    double st_dust = 0, st_fb = 0, st_judged = 0, st_sum = 0, st_max = 0;

    for (unsigned tile = t_begin; tile < t_end; ++tile) {
        const unsigned cell = tile * 128u + (unsigned)r;
        const bool valid = tid < 128 && cell < p.ncells;
        unsigned ray = 0, k = 0;
        float rho = 0.0f, td = 0.0f, d = 0.0f;
        float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        bool dust = false;
        if (valid) {
            ray = p.nrdiv.div(cell);
            k = cell - ray * p.nr;
            rho = p.rho[cell];
            td = p.tdust[cell];
            g = __ldg(p.rtab + k);
            dust = td <= p.t_sub;
            d = dust ? rho * g.x : 0.0f;
        }
        const bool bad = valid && (!(rho >= 0.0f && rho <= FLT_MAX) || td != td);
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(p.bad_input, p.seq);
        const bool head = !valid || k == 0u;

        // segmented inclusive scan over the tile (threads 0..127), compensated
        KahanSum v;
        v.zero();
        v.add(d);
        bool f = head;
        for (int o = 1; o < 32; o <<= 1) {
            const KahanSum vo = v.shfl_up(o);
            const bool fo = __shfl_up_sync(0xffffffffu, f, o);
            if (lane >= o) {
                if (!f) v.add(vo);
                f = f || fo;
            }
        }
        if (lane == 31 && warp < 4) {
            s_wv[warp] = v;
            s_wf[warp] = f;
        }
        __syncthreads();
        KahanSum pre = carry;
        if (warp < 4)
            for (int w2 = 0; w2 < warp; ++w2) {
                if (s_wf[w2]) pre = s_wv[w2];
                else pre.add(s_wv[w2]);
            }
        KahanSum incl = v;
        if (!f) incl.add(pre);
        KahanSum ex = incl.shfl_up(1);
        if (lane == 0) ex = pre;
        if (head) ex.zero();
        if (tid == 127) s_next = incl;
        const float n_in = ex.value();

        float x[kNF];
        sur::features(n_in, d, td, p.net.fc, x);
        float y = 0.0f;
        if (!mlp_tile(dsm, S, phase, x, valid, b3, y)) {
            mlp_drain(S, phase, p.timeout);
            break;
        }
        carry = s_next;  // written before the network's barriers

        if (valid) {
            const float dom = __ldg(p.domega32 + ray);
            float qv = 0.0f, av = 0.0f, acc = 0.0f;
            if (dust) {
                st_dust += 1.0;
                const float gg = sur::ex2f((p.net.mu + p.net.sigma * y) * (float)kLog2e);
                acc = gg * k550 * d;
                qv = g.y * acc;
                av = g.z * gg * k550;
                bool use_exact = false;
                float qx = 0.0f, ax = 0.0f;
                if (p.mode == 0) {
                    // an empty column (log2 0 = -inf) falls into bin 0
                    const float u = fmaxf(sur::lg2f(k550 * n_in), kTrustU0 - 1.0f);
                    const float w = fmaxf(sur::lg2f(k550 * d), kTrustV0 - 1.0f);
                    const int iu = max(0, (int)floorf((u - kTrustU0) * (1.0f / kTrustDU)));
                    const int iv = max(0, (int)floorf((w - kTrustV0) * (1.0f / kTrustDV)));
                    bool trusted = false;
                    if (iu < kTrustBins && iv < kTrustBins) {
                        const int b = iu * kTrustBins + iv;
                        trusted = (s_trust[b >> 5] >> (b & 31)) & 1u;
                    }
                    if (!trusted) {
                        float e1, e0;
                        exact_cell(s_nu, s_kap, p.n_active, n_in, d, e1, e0);
                        acc = e1;
                        qx = g.y * e1;
                        ax = g.z * (d > 0.0f ? __fdividef(e1, d) : e0);
                        use_exact = true;
                    }
                } else if (p.mode == 1) {
                    qx = p.q_ref[cell];
                    ax = p.a_ref[cell];
                    const float accx = qx / g.y;
                    if (accx * dom > p.acc_mask) {
                        const double rel = fabs((double)qv / (double)qx - 1.0);
                        st_judged += 1.0;
                        st_sum += rel;
                        st_max = fmax(st_max, rel);
                        if (!(rel <= p.tol)) use_exact = true;
                    }
                    if (use_exact) acc = accx;
                }
                if (use_exact) {
                    st_fb += 1.0;
                    qv = qx;
                    av = ax;
                }
                if (!(qv >= 0.0f && qv <= FLT_MAX)) qv = 0.0f;  // a non-finite network answer
            }
            p.q[cell] = qv;
            p.a[cell] = av;
            eabs.add(acc * dom);
            if (k == p.nr - 1u) {  // the ray leaves the grid: escaping power (Eqs. 33-35)
                const float ntot = incl.value();
                float s = 0.0f;
                for (int i = 0; i < p.n_active; ++i) s += sur::ex2f(fmaf(s_nu[i].x, ntot, s_nu[i].y));
                eesc.add(s * dom);
            }
        }
    }

    // per-CTA energy and statistics
    for (int o = 16; o > 0; o >>= 1) {
        eabs.add(eabs.shfl_xor(o));
        eesc.add(eesc.shfl_xor(o));
        st_dust += __shfl_xor_sync(0xffffffffu, st_dust, o);
        st_fb += __shfl_xor_sync(0xffffffffu, st_fb, o);
        st_judged += __shfl_xor_sync(0xffffffffu, st_judged, o);
        st_sum += __shfl_xor_sync(0xffffffffu, st_sum, o);
        st_max = fmax(st_max, __shfl_xor_sync(0xffffffffu, st_max, o));
    }
    __shared__ double s_st[8][5];
    __shared__ KahanSum s_e[8][2];
    if (lane == 0) {
        s_e[warp][0] = eabs;
        s_e[warp][1] = eesc;
        s_st[warp][0] = st_dust;
        s_st[warp][1] = st_fb;
        s_st[warp][2] = st_judged;
        s_st[warp][3] = st_sum;
        s_st[warp][4] = st_max;
    }
    mlp_release(S);  // includes a block barrier
    if (tid == 0) {
        KahanSum a = s_e[0][0], e = s_e[0][1];
        double st[5] = {s_st[0][0], s_st[0][1], s_st[0][2], s_st[0][3], s_st[0][4]};
        for (int w2 = 1; w2 < kInfThreads / 32; ++w2) {
            a.add(s_e[w2][0]);
            e.add(s_e[w2][1]);
            for (int j = 0; j < 4; ++j) st[j] += s_st[w2][j];
            st[4] = fmax(st[4], s_st[w2][4]);
        }
        p.partials[blockIdx.x] = make_double2(to_double(a), to_double(e));
        for (int j = 0; j < 5; ++j) p.stats[blockIdx.x * 5 + j] = st[j];
    }
}

// ---------------------------------------------------------------------------
// trust map: which (u, v) bins the network answers within the tolerance
// ---------------------------------------------------------------------------
__global__ void k_trust_points(const sur::FeatConst fc, float t_sub, unsigned long long seed, float *X, float2 *nd)
{
    const int pt = blockIdx.x * blockDim.x + threadIdx.x;
    if (pt >= kTrustBins * kTrustBins * kTrustSamples) return;
    const int b = pt / kTrustSamples, j = pt % kTrustSamples;
    const int iu = b / kTrustBins, iv = b % kTrustBins;
    const float r1 = sur::u01(seed, 1, pt), r2 = sur::u01(seed, 2, pt), r3 = sur::u01(seed, 3, pt);
    // bin 0 also covers everything below the range, down to an empty column
    const float ulo = iu == 0 ? kTrustU0 - 8.0f : kTrustU0 + iu * kTrustDU;
    const float vlo = iv == 0 ? kTrustV0 - 8.0f : kTrustV0 + iv * kTrustDV;
    const float uhi = kTrustU0 + (iu + 1) * kTrustDU, vhi = kTrustV0 + (iv + 1) * kTrustDV;
    float n_in = exp2f(ulo + r1 * (uhi - ulo)) / fc.k550;
    float dn = exp2f(vlo + r2 * (vhi - vlo)) / fc.k550;
    if (iu == 0 && j == 0) n_in = 0.0f;
    if (iv == 0 && j == 1) dn = 0.0f;
    float x[kNF];
    sur::features(n_in, dn, r3 * t_sub, fc, x);
    for (int m = 0; m < kNF; ++m) X[(size_t)pt * kNF + m] = x[m];
    nd[pt] = make_float2(n_in, dn);
}

// One warp per bin (32 points): trusted iff every point is either within tol/2 in
// ln g or absorbs far too little to be judged (acc dOmega_max at least 1000 times
// below the mask, so cells elsewhere in the bin stay below it too).
__global__ void k_trust_judge(const float2 *nd, const float *y, float mu, float sigma, const NuEntry *nu,
                              const float *kap, int na, float k550, float tol, float acc_mask_over_dom,
                              uint32_t *bits)
{
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= kTrustBins * kTrustBins) return;
    const int pt = b * kTrustSamples + lane;
    const float2 v = nd[pt];
    float g = 0.0f;
    for (int i = 0; i < na; ++i) {
        const float e = sur::ex2f(fmaf(nu[i].nk, v.x, nu[i].lf));
        const float xk = kap[i] * v.y;
        const float phi = xk > 0.0f ? -expm1f(-xk) / xk : 1.0f;
        g = fmaf(e * kap[i], phi, g);
    }
    g /= k550;
    const float lng = logf(g);
    const float pred = mu + sigma * y[pt];
    const float err = fabsf(pred - lng);
    const bool relevant = 1e3f * g * k550 * v.y > acc_mask_over_dom;
    const bool badp = relevant && !(err <= 0.5f * tol);
    const unsigned anybad = __ballot_sync(0xffffffffu, badp);
    if (lane == 0 && anybad == 0u) atomicOr(bits + (b >> 5), 1u << (b & 31));
}

// Inference operands from the masters: W1b^T and W2^T in the tensor-core layout.
__global__ void k_pack_infer(const float *master, uint16_t *w1t, uint16_t *w2t)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < kHid * kK1) {  // W1 operand: B[n][k] = W1b[k][n]
        const int n = t / kK1, k = t % kK1;
        float w = 0.0f;
        if (k < 24) w = master[sur::kOffW1 + (k % 8) * kHid + n];
        else if (k == sur::kBiasCol) w = master[sur::kOffB1 + n];
        w1t[umma::kmajor_offset(n, k, 128) / 2] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
    }
    if (t < kHid * kHid) {  // W2 operand: B[n][k] = W2[k][n]
        const int n = t / kHid, k = t % kHid;
        w2t[umma::kmajor_offset(n, k, 128) / 2] =
            __bfloat16_as_ushort(__float2bfloat16_rn(master[sur::kOffW2 + k * kHid + n]));
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct SurState {
    int dev = 0;
    // network (device): FP32 masters (public layout), Adam moments, operand copies
    float *master = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    bf16 *W1b = nullptr, *W2b = nullptr;
    uint16_t *w1t = nullptr, *w2t = nullptr;
    double mu = 0.0, sigma = 1.0;
    sur::FeatConst fc{};
    unsigned long long fingerprint = 0;
    bool packed = false;
    // trust map for one tolerance and one grid
    uint32_t *trust = nullptr;
    float trust_tol = -1.0f;
    double trust_mask = -1.0;
    // scratch
    double2 *partials = nullptr;
    double *stats = nullptr;
    long long part_cap = 0;
    unsigned *timeout = nullptr;
    unsigned *bad = nullptr;      // input validity word
    float dom_max = -1.0f;        // largest ray solid angle of the context's grid
    float *q_ref = nullptr, *a_ref = nullptr;
    long long ref_cap = 0;
    std::vector<float> loss_hist;
};

void sur_free(SurState *s)
{
    if (!s) return;
    void *ptrs[] = {s->master, s->adam_m, s->adam_v, s->W1b, s->W2b, s->w1t, s->w2t, s->trust,
                    s->partials, s->stats, s->timeout, s->bad, s->q_ref, s->a_ref};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete s;
}

namespace {

#define SUR_CK(ctx, call)                                                                        \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return ctx_fail(ctx, RT_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

// reference opacities of the features: nearest bins in |ln nu| (first on ties)
bool feature_constants(const CtxInfo &in, sur::FeatConst *fc)
{
    auto nearest = [&](double nu) {
        int best = 0;
        double bd = INFINITY;
        for (int i = 0; i < in.n_nu; ++i) {
            const double d = fabs(log(in.nu_h[i]) - log(nu));
            if (d < bd) {
                bd = d;
                best = i;
            }
        }
        return in.kappa_h[best];
    };
    for (int m = 0; m < 6; ++m) fc->kref[m] = (float)nearest(1e11 * pow(10.0, m));
    fc->k550 = (float)nearest(kC / 550e-7);
    return fc->k550 > 0.0f;
}

int sur_alloc(rt_ctx *ctx, SurState **out)
{
    SurState *s = new SurState();
    cudaGetDevice(&s->dev);
    bool ok = cudaMalloc(&s->master, sizeof(float) * kNParams) == cudaSuccess &&
              cudaMalloc(&s->adam_m, sizeof(float) * kNParams) == cudaSuccess &&
              cudaMalloc(&s->adam_v, sizeof(float) * kNParams) == cudaSuccess &&
              cudaMalloc(&s->W1b, sizeof(bf16) * kK1 * kHid) == cudaSuccess &&
              cudaMalloc(&s->W2b, sizeof(bf16) * 2 * kHid * kHid) == cudaSuccess &&
              cudaMalloc(&s->w1t, 2 * kHid * kK1) == cudaSuccess &&
              cudaMalloc(&s->w2t, 2 * kHid * kHid) == cudaSuccess &&
              cudaMalloc(&s->trust, sizeof(uint32_t) * kTrustWords) == cudaSuccess &&
              cudaMalloc(&s->timeout, sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&s->bad, sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMemset(s->W1b, 0, sizeof(bf16) * kK1 * kHid) == cudaSuccess &&
         cudaMemset(s->adam_m, 0, sizeof(float) * kNParams) == cudaSuccess &&
         cudaMemset(s->adam_v, 0, sizeof(float) * kNParams) == cudaSuccess &&
         cudaMemset(s->timeout, 0, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        sur_free(s);
        return ctx_fail(ctx, RT_ERR_NO_MEMORY, "cannot allocate the surrogate's device state");
    }
    *out = s;
    return RT_OK;
}

// the BF16 copies for training and the tensor-core operands for inference
int sur_refresh(rt_ctx *ctx, SurState *s, cudaStream_t st)
{
    UpdateArgs u{};
    u.mode = 2;
    u.master = s->master;
    u.W1b = s->W1b;
    u.W2b = s->W2b;
    k_update<<<(kNParams + 255) / 256, 256, 0, st>>>(u);
    k_pack_infer<<<(kHid * kHid + 255) / 256, 256, 0, st>>>(s->master, s->w1t, s->w2t);
    SUR_CK(ctx, cudaGetLastError());
    s->packed = true;
    s->trust_tol = -1.0f;
    return RT_OK;
}

// Training-step workspace for minibatches of up to B rows.
struct Work {
    int B = 0, S = 0, G = 0;
    bf16 *Xb = nullptr, *H1 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    float *Tb = nullptr, *Z1 = nullptr, *Z2 = nullptr, *dW1p = nullptr, *dW2p = nullptr, *hp = nullptr;
    float *loss = nullptr, *grad = nullptr, *y = nullptr;
    ~Work()
    {
        void *ptrs[] = {Xb, H1, dZ2, dZ1, Tb, Z1, Z2, dW1p, dW2p, hp, loss, grad, y};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    }
    bool alloc(int b)
    {
        B = b;
        S = std::max(1, B / 256);
        G = std::min(128, std::max(1, B / (kHeadWarps * 8)));
        return cudaMalloc(&Xb, sizeof(bf16) * B * kK1) == cudaSuccess &&
               cudaMalloc(&H1, sizeof(bf16) * B * 2 * kHid) == cudaSuccess &&
               cudaMalloc(&dZ2, sizeof(bf16) * B * kHid) == cudaSuccess &&
               cudaMalloc(&dZ1, sizeof(bf16) * B * kHid) == cudaSuccess &&
               cudaMalloc(&Tb, sizeof(float) * B) == cudaSuccess &&
               cudaMalloc(&Z1, sizeof(float) * B * kHid) == cudaSuccess &&
               cudaMalloc(&Z2, sizeof(float) * B * kHid) == cudaSuccess &&
               cudaMalloc(&dW1p, sizeof(float) * S * kK1 * kHid) == cudaSuccess &&
               cudaMalloc(&dW2p, sizeof(float) * S * 2 * kHid * kHid) == cudaSuccess &&
               cudaMalloc(&hp, sizeof(float) * G * kHeadPart) == cudaSuccess &&
               cudaMalloc(&loss, sizeof(float)) == cudaSuccess &&
               cudaMalloc(&grad, sizeof(float) * kNParams) == cudaSuccess &&
               cudaMalloc(&y, sizeof(float) * B) == cudaSuccess;
    }
};

// Forward and backward of one minibatch already in w.Xb / w.Tb (n valid rows):
// leaves the split-K and head partials for k_update.
void fwd_bwd(SurState *s, Work &w, int n, cudaStream_t st)
{
    const int B = w.B;
    GemmArgs g{};
    // Z1 = Xb W1b, H1 = SiLU(Z1) (hi, lo)
    g.A = w.Xb; g.lda = kK1; g.B = s->W1b; g.ldb = kHid; g.M = B; g.K = kK1; g.kchunk = kK1;
    g.C = w.Z1; g.Cb = w.H1;
    k_gemm<false, false, kEpiZ1><<<dim3(B / 64, 1), 128, 0, st>>>(g);
    // Z2 = H1 [W2; W2] + b2
    g = GemmArgs{};
    g.A = w.H1; g.lda = 2 * kHid; g.B = s->W2b; g.ldb = kHid; g.M = B; g.K = 2 * kHid; g.kchunk = 2 * kHid;
    g.C = w.Z2; g.bias = s->master + sur::kOffB2;
    k_gemm<false, false, kEpiZ2><<<dim3(B / 64, 1), 128, 0, st>>>(g);
    // output layer, loss, dZ2
    k_head<<<w.G, kHeadWarps * 32, 0, st>>>(w.Z2, w.Tb, s->master, n, B, 2.0f / (float)n, w.dZ2, w.hp, w.y);
    // dZ1 = (dZ2 W2^T) SiLU'(Z1)
    g = GemmArgs{};
    g.A = w.dZ2; g.lda = kHid; g.B = s->W2b; g.ldb = kHid; g.M = B; g.K = kHid; g.kchunk = kHid;
    g.Cb = w.dZ1; g.aux = w.Z1;
    k_gemm<false, true, kEpiDZ1><<<dim3(B / 64, 1), 128, 0, st>>>(g);
    // dW2 partials = H1^T dZ2 over K slices of the batch
    const int kc = B / w.S;
    g = GemmArgs{};
    g.A = w.H1; g.lda = 2 * kHid; g.B = w.dZ2; g.ldb = kHid; g.M = 2 * kHid; g.K = B; g.kchunk = kc;
    g.C = w.dW2p;
    k_gemm<true, false, kEpiPart><<<dim3(2 * kHid / 64, w.S), 128, 0, st>>>(g);
    // dW1 partials = Xb^T dZ1
    g = GemmArgs{};
    g.A = w.Xb; g.lda = kK1; g.B = w.dZ1; g.ldb = kHid; g.M = kK1; g.K = B; g.kchunk = kc;
    g.C = w.dW1p;
    k_gemm<true, false, kEpiPart><<<dim3(1, w.S), 128, 0, st>>>(g);
}

UpdateArgs update_args(SurState *s, Work &w, int mode, int n)
{
    UpdateArgs u{};
    u.mode = mode;
    u.master = s->master;
    u.m = s->adam_m;
    u.v = s->adam_v;
    u.dW1p = w.dW1p;
    u.dW2p = w.dW2p;
    u.hp = w.hp;
    u.S = w.S;
    u.G = w.G;
    u.grad_out = w.grad;
    u.loss_out = w.loss;
    u.inv_n = 1.0f / (float)n;
    u.W1b = s->W1b;
    u.W2b = s->W2b;
    return u;
}

SurNet net_of(const SurState *s)
{
    SurNet n{};
    n.w1t = reinterpret_cast<const uint4 *>(s->w1t);
    n.w2t = reinterpret_cast<const uint4 *>(s->w2t);
    n.master = s->master;
    n.mu = (float)s->mu;
    n.sigma = (float)s->sigma;
    n.fc = s->fc;
    return n;
}

int set_smem(rt_ctx *ctx)
{
    static bool done[16] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 16 && done[dev]) return RT_OK;
    SUR_CK(ctx, cudaFuncSetAttribute(k_sur_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmDyn));
    SUR_CK(ctx, cudaFuncSetAttribute(k_sur_ray, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmDyn));
    if (dev < 16) done[dev] = true;
    return RT_OK;
}

// y = network(X) for n feature rows on the device (inference arithmetic)
int eval_rows(rt_ctx *ctx, SurState *s, const float *X, int n, float *y, cudaStream_t st)
{
    int rc = set_smem(ctx);
    if (rc != RT_OK) return rc;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->dev);
    const int ntiles = (n + 127) / 128;
    const int grid = std::max(1, std::min(ntiles, nsm));
    SUR_CK(ctx, cudaMemsetAsync(s->timeout, 0, sizeof(unsigned), st));
    k_sur_eval<<<grid, kInfThreads, kSmDyn, st>>>(net_of(s), X, n, y, s->timeout);
    SUR_CK(ctx, cudaGetLastError());
    unsigned to = 0;
    SUR_CK(ctx, cudaMemcpyAsync(&to, s->timeout, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SUR_CK(ctx, cudaStreamSynchronize(st));
    if (to) return ctx_fail(ctx, RT_ERR_TIMEOUT, "tensor-core product did not complete within the bounded wait");
    return RT_OK;
}

double acc_mask_of(const CtxInfo &in)
{
    // a cell is judged when it absorbs more than 1e-12 of the star's power
    // reaching the grid: acc dOmega R*^2 F_max > 1e-12 L_grid
    return 1e-12 * in.sc.l_grid / (in.sc.r2 * in.sc.f_max);
}

int build_trust(rt_ctx *ctx, SurState *s, const CtxInfo &in, float tol, float dom_max, cudaStream_t st)
{
    const int npts = kTrustBins * kTrustBins * kTrustSamples;
    float *X = nullptr, *y = nullptr;
    float2 *nd = nullptr;
    if (cudaMalloc(&X, sizeof(float) * npts * kNF) != cudaSuccess || cudaMalloc(&y, sizeof(float) * npts) != cudaSuccess ||
        cudaMalloc(&nd, sizeof(float2) * npts) != cudaSuccess) {
        cudaFree(X);
        cudaFree(y);
        cudaFree(nd);
        cudaGetLastError();
        return ctx_fail(ctx, RT_ERR_NO_MEMORY, "trust map scratch");
    }
    k_trust_points<<<(npts + 255) / 256, 256, 0, st>>>(s->fc, (float)in.t_sub, 12345ULL, X, nd);
    int rc = eval_rows(ctx, s, X, npts, y, st);
    if (rc == RT_OK) {
        const double mask = acc_mask_of(in);
        cudaMemsetAsync(s->trust, 0, sizeof(uint32_t) * kTrustWords, st);
        k_trust_judge<<<kTrustBins * kTrustBins / 8, 256, 0, st>>>(nd, y, (float)s->mu, (float)s->sigma, in.nu_tab,
                                                                  in.kap, in.sc.n_active, s->fc.k550, tol,
                                                                  (float)(mask / dom_max), s->trust);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
            rc = ctx_fail(ctx, RT_ERR_CUDA, "trust map kernels");
        else {
            s->trust_tol = tol;
            s->trust_mask = mask / dom_max;
        }
    }
    cudaFree(X);
    cudaFree(y);
    cudaFree(nd);
    return rc;
}

int begin(rt_ctx *ctx, CtxInfo *in)
{
    if (!ctx) return RT_ERR_INVALID_ARG;
    ctx_info(ctx, in);
    if (!in->configured) return ctx_fail(ctx, RT_ERR_NOT_CONFIGURED, "call rt_set_star and rt_set_opacity_table first");
    if (in->n_t > 0)
        return ctx_fail(ctx, RT_ERR_INVALID_ARG,
                        "the surrogate's inputs assume a temperature-independent table (rt_set_opacity_table)");
    if (cudaSetDevice(in->dev) != cudaSuccess) return ctx_fail(ctx, RT_ERR_CUDA, "cudaSetDevice");
    return RT_OK;
}

int need_surrogate(rt_ctx *ctx, const CtxInfo &in, SurState **s)
{
    *s = ctx_surrogate(ctx);
    if (!*s) return ctx_fail(ctx, RT_ERR_NOT_CONFIGURED, "no surrogate: train, load or set its parameters first");
    if ((*s)->fingerprint != in.table_fingerprint)
        return ctx_fail(ctx, RT_ERR_NOT_CONFIGURED,
                        "the surrogate was made for another opacity table, sublimation temperature or star");
    return RT_OK;
}

// a fresh surrogate bound to this context's table
int sur_create(rt_ctx *ctx, const CtxInfo &in, SurState **out)
{
    sur::FeatConst fc;
    if (!feature_constants(in, &fc))
        return ctx_fail(ctx, RT_ERR_INVALID_ARG, "the opacity at 550 nm is zero: the surrogate's inputs are undefined");
    SurState *&slot = ctx_surrogate(ctx);
    if (slot) {
        sur_free(slot);
        slot = nullptr;
    }
    int rc = sur_alloc(ctx, &slot);
    if (rc != RT_OK) return rc;
    slot->fc = fc;
    slot->fingerprint = in.table_fingerprint;
    *out = slot;
    return RT_OK;
}

float dom_max_of(rt_ctx *ctx, const CtxInfo &in)
{
    std::vector<float> d((size_t)in.nrays);
    if (cudaMemcpy(d.data(), in.domega32, sizeof(float) * in.nrays, cudaMemcpyDeviceToHost) != cudaSuccess) return -1.0f;
    float m = 0.0f;
    for (float v : d) m = std::max(m, v);
    (void)ctx;
    return m;
}

}  // namespace
}  // namespace rt

using namespace rt;

extern "C" {

int rt_surrogate_set_params(rt_ctx *ctx, const float *params, double mu, double sigma)
{
    CtxInfo in;
    int rc = begin(ctx, &in);
    if (rc != RT_OK) return rc;
    if (!params || !(sigma > 0.0) || !isfinite(mu) || !isfinite(sigma))
        return ctx_fail(ctx, RT_ERR_INVALID_ARG, "params must be non-NULL, sigma > 0 and finite");
    for (int i = 0; i < kNParams; ++i)
        if (!isfinite(params[i])) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "non-finite parameter");
    SurState *s = ctx_surrogate(ctx);
    if (!s || s->fingerprint != in.table_fingerprint) {
        rc = sur_create(ctx, in, &s);
        if (rc != RT_OK) return rc;
    }
    SUR_CK(ctx, cudaMemcpyAsync(s->master, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice, in.stream));
    s->mu = mu;
    s->sigma = sigma;
    rc = sur_refresh(ctx, s, in.stream);
    if (rc != RT_OK) return rc;
    SUR_CK(ctx, cudaStreamSynchronize(in.stream));
    return RT_OK;
}

int rt_surrogate_get_params(rt_ctx *ctx, float *params, double *mu, double *sigma)
{
    CtxInfo in;
    int rc = begin(ctx, &in);
    if (rc != RT_OK) return rc;
    if (!params) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "params is NULL");
    SurState *s = ctx_surrogate(ctx);
    if (!s) return ctx_fail(ctx, RT_ERR_NOT_CONFIGURED, "no surrogate");
    SUR_CK(ctx, cudaMemcpyAsync(params, s->master, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, in.stream));
    SUR_CK(ctx, cudaStreamSynchronize(in.stream));
    if (mu) *mu = s->mu;
    if (sigma) *sigma = s->sigma;
    return RT_OK;
}

int rt_surrogate_grad(rt_ctx *ctx, const float *x, const float *t, int n, float *grad, double *loss)
{
    CtxInfo in;
    int rc = begin(ctx, &in);
    if (rc != RT_OK) return rc;
    if (!x || !t || !grad || n < 1 || n > (1 << 20)) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "need 1 <= n <= 2^20 and non-NULL buffers");
    SurState *s = nullptr;
    rc = need_surrogate(ctx, in, &s);
    if (rc != RT_OK) return rc;
    const int B = ((n + 255) / 256) * 256;
    Work w;
    if (!w.alloc(B)) {
        cudaGetLastError();
        return ctx_fail(ctx, RT_ERR_NO_MEMORY, "gradient workspace");
    }
    float *xd = nullptr, *td = nullptr;
    if (cudaMalloc(&xd, sizeof(float) * n * kNF) != cudaSuccess || cudaMalloc(&td, sizeof(float) * n) != cudaSuccess) {
        cudaFree(xd);
        cudaGetLastError();
        return ctx_fail(ctx, RT_ERR_NO_MEMORY, "gradient inputs");
    }
    cudaStream_t st = in.stream;
    cudaMemcpyAsync(xd, x, sizeof(float) * n * kNF, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(td, t, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    k_rows<<<(B + 255) / 256, 256, 0, st>>>(xd, td, n, B, w.Xb, w.Tb);
    fwd_bwd(s, w, n, st);
    k_update<<<(kNParams + 255) / 256, 256, 0, st>>>(update_args(s, w, 0, n));
    float lh = 0.0f;
    cudaMemcpyAsync(grad, w.grad, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&lh, w.loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(xd);
    cudaFree(td);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return ctx_fail(ctx, RT_ERR_CUDA, std::string("gradient kernels: ") + cudaGetErrorString(e));
    if (loss) *loss = lh;
    return RT_OK;
}

int rt_surrogate_eval(rt_ctx *ctx, const float *x, int n, float *y)
{
    CtxInfo in;
    int rc = begin(ctx, &in);
    if (rc != RT_OK) return rc;
    if (!x || !y || n < 1 || n > (1 << 26)) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "need 1 <= n <= 2^26 and non-NULL buffers");
    SurState *s = nullptr;
    rc = need_surrogate(ctx, in, &s);
    if (rc != RT_OK) return rc;
    float *xd = nullptr, *yd = nullptr;
    if (cudaMalloc(&xd, sizeof(float) * (size_t)n * kNF) != cudaSuccess || cudaMalloc(&yd, sizeof(float) * n) != cudaSuccess) {
        cudaFree(xd);
        cudaGetLastError();
        return ctx_fail(ctx, RT_ERR_NO_MEMORY, "evaluation buffers");
    }
    cudaMemcpyAsync(xd, x, sizeof(float) * (size_t)n * kNF, cudaMemcpyHostToDevice, in.stream);
    rc = eval_rows(ctx, s, xd, n, yd, in.stream);
    if (rc == RT_OK) {
        cudaMemcpyAsync(y, yd, sizeof(float) * n, cudaMemcpyDeviceToHost, in.stream);
        if (cudaStreamSynchronize(in.stream) != cudaSuccess) rc = ctx_fail(ctx, RT_ERR_CUDA, "evaluation copy");
    }
    cudaFree(xd);
    cudaFree(yd);
    return rc;
}

int rt_surrogate_train(rt_ctx *ctx, const rt_train_cfg *cfg, const float *const *rho, const float *const *t_dust,
                       int ngrids, rt_train_stats *stats)
{
    CtxInfo in;
    int rc = begin(ctx, &in);
    if (rc != RT_OK) return rc;
    if (!cfg || !rho || !t_dust || ngrids < 1) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "cfg, rho, t_dust and ngrids >= 1 required");
    for (int i = 0; i < ngrids; ++i)
        if (!rho[i] || !t_dust[i]) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "NULL training field");
    const long long n_target = cfg->n_samples > 0 ? cfg->n_samples : 20000000LL;
    const int B = cfg->batch > 0 ? cfg->batch : 8192;
    const int steps = cfg->steps > 0 ? cfg->steps : 30000;
    const float lr = cfg->lr > 0.0f ? cfg->lr : 2e-3f;
    if (B % 256 != 0 || B > (1 << 20)) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "batch must be a multiple of 256, at most 2^20");
    SurState *s = nullptr;
    rc = sur_create(ctx, in, &s);
    if (rc != RT_OK) return rc;
    cudaStream_t st = in.stream;

    // scratch: one grid's exact outputs, per-ray counts and offsets
    const long long nc = in.ncells, nrays = in.nrays;
    float *q = nullptr, *a = nullptr;
    unsigned *cnt = nullptr;
    long long *off = nullptr, *base = nullptr;
    bool ok = cudaMalloc(&q, sizeof(float) * nc) == cudaSuccess && cudaMalloc(&a, sizeof(float) * nc) == cudaSuccess &&
              cudaMalloc(&cnt, sizeof(unsigned) * 2 * nrays) == cudaSuccess &&
              cudaMalloc(&off, sizeof(long long) * 2 * nrays) == cudaSuccess &&
              cudaMalloc(&base, sizeof(long long) * 2) == cudaSuccess;
    float *X = nullptr, *Y = nullptr, *Xv = nullptr, *Yv = nullptr;
    auto cleanup = [&]() {
        void *ptrs[] = {q, a, cnt, off, base, X, Y, Xv, Yv};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    };
    if (!ok) {
        cleanup();
        cudaGetLastError();
        return ctx_fail(ctx, RT_ERR_NO_MEMORY, "training scratch");
    }
    CollectArgs ca{};
    ca.rtab = in.rtab;
    ca.domega32 = in.domega32;
    ca.nr = in.nr;
    ca.nrays = nrays;
    ca.t_sub = (float)in.t_sub;
    ca.acc_mask = (float)acc_mask_of(in);
    ca.fc = s->fc;
    ca.seed = cfg->seed;
    ca.cnt = cnt;
    ca.off = off;
    ca.q = q;
    const int cb = 128, cg = (int)((nrays + cb - 1) / cb);
    std::vector<unsigned> cnt_h((size_t)2 * nrays);

    // pass 0: eligible cells of every grid (the exact tracer judges each cell)
    long long eligible = 0;
    for (int gi = 0; gi < ngrids && rc == RT_OK; ++gi) {
        rc = rt_irradiate(ctx, rho[gi], t_dust[gi], q, a, nullptr);
        if (rc != RT_OK) break;
        ca.pass = 0;
        ca.rho = rho[gi];
        ca.tdust = t_dust[gi];
        k_collect<<<cg, cb, 0, st>>>(ca);
        if (cudaMemcpyAsync(cnt_h.data(), cnt, sizeof(unsigned) * 2 * nrays, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = ctx_fail(ctx, RT_ERR_CUDA, "sample count");
            break;
        }
        for (long long i = 0; i < nrays; ++i) eligible += cnt_h[2 * i];
    }
    if (rc == RT_OK && eligible < 1024) rc = ctx_fail(ctx, RT_ERR_INVALID_ARG, "fewer than 1024 cells absorb enough to train on");
    if (rc != RT_OK) {
        cleanup();
        return rc;
    }
    // at most 95 % of the eligible cells train; a held-out share of 2-5 % judges
    ca.p_keep = (float)std::min(0.95, (double)n_target / (double)eligible);
    ca.p_val = (float)std::min(1.0 - ca.p_keep, std::max(0.02, 0.05 * ca.p_keep));
    // passes 1 and 2: select, count, scan, write
    long long n_train = 0, n_val = 0;
    for (int round = 0; round < 2 && rc == RT_OK; ++round) {
        if (round == 1) {
            if (cudaMalloc(&X, sizeof(float) * kNF * std::max(1LL, n_train)) != cudaSuccess ||
                cudaMalloc(&Y, sizeof(float) * std::max(1LL, n_train)) != cudaSuccess ||
                cudaMalloc(&Xv, sizeof(float) * kNF * std::max(1LL, n_val)) != cudaSuccess ||
                cudaMalloc(&Yv, sizeof(float) * std::max(1LL, n_val)) != cudaSuccess) {
                cudaGetLastError();
                rc = ctx_fail(ctx, RT_ERR_NO_MEMORY, "training set");
                break;
            }
            ca.X = X;
            ca.Y = Y;
            ca.Xv = Xv;
            ca.Yv = Yv;
            ca.cap_train = n_train;
            ca.cap_val = n_val;
        }
        cudaMemsetAsync(base, 0, sizeof(long long) * 2, st);
        for (int gi = 0; gi < ngrids && rc == RT_OK; ++gi) {
            rc = rt_irradiate(ctx, rho[gi], t_dust[gi], q, a, nullptr);
            if (rc != RT_OK) break;
            ca.rho = rho[gi];
            ca.tdust = t_dust[gi];
            ca.cell_base = (long long)gi * nc;
            ca.pass = 1;
            k_collect<<<cg, cb, 0, st>>>(ca);
            k_scan_counts<<<1, 1024, 0, st>>>(cnt, nrays, off, base);
            if (round == 1) {
                ca.pass = 2;
                k_collect<<<cg, cb, 0, st>>>(ca);
            }
        }
        if (rc != RT_OK) break;
        long long tot[2] = {0, 0};
        if (cudaMemcpyAsync(tot, base, sizeof(tot), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = ctx_fail(ctx, RT_ERR_CUDA, "sample selection");
            break;
        }
        // the second round selects the same cells; never count past what was allocated
        n_train = round == 0 ? tot[0] : std::min(tot[0], ca.cap_train);
        n_val = round == 0 ? tot[1] : std::min(tot[1], ca.cap_val);
    }
    if (rc == RT_OK && n_train < 256) rc = ctx_fail(ctx, RT_ERR_INVALID_ARG, "too few training cells selected");
    if (rc != RT_OK) {
        cleanup();
        return rc;
    }

    // standardisation of the targets
    double mom[2] = {0.0, 1.0};
    {
        double *md = nullptr;
        cudaMalloc(&md, sizeof(double) * 2);
        k_moments<<<1, 1024, 0, st>>>(Y, n_train, md);
        cudaMemcpyAsync(mom, md, sizeof(mom), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        cudaFree(md);
    }
    s->mu = mom[0];
    s->sigma = mom[1];

    // initial parameters: uniform fan-in initialisation from a counter hash, zero biases
    std::vector<float> init(kNParams, 0.0f);
    for (int i = 0; i < kNParams; ++i) {
        float fan = 0.0f;
        if (i < sur::kOffB1) fan = (float)kNF;
        else if (i >= sur::kOffW2 && i < sur::kOffB2) fan = (float)kHid;
        else if (i >= sur::kOffW3 && i < sur::kOffB3) fan = (float)kHid;
        if (fan > 0.0f) init[i] = (2.0f * sur::u01(cfg->seed, 99, (uint64_t)i) - 1.0f) / sqrtf(fan);
    }
    SUR_CK(ctx, cudaMemcpyAsync(s->master, init.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice, st));
    rc = sur_refresh(ctx, s, st);
    if (rc != RT_OK) {
        cleanup();
        return rc;
    }

    Work w;
    if (!w.alloc(B)) {
        cleanup();
        cudaGetLastError();
        return ctx_fail(ctx, RT_ERR_NO_MEMORY, "training workspace");
    }
    float *loss_d = nullptr;
    cudaMalloc(&loss_d, sizeof(float) * steps);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    const float inv_sigma = (float)(1.0 / s->sigma);
    const int warm = std::max(1, steps / 50);
    double c1 = 1.0, c2 = 1.0;
    for (int step = 0; step < steps; ++step) {
        // linear warm-up, then cosine decay to 1 % of the peak rate
        float lr_t;
        if (step < warm) lr_t = lr * (float)(step + 1) / (float)warm;
        else {
            const double ph = (double)(step - warm) / (double)std::max(1, steps - warm);
            lr_t = (float)(lr * (0.01 + 0.99 * 0.5 * (1.0 + cos(kPi * ph))));
        }
        c1 *= 0.9;
        c2 *= 0.999;
        k_gather<<<(B + 255) / 256, 256, 0, st>>>(X, Y, n_train, (float)s->mu, inv_sigma, cfg->seed, step, B, B,
                                                  w.Xb, w.Tb);
        fwd_bwd(s, w, B, st);
        UpdateArgs u = update_args(s, w, 1, B);
        u.lr = lr_t;
        u.c1 = (float)(1.0 - c1);
        u.c2 = (float)(1.0 - c2);
        u.loss_out = loss_d + step;
        k_update<<<(kNParams + 255) / 256, 256, 0, st>>>(u);
    }
    cudaEventRecord(e1, st);
    SUR_CK(ctx, cudaGetLastError());
    s->loss_hist.assign(steps, 0.0f);
    cudaMemcpyAsync(s->loss_hist.data(), loss_d, sizeof(float) * steps, cudaMemcpyDeviceToHost, st);
    rc = sur_refresh(ctx, s, st);
    float train_ms = 0.0f;
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = ctx_fail(ctx, RT_ERR_CUDA, "training loop");
    cudaEventElapsedTime(&train_ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(loss_d);

    // held-out error of ln g with the inference arithmetic
    double vrms = 0.0, vmax = 0.0;
    if (rc == RT_OK && n_val > 0) {
        float *yv = nullptr;
        if (cudaMalloc(&yv, sizeof(float) * n_val) == cudaSuccess) {
            rc = eval_rows(ctx, s, Xv, (int)std::min<long long>(n_val, 1LL << 26), yv, st);
            if (rc == RT_OK) {
                std::vector<float> yh((size_t)n_val), th((size_t)n_val);
                cudaMemcpy(yh.data(), yv, sizeof(float) * n_val, cudaMemcpyDeviceToHost);
                cudaMemcpy(th.data(), Yv, sizeof(float) * n_val, cudaMemcpyDeviceToHost);
                for (long long i = 0; i < n_val; ++i) {
                    const double err = fabs(s->mu + s->sigma * (double)yh[i] - (double)th[i]);
                    vrms += err * err;
                    vmax = std::max(vmax, err);
                }
                vrms = sqrt(vrms / (double)n_val);
            }
            cudaFree(yv);
        } else {
            cudaGetLastError();
        }
    }
    cleanup();
    if (rc != RT_OK) return rc;
    if (stats) {
        stats->n_train = n_train;
        stats->n_val = n_val;
        stats->mu = s->mu;
        stats->sigma = s->sigma;
        double fl = 0.0;
        const int tail = std::max(1, steps / 100);
        for (int i = steps - tail; i < steps; ++i) fl += s->loss_hist[i];
        stats->final_loss = fl / tail;
        stats->val_rms = vrms;
        stats->val_max = vmax;
        stats->train_ms = train_ms;
    }
    return RT_OK;
}

int rt_surrogate_loss_history(rt_ctx *ctx, float *loss, int max)
{
    if (!ctx || max < 0 || (max > 0 && !loss)) return RT_ERR_INVALID_ARG;
    SurState *s = ctx_surrogate(ctx);
    if (!s) return ctx_fail(ctx, RT_ERR_NOT_CONFIGURED, "no surrogate");
    const int n = (int)s->loss_hist.size();
    for (int i = 0; i < n && i < max; ++i) loss[i] = s->loss_hist[i];
    return n;
}

int rt_irradiate_surrogate(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs, float *a_rad,
                           float err_tol, int validate, rt_surrogate_stats *stats)
{
    CtxInfo in;
    int rc = begin(ctx, &in);
    if (rc != RT_OK) return rc;
    if (!rho || !t_dust || !q_abs || !a_rad) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "NULL field pointer");
    if (validate < 0 || validate > 2) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "validate must be 0, 1 or 2");
    if (!(err_tol > 0.0f) || !isfinite(err_tol)) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "err_tol must be > 0");
    if (in.nr < 1 || in.ncells >= (1LL << 31)) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "the surrogate path takes grids below 2^31 cells");
    SurState *s = nullptr;
    rc = need_surrogate(ctx, in, &s);
    if (rc != RT_OK) return rc;
    cudaStream_t st = in.stream;
    rc = set_smem(ctx);
    if (rc != RT_OK) return rc;
    const double mask = acc_mask_of(in);
    if (validate == 0) {
        if (!(s->dom_max > 0.0f)) s->dom_max = dom_max_of(ctx, in);
        const float dom_max = s->dom_max;
        if (!(dom_max > 0.0f)) return ctx_fail(ctx, RT_ERR_CUDA, "solid angles");
        if (s->trust_tol != err_tol || s->trust_mask != mask / dom_max) {
            rc = build_trust(ctx, s, in, err_tol, dom_max, st);
            if (rc != RT_OK) return rc;
        }
    } else if (validate == 1) {
        if (s->ref_cap < in.ncells) {
            if (s->q_ref) cudaFree(s->q_ref);
            if (s->a_ref) cudaFree(s->a_ref);
            s->q_ref = s->a_ref = nullptr;
            s->ref_cap = 0;
            if (cudaMalloc(&s->q_ref, sizeof(float) * in.ncells) != cudaSuccess ||
                cudaMalloc(&s->a_ref, sizeof(float) * in.ncells) != cudaSuccess) {
                cudaGetLastError();
                return ctx_fail(ctx, RT_ERR_NO_MEMORY, "validation buffers");
            }
            s->ref_cap = in.ncells;
        }
        rc = rt_irradiate(ctx, rho, t_dust, s->q_ref, s->a_ref, nullptr);
        if (rc != RT_OK) return rc;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, in.dev);
    const unsigned ntiles = (unsigned)((in.ncells + 127) / 128);
    const int grid = (int)std::max(1u, std::min(ntiles, (unsigned)(2 * nsm)));
    if (s->part_cap < grid) {
        if (s->partials) cudaFree(s->partials);
        if (s->stats) cudaFree(s->stats);
        s->partials = nullptr;
        s->stats = nullptr;
        s->part_cap = 0;
        if (cudaMalloc(&s->partials, sizeof(double2) * grid) != cudaSuccess ||
            cudaMalloc(&s->stats, sizeof(double) * 5 * grid) != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(ctx, RT_ERR_NO_MEMORY, "surrogate partials");
        }
        s->part_cap = grid;
    }
    // validity word of the inputs, cleared for this call
    unsigned *bad = s->bad;
    cudaMemsetAsync(bad, 0, sizeof(unsigned), st);
    cudaMemsetAsync(s->timeout, 0, sizeof(unsigned), st);
    SurRayArgs p{};
    p.rho = rho;
    p.tdust = t_dust;
    p.q = q_abs;
    p.a = a_rad;
    p.q_ref = s->q_ref;
    p.a_ref = s->a_ref;
    p.rtab = in.rtab;
    p.domega32 = in.domega32;
    p.nu = in.nu_tab;
    p.kap = in.kap;
    p.n_active = in.sc.n_active;
    p.nnu_pad = in.sc.nnu_pad;
    p.trust = validate == 0 ? s->trust : nullptr;
    p.net = net_of(s);
    p.tol = err_tol;
    p.acc_mask = (float)mask;
    p.t_sub = (float)in.t_sub;
    p.mode = validate;
    p.partials = s->partials;
    p.stats = s->stats;
    p.bad_input = bad;
    p.seq = 1u;
    p.timeout = s->timeout;
    p.ncells = (unsigned)in.ncells;
    p.nr = (unsigned)in.nr;
    p.ntiles = ntiles;
    p.nrdiv = FastDiv::make((unsigned)in.nr);
    k_sur_ray<<<grid, kInfThreads, kSmDyn, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return ctx_fail(ctx, RT_ERR_CUDA, std::string("surrogate kernel launch: ") + cudaGetErrorString(e));
    if (!stats) return RT_OK;  // asynchronous, like rt_irradiate
    std::vector<double2> part(grid);
    std::vector<double> sth((size_t)5 * grid);
    unsigned bad_h = 0, to = 0;
    cudaMemcpyAsync(part.data(), s->partials, sizeof(double2) * grid, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(sth.data(), s->stats, sizeof(double) * 5 * grid, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&bad_h, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&to, s->timeout, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ctx_fail(ctx, RT_ERR_CUDA, std::string("surrogate kernel: ") + cudaGetErrorString(e));
    if (to) return ctx_fail(ctx, RT_ERR_TIMEOUT, "tensor-core product did not complete within the bounded wait");
    if (bad_h == p.seq) return ctx_fail(ctx, RT_ERR_NONFINITE_INPUT, "input field holds NaN/Inf/negative density or NaN temperature");
    double sa = 0.0, se = 0.0, sd = 0.0, sf = 0.0, sj = 0.0, ss = 0.0, sm = 0.0;
    for (int i = 0; i < grid; ++i) {
        sa += part[i].x;
        se += part[i].y;
        sd += sth[5 * i];
        sf += sth[5 * i + 1];
        sj += sth[5 * i + 2];
        ss += sth[5 * i + 3];
        sm = std::max(sm, sth[5 * i + 4]);
    }
    const double scale = in.sc.r2 * in.sc.f_max;
    stats->n_dust = (long long)sd;
    stats->n_fallback = (long long)sf;
    stats->n_judged = (long long)sj;
    stats->max_rel_err = sm;
    stats->mean_rel_err = sj > 0 ? ss / sj : 0.0;
    stats->e_abs = scale * sa;
    stats->e_esc = scale * se + in.sc.r2 * in.sc.f_transparent * in.sc.sum_domega;
    stats->rel_err = (stats->e_abs + stats->e_esc) / in.sc.l_grid - 1.0;
    return RT_OK;
}

int rt_surrogate_trust_map(rt_ctx *ctx, float err_tol, unsigned *bits, float *ranges)
{
    CtxInfo in;
    int rc = begin(ctx, &in);
    if (rc != RT_OK) return rc;
    if (!bits || !(err_tol > 0.0f)) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "bits must be non-NULL and err_tol > 0");
    SurState *s = nullptr;
    rc = need_surrogate(ctx, in, &s);
    if (rc != RT_OK) return rc;
    if (!(s->dom_max > 0.0f)) s->dom_max = dom_max_of(ctx, in);
    const float dom_max = s->dom_max;
    if (!(dom_max > 0.0f)) return ctx_fail(ctx, RT_ERR_CUDA, "solid angles");
    rc = build_trust(ctx, s, in, err_tol, dom_max, in.stream);
    if (rc != RT_OK) return rc;
    SUR_CK(ctx, cudaMemcpy(bits, s->trust, sizeof(uint32_t) * kTrustWords, cudaMemcpyDeviceToHost));
    if (ranges) {
        ranges[0] = kTrustU0;
        ranges[1] = kTrustDU;
        ranges[2] = kTrustV0;
        ranges[3] = kTrustDV;
    }
    return RT_OK;
}

// File: "RTSURR01", the table fingerprint, mu, sigma, the feature constants, then
// the FP32 parameters in the public flat order.
int rt_surrogate_save(rt_ctx *ctx, const char *path)
{
    CtxInfo in;
    int rc = begin(ctx, &in);
    if (rc != RT_OK) return rc;
    if (!path) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "path is NULL");
    SurState *s = ctx_surrogate(ctx);
    if (!s) return ctx_fail(ctx, RT_ERR_NOT_CONFIGURED, "no surrogate");
    std::vector<float> prm(kNParams);
    SUR_CK(ctx, cudaMemcpy(prm.data(), s->master, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    if (!f) return ctx_fail(ctx, RT_ERR_INVALID_ARG, std::string("cannot open ") + path);
    const char magic[8] = {'R', 'T', 'S', 'U', 'R', 'R', '0', '1'};
    const int np = kNParams;
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&s->fingerprint, sizeof(s->fingerprint), 1, f) == 1 &&
              fwrite(&s->mu, sizeof(double), 1, f) == 1 && fwrite(&s->sigma, sizeof(double), 1, f) == 1 &&
              fwrite(&s->fc, sizeof(s->fc), 1, f) == 1 && fwrite(&np, sizeof(int), 1, f) == 1 &&
              fwrite(prm.data(), sizeof(float), kNParams, f) == (size_t)kNParams;
    ok = (fclose(f) == 0) && ok;
    return ok ? RT_OK : ctx_fail(ctx, RT_ERR_INVALID_ARG, std::string("write failed: ") + path);
}

int rt_surrogate_load(rt_ctx *ctx, const char *path)
{
    CtxInfo in;
    int rc = begin(ctx, &in);
    if (rc != RT_OK) return rc;
    if (!path) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "path is NULL");
    FILE *f = fopen(path, "rb");
    if (!f) return ctx_fail(ctx, RT_ERR_INVALID_ARG, std::string("cannot open ") + path);
    char magic[8];
    unsigned long long fp = 0;
    double mu = 0.0, sigma = 0.0;
    sur::FeatConst fc;
    int np = 0;
    std::vector<float> prm(kNParams);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "RTSURR01", 8) == 0 &&
              fread(&fp, sizeof(fp), 1, f) == 1 && fread(&mu, sizeof(double), 1, f) == 1 &&
              fread(&sigma, sizeof(double), 1, f) == 1 && fread(&fc, sizeof(fc), 1, f) == 1 &&
              fread(&np, sizeof(int), 1, f) == 1 && np == kNParams &&
              fread(prm.data(), sizeof(float), kNParams, f) == (size_t)kNParams;
    fclose(f);
    if (!ok) return ctx_fail(ctx, RT_ERR_INVALID_ARG, std::string("not a surrogate file: ") + path);
    if (fp != in.table_fingerprint)
        return ctx_fail(ctx, RT_ERR_NOT_CONFIGURED, "the file's surrogate was made for another opacity table or star");
    return rt_surrogate_set_params(ctx, prm.data(), mu, sigma);
}

}  // extern "C"
