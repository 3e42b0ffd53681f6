// fpt_mlp.cuh -- device side of the learned importance-sampling proposal.
//
// alpha(x, pi, N) = clamp((o1 + t o2) / sqrt(1 + t^2), +-alpha_max), with
// (o1, o2) = W3 silu(W2 silu(W1 s + b1) + b2) + b3, s the normalised state
// and t = tan(theta_n): the bias amplitude along the noise vector (1, t) of
// the 1-D-noise system (Sec. 4.1 of arXiv:2410.13683: the bias must lie along
// (1, tan theta_n) for the two one-dimensional weights to agree).
//
// One warp evaluates 32 trajectories (two 16-row M tiles) with
// mma.sync.m16n8k16 (bf16 operands, fp32 accumulation). The accumulator
// fragment of one layer is, element for element, the A fragment of the next
// (rows g, g+8; columns 2t, 2t+1 of each 8-wide N tile), so activations stay
// in registers between layers.
//
// Packed weights ("blob", 16-byte aligned, kMlpBlobBytes): 44 fragment tiles
// of 32 lanes x uint2 (layer 1: 8 N tiles x 1 K tile; layer 2: 8 x 4; layer 3:
// 1 x 4), tile (nt, kt) lane (g, t) holding
//   .x = bf16x2(B[16kt + 2t][8nt + g], B[16kt + 2t + 1][8nt + g]),
//   .y = bf16x2(B[16kt + 2t + 8][8nt + g], B[16kt + 2t + 9][8nt + g]),
// B[k][n] = W[n][k] zero-padded (layer-1 inputs 3 -> 16, layer-3 outputs 2 -> 8);
// then fp32 biases b1[64], b2[64], b3[8] (b3[2..7] = 0).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace fpt_dev {

constexpr int kMlpIn = 3, kMlpH = 64, kMlpOut = 2;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpOut * kMlpH + kMlpOut;  // 4546
constexpr int kTilesL1 = 8, kTilesL2 = 32, kTilesL3 = 4;
constexpr int kMlpTiles = kTilesL1 + kTilesL2 + kTilesL3;                 // 44
constexpr int kMlpBiasFloats = kMlpH + kMlpH + 8;                          // 136
constexpr int kMlpBlobBytes = kMlpTiles * 32 * 8 + kMlpBiasFloats * 4;    // 11808

// Offsets of the canonical fp32 parameter vector (row-major (out, in)).
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpH * kMlpIn, kOffW2 = kOffB1 + kMlpH,
              kOffB2 = kOffW2 + kMlpH * kMlpH, kOffW3 = kOffB2 + kMlpH, kOffB3 = kOffW3 + kMlpOut * kMlpH;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float d[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                               uint32_t a3, uint2 b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b.x), "r"(b.y));
}

// silu(v) = v sigmoid(v) = v / (1 + e^{-v}), with the hardware exponential and
// reciprocal (relative error ~1e-7). The activations are rounded to bf16 next,
// so the SiLU's own error decides how often that rounding goes the other way
// than for the exact function: at ~1e-7 only values within ~1e-7 of a rounding
// boundary are affected (a tanh.approx-based sigmoid, with ~2^-11 relative
// error, changed about one activation in eight).
__device__ __forceinline__ float silu_f(float v)
{
    return __fdividef(v, 1.0f + __expf(-v));
}

// MLP outputs (o1, o2) of this lane's trajectory; all 32 lanes must call.
// `tiles` / `bias` may point to shared or global memory.
__device__ __forceinline__ void mlp_forward_warp(const uint2 *tiles, const float *bias, float in0,
                                                 float in1, float in2, float &o1, float &o2)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float *b1 = bias, *b2 = bias + kMlpH, *b3 = bias + 2 * kMlpH;
    o1 = 0.0f;
    o2 = 0.0f;
#pragma unroll 1
    for (int m = 0; m < 2; ++m) {
        const int r0 = 16 * m + g, r1 = r0 + 8;
        const float x0 = __shfl_sync(FULL, in0, r0), y0 = __shfl_sync(FULL, in1, r0), z0 = __shfl_sync(FULL, in2, r0);
        const float x1 = __shfl_sync(FULL, in0, r1), y1 = __shfl_sync(FULL, in1, r1), z1 = __shfl_sync(FULL, in2, r1);
        // layer-1 A fragment: row r, columns (2t, 2t+1) of (s0, s1, s2, 0, ..., 0)
        const uint32_t a0 = pack_bf16x2(t == 0 ? x0 : (t == 1 ? z0 : 0.0f), t == 0 ? y0 : 0.0f);
        const uint32_t a1 = pack_bf16x2(t == 0 ? x1 : (t == 1 ? z1 : 0.0f), t == 0 ? y1 : 0.0f);
        // layer 1, two N tiles at a time -> the four K tiles of layer 2's A operand
        uint32_t A[4][4];
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            float d0[4], d1[4];
            const float2 c0 = *reinterpret_cast<const float2 *>(b1 + 16 * kt + 2 * t);
            const float2 c1 = *reinterpret_cast<const float2 *>(b1 + 16 * kt + 8 + 2 * t);
            d0[0] = c0.x; d0[1] = c0.y; d0[2] = c0.x; d0[3] = c0.y;
            d1[0] = c1.x; d1[1] = c1.y; d1[2] = c1.x; d1[3] = c1.y;
            mma_bf16_16816(d0, a0, a1, 0u, 0u, tiles[(2 * kt) * 32 + lane]);
            mma_bf16_16816(d1, a0, a1, 0u, 0u, tiles[(2 * kt + 1) * 32 + lane]);
            A[kt][0] = pack_bf16x2(silu_f(d0[0]), silu_f(d0[1]));
            A[kt][1] = pack_bf16x2(silu_f(d0[2]), silu_f(d0[3]));
            A[kt][2] = pack_bf16x2(silu_f(d1[0]), silu_f(d1[1]));
            A[kt][3] = pack_bf16x2(silu_f(d1[2]), silu_f(d1[3]));
        }
        // layers 2 and 3 streamed: each pair of layer-2 N tiles is one K tile of
        // layer 3, consumed as soon as it is formed
        const uint2 *t2 = tiles + kTilesL1 * 32;
        const uint2 *t3 = tiles + (kTilesL1 + kTilesL2) * 32;
        const float2 c3 = *reinterpret_cast<const float2 *>(b3 + 2 * t);
        float d3[4] = {c3.x, c3.y, c3.x, c3.y};
#pragma unroll
        for (int k3 = 0; k3 < 4; ++k3) {
            float e0[4], e1[4];
            const float2 c0 = *reinterpret_cast<const float2 *>(b2 + 16 * k3 + 2 * t);
            const float2 c1 = *reinterpret_cast<const float2 *>(b2 + 16 * k3 + 8 + 2 * t);
            e0[0] = c0.x; e0[1] = c0.y; e0[2] = c0.x; e0[3] = c0.y;
            e1[0] = c1.x; e1[1] = c1.y; e1[2] = c1.x; e1[3] = c1.y;
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                mma_bf16_16816(e0, A[kt][0], A[kt][1], A[kt][2], A[kt][3], t2[((2 * k3) * 4 + kt) * 32 + lane]);
                mma_bf16_16816(e1, A[kt][0], A[kt][1], A[kt][2], A[kt][3], t2[((2 * k3 + 1) * 4 + kt) * 32 + lane]);
            }
            const uint32_t h0 = pack_bf16x2(silu_f(e0[0]), silu_f(e0[1]));
            const uint32_t h1 = pack_bf16x2(silu_f(e0[2]), silu_f(e0[3]));
            const uint32_t h2 = pack_bf16x2(silu_f(e1[0]), silu_f(e1[1]));
            const uint32_t h3 = pack_bf16x2(silu_f(e1[2]), silu_f(e1[3]));
            mma_bf16_16816(d3, h0, h1, h2, h3, t3[k3 * 32 + lane]);
        }
        // lanes with t == 0 hold (o1, o2) of rows g (d3[0..1]) and g + 8 (d3[2..3])
        const int src = 4 * (lane & 7);
        const float s0 = __shfl_sync(FULL, d3[0], src), s1 = __shfl_sync(FULL, d3[1], src);
        const float s2 = __shfl_sync(FULL, d3[2], src), s3 = __shfl_sync(FULL, d3[3], src);
        if ((lane >> 4) == m) {
            const bool upper = (lane >> 3) & 1;
            o1 = upper ? s2 : s0;
            o2 = upper ? s3 : s1;
        }
    }
}

// Bias amplitude from the outputs: projection on the noise direction, clamp.
__device__ __forceinline__ float mlp_alpha_of(float o1, float o2, float tan_t, float amax, float &raw)
{
    raw = (o1 + tan_t * o2) * rsqrtf(fmaf(tan_t, tan_t, 1.0f));
    return fminf(fmaxf(raw, -amax), amax);
}

}  // namespace fpt_dev
