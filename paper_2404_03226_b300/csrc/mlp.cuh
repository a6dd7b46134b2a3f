// Learned proposal scorer: packed weights and the warp-level tensor-core tile
// (shared by the batched scoring kernel and the simulation's learned pop).
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace insp {

constexpr int MLP_IN = 16, MLP_H = 64;
constexpr int MLP_NW = MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;  // 5313

// Weights laid out for mma.sync B fragments: transposed (output-major) BF16
// rows, so a thread's two consecutive k values are one 32-bit word.
struct ScorerPacked {
    uint16_t w1t[MLP_H][MLP_IN];  // w1t[n][k] = W1[k][n]
    uint16_t w2t[MLP_H][MLP_H];   // w2t[n][k] = W2[k][n]
    uint16_t w3t[8][MLP_H];       // row 0 = W3, rows 1..7 zero (N padded to 8)
    float b1[MLP_H], b2[MLP_H], b3[4];
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Hidden unit of the inference network: min(floor(max(z, 0)), 255).
__device__ __forceinline__ float mlp_act(float z) { return fminf(floorf(fmaxf(z, 0.f)), 255.f); }

// D = A(16x16, row) * B(16x8, col) + C, BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma_bf16_16816(float *c, const uint32_t *a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Scores of a 16-row tile; `feat` holds 16 rows x 8 words (BF16 pairs of the
// 16 features).  Lanes with lane % 4 == 0 return rows lane/4 (s0) and
// lane/4 + 8 (s1).  Fragment layouts follow the PTX ISA description of
// mma.m16n8k16: A rows g and g+8 with columns 2t, 2t+1 and 2t+8, 2t+9; B
// column g with rows 2t, 2t+1 and 2t+8, 2t+9; C rows g, g+8 and columns 2t,
// 2t+1 (g = lane / 4, t = lane % 4).  The C fragments of two adjacent 8-column
// tiles form the A fragment of the next layer's 16-wide k tile.
__device__ __forceinline__ void mlp_score_tile(const ScorerPacked *P, const uint32_t *feat, int lane, float &s0,
                                               float &s1) {
    const int g = lane >> 2, t = lane & 3;
    uint32_t a[4] = {feat[g * 8 + t], feat[(g + 8) * 8 + t], feat[g * 8 + t + 4], feat[(g + 8) * 8 + t + 4]};
    uint32_t h1[16], h2[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float c[4] = {P->b1[8 * j + 2 * t], P->b1[8 * j + 2 * t + 1], P->b1[8 * j + 2 * t], P->b1[8 * j + 2 * t + 1]};
        const uint32_t *w = reinterpret_cast<const uint32_t *>(&P->w1t[8 * j + g][0]);
        mma_bf16_16816(c, a, w[t], w[t + 4]);
        h1[(j >> 1) * 4 + (j & 1) * 2 + 0] = pack_bf16x2(mlp_act(c[0]), mlp_act(c[1]));
        h1[(j >> 1) * 4 + (j & 1) * 2 + 1] = pack_bf16x2(mlp_act(c[2]), mlp_act(c[3]));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float c[4] = {P->b2[8 * j + 2 * t], P->b2[8 * j + 2 * t + 1], P->b2[8 * j + 2 * t], P->b2[8 * j + 2 * t + 1]};
        const uint32_t *w = reinterpret_cast<const uint32_t *>(&P->w2t[8 * j + g][0]);
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma_bf16_16816(c, &h1[kt * 4], w[kt * 8 + t], w[kt * 8 + t + 4]);
        h2[(j >> 1) * 4 + (j & 1) * 2 + 0] = pack_bf16x2(mlp_act(c[0]), mlp_act(c[1]));
        h2[(j >> 1) * 4 + (j & 1) * 2 + 1] = pack_bf16x2(mlp_act(c[2]), mlp_act(c[3]));
    }
    float c[4] = {P->b3[0], P->b3[0], P->b3[0], P->b3[0]};
    const uint32_t *w = reinterpret_cast<const uint32_t *>(&P->w3t[g][0]);
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) mma_bf16_16816(c, &h2[kt * 4], w[kt * 8 + t], w[kt * 8 + t + 4]);
    s0 = c[0];
    s1 = c[2];
}

}  // namespace insp
