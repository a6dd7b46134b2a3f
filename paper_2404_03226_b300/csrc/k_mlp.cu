// Learned proposal scorer (no counterpart in the paper): MLP 16 -> 64 -> 64 -> 1.
//
// Batched inference runs on the fifth-generation tensor cores (tcgen05, in
// k_scorer_tc.cu); the simulation's learned pop scores its candidates with the
// warp-level mma.sync m16n8k16 tile of mlp.cuh (BF16 operands, FP32
// accumulation, one 16-candidate tile per warp).  Both are exact by
// construction: features are integers in [0, 255], weights and biases are
// k / 64 with |k| <= 128 (both exact in BF16), hidden units are
// min(floor(max(z, 0)), 255) (integers again), so every partial sum is a
// multiple of 1/64 below 2^15 in magnitude -- exact in FP32 in any summation
// order.  The score is returned as an integer count of 1/64.
//
// Training (loss and gradient of a squared-error objective; quantisation-aware
// mode rounds weights to the grid and floors activations in the forward pass
// and passes gradients straight through) has two forms: FP32 on the CUDA cores
// (a per-sample kernel and a gradient kernel that reduces over the samples in a
// fixed order), and the tensor-core form (k_mlp_tc: every matrix product as
// BF16 mma.sync with FP32 accumulation, per-tile partial gradients summed in
// tile order).  Both are deterministic.  Then AdamW and grid quantisation.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "mlp.cuh"

namespace insp {

// --------------------------------------------------------------- training
__device__ __forceinline__ float q_weight(float w) {
    float k = w * 64.0f;
    k = k >= 0.f ? floorf(k + 0.5f) : -floorf(-k + 0.5f);
    return fminf(fmaxf(k, -128.f), 128.f) / 64.0f;
}

// Per sample (one warp each): forward pass, squared error and the backward
// pass through the activations.  work[s] holds a1[h1], d1[h1], a2[h2], d2[h2],
// dy, e^2.  Dimensions: in <= 32, h1, h2 <= 64.
__global__ void __launch_bounds__(256) k_mlp_samples(int32_t in, int32_t h1, int32_t h2, const float *w,
                                                     int32_t mode, int64_t n, const float *x, const float *target,
                                                     float *work) {
    extern __shared__ float sh[];
    const int32_t nw = in * h1 + h1 + h1 * h2 + h2 + h2 + 1;
    float *wq = sh;                       // weights used by the forward pass
    float *per = sh + nw;                 // per warp: x[32], a1[64], d2[64]
    for (int i = threadIdx.x; i < nw; i += blockDim.x) wq[i] = mode ? q_weight(w[i]) : w[i];
    __syncthreads();
    const float *W1 = wq, *B1 = W1 + in * h1, *W2 = B1 + h1, *B2 = W2 + h1 * h2, *W3 = B2 + h2, *B3 = W3 + h2;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *xs = per + wib * 160, *a1s = xs + 32, *d2s = a1s + 64;
    const int64_t stride = 2 * int64_t(h1) + 2 * h2 + 2;
    const float hi = mode ? 256.f : 255.f;
    for (int64_t s = int64_t(blockIdx.x) * 8 + wib; s < n; s += int64_t(gridDim.x) * 8) {
        float *ws = work + s * stride;
        if (lane < in) xs[lane] = x[s * in + lane];
        __syncwarp();
        float z1v[2] = {0, 0};
        for (int r = 0; r < 2; ++r) {
            const int j = lane + 32 * r;
            if (j < h1) {
                float z = B1[j];
                for (int i = 0; i < in; ++i) z += W1[i * h1 + j] * xs[i];
                z1v[r] = z;
                float a = fmaxf(z, 0.f);
                if (mode) a = floorf(a);
                a = fminf(a, 255.f);
                a1s[j] = a;
                ws[j] = a;
            }
        }
        __syncwarp();
        float z2v[2] = {0, 0}, part = 0.f;
        for (int r = 0; r < 2; ++r) {
            const int j = lane + 32 * r;
            if (j < h2) {
                float z = B2[j];
                for (int i = 0; i < h1; ++i) z += W2[i * h2 + j] * a1s[i];
                z2v[r] = z;
                float a = fmaxf(z, 0.f);
                if (mode) a = floorf(a);
                a = fminf(a, 255.f);
                ws[2 * h1 + j] = a;
                part += W3[j] * a;
            }
        }
        for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(FULL, part, off);
        const float y = B3[0] + part;
        const float e = y - target[s];
        const float dy = 2.f * e / float(n);
        if (lane == 0) {
            ws[2 * h1 + 2 * h2] = dy;
            ws[2 * h1 + 2 * h2 + 1] = e * e;
        }
        for (int r = 0; r < 2; ++r) {
            const int j = lane + 32 * r;
            if (j < h2) {
                const float d = (z2v[r] > 0.f && z2v[r] < hi) ? dy * W3[j] : 0.f;
                d2s[j] = d;
                ws[2 * h1 + h2 + j] = d;
            }
        }
        __syncwarp();
        for (int r = 0; r < 2; ++r) {
            const int i = lane + 32 * r;
            if (i < h1) {
                float g = 0.f;
                for (int j = 0; j < h2; ++j) g += W2[i * h2 + j] * d2s[j];
                ws[h1 + i] = (z1v[r] > 0.f && z1v[r] < hi) ? g : 0.f;
            }
        }
        __syncwarp();
    }
}

// One thread per weight: gradient as a fixed-order sum over the samples; the
// last thread also reduces the loss.  Quantisation-aware mode zeroes the
// gradient of weights clamped off the grid (|64 w| > 128.5).
__global__ void __launch_bounds__(256) k_mlp_grad(int32_t in, int32_t h1, int32_t h2, const float *w, int32_t mode,
                                                  int64_t n, const float *x, const float *work, float *grad,
                                                  float *loss) {
    const int32_t nw = in * h1 + h1 + h1 * h2 + h2 + h2 + 1;
    const int64_t stride = 2 * int64_t(h1) + 2 * h2 + 2;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nw) return;
    if (k == nw) {  // loss
        double acc = 0.0;
        for (int64_t s = 0; s < n; ++s) acc += work[s * stride + 2 * h1 + 2 * h2 + 1];
        *loss = float(acc / double(n));
        return;
    }
    // which tensor does weight k belong to: product of an input side and an output side
    const int o_a1 = 0, o_d1 = h1, o_a2 = 2 * h1, o_d2 = 2 * h1 + h2, o_dy = 2 * h1 + 2 * h2;
    float acc = 0.f;
    int r = k;
    if (r < in * h1) {                       // W1[i][j] += x_i d1_j
        const int i = r / h1, j = r % h1;
        for (int64_t s = 0; s < n; ++s) acc += x[s * in + i] * work[s * stride + o_d1 + j];
    } else if ((r -= in * h1) < h1) {        // b1[j] += d1_j
        for (int64_t s = 0; s < n; ++s) acc += work[s * stride + o_d1 + r];
    } else if ((r -= h1) < h1 * h2) {        // W2[i][j] += a1_i d2_j
        const int i = r / h2, j = r % h2;
        for (int64_t s = 0; s < n; ++s) acc += work[s * stride + o_a1 + i] * work[s * stride + o_d2 + j];
    } else if ((r -= h1 * h2) < h2) {        // b2[j] += d2_j
        for (int64_t s = 0; s < n; ++s) acc += work[s * stride + o_d2 + r];
    } else if ((r -= h2) < h2) {             // W3[j] += dy a2_j
        for (int64_t s = 0; s < n; ++s) acc += work[s * stride + o_dy] * work[s * stride + o_a2 + r];
    } else {                                 // b3 += dy
        for (int64_t s = 0; s < n; ++s) acc += work[s * stride + o_dy];
    }
    if (mode) {
        const float kk = w[k] * 64.f;
        if (kk > 128.5f || kk < -128.5f) acc = 0.f;
    }
    grad[k] = acc;
}

// --------------------------------------------------- training on tensor cores
// The same loss and gradient with every matrix product on the tensor cores (mma.sync
// m16n8k16, BF16 operands, FP32 accumulation).  One warp takes a tile of 16 samples:
//   forward   Z1 = X W1 + b1, Z2 = A1 W2 + b2, y = A2 W3 + b3   (M = 16 samples)
//   backward  D2 = (dy W3^T) * act'(Z2), D1 = (D2 W2^T) * act'(Z1)
//   gradients W1 += X^T D1, W2 += A1^T D2 (K = the 16 samples), biases and W3 by warp sums.
// Each FP32 operand x enters as two BF16 numbers hi = bf16(x), lo = bf16(x - hi), and each
// product as hi*hi + hi*lo + lo*hi: only lo*lo (below 2^-16 of the product) is dropped, so a
// product keeps about 16 significant bits.  In the quantisation-aware mode the weights (k/64),
// the integer features and the floored activations are exact in BF16 (their lo parts are 0), so
// the forward pass and the loss are exact; only the backward signals are split.  Dimensions are
// padded to in 32, h1 64, h2 64 with zero weights (padded units stay at 0 and pass no gradient).
// Every tile writes its partial gradient (and squared error) to its own slice of `part`; a
// second kernel sums the slices in tile order, so the result is deterministic.
constexpr int TC_IN = 32, TC_H = 64, TC_WARPS = 4;

struct TcWeights {  // CTA-shared BF16 packs of the weights in use (B operands stored [n][k])
    uint16_t w1t[2][TC_H][TC_IN];  // [hi/lo][j][i] = W1[i][j]
    uint16_t w2t[2][TC_H][TC_H];   // [hi/lo][j][i] = W2[i][j]   (forward)
    uint16_t w2[2][TC_H][TC_H];    // [hi/lo][i][j] = W2[i][j]   (backward)
    uint16_t w3[2][8][TC_H];       // [hi/lo][0][j] = W3[j], rows 1..7 zero
    float b1[TC_H], b2[TC_H], w3f[TC_H], b3;
};
struct TcTile {  // per-warp staging of one 16-sample tile
    uint16_t x[2][16][TC_IN], xt[2][TC_IN][16];
    uint16_t a1[2][16][TC_H], a1t[2][TC_H][16];
    uint16_t a2[2][16][TC_H];
    uint16_t d2[2][16][TC_H], d2t[2][TC_H][16];
    uint16_t d1t[2][TC_H][16];
    float dy[16];
};

__device__ __forceinline__ void split_bf16(float x, uint16_t &hi, uint16_t &lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = *reinterpret_cast<const uint16_t *>(&h);
    lo = *reinterpret_cast<const uint16_t *>(&l);
}
__device__ __forceinline__ uint32_t ld_pair(const uint16_t *p) { return *reinterpret_cast<const uint32_t *>(p); }

// C(16x8) += A(16x16 at column k0 of a [16][ld] pair of hi/lo buffers) * B(16x8: rows n0.. of a
// [n][ldb] pair of hi/lo buffers, k from k0), three products per the split above.
__device__ __forceinline__ void mma3(float *c, const uint16_t *ahi, const uint16_t *alo, int lda, int m0, int k0,
                                     const uint16_t *bhi, const uint16_t *blo, int ldb, int n0, int lane) {
    const int g = lane >> 2, t = lane & 3;
    const int r0 = (m0 + g) * lda + k0 + 2 * t, r1 = (m0 + g + 8) * lda + k0 + 2 * t;
    const uint32_t ah[4] = {ld_pair(ahi + r0), ld_pair(ahi + r1), ld_pair(ahi + r0 + 8), ld_pair(ahi + r1 + 8)};
    const uint32_t al[4] = {ld_pair(alo + r0), ld_pair(alo + r1), ld_pair(alo + r0 + 8), ld_pair(alo + r1 + 8)};
    const int q = (n0 + g) * ldb + k0 + 2 * t;
    const uint32_t bh0 = ld_pair(bhi + q), bh1 = ld_pair(bhi + q + 8);
    const uint32_t bl0 = ld_pair(blo + q), bl1 = ld_pair(blo + q + 8);
    mma_bf16_16816(c, ah, bh0, bh1);
    mma_bf16_16816(c, ah, bl0, bl1);
    mma_bf16_16816(c, al, bh0, bh1);
}

// sum over the 8 row groups g of a value held per lane (lanes with equal t = lane % 4)
__device__ __forceinline__ float sum_rows(float v) {
    v += __shfl_xor_sync(FULL, v, 4);
    v += __shfl_xor_sync(FULL, v, 8);
    v += __shfl_xor_sync(FULL, v, 16);
    return v;
}

__global__ void __launch_bounds__(TC_WARPS * 32) k_mlp_tc(int32_t in, int32_t h1, int32_t h2, const float *w,
                                                          int32_t mode, int64_t n, const float *x,
                                                          const float *target, float *part) {
    extern __shared__ __align__(16) unsigned char tc_smem[];
    TcWeights &W = *reinterpret_cast<TcWeights *>(tc_smem);
    TcTile &T = reinterpret_cast<TcTile *>(tc_smem + (sizeof(TcWeights) + 15) / 16 * 16)[threadIdx.x >> 5];
    const int32_t nw = in * h1 + h1 + h1 * h2 + h2 + h2 + 1;
    const float *W1 = w, *B1 = W1 + in * h1, *W2 = B1 + h1, *B2 = W2 + h1 * h2, *W3 = B2 + h2, *B3 = W3 + h2;
    auto wv = [&](float v) { return mode ? q_weight(v) : v; };
    // CTA: the weight packs (zero padding outside in x h1 x h2)
    for (int e = threadIdx.x; e < TC_H * TC_IN; e += blockDim.x) {
        const int j = e / TC_IN, i = e % TC_IN;
        split_bf16(i < in && j < h1 ? wv(W1[i * h1 + j]) : 0.f, W.w1t[0][j][i], W.w1t[1][j][i]);
    }
    for (int e = threadIdx.x; e < TC_H * TC_H; e += blockDim.x) {
        const int a = e / TC_H, b = e % TC_H;  // w2t[a = j][b = i], w2[a = i][b = j]
        split_bf16(b < h1 && a < h2 ? wv(W2[b * h2 + a]) : 0.f, W.w2t[0][a][b], W.w2t[1][a][b]);
        split_bf16(a < h1 && b < h2 ? wv(W2[a * h2 + b]) : 0.f, W.w2[0][a][b], W.w2[1][a][b]);
    }
    for (int e = threadIdx.x; e < 8 * TC_H; e += blockDim.x) {
        const int r = e / TC_H, j = e % TC_H;
        split_bf16(r == 0 && j < h2 ? wv(W3[j]) : 0.f, W.w3[0][r][j], W.w3[1][r][j]);
    }
    for (int j = threadIdx.x; j < TC_H; j += blockDim.x) {
        W.b1[j] = j < h1 ? wv(B1[j]) : 0.f;
        W.b2[j] = j < h2 ? wv(B2[j]) : 0.f;
        W.w3f[j] = j < h2 ? wv(W3[j]) : 0.f;
    }
    if (threadIdx.x == 0) W.b3 = wv(B3[0]);
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float hi_act = mode ? 256.f : 255.f;
    auto act = [&](float z) {
        float a = fmaxf(z, 0.f);
        if (mode) a = floorf(a);
        return fminf(a, 255.f);
    };
    const int64_t tiles = (n + 15) / 16;
    const int64_t stride = int64_t(nw) + 1;
    for (int64_t tile = int64_t(blockIdx.x) * TC_WARPS + (threadIdx.x >> 5); tile < tiles;
         tile += int64_t(gridDim.x) * TC_WARPS) {
        const int64_t s0 = tile * 16;
        float *P = part + tile * stride;
        // ---- inputs
        for (int e = lane; e < 16 * TC_IN; e += 32) {
            const int r = e / TC_IN, i = e % TC_IN;
            const float v = (s0 + r < n && i < in) ? x[(s0 + r) * in + i] : 0.f;
            uint16_t h, l;
            split_bf16(v, h, l);
            T.x[0][r][i] = h; T.x[1][r][i] = l;
            T.xt[0][i][r] = h; T.xt[1][i][r] = l;
        }
        __syncwarp();
        // ---- layer 1
        uint32_t mask1 = 0;  // bit 4 nt + e: act' of C element e of n tile nt
        for (int nt = 0; nt < 8; ++nt) {
            const int c = 8 * nt + 2 * t;
            float z[4] = {W.b1[c], W.b1[c + 1], W.b1[c], W.b1[c + 1]};
            for (int kt = 0; kt < TC_IN / 16; ++kt)
                mma3(z, &T.x[0][0][0], &T.x[1][0][0], TC_IN, 0, 16 * kt, &W.w1t[0][0][0], &W.w1t[1][0][0], TC_IN,
                     8 * nt, lane);
            for (int e = 0; e < 4; ++e) {
                const int r = g + 8 * (e >> 1), col = c + (e & 1);
                if (z[e] > 0.f && z[e] < hi_act) mask1 |= 1u << (4 * nt + e);
                uint16_t h, l;
                split_bf16(act(z[e]), h, l);
                T.a1[0][r][col] = h; T.a1[1][r][col] = l;
                T.a1t[0][col][r] = h; T.a1t[1][col][r] = l;
            }
        }
        __syncwarp();
        // ---- layer 2
        uint32_t mask2 = 0;
        float a2v[32];
        for (int nt = 0; nt < 8; ++nt) {
            const int c = 8 * nt + 2 * t;
            float z[4] = {W.b2[c], W.b2[c + 1], W.b2[c], W.b2[c + 1]};
            for (int kt = 0; kt < TC_H / 16; ++kt)
                mma3(z, &T.a1[0][0][0], &T.a1[1][0][0], TC_H, 0, 16 * kt, &W.w2t[0][0][0], &W.w2t[1][0][0], TC_H,
                     8 * nt, lane);
            for (int e = 0; e < 4; ++e) {
                const int r = g + 8 * (e >> 1), col = c + (e & 1);
                if (z[e] > 0.f && z[e] < hi_act) mask2 |= 1u << (4 * nt + e);
                a2v[4 * nt + e] = act(z[e]);
                uint16_t h, l;
                split_bf16(a2v[4 * nt + e], h, l);
                T.a2[0][r][col] = h; T.a2[1][r][col] = l;
            }
        }
        __syncwarp();
        // ---- output, error and dy (column 0 of the 16 x 8 product: lanes t == 0)
        float yv[4] = {W.b3, W.b3, W.b3, W.b3};
        for (int kt = 0; kt < TC_H / 16; ++kt)
            mma3(yv, &T.a2[0][0][0], &T.a2[1][0][0], TC_H, 0, 16 * kt, &W.w3[0][0][0], &W.w3[1][0][0], TC_H, 0, lane);
        float sq = 0.f;
        if (t == 0) {
            for (int h = 0; h < 2; ++h) {
                const int r = g + 8 * h;
                const bool live = s0 + r < n;
                const float e = live ? yv[2 * h] - target[s0 + r] : 0.f;
                T.dy[r] = live ? 2.f * e / float(n) : 0.f;
                sq += e * e;
            }
        }
        sq = sum_rows(sq);
        __syncwarp();
        // ---- D2, the layer-3 and layer-2 bias / W3 gradients
        float dy_r[2] = {T.dy[g], T.dy[g + 8]};
        for (int nt = 0; nt < 8; ++nt) {
            const int c = 8 * nt + 2 * t;
            float gb2[2] = {0.f, 0.f}, gw3[2] = {0.f, 0.f};
            for (int e = 0; e < 4; ++e) {
                const int r = g + 8 * (e >> 1), col = c + (e & 1);
                const float d = ((mask2 >> (4 * nt + e)) & 1u) ? dy_r[e >> 1] * W.w3f[col] : 0.f;
                gb2[e & 1] += d;
                gw3[e & 1] += dy_r[e >> 1] * a2v[4 * nt + e];
                uint16_t h, l;
                split_bf16(d, h, l);
                T.d2[0][r][col] = h; T.d2[1][r][col] = l;
                T.d2t[0][col][r] = h; T.d2t[1][col][r] = l;
            }
            for (int k = 0; k < 2; ++k) {
                gb2[k] = sum_rows(gb2[k]);
                gw3[k] = sum_rows(gw3[k]);
            }
            if (g == 0) {
                for (int k = 0; k < 2; ++k) {
                    if (c + k < h2) {
                        P[in * h1 + h1 + h1 * h2 + c + k] = gb2[k];
                        P[in * h1 + h1 + h1 * h2 + h2 + c + k] = gw3[k];
                    }
                }
            }
        }
        if (lane == 0) {
            float gb3 = 0.f;
            for (int r = 0; r < 16; ++r) gb3 += T.dy[r];
            P[nw - 1] = gb3;
            P[nw] = sq;
        }
        __syncwarp();
        // ---- D1 and the layer-1 bias gradient
        for (int nt = 0; nt < 8; ++nt) {
            const int c = 8 * nt + 2 * t;
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            for (int kt = 0; kt < TC_H / 16; ++kt)
                mma3(d, &T.d2[0][0][0], &T.d2[1][0][0], TC_H, 0, 16 * kt, &W.w2[0][0][0], &W.w2[1][0][0], TC_H,
                     8 * nt, lane);
            float gb1[2] = {0.f, 0.f};
            for (int e = 0; e < 4; ++e) {
                const int r = g + 8 * (e >> 1), col = c + (e & 1);
                const float v = ((mask1 >> (4 * nt + e)) & 1u) ? d[e] : 0.f;
                gb1[e & 1] += v;
                uint16_t h, l;
                split_bf16(v, h, l);
                T.d1t[0][col][r] = h; T.d1t[1][col][r] = l;
            }
            for (int k = 0; k < 2; ++k) gb1[k] = sum_rows(gb1[k]);
            if (g == 0)
                for (int k = 0; k < 2; ++k)
                    if (c + k < h1) P[in * h1 + c + k] = gb1[k];
        }
        __syncwarp();
        // ---- weight gradients over the tile's samples: W1 (in x h1), W2 (h1 x h2)
        for (int mt = 0; mt < TC_IN / 16; ++mt)
            for (int nt = 0; nt < 8; ++nt) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma3(c, &T.xt[0][0][0], &T.xt[1][0][0], 16, 16 * mt, 0, &T.d1t[0][0][0], &T.d1t[1][0][0], 16, 8 * nt,
                     lane);
                for (int e = 0; e < 4; ++e) {
                    const int i = 16 * mt + g + 8 * (e >> 1), j = 8 * nt + 2 * t + (e & 1);
                    if (i < in && j < h1) P[i * h1 + j] = c[e];
                }
            }
        for (int mt = 0; mt < TC_H / 16; ++mt)
            for (int nt = 0; nt < 8; ++nt) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma3(c, &T.a1t[0][0][0], &T.a1t[1][0][0], 16, 16 * mt, 0, &T.d2t[0][0][0], &T.d2t[1][0][0], 16,
                     8 * nt, lane);
                for (int e = 0; e < 4; ++e) {
                    const int i = 16 * mt + g + 8 * (e >> 1), j = 8 * nt + 2 * t + (e & 1);
                    if (i < h1 && j < h2) P[in * h1 + h1 + i * h2 + j] = c[e];
                }
            }
        __syncwarp();
    }
}

// Sum of the per-tile partials in tile order (one thread per weight; the last one the loss).
__global__ void __launch_bounds__(256) k_mlp_tc_reduce(int32_t nw, int64_t tiles, int64_t n, int32_t mode,
                                                       const float *w, const float *part, float *grad, float *loss) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nw) return;
    const int64_t stride = int64_t(nw) + 1;
    if (k == nw) {
        double acc = 0.0;
        for (int64_t s = 0; s < tiles; ++s) acc += part[s * stride + nw];
        *loss = float(acc / double(n));
        return;
    }
    float acc = 0.f;
    for (int64_t s = 0; s < tiles; ++s) acc += part[s * stride + k];
    if (mode) {
        const float kk = w[k] * 64.f;
        if (kk > 128.5f || kk < -128.5f) acc = 0.f;
    }
    grad[k] = acc;
}

// AdamW (decoupled weight decay), step t >= 1.
__global__ void k_adamw(int64_t nw, float *w, float *m, float *v, const float *g, float c1, float c2, float lr,
                        float b1, float b2, float eps, float wd) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nw) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * w[i]);
}

// Grid quantisation of real weights: BF16 bits of clamp(round(64 w), -128, 128) / 64.
__global__ void k_quantize(int64_t nw, const float *w, uint16_t *out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nw) return;
    const __nv_bfloat16 b = __float2bfloat16_rn(q_weight(w[i]));
    out[i] = *reinterpret_cast<const uint16_t *>(&b);
}

// ----------------------------------------------------------------- launch

void launch_mlp_train_grad(int32_t in, int32_t h1, int32_t h2, const float *w, int32_t mode, int64_t n,
                           const float *x, const float *target, float *work, float *grad, float *loss,
                           cudaStream_t s) {
    const int32_t nw = in * h1 + h1 + h1 * h2 + h2 + h2 + 1;
    const size_t smem = size_t(nw + 8 * 160) * 4;
    cudaFuncSetAttribute(k_mlp_samples, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    const int grid = int(std::min<int64_t>(std::max<int64_t>((n + 7) / 8, 1), 148 * 4));
    k_mlp_samples<<<grid, 256, smem, s>>>(in, h1, h2, w, mode, n, x, target, work);
    k_mlp_grad<<<(nw + 1 + 255) / 256, 256, 0, s>>>(in, h1, h2, w, mode, n, x, work, grad, loss);
}

void launch_mlp_train_grad_tc(int32_t in, int32_t h1, int32_t h2, const float *w, int32_t mode, int64_t n,
                              const float *x, const float *target, float *part, float *grad, float *loss,
                              cudaStream_t s) {
    const int32_t nw = in * h1 + h1 + h1 * h2 + h2 + h2 + 1;
    const int64_t tiles = (n + 15) / 16;
    const size_t smem = (sizeof(TcWeights) + 15) / 16 * 16 + TC_WARPS * sizeof(TcTile);
    cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    const int grid = int(std::min<int64_t>(std::max<int64_t>((tiles + TC_WARPS - 1) / TC_WARPS, 1), 148 * 2));
    k_mlp_tc<<<grid, TC_WARPS * 32, smem, s>>>(in, h1, h2, w, mode, n, x, target, part);
    k_mlp_tc_reduce<<<(nw + 1 + 255) / 256, 256, 0, s>>>(nw, tiles, n, mode, w, part, grad, loss);
}

void launch_adamw(int64_t nw, float *w, float *m, float *v, const float *g, int32_t t, float lr, float b1, float b2,
                  float eps, float wd, cudaStream_t s) {
    double c1 = 1.0, c2 = 1.0;
    for (int i = 0; i < t; ++i) { c1 *= b1; c2 *= b2; }
    k_adamw<<<int((nw + 255) / 256), 256, 0, s>>>(nw, w, m, v, g, float(1.0 - c1), float(1.0 - c2), lr, b1, b2, eps,
                                                   wd);
}

void launch_quantize(int64_t nw, const float *w, uint16_t *out, cudaStream_t s) {
    k_quantize<<<int((nw + 255) / 256), 256, 0, s>>>(nw, w, out);
}

}  // namespace insp
