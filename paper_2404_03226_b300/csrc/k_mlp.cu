// Learned proposal scorer (no counterpart in the paper): MLP 16 -> 64 -> 64 -> 1.
//
// Inference runs on the tensor cores with mma.sync m16n8k16 (BF16 operands,
// FP32 accumulation), one 16-candidate tile per warp.  It is exact by
// construction: features are integers in [0, 255], weights and biases are
// k / 64 with |k| <= 128 (both exact in BF16), hidden units are
// min(floor(max(z, 0)), 255) (integers again), so every partial sum is a
// multiple of 1/64 below 2^15 in magnitude -- exact in FP32 in any summation
// order.  The score is returned as an integer count of 1/64.
//
// Training is FP32 on the CUDA cores: a per-sample kernel (forward, loss,
// backward through the activations; quantisation-aware mode rounds weights to
// the grid and floors activations in the forward pass and passes gradients
// straight through) and a gradient kernel that reduces over the samples in a
// fixed order (deterministic), then AdamW and grid quantisation kernels.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "mlp.cuh"

namespace insp {

// ------------------------------------------------------------- inference
// Batched scoring of feature rows feat[n][16] (int32, clamped to [0, 255]).
__global__ void __launch_bounds__(128) k_scorer_eval(const ScorerPacked *Pg, const int32_t *feat, int64_t n,
                                                     int64_t *score) {
    __shared__ ScorerPacked P;
    __shared__ uint32_t tile[4][16 * 8];
    for (int i = threadIdx.x; i < int(sizeof(ScorerPacked) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t *>(&P)[i] = reinterpret_cast<const uint32_t *>(Pg)[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *my = tile[wib];
    const int64_t tiles = (n + 15) / 16;
    for (int64_t tt = int64_t(blockIdx.x) * 4 + wib; tt < tiles; tt += int64_t(gridDim.x) * 4) {
        // lane r < 16 packs row r
        if (lane < 16) {
            const int64_t row = tt * 16 + lane;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                int f0 = 0, f1 = 0;
                if (row < n) {
                    f0 = min(max(feat[row * 16 + 2 * c], 0), 255);
                    f1 = min(max(feat[row * 16 + 2 * c + 1], 0), 255);
                }
                my[lane * 8 + c] = pack_bf16x2(float(f0), float(f1));
            }
        }
        __syncwarp();
        float s0, s1;
        mlp_score_tile(&P, my, lane, s0, s1);
        if ((lane & 3) == 0) {
            const int64_t r0 = tt * 16 + (lane >> 2), r1 = r0 + 8;
            if (r0 < n) score[r0] = int64_t(s0 * 64.0f);
            if (r1 < n) score[r1] = int64_t(s1 * 64.0f);
        }
        __syncwarp();
    }
}

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
void launch_scorer_eval(const ScorerPacked *P, const int32_t *feat, int64_t n, int64_t *score, cudaStream_t s) {
    const int64_t tiles = (n + 15) / 16;
    const int grid = int(std::min<int64_t>(std::max<int64_t>((tiles + 3) / 4, 1), 148 * 8));
    k_scorer_eval<<<grid, 128, 0, s>>>(P, feat, n, score);
}

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
