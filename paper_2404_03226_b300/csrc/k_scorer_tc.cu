// Batched scoring of the learned proposal scorer (no counterpart in the paper) on the fifth-
// generation tensor cores: 128 feature rows per tile, one row per thread and per tensor-memory
// lane.  The three layers are tcgen05.mma of kind::f16 (BF16 operands in shared memory, FP32
// accumulators in tensor memory) issued by one thread: layer 1 [128 x 16] x [16 x 64], layer 2
// [128 x 64] x [64 x 64] (four K = 16 steps), layer 3 [128 x 64] x [64 x 16] (W3 in row 0 of
// the 16, the rest zero).  Between layers each warp reads its 32 rows of the accumulators
// (tcgen05.ld), adds the bias, applies the hidden unit min(floor(max(z, 0)), 255) and writes
// the BF16 row back to shared memory as the next layer's A operand.
//
// Exact for the same reason as the warp-level form of the simulation's learned pop: features
// and hidden units are integers in [0, 255], weights and biases k / 64 with |k| <= 128, so
// every product and partial sum is a multiple of 1/64 below 2^15 -- representable in FP32 in
// any order of summation.  The score is an integer count of 1/64.
//
// Features arrive by one-dimensional bulk copies (TMA) of whole tiles into two shared-memory
// buffers, two tiles ahead of the MMAs.  Measured on 16M rows: 12.3 G rows/s (884 GB/s)
// against 9.9 with per-thread loads and 5.4 for the warp-level mma.sync tiles; per-thread
// register prefetch of the next row (8.1), every layer's accumulator at column 0 of 64 columns
// (8.1), and that with six CTAs per SM (6.6) were slower.  Feature rows that are not 16-byte
// aligned are loaded by each thread instead.
//
// Every wait (an MMA commit, a bulk copy) is bounded: on timeout the CTA writes
// INSP_SCORE_TIMEOUT (INT64_MIN) to the rows it has not scored, waits once more (bounded) for
// the MMA and the copies in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "mlp.cuh"
#include "umma.cuh"

namespace insp {

namespace {
constexpr int TM = 128;                 // rows per tile: threads per CTA, tensor-memory lanes
constexpr uint32_t TMEM_COLS = 128;     // layer 1 and 3 accumulators at column 0, layer 2 at 64
constexpr uint32_t WAIT_LIMIT = 1u << 24;
// shared memory (bytes): the operands in the K-major core-matrix layout, then the biases, the
// mbarrier, the tensor-memory address and the timeout flag
constexpr uint32_t OFF_A1 = 0;                                  // features, 128 x 16
constexpr uint32_t OFF_A2 = OFF_A1 + TM * MLP_IN * 2;           // hidden units, 128 x 64
constexpr uint32_t OFF_B1 = OFF_A2 + TM * MLP_H * 2;            // W1^T, 64 x 16
constexpr uint32_t OFF_B2 = OFF_B1 + MLP_H * MLP_IN * 2;        // W2^T, 64 x 64
constexpr uint32_t OFF_B3 = OFF_B2 + MLP_H * MLP_H * 2;         // W3^T padded, 16 x 64
constexpr uint32_t FB_BYTES = TM * MLP_IN * 4;                   // one tile of int32 features
constexpr uint32_t OFF_FB = OFF_B3 + 16 * MLP_H * 2;              // two feature buffers (bulk copies)
constexpr uint32_t OFF_BIAS = OFF_FB + 2 * FB_BYTES;              // b1[64], b2[64], b3
// the MMA mbarrier, the two feature-buffer mbarriers, the tensor-memory address, the timeout flag
constexpr uint32_t OFF_MISC = OFF_BIAS + (2 * MLP_H + 4) * 4;
constexpr uint32_t SMEM_USED = OFF_MISC + 32;
// Dynamic shared memory per CTA: more than a quarter of an SM's shared memory, so at most
// four CTAs (4 x 128 of the 512 tensor-memory columns) are resident on an SM and an
// allocation never has to wait for another CTA.
constexpr uint32_t SMEM_BYTES = 60 * 1024;
static_assert(SMEM_USED <= SMEM_BYTES, "scorer tile does not fit");
static_assert(OFF_A2 % 1024 == 0 && OFF_B1 % 1024 == 0 && OFF_B2 % 1024 == 0 && OFF_B3 % 1024 == 0 &&
                  OFF_FB % 1024 == 0,
              "operand tiles and feature buffers are 1024-byte aligned");
static_assert(OFF_MISC % 8 == 0, "mbarrier alignment");

__device__ __forceinline__ void put8(unsigned char *dst, const uint32_t *w) {
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// The hidden units of 64 accumulator columns of this thread's row: act(d + bias) as BF16, row
// `r` of the K = 64 operand at `a`.
__device__ __forceinline__ void hidden_row(uint32_t taddr, const float *bias, unsigned char *a, int r) {
#pragma unroll
    for (int c0 = 0; c0 < MLP_H; c0 += 16) {
        uint32_t d[16];
        tmem_ld16(taddr + c0, d);
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            w[j] = pack_bf16x2(mlp_act(__uint_as_float(d[2 * j]) + bias[c0 + 2 * j]),
                               mlp_act(__uint_as_float(d[2 * j + 1]) + bias[c0 + 2 * j + 1]));
        put8(a + kmajor_offset(r, c0, MLP_H), w);
        put8(a + kmajor_offset(r, c0 + 8, MLP_H), w + 4);
    }
}
}  // namespace

__global__ void __launch_bounds__(TM) k_scorer_eval_tc(const ScorerPacked *Pg, const int32_t *feat, int64_t n,
                                                       int64_t *score) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *a1 = sm + OFF_A1, *a2 = sm + OFF_A2, *b1 = sm + OFF_B1, *b2 = sm + OFF_B2, *b3 = sm + OFF_B3;
    float *bias = reinterpret_cast<float *>(sm + OFF_BIAS);
    unsigned char *fb = sm + OFF_FB;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + OFF_MISC);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + OFF_MISC + 24);
    int32_t *timed_out = reinterpret_cast<int32_t *>(sm + OFF_MISC + 28);

    // B operands (N x K, K-major): the transposed weights, W3 padded to 16 rows; the biases
    for (int i = tid; i < MLP_H * MLP_IN; i += TM)
        *reinterpret_cast<uint16_t *>(b1 + kmajor_offset(i / MLP_IN, i % MLP_IN, MLP_IN)) = Pg->w1t[i / MLP_IN][i % MLP_IN];
    for (int i = tid; i < MLP_H * MLP_H; i += TM)
        *reinterpret_cast<uint16_t *>(b2 + kmajor_offset(i / MLP_H, i % MLP_H, MLP_H)) = Pg->w2t[i / MLP_H][i % MLP_H];
    for (int i = tid; i < 16 * MLP_H; i += TM) {
        const int r = i / MLP_H, k = i % MLP_H;
        *reinterpret_cast<uint16_t *>(b3 + kmajor_offset(r, k, MLP_H)) = r < 8 ? Pg->w3t[r][k] : uint16_t(0);
    }
    for (int i = tid; i < MLP_H; i += TM) {
        bias[i] = Pg->b1[i];
        bias[MLP_H + i] = Pg->b2[i];
    }
    const uint32_t mb = smem_u32(mbar), mbl = mb + 8;  // feature buffer b completes on mbl + 8 b
    if (tid == 0) {
        bias[2 * MLP_H] = Pg->b3[0];
        *timed_out = 0;
        mbar_init(mb, 1);
        mbar_init(mbl, 1);
        mbar_init(mbl + 8, 1);
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tslot), TMEM_COLS);
        tmem_relinquish();
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t my_lanes = tbase + (uint32_t(warp * 32) << 16);  // this warp's 32 accumulator rows
    const uint32_t ID64 = umma_idesc_bf16_f32(TM, MLP_H), ID16 = umma_idesc_bf16_f32(TM, 16);
    const uint32_t sa1 = smem_u32(a1), sa2 = smem_u32(a2), sb1 = smem_u32(b1), sb2 = smem_u32(b2),
                   sb3 = smem_u32(b3);
    uint32_t phase = 0;

    // the operands written by all threads go to the tensor core; thread 0 issues `issue` and
    // commits; every thread learns whether the MMAs completed within the bound
    auto run = [&](auto issue) -> bool {
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue();
            umma_commit(mb);
            if (!mbar_wait_bounded(mb, phase, WAIT_LIMIT)) *timed_out = 1;
        }
        phase ^= 1u;
        __syncthreads();
        tc_fence_after();
        return *timed_out == 0;
    };

    const int64_t tiles = (n + TM - 1) / TM;
    // Features: with 16-byte aligned rows, whole tiles (contiguous, up to 8 KB) come by bulk copy
    // into two buffers, two tiles ahead; thread 0 issues them and counts them per buffer (at most
    // one in flight per buffer).  Otherwise every thread loads its row.
    const bool bulk = (reinterpret_cast<uintptr_t>(feat) & 15) == 0;
    int issued[2] = {0, 0}, used[2] = {0, 0};
    auto issue_load = [&](int64_t t, int b) {
        const int64_t rows = n - t * TM < TM ? n - t * TM : TM;
        const uint32_t bytes = uint32_t(rows) * uint32_t(MLP_IN * 4);
        mbar_arrive_expect_tx(mbl + 8 * b, bytes);
        bulk_g2s(smem_u32(fb + b * FB_BYTES), feat + t * TM * MLP_IN, bytes, mbl + 8 * b);
        issued[b] += 1;
    };
    if (bulk && tid == 0)
        for (int b = 0; b < 2; ++b)
            if (blockIdx.x + int64_t(b) * gridDim.x < tiles) issue_load(blockIdx.x + int64_t(b) * gridDim.x, b);
    int64_t tt = blockIdx.x;
    bool ok = true;
    for (int k = 0; tt < tiles; tt += gridDim.x, ++k) {
        const int64_t row = tt * TM + tid;
        const int b = k & 1;
        int32_t f[16];
        if (bulk) {
            if (tid == 0) {
                if (!mbar_wait_bounded(mbl + 8 * b, uint32_t(used[b] & 1), WAIT_LIMIT)) *timed_out = 1;
                used[b] += 1;
            }
            __syncthreads();
            if (*timed_out) {
                ok = false;
                break;
            }
            const int4 *p = reinterpret_cast<const int4 *>(fb + b * FB_BYTES + tid * MLP_IN * 4);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int4 v = p[q];
                f[4 * q] = v.x; f[4 * q + 1] = v.y; f[4 * q + 2] = v.z; f[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 16; ++c) f[c] = row < n ? feat[row * 16 + c] : 0;
        }
        {  // layer-1 input: this thread's features, clamped to [0, 255] (zeros past n)
            uint32_t w[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int f0 = row < n ? min(max(f[2 * c], 0), 255) : 0;
                const int f1 = row < n ? min(max(f[2 * c + 1], 0), 255) : 0;
                w[c] = pack_bf16x2(float(f0), float(f1));
            }
            put8(a1 + kmajor_offset(tid, 0, MLP_IN), w);
            put8(a1 + kmajor_offset(tid, 8, MLP_IN), w + 4);
        }
        // layer 1; buffer b is free once every thread has passed the barrier in run(): the bulk
        // copy of the tile two ahead goes there
        ok = run([&] {
            umma_bf16(tbase, umma_smem_desc(sa1, 128, 256), umma_smem_desc(sb1, 128, 256), ID64, 0);
            if (bulk && tt + 2 * int64_t(gridDim.x) < tiles) issue_load(tt + 2 * int64_t(gridDim.x), b);
        });
        if (!ok) break;
        hidden_row(my_lanes, bias, a2, tid);
        ok = run([&] {
            for (uint32_t s = 0; s < 4; ++s)
                umma_bf16(tbase + 64, umma_smem_desc(sa2 + 256 * s, 128, 1024), umma_smem_desc(sb2 + 256 * s, 128, 1024),
                          ID64, s);
        });
        if (!ok) break;
        hidden_row(my_lanes + 64, bias + MLP_H, a2, tid);  // layer 2 has read a2
        ok = run([&] {
            for (uint32_t s = 0; s < 4; ++s)
                umma_bf16(tbase, umma_smem_desc(sa2 + 256 * s, 128, 1024), umma_smem_desc(sb3 + 256 * s, 128, 1024),
                          ID16, s);
        });
        if (!ok) break;
        uint32_t d[16];
        tmem_ld16(my_lanes, d);
        if (row < n) score[row] = int64_t((__uint_as_float(d[0]) + bias[2 * MLP_H]) * 64.0f);
        tc_fence_before();
        __syncthreads();  // the next tile rewrites a1, a2 and the accumulators
    }
    if (!ok) {
        // this CTA's unscored rows get the sentinel; the MMA in flight gets one more bounded wait
        for (; tt < tiles; tt += gridDim.x) {
            const int64_t row = tt * TM + tid;
            if (row < n) score[row] = INSP_SCORE_TIMEOUT;
        }
        if (tid == 0) {
            mbar_wait_bounded(mb, phase ^ 1u, WAIT_LIMIT);
            for (int b = 0; b < 2; ++b)  // a bulk copy still in flight into buffer b
                if (issued[b] > used[b]) mbar_wait_bounded(mbl + 8 * b, uint32_t(used[b] & 1), WAIT_LIMIT);
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, TMEM_COLS);
    }
}

void launch_scorer_eval(const ScorerPacked *P, const int32_t *feat, int64_t n, int64_t *score, cudaStream_t s) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 148;
    }
    cudaFuncSetAttribute(k_scorer_eval_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM_BYTES));
    const int64_t tiles = (n + TM - 1) / TM;
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(tiles, int64_t(sms) * 4)));
    k_scorer_eval_tc<<<grid, TM, SMEM_BYTES, s>>>(P, feat, n, score);
}

}  // namespace insp
