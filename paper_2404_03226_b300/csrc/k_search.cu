// Automatic unit time (the paper tunes T of Sec. 4.3 by hand, iteratively;
// this is the batched search that replaces it).  Candidates per DAG:
// T_k = med * 2^k, k = 0..k_max (med = the lower median GPU cost, so T_2 is
// the default unit time; saturating at 2^62).  The chosen T is the smallest
// candidate whose IE takes at least
//     target = min(#distinct (topological layer, type) pairs, #distinct IA)
// distinct values over the DAG's tasks, else T_{k_max}.
//
// Kernels (one warp per DAG, DAGs in size order through a work counter):
//   k_search_target  layers (forward sweep in id order, lanes over a task's
//                    successors) and the two distinct counts, by marking bits
//                    in the DAG's slice of a bitmap and counting them;
//   k_search_ut      the candidate T_k of every DAG not yet decided (0 for a
//                    decided DAG, which makes its efficiency sweep trivial);
//   k_search_step    distinct IE values at T_k; decide the DAG if enough;
//   k_search_final   undecided DAGs take T_{k_max}.
#include "common.cuh"
#include "kernels.h"

namespace insp {

namespace {

// Clear, mark and count bits in words [0, nw) of bm: value v sets bit v.
__device__ __forceinline__ void bm_clear(uint32_t *bm, int64_t nw, int lane) {
    for (int64_t i = lane; i < nw; i += 32) bm[i] = 0;
    __syncwarp();
}
__device__ __forceinline__ int64_t bm_count(const uint32_t *bm, int64_t nw, int lane) {
    int64_t c = 0;
    for (int64_t i = lane; i < nw; i += 32) c += __popc(bm[i]);
    for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
    return c;
}

__device__ __forceinline__ int next_dag(int32_t *counter, const int32_t *order, int ndag, int lane) {
    int k = 0;
    if (lane == 0) k = atomicAdd(counter, 1);
    k = __shfl_sync(FULL, k, 0);
    return k < ndag ? order[k] : -1;
}

}  // namespace

__global__ void __launch_bounds__(256) k_search_target(DevBatch B, const int32_t *order, int32_t *counter,
                                                       const int32_t *ia, int32_t *layer, uint32_t *bitmap,
                                                       const int64_t *bm_base, int64_t *target) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        const int d = next_dag(counter, order, B.ndag, lane);
        if (d < 0) return;
        const int64_t tb = B.task_base[d], eb = B.edge_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        const int32_t *rp = B.row_ptr + tb + d;
        const int32_t *col = B.col_idx + eb;
        int32_t *ly = layer + tb;
        for (int32_t t = lane; t < n; t += 32) ly[t] = 0;
        __syncwarp();
        for (int32_t u = 0; u < n; ++u) {  // ids are topological: u's layer is final here
            const int32_t lu = ly[u] + 1;
            for (int32_t e = rp[u] + lane; e < rp[u + 1]; e += 32) ly[col[e]] = max(ly[col[e]], lu);
            __syncwarp();
        }
        // distinct IA values (in [0, n)), then distinct (layer, type) pairs (layer * n_types + type)
        uint32_t *bm = bitmap + bm_base[d];
        const int64_t nw_ia = (int64_t(n) + 31) / 32, nw_pair = (int64_t(n) * B.n_types + 31) / 32;
        bm_clear(bm, nw_ia, lane);
        for (int32_t t = lane; t < n; t += 32) {
            const int32_t v = ia[tb + t];  // in [0, n) unless the ability sweep failed (status set)
            if (uint32_t(v) < uint32_t(n)) atomicOr(&bm[v >> 5], 1u << (v & 31));
        }
        __syncwarp();
        const int64_t d_ia = bm_count(bm, nw_ia, lane);
        __syncwarp();
        bm_clear(bm, nw_pair, lane);
        for (int32_t t = lane; t < n; t += 32) {  // layer < n and type < n_types (checked at load)
            const int64_t key = int64_t(ly[t]) * B.n_types + B.type[tb + t];
            if (key < int64_t(n) * B.n_types) atomicOr(&bm[key >> 5], 1u << (key & 31));
        }
        __syncwarp();
        const int64_t d_pair = bm_count(bm, nw_pair, lane);
        if (lane == 0) target[d] = min(d_ia, d_pair);
        __syncwarp();
    }
}

__global__ void k_search_ut(int32_t ndag, int32_t k, const int64_t *unit_time_def, const int32_t *done,
                            int64_t *ut) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndag) return;
    const int64_t med = max(int64_t(1), unit_time_def[d] / 4);  // the default is 4 x the lower median
    const int64_t cap = int64_t(1) << 62;
    ut[d] = done[d] ? 0 : (med > (cap >> k) ? cap : med << k);
}

__global__ void __launch_bounds__(256) k_search_step(DevBatch B, const int32_t *order, int32_t *counter,
                                                     const int32_t *ie, uint32_t *bitmap, const int64_t *bm_base,
                                                     const int64_t *target, const int64_t *ut, int32_t *done,
                                                     int64_t *chosen, int32_t *n_done) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        const int d = next_dag(counter, order, B.ndag, lane);
        if (d < 0) return;
        if (done[d]) continue;
        const int64_t tb = B.task_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        uint32_t *bm = bitmap + bm_base[d];
        const int64_t nw = (int64_t(n) + 31) / 32;
        bm_clear(bm, nw, lane);
        for (int32_t t = lane; t < n; t += 32) {
            const int32_t v = ie[tb + t];  // in [0, n) unless the efficiency sweep failed (status set)
            if (uint32_t(v) < uint32_t(n)) atomicOr(&bm[v >> 5], 1u << (v & 31));
        }
        __syncwarp();
        const int64_t c = bm_count(bm, nw, lane);
        if (lane == 0 && c >= target[d]) {
            chosen[d] = ut[d];
            done[d] = 1;
            atomicAdd(n_done, 1);
        }
        __syncwarp();
    }
}

__global__ void k_search_final(int32_t ndag, int32_t k_max, const int64_t *unit_time_def, const int32_t *done,
                               int64_t *chosen) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndag || done[d]) return;
    const int64_t med = max(int64_t(1), unit_time_def[d] / 4);
    const int64_t cap = int64_t(1) << 62;
    chosen[d] = med > (cap >> k_max) ? cap : med << k_max;
}

void launch_search_target(const DevBatch &B, const int32_t *order, int32_t *counter, const int32_t *ia,
                          int32_t *layer, uint32_t *bitmap, const int64_t *bm_base, int64_t *target, int grid,
                          cudaStream_t s) {
    k_search_target<<<grid, 256, 0, s>>>(B, order, counter, ia, layer, bitmap, bm_base, target);
}
void launch_search_ut(int32_t ndag, int32_t k, const int64_t *unit_time_def, const int32_t *done, int64_t *ut,
                      cudaStream_t s) {
    k_search_ut<<<(ndag + 255) / 256, 256, 0, s>>>(ndag, k, unit_time_def, done, ut);
}
void launch_search_step(const DevBatch &B, const int32_t *order, int32_t *counter, const int32_t *ie,
                        uint32_t *bitmap, const int64_t *bm_base, const int64_t *target, const int64_t *ut,
                        int32_t *done, int64_t *chosen, int32_t *n_done, int grid, cudaStream_t s) {
    k_search_step<<<grid, 256, 0, s>>>(B, order, counter, ie, bitmap, bm_base, target, ut, done, chosen, n_done);
}
void launch_search_final(int32_t ndag, int32_t k_max, const int64_t *unit_time_def, const int32_t *done,
                         int64_t *chosen, cudaStream_t s) {
    k_search_final<<<(ndag + 255) / 256, 256, 0, s>>>(ndag, k_max, unit_time_def, done, chosen);
}

}  // namespace insp
