// Bottom levels, the static priority of the DMDAP baseline (Sec. 2.1: DMDA
// with task priorities; Sec. 3 Observation 1): HEFT's upward rank over the
// machine's mean costs,
//     bl(v) = wbar(v) + max over successors s of (cbar + bl(s)),   a sink: wbar(v),
//     wbar(v) = floor((n_cpu * c_cpu(v) + n_gpu * c_gpu(v)) / P),
// with cbar (the mean transfer cost over ordered worker pairs) from the host.
// One warp per DAG sweeps its tasks in descending id (ids are a topological
// order, so every successor is done first); lanes split a task's successor
// row and combine by a warp max.  Values stay below 2^54 (the load-time bound
// on sum of (max cost + transfer)), so n_cpu * c_cpu + n_gpu * c_gpu < 2^61.
#include "common.cuh"
#include "kernels.h"

namespace insp {

__global__ void __launch_bounds__(256) k_blevel(DevBatch B, int32_t n_cpu, int32_t n_gpu, int64_t cbar,
                                                const int32_t *order, int32_t *counter, int64_t *bl) {
    const int lane = threadIdx.x & 31;
    const int64_t P = int64_t(n_cpu) + n_gpu;
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(counter, 1);
        k = __shfl_sync(FULL, k, 0);
        if (k >= B.ndag) return;
        const int d = order[k];
        const int64_t tb = B.task_base[d], eb = B.edge_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        const int32_t *rp = B.row_ptr + tb + d;
        const int32_t *col = B.col_idx + eb;
        int64_t *out = bl + tb;
        for (int32_t v = n - 1; v >= 0; --v) {
            const int32_t lo = rp[v], hi = rp[v + 1];
            uint64_t m = 0;  // 1 + the largest successor level (0: no successor)
            for (int32_t e = lo + lane; e < hi; e += 32) m = max(m, uint64_t(out[col[e]]) + 1);
            m = warp_max_u64(m);
            if (lane == 0) {
                const int64_t wbar = (n_cpu * task_cost(B, d, tb + v, 0) + n_gpu * task_cost(B, d, tb + v, 1)) / P;
                out[v] = wbar + (m ? cbar + int64_t(m - 1) : 0);
            }
            __syncwarp();  // the level is read by the whole warp at the next tasks
        }
    }
}

void launch_blevel(const DevBatch &B, int32_t n_cpu, int32_t n_gpu, int64_t cbar, const int32_t *order,
                   int32_t *counter, int64_t *bl, int grid, cudaStream_t s) {
    k_blevel<<<grid, 256, 0, s>>>(B, n_cpu, n_gpu, cbar, order, counter, bl);
}

}  // namespace insp
