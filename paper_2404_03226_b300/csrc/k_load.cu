// DAG ingest: validation of the CSR and cost tables, in-degrees, the largest
// edge span per DAG and over the batch (window sizes of the inspiring-efficiency
// sweep) and each DAG's default unit time (4 x the lower median of its GPU costs).
#include "common.cuh"
#include "kernels.h"

namespace insp {

// One CTA per DAG (grid-stride over DAGs).  Error precedence matches the
// header: INSP_EINVAL, then INSP_ENOTTOPO, then INSP_EOVERFLOW.
__global__ void __launch_bounds__(256) k_validate(DevBatch B, int64_t xfer, int32_t *status, int32_t *indeg0,
                                                  int32_t *max_span, int32_t *dag_span) {
    __shared__ uint32_t s_flags;
    __shared__ unsigned long long s_sum;
    __shared__ int32_t s_span;
    for (int d = blockIdx.x; d < B.ndag; d += gridDim.x) {
        const int64_t tb = B.task_base[d], eb = B.edge_base[d];
        const int64_t n64 = B.task_base[d + 1] - tb, m64 = B.edge_base[d + 1] - eb;
        if (threadIdx.x == 0) { s_flags = 0; s_sum = 0; s_span = 0; }
        __syncthreads();
        uint32_t flags = 0;
        unsigned long long sum = 0;
        int32_t span = 0;
        if (n64 < 0 || n64 > MAX_DAG_TASKS || m64 < 0 || m64 > 0x7fffffffLL) {
            flags |= 1;
        } else {
            const int32_t n = int32_t(n64), m = int32_t(m64);
            const int32_t *rp = B.row_ptr + tb + d;
            const int32_t *col = B.col_idx + eb;
            if (threadIdx.x == 0 && (rp[0] != 0 || rp[n] != m)) flags |= 1;
            for (int32_t t = threadIdx.x; t < n; t += blockDim.x) {
                int32_t lo = rp[t], hi = rp[t + 1];
                if (lo < 0 || hi < lo || hi > m) { flags |= 1; continue; }
                int32_t prev = -1;
                for (int32_t e = lo; e < hi; ++e) {
                    int32_t v = col[e];
                    if (v < 0 || v >= n) { flags |= 1; break; }
                    if (v <= prev) flags |= 1;
                    prev = v;
                    if (v <= t) flags |= 2;
                    else span = max(span, v - t);
                }
                if (B.type[tb + t] >= B.n_types) { flags |= 1; continue; }
                int64_t cc = task_cost(B, d, tb + t, 0), cg = task_cost(B, d, tb + t, 1);
                if (cc < 1 || cg < 1) { flags |= 1; continue; }
                int64_t c = cc > cg ? cc : cg;
                if (c > TIME_BOUND) flags |= 4;
                else if (sum <= (unsigned long long)TIME_BOUND) sum += (unsigned long long)(c + xfer);
            }
            if (sum > (unsigned long long)TIME_BOUND) flags |= 4;
        }
        if (flags) atomicOr(&s_flags, flags);
        if (sum) atomicAdd(&s_sum, sum < (1ull << 55) ? sum : (1ull << 55));
        if (span) atomicMax(&s_span, span);
        __syncthreads();
        uint32_t f = s_flags;
        if (s_sum > (unsigned long long)TIME_BOUND) f |= 4;
        int32_t st = (f & 1) ? INSP_EINVAL : (f & 2) ? INSP_ENOTTOPO : (f & 4) ? INSP_EOVERFLOW : INSP_OK;
        if (threadIdx.x == 0) {
            status[d] = st;
            atomicMax(max_span, s_span);
            if (dag_span) dag_span[d] = s_span;
        }
        // in-degrees (only meaningful for valid DAGs)
        if (st == INSP_OK) {
            const int32_t n = int32_t(n64);
            const int32_t *rp = B.row_ptr + tb + d;
            for (int32_t t = threadIdx.x; t < n; t += blockDim.x)
                for (int32_t e = rp[t]; e < rp[t + 1]; ++e) atomicAdd(&indeg0[tb + B.col_idx[eb + e]], 1);
        }
        __syncthreads();
    }
}

// Lower median of the GPU costs by an 8-bit radix select (values < 2^56),
// one CTA per valid DAG; writes 4 x median (>= 1).
__global__ void __launch_bounds__(256) k_unit_time(DevBatch B, const int32_t *status, int64_t *unit_time) {
    __shared__ uint32_t hist[256];
    __shared__ uint64_t s_prefix, s_mask;
    __shared__ int64_t s_rank;
    for (int d = blockIdx.x; d < B.ndag; d += gridDim.x) {
        const int64_t tb = B.task_base[d];
        const int64_t n = B.task_base[d + 1] - tb;
        if (status[d] != INSP_OK || n <= 0) {
            if (threadIdx.x == 0) unit_time[d] = 1;
            continue;
        }
        if (threadIdx.x == 0) { s_prefix = 0; s_mask = 0; s_rank = (n - 1) / 2; }
        __syncthreads();
        for (int shift = 48; shift >= 0; shift -= 8) {
            for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
            __syncthreads();
            const uint64_t prefix = s_prefix, mask = s_mask;
            for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
                uint64_t v = uint64_t(task_cost(B, d, tb + t, 1));
                if ((v & mask) == prefix) atomicAdd(&hist[(v >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int64_t r = s_rank;
                int b = 0;
                for (; b < 256; ++b) {
                    if (r < int64_t(hist[b])) break;
                    r -= hist[b];
                }
                s_rank = r;
                s_prefix = prefix | (uint64_t(b) << shift);
                s_mask = mask | (uint64_t(255) << shift);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            int64_t T = 4 * int64_t(s_prefix);
            unit_time[d] = T < 1 ? 1 : T;
        }
        __syncthreads();
    }
}

void launch_validate(const DevBatch &B, int64_t xfer, int32_t *status, int32_t *indeg0, int32_t *max_span,
                     int32_t *dag_span,
                     int grid, cudaStream_t s) {
    k_validate<<<grid, 256, 0, s>>>(B, xfer, status, indeg0, max_span, dag_span);
}
void launch_unit_time(const DevBatch &B, const int32_t *status, int64_t *unit_time, int grid, cudaStream_t s) {
    k_unit_time<<<grid, 256, 0, s>>>(B, status, unit_time);
}

}  // namespace insp
