// DAG ingest: validation of the CSR and cost tables, in-degrees, the largest
// edge span per DAG and over the batch (window sizes of the inspiring-efficiency
// sweep) and each DAG's default unit time (4 x the lower median of its GPU costs).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace insp {

// Structure fingerprint terms (splitmix64 finaliser): a DAG's fingerprint is the wrapping sum of
// mix64 over its task and edge counts, every row offset with its index and every successor id
// with its edge index.  Equal structures have equal fingerprints; the load compares candidate
// pairs exactly before sharing anything.
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// Per DAG (one CTA each, grid-stride over DAGs): validation (error precedence as in the header:
// INSP_EINVAL, then INSP_ENOTTOPO, then INSP_EOVERFLOW), then -- for DAGs whose edges are in range -- one coalesced
// pass over the flat successor array that counts in-degrees (in shared memory for DAGs of up to
// smem_n tasks, else by global atomics) and sums the structure fingerprint (hash may be NULL).
__global__ void __launch_bounds__(256) k_validate(DevBatch B, int64_t xfer, int32_t *status, int32_t *indeg0,
                                                  int32_t *max_span, int32_t *dag_span, unsigned long long *hash,
                                                  int32_t smem_n) {
    extern __shared__ int32_t s_indeg[];  // smem_n counters
    __shared__ uint32_t s_flags;
    __shared__ unsigned long long s_sum, s_h;
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
        // in-degrees and fingerprint (valid DAGs, and DAGs whose numbering is not topological:
        // renumbering uses the in-degrees, and they are validated again afterwards)
        if (st == INSP_OK || st == INSP_ENOTTOPO) {
            const int32_t n = int32_t(n64), m = int32_t(m64);
            const int32_t *rp = B.row_ptr + tb + d;
            const int32_t *col = B.col_idx + eb;
            const bool in_smem = n <= smem_n;
            if (in_smem)
                for (int32_t t = threadIdx.x; t < n; t += blockDim.x) s_indeg[t] = 0;
            if (threadIdx.x == 0) s_h = 0;
            __syncthreads();
            unsigned long long h = threadIdx.x == 0 ? mix64(uint64_t(n) * 0x100000001ull + uint64_t(m)) : 0ull;
            for (int32_t i = threadIdx.x; i <= n; i += blockDim.x) h += mix64((uint64_t(i) << 32) ^ uint32_t(rp[i]));
            for (int32_t e = threadIdx.x; e < m; e += blockDim.x) {
                const int32_t v = col[e];
                if (in_smem) atomicAdd(&s_indeg[v], 1);
                else atomicAdd(&indeg0[tb + v], 1);
                h += mix64(((uint64_t(e) + 0x80000000ull) << 32) ^ uint32_t(v) ^ 0x5bd1e995ull);
            }
            atomicAdd(&s_h, h);
            __syncthreads();
            if (in_smem)
                for (int32_t t = threadIdx.x; t < n; t += blockDim.x) indeg0[tb + t] = s_indeg[t];
            if (hash && threadIdx.x == 0) hash[d] = s_h;
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

// ------------------------------------------------------------- renumbering
// A DAG whose ids are not a topological order is renumbered by Kahn's algorithm in rounds
// (round 0: the tasks without predecessors; round r + 1: the tasks whose predecessors all lie
// in rounds <= r), consecutive new ids within a round in ascending old id.  One CTA per listed
// DAG; cnt, level, qa, qb: per-task scratch in the batch's global task indexing.

// Rounds by frontier queues: level[t] = the round of t; a cycle leaves tasks in no round
// (status INSP_ECYCLE).  n_levels[k] = the number of rounds of listed DAG k.
__global__ void __launch_bounds__(256) k_kahn(DevBatch B, const int32_t *dags, int32_t n_dags, const int32_t *indeg0,
                                              int32_t *cnt, int32_t *level, int32_t *qa, int32_t *qb,
                                              int32_t *n_levels, int32_t *status) {
    __shared__ int32_t s_na, s_nb, s_total;
    for (int k = blockIdx.x; k < n_dags; k += gridDim.x) {
        const int d = dags[k];
        const int64_t tb = B.task_base[d], eb = B.edge_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        const int32_t *rp = B.row_ptr + tb + d;
        const int32_t *col = B.col_idx + eb;
        int32_t *a = qa + tb, *b = qb + tb;
        if (threadIdx.x == 0) s_na = 0;
        __syncthreads();
        for (int32_t t = threadIdx.x; t < n; t += blockDim.x) {
            const int32_t c = indeg0[tb + t];
            cnt[tb + t] = c;
            level[tb + t] = -1;
            if (c == 0) {
                level[tb + t] = 0;
                a[atomicAdd(&s_na, 1)] = t;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_total = s_na;
        int32_t round = 0;
        for (;;) {
            __syncthreads();
            const int32_t na = s_na;
            if (na == 0) break;
            if (threadIdx.x == 0) s_nb = 0;
            __syncthreads();
            for (int32_t i = threadIdx.x; i < na; i += blockDim.x) {
                const int32_t u = a[i];
                for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
                    const int32_t v = col[e];
                    if (atomicSub(&cnt[tb + v], 1) == 1) {
                        level[tb + v] = round + 1;
                        b[atomicAdd(&s_nb, 1)] = v;
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                s_na = s_nb;
                s_total += s_nb;
            }
            int32_t *x = a;
            a = b;
            b = x;
            ++round;
        }
        if (threadIdx.x == 0) {
            n_levels[k] = round;
            status[d] = s_total == n ? INSP_OK : INSP_ECYCLE;
        }
        __syncthreads();
    }
}

// New ids from the rounds: a counting sort by round, stable in old id.  old_of_new[tb + p] =
// the old local id of new task p; new_of_old[tb + t] = the new id of old task t.  The counts
// and cursors reuse cnt.  One CTA per listed DAG; warp 0 places the tasks 32 at a time in
// ascending old id (equal rounds matched within the warp), so the order is deterministic.
__global__ void __launch_bounds__(256) k_kahn_order(DevBatch B, const int32_t *dags, int32_t n_dags,
                                                    const int32_t *n_levels, const int32_t *level, int32_t *cnt,
                                                    int32_t *new_of_old, int32_t *old_of_new, const int32_t *status) {
    for (int k = blockIdx.x; k < n_dags; k += gridDim.x) {
        const int d = dags[k];
        if (status[d] != INSP_OK) continue;
        const int64_t tb = B.task_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        const int32_t nl = n_levels[k];
        int32_t *c = cnt + tb;  // per round: count, then the next free new id
        for (int32_t i = threadIdx.x; i < nl; i += blockDim.x) c[i] = 0;
        __syncthreads();
        for (int32_t t = threadIdx.x; t < n; t += blockDim.x) atomicAdd(&c[level[tb + t]], 1);
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int32_t carry = 0;  // exclusive scan of the counts over the rounds
            for (int32_t base = 0; base < nl; base += 32) {
                const int32_t i = base + lane;
                const int32_t v = i < nl ? c[i] : 0;
                int32_t x = v;
                for (int off = 1; off < 32; off <<= 1) {
                    const int32_t y = __shfl_up_sync(FULL, x, off);
                    if (lane >= off) x += y;
                }
                if (i < nl) c[i] = carry + x - v;
                carry += __shfl_sync(FULL, x, 31);
            }
            __syncwarp();
            for (int32_t base = 0; base < n; base += 32) {
                const int32_t t = base + lane;
                const int32_t L = t < n ? level[tb + t] : -1;
                const uint32_t same = __match_any_sync(FULL, L);
                int32_t pos = 0;
                if (t < n) {
                    pos = c[L] + __popc(same & ((1u << lane) - 1));
                    new_of_old[tb + t] = pos;
                    old_of_new[tb + pos] = t;
                }
                __syncwarp();
                if (t < n && lane == __ffs(same) - 1) c[L] += __popc(same);
                __syncwarp();
            }
        }
        __syncthreads();
    }
}

// The renumbered DAGs' arrays: new row p is old task old_of_new[p] with its successors mapped
// by new_of_old and sorted ascending (one warp per row: a rank among the row's values, which
// are distinct); types and per-task costs move with their tasks.  `out` arrays already hold a
// copy of the whole batch (the other DAGs stay as they are); out_rp must hold the new row
// offsets (filled by k_renumber_rows first).
__global__ void __launch_bounds__(256) k_renumber_degrees(DevBatch B, const int32_t *dags, int32_t n_dags,
                                                          const int32_t *old_of_new, int32_t *out_rp,
                                                          const int32_t *status) {
    __shared__ int32_t s_carry;
    for (int k = blockIdx.x; k < n_dags; k += gridDim.x) {
        const int d = dags[k];
        if (status[d] != INSP_OK) continue;
        const int64_t tb = B.task_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        const int32_t *rp = B.row_ptr + tb + d;
        int32_t *orp = out_rp + tb + d;
        if (threadIdx.x == 0) { s_carry = 0; orp[0] = 0; }
        __syncthreads();
        // inclusive block scan of the new rows' degrees, 256 rows at a time
        __shared__ int32_t s_w[8];
        for (int32_t base = 0; base < n; base += blockDim.x) {
            const int32_t p = base + threadIdx.x;
            const int32_t u = p < n ? old_of_new[tb + p] : 0;
            const int32_t deg = p < n ? rp[u + 1] - rp[u] : 0;
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            int32_t x = deg;
            for (int off = 1; off < 32; off <<= 1) {
                const int32_t y = __shfl_up_sync(FULL, x, off);
                if (lane >= off) x += y;
            }
            if (lane == 31) s_w[w] = x;
            __syncthreads();
            int32_t before = s_carry;
            for (int i = 0; i < w; ++i) before += s_w[i];
            if (p < n) orp[p + 1] = before + x;
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1) s_carry = before + x;
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256) k_renumber_rows(DevBatch B, const int32_t *dags, int32_t n_dags,
                                                       const int32_t *old_of_new, const int32_t *new_of_old,
                                                       const int32_t *out_rp, int32_t *out_col, uint8_t *out_type,
                                                       int64_t *out_task_cost, const int32_t *status) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = blockIdx.x; k < n_dags; k += gridDim.x) {
        const int d = dags[k];
        if (status[d] != INSP_OK) continue;
        const int64_t tb = B.task_base[d], eb = B.edge_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        const int32_t *rp = B.row_ptr + tb + d, *col = B.col_idx + eb;
        const int32_t *orp = out_rp + tb + d;
        for (int32_t p = wib; p < n; p += nw) {
            const int32_t u = old_of_new[tb + p];
            const int32_t lo = rp[u], deg = rp[u + 1] - lo, o = orp[p];
            if (lane == 0) {
                out_type[tb + p] = B.type[tb + u];
                if (out_task_cost) {
                    out_task_cost[2 * (tb + p)] = B.task_cost[2 * (tb + u)];
                    out_task_cost[2 * (tb + p) + 1] = B.task_cost[2 * (tb + u) + 1];
                }
            }
            for (int32_t i = lane; i < deg; i += 32) {
                const int32_t x = new_of_old[tb + col[lo + i]];
                int32_t rank = 0;
                for (int32_t j = 0; j < deg; ++j) rank += new_of_old[tb + col[lo + j]] < x;
                out_col[eb + o + rank] = x;
            }
        }
    }
}

// Caller order <-> batch order of per-task arrays: dst[tb + old_of_new[tb + p]] = src[tb + p]
// (to the caller's numbering) or dst[tb + p] = src[tb + old_of_new[tb + p]] (from it).
template <typename T>
__global__ void k_permute(const int64_t *task_base, int32_t ndag, const int32_t *old_of_new, const T *src, T *dst,
                          int to_caller) {
    for (int d = blockIdx.x; d < ndag; d += gridDim.x) {
        const int64_t tb = task_base[d], n = task_base[d + 1] - tb;
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
            const int64_t q = tb + old_of_new[tb + p];
            if (to_caller) dst[q] = src[tb + p];
            else dst[tb + p] = src[q];
        }
    }
}

// old_of_new[tb + p] = p for every task (the DAGs that keep their numbering).
__global__ void k_local_iota(const int64_t *task_base, int32_t ndag, int32_t *out) {
    for (int d = blockIdx.x; d < ndag; d += gridDim.x) {
        const int64_t tb = task_base[d], n = task_base[d + 1] - tb;
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) out[tb + p] = int32_t(p);
    }
}
void launch_local_iota(const int64_t *task_base, int32_t ndag, int32_t *out, cudaStream_t s) {
    if (ndag > 0) k_local_iota<<<ndag < 4096 ? ndag : 4096, 256, 0, s>>>(task_base, ndag, out);
}

void launch_kahn(const DevBatch &B, const int32_t *dags, int32_t n_dags, const int32_t *indeg0, int32_t *cnt,
                 int32_t *level, int32_t *qa, int32_t *qb, int32_t *n_levels, int32_t *new_of_old,
                 int32_t *old_of_new, int32_t *status, cudaStream_t s) {
    if (n_dags <= 0) return;
    const int grid = n_dags < 1024 ? n_dags : 1024;
    k_kahn<<<grid, 256, 0, s>>>(B, dags, n_dags, indeg0, cnt, level, qa, qb, n_levels, status);
    k_kahn_order<<<grid, 256, 0, s>>>(B, dags, n_dags, n_levels, level, cnt, new_of_old, old_of_new, status);
}
void launch_renumber(const DevBatch &B, const int32_t *dags, int32_t n_dags, const int32_t *old_of_new,
                     const int32_t *new_of_old, int32_t *out_rp, int32_t *out_col, uint8_t *out_type,
                     int64_t *out_task_cost, const int32_t *status, cudaStream_t s) {
    if (n_dags <= 0) return;
    const int grid = n_dags < 1024 ? n_dags : 1024;
    k_renumber_degrees<<<grid, 256, 0, s>>>(B, dags, n_dags, old_of_new, out_rp, status);
    k_renumber_rows<<<grid, 256, 0, s>>>(B, dags, n_dags, old_of_new, new_of_old, out_rp, out_col, out_type,
                                         out_task_cost, status);
}
void launch_permute(const int64_t *task_base, int32_t ndag, const int32_t *old_of_new, const void *src, void *dst,
                    int elem_bytes, bool to_caller, cudaStream_t s) {
    if (ndag <= 0) return;
    const int grid = ndag < 4096 ? ndag : 4096;
    if (elem_bytes == 4)
        k_permute<int32_t><<<grid, 256, 0, s>>>(task_base, ndag, old_of_new, (const int32_t *)src, (int32_t *)dst,
                                                to_caller);
    else
        k_permute<int64_t><<<grid, 256, 0, s>>>(task_base, ndag, old_of_new, (const int64_t *)src, (int64_t *)dst,
                                                to_caller);
}

void launch_validate(const DevBatch &B, int64_t xfer, int32_t *status, int32_t *indeg0, int32_t *max_span,
                     int32_t *dag_span, unsigned long long *hash, int32_t max_n, int grid, cudaStream_t s) {
    const int32_t smem_n = std::max(0, std::min(max_n, VALIDATE_SMEM_TASKS));
    cudaFuncSetAttribute(k_validate, cudaFuncAttributeMaxDynamicSharedMemorySize, VALIDATE_SMEM_TASKS * 4);
    k_validate<<<grid, 256, size_t(smem_n) * 4, s>>>(B, xfer, status, indeg0, max_span, dag_span, hash, smem_n);
}
void launch_unit_time(const DevBatch &B, const int32_t *status, int64_t *unit_time, int grid, cudaStream_t s) {
    k_unit_time<<<grid, 256, 0, s>>>(B, status, unit_time);
}

}  // namespace insp
