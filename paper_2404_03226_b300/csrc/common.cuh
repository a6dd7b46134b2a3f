// Device-side building blocks shared by the library's kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/inspirit.h"

namespace insp {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int MAX_WORKERS = 64;
constexpr int MAX_TYPES_SMEM = 16;
constexpr int32_t MAX_DAG_TASKS = (1 << 24) - 1;
constexpr int64_t TIME_BOUND = int64_t(1) << 54;
constexpr int64_t NEG_TIME = -(int64_t(1) << 60);
// Spin iterations (each ~ >= 64 ns of sleep) before a device-side wait gives up.
constexpr int SPIN_LIMIT = 1 << 22;

// A batch of DAGs in device memory (see insp_batch_load_csr for the layout).
struct DevBatch {
    int32_t ndag;
    int32_t n_types;
    const int64_t *task_base;  // ndag+1
    const int64_t *edge_base;  // ndag+1
    const int32_t *row_ptr;    // n_total + ndag
    const int32_t *col_idx;    // m_total
    const uint8_t *type;       // n_total
    const int64_t *type_cost;  // ndag * n_types * 2
    const int64_t *task_cost;  // n_total * 2, or nullptr
};

// Cost of global task g (local id t of DAG d) on a CPU (kind 0) or GPU (kind 1).
__device__ __forceinline__ int64_t task_cost(const DevBatch &B, int d, int64_t g, int kind) {
    if (B.task_cost) return B.task_cost[2 * g + kind];
    return B.type_cost[(int64_t(d) * B.n_types + B.type[g]) * 2 + kind];
}

// ---------------------------------------------------------------- warp ops
// 64-bit warp min / max from two 32-bit redux steps (sm_80+ redux.sync).
__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
    uint32_t hi = uint32_t(v >> 32);
    uint32_t mh = __reduce_min_sync(FULL, hi);
    uint32_t lo = (hi == mh) ? uint32_t(v) : 0xffffffffu;
    uint32_t ml = __reduce_min_sync(FULL, lo);
    return (uint64_t(mh) << 32) | ml;
}
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
    uint32_t hi = uint32_t(v >> 32);
    uint32_t mh = __reduce_max_sync(FULL, hi);
    uint32_t lo = (hi == mh) ? uint32_t(v) : 0u;
    uint32_t ml = __reduce_max_sync(FULL, lo);
    return (uint64_t(mh) << 32) | ml;
}
__device__ __forceinline__ int64_t warp_min_i64(int64_t v) {
    // order-preserving map of int64 onto uint64
    uint64_t u = uint64_t(v) ^ 0x8000000000000000ull;
    return int64_t(warp_min_u64(u) ^ 0x8000000000000000ull);
}

__device__ __forceinline__ int ld_volatile(const int32_t *p) { return *(const volatile int32_t *)p; }
__device__ __forceinline__ void st_volatile(int32_t *p, int v) { *(volatile int32_t *)p = v; }

// Debug bounds checks (built with -DINSP_CHECK): a failed check records INSP_ECHECK in the
// given status word and the guarded access is skipped.  Release builds compile them away.
#ifdef INSP_CHECK
__device__ __forceinline__ bool insp_check(bool ok, int32_t *status) {
    if (!ok) atomicExch(status, INSP_ECHECK);
    return ok;
}
#else
__device__ __forceinline__ bool insp_check(bool, int32_t *) { return true; }
#endif

// Bounded wait until *flag == value: gives up (returns false) after `limit` polls, or at
// once when *abort is set (another waiter gave up), and then sets *abort.  Every
// device-side wait of the library goes through here, so none can hang the GPU.
__device__ __forceinline__ bool wait_flag(const int32_t *flag, int32_t value, int32_t *abort, int limit) {
    int it = 0;
    while (ld_volatile(flag) != value) {
        if (++it > limit || ld_volatile(abort)) {
            st_volatile(abort, 1);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// Index of the last element of a[0..n) that is <= x (a ascending, a[0] <= x).
__device__ __forceinline__ int upper_index(const int64_t *a, int n, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (a[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace insp
