// Task attributes of Sec. 4.2 / Sec. 4.3.
//
// Inspiring ability, IA(v) = |strict descendants of v|.  Reverse sweep over a
// DAG in descending id (ids are topological): desc(v) = union over successors
// s of ({s} + desc(s)), kept as one bitset row per task in global scratch.  A
// CTA owns one DAG at a time; its warps claim tasks in descending id and each
// waits (bounded) until the rows of its successors are published.
//
// Inspiring efficiency, IE_T(v) = |{u != v : every path v ~> u, weighted by GPU
// costs with both ends included, weighs <= T}|.  A warp owns 32 consecutive
// sources (lane j <-> v0 + j) and sweeps ids upward from v0 -- the "sliding
// window" of Sec. 4.3 -- keeping per task a reach mask (sources whose cone
// holds it), an over mask (sources for which some path to it already exceeds
// T) and, in a ring buffer of W >= max edge span + 1 slots, the running max of
// its in-cone predecessors' path weights per source.  The sweep stops after
// the last task that received an in-window contribution.
#include "common.cuh"
#include "kernels.h"

namespace insp {

// --------------------------------------------------------- inspiring ability
constexpr int IA_MAX_WARPS = 32;  // warps per CTA: blockDim / 32, up to 32 (autotuned)

// Descendant rows are bitsets of 64-bit words (half the word operations of 32-bit ones).
__global__ void __launch_bounds__(IA_MAX_WARPS * 32) k_ia(DevBatch B, const int32_t *order, int32_t n_order,
                                                          int32_t *counter, uint64_t *bits, int64_t slot_words,
                                                          int32_t *done, const int32_t *epoch_ptr, int32_t *ia_out,
                                                          int32_t *status) {
    const int32_t epoch = *epoch_ptr;  // this step's value of the done flags
    __shared__ int32_t s_dag;
    __shared__ int32_t s_next;
    __shared__ int32_t s_abort;  // a wait gave up: later waits of this DAG return at once
    const int lane = threadIdx.x & 31;
    uint64_t *slot = bits + int64_t(blockIdx.x) * slot_words;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int k = atomicAdd(counter, 1);
            int d = k < n_order ? order[k] : -1;
            s_dag = d;
            s_next = d >= 0 ? int32_t(B.task_base[d + 1] - B.task_base[d]) - 1 : -1;
            s_abort = 0;
        }
        __syncthreads();
        const int d = s_dag;
        if (d < 0) return;
        const int64_t tb = B.task_base[d], eb = B.edge_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        const int32_t NW = (n + 63) >> 6;
        const int32_t *rp = B.row_ptr + tb + d;
        const int32_t *col = B.col_idx + eb;
        bool timed_out = false;
        for (;;) {
            int32_t v = 0;
            if (lane == 0) v = atomicSub(&s_next, 1);
            v = __shfl_sync(FULL, v, 0);
            if (v < 0) break;
            const int32_t lo = rp[v], deg = rp[v + 1] - lo;
            // wait until every successor's row is published (bounded)
            for (int32_t i = lane; i < deg; i += 32) {
                const int32_t s = col[lo + i];
                if (!wait_flag(done + tb + s, epoch, &s_abort, SPIN_LIMIT)) timed_out = true;
            }
            __syncwarp();
            __threadfence_block();
            // Words wlo..NW-1 of the row are needed.  The warp splits into
            // 32/g groups of g lanes (g = words per chunk, a power of two);
            // groups OR different successors, then combine by shuffle-xor.
            // Stored rows hold the task itself too: row(s) = {s} and its descendants, so a row is
            // the plain OR of its successors' rows plus its own bit, and IA = popcount - 1.
            // Words v/64 .. NW-1 of the row are needed.
            const int32_t wlo = v >> 6;
            const int32_t span_w = NW - wlo;
            // g = the power of two >= span_w, at most 32 (shifts and masks: g is not known to the
            // compiler to be a power of two, so / and % would be full integer divisions)
            const int32_t lg = span_w >= 32 ? 5 : (span_w <= 1 ? 0 : 32 - __clz(span_w - 1));
            const int32_t g = 1 << lg;
            const int32_t G = 32 >> lg, grp = lane >> lg, wl = lane & (g - 1);
            uint64_t *row_v = slot + int64_t(v) * NW;
            int32_t count = 0;
            for (int32_t cw = wlo; cw < NW; cw += g) {
                const int32_t w = cw + wl;
                uint64_t acc = (grp == 0 && w == wlo) ? (1ull << (v & 63)) : 0ull;
#pragma unroll 4
                for (int32_t i = grp; i < deg; i += G) {
                    const int32_t s = col[lo + i];
                    // successors come after v (topological ids, checked at load) and before n
                    if (w >= (s >> 6) && w < NW && insp_check(s > v && s < n, status + d))
                        acc |= slot[int64_t(s) * NW + w];
                }
                for (int32_t off = g; off < 32; off <<= 1) acc |= __shfl_xor_sync(FULL, acc, off);
                if (grp == 0 && w < NW) {
                    row_v[w] = acc;
                    count += __popcll(acc);
                }
            }
            count = __reduce_add_sync(FULL, count) - 1;  // the task's own bit
            __threadfence_block();
            __syncwarp();
            if (lane == 0) {
                ia_out[tb + v] = count;
                st_volatile(done + tb + v, epoch);
            }
        }
        timed_out = __syncthreads_or(timed_out);
        if (timed_out && threadIdx.x == 0) status[d] = INSP_ETIMEOUT;
    }
}

// ------------------------------------------------------ inspiring efficiency
// Per-task record of the sweep: {tag low, reach mask, over mask, tag high}.  A
// record whose 64-bit tag differs from the current work item's is empty (no
// reset needed; tags grow by the number of work items every step).
template <typename V>
__global__ void __launch_bounds__(256) k_ie(DevBatch B, const int64_t *item_base, int64_t n_items, int32_t *counter,
                                            const int64_t *unit_time, uint4 *rec, int64_t rec_stride, V *acc,
                                            int32_t W, const uint64_t *tag_base_ptr, int32_t *ie_out) {
    const uint64_t tag_base = *tag_base_ptr;
    const int lane = threadIdx.x & 31;
    const int64_t warp_id = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    uint4 *my_rec = rec + warp_id * rec_stride;
    V *my_acc = acc + warp_id * int64_t(W) * 32;
    const int32_t wmask = W - 1;
    for (;;) {
        int64_t item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(FULL, item, 0);
        if (item >= n_items) return;
        const int d = upper_index(item_base, B.ndag + 1, item);
        const int64_t tb = B.task_base[d], eb = B.edge_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        const int32_t v0 = int32_t(item - item_base[d]) * 32;
        const int32_t n_src = min(32, n - v0);
        const int32_t *rp = B.row_ptr + tb + d;
        const int32_t *col = B.col_idx + eb;
        const int64_t T = unit_time[d];
        const uint64_t tag64 = tag_base + uint64_t(item);
        const uint32_t tag = uint32_t(tag64), tag_hi = uint32_t(tag64 >> 32);
        int32_t cnt = 0;
        int32_t hi = v0 + n_src - 1;
        for (int32_t x = v0; x <= hi; ++x) {
            const uint4 r = my_rec[x];
            const bool mine = r.x == tag && r.w == tag_hi;
            const uint32_t reach = mine ? r.y : 0u;
            const uint32_t over = mine ? r.z : 0u;
            const uint32_t src = (x - v0 < n_src) ? (1u << (x - v0)) : 0u;
            const uint32_t pmask = reach | src;
            if (pmask == 0) continue;
            const int64_t c = task_cost(B, d, tb + x, 1);
            bool under = false;
            int64_t L = 0;
            if ((src >> lane) & 1u) {
                L = c;
                under = (L <= T);
            } else if (((reach >> lane) & 1u) && !((over >> lane) & 1u)) {
                L = int64_t(my_acc[(x & wmask) * 32 + lane]) + c;
                under = (L <= T);
                cnt += under;
            }
            const uint32_t umask = __ballot_sync(FULL, under);
            const uint32_t omask = pmask & ~umask;
            const int32_t elo = rp[x], ehi = rp[x + 1];
            for (int32_t base = elo; base < ehi; base += 32) {
                const int32_t i = base + lane;
                int32_t s = 0;
                uint32_t old_reach = 0, old_over = 0;
                if (i < ehi) {
                    s = col[i];
                    uint4 q = my_rec[s];
                    if (q.x != tag || q.w != tag_hi) q = make_uint4(tag, 0u, 0u, tag_hi);
                    old_reach = q.y;
                    old_over = q.z;
                    q.y |= pmask;
                    q.z |= omask;
                    my_rec[s] = q;
                }
                if (umask) {
                    const int k = min(32, ehi - base);
                    for (int j = 0; j < k; ++j) {
                        const int32_t sj = __shfl_sync(FULL, s, j);
                        const uint32_t orj = __shfl_sync(FULL, old_reach, j);
                        const uint32_t ooj = __shfl_sync(FULL, old_over, j);
                        if (under && !((ooj >> lane) & 1u)) {
                            V *a = my_acc + (sj & wmask) * 32 + lane;
                            if ((orj >> lane) & 1u) {
                                if (V(L) > *a) *a = V(L);
                            } else {
                                *a = V(L);
                            }
                        }
                        hi = max(hi, sj);
                    }
                }
            }
            __syncwarp();
        }
        if (lane < n_src) ie_out[tb + v0 + lane] = cnt;
        __syncwarp();
    }
}

// Self-test of the bounded wait (failure detection without a GPU fault): one
// warp waits for flag == value with at most `limit` polls; status gets
// INSP_ETIMEOUT if the wait gave up.
__global__ void k_wait_probe(const int32_t *flag, int32_t value, int32_t limit, int32_t *status) {
    __shared__ int32_t s_abort;
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    const bool ok = wait_flag(flag, value, &s_abort, limit);
    if (threadIdx.x == 0) *status = ok ? INSP_OK : INSP_ETIMEOUT;
}

void launch_wait_probe(const int32_t *flag, int32_t value, int32_t limit, int32_t *status, cudaStream_t s) {
    k_wait_probe<<<1, 32, 0, s>>>(flag, value, limit, status);
}

// Start of an attributes step: the done-flag epoch and the record tags advance
// (device-side, so a recorded CUDA graph replays correctly).
__global__ void k_step_begin(StepCounters *c, int64_t n_items) {
    c->epoch += 1;
    c->tag_base += uint64_t(n_items);
}

void launch_step_begin(StepCounters *c, int64_t n_items, cudaStream_t s) { k_step_begin<<<1, 1, 0, s>>>(c, n_items); }

void launch_ia(const DevBatch &B, const int32_t *order, int32_t n_order, int32_t *counter, uint64_t *bits,
               int64_t slot_words, int32_t *done, const int32_t *epoch, int32_t *ia, int32_t *status, int grid,
               int warps, cudaStream_t s) {
    k_ia<<<grid, 32 * warps, 0, s>>>(B, order, n_order, counter, bits, slot_words, done, epoch, ia, status);
}

void launch_ie(const DevBatch &B, const int64_t *item_base, int64_t n_items, int32_t *counter,
               const int64_t *unit_time, uint4 *rec, int64_t rec_stride, void *acc, int32_t W, bool wide,
               const uint64_t *tag_base, int32_t *ie, int grid, cudaStream_t s) {
    if (wide)
        k_ie<int64_t><<<grid, 256, 0, s>>>(B, item_base, n_items, counter, unit_time, rec, rec_stride,
                                           (int64_t *)acc, W, tag_base, ie);
    else
        k_ie<int32_t><<<grid, 256, 0, s>>>(B, item_base, n_items, counter, unit_time, rec, rec_stride,
                                           (int32_t *)acc, W, tag_base, ie);
}

int ia_max_warps() { return IA_MAX_WARPS; }
int ie_threads() { return 256; }
int ia_occupancy(int warps) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ia, 32 * warps, 0) != cudaSuccess) return 0;
    return nb;
}
int ie_occupancy() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ie<int64_t>, 256, 0) != cudaSuccess) return 0;
    return nb;
}

}  // namespace insp
