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

#include <algorithm>

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

// Inspiring ability at any DAG size: the target ids are cut into blocks of IA_BLK_BITS, and one
// CTA sweeps one (DAG, block) work item.  Within block j = [b0, b1) the row of task v is
// row_j(v) = ({v} if v is in the block) | OR over successors s of row_j(s); a successor at or
// above b1 adds nothing (its descendants come after it), so the sweep runs from b1 - 1 down to
// task 0, and IA(v) = sum over blocks of popcount(row_j(v)) - 1.  A row is read only by
// predecessors at most `span` ids below it (the DAG's longest edge), so rows live in a ring of
// R >= span + warps slots: the CTA's warps take the tasks in waves of one task per warp, the
// waves separated by a barrier, so when a slot is overwritten every reader of its previous row
// has finished.  Within a wave a task waits (bounded) for its successors' publish flags, which
// carry the item's tag and the task id.  Memory per CTA: R x (IA_BLK_BITS / 8 + 8) bytes,
// independent of the DAG's size.  Partial counts are added to ia (zeroed first) atomically.
// Full rows: a row holding the whole block (every target id a descendant) is published with a
// full mark and never written; a task with a full successor is full itself (its row contains
// the successor's), so the long stretch of a sweep below a block -- where most tasks reach all
// of it -- costs a flag read per successor instead of the successors' rows.
constexpr unsigned long long IA_FULL = 1ull << 31;  // in the task-id half of a flag (ids < 2^24)
__device__ __forceinline__ bool wait_key(const unsigned long long *flag, unsigned long long key, int32_t *abort,
                                         int limit, bool &full) {
    int it = 0;
    unsigned long long f;
    while (((f = *(const volatile unsigned long long *)flag) & ~IA_FULL) != key) {
        if (++it > limit || ld_volatile(abort)) {
            st_volatile(abort, 1);
            return false;
        }
        __nanosleep(64);
    }
    full = (f & IA_FULL) != 0;
    return true;
}

__global__ void __launch_bounds__(IA_MAX_WARPS * 32) k_ia_blk(DevBatch B, const int2 *items, int32_t n_items,
                                                              int32_t *counter, uint64_t *ring,
                                                              unsigned long long *flags, int32_t ring_rows,
                                                              uint32_t *slot_seq, int32_t *ia_out, int32_t *status) {
    __shared__ int32_t s_item;
    __shared__ uint32_t s_tag;
    __shared__ int32_t s_abort;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint64_t *R = ring + int64_t(blockIdx.x) * ring_rows * IA_BLK_WORDS;
    unsigned long long *F = flags + int64_t(blockIdx.x) * ring_rows;
    const int32_t rmask = ring_rows - 1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int k = atomicAdd(counter, 1);
            s_item = k < n_items ? k : -1;
            if (k < n_items) {
                s_tag = slot_seq[blockIdx.x] + 1;  // unique per item of this CTA (flags start at 0)
                slot_seq[blockIdx.x] = s_tag;
            }
            s_abort = 0;
        }
        __syncthreads();
        if (s_item < 0) return;
        const int2 it = items[s_item];
        const int d = it.x;
        const int64_t tb = B.task_base[d], eb = B.edge_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        const int32_t b0 = it.y * IA_BLK_BITS, b1 = min(n, b0 + IA_BLK_BITS);
        const int32_t NWb = (b1 - b0 + 63) >> 6;
        const int32_t *rp = B.row_ptr + tb + d;
        const int32_t *col = B.col_idx + eb;
        const unsigned long long tag = (unsigned long long)s_tag << 32;
        bool timed_out = false;
        for (int32_t top = b1 - 1; top >= 0; top -= nwarps) {
            const int32_t v = top - wib;
            if (v >= 0) {
                const int32_t lo = rp[v], hi = rp[v + 1];
                // successors below b1 (the list is ascending), each waited for (bounded)
                int32_t deg = 0;
                bool any_full = false;
                for (int32_t base = lo; base < hi; base += 32) {
                    const int32_t i = base + lane;
                    const int32_t s = i < hi ? col[i] : b1;
                    const bool in = s < b1;
                    bool full = false;
                    if (in && insp_check(s > v && s - v < ring_rows, status + d) &&
                        !wait_key(F + (s & rmask), tag | uint32_t(s), &s_abort, SPIN_LIMIT, full))
                        timed_out = true;
                    any_full |= __ballot_sync(FULL, full) != 0;
                    const uint32_t m = __ballot_sync(FULL, in);
                    deg += __popc(m);
                    if (m != FULL) break;
                }
                __syncwarp();
                __threadfence_block();
                if (any_full) {  // v reaches the whole block (so v < b0: a row at or above b0 holds no id below it)
                    if (lane == 0) {
                        *(volatile unsigned long long *)(F + (v & rmask)) = tag | uint32_t(v) | IA_FULL;
                        atomicAdd(ia_out + tb + v, b1 - b0 - (v >= b0 ? 1 : 0));
                    }
                } else {
                    const bool own = v >= b0;
                    const int32_t wlo = own ? (v - b0) >> 6 : 0;
                    const int32_t span_w = NWb - wlo;
                    const int32_t lg = span_w >= 32 ? 5 : (span_w <= 1 ? 0 : 32 - __clz(span_w - 1));
                    const int32_t g = 1 << lg;
                    const int32_t G = 32 >> lg, grp = lane >> lg, wl = lane & (g - 1);
                    uint64_t *row_v = R + int64_t(v & rmask) * IA_BLK_WORDS;
                    int32_t count = 0;
                    for (int32_t cw = wlo; cw < NWb; cw += g) {
                        const int32_t w = cw + wl;
                        uint64_t acc = (own && grp == 0 && w == wlo) ? (1ull << ((v - b0) & 63)) : 0ull;
#pragma unroll 4
                        for (int32_t i = grp; i < deg; i += G) {
                            const int32_t s = col[lo + i];
                            // words of row(s) below its own first word were not written for it
                            const int32_t ws = s >= b0 ? (s - b0) >> 6 : 0;
                            if (w >= ws && w < NWb) acc |= R[int64_t(s & rmask) * IA_BLK_WORDS + w];
                        }
                        for (int32_t off = g; off < 32; off <<= 1) acc |= __shfl_xor_sync(FULL, acc, off);
                        if (grp == 0 && w < NWb) {
                            row_v[w] = acc;
                            count += __popcll(acc);
                        }
                    }
                    count = __reduce_add_sync(FULL, count);
                    const bool full = count == b1 - b0;
                    count -= own ? 1 : 0;
                    __threadfence_block();
                    __syncwarp();
                    if (lane == 0) {
                        *(volatile unsigned long long *)(F + (v & rmask)) = tag | uint32_t(v) | (full ? IA_FULL : 0ull);
                        if (count > 0) atomicAdd(ia_out + tb + v, count);
                    }
                }
            }
            __syncthreads();
        }
        timed_out = __syncthreads_or(timed_out);
        if (timed_out && threadIdx.x == 0) status[d] = INSP_ETIMEOUT;
    }
}

// Zero the inspiring ability of the listed DAGs (before k_ia_blk adds its partial counts).
__global__ void k_ia_zero(DevBatch B, const int32_t *dags, int32_t n_dags, int32_t *ia) {
    for (int k = blockIdx.x; k < n_dags; k += gridDim.x) {
        const int d = dags[k];
        const int64_t tb = B.task_base[d], te = B.task_base[d + 1];
        for (int64_t t = tb + threadIdx.x; t < te; t += blockDim.x) ia[t] = 0;
    }
}

// A DAG whose structure (tasks, successor lists) equals an earlier one's takes its inspiring
// ability, which depends on nothing else: pairs[k] = {dag, representative}.
__global__ void k_ia_copy(DevBatch B, const int2 *pairs, int32_t n_pairs, int32_t *ia) {
    for (int k = blockIdx.x; k < n_pairs; k += gridDim.x) {
        const int2 p = pairs[k];
        const int64_t td = B.task_base[p.x], tr = B.task_base[p.y];
        const int64_t n = B.task_base[p.x + 1] - td;
        for (int64_t t = threadIdx.x; t < n; t += blockDim.x) ia[td + t] = ia[tr + t];
    }
}

// Exact comparison of candidate pairs {dag, representative} of equal fingerprints, task counts
// and edge counts: same[k] = 1 when their row offsets and successor ids are equal.
__global__ void __launch_bounds__(256) k_dag_equal(DevBatch B, const int2 *pairs, int32_t n_pairs, int32_t *same) {
    __shared__ int32_t s_diff;
    for (int k = blockIdx.x; k < n_pairs; k += gridDim.x) {
        if (threadIdx.x == 0) s_diff = 0;
        __syncthreads();
        const int2 p = pairs[k];
        const int64_t ta = B.task_base[p.x], tr = B.task_base[p.y];
        const int64_t n = B.task_base[p.x + 1] - ta, m = B.edge_base[p.x + 1] - B.edge_base[p.x];
        const int32_t *ra = B.row_ptr + ta + p.x, *rr = B.row_ptr + tr + p.y;
        const int32_t *ca = B.col_idx + B.edge_base[p.x], *cr = B.col_idx + B.edge_base[p.y];
        bool diff = n != B.task_base[p.y + 1] - tr || m != B.edge_base[p.y + 1] - B.edge_base[p.y];
        if (!diff) {
            for (int64_t i = threadIdx.x; i <= n && !diff; i += blockDim.x) diff = ra[i] != rr[i];
            for (int64_t e = threadIdx.x; e < m && !diff; e += blockDim.x) diff = ca[e] != cr[e];
        }
        if (diff) s_diff = 1;
        __syncthreads();
        if (threadIdx.x == 0) same[k] = s_diff ? 0 : 1;
        __syncthreads();
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

void launch_ia_blk(const DevBatch &B, const int2 *items, int32_t n_items, int32_t *counter, uint64_t *ring,
                   unsigned long long *flags, int32_t ring_rows, uint32_t *slot_seq, int32_t *ia, int32_t *status,
                   int grid, int warps, cudaStream_t s) {
    k_ia_blk<<<grid, 32 * warps, 0, s>>>(B, items, n_items, counter, ring, flags, ring_rows, slot_seq, ia, status);
}
void launch_ia_zero(const DevBatch &B, const int32_t *dags, int32_t n_dags, int32_t *ia, cudaStream_t s) {
    if (n_dags > 0) k_ia_zero<<<std::min(n_dags, 4096), 256, 0, s>>>(B, dags, n_dags, ia);
}
void launch_ia_copy(const DevBatch &B, const int2 *pairs, int32_t n_pairs, int32_t *ia, cudaStream_t s) {
    if (n_pairs > 0) k_ia_copy<<<std::min(n_pairs, 4096), 256, 0, s>>>(B, pairs, n_pairs, ia);
}
void launch_dag_equal(const DevBatch &B, const int2 *pairs, int32_t n_pairs, int32_t *same, cudaStream_t s) {
    if (n_pairs > 0) k_dag_equal<<<std::min(n_pairs, 4096), 256, 0, s>>>(B, pairs, n_pairs, same);
}
int ia_blk_occupancy(int warps) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ia_blk, 32 * warps, 0) != cudaSuccess) return 0;
    return nb;
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
