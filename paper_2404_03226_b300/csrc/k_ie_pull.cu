// Inspiring efficiency (Sec. 4.2 / Sec. 4.3), "pull" form of the window sweep.
//
// A warp owns IE_PULL_SOURCES = 64 consecutive sources (two codes per lane) and
// visits every task u = v0, v0+1, ... in id order (a topological order).  It
// keeps, per task, the 64 codes in a row of a ring of W rows (W a power of two
// above every edge span, so every predecessor of u is still in the ring):
//     "out"      u is not in the source's cone,
//     L in 1..T  u is in the cone and every path from the source to u weighs L
//                or less (L = the longest path weight, GPU costs, both ends),
//     OVER       u is in the cone but some path weighs more than T.
// The codes are ordered out < 1..T < OVER, so a plain max over predecessors
// combines them:
//     val_j(u) = source ? (c(u) <= T ? c(u) : OVER)
//              : m = max over predecessors q >= v0 of val_j(q);
//                m = out ? out : (m == OVER ? OVER : (m + c(u) <= T ? m + c(u) : OVER))
// and IE(v_j) counts the tasks whose value lands in 1..T (the source excluded).
// With T < 2^16 - 1 a code is 16 bits (out = 0, OVER = 0xffff) and a lane's two
// codes share one word, combined by a packed max; otherwise 32 bits (out = -1,
// OVER = 2^31 - 1).  The choice is made per work item from its DAG's T.
// The sweep stops after the last task that received an in-window value from a
// predecessor (tracked through each in-window task's largest successor id).
// Predecessor lists (built at ingest) and GPU costs of the next 32 tasks are
// staged into shared memory with coalesced loads; predecessors older than the
// sources (outside every source's cone) are dropped while staging.  The ring is a
// per-warp slice of global memory meant to stay in L2 (a shared-memory ring was
// measured slower: at 33 KB per warp it caps residency at 6 warps per SM).  With
// 32-bit codes each lane only reads its own column (its own earlier writes); with
// 16-bit codes lanes read words other lanes wrote, so a __syncwarp orders every
// row's store before the later visits' loads.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace insp {

constexpr int PULL_MAX_WARPS = 16;  // warps per CTA: blockDim / 32 (autotuned)
constexpr int PCH = 32;      // tasks per staged chunk
constexpr int PCOL = 768;    // staged predecessor ids per chunk (longer chunks read the rest from global)
constexpr int32_t OVER = 0x7fffffff;
constexpr int SPW = IE_PULL_SOURCES;  // sources per warp: lane j owns v0 + j + 32 q, q < NV
constexpr int NV = SPW / 32;          // codes per lane
// Predecessor rows loaded per round before they are combined, and the register cap that
// holds them (8 rows at 56 registers, 36 resident warps per SM, measured best of 4/48,
// 6/56, 8/56 and 8/64 on the layered workload).
#ifndef IE_PULL_MAXREG
#define IE_PULL_MAXREG 56
#endif
#ifndef IE_PULL_INFLIGHT
#define IE_PULL_INFLIGHT 8
#endif
// Narrow codes: 16-byte loads per lane, so one load instruction of the warp fetches four
// predecessor rows (lanes 8 g .. 8 g + 7 read row e + g); IE_PULL_NARROW_LOADS of them per lane
// are in flight per round (4 x that many rows; on the layered workload 2 and 4 alike, 8
// slower).  The same gather for 32-bit codes (two 256-byte rows per load, six or four rows in
// flight) was measured slower than the lane-owned rows below: tiled 16 + 32 sweep 36.4 against
// 34.0 ms.
#ifndef IE_PULL_NARROW_LOADS
#define IE_PULL_NARROW_LOADS 4
#endif

// NV codes per lane, moved as one vector
template <int V> struct CodeVec;
template <> struct CodeVec<2> { using T = int2; };
template <> struct CodeVec<4> { using T = int4; };
using Codes = CodeVec<NV>::T;
__device__ __forceinline__ int32_t cget(const int2 &a, int q) { return q == 0 ? a.x : a.y; }
__device__ __forceinline__ int32_t cget(const int4 &a, int q) { return q == 0 ? a.x : q == 1 ? a.y : q == 2 ? a.z : a.w; }
__device__ __forceinline__ int2 cmake(const int32_t (&v)[2]) { return make_int2(v[0], v[1]); }
__device__ __forceinline__ int4 cmake(const int32_t (&v)[4]) { return make_int4(v[0], v[1], v[2], v[3]); }

// Narrow codes: when T <= NARROW_T_MAX a code fits 16 bits, unsigned and ordered the same way
// (0 = outside the cone, 1..T = in the window, 0xffff = OVER), two to a 32-bit word: half the
// ring bytes, and one packed max per word.  A narrow row is 32 words, word w holding sources
// 2w and 2w + 1 (low half first).  Lane 8 g + s gathers with 16-byte loads: bytes 16 s .. 16 s + 15
// of the rows e + g, e + 4 + g, ..., so one load instruction covers four rows; a reduce-scatter
// over the four lane groups then leaves lane 8 g + s with word 4 s + g, i.e. sources
// 8 s + 2 g and 8 s + 2 g + 1, which it combines with the task's cost and stores.
constexpr int64_t NARROW_T_MAX = 0xfffe;
constexpr uint32_t NOVER = 0xffff;
static_assert(NV == 2, "narrow codes pack the two codes of a lane into one word");
__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// ring of W rows of 32 lanes x NV values (the narrow rows use the first half)
__host__ __device__ constexpr int64_t ie_ring_bytes(int32_t W) { return int64_t(W) * 32 * 4 * NV; }
// per warp shared memory: the chunk staging
constexpr int64_t IE_PULL_STAGE_BYTES = ((PCH + 1 + PCH + PCH + PCOL + PCH + 1) * 4 + 15) / 16 * 16;
// DAGs whose longest edge spans more tasks than this take the sparse sweep.  With long edges the
// in-window tasks' far successors stretch the sweep over many tasks outside every cone (tiled LU
// at 32 tiles: 22 % of the visited tasks in a cone, 83 % of the predecessor rows read all
// "out").  There a W-bit ring bitmap records which rows hold codes (the task is in some cone);
// a task reads only those predecessors' rows, and a task with none (not a source) is outside
// every cone: its row is neither computed nor stored.
constexpr int32_t SPARSE_SPAN = 256;
// per warp shared memory of a launch with window W: the staging, then the row bitmap when some
// DAG may take the sparse sweep (W > SPARSE_SPAN + 1)
__host__ __device__ constexpr int64_t ie_stage_bytes(int32_t W) {
    return IE_PULL_STAGE_BYTES + (W > SPARSE_SPAN + 1 ? (int64_t(W) / 8 + 15) / 16 * 16 : 0);
}

// One work item's sweep state and the warp's chunk staging.
struct PullItem {
    const int32_t *pp, *pc, *rp, *col;
    int64_t tb, T;
    int32_t d, n, v0, n_src, wmask;
    int32_t *c_pp, *c_cost, *c_msucc, *c_off, *c_kp;
    uint32_t *live;  // sparse sweep: W-bit ring bitmap of the rows that hold codes
};

// Stage the chunk of tasks u .. u + PCH - 1: predecessor offsets, GPU costs (clamped to
// T + 1), largest successor ids, and the first `ne` predecessor ids of the chunk, keeping
// only those >= v0 (older ones are outside every source's cone) compacted by ballot as ring
// row offsets; each task's first kept entry is found from its boundary b_k (lane k; lane 0
// also the chunk's end).  Returns e0 (the chunk's first edge) and ne.
__device__ __forceinline__ void stage_chunk(const DevBatch &B, const PullItem &I, int32_t u, int lane, int32_t &e0,
                                            int32_t &ne) {
    __syncwarp();
    const int32_t t = min(u + lane, I.n);
    I.c_pp[lane] = I.pp[t];
    if (lane == 0) I.c_pp[PCH] = I.pp[min(u + PCH, I.n)];
    if (u + lane < I.n) {
        const int64_t cg = task_cost(B, I.d, I.tb + u + lane, 1);
        I.c_cost[lane] = int32_t(cg > I.T ? I.T + 1 : cg);
        const int32_t r0 = I.rp[u + lane], r1 = I.rp[u + lane + 1];
        I.c_msucc[lane] = r1 > r0 ? I.col[r1 - 1] : -1;
    }
    __syncwarp();
    e0 = I.c_pp[0];
    ne = min(I.c_pp[PCH] - e0, PCOL);
    const int32_t b_k = I.c_pp[lane] - e0;
    int32_t kp = 0, base = 0;
    for (int r0 = 0; r0 < PCOL / 32 && 32 * r0 < ne; r0 += 8) {
        int32_t qv[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int32_t i = lane + 32 * (r0 + r);
            qv[r] = i < ne ? __ldg(I.pc + e0 + i) : -1;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int32_t i0 = 32 * (r0 + r);
            const bool keep = qv[r] >= I.v0;  // -1 past ne
            const uint32_t bal = __ballot_sync(FULL, keep);
            if (keep) I.c_off[base + __popc(bal & ((1u << lane) - 1))] = (qv[r] & I.wmask) * 32;
            if (b_k >= i0 && b_k < i0 + 32) kp = base + __popc(bal & ((1u << (b_k - i0)) - 1));
            base += __popc(bal);
        }
    }
    I.c_kp[lane] = b_k >= ne ? base : kp;
    if (lane == 0) I.c_kp[PCH] = base;
    __syncwarp();
}

// The sweep of one work item.  R: the ring's row element per lane (Codes: NV int32 codes;
// uint32_t: two narrow codes).  Adds each source's count to cnt.
template <bool NARROW, bool SPARSE>
__device__ __forceinline__ void sweep_item(const DevBatch &B, const PullItem &I, void *ring, int lane,
                                           int32_t (&cnt)[NV]) {
    using R = typename std::conditional<NARROW, uint32_t, Codes>::type;
    R *__restrict__ val = reinterpret_cast<R *>(ring);
    int32_t hi = I.v0 + I.n_src - 1;
    int32_t uc = -1, e0 = 0, ne = 0;  // first task, first predecessor edge and staged entries of the chunk
    for (int32_t u = I.v0; u <= hi; ++u) {
        if (uc < 0 || u - uc >= PCH) {
            uc = u;
            stage_chunk(B, I, u, lane, e0, ne);
        }
        const int32_t k = u - uc;
        const int32_t lo = I.c_pp[k] - e0, hi_p = I.c_pp[k + 1] - e0;
        // staged entries of this task (compacted), then any beyond the staging from global
        const int32_t clo = I.c_kp[k];
        int32_t chi = hi_p <= ne ? I.c_kp[k + 1] : I.c_kp[PCH];
        const int32_t r_u = u & I.wmask;
        if (SPARSE) {
            // keep the staged predecessors whose rows hold codes, compacted in place (a round's
            // writes land at or below its reads; every row read was visited earlier in this item)
            int32_t nl = 0;
            for (int32_t e = clo; e < chi; e += 32) {
                const int32_t i = e + lane;
                int32_t off = 0;
                bool keep = false;
                if (i < chi) {
                    off = I.c_off[i];
                    const int32_t r = off >> 5;
                    keep = (I.live[r >> 5] >> (r & 31)) & 1u;
                }
                const uint32_t bal = __ballot_sync(FULL, keep);
                if (keep) I.c_off[clo + nl + __popc(bal & ((1u << lane) - 1))] = off;
                nl += __popc(bal);
            }
            __syncwarp();
            chi = clo + nl;
            if (nl == 0 && hi_p <= ne && u - I.v0 >= SPW) {  // outside every cone: no row
                if (lane == 0) I.live[r_u >> 5] &= ~(1u << (r_u & 31));
                __syncwarp();
                continue;
            }
        }
        // wide codes: predecessor rows in flight per round; the last round's loads are predicated
        constexpr int U = IE_PULL_INFLIGHT;
        const int32_t c = I.c_cost[k];
        int32_t vv[NV];
        bool any_in = false, any_cone = false;
        if (NARROW) {
            // gather: lane 8 g + s folds bytes 16 s .. 16 s + 15 of the rows e + 4 i + g (0 = outside,
            // the max's identity, for the rows past the task's list)
            constexpr int NL = IE_PULL_NARROW_LOADS;
            const int s8 = lane & 7, g4 = lane >> 3;
            const uint4 *__restrict__ v4 = reinterpret_cast<const uint4 *>(val) + s8;
            uint4 acc = make_uint4(0u, 0u, 0u, 0u);
            for (int32_t e = clo; e < chi; e += 4 * NL) {
                uint4 pv[NL];
#pragma unroll
                for (int r = 0; r < NL; ++r) {
                    const int32_t i = e + 4 * r + g4;
                    pv[r] = i < chi ? v4[I.c_off[i] >> 2] : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int r = 0; r < NL; ++r) {
                    acc.x = max_u16x2(acc.x, pv[r].x);
                    acc.y = max_u16x2(acc.y, pv[r].y);
                    acc.z = max_u16x2(acc.z, pv[r].z);
                    acc.w = max_u16x2(acc.w, pv[r].w);
                }
            }
            // predecessors beyond the staging, from global: lane group g takes every fourth
            for (int32_t f = max(lo, ne) + g4; f < hi_p; f += 4) {
                const int32_t qd = I.pc[e0 + f];
                const int32_t rq = qd & I.wmask;
                if (qd >= I.v0 && (!SPARSE || ((I.live[rq >> 5] >> (rq & 31)) & 1u))) {
                    const uint4 x = v4[rq * 8];
                    acc.x = max_u16x2(acc.x, x.x);
                    acc.y = max_u16x2(acc.y, x.y);
                    acc.z = max_u16x2(acc.z, x.z);
                    acc.w = max_u16x2(acc.w, x.w);
                }
            }
            // reduce-scatter over the four lane groups: first groups g and g ^ 2 keep words
            // 2 (g >> 1) and 2 (g >> 1) + 1 of the slice, then g and g ^ 1 keep word g
            const bool hi2 = (g4 >> 1) != 0, hi1 = (g4 & 1) != 0;
            uint32_t k0 = hi2 ? acc.z : acc.x, k1 = hi2 ? acc.w : acc.y;
            k0 = max_u16x2(k0, __shfl_xor_sync(FULL, hi2 ? acc.x : acc.z, 16));
            k1 = max_u16x2(k1, __shfl_xor_sync(FULL, hi2 ? acc.y : acc.w, 16));
            const uint32_t m2 = max_u16x2(hi1 ? k1 : k0, __shfl_xor_sync(FULL, hi1 ? k0 : k1, 8));
            // T <= 0xfffe and c <= T + 1: m + c fits 32 bits and fits the window iff <= T
            const uint32_t own = uint32_t(c) <= uint32_t(I.T) ? uint32_t(c) : NOVER;
            const int32_t j0 = 8 * s8 + 2 * g4;  // this lane's sources: v0 + j0, v0 + j0 + 1
            uint32_t packed = 0;
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const uint32_t m = (m2 >> (16 * q)) & 0xffffu;
                const bool live = m != 0 && m != NOVER;
                const uint32_t L = m + uint32_t(c);
                const bool fits = live && L <= uint32_t(I.T);
                uint32_t v = live ? (fits ? L : NOVER) : m;
                if (u - I.v0 == j0 + q) v = own;
                cnt[q] += fits;
                any_in |= v != 0 && v != NOVER;
                any_cone |= v != 0;
                packed |= v << (16 * q);
            }
            if (!SPARSE || __any_sync(FULL, any_cone))
                reinterpret_cast<uint32_t *>(val)[r_u * 32 + 4 * s8 + g4] = packed;
            __syncwarp();  // the row is read by other lanes at later visits
            (void)vv;
        } else {
            int32_t ma[NV], mb[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) ma[q] = mb[q] = -1;
            int32_t e = clo;
            for (; e + U <= chi; e += U) {
                Codes pv[U];
#pragma unroll
                for (int r = 0; r < U; ++r) pv[r] = reinterpret_cast<const Codes *>(val)[I.c_off[e + r] + lane];
#pragma unroll
                for (int r = 0; r < U; r += 2)
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        ma[q] = max(ma[q], cget(pv[r], q));
                        mb[q] = max(mb[q], cget(pv[r + 1], q));
                    }
            }
            if (e < chi) {
                Codes pv[U];
#pragma unroll
                for (int r = 0; r < U; ++r)
                    pv[r] = e + r < chi ? reinterpret_cast<const Codes *>(val)[I.c_off[e + r] + lane] : cmake({-1, -1});
#pragma unroll
                for (int r = 0; r < U; r += 2)
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        ma[q] = max(ma[q], cget(pv[r], q));
                        mb[q] = max(mb[q], cget(pv[r + 1], q));
                    }
            }
            for (int32_t f = max(lo, ne); f < hi_p; ++f) {
                const int32_t qd = I.pc[e0 + f];
                const int32_t rq = qd & I.wmask;
                if (qd >= I.v0 && (!SPARSE || ((I.live[rq >> 5] >> (rq & 31)) & 1u))) {
                    const Codes x = reinterpret_cast<const Codes *>(val)[rq * 32 + lane];
#pragma unroll
                    for (int q = 0; q < NV; ++q) ma[q] = max(ma[q], cget(x, q));
                }
            }
            const int32_t own = c <= int32_t(I.T) ? c : OVER;
            // branch-free: T < 2^31 here, so m + c (both <= T + 1) fits in 32 unsigned bits.  A
            // source's own m is -1 (tasks before a source are outside its cone).
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const int32_t m = max(ma[q], mb[q]);
                const bool live = m >= 0 && m != OVER;
                const uint32_t L = uint32_t(m) + uint32_t(c);
                const bool fits = live && L <= uint32_t(I.T);
                int32_t v = live ? (fits ? int32_t(L) : OVER) : m;
                if (u - I.v0 == lane + 32 * q) v = own;
                cnt[q] += fits;
                vv[q] = v;
                any_in |= v >= 0 && v != OVER;
                any_cone |= v >= 0;
            }
            if (!SPARSE || __any_sync(FULL, any_cone)) reinterpret_cast<Codes *>(val)[r_u * 32 + lane] = cmake(vv);
        }
        if (SPARSE) {
            const bool cone = __any_sync(FULL, any_cone);
            if (lane == 0) {
                const uint32_t bit = 1u << (r_u & 31);
                I.live[r_u >> 5] = cone ? (I.live[r_u >> 5] | bit) : (I.live[r_u >> 5] & ~bit);
            }
            __syncwarp();
        }
        if (__any_sync(FULL, any_in)) hi = max(hi, I.c_msucc[k]);
    }
}

// A register cap keeps more warps resident than the 64 registers a free compile takes.
__global__ void __maxnreg__(IE_PULL_MAXREG)
    k_ie_pull(DevBatch B, const int32_t *pr_ptr, const int32_t *pcol, const int64_t *item_base,
              const int32_t *item_dag, int64_t item_lo, int64_t item_hi, int32_t *counter,
              const int64_t *unit_time, const int32_t *dag_span, int32_t W, int32_t *gring, int32_t *ie_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char *mine = smem + int64_t(wib) * ie_stage_bytes(W);
    void *ring = reinterpret_cast<unsigned char *>(gring) +
                 (int64_t(blockIdx.x) * (blockDim.x >> 5) + wib) * ie_ring_bytes(W);
    PullItem I;
    I.c_pp = reinterpret_cast<int32_t *>(mine);  // chunk predecessor offsets
    I.c_cost = I.c_pp + PCH + 1;                 // GPU costs, clamped to T + 1
    I.c_msucc = I.c_cost + PCH;                  // largest successor id (-1: none)
    I.c_off = I.c_msucc + PCH;                   // ring row offsets of the staged predecessors >= v0
    I.c_kp = I.c_off + PCOL;                     // per task: its first entry in c_off
    I.live = reinterpret_cast<uint32_t *>(mine + IE_PULL_STAGE_BYTES);

    for (;;) {
        int64_t item = 0;
        if (lane == 0) item = item_lo + atomicAdd(counter, 1);
        item = __shfl_sync(FULL, item, 0);
        if (item >= item_hi) return;
        I.d = item_dag[item];
        I.tb = B.task_base[I.d];
        const int64_t eb = B.edge_base[I.d];
        I.n = int32_t(B.task_base[I.d + 1] - I.tb);
        I.v0 = int32_t(item - item_base[I.d]) * SPW;
        I.n_src = min(SPW, I.n - I.v0);
        I.rp = B.row_ptr + I.tb + I.d;
        I.col = B.col_idx + eb;
        I.pp = pr_ptr + I.tb + I.d;
        I.pc = pcol + eb;
        I.T = unit_time[I.d];
        // this DAG's own window: a power of two above its longest edge span (at most W), so a DAG
        // with short edges touches only the first rows of the ring
        I.wmask = (1 << (32 - __clz(dag_span[I.d]))) - 1;

        int32_t cnt[NV];  // per source v0 + lane + 32 q
#pragma unroll
        for (int q = 0; q < NV; ++q) cnt[q] = 0;
        const bool sparse = dag_span[I.d] > SPARSE_SPAN;  // then W > SPARSE_SPAN + 1: the bitmap exists
        const bool narrow = I.T <= NARROW_T_MAX;
        if (narrow) {
            if (sparse) sweep_item<true, true>(B, I, ring, lane, cnt);
            else sweep_item<true, false>(B, I, ring, lane, cnt);
        } else {
            if (sparse) sweep_item<false, true>(B, I, ring, lane, cnt);
            else sweep_item<false, false>(B, I, ring, lane, cnt);
        }
        // the sources of this lane's counts: 8 s + 2 g + q with narrow codes (lane 8 g + s), else lane + 32 q
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const int32_t j = narrow ? 8 * (lane & 7) + 2 * (lane >> 3) + q : lane + 32 * q;
            if (j < I.n_src) ie_out[I.tb + I.v0 + j] = cnt[q];
        }
        __syncwarp();
    }
}

// Exclusive prefix sum over the 256 threads of a CTA (8 warps): returns this thread's offset and
// the CTA total.  s_w: 8 ints of shared memory, free again when the call returns.
__device__ __forceinline__ int32_t cta_exclusive_scan(int32_t x, int32_t *s_w, int32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < 8 ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const int32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < 8) s_w[lane] = w;
    }
    __syncthreads();
    const int32_t before = warp ? s_w[warp - 1] : 0;
    total = s_w[7];
    __syncthreads();
    return before + incl - x;
}

// Predecessor lists of every DAG (CSR of the reversed edges, same layout as row_ptr / col_idx),
// one CTA of 256 threads per DAG: exclusive scan of the in-degrees (each thread a contiguous
// chunk, then a CTA scan of the chunk sums), then a scatter by one warp per row, its lanes over
// the row's successors (coalesced), with the insertion cursors in shared memory for DAGs of up to
// smem_n tasks (else in `cursor`).  Order within a list is irrelevant to the max.
__global__ void __launch_bounds__(256) k_reverse_csr(DevBatch B, const int32_t *indeg0, int32_t *pr_ptr,
                                                     int32_t *cursor, int32_t *pcol, int32_t smem_n) {
    extern __shared__ int32_t s_cur[];  // smem_n cursors
    __shared__ int32_t s_w[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = blockIdx.x; d < B.ndag; d += gridDim.x) {
        const int64_t tb = B.task_base[d], eb = B.edge_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        int32_t *pp = pr_ptr + tb + d;
        const bool in_smem = n <= smem_n;
        int32_t *cur = in_smem ? s_cur : cursor + tb;
        const int32_t chunk = (n + 255) / 256, c0 = min(n, int32_t(threadIdx.x) * chunk), c1 = min(n, c0 + chunk);
        int32_t sum = 0;
        for (int32_t i = c0; i < c1; ++i) sum += indeg0[tb + i];
        int32_t total;
        int32_t off = cta_exclusive_scan(sum, s_w, total);
        for (int32_t i = c0; i < c1; ++i) {
            pp[i] = off;
            cur[i] = off;
            off += indeg0[tb + i];
        }
        if (threadIdx.x == 0) pp[n] = total;
        __syncthreads();
        const int32_t *rp = B.row_ptr + tb + d;
        const int32_t *col = B.col_idx + eb;
        for (int32_t u = warp; u < n; u += 8) {
            const int32_t lo = rp[u], hi = rp[u + 1];
            for (int32_t e = lo + lane; e < hi; e += 32) {
                const int32_t v = col[e];
                pcol[eb + atomicAdd(&cur[v], 1)] = u;
            }
        }
        __syncthreads();
    }
}

int ie_pull_max_warps() { return PULL_MAX_WARPS; }
int64_t ie_pull_ring_bytes(int32_t W) { return ie_ring_bytes(W); }

int ie_pull_occupancy(int warps, int32_t W) {
    const int64_t bytes = ie_stage_bytes(W) * warps;
    int nb = 0;
    cudaFuncSetAttribute(k_ie_pull, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(ie_stage_bytes(IE_PULL_MAX_W) * PULL_MAX_WARPS));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ie_pull, warps * 32, size_t(bytes)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

void launch_ie_pull(const DevBatch &B, const int32_t *pr_ptr, const int32_t *pcol, const int64_t *item_base,
                    const int32_t *item_dag, int64_t item_lo, int64_t item_hi, int32_t *counter,
                    const int64_t *unit_time, const int32_t *dag_span, int32_t W, int32_t *gring, int32_t *ie,
                    int grid, int warps, cudaStream_t s) {
    cudaFuncSetAttribute(k_ie_pull, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(ie_stage_bytes(IE_PULL_MAX_W) * PULL_MAX_WARPS));
    k_ie_pull<<<grid, warps * 32, size_t(ie_stage_bytes(W) * warps), s>>>(B, pr_ptr, pcol, item_base, item_dag,
                                                                         item_lo, item_hi, counter, unit_time,
                                                                         dag_span, W, gring, ie);
}

void launch_reverse_csr(const DevBatch &B, const int32_t *indeg0, int32_t *pr_ptr, int32_t *cursor, int32_t *pcol,
                        int32_t max_n, int grid, cudaStream_t s) {
    const int32_t smem_n = std::max(0, std::min(max_n, VALIDATE_SMEM_TASKS));
    cudaFuncSetAttribute(k_reverse_csr, cudaFuncAttributeMaxDynamicSharedMemorySize, VALIDATE_SMEM_TASKS * 4);
    k_reverse_csr<<<grid, 256, size_t(smem_n) * 4, s>>>(B, indeg0, pr_ptr, cursor, pcol, smem_n);
}

}  // namespace insp
