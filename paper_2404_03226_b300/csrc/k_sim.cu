// The list-scheduling run of INSPIRIT (Sec. 2.1 push/pop, Sec. 4.1, Sec. 4.4),
// one warp per DAG.
//
// Lane l owns workers l and l + 32: their busy-until time, queued work,
// running task and queue count live in registers.  The ready tasks of all
// workers form one pool (Nready = pool size): the first POOL_C entries in
// shared memory, the rest spilled to the DAG's slice of a global pool.  Per
// task the warp keeps in global scratch the remaining in-degree and the two
// latest completion times of its predecessors on distinct memory nodes, which
// give the data-arrival time on any worker in O(1).
//
// Event loop (all lanes in lockstep, every decision warp-uniform):
//   completions at `now` release successors (lanes over the CSR row);
//   released tasks are pushed in ascending id (a P-way merge of the per
//   completion runs), each to the worker of minimum expected finish
//   (argmin of (finish << 6 | worker) by redux);
//   idle workers pop in ascending id: the Nready controller picks the mode
//   and an argmax over the pool of a 64-bit key (mode key, then lowest id)
//   selects the task.
#include "common.cuh"
#include "kernels.h"

#include <algorithm>

namespace insp {

constexpr int SIM_WARPS = 8;  // most warps per CTA (the autotuner may launch fewer)
// Successor row of a started task toward L1 (no register, no wait); its completion
// reads it several events later.  Measured 6 % off the simulation; prefetching the
// successors' release state and push inputs one event later as well cost more than it saved.
__device__ __forceinline__ void prefetch_row(const int32_t *p, int32_t lo, int32_t hi) {
    for (int32_t o = lo; o < hi; o += 32) asm volatile("prefetch.global.L1 [%0];" ::"l"(p + o));
    if (hi > lo) asm volatile("prefetch.global.L1 [%0];" ::"l"(p + hi - 1));
}
constexpr int NL_C = 128;     // released-task buffer per warp in shared memory
constexpr int NODE_NONE = 0xff;

enum { MODE_FIFO = 0, MODE_ABILITY = 1, MODE_EFI = 2, MODE_EFI_LOC = 3, MODE_LEARNED = 4, MODE_PRIO = 5 };
enum { ST_INC = 0, ST_DEC = 1 };

// Pools of at least MASK_MIN shared-memory entries keep, per worker, a bitmap of its entries
// there, so a pop visits only the popping worker's entries instead of the whole pool (the tiled
// DAGs hold hundreds of ready tasks over 20 workers, the 1,000,000-task layered DAG ~500 over
// 40).  Rows for 32 workers, or 64 when lanes own two workers (TWO).
constexpr int MASK_MIN = 128;
template <int POOL_C>
constexpr int mask_words() { return POOL_C >= MASK_MIN ? POOL_C / 32 : 1; }
template <int POOL_C, bool TWO>
constexpr int mask_rows() { return POOL_C >= MASK_MIN ? (TWO ? 64 : 32) : 1; }

// POOL_C: ready-pool entries per warp kept in shared memory (the queue
// capacity the autotuner picks; entries beyond it spill to global memory).
template <int POOL_C, bool TWO>
struct WarpSmem {
    int32_t idw[POOL_C];  // task id | worker << 24
    int32_t seq[POOL_C];
    int32_t ia[POOL_C];
    int32_t ie[POOL_C];
    int64_t dr[POOL_C];   // data arrival time on the queued worker
    int64_t cost[POOL_C]; // cost on the queued worker
    int32_t newly[NL_C];
    int32_t run_end[MAX_WORKERS];
    int64_t tcost[MAX_TYPES_SMEM * 2];
    uint32_t wmask[mask_rows<POOL_C, TWO>()][mask_words<POOL_C>()];  // entry bitmaps per worker
};

template <int POOL_C, bool TWO>
struct Pool {
    WarpSmem<POOL_C, TWO> *sm;
    int32_t *g_idw, *g_seq, *g_ia, *g_ie;
    int64_t *g_dr, *g_cost;
    __device__ __forceinline__ int32_t idw(int i) const { return i < POOL_C ? sm->idw[i] : g_idw[i - POOL_C]; }
    __device__ __forceinline__ int32_t seq(int i) const { return i < POOL_C ? sm->seq[i] : g_seq[i - POOL_C]; }
    __device__ __forceinline__ int32_t ia(int i) const { return i < POOL_C ? sm->ia[i] : g_ia[i - POOL_C]; }
    __device__ __forceinline__ int32_t ie(int i) const { return i < POOL_C ? sm->ie[i] : g_ie[i - POOL_C]; }
    __device__ __forceinline__ int64_t dr(int i) const { return i < POOL_C ? sm->dr[i] : g_dr[i - POOL_C]; }
    __device__ __forceinline__ int64_t cost(int i) const { return i < POOL_C ? sm->cost[i] : g_cost[i - POOL_C]; }
    __device__ __forceinline__ void set(int i, int32_t idw_, int32_t seq_, int32_t ia_, int32_t ie_, int64_t dr_,
                                        int64_t cost_) const {
        if (i < POOL_C) {
            sm->idw[i] = idw_; sm->seq[i] = seq_; sm->ia[i] = ia_; sm->ie[i] = ie_; sm->dr[i] = dr_; sm->cost[i] = cost_;
        } else {
            int j = i - POOL_C;
            g_idw[j] = idw_; g_seq[j] = seq_; g_ia[j] = ia_; g_ie[j] = ie_; g_dr[j] = dr_; g_cost[j] = cost_;
        }
    }
    // copy entry `from` into slot `to`: one lane (lane 0, or the caller's lane when `mine`),
    // its six independent loads in flight together (one lane per field would serialise six
    // divergent paths)
    __device__ __forceinline__ void move(int from, int to, int lane, bool mine = false) const {
        if (mine || lane == 0) set(to, idw(from), seq(from), ia(from), ie(from), dr(from), cost(from));
    }
};

// Nready controller (Sec. 4.4 pseudocode), warp-uniform state.
struct Ctrl {
    int64_t peak, prev_n, prev_t, count;
    int32_t mode, state;
};

__device__ __forceinline__ void ctrl_step(Ctrl &S, int64_t cur, int64_t now, int32_t tw, int32_t s_inc,
                                          int32_t s_dec, int32_t dec_step, int32_t c, int64_t kt, int64_t kns) {
    if (cur > S.peak) { S.peak = cur; S.count = 0; }
    int64_t moved = cur - S.prev_n;
    if (moved < 0) moved = -moved;
    if (moved < tw) return;
    S.state = (cur >= S.peak - dec_step) ? ST_INC : ST_DEC;
    if (S.state == ST_INC) {
        const int64_t growth = cur - S.prev_n, elapsed = now - S.prev_t;
        if (growth >= s_inc) {
            if (elapsed == 0) {
                S.mode = MODE_ABILITY;
            } else {
                const __int128 lhs = (__int128)growth * kns, rhs = (__int128)kt * elapsed;
                S.mode = lhs < rhs ? MODE_EFI : (lhs > rhs ? MODE_ABILITY : MODE_FIFO);
            }
        } else {
            S.mode = MODE_FIFO;
        }
    } else {
        const int64_t stage = S.peak - int64_t(s_dec) * S.count;
        const int64_t next = S.peak - int64_t(s_dec) * (S.count + 1);
        if (cur > stage) {
            S.mode = MODE_ABILITY;
        } else if (cur <= next + c) {
            S.mode = MODE_EFI_LOC;
            if (cur <= next) S.count += 1;
        } else {
            S.mode = MODE_FIFO;
        }
    }
    S.prev_n = cur;
    S.prev_t = now;
}

__device__ __forceinline__ int32_t node_of(int32_t w, int32_t n_cpu) { return w < n_cpu ? 0 : 1 + (w - n_cpu); }

__device__ __forceinline__ int32_t bitlen64(int64_t x) { return x > 0 ? 64 - __clzll(x) : 0; }
__device__ __forceinline__ int32_t clamp255(int64_t x) { return x < 0 ? 0 : (x > 255 ? 255 : int32_t(x)); }

// The 16 integer features of a candidate at a pop (all in [0, 255]): inspiring
// ability and efficiency (bit lengths and their ratio), CPU / GPU costs (bit
// lengths and ratio), whether the popping worker is a GPU, data locality and
// remaining wait, Nready, the worker's queue length, the controller's mode,
// state and peak, the out-degree and the number of pushes since the task was
// pushed.
__device__ __forceinline__ void cand_features(int32_t *f, int32_t ia, int32_t ie, int64_t ccpu, int64_t cgpu,
                                              int32_t is_gpu, int64_t dr, int64_t now, int64_t nready, int64_t qlen,
                                              int32_t mode, int32_t state, int64_t peak, int32_t outdeg,
                                              int64_t age) {
    f[0] = clamp255(bitlen64(ia));
    f[1] = clamp255(bitlen64(ie));
    f[2] = clamp255(int64_t(ie) * 255 / (ia > 1 ? ia : 1));
    f[3] = clamp255(bitlen64(ccpu));
    f[4] = clamp255(bitlen64(cgpu));
    f[5] = clamp255(16 * ccpu / cgpu);
    f[6] = is_gpu;
    f[7] = dr <= now;
    f[8] = clamp255(bitlen64(dr > now ? dr - now : 0));
    f[9] = clamp255(bitlen64(nready));
    f[10] = clamp255(bitlen64(qlen));
    f[11] = mode;
    f[12] = state;
    f[13] = clamp255(bitlen64(peak));
    f[14] = clamp255(bitlen64(outdeg));
    f[15] = clamp255(bitlen64(age));
}

// Per-warp shared memory of the learned pop: 32 candidate rows of 16 BF16
// features and their pool indices.
struct LearnSmem {
    uint32_t tile[32 * 8];
    int32_t cidx[32];
};

// TWO: more than 32 workers, so every lane owns a second worker (lane + 32); with 32 or
// fewer that slot and all its code drop out at compile time.  EX: rollout controls or the
// push/pop trace are in use; without them their checks drop out too.
template <bool LEARNED, int POOL_C, bool TWO, bool EX>
__global__ void __launch_bounds__(SIM_WARPS * 32) k_sim(SimArgs A) {
    // dynamic shared memory: every warp's pool and buffers, then the learned scorer's
    // weights and per-warp tiles (sized by the warps actually launched)
    extern __shared__ __align__(16) unsigned char dyn[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    WarpSmem<POOL_C, TWO> *sm = reinterpret_cast<WarpSmem<POOL_C, TWO> *>(dyn) + wib;
    unsigned char *dyn_l = dyn + (size_t(blockDim.x >> 5) * sizeof(WarpSmem<POOL_C, TWO>) + 15) / 16 * 16;
    ScorerPacked *SP = reinterpret_cast<ScorerPacked *>(dyn_l);
    LearnSmem *LS = reinterpret_cast<LearnSmem *>(dyn_l + sizeof(ScorerPacked)) + wib;
    if (LEARNED) {
        for (int i = threadIdx.x; i < int(sizeof(ScorerPacked) / 4); i += blockDim.x)
            reinterpret_cast<uint32_t *>(SP)[i] = reinterpret_cast<const uint32_t *>(A.scorer)[i];
        __syncthreads();
    }
    const DevBatch &B = A.B;
    constexpr bool USE_MASK = POOL_C >= MASK_MIN;
    const int32_t P = A.n_cpu + A.n_gpu, n_cpu = A.n_cpu;
    const int64_t xfer = A.xfer;
    const bool smem_types = (A.B.task_cost == nullptr) && (B.n_types <= MAX_TYPES_SMEM);

    for (int32_t iter = 0;; ++iter) {
        int d;
        if (A.single_dag >= 0) {
            if (iter > 0 || blockIdx.x != 0 || wib != 0) return;
            d = A.single_dag;
        } else {
            // first DAG of every warp transposed over the grid (warp j of every CTA takes the j-th
            // stripe of gridDim DAGs), so the largest DAGs start on different SMs instead of filling
            // one CTA; later DAGs through the work counter
            const int nw = gridDim.x * (blockDim.x >> 5);
            int k = 0;
            if (iter == 0) {
                k = wib * gridDim.x + blockIdx.x;
            } else {
                if (lane == 0) k = nw + atomicAdd(A.counter, 1);
                k = __shfl_sync(FULL, k, 0);
            }
            if (k >= A.n_order) return;
            d = A.order[k];
        }
        const int64_t tb = B.task_base[d], eb = B.edge_base[d];
        const int32_t n = int32_t(B.task_base[d + 1] - tb);
        const int32_t *rp = B.row_ptr + tb + d;
        const int32_t *col = B.col_idx + eb;
        int2 *st_a = A.st_a + tb;
        longlong2 *st_b = A.st_b + tb;
        const int32_t *g_ia = A.ia + tb, *g_ie = A.ie + tb;
        Pool<POOL_C, TWO> pool{sm, A.p_idw + tb, A.p_seq + tb, A.p_ia + tb, A.p_ie + tb, A.p_dr + tb, A.p_cost + tb};
        int32_t *nl_g = A.nl + tb;

        // resolved policy parameters (zero = default for P workers and the attributes' unit time T)
        const int32_t tw = A.task_window > 0 ? A.task_window : P;
        const int32_t s_inc = A.s_inc > 0 ? A.s_inc : P;
        const int32_t s_dec = A.s_dec > 0 ? A.s_dec : P;
        const int32_t dec_step = A.dec_step > 0 ? A.dec_step : P;
        const int32_t cslack = A.c > 0 ? A.c : (P / 2 > 1 ? P / 2 : 1);
        const int64_t kt = A.k_inc_tasks > 0 ? A.k_inc_tasks : P;
        const int64_t kns = A.k_inc_ns > 0 ? A.k_inc_ns : A.unit_time[d];
        // static pick modes: DMDA (FIFO) and the DMDAP baselines; -1: the Nready controller decides
        const int32_t static_mode = A.policy == INSP_POLICY_FIFO       ? MODE_FIFO
                                    : A.policy == INSP_POLICY_DMDAP_IA ? MODE_ABILITY
                                    : A.policy == INSP_POLICY_DMDAP_BL ? MODE_PRIO
                                                                       : -1;
        const bool by_level = A.policy == INSP_POLICY_DMDAP_BL;

        // per-DAG init: cost table, per-task release state
        if (smem_types) {
            for (int i = lane; i < B.n_types * 2; i += 32) sm->tcost[i] = B.type_cost[int64_t(d) * B.n_types * 2 + i];
        }
        if (USE_MASK)
            for (int i = lane; i < mask_rows<POOL_C, TWO>() * mask_words<POOL_C>(); i += 32) (&sm->wmask[0][0])[i] = 0u;
        for (int32_t t = lane; t < n; t += 32) {
            st_a[t] = make_int2(A.indeg0[tb + t], NODE_NONE);
            st_b[t] = make_longlong2(NEG_TIME, NEG_TIME);
        }
        __syncwarp();

        auto cost_of = [&](int32_t t, int kind) -> int64_t {
            if (smem_types) return sm->tcost[int(B.type[tb + t]) * 2 + kind];
            return task_cost(B, d, tb + t, kind);
        };

        // lane-owned worker state, workers w0 = lane and w1 = lane + 32
        const int32_t w0 = lane, w1 = lane + 32;
        int64_t busy0 = 0, busy1 = 0, qc0 = 0, qc1 = 0;
        int32_t run0 = -1, run1 = -1, qn0 = 0, qn1 = 0;
        // successor-row bounds of the running task, loaded when it starts (used at its completion)
        int32_t rlo0 = 0, rhi0 = 0, rlo1 = 0, rhi1 = 0;
        bool pf0 = false, pf1 = false;  // started since the last event: prefetch its row
        int32_t nready = 0, seq = 0, done = 0, npop = 0;
        int64_t now = 0;
        Ctrl ctl{0, 0, 0, 0, MODE_FIFO, ST_INC};

        // push(t): earliest expected finish over all workers (DMDA with transfer)
        auto push = [&](int32_t t) {
            const int2 a = st_a[t];
            const longlong2 b = st_b[t];
            int32_t tia, tie;
            if (by_level) {  // the pool's two priority fields carry the bottom level (< 2^54)
                const int64_t l = A.blevel[tb + t];
                tia = int32_t(l >> 31);
                tie = int32_t(l & 0x7fffffff);
            } else {
                tia = g_ia[t];
                tie = g_ie[t];
            }
            const int64_t cc = cost_of(t, 0), cg = cost_of(t, 1);
            uint64_t k0 = ~0ull, k1 = ~0ull;
            int64_t dr0 = 0, dr1 = 0;
            if (w0 < P) {
                const int32_t nd = node_of(w0, n_cpu);
                dr0 = a.y == NODE_NONE ? 0 : (nd == a.y ? max(b.x, b.y + xfer) : b.x + xfer);
                const int64_t avail = max(now, busy0) + qc0;
                const int64_t ef = max(avail, dr0) + (w0 < n_cpu ? cc : cg);
                k0 = (uint64_t(ef) << 6) | uint64_t(w0);
            }
            if (TWO && w1 < P) {
                const int32_t nd = node_of(w1, n_cpu);
                dr1 = a.y == NODE_NONE ? 0 : (nd == a.y ? max(b.x, b.y + xfer) : b.x + xfer);
                const int64_t avail = max(now, busy1) + qc1;
                const int64_t ef = max(avail, dr1) + (w1 < n_cpu ? cc : cg);
                k1 = (uint64_t(ef) << 6) | uint64_t(w1);
            }
            const uint64_t kmin = warp_min_u64(k0 < k1 ? k0 : k1);
            const int32_t ws = int32_t(kmin & 63);
            if (lane == (ws & 31)) {
                const bool hi = ws >= 32;
                const int64_t c = ws < n_cpu ? cc : cg;
                if (TWO && hi) { qc1 += c; qn1 += 1; } else { qc0 += c; qn0 += 1; }
                if (insp_check(nready < n, A.status + d))  // the pool never holds more than n tasks
                    pool.set(nready, t | (ws << 24), seq, tia, tie, hi ? dr1 : dr0, c);
                if (USE_MASK && nready < POOL_C) sm->wmask[ws][nready >> 5] |= 1u << (nready & 31);
                if (EX && A.tr_push_time) {
                    const int64_t r = tb + seq;
                    A.tr_push_time[r] = now;
                    A.tr_push_task[r] = t;
                    A.tr_push_worker[r] = ws;
                    A.tr_push_nready[r] = nready + 1;
                }
            }
            seq += 1;
            nready += 1;
            __syncwarp();
        };

        // features of pool entry i as a candidate of worker w at this pop
        auto features_of = [&](int32_t i, int32_t w, int64_t cur, int32_t qlen, int32_t *f) {
            const int32_t t = pool.idw(i) & 0xffffff;
            cand_features(f, pool.ia(i), pool.ie(i), cost_of(t, 0), cost_of(t, 1), w >= n_cpu, pool.dr(i), now, cur,
                          qlen, ctl.mode, ctl.state, ctl.peak, rp[t + 1] - rp[t], int64_t(seq) - pool.seq(i));
        };

        // pop(w): controller judgement, then the pick (forced / learned / mode key).
        // Returns false (no fault) if w has no entry, which would be a bookkeeping error.
        auto pop = [&](int32_t w) -> bool {
            const int64_t cur = nready;
            int32_t mode = static_mode;
            if (static_mode < 0) {
                ctrl_step(ctl, cur, now, tw, s_inc, s_dec, dec_step, cslack, kt, kns);
                mode = ctl.mode;
            }
            const int32_t qlen = __shfl_sync(FULL, (TWO && w >= 32) ? qn1 : qn0, w & 31);
            // rollouts: candidate features in push order
            if (EX && A.feat_pop != nullptr && npop == A.feat_pop[d]) {
                int32_t last = -1, nd = 0;
                for (int k = 0; k < A.feat_cap; ++k) {
                    int32_t ms = 0x7fffffff, mi = -1;
                    for (int32_t i = lane; i < nready; i += 32) {
                        if ((pool.idw(i) >> 24) != w) continue;
                        const int32_t sq = pool.seq(i);
                        if (sq > last && sq < ms) { ms = sq; mi = i; }
                    }
                    const int32_t wm = int32_t(__reduce_min_sync(FULL, uint32_t(ms)));
                    if (wm == 0x7fffffff) break;
                    const uint32_t ol = __ballot_sync(FULL, ms == wm && mi >= 0);
                    const int32_t i = __shfl_sync(FULL, mi, __ffs(ol) - 1);
                    if (lane == 0) {
                        int32_t f[16];
                        features_of(i, w, cur, qlen, f);
                        int32_t *o = A.feat + (int64_t(d) * A.feat_cap + k) * 16;
                        for (int q = 0; q < 16; ++q) o[q] = f[q];
                        A.feat_task[int64_t(d) * A.feat_cap + k] = pool.idw(i) & 0xffffff;
                    }
                    last = wm;
                    nd += 1;
                }
                if (lane == 0) A.feat_n[d] = nd;
                __syncwarp();
            }
            uint64_t best = 0;
            int32_t bi = -1;
            const bool forcing = EX && A.force_pop != nullptr && npop == A.force_pop[d];
            if (forcing) {
                const int32_t ft = A.force_task[d];
                for (int32_t i = lane; i < nready; i += 32) {
                    const int32_t e = pool.idw(i);
                    if ((e >> 24) == w && (e & 0xffffff) == ft) { best = 1; bi = i; }
                }
            }
            if (!EX || __ballot_sync(FULL, bi >= 0) == 0) {
                if (LEARNED) {
                    // score w's candidates 32 at a time on the tensor cores
                    for (int32_t base = 0; base < nready; base += 32) {
                        const int32_t i = base + lane;
                        const bool match = i < nready && (pool.idw(i) >> 24) == w;
                        const uint32_t mm = __ballot_sync(FULL, match);
                        if (!mm) continue;
                        if (match) {
                            const int r = __popc(mm & ((1u << lane) - 1));
                            int32_t f[16];
                            features_of(i, w, cur, qlen, f);
#pragma unroll
                            for (int c = 0; c < 8; ++c) LS->tile[r * 8 + c] = pack_bf16x2(float(f[2 * c]), float(f[2 * c + 1]));
                            LS->cidx[r] = i;
                        }
                        __syncwarp();
                        const int nc = __popc(mm);
                        for (int mt = 0; mt < nc; mt += 16) {
                            float s0, s1;
                            mlp_score_tile(SP, LS->tile + mt * 8, lane, s0, s1);
                            if ((lane & 3) == 0) {
                                const int r0 = mt + (lane >> 2), r1 = r0 + 8;
                                if (r0 < nc) {
                                    const int32_t pi = LS->cidx[r0];
                                    const uint64_t key = (1ull << 63) | (uint64_t(int64_t(s0 * 64.0f) + 0x80000000LL) << 31) |
                                                         uint64_t(0x7fffffffu - uint32_t(pool.idw(pi) & 0xffffff));
                                    if (key > best) { best = key; bi = pi; }
                                }
                                if (r1 < nc) {
                                    const int32_t pi = LS->cidx[r1];
                                    const uint64_t key = (1ull << 63) | (uint64_t(int64_t(s1 * 64.0f) + 0x80000000LL) << 31) |
                                                         uint64_t(0x7fffffffu - uint32_t(pool.idw(pi) & 0xffffff));
                                    if (key > best) { best = key; bi = pi; }
                                }
                            }
                        }
                        __syncwarp();
                    }
                } else if (mode == MODE_PRIO) {
                    // highest bottom level (54 bits), then lowest id: the lane's best by both, then
                    // a warp max of the level and, among the lanes holding it, of the id key
                    uint32_t lo_best = 0;
                    for (int32_t i = lane; i < nready; i += 32) {
                        const int32_t e = pool.idw(i);
                        if ((e >> 24) != w) continue;
                        const uint64_t lvl = (1ull << 63) | (uint64_t(uint32_t(pool.ia(i))) << 31) |
                                             uint64_t(uint32_t(pool.ie(i)));
                        const uint32_t lo = 0x7fffffffu - uint32_t(e & 0xffffff);
                        if (lvl > best || (lvl == best && lo > lo_best)) { best = lvl; lo_best = lo; bi = i; }
                    }
                    const uint64_t top = warp_max_u64(best);
                    const uint32_t lo_top = __reduce_max_sync(FULL, best == top ? lo_best : 0u);
                    if (best != top || lo_best != lo_top) { best = 0; bi = -1; }
                } else {
                    // one loop per pick mode (the mode is fixed for the pop): the entries of
                    // worker w, keyed by the mode's priority, ties to the lowest id (FIFO: the
                    // oldest push)
                    auto scan = [&](auto key_of) {
                        int32_t i0 = 0;
                        if (USE_MASK) {
                            // shared-memory entries: the set bits of w's bitmap, word j by lane j
                            const int32_t ns = min(nready, POOL_C);
                            if (lane < ((ns + 31) >> 5)) {
                                for (uint32_t m = sm->wmask[w][lane]; m; m &= m - 1) {
                                    const int32_t i = lane * 32 + __ffs(m) - 1;
                                    const int32_t e = pool.idw(i);
                                    const uint64_t key = key_of(i, uint64_t(0x7fffffffu - uint32_t(e & 0xffffff)));
                                    if (key > best) { best = key; bi = i; }
                                }
                            }
                            i0 = POOL_C;  // then the spilled entries
                        }
                        for (int32_t i = i0 + lane; i < nready; i += 32) {
                            const int32_t e = pool.idw(i);
                            if ((e >> 24) != w) continue;
                            const uint64_t key = key_of(i, uint64_t(0x7fffffffu - uint32_t(e & 0xffffff)));
                            if (key > best) { best = key; bi = i; }
                        }
                    };
                    constexpr uint64_t TOP = 1ull << 63;
                    if (mode == MODE_FIFO) {
                        scan([&](int32_t i, uint64_t) { return TOP | uint64_t(0xffffffffu - uint32_t(pool.seq(i))); });
                    } else if (mode == MODE_ABILITY) {
                        scan([&](int32_t i, uint64_t lo) { return TOP | (uint64_t(uint32_t(pool.ia(i))) << 31) | lo; });
                    } else if (mode == MODE_EFI) {
                        scan([&](int32_t i, uint64_t lo) { return TOP | (uint64_t(uint32_t(pool.ie(i))) << 31) | lo; });
                    } else {
                        scan([&](int32_t i, uint64_t lo) {
                            return TOP | (uint64_t(pool.dr(i) <= now) << 62) | (uint64_t(uint32_t(pool.ie(i))) << 31) | lo;
                        });
                    }
                }
            }
            const uint64_t wbest = warp_max_u64(best);
            const uint32_t wl = __ballot_sync(FULL, best == wbest && bi >= 0);
            if (wl == 0) return false;
            const int32_t src_lane = __ffs(wl) - 1;
            const int32_t idx = __shfl_sync(FULL, bi, src_lane);
            const int32_t last = nready - 1;
            nready -= 1;
            npop += 1;
            // the rest by the lane that owns worker w: read the entry, fill its slot with the
            // last entry, start the task, write its schedule
            if (lane == (w & 31)) {
                const int32_t t = pool.idw(idx) & 0xffffff;
                const int64_t dr = pool.dr(idx), c = pool.cost(idx);
                if (USE_MASK) {  // idx leaves w's bitmap; the last entry moves into idx
                    if (idx < POOL_C) sm->wmask[w][idx >> 5] &= ~(1u << (idx & 31));
                    if (idx != last) {
                        const int32_t w2 = pool.idw(last) >> 24;
                        if (last < POOL_C) sm->wmask[w2][last >> 5] &= ~(1u << (last & 31));
                        if (idx < POOL_C) sm->wmask[w2][idx >> 5] |= 1u << (idx & 31);
                    }
                }
                if (idx != last) pool.move(last, idx, lane, true);
                const int64_t s = max(now, dr), e = s + c;
                if (TWO && w >= 32) { qc1 -= c; qn1 -= 1; run1 = t; busy1 = e; rlo1 = rp[t]; rhi1 = rp[t + 1]; pf1 = true; }
                else { qc0 -= c; qn0 -= 1; run0 = t; busy0 = e; rlo0 = rp[t]; rhi0 = rp[t + 1]; pf0 = true; }
                A.worker[tb + t] = w;
                A.start[tb + t] = s;
                A.end[tb + t] = e;
                if (EX && A.tr_pop_time) {
                    const int64_t r = tb + npop - 1;
                    A.tr_pop_time[r] = now;
                    A.tr_pop_task[r] = t;
                    A.tr_pop_worker[r] = w;
                    A.tr_pop_nready[r] = int32_t(cur);
                    A.tr_pop_mode[r] = LEARNED ? MODE_LEARNED : mode;
                }
            }
            __syncwarp();
            return true;
        };

        auto dispatch = [&]() -> bool {
            const uint32_t m0 = __ballot_sync(FULL, w0 < P && run0 < 0 && qn0 > 0);
            const uint32_t m1 = TWO ? __ballot_sync(FULL, w1 < P && run1 < 0 && qn1 > 0) : 0u;
            bool ok = true;
            for (uint32_t m = m0; m && ok; m &= m - 1) ok = pop(__ffs(m) - 1);
            for (uint32_t m = m1; m && ok; m &= m - 1) ok = pop(32 + __ffs(m) - 1);
            return ok;
        };

        // initial pushes: tasks without predecessors, ascending id
        for (int32_t base = 0; base < n; base += 32) {
            const int32_t t = base + lane;
            const uint32_t m = __ballot_sync(FULL, t < n && A.indeg0[tb + t] == 0);
            for (uint32_t mm = m; mm; mm &= mm - 1) push(base + __ffs(mm) - 1);
        }
        bool bad = !dispatch();

        int64_t guard = 0;
        while (!bad && done < n) {
            if (++guard > 2 * int64_t(n) + 2) { bad = true; break; }
            if (pf0) { prefetch_row(col, rlo0, rhi0); pf0 = false; }
            if (TWO && pf1) { prefetch_row(col, rlo1, rhi1); pf1 = false; }
            // next event: earliest completion
            const int64_t e0 = (w0 < P && run0 >= 0) ? busy0 : INT64_MAX;
            const int64_t e1 = (TWO && w1 < P && run1 >= 0) ? busy1 : INT64_MAX;
            now = warp_min_i64(min(e0, e1));
            if (now == INT64_MAX) { bad = true; break; }
            const uint32_t c0 = __ballot_sync(FULL, w0 < P && run0 >= 0 && busy0 == now);
            const uint32_t c1 = TWO ? __ballot_sync(FULL, w1 < P && run1 >= 0 && busy1 == now) : 0u;
            // release successors of every completed task; one run of released ids per completion
            int32_t nl = 0, nruns = 0;
            for (int half = 0; half < (TWO ? 2 : 1); ++half) {
                for (uint32_t m = half ? c1 : c0; m; m &= m - 1) {
                    const int32_t wl = __ffs(m) - 1;
                    const int32_t w = wl + 32 * half;
                    const int32_t p = __shfl_sync(FULL, half ? run1 : run0, wl);
                    const int32_t nd = node_of(w, n_cpu);
                    const int32_t lo = __shfl_sync(FULL, half ? rlo1 : rlo0, wl);
                    const int32_t hi = __shfl_sync(FULL, half ? rhi1 : rhi0, wl);
                    for (int32_t base = lo; base < hi; base += 32) {
                        const int32_t i = base + lane;
                        bool ready = false;
                        int32_t s = 0;
                        if (i < hi) {
                            s = col[i];
                            int2 a = st_a[s];
                            longlong2 b = st_b[s];
                            a.x -= 1;
                            // latest completion per node, top two nodes (now never decreases):
                            // same node -> new latest; another node and later -> the old latest
                            // becomes the runner-up; another node at the same time -> runner-up
                            const bool same = a.y == nd, later = now > b.x;
                            b.y = same ? b.y : (later ? b.x : now);
                            a.y = (same || !later) ? a.y : nd;
                            b.x = (same || later) ? now : b.x;
                            st_a[s] = a;
                            st_b[s] = b;
                            ready = (a.x == 0);
                        }
                        __syncwarp();  // the next row may release the same successor from another lane
                        const uint32_t rm = __ballot_sync(FULL, ready);
                        if (ready) {
                            const int32_t pos = nl + __popc(rm & ((1u << lane) - 1));
                            if (pos < NL_C) sm->newly[pos] = s;
                            else if (insp_check(pos - NL_C < n, A.status + d)) nl_g[pos - NL_C] = s;
                        }
                        nl += __popc(rm);
                    }
                    if (lane == 0) sm->run_end[nruns] = nl;
                    nruns += 1;
                }
            }
            if (c0 & (1u << lane)) run0 = -1;
            if (c1 & (1u << lane)) run1 = -1;
            done += __popc(c0) + __popc(c1);
            __syncwarp();
            // push released tasks in ascending id: merge of the sorted runs
            if (nl > 0) {
                int32_t runs_nonempty = 0;
                for (int r = 0; r < nruns; ++r) {
                    const int32_t b0 = r ? sm->run_end[r - 1] : 0;
                    runs_nonempty += sm->run_end[r] > b0;
                }
                if (runs_nonempty <= 1) {
                    for (int32_t k = 0; k < nl; ++k) push(k < NL_C ? sm->newly[k] : nl_g[k - NL_C]);
                } else {
                    // lane r owns run r (and r + 32): cursor and end
                    int32_t cur0 = 0, end0 = 0, cur1 = 0, end1 = 0;
                    if (lane < nruns) { cur0 = lane ? sm->run_end[lane - 1] : 0; end0 = sm->run_end[lane]; }
                    if (lane + 32 < nruns) { cur1 = sm->run_end[lane + 31]; end1 = sm->run_end[lane + 32]; }
                    __syncwarp();
                    for (int32_t k = 0; k < nl; ++k) {
                        const uint32_t h0 = cur0 < end0 ? uint32_t(cur0 < NL_C ? sm->newly[cur0] : nl_g[cur0 - NL_C])
                                                        : 0xffffffffu;
                        const uint32_t h1 = cur1 < end1 ? uint32_t(cur1 < NL_C ? sm->newly[cur1] : nl_g[cur1 - NL_C])
                                                        : 0xffffffffu;
                        const uint32_t hm = __reduce_min_sync(FULL, min(h0, h1));
                        if (h0 == hm) cur0 += 1;
                        else if (h1 == hm) cur1 += 1;
                        push(int32_t(hm));
                    }
                }
            }
            if (!dispatch()) bad = true;
        }
        if (lane == 0) {
            A.makespan[d] = (n > 0 && !bad) ? now : 0;
            if (bad) A.status[d] = INSP_ETIMEOUT;
        }
        __syncwarp();
    }
}

// dynamic shared memory of a launch with `warps` warps per CTA
template <bool L, int Q, bool TWO>
static size_t sim_dyn_bytes(int warps) {
    return (size_t(warps) * sizeof(WarpSmem<Q, TWO>) + 15) / 16 * 16 +
           (L ? sizeof(ScorerPacked) + warps * sizeof(LearnSmem) : 0);
}

// the device's opt-in limit of dynamic shared memory per CTA
static size_t smem_optin() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 48 * 1024;
    }
    return size_t(v);
}
// the largest CTA of this variant that fits (large queues hold fewer warps per CTA)
template <bool L, int Q, bool TWO>
static size_t sim_dyn_max() {
    return std::min(sim_dyn_bytes<L, Q, TWO>(SIM_WARPS), smem_optin());
}

template <bool L, int Q, bool TWO, bool EX>
static void launch_q(const SimArgs &A, int grid, int threads, cudaStream_t s) {
    cudaFuncSetAttribute(k_sim<L, Q, TWO, EX>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sim_dyn_max<L, Q, TWO>()));
    k_sim<L, Q, TWO, EX><<<grid, threads, sim_dyn_bytes<L, Q, TWO>(threads / 32), s>>>(A);
}

template <bool L, bool TWO, bool EX>
static void launch_l(const SimArgs &A, int grid, int threads, int queue, cudaStream_t s) {
    if (queue <= 32) launch_q<L, 32, TWO, EX>(A, grid, threads, s);
    else if (queue <= 64) launch_q<L, 64, TWO, EX>(A, grid, threads, s);
    else if (queue <= 128) launch_q<L, 128, TWO, EX>(A, grid, threads, s);
    else if (queue <= 256) launch_q<L, 256, TWO, EX>(A, grid, threads, s);
    else if (queue <= 512) launch_q<L, 512, TWO, EX>(A, grid, threads, s);
    else launch_q<L, 1024, TWO, EX>(A, grid, threads, s);
}

template <bool EX>
static void launch_ex(const SimArgs &A, int grid, int threads, int queue, cudaStream_t s) {
    const bool two = A.n_cpu + A.n_gpu > 32;
    if (A.policy == INSP_POLICY_LEARNED) {
        if (two) launch_l<true, true, EX>(A, grid, threads, queue, s);
        else launch_l<true, false, EX>(A, grid, threads, queue, s);
    } else {
        if (two) launch_l<false, true, EX>(A, grid, threads, queue, s);
        else launch_l<false, false, EX>(A, grid, threads, queue, s);
    }
}

static void launch_any(const SimArgs &A, int grid, int threads, int queue, cudaStream_t s) {
    const bool ex = A.feat_pop || A.force_pop || A.tr_push_time || A.tr_pop_time;
    if (ex) launch_ex<true>(A, grid, threads, queue, s);
    else launch_ex<false>(A, grid, threads, queue, s);
}

void launch_sim(const SimArgs &A, int grid, int warps, int queue, cudaStream_t s) {
    launch_any(A, grid, 32 * std::max(1, std::min(warps, SIM_WARPS)), queue, s);
}
// The unbatched form: one launch, one warp, one DAG.
void launch_sim_single(const SimArgs &A, cudaStream_t s) { launch_any(A, 1, 32, 64, s); }
int sim_max_warps() { return SIM_WARPS; }

template <bool L, int Q, bool TWO>
static int occ_q(int threads) {
    int nb = 0;
    if (sim_dyn_bytes<L, Q, TWO>(threads / 32) > sim_dyn_max<L, Q, TWO>()) return 0;  // the CTA does not fit
    cudaFuncSetAttribute(k_sim<L, Q, TWO, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sim_dyn_max<L, Q, TWO>()));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sim<L, Q, TWO, false>, threads,
                                                      sim_dyn_bytes<L, Q, TWO>(threads / 32)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}
template <bool L, bool TWO>
static int occ_l(int threads, int queue) {
    return queue <= 32    ? occ_q<L, 32, TWO>(threads)
           : queue <= 64  ? occ_q<L, 64, TWO>(threads)
           : queue <= 128 ? occ_q<L, 128, TWO>(threads)
           : queue <= 256 ? occ_q<L, 256, TWO>(threads)
           : queue <= 512 ? occ_q<L, 512, TWO>(threads)
                          : occ_q<L, 1024, TWO>(threads);
}
int sim_occupancy(bool learned, int n_workers, int warps, int queue) {
    const int threads = 32 * std::max(1, std::min(warps, SIM_WARPS));
    const bool two = n_workers > 32;
    if (learned) return two ? occ_l<true, true>(threads, queue) : occ_l<true, false>(threads, queue);
    return two ? occ_l<false, true>(threads, queue) : occ_l<false, false>(threads, queue);
}

}  // namespace insp
