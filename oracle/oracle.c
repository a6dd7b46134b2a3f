/*
 * CPU ORACLE -- test infrastructure only.
 *
 * A plain, slow, single-threaded restatement of INSPIRIT's schedule evaluation
 * (arxiv 2404.03226).  Only the tests, the smoke check and the benchmark's CPU
 * baseline use it; the library never calls it.  It shares no code, header or
 * table with the CUDA path.
 *
 * What it computes, with the reading of the paper each part follows:
 *
 *  orc_ia        inspiring ability (Sec. 4.2 definition, Sec. 4.3 computation):
 *                the number of strict descendants of a task -- the dependencies
 *                its completion eventually releases.  Plain DFS from every task.
 *  orc_ie        inspiring efficiency (Sec. 4.2, Sec. 4.3): the number of
 *                strict descendants u whose longest path from the start of v
 *                (GPU execution times, v's own time included, unlimited
 *                workers, tasks outside v's cone treated as done) finishes
 *                within the unit time T.  Plain longest-path DP over the cone.
 *  orc_unit_time_search  automatic choice of the unit time T of Sec. 4.3 (the
 *                paper tunes it by hand): the smallest T = med * 2^k whose IE
 *                separates as many tasks as the DAG's structure does.
 *  orc_bottom_level  the static priority of the DMDAP baseline (Sec. 2.1,
 *                Sec. 3 Observation 1): HEFT's upward rank (Topcuoglu et al.,
 *                2002, cited in Sec. 2) over mean worker costs.
 *  orc_simulate  the list-scheduling run (Sec. 2.1 push/pop, Sec. 4.1 steps
 *                1-3, Sec. 4.4 Nready regulation with the adaptive-priority
 *                pseudocode): in-degree countdown, earliest-finish push with
 *                transfer cost (DMDA, Sec. 2.1), pop by the Nready controller;
 *                or the baselines: DMDA (FIFO pop) and DMDAP with a static
 *                priority (IA, or the bottom level), optionally with a trace
 *                of every push and pop (Sec. 4.4 "Implementation details":
 *                the Nready time piling of push and pop).
 *  orc_renumber  a topological numbering for a DAG given in another one (Kahn
 *                rounds, ascending old id within a round).
 *  orc_validate  an independent check of a schedule's feasibility.
 *  orc_optimum   exhaustive optimum makespan for tiny DAGs.
 *  orc_mlp_*     integer restatement of the learned proposal scorer (fixed
 *                grid BF16 weights; see the scorer section below) and an
 *                fp64 restatement of its training loss, gradient and AdamW.
 *
 * Readings where the paper is silent (each is also listed in the design
 * notes): self excluded from IA; IE counts a descendant only if every path to
 * it fits in T; unit time T is an explicit argument, default 4 x the lower
 * median GPU cost; memory nodes: all CPUs share node 0, GPU g is node 1+g, an
 * edge whose endpoints run on different nodes costs xfer ns; push ties go to
 * the lowest worker; completions, pushes and idle-worker pops are processed by
 * ascending task / task / worker id; the controller is global (Nready counts
 * ready tasks in all worker queues); its state is re-judged only when Nready
 * moved by at least task_window since the last judgement, the count of
 * downward steps resets when a new peak is seen.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EXPORT __attribute__((visibility("default")))

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOTTOPO = 2, ORC_ENOMEM = 3, ORC_EOVERFLOW = 6, ORC_ECYCLE = 8 };
enum { POL_INSPIRIT = 0, POL_FIFO = 1, POL_LEARNED = 2, POL_DMDAP_IA = 3, POL_DMDAP_BL = 4 };
enum { MODE_FIFO = 0, MODE_ABILITY = 1, MODE_EFI = 2, MODE_EFI_LOC = 3, MODE_LEARNED = 4, MODE_PRIO = 5 };
enum { ST_INC = 0, ST_DEC = 1 };

/* ------------------------------------------------------------ DAG checks */

/* Bound on every time value: makespan <= sum_t (max cost + xfer) (each
 * popped task keeps its worker busy for at most one transfer plus its cost and
 * some worker is always busy), so a DAG within this bound never overflows. */
#define TIME_BOUND (((int64_t)1) << 54)

EXPORT int orc_check_dag(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                         const int64_t *c_cpu, const int64_t *c_gpu, int64_t xfer) {
    /* Precedence when several rules fail: malformed input (EINVAL) first, then
     * a non-topological numbering, then a possible time overflow. */
    if (n < 0 || xfer < 0) return ORC_EINVAL;
    if (n == 0) return ORC_OK;
    int bad = 0, nottopo = 0, overflow = 0;
    if (row_ptr[0] != 0) return ORC_EINVAL;
    for (int32_t u = 0; u < n; ++u)
        if (row_ptr[u + 1] < row_ptr[u]) return ORC_EINVAL;
    for (int32_t u = 0; u < n; ++u) {
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col_idx[e];
            if (v < 0 || v >= n) bad = 1;
            else if (e > row_ptr[u] && v <= col_idx[e - 1]) bad = 1;
            else if (v <= u) nottopo = 1;
        }
    }
    int64_t total = 0;
    for (int32_t t = 0; t < n; ++t) {
        if (c_cpu[t] < 1 || c_gpu[t] < 1) { bad = 1; continue; }
        int64_t c = c_cpu[t] > c_gpu[t] ? c_cpu[t] : c_gpu[t];
        if (c > TIME_BOUND || xfer > TIME_BOUND) { overflow = 1; continue; }
        if (total <= TIME_BOUND) total += c + xfer;
    }
    if (total > TIME_BOUND) overflow = 1;
    if (bad) return ORC_EINVAL;
    if (nottopo) return ORC_ENOTTOPO;
    if (overflow) return ORC_EOVERFLOW;
    return ORC_OK;
}

/* ------------------------------------------------------------ renumbering */

/* Task ids must be a topological order for the rest of the method (a task's
 * predecessors come before it).  A DAG given in another numbering (tasks as a
 * runtime's dependency manager lists them, Sec. 2.1) keeps its ids when they
 * are already topological; otherwise it is renumbered by Kahn's algorithm in
 * rounds: round 0 takes every task without predecessors, round r + 1 every
 * task whose predecessors all lie in rounds <= r, and within a round the tasks
 * get consecutive new ids in ascending old id.  new_id[old] receives the new
 * id.  A cycle leaves tasks that no round takes: ORC_ECYCLE.  Duplicate or
 * out-of-range successors: ORC_EINVAL. */
EXPORT int orc_renumber(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t *new_id) {
    if (n < 0) return ORC_EINVAL;
    if (n == 0) return ORC_OK;
    if (row_ptr[0] != 0) return ORC_EINVAL;
    int topo = 1;
    for (int32_t u = 0; u < n; ++u) {
        if (row_ptr[u + 1] < row_ptr[u]) return ORC_EINVAL;
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col_idx[e];
            if (v < 0 || v >= n || (e > row_ptr[u] && v <= col_idx[e - 1])) return ORC_EINVAL;
            if (v <= u) topo = 0;
        }
    }
    if (topo) {
        for (int32_t t = 0; t < n; ++t) new_id[t] = t;
        return ORC_OK;
    }
    int32_t *indeg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *round = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!indeg || !round) { free(indeg); free(round); return ORC_ENOMEM; }
    for (int32_t e = 0; e < row_ptr[n]; ++e) indeg[col_idx[e]]++;
    for (int32_t t = 0; t < n; ++t) round[t] = -1;
    int32_t next = 0, r = 0;
    for (;;) {
        /* this round: every untaken task whose in-degree has reached 0, ascending id */
        int32_t taken = 0;
        for (int32_t t = 0; t < n; ++t)
            if (round[t] < 0 && indeg[t] == 0) { round[t] = r; new_id[t] = next++; ++taken; }
        if (taken == 0) break;
        for (int32_t t = 0; t < n; ++t)
            if (round[t] == r)
                for (int32_t e = row_ptr[t]; e < row_ptr[t + 1]; ++e) indeg[col_idx[e]]--;
        ++r;
    }
    free(indeg);
    free(round);
    return next == n ? ORC_OK : ORC_ECYCLE;
}

/* ------------------------------------------------------- inspiring ability */

/* IA(v) = |{u != v : v reaches u}| by a depth-first search from every v. */
EXPORT int orc_ia(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t *ia) {
    if (n <= 0) return n < 0 ? ORC_EINVAL : ORC_OK;
    int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!stamp || !stack) { free(stamp); free(stack); return ORC_ENOMEM; }
    for (int32_t i = 0; i < n; ++i) stamp[i] = -1;
    for (int32_t v = 0; v < n; ++v) {
        int32_t count = 0, top = 0;
        stamp[v] = v;
        stack[top++] = v;
        while (top > 0) {
            int32_t x = stack[--top];
            for (int32_t e = row_ptr[x]; e < row_ptr[x + 1]; ++e) {
                int32_t s = col_idx[e];
                if (stamp[s] != v) {
                    stamp[s] = v;
                    ++count;
                    stack[top++] = s;
                }
            }
        }
        ia[v] = count;
    }
    free(stamp); free(stack);
    return ORC_OK;
}

/* ----------------------------------------------------- inspiring efficiency */

/* For each v: mark its cone (DFS), then walk the cone in ascending id (ids are
 * a topological order) computing L(u) = c(u) + max L over u's predecessors in
 * the cone, with L(v) = c(v).  IE(v) counts cone members u != v with L(u) <= T.
 * Predecessors are found through a reverse adjacency built here. */
EXPORT int orc_ie(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int64_t *c_gpu,
                  int64_t T, int32_t *ie) {
    if (n <= 0) return n < 0 ? ORC_EINVAL : ORC_OK;
    int32_t m = row_ptr[n];
    int32_t *pr = (int32_t *)calloc((size_t)n + 2, sizeof(int32_t));
    int32_t *pc = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m + 1));
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *in_cone = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int64_t *L = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!pr || !pc || !fill || !in_cone || !stack || !L) {
        free(pr); free(pc); free(fill); free(in_cone); free(stack); free(L);
        return ORC_ENOMEM;
    }
    for (int32_t e = 0; e < m; ++e) pr[col_idx[e] + 1]++;
    for (int32_t i = 0; i < n; ++i) pr[i + 1] += pr[i];
    memcpy(fill, pr, sizeof(int32_t) * (size_t)n);
    for (int32_t u = 0; u < n; ++u)
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) pc[fill[col_idx[e]]++] = u;
    for (int32_t i = 0; i < n; ++i) in_cone[i] = -1;
    for (int32_t v = 0; v < n; ++v) {
        int32_t top = 0, hi = v;
        in_cone[v] = v;
        stack[top++] = v;
        while (top > 0) {
            int32_t x = stack[--top];
            for (int32_t e = row_ptr[x]; e < row_ptr[x + 1]; ++e) {
                int32_t s = col_idx[e];
                if (in_cone[s] != v) {
                    in_cone[s] = v;
                    if (s > hi) hi = s;
                    stack[top++] = s;
                }
            }
        }
        int32_t count = 0;
        L[v] = c_gpu[v];
        for (int32_t u = v + 1; u <= hi; ++u) {
            if (in_cone[u] != v) continue;
            int64_t best = INT64_MIN;
            for (int32_t e = pr[u]; e < pr[u + 1]; ++e) {
                int32_t q = pc[e];
                if (in_cone[q] == v && L[q] > best) best = L[q];
            }
            L[u] = c_gpu[u] + best; /* best is set: u in the cone has an in-cone predecessor */
            if (L[u] <= T) ++count;
        }
        ie[v] = count;
    }
    free(pr); free(pc); free(fill); free(in_cone); free(stack); free(L);
    return ORC_OK;
}

/* Default unit time: 4 x the lower median of the GPU costs (at least 1). */
static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}
EXPORT int64_t orc_default_unit_time(int32_t n, const int64_t *c_gpu) {
    if (n <= 0) return 1;
    int64_t *s = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!s) return -1;
    memcpy(s, c_gpu, sizeof(int64_t) * (size_t)n);
    qsort(s, (size_t)n, sizeof(int64_t), cmp_i64);
    int64_t med = s[(n - 1) / 2];
    free(s);
    int64_t T = 4 * med;
    return T < 1 ? 1 : T;
}

/* ------------------------------------------------------- unit-time search */

static int64_t count_distinct_i64(int64_t *v, int32_t n) {
    if (n <= 0) return 0;
    qsort(v, (size_t)n, sizeof(int64_t), cmp_i64);
    int64_t c = 1;
    for (int32_t i = 1; i < n; ++i) c += v[i] != v[i - 1];
    return c;
}

/* Automatic choice of the unit time T (Sec. 4.3 tunes T by hand, iteratively;
 * this is the batched search that replaces the hand tuning): candidates
 * T_k = med * 2^k for k = 0..k_max (med = the lower median GPU cost, so T_2 is
 * the default unit time; saturating at 2^62), and the chosen T is the smallest
 * candidate whose IE takes at least
 *     target = min(#distinct (topological layer, type) pairs, #distinct IA)
 * distinct values over the DAG's tasks, else T_{k_max}.  The topological layer
 * of a task is the number of edges on the longest path reaching it from a
 * source.  An empty DAG gets T = 1.  Outputs T and its k. */
EXPORT int orc_unit_time_search(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int64_t *c_gpu,
                                const uint8_t *type, int32_t k_max, int64_t *T_out, int32_t *k_out) {
    if (n < 0 || k_max < 0 || k_max > 62) return ORC_EINVAL;
    *T_out = 1;
    *k_out = 0;
    if (n == 0) return ORC_OK;
    int64_t med = orc_default_unit_time(n, c_gpu) / 4; /* the default is 4 x the lower median */
    int32_t *ia = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *ie = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *layer = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!ia || !ie || !layer || !tmp) { free(ia); free(ie); free(layer); free(tmp); return ORC_ENOMEM; }
    orc_ia(n, row_ptr, col_idx, ia);
    for (int32_t u = 0; u < n; ++u) /* ids are topological: u's layer is final here */
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if (layer[col_idx[e]] < layer[u] + 1) layer[col_idx[e]] = layer[u] + 1;
    for (int32_t i = 0; i < n; ++i) tmp[i] = ia[i];
    int64_t d_ia = count_distinct_i64(tmp, n);
    for (int32_t i = 0; i < n; ++i) tmp[i] = (int64_t)layer[i] * 256 + type[i];
    int64_t d_pairs = count_distinct_i64(tmp, n);
    int64_t target = d_ia < d_pairs ? d_ia : d_pairs;
    const int64_t cap = ((int64_t)1) << 62;
    for (int32_t k = 0; k <= k_max; ++k) {
        int64_t T = med > (cap >> k) ? cap : med << k;
        orc_ie(n, row_ptr, col_idx, c_gpu, T, ie);
        for (int32_t i = 0; i < n; ++i) tmp[i] = ie[i];
        *T_out = T;
        *k_out = k;
        if (count_distinct_i64(tmp, n) >= target) break;
    }
    free(ia); free(ie); free(layer); free(tmp);
    return ORC_OK;
}

/* ------------------------------------------------------------ bottom level */

/* HEFT upward rank with integer means, ids being a topological order:
 *   rank(v) = wbar(v) + max over successors s of (cbar + rank(s))  (no successor: wbar(v)),
 *   wbar(v) = floor((n_cpu * c_cpu(v) + n_gpu * c_gpu(v)) / P), the mean cost over the P workers,
 *   cbar    = floor(xfer * D / P^2), the mean transfer cost over ordered worker pairs, D of the
 *             P^2 pairs being on distinct memory nodes (CPUs share one node, each GPU has its own):
 *             D = P^2 - n_cpu^2 - n_gpu. */
EXPORT int orc_bottom_level(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int64_t *c_cpu,
                            const int64_t *c_gpu, int32_t n_cpu, int32_t n_gpu, int64_t xfer, int64_t *bl) {
    int32_t P = n_cpu + n_gpu;
    if (n < 0 || n_cpu < 0 || n_gpu < 0 || P < 1 || xfer < 0) return ORC_EINVAL;
    __int128 D = (__int128)P * P - (__int128)n_cpu * n_cpu - n_gpu;
    int64_t cbar = (int64_t)(((__int128)xfer * D) / ((__int128)P * P));
    for (int32_t v = n - 1; v >= 0; --v) {
        int64_t wbar = (int64_t)(((__int128)n_cpu * c_cpu[v] + (__int128)n_gpu * c_gpu[v]) / P);
        int64_t tail = 0;
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            int64_t x = cbar + bl[col_idx[e]];
            if (x > tail) tail = x;
        }
        bl[v] = wbar + tail;
    }
    return ORC_OK;
}

/* ----------------------------------------------------------- the policy */

typedef struct {
    int32_t policy;                   /* POL_* */
    int32_t task_window, s_inc, s_dec, dec_step, c;
    int64_t k_inc_tasks, k_inc_ns;    /* ascending slope threshold k_inc = tasks / ns */
} orc_policy;

/* Zero fields take the defaults for P workers and unit time T: task window,
 * s_inc, s_dec and dec_step = P; c = max(1, P/2); k_inc = P tasks per T ns. */
EXPORT void orc_resolve_policy(const orc_policy *in, int32_t P, int64_t T, orc_policy *out) {
    *out = *in;
    if (out->task_window <= 0) out->task_window = P;
    if (out->s_inc <= 0) out->s_inc = P;
    if (out->s_dec <= 0) out->s_dec = P;
    if (out->dec_step <= 0) out->dec_step = P;
    if (out->c <= 0) out->c = P / 2 > 1 ? P / 2 : 1;
    if (out->k_inc_tasks <= 0) out->k_inc_tasks = P;
    if (out->k_inc_ns <= 0) out->k_inc_ns = T;
}

/* Nready controller state (Sec. 4.4). */
typedef struct {
    int64_t peak, prev_n, prev_t, count;
    int32_t mode, state;
} orc_ctrl;

/* One judgement at a pop, with cur = Nready before the pop and now = current
 * time.  Follows the adaptive-priority pseudocode of Sec. 4.4:
 *   - a new peak is recorded (and the downward-step count restarts);
 *   - only when |cur - prev_n| >= task_window is the state re-judged:
 *       INC if cur >= peak - dec_step, else DEC;
 *       INC: with growth cur - prev_n >= s_inc the slope k = growth / elapsed
 *            is compared with k_inc: slower -> efficiency pick, faster ->
 *            ability pick, equal -> default (FIFO) pop; smaller growth ->
 *            default pop;
 *       DEC: cur above the current stage threshold peak - s_dec*count ->
 *            ability pick; cur at or below the next stage threshold plus the
 *            slack c -> efficiency-with-locality pick, and when cur is at or
 *            below the next stage threshold itself the stage count advances;
 *            otherwise default pop;
 *     and the reference point (prev_n, prev_t) moves to (cur, now);
 *   - otherwise the previous pick mode is kept. */
EXPORT void orc_ctrl_step(orc_ctrl *S, const orc_policy *p, int64_t cur, int64_t now) {
    if (cur > S->peak) {
        S->peak = cur;
        S->count = 0;
    }
    int64_t moved = cur - S->prev_n;
    if (moved < 0) moved = -moved;
    if (moved < p->task_window) return;
    S->state = (cur >= S->peak - p->dec_step) ? ST_INC : ST_DEC;
    if (S->state == ST_INC) {
        int64_t growth = cur - S->prev_n;
        int64_t elapsed = now - S->prev_t;
        if (growth >= p->s_inc) {
            if (elapsed == 0) {
                S->mode = MODE_ABILITY; /* an instantaneous rise: infinite slope */
            } else {
                __int128 lhs = (__int128)growth * p->k_inc_ns;    /* k * k_inc_ns * elapsed */
                __int128 rhs = (__int128)p->k_inc_tasks * elapsed; /* k_inc * k_inc_ns * elapsed */
                if (lhs < rhs) S->mode = MODE_EFI;
                else if (lhs > rhs) S->mode = MODE_ABILITY;
                else S->mode = MODE_FIFO;
            }
        } else {
            S->mode = MODE_FIFO;
        }
    } else {
        int64_t stage = S->peak - (int64_t)p->s_dec * S->count;
        int64_t next_stage = S->peak - (int64_t)p->s_dec * (S->count + 1);
        if (cur > stage) {
            S->mode = MODE_ABILITY;
        } else if (cur <= next_stage + p->c) {
            S->mode = MODE_EFI_LOC;
            if (cur <= next_stage) S->count += 1;
        } else {
            S->mode = MODE_FIFO;
        }
    }
    S->prev_n = cur;
    S->prev_t = now;
}

/* --------------------------------------------------------- learned scorer */
/*
 * Proposal scorer: an MLP 16 -> 64 -> 64 -> 1 over integer features in
 * [0, 255].  Weights and biases lie on the grid k / 64 with |k| <= 128, so
 * they are exact in BF16; hidden units are floor(max(0, x)) clamped to 255.
 * With integer inputs every partial sum is a multiple of 1/64 below 2^15 in
 * magnitude, so FP32 accumulation in any order is exact, and this integer
 * restatement (sums of k * x in units of 1/64) gives the same result.
 * Weight layout (int16 grid numerators k):
 *   W1[16][64], b1[64], W2[64][64], b2[64], W3[64], b3[1]  (5313 values).
 * The score is returned in units of 1/64.
 */
#define MLP_IN 16
#define MLP_H 64
#define MLP_NW (MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)

EXPORT int32_t orc_mlp_nweights(void) { return MLP_NW; }

static int64_t floor_div64(int64_t a) { /* floor(a / 64) */
    return a >= 0 ? a / 64 : -((-a + 63) / 64);
}

EXPORT int64_t orc_mlp_score(const int16_t *w, const int32_t *feat) {
    const int16_t *W1 = w, *b1 = W1 + MLP_IN * MLP_H, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const int16_t *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    int64_t h1[MLP_H], h2[MLP_H];
    for (int j = 0; j < MLP_H; ++j) {
        int64_t acc = b1[j];
        for (int i = 0; i < MLP_IN; ++i) acc += (int64_t)W1[i * MLP_H + j] * feat[i];
        int64_t h = acc <= 0 ? 0 : floor_div64(acc);
        h1[j] = h > 255 ? 255 : h;
    }
    for (int j = 0; j < MLP_H; ++j) {
        int64_t acc = b2[j];
        for (int i = 0; i < MLP_H; ++i) acc += (int64_t)W2[i * MLP_H + j] * h1[i];
        int64_t h = acc <= 0 ? 0 : floor_div64(acc);
        h2[j] = h > 255 ? 255 : h;
    }
    int64_t acc = b3[0];
    for (int i = 0; i < MLP_H; ++i) acc += (int64_t)W3[i] * h2[i];
    return acc;
}

/* floor(log2(x)) + 1 for x >= 1, 0 for x <= 0 */
static int32_t bitlen(int64_t x) {
    int32_t b = 0;
    while (x > 0) { ++b; x >>= 1; }
    return b;
}
static int32_t clamp255(int64_t x) { return x < 0 ? 0 : (x > 255 ? 255 : (int32_t)x); }

/*
 * The 16 integer features of a candidate task t for worker w at a pop
 * (all clamped to [0, 255]):
 *   0 bitlen(IA)            1 bitlen(IE)            2 min(IE*255/max(IA,1), 255)
 *   3 bitlen(c_cpu)         4 bitlen(c_gpu)         5 min(16*c_cpu/c_gpu, 255)
 *   6 worker is a GPU       7 data local (ready time <= now)
 *   8 bitlen(ready wait)    9 bitlen(Nready)        10 bitlen(queue length of w)
 *  11 controller mode      12 controller state      13 bitlen(peak)
 *  14 bitlen(out-degree)   15 bitlen(age), age = pushes since t was pushed
 * where ready wait = max(0, data_ready - now).
 */
static void mlp_features(int32_t *f, int32_t ia, int32_t ie, int64_t ccpu, int64_t cgpu, int32_t is_gpu,
                         int64_t dr, int64_t now, int64_t nready, int64_t qlen, int32_t mode, int32_t state,
                         int64_t peak, int32_t outdeg, int64_t age) {
    f[0] = clamp255(bitlen(ia));
    f[1] = clamp255(bitlen(ie));
    f[2] = clamp255((int64_t)ie * 255 / (ia > 1 ? ia : 1));
    f[3] = clamp255(bitlen(ccpu));
    f[4] = clamp255(bitlen(cgpu));
    f[5] = clamp255(16 * ccpu / cgpu);
    f[6] = is_gpu;
    f[7] = dr <= now;
    f[8] = clamp255(bitlen(dr > now ? dr - now : 0));
    f[9] = clamp255(bitlen(nready));
    f[10] = clamp255(bitlen(qlen));
    f[11] = mode;
    f[12] = state;
    f[13] = clamp255(bitlen(peak));
    f[14] = clamp255(bitlen(outdeg));
    f[15] = clamp255(bitlen(age));
}

/* -------------------------------------------------------- the simulation */

typedef struct {
    /* per pop (capacity n): time, Nready before the pop, mode, task, worker */
    int64_t *t;
    int32_t *nready, *mode, *task, *worker;
    int32_t npop;
    /* candidate features at pop number feat_pop (< 0: none): up to feat_cap
     * candidates of the popping worker's queue, in push order */
    int32_t feat_pop, feat_cap, n_feat;
    int32_t *feat_task; /* feat_cap */
    int32_t *feat;      /* feat_cap * 16 */
    /* per push (capacity n; push_t NULL: not recorded): time, task, chosen
     * worker, Nready after the push */
    int64_t *push_t;
    int32_t *push_task, *push_worker, *push_nready;
    int32_t npush;
} orc_trace;

typedef struct {
    /* Optional forced decision for rollouts: at pop number force_pop, take
     * task force_task if it is in the popping worker's queue, instead of the
     * policy's pick.  force_pop < 0 disables it. */
    int32_t force_pop, force_task;
} orc_force;

typedef struct { int32_t task; int64_t seq; } qent;

static int32_t node_of(int32_t w, int32_t n_cpu) { return w < n_cpu ? 0 : 1 + (w - n_cpu); }

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* data_ready(t, w) = max over predecessors p of end(p) + xfer * [node(p) != node(w)]; 0 without predecessors. */
static int64_t data_ready(int32_t t, int32_t w, const int32_t *pr, const int32_t *pc, const int32_t *worker,
                          const int64_t *end, int32_t n_cpu, int64_t xfer) {
    int64_t r = 0;
    int32_t nw = node_of(w, n_cpu);
    for (int32_t e = pr[t]; e < pr[t + 1]; ++e) {
        int32_t p = pc[e];
        int64_t x = end[p] + (node_of(worker[p], n_cpu) != nw ? xfer : 0);
        if (x > r) r = x;
    }
    return r;
}

EXPORT int orc_simulate(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                        const int64_t *c_cpu, const int64_t *c_gpu,
                        int32_t n_cpu, int32_t n_gpu, int64_t xfer,
                        const orc_policy *pol_in, int64_t unit_time,
                        const int32_t *ia, const int32_t *ie, const int16_t *mlp_w,
                        const orc_force *force,
                        int32_t *worker, int64_t *start, int64_t *end, int64_t *makespan,
                        orc_trace *trace) {
    int32_t P = n_cpu + n_gpu;
    if (n_cpu < 0 || n_gpu < 0 || P < 1 || P > 64) return ORC_EINVAL;
    int rc = orc_check_dag(n, row_ptr, col_idx, c_cpu, c_gpu, xfer);
    if (rc) return rc;
    if (pol_in->policy < POL_INSPIRIT || pol_in->policy > POL_DMDAP_BL) return ORC_EINVAL;
    if (pol_in->policy == POL_LEARNED && !mlp_w) return ORC_EINVAL;
    /* unit_time is the unit time T the attributes were computed with; it sets
     * k_inc's default, P tasks per T ns (<= 0 selects the DAG's default unit
     * time). */
    if (unit_time <= 0) unit_time = orc_default_unit_time(n, c_gpu);
    orc_policy pol;
    orc_resolve_policy(pol_in, P, unit_time, &pol);
    *makespan = 0;
    if (trace) { trace->npop = 0; trace->npush = 0; }
    if (n == 0) return ORC_OK;

    int32_t m = row_ptr[n];
    int32_t *pr = (int32_t *)calloc((size_t)n + 2, sizeof(int32_t));
    int32_t *pc = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m + 1));
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *indeg = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *newly = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *completed = (int32_t *)malloc(sizeof(int32_t) * ((size_t)P + 1));
    qent *queue = (qent *)malloc(sizeof(qent) * (size_t)P * (size_t)n);
    int32_t *qlen = (int32_t *)calloc((size_t)P, sizeof(int32_t));
    int64_t *busy_end = (int64_t *)calloc((size_t)P, sizeof(int64_t));
    int64_t *queued_cost = (int64_t *)calloc((size_t)P, sizeof(int64_t));
    int32_t *running = (int32_t *)malloc(sizeof(int32_t) * (size_t)P);
    int64_t *bl = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!pr || !pc || !fill || !indeg || !newly || !completed || !queue || !qlen || !busy_end ||
        !queued_cost || !running || !bl) {
        rc = ORC_ENOMEM;
        goto out;
    }
    if (pol.policy == POL_DMDAP_BL) orc_bottom_level(n, row_ptr, col_idx, c_cpu, c_gpu, n_cpu, n_gpu, xfer, bl);
    for (int32_t e = 0; e < m; ++e) pr[col_idx[e] + 1]++;
    for (int32_t i = 0; i < n; ++i) pr[i + 1] += pr[i];
    for (int32_t i = 0; i < n; ++i) fill[i] = pr[i];
    for (int32_t u = 0; u < n; ++u)
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) pc[fill[col_idx[e]]++] = u;
    for (int32_t t = 0; t < n; ++t) {
        indeg[t] = pr[t + 1] - pr[t];
        worker[t] = -1;
        start[t] = -1;
        end[t] = -1;
    }
    for (int32_t w = 0; w < P; ++w) running[w] = -1;

    int64_t now = 0, nready = 0, seq = 0;
    int32_t done = 0, npop = 0;
    orc_ctrl ctl = {0, 0, 0, 0, MODE_FIFO, ST_INC};

#define COST(t, w) ((w) < n_cpu ? c_cpu[t] : c_gpu[t])

    /* push(t): earliest expected finish over all workers (DMDA, Sec. 2.1). */
#define PUSH(t_)                                                                         \
    do {                                                                                 \
        int32_t pt_ = (t_), best = -1;                                                     \
        int64_t best_ef = 0;                                                             \
        for (int32_t w = 0; w < P; ++w) {                                                \
            int64_t avail = (now > busy_end[w] ? now : busy_end[w]) + queued_cost[w];    \
            int64_t dr = data_ready(pt_, w, pr, pc, worker, end, n_cpu, xfer);             \
            int64_t ef = (avail > dr ? avail : dr) + COST(pt_, w);                         \
            if (best < 0 || ef < best_ef) { best = w; best_ef = ef; }                    \
        }                                                                                \
        queue[(size_t)best * n + qlen[best]].task = pt_;                                   \
        queue[(size_t)best * n + qlen[best]].seq = seq++;                                \
        qlen[best]++;                                                                    \
        queued_cost[best] += COST(pt_, best);                                              \
        nready++;                                                                        \
        if (trace && trace->push_t) {                                                    \
            trace->push_t[trace->npush] = now;                                           \
            trace->push_task[trace->npush] = pt_;                                          \
            trace->push_worker[trace->npush] = best;                                     \
            trace->push_nready[trace->npush] = (int32_t)nready;                          \
            trace->npush++;                                                              \
        }                                                                                \
    } while (0)

    /* initial pushes: every task without predecessors, ascending id */
    for (int32_t t = 0; t < n; ++t)
        if (indeg[t] == 0) PUSH(t);

    for (;;) {
        /* dispatch: idle workers with a non-empty queue pop, ascending worker id */
        for (int32_t w = 0; w < P; ++w) {
            if (running[w] >= 0 || qlen[w] == 0) continue;
            int64_t cur = nready;
            int32_t mode = MODE_FIFO;
            if (pol.policy == POL_DMDAP_IA) {
                mode = MODE_ABILITY; /* static priority: inspiring ability */
            } else if (pol.policy == POL_DMDAP_BL) {
                mode = MODE_PRIO; /* static priority: bottom level */
            } else if (pol.policy != POL_FIFO) {
                orc_ctrl_step(&ctl, &pol, cur, now);
                mode = ctl.mode;
            }
            qent *Q = queue + (size_t)w * n;
            int32_t pick = 0; /* queue is kept in push order: index 0 = oldest */
            int want_feat = (pol.policy == POL_LEARNED) || (trace && trace->feat_pop == npop);
            int64_t best_sc = 0;
            if (trace && trace->feat_pop == npop) trace->n_feat = 0;
            for (int32_t i = 0; want_feat && i < qlen[w]; ++i) {
                int32_t t = Q[i].task;
                int32_t f[MLP_IN];
                int64_t dr = data_ready(t, w, pr, pc, worker, end, n_cpu, xfer);
                mlp_features(f, ia[t], ie[t], c_cpu[t], c_gpu[t], w >= n_cpu, dr, now, nready, qlen[w],
                             ctl.mode, ctl.state, ctl.peak, row_ptr[t + 1] - row_ptr[t], seq - Q[i].seq);
                if (trace && trace->feat_pop == npop && trace->n_feat < trace->feat_cap) {
                    trace->feat_task[trace->n_feat] = t;
                    memcpy(trace->feat + (size_t)trace->n_feat * MLP_IN, f, sizeof(f));
                    trace->n_feat++;
                }
                if (pol.policy == POL_LEARNED) {
                    int64_t sc = orc_mlp_score(mlp_w, f);
                    if (i == 0 || sc > best_sc || (sc == best_sc && t < Q[pick].task)) { best_sc = sc; pick = i; }
                }
            }
            int32_t forced = -1;
            if (force && force->force_pop == npop)
                for (int32_t i = 0; i < qlen[w]; ++i)
                    if (Q[i].task == force->force_task) forced = i;
            if (forced >= 0) {
                pick = forced;
            } else if (pol.policy == POL_LEARNED) {
                /* pick already chosen by the scorer */
            } else if (mode == MODE_ABILITY || mode == MODE_EFI || mode == MODE_EFI_LOC || mode == MODE_PRIO) {
                int64_t best_key = 0;
                int32_t best_loc = 0;
                for (int32_t i = 0; i < qlen[w]; ++i) {
                    int32_t t = Q[i].task;
                    int64_t key = (mode == MODE_ABILITY) ? ia[t] : (mode == MODE_PRIO ? bl[t] : ie[t]);
                    int32_t loc = 0;
                    if (mode == MODE_EFI_LOC)
                        loc = data_ready(t, w, pr, pc, worker, end, n_cpu, xfer) <= now;
                    int better;
                    if (i == 0) better = 1;
                    else if (loc != best_loc) better = loc > best_loc;
                    else if (key != best_key) better = key > best_key;
                    else better = t < Q[pick].task;
                    if (better) { pick = i; best_key = key; best_loc = loc; }
                }
            }
            int32_t t = Q[pick].task;
            for (int32_t i = pick; i + 1 < qlen[w]; ++i) Q[i] = Q[i + 1];
            qlen[w]--;
            queued_cost[w] -= COST(t, w);
            nready--;
            int64_t dr = data_ready(t, w, pr, pc, worker, end, n_cpu, xfer);
            int64_t s = now > dr ? now : dr;
            worker[t] = w;
            start[t] = s;
            end[t] = s + COST(t, w);
            running[w] = t;
            busy_end[w] = end[t];
            if (trace) {
                trace->t[npop] = now;
                trace->nready[npop] = (int32_t)cur;
                trace->mode[npop] = (pol.policy == POL_LEARNED) ? MODE_LEARNED : mode;
                trace->task[npop] = t;
                trace->worker[npop] = w;
            }
            npop++;
        }
        if (done == n) break;
        /* advance to the earliest completion */
        int64_t next = INT64_MAX;
        for (int32_t w = 0; w < P; ++w)
            if (running[w] >= 0 && busy_end[w] < next) next = busy_end[w];
        if (next == INT64_MAX) { rc = ORC_EINVAL; goto out; } /* unreachable for a DAG */
        now = next;
        int32_t nc = 0;
        for (int32_t w = 0; w < P; ++w)
            if (running[w] >= 0 && busy_end[w] == now) { completed[nc++] = running[w]; running[w] = -1; }
        qsort(completed, (size_t)nc, sizeof(int32_t), cmp_i32);
        int32_t nn = 0;
        for (int32_t i = 0; i < nc; ++i) {
            int32_t p = completed[i];
            done++;
            if (end[p] > *makespan) *makespan = end[p];
            for (int32_t e = row_ptr[p]; e < row_ptr[p + 1]; ++e) {
                int32_t s = col_idx[e];
                if (--indeg[s] == 0) newly[nn++] = s;
            }
        }
        qsort(newly, (size_t)nn, sizeof(int32_t), cmp_i32);
        for (int32_t i = 0; i < nn; ++i) PUSH(newly[i]);
    }
    if (trace) trace->npop = npop;
#undef PUSH
#undef COST
out:
    free(pr); free(pc); free(fill); free(indeg); free(newly); free(completed); free(queue);
    free(qlen); free(busy_end); free(queued_cost); free(running); free(bl);
    return rc;
}

/* ------------------------------------------------------------ validator */

/* 0 if the schedule is feasible for the DAG and machine, else a code naming
 * the first violated rule: 1 worker out of range, 2 end != start + cost,
 * 3 start before data arrives (precedence + transfer), 4 two tasks overlap on
 * a worker, 5 makespan != max end, 6 negative start. */
EXPORT int orc_validate(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                        const int64_t *c_cpu, const int64_t *c_gpu, int32_t n_cpu, int32_t n_gpu, int64_t xfer,
                        const int32_t *worker, const int64_t *start, const int64_t *end, int64_t makespan,
                        int32_t *bad_task) {
    int32_t P = n_cpu + n_gpu;
    int64_t mx = 0;
    *bad_task = -1;
    for (int32_t t = 0; t < n; ++t) {
        if (worker[t] < 0 || worker[t] >= P) { *bad_task = t; return 1; }
        int64_t c = worker[t] < n_cpu ? c_cpu[t] : c_gpu[t];
        if (end[t] != start[t] + c) { *bad_task = t; return 2; }
        if (start[t] < 0) { *bad_task = t; return 6; }
        if (end[t] > mx) mx = end[t];
    }
    for (int32_t u = 0; u < n; ++u) {
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col_idx[e];
            int64_t arrive = end[u] + (node_of(worker[u], n_cpu) != node_of(worker[v], n_cpu) ? xfer : 0);
            if (start[v] < arrive) { *bad_task = v; return 3; }
        }
    }
    /* overlap: for each worker, intervals sorted by start must not intersect */
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!idx) return ORC_ENOMEM;
    for (int32_t w = 0; w < P; ++w) {
        int32_t k = 0;
        for (int32_t t = 0; t < n; ++t) if (worker[t] == w) idx[k++] = t;
        for (int32_t a = 1; a < k; ++a) { /* insertion sort by start */
            int32_t x = idx[a], b = a - 1;
            while (b >= 0 && start[idx[b]] > start[x]) { idx[b + 1] = idx[b]; --b; }
            idx[b + 1] = x;
        }
        for (int32_t a = 1; a < k; ++a)
            if (start[idx[a]] < end[idx[a - 1]]) { *bad_task = idx[a]; free(idx); return 4; }
    }
    free(idx);
    if (n > 0 && makespan != mx) return 5;
    if (n == 0 && makespan != 0) return 5;
    return 0;
}

/* -------------------------------------------------------- exact optimum */

/* Branch and bound over (ready task, worker) sequences, each task starting as
 * early as its worker and its data allow.  Any schedule ordered by start time
 * is such a sequence after left-shifting, so the minimum over sequences is the
 * optimum makespan.  Intended for n <= 10. */
typedef struct {
    int32_t n, n_cpu, P;
    const int32_t *row_ptr, *col_idx, *pr, *pc;
    const int64_t *c_cpu, *c_gpu;
    int64_t xfer, best;
    int32_t *worker, *indeg;
    int64_t *end, *free_at;
} bb_state;

static void bb(bb_state *S, int32_t placed, int64_t cur_max) {
    if (cur_max >= S->best) return;
    if (placed == S->n) { S->best = cur_max; return; }
    for (int32_t t = 0; t < S->n; ++t) {
        if (S->worker[t] >= 0 || S->indeg[t] != 0) continue;
        for (int32_t w = 0; w < S->P; ++w) {
            int64_t dr = data_ready(t, w, S->pr, S->pc, S->worker, S->end, S->n_cpu, S->xfer);
            int64_t s = S->free_at[w] > dr ? S->free_at[w] : dr;
            int64_t e = s + (w < S->n_cpu ? S->c_cpu[t] : S->c_gpu[t]);
            int64_t saved_free = S->free_at[w];
            S->worker[t] = w; S->end[t] = e; S->free_at[w] = e;
            for (int32_t k = S->row_ptr[t]; k < S->row_ptr[t + 1]; ++k) S->indeg[S->col_idx[k]]--;
            bb(S, placed + 1, e > cur_max ? e : cur_max);
            for (int32_t k = S->row_ptr[t]; k < S->row_ptr[t + 1]; ++k) S->indeg[S->col_idx[k]]++;
            S->worker[t] = -1; S->end[t] = -1; S->free_at[w] = saved_free;
        }
    }
}

EXPORT int64_t orc_optimum(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                           const int64_t *c_cpu, const int64_t *c_gpu, int32_t n_cpu, int32_t n_gpu, int64_t xfer,
                           int64_t upper_bound) {
    if (n <= 0) return 0;
    int32_t m = row_ptr[n];
    int32_t pr[64], pc[1024], fill[64], worker[64], indeg[64];
    int64_t end[64], free_at[64];
    if (n > 16 || m > 1024 || n_cpu + n_gpu > 64) return -1;
    memset(pr, 0, sizeof(pr));
    for (int32_t e = 0; e < m; ++e) pr[col_idx[e] + 1]++;
    for (int32_t i = 0; i < n; ++i) pr[i + 1] += pr[i];
    memcpy(fill, pr, sizeof(int32_t) * (size_t)n);
    for (int32_t u = 0; u < n; ++u)
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) pc[fill[col_idx[e]]++] = u;
    for (int32_t t = 0; t < n; ++t) { worker[t] = -1; end[t] = -1; indeg[t] = pr[t + 1] - pr[t]; }
    for (int32_t w = 0; w < n_cpu + n_gpu; ++w) free_at[w] = 0;
    bb_state S = {n, n_cpu, n_cpu + n_gpu, row_ptr, col_idx, pr, pc, c_cpu, c_gpu, xfer,
                  upper_bound > 0 ? upper_bound + 1 : INT64_MAX, worker, indeg, end, free_at};
    bb(&S, 0, 0);
    return S.best;
}

/* ------------------------------------------------------ scorer training */
/*
 * fp64 restatement of the scorer's training loss and gradient, for checking
 * the training kernels.  Network in -> h1 -> h2 -> 1, weights laid out as
 * W1[in][h1], b1[h1], W2[h1][h2], b2[h2], W3[h2], b3[1] (real values).
 * Loss = mean over samples of (y - target)^2.
 *
 * mode 0 (smooth): h = min(max(z, 0), 255), derivative 1 on 0 < z < 255.
 * mode 1 (quantisation-aware, the inference network): the forward pass uses
 *   w_q = clamp(round(64 w), -128, 128) / 64 and h = min(floor(max(z, 0)), 255),
 *   i.e. exactly orc_mlp_score / 64 for the rounded weights; the backward pass
 *   uses straight-through estimators: d w_q / d w = 1 when |64 w| <= 128.5,
 *   else 0; d h / d z = 1 when 0 < z < 256, else 0 (round: half away from zero).
 */
static double q_weight(double w) {
    double k = w * 64.0;
    k = k >= 0 ? (double)(int64_t)(k + 0.5) : -(double)(int64_t)(-k + 0.5);
    if (k > 128) k = 128;
    if (k < -128) k = -128;
    return k / 64.0;
}
static int q_pass(double w) { double k = w * 64.0; return k <= 128.5 && k >= -128.5; }

EXPORT double orc_mlp_loss_grad(int32_t in, int32_t h1, int32_t h2, const double *w, int32_t mode, int32_t n,
                                const double *x, const double *target, double *grad) {
    const int32_t nw = in * h1 + h1 + h1 * h2 + h2 + h2 + 1;
    const double *W1 = w, *B1 = W1 + in * h1, *W2 = B1 + h1, *B2 = W2 + h1 * h2, *W3 = B2 + h2, *B3 = W3 + h2;
    double *gW1 = grad, *gB1 = gW1 + in * h1, *gW2 = gB1 + h1, *gB2 = gW2 + h1 * h2, *gW3 = gB2 + h2, *gB3 = gW3 + h2;
    double *wq = (double *)malloc(sizeof(double) * (size_t)nw);
    double *z1 = (double *)malloc(sizeof(double) * (size_t)h1), *a1 = (double *)malloc(sizeof(double) * (size_t)h1);
    double *z2 = (double *)malloc(sizeof(double) * (size_t)h2), *a2 = (double *)malloc(sizeof(double) * (size_t)h2);
    double *d1 = (double *)malloc(sizeof(double) * (size_t)h1), *d2 = (double *)malloc(sizeof(double) * (size_t)h2);
    if (!wq || !z1 || !a1 || !z2 || !a2 || !d1 || !d2) return -1.0;
    for (int32_t i = 0; i < nw; ++i) { wq[i] = mode ? q_weight(w[i]) : w[i]; grad[i] = 0.0; }
    const double *Q1 = wq, *QB1 = Q1 + in * h1, *Q2 = QB1 + h1, *QB2 = Q2 + h1 * h2, *Q3 = QB2 + h2, *QB3 = Q3 + h2;
    (void)W1; (void)B1; (void)W2; (void)B2; (void)W3; (void)B3;
    double loss = 0.0;
    for (int32_t s = 0; s < n; ++s) {
        const double *xs = x + (size_t)s * in;
        for (int32_t j = 0; j < h1; ++j) {
            double z = QB1[j];
            for (int32_t i = 0; i < in; ++i) z += Q1[i * h1 + j] * xs[i];
            z1[j] = z;
            double h = z > 0 ? z : 0;
            if (mode) h = (double)(int64_t)h;
            a1[j] = h > 255 ? 255 : h;
        }
        for (int32_t j = 0; j < h2; ++j) {
            double z = QB2[j];
            for (int32_t i = 0; i < h1; ++i) z += Q2[i * h2 + j] * a1[i];
            z2[j] = z;
            double h = z > 0 ? z : 0;
            if (mode) h = (double)(int64_t)h;
            a2[j] = h > 255 ? 255 : h;
        }
        double y = QB3[0];
        for (int32_t i = 0; i < h2; ++i) y += Q3[i] * a2[i];
        const double e = y - target[s];
        loss += e * e;
        const double dy = 2.0 * e / n;
        const double hi = mode ? 256.0 : 255.0;
        gB3[0] += dy;
        for (int32_t i = 0; i < h2; ++i) {
            gW3[i] += dy * a2[i];
            d2[i] = (z2[i] > 0 && z2[i] < hi) ? dy * Q3[i] : 0.0;
            gB2[i] += d2[i];
        }
        for (int32_t i = 0; i < h1; ++i) {
            double g = 0.0;
            for (int32_t j = 0; j < h2; ++j) {
                gW2[i * h2 + j] += a1[i] * d2[j];
                g += Q2[i * h2 + j] * d2[j];
            }
            d1[i] = (z1[i] > 0 && z1[i] < hi) ? g : 0.0;
            gB1[i] += d1[i];
        }
        for (int32_t i = 0; i < in; ++i)
            for (int32_t j = 0; j < h1; ++j) gW1[i * h1 + j] += xs[i] * d1[j];
    }
    if (mode)
        for (int32_t i = 0; i < nw; ++i)
            if (!q_pass(w[i])) grad[i] = 0.0;
    free(wq); free(z1); free(a1); free(z2); free(a2); free(d1); free(d2);
    return loss / n;
}

/* One AdamW step (decoupled weight decay, Loshchilov and Hutter, ICLR 2019),
 * step counter t >= 1: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * w -= lr (m / (1-b1^t) / (sqrt(v / (1-b2^t)) + eps) + wd w). */
EXPORT void orc_adamw(int32_t nw, double *w, double *m, double *v, const double *g, int32_t t, double lr,
                      double b1, double b2, double eps, double wd) {
    double c1 = 1.0, c2 = 1.0;
    for (int32_t i = 0; i < t; ++i) { c1 *= b1; c2 *= b2; }
    c1 = 1.0 - c1;
    c2 = 1.0 - c2;
    for (int32_t i = 0; i < nw; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        w[i] -= lr * ((m[i] / c1) / (sqrt(v[i] / c2) + eps) + wd * w[i]);
    }
}
