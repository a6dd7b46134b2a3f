/*
 * Seeded synthetic task-DAG generators shared by the tests, the benchmark and
 * the oracle.  This file holds no scheduling arithmetic: it only builds task
 * graphs (CSR, successor lists sorted ascending, ids in a topological order)
 * and integer nanosecond cost tables.
 *
 * Workloads (stand-ins for the evaluation section of the paper):
 *   - random layered DAGs, the "logically layered" auto-generated graphs the
 *     authors fed to their Taskbench extension (Sec. 4.4 "Implementation
 *     details", Sec. 5.2), with random task types or, as the authors did,
 *     types by in/out degree;
 *   - tiled Cholesky / LU / QR DAGs (Sec. 5.3: Cholesky with 960x960 tiles,
 *     LU with 160x160 tiles; QR is added as a third dense factorisation),
 *     whose edges are inferred from tile reads and writes the way a
 *     task-based runtime infers them from data handles and access modes
 *     (Sec. 2.1): read-after-write, write-after-write, write-after-read.
 *
 * Random numbers: splitmix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).  DAG i of workload cfg uses
 * the stream seeded with splitmix64(base ^ (cfg << 32) ^ i).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ rng -- */
static inline uint64_t sm64_next(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline double u01(uint64_t *s) { return (double)(sm64_next(s) >> 11) * 0x1.0p-53; }
/* inclusive integer range [lo, hi] */
static inline int64_t urange(uint64_t *s, int64_t lo, int64_t hi) {
    uint64_t span = (uint64_t)(hi - lo) + 1u;
    return lo + (int64_t)(sm64_next(s) % span);
}
/* standard normal by the Box-Muller transform */
static double std_normal(uint64_t *s) {
    double u1 = 1.0 - u01(s); /* (0, 1] */
    double u2 = u01(s);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

EXPORT uint64_t insg_dag_seed(uint64_t base, uint32_t cfg, uint64_t index) {
    uint64_t s = base ^ ((uint64_t)cfg << 32) ^ index;
    return sm64_next(&s);
}

/* -------------------------------------------------------------- batches -- */
typedef struct {
    int32_t ndag, n_types;
    int64_t n_total, m_total;
    int64_t *task_base; /* ndag+1 */
    int64_t *edge_base; /* ndag+1 */
    int32_t *row_ptr;   /* n_total + ndag: per DAG n_d+1 local offsets */
    int32_t *col_idx;   /* m_total local successor ids */
    uint8_t *type;      /* n_total */
    int64_t *type_cost; /* ndag * n_types * 2 (cpu, gpu) or NULL */
    int64_t *task_cost; /* n_total * 2 (cpu, gpu) or NULL */
} insg_batch;

/* one generated DAG before concatenation */
typedef struct {
    int32_t n, m;
    int32_t *row_ptr, *col_idx;
    uint8_t *type;
    int64_t type_cost[2 * 16];
    int64_t *task_cost;
} one_dag;

static void one_free(one_dag *d) {
    free(d->row_ptr); free(d->col_idx); free(d->type); free(d->task_cost);
    memset(d, 0, sizeof(*d));
}

/* Edge list (u, v) -> CSR with each row sorted ascending. */
static int build_csr(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, one_dag *d) {
    d->n = n; d->m = (int32_t)m;
    d->row_ptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    d->col_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!d->row_ptr || !d->col_idx) return -1;
    for (int64_t e = 0; e < m; ++e) d->row_ptr[eu[e] + 1]++;
    for (int32_t i = 0; i < n; ++i) d->row_ptr[i + 1] += d->row_ptr[i];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!fill) return -1;
    memcpy(fill, d->row_ptr, sizeof(int32_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; ++e) d->col_idx[fill[eu[e]]++] = ev[e];
    free(fill);
    for (int32_t i = 0; i < n; ++i) { /* insertion sort: rows are nearly sorted */
        int32_t *r = d->col_idx + d->row_ptr[i];
        int32_t len = d->row_ptr[i + 1] - d->row_ptr[i];
        for (int32_t a = 1; a < len; ++a) {
            int32_t x = r[a], b = a - 1;
            while (b >= 0 && r[b] > x) { r[b + 1] = r[b]; --b; }
            r[b + 1] = x;
        }
    }
    return 0;
}

/* growable edge list */
typedef struct { int32_t *u, *v; int64_t m, cap; } edges;
static int edges_push(edges *E, int32_t u, int32_t v) {
    if (E->m == E->cap) {
        int64_t nc = E->cap ? E->cap * 2 : 1024;
        int32_t *nu = (int32_t *)realloc(E->u, sizeof(int32_t) * (size_t)nc);
        if (!nu) return -1;
        E->u = nu;
        int32_t *nv = (int32_t *)realloc(E->v, sizeof(int32_t) * (size_t)nc);
        if (!nv) return -1;
        E->v = nv; E->cap = nc;
    }
    E->u[E->m] = u; E->v[E->m] = v; E->m++;
    return 0;
}
static void edges_free(edges *E) { free(E->u); free(E->v); memset(E, 0, sizeof(*E)); }

/* ------------------------------------------------------- layered DAGs -- */
typedef struct {
    int32_t n_min, n_max;     /* task count ~ U{n_min..n_max} */
    int32_t w_min, w_max;     /* layer width ~ U{w_min..w_max}, last layer truncated */
    double p_min, p_max;      /* per-DAG edge probability ~ U[p_min, p_max) */
    int32_t d_min, d_max;     /* per-DAG layer span ~ U{d_min..d_max} */
    int32_t n_types;          /* task type ~ U{0..n_types-1} (<= 16) */
    double cost_median_ns;    /* CPU cost per type: round(exp(ln median + sigma N(0,1))) */
    double cost_sigma;
    double speed_min, speed_max; /* GPU cost = max(1, round(cpu / U[speed_min, speed_max))) */
    int32_t typing;           /* 0: type ~ U{0..n_types-1}; 1: by in/out degree (n_types must be 16) */
} insg_layered_params;

/* Degree-based codelet of a task (the authors gave their generated tasks
 * codelets by inbound and outbound degree, Sec. 4.4 "Implementation details"):
 * 4 x bucket(in-degree) + bucket(out-degree), bucket(k) = min(3, bit length of k),
 * i.e. buckets {0}, {1}, {2, 3}, {4, ...}: 16 types. */
static uint8_t degree_type(int32_t indeg, int32_t outdeg) {
    int32_t bi = 0, bo = 0;
    while (bi < 3 && (indeg >> bi) != 0) ++bi;
    while (bo < 3 && (outdeg >> bo) != 0) ++bo;
    return (uint8_t)(4 * bi + bo);
}

/* Draw order per DAG (fixed): n, p, d, layer widths, edge coin flips in
 * (u ascending, layer ascending, v ascending) order, the fix-up parent of
 * every parentless non-first-layer node in id order, task types in id order
 * (random typing only; degree typing draws none), then per type: normal
 * deviate for CPU cost, then GPU speed-up. */
static int gen_layered_one(uint64_t seed, const insg_layered_params *P, one_dag *d) {
    uint64_t s = seed;
    int32_t n = (int32_t)urange(&s, P->n_min, P->n_max);
    double p = P->p_min + (P->p_max - P->p_min) * u01(&s);
    int32_t span = (int32_t)urange(&s, P->d_min, P->d_max);
    /* layers */
    int32_t cap_layers = n + 1, L = 0;
    int32_t *lstart = (int32_t *)malloc(sizeof(int32_t) * ((size_t)cap_layers + 1));
    if (!lstart) return -1;
    int32_t pos = 0;
    while (pos < n) {
        int32_t w = (int32_t)urange(&s, P->w_min, P->w_max);
        if (pos + w > n) w = n - pos;
        lstart[L++] = pos;
        pos += w;
    }
    lstart[L] = n;
    edges E = {0};
    uint8_t *has_pred = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!has_pred) return -1;
    for (int32_t l = 0; l < L; ++l) {
        for (int32_t u = lstart[l]; u < lstart[l + 1]; ++u) {
            for (int32_t l2 = l + 1; l2 <= l + span && l2 < L; ++l2) {
                for (int32_t v = lstart[l2]; v < lstart[l2 + 1]; ++v) {
                    if (u01(&s) < p) {
                        if (edges_push(&E, u, v)) return -1;
                        has_pred[v] = 1;
                    }
                }
            }
        }
    }
    for (int32_t l = 1; l < L; ++l) {
        int32_t pw = lstart[l] - lstart[l - 1];
        for (int32_t v = lstart[l]; v < lstart[l + 1]; ++v) {
            if (!has_pred[v]) {
                int32_t u = lstart[l - 1] + (int32_t)urange(&s, 0, pw - 1);
                if (edges_push(&E, u, v)) return -1;
            }
        }
    }
    free(has_pred);
    free(lstart);
    if (build_csr(n, E.m, E.u, E.v, d)) return -1;
    edges_free(&E);
    d->type = (uint8_t *)malloc((size_t)n + 1);
    if (!d->type) return -1;
    if (P->typing == 1) {
        int32_t *indeg = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        if (!indeg) return -1;
        for (int32_t e = 0; e < d->m; ++e) indeg[d->col_idx[e]]++;
        for (int32_t i = 0; i < n; ++i) d->type[i] = degree_type(indeg[i], d->row_ptr[i + 1] - d->row_ptr[i]);
        free(indeg);
    } else {
        for (int32_t i = 0; i < n; ++i) d->type[i] = (uint8_t)urange(&s, 0, P->n_types - 1);
    }
    for (int32_t k = 0; k < P->n_types; ++k) {
        double z = std_normal(&s);
        double cpu = exp(log(P->cost_median_ns) + P->cost_sigma * z);
        int64_t c = (int64_t)llround(cpu);
        if (c < 1) c = 1;
        double sp = P->speed_min + (P->speed_max - P->speed_min) * u01(&s);
        int64_t g = (int64_t)llround((double)c / sp);
        if (g < 1) g = 1;
        d->type_cost[2 * k + 0] = c;
        d->type_cost[2 * k + 1] = g;
    }
    d->task_cost = NULL;
    return 0;
}

/* --------------------------------------------------------- tiled DAGs -- */
/* Tile-level dependency inference with sequential consistency: a task that
 * reads tile X depends on X's last writer; a task that writes X depends on the
 * last writer and on every reader since that write. */
typedef struct {
    int32_t N;
    int32_t *last_writer;   /* N*N */
    int32_t **readers;      /* N*N lists of readers since the last write */
    int32_t *nread, *capread;
} tile_tracker;

static int tt_init(tile_tracker *T, int32_t N) {
    T->N = N;
    size_t k = (size_t)N * (size_t)N;
    T->last_writer = (int32_t *)malloc(sizeof(int32_t) * k);
    T->readers = (int32_t **)calloc(k, sizeof(int32_t *));
    T->nread = (int32_t *)calloc(k, sizeof(int32_t));
    T->capread = (int32_t *)calloc(k, sizeof(int32_t));
    if (!T->last_writer || !T->readers || !T->nread || !T->capread) return -1;
    for (size_t i = 0; i < k; ++i) T->last_writer[i] = -1;
    return 0;
}
static void tt_free(tile_tracker *T) {
    size_t k = (size_t)T->N * (size_t)T->N;
    for (size_t i = 0; i < k; ++i) free(T->readers[i]);
    free(T->readers); free(T->last_writer); free(T->nread); free(T->capread);
}

/* Accumulates the predecessor set of the task being submitted. */
typedef struct { int32_t *p; int32_t n, cap; } predset;
static int ps_add(predset *S, int32_t u) {
    for (int32_t i = 0; i < S->n; ++i) if (S->p[i] == u) return 0;
    if (S->n == S->cap) {
        int32_t nc = S->cap ? S->cap * 2 : 16;
        int32_t *np = (int32_t *)realloc(S->p, sizeof(int32_t) * (size_t)nc);
        if (!np) return -1;
        S->p = np; S->cap = nc;
    }
    S->p[S->n++] = u;
    return 0;
}

typedef struct { int32_t tile; int write; } access;

static int submit(tile_tracker *T, edges *E, predset *S, int32_t task, const access *acc, int na) {
    S->n = 0;
    for (int a = 0; a < na; ++a) {
        int32_t x = acc[a].tile;
        if (T->last_writer[x] >= 0 && ps_add(S, T->last_writer[x])) return -1;
        if (acc[a].write)
            for (int32_t r = 0; r < T->nread[x]; ++r)
                if (T->readers[x][r] != task && ps_add(S, T->readers[x][r])) return -1;
    }
    for (int32_t i = 0; i < S->n; ++i)
        if (edges_push(E, S->p[i], task)) return -1;
    for (int a = 0; a < na; ++a) {
        int32_t x = acc[a].tile;
        if (acc[a].write) {
            T->last_writer[x] = task;
            T->nread[x] = 0;
        } else {
            if (T->nread[x] == T->capread[x]) {
                int32_t nc = T->capread[x] ? T->capread[x] * 2 : 4;
                int32_t *nr = (int32_t *)realloc(T->readers[x], sizeof(int32_t) * (size_t)nc);
                if (!nr) return -1;
                T->readers[x] = nr; T->capread[x] = nc;
            }
            T->readers[x][T->nread[x]++] = task;
        }
    }
    return 0;
}

enum { TILED_CHOLESKY = 0, TILED_LU = 1, TILED_QR = 2 };

/* Task counts: Cholesky N + N(N-1) + N(N-1)(N-2)/6; LU and QR
 * N + N(N-1) + (N-1)N(2N-1)/6. */
EXPORT int64_t insg_tiled_count(int32_t kind, int32_t N) {
    int64_t n = N;
    if (kind == TILED_CHOLESKY) return n + n * (n - 1) + n * (n - 1) * (n - 2) / 6;
    return n + n * (n - 1) + (n - 1) * n * (2 * n - 1) / 6;
}

static int gen_tiled_one(int32_t kind, int32_t N, one_dag *d, uint8_t *type_out_buf) {
    (void)type_out_buf;
    int64_t ntask = insg_tiled_count(kind, N);
    tile_tracker T;
    if (tt_init(&T, N)) return -1;
    edges E = {0};
    predset S = {0};
    uint8_t *ty = (uint8_t *)malloc((size_t)ntask + 1);
    if (!ty) return -1;
    int32_t t = 0;
#define TILE(i, j) ((i) * N + (j))
#define SUBMIT(tp, ...)                                                     \
    do {                                                                    \
        access a_[] = {__VA_ARGS__};                                        \
        if (submit(&T, &E, &S, t, a_, (int)(sizeof(a_) / sizeof(a_[0])))) \
            return -1;                                                      \
        ty[t++] = (uint8_t)(tp);                                            \
    } while (0)
    for (int32_t k = 0; k < N; ++k) {
        if (kind == TILED_CHOLESKY) {
            /* types: 0 POTRF, 1 TRSM, 2 SYRK, 3 GEMM */
            SUBMIT(0, {TILE(k, k), 1});
            for (int32_t i = k + 1; i < N; ++i) SUBMIT(1, {TILE(k, k), 0}, {TILE(i, k), 1});
            for (int32_t i = k + 1; i < N; ++i) {
                SUBMIT(2, {TILE(i, k), 0}, {TILE(i, i), 1});
                for (int32_t j = k + 1; j < i; ++j)
                    SUBMIT(3, {TILE(i, k), 0}, {TILE(j, k), 0}, {TILE(i, j), 1});
            }
        } else if (kind == TILED_LU) {
            /* types: 0 GETRF, 1 TRSM (row and column panels), 2 GEMM */
            SUBMIT(0, {TILE(k, k), 1});
            for (int32_t j = k + 1; j < N; ++j) SUBMIT(1, {TILE(k, k), 0}, {TILE(k, j), 1});
            for (int32_t i = k + 1; i < N; ++i) SUBMIT(1, {TILE(k, k), 0}, {TILE(i, k), 1});
            for (int32_t i = k + 1; i < N; ++i)
                for (int32_t j = k + 1; j < N; ++j)
                    SUBMIT(2, {TILE(i, k), 0}, {TILE(k, j), 0}, {TILE(i, j), 1});
        } else {
            /* types: 0 GEQRT, 1 UNMQR, 2 TSQRT, 3 TSMQR (flat reduction tree) */
            SUBMIT(0, {TILE(k, k), 1});
            for (int32_t j = k + 1; j < N; ++j) SUBMIT(1, {TILE(k, k), 0}, {TILE(k, j), 1});
            for (int32_t i = k + 1; i < N; ++i) {
                SUBMIT(2, {TILE(k, k), 1}, {TILE(i, k), 1});
                for (int32_t j = k + 1; j < N; ++j)
                    SUBMIT(3, {TILE(i, k), 0}, {TILE(k, j), 1}, {TILE(i, j), 1});
            }
        }
    }
#undef SUBMIT
#undef TILE
    tt_free(&T);
    free(S.p);
    if (t != ntask) return -2;
    if (build_csr((int32_t)ntask, E.m, E.u, E.v, d)) return -1;
    edges_free(&E);
    d->type = ty;
    return 0;
}

/* ------------------------------------------------------- concatenation -- */
static insg_batch *concat(one_dag *D, int32_t ndag, int32_t n_types, int with_type_cost, int with_task_cost) {
    insg_batch *B = (insg_batch *)calloc(1, sizeof(insg_batch));
    if (!B) return NULL;
    B->ndag = ndag; B->n_types = n_types;
    B->task_base = (int64_t *)malloc(sizeof(int64_t) * ((size_t)ndag + 1));
    B->edge_base = (int64_t *)malloc(sizeof(int64_t) * ((size_t)ndag + 1));
    if (!B->task_base || !B->edge_base) return NULL;
    B->task_base[0] = 0; B->edge_base[0] = 0;
    for (int32_t i = 0; i < ndag; ++i) {
        B->task_base[i + 1] = B->task_base[i] + D[i].n;
        B->edge_base[i + 1] = B->edge_base[i] + D[i].m;
    }
    B->n_total = B->task_base[ndag];
    B->m_total = B->edge_base[ndag];
    B->row_ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(B->n_total + ndag + 1));
    B->col_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(B->m_total + 1));
    B->type = (uint8_t *)malloc((size_t)B->n_total + 1);
    if (!B->row_ptr || !B->col_idx || !B->type) return NULL;
    if (with_type_cost) {
        B->type_cost = (int64_t *)malloc(sizeof(int64_t) * (size_t)ndag * (size_t)n_types * 2);
        if (!B->type_cost) return NULL;
    }
    if (with_task_cost) {
        B->task_cost = (int64_t *)malloc(sizeof(int64_t) * (size_t)(B->n_total * 2 + 1));
        if (!B->task_cost) return NULL;
    }
    for (int32_t i = 0; i < ndag; ++i) {
        int64_t tb = B->task_base[i], eb = B->edge_base[i];
        memcpy(B->row_ptr + tb + i, D[i].row_ptr, sizeof(int32_t) * ((size_t)D[i].n + 1));
        if (D[i].m) memcpy(B->col_idx + eb, D[i].col_idx, sizeof(int32_t) * (size_t)D[i].m);
        if (D[i].n) memcpy(B->type + tb, D[i].type, (size_t)D[i].n);
        if (with_type_cost)
            memcpy(B->type_cost + (size_t)i * n_types * 2, D[i].type_cost, sizeof(int64_t) * (size_t)n_types * 2);
        if (with_task_cost && D[i].n)
            memcpy(B->task_cost + tb * 2, D[i].task_cost, sizeof(int64_t) * (size_t)D[i].n * 2);
    }
    return B;
}

EXPORT void insg_free(insg_batch *B) {
    if (!B) return;
    free(B->task_base); free(B->edge_base); free(B->row_ptr); free(B->col_idx);
    free(B->type); free(B->type_cost); free(B->task_cost);
    free(B);
}

/* DAG i (i = first .. first+ndag-1) of workload cfg, each from its own stream. */
EXPORT insg_batch *insg_layered(uint64_t base, uint32_t cfg, uint64_t first, int32_t ndag,
                                const insg_layered_params *P) {
    if (ndag < 0 || P->n_types < 1 || P->n_types > 16 || P->n_min < 0 || P->n_max < P->n_min ||
        P->w_min < 1 || P->w_max < P->w_min || P->d_min < 1 || P->d_max < P->d_min ||
        (P->typing != 0 && P->typing != 1) || (P->typing == 1 && P->n_types != 16))
        return NULL;
    one_dag *D = (one_dag *)calloc((size_t)ndag + 1, sizeof(one_dag));
    if (!D) return NULL;
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : fail)
    for (int32_t i = 0; i < ndag; ++i)
        fail |= gen_layered_one(insg_dag_seed(base, cfg, first + (uint64_t)i), P, &D[i]) != 0;
    insg_batch *B = fail ? NULL : concat(D, ndag, P->n_types, 1, 0);
    for (int32_t i = 0; i < ndag; ++i) one_free(&D[i]);
    free(D);
    return B;
}

/* ndag instances of one tiled factorisation DAG.  base_cost[type][cpu, gpu]
 * in ns.  perturb != 0: every task's two costs are scaled by the integer-exact
 * factor (800000 + r mod 400001) / 1e6 (uniform within +-20 %), r drawn per
 * task from the instance's stream; otherwise costs come from the type table. */
EXPORT insg_batch *insg_tiled(int32_t kind, int32_t N, uint64_t base, uint32_t cfg, uint64_t first,
                              int32_t ndag, const int64_t *base_cost, int32_t perturb) {
    if (kind < 0 || kind > 2 || N < 1 || ndag < 0) return NULL;
    int32_t n_types = (kind == TILED_LU) ? 3 : 4;
    one_dag *D = (one_dag *)calloc((size_t)ndag + 1, sizeof(one_dag));
    if (!D) return NULL;
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
    for (int32_t i = 0; i < ndag; ++i) {
        if (gen_tiled_one(kind, N, &D[i], NULL)) { fail = 1; continue; }
        for (int32_t k = 0; k < n_types; ++k) {
            D[i].type_cost[2 * k] = base_cost[2 * k];
            D[i].type_cost[2 * k + 1] = base_cost[2 * k + 1];
        }
        if (perturb) {
            uint64_t s = insg_dag_seed(base, cfg, first + (uint64_t)i);
            D[i].task_cost = (int64_t *)malloc(sizeof(int64_t) * (size_t)D[i].n * 2 + 8);
            if (!D[i].task_cost) { fail = 1; continue; }
            for (int32_t t = 0; t < D[i].n; ++t) {
                int64_t f = 800000 + (int64_t)(sm64_next(&s) % 400001u);
                for (int c = 0; c < 2; ++c) {
                    int64_t v = base_cost[2 * D[i].type[t] + c] * f / 1000000;
                    D[i].task_cost[2 * t + c] = v < 1 ? 1 : v;
                }
            }
        }
    }
    insg_batch *B = fail ? NULL : concat(D, ndag, n_types, 1, perturb ? 1 : 0);
    for (int32_t i = 0; i < ndag; ++i) one_free(&D[i]);
    free(D);
    return B;
}

/* Concatenate already generated batches (e.g. a mixed-size workload). */
EXPORT insg_batch *insg_concat(insg_batch *const *parts, int32_t nparts) {
    int32_t ndag = 0, n_types = 1, any_task_cost = 0;
    for (int32_t p = 0; p < nparts; ++p) {
        ndag += parts[p]->ndag;
        if (parts[p]->n_types > n_types) n_types = parts[p]->n_types;
        if (parts[p]->task_cost) any_task_cost = 1;
    }
    one_dag *D = (one_dag *)calloc((size_t)ndag + 1, sizeof(one_dag));
    if (!D) return NULL;
    int32_t k = 0;
    for (int32_t p = 0; p < nparts; ++p) {
        const insg_batch *B = parts[p];
        for (int32_t i = 0; i < B->ndag; ++i, ++k) {
            int64_t tb = B->task_base[i];
            D[k].n = (int32_t)(B->task_base[i + 1] - tb);
            D[k].m = (int32_t)(B->edge_base[i + 1] - B->edge_base[i]);
            D[k].row_ptr = B->row_ptr + tb + i;
            D[k].col_idx = B->col_idx + B->edge_base[i];
            D[k].type = B->type + tb;
            for (int32_t t = 0; t < 2 * 16; ++t) D[k].type_cost[t] = 1;
            for (int32_t t = 0; t < 2 * B->n_types; ++t) D[k].type_cost[t] = B->type_cost[(size_t)i * B->n_types * 2 + t];
            if (any_task_cost) {
                D[k].task_cost = (int64_t *)malloc(sizeof(int64_t) * (size_t)D[k].n * 2 + 8);
                if (!D[k].task_cost) return NULL;
                for (int32_t t = 0; t < D[k].n; ++t)
                    for (int c = 0; c < 2; ++c)
                        D[k].task_cost[2 * t + c] = B->task_cost ? B->task_cost[(tb + t) * 2 + c]
                                                                 : B->type_cost[((size_t)i * B->n_types + D[k].type[t]) * 2 + c];
            }
        }
    }
    insg_batch *R = concat(D, ndag, n_types, 1, any_task_cost);
    for (int32_t i = 0; i < ndag; ++i) free(D[i].task_cost);
    free(D);
    return R;
}

/* The mixed-size stress workload: DAG i (i = first .. first+ndag-1) draws from its own stream a
 * task count n* = round(exp(U[ln n_lo, ln n_hi))) (log-uniform); even i give a random layered
 * DAG of exactly n* tasks (shape parameters P, its n range ignored), odd i a tiled Cholesky, LU
 * or QR DAG (kind uniform) of the largest tile count whose task count is at most n* (at least
 * one tile).  Costs are per task: a layered task's from its DAG's type table, a tiled task's
 * from base_cost[kind][type] scaled by (800000 + r mod 400001) / 1e6 as in insg_tiled.  Draw
 * order per DAG: n*, then (tiled) kind, then the generator's own draws from a second stream
 * seeded by the DAG's seed plus one. */
EXPORT insg_batch *insg_mixed(uint64_t base, uint32_t cfg, uint64_t first, int32_t ndag, int64_t n_lo, int64_t n_hi,
                              const insg_layered_params *P, const int64_t *base_cost /* [3][4][2] */) {
    if (ndag < 0 || n_lo < 1 || n_hi < n_lo || n_hi > (1 << 24) - 1 || P->n_types < 1 || P->n_types > 16 ||
        P->typing != 0)
        return NULL;
    one_dag *D = (one_dag *)calloc((size_t)ndag + 1, sizeof(one_dag));
    if (!D) return NULL;
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
    for (int32_t i = 0; i < ndag; ++i) {
        uint64_t seed = insg_dag_seed(base, cfg, first + (uint64_t)i);
        uint64_t s = seed;
        double ln = log((double)n_lo) + (log((double)n_hi) - log((double)n_lo)) * u01(&s);
        int64_t want = (int64_t)llround(exp(ln));
        if (want < n_lo) want = n_lo;
        if (want > n_hi) want = n_hi;
        one_dag *d = &D[i];
        if (((first + (uint64_t)i) & 1u) == 0) {
            insg_layered_params Q = *P;
            Q.n_min = Q.n_max = (int32_t)want;
            if (gen_layered_one(seed + 1, &Q, d)) { fail = 1; continue; }
            d->task_cost = (int64_t *)malloc(sizeof(int64_t) * (size_t)d->n * 2 + 8);
            if (!d->task_cost) { fail = 1; continue; }
            for (int32_t t = 0; t < d->n; ++t)
                for (int c = 0; c < 2; ++c) d->task_cost[2 * t + c] = d->type_cost[2 * d->type[t] + c];
        } else {
            int32_t kind = (int32_t)urange(&s, 0, 2);
            int32_t N = 1;
            while (insg_tiled_count(kind, N + 1) <= want) ++N;
            if (gen_tiled_one(kind, N, d, NULL)) { fail = 1; continue; }
            uint64_t r = seed + 1;
            d->task_cost = (int64_t *)malloc(sizeof(int64_t) * (size_t)d->n * 2 + 8);
            if (!d->task_cost) { fail = 1; continue; }
            const int64_t *bc = base_cost + (size_t)kind * 8;
            for (int32_t t = 0; t < d->n; ++t) {
                int64_t f = 800000 + (int64_t)(sm64_next(&r) % 400001u);
                for (int c = 0; c < 2; ++c) {
                    int64_t v = bc[2 * d->type[t] + c] * f / 1000000;
                    d->task_cost[2 * t + c] = v < 1 ? 1 : v;
                }
            }
            for (int32_t k = 0; k < 16; ++k) { d->type_cost[2 * k] = 1; d->type_cost[2 * k + 1] = 1; }
        }
    }
    insg_batch *B = fail ? NULL : concat(D, ndag, P->n_types, 1, 1);
    for (int32_t i = 0; i < ndag; ++i) one_free(&D[i]);
    free(D);
    return B;
}

/* The task count insg_mixed draws for DAG i (before tiling rounds it down): n*[i - first]. */
EXPORT void insg_mixed_sizes(uint64_t base, uint32_t cfg, uint64_t first, int32_t ndag, int64_t n_lo, int64_t n_hi,
                             int64_t *out) {
    for (int32_t i = 0; i < ndag; ++i) {
        uint64_t s = insg_dag_seed(base, cfg, first + (uint64_t)i);
        double ln = log((double)n_lo) + (log((double)n_hi) - log((double)n_lo)) * u01(&s);
        int64_t want = (int64_t)llround(exp(ln));
        out[i] = want < n_lo ? n_lo : (want > n_hi ? n_hi : want);
    }
}
