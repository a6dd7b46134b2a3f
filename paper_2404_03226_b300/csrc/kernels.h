// Launch interface between the host runtime (insp_api.cu) and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "mlp.cuh"

namespace insp {

struct SimArgs {
    DevBatch B;
    int32_t n_cpu, n_gpu;
    int64_t xfer;
    int32_t policy, task_window, s_inc, s_dec, dec_step, c;
    int64_t k_inc_tasks, k_inc_ns;
    const int64_t *unit_time;      // per DAG unit time T of the attributes (k_inc default: P tasks per T)
    const int32_t *indeg0;
    const int32_t *ia, *ie;
    int32_t *worker;
    int64_t *start, *end, *makespan;
    int32_t *status;
    // scratch, indexed by global task id
    int2 *st_a;         // {remaining in-degree, node of the latest predecessor completion}
    longlong2 *st_b;    // {latest completion time, latest on another node}
    int32_t *p_idw, *p_seq, *p_ia, *p_ie;  // pool spill
    int64_t *p_dr, *p_cost;
    int32_t *nl;        // released-task spill
    // work distribution
    const int32_t *order;  // DAGs by descending size (or a contiguous part of that order)
    int32_t n_order;       // DAGs in order[]
    int32_t *counter;
    int32_t single_dag;    // >= 0: only that DAG, one warp
    // learned scorer (policy INSP_POLICY_LEARNED)
    const ScorerPacked *scorer;
    // rollouts: per DAG, at pop number force_pop[d] take task force_task[d] if it is
    // in the popping worker's queue; at pop number feat_pop[d] record the features
    // of up to feat_cap candidates of that queue in push order
    const int32_t *force_pop, *force_task, *feat_pop;
    int32_t feat_cap;
    int32_t *feat_task, *feat, *feat_n;
    // static priority of INSP_POLICY_DMDAP_BL (bottom level per task, global index)
    const int64_t *blevel;
    // push/pop trace (null: off), indexed by task_base[d] + k for the k-th push / pop of DAG d
    int64_t *tr_push_time, *tr_pop_time;
    int32_t *tr_push_task, *tr_push_worker, *tr_push_nready;
    int32_t *tr_pop_task, *tr_pop_worker, *tr_pop_nready, *tr_pop_mode;
};

// DAGs of up to this many tasks count their in-degrees (validation) and predecessor-list cursors
// in shared memory; larger ones use global atomics
constexpr int32_t VALIDATE_SMEM_TASKS = 16384;
// validation, in-degrees, spans and (hash != NULL) structure fingerprints; max_n: the largest DAG
void launch_validate(const DevBatch &B, int64_t xfer, int32_t *status, int32_t *indeg0, int32_t *max_span,
                     int32_t *dag_span, unsigned long long *hash, int32_t max_n, int grid, cudaStream_t s);
void launch_unit_time(const DevBatch &B, const int32_t *status, int64_t *unit_time, int grid, cudaStream_t s);
// Renumbering of the listed DAGs (ids not topological): Kahn rounds, ascending old id within a
// round (k_load.cu).  Scratch cnt, level, qa, qb: per task (global indexing); n_levels: per
// listed DAG.  status[d] becomes INSP_OK or INSP_ECYCLE.
void launch_kahn(const DevBatch &B, const int32_t *dags, int32_t n_dags, const int32_t *indeg0, int32_t *cnt,
                 int32_t *level, int32_t *qa, int32_t *qb, int32_t *n_levels, int32_t *new_of_old,
                 int32_t *old_of_new, int32_t *status, cudaStream_t s);
// The renumbered arrays of the listed DAGs into out_* (which hold a copy of the batch).
void launch_renumber(const DevBatch &B, const int32_t *dags, int32_t n_dags, const int32_t *old_of_new,
                     const int32_t *new_of_old, int32_t *out_rp, int32_t *out_col, uint8_t *out_type,
                     int64_t *out_task_cost, const int32_t *status, cudaStream_t s);
void launch_local_iota(const int64_t *task_base, int32_t ndag, int32_t *out, cudaStream_t s);
// Per-task arrays between the batch's numbering and the caller's (4- or 8-byte elements).
void launch_permute(const int64_t *task_base, int32_t ndag, const int32_t *old_of_new, const void *src, void *dst,
                    int elem_bytes, bool to_caller, cudaStream_t s);
// Device-side step counters of the attribute kernels: the done-flag epoch of
// the ability sweep and the 64-bit record tag base of the efficiency sweep.
struct StepCounters {
    int32_t epoch;
    int32_t pad;
    uint64_t tag_base;
};
void launch_step_begin(StepCounters *c, int64_t n_items, cudaStream_t s);
void launch_wait_probe(const int32_t *flag, int32_t value, int32_t limit, int32_t *status, cudaStream_t s);
void launch_ia(const DevBatch &B, const int32_t *order, int32_t n_order, int32_t *counter, uint64_t *bits,
               int64_t slot_words, int32_t *done, const int32_t *epoch, int32_t *ia, int32_t *status, int grid,
               int warps, cudaStream_t s);
void launch_ie(const DevBatch &B, const int64_t *item_base, int64_t n_items, int32_t *counter,
               const int64_t *unit_time, uint4 *rec, int64_t rec_stride, void *acc, int32_t W, bool wide,
               const uint64_t *tag_base, int32_t *ie, int grid, cudaStream_t s);
// Inspiring ability by target blocks (any DAG size): work items {dag, block} of IA_BLK_BITS
// target ids, per CTA a ring of ring_rows rows (a power of two >= the DAG's longest edge span
// + warps per CTA) and publish flags; slot_seq[grid] per-CTA item tags (start at 0).
constexpr int32_t IA_BLK_BITS = 8192;
constexpr int32_t IA_BLK_WORDS = IA_BLK_BITS / 64;
void launch_ia_blk(const DevBatch &B, const int2 *items, int32_t n_items, int32_t *counter, uint64_t *ring,
                   unsigned long long *flags, int32_t ring_rows, uint32_t *slot_seq, int32_t *ia, int32_t *status,
                   int grid, int warps, cudaStream_t s);
void launch_ia_zero(const DevBatch &B, const int32_t *dags, int32_t n_dags, int32_t *ia, cudaStream_t s);
void launch_ia_copy(const DevBatch &B, const int2 *pairs, int32_t n_pairs, int32_t *ia, cudaStream_t s);
void launch_dag_equal(const DevBatch &B, const int2 *pairs, int32_t n_pairs, int32_t *same, cudaStream_t s);
int ia_blk_occupancy(int warps);
// inspiring efficiency, pull form (k_ie_pull.cu)
// Longest window (ring rows, a power of two above the batch's longest edge span) of the
// pull form: its per-warp ring is W x 128 bytes, so long spans only cost ring memory (the
// tuning's ring budget then admits fewer warps); beyond it the global form runs.
constexpr int32_t IE_PULL_MAX_W = 8192;
// Sources per work item of the pull form (one warp; 64 = two per lane).  128 (four per lane,
// int4 ring rows) runs 24 % fewer instructions but was measured 1.5x slower: the ring
// traffic then bounds the sweep.
constexpr int32_t IE_PULL_SOURCES = 64;
int ie_pull_max_warps();
int64_t ie_pull_ring_bytes(int32_t W);
int ie_pull_occupancy(int warps, int32_t W);
// gring: per-warp rings of ie_pull_ring_bytes(W) in global memory
void launch_ie_pull(const DevBatch &B, const int32_t *pr_ptr, const int32_t *pcol, const int64_t *item_base,
                    const int32_t *item_dag, int64_t item_lo, int64_t item_hi, int32_t *counter,
                    const int64_t *unit_time, const int32_t *dag_span, int32_t W, int32_t *gring, int32_t *ie,
                    int grid, int warps, cudaStream_t s);
void launch_reverse_csr(const DevBatch &B, const int32_t *indeg0, int32_t *pr_ptr, int32_t *cursor, int32_t *pcol,
                        int32_t max_n, int grid, cudaStream_t s);
// learned scorer (k_mlp.cu)
void launch_scorer_eval(const ScorerPacked *P, const int32_t *feat, int64_t n, int64_t *score, cudaStream_t s);
void launch_mlp_train_grad(int32_t in, int32_t h1, int32_t h2, const float *w, int32_t mode, int64_t n,
                           const float *x, const float *target, float *work, float *grad, float *loss,
                           cudaStream_t s);
// the tensor-core form: part = caller scratch of ceil(n / 16) x (nweights + 1) floats
void launch_mlp_train_grad_tc(int32_t in, int32_t h1, int32_t h2, const float *w, int32_t mode, int64_t n,
                              const float *x, const float *target, float *part, float *grad, float *loss,
                              cudaStream_t s);
void launch_adamw(int64_t nw, float *w, float *m, float *v, const float *g, int32_t t, float lr, float b1, float b2,
                  float eps, float wd, cudaStream_t s);
void launch_quantize(int64_t nw, const float *w, uint16_t *out, cudaStream_t s);
void launch_sim(const SimArgs &A, int grid, int warps, int queue, cudaStream_t s);
// Unit-time search (k_search.cu).
void launch_search_target(const DevBatch &B, const int32_t *order, int32_t *counter, const int32_t *ia,
                          int32_t *layer, uint32_t *bitmap, const int64_t *bm_base, int64_t *target, int grid,
                          cudaStream_t s);
void launch_search_ut(int32_t ndag, int32_t k, const int64_t *unit_time_def, const int32_t *done, int64_t *ut,
                      cudaStream_t s);
void launch_search_step(const DevBatch &B, const int32_t *order, int32_t *counter, const int32_t *ie,
                        uint32_t *bitmap, const int64_t *bm_base, const int64_t *target, const int64_t *ut,
                        int32_t *done, int64_t *chosen, int32_t *n_done, int grid, cudaStream_t s);
void launch_search_final(int32_t ndag, int32_t k_max, const int64_t *unit_time_def, const int32_t *done,
                         int64_t *chosen, cudaStream_t s);
// Bottom levels (HEFT upward rank over mean costs) of every task; cbar = the mean
// transfer cost (computed by the host).  One warp per DAG, DAGs in size order.
void launch_blevel(const DevBatch &B, int32_t n_cpu, int32_t n_gpu, int64_t cbar, const int32_t *order,
                   int32_t *counter, int64_t *bl, int grid, cudaStream_t s);
int sim_occupancy(bool learned, int n_workers, int warps, int queue);
int sim_max_warps();
void launch_sim_single(const SimArgs &A, cudaStream_t s);
int ia_max_warps();
int ia_occupancy(int warps);
int ie_threads();
int ie_occupancy();

}  // namespace insp
