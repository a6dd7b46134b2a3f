/*
 * inspirit.h -- C ABI of the B300 INSPIRIT schedule evaluator.
 *
 * Evaluates the INSPIRIT scheduling policy (arxiv 2404.03226) on task DAGs and
 * a modelled heterogeneous machine, entirely in CUDA kernels for sm_103a:
 *
 *   insp_attributes*  inspiring ability and inspiring efficiency of every task
 *                     (Sec. 4.2 definitions, Sec. 4.3 computation);
 *   insp_simulate*    the list-scheduling run (Sec. 2.1 push/pop over per-worker
 *                     queues, Sec. 4.1 steps 1-3, Sec. 4.4 Nready regulation by
 *                     adaptive priority) returning each task's worker, start and
 *                     end time and each DAG's makespan.
 *
 * Conventions for every entry point
 *   - Status: every function returns INSP_OK (0) or one of the INSP_E* codes
 *     below; nothing aborts.  insp_last_error() returns a thread-local message
 *     for the last failure on the calling thread.
 *   - Ownership: load functions copy their inputs into library-owned device
 *     memory; the caller may free its arrays after the call returns.  Output
 *     arrays are caller-owned.
 *   - Pointers: inputs and outputs may be host or device pointers (detected
 *     with cudaPointerGetAttributes).  When every output is a device pointer
 *     the call only enqueues work on `stream` and returns; results and the
 *     per-DAG status (insp_batch_status) are valid after the caller
 *     synchronises the stream.  When any array is a host pointer the call
 *     stages through device buffers, synchronises `stream` and returns the
 *     final status, including device-side errors.
 *   - Streams: `stream` is a cudaStream_t passed as void*; NULL means the
 *     legacy default stream.  Calls on one batch must not overlap in time.
 *   - Numbering: tasks of a DAG are 0..n-1; successor lists are strictly
 *     increasing.  The method needs ids in a topological order (every edge
 *     (u, v) with u < v).  A DAG loaded in another numbering (as a runtime's
 *     dependency manager lists its tasks, Sec. 2.1) is renumbered at load by
 *     Kahn's algorithm in rounds -- round 0 the tasks without predecessors,
 *     round r + 1 the tasks whose predecessors all lie in rounds <= r, new ids
 *     consecutive within a round in ascending old id -- and evaluated in that
 *     numbering (every tie broken by the lowest id means the lowest new id);
 *     all per-task inputs and outputs stay in the caller's numbering.  A DAG
 *     whose ids are already topological keeps them.  A cycle: INSP_ECYCLE.
 *     Workers 0..n_cpu-1 are CPUs, n_cpu..n_cpu+n_gpu-1 GPUs.
 *   - Time: all costs and times are int64 nanoseconds; costs are >= 1.
 */
#ifndef INSPIRIT_H
#define INSPIRIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define INSP_OK 0
#define INSP_EINVAL 1    /* malformed argument: bad CSR, id out of range, duplicate or unsorted successor, cost < 1, type >= n_types, bad size */
#define INSP_ENOTTOPO 2  /* an edge (u, v) with v <= u where a topological numbering is required
                            (insp_simulate_noalloc); the load functions renumber instead */
#define INSP_ENOMEM 3    /* device or host allocation failed */
#define INSP_ECUDA 4     /* a CUDA runtime call failed (message in insp_last_error) */
#define INSP_ETIMEOUT 5  /* a bounded device-side wait gave up (no GPU hang; the DAG's outputs are invalid) */
#define INSP_EOVERFLOW 6 /* sum over tasks of (max cost + transfer) exceeds 2^54 ns, so times could overflow */
#define INSP_ECHECK 7    /* debug builds only (INSP_CHECK): an internal bounds check failed; outputs invalid */
#define INSP_ECYCLE 8    /* the successor lists contain a cycle: no topological numbering exists */

/* insp_scorer_eval's score of a row whose tensor-core tile did not complete in time */
#define INSP_SCORE_TIMEOUT INT64_MIN

/* ---------------------------------------------------------------- policy */
#define INSP_POLICY_INSPIRIT 0 /* adaptive priority by the Nready controller (default) */
#define INSP_POLICY_FIFO 1     /* DMDA without priorities: pop in push order (Sec. 2.1) */
#define INSP_POLICY_LEARNED 2  /* controller runs, but the pop takes the learned scorer's best candidate
                                  (highest score, ties to the lowest id); needs insp_set_scorer */
/* DMDAP baselines (Sec. 2.1: DMDA with task priorities; Sec. 3 Observation 1):
 * the pop always takes the highest static priority of the worker's queue, ties
 * to the lowest id, with no Nready controller. */
#define INSP_POLICY_DMDAP_IA 3 /* priority = inspiring ability (the ia input) */
#define INSP_POLICY_DMDAP_BL 4 /* priority = bottom level, HEFT's upward rank (insp_bottom_level_batch);
                                  the library computes it, the ia / ie inputs are not read */

/* Controller parameters of Sec. 4.4 (the paper gives no values).  A zero
 * field takes its default for P = n_cpu + n_gpu workers and the unit time T
 * of the DAG's inspiring efficiency (Sec. 4.2-4.3: the ascending slope is a
 * task count per that same unit time window):
 *   task_window = s_inc = s_dec = dec_step = P, c = max(1, P / 2),
 *   k_inc = k_inc_tasks / k_inc_ns = P tasks per T ns.
 * T is the DAG's unit time in the batch's last insp_attributes* or
 * insp_evaluate_batch* call (before any: the DAG's default unit time, 4 x the
 * lower median of its GPU costs); insp_simulate_noalloc takes the default
 * unit time.  Simulating with attributes computed elsewhere at another T needs
 * k_inc set explicitly. */
typedef struct {
    int32_t policy;      /* INSP_POLICY_* */
    int32_t task_window; /* re-judge the state when Nready moved by at least this much */
    int32_t s_inc;       /* minimum Nready growth before the slope is tested (ascending state) */
    int32_t s_dec;       /* stage size of the descending peak threshold */
    int32_t dec_step;    /* INC if Nready >= peak - dec_step, else DEC */
    int32_t c;           /* slack below the next stage threshold for efficiency+locality picks */
    int64_t k_inc_tasks; /* ascending slope threshold, numerator (tasks) */
    int64_t k_inc_ns;    /* ascending slope threshold, denominator (ns) */
} insp_policy;

/* --------------------------------------------------------------- objects */
typedef struct insp_machine insp_machine; /* workers, transfer cost, policy, scorer */
typedef struct insp_batch insp_batch;     /* one or more DAGs resident in device memory */
typedef struct insp_batch insp_dag;       /* a batch holding exactly one DAG */

/* Create a machine of n_cpu CPU workers (memory node 0) and n_gpu GPU workers
 * (GPU g is memory node 1+g); an edge whose two tasks run on different memory
 * nodes costs xfer_ns before the successor can start (DMDA's transfer-aware
 * placement, Sec. 2.1).  1 <= n_cpu + n_gpu <= 64, xfer_ns >= 0.  `policy`
 * may be NULL (all defaults).  Errors: INSP_EINVAL, INSP_ENOMEM. */
int insp_machine_create(int32_t n_cpu, int32_t n_gpu, int64_t xfer_ns, const insp_policy *policy,
                        insp_machine **out);
/* Destroy a machine.  A destroyed batch hands its kernel scratch and its device
 * buffers back to its machine for reuse by the next load (up to two sets are
 * kept; they are freed here).  Batches loaded on the machine may still be alive
 * (a garbage collector may finalise the two handles in either order): they stay
 * usable, and the machine's memory is released when the last of them is
 * destroyed.  No call may use `m` itself afterwards.  NULL is ignored. */
void insp_machine_destroy(insp_machine *m);

/* Install the learned proposal scorer used by INSP_POLICY_LEARNED: an MLP
 * 16 -> 64 -> 64 -> 1 with BF16 weights and FP32 accumulation (no
 * counterpart in the paper).  `bf16_weights` holds, in this order, W1[16][64],
 * b1[64], W2[64][64], b2[64], W3[64], b3[1] as raw BF16 bit patterns
 * (nbytes = 5313 * 2); every value must be k / 64 with integer |k| <= 128.
 * Host pointer.  Call it before loading batches on the machine, not while its
 * batches load or evaluate on other threads.  Errors: INSP_EINVAL (size or
 * off-grid value). */
int insp_set_scorer(insp_machine *m, const uint16_t *bf16_weights, size_t nbytes);

/* Load one DAG of n tasks (CSR, Sec. 2.1 task graph).
 *   row_ptr[n+1] int32, row_ptr[0] = 0, non-decreasing; col_idx[row_ptr[n]]
 *   int32 successor ids; type[n] uint8 < n_types (<= 64);
 *   type_cost[n_types][2] int64 (CPU ns, GPU ns) used when task_cost is NULL;
 *   task_cost[n][2] int64 per-task (CPU ns, GPU ns), overrides type_cost.
 * Validation (and renumbering, see Numbering above) runs on the device;
 * errors: INSP_EINVAL, INSP_ECYCLE, INSP_EOVERFLOW, INSP_ENOMEM, INSP_ECUDA.
 * n <= 2^24 - 1.  Synchronous. */
int insp_dag_load_csr(insp_machine *m, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                      const uint8_t *type, int32_t n_types, const int64_t *type_cost, const int64_t *task_cost,
                      insp_dag **out);

/* Load ndag DAGs at once (the batched form).  Arrays are the per-DAG arrays
 * of insp_dag_load_csr concatenated:
 *   task_base[ndag+1], edge_base[ndag+1] int64 prefix sums of task and edge
 *   counts; row_ptr[task_base[ndag] + ndag]: DAG d's n_d+1 local offsets start
 *   at task_base[d] + d; col_idx[edge_base[ndag]] local successor ids;
 *   type[task_base[ndag]]; type_cost[ndag][n_types][2] (one table per DAG) or
 *   NULL when task_cost[task_base[ndag]][2] is given.
 * The first invalid DAG's error is returned.  Synchronous for the calling
 * thread, but its copies and kernels run on the batch's own non-blocking stream
 * and it waits for that stream alone: a load may run on one host thread while
 * batches of the same machine evaluate on other streams (their kernels overlap),
 * and loads and destroys of one machine may come from several threads.  Host
 * inputs in pinned memory are read by DMA (the fastest path); pageable ones are
 * staged by the CUDA driver.
 * Device memory: the inputs, predecessor lists (another m int32) and the
 * kernels' scratch; the exact ability sweep holds n_max x ceil(n_max / 64)
 * 64-bit words per concurrent DAG (n_max the largest DAG).  Its concurrency
 * shrinks to keep that under 24 GB, down to one DAG at a time (a single bitset
 * passes 24 GB beyond about 450,000 tasks); past the device's free memory the
 * load fails with INSP_ENOMEM. */
int insp_batch_load_csr(insp_machine *m, int32_t ndag, const int64_t *task_base, const int64_t *edge_base,
                        const int32_t *row_ptr, const int32_t *col_idx, const uint8_t *type, int32_t n_types,
                        const int64_t *type_cost, const int64_t *task_cost, insp_batch **out);
void insp_batch_destroy(insp_batch *b);
void insp_dag_destroy(insp_dag *d);

/* Inspiring ability and efficiency (Sec. 4.2, Sec. 4.3):
 *   ia[t] = number of strict descendants of t (the dependencies its completion
 *           eventually releases);
 *   ie[t] = number of strict descendants u whose longest path from the start
 *           of t, over GPU execution times with t's own time included, fits in
 *           the unit time T (every path from t to u takes at most T).
 * unit_time_ns <= 0 selects the DAG's default T (4 x lower median GPU cost).
 * ia, ie: int32[n] (batch: int32[task_base[ndag]] in concatenated order). */
int insp_attributes(insp_dag *d, int64_t unit_time_ns, int32_t *ia, int32_t *ie, void *stream);
/* unit_time_ns: int64[ndag] per-DAG unit times (host or device), or NULL for defaults. */
int insp_attributes_batch(insp_batch *b, const int64_t *unit_time_ns, int32_t *ia, int32_t *ie, void *stream);

/* The schedule (Sec. 2.1 push/pop, Sec. 4.4), with the machine's policy:
 *   - completions at time t are processed together; released tasks are pushed
 *     in ascending id to the worker with the earliest expected finish
 *     (max(now, busy) + queued work, data arrival incl. transfer, plus cost;
 *     ties to the lowest worker);
 *   - idle workers pop in ascending worker id; the Nready controller picks
 *     FIFO / highest IA / highest IE / local-then-highest IE (ties: lowest id);
 *   - a task starts when its worker pops it and its data has arrived.
 * Inputs ia, ie: int32 per task (from insp_attributes or the caller's own).
 * Outputs: worker int32, start int64, end int64 per task; makespan int64 per DAG. */
int insp_simulate(insp_dag *d, const int32_t *ia, const int32_t *ie, int32_t *worker, int64_t *start,
                  int64_t *end, int64_t *makespan, void *stream);
int insp_simulate_batch(insp_batch *b, const int32_t *ia, const int32_t *ie, int32_t *worker, int64_t *start,
                        int64_t *end, int64_t *makespan, void *stream);

/* The whole evaluation step: insp_attributes_batch, then insp_simulate_batch
 * with its results, in one call with the same outputs.  With device arrays the
 * step is pipelined (the batch's tuning, field groups): the DAGs are cut into
 * size groups along descending size, and the simulation of a group starts on
 * its own stream once the group's attributes are done, concurrently with the
 * attribute sweeps of the later groups.  Outputs may be device or host arrays
 * (host arrays are staged through library-owned device memory; the call then
 * synchronises `stream` and returns the first per-DAG status).  Stream-ordered
 * on `stream`.  Errors: as the two calls. */
int insp_evaluate_batch(insp_batch *b, const int64_t *unit_time_ns, int32_t *ia, int32_t *ie, int32_t *worker,
                        int64_t *start, int64_t *end, int64_t *makespan, void *stream);
/* As insp_evaluate_batch, but host output arrays must be pinned (page-locked,
 * e.g. cudaHostAlloc) and are filled asynchronously: the call returns once the
 * step and its device-to-host copies are enqueued on `stream`.  The outputs and
 * the per-DAG status (insp_batch_status) are valid after `stream` is
 * synchronised; until then the batch's staging memory is in use, so the batch
 * must not be evaluated again on another stream, and insp_batch_destroy waits
 * for it.  A serving loop overlaps one batch's copies with the next batch's
 * kernels this way.  Errors: INSP_EINVAL for a pageable host output, else as
 * insp_evaluate_batch (device-side errors show in the status). */
int insp_evaluate_batch_async(insp_batch *b, const int64_t *unit_time_ns, int32_t *ia, int32_t *ie,
                              int32_t *worker, int64_t *start, int64_t *end, int64_t *makespan, void *stream);

/* Automatic unit time per DAG (Sec. 4.3 tunes T by hand, iteratively; this
 * search replaces the hand tuning): candidates T_k = med * 2^k for
 * k = 0..k_max (med = the lower median GPU cost, so T_2 is the default;
 * saturating at 2^62); the chosen T is the smallest candidate whose IE takes at
 * least min(#distinct (topological layer, type) pairs, #distinct IA) distinct
 * values over the DAG's tasks, else T_{k_max}.  The topological layer of a
 * task is the most edges on a path reaching it from a source.  An empty DAG
 * gets T = 1.  unit_time_ns: int64[ndag] (device or host), ready to pass to
 * insp_attributes_batch / insp_evaluate_batch.  Synchronous; allocates its
 * scratch for the call.  Errors: INSP_EINVAL (k_max outside 0..62),
 * INSP_ENOMEM, INSP_ECUDA, INSP_ETIMEOUT. */
int insp_unit_time_search(insp_batch *b, int32_t k_max, int64_t *unit_time_ns, void *stream);

/* Bottom level of every task, the static priority of INSP_POLICY_DMDAP_BL:
 * HEFT's upward rank (Topcuoglu et al. 2002, cited in Sec. 2) over the
 * machine's mean costs, ids being a topological order:
 *   bl[v] = wbar(v) + max over successors s of (cbar + bl[s])  (no successor: wbar(v)),
 *   wbar(v) = floor((n_cpu * c_cpu(v) + n_gpu * c_gpu(v)) / P),
 *   cbar = floor(xfer * D / P^2), D = P^2 - n_cpu^2 - n_gpu the ordered worker
 *          pairs on distinct memory nodes (CPUs share one node, each GPU has its own).
 * bl: int64[task_base[ndag]] (device or host). */
int insp_bottom_level_batch(insp_batch *b, int64_t *bl, void *stream);

/* Push/pop trace of a simulation (the Nready time piling of Sec. 4.4
 * "Implementation details"), a tracing aid.  Device arrays of
 * task_base[ndag] entries; the k-th push and the k-th pop of DAG d sit at
 * task_base[d] + k (each DAG pushes and pops each of its tasks once):
 *   push_*: time, task (local id), chosen worker, Nready after the push;
 *   pop_*:  time, task, worker, Nready before the pop, pick mode
 *           (0 FIFO, 1 ability, 2 efficiency, 3 locality then efficiency,
 *           4 learned, 5 bottom level).
 * At one event time the pushes come before the pops. */
typedef struct {
    int64_t *push_time;
    int32_t *push_task, *push_worker, *push_nready;
    int64_t *pop_time;
    int32_t *pop_task, *pop_worker, *pop_nready, *pop_mode;
} insp_trace;
/* insp_simulate_batch that also writes the trace (device pointers only; the
 * batch's DAGs must have been loaded in a topological numbering, INSP_EINVAL
 * otherwise, and so for insp_simulate_rollout). */
int insp_simulate_trace(insp_batch *b, const int32_t *ia, const int32_t *ie, int32_t *worker, int64_t *start,
                        int64_t *end, int64_t *makespan, const insp_trace *trace, void *stream);

/* The same simulation launched once per DAG (one warp on the GPU per launch,
 * serial on `stream`): the unbatched form used as the throughput baseline. */
int insp_simulate_per_dag(insp_batch *b, const int32_t *ia, const int32_t *ie, int32_t *worker, int64_t *start,
                          int64_t *end, int64_t *makespan, void *stream);

/* Per-DAG device-side status of the last attributes / simulate call on the
 * batch (INSP_OK or INSP_ETIMEOUT), copied to the host array status[ndag].
 * Synchronises the batch's last stream.  Returns the first non-OK status. */
int insp_batch_status(insp_batch *b, int32_t *status);

/* ------------------------------------------------ learned proposal scorer
 * No counterpart in the paper: a small network that can replace the adaptive
 * priority's pick (INSP_POLICY_LEARNED), trained on rollouts of this
 * simulator.  All pointers below are device pointers (INSP_EINVAL otherwise).
 *
 * insp_scorer_eval: scores of n candidates, feat[n][16] int32 features (each
 *   clamped to [0, 255]) -> score[n] int64 in units of 1/64, with the scorer
 *   installed on m; the same network, bit for bit, as the learned pop's.  Runs
 *   asynchronously on the fifth-generation tensor cores (tcgen05 MMAs on tiles
 *   of 128 rows, accumulators in tensor memory).  Its waits for the MMAs are
 *   bounded: a row whose tile did not complete gets INSP_SCORE_TIMEOUT (no
 *   score is that low; |score| < 2^22), so check for it where that matters.
 *
 * insp_simulate_rollout: insp_simulate_batch plus rollout controls, each
 *   optional (NULL): at pop number force_pop[d] (0-based count of pops in DAG
 *   d) take task force_task[d] if it is queued on the popping worker; at pop
 *   number feat_pop[d] write the 16 features of up to feat_cap candidates of
 *   that worker's queue, oldest push first, to feat[d][feat_cap][16], their
 *   task ids to feat_task[d][feat_cap] and the count to feat_n[d].  The
 *   features are: bit lengths of IA and IE, min(255 * IE / max(IA, 1), 255),
 *   bit lengths of the CPU and GPU costs, min(16 * cpu / gpu, 255), worker is a
 *   GPU, data already local, bit length of the remaining data wait, of Nready,
 *   of the worker's queue length, the controller mode (0 FIFO, 1 ability,
 *   2 efficiency, 3 efficiency + locality) and state (0 ascending,
 *   1 descending), bit lengths of the peak, of the out-degree and of the number
 *   of pushes since the task was pushed.
 *
 * insp_scorer_train_grad: FP32 loss and gradient of an in -> h1 -> h2 -> 1
 *   network (in <= 32, h1, h2 <= 64; weights w laid out W1[in][h1], b1[h1],
 *   W2[h1][h2], b2[h2], W3[h2], b3) on n samples x[n][in] with targets[n]:
 *   loss = mean (y - target)^2.  mode 0: smooth network (h = clamp(z, 0, 255));
 *   mode 1: quantisation-aware -- the forward pass is the installed-scorer
 *   network (weights rounded to k/64 with |k| <= 128, h = min(floor(max(z,0)),
 *   255)) and gradients pass straight through the rounding and the floor.
 *   work: caller scratch of n * (2*h1 + 2*h2 + 2) floats; grad[nw], loss[1].
 *   Gradients are reduced over samples in a fixed order (deterministic).
 *
 * insp_scorer_train_grad_tc: the same loss and gradient with every matrix
 *   product on the tensor cores (BF16 mma.sync, FP32 accumulation, FP32 master
 *   weights w): each FP32 operand enters as two BF16 numbers hi + lo and each
 *   product as hi*hi + hi*lo + lo*hi, about 16 significant bits; in mode 1 the
 *   weights on the k/64 grid, integer features and floored activations are exact
 *   in BF16, so the forward pass and the loss are exact.  part: caller scratch of
 *   ceil(n / 16) * (nw + 1) floats, nw = in*h1 + h1 + h1*h2 + h2 + h2 + 1 (one
 *   partial gradient per tile of 16 samples, summed in tile order:
 *   deterministic).  Same dimension limits and errors.
 *
 * insp_adamw: one AdamW step (decoupled weight decay), step t >= 1, in place
 *   on w, m, v with gradient g.
 *
 * insp_scorer_quantize: BF16 bit patterns of clamp(round(64 w), -128, 128)/64
 *   (ties away from zero), ready for insp_set_scorer. */
int insp_scorer_eval(insp_machine *m, const int32_t *feat, int64_t n, int64_t *score, void *stream);
int insp_simulate_rollout(insp_batch *b, const int32_t *ia, const int32_t *ie, int32_t *worker, int64_t *start,
                          int64_t *end, int64_t *makespan, const int32_t *force_pop, const int32_t *force_task,
                          const int32_t *feat_pop, int32_t feat_cap, int32_t *feat_task, int32_t *feat,
                          int32_t *feat_n, void *stream);
int insp_scorer_train_grad(int32_t in, int32_t h1, int32_t h2, const float *w, int32_t mode, int64_t n,
                           const float *x, const float *target, float *work, float *grad, float *loss, void *stream);
int insp_scorer_train_grad_tc(int32_t in, int32_t h1, int32_t h2, const float *w, int32_t mode, int64_t n,
                              const float *x, const float *target, float *part, float *grad, float *loss,
                              void *stream);
int insp_adamw(int64_t nw, float *w, float *m, float *v, const float *g, int32_t t, float lr, float b1, float b2,
               float eps, float wd, void *stream);
int insp_scorer_quantize(int64_t nw, const float *w, uint16_t *bf16_out, void *stream);

/* One evaluation step as a CUDA graph.  insp_batch_record captures, on
 * `stream` (not the legacy default stream), the kernels of
 * insp_attributes_batch (default unit times) followed by insp_simulate_batch
 * with the given device outputs, and keeps the instantiated graph in the batch
 * (replacing an earlier one); it does not run the step.  insp_batch_replay
 * launches the recorded step on `stream` -- the same results as the two calls,
 * with one graph launch per step.  The output arrays must stay valid while the
 * graph is used; calls on the batch must not overlap in time.
 * Errors: INSP_EINVAL (host pointers, default stream, nothing recorded), INSP_ECUDA. */
int insp_batch_record(insp_batch *b, int32_t *ia, int32_t *ie, int32_t *worker, int64_t *start, int64_t *end,
                      int64_t *makespan, void *stream);
int insp_batch_replay(insp_batch *b, void *stream);

/* ------------------------------------------------------------- tuning
 * Launch shapes of the batched kernels and the pipelining of the evaluation
 * step, picked per batch by the library's own autotuner (no counterpart in the
 * paper).  None of them changes a result. */
typedef struct {
    int32_t groups;        /* size groups of insp_evaluate_batch (1..16; 1: all attributes, then the simulation) */
    int32_t attr_overlap;  /* 1: ability and efficiency sweeps on two streams, concurrently; 0: one after the other */
    int32_t ia_warps;      /* warps per CTA of the ability sweep (1..32) */
    int32_t ie_warps;      /* warps per CTA of the efficiency sweep (1..16) */
    int32_t ie_ring_mb;    /* device memory for the efficiency sweep's window rings, MB (1..65536); it
                              bounds the warps in flight, and rings beyond L2 spill to HBM */
    int32_t sim_warps;     /* warps (= DAGs in flight) per CTA of the simulation (1..8) */
    int32_t sim_queue;     /* ready-pool entries per warp kept in shared memory: 32, 64, 128, 256, 512 or
                              1024 (more spill to global memory); 1024 fits CTAs of at most 6 warps (5 above
                              32 workers, one less with the learned scorer): a simulation whose CTA does not
                              fit fails with INSP_EINVAL */
    int32_t group_split;   /* 0: groups of equal DAG counts; 1: geometric, each group 4x the DAGs of the
                              one before (the largest DAGs, whose simulations take longest, start first);
                              2: the first group holds one DAG per SM (the largest), the others split the
                              rest equally, so the longest simulations run beside the others' sweeps */
    int32_t ia_block;      /* ability sweep: 0: DAGs of up to 16384 tasks keep one bitset row of n bits per task
                              in one CTA (n x n bits), larger ones are cut into target blocks; 1: every DAG
                              is cut into blocks of 8192 target ids, one CTA per (DAG, block), rows in a ring
                              of (longest edge span + warps) slots per CTA, so memory does not grow with n */
} insp_tuning;

/* Time a fixed candidate set of tunings on this batch (the fastest of three
 * insp_evaluate_batch steps each after a warm-up step, CUDA events on `stream`; the library's own
 * scratch holds the outputs), in a coordinate search over the fields, keep the
 * fastest and return it in *chosen (may be NULL).  The results of later calls
 * do not depend on the tuning.  Synchronous. */
int insp_batch_autotune(insp_batch *b, void *stream, insp_tuning *chosen);
/* Set or read the tuning explicitly (set: INSP_EINVAL on out-of-range fields;
 * may allocate, INSP_ENOMEM).  insp_machine_set_tuning sets the tuning that
 * batches loaded later on the machine start with (the default is the library's
 * fixed choice), e.g. one found by insp_batch_autotune on a batch of the same
 * shape. */
int insp_batch_set_tuning(insp_batch *b, const insp_tuning *t);
int insp_batch_get_tuning(const insp_batch *b, insp_tuning *t);
int insp_machine_set_tuning(insp_machine *m, const insp_tuning *t);

/* Self-test of failure detection, no GPU fault involved: one warp waits, with
 * the library's bounded device-side wait (the one the ability sweep uses for
 * its done flags), until a device flag holding flag_value equals wait_value,
 * polling at most `limit` times.  Returns INSP_OK when the values match and
 * INSP_ETIMEOUT when the wait gave up (the context stays usable).  No
 * counterpart in the paper.  Synchronous.  Errors: INSP_EINVAL (limit < 1). */
int insp_selftest_wait(int32_t flag_value, int32_t wait_value, int32_t limit, void *stream);

/* Kernel timing, a tracing aid.  While enabled, every attributes / simulate
 * call on the batch records CUDA events on its stream around each kernel.
 * insp_batch_timing waits for them and returns the summed milliseconds and
 * launch counts since the last reset, per kernel: [0] inspiring ability,
 * [1] inspiring efficiency, [2] batched simulation, [3] per-DAG simulation
 * launches.  ms and launches may be NULL; reset != 0 clears the sums.  (Each
 * attributes call also runs one single-thread step-counter kernel, not timed.)
 * Steps replayed from a recorded graph are not timed. */
int insp_batch_set_timing(insp_batch *b, int32_t enable);
int insp_batch_timing(insp_batch *b, double *ms, int64_t *launches, int32_t reset);

/* Replace the policy a batch was loaded with (its machine's), e.g. to sweep the
 * controller parameters of Sec. 4.4 over resident DAGs without reloading them.
 * Same rules as insp_machine_create's policy; INSP_POLICY_LEARNED needs a
 * scorer installed on the batch's machine.  Later simulate / evaluate calls use
 * it (a recorded graph keeps the old one: record again).  Errors: INSP_EINVAL,
 * INSP_ENOMEM. */
int insp_batch_set_policy(insp_batch *b, const insp_policy *policy);

/* Number of distinct DAG structures (tasks and successor lists) in the batch:
 * repeated structures share one inspiring-ability sweep. */
int insp_batch_structures(const insp_batch *b, int32_t *n_distinct);

/* Batch facts: number of DAGs, total tasks, total edges. */
int insp_batch_info(const insp_batch *b, int32_t *ndag, int64_t *n_tasks, int64_t *n_edges);

/* ------------------------------------------------ no-allocation entry point
 * insp_simulate_noalloc -- the paper has no counterpart; this is a service for
 * callers that cannot allocate device memory: code running inside a framework
 * whose allocator owns all of the GPU's memory (a stray cudaMalloc may fail or
 * fragment it) and latency-critical loops that cannot afford the implicit
 * synchronisation of cudaMalloc / cudaFree.
 *
 * Same result as insp_dag_load_csr + insp_simulate on one DAG with the same
 * arguments (validation included), but it allocates nothing: its scratch is
 * a fixed array of INSP_NOALLOC_SCRATCH_BYTES reserved in every GPU that loads
 * the library, held until the process exits.  The caller passes device
 * pointers only (a host pointer gives INSP_EINVAL): row_ptr[n+1], col_idx,
 * type[n], type_cost[n_types][2] or task_cost[n][2], ia[n], ie[n] (from
 * insp_attributes or the caller's own) and the outputs worker[n], start[n],
 * end[n], makespan[1].  n above INSP_NOALLOC_MAX_TASKS gives INSP_EINVAL.
 * policy may be NULL; INSP_POLICY_LEARNED and INSP_POLICY_DMDAP_BL are not
 * accepted.
 *
 * Every array must be device memory of the current device (or managed
 * memory) at least as long as stated above, counted from the pointer to the
 * end of its allocation (checked with the driver's cuMemGetAddressRange):
 * host memory, another device's memory or a shorter array gives INSP_EINVAL
 * before any kernel runs.  A short array inside a larger allocation (e.g. a
 * caching allocator's block) passes this check; its extra elements are read.
 * The k_inc default takes the DAG's default unit time (see insp_policy).
 *
 * The first call on a device looks up the array's device address on that
 * device; make that first call before any stream capture.  Every call reuses
 * the same array (it keeps the previous call's contents and clears what must
 * start at zero), so calls whose work overlaps on the GPU -- two streams or
 * two host threads -- race and must be serialised by the caller.  Every call
 * waits for `stream` (the validation status and the final status are read
 * back) before it returns the final status. */
#define INSP_NOALLOC_MAX_TASKS 65536
#define INSP_NOALLOC_SCRATCH_BYTES 4194560
int insp_simulate_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const uint8_t *type,
                          int32_t n_types, const int64_t *type_cost, const int64_t *task_cost, int32_t n_cpu,
                          int32_t n_gpu, int64_t xfer_ns, const insp_policy *policy, const int32_t *ia,
                          const int32_t *ie, int32_t *worker, int64_t *start, int64_t *end, int64_t *makespan,
                          void *stream);

/* Thread-local description of the last error on the calling thread ("" if none). */
const char *insp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* INSPIRIT_H */
