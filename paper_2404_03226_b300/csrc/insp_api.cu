// Host runtime behind the C ABI of include/inspirit.h: object lifetimes,
// device residency of the DAGs, scratch sizing, launch configuration and
// host/device pointer staging.  All scheduling arithmetic runs in the kernels.
#include <algorithm>
#include <memory>
#include <cstdio>
#include <cstring>
#include <string>
#include <mutex>
#include <tuple>
#include <vector>

#include "kernels.h"

#define INSP_API extern "C" __attribute__((visibility("default")))

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(INSP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Device buffer owned by the library.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    int alloc(size_t n, bool *fresh = nullptr) {
        if (fresh) *fresh = false;
        if (n <= bytes && p) return INSP_OK;
        if (fresh) *fresh = true;
        release();
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(INSP_ENOMEM, "cudaMalloc(" + std::to_string(n) + " bytes): " + cudaGetErrorString(e));
        }
        bytes = n;
        return INSP_OK;
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DeviceInfo {
    int sms = 0;
    int occ_ie = 0;  // the global-memory efficiency sweep
};

// SM count and occupancy of the current device, queried once per device.
int device_info(DeviceInfo &di) {
    constexpr int MAX_DEV = 64;
    static DeviceInfo cache[MAX_DEV];
    static std::mutex mu;
    int dev = 0;
    CU(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < MAX_DEV && cache[dev].sms > 0) {
        di = cache[dev];
        return INSP_OK;
    }
    CU(cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev));
    di.occ_ie = insp::ie_occupancy();
    if (di.occ_ie < 1) return fail(INSP_ECUDA, "occupancy query failed");
    if (dev >= 0 && dev < MAX_DEV) cache[dev] = di;
    return INSP_OK;
}

constexpr int MAX_GROUPS = 16;
// The tuning a batch starts with: what the autotuner picks on the 4096-DAG layered workload
// (one group, overlapped attribute sweeps, 4-warp efficiency CTAs, 2-warp simulation CTAs with
// 32-entry pools, whole-DAG bitsets for the ability sweep), with a 16 GB ring budget for the
// efficiency sweep: enough for every resident warp up to the largest window (8192 rows, 2 MB
// per warp), where a 1 GB budget left DAGs with long edges at a tenth of the warps (tiled and
// mixed-size workloads 2.5x and 10x slower); with short windows the grid stops at occupancy.
const insp_tuning kDefaultTuning = {1, 1, 16, 4, 16384, 2, 32, 0, 0};
// Largest DAG whose inspiring ability takes whole-DAG bitset rows (n x n bits in one CTA slot)
// when the tuning's ia_block is 0; larger DAGs always take the target-block sweep.
constexpr int32_t IA_FULL_MAX = 16384;

bool tuning_ok(const insp_tuning &t) {
    return t.groups >= 1 && t.groups <= MAX_GROUPS && (t.attr_overlap == 0 || t.attr_overlap == 1) &&
           t.ia_warps >= 1 && t.ia_warps <= insp::ia_max_warps() && t.ie_warps >= 1 &&
           t.ie_warps <= insp::ie_pull_max_warps() && t.ie_ring_mb >= 1 && t.ie_ring_mb <= 65536 &&
           t.sim_warps >= 1 && t.sim_warps <= insp::sim_max_warps() &&
           (t.sim_queue == 32 || t.sim_queue == 64 || t.sim_queue == 128 || t.sim_queue == 256 ||
            t.sim_queue == 512 || t.sim_queue == 1024) &&
           (t.group_split >= 0 && t.group_split <= 2) && (t.ia_block == 0 || t.ia_block == 1);
}

// First DAG rank of size group g of G (g = G: ndag): equal DAG counts (split 0), geometric
// (1: group g holds 4x the DAGs of group g - 1), or head first (2: group 0 holds the `head`
// largest DAGs -- one per SM, whose simulations are the step's longest chains and then run
// beside the attribute sweeps of all the others -- and the rest is cut into equal groups).
int group_begin(int g, int G, int ndag, int split, int head) {
    if (g <= 0) return 0;
    if (g >= G) return ndag;
    if (split == 0) return int(int64_t(g) * ndag / G);
    if (split == 2) {
        const int h = std::min(head, ndag);
        return h + int(int64_t(g - 1) * (ndag - h) / (G - 1));
    }
    int64_t denom = 1;
    for (int k = g; k < G; ++k) denom *= 4;
    return int(int64_t(ndag) / denom);
}

}  // namespace

// Scratch of the kernels.  A batch borrows one set from its machine at load
// and hands it back when destroyed, so reloading batches through the public
// API reuses device memory instead of allocating it again.
struct Scratch {
    DBuf st_a, st_b, p_idw, p_seq, p_ia, p_ie, p_dr, p_cost, nl;  // simulation
    DBuf ia_bits, ia_done;                                         // inspiring ability, whole-DAG rows
    DBuf ia_ring, ia_flags, ia_seq;                                // inspiring ability, target blocks
    DBuf ie_rec, ie_acc;                                           // inspiring efficiency
    DBuf s_ia, s_ie, s_worker, s_start, s_end, s_makespan;         // staging of host arrays
    DBuf s_perm, s_bl;  // reordering into or out of the caller's numbering; bottom levels
    DBuf ie_ring;  // per-warp window rings of the pull efficiency sweep (global, meant to stay in L2)
    DBuf blevel;   // bottom levels (INSP_POLICY_DMDAP_BL)
    DBuf step;              // insp::StepCounters (device-side epoch and record tags)
    // streams and events of the pipelined step: q[0] runs the efficiency sweep
    // when it overlaps the ability sweep, q[1 + g] the simulation of size group g
    cudaStream_t q[1 + MAX_GROUPS] = {};
    cudaEvent_t ev_ia[MAX_GROUPS] = {}, ev_ie[MAX_GROUPS] = {}, ev_sim[MAX_GROUPS] = {}, ev_fork = nullptr;
    bool streams_ready = false;
    int make_streams() {
        if (streams_ready) return INSP_OK;
        for (auto &x : q) CU(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        for (int g = 0; g < MAX_GROUPS; ++g) {
            CU(cudaEventCreateWithFlags(&ev_ia[g], cudaEventDisableTiming));
            CU(cudaEventCreateWithFlags(&ev_ie[g], cudaEventDisableTiming));
            CU(cudaEventCreateWithFlags(&ev_sim[g], cudaEventDisableTiming));
        }
        CU(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        streams_ready = true;
        return INSP_OK;
    }
    ~Scratch() {
        for (auto x : q)
            if (x) cudaStreamDestroy(x);
        for (int g = 0; g < MAX_GROUPS; ++g) {
            if (ev_ia[g]) cudaEventDestroy(ev_ia[g]);
            if (ev_ie[g]) cudaEventDestroy(ev_ie[g]);
            if (ev_sim[g]) cudaEventDestroy(ev_sim[g]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
    }
};

// Device copies of a batch's inputs and what the load derives from them.  A batch borrows
// one set from its machine at load and hands it back when destroyed (like Scratch), so
// loading batch after batch reuses the allocations instead of paying cudaMalloc / cudaFree.
struct BatchBufs {
    DBuf task_base, edge_base, row_ptr, col_idx, type, type_cost, task_cost;
    DBuf indeg0, unit_time_def, unit_time_user, order, item_base, status, max_span, counters, dag_span;
    DBuf pr_ptr, pcol, cursor;
    // DAGs renumbered at load: old_of_new[task_base[d] + p] = the caller's id of task p (identity
    // for the DAGs that kept their numbering)
    DBuf old_of_new;
    DBuf item_dag, item_dag_lpt, item_base_lpt;
    // inspiring-ability plan: DAGs of the whole-row sweep, work items and zeroed DAGs of the
    // target-block sweep, {dag, representative} pairs of repeated structures; fingerprints
    DBuf ia_small_order, ia_items, ia_blk_dags, ia_pairs, dag_hash;
    // The load's own non-blocking stream: a load orders its copies and kernels on it and waits
    // for it alone, so it can run while other batches evaluate on other streams.
    cudaStream_t ls = nullptr;
    BatchBufs() = default;
    BatchBufs(const BatchBufs &) = delete;
    BatchBufs &operator=(const BatchBufs &) = delete;
    ~BatchBufs() {
        if (ls) cudaStreamDestroy(ls);
    }
};

struct insp_machine {
    int32_t n_cpu = 0, n_gpu = 0;
    int64_t xfer = 0;
    insp_policy pol{};
    bool has_scorer = false;
    DBuf scorer;  // insp::ScorerPacked in device memory
    std::mutex mu;  // guards the spare lists and the tuning: batches of one machine may load and die on several threads
    std::vector<std::unique_ptr<Scratch>> spare;
    std::vector<std::unique_ptr<BatchBufs>> spare_bufs;
    insp_tuning tun = kDefaultTuning;  // the tuning batches loaded on this machine start with
    // Batches loaded on this machine and not yet destroyed.  A machine destroyed while some are
    // alive (a garbage collector may finalise the handles in any order) is only marked; the last
    // of its batches frees it.
    int64_t live_batches = 0;
    bool destroyed = false;
};

enum { TK_IA = 0, TK_IE = 1, TK_SIM = 2, TK_SIM_SINGLE = 3, TK_N = 4 };

struct insp_batch {
    insp_machine *owner = nullptr;
    std::unique_ptr<BatchBufs> bufs;  // declared before the references into it
    insp_machine mach_params;
    const insp_machine &mach = mach_params;
    int32_t ndag = 0, n_types = 1;
    int64_t n_total = 0, m_total = 0;
    std::vector<int64_t> h_task_base, h_edge_base;
    std::vector<int32_t> h_order;  // DAGs by descending size
    DBuf &task_base = bufs->task_base, &edge_base = bufs->edge_base, &row_ptr = bufs->row_ptr,
         &col_idx = bufs->col_idx, &type = bufs->type, &type_cost = bufs->type_cost, &task_cost = bufs->task_cost;
    DBuf &indeg0 = bufs->indeg0, &unit_time_def = bufs->unit_time_def, &unit_time_user = bufs->unit_time_user,
         &order = bufs->order, &item_base = bufs->item_base, &status = bufs->status, &max_span = bufs->max_span,
         &counters = bufs->counters, &dag_span = bufs->dag_span;  // longest edge span per DAG
    DBuf &pr_ptr = bufs->pr_ptr, &pcol = bufs->pcol;  // predecessor lists (pull form of the efficiency sweep)
    bool pull = false;      // predecessor lists built: the pull sweep is used (window ring W <= IE_PULL_MAX_W)
    int grid_ie_pull = 0;   // its grid for the current tuning
    DBuf &item_dag = bufs->item_dag;  // DAG of every 32-source work item (items numbered by DAG id)
    // the pull sweep's items numbered along the size order
    DBuf &item_dag_lpt = bufs->item_dag_lpt, &item_base_lpt = bufs->item_base_lpt;
    std::vector<int64_t> h_rank_item;  // first item (size-order numbering) of the DAG at each rank
    bool has_task_cost = false;
    bool renumbered = false;  // some DAG was renumbered at load: per-task arrays are reordered
    int32_t max_n = 0, max_span_h = 0, W = 1;
    int64_t max_unit_def = 1, n_items = 0;  // 32-source items (global efficiency sweep)
    // per-DAG unit times of the last attributes call (device; the defaults before any): the
    // simulation's default ascending slope k_inc is P tasks per this T
    const int64_t *ut_attr = nullptr;
    int64_t n_items_pull = 0;                 // IE_PULL_SOURCES-source items (pull sweep)
    std::unique_ptr<Scratch> sc;
    int64_t ie_rec_stride = 0;
    // tuning and the launch shapes derived from it
    insp_tuning tun = kDefaultTuning;
    int64_t ia_slot = 1;  // 64-bit bitset words per CTA slot of the ability sweep
    int grid_ia = 0;
    // The inspiring-ability plan (build_ia_plan).  IA depends only on a DAG's structure, so DAGs
    // whose tasks and successor lists equal an earlier DAG's (found at load by fingerprint, then
    // compared exactly) take their representative's IA.  Representatives of up to IA_FULL_MAX
    // tasks take the whole-row sweep unless the tuning asks for target blocks; the rest are cut
    // into target blocks.  Per size rank r, prefix counts of the entries of each list.
    std::vector<int32_t> h_ia_rep, h_dag_span;
    bool ia_dups = false;
    std::vector<int32_t> h_rank_small, h_rank_blk, h_rank_blkdag;
    int32_t ia_n_pairs = 0, ia_small_max_n = 0, ia_blk_max_span = 0;
    int32_t ia_ring_rows = 0;  // ring slots per CTA of the target-block sweep
    int grid_ia_blk = 0;
    bool ie_global_ready = false;
    int grid_ie = 1;
    cudaStream_t last_stream = nullptr;
    // kernel timing (tracing aid)
    bool timing = false;
    struct Pending { int kind; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    double ms[TK_N] = {0, 0, 0, 0};
    int64_t launches[TK_N] = {0, 0, 0, 0};
    cudaGraphExec_t graph = nullptr;  // recorded evaluation step (insp_batch_record)

    explicit insp_batch(std::unique_ptr<BatchBufs> bb) : bufs(std::move(bb)) {}
    insp_batch(const insp_batch &) = delete;
    insp_batch &operator=(const insp_batch &) = delete;

    ~insp_batch() {
        if (graph) cudaGraphExecDestroy(graph);
        for (auto &p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        if (!owner) return;
        bool last = false;
        {
            std::lock_guard<std::mutex> lk(owner->mu);
            if (!owner->destroyed) {
                if (sc && owner->spare.size() < 2) owner->spare.push_back(std::move(sc));
                if (bufs && owner->spare_bufs.size() < 2) owner->spare_bufs.push_back(std::move(bufs));
            }
            last = --owner->live_batches == 0 && owner->destroyed;
        }
        if (last) delete owner;  // its destroy call came first
    }

    insp::DevBatch dev() const {
        insp::DevBatch B;
        B.ndag = ndag;
        B.n_types = n_types;
        B.task_base = task_base.as<int64_t>();
        B.edge_base = edge_base.as<int64_t>();
        B.row_ptr = row_ptr.as<int32_t>();
        B.col_idx = col_idx.as<int32_t>();
        B.type = type.as<uint8_t>();
        B.type_cost = type_cost.as<int64_t>();
        B.task_cost = has_task_cost ? task_cost.as<int64_t>() : nullptr;
        return B;
    }
};

namespace {

// Stream-ordered copy into dst (grown as needed).  A pageable host source is staged by the
// driver before the call returns; a pinned or device source must stay valid until s is synced.
int copy_in(DBuf &dst, const void *src, size_t bytes, cudaStream_t s) {
    int rc = dst.alloc(bytes);
    if (rc) return rc;
    if (bytes) CU(cudaMemcpyAsync(dst.p, src, bytes, cudaMemcpyDefault, s));
    return INSP_OK;
}

int alloc_ie_global(insp_batch *b);

// Validation statuses after the load's validation kernels: the first DAG with an error other
// than a non-topological numbering fails the load; those DAGs are renumbered instead.
int validation_status(insp_batch *b, std::vector<int32_t> &st, cudaStream_t s) {
    st.assign(std::max(b->ndag, 0), 0);
    if (b->ndag) {
        CU(cudaMemcpyAsync(st.data(), b->status.p, size_t(b->ndag) * 4, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    for (int d = 0; d < b->ndag; ++d)
        if (st[d] != INSP_OK && st[d] != INSP_ENOTTOPO)
            return fail(st[d], "DAG validation failed: DAG " + std::to_string(d) + ": device-side error");
    return INSP_OK;
}

void swap_buf(DBuf &a, DBuf &c) {
    std::swap(a.p, c.p);
    std::swap(a.bytes, c.bytes);
}

// Renumber the listed DAGs (ids not topological) on the device: Kahn rounds, then new row
// offsets, mapped and sorted successor rows, types and per-task costs in new arrays that
// replace the batch's; old_of_new keeps the caller's ids.  A cycle fails with INSP_ECYCLE.
int renumber_dags(insp_batch *b, const std::vector<int32_t> &dags, cudaStream_t s) {
    const int64_t N = std::max<int64_t>(b->n_total, 1);
    const int32_t k = int32_t(dags.size());
    DBuf list, cnt, level, qa, qb, nlev, new_of_old, rp2, col2, type2, cost2;
    int rc;
    if ((rc = copy_in(list, dags.data(), dags.size() * 4, s)) || (rc = cnt.alloc(N * 4)) ||
        (rc = level.alloc(N * 4)) || (rc = qa.alloc(N * 4)) || (rc = qb.alloc(N * 4)) || (rc = nlev.alloc(k * 4)) ||
        (rc = new_of_old.alloc(N * 4)) || (rc = b->bufs->old_of_new.alloc(N * 4)))
        return rc;
    insp::DevBatch B = b->dev();
    insp::launch_local_iota(b->task_base.as<int64_t>(), b->ndag, b->bufs->old_of_new.as<int32_t>(), s);
    insp::launch_kahn(B, list.as<int32_t>(), k, b->indeg0.as<int32_t>(), cnt.as<int32_t>(), level.as<int32_t>(),
                      qa.as<int32_t>(), qb.as<int32_t>(), nlev.as<int32_t>(), new_of_old.as<int32_t>(),
                      b->bufs->old_of_new.as<int32_t>(), b->status.as<int32_t>(), s);
    CU(cudaGetLastError());
    std::vector<int32_t> st(b->ndag);
    CU(cudaMemcpyAsync(st.data(), b->status.p, size_t(b->ndag) * 4, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (int32_t d : dags)
        if (st[d] != INSP_OK)
            return fail(INSP_ECYCLE, "DAG " + std::to_string(d) + " has a cycle: no topological numbering exists");
    const size_t rp_bytes = size_t(b->n_total + b->ndag) * 4, col_bytes = size_t(b->m_total) * 4;
    if ((rc = rp2.alloc(rp_bytes)) || (rc = col2.alloc(col_bytes)) || (rc = type2.alloc(size_t(b->n_total))) ||
        (b->has_task_cost && (rc = cost2.alloc(size_t(b->n_total) * 16))))
        return rc;
    if (rp_bytes) CU(cudaMemcpyAsync(rp2.p, b->row_ptr.p, rp_bytes, cudaMemcpyDeviceToDevice, s));
    if (col_bytes) CU(cudaMemcpyAsync(col2.p, b->col_idx.p, col_bytes, cudaMemcpyDeviceToDevice, s));
    if (b->n_total) CU(cudaMemcpyAsync(type2.p, b->type.p, size_t(b->n_total), cudaMemcpyDeviceToDevice, s));
    if (b->has_task_cost && b->n_total)
        CU(cudaMemcpyAsync(cost2.p, b->task_cost.p, size_t(b->n_total) * 16, cudaMemcpyDeviceToDevice, s));
    insp::launch_renumber(B, list.as<int32_t>(), k, b->bufs->old_of_new.as<int32_t>(), new_of_old.as<int32_t>(),
                          rp2.as<int32_t>(), col2.as<int32_t>(), type2.as<uint8_t>(),
                          b->has_task_cost ? cost2.as<int64_t>() : nullptr, b->status.as<int32_t>(), s);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(s));
    swap_buf(b->row_ptr, rp2);
    swap_buf(b->col_idx, col2);
    swap_buf(b->type, type2);
    if (b->has_task_cost) swap_buf(b->task_cost, cost2);
    b->renumbered = true;
    return INSP_OK;
}

// Longest edge span of every DAG (host copy) and the representative of every DAG's structure:
// DAGs with equal fingerprints, task counts and edge counts are compared exactly on the device,
// and a DAG equal to an earlier one takes that one as its representative.
int find_repeated_structures(insp_batch *b, cudaStream_t s) {
    const int32_t nd = b->ndag;
    b->h_ia_rep.resize(nd);
    b->h_dag_span.assign(nd, 0);
    for (int d = 0; d < nd; ++d) b->h_ia_rep[d] = d;
    if (nd == 0) return INSP_OK;
    DeviceInfo di;
    int rc = device_info(di);
    if (rc) return rc;
    DBuf &hash = b->bufs->dag_hash;  // fingerprints, summed by the validation pass
    std::vector<unsigned long long> h(nd);
    CU(cudaMemcpyAsync(h.data(), hash.p, size_t(nd) * 8, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(b->h_dag_span.data(), b->dag_span.p, size_t(nd) * 4, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    std::vector<int32_t> idx(nd);
    for (int d = 0; d < nd; ++d) idx[d] = d;
    auto key = [&](int d) {
        return std::make_tuple(h[d], b->h_task_base[d + 1] - b->h_task_base[d], b->h_edge_base[d + 1] - b->h_edge_base[d]);
    };
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return key(x) < key(y) || (key(x) == key(y) && x < y); });
    std::vector<int2> cand;
    for (int k = 1; k < nd; ++k) {
        int first = k;
        while (first > 0 && key(idx[first - 1]) == key(idx[k])) --first;
        if (first < k && b->h_task_base[idx[k] + 1] > b->h_task_base[idx[k]]) cand.push_back(make_int2(idx[k], idx[first]));
    }
    if (cand.empty()) return INSP_OK;
    DBuf pairs, same;
    if ((rc = copy_in(pairs, cand.data(), cand.size() * 8, s)) || (rc = same.alloc(cand.size() * 4))) return rc;
    insp::launch_dag_equal(b->dev(), pairs.as<int2>(), int32_t(cand.size()), same.as<int32_t>(), s);
    std::vector<int32_t> eq(cand.size());
    CU(cudaMemcpyAsync(eq.data(), same.p, cand.size() * 4, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (size_t k = 0; k < cand.size(); ++k)
        if (eq[k]) b->h_ia_rep[cand[k].x] = cand[k].y;
    return INSP_OK;
}

// The inspiring-ability plan for the current tuning's ia_block (see insp_batch): which
// representatives take the whole-row sweep and which the target-block sweep, the block work
// items along the size order (largest DAGs first, a DAG's last block -- the longest sweep --
// first), and the pairs whose IA is copied from their representative.  Uploaded on stream s.
int build_ia_plan(insp_batch *b, cudaStream_t s) {
    const int32_t nd = b->ndag;
    const int32_t full_max = b->tun.ia_block ? 0 : IA_FULL_MAX;
    std::vector<int32_t> small, blkdags;
    std::vector<int2> items, pairs;
    b->h_rank_small.assign(nd + 1, 0);
    b->h_rank_blk.assign(nd + 1, 0);
    b->h_rank_blkdag.assign(nd + 1, 0);
    b->ia_small_max_n = 0;
    b->ia_blk_max_span = 0;
    for (int r = 0; r < nd; ++r) {
        const int d = b->h_order[r];
        const int32_t n = int32_t(b->h_task_base[d + 1] - b->h_task_base[d]);
        if (b->h_ia_rep[d] == d && n > 0) {
            if (n <= full_max) {
                small.push_back(d);
                b->ia_small_max_n = std::max(b->ia_small_max_n, n);
            } else {
                blkdags.push_back(d);
                b->ia_blk_max_span = std::max(b->ia_blk_max_span, b->h_dag_span[d]);
                for (int32_t j = (n + insp::IA_BLK_BITS - 1) / insp::IA_BLK_BITS - 1; j >= 0; --j)
                    items.push_back(make_int2(d, j));
            }
        }
        b->h_rank_small[r + 1] = int32_t(small.size());
        b->h_rank_blk[r + 1] = int32_t(items.size());
        b->h_rank_blkdag[r + 1] = int32_t(blkdags.size());
    }
    for (int d = 0; d < nd; ++d)
        if (b->h_ia_rep[d] != d) pairs.push_back(make_int2(d, b->h_ia_rep[d]));
    b->ia_dups = !pairs.empty();
    b->ia_n_pairs = int32_t(pairs.size());
    // (an empty list still gets a small buffer; nothing is copied from it)
    auto put = [&](DBuf &dst, const void *src, size_t bytes) {
        return bytes ? copy_in(dst, src, bytes, s) : dst.alloc(16);
    };
    int rc;
    if ((rc = put(b->bufs->ia_small_order, small.data(), small.size() * 4)) ||
        (rc = put(b->bufs->ia_items, items.data(), items.size() * 8)) ||
        (rc = put(b->bufs->ia_blk_dags, blkdags.data(), blkdags.size() * 4)) ||
        (rc = put(b->bufs->ia_pairs, pairs.data(), pairs.size() * 8)))
        return rc;
    return INSP_OK;
}

// Inspiring-ability scratch for the current tuning and plan: for the whole-row sweep one bitset
// slot per CTA sized by its largest DAG (n x ceil(n/64) words); for the target-block sweep one
// ring per CTA of ring_rows x (IA_BLK_BITS / 8 + 8) bytes, ring_rows a power of two above the
// longest edge span of its DAGs plus the warps of a CTA (each wave of warps takes one task per
// warp), with its publish flags and item tags zeroed.
int alloc_ia(insp_batch *b) {
    DeviceInfo di;
    int rc = device_info(di);
    if (rc) return rc;
    const int64_t budget = int64_t(24) << 30;  // bytes of bitset scratch at most
    const int64_t n = b->ia_small_max_n;
    b->ia_slot = std::max<int64_t>(n * ((n + 63) / 64), 1);  // 64-bit words
    const int occ = std::max(1, insp::ia_occupancy(b->tun.ia_warps));
    const int64_t n_small = b->h_rank_small.empty() ? 0 : b->h_rank_small.back();
    int64_t g = std::min<int64_t>(int64_t(di.sms) * occ, std::max<int64_t>(n_small, 1));
    g = std::max<int64_t>(1, std::min(g, budget / (b->ia_slot * 8)));
    b->grid_ia = int(g);
    if ((rc = b->sc->ia_bits.alloc(size_t(g * b->ia_slot) * 8 + 16))) return rc;
    const int64_t n_items = b->h_rank_blk.empty() ? 0 : b->h_rank_blk.back();
    if (n_items == 0) {
        b->grid_ia_blk = 0;
        return INSP_OK;
    }
    int32_t rows = 1;
    while (rows < b->ia_blk_max_span + b->tun.ia_warps + 1) rows <<= 1;
    b->ia_ring_rows = rows;
    const int64_t per_cta = int64_t(rows) * (insp::IA_BLK_WORDS * 8 + 8);
    const int occ_b = std::max(1, insp::ia_blk_occupancy(b->tun.ia_warps));
    int64_t gb = std::min<int64_t>(int64_t(di.sms) * occ_b, n_items);
    gb = std::max<int64_t>(1, std::min(gb, budget / per_cta));
    b->grid_ia_blk = int(gb);
    Scratch &S = *b->sc;
    if ((rc = S.ia_ring.alloc(size_t(gb) * rows * insp::IA_BLK_WORDS * 8)) ||
        (rc = S.ia_flags.alloc(size_t(gb) * rows * 8)) || (rc = S.ia_seq.alloc(size_t(gb) * 4)))
        return rc;
    // flags of 0 never match a key (item tags start at 1); the tags restart with the flags.  No
    // sweep of this batch may run meanwhile, and the zeroing completes before the next one starts.
    if (b->last_stream) CU(cudaStreamSynchronize(b->last_stream));
    CU(cudaMemset(S.ia_flags.p, 0, size_t(gb) * rows * 8));
    CU(cudaMemset(S.ia_seq.p, 0, size_t(gb) * 4));
    CU(cudaStreamSynchronize(nullptr));
    return INSP_OK;
}

// Window rings of the pull efficiency sweep for the current tuning (L2 budget).
int alloc_pull_ring(insp_batch *b) {
    DeviceInfo di;
    int rc = device_info(di);
    if (rc) return rc;
    const int wpc = b->tun.ie_warps;
    const int occ = insp::ie_pull_occupancy(wpc, b->W);
    if (occ < 1) return fail(INSP_ECUDA, "occupancy query failed");
    const int64_t ring = insp::ie_pull_ring_bytes(b->W);
    const int64_t l2_ctas = std::max<int64_t>(1, (int64_t(b->tun.ie_ring_mb) << 20) / (ring * wpc));
    b->grid_ie_pull =
        int(std::max<int64_t>(1, std::min({int64_t(di.sms) * occ, (b->n_items_pull + wpc - 1) / wpc, l2_ctas})));
    // (the kernel writes every ring row before reading it, row W included)
    return b->sc->ie_ring.alloc(size_t(b->grid_ie_pull) * wpc * ring);
}

int alloc_scratch(insp_batch *b, cudaStream_t s) {
    DeviceInfo di;
    int rc = device_info(di);
    if (rc) return rc;
    if (!b->sc && b->owner) {
        std::lock_guard<std::mutex> lk(b->owner->mu);
        if (!b->owner->spare.empty()) {
            b->sc = std::move(b->owner->spare.back());
            b->owner->spare.pop_back();
        }
    }
    if (!b->sc) {
        b->sc.reset(new (std::nothrow) Scratch);
        if (!b->sc) return fail(INSP_ENOMEM, "host allocation");
    }
    Scratch &S = *b->sc;
    const int64_t N = std::max<int64_t>(b->n_total, 1);
    // simulation: per task release state, pool spill, released-task spill
    if ((rc = S.st_a.alloc(N * sizeof(int2))) || (rc = S.st_b.alloc(N * sizeof(longlong2))) ||
        (rc = S.p_idw.alloc(N * 4)) || (rc = S.p_seq.alloc(N * 4)) || (rc = S.p_ia.alloc(N * 4)) ||
        (rc = S.p_ie.alloc(N * 4)) || (rc = S.p_dr.alloc(N * 8)) || (rc = S.p_cost.alloc(N * 8)) ||
        (rc = S.nl.alloc(N * 4)))
        return rc;
    bool fresh = false;
    if ((rc = S.ia_done.alloc(N * 4, &fresh))) return rc;
    if (fresh) CU(cudaMemsetAsync(S.ia_done.p, 0, S.ia_done.bytes, s));
    if ((rc = S.step.alloc(sizeof(insp::StepCounters), &fresh))) return rc;
    if (fresh) {
        const insp::StepCounters c0{0, 0, 1};  // epoch 0 is never published; tag 0 marks empty records
        CU(cudaMemcpyAsync(S.step.p, &c0, sizeof(c0), cudaMemcpyHostToDevice, s));
        CU(cudaStreamSynchronize(s));  // c0 is a local
    }
    if ((rc = S.make_streams())) return rc;
    if (b->mach.pol.policy == INSP_POLICY_DMDAP_BL && (rc = S.blevel.alloc(N * 8))) return rc;
    if ((rc = alloc_ia(b))) return rc;
    // inspiring efficiency: global-memory sweep scratch unless the pull form applies
    // (allocated later if a call needs the global form)
    b->ie_rec_stride = std::max<int32_t>(b->max_n, 1);
    return b->pull ? alloc_pull_ring(b) : alloc_ie_global(b);
}

// Scratch of the global-memory inspiring-efficiency sweep: per warp one record
// per task of the largest DAG and a W x 32 ring of int64 path weights.
int alloc_ie_global(insp_batch *b) {
    DeviceInfo di;
    int rc = device_info(di);
    if (rc) return rc;
    Scratch &S = *b->sc;
    const int ie_warps_per_cta = insp::ie_threads() / 32;
    const int64_t budget = int64_t(24) << 30;
    int64_t gie = std::min<int64_t>(int64_t(di.sms) * di.occ_ie,
                                    (std::max<int64_t>(b->n_items, 1) + ie_warps_per_cta - 1) / ie_warps_per_cta);
    const int64_t per_warp = b->ie_rec_stride * 16 + int64_t(b->W) * 32 * 8;
    gie = std::max<int64_t>(1, std::min<int64_t>(gie, budget / (per_warp * ie_warps_per_cta)));
    b->grid_ie = int(gie);
    const int64_t warps = gie * ie_warps_per_cta;
    bool fresh = false;
    if ((rc = S.ie_rec.alloc(size_t(warps) * b->ie_rec_stride * 16, &fresh))) return rc;
    if (fresh) CU(cudaMemset(S.ie_rec.p, 0, S.ie_rec.bytes));
    if ((rc = S.ie_acc.alloc(size_t(warps) * b->W * 32 * 8))) return rc;
    b->ie_global_ready = true;
    return INSP_OK;
}

// Events around one kernel launch when timing is enabled.
struct TimedLaunch {
    insp_batch *b;
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr, e = nullptr;
    TimedLaunch(insp_batch *b_, int kind_, cudaStream_t s_) : b(b_), kind(kind_), s(s_) {
        if (b->timing && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&e) == cudaSuccess)
            cudaEventRecord(a, s);
    }
    ~TimedLaunch() {
        b->launches[kind] += 1;
        if (a && e) {
            cudaEventRecord(e, s);
            b->pending.push_back({kind, a, e});
        }
    }
};

// Per-task arrays cross the boundary in the caller's numbering.  Stage a caller input into a
// device buffer when it lives on the host or the batch was renumbered at load (then reorder it
// into the batch's numbering).
template <typename T>
int stage_in(insp_batch *b, DBuf &buf, const T *src, int64_t count, cudaStream_t s, const T *&dev) {
    const bool host = !is_device_ptr(src);
    if (!host && !b->renumbered) { dev = src; return INSP_OK; }
    int rc = buf.alloc(std::max<int64_t>(count, 1) * sizeof(T));
    if (rc) return rc;
    dev = buf.as<T>();
    if (!b->renumbered) {
        if (count) CU(cudaMemcpyAsync(buf.p, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
        return INSP_OK;
    }
    const T *from = src;
    if (host) {
        if ((rc = b->sc->s_perm.alloc(std::max<int64_t>(count, 1) * 8))) return rc;
        if (count) CU(cudaMemcpyAsync(b->sc->s_perm.p, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
        from = b->sc->s_perm.as<T>();
    }
    insp::launch_permute(b->task_base.as<int64_t>(), b->ndag, b->bufs->old_of_new.as<int32_t>(), from, buf.p,
                         int(sizeof(T)), false, s);
    return INSP_OK;
}

// Where the kernels write an output: the caller's array itself when it is device memory (and,
// for a per-task array, the batch kept the caller's numbering), else a staging buffer that
// finish_out delivers.
template <typename T>
int stage_out(insp_batch *b, DBuf &buf, T *dst, int64_t count, T *&dev, bool &staged, bool per_task = true) {
    if (is_device_ptr(dst) && !(per_task && b->renumbered)) { dev = dst; staged = false; return INSP_OK; }
    int rc = buf.alloc(std::max<int64_t>(count, 1) * sizeof(T));
    if (rc) return rc;
    dev = buf.as<T>();
    staged = true;
    return INSP_OK;
}

// Deliver a staged output after the kernels that write it (stream-ordered): reorder a per-task
// array into the caller's numbering, copy to the host.
template <typename T>
int finish_out(insp_batch *b, T *dst, const T *dev, int64_t count, cudaStream_t s, bool per_task = true) {
    const bool host = !is_device_ptr(dst);
    const T *src = dev;
    if (per_task && b->renumbered) {
        T *to = dst;
        if (host) {
            int rc = b->sc->s_perm.alloc(std::max<int64_t>(count, 1) * 8);
            if (rc) return rc;
            to = b->sc->s_perm.as<T>();
        }
        insp::launch_permute(b->task_base.as<int64_t>(), b->ndag, b->bufs->old_of_new.as<int32_t>(), dev, to,
                             int(sizeof(T)), true, s);
        src = to;
    }
    if (host && count) CU(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    return INSP_OK;
}

// The batch's per-DAG status words, read on stream s (after the work that wrote them).
int first_status(insp_batch *b, std::vector<int32_t> &st, cudaStream_t s) {
    st.assign(std::max(b->ndag, 0), 0);
    if (b->ndag) {
        CU(cudaMemcpyAsync(st.data(), b->status.p, size_t(b->ndag) * 4, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    for (int d = 0; d < b->ndag; ++d)
        if (st[d] != INSP_OK) {
            const char *what = st[d] == INSP_ETIMEOUT ? "a bounded device wait gave up" : "device-side error";
            return fail(st[d], "DAG " + std::to_string(d) + ": " + what);
        }
    return INSP_OK;
}

}  // namespace

namespace insp {
// Lets other translation units of the library report through insp_last_error.
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace insp

// ===================================================================== ABI
INSP_API const char *insp_last_error(void) { return g_err.c_str(); }

INSP_API int insp_machine_create(int32_t n_cpu, int32_t n_gpu, int64_t xfer_ns, const insp_policy *policy,
                                 insp_machine **out) {
    if (!out) return fail(INSP_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_cpu < 0 || n_gpu < 0 || n_cpu + n_gpu < 1 || n_cpu + n_gpu > insp::MAX_WORKERS)
        return fail(INSP_EINVAL, "need 1 <= n_cpu + n_gpu <= 64 workers");
    if (xfer_ns < 0 || xfer_ns > insp::TIME_BOUND) return fail(INSP_EINVAL, "xfer_ns out of range");
    insp_policy p{};
    if (policy) p = *policy;
    if (p.policy < INSP_POLICY_INSPIRIT || p.policy > INSP_POLICY_DMDAP_BL) return fail(INSP_EINVAL, "unknown policy");
    if (p.task_window < 0 || p.s_inc < 0 || p.s_dec < 0 || p.dec_step < 0 || p.c < 0 || p.k_inc_tasks < 0 ||
        p.k_inc_ns < 0)
        return fail(INSP_EINVAL, "policy parameters must be >= 0 (0 = default)");
    auto *m = new (std::nothrow) insp_machine;
    if (!m) return fail(INSP_ENOMEM, "host allocation");
    m->n_cpu = n_cpu;
    m->n_gpu = n_gpu;
    m->xfer = xfer_ns;
    m->pol = p;
    *out = m;
    return INSP_OK;
}

INSP_API void insp_machine_destroy(insp_machine *m) {
    if (!m) return;
    {
        std::lock_guard<std::mutex> lk(m->mu);
        if (m->live_batches > 0) {  // the last batch's destroy frees it
            m->destroyed = true;
            m->spare.clear();
            m->spare_bufs.clear();
            return;
        }
    }
    delete m;
}

INSP_API int insp_set_scorer(insp_machine *m, const uint16_t *w, size_t nbytes) {
    if (!m || !w) return fail(INSP_EINVAL, "NULL argument");
    if (nbytes != size_t(insp::MLP_NW) * 2) return fail(INSP_EINVAL, "expected 5313 BF16 weights (10626 bytes)");
    // every value must be k / 64 with integer |k| <= 128
    std::vector<float> v(insp::MLP_NW);
    for (int i = 0; i < insp::MLP_NW; ++i) {
        uint32_t bits = uint32_t(w[i]) << 16;
        float f;
        std::memcpy(&f, &bits, 4);
        const float k = f * 64.0f;
        if (!(k >= -128.0f && k <= 128.0f) || k != float(int(k)))
            return fail(INSP_EINVAL, "weight " + std::to_string(i) + " is not k/64 with |k| <= 128");
        v[i] = f;
    }
    // pack for the tensor-core tile (see mlp.cuh): transposed BF16 rows, FP32 biases
    insp::ScorerPacked P;
    std::memset(&P, 0, sizeof(P));
    const uint16_t *W1 = w, *W2 = w + insp::MLP_IN * insp::MLP_H + insp::MLP_H;
    const uint16_t *W3 = W2 + insp::MLP_H * insp::MLP_H + insp::MLP_H;
    const float *B1 = v.data() + insp::MLP_IN * insp::MLP_H;
    const float *B2 = B1 + insp::MLP_H + insp::MLP_H * insp::MLP_H;
    const float *B3 = B2 + insp::MLP_H + insp::MLP_H;
    for (int k = 0; k < insp::MLP_IN; ++k)
        for (int n = 0; n < insp::MLP_H; ++n) P.w1t[n][k] = W1[k * insp::MLP_H + n];
    for (int k = 0; k < insp::MLP_H; ++k)
        for (int n = 0; n < insp::MLP_H; ++n) P.w2t[n][k] = W2[k * insp::MLP_H + n];
    for (int k = 0; k < insp::MLP_H; ++k) P.w3t[0][k] = W3[k];
    for (int n = 0; n < insp::MLP_H; ++n) { P.b1[n] = B1[n]; P.b2[n] = B2[n]; }
    P.b3[0] = P.b3[1] = P.b3[2] = P.b3[3] = B3[0];
    int rc = m->scorer.alloc(sizeof(P));
    if (rc) return rc;
    CU(cudaMemcpy(m->scorer.p, &P, sizeof(P), cudaMemcpyHostToDevice));
    m->has_scorer = true;
    return INSP_OK;
}

INSP_API int insp_scorer_eval(insp_machine *m, const int32_t *feat, int64_t n, int64_t *score, void *stream) {
    if (!m || n < 0 || (n > 0 && (!feat || !score))) return fail(INSP_EINVAL, "bad argument");
    if (!m->has_scorer) return fail(INSP_EINVAL, "no scorer installed (insp_set_scorer)");
    if (n > 0 && (!is_device_ptr(feat) || !is_device_ptr(score))) return fail(INSP_EINVAL, "device pointers required");
    if (n == 0) return INSP_OK;
    insp::launch_scorer_eval(m->scorer.as<insp::ScorerPacked>(), feat, n, score, static_cast<cudaStream_t>(stream));
    CU(cudaGetLastError());
    return INSP_OK;
}

INSP_API int insp_scorer_train_grad(int32_t in, int32_t h1, int32_t h2, const float *w, int32_t mode, int64_t n,
                                    const float *x, const float *target, float *work, float *grad, float *loss,
                                    void *stream) {
    if (in < 1 || in > 32 || h1 < 1 || h1 > 64 || h2 < 1 || h2 > 64 || n < 1 || (mode != 0 && mode != 1))
        return fail(INSP_EINVAL, "need 1 <= in <= 32, 1 <= h1, h2 <= 64, n >= 1, mode 0 or 1");
    const void *ptrs[] = {w, x, target, work, grad, loss};
    for (const void *q : ptrs)
        if (!is_device_ptr(q)) return fail(INSP_EINVAL, "device pointers required");
    insp::launch_mlp_train_grad(in, h1, h2, w, mode, n, x, target, work, grad, loss,
                                static_cast<cudaStream_t>(stream));
    CU(cudaGetLastError());
    return INSP_OK;
}

INSP_API int insp_scorer_train_grad_tc(int32_t in, int32_t h1, int32_t h2, const float *w, int32_t mode, int64_t n,
                                       const float *x, const float *target, float *part, float *grad, float *loss,
                                       void *stream) {
    if (in < 1 || in > 32 || h1 < 1 || h1 > 64 || h2 < 1 || h2 > 64 || n < 1 || (mode != 0 && mode != 1))
        return fail(INSP_EINVAL, "need 1 <= in <= 32, 1 <= h1, h2 <= 64, n >= 1, mode 0 or 1");
    const void *ptrs[] = {w, x, target, part, grad, loss};
    for (const void *q : ptrs)
        if (!is_device_ptr(q)) return fail(INSP_EINVAL, "device pointers required");
    insp::launch_mlp_train_grad_tc(in, h1, h2, w, mode, n, x, target, part, grad, loss,
                                   static_cast<cudaStream_t>(stream));
    CU(cudaGetLastError());
    return INSP_OK;
}

INSP_API int insp_adamw(int64_t nw, float *w, float *m_, float *v, const float *g, int32_t t, float lr, float b1,
                        float b2, float eps, float wd, void *stream) {
    if (nw < 1 || t < 1) return fail(INSP_EINVAL, "need nw >= 1 and step t >= 1");
    const void *ptrs[] = {w, m_, v, g};
    for (const void *q : ptrs)
        if (!is_device_ptr(q)) return fail(INSP_EINVAL, "device pointers required");
    insp::launch_adamw(nw, w, m_, v, g, t, lr, b1, b2, eps, wd, static_cast<cudaStream_t>(stream));
    CU(cudaGetLastError());
    return INSP_OK;
}

INSP_API int insp_scorer_quantize(int64_t nw, const float *w, uint16_t *bf16_out, void *stream) {
    if (nw < 1) return fail(INSP_EINVAL, "need nw >= 1");
    if (!is_device_ptr(w) || !is_device_ptr(bf16_out)) return fail(INSP_EINVAL, "device pointers required");
    insp::launch_quantize(nw, w, bf16_out, static_cast<cudaStream_t>(stream));
    CU(cudaGetLastError());
    return INSP_OK;
}

INSP_API int insp_batch_load_csr(insp_machine *m, int32_t ndag, const int64_t *task_base, const int64_t *edge_base,
                                 const int32_t *row_ptr, const int32_t *col_idx, const uint8_t *type,
                                 int32_t n_types, const int64_t *type_cost, const int64_t *task_cost,
                                 insp_batch **out) {
    if (!out) return fail(INSP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!m) return fail(INSP_EINVAL, "machine is NULL");
    if (ndag < 0 || !task_base || !edge_base) return fail(INSP_EINVAL, "bad ndag or base arrays");
    if (n_types < 1 || n_types > 64) return fail(INSP_EINVAL, "n_types must be in 1..64");
    if (!type_cost && !task_cost) return fail(INSP_EINVAL, "need type_cost or task_cost");
    std::unique_ptr<BatchBufs> bb;
    {
        std::lock_guard<std::mutex> lk(m->mu);
        if (!m->spare_bufs.empty()) {
            bb = std::move(m->spare_bufs.back());
            m->spare_bufs.pop_back();
        }
    }
    if (!bb) {
        bb.reset(new (std::nothrow) BatchBufs);
        if (!bb) return fail(INSP_ENOMEM, "host allocation");
    }
    if (!bb->ls && cudaStreamCreateWithFlags(&bb->ls, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        bb->ls = nullptr;
        return fail(INSP_ECUDA, "creating the load stream");
    }
    cudaStream_t ls = bb->ls;
    auto *b = new (std::nothrow) insp_batch(std::move(bb));
    if (!b) return fail(INSP_ENOMEM, "host allocation");
    auto bail = [&](int rc) { delete b; return rc; };
    {
        std::lock_guard<std::mutex> lk(m->mu);
        b->owner = m;
        ++m->live_batches;
        b->tun = m->tun;
    }
    b->mach_params.n_cpu = m->n_cpu;
    b->mach_params.n_gpu = m->n_gpu;
    b->mach_params.xfer = m->xfer;
    b->mach_params.pol = m->pol;
    b->mach_params.has_scorer = m->has_scorer;
    b->ndag = ndag;
    b->n_types = n_types;
    b->h_task_base.resize(ndag + 1);
    b->h_edge_base.resize(ndag + 1);
    if (is_device_ptr(task_base) || is_device_ptr(edge_base)) {
        if (cudaMemcpyAsync(b->h_task_base.data(), task_base, (ndag + 1) * 8, cudaMemcpyDefault, ls) != cudaSuccess ||
            cudaMemcpyAsync(b->h_edge_base.data(), edge_base, (ndag + 1) * 8, cudaMemcpyDefault, ls) != cudaSuccess ||
            cudaStreamSynchronize(ls) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(INSP_ECUDA, "reading task_base / edge_base"));
        }
    } else {
        std::memcpy(b->h_task_base.data(), task_base, size_t(ndag + 1) * 8);
        std::memcpy(b->h_edge_base.data(), edge_base, size_t(ndag + 1) * 8);
    }
    if (b->h_task_base[0] != 0 || b->h_edge_base[0] != 0) return bail(fail(INSP_EINVAL, "bases must start at 0"));
    for (int d = 0; d < ndag; ++d) {
        int64_t n = b->h_task_base[d + 1] - b->h_task_base[d], e = b->h_edge_base[d + 1] - b->h_edge_base[d];
        if (n < 0 || e < 0) return bail(fail(INSP_EINVAL, "bases must be non-decreasing"));
        if (n > insp::MAX_DAG_TASKS) return bail(fail(INSP_EINVAL, "a DAG has more than 2^24-1 tasks"));
        if (e > 0x7fffffffLL) return bail(fail(INSP_EINVAL, "a DAG has more than 2^31-1 edges"));
        b->max_n = std::max<int32_t>(b->max_n, int32_t(n));
    }
    b->n_total = b->h_task_base[ndag];
    b->m_total = b->h_edge_base[ndag];
    if (b->n_total > 0 && (!row_ptr || !type)) return bail(fail(INSP_EINVAL, "row_ptr and type are required"));
    if (b->m_total > 0 && !col_idx) return bail(fail(INSP_EINVAL, "col_idx is required"));
    int rc;
    if ((rc = copy_in(b->task_base, b->h_task_base.data(), (ndag + 1) * 8, ls)) ||
        (rc = copy_in(b->edge_base, b->h_edge_base.data(), (ndag + 1) * 8, ls)) ||
        (rc = copy_in(b->row_ptr, row_ptr, (b->n_total + ndag) * 4, ls)) ||
        (rc = copy_in(b->col_idx, col_idx, b->m_total * 4, ls)) || (rc = copy_in(b->type, type, b->n_total, ls)))
        return bail(rc);
    if (type_cost) {
        if ((rc = copy_in(b->type_cost, type_cost, size_t(ndag) * n_types * 16, ls))) return bail(rc);
    } else if ((rc = b->type_cost.alloc(16))) {
        return bail(rc);
    }
    if (task_cost) {
        if ((rc = copy_in(b->task_cost, task_cost, b->n_total * 16, ls))) return bail(rc);
        b->has_task_cost = true;
    } else if (!type_cost) {
        return bail(fail(INSP_EINVAL, "need type_cost or task_cost"));
    }
    if ((rc = b->indeg0.alloc(std::max<int64_t>(b->n_total, 1) * 4)) ||
        (rc = b->unit_time_def.alloc(std::max(ndag, 1) * 8)) || (rc = b->unit_time_user.alloc(std::max(ndag, 1) * 8)) ||
        (rc = b->status.alloc(std::max(ndag, 1) * 4)) || (rc = b->max_span.alloc(4)) || (rc = b->counters.alloc(512)) ||
        (rc = b->dag_span.alloc(std::max(ndag, 1) * 4)) || (rc = b->bufs->dag_hash.alloc(std::max(ndag, 1) * 8)))
        return bail(rc);
    if (cudaMemsetAsync(b->indeg0.p, 0, std::max<int64_t>(b->n_total, 1) * 4, ls) != cudaSuccess ||
        cudaMemsetAsync(b->max_span.p, 0, 4, ls) != cudaSuccess)
        return bail(fail(INSP_ECUDA, "memset"));
    DeviceInfo di;
    if ((rc = device_info(di))) return bail(rc);
    insp::DevBatch B = b->dev();
    const int grid = std::max(1, std::min(ndag, di.sms * 8));
    if (ndag > 0) {
        insp::launch_validate(B, b->mach.xfer, b->status.as<int32_t>(), b->indeg0.as<int32_t>(),
                              b->max_span.as<int32_t>(), b->dag_span.as<int32_t>(),
                              b->bufs->dag_hash.as<unsigned long long>(), b->max_n, grid, ls);
        insp::launch_unit_time(B, b->status.as<int32_t>(), b->unit_time_def.as<int64_t>(), grid, ls);
    }
    if (cudaStreamSynchronize(ls) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return bail(fail(INSP_ECUDA, "validation kernels failed"));
    std::vector<int32_t> st;
    if ((rc = validation_status(b, st, ls))) return bail(rc);
    std::vector<int32_t> renum;
    for (int d = 0; d < ndag; ++d)
        if (st[d] == INSP_ENOTTOPO) renum.push_back(d);
    if (!renum.empty()) {
        if ((rc = renumber_dags(b, renum, ls))) return bail(rc);
        // validate the renumbered batch again: in-degrees, spans and unit times of the new ids
        B = b->dev();
        if (cudaMemsetAsync(b->indeg0.p, 0, std::max<int64_t>(b->n_total, 1) * 4, ls) != cudaSuccess ||
            cudaMemsetAsync(b->max_span.p, 0, 4, ls) != cudaSuccess)
            return bail(fail(INSP_ECUDA, "memset"));
        insp::launch_validate(B, b->mach.xfer, b->status.as<int32_t>(), b->indeg0.as<int32_t>(),
                              b->max_span.as<int32_t>(), b->dag_span.as<int32_t>(),
                              b->bufs->dag_hash.as<unsigned long long>(), b->max_n, grid, ls);
        insp::launch_unit_time(B, b->status.as<int32_t>(), b->unit_time_def.as<int64_t>(), grid, ls);
        if (cudaStreamSynchronize(ls) != cudaSuccess || cudaGetLastError() != cudaSuccess)
            return bail(fail(INSP_ECUDA, "validation kernels failed"));
        if ((rc = first_status(b, st, ls))) {
            g_err = "renumbered DAG failed validation: " + g_err;
            return bail(rc);
        }
    }
    std::vector<int64_t> ut(std::max(ndag, 1), 1);
    if (cudaMemcpyAsync(&b->max_span_h, b->max_span.p, 4, cudaMemcpyDeviceToHost, ls) != cudaSuccess ||
        (ndag && cudaMemcpyAsync(ut.data(), b->unit_time_def.p, ndag * 8, cudaMemcpyDeviceToHost, ls) != cudaSuccess) ||
        cudaStreamSynchronize(ls) != cudaSuccess)
        return bail(fail(INSP_ECUDA, "reading max span and unit times"));
    b->max_unit_def = *std::max_element(ut.begin(), ut.end());
    // window of the efficiency sweep: a power of two above every edge span
    b->W = 1;
    while (b->W <= b->max_span_h) b->W <<= 1;
    // DAG order for the persistent kernels: descending size (longest first)
    std::vector<int32_t> order(ndag);
    for (int d = 0; d < ndag; ++d) order[d] = d;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (b->h_task_base[a + 1] - b->h_task_base[a]) > (b->h_task_base[c + 1] - b->h_task_base[c]);
    });
    b->h_order = order;
    if ((rc = find_repeated_structures(b, ls))) return bail(rc);
    if ((rc = build_ia_plan(b, ls))) return bail(rc);
    std::vector<int64_t> items(ndag + 1, 0);
    for (int d = 0; d < ndag; ++d) items[d + 1] = items[d] + (b->h_task_base[d + 1] - b->h_task_base[d] + 31) / 32;
    b->n_items = items[ndag];
    std::vector<int32_t> idag(std::max<int64_t>(b->n_items, 1));
    for (int d = 0; d < ndag; ++d)
        for (int64_t k = items[d]; k < items[d + 1]; ++k) idag[k] = d;
    // the pull sweep's items (IE_PULL_SOURCES sources each) numbered along the size order: a
    // size group's items are a contiguous range
    b->h_rank_item.assign(ndag + 1, 0);
    std::vector<int64_t> base_lpt(std::max(ndag, 1), 0);
    for (int r = 0; r < ndag; ++r) {
        const int d = order[r];
        const int64_t nd = b->h_task_base[d + 1] - b->h_task_base[d];
        base_lpt[d] = b->h_rank_item[r];
        b->h_rank_item[r + 1] = b->h_rank_item[r] + (nd + insp::IE_PULL_SOURCES - 1) / insp::IE_PULL_SOURCES;
    }
    b->n_items_pull = b->h_rank_item[ndag];
    std::vector<int32_t> idag_lpt(std::max<int64_t>(b->n_items_pull, 1));
    for (int r = 0; r < ndag; ++r)
        for (int64_t k = b->h_rank_item[r]; k < b->h_rank_item[r + 1]; ++k) idag_lpt[k] = order[r];
    if ((rc = copy_in(b->order, order.data(), size_t(std::max(ndag, 1)) * 4, ls)) ||
        (rc = copy_in(b->item_base, items.data(), size_t(ndag + 1) * 8, ls)) ||
        (rc = copy_in(b->item_dag, idag.data(), idag.size() * 4, ls)) ||
        (rc = copy_in(b->item_base_lpt, base_lpt.data(), base_lpt.size() * 8, ls)) ||
        (rc = copy_in(b->item_dag_lpt, idag_lpt.data(), idag_lpt.size() * 4, ls)))
        return bail(rc);
    // pull form of the efficiency sweep when its window is at most IE_PULL_MAX_W
    if (b->W <= insp::IE_PULL_MAX_W && ndag > 0) {
        DBuf &cursor = b->bufs->cursor;
        if ((rc = b->pr_ptr.alloc((b->n_total + ndag) * 4)) || (rc = b->pcol.alloc(std::max<int64_t>(b->m_total, 1) * 4)) ||
            (rc = cursor.alloc(std::max<int64_t>(b->n_total, 1) * 4)))
            return bail(rc);
        insp::launch_reverse_csr(B, b->indeg0.as<int32_t>(), b->pr_ptr.as<int32_t>(), cursor.as<int32_t>(),
                                 b->pcol.as<int32_t>(), b->max_n, grid, ls);
        b->pull = true;
    }
    if ((rc = alloc_scratch(b, ls))) return bail(rc);
    // the host vectors above were staged by the driver; the device-side work of the load ends here
    if (cudaStreamSynchronize(ls) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return bail(fail(INSP_ECUDA, "building predecessor lists failed"));
    *out = b;
    return INSP_OK;
}

INSP_API int insp_dag_load_csr(insp_machine *m, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                               const uint8_t *type, int32_t n_types, const int64_t *type_cost,
                               const int64_t *task_cost, insp_dag **out) {
    if (!out) return fail(INSP_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 0 || n > insp::MAX_DAG_TASKS) return fail(INSP_EINVAL, "n out of range");
    if (!row_ptr) return fail(INSP_EINVAL, "row_ptr is NULL");
    int32_t m_edges = 0;
    if (cudaMemcpy(&m_edges, row_ptr + n, 4, cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        return fail(INSP_ECUDA, "reading row_ptr[n]");
    }
    if (m_edges < 0) return fail(INSP_EINVAL, "row_ptr[n] < 0");
    int64_t tb[2] = {0, n}, eb[2] = {0, m_edges};
    std::vector<uint8_t> zeros;
    if (!type) {
        zeros.assign(std::max(n, 1), 0);
        type = zeros.data();
    }
    return insp_batch_load_csr(m, 1, tb, eb, row_ptr, col_idx, type, n_types, type_cost, task_cost, out);
}

INSP_API void insp_batch_destroy(insp_batch *b) {
    if (b && b->last_stream) cudaStreamSynchronize(b->last_stream);
    delete b;
}
INSP_API void insp_dag_destroy(insp_dag *d) { insp_batch_destroy(d); }

INSP_API int insp_batch_set_policy(insp_batch *b, const insp_policy *policy) {
    if (!b || !policy) return fail(INSP_EINVAL, "NULL argument");
    const insp_policy &p = *policy;
    if (p.policy < INSP_POLICY_INSPIRIT || p.policy > INSP_POLICY_DMDAP_BL) return fail(INSP_EINVAL, "unknown policy");
    if (p.task_window < 0 || p.s_inc < 0 || p.s_dec < 0 || p.dec_step < 0 || p.c < 0 || p.k_inc_tasks < 0 ||
        p.k_inc_ns < 0)
        return fail(INSP_EINVAL, "policy parameters must be >= 0 (0 = default)");
    if (p.policy == INSP_POLICY_LEARNED && !(b->owner && b->owner->has_scorer))
        return fail(INSP_EINVAL, "INSP_POLICY_LEARNED needs a scorer installed with insp_set_scorer");
    if (p.policy == INSP_POLICY_DMDAP_BL) {
        const int rc = b->sc->blevel.alloc(std::max<int64_t>(b->n_total, 1) * 8);
        if (rc) return rc;
    }
    b->mach_params.pol = p;
    b->mach_params.has_scorer = b->owner && b->owner->has_scorer;
    return INSP_OK;
}

INSP_API int insp_batch_structures(const insp_batch *b, int32_t *n_distinct) {
    if (!b || !n_distinct) return fail(INSP_EINVAL, "NULL argument");
    *n_distinct = b->ndag - b->ia_n_pairs;
    return INSP_OK;
}

INSP_API int insp_batch_info(const insp_batch *b, int32_t *ndag, int64_t *n_tasks, int64_t *n_edges) {
    if (!b) return fail(INSP_EINVAL, "batch is NULL");
    if (ndag) *ndag = b->ndag;
    if (n_tasks) *n_tasks = b->n_total;
    if (n_edges) *n_edges = b->m_total;
    return INSP_OK;
}

namespace {

// The per-DAG unit time T of the efficiency sweep: the defaults, or the
// caller's array (entries <= 0 take the default).  *wide: some T >= 2^31.
int prep_unit_time(insp_batch *b, const int64_t *unit_time_ns, cudaStream_t s, const int64_t *&ut, bool &wide) {
    ut = b->unit_time_def.as<int64_t>();
    b->ut_attr = ut;
    wide = b->max_unit_def >= 0x7fffffffLL;
    if (!unit_time_ns) return INSP_OK;
    if (is_device_ptr(unit_time_ns)) {
        CU(cudaMemcpyAsync(b->unit_time_user.p, unit_time_ns, size_t(b->ndag) * 8, cudaMemcpyDeviceToDevice, s));
        wide = true;
    } else {
        std::vector<int64_t> h(unit_time_ns, unit_time_ns + b->ndag);
        std::vector<int64_t> def(std::max(b->ndag, 1));
        bool need_def = false;
        for (auto v : h) need_def |= v <= 0;
        if (need_def && b->ndag) {
            CU(cudaMemcpyAsync(def.data(), b->unit_time_def.p, size_t(b->ndag) * 8, cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
        }
        int64_t mx = 1;
        for (int d = 0; d < b->ndag; ++d) {
            if (h[d] <= 0) h[d] = def[d];
            mx = std::max(mx, h[d]);
        }
        wide = mx >= 0x7fffffffLL;
        if (b->ndag)
            CU(cudaMemcpyAsync(b->unit_time_user.p, h.data(), size_t(b->ndag) * 8, cudaMemcpyHostToDevice, s));
        if (b->ndag) CU(cudaStreamSynchronize(s));  // h is a local vector
    }
    ut = b->unit_time_user.as<int64_t>();
    b->ut_attr = ut;
    return INSP_OK;
}

// The inspiring ability of the DAGs at ranks [r0, r1) of the size order on stream s (counters
// c_small and c_blk zeroed): the whole-row sweep over its representatives, the zeroing and the
// target-block sweep of the others, then the copies for repeated structures.  With repeated
// structures, all of it runs with the first range (r0 == 0), for every rank.
void launch_ia_ranks(insp_batch *b, int r0, int r1, int32_t *c_small, int32_t *c_blk, int32_t *d_ia,
                     cudaStream_t s) {
    if (b->ia_dups) {
        if (r0 != 0) return;
        r1 = b->ndag;
    }
    Scratch &S = *b->sc;
    insp::StepCounters *sc = S.step.as<insp::StepCounters>();
    const insp::DevBatch B = b->dev();
    const int32_t s0 = b->h_rank_small[r0], s1 = b->h_rank_small[r1];
    if (s1 > s0)
        insp::launch_ia(B, b->bufs->ia_small_order.as<int32_t>() + s0, s1 - s0, c_small, S.ia_bits.as<uint64_t>(),
                        b->ia_slot, S.ia_done.as<int32_t>(), &sc->epoch, d_ia, b->status.as<int32_t>(),
                        std::min(b->grid_ia, s1 - s0), b->tun.ia_warps, s);
    const int32_t i0 = b->h_rank_blk[r0], i1 = b->h_rank_blk[r1];
    if (i1 > i0) {
        const int32_t z0 = b->h_rank_blkdag[r0], z1 = b->h_rank_blkdag[r1];
        insp::launch_ia_zero(B, b->bufs->ia_blk_dags.as<int32_t>() + z0, z1 - z0, d_ia, s);
        insp::launch_ia_blk(B, b->bufs->ia_items.as<int2>() + i0, i1 - i0, c_blk, S.ia_ring.as<uint64_t>(),
                            S.ia_flags.as<unsigned long long>(), b->ia_ring_rows, S.ia_seq.as<uint32_t>(), d_ia,
                            b->status.as<int32_t>(), std::min(b->grid_ia_blk, i1 - i0), b->tun.ia_warps, s);
    }
    if (b->ia_dups) insp::launch_ia_copy(B, b->bufs->ia_pairs.as<int2>(), b->ia_n_pairs, d_ia, s);
}

// The attribute sweeps of the DAGs at ranks [r0, r1) of the size order: the
// ability sweep on s_ia, the efficiency sweep on s_ie (the two are
// independent).  ctr: this launch pair's two work counters (zeroed).  The
// global-memory efficiency sweep (wide unit times or long edges) only runs over
// the whole batch.
int launch_attr(insp_batch *b, int r0, int r1, int32_t *ctr, const int64_t *ut, bool pull, bool wide, int32_t *d_ia,
                int32_t *d_ie, cudaStream_t s_ia, cudaStream_t s_ie) {
    Scratch &S = *b->sc;
    insp::StepCounters *sc = S.step.as<insp::StepCounters>();
    const insp::DevBatch B = b->dev();
    const int nd = r1 - r0;
    if (nd <= 0) return INSP_OK;
    {
        TimedLaunch tl(b, TK_IA, s_ia);
        launch_ia_ranks(b, r0, r1, ctr + 0, ctr + 3, d_ia, s_ia);
    }
    {
        TimedLaunch tl(b, TK_IE, s_ie);
        if (pull) {
            const int64_t i0 = b->h_rank_item[r0], i1 = b->h_rank_item[r1];
            const int wpc = b->tun.ie_warps;
            const int grid = int(std::max<int64_t>(1, std::min<int64_t>(b->grid_ie_pull, (i1 - i0 + wpc - 1) / wpc)));
            insp::launch_ie_pull(B, b->pr_ptr.as<int32_t>(), b->pcol.as<int32_t>(), b->item_base_lpt.as<int64_t>(),
                                 b->item_dag_lpt.as<int32_t>(), i0, i1, ctr + 1, ut, b->dag_span.as<int32_t>(), b->W, S.ie_ring.as<int32_t>(),
                                 d_ie, grid, wpc, s_ie);
        } else {
            if (r0 != 0 || r1 != b->ndag) return fail(INSP_EINVAL, "internal: global efficiency sweep over a part");
            insp::launch_ie(B, b->item_base.as<int64_t>(), b->n_items, ctr + 1, ut, S.ie_rec.as<uint4>(),
                            b->ie_rec_stride, S.ie_acc.p, b->W, wide, &sc->tag_base, d_ie, b->grid_ie, s_ie);
        }
    }
    CU(cudaGetLastError());
    return INSP_OK;
}

}  // namespace

INSP_API int insp_attributes_batch(insp_batch *b, const int64_t *unit_time_ns, int32_t *ia, int32_t *ie,
                                   void *stream) {
    if (!b || !ia || !ie) return fail(INSP_EINVAL, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    b->last_stream = s;
    int rc;
    const int64_t N = b->n_total;
    int32_t *d_ia, *d_ie;
    bool st_ia, st_ie;
    Scratch &S = *b->sc;
    if ((rc = stage_out(b, S.s_ia, ia, N, d_ia, st_ia)) || (rc = stage_out(b, S.s_ie, ie, N, d_ie, st_ie))) return rc;
    const int64_t *ut;
    bool wide;
    if ((rc = prep_unit_time(b, unit_time_ns, s, ut, wide))) return rc;
    if (b->ndag == 0) return INSP_OK;
    CU(cudaMemsetAsync(b->counters.p, 0, b->counters.bytes, s));
    CU(cudaMemsetAsync(b->status.p, 0, size_t(b->ndag) * 4, s));
    const bool pull = !wide && b->pull;
    if (!pull && !b->ie_global_ready && (rc = alloc_ie_global(b))) return rc;
    insp::launch_step_begin(S.step.as<insp::StepCounters>(), b->n_items, s);
    const bool ov = b->tun.attr_overlap != 0;
    if (ov) {
        CU(cudaEventRecord(S.ev_fork, s));
        CU(cudaStreamWaitEvent(S.q[0], S.ev_fork, 0));
    }
    if ((rc = launch_attr(b, 0, b->ndag, b->counters.as<int32_t>() + 16, ut, pull, wide, d_ia, d_ie, s,
                          ov ? S.q[0] : s)))
        return rc;
    if (ov) {
        CU(cudaEventRecord(S.ev_ie[0], S.q[0]));
        CU(cudaStreamWaitEvent(s, S.ev_ie[0], 0));
    }
    CU(cudaGetLastError());
    if ((st_ia && (rc = finish_out(b, ia, d_ia, N, s))) || (st_ie && (rc = finish_out(b, ie, d_ie, N, s)))) return rc;
    if (!is_device_ptr(ia) || !is_device_ptr(ie)) {
        CU(cudaStreamSynchronize(s));
        std::vector<int32_t> st;
        return first_status(b, st, s);
    }
    return INSP_OK;
}

INSP_API int insp_attributes(insp_dag *d, int64_t unit_time_ns, int32_t *ia, int32_t *ie, void *stream) {
    if (!d) return fail(INSP_EINVAL, "dag is NULL");
    if (unit_time_ns <= 0) return insp_attributes_batch(d, nullptr, ia, ie, stream);
    std::vector<int64_t> t(std::max(d->ndag, 1), unit_time_ns);
    return insp_attributes_batch(d, t.data(), ia, ie, stream);
}

namespace {

struct Rollout {
    const int32_t *force_pop = nullptr, *force_task = nullptr, *feat_pop = nullptr;
    int32_t feat_cap = 0;
    int32_t *feat_task = nullptr, *feat = nullptr, *feat_n = nullptr;
};

// Bottom levels of every task of the batch into bl (device), counter slot 12.
int launch_blevel_all(insp_batch *b, int64_t *bl, cudaStream_t s) {
    if (b->ndag == 0) return INSP_OK;
    DeviceInfo di;
    int rc = device_info(di);
    if (rc) return rc;
    const int32_t nc = b->mach.n_cpu, ng = b->mach.n_gpu;
    const __int128 P = nc + ng;
    const __int128 D = P * P - __int128(nc) * nc - ng;  // ordered worker pairs on distinct memory nodes
    const int64_t cbar = int64_t(__int128(b->mach.xfer) * D / (P * P));
    int32_t *ctr = b->counters.as<int32_t>() + 12;
    CU(cudaMemsetAsync(ctr, 0, 4, s));
    const int grid = std::max(1, std::min(di.sms * 8, (b->ndag + 7) / 8));
    insp::launch_blevel(b->dev(), nc, ng, cbar, b->order.as<int32_t>(), ctr, bl, grid, s);
    CU(cudaGetLastError());
    return INSP_OK;
}

// Arguments of the simulation kernel over the whole batch (size order, counter 8).
void fill_sim_args(insp_batch *b, insp::SimArgs &A, const int32_t *d_ia, const int32_t *d_ie, int32_t *d_worker,
                   int64_t *d_start, int64_t *d_end, int64_t *d_mk, const Rollout &ro) {
    const bool learned = b->mach.pol.policy == INSP_POLICY_LEARNED;
    Scratch &S = *b->sc;
    A.B = b->dev();
    A.n_cpu = b->mach.n_cpu;
    A.n_gpu = b->mach.n_gpu;
    A.xfer = b->mach.xfer;
    A.policy = b->mach.pol.policy;
    A.task_window = b->mach.pol.task_window;
    A.s_inc = b->mach.pol.s_inc;
    A.s_dec = b->mach.pol.s_dec;
    A.dec_step = b->mach.pol.dec_step;
    A.c = b->mach.pol.c;
    A.k_inc_tasks = b->mach.pol.k_inc_tasks;
    A.k_inc_ns = b->mach.pol.k_inc_ns;
    A.unit_time = b->ut_attr ? b->ut_attr : b->unit_time_def.as<int64_t>();
    A.indeg0 = b->indeg0.as<int32_t>();
    A.ia = d_ia;
    A.ie = d_ie;
    A.worker = d_worker;
    A.start = d_start;
    A.end = d_end;
    A.makespan = d_mk;
    A.status = b->status.as<int32_t>();
    A.st_a = S.st_a.as<int2>();
    A.st_b = S.st_b.as<longlong2>();
    A.p_idw = S.p_idw.as<int32_t>();
    A.p_seq = S.p_seq.as<int32_t>();
    A.p_ia = S.p_ia.as<int32_t>();
    A.p_ie = S.p_ie.as<int32_t>();
    A.p_dr = S.p_dr.as<int64_t>();
    A.p_cost = S.p_cost.as<int64_t>();
    A.nl = S.nl.as<int32_t>();
    A.order = b->order.as<int32_t>();
    A.counter = b->counters.as<int32_t>() + 8;
    A.scorer = learned ? b->owner->scorer.as<insp::ScorerPacked>() : nullptr;
    A.force_pop = ro.force_pop;
    A.force_task = ro.force_task;
    A.feat_pop = ro.feat_pop;
    A.feat_cap = ro.feat_cap;
    A.feat_task = ro.feat_task;
    A.feat = ro.feat;
    A.feat_n = ro.feat_n;
    A.n_order = b->ndag;
    A.single_dag = -1;
    A.blevel = b->mach.pol.policy == INSP_POLICY_DMDAP_BL ? S.blevel.as<int64_t>() : nullptr;
}

// The batched simulation of the DAGs A.order[0, A.n_order) on stream s.
int launch_sim_part(insp_batch *b, const insp::SimArgs &A, cudaStream_t s) {
    if (A.n_order <= 0) return INSP_OK;
    TimedLaunch tl(b, TK_SIM, s);
    DeviceInfo di;
    int rc = device_info(di);
    if (rc) return rc;
    const bool learned = A.policy == INSP_POLICY_LEARNED;
    const int wpc = b->tun.sim_warps;
    const int occ = insp::sim_occupancy(learned, b->mach.n_cpu + b->mach.n_gpu, wpc, b->tun.sim_queue);
    if (occ < 1)
        return fail(INSP_EINVAL, "the simulation CTA (sim_warps x sim_queue) does not fit in shared memory");
    const int grid = std::max(1, std::min(di.sms * occ, (A.n_order + wpc - 1) / wpc));
    insp::launch_sim(A, grid, wpc, b->tun.sim_queue, s);
    CU(cudaGetLastError());
    return INSP_OK;
}

int simulate_impl(insp_batch *b, const int32_t *ia, const int32_t *ie, int32_t *worker, int64_t *start,
                  int64_t *end, int64_t *makespan, void *stream, bool per_dag, const Rollout &ro = Rollout(),
                  const insp_trace *tr = nullptr) {
    if (!b || !ia || !ie || !worker || !start || !end || !makespan) return fail(INSP_EINVAL, "NULL argument");
    const bool learned = b->mach.pol.policy == INSP_POLICY_LEARNED;
    if (learned && !(b->owner && b->owner->has_scorer))
        return fail(INSP_EINVAL, "INSP_POLICY_LEARNED needs a scorer installed with insp_set_scorer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    b->last_stream = s;
    const int64_t N = b->n_total;
    int rc;
    const int32_t *d_ia, *d_ie;
    Scratch &S = *b->sc;
    if ((rc = stage_in(b, S.s_ia, ia, N, s, d_ia)) || (rc = stage_in(b, S.s_ie, ie, N, s, d_ie))) return rc;
    int32_t *d_worker;
    int64_t *d_start, *d_end, *d_mk;
    bool sw, ss, se, sm;
    if ((rc = stage_out(b, S.s_worker, worker, N, d_worker, sw)) ||
        (rc = stage_out(b, S.s_start, start, N, d_start, ss)) || (rc = stage_out(b, S.s_end, end, N, d_end, se)) ||
        (rc = stage_out(b, S.s_makespan, makespan, b->ndag, d_mk, sm, false)))
        return rc;
    if (b->ndag > 0) {
        CU(cudaMemsetAsync(b->counters.p, 0, 64, s));
        CU(cudaMemsetAsync(b->status.p, 0, size_t(b->ndag) * 4, s));
        insp::SimArgs A{};
        fill_sim_args(b, A, d_ia, d_ie, d_worker, d_start, d_end, d_mk, ro);
        if (tr) {
            A.tr_push_time = tr->push_time;
            A.tr_push_task = tr->push_task;
            A.tr_push_worker = tr->push_worker;
            A.tr_push_nready = tr->push_nready;
            A.tr_pop_time = tr->pop_time;
            A.tr_pop_task = tr->pop_task;
            A.tr_pop_worker = tr->pop_worker;
            A.tr_pop_nready = tr->pop_nready;
            A.tr_pop_mode = tr->pop_mode;
        }
        if (A.blevel && (rc = launch_blevel_all(b, S.blevel.as<int64_t>(), s))) return rc;
        if (per_dag) {
            for (int d = 0; d < b->ndag; ++d) {
                A.single_dag = d;
                TimedLaunch tl(b, TK_SIM_SINGLE, s);
                insp::launch_sim_single(A, s);
            }
        } else if ((rc = launch_sim_part(b, A, s))) {
            return rc;
        }
        CU(cudaGetLastError());
    }
    if ((sw && (rc = finish_out(b, worker, d_worker, N, s))) || (ss && (rc = finish_out(b, start, d_start, N, s))) ||
        (se && (rc = finish_out(b, end, d_end, N, s))) ||
        (sm && (rc = finish_out(b, makespan, d_mk, b->ndag, s, false))))
        return rc;
    if (!is_device_ptr(worker) || !is_device_ptr(start) || !is_device_ptr(end) || !is_device_ptr(makespan)) {
        CU(cudaStreamSynchronize(s));
        std::vector<int32_t> st;
        return first_status(b, st, s);
    }
    return INSP_OK;
}

}  // namespace

INSP_API int insp_simulate_batch(insp_batch *b, const int32_t *ia, const int32_t *ie, int32_t *worker,
                                 int64_t *start, int64_t *end, int64_t *makespan, void *stream) {
    return simulate_impl(b, ia, ie, worker, start, end, makespan, stream, false);
}

INSP_API int insp_simulate_trace(insp_batch *b, const int32_t *ia, const int32_t *ie, int32_t *worker,
                                 int64_t *start, int64_t *end, int64_t *makespan, const insp_trace *trace,
                                 void *stream) {
    if (!b || !trace) return fail(INSP_EINVAL, "NULL argument");
    if (b->renumbered) return fail(INSP_EINVAL, "the trace needs DAGs loaded in a topological numbering");
    const void *ptrs[] = {ia, ie, worker, start, end, makespan, trace->push_time, trace->push_task,
                          trace->push_worker, trace->push_nready, trace->pop_time, trace->pop_task,
                          trace->pop_worker, trace->pop_nready, trace->pop_mode};
    if (b->ndag > 0 && b->n_total > 0)
        for (const void *q : ptrs)
            if (!is_device_ptr(q)) return fail(INSP_EINVAL, "device pointers required");
    return simulate_impl(b, ia, ie, worker, start, end, makespan, stream, false, Rollout(), trace);
}

INSP_API int insp_unit_time_search(insp_batch *b, int32_t k_max, int64_t *unit_time_ns, void *stream) {
    if (!b || !unit_time_ns) return fail(INSP_EINVAL, "NULL argument");
    if (k_max < 0 || k_max > 62) return fail(INSP_EINVAL, "k_max must be in 0..62");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    b->last_stream = s;
    const int nd = b->ndag;
    if (nd == 0) return INSP_OK;
    int rc;
    DeviceInfo di;
    if ((rc = device_info(di))) return rc;
    Scratch &S = *b->sc;
    const int64_t N = std::max<int64_t>(b->n_total, 1);
    // the DAGs' bitmap slices: n * n_types bits each (the IA and IE marks use the first n)
    std::vector<int64_t> bm_base(nd + 1, 0);
    for (int d = 0; d < nd; ++d) {
        const int64_t n = b->h_task_base[d + 1] - b->h_task_base[d];
        bm_base[d + 1] = bm_base[d] + (n * std::max(b->n_types, 1) + 31) / 32;
    }
    DBuf ia, ie, layer, bm, bmb, target, done, chosen, ut, ctr;
    if ((rc = ia.alloc(N * 4)) || (rc = ie.alloc(N * 4)) || (rc = layer.alloc(N * 4)) ||
        (rc = bm.alloc(std::max<int64_t>(bm_base[nd], 1) * 4)) || (rc = target.alloc(nd * 8)) ||
        (rc = done.alloc(nd * 4)) || (rc = chosen.alloc(nd * 8)) || (rc = ut.alloc(nd * 8)) || (rc = ctr.alloc(256)) ||
        (rc = copy_in(bmb, bm_base.data(), bm_base.size() * 8, s)))
        return rc;
    if (!b->pull && !b->ie_global_ready && (rc = alloc_ie_global(b))) return rc;
    CU(cudaMemsetAsync(done.p, 0, size_t(nd) * 4, s));
    CU(cudaMemsetAsync(ctr.p, 0, 256, s));
    CU(cudaMemsetAsync(b->status.p, 0, size_t(nd) * 4, s));
    const insp::DevBatch B = b->dev();
    insp::StepCounters *sc = S.step.as<insp::StepCounters>();
    int32_t *c = ctr.as<int32_t>();  // 0, 2: ability, 1: targets, 8 + 4k..: per candidate, 63: decided DAGs
    const int32_t *order = b->order.as<int32_t>();
    const int grid = std::max(1, std::min(di.sms * 8, (nd + 7) / 8));
    insp::launch_step_begin(sc, b->n_items, s);
    launch_ia_ranks(b, 0, nd, c + 0, c + 2, ia.as<int32_t>(), s);
    insp::launch_search_target(B, order, c + 1, ia.as<int32_t>(), layer.as<int32_t>(), bm.as<uint32_t>(),
                               bmb.as<int64_t>(), target.as<int64_t>(), grid, s);
    const int64_t max_med = std::max<int64_t>(1, b->max_unit_def / 4), cap = int64_t(1) << 62;
    for (int32_t k = 0; k <= k_max; ++k) {
        int32_t *ck = c + 8 + 4 * (k % 12);
        CU(cudaMemsetAsync(ck, 0, 16, s));
        insp::launch_search_ut(nd, k, b->unit_time_def.as<int64_t>(), done.as<int32_t>(), ut.as<int64_t>(), s);
        const int64_t t_max = max_med > (cap >> k) ? cap : max_med << k;
        const bool wide = t_max >= 0x7fffffffLL;
        insp::launch_step_begin(sc, b->n_items, s);
        if (b->pull && !wide) {
            const int wpc = b->tun.ie_warps;
            insp::launch_ie_pull(B, b->pr_ptr.as<int32_t>(), b->pcol.as<int32_t>(), b->item_base_lpt.as<int64_t>(),
                                 b->item_dag_lpt.as<int32_t>(), 0, b->n_items_pull, ck + 0, ut.as<int64_t>(),
                                 b->dag_span.as<int32_t>(), b->W, S.ie_ring.as<int32_t>(), ie.as<int32_t>(), b->grid_ie_pull, wpc, s);
        } else {
            if (!b->ie_global_ready && (rc = alloc_ie_global(b))) return rc;
            insp::launch_ie(B, b->item_base.as<int64_t>(), b->n_items, ck + 0, ut.as<int64_t>(), S.ie_rec.as<uint4>(),
                            b->ie_rec_stride, S.ie_acc.p, b->W, wide, &sc->tag_base, ie.as<int32_t>(), b->grid_ie, s);
        }
        insp::launch_search_step(B, order, ck + 1, ie.as<int32_t>(), bm.as<uint32_t>(), bmb.as<int64_t>(),
                                 target.as<int64_t>(), ut.as<int64_t>(), done.as<int32_t>(), chosen.as<int64_t>(),
                                 c + 63, grid, s);
        CU(cudaGetLastError());
        int32_t n_done = 0;
        CU(cudaMemcpyAsync(&n_done, c + 63, 4, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (n_done >= nd) break;
    }
    insp::launch_search_final(nd, k_max, b->unit_time_def.as<int64_t>(), done.as<int32_t>(), chosen.as<int64_t>(), s);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(unit_time_ns, chosen.p, size_t(nd) * 8, cudaMemcpyDefault, s));
    CU(cudaStreamSynchronize(s));
    std::vector<int32_t> st;
    return first_status(b, st, s);
}

INSP_API int insp_bottom_level_batch(insp_batch *b, int64_t *bl, void *stream) {
    if (!b || !bl) return fail(INSP_EINVAL, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    b->last_stream = s;
    int64_t *d_bl;
    bool staged;
    int rc = stage_out(b, b->sc->s_bl, bl, b->n_total, d_bl, staged);
    if (rc) return rc;
    if ((rc = launch_blevel_all(b, d_bl, s))) return rc;
    if (staged && (rc = finish_out(b, bl, d_bl, b->n_total, s))) return rc;
    if (!is_device_ptr(bl)) CU(cudaStreamSynchronize(s));
    return INSP_OK;
}

namespace {
bool is_pinned_host(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

int evaluate_impl(insp_batch *b, const int64_t *unit_time_ns, int32_t *ia, int32_t *ie, int32_t *worker,
                  int64_t *start, int64_t *end, int64_t *makespan, void *stream, bool async);
}  // namespace

INSP_API int insp_evaluate_batch(insp_batch *b, const int64_t *unit_time_ns, int32_t *ia, int32_t *ie,
                                 int32_t *worker, int64_t *start, int64_t *end, int64_t *makespan, void *stream) {
    return evaluate_impl(b, unit_time_ns, ia, ie, worker, start, end, makespan, stream, false);
}

INSP_API int insp_evaluate_batch_async(insp_batch *b, const int64_t *unit_time_ns, int32_t *ia, int32_t *ie,
                                       int32_t *worker, int64_t *start, int64_t *end, int64_t *makespan,
                                       void *stream) {
    if (!b || !ia || !ie || !worker || !start || !end || !makespan) return fail(INSP_EINVAL, "NULL argument");
    const void *outs[6] = {ia, ie, worker, start, end, makespan};
    for (const void *o : outs)
        if (!is_device_ptr(o) && !is_pinned_host(o))
            return fail(INSP_EINVAL, "insp_evaluate_batch_async needs device or pinned host outputs");
    return evaluate_impl(b, unit_time_ns, ia, ie, worker, start, end, makespan, stream, true);
}

namespace {
int evaluate_impl(insp_batch *b, const int64_t *unit_time_ns, int32_t *ia, int32_t *ie, int32_t *worker,
                  int64_t *start, int64_t *end, int64_t *makespan, void *stream, bool async) {
    if (!b || !ia || !ie || !worker || !start || !end || !makespan) return fail(INSP_EINVAL, "NULL argument");
    if (b->mach.pol.policy == INSP_POLICY_LEARNED && !(b->owner && b->owner->has_scorer))
        return fail(INSP_EINVAL, "INSP_POLICY_LEARNED needs a scorer installed with insp_set_scorer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    b->last_stream = s;
    int rc;
    Scratch &S = *b->sc;
    // host arrays are staged through the batch's scratch and copied back at the end
    const int64_t N = b->n_total;
    int32_t *d_ia, *d_ie, *d_worker;
    int64_t *d_start, *d_end, *d_mk;
    bool h[6];
    if ((rc = stage_out(b, S.s_ia, ia, N, d_ia, h[0])) || (rc = stage_out(b, S.s_ie, ie, N, d_ie, h[1])) ||
        (rc = stage_out(b, S.s_worker, worker, N, d_worker, h[2])) ||
        (rc = stage_out(b, S.s_start, start, N, d_start, h[3])) || (rc = stage_out(b, S.s_end, end, N, d_end, h[4])) ||
        (rc = stage_out(b, S.s_makespan, makespan, b->ndag, d_mk, h[5], false)))
        return rc;
    const int64_t *ut;
    bool wide;
    if ((rc = prep_unit_time(b, unit_time_ns, s, ut, wide))) return rc;
    if (b->ndag == 0) return INSP_OK;
    const bool pull = !wide && b->pull;
    if (!pull && !b->ie_global_ready && (rc = alloc_ie_global(b))) return rc;
    const int G = pull ? std::min(b->tun.groups, b->ndag) : 1;
    const bool ov = b->tun.attr_overlap != 0;
    int32_t *ctr = b->counters.as<int32_t>();
    CU(cudaMemsetAsync(b->counters.p, 0, b->counters.bytes, s));
    CU(cudaMemsetAsync(b->status.p, 0, size_t(b->ndag) * 4, s));
    insp::launch_step_begin(S.step.as<insp::StepCounters>(), b->n_items, s);
    insp::SimArgs A{};
    fill_sim_args(b, A, d_ia, d_ie, d_worker, d_start, d_end, d_mk, Rollout());
    if (A.blevel && (rc = launch_blevel_all(b, S.blevel.as<int64_t>(), s))) return rc;
    cudaStream_t s_ie = ov ? S.q[0] : s;
    if (ov) {
        CU(cudaEventRecord(S.ev_fork, s));
        CU(cudaStreamWaitEvent(S.q[0], S.ev_fork, 0));
    }
    // size groups along the size order (largest DAGs first; see group_begin): the
    // simulation of group g starts on its own stream as soon as the attributes of
    // group g are done, while the attributes of the later groups still run
    DeviceInfo di;
    if ((rc = device_info(di))) return rc;
    const int head = di.sms;
    for (int g = 0; g < G; ++g) {
        const int r0 = group_begin(g, G, b->ndag, b->tun.group_split, head);
        const int r1 = group_begin(g + 1, G, b->ndag, b->tun.group_split, head);
        int32_t *cg = ctr + 16 + 4 * g;
        if ((rc = launch_attr(b, r0, r1, cg, ut, pull, wide, d_ia, d_ie, s, s_ie))) return rc;
        A.order = b->order.as<int32_t>() + r0;
        A.n_order = r1 - r0;
        A.counter = cg + 2;
        if (G == 1) {
            if (ov) {
                CU(cudaEventRecord(S.ev_ie[0], s_ie));
                CU(cudaStreamWaitEvent(s, S.ev_ie[0], 0));
            }
            if ((rc = launch_sim_part(b, A, s))) return rc;
        } else {
            cudaStream_t qg = S.q[1 + g];
            CU(cudaEventRecord(S.ev_ia[g], s));
            CU(cudaStreamWaitEvent(qg, S.ev_ia[g], 0));
            if (ov) {
                CU(cudaEventRecord(S.ev_ie[g], s_ie));
                CU(cudaStreamWaitEvent(qg, S.ev_ie[g], 0));
            }
            if ((rc = launch_sim_part(b, A, qg))) return rc;
            CU(cudaEventRecord(S.ev_sim[g], qg));
        }
    }
    if (G > 1) {
        for (int g = 0; g < G; ++g) CU(cudaStreamWaitEvent(s, S.ev_sim[g], 0));
        if (ov) {
            CU(cudaEventRecord(S.ev_ie[0], s_ie));
            CU(cudaStreamWaitEvent(s, S.ev_ie[0], 0));
        }
    }
    CU(cudaGetLastError());
    if ((h[0] && (rc = finish_out(b, ia, d_ia, N, s))) || (h[1] && (rc = finish_out(b, ie, d_ie, N, s))) ||
        (h[2] && (rc = finish_out(b, worker, d_worker, N, s))) || (h[3] && (rc = finish_out(b, start, d_start, N, s))) ||
        (h[4] && (rc = finish_out(b, end, d_end, N, s))) || (h[5] && (rc = finish_out(b, makespan, d_mk, b->ndag, s, false))))
        return rc;
    const void *outs[6] = {ia, ie, worker, start, end, makespan};
    bool any_host = false;
    for (const void *o : outs) any_host |= !is_device_ptr(o);
    if (any_host) {
        if (async) return INSP_OK;
        CU(cudaStreamSynchronize(s));
        std::vector<int32_t> st;
        return first_status(b, st, s);
    }
    return INSP_OK;
}
}  // namespace

INSP_API int insp_simulate(insp_dag *d, const int32_t *ia, const int32_t *ie, int32_t *worker, int64_t *start,
                           int64_t *end, int64_t *makespan, void *stream) {
    return simulate_impl(d, ia, ie, worker, start, end, makespan, stream, false);
}

INSP_API int insp_simulate_rollout(insp_batch *b, const int32_t *ia, const int32_t *ie, int32_t *worker,
                                   int64_t *start, int64_t *end, int64_t *makespan, const int32_t *force_pop,
                                   const int32_t *force_task, const int32_t *feat_pop, int32_t feat_cap,
                                   int32_t *feat_task, int32_t *feat, int32_t *feat_n, void *stream) {
    if (!b) return fail(INSP_EINVAL, "batch is NULL");
    if (b->renumbered) return fail(INSP_EINVAL, "rollouts need DAGs loaded in a topological numbering");
    if ((force_pop == nullptr) != (force_task == nullptr)) return fail(INSP_EINVAL, "force_pop and force_task go together");
    if (feat_pop && (feat_cap < 1 || !feat_task || !feat || !feat_n)) return fail(INSP_EINVAL, "feature capture needs outputs");
    const void *ptrs[] = {ia, ie, worker, start, end, makespan};
    for (const void *q : ptrs)
        if (!is_device_ptr(q)) return fail(INSP_EINVAL, "device pointers required");
    const void *opt[] = {force_pop, force_task, feat_pop, feat_task, feat, feat_n};
    for (const void *q : opt)
        if (q && !is_device_ptr(q)) return fail(INSP_EINVAL, "device pointers required");
    Rollout ro;
    ro.force_pop = force_pop;
    ro.force_task = force_task;
    ro.feat_pop = feat_pop;
    ro.feat_cap = feat_pop ? feat_cap : 0;
    ro.feat_task = feat_task;
    ro.feat = feat;
    ro.feat_n = feat_n;
    return simulate_impl(b, ia, ie, worker, start, end, makespan, stream, false, ro);
}

INSP_API int insp_simulate_per_dag(insp_batch *b, const int32_t *ia, const int32_t *ie, int32_t *worker,
                                   int64_t *start, int64_t *end, int64_t *makespan, void *stream) {
    return simulate_impl(b, ia, ie, worker, start, end, makespan, stream, true);
}

INSP_API int insp_batch_status(insp_batch *b, int32_t *status) {
    if (!b) return fail(INSP_EINVAL, "batch is NULL");
    CU(cudaStreamSynchronize(b->last_stream));
    std::vector<int32_t> st;
    int rc = first_status(b, st, b->last_stream);
    if (status) std::copy(st.begin(), st.end(), status);
    return rc;
}

INSP_API int insp_batch_record(insp_batch *b, int32_t *ia, int32_t *ie, int32_t *worker, int64_t *start,
                               int64_t *end, int64_t *makespan, void *stream) {
    if (!b || !stream) return fail(INSP_EINVAL, "batch and a non-default stream are required");
    const void *ptrs[] = {ia, ie, worker, start, end, makespan};
    for (const void *q : ptrs)
        if (!is_device_ptr(q)) return fail(INSP_EINVAL, "device pointers required");
    if (b->mach.pol.policy == INSP_POLICY_LEARNED && !(b->owner && b->owner->has_scorer))
        return fail(INSP_EINVAL, "INSP_POLICY_LEARNED needs a scorer installed with insp_set_scorer");
    // scratch the step may need is allocated before recording
    if (!b->pull && !b->ie_global_ready) {
        int rc = alloc_ie_global(b);
        if (rc) return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool timing = b->timing;
    b->timing = false;
    CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    int rc = insp_evaluate_batch(b, nullptr, ia, ie, worker, start, end, makespan, stream);
    const std::string err = g_err;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    b->timing = timing;
    if (rc != INSP_OK) {
        if (g) cudaGraphDestroy(g);
        return fail(rc, "recording failed: " + err);
    }
    if (e != cudaSuccess) return fail(INSP_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return fail(INSP_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    return INSP_OK;
}

INSP_API int insp_batch_replay(insp_batch *b, void *stream) {
    if (!b || !b->graph) return fail(INSP_EINVAL, "nothing recorded on this batch (insp_batch_record)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    b->last_stream = s;
    CU(cudaGraphLaunch(b->graph, s));
    return INSP_OK;
}

INSP_API int insp_batch_set_tuning(insp_batch *b, const insp_tuning *t) {
    if (!b || !t) return fail(INSP_EINVAL, "NULL argument");
    if (!tuning_ok(*t)) return fail(INSP_EINVAL, "tuning field out of range");
    const insp_tuning old = b->tun;
    b->tun = *t;
    int rc = INSP_OK;
    if (old.ia_block != t->ia_block) rc = build_ia_plan(b, nullptr);
    if (rc == INSP_OK && (old.ia_warps != t->ia_warps || old.ia_block != t->ia_block)) rc = alloc_ia(b);
    if (rc == INSP_OK && b->pull && (old.ie_warps != t->ie_warps || old.ie_ring_mb != t->ie_ring_mb))
        rc = alloc_pull_ring(b);
    if (rc != INSP_OK) {
        // back to the old shapes: reallocate what the failed attempt may have released (the
        // old sizes fitted before); the batch stays usable with its previous tuning
        const std::string err = g_err;
        b->tun = old;
        const int r1 = build_ia_plan(b, nullptr);
        const int r2 = r1 ? r1 : alloc_ia(b);
        const int r3 = b->pull ? alloc_pull_ring(b) : INSP_OK;
        if (r2 || r3) return fail(rc, err + "; restoring the previous tuning failed too");
        g_err = err;
    }
    if (b->graph) {  // a recorded step holds the old launch shapes
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return rc;
}

INSP_API int insp_machine_set_tuning(insp_machine *m, const insp_tuning *t) {
    if (!m || !t) return fail(INSP_EINVAL, "NULL argument");
    if (!tuning_ok(*t)) return fail(INSP_EINVAL, "tuning field out of range");
    std::lock_guard<std::mutex> lk(m->mu);
    m->tun = *t;
    return INSP_OK;
}

INSP_API int insp_batch_get_tuning(const insp_batch *b, insp_tuning *t) {
    if (!b || !t) return fail(INSP_EINVAL, "NULL argument");
    *t = b->tun;
    return INSP_OK;
}

INSP_API int insp_batch_autotune(insp_batch *b, void *stream, insp_tuning *chosen) {
    if (!b) return fail(INSP_EINVAL, "batch is NULL");
    if (b->ndag == 0) {
        if (chosen) *chosen = b->tun;
        return INSP_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch &S = *b->sc;
    const int64_t N = std::max<int64_t>(b->n_total, 1);
    int rc;
    int32_t *ia, *ie, *worker;
    int64_t *start, *end, *mk;
    if ((rc = S.s_ia.alloc(N * 4)) || (rc = S.s_ie.alloc(N * 4)) || (rc = S.s_worker.alloc(N * 4)) ||
        (rc = S.s_start.alloc(N * 8)) || (rc = S.s_end.alloc(N * 8)) || (rc = S.s_makespan.alloc(b->ndag * 8)))
        return rc;
    ia = S.s_ia.as<int32_t>();
    ie = S.s_ie.as<int32_t>();
    worker = S.s_worker.as<int32_t>();
    start = S.s_start.as<int64_t>();
    end = S.s_end.as<int64_t>();
    mk = S.s_makespan.as<int64_t>();
    const bool timing = b->timing;
    b->timing = false;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    // the fastest of three evaluation steps, after a warm-up step (one step alone varies by a
    // few per cent, as much as the candidates differ)
    auto time_step = [&](float &ms) -> int {
        ms = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            CU(cudaEventRecord(e0, s));
            const int r = insp_evaluate_batch(b, nullptr, ia, ie, worker, start, end, mk, stream);
            if (r) return r;
            CU(cudaEventRecord(e1, s));
            CU(cudaEventSynchronize(e1));
            float t = 0;
            CU(cudaEventElapsedTime(&t, e0, e1));
            if (rep > 0) ms = std::min(ms, t);
        }
        return INSP_OK;
    };
    insp_tuning best = b->tun;
    // coordinate search: each stage varies some fields of the best tuning so far
    auto search = [&](const std::vector<insp_tuning> &cands) -> int {
        float best_ms = 1e30f;
        for (const insp_tuning &c : cands) {
            int r = insp_batch_set_tuning(b, &c);
            if (r == INSP_ENOMEM) continue;  // a candidate that does not fit is skipped
            if (r) return r;
            float ms = 0;
            if ((r = time_step(ms))) return r;
            if (ms < best_ms) { best_ms = ms; best = c; }
        }
        return insp_batch_set_tuning(b, &best);
    };
    std::vector<insp_tuning> c;
    // 1. simulation: DAGs per CTA and queue capacity
    for (int w : {1, 2, 4, 8})
        for (int q : {32, 64, 128, 256, 512, 1024}) {
            if (q == 1024 && w > 4) continue;  // does not fit in shared memory
            insp_tuning t = best;
            t.sim_warps = w; t.sim_queue = q;
            c.push_back(t);
        }
    rc = search(c);
    // 2. efficiency sweep: CTA size and ring budget (only the pull form has them)
    if (rc == INSP_OK && b->pull) {
        c.clear();
        for (int w : {4, 8, 16})
            for (int mb : {128, 256, 512, 1024, 4096, 16384}) {
                insp_tuning t = best;
                t.ie_warps = w; t.ie_ring_mb = mb;
                c.push_back(t);
            }
        rc = search(c);
    }
    // 3. ability sweep: CTA size, whole-DAG rows or target blocks
    if (rc == INSP_OK) {
        c.clear();
        for (int blk : {0, 1})
            for (int w : {8, 16, 32}) {
                insp_tuning t = best;
                t.ia_warps = w;
                t.ia_block = blk;
                c.push_back(t);
            }
        rc = search(c);
    }
    // 4. pipelining: size groups and concurrent attribute sweeps
    if (rc == INSP_OK) {
        c.clear();
        for (int ov : {0, 1}) {
            for (int g : {1, 2, 4, 8, 16}) {
                insp_tuning t = best;
                t.groups = g; t.attr_overlap = ov; t.group_split = 0;
                c.push_back(t);
            }
            for (int g : {2, 3, 4}) {
                insp_tuning t = best;
                t.groups = g; t.attr_overlap = ov; t.group_split = 1;
                c.push_back(t);
                t.group_split = 2;
                c.push_back(t);
            }
        }
        rc = search(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->timing = timing;
    if (rc) return rc;
    if (chosen) *chosen = b->tun;
    std::vector<int32_t> st;
    return first_status(b, st, s);
}

INSP_API int insp_selftest_wait(int32_t flag_value, int32_t wait_value, int32_t limit, void *stream) {
    if (limit < 1) return fail(INSP_EINVAL, "limit must be >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DBuf buf;
    int rc = buf.alloc(8);
    if (rc) return rc;
    int32_t *d = buf.as<int32_t>();
    const int32_t h[2] = {flag_value, -1};
    CU(cudaMemcpyAsync(d, h, 8, cudaMemcpyHostToDevice, s));
    insp::launch_wait_probe(d, wait_value, limit, d + 1, s);
    CU(cudaGetLastError());
    int32_t st = -1;
    CU(cudaMemcpyAsync(&st, d + 1, 4, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (st == INSP_ETIMEOUT) return fail(INSP_ETIMEOUT, "a bounded device-side wait gave up");
    return st == INSP_OK ? INSP_OK : fail(INSP_ECUDA, "wait probe wrote no status");
}

INSP_API int insp_batch_set_timing(insp_batch *b, int32_t enable) {
    if (!b) return fail(INSP_EINVAL, "batch is NULL");
    b->timing = enable != 0;
    return INSP_OK;
}

INSP_API int insp_batch_timing(insp_batch *b, double *ms, int64_t *launches, int32_t reset) {
    if (!b) return fail(INSP_EINVAL, "batch is NULL");
    for (auto &p : b->pending) {
        CU(cudaEventSynchronize(p.b));
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, p.a, p.b));
        b->ms[p.kind] += t;
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    b->pending.clear();
    for (int k = 0; k < TK_N; ++k) {
        if (ms) ms[k] = b->ms[k];
        if (launches) launches[k] = b->launches[k];
        if (reset) { b->ms[k] = 0; b->launches[k] = 0; }
    }
    return INSP_OK;
}
