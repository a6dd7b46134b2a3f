// insp_simulate_noalloc: the single-DAG simulation for callers that must not
// allocate device memory.
//
// Who needs it: code that runs inside a host framework which owns the GPU's
// memory (a caching allocator hands out every byte, so a stray cudaMalloc can
// fail or fragment it), and latency-critical loops where cudaMalloc/cudaFree
// would add their implicit device synchronisation.  Such callers can hand us
// their own device buffers for inputs and outputs but cannot let the library
// grab scratch of its own.
//
// How: the kernels' scratch lives in one file-scope __device__ array of a
// fixed size, reserved when the library is loaded; every GPU that loads the
// library keeps it until the process exits.  Host code cannot use the array's
// name as a device address (in host code it names a host-side stand-in), so
// the address is looked up once per device with cudaGetSymbolAddress.  All
// calls share the array: calls whose work overlaps on the GPU (two streams, or
// two threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.h"

namespace insp {
void set_last_error(const std::string &msg);  // insp_api.cu
}

#define INSP_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr int64_t NA_MAX = INSP_NOALLOC_MAX_TASKS;

// Layout of the array (every region 256-byte aligned):
//   header: task_base[2], edge_base[2], unit_time[1], status[1], max_span[1]
//   per task: indeg0, st_a, st_b, pool spill (idw, seq, ia, ie, dr, cost), released spill
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_HDR = 0;
constexpr size_t OFF_INDEG = align256(OFF_HDR + 64);
constexpr size_t OFF_STA = align256(OFF_INDEG + 4 * NA_MAX);
constexpr size_t OFF_STB = align256(OFF_STA + 8 * NA_MAX);
constexpr size_t OFF_PIDW = align256(OFF_STB + 16 * NA_MAX);
constexpr size_t OFF_PSEQ = align256(OFF_PIDW + 4 * NA_MAX);
constexpr size_t OFF_PIA = align256(OFF_PSEQ + 4 * NA_MAX);
constexpr size_t OFF_PIE = align256(OFF_PIA + 4 * NA_MAX);
constexpr size_t OFF_PDR = align256(OFF_PIE + 4 * NA_MAX);
constexpr size_t OFF_PCOST = align256(OFF_PDR + 8 * NA_MAX);
constexpr size_t OFF_NL = align256(OFF_PCOST + 8 * NA_MAX);
constexpr size_t NA_BYTES = align256(OFF_NL + 4 * NA_MAX);
static_assert(NA_BYTES == INSP_NOALLOC_SCRATCH_BYTES, "scratch size out of sync with the header");

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {

int na_fail(int code, const std::string &msg) {
    insp::set_last_error(msg);
    return code;
}

constexpr int MAX_DEV = 64;
std::mutex g_mu;
unsigned char *g_addr[MAX_DEV] = {};

// The array's device address on the current device, looked up once per device.
int scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(INSP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEV) return na_fail(INSP_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(INSP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return INSP_OK;
}

// The driver's cuMemGetAddressRange (looked up through the runtime, so the library does not
// link libcuda itself): base and size of the allocation that holds a device address.
typedef int (*AddressRangeFn)(unsigned long long *base, size_t *size, unsigned long long ptr);
AddressRangeFn address_range_fn() {
    static AddressRangeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<AddressRangeFn>(f);
        else
            cudaGetLastError();
    });
    return fn;
}

// A caller array must be device memory of the current device (or managed memory) whose
// allocation holds at least `bytes` bytes from p on.  Without a staging copy, an array on
// another GPU or a short one would otherwise reach the kernels, which would read or write
// outside it.  Returns an empty string when the array is fine, else what is wrong.
std::string check_array(const char *name, const void *p, size_t bytes) {
    if (!p) return std::string(name) + " is NULL";
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return std::string(name) + " is not a device pointer";
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return std::string(name) + " is not a device pointer (every array must be a device pointer)";
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return "cudaGetDevice failed";
    }
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return std::string(name) + " lives on device " + std::to_string(a.device) + ", not on the current device " +
               std::to_string(dev);
    AddressRangeFn fn = address_range_fn();
    unsigned long long base = 0;
    size_t size = 0;
    const unsigned long long addr = reinterpret_cast<unsigned long long>(p);
    if (!fn || fn(&base, &size, addr) != 0)
        return std::string("cannot determine the extent of ") + name + " (cuMemGetAddressRange failed)";
    if (addr < base || addr - base > size || size - (addr - base) < bytes)
        return std::string(name) + " is shorter than the " + std::to_string(bytes) + " bytes it must hold";
    return std::string();
}

#define NA_CU(call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return na_fail(INSP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

INSP_API int insp_simulate_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const uint8_t *type,
                                   int32_t n_types, const int64_t *type_cost, const int64_t *task_cost,
                                   int32_t n_cpu, int32_t n_gpu, int64_t xfer_ns, const insp_policy *policy,
                                   const int32_t *ia, const int32_t *ie, int32_t *worker, int64_t *start,
                                   int64_t *end, int64_t *makespan, void *stream) {
    if (n < 0 || n > NA_MAX)
        return na_fail(INSP_EINVAL, "n = " + std::to_string(n) + " is outside 0.." + std::to_string(NA_MAX) +
                                        " (the fixed scratch of insp_simulate_noalloc)");
    if (n_cpu < 0 || n_gpu < 0 || n_cpu + n_gpu < 1 || n_cpu + n_gpu > insp::MAX_WORKERS)
        return na_fail(INSP_EINVAL, "need 1 <= n_cpu + n_gpu <= 64 workers");
    if (xfer_ns < 0 || xfer_ns > insp::TIME_BOUND) return na_fail(INSP_EINVAL, "xfer_ns out of range");
    if (n_types < 1 || n_types > 64) return na_fail(INSP_EINVAL, "n_types must be in 1..64");
    insp_policy p{};
    if (policy) p = *policy;
    if (p.policy != INSP_POLICY_INSPIRIT && p.policy != INSP_POLICY_FIFO && p.policy != INSP_POLICY_DMDAP_IA)
        return na_fail(INSP_EINVAL, "policy must be INSP_POLICY_INSPIRIT, INSP_POLICY_FIFO or INSP_POLICY_DMDAP_IA");
    if (p.task_window < 0 || p.s_inc < 0 || p.s_dec < 0 || p.dec_step < 0 || p.c < 0 || p.k_inc_tasks < 0 ||
        p.k_inc_ns < 0)
        return na_fail(INSP_EINVAL, "policy parameters must be >= 0 (0 = default)");
    // every array must already live on the current device and be long enough: staging a host
    // array would need an allocation, and nothing else stands between a short array and the kernels
    if (!type_cost && !task_cost) return na_fail(INSP_EINVAL, "need type_cost or task_cost");
    const size_t N = size_t(n);
    struct Need { const char *name; const void *p; size_t bytes; };
    const Need need[] = {{"row_ptr", row_ptr, 4 * (N + 1)}, {"type", type, N},
                         {"ia", ia, 4 * N}, {"ie", ie, 4 * N}, {"worker", worker, 4 * N},
                         {"start", start, 8 * N}, {"end", end, 8 * N}, {"makespan", makespan, 8}};
    for (const Need &q : need) {
        if (q.bytes == 0 && q.p == nullptr) continue;
        const std::string why = check_array(q.name, q.p, q.bytes);
        if (!why.empty()) return na_fail(INSP_EINVAL, why);
    }
    {
        const std::string why = task_cost ? check_array("task_cost", task_cost, 16 * N)
                                          : check_array("type_cost", type_cost, 16 * size_t(n_types));
        if (!why.empty()) return na_fail(INSP_EINVAL, why);
    }

    unsigned char *S = nullptr;
    int rc = scratch_address(&S);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    int32_t m = 0;
    NA_CU(cudaMemcpyAsync(&m, row_ptr + n, 4, cudaMemcpyDeviceToHost, s));
    NA_CU(cudaStreamSynchronize(s));
    if (m < 0) return na_fail(INSP_EINVAL, "row_ptr[n] < 0");
    if (m > 0) {
        const std::string why = check_array("col_idx", col_idx, 4 * size_t(m));
        if (!why.empty()) return na_fail(INSP_EINVAL, why);
    }

    // header: bases of the one-DAG batch; status, span and in-degrees start at zero
    const int64_t hdr[4] = {0, n, 0, m};
    int64_t *task_base = reinterpret_cast<int64_t *>(S + OFF_HDR);
    int64_t *edge_base = task_base + 2;
    int64_t *unit_time = task_base + 4;
    int32_t *status = reinterpret_cast<int32_t *>(task_base + 5);
    int32_t *max_span = status + 1;
    NA_CU(cudaMemcpyAsync(task_base, hdr, sizeof(hdr), cudaMemcpyHostToDevice, s));
    NA_CU(cudaMemsetAsync(status, 0, 8, s));
    NA_CU(cudaMemsetAsync(S + OFF_INDEG, 0, 4 * size_t(n > 0 ? n : 1), s));

    insp::DevBatch B;
    B.ndag = 1;
    B.n_types = n_types;
    B.task_base = task_base;
    B.edge_base = edge_base;
    B.row_ptr = row_ptr;
    B.col_idx = col_idx;
    B.type = type;
    B.type_cost = type_cost;
    B.task_cost = task_cost;
    int32_t *indeg0 = reinterpret_cast<int32_t *>(S + OFF_INDEG);
    insp::launch_validate(B, xfer_ns, status, indeg0, max_span, nullptr, nullptr, n, 1, s);
    insp::launch_unit_time(B, status, unit_time, 1, s);
    int32_t st = 0;
    NA_CU(cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s));
    NA_CU(cudaStreamSynchronize(s));
    if (st != INSP_OK) return na_fail(st, "DAG validation failed");

    insp::SimArgs A{};
    A.B = B;
    A.n_cpu = n_cpu;
    A.n_gpu = n_gpu;
    A.xfer = xfer_ns;
    A.policy = p.policy;
    A.task_window = p.task_window;
    A.s_inc = p.s_inc;
    A.s_dec = p.s_dec;
    A.dec_step = p.dec_step;
    A.c = p.c;
    A.k_inc_tasks = p.k_inc_tasks;
    A.k_inc_ns = p.k_inc_ns;
    A.unit_time = unit_time;  // the default unit time: the attributes are taken to use it
    A.indeg0 = indeg0;
    A.ia = ia;
    A.ie = ie;
    A.worker = worker;
    A.start = start;
    A.end = end;
    A.makespan = makespan;
    A.status = status;
    A.st_a = reinterpret_cast<int2 *>(S + OFF_STA);
    A.st_b = reinterpret_cast<longlong2 *>(S + OFF_STB);
    A.p_idw = reinterpret_cast<int32_t *>(S + OFF_PIDW);
    A.p_seq = reinterpret_cast<int32_t *>(S + OFF_PSEQ);
    A.p_ia = reinterpret_cast<int32_t *>(S + OFF_PIA);
    A.p_ie = reinterpret_cast<int32_t *>(S + OFF_PIE);
    A.p_dr = reinterpret_cast<int64_t *>(S + OFF_PDR);
    A.p_cost = reinterpret_cast<int64_t *>(S + OFF_PCOST);
    A.nl = reinterpret_cast<int32_t *>(S + OFF_NL);
    A.order = nullptr;
    A.counter = nullptr;
    A.single_dag = 0;
    insp::launch_sim_single(A, s);
    NA_CU(cudaGetLastError());
    NA_CU(cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s));
    NA_CU(cudaStreamSynchronize(s));
    if (st == INSP_ETIMEOUT) return na_fail(st, "a bounded device-side wait gave up");
    if (st == INSP_ECHECK) return na_fail(st, "an internal bounds check of the debug build failed");
    if (st != INSP_OK) return na_fail(st, "device-side error " + std::to_string(st));
    return INSP_OK;
}
