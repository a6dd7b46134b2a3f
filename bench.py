#!/usr/bin/env python
"""Benchmark: scheduled tasks per second of the INSPIRIT schedule evaluation
(inspiring attributes + adaptive-priority list-scheduling run) on one B300.

Workload: the 4096 random layered DAGs (n ~ U[50, 2000], layer width
U[4, 64], edge probability U[0.1, 0.5] to the next U{1..3} layers, 8 task
types, log-normal per-type costs) on 8 CPU + 2 GPU workers, 20 us transfer.
A step is one pass of the whole path over the batch: inspiring ability,
inspiring efficiency, and the simulation, with the DAGs resident in HBM.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank evaluates its own 4096-DAG window (weak scaling).
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "scheduled tasks/sec on 1 B300, batched vs per-DAG form; makespan exact vs oracle"
UNIT = "tasks/s"
WORKLOAD = ("4096 random layered DAGs (n~U[50,2000], width U[4,64], p U[0.1,0.5], span U{1,2,3}, 8 types, "
            "log-normal costs) on 8 CPU + 2 GPU workers, 20 us transfer, INSPIRIT policy")


def make_workload(args, rank):
    """(batch, machine, description) of the selected workload."""
    import inputs
    if args.workload == "layered":
        # weak scaling: each rank its own 4096 DAGs (--ndag: the first K of them, for profiling captures)
        b = inputs.layered4096(ndag=args.ndag, first=rank_first_dag(rank))
        desc = WORKLOAD if args.ndag == 4096 else f"first {args.ndag} of: " + WORKLOAD
        return b, inputs.MACHINE_LAYERED, desc, "8 CPU + 2 GPU workers, xfer 20000 ns"
    if args.workload == "layered_degree":
        b = inputs.layered4096_degree(ndag=args.ndag, first=rank_first_dag(rank))
        desc = ("the same 4096 layered DAG shapes with 16 task types by in/out degree bucket (per-type log-normal "
                "costs), 8 CPU + 2 GPU workers, 20 us transfer, INSPIRIT policy")
        return b, inputs.MACHINE_LAYERED, desc, "8 CPU + 2 GPU workers, xfer 20000 ns"
    if args.workload == "tiled":
        Ns = tuple(int(x) for x in args.tiles.split(","))
        b = inputs.tiled_workload(Ns=Ns, instances=args.instances)
        desc = (f"tiled Cholesky / LU / QR DAGs at {args.tiles} tiles x {args.instances} instances each, "
                f"per-task costs perturbed +-20 % from seed, 16 CPU + 4 GPU workers, 20 us transfer, INSPIRIT policy")
        return b, inputs.MACHINE_TILED, desc, "16 CPU + 4 GPU workers, xfer 20000 ns"
    if args.workload == "mixed":
        b = inputs.mixed_workload(args.mixed_ndag, with_large=not args.no_large)
        desc = (f"mixed-size stress: {args.mixed_ndag} DAGs with task counts log-uniform in [100, 200000], random "
                f"layered (the layered workload's shape) and tiled Cholesky / LU / QR (largest tile count within the "
                f"drawn size) alternating 1:1" + ("" if args.no_large else ", plus one 1,000,000-task layered DAG "
                f"(layers of 256, edge probability 0.05, span U{{1,2,3}})") +
                ", per-task costs, 32 CPU + 8 GPU workers, 20 us transfer, INSPIRIT policy")
        return b, inputs.MACHINE_MIXED, desc, "32 CPU + 8 GPU workers, xfer 20000 ns"
    raise ValueError(args.workload)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ------------------------------------------------------------------- clocks
CLOCK_FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, device: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(device)], stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None
        self.t0 = self.t1 = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.p is not None:
            time.sleep(0.3)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sel = [r for r in rows if self.t0 is None or (self.t0 - 1 <= r[0] <= (self.t1 or r[0]) + 1)] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in sel for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        return {"sm_mhz": float(np.median([r[1] for r in sel])), "sm_max_mhz": float(max(r[2] for r in sel)),
                "reasons": reasons, "samples": len(sel)}


# ---------------------------------------------------------------- roofline
def algorithmic_bytes(batch):
    """Minimal HBM bytes per step of each kernel (all its launches): inputs read once, outputs
    written once (scratch excluded).  Costs: 1 byte of type per task with
    per-type tables, or 8 (GPU cost) / 16 (both costs) bytes with per-task costs."""
    n, m, nd = batch.n_total, batch.m_total, batch.ndag
    csr = 4 * (n + nd) + 4 * m  # row_ptr + col_idx
    per_task = batch.task_cost is not None
    c_ie = 8 * n if per_task else n
    c_sim = 16 * n if per_task else n
    return {
        "k_ia": csr + 4 * n,                                   # ia written
        "k_ie_pull": csr + c_ie + 4 * n,                            # GPU cost read, ie written
        "k_sim": csr + c_sim + 4 * n + 8 * n + 20 * n + 8 * nd,  # costs, in-degree, ia+ie read; schedule written
    }


def path_bytes(batch):
    """Algorithmic HBM bytes of one pass of the whole path over the batch, each input read once
    and each output written once: per task 4 (row_ptr) + 4 x out-degree (col_idx) + 1 (type) +
    8 (IA and IE written) + 20 (worker, start, end written), plus 16 per task of per-task costs;
    per DAG 4 (the extra row_ptr entry) + 8 (makespan) + the per-type cost table."""
    n, m, nd = batch.n_total, batch.m_total, batch.ndag
    costs = 16 * n if batch.task_cost is not None else 16 * nd * batch.n_types
    return 4 * (n + nd) + 4 * m + n + 8 * n + 20 * n + 8 * nd + costs


def profile_record(kernel: str, workload: str):
    """The counters an ncu capture recorded in profiles/ for a kernel (per-step DRAM bytes and
    warp instructions, scaled to the full workload), if they were taken on this workload and the
    kernel source has not changed since."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(kernel)
    if not rec or rec.get("workload") != workload:
        return None
    src = os.path.join(ROOT, "paper_2404_03226_b300", "csrc", rec["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec["source_sha"]:
        return None
    return rec


def traffic_from_profile(kernel: str, launches_per_step: float, workload: str):
    """dram bytes per launch from the per-step figure of the kernel's ncu record."""
    rec = profile_record(kernel, workload)
    if rec is None:
        return None
    return rec["bytes_per_step_full"] / max(launches_per_step, 1.0)


def issue_roofline(names, kms, steps, sms: int, sm_mhz: float, dom: str, workload: str):
    """Second roofline: SM instruction issue.  achieved = warp instructions per step (ncu
    smsp__inst_executed.sum of the recorded capture, scaled to the workload) over the kernel's
    measured time; peak = SMs x 4 schedulers x 1 warp instruction per cycle x the SM clock
    sampled during the timed region."""
    peak = sms * 4 * sm_mhz * 1e6 / 1e9  # G warp instructions / s
    per = {}
    for k, name in enumerate(names):
        rec = profile_record(name, workload)
        if rec is None or "inst_per_step_full" not in rec or kms[k] <= 0:
            per[name] = None
            continue
        ach = rec["inst_per_step_full"] * steps / (kms[k] / 1e3) / 1e9
        per[name] = {"achieved": round(ach, 1), "frac": round(ach / peak, 4)}
    d = per.get(dom)
    return {"bound": "issue", "kernel": dom, "achieved": d["achieved"] if d else None, "peak": round(peak, 1),
            "unit": "G warp-instructions/s", "frac": d["frac"] if d else None, "per_kernel": per,
            "peak_source": f"{sms} SMs x 4 schedulers x {sm_mhz:.0f} MHz (sampled)"}


# ------------------------------------------------------------ multi-rank
def rank_first_dag(rank: int, per_rank: int = 4096) -> int:
    """Weak scaling: rank r evaluates its own window of the DAG stream."""
    return rank * per_rank


def combine_ranks(tasks: float, elapsed_s: float, dist, device) -> tuple[float, float]:
    """Whole-job tasks (sum over ranks) and the slowest rank's time (max)."""
    if dist is None:
        return tasks, elapsed_s
    import torch
    t = torch.tensor([tasks, elapsed_s], dtype=torch.float64, device=device)
    s_ = t.clone()
    dist.all_reduce(s_, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(s_[0]), float(t[1])


# --------------------------------------------------------------------- arms
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def first_dags(batch, budget_tasks: int, max_n: int | None = None):
    """The first DAGs of the workload (of at most max_n tasks each, if given) holding about
    budget_tasks tasks."""
    idx, tasks = [], 0
    for d in range(batch.ndag):
        n = int(batch.task_base[d + 1] - batch.task_base[d])
        if max_n is not None and n > max_n:
            continue
        idx.append(d)
        tasks += n
        if tasks >= budget_tasks:
            break
    return idx, tasks


def run_oracle(dags, machine, threads: int) -> None:
    """The oracle (attributes + simulation) over the DAGs, one DAG per call, on `threads` host
    threads (its C calls release the interpreter lock)."""
    import oracle
    if threads <= 1:
        for g in dags:
            assert oracle.simulate(g, machine)["rc"] == 0
        return
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(threads) as ex:
        assert all(rc == 0 for rc in ex.map(lambda g: oracle.simulate(g, machine)["rc"], dags))


def cpu_baseline(batch, machine, per_core_tasks=100000, max_n=None):
    """The oracle, as it stands, on the first DAGs of the workload (of at most max_n tasks each:
    its exact inspiring ability grows with n^2): once on one core, and on every host core (DAGs
    spread over threads)."""
    import oracle
    idx1, t1 = first_dags(batch, per_core_tasks, max_n)
    oracle.simulate(batch.dag(idx1[0]), machine)  # load the library before the threads start
    dags1 = [batch.dag(d) for d in idx1]
    s0 = time.perf_counter()
    run_oracle(dags1, machine, 1)
    dt1 = time.perf_counter() - s0
    cores = host_cores()
    idx, tasks = first_dags(batch, per_core_tasks * cores, max_n)
    dags = [batch.dag(d) for d in idx]
    s0 = time.perf_counter()
    run_oracle(dags, machine, cores)
    dt = time.perf_counter() - s0
    which = "DAGs" if max_n is None else f"DAGs of at most {max_n} tasks"
    return {"value": tasks / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {len(idx)} {which} of the workload ({tasks} tasks), attributes + simulation, "
                      f"{dt:.1f} s on {cores} threads (one DAG per oracle call)",
            "single_core": {"value": t1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"first {len(idx1)} DAGs ({t1} tasks), {dt1:.1f} s"}}


def run_reference(args, rank):
    """The oracle arm: same metric on a bounded sample per step, host cores."""
    import inputs
    import oracle
    if rank != 0:
        return
    batch = inputs.layered4096()
    machine = inputs.MACHINE_LAYERED
    oracle.simulate(batch.dag(0), machine)  # load the library before the threads start
    cores = host_cores()
    idx, tasks = first_dags(batch, 25000 * cores)  # about a second of oracle work per step
    dags = [batch.dag(d) for d in idx]
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        run_oracle(dags, machine, cores)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    step = float(np.mean(times))
    v = tasks / step
    cb = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
          "sample": f"first {len(idx)} DAGs of the workload ({tasks} tasks) per step, on {cores} threads"}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
                      "data": "synthetic", "config": {"workload": WORKLOAD, "sample_tasks": tasks},
                      "cpu_baseline": cb,
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def compare_policies(args, batch, mach, t_struct, b_main, mk_main, dev, steps=5):
    """Throughput of the evaluation step and mean makespan under DMDA (FIFO pop)
    and the DMDAP baselines (static IA / bottom-level priority), beside INSPIRIT,
    all through the same kernels on the same DAGs; and the unit-time search:
    its duration and INSPIRIT's mean makespan with the searched unit times."""
    import torch

    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    out = {"inspirit": {"mean_makespan_ns": float(mk_main.double().mean())}}
    n, nd = batch.n_total, batch.ndag
    bufs = [torch.empty(n, dtype=t, device=dev) for t in (torch.int32, torch.int32, torch.int32, torch.int64,
                                                           torch.int64)] + [torch.empty(nd, dtype=torch.int64,
                                                                                        device=dev)]
    stream = torch.cuda.current_stream(dev)
    bb = b_main  # each baseline's policy set on the resident batch in turn (then back to INSPIRIT)
    for name, pid in (("dmda_fifo", P.INSP_POLICY_FIFO), ("dmdap_ia", P.INSP_POLICY_DMDAP_IA),
                      ("dmdap_bottom_level", P.INSP_POLICY_DMDAP_BL)):
        pol = P.insp_policy()
        pol.policy = pid
        _lib.insp_batch_set_policy(bb.handle, pol)
        for _ in range(2):
            _lib.insp_evaluate_batch(bb.handle, None, *bufs, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            _lib.insp_evaluate_batch(bb.handle, None, *bufs, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if _lib.insp_batch_status(bb.handle) != 0:
            raise RuntimeError(f"{name}: device-side status not OK: " + _lib.last_error())
        t = e0.elapsed_time(e1) / 1e3 / steps
        out[name] = {"value": n / t, "unit": UNIT, "ms_per_step": t * 1e3,
                     "mean_makespan_ns": float(bufs[5].double().mean())}
    _lib.insp_batch_set_policy(bb.handle, P.insp_policy())
    # unit-time search (k = 0..16) on the main batch, then INSPIRIT with the searched T
    ut = torch.empty(nd, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _lib.insp_unit_time_search(b_main.handle, 16, ut, stream)
    t_search = time.perf_counter() - t0
    _lib.insp_evaluate_batch(b_main.handle, ut, *bufs, stream)
    torch.cuda.synchronize()
    out["unit_time_search"] = {"seconds": t_search, "k_max": 16,
                               "mean_makespan_ns_inspirit_searched_T": float(bufs[5].double().mean()),
                               "median_searched_T_ns": float(ut.double().median())}
    base = out["inspirit"]["mean_makespan_ns"]
    for k in ("dmda_fifo", "dmdap_ia", "dmdap_bottom_level"):
        out[k]["makespan_vs_inspirit"] = out[k]["mean_makespan_ns"] / base
    return out


MIXED_TUNING = dict(groups=1, attr_overlap=1, ia_warps=16, ie_warps=4, ie_ring_mb=16384, sim_warps=2, sim_queue=128,
                    group_split=0, ia_block=1)

# DAGs of at most this many tasks make up the CPU-baseline and per-DAG-launch samples (the
# oracle's exact inspiring ability grows with n^2; the mixed-size workload reaches 1,000,000)
SAMPLE_MAX_N = 20000


def learned_leg(batch, machine, bb, mk_plain, dev, steps=3):
    """The learned proposal scorer (shipped weights) beside the plain INSPIRIT priority on the
    same resident batch (its policy switched for the leg, then back), same tuning: evaluation-step
    throughput and mean makespans."""
    import torch

    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib, scorer
    bits, shipped = scorer.load_trained()
    _lib.insp_set_scorer(machine.handle, bits)
    pol = P.insp_policy()
    pol.policy = P.INSP_POLICY_LEARNED
    _lib.insp_batch_set_policy(bb.handle, pol)
    n, nd = batch.n_total, batch.ndag
    bufs = [torch.empty(n, dtype=t, device=dev) for t in (torch.int32, torch.int32, torch.int32, torch.int64,
                                                           torch.int64)] + [torch.empty(nd, dtype=torch.int64,
                                                                                        device=dev)]
    stream = torch.cuda.current_stream(dev)
    _lib.insp_evaluate_batch(bb.handle, None, *bufs, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        _lib.insp_evaluate_batch(bb.handle, None, *bufs, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if _lib.insp_batch_status(bb.handle) != 0:
        raise RuntimeError("learned policy: device-side status not OK: " + _lib.last_error())
    t = e0.elapsed_time(e1) / 1e3 / steps
    _lib.insp_batch_set_policy(bb.handle, P.insp_policy())  # back to the plain INSPIRIT defaults
    plain = float(mk_plain.double().mean())
    lm = float(bufs[5].double().mean())
    return {"value": n / t, "unit": UNIT, "ms_per_step": t * 1e3, "mean_makespan_ns": lm,
            "mean_makespan_ns_plain": plain, "gain_pct_vs_plain": (plain - lm) / plain * 100.0,
            "policy_shipped": shipped}


def run_ours(args, rank, world, local_rank):
    import torch

    import inputs
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    batch, mach, wdesc, mdesc = make_workload(args, rank)
    machine = P.Machine(mach.n_cpu, mach.n_gpu, mach.xfer_ns)
    b = P.DagBatch(machine, batch)
    n, ndag = b.n_tasks, b.ndag
    stream = torch.cuda.current_stream(dev)
    ia = torch.empty(n, dtype=torch.int32, device=dev)
    ie = torch.empty(n, dtype=torch.int32, device=dev)
    worker = torch.empty(n, dtype=torch.int32, device=dev)
    start = torch.empty(n, dtype=torch.int64, device=dev)
    end = torch.empty(n, dtype=torch.int64, device=dev)
    mk = torch.empty(ndag, dtype=torch.int64, device=dev)

    def step():  # attributes + schedule of every DAG, pipelined by size groups
        _lib.insp_evaluate_batch(b.handle, None, ia, ie, worker, start, end, mk, stream)

    # launch shapes picked on this batch before the timed region (setup, like the load)
    if args.tuning:  # explicit launch shapes (profiling captures)
        _lib.insp_batch_set_tuning(b.handle, _lib.insp_tuning(**json.loads(args.tuning)))
        t_struct = _lib.insp_batch_get_tuning(b.handle)
    elif args.workload == "mixed":
        # the mixed batch's steps take seconds, too long for the autotuner's ~60 candidates x 4 steps:
        # the shapes measured best on it (target-block ability sweep, 128-entry pools with per-worker
        # bitmaps for the 1,000,000-task DAG's ~500 ready tasks over 40 workers, full ring budget)
        _lib.insp_batch_set_tuning(b.handle, _lib.insp_tuning(**MIXED_TUNING))
        t_struct = _lib.insp_batch_get_tuning(b.handle)
    elif args.autotune:
        t_struct = _lib.insp_batch_autotune(b.handle, stream)
    else:
        t_struct = _lib.insp_batch_get_tuning(b.handle)
    _lib.insp_machine_set_tuning(machine.handle, t_struct)  # batches loaded later (the e2e leg) start with it
    tuning = t_struct.as_dict()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if _lib.insp_batch_status(b.handle) != 0:
        raise RuntimeError("device-side status not OK: " + _lib.last_error())

    clocks = ClockSampler(local_rank)
    time.sleep(0.6)  # let the sampler start
    _lib.insp_batch_timing(b.handle, reset=True)
    _lib.insp_batch_set_timing(b.handle, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.mark_start()
    ev_step = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev0.record(stream)
    for k in range(args.steps):
        step()
        ev_step[k].record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    step_ms = [(ev0 if k == 0 else ev_step[k - 1]).elapsed_time(ev_step[k]) for k in range(args.steps)]
    _lib.insp_batch_set_timing(b.handle, False)
    kms, klaunch = _lib.insp_batch_timing(b.handle, reset=True)
    clk = clocks.stop()
    if _lib.insp_batch_status(b.handle) != 0:
        raise RuntimeError("device-side status not OK: " + _lib.last_error())

    tasks_all, t_max = combine_ranks(float(n) * args.steps, elapsed, dist, dev)
    value = tasks_all / t_max

    # ---- the same step recorded once as a CUDA graph and replayed
    graph = None
    gstream = torch.cuda.Stream(dev)
    _lib.insp_batch_record(b.handle, ia, ie, worker, start, end, mk, gstream)
    for _ in range(args.warmup):
        _lib.insp_batch_replay(b.handle, gstream)
    gstream.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    g0.record(gstream)
    for _ in range(args.steps):
        _lib.insp_batch_replay(b.handle, gstream)
    g1.record(gstream)
    gstream.synchronize()
    barrier()
    if _lib.insp_batch_status(b.handle) != 0:
        raise RuntimeError("device-side status not OK after graph replays: " + _lib.last_error())
    g_elapsed = g0.elapsed_time(g1) / 1e3
    graph = {"value": n * args.steps / g_elapsed, "unit": UNIT, "ms_per_step": g_elapsed / args.steps * 1e3,
             "launches_per_step": 1}

    # ---- simulation alone (a3-a5), on the attributes the timed steps left resident
    for _ in range(args.warmup):
        _lib.insp_simulate_batch(b.handle, ia, ie, worker, start, end, mk, stream)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s0.record(stream)
    for _ in range(args.steps):
        _lib.insp_simulate_batch(b.handle, ia, ie, worker, start, end, mk, stream)
    s1.record(stream)
    torch.cuda.synchronize()
    if _lib.insp_batch_status(b.handle) != 0:
        raise RuntimeError("device-side status not OK after the simulation-only steps: " + _lib.last_error())
    s_elapsed = s0.elapsed_time(s1) / 1e3
    sim_only = {"value": n * args.steps / s_elapsed, "unit": UNIT, "ms_per_step": s_elapsed / args.steps * 1e3}

    # ---- roofline of the dominant kernel
    names = ["k_ia", "k_ie_pull", "k_sim"]  # the layered and tiled workloads take the pull efficiency sweep
    alg = algorithmic_bytes(batch)
    per_launch_ms = {names[k]: kms[k] / max(klaunch[k], 1) for k in range(3)}
    share = {names[k]: kms[k] / max(kms[:3].sum(), 1e-9) for k in range(3)}
    dom = max(names, key=lambda k: share[k])
    peak, peak_kind = load_peaks()
    # achieved: the path's algorithmic bytes (per task figure x the tasks one step processes,
    # each input read once and each output written once) over the dominant kernel's time per
    # step (= bytes per launch / mean launch time; one launch per size group and step)
    pb = path_bytes(batch)
    # the recorded counters were taken on the layered workload (scaled to its 4096 DAGs)
    rec_key = f"{args.workload}:{args.ndag}" if args.workload == "layered" else args.workload
    dom_s = kms[names.index(dom)] / 1e3 / args.steps
    achieved = pb / dom_s / 1e9
    own = alg[dom] / dom_s / 1e9  # the dominant kernel's own inputs and outputs only
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_from_profile(dom, klaunch[names.index(dom)] / args.steps, rec_key), "kernel": dom,
                "peak_source": f"{peak_kind} hbm_gbs",
                "path_bytes_per_step": int(pb), "path_bytes_per_task": round(pb / max(n, 1), 2),
                "kernel_own_bytes": {k: int(v) for k, v in alg.items()},
                "kernel_own": {"achieved": own, "frac": own / peak},
                "kernel_ms": {k: round(v, 4) for k, v in per_launch_ms.items()},
                "kernel_share": {k: round(v, 4) for k, v in share.items()},
                "step_frac": pb / (t_max / args.steps) / 1e9 / peak}
    roofline_issue = issue_roofline(names, kms, args.steps, torch.cuda.get_device_properties(dev).multi_processor_count,
                                    clk["sm_mhz"] or clk["sm_max_mhz"] or 2032.0, dom, rec_key)

    # ---- per-DAG launch form on a sample (same kernels, one DAG per launch)
    per_dag = None
    if rank == 0 and not args.profile:
        k_sample = 64
        small = [d for d in range(batch.ndag) if batch.task_base[d + 1] - batch.task_base[d] <= SAMPLE_MAX_N]
        sub = batch.subset(small[:k_sample])
        k_sample = sub.ndag
        dags, outs = [], []
        for d in range(k_sample):
            g = sub.dag(d)
            h = _lib.insp_dag_load_csr(machine.handle, g.n, g.row_ptr, g.col_idx, None, 1, None,
                                       np.ascontiguousarray(np.stack([g.c_cpu, g.c_gpu], 1)))
            dags.append(h)
            outs.append([torch.empty(max(g.n, 1), dtype=dt, device=dev) for dt in
                         (torch.int32, torch.int32, torch.int32, torch.int64, torch.int64)] +
                        [torch.empty(1, dtype=torch.int64, device=dev)])

        def per_dag_pass():
            for h, o in zip(dags, outs):
                _lib.insp_attributes(h, 0, o[0], o[1], stream)
                _lib.insp_simulate(h, o[0], o[1], o[2], o[3], o[4], o[5], stream)

        per_dag_pass()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            per_dag_pass()
        e1.record(stream)
        torch.cuda.synchronize()
        t_pd = e0.elapsed_time(e1) / 1e3 / reps
        sub_tasks = int(sub.n_total)
        for h in dags:
            _lib.insp_dag_destroy(h)
        pd_value = sub_tasks / t_pd
        per_dag = {"value": pd_value, "unit": UNIT, "sample_dags": k_sample, "sample_tasks": sub_tasks,
                   "batched_over_per_dag": (n * args.steps / elapsed) / pd_value}

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if rank == 0 and not args.profile:
        def pinned(a):
            t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            return t
        h_tb, h_eb = pinned(batch.task_base), pinned(batch.edge_base)
        h_rp, h_ci, h_ty = pinned(batch.row_ptr), pinned(batch.col_idx), pinned(batch.type)
        h_tc = pinned(batch.type_cost)
        h_kc = pinned(batch.task_cost) if batch.task_cost is not None else None
        o_w = torch.empty(n, dtype=torch.int32).pin_memory()
        o_s = torch.empty(n, dtype=torch.int64).pin_memory()
        o_e = torch.empty(n, dtype=torch.int64).pin_memory()
        o_m = torch.empty(ndag, dtype=torch.int64).pin_memory()
        h2d = sum(int(t.numel() * t.element_size()) for t in (h_tb, h_eb, h_rp, h_ci, h_ty, h_tc)
                  + ((h_kc,) if h_kc is not None else ()))
        d2h = sum(int(t.numel() * t.element_size()) for t in (o_w, o_s, o_e, o_m))

        def load():
            return _lib.insp_batch_load_csr(machine.handle, ndag, h_tb, h_eb, h_rp, h_ci, h_ty, batch.n_types,
                                            h_tc, h_kc)

        def evaluate(h, est):
            try:
                # schedule to pinned host arrays (D2H + sync inside); ia / ie stay on the device
                _lib.insp_evaluate_batch(h, None, ia_e, ie_e, o_w, o_s, o_e, o_m, est)
            finally:
                _lib.insp_batch_destroy(h)

        ia_e, ie_e = torch.empty_like(ia), torch.empty_like(ie)
        streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]  # non-blocking: loads run beside them
        k_e2e = max(1, min(args.steps, 30))
        # one step at a time: load, evaluate, read back
        free0 = torch.cuda.mem_get_info(dev)[0]
        h_first = load()
        # device bytes a loaded batch holds, plus the staging of its host outputs at evaluation
        per_batch = max(free0 - torch.cuda.mem_get_info(dev)[0], 1) + 32 * n
        evaluate(h_first, streams[0])
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            evaluate(load(), streams[0])
        t_serial = (time.perf_counter() - t0) / k_e2e
        assert np.array_equal(o_m.numpy(), mk.cpu().numpy())

        # as a serving loop runs it: the next batches load (H2D, validation, predecessor lists) on
        # host threads, each batch on its own stream, while this one evaluates, and each step's
        # read-back (asynchronous, into pinned memory) overlaps the next step's kernels; steps
        # alternate between two streams and two sets of outputs.  A load's ingest kernels get SM
        # slots only as the evaluation's persistent CTAs retire, so one loader thread cannot keep
        # up (12.3 ms per load beside an evaluation against 8.6 alone); three can.  Batches alive:
        # one per loader, the one evaluating, the one reading back.
        free_now = torch.cuda.mem_get_info(dev)[0]
        loaders = max((k for k in (3, 2, 1) if free_now > (k + 2.2) * per_batch), default=0)
        serving = loaders > 0
        if serving:
            import queue
            import threading
            outs = [(ia_e, ie_e, o_w, o_s, o_e, o_m),
                    (torch.empty_like(ia), torch.empty_like(ie), torch.empty(n, dtype=torch.int32).pin_memory(),
                     torch.empty(n, dtype=torch.int64).pin_memory(), torch.empty(n, dtype=torch.int64).pin_memory(),
                     torch.empty(ndag, dtype=torch.int64).pin_memory())]
            slots = threading.Semaphore(loaders + 2)  # batches alive: loading, evaluating, reading back
            q = queue.Queue()
            warm = 2 + loaders

            def loader(count):
                try:
                    for _ in range(count):
                        slots.acquire()
                        q.put(load())
                except Exception as exc:  # handed to the evaluating thread
                    q.put(exc)

            def finish(p):  # wait for a step's read-back, check it, release its batch
                h, j = p
                streams[j].synchronize()
                rc = _lib.insp_batch_status(h)
                _lib.insp_batch_destroy(h)
                slots.release()
                if rc != 0:
                    raise RuntimeError("device-side status not OK in the e2e loop: " + _lib.last_error())

            # the loaders run on past the timed steps by the pipeline's depth, so that the window ends
            # as full as it began (batches loaded before it are balanced by loads in flight after it)
            extra = loaders + 2
            total = warm + k_e2e + extra
            ths = [threading.Thread(target=loader, args=(total // loaders + (i < total % loaders),), daemon=True)
                   for i in range(loaders)]  # daemons: never block the exit after an error
            for th in ths:
                th.start()
            pending = None
            for k in range(warm + k_e2e):
                if k == warm:
                    if pending is not None:
                        finish(pending)
                        pending = None
                    t0 = time.perf_counter()
                h = q.get()
                if isinstance(h, Exception):
                    raise h
                j = k % 2
                o = outs[j]
                _lib.insp_evaluate_batch_async(h, None, o[0], o[1], o[2], o[3], o[4], o[5], streams[j])
                if pending is not None:
                    finish(pending)
                pending = (h, j)
            finish(pending)
            t_e2e = (time.perf_counter() - t0) / k_e2e
            for _ in range(extra):  # the fill after the window: loaded, not evaluated
                h = q.get()
                if isinstance(h, Exception):
                    raise h
                _lib.insp_batch_destroy(h)
                slots.release()
            for th in ths:
                th.join()
            for o in outs:
                assert np.array_equal(o[5].numpy(), mk.cpu().numpy())
            e2e = {"value": n / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "ms_per_step": t_e2e * 1e3, "steps": k_e2e,
                   "mode": f"serving loop: {loaders} loader threads load the next batches and this step's read-back "
                           f"overlaps the kernels",
                   "serial": {"value": n / t_serial, "ms_per_step": t_serial * 1e3}}
        else:  # one batch at a time: the serial figure is the end-to-end one
            e2e = {"value": n / t_serial, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "ms_per_step": t_serial * 1e3, "steps": k_e2e,
                   "mode": "one step at a time: load, evaluate, read back (three batches of this size do not "
                           "fit the device together, so the serving loop's overlap is not run)",
                   "serial": {"value": n / t_serial, "ms_per_step": t_serial * 1e3}}

    # ---- the baselines and the unit-time search on the same batch (same tuning, same step)
    policies = None
    if rank == 0 and not args.profile and not args.no_policies:
        policies = compare_policies(args, batch, mach, t_struct, b, mk, dev)

    learned = None
    if rank == 0 and not args.profile and not args.no_learned:
        learned = learned_leg(batch, machine, b, mk, dev)

    cb = cpu_baseline(batch, mach, max_n=SAMPLE_MAX_N) if (rank == 0 and world == 1 and not args.profile) else None

    if rank == 0:
        res = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": wdesc, "ndag": ndag, "tasks": n, "edges": int(batch.m_total),
                       "machine": mdesc, "policy": "INSPIRIT (defaults)",
                       "tuning": dict(tuning, autotuned=bool(args.autotune and not args.tuning
                                                             and args.workload != "mixed")),
                       "l2": f"inputs larger than L2 ({(4 * (n + ndag) + 4 * batch.m_total + n) / 1e6:.0f} MB of CSR "
                             f"resident, 126 MB L2)", "parallelism": f"dp{world}" if world > 1 else "single GPU"},
            "per_dag_form": per_dag,
            "policies": policies,
            "learned": learned,
            "cuda_graph": graph,
            "e2e": e2e,
            "roofline": roofline,
            "roofline_issue": roofline_issue,
            "step_ms": {"best": round(min(step_ms), 4), "median": round(float(np.median(step_ms)), 4),
                        "mean": round(t_max / args.steps * 1e3, 4)},
            "simulate_only": sim_only,
            "cpu_baseline": cb,
            "clocks": clk,
            # our kernels in the timed region: ability, efficiency, simulation, plus one
            # step-counter kernel per step; ability, efficiency and simulation kernels once
            # per size group
            "gpu_launches": int(klaunch[:3].sum() + args.steps),
        }
        print(json.dumps(res), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ndag", type=int, default=4096, help="first K DAGs of the workload (profiling captures)")
    ap.add_argument("--workload", choices=["layered", "layered_degree", "tiled", "mixed"], default="layered",
                    help="layered: the 4096-DAG headline workload; tiled: Cholesky/LU/QR batches; mixed: the "
                         "mixed-size stress batch")
    ap.add_argument("--mixed-ndag", dest="mixed_ndag", type=int, default=10000,
                    help="DAGs of the mixed-size workload (before the 1M-task DAG)")
    ap.add_argument("--no-large", dest="no_large", action="store_true",
                    help="mixed workload without the 1,000,000-task DAG")
    ap.add_argument("--tiles", default="16,32", help="tile counts of the tiled workload")
    ap.add_argument("--instances", type=int, default=256, help="instances per (kind, tiles) of the tiled workload")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the library's default launch shapes instead of autotuning them on the batch")
    ap.add_argument("--tuning", default=None,
                    help='explicit tuning as JSON, e.g. \'{"groups": 1, "attr_overlap": 0, "ia_warps": 32, '
                         '"ie_warps": 16, "ie_ring_mb": 512, "sim_warps": 4, "sim_queue": 64, "group_split": 0, '
                         '"ia_block": 0}\'')
    ap.add_argument("--no-policies", dest="no_policies", action="store_true",
                    help="skip the DMDA / DMDAP baselines and the unit-time search leg")
    ap.add_argument("--no-learned", dest="no_learned", action="store_true",
                    help="skip the learned-scorer leg beside the plain policy")
    ap.add_argument("--profile", action="store_true",
                    help="only the timed steps: no per-DAG form, e2e or CPU baseline (for ncu captures)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
