#!/usr/bin/env python
"""Benchmark of the CFPQ closure engine on B300.

Workload (one GPU): the same-generation hierarchy of n = 16384 nodes (5000 classes,
11384 instances, seed 0) with both same-generation grammars on the same graph (Query 1
and the subClassOf-only query). One step = one pass of the whole path for both queries:
matrix initialisation, the closure loop to the fixpoint, and extraction of every R_A
into device memory. The timed path is, by default, Algorithm 1 itself (Jacobi schedule,
T <- T u T x T) with every Boolean product on the tcgen05 tensor cores; the in-place
tensor schedule and the automatic path (sparse bit-gather products) are timed on the same
workload and reported beside it.

metric: Boolean GOPS. The work of a step is the work of Algorithm 1 on the workload:
sum over queries of (loop executions of Algorithm 1) x (binary productions) x 2 n^3, a
fixed number for the workload (both arms count it the same way), divided by the step
time. `value` is device-timed (CUDA events on the launching stream, inputs resident in
HBM); `e2e` is the same metric through the C ABI with host buffers (edge upload, solve,
triples copied back) inside the timed region.

Every relation of the timed leg is compared with the CPU oracle's (`parity`; a mismatch
ends the run with exit status 3). Beside the main workload the line carries the default
path of cfpq_solve (`default_path`: its time, roofline and e2e) and the other workload
configurations (`configs`): Query 1 on n = 1024 hierarchies (seeds 0-4), the two-cycle
closure (n = 8190), 256 batched queries in one grouped launch, and the served Poisson
stream at two loads over three arrival draws.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--path tensor|auto|gather]
                    [--schedule jacobi|inplace] [--no-configs] [--no-alternatives]
    python bench.py --impl reference ...      # the CPU oracle on the same workload
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import cfpq_synth as synth  # noqa: E402

N_NODES, N_CLASSES, SEED = 16384, 5000, 0
WORKLOAD = "hierarchy n=16384 (5000 classes), Query 1 + sc-only query on one graph, closure + extraction"
METRIC = "Boolean GOPS (2n^3 per product of Algorithm 1) over the closure"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--path", default="tensor", choices=["auto", "tensor", "gather"])
    ap.add_argument("--schedule", default="jacobi", choices=["jacobi", "inplace"])
    ap.add_argument("--tensor", default="dense", choices=["dense", "skip"],
                    help="tensor products of the timed leg: every K step (Algorithm 1's dense product) or "
                         "only the K steps whose operand tiles are both non-zero")
    ap.add_argument("--tensor-kind", default="auto", choices=["auto", "fp8", "fp4"],
                    help="operand format of the tensor products: E4M3 bytes (kind::f8f6f4) or E2M1 nibbles "
                         "(kind::mxf4, unit scales); auto = the library's default (fp4)")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "rows"],
                    help="with N > 1 ranks: replicas (every rank solves the whole workload, weak scaling) or "
                         "rows (every query split into N row blocks, one per rank, new pairs exchanged by NCCL "
                         "after each loop execution; strong scaling)")
    ap.add_argument("--no-alternatives", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave out the other workload configurations (n = 1024 seeds, two cycles, 256 batched "
                         "queries, served stream) that the default line reports beside the main workload")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="hier16k",
                    choices=["hier16k", "sg16k", "batch256", "serve", "cycles", "lengths16k", "blockdiag32k"],
                    help="hier16k: the default line; sg16k: the same hierarchy with the same-generation "
                         "query (denser result); batch256 / serve / cycles: the batched, served and "
                         "two-cycle workloads; lengths16k: single-path lengths (Section 5) on the hierarchy")
    ap.add_argument("--n", type=int, default=None, help="smaller hierarchy for profiling captures")
    ap.add_argument("--classes", type=int, default=None)
    ap.add_argument("--cycle-p", type=int, default=None, help="a-cycle length of the cycles workload (profiling)")
    a = ap.parse_args()
    global N_NODES, N_CLASSES, WORKLOAD, GRAMMARS
    if a.workload == "sg16k":
        GRAMMARS = [("SG", synth.GRAMMAR_SG)]
        WORKLOAD = WORKLOAD.replace("Query 1 + sc-only query", "same-generation query (sc up, then down)")
    if a.n:
        N_NODES = a.n
        N_CLASSES = a.classes or max(1, round(N_NODES * 5000 / 16384))
        WORKLOAD = WORKLOAD.replace("n=16384 (5000 classes)", f"n={N_NODES} ({N_CLASSES} classes)")
    return a


GRAMMARS = [("Q1", synth.GRAMMAR_Q1), ("QSC", synth.GRAMMAR_QSC)]


def max_over_ranks(x: float, device: str = "cuda") -> float:
    """The job's time: the slowest rank's (max over the default process group); the value
    itself when there is no group (one process)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput of replicas: every rank processes its own units (weak scaling),
    the job takes the slowest rank's time."""
    return world * units_per_rank / seconds


def workload():
    g = synth.hierarchy(N_NODES, N_CLASSES, seed=SEED)
    return g, list(GRAMMARS)


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx, self.proc, self.lines = gpu_index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------ CPU arm

def oracle_step(graph, grammars):
    import oracle

    return [oracle.hellings(graph, text) for _, text in grammars]


def oracle_work(graph, grammars):
    """Products of Algorithm 1 on the workload, counted by the oracle's own sparse form of
    Algorithm 1 (loop executions x binary productions)."""
    import oracle

    total = 0
    for _, text in grammars:
        cnf, _, k = oracle.matrix_closure_sparse(graph, text)
        total += k * len(set(map(tuple, cnf.binary)))
    return total


def check_against_oracle(graph, grammars, engine_pairs):
    """Every relation the engine computed on the workload against the oracle's, element by
    element; a mismatch ends the run (exit status 3) instead of printing a number."""
    refs = oracle_step(graph, grammars)
    rel = pairs = 0
    for (label, _), ref, got in zip(grammars, refs, engine_pairs):
        for nm, arr in got.items():
            exp = ref.pairs(nm)
            if arr.shape != exp.shape or not np.array_equal(arr, exp):
                print(f"bench: {label} R_{nm} differs from the oracle ({arr.shape[0]} vs {exp.shape[0]} pairs)",
                      file=sys.stderr)
                sys.exit(3)
            rel += 1
            pairs += int(exp.shape[0])
    return {"reference": "oracle (Hellings worklist on the CPU)", "relations_compared": rel,
            "pairs_compared": pairs, "equal": True}


def reference_arm(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    graph, grammars = workload()
    products = oracle_work(graph, grammars)
    ops = products * 2.0 * float(N_NODES) ** 3
    for _ in range(args.warmup):
        oracle_step(graph, grammars)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(graph, grammars)
    dt = (time.perf_counter() - t0) / args.steps
    value = ops / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GOPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64 bitsets (CPU worklist)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_NODES, "classes": N_CLASSES, "seed": SEED,
                   "grammars": [nm for nm, _ in grammars], "products_per_step": products},
        "cpu_baseline": {"value": value, "unit": "GOPS", "cores": 1, "kind": "oracle",
                         "sample": f"full workload, {args.steps} timed steps, one host thread"},
        "e2e": {"value": value, "unit": "GOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------------ GPU arm

TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_tc_bool_gemm_hier16k_dram.txt")
TC_SOURCE = os.path.join(ROOT, "paper_1707_01007_b300", "csrc", "cfpq_tensor.cu")


def tc_traffic_per_launch(dense=True, tkind="fp8"):
    """DRAM bytes per k_tc_bool_gemm launch (dense products, or with tile skipping; E4M3 or,
    with the key suffix _fp4, E2M1 operands) from the committed ncu summary, or None when the
    summary is missing or the kernel source changed since the counters were taken."""
    import hashlib

    try:
        vals = {}
        for ln in open(TRAFFIC_FILE):
            if ":" in ln:
                k, v = ln.split(":", 1)
                vals[k.strip()] = v.strip()
        src = hashlib.sha256(open(TC_SOURCE, "rb").read()).hexdigest()
        if vals.get("source_sha256") != src:
            return None
        key = "dram_bytes_per_launch_avg" if dense else "dram_bytes_per_launch_skip_avg"
        return float(vals[key + ("_fp4" if tkind == "fp4" else "")])
    except (OSError, KeyError, ValueError):
        return None


# dense tcgen05 ops (2 per multiply-add) per SM clock, measured by cfpq_measure_tensor_peaks
# (clock64 around back-to-back MMAs): kind::f8f6f4 16384, kind::mxf4 32768
OPS_PER_CLK_SM = {"fp8": 16384, "fp4": 32768}
# the recipe's nominal dense ratios to bf16 (2.25 PFLOP/s): fp8 4.5, fp4 13.5
NOMINAL_RATIO_TO_BF16 = {"fp8": 2.0, "fp4": 6.0}


def effective_kind(name):
    """The operand format a tensor_kind option runs with (the library's default is FP4)."""
    return "fp4" if name == "auto" else name


def nominal_tflops(sm_mhz, tkind="fp8"):
    """The dense tensor rate of this device for an operand kind at an SM clock (SMs x ops per
    clock x clock)."""
    import torch

    if not sm_mhz:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * OPS_PER_CLK_SM[effective_kind(tkind)] * sm_mhz * 1e6 / 1e12


def kind_code(eng, name):
    return {"auto": eng.TENSOR_AUTO, "fp8": eng.TENSOR_FP8, "fp4": eng.TENSOR_FP4}[name]


def roofline(eng, graph, gs, path, schedule, stream, dense=True, sm_mhz=None, tkind="auto"):
    """Dominant product kernel: every product launch of a solve with the timed options is
    bracketed by CUDA events on the launching stream (profile mode); algorithmic work per
    launch is 2 n^3 per production of the group (tensor; with tile skipping, the K steps the
    launch issued) or the counted words (gather). A tensor product's peak is that of its
    operand kind: the measured bf16 burst x the nominal ratio of the kind, with the kind's
    measured MMA-only rate (cfpq_measure_tensor_peaks, same run) and its nominal per-clock
    rate at the sampled clock beside it."""
    peaks, source = load_peaks()
    ek = effective_kind(tkind)
    prod_ms = prod_l = tens_ms = tens_l = 0
    flops = bytes_ = useful = 0.0
    for g in gs:
        q = eng.Query(g, graph.n, graph.edges, path=path, schedule=schedule, profile=True, timeout_s=300.0,
                      dense_tensor=dense, tensor_kind=kind_code(eng, tkind))
        q.solve(stream)
        s = q.stats()
        prod_ms += s["product_ms"]
        prod_l += s["product_launches"]
        tens_ms += s["tensor_ms"]
        tens_l += s["tensor_launches"]
        flops += s["tensor_live_ops"]
        bytes_ += s["product_bytes"]
        useful += s["useful_ops"]
        q.close()
    if tens_l > 0 and tens_ms >= 0.5 * prod_ms:
        achieved = flops / (tens_ms / 1e3) / 1e12
        ratio = NOMINAL_RATIO_TO_BF16[ek]
        peak = ratio * peaks["bf16_tflops"]
        sustained = ratio * peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        # the integer tensor references of this device (sm_103a has no 8-bit integer tcgen05 kind)
        mma = eng.measure_mma_sync_peaks()
        tp = eng.measure_tensor_peaks()
        mma_only = tp["mxf4_tflops"] if ek == "fp4" else tp["f8f6f4_tflops"]
        nominal = nominal_tflops(sm_mhz, ek)
        nominal8 = nominal_tflops(sm_mhz, "fp8")
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": tc_traffic_per_launch(dense, ek), "kernel": f"k_tc_bool_gemm<{ek}>",
                "operands": "E2M1 0/1 nibbles, kind::mxf4, unit UE8M0 scales" if ek == "fp4"
                            else "E4M3 0/1 bytes, kind::f8f6f4",
                "tile_skipping": not dense, "launches": tens_l,
                "launch_ms": tens_ms / tens_l, "flops_per_launch": flops / tens_l,
                "peak_note": f"{source} bf16 dense burst x {ratio:g} (the {ek} : bf16 nominal ratio); "
                             f"frac against the sustained figure x {ratio:g}: {achieved / sustained:.3f}",
                "useful_ops_per_step": useful,
                "measured_mma_only": {"peak": mma_only, "frac": achieved / mma_only,
                                      "note": "the same kind's MMAs back to back in the kernel's tile shape, "
                                              "no unpacking (cfpq_measure_tensor_peaks, this run)",
                                      "probe": tp},
                "nominal_at_clock": {"peak": nominal, "sm_mhz": sm_mhz,
                                     "frac": (achieved / nominal) if nominal else None,
                                     "ops_per_clk_sm": OPS_PER_CLK_SM[ek],
                                     "note": "SMs x the kind's dense ops per clock x the median SM clock "
                                             "sampled during the timed region"},
                "vs_fp8_at_clock": {"peak": nominal8, "frac": (achieved / nominal8) if nominal8 else None,
                                    "note": "the E4M3 kind's dense rate at the same clock: the ceiling of an "
                                            "FP8 product kernel"},
                "int_tensor_refs": {"mma_sync_s8_tops": mma["s8_tops"], "frac_of_mma_sync_s8": achieved / mma["s8_tops"],
                                    "mma_sync_b1_tops": mma["b1_tops"],
                                    "frac_of_mma_sync_b1": achieved / mma["b1_tops"],
                                    "note": "measured on this device (cfpq_measure_mma_sync_peaks)"}}
    gather_ms = prod_ms - tens_ms
    launches = max(1, prod_l - tens_l)
    achieved = bytes_ / (gather_ms / 1e3) / 1e9 if gather_ms > 0 else None
    peak = peaks["hbm_gbs"]
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "traffic": None, "kernel": "k_scan_rows + k_gather_list",
            "launches": launches, "launch_ms": gather_ms / launches, "bytes_per_launch": bytes_ / launches,
            "peak_note": f"{source} HBM copy bandwidth"}


class Leg:
    """The queries of the workload resident on the device with one set of options."""

    def __init__(self, eng, torch, graph, gs, path, schedule, stream, dense=True, kind="auto"):
        self.eng, self.torch, self.gs, self.stream = eng, torch, gs, stream
        self.qs = [eng.Query(g, graph.n, graph.edges, path=path, schedule=schedule, timeout_s=300.0,
                             dense_tensor=dense, tensor_kind=kind_code(eng, kind)) for g in gs]
        self.bufs = []
        for q in self.qs:
            q.solve(stream)
            self.bufs.append(torch.empty(max(1, q.get_all_device(0, 0)) * 3, dtype=torch.int32, device="cuda"))

    def step(self):
        for q, b in zip(self.qs, self.bufs):
            q.solve(self.stream)
            q.get_all_device(b.data_ptr(), b.numel() // 3)

    def time(self, steps):
        torch = self.torch
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(self.stream)
        for i in range(steps):
            self.step()
            ev[i + 1].record(self.stream)  # per-step boundaries (best and median beside the mean)
        torch.cuda.synchronize()
        self.step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        return ev[0].elapsed_time(ev[steps]) / steps

    def close(self):
        for q in self.qs:
            q.close()


class RowBlockLeg:
    """The queries of the workload as row blocks of a sharded solve (Jacobi schedule, the
    timed leg's product path). exchange=None: `parts` blocks of each query on this one device,
    the records copied between them (shard.solve_local); otherwise this rank's block of each
    query, the records all-gathered over the process group (shard.solve_sharded)."""

    def __init__(self, eng, torch, graph, gs, path, stream, dense, kind, parts, rank=0, exchange=None):
        from paper_1707_01007_b300 import shard

        self.shard, self.torch, self.stream, self.exchange = shard, torch, stream, exchange
        blocks = shard.row_blocks(graph.n, parts)
        mine = range(len(blocks)) if exchange is None else [rank]
        self.per_query = []
        for g in gs:
            bl = []
            for r in mine:
                b0, b1 = blocks[r]
                q = eng.Query(g, graph.n, graph.edges, path=path, schedule=eng.SCHED_JACOBI, timeout_s=300.0,
                              dense_tensor=dense, tensor_kind=kind_code(eng, kind), row_begin=b0, row_end=b1)
                bl.append(shard.EngineBlock(q, b0, b1, len(g.names)))
            self.per_query.append(bl)
        self.executions = [self._solve(bl) for bl in self.per_query]
        self.bufs = [torch.empty(max(1, bl[0].q.get_all_device(0, 0)) * 3, dtype=torch.int32, device="cuda")
                     for bl in self.per_query]

    def _solve(self, bl):
        return self.shard.solve_local(bl) if self.exchange is None else self.shard.solve_sharded(bl[0], self.exchange)

    def step(self):
        # every query's closure, then every relation of it extracted into device memory
        for bl, buf in zip(self.per_query, self.bufs):
            self._solve(bl)
            bl[0].q.get_all_device(buf.data_ptr(), buf.numel() // 3)

    @property
    def qs(self):
        return [bl[0].q for bl in self.per_query]

    def time(self, steps):
        torch = self.torch
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(self.stream)
        for i in range(steps):
            self.step()
            ev[i + 1].record(self.stream)
        torch.cuda.synchronize()
        self.step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        return ev[0].elapsed_time(ev[steps]) / steps

    def relations(self):
        return [{nm: bl[0].q.get(nm) for nm in bl[0].q.grammar.names} for bl in self.per_query]

    def close(self):
        for bl in self.per_query:
            for b in bl:
                b.q.close()


def engine_arm(args):
    import torch
    import torch.distributed as dist

    import paper_1707_01007_b300 as eng

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    paths = {"tensor": eng.PATH_TENSOR, "gather": eng.PATH_GATHER, "auto": eng.PATH_AUTO}
    path = paths[args.path]
    schedule = eng.SCHED_JACOBI if args.schedule == "jacobi" else eng.SCHED_INPLACE

    graph, grammars = workload()
    gs = [eng.Grammar(t, graph.labels) for _, t in grammars]
    stream = torch.cuda.current_stream()
    # work of Algorithm 1 on this workload: loop executions x productions, from a Jacobi solve
    products = 0
    for g in gs:
        qj = eng.Query(g, graph.n, graph.edges, schedule=eng.SCHED_JACOBI, path=eng.PATH_GATHER, timeout_s=300.0)
        qj.solve(stream)
        nprod = len({(g.cnf.contents.binary[i].lhs, g.cnf.contents.binary[i].b, g.cnf.contents.binary[i].c)
                     for i in range(g.cnf.contents.n_binary)})
        products += qj.stats()["iterations"] * nprod
        qj.close()
    ops_per_step = products * 2.0 * float(N_NODES) ** 3

    dense = args.tensor == "dense"
    sharded = world > 1 and args.shard == "rows"
    if sharded:
        # every query split into `world` row blocks, this rank's block here; NCCL all-gathers
        # the new pairs after each loop execution (Jacobi schedule)
        from paper_1707_01007_b300 import shard as shardmod
        main = RowBlockLeg(eng, torch, graph, gs, path, stream, dense, args.tensor_kind, world, rank,
                           shardmod.TorchExchange("cuda"))
    else:
        main = Leg(eng, torch, graph, gs, path, schedule, stream, dense, args.tensor_kind)
    for _ in range(args.warmup):
        main.step()
    st = [q.stats() for q in main.qs]
    # the solve's kernels plus the extraction of every relation (count, three scan passes,
    # offsets per non-terminal, emission)
    launches_per_step = sum(s["kernel_launches"] + 6 for s in st)

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    ms = main.time(args.steps)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ms)
    step_ms = {"best": min(main.step_ms), "median": float(np.median(main.step_ms)), "worst": max(main.step_ms)}
    # replicas: every rank's workload counts; row blocks: the ranks solve one workload together
    value = (ops_per_step / (ms / 1e3) if sharded else job_rate(ops_per_step, ms / 1e3, world)) / 1e9
    executed_dense = sum(s["dense_ops"] for s in st)
    results = {f"{label}:{g.names[0]}": q.count(g.names[0]) for (label, _), g, q in zip(grammars, gs, main.qs)}
    # every relation of the timed leg, for the check against the oracle below
    timed_pairs = [{nm: q.get(nm) for nm in g.names} for g, q in zip(gs, main.qs)]
    main.close()
    if sharded:
        dist.barrier()
    parity = check_against_oracle(graph, grammars, timed_pairs)

    # the same closure with the other schedules / product paths (exact results in all)
    alternatives = {}
    if not args.no_alternatives and not sharded:
        for name, (pth, sch, dns) in {"tensor_tile_skip": (eng.PATH_TENSOR, eng.SCHED_JACOBI, False),
                                      "tensor_inplace": (eng.PATH_TENSOR, eng.SCHED_INPLACE, True),
                                      "tensor_inplace_tile_skip": (eng.PATH_TENSOR, eng.SCHED_INPLACE, False),
                                      "auto_inplace": (eng.PATH_AUTO, eng.SCHED_INPLACE, False)}.items():
            if pth == path and sch == schedule and dns == dense:
                continue
            leg = Leg(eng, torch, graph, gs, pth, sch, stream, dns, args.tensor_kind)
            leg.step()
            ams = leg.time(max(2, min(args.steps, 5)))
            alternatives[name] = {"ms_per_step": ams, "value": world * ops_per_step / (ams / 1e3) / 1e9,
                                  "step_ms": {"best": min(leg.step_ms), "median": float(np.median(leg.step_ms)),
                                              "worst": max(leg.step_ms)},
                                  "iterations": [q.stats()["iterations"] for q in leg.qs],
                                  "tensor_products": sum(q.stats()["tensor_products"] for q in leg.qs),
                                  "gather_products": sum(q.stats()["gather_products"] for q in leg.qs),
                                  "tensor_ops_executed": sum(q.stats()["tensor_live_ops"] for q in leg.qs)}
            leg.close()
            if name == "tensor_tile_skip":
                r = roofline(eng, graph, gs, pth, sch, stream, dense=False, tkind=args.tensor_kind)
                alternatives[name]["roofline_executed"] = {k: r.get(k) for k in
                                                           ("achieved", "peak", "unit", "frac", "launches", "launch_ms")}

    if not args.no_alternatives and world == 1 and schedule == eng.SCHED_JACOBI and path != eng.PATH_WORKLIST:
        # the timed solve as two row blocks of a sharded solve, both on this device: the same
        # products split by rows, plus the per-execution export and import of the new pairs
        rb = RowBlockLeg(eng, torch, graph, gs, path, stream, dense, args.tensor_kind, 2)
        rbs = rb.time(max(2, min(args.steps, 3)))
        same = all(set(a) == set(b) and all(np.array_equal(a[k], b[k]) for k in a)
                   for a, b in zip(rb.relations(), timed_pairs))
        alternatives["row_blocks_2_one_gpu"] = {
            "ms_per_step": rbs, "value": ops_per_step / (rbs / 1e3) / 1e9, "executions": rb.executions,
            "relations_equal_timed_leg": bool(same),
            "note": "each query split into 2 row blocks (contexts), both on this GPU, new pairs exchanged as "
                    "records after every loop execution; the multi-GPU form runs one block per rank (NCCL)"}
        rb.close()
        if not same:
            print("bench: the row-block solve differs from the timed leg", file=sys.stderr)
            sys.exit(3)

    # e2e through the C ABI with host buffers: create (edge upload), solve, copy triples back
    h2d = graph.n_edges * 12 * len(grammars)
    d2h = 0
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    # untimed warm-up steps first (as for the device-timed loop): the first steps pay one-time
    # costs (the library's memory pool growing, first-touch of host pages)
    e2e_warmup = max(1, min(args.warmup, 2))
    e2e_times = []
    for it in range(e2e_warmup + e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if it >= e2e_warmup + 1:
            e2e_times.append(t0 - t_prev)
        t_prev = t0
        d2h = 0
        if sharded:  # this rank's row blocks created, the sharded solve, the whole closure copied back
            leg = RowBlockLeg(eng, torch, graph, gs, path, stream, dense, args.tensor_kind, world, rank,
                              shardmod.TorchExchange("cuda"))
            for q in leg.qs:
                d2h += q.triples_all().shape[0] * 12
            leg.close()
            continue
        for g in gs:
            q = eng.Query(g, graph.n, graph.edges, path=path, schedule=schedule, timeout_s=300.0, dense_tensor=dense,
                          tensor_kind=kind_code(eng, args.tensor_kind))
            q.solve()
            for nm in g.names:
                d2h += q.triples(nm).shape[0] * 12
            q.close()
    torch.cuda.synchronize()
    e2e_times.append(time.perf_counter() - t_prev)
    e2e_s = max_over_ranks(float(np.mean(e2e_times)))
    e2e_spread = {"best": min(e2e_times) * 1e3, "median": float(np.median(e2e_times)) * 1e3,
                  "worst": max(e2e_times) * 1e3}
    e2e_val = (ops_per_step / e2e_s if sharded else job_rate(ops_per_step, e2e_s, world)) / 1e9

    roof = roofline(eng, graph, gs, path, schedule, stream, dense, sm_mhz=clk.get("sm_mhz"), tkind=args.tensor_kind)

    # the default path of cfpq_solve (automatic product choice, in-place schedule): its
    # dominant kernels' roofline and its own end-to-end figure
    default_path = None
    if not args.no_alternatives and not sharded:
        droof = roofline(eng, graph, gs, eng.PATH_AUTO, eng.SCHED_INPLACE, stream, dense=False)
        d_d2h = 0
        d_steps = 5  # a few milliseconds each: more steps against host noise
        d_times = []
        for it in range(e2e_warmup + d_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d_d2h = 0
            for g in gs:
                q = eng.Query(g, graph.n, graph.edges, timeout_s=300.0)
                q.solve()
                d_d2h += q.triples_all().shape[0] * 12
                q.close()
            if it >= e2e_warmup:
                d_times.append(time.perf_counter() - t0)
        de2e_s = max_over_ranks(float(np.mean(d_times)))
        auto = alternatives.get("auto_inplace", {})
        default_path = {"options": "path auto, schedule in-place, tile skipping (the cfpq_solve defaults)",
                        "ms_per_step": auto.get("ms_per_step"), "value": auto.get("value"), "unit": "GOPS",
                        "roofline": droof,
                        "e2e": {"value": job_rate(ops_per_step, de2e_s, world) / 1e9, "unit": "GOPS",
                                "ms_per_step": de2e_s * 1e3, "h2d_bytes_per_step": h2d,
                                "d2h_bytes_per_step": d_d2h, "steps": d_steps, "warmup": e2e_warmup,
                                "step_ms": {"best": min(d_times) * 1e3, "median": float(np.median(d_times)) * 1e3,
                                            "worst": max(d_times) * 1e3}}}

    line = {
        "metric": METRIC, "value": value, "unit": "GOPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "step_ms_this_rank": step_ms, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": ("fp4e2m1" if effective_kind(args.tensor_kind) == "fp4" else "fp8e4m3") +
                 " 0/1 operands, f32 accumulate (tensor path); u32 bit-packed storage",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_NODES, "classes": N_CLASSES, "seed": SEED,
                   "grammars": [nm for nm, _ in grammars], "path": args.path, "schedule": args.schedule,
                   "tensor_products": args.tensor, "tensor_kind": effective_kind(args.tensor_kind),
                   "parallelism": f"row blocks x{world} (NCCL exchange)" if sharded else f"replicas x{world}",
                   "l2": "inputs larger than L2 (per query 3 x 7 x 32 MiB bit planes + 7 x 32 MiB transposes)",
                   "products_per_step": products, "dense_ops_executed_per_step": executed_dense,
                   "iterations": [s["iterations"] for s in st], "results_start_symbol": results},
        "e2e": {"value": e2e_val, "unit": "GOPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3, "steps": e2e_steps, "warmup": e2e_warmup, "step_ms": e2e_spread},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "roofline": roof,
        "parity": parity,
        "headline": "Algorithm 1 with every Boolean product on the tcgen05 tensor cores (dense products: the "
                    "work the metric counts is executed); the default path's figure is under default_path",
        "alternatives": alternatives,
    }
    if default_path:
        line["default_path"] = default_path
    if roof.get("useful_ops_per_step"):
        # Boolean ops whose operands are both 1 (sum_k nnz(col k of T_B) nnz(row k of T_C) per
        # product, counted in profile mode on the same closure), beside the dense count
        u = roof.pop("useful_ops_per_step")
        line["useful_work"] = {"ops_per_step": u, "fraction_of_dense": u / ops_per_step,
                               "gops": world * u / (ms / 1e3) / 1e9}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        reps = 0
        while True:
            oracle_step(graph, grammars)
            reps += 1
            if time.perf_counter() - t0 >= args.cpu_seconds:
                break
        per = (time.perf_counter() - t0) / reps
        line["cpu_baseline"] = {"value": ops_per_step / per / 1e9, "unit": "GOPS", "cores": 1, "kind": "oracle",
                                "sample": f"full workload x{reps} ({per * 1e3:.0f} ms per step), one host thread"}
        cpu_v = line["cpu_baseline"]["value"]
        line["vs_cpu_baseline"] = {"value": value / cpu_v, "e2e": e2e_val / cpu_v,
                                   "default_path": (default_path["value"] / cpu_v) if default_path else None,
                                   "default_path_e2e": (default_path["e2e"]["value"] / cpu_v) if default_path else None}
    if rank == 0 and world == 1 and not args.no_configs:
        line["configs"] = {
            "n1024_seeds": small_hierarchy_measure(eng, torch),
            "two_cycles": cycles_measure(eng, torch, 4096, 3, 1, cpu=not args.no_cpu_baseline),
            "batch256": batch_measure(eng, torch, 5, 3),
            "serve": serve_measure(eng),
        }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------------------ batched / served

def batch_measure(eng, torch, steps, warmup):
    """256 independent hierarchy queries (n log-uniform in [64, 4096], class fraction 0.3,
    grammar Q1 or sc-only uniformly, seed 0): one grouped persistent launch (built-in and
    autotuned launch configuration) vs the same queries solved one at a time with the
    single-query path."""
    work = synth.batch_queries(256, 64, 4096, 0.3, seed=0)
    gs = [eng.Grammar(t, g.labels) for g, t in work]
    qs = [eng.Query(gr, g.n, g.edges, path=eng.PATH_GATHER, schedule=eng.SCHED_AUTO) for (g, _), gr in zip(work, gs)]
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    default = eng.batch_tuning_default()
    for _ in range(warmup):
        eng.solve_batch(qs, stream, tuning=default)
    ms_default = timed(lambda: eng.solve_batch(qs, stream, tuning=default), steps)
    # the autotuner times candidate launch configurations on this batch and installs the best
    best, report = eng.autotune_batch(qs, stream)
    for _ in range(warmup):
        eng.solve_batch(qs, stream)
    ms_batch = timed(lambda: eng.solve_batch(qs, stream), steps)
    phases = eng.batch_last_profile()
    # bytes the products phase moves: the same batch once more with word counting on
    # (profile mode: scanned left rows, gathered right-row chunks, merged result chunks)
    prof_qs = [eng.Query(gr, g.n, g.edges, path=eng.PATH_GATHER, schedule=eng.SCHED_AUTO, profile=True)
               for (g, _), gr in zip(work, gs)]
    eng.solve_batch(prof_qs, stream)
    product_bytes = sum(q.stats()["product_bytes"] for q in prof_qs)
    for q in prof_qs:
        q.close()

    def serial():
        for q in qs:
            q.solve(stream)
    serial()
    ms_serial = timed(serial, max(1, min(steps, 3)))
    for q in qs:
        q.close()
    # a batch with dense members: 24 sparse hierarchy queries (n 64..1500) and five
    # block-diagonal closures of 2,048-8,192 nodes (communities of 512, S -> S S | t0): the
    # tuner may take size classes out of the grouped launch, to be solved alone beside it by
    # the single-query automatic path (tensor-core products with tile skipping where cheaper)
    dense_work = [(eng.Grammar(t, g.labels), g) for g, t in synth.batch_queries(24, 64, 1500, 0.3, seed=31)]
    for j, n in enumerate([2048, 3000, 4096, 6000, 8192]):
        g = synth.communities(n, max(1, n // 512), 2, seed=40 + j)
        dense_work.append((eng.Grammar("S S S\nS t0\n", g.labels), g))
    dqs = [eng.Query(gr, g.n, g.edges) for gr, g in dense_work]
    saved = eng.batch_tuning()
    for _ in range(warmup):
        eng.solve_batch(dqs, stream, tuning=default)
    d_default = timed(lambda: eng.solve_batch(dqs, stream, tuning=default), steps)
    d_best, d_report = eng.autotune_batch(dqs, stream)
    for _ in range(warmup):
        eng.solve_batch(dqs, stream, tuning=d_best)
    d_tuned = timed(lambda: eng.solve_batch(dqs, stream, tuning=d_best), steps)
    d_tensor = sum(q.stats()["tensor_products"] for q in dqs)
    for q in dqs:
        q.close()
    eng.set_batch_tuning(saved)
    dense_mix = {"workload": "24 hierarchy queries (n 64..1500) + 5 block-diagonal closures (n 2048..8192)",
                 "built_in_ms": d_default, "tuned_ms": d_tuned, "speedup": d_default / d_tuned,
                 "tuned_config": d_best.as_dict(), "tensor_products_tuned": d_tensor, "tuner": d_report}
    return {"queries_per_s": 256 / (ms_batch / 1e3), "ms_per_batch": ms_batch,
            "workload": "256 hierarchy queries, n log-uniform [64, 4096], class fraction 0.3, "
                        "Q1 or sc-only uniformly, seed 0",
            "path": "gather (grouped launch)",
            "launch_config": "autotuned on this batch (grid, tile width per size class, schedule)",
            "serial_ms": ms_serial, "serial_queries_per_s": 256 / (ms_serial / 1e3),
            "speedup_vs_serial": ms_serial / ms_batch,
            "built_in_config_ms": ms_default, "tuned_config": best.as_dict(), "tuner": report,
            "phase_ms": {k: (round(v, 3) if isinstance(v, float) else
                             ([round(x, 3) for x in v] if isinstance(v, list) else v)) for k, v in phases.items()},
            "products_phase": {"bytes": product_bytes,
                               "gbs": product_bytes / (phases["products"] * 1e6) if phases["products"] else None},
            "dense_mix": dense_mix}


def batch_arm(args):
    import torch

    import paper_1707_01007_b300 as eng

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    b = batch_measure(eng, torch, args.steps, args.warmup)
    line = {"metric": "queries/s, 256 batched hierarchy queries (closure to fixpoint)",
            "value": b["queries_per_s"], "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32 bit-packed", "data": "synthetic",
            "config": {"workload": b["workload"], "path": b["path"], "launch_config": b["launch_config"]}}
    line.update({k: v for k, v in b.items() if k not in ("workload", "path", "launch_config")})
    print(json.dumps(line))
    return 0


SERVE_ARRIVAL_SEEDS = (17, 18, 19)


def serve_measure(eng, count=2000, seeds=SERVE_ARRIVAL_SEEDS):
    """Poisson stream of `count` hierarchy queries (n log-uniform in [128, 32768], both
    grammars) plus one n = 65536 Query 1 query, at 0.7x and 1.5x the measured serial
    throughput: the continuous-batching server against serial FIFO solves of the same stream,
    one run per arrival draw (seeds), with the spread of p50 / p99 over the draws."""
    from paper_1707_01007_b300 import serve

    work = synth.batch_queries(count, 128, 32768, 0.3, seed=5)
    big = synth.hierarchy(65536, round(65536 * 0.3), seed=5)
    work = work[: count // 2] + [(big, synth.GRAMMAR_Q1)] + work[count // 2:]
    queries = [(eng.Grammar(t, g.labels), g.n, g.edges) for g, t in work]
    # serial throughput on the stream's first 200 queries, all available at time 0
    probe = queries[:200]
    sp = serve.run_serial(probe, np.zeros(len(probe)))
    thr = sp["queries_per_s"]
    out = {"workload": f"{len(queries)} hierarchy queries, n log-uniform [128, 32768] + one n=65536 Q1, "
                       "Poisson arrivals at 0.7x and 1.5x serial throughput",
           "serial_probe_queries_per_s": thr, "arrival_seeds": list(seeds), "rounds_per_step": 8}
    for load in (0.7, 1.5):
        runs = []
        for sd in seeds:
            arr = synth.poisson_arrivals(len(queries), rate_per_s=load * thr, seed=sd)
            srv = eng.Server(rounds_per_step=8)
            s_sum, _ = serve.run_server(srv, queries, arr)
            stats = srv.stats()
            srv.close()
            f_sum = serve.run_serial(queries, arr)
            runs.append({"seed": sd, "server": s_sum, "serial_fifo": f_sum, "server_launches": stats["launches"],
                         "server_steps": stats["steps"],
                         "server_host_ms": {k: stats[k] for k in ("admit_ms", "launch_ms", "retire_ms")},
                         "peak_hbm_bytes": stats["peak_used_bytes"], "budget_bytes": stats["budget_bytes"]})

        def spread(who, key):
            v = [r[who][key] for r in runs]
            return {"mean": float(np.mean(v)), "min": float(min(v)), "max": float(max(v))}
        out[f"load_{load}"] = {
            "runs": runs,
            "server": {k: spread("server", k) for k in ("queries_per_s", "p50_ms", "p99_ms", "mean_ms")},
            "serial_fifo": {k: spread("serial_fifo", k) for k in ("queries_per_s", "p50_ms", "p99_ms", "mean_ms")}}
    return out


def serve_arm(args):
    import torch

    import paper_1707_01007_b300 as eng

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    out = serve_measure(eng, count=2000 if args.n is None else args.n)
    top = out["load_1.5"]["server"]
    line = {"metric": "queries/s and p50/p99 latency, served Poisson stream", "value": top["queries_per_s"]["mean"],
            "unit": "queries/s", "n_gpus": 1, "steps": len(SERVE_ARRIVAL_SEEDS), "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32 bit-packed",
            "data": "synthetic", "config": {"workload": out["workload"], "rounds_per_step": 8}, "detail": out}
    print(json.dumps(line))
    return 0


def cycles_measure(eng, torch, p, steps, warmup, cpu=True):
    """Two directed cycles of p and p - 1 nodes sharing node 0, S -> a S b | a b: closure by
    the worklist path (on-device) and by the automatic path (matrix loop, then the hand-over
    to the worklist), timed with CUDA events inside the library (solve_ms); the results are
    checked against the closed form R_S = R_S1 = (a-cycle) x (b-cycle). The set-up of the
    worklist path (CSR adjacency of the static relations, unique-successor and period power
    tables, built by kernels from the seeded matrices) runs when the context is created
    (worklist path) or at the first hand-over (automatic path); its wall time
    (cfpq_stats.worklist_setup_ms) is reported beside the solve times."""
    q = p - 1
    graph = synth.two_cycles(p, q)
    g = eng.Grammar(synth.GRAMMAR_C3, graph.labels)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qy = eng.Query(g, graph.n, graph.edges, path=eng.PATH_WORKLIST, timeout_s=600.0)
    torch.cuda.synchronize()
    create_ms = (time.perf_counter() - t0) * 1e3
    for _ in range(max(1, min(warmup, 1))):
        qy.solve(stream)
    times = []
    for _ in range(max(1, min(steps, 3))):
        qy.solve(stream)
        times.append(qy.stats()["solve_ms"])
    ok = qy.count("S") == p * q and qy.count("S1") == p * q
    st = qy.stats()
    setup_ms = st["worklist_setup_ms"]
    ms = float(np.median(times))
    qy.close()
    qa = eng.Query(g, graph.n, graph.edges, path=eng.PATH_AUTO, timeout_s=600.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qa.solve(stream)  # the first solve builds the worklist tables at the hand-over
    torch.cuda.synchronize()
    first_ms = (time.perf_counter() - t0) * 1e3
    auto_times = []
    for _ in range(max(1, min(steps, 3))):
        qa.solve(stream)
        auto_times.append(qa.stats()["solve_ms"])
    auto = {"ms": float(np.median(auto_times)), "loop_executions_before_hand_over": qa.stats()["iterations"],
            "first_solve_wall_ms_with_setup": first_ms, "worklist_setup_ms": qa.stats()["worklist_setup_ms"],
            "closed_form_count_ok": bool(qa.count("S") == p * q)}
    qa.close()
    out = {"workload": f"two cycles {p} / {q} sharing node 0, S -> a S b | a b (n = {graph.n})",
           "worklist_ms": ms, "pairs_S": p * q if ok else None, "closed_form_count_ok": bool(ok),
           "worklist_items": st["worklist_items"], "ns_per_item": ms * 1e6 / max(1, st["worklist_items"]),
           "worklist_create_wall_ms": create_ms, "worklist_setup_ms": setup_ms, "automatic_path": auto}
    if cpu:
        import oracle
        t0 = time.perf_counter()
        oracle.hellings(graph, synth.GRAMMAR_C3)
        out["cpu_baseline"] = {"value": time.perf_counter() - t0, "unit": "s", "cores": 1, "kind": "oracle",
                               "sample": "full workload once, one host thread"}
    return out


def cycles_arm(args):
    import torch

    import paper_1707_01007_b300 as eng

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    p = args.cycle_p or 4096
    c = cycles_measure(eng, torch, p, args.steps, args.warmup, cpu=not args.no_cpu_baseline)
    line = {"metric": "two-cycle closure time (worklist path)", "value": c["worklist_ms"] / 1e3, "unit": "s",
            "n_gpus": 1, "steps": max(1, min(args.steps, 3)), "warmup": 1, "ms_per_step": c["worklist_ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32 bit-packed",
            "data": "synthetic", "config": {"workload": c["workload"]}}
    line.update({k: v for k, v in c.items() if k != "workload"})
    print(json.dumps(line))
    return 0


def small_hierarchy_measure(eng, torch, seeds=range(5), reps=5):
    """Query 1 on the hierarchy of n = 1024 nodes (300 classes), one per seed: Algorithm 1's
    loop count, and the solve time (CUDA events inside the library, median of reps) of the
    automatic path and of Algorithm 1 with dense tensor-core products, with the Boolean GOPS
    of the latter (loop executions x productions x 2 n^3 / time)."""
    n, c = 1024, 300
    stream = torch.cuda.current_stream()
    per = []
    for sd in seeds:
        graph = synth.hierarchy(n, c, seed=sd)
        g = eng.Grammar(synth.GRAMMAR_Q1, graph.labels)
        nprod = len({(g.cnf.contents.binary[i].lhs, g.cnf.contents.binary[i].b, g.cnf.contents.binary[i].c)
                     for i in range(g.cnf.contents.n_binary)})
        row = {"seed": sd}
        for label, kw in (("auto", dict(path=eng.PATH_AUTO)),
                          ("tensor_dense_jacobi", dict(path=eng.PATH_TENSOR, schedule=eng.SCHED_JACOBI,
                                                       dense_tensor=True))):
            q = eng.Query(g, graph.n, graph.edges, timeout_s=60.0, **kw)
            q.solve(stream)
            ts = []
            for _ in range(reps):
                q.solve(stream)
                ts.append(q.stats()["solve_ms"])
            row[label + "_ms"] = float(np.median(ts))
            if label == "tensor_dense_jacobi":
                row["jacobi_iterations"] = q.stats()["iterations"]
                row["tensor_gops"] = q.stats()["iterations"] * nprod * 2.0 * n ** 3 / (row[label + "_ms"] / 1e3) / 1e9
            row["pairs_S_" + label] = q.count("S")
            q.close()
        per.append(row)
    return {"workload": "hierarchy n=1024 (300 classes), Query 1, seeds 0-4", "per_seed": per,
            "auto_ms_median": float(np.median([r["auto_ms"] for r in per])),
            "tensor_dense_jacobi_ms_median": float(np.median([r["tensor_dense_jacobi_ms"] for r in per]))}


def lengths_arm(args):
    """Single-path semantics (Section 5) on the n = 16384 hierarchy: Query 1 and the
    same-generation query with a length per pair, Jacobi schedule, automatic product path.
    Reported: the device time of the closure with lengths, the same closure without them, the
    length kernels' own time and splits (profile mode), and Query 1's pairs and lengths checked
    one by one against the oracle (whose run is the CPU baseline)."""
    import torch

    import paper_1707_01007_b300 as eng

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    graph, _ = workload()
    stream = torch.cuda.current_stream()
    queries = [("Q1", synth.GRAMMAR_Q1), ("SG", synth.GRAMMAR_SG)]
    per, total_ms, kept = {}, 0.0, {}
    for nm, text in queries:
        g = eng.Grammar(text, graph.labels)
        mk = lambda **kw: eng.Query(g, graph.n, graph.edges, path=eng.PATH_AUTO, schedule=eng.SCHED_JACOBI,
                                    timeout_s=600.0, **kw)
        out = {}
        for label, q in (("with_lengths", mk(lengths=True)), ("without", mk())):
            for _ in range(args.warmup):
                q.solve(stream)
            ts = []
            for _ in range(args.steps):
                q.solve(stream)
                ts.append(q.stats()["solve_ms"])
            out[label + "_ms"] = float(np.median(ts))
            if label == "with_lengths":
                kept[nm] = (g, q)
        qp = mk(lengths=True, profile=True)
        qp.solve(stream)
        st = qp.stats()
        out.update({"iterations": st["iterations"], "new_pairs": st["new_bits"], "lengths_kernel_ms": st["lengths_ms"],
                    "lengths_launches": st["lengths_launches"], "splits": st["lengths_splits"],
                    "ns_per_new_pair": st["lengths_ms"] * 1e6 / max(1, st["new_bits"])})
        qp.close()
        per[nm] = out
        total_ms += out["with_lengths_ms"]
    line = {"metric": "single-path closure time (Query 1 + same-generation query, lengths per pair)",
            "value": total_ms / 1e3, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32 bit-packed + u32 lengths", "data": "synthetic",
            "config": {"workload": f"hierarchy n={N_NODES} ({N_CLASSES} classes, seed {SEED}), Query 1 + "
                                   "same-generation query, single-path lengths, Jacobi schedule, automatic path"},
            "queries": per}
    if not args.no_cpu_baseline:
        import oracle
        g, q = kept["Q1"]
        t0 = time.perf_counter()
        cnf, L, _ = oracle.single_path_lengths(graph, synth.GRAMMAR_Q1)
        dt = time.perf_counter() - t0
        same = True
        for a, name in enumerate(cnf.names):
            pairs, lens = q.lengths(name)
            got = {(int(m), int(n)): int(l) for (m, n), l in zip(pairs.tolist(), lens.tolist())}
            same &= got == L[a]
        line["parity_Q1_vs_oracle"] = bool(same)
        line["cpu_baseline"] = {"value": dt, "unit": "s", "cores": 1, "kind": "oracle",
                                "sample": "Query 1 only (the same-generation query takes minutes), one host thread"}
    print(json.dumps(line))
    return 0


def blockdiag_arm(args):
    """A transitive closure (S -> S S | t0) over 64 communities of 512 nodes, n = 32768: the
    matrices are block-diagonal, so tensor products with tile skipping execute 0.1 % of the
    dense product. The automatic path (cost model pricing the live K steps once the tile
    counts are known) against the gather alone and the tensor path alone; results checked
    equal between them (and, with the CPU baseline, against the oracle)."""
    import torch

    import paper_1707_01007_b300 as eng

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    graph = synth.communities(32768, 64, 2, seed=4)
    text = "S S S\nS t0\n"
    g = eng.Grammar(text, graph.labels)
    stream = torch.cuda.current_stream()
    legs, first = {}, None
    for name, kw in (("auto", dict(path=eng.PATH_AUTO)), ("gather", dict(path=eng.PATH_GATHER)),
                     ("tensor_tile_skip", dict(path=eng.PATH_TENSOR)),
                     ("tensor_tile_skip_jacobi", dict(path=eng.PATH_TENSOR, schedule=eng.SCHED_JACOBI))):
        q = eng.Query(g, graph.n, graph.edges, timeout_s=300.0, **kw)
        for _ in range(max(1, args.warmup)):
            q.solve(stream)
        ts = []
        for _ in range(max(1, args.steps)):
            q.solve(stream)
            ts.append(q.stats()["solve_ms"])
        st = q.stats()
        got = q.get("S")
        if first is None:
            first = got
        elif not np.array_equal(got, first):
            print(f"bench: {name} differs from the automatic path", file=sys.stderr)
            return 3
        legs[name] = {"ms": float(np.median(ts)), "iterations": st["iterations"],
                      "tensor_products": st["tensor_products"], "gather_products": st["gather_products"],
                      "tensor_live_fraction": (st["tensor_live_ops"] / st["dense_ops"]) if st["dense_ops"] else None}
        q.close()
    line = {"metric": "closure time, block-diagonal transitive closure", "value": legs["auto"]["ms"] / 1e3,
            "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": legs["auto"]["ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32 bit-packed",
            "data": "synthetic",
            "config": {"workload": "64 communities of 512 nodes (n = 32768, 2 out-edges per node inside its "
                                   "community), S -> S S | t0"},
            "pairs_S": int(first.shape[0]), "paths": legs,
            "speedup_vs_gather": legs["gather"]["ms"] / legs["auto"]["ms"]}
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        ref = oracle.hellings(graph, text)
        line["cpu_baseline"] = {"value": time.perf_counter() - t0, "unit": "s", "cores": 1, "kind": "oracle",
                                "sample": "full workload once, one host thread"}
        if not np.array_equal(ref.pairs("S"), first):
            print("bench: the closure differs from the oracle", file=sys.stderr)
            return 3
        line["parity"] = {"reference": "oracle", "equal": True}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batch256":
        return batch_arm(args)
    if args.workload == "serve":
        return serve_arm(args)
    if args.workload == "cycles":
        return cycles_arm(args)
    if args.workload == "lengths16k":
        return lengths_arm(args)
    if args.workload == "blockdiag32k":
        return blockdiag_arm(args)
    return engine_arm(args)


if __name__ == "__main__":
    sys.exit(main())
