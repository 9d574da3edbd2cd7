#!/usr/bin/env python3
"""Throughput of the uplink receiver hot path on GB300: MMSE-detected REs/s.

One step = one pass of the whole path over one batch: DMRS LS estimation (phy_chest), then
interpolation, Gram and matched-filter products (tensor cores in the headline form), Cholesky,
solves, SINR and max-log LLRs for 8 cells x 273 PRB x 14 symbols, 64 Rx x 16 layers, 256-QAM,
Kronecker rho = 0.7 (the massive-MIMO workload). The headline runs that workload as it is
specified: FP16 tensor-core products with FP32 accumulation, FP32 Cholesky/solve/LLR, FP64
re-computation of ill-conditioned REs. Plain FP32 and BF16 products are timed beside it on the same
inputs (`variants`, `vs_plain_fp32`). Inputs are seeded synthetic slots resident in HBM. Prints
one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import tempfile
import sys
import time

# The oracle baseline runs single-threaded numpy; pin BLAS before numpy loads.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_07843_gb300 import synth as S  # noqa: E402

METRIC = "MMSE-detected REs/s (64Rx×16L, 273 PRB) & p99 slot latency vs plain FP32"


def workload(name: str) -> S.SlotSpec:
    if name == "massive":
        return S.spec_massive_mimo()
    if name == "carrier":
        return S.spec_carrier_273prb(n_cells=8)
    if name == "small":
        return S.spec_small_51prb(n_cells=8)
    raise SystemExit(f"unknown workload {name}")


def rank_seed(rank: int) -> int:
    """Each rank draws its own cells (weak scaling: every rank owns a full batch)."""
    return 3000 + 1000 * rank


def max_over_ranks(ms: float, device=None) -> float:
    """The slowest rank's time (the job's time); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, steps: int, ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank's time."""
    return world * units_per_rank * steps / (ms / 1e3)


def anchor_bytes(spec: S.SlotSpec) -> int:
    n_comb = spec.n_sc // 2
    G = -(-n_comb // spec.occ)
    return spec.n_cells * len(spec.dmrs_sym) * G * spec.n_layers * spec.n_rx * 8


def n_data_res(spec: S.SlotSpec) -> int:
    return spec.n_cells * spec.n_sc * len(spec.data_sym)


def algorithmic_bytes(spec: S.SlotSpec) -> dict:
    """Bytes the path must move once per step: the grid and pilots in, every output out."""
    C, K, R, L, qm = spec.n_cells, spec.n_sc, spec.n_rx, spec.n_layers, spec.qm
    J, nd = len(spec.data_sym), len(spec.dmrs_sym)
    y_data = C * J * R * K * 8
    y_dmrs = C * nd * R * K * 8
    pilots = C * nd * L * K * 8
    n_re = C * J * K
    outs = n_re * (L * 8 + L * 4 + L * qm * 4 + 1)
    return dict(y_data=y_data, y_dmrs=y_dmrs, pilots=pilots, outputs=outs,
                step=y_data + y_dmrs + pilots + outs)


def detect_chunks(spec: S.SlotSpec) -> int:
    """Chunks of cells the detection stage runs in (two kernel launches each) with the full
    phy_workspace_size() workspace: the library prefers chunks whose intermediates (Gram blocks
    and matched filter) stay within 256 MiB (PHY_CHUNK_MB overrides)."""
    nl = next(c for c in (2, 4, 8, 16) if spec.n_layers <= c)
    n_comb = spec.n_sc // 2
    n_seg = max(-(-n_comb // spec.occ) - 1, 1)
    J = len(spec.data_sym)
    per_cell = n_seg * J * nl * (nl + 1) // 2 * 32 + J * spec.n_sc * nl * 8
    budget = int(os.environ.get("PHY_CHUNK_MB", "256")) << 20
    chunk = min(max(1, budget // per_cell), spec.n_cells)
    return -(-spec.n_cells // chunk)


def detect_flops(spec: S.SlotSpec) -> dict:
    """Floating-point operations of the segment-factored LMMSE per launch (FMA = 2).

    Counts what the method needs, not what the kernels issue: Hermitian halves only, no layer
    padding. 'products': per segment the corner cross-Gram X = C^H C (NX = 2 n_dmrs n_layers,
    Hermitian) and per RE the matched filter (two n_rx x n_layers products against the
    time-interpolated anchors); these run on the tensor cores in the TF32/FP16/BF16 variants.
    'solve': per segment and data symbol the time folding of X, per RE the weighted Gram,
    Cholesky (n^3/6 complex MACs), forward and backward solves (n^2), the inverse diagonal
    (n^3/6 + n^2/2), SINR and the max-log demapper (H folds per axis).
    """
    nr, nl, qm = spec.n_rx, spec.n_layers, spec.qm
    nd = len(spec.dmrs_sym)
    L = spec.occ
    n_comb = spec.n_sc // 2
    G = -(-n_comb // L)
    n_seg = max(G - 1, 1)
    J = len(spec.data_sym)
    cm = 8.0  # flops per complex multiply-add
    nx = 2 * nd * nl
    n_re = n_data_res(spec)
    products = spec.n_cells * n_seg * nx * (nx + 1) / 2 * nr * cm + n_re * 2 * nl * nr * cm
    per_seg_sym = (2 * nl * (nl + 1) / 2 + nl * nl) * (4 if nd == 2 else 1) * 4
    per_re = (nl * 6 + nl * (nl + 1) / 2 * 4 * 6
              + (nl ** 3 / 6) * cm + nl ** 2 * cm + (nl ** 3 / 6 + nl ** 2 / 2) * cm
              + nl * 10 + nl * 2 * (qm // 2) * 8)
    solve = spec.n_cells * n_seg * J * per_seg_sym + n_re * per_re
    return {"products": products, "solve": solve}


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, log_dir: str = ""):
        self.idx = gpu_index
        self.proc = None
        self.path = None
        self.log_dir = log_dir  # keep the raw samples there; "" = a temporary file

    def start(self):
        try:
            if self.log_dir:
                os.makedirs(self.log_dir, exist_ok=True)
                self.path = os.path.join(self.log_dir, f"clocks_bench_{os.getpid()}.csv")
                self.temp = False
            else:
                fd, self.path = tempfile.mkstemp(prefix="clocks_bench_", suffix=".csv")
                os.close(fd)
                self.temp = True
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if self.temp:
            os.remove(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# profiles: DRAM traffic of the dominant kernel from a committed ncu summary
# ---------------------------------------------------------------------------------------------

# translation unit that defines each profiled kernel
KERNEL_SOURCE = {"seg_prep_tc": "detect_tc.cu", "re_solve": "detect_fp32.cu",
                 "seg_prep_fp32": "detect_fp32.cu", "chest": "chest.cu"}


def kernel_source_hash(kernel: str) -> str:
    """Hash of the device code a kernel is built from: its translation unit and every local
    .cuh header it includes, transitively (the .h headers on the way, the C ABI and the host
    launchers' declarations, are followed but not hashed: they hold no device code).

    Counters recorded for one hash stay valid while none of those files changes."""
    csrc = os.path.join(ROOT, "paper_2510_07843_gb300", "csrc")
    seen, todo = [], [os.path.join(csrc, KERNEL_SOURCE[kernel])]
    while todo:
        path = os.path.normpath(todo.pop())
        if path in seen:
            continue
        seen.append(path)
        for line in open(path):
            m = re.match(r'\s*#include\s+"([^"]+)"', line)
            if m:
                todo.append(os.path.join(os.path.dirname(path), m.group(1)))
    h = hashlib.sha256()
    for path in sorted(seen):
        if path.endswith(".h"):
            continue
        h.update(os.path.relpath(path, ROOT).encode())
        h.update(open(path, "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, workload_name: str):
    """Per-launch DRAM bytes from profiles/traffic.txt if recorded for the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash(kernel)
    for line in open(path):
        p = line.split()
        if len(p) >= 4 and not line.startswith("#") and p[0] == kernel and p[1] == workload_name \
                and p[3] == src:
            return float(p[2])
    return None


# ---------------------------------------------------------------------------------------------
# oracle baseline
# ---------------------------------------------------------------------------------------------

ORACLE_CHUNK = 256  # subcarriers of one data symbol per oracle detection call


def oracle_chunk_res(spec: S.SlotSpec, anchors, slot, chunk: int) -> int:
    """Detect one chunk (data symbol chunk % J, subcarriers 256 (chunk // J) ...) of cell 0."""
    from oracle import phy_oracle as O
    data = spec.data_sym
    j = chunk % len(data)
    k0 = (chunk // len(data)) * ORACLE_CHUNK % spec.n_sc
    ks = np.arange(k0, min(k0 + ORACLE_CHUNK, spec.n_sc))
    O.detect_res(anchors[0], slot.Y[0], spec.dmrs_sym, spec.n_layers, spec.occ, spec.qm,
                 float(slot.sigma2[0]), data[j], ks)
    return int(ks.size)


def oracle_sample_rate(spec: S.SlotSpec, slot, budget_s: float) -> dict:
    """Time the FP64 oracle on one core on a bounded sample of the workload: LS estimation of
    cell 0, then detection of whole data symbols of cell 0, 256 subcarriers at a time, until
    budget_s."""
    from oracle import phy_oracle as O
    t0 = time.perf_counter()
    anchors = O.ls_anchors(slot.Y[:1], slot.pilots[:1], spec.dmrs_sym, spec.n_layers, spec.occ)
    n = chunks = 0
    while True:
        n += oracle_chunk_res(spec, anchors, slot, chunks)
        chunks += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n / dt, "res": n, "seconds": dt, "cores": 1}


_ORACLE_WORKER = {}


def _oracle_worker_init(spec: S.SlotSpec, seed: int):
    """Pool worker set-up (untimed): its own copy of cell 0 and its LS anchors."""
    from oracle import phy_oracle as O
    sl = S.make_slot(dataclasses.replace(spec, n_cells=1), seed, keep_h=False)
    _ORACLE_WORKER.update(spec=spec, slot=sl, anchors=O.ls_anchors(
        sl.Y[:1], sl.pilots[:1], spec.dmrs_sym, spec.n_layers, spec.occ))


def _oracle_worker_run(arg) -> int:
    """Detect chunks first, first + stride, ... until the wall-clock deadline; REs detected."""
    first, stride, deadline = arg
    w = _ORACLE_WORKER
    n, c = 0, first
    while time.time() < deadline:
        n += oracle_chunk_res(w["spec"], w["anchors"], w["slot"], c)
        c += stride
    return n


class OraclePool:
    """The oracle on every core this process may use (os.sched_getaffinity): one spawned worker
    process per core, each detecting its own share of cell 0's chunks. Spawned (not forked), so
    it is safe next to a CUDA context."""

    def __init__(self, spec: S.SlotSpec, seed: int):
        import multiprocessing as mp
        self.cores = len(os.sched_getaffinity(0))
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init,
                                                 initargs=(spec, seed))
        # every worker set up before the first timing
        self.pool.map(_oracle_worker_run, [(0, 1, 0.0)] * self.cores, chunksize=1)

    def rate(self, budget_s: float) -> dict:
        t0 = time.time()
        deadline = t0 + budget_s
        ns = self.pool.map(_oracle_worker_run,
                           [(w, self.cores, deadline) for w in range(self.cores)], chunksize=1)
        dt = time.time() - t0
        return {"value": sum(ns) / dt, "res": int(sum(ns)), "seconds": dt, "cores": self.cores}

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(spec: S.SlotSpec, budget_s: float) -> dict:
    """The oracle as it stands on the host cores: one core (LS of cell 0 included) and every
    allowed core (workers set up outside the timing), each for about budget_s / 2."""
    half = max(budget_s / 2.0, 1.0)
    one = oracle_sample_rate(spec, S.make_slot(dataclasses.replace(spec, n_cells=1), 3000,
                                               keep_h=False), half)
    pool = OraclePool(spec, 3000)
    try:
        allc = pool.rate(half)
    finally:
        pool.close()
    return {"value": allc["value"], "unit": "REs/s", "cores": allc["cores"], "kind": "oracle",
            "sample": f"cell 0 of the workload, whole data symbols {ORACLE_CHUNK} subcarriers at "
                      f"a time, numpy float64: {allc['res']} REs in {allc['seconds']:.1f} s on "
                      f"{allc['cores']} worker processes (one per allowed core, LS done per "
                      f"worker before the timing); single core {one['value']:.0f} REs/s "
                      f"({one['res']} REs in {one['seconds']:.1f} s, LS included)",
            "single_core": {"value": one["value"], "cores": 1, "res": one["res"],
                            "seconds": one["seconds"]},
            "all_cores": {"value": allc["value"], "cores": allc["cores"], "res": allc["res"],
                          "seconds": allc["seconds"]}}


# ---------------------------------------------------------------------------------------------
# measured arithmetic peaks
# ---------------------------------------------------------------------------------------------

def measured_fma_peaks(dev, st) -> dict:
    """FMA throughput of this GPU, measured in-process by the library's probe kernel (8 CTAs of
    256 threads per SM, eight independent chains per thread), CUDA events, best of 5 launches
    after 2 warm-up launches: FP32 (fma.rn.f32), FP32 pairs (fma.rn.f32x2) and FP64."""
    import torch
    from paper_2510_07843_gb300 import phy
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(512, dtype=torch.float64, device=dev)
    out = {"sm_count": sms, "how": "phy_fma_probe, 8 x 256-thread CTAs per SM, best of 5"}
    for kind, iters in (("fp32", 4096), ("fp32x2", 2048), ("fp64", 64)):
        best = 0.0
        for rep in range(7):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fl = phy.fma_probe(kind, 8 * sms, iters, sink, stream=st)
            b.record(st)
            torch.cuda.synchronize()
            if rep >= 2:
                best = max(best, fl / (a.elapsed_time(b) * 1e-3) / 1e12)
        out[f"{kind}_tflops"] = best
    return out


# ---------------------------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="massive", choices=["massive", "carrier", "small"])
    ap.add_argument("--cells", type=int, default=0,
                    help="override the workload's cells per GPU (smaller cases for profiling)")
    ap.add_argument("--precision", default="fp16", choices=["fp32", "tf32", "fp16", "bf16"],
                    help="products of the headline step (the massive configuration specifies "
                         "FP16/BF16 tensor-core products with an FP32 solve)")
    ap.add_argument("--variants", default="fp32,bf16",
                    help="other precisions timed on the same workload ('' for none)")
    ap.add_argument("--no-refactor", action="store_true",
                    help="headline without the FP64 re-computation of flagged REs")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle timing")
    ap.add_argument("--llr", default="f32", choices=["f32", "f16"], help="LLR output format")
    ap.add_argument("--streams", type=int, default=4,
                    help="streams the pipelined steps rotate over (1: strictly serial)")
    ap.add_argument("--serving-lanes", type=int, default=2,
                    help="slot batches the serving run keeps in flight")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop latency run")
    ap.add_argument("--no-noise", action="store_true",
                    help="skip the noise-variance estimate timing")
    ap.add_argument("--no-bfp", action="store_true",
                    help="skip the block-floating-point fronthaul timing")
    ap.add_argument("--clock-log", default="", metavar="DIR",
                    help="keep the raw nvidia-smi clock samples of the timed region in DIR")
    ap.add_argument("--no-cnn", action="store_true",
                    help="skip training and evaluating the learned channel denoiser")
    ap.add_argument("--aux-probe", type=int, default=0, metavar="REPS",
                    help="only time the auxiliary paths (noise estimate, BFP decoder, denoiser)")
    ap.add_argument("--batch-probe", type=int, default=0, metavar="JOBS",
                    help="only time batches of JOBS jobs of the serving mix through the batched "
                         "receiver (1 to 64; small enough to run under ncu)")
    ap.add_argument("--cnn-slots", type=int, default=24,
                    help="generated 12-PRB training slots for the denoiser (3,072 tiles each; "
                         "651 slots = 2.0 M tiles)")
    ap.add_argument("--cnn-epochs", type=int, default=8)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default tile shapes (no tuning launches before the timing; "
                         "for launch-list captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    spec = workload(args.workload)
    if args.cells > 0:
        spec = dataclasses.replace(spec, n_cells=args.cells)
    if args.impl == "reference":
        return run_reference(args, spec, rank, world)
    if args.aux_probe:
        return aux_probe(spec, args.aux_probe)
    if args.batch_probe:
        return batch_probe(args.batch_probe, max(args.steps, 1))
    return run_ours(args, spec, rank, world, local)


def aux_probe(spec, reps: int) -> int:
    """Times the auxiliary paths alone (CUDA events, `reps` calls each after two warm-up calls):
    the noise estimate and the 9-bit BFP decoder on `spec` (use --cells to size it), the
    denoiser forward pass (FP32, then BF16 on the tensor cores) on 16,384 tiles and its training
    step on 1,024 tiles. Small enough to run under ncu; prints one JSON line."""
    import torch
    from paper_2510_07843_gb300 import denoise as D
    from paper_2510_07843_gb300 import phy
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(2):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps * 1e3

    sl = S.make_slot(spec, 3000, keep_h=False)
    cfg = phy.SlotConfig.from_spec(spec, precision="fp16")
    b = phy.SlotBuffers(cfg, device=dev)
    b.Y.copy_(torch.from_numpy(sl.Y))
    b.pilots.copy_(torch.from_numpy(sl.pilots))
    b.sigma2.copy_(torch.from_numpy(sl.sigma2))
    phy.chest(cfg, b.Y, b.pilots, b.anchors)
    s2 = torch.empty(spec.n_cells, device=dev)
    out = {"noise_est_us": timed(lambda: phy.noise_est(cfg, "min", b.anchors, b.pilots, s2,
                                                        b.workspace))}
    c = torch.from_numpy(S.bfp_compress(sl.Y, 9, 2.0 ** -10)).to(dev)
    Yd = torch.empty_like(b.Y)
    out["bfp_decompress_us"] = timed(lambda: phy.bfp_decompress(cfg, c, 9, 2.0 ** -10, Yd))
    rng = np.random.default_rng(0)
    n = 16384
    p = torch.from_numpy(D.init_params(0) + (0.01 * rng.standard_normal(19682)).astype(
        np.float32)).to(dev)
    x = torch.from_numpy(rng.standard_normal((n, 2, 14, 12)).astype(np.float32)).to(dev)
    y = torch.empty_like(x)
    ws = torch.empty(phy.cnn_workspace_size(n), dtype=torch.uint8, device=dev)
    out["cnn_forward_us_16384_tiles"] = timed(lambda: phy.cnn_forward(n, p, x, y, ws))
    err = torch.zeros(64, dtype=torch.int32, device=dev)
    out["cnn_forward_bf16_tc_us_16384_tiles"] = timed(
        lambda: phy.cnn_forward_bf16(n, p, x, y, err))
    if int(err[0].item()) != 0:
        raise RuntimeError("tensor-core denoiser forward: a bounded wait ran out")
    nb = 1024
    m, v, g = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    wsb = torch.empty(phy.cnn_workspace_size(nb), dtype=torch.uint8, device=dev)
    step = [0]

    def train():
        step[0] += 1
        phy.cnn_train_step(nb, p, m, v, step[0], 1e-4, x[:nb], y[:nb], g, None, None, wsb)

    out["cnn_train_step_us_1024_tiles"] = timed(train)
    print(json.dumps(out))
    return 0


def run_reference(args, spec, rank, world):
    """The oracle (the FP64 CPU definition of the method) timed on this host's cores: one spawned
    worker per allowed core, each step a bounded sample of the workload."""
    if rank != 0:
        return 0
    per_step = max(args.cpu_budget / max(args.steps + args.warmup, 1), 0.5)
    pool = OraclePool(spec, 3000)
    try:
        for _ in range(args.warmup):
            pool.rate(per_step)
        vals, secs, res = [], 0.0, 0
        for _ in range(args.steps):
            r = pool.rate(per_step)
            vals.append(r["value"])
            secs += r["seconds"]
            res += r["res"]
    finally:
        pool.close()
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "REs/s", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(spec, args, world),
        "cpu_baseline": {"value": value, "unit": "REs/s", "cores": pool.cores, "kind": "oracle",
                         "sample": f"cell 0 of the workload, whole data symbols {ORACLE_CHUNK} "
                                   f"subcarriers at a time, {per_step:.1f} s per step on "
                                   f"{pool.cores} worker processes (one per allowed core); "
                                   f"{res} REs over the timed steps"},
        "e2e": {"value": value, "unit": "REs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_dict(spec, args, world):
    return {"workload": f"{args.workload}: {spec.n_cells} cells x {spec.n_prb} PRB x "
                        f"{spec.n_sym} sym, {spec.n_rx} Rx x {spec.n_layers} layers, "
                        f"{2 ** spec.qm}-QAM, DMRS {list(spec.dmrs_sym)}",
            "n_cells_per_gpu": spec.n_cells, "n_prb": spec.n_prb, "n_rx": spec.n_rx,
            "n_layers": spec.n_layers, "qm": spec.qm, "snr_db": spec.snr_db,
            "precision": f"{args.precision} products on tensor cores, FP32 accumulation, "
                         f"FP32 Cholesky/solve/LLR"
                         + ("" if args.no_refactor else ", FP64 re-computation of flagged REs")
            if args.precision != "fp32" else "fp32 throughout",
            "llr_format": args.llr,
            "pipelining": (f"{args.streams} streams: consecutive steps overlap, own buffers"
                           if args.streams > 1 else "serial"),
            "parallelism": f"replicas x{world} (cells per rank)",
            "l2": "working set per step larger than the 129 MB L2 (no flush needed)"}


def noise_estimate_run(cfg, spec, buf, st, reps: int = 50) -> dict:
    """Noise-variance estimate (phy_noise_est, 'min' mode) on the step's LS anchors: CUDA-event
    time per call (two launches; the anchors are L2-resident, as right after the LS stage) and
    the estimates against the noise level the grid was drawn with."""
    import torch
    from paper_2510_07843_gb300 import phy
    s2 = torch.empty(spec.n_cells, dtype=torch.float32, device=buf.Y.device)
    phy.chest(cfg, buf.Y, buf.pilots, buf.anchors, stream=st)

    def call():
        phy.noise_est(cfg, "min", buf.anchors, buf.pilots, s2, buf.workspace, stream=st)

    for _ in range(3):
        call()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        call()
    b.record(st)
    torch.cuda.synchronize()
    est = s2.cpu().numpy().astype(np.float64)
    return {"api": "phy_noise_est", "mode": "min", "us_per_call": a.elapsed_time(b) / reps * 1e3,
            "launches_per_call": 2, "sigma2_true": spec.sigma2,
            "estimate_rel_err_max": float(np.max(np.abs(est / spec.sigma2 - 1.0)))}


def bfp_run(cfg, spec, slot, buf, st, hbm_peak: float, iq_width: int = 9, reps: int = 20) -> dict:
    """Block-floating-point fronthaul input (9-bit mantissas) on the same batch: decompression of
    the whole grid (stream read + grid written, inputs larger than L2) and the receiver fed from
    the stream (phy_slot_run_bfp) next to the grid-fed one, CUDA events on the launch stream."""
    import torch
    from paper_2510_07843_gb300 import phy
    scale = 2.0 ** -10
    c = torch.from_numpy(S.bfp_compress(slot.Y, iq_width, scale)).to(buf.Y.device)
    Yd = torch.empty_like(buf.Y)

    def timed(fn):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    dec_ms = timed(lambda: phy.bfp_decompress(cfg, c, iq_width, scale, Yd, stream=st))
    bfp_ms = timed(lambda: phy.slot_run_bfp(cfg, c, iq_width, scale, Yd, buf.pilots, buf.sigma2,
                                            buf.x_hat, buf.sinr, buf.llr, buf.flags,
                                            buf.workspace, stream=st))
    run_ms = timed(lambda: phy.slot_run(cfg, buf.Y, buf.pilots, buf.sigma2, buf.x_hat, buf.sinr,
                                        buf.llr, buf.flags, buf.workspace, stream=st))
    moved = c.numel() + Yd.numel() * 8
    gbs = moved / (dec_ms * 1e-3) / 1e9
    # end to end with the compressed stream in pinned host memory (phy_slot_run_bfp_host): what
    # crosses to the device per step is the stream, pilots and noise levels; LLRs and flags back
    ch = c.cpu().pin_memory()
    Ph = buf.pilots.cpu().pin_memory()
    sh = buf.sigma2.cpu().pin_memory()
    # the steps rotate over E2E_SETS streams with their own device and pinned output buffers,
    # as the grid-fed end-to-end measurement does
    esets = []
    for i in range(E2E_SETS):
        b_ = buf if i == 0 else phy.SlotBuffers(cfg, device=buf.Y.device)
        s_ = st if i == 0 else torch.cuda.Stream(device=buf.Y.device)
        esets.append((b_, s_, torch.empty_like(c), torch.empty_like(Yd),
                      torch.empty(buf.llr.shape, dtype=buf.llr.dtype).pin_memory(),
                      torch.empty(buf.flags.shape, dtype=torch.uint8).pin_memory()))
    lh, fh = esets[0][4], esets[0][5]

    def e2e_step(i):
        b_, s_, cd, yd, lh_, fh_ = esets[i % len(esets)]
        phy.slot_run_bfp_host(cfg, ch, iq_width, scale, Ph, sh, lh_, fh_, cd, yd, b_.pilots,
                              b_.sigma2, b_.x_hat, b_.sinr, b_.llr, b_.flags, b_.workspace,
                              stream=s_)

    for i in range(2 * len(esets)):
        e2e_step(i)
    torch.cuda.synchronize()
    k2 = max(reps, 3 * len(esets))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _, s_, *_ in esets[1:]:
        s_.wait_event(a)
    for i in range(k2):
        e2e_step(i)
    for _, s_, *_ in esets[1:]:
        st.wait_stream(s_)
    b.record(st)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / k2
    del esets
    n_re = spec.n_cells * len(spec.data_sym) * spec.n_sc
    return {"iq_width": iq_width, "stream_mb": c.numel() / 1e6,
            "decompress_us": dec_ms * 1e3, "decompress_gbs": gbs,
            "decompress_hbm_frac": gbs / hbm_peak,
            "slot_run_bfp_ms": bfp_ms, "slot_run_ms": run_ms,
            "e2e_bfp": {"value": n_re / (e2e_ms * 1e-3), "unit": "REs/s",
                        "h2d_bytes_per_step": int(ch.numel() + Ph.numel() * 8 + sh.numel() * 4),
                        "d2h_bytes_per_step": int(lh.numel() * lh.element_size() + fh.numel()),
                        "api": "phy_slot_run_bfp_host (pinned host buffers)"}}


E2E_SETS = 3  # streams (with their own buffers) the end-to-end steps rotate over
CNN_MACS_FWD = 168 * (32 * 18 + 2 * 32 * 288 + 2 * 288)  # per tile: the four 3x3 layers
CNN_MACS_TRAIN = 2 * CNN_MACS_FWD + 168 * (2 * 288 + 2 * 32 * 288)  # + dW all, dX layers 2-4


def cnn_run(dev, st, fp32_peak_tf: float, bf16_peak_tf: float, slots: int = 24,
            epochs: int = 8) -> dict:
    """The learned denoiser: trained on the GPU by the library's kernels on generated slots
    (`slots` slots of 12 PRB, 32 Rx x 8 layers = 3,072 tiles each, 0-30 dB, 0-500 Hz Doppler;
    `epochs` epochs of Adam), then evaluated on one 273-PRB 32 Rx x 8 layer 64-QAM slot at 5 dB
    and 300 Hz against LS + interpolation (channel MSE, uncoded BER of LMMSE detection), and with
    more than 24 training slots also at 0 and 20 dB. Times by CUDA events."""
    import torch
    from paper_2510_07843_gb300 import denoise as D
    from paper_2510_07843_gb300 import phy
    workers = 0 if slots <= 24 else max(1, min(16, len(os.sched_getaffinity(0))))
    g0 = time.perf_counter()
    x, y = D.training_set(n_slots=slots, n_prb=12, seed=11, dev=dev, workers=workers)
    gen_s = time.perf_counter() - g0
    tr = D.Trainer(D.init_params(0), batch=256, dev=dev, lr=2e-3)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for ep in range(epochs):
        tr.epoch(x, y, seed=ep)
    b.record(st)
    torch.cuda.synchronize()
    train_s = a.elapsed_time(b) * 1e-3
    tiles = tr.step * tr.batch
    # the same schedule with the mixed-precision step (tensor-core BF16 forward, FP32 backward
    # and master weights)
    trm = D.Trainer(D.init_params(0), batch=256, dev=dev, lr=2e-3, bf16=True)
    a.record(st)
    for ep in range(epochs):
        trm.epoch(x, y, seed=ep)
    b.record(st)
    torch.cuda.synchronize()
    train_mixed_s = a.elapsed_time(b) * 1e-3
    ev = D.slot_tiles(D.train_spec(n_prb=273, snr_db=5.0, doppler_hz=300.0), 4000, dev)
    n_tiles = phy.cnn_n_tiles(ev.cfg)
    H = torch.empty((1, len(ev.spec.data_sym), ev.spec.n_sc, 32, 8), dtype=torch.complex64,
                    device=dev)
    ws = torch.empty(phy.cnn_denoise_workspace_size(ev.cfg), dtype=torch.uint8, device=dev)
    for _ in range(3):
        phy.cnn_denoise(ev.cfg, tr.p, ev.anchors, H, ws, stream=st)
    a.record(st)
    for _ in range(10):
        phy.cnn_denoise(ev.cfg, tr.p, ev.anchors, H, ws, stream=st)
    b.record(st)
    torch.cuda.synchronize()
    inf_s = a.elapsed_time(b) * 1e-3 / 10
    # the same slot through the tensor-core forward pass (BF16 operands, FP32 sums), and the
    # forward pass alone on the slot's tiles for both forms
    for _ in range(3):
        phy.cnn_denoise_bf16(ev.cfg, tr.p, ev.anchors, H, ws, stream=st)
    a.record(st)
    for _ in range(10):
        phy.cnn_denoise_bf16(ev.cfg, tr.p, ev.anchors, H, ws, stream=st)
    b.record(st)
    torch.cuda.synchronize()
    inf_tc_s = a.elapsed_time(b) * 1e-3 / 10
    tiles_in = ev.x
    tiles_out = torch.empty_like(tiles_in)
    wsf = torch.empty(phy.cnn_workspace_size(n_tiles), dtype=torch.uint8, device=dev)
    fwd = {}
    for name, fn in (("fp32", lambda: phy.cnn_forward(n_tiles, tr.p, tiles_in, tiles_out, wsf,
                                                      stream=st)),
                     ("bf16_tensor_core", lambda: phy.cnn_forward_bf16(n_tiles, tr.p, tiles_in,
                                                                        tiles_out, wsf,
                                                                        stream=st))):
        for _ in range(3):
            fn()
        a.record(st)
        for _ in range(10):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        fwd[name] = a.elapsed_time(b) / 10
    train_tf = tiles * CNN_MACS_TRAIN * 2 / train_s / 1e12
    inf_tf = n_tiles * CNN_MACS_FWD * 2 / inf_s / 1e12
    fwd_flops = n_tiles * CNN_MACS_FWD * 2
    res = D.evaluate(tr.p, ev, dev, tensor_cores=True)
    res_mixed = D.evaluate(trm.p, ev, dev)
    more = {}
    if slots > 24:
        for snr in (0.0, 20.0):
            evs = D.slot_tiles(D.train_spec(n_prb=273, snr_db=snr, doppler_hz=300.0),
                               4000 + int(snr), dev)
            more[f"{snr:g}dB"] = D.evaluate(tr.p, evs, dev, tensor_cores=True)
    return {"train": {"tiles": int(tiles), "steps": tr.step, "batch": tr.batch,
                      "set_tiles": int(x.shape[0]), "epochs": epochs,
                      "generation_s": gen_s, "generation_workers": workers,
                      "seconds": train_s, "tiles_per_s": tiles / train_s,
                      "tflops": train_tf, "fp32_peak_frac": train_tf / fp32_peak_tf,
                      "mixed_precision": {"seconds": train_mixed_s,
                                          "tiles_per_s": trm.step * trm.batch / train_mixed_s,
                                          "what": "phy_cnn_train_step_bf16: BF16 forward on "
                                                  "the tensor cores, FP32 backward and Adam",
                                          "eval_5db": {k: res_mixed[k] for k in
                                                       ("mse_ls", "mse_cnn", "ber_ls",
                                                        "ber_cnn")}}},
            "denoise_slot": {"tiles": n_tiles, "ms": inf_s * 1e3, "tflops": inf_tf,
                             "fp32_peak_frac": inf_tf / fp32_peak_tf,
                             "ms_bf16_tensor_core": inf_tc_s * 1e3,
                             "what": "interpolation, tiles, 4 conv layers, untile (273 PRB, "
                                     "32 Rx x 8 layers)"},
            "forward_only": {"tiles": n_tiles,
                             "ms": fwd,
                             "tflops": {k: fwd_flops / (v * 1e-3) / 1e12 for k, v in fwd.items()},
                             "bf16_peak_frac": fwd_flops / (fwd["bf16_tensor_core"] * 1e-3)
                             / 1e12 / bf16_peak_tf,
                             "peak": {"fp32_tflops": fp32_peak_tf, "bf16_tflops": bf16_peak_tf,
                                      "bf16_source": "MEASURED_PEAKS.json bf16_tflops"}},
            "eval": {"snr_db": 5.0, "doppler_hz": 300.0, **res},
            **({"eval_more": more} if more else {})}


def serving_run(spec, precision, dev, buf, slots=100, llr="f32", streams=2):
    """Per-job latency in the serving loop: every 0.5 ms slot the batch's cells arrive as jobs
    (one cell each, inputs resident on the device) and are served by captured receiver graphs."""
    import dataclasses
    from paper_2510_07843_gb300 import phy, serve
    cfg1 = dataclasses.replace(phy.SlotConfig.from_spec(spec, precision=precision,
                                                        llr_format=llr), n_cells=1)
    s2 = buf.sigma2.cpu().tolist()
    jobs = [serve.Job(cfg1, buf.Y[c:c + 1], buf.pilots[c:c + 1], s2[c],
                      arrival=s * serve.DEADLINE_S, job_id=s * spec.n_cells + c,
                      sigma2_dev=buf.sigma2[c:c + 1])
            for s in range(slots) for c in range(spec.n_cells)]
    srv = serve.SlotServer(device=dev, max_cells=spec.n_cells, streams=streams)
    srv.prepare([cfg1])
    # captures the in-place receiver on every lane
    srv.run(jobs[:spec.n_cells * streams], realtime=False, keep=False)
    srv.service.clear()
    srv.batches = 0
    done = srv.run(jobs, realtime=True, keep=False)
    out = serve.latency_summary(done, service=srv.service)
    out.update(workload=f"{spec.n_cells} cells per {serve.DEADLINE_S * 1e3:g} ms slot, "
                        "slot-synchronous arrivals, inputs resident (read in place), "
                        f"{streams} batches in flight",
               slots=slots, batches=srv.batches)
    return out


def time_variant(spec, precision, refactor, llr, args, slot, dev, world, fl_peak_tf,
                 hbm_peak, first_buf=None):
    """One precision of the receiver on the workload, inputs resident in HBM.

    Serial pass: every step's stages bracketed by CUDA events on the launch stream (per-stage
    times, step latency p50/p99, per-kernel rooflines). Pipelined pass (the throughput): the
    steps rotate over `args.streams` streams (default four) with their own buffers, so one
    step's solve overlaps the next steps' estimation and Gram kernels, as a continuous stream of
    slots runs.
    Returns the variant's record and its buffers."""
    import torch
    from paper_2510_07843_gb300 import phy
    cfg = phy.SlotConfig.from_spec(spec, precision=precision, llr_format=llr,
                                   fp64_refactor=refactor)
    buf = first_buf if first_buf is not None else phy.SlotBuffers(cfg, device=dev)
    if first_buf is None:
        buf.Y.copy_(torch.from_numpy(slot.Y))
        buf.pilots.copy_(torch.from_numpy(slot.pilots))
        buf.sigma2.copy_(torch.from_numpy(slot.sigma2))
    st = torch.cuda.Stream(device=dev)
    n_re = n_data_res(spec)
    split = phy.stage_supported(cfg)
    args_ = (buf.anchors, buf.Y, buf.sigma2, buf.x_hat, buf.sinr, buf.llr, buf.flags,
             buf.workspace)

    def step(e1=None, e2=None):
        phy.chest(cfg, buf.Y, buf.pilots, buf.anchors, stream=st)
        if e1 is not None:
            e1.record(st)
        if split:  # the two detection kernels as separate calls, timed apart
            phy.detect_stage(cfg, phy.STAGE_GRAM_MF, *args_, stream=st)
            if e2 is not None:
                e2.record(st)
            phy.detect_stage(cfg, phy.STAGE_SOLVE, *args_, stream=st)
        else:
            if e2 is not None:
                e2.record(st)
            phy.detect_anchors(cfg, *args_, stream=st)

    # tile shapes (cells per chunk, solve CTA width, tensor-core ring depth) chosen by the
    # library's autotuner on these buffers, before anything is timed; outputs do not depend on them
    phy.autotune_clear()
    if not args.no_autotune:
        phy.autotune(cfg, buf.Y, buf.pilots, buf.sigma2, buf.x_hat, buf.sinr, buf.llr, buf.flags,
                     buf.workspace, stream=st)
    tiles = phy.autotune_tiles(cfg)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4))
          for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(st)
    for i in range(args.steps):
        ev[i][0].record(st)
        step(ev[i][1], ev[i][2])
        ev[i][3].record(st)
    t1.record(st)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    serial_ms = max_over_ranks(t0.elapsed_time(t1), dev)
    fl = buf.flags.cpu().numpy()
    flag_stats = {"flagged_frac": float(np.mean((fl & 1) != 0)),
                  "fp64_refactored": int(np.count_nonzero(fl & 2)),
                  "fp64_refactored_frac": float(np.mean((fl & 2) != 0)),
                  "nonfinite": int(np.count_nonzero(fl & 4)),
                  "timed_out": int(np.count_nonzero(fl & 8))}

    pipe_ms = None
    sets = [(buf, st)]
    if args.streams > 1:
        for _ in range(args.streams - 1):
            b2 = phy.SlotBuffers(cfg, device=dev)
            b2.Y.copy_(buf.Y)
            b2.pilots.copy_(buf.pilots)
            b2.sigma2.copy_(buf.sigma2)
            sets.append((b2, torch.cuda.Stream(device=dev)))

        def pstep(i):
            b, s_ = sets[i % len(sets)]
            phy.slot_run(cfg, b.Y, b.pilots, b.sigma2, b.x_hat, b.sinr, b.llr, b.flags,
                         b.workspace, stream=s_)

        for i in range(max(args.warmup, 3) * len(sets)):
            pstep(i)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(st)
        for _, s_ in sets[1:]:
            s_.wait_event(p0)
        for i in range(args.steps):
            pstep(i)
        for _, s_ in sets[1:]:
            st.wait_stream(s_)
        p1.record(st)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        pipe_ms = max_over_ranks(p0.elapsed_time(p1), dev)
    step_ms = [a.elapsed_time(d) for a, b, c, d in ev]
    chest_ms = statistics.mean(a.elapsed_time(b) for a, b, c, d in ev)
    gram_ms = statistics.mean(b.elapsed_time(c) for a, b, c, d in ev)
    solve_ms = statistics.mean(c.elapsed_time(d) for a, b, c, d in ev)
    det_ms = statistics.mean(b.elapsed_time(d) for a, b, c, d in ev)

    flops = detect_flops(spec)
    ab = algorithmic_bytes(spec)
    on_tc = precision != "fp32"
    peak_src = "measured in this run: phy_fma_probe FP32 (fma.rn.f32 / f32x2, the larger)"
    solve_roof = {"bound": "alu", "kernel": f"re_solve_fp32_kernel<16,{spec.qm}>",
                  "achieved": flops["solve"] / (solve_ms * 1e-3) / 1e12, "peak": fl_peak_tf,
                  "unit": "TFLOP/s", "peak_source": peak_src, "flops_per_launch": flops["solve"],
                  "ms": solve_ms, "traffic": committed_traffic("re_solve", args.workload)}
    gram_bytes = ab["y_data"] + anchor_bytes(spec)
    if on_tc:
        gram_roof = {"bound": "hbm", "kernel": f"seg_prep_tc_kernel ({precision})",
                     "achieved": gram_bytes / (gram_ms * 1e-3) / 1e9, "peak": hbm_peak,
                     "unit": "GB/s", "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                     "bytes_per_launch": gram_bytes,
                     "tensor_flops_per_launch": flops["products"], "ms": gram_ms,
                     "traffic": committed_traffic("seg_prep_tc", args.workload)}
    else:
        gram_roof = {"bound": "alu", "kernel": "seg_prep_fp32_kernel<16>",
                     "achieved": flops["products"] / (gram_ms * 1e-3) / 1e12, "peak": fl_peak_tf,
                     "unit": "TFLOP/s", "peak_source": peak_src,
                     "flops_per_launch": flops["products"], "ms": gram_ms,
                     "traffic": committed_traffic("seg_prep_fp32", args.workload)}
    for r in (solve_roof, gram_roof):
        r["frac"] = r["achieved"] / r["peak"]
    dominant = solve_roof if solve_ms >= gram_ms else gram_roof
    timed_ms = pipe_ms if pipe_ms is not None else serial_ms
    rec = {"precision": precision, "fp64_refactor": bool(refactor), "tiles": tiles,
           "value": whole_job_rate(world, n_re, args.steps, timed_ms), "unit": "REs/s",
           "ms_per_step": timed_ms / args.steps,
           "serial_ms_per_step": serial_ms / args.steps,
           "serial_value": whole_job_rate(world, n_re, args.steps, serial_ms),
           "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                          "p99": float(np.percentile(step_ms, 99)), "deadline_ms": 0.5,
                          "what": "one step (whole batch) on an idle GPU, CUDA events"},
           "stages_ms": {"chest": chest_ms, "gram_mf": gram_ms, "solve": solve_ms,
                         "detect": det_ms},
           "dominant": dominant, "per_kernel": {"solve": solve_roof, "gram_mf": gram_roof},
           "split_stages": bool(split), "flags": flag_stats,
           "gpu_launches": (1 + 2 * detect_chunks(spec)) * args.steps}
    return rec, cfg, buf, st


def serving_pool(dev, pool_size: int = 48, seed: int = 5):
    """Distinct seeded jobs of the serving configuration, resident on the device: FP16
    tensor-core products for 5 or more layers, the direct FP32 form below that."""
    import torch
    from paper_2510_07843_gb300 import phy
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(pool_size):
        sp = S.spec_serving_job(rng)
        sl = S.make_slot(sp, 7000 + i, keep_h=False)
        cfg = phy.SlotConfig.from_spec(sp, precision="fp16" if sp.n_layers > 4 else "fp32")
        pool.append((cfg, *(torch.from_numpy(a).to(dev) for a in (sl.Y, sl.pilots, sl.sigma2))))
    return pool


def batch_probe(n_jobs: int, reps: int) -> int:
    """Times `reps` batches of `n_jobs` jobs of the serving mix (consecutive pool entries) through
    one lane of the batching server (post, then a replay of the captured batched receiver), after
    one warm-up batch; prints one JSON line with the GPU time per batch (CUDA events)."""
    import torch
    from paper_2510_07843_gb300 import build, phy, serve
    if not 1 <= n_jobs <= phy.BATCH_MAX_JOBS:
        raise SystemExit(f"--batch-probe takes 1 to {phy.BATCH_MAX_JOBS} jobs")
    build.build()
    dev = torch.device("cuda:0")
    pool = serving_pool(dev)
    srv = serve.BatchServer(device=dev, lanes=1)
    srv.prepare(serve.MixedJob(*pool[0]))
    ln = srv.lanes[0]
    ms, res = [], 0
    for rep in range(reps + 1):
        jobs = [serve.MixedJob(*pool[(rep * n_jobs + k) % len(pool)]) for k in range(n_jobs)]
        ln.post(jobs, srv._layout)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ln.stream)
        with torch.cuda.stream(ln.stream):
            ln.graph.replay()
        e1.record(ln.stream)
        torch.cuda.synchronize()
        if phy.batch_status(ln.host) != 0:
            raise RuntimeError("batch did not complete")
        if rep > 0:
            ms.append(e0.elapsed_time(e1))
            res += sum(j.n_res for j in jobs)
    print(json.dumps({"batch_jobs": n_jobs, "batches": reps, "ms_per_batch_p50":
                      float(np.median(ms)), "res_per_s": res / (sum(ms) * 1e-3)}))
    return 0


def serving_mixed_run(dev, slots: int = 100, n_cells=(32, 16), rate_hz: float = 2000.0,
                      pool_size: int = 48, lanes: int = 2, seed: int = 5) -> dict:
    """The serving configuration: uplink jobs of 32 cells arriving as Poisson streams at 2000
    slots/s per cell, each of its own shape (4-273 PRB, 4/16/32/64 Rx, 1-16 layers, QPSK to
    256-QAM, 23-tap 300 ns TDL with Jakes 100 Hz), served by continuous heterogeneous batching
    (BatchServer over the batched receiver: FP16 tensor-core products for jobs of 5 or more
    layers, the direct FP32 form below that) for `slots` 0.5 ms slots in real
    time. Job inputs come from a pool of `pool_size` distinct seeded jobs resident on the device
    (arrivals pick pool entries uniformly). Each load runs twice: with every cell keeping its
    noise level on the device across its slots (phy_job.noise_state, alpha 0.5, the smaller of
    the two DMRS estimates; a cell's next slot then waits for its previous one, since its
    detection uses the state that slot updated), and with the noise levels given. Latency is
    per job, arrival to completion seen by the host; throughput counts the REs of every served
    job over the run's span."""
    import torch
    from paper_2510_07843_gb300 import serve
    pool = serving_pool(dev, pool_size, seed)
    duration = slots * serve.DEADLINE_S
    srv = serve.BatchServer(device=dev, lanes=lanes)
    srv.prepare(serve.MixedJob(*pool[0], arrival=0.0, job_id=-1))
    # a short untimed stream first (kernels warm, lanes in use), then the measured ones
    srv.run([serve.MixedJob(*pool[p], arrival=0.0, job_id=-1) for p in range(min(8, pool_size))],
            realtime=False)
    runs = []
    for cells, track in [(c, tr) for c in n_cells for tr in (True, False)]:
        arrivals = S.serving_arrivals(cells, rate_hz, duration, seed + cells)
        pick = np.random.default_rng(seed + 100 + cells).integers(0, pool_size, len(arrivals))
        state = torch.zeros(cells, dtype=torch.float32, device=dev)  # unset: first slot sets it
        jobs = [serve.MixedJob(*pool[p], arrival=t, job_id=k,
                               noise_state=state[c:c + 1] if track else None,
                               noise_alpha=0.5 if track else 0.0, noise_mode="min")
                for k, ((t, c), p) in enumerate(zip(arrivals, pick))]
        srv.batches, srv.batch_sizes, srv.service, srv.host_post = 0, [], [], []
        done = srv.run(jobs, realtime=True)
        out = serve.latency_summary(done, service=srv.service)
        n_res = sum(j.n_res for j in done)
        span = max(j.done for j in done) - min(j.arrival for j in done)
        out.update(cells=cells, noise_state_on_device=track,
                   res_per_s=n_res / span, offered_res_per_s=n_res / duration,
                   res=int(n_res), batches=srv.batches,
                   mean_batch=float(np.mean(srv.batch_sizes)),
                   max_batch=int(max(srv.batch_sizes)),
                   host_post_us_p50=float(np.median(srv.host_post)) * 1e6)
        runs.append(out)
    return {"workload": f"Poisson {rate_hz:g} slots/s per cell for {slots} slots of 0.5 ms; per "
                        f"job 4-273 PRB, 4/16/32/64 Rx, 1-16 layers, QPSK-256QAM; pool of "
                        f"{pool_size} distinct resident jobs; FP16 tensor-core products for 5-16 "
                        f"layers, FP32 for 1-4; the configuration's 32 cells, then 16, each "
                        f"with and without the noise level tracked per cell on the device",
            "runs": runs, "lanes": lanes, "arena_bytes_per_lane": srv.arena_bytes,
            "api": "phy_batch_post / phy_batch_launch (captured graph per lane)"}


def run_ours(args, spec, rank, world, local):
    import torch
    from paper_2510_07843_gb300 import build, phy

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    phy.load()
    slot = S.make_slot(spec, rank_seed(rank), keep_h=False)
    n_re = n_data_res(spec)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    probe_st = torch.cuda.Stream(device=dev)

    clocks = ClockSampler(local, args.clock_log)
    clocks.start()
    time.sleep(0.3)  # let the sampler start before the GPU gets busy
    fma = measured_fma_peaks(dev, probe_st)
    fl_peak = max(fma["fp32_tflops"], fma["fp32x2_tflops"])
    refactor = not args.no_refactor and args.precision != "fp32"
    head, cfg, buf, st = time_variant(spec, args.precision, refactor, args.llr, args, slot, dev,
                                      world, fl_peak, hbm_peak)
    variants = {}
    for v in [x for x in args.variants.split(",") if x and x != args.precision]:
        rec, _, vbuf, _ = time_variant(spec, v, False, args.llr, args, slot, dev, world, fl_peak,
                                       hbm_peak)
        variants[v] = rec
        del vbuf
    torch.cuda.synchronize()
    clk = clocks.stop()

    # e2e through the C ABI with host buffers (pinned), copies inside the timed region. Steps
    # rotate over E2E_SETS streams, each with its own device buffers and pinned output buffers,
    # so that one step's input copy, another's kernels and a third's result copy overlap (the
    # two copy directions use separate copy engines), as a stream of slots runs in service.
    e2e = None
    if not args.no_e2e:
        Yh = torch.from_numpy(slot.Y).pin_memory()
        Ph = torch.from_numpy(slot.pilots).pin_memory()
        sh = torch.from_numpy(slot.sigma2).pin_memory()
        esets = []
        for i in range(E2E_SETS):
            b_ = buf if i == 0 else phy.SlotBuffers(cfg, device=dev)
            s_ = st if i == 0 else torch.cuda.Stream(device=dev)
            lh = torch.empty(buf.llr.shape, dtype=buf.llr.dtype).pin_memory()
            fh = torch.empty(buf.flags.shape, dtype=torch.uint8).pin_memory()
            esets.append((b_, s_, lh, fh))

        def e2e_step(i):
            b_, s_, lh, fh = esets[i % len(esets)]
            phy.slot_run_host(cfg, Yh, Ph, sh, lh, fh, b_.Y, b_.pilots, b_.sigma2, b_.x_hat,
                              b_.sinr, b_.llr, b_.flags, b_.workspace, stream=s_)

        for i in range(2 * len(esets)):
            e2e_step(i)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        k2 = max(min(args.steps, 30), 3 * len(esets))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _, s_, _, _ in esets[1:]:
            s_.wait_event(a)
        for i in range(k2):
            e2e_step(i)
        for _, s_, _, _ in esets[1:]:
            st.wait_stream(s_)
        b.record(st)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(a.elapsed_time(b), dev)
        lh0, fh0 = esets[0][2], esets[0][3]
        h2d = Yh.numel() * 8 + Ph.numel() * 8 + sh.numel() * 4
        d2h = lh0.numel() * lh0.element_size() + fh0.numel()
        e2e = {"value": whole_job_rate(world, n_re, k2, e_ms), "unit": "REs/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "h2d_d2h_gbs": (h2d + d2h) * k2 / (e_ms * 1e-3) / 1e9,
               "streams": len(esets), "steps": k2,
               "api": "phy_slot_run_host (pinned host buffers)"}
        del esets

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    serving = None
    if not args.no_serving:
        serving = serving_run(spec, args.precision, dev, buf, llr=args.llr,
                              streams=args.serving_lanes)

    serving_mixed = None
    if not args.no_serving:
        serving_mixed = serving_mixed_run(dev)

    noise = None
    if not args.no_noise:
        noise = noise_estimate_run(cfg, spec, buf, st)

    bfp = None
    if not args.no_bfp:
        bfp = bfp_run(cfg, spec, slot, buf, st, hbm_peak)
    learned = None
    if not args.no_cnn:
        learned = cnn_run(dev, st, fl_peak, peaks.get("bf16_tflops", 1900.0),
                          slots=args.cnn_slots, epochs=args.cnn_epochs)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(spec, args.cpu_budget)

    dominant = head["dominant"]
    roofline = {k: dominant[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    roofline.update(kernel=dominant["kernel"], peak_source=dominant["peak_source"],
                    per_kernel=head["per_kernel"], split_stages=head["split_stages"],
                    measured_peaks={"fma": fma, "hbm_gbs": hbm_peak})
    ab = algorithmic_bytes(spec)
    plain = variants.get("fp32")
    vs_plain = None
    if plain is not None:
        vs_plain = {"value_ratio": head["value"] / plain["value"],
                    "serial_ratio": head["serial_value"] / plain["serial_value"],
                    "p99_ms": {args.precision: head["latency_ms"]["p99"],
                               "fp32": plain["latency_ms"]["p99"]},
                    "what": "headline form over plain FP32 on the same workload and buffers"}
    strip = lambda r: {k: v for k, v in r.items() if k not in ("dominant",)}
    line = {
        "metric": METRIC, "value": head["value"], "unit": "REs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": (f"{args.precision} tensor-core products (fp32 accumulate), f32 solve"
                  if args.precision != "fp32" else "f32"),
        "data": "synthetic", "config": dict(config_dict(spec, args, world),
                                            tiles=dict(head["tiles"], chosen_by=(
                                                "defaults" if args.no_autotune
                                                else "phy_autotune"))),
        "serial_ms_per_step": head["serial_ms_per_step"],
        "latency_ms": head["latency_ms"],
        "stages_ms": head["stages_ms"],
        "flags": head["flags"],
        "roofline": roofline,
        "step_hbm": {"algorithmic_bytes": ab["step"],
                     "achieved_gbs": ab["step"] / (head["serial_ms_per_step"] * 1e-3) / 1e9,
                     "peak_gbs": hbm_peak,
                     "frac": ab["step"] / (head["serial_ms_per_step"] * 1e-3) / 1e9 / hbm_peak},
        "vs_plain_fp32": vs_plain,
        "variants": {k: strip(v) for k, v in variants.items()},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "serving": serving,
        "serving_mixed": serving_mixed,
        "noise_estimate": noise,
        "bfp_fronthaul": bfp,
        "learned_denoiser": learned,
        "gpu_launches": head["gpu_launches"],
        "clocks": clk,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
