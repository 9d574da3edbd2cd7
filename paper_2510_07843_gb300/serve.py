"""Serving slot loop: continuous batching of uplink receiver jobs on one GPU.

Two servers, both measuring latency per job from its arrival to the host seeing its batch
complete, against the slot deadline.

SlotServer batches jobs of equal configuration: a job is one cell's slot (received grid, DMRS
pilots, noise variance) with its receiver configuration (a SlotConfig with n_cells = 1). Cells
are independent, so jobs with equal configurations batch by placing their cells side by side in
one phy_slot_run call. The server keeps, per (configuration, batch size), persistent device
buffers and a CUDA graph of the whole receiver captured on them; a batch copies its jobs' inputs
into the buffers, replays the graph and copies each job's LLRs and flags out; when a batch's
inputs already sit side by side in device memory (consecutive cells of one resident input), a
receiver captured on those addresses reads them in place instead. Batch sizes are powers of two
up to a limit that the configuration's device memory (buffers plus workspace) sets against a
budget, so admission is by device memory.

BatchServer batches jobs of any shape together through the batched receiver (phy_batch_post /
phy_batch_launch): whatever has arrived goes into the next free lane's batch, up to 64 jobs and
the lane arena's bytes (arenas sized from the device's free memory), served by one replay of the
lane's captured graph.

Everything on the device runs in libphy.so; this module only schedules and marshals.
"""
from __future__ import annotations

import dataclasses
import struct
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import phy

DEADLINE_S = 0.5e-3  # one 30 kHz slot


def config_key(cfg: phy.SlotConfig) -> Tuple:
    """Hashable identity of a per-cell configuration (n_cells excluded)."""
    d = dataclasses.asdict(cfg)
    d.pop("n_cells")
    d["dmrs_sym"] = tuple(d["dmrs_sym"])
    return tuple(sorted(d.items()))


@dataclass
class Job:
    cfg: phy.SlotConfig        # per-cell configuration (n_cells is ignored)
    Y: object                  # device tensor [1][sym][rx][sc] complex64
    pilots: object             # device tensor [1][dmrs][layer][sc] complex64
    sigma2: float
    arrival: float = 0.0       # seconds on the server clock
    job_id: int = 0
    sigma2_dev: object = None  # optional device view [1] float32 of sigma2 (zero-copy batches)
    # > 0: estimate the noise level from the DMRS and track it in sigma2_dev, a per-cell device
    # state kept across slots (state = alpha estimate + (1 - alpha) state); the batch must read
    # resident inputs in place (consecutive cells, see _direct)
    noise_alpha: float = 0.0
    llr: object = None         # filled: device tensor [1][dsym][sc][layer][qm]
    flags: object = None       # filled: device tensor [1][dsym][sc]
    done: float = field(default=float("nan"))

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def batch_sizes(max_cells: int) -> List[int]:
    """Powers of two up to max_cells (at least 1)."""
    out, b = [], 1
    while b <= max(1, max_cells):
        out.append(b)
        b *= 2
    return out


def pick_batch(n_waiting: int, max_cells: int) -> int:
    """Largest power of two not above the waiting count and the admission limit."""
    b = 1
    while b * 2 <= min(n_waiting, max_cells):
        b *= 2
    return b


def bytes_per_cell(cfg: phy.SlotConfig) -> int:
    """Device bytes one cell of cfg takes in a batch: inputs, outputs and workspace share."""
    one = dataclasses.replace(cfg, n_cells=1)
    K, nds, nl = one.n_sc, one.n_dsym, one.n_layers
    io = (one.n_sym * one.n_rx * K * 8 + len(one.dmrs_sym) * nl * K * 8 + 4
          + nds * K * nl * (8 + 4 + 4 * one.qm) + nds * K
          + len(one.dmrs_sym) * phy.n_groups(one) * nl * one.n_rx * 8)
    return io + phy.workspace_size(one)


def admission_limit(cfg: phy.SlotConfig, budget_bytes: int, max_cells: int) -> int:
    """Cells of cfg one batch may hold under the device-memory budget (at least 1)."""
    return max(1, min(max_cells, budget_bytes // max(1, bytes_per_cell(cfg))))


def _follows(a, b) -> bool:
    """b is the cell right after a in the same storage (both [1][...] views)."""
    return (a.untyped_storage().data_ptr() == b.untyped_storage().data_ptr() and
            b.data_ptr() == a.data_ptr() + a.numel() * a.element_size() and a.is_contiguous()
            and b.is_contiguous())


def _direct(jobs: Sequence[Job]) -> bool:
    """All inputs of the batch are consecutive cells of their sources (and the source grid is
    16-byte aligned), so the receiver can read them in place."""
    if any(j.sigma2_dev is None for j in jobs) or jobs[0].Y.data_ptr() % 16:
        return False
    return all(_follows(a.Y, b.Y) and _follows(a.pilots, b.pilots) and
               _follows(a.sigma2_dev, b.sigma2_dev) for a, b in zip(jobs, jobs[1:]))


def _span(first, n: int):
    """The n consecutive cells starting at view `first` as one [n][...] tensor."""
    if n == 1:
        return first
    return first.as_strided((n,) + tuple(first.shape[1:]), first.stride())


class _Graph:
    """Persistent buffers and the captured receiver for one (configuration, batch size)."""

    def __init__(self, cfg: phy.SlotConfig, n_cells: int, device, stream):
        import torch
        self.cfg = dataclasses.replace(cfg, n_cells=n_cells)
        self.buf = phy.SlotBuffers(self.cfg, device=device)
        self.buf.Y.zero_()
        self.buf.pilots.zero_()
        self.buf.sigma2.fill_(1.0)
        self.stream = stream
        args = (self.buf.Y, self.buf.pilots, self.buf.sigma2, self.buf.x_hat, self.buf.sinr,
                self.buf.llr, self.buf.flags, self.buf.workspace)
        with torch.cuda.stream(stream):
            phy.slot_run(self.cfg, *args, stream=stream)  # configures kernels before capture
        stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=stream):
            phy.slot_run(self.cfg, *args, stream=stream)
        self.direct = {}  # captured receivers reading resident inputs in place, by address

    def launch(self, jobs: Sequence[Job], keep: bool = True):
        """Enqueues the batch on this graph's stream (no host synchronisation)."""
        import torch
        if _direct(jobs):  # inputs already side by side in device memory: read in place
            b, n = self.buf, len(jobs)
            alpha = jobs[0].noise_alpha
            key = (jobs[0].Y.data_ptr(), jobs[0].pilots.data_ptr(), jobs[0].sigma2_dev.data_ptr(),
                   alpha)
            g = self.direct.get(key)
            if g is None:  # one captured receiver per input location (a ring has few)
                ins = (_span(jobs[0].Y, n), _span(jobs[0].pilots, n), _span(jobs[0].sigma2_dev, n))
                outs = (b.x_hat, b.sinr, b.llr, b.flags, b.workspace)
                if len(self.direct) >= 64:
                    self.direct.clear()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=self.stream):
                    if alpha > 0.0:  # the noise state is updated in place, then detected with
                        phy.slot_run_track(self.cfg, "min", alpha, *ins, *outs,
                                           stream=self.stream)
                    else:
                        phy.slot_run(self.cfg, *ins, *outs, stream=self.stream)
                self.direct[key] = g
            with torch.cuda.stream(self.stream):
                g.replay()
                if keep:
                    for i, j in enumerate(jobs):
                        j.llr = b.llr[i:i + 1].clone()
                        j.flags = b.flags[i:i + 1].clone()
            return
        if any(j.noise_alpha > 0.0 for j in jobs):
            raise ValueError("noise tracking needs the batch's inputs resident side by side")
        with torch.cuda.stream(self.stream):
            # inputs into the batch buffers: one copy per run of jobs whose tensors are
            # consecutive cells of one source (the common case of a cell-major input ring)
            i = 0
            while i < len(jobs):
                e = i + 1
                while (e < len(jobs) and _follows(jobs[e - 1].Y, jobs[e].Y) and
                       _follows(jobs[e - 1].pilots, jobs[e].pilots)):
                    e += 1
                src_y = _span(jobs[i].Y, e - i)
                src_p = _span(jobs[i].pilots, e - i)
                self.buf.Y[i:e].copy_(src_y, non_blocking=True)
                self.buf.pilots[i:e].copy_(src_p, non_blocking=True)
                i = e
            s2 = torch.tensor([float(j.sigma2) for j in jobs], dtype=torch.float32)
            self.buf.sigma2[:len(jobs)].copy_(s2.pin_memory(), non_blocking=True)
            self.graph.replay()
            if keep:
                for i, j in enumerate(jobs):
                    j.llr = self.buf.llr[i:i + 1].clone()
                    j.flags = self.buf.flags[i:i + 1].clone()


class SlotServer:
    """Continuous batching over captured receiver graphs (see the module docstring)."""

    def __init__(self, device="cuda", max_cells: int = 8, memory_budget: int = 2 << 30,
                 clock: Callable[[], float] = time.perf_counter, streams: int = 1):
        self.device = device
        self.max_cells = max_cells
        self.budget = memory_budget
        self.clock = clock
        self.lanes = max(1, streams)  # batches in flight at once, one stream each
        self.streams = None  # created with the first graph
        self.graphs: Dict[Tuple, _Graph] = {}
        self.limits: Dict[Tuple, int] = {}
        self.batches = 0
        self.service: List[float] = []  # seconds per batch on the GPU (start to end event)

    def _event(self):
        import torch
        return torch.cuda.Event(enable_timing=True)

    def _sync(self):
        import torch
        torch.cuda.synchronize(self.device)

    def limit(self, cfg: phy.SlotConfig) -> int:
        k = config_key(cfg)
        if k not in self.limits:
            self.limits[k] = admission_limit(cfg, self.budget, self.max_cells)
        return self.limits[k]

    def prepare(self, cfgs: Sequence[phy.SlotConfig]):
        """Captures the graphs of every batch size each configuration may use (before timing)."""
        for cfg in cfgs:
            for b in batch_sizes(self.limit(cfg)):
                for lane in range(self.lanes):
                    self._graph(cfg, b, lane)

    def _graph(self, cfg: phy.SlotConfig, n: int, lane: int = 0) -> _Graph:
        k = (config_key(cfg), n, lane)
        if k not in self.graphs:
            import torch
            if self.streams is None:
                self.device = torch.device(self.device)
                self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.lanes)]
            self.graphs[k] = _Graph(cfg, n, self.device, self.streams[lane])
        return self.graphs[k]

    def run(self, jobs: Sequence[Job], realtime: bool = True, keep: bool = True) -> List[Job]:
        """Serves jobs in arrival order. With realtime, job.arrival is an offset in seconds from
        the start of the call and jobs are not seen before they arrive; otherwise all are
        waiting at once (done then counts from the start). Up to `streams` batches are in
        flight at once, each on its own stream with its own buffers; a batch's completion time
        is its end event on the GPU clock, placed on the host clock by an event recorded at the
        start. Returns the jobs with done (and, with keep, their own copies of llr and flags)
        filled, in completion order."""
        import collections
        pending = sorted(jobs, key=lambda j: j.arrival)
        queues: Dict[Tuple, List[Job]] = {}
        finished: List[Job] = []
        inflight = collections.deque()  # (lane, start event, end event, batch)
        free = list(range(self.lanes))
        if self.streams is None and pending:
            self._graph(pending[0].cfg, 1)  # creates the streams
        self._sync()
        ref = self._event()
        ref.record(self.streams[0])
        t0 = self.clock()
        ref.synchronize()

        def retire(block: bool):
            while inflight and (block or inflight[0][2].query()):
                lane, e0, e1, batch = inflight.popleft()
                e1.synchronize()
                t = ref.elapsed_time(e1) * 1e-3
                self.service.append(e0.elapsed_time(e1) * 1e-3)
                for j in batch:
                    j.done = t
                finished.extend(batch)
                free.append(lane)
                block = False

        i = 0
        while i < len(pending) or any(queues.values()):
            now = self.clock() - t0
            while i < len(pending) and (not realtime or pending[i].arrival <= now):
                queues.setdefault((config_key(pending[i].cfg), pending[i].noise_alpha),
                                  []).append(pending[i])
                i += 1
            retire(False)
            ready = [(q[0].arrival, k) for k, q in queues.items() if q]
            if not ready:  # idle until the next arrival
                if realtime and i < len(pending):
                    while self.clock() - t0 < pending[i].arrival:
                        retire(False)
                continue
            if not free:  # every lane busy: wait for the oldest batch
                retire(True)
            _, key = min(ready)  # the configuration whose oldest job has waited longest
            q = queues[key]
            cfg = q[0].cfg
            b = pick_batch(len(q), self.limit(cfg))
            batch, queues[key] = q[:b], q[b:]
            lane = free.pop(0)
            g = self._graph(cfg, b, lane)
            e0, e1 = self._event(), self._event()
            e0.record(g.stream)
            g.launch(batch, keep=keep)
            e1.record(g.stream)
            inflight.append((lane, e0, e1, batch))
            self.batches += 1
        while inflight:
            retire(True)
        return finished


def latency_summary(jobs: Sequence[Job], deadline: float = DEADLINE_S,
                    service: Optional[Sequence[float]] = None) -> dict:
    """Per-job latency (arrival to completion seen by the host) percentiles against the
    deadline; with `service`, also the per-batch service time (launch to completion)."""
    import numpy as np
    lat = np.array([j.latency for j in jobs]) * 1e3
    out = {"jobs": len(jobs), "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
           "deadline_ms": deadline * 1e3, "missed": int((lat > deadline * 1e3).sum())}
    if service:
        sv = np.array(service) * 1e3
        out.update(service_p50_ms=float(np.percentile(sv, 50)),
                   service_p99_ms=float(np.percentile(sv, 99)))
    return out


# ---------------------------------------------------------------------------------------------
# Heterogeneous continuous batching over the batched receiver (phy_batch_*)
# ---------------------------------------------------------------------------------------------

_ALIGN = 256


def _up(v: int) -> int:
    return (v + _ALIGN - 1) // _ALIGN * _ALIGN


@dataclass
class MixedJob:
    """One cell's slot with its own shape; inputs are device tensors [1][...] that stay resident
    until the job completes. The server fills llr and flags (views into its lane arena, valid
    until that lane's next batch, or copies with keep) and done."""
    cfg: phy.SlotConfig
    Y: object
    pilots: object
    sigma2: object           # device tensor [1] float32
    arrival: float = 0.0
    job_id: int = 0
    # the cell's noise level tracked on the device (phy_job.noise_state): a device tensor of
    # n_cells floats kept by the caller from slot to slot; sigma2 is then not read
    noise_state: object = None
    noise_alpha: float = 0.0
    noise_mode: str = "min"
    done: float = field(default=float("nan"))
    _out: object = field(default=None, repr=False)    # (arena, LLR offset, flag offset)
    _views: object = field(default=None, repr=False)  # (llr, flags) once built or kept

    def __post_init__(self):
        # input addresses, taken once (the inputs stay where they are until the job is done)
        self._addr = (phy._ptr(self.Y), phy._ptr(self.pilots), phy._ptr(self.sigma2),
                      phy._ptr(self.noise_state), float(self.noise_alpha),
                      phy.NOISE_MODE.get(self.noise_mode, self.noise_mode))

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def n_res(self) -> int:
        return self.cfg.n_cells * self.cfg.n_dsym * self.cfg.n_sc

    def _results(self):
        if self._views is None and self._out is not None:
            import torch
            arena, lo, fo = self._out
            c = self.cfg
            n_re = c.n_cells * c.n_dsym * c.n_sc
            dt, el = (torch.float16, 2) if c.llr_format == "f16" else (torch.float32, 4)
            n = n_re * c.n_layers * c.qm * el
            llr = arena[lo:lo + n].view(dt).view(c.n_cells, c.n_dsym, c.n_sc, c.n_layers, c.qm)
            self._views = (llr, arena[fo:fo + n_re].view(c.n_cells, c.n_dsym, c.n_sc))
        return self._views

    @property
    def llr(self):
        v = self._results()
        return None if v is None else v[0]

    @property
    def flags(self):
        v = self._results()
        return None if v is None else v[1]


class _JobLayout:
    """Per-configuration constants of the batched path: the phy_slot_cfg record and the bytes a
    job takes (intermediates, LLRs, flags)."""
    __slots__ = ("cfg", "record", "ws", "llr", "flags", "total")

    def __init__(self, cfg: phy.SlotConfig):
        self.cfg = cfg
        self.record = bytes(cfg.c())
        self.ws = phy.batch_workspace_size([(cfg, None, None, None, None, None, None, None)])
        if self.ws == 0:
            raise ValueError(f"configuration not accepted by the batched receiver: {cfg}")
        n_re = cfg.n_cells * cfg.n_dsym * cfg.n_sc
        self.llr = n_re * cfg.n_layers * cfg.qm * (2 if cfg.llr_format == "f16" else 4)
        self.flags = n_re
        self.total = self.ws + _up(self.llr) + _up(self.flags)


def mixed_job_bytes(cfg: phy.SlotConfig) -> int:
    """Device bytes a job takes in a lane's arena: its intermediates and its LLR and flag
    outputs (x_hat and SINR are not kept by the server)."""
    return _JobLayout(cfg).total


class _Lane:
    """One batch in flight: its arena, its pinned job table and device copy, its stream and the
    CUDA graph captured on phy_batch_launch for them."""

    def __init__(self, device, arena_bytes: int, poll_limit: int):
        import ctypes
        import torch
        self.stream = torch.cuda.Stream(device=device)
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=device)
        self.base = self.arena.data_ptr()
        n = phy.batch_table_bytes()
        self.host = torch.zeros(n, dtype=torch.uint8).pin_memory()
        self.host_addr = self.host.data_ptr()
        self.devt = torch.zeros(n, dtype=torch.uint8, device=device)
        self.poll_limit = poll_limit
        self.graph = None
        # the job records of a batch, filled in place (no ctypes objects per job)
        self.records = (ctypes.c_char * (phy.BATCH_MAX_JOBS * phy.JOB_BYTES))()
        self.rec_view = memoryview(self.records).cast("B")

    def capture(self, warm: Sequence["MixedJob"], layout):
        """Runs one real batch (configures the kernels), then captures the launch."""
        import torch
        self.post(warm, layout)
        phy.batch_launch(self.host, self.devt, self.poll_limit, stream=self.stream)
        self.stream.synchronize()
        if phy.batch_status(self.host) != 0:
            raise RuntimeError("warm-up batch did not run")
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            phy.batch_launch(self.host, self.devt, self.poll_limit, stream=self.stream)

    def post(self, jobs: Sequence["MixedJob"], layout):
        """Lays the batch out in the arena (intermediates, then each job's LLRs and flags),
        writes the job records and rings the table's doorbell. layout(cfg) -> _JobLayout."""
        lays = [layout(j.cfg) for j in jobs]
        ws, outs, end = write_records(self.rec_view, lays, [j._addr for j in jobs], self.base)
        if end > self.arena.numel():
            raise ValueError("batch larger than the lane arena")
        for j, o in zip(jobs, outs):
            j._out, j._views = (self.arena,) + o, None
        st = phy.batch_post_records(self.records, len(jobs), self.host_addr, self.base, ws)
        if st != 0:
            raise RuntimeError(f"phy_batch_post failed: {phy.STATUS.get(st, st)}")


# the phy_job fields after the configuration: eight addresses, noise_alpha, noise_mode
_ADDR = struct.Struct("<8Qfi")


def write_records(rec, lays: Sequence[_JobLayout], addrs, base: int):
    """Writes the phy_job records of a batch into `rec` (a writable byte buffer) for an arena at
    device address `base`: the intermediates first (phy_batch_post lays them out from `base`),
    then per job its LLRs and flags. addrs: per job the (Y, pilots, sigma2) addresses, optionally
    followed by (noise_state, noise_alpha, noise_mode code). Returns the intermediates' bytes,
    per job the (LLR, flag) arena offsets, and the end offset."""
    ws = _up(sum(l.ws for l in lays))
    off, jb, ao, pack = ws, phy.JOB_BYTES, phy.JOB_ADDR_OFFSET, _ADDR.pack_into
    outs = []
    for i, (l, a) in enumerate(zip(lays, addrs)):
        y, p, s2 = a[:3]
        st, alpha, mode = a[3:6] if len(a) >= 6 else (None, 0.0, 2)
        lo = off
        fo = _up(lo + l.llr)
        off = _up(fo + l.flags)
        o = i * jb
        rec[o:o + ao] = l.record
        pack(rec, o + ao, y or 0, p or 0, s2 or 0, 0, 0, base + lo, base + fo, st or 0,
             alpha, mode)
        outs.append((lo, fo))
    return ws, outs, off


class BatchServer:
    """Continuous batching of jobs of any shape: whatever has arrived goes into the next free
    lane's batch (arrival order, up to 64 jobs and the lane arena's bytes), served by one replay
    of the lane's captured graph of the batched receiver. The arenas are sized from the device's
    free memory when the server starts (admission by device memory). Up to `lanes` batches are
    in flight at once; a batch's completion is its end event on the GPU clock, mapped to the host
    clock by an event recorded when serving starts."""

    def __init__(self, device="cuda", lanes: int = 2, memory_fraction: float = 0.25,
                 max_arena: int = 4 << 30, max_jobs: int = phy.BATCH_MAX_JOBS,
                 poll_limit: int = -1, clock: Callable[[], float] = time.perf_counter):
        import torch
        self.device = torch.device(device)
        free, _ = torch.cuda.mem_get_info(self.device)
        self.arena_bytes = int(min(free * memory_fraction / max(1, lanes), max_arena))
        self.max_jobs = min(max_jobs, phy.BATCH_MAX_JOBS)
        self.clock = clock
        self.lanes = [_Lane(self.device, self.arena_bytes, poll_limit) for _ in range(lanes)]
        self.batches = 0
        self.batch_sizes: List[int] = []
        self.service: List[float] = []
        self.host_post: List[float] = []  # host seconds per batch: records, table, doorbell
        self._layouts: Dict[int, _JobLayout] = {}

    def _layout(self, cfg: phy.SlotConfig) -> _JobLayout:
        """The configuration's layout, cached by object (configurations are shared by the jobs
        of one stream; the cache keeps each object alive, so its id is not reused)."""
        lay = self._layouts.get(id(cfg))
        if lay is None or lay.cfg is not cfg:
            lay = self._layouts[id(cfg)] = _JobLayout(cfg)
        return lay

    def job_bytes(self, cfg: phy.SlotConfig) -> int:
        return self._layout(cfg).total

    def prepare(self, warm: "MixedJob"):
        """Captures every lane's graph (before timing), warming each on one job."""
        for ln in self.lanes:
            ln.capture([warm], self._layout)

    def _take(self, waiting: "collections.deque", busy=frozenset()) -> List["MixedJob"]:
        """The arrival-order jobs that fit one lane: up to max_jobs and the arena's bytes. A job
        that tracks its noise level waits (keeping its place) while an earlier job of this batch
        updates the same state, or a batch in flight does (`busy`): one cell's slots then update
        its state in arrival order. When every waiting job waits on a batch in flight, they form
        a batch anyway, and run() starts it on the GPU after those batches (the lanes' streams
        are chained) instead of waiting for them on the host."""
        batch, used, states, skipped = [], 0, set(busy), []

        def fill():
            nonlocal used
            while waiting and len(batch) < self.max_jobs:
                j = waiting[0]
                st = j._addr[3]
                if st is not None and st in states:
                    skipped.append(waiting.popleft())
                    continue
                b = self.job_bytes(j.cfg)
                if b > self.arena_bytes:
                    raise ValueError(f"job {j.job_id} needs {b} bytes, above the arena")
                if used + b + _ALIGN > self.arena_bytes:
                    break
                used += b
                if st is not None:
                    states.add(st)
                batch.append(waiting.popleft())
            waiting.extendleft(reversed(skipped))
            skipped.clear()

        fill()
        if not batch and busy:  # all waiting on batches in flight: chain on the GPU
            states.clear()
            fill()
        return batch

    def run(self, jobs: Sequence["MixedJob"], realtime: bool = True,
            keep: bool = False) -> List["MixedJob"]:
        """Serves jobs in arrival order (see SlotServer.run for realtime and the clock)."""
        import collections
        import torch
        pending = sorted(jobs, key=lambda j: j.arrival)
        waiting: collections.deque = collections.deque()
        finished: List[MixedJob] = []
        inflight = collections.deque()  # (lane, start event, end event, batch)
        free = list(range(len(self.lanes)))
        torch.cuda.synchronize(self.device)
        ref = torch.cuda.Event(enable_timing=True)
        ref.record(self.lanes[0].stream)
        t0 = self.clock()
        ref.synchronize()

        def retire(block: bool):
            while inflight and (block or inflight[0][2].query()):
                li, e0, e1, batch = inflight.popleft()
                e1.synchronize()
                st = phy.batch_status(self.lanes[li].host)
                if st != 0:
                    raise RuntimeError(f"batch of {len(batch)} jobs ended with status {st}")
                t = ref.elapsed_time(e1) * 1e-3
                self.service.append(e0.elapsed_time(e1) * 1e-3)
                for j in batch:
                    j.done = t
                    if keep:
                        j._views = (j.llr.clone(), j.flags.clone())
                        j._out = None
                finished.extend(batch)
                free.append(li)
                block = False

        i = 0
        while i < len(pending) or waiting:
            now = self.clock() - t0
            while i < len(pending) and (not realtime or pending[i].arrival <= now):
                waiting.append(pending[i])
                i += 1
            retire(False)
            if not waiting:
                if realtime and i < len(pending):
                    while self.clock() - t0 < pending[i].arrival:
                        retire(False)
                continue
            if not free:
                retire(True)
            busy = frozenset(j._addr[3] for f in inflight for j in f[3] if j._addr[3] is not None)
            batch = self._take(waiting, busy)
            if not batch:
                raise ValueError(f"job {waiting[0].job_id} does not fit a lane's arena")
            # the latest batch in flight that updates each noise state this batch reads
            last = {j._addr[3]: f[2] for f in inflight for j in f[3] if j._addr[3] is not None}
            deps = {id(e): e for e in (last.get(j._addr[3]) for j in batch
                                       if j._addr[3] is not None) if e is not None}
            li = free.pop(0)
            ln = self.lanes[li]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h0 = self.clock()
            ln.post(batch, self._layout)
            self.host_post.append(self.clock() - h0)
            for e in deps.values():  # ordered on the GPU, not by the host
                ln.stream.wait_event(e)
            e0.record(ln.stream)
            with torch.cuda.stream(ln.stream):
                ln.graph.replay()
            e1.record(ln.stream)
            inflight.append((li, e0, e1, batch))
            self.batches += 1
            self.batch_sizes.append(len(batch))
        while inflight:
            retire(True)
        return finished
