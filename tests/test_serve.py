"""Serving slot loop: host-side batching and admission (CPU), and on the GPU that every job's
result in a mixed, batched stream equals its result alone."""
import dataclasses

import numpy as np
import pytest

from paper_2510_07843_gb300 import phy, serve
from paper_2510_07843_gb300 import synth as S

SMALL = phy.SlotConfig(n_cells=1, n_prb=51, n_rx=4, n_layers=2, qm=4, dmrs_sym=(2,))
CARRIER = phy.SlotConfig(n_cells=1, n_prb=25, n_rx=16, n_layers=4, qm=6, dmrs_sym=(2, 11))
MASSIVE = phy.SlotConfig(n_cells=1, n_prb=273, n_rx=64, n_layers=16, qm=8, dmrs_sym=(2, 11))


def test_batch_sizes_and_pick():
    assert serve.batch_sizes(8) == [1, 2, 4, 8]
    assert serve.batch_sizes(6) == [1, 2, 4]
    assert serve.batch_sizes(0) == [1]
    assert [serve.pick_batch(n, 8) for n in (1, 2, 3, 5, 8, 20)] == [1, 2, 2, 4, 8, 8]
    assert serve.pick_batch(7, 3) == 2


def test_config_key_ignores_cell_count():
    a = dataclasses.replace(MASSIVE, n_cells=3)
    assert serve.config_key(a) == serve.config_key(MASSIVE)
    assert serve.config_key(SMALL) != serve.config_key(CARRIER)
    assert serve.config_key(dataclasses.replace(MASSIVE, precision="fp16")) != \
        serve.config_key(MASSIVE)


def test_admission_by_device_memory():
    phy.load()
    per = serve.bytes_per_cell(MASSIVE)
    assert per > serve.bytes_per_cell(CARRIER) > serve.bytes_per_cell(SMALL)
    assert serve.admission_limit(MASSIVE, 3 * per + 1, 8) == 3
    assert serve.admission_limit(MASSIVE, per // 2, 8) == 1  # one cell is always admitted
    assert serve.admission_limit(SMALL, 1 << 40, 8) == 8


class _FakeGraph:
    stream = None

    def __init__(self, log, key, n):
        self.log, self.key, self.n = log, key, n

    def launch(self, jobs, keep=True):
        assert len(jobs) == self.n
        self.log.append((self.key, [j.job_id for j in jobs]))


class _FakeEvent:
    def record(self, stream):
        pass

    def query(self):
        return True

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 0.0


def test_scheduling_oldest_first_powers_of_two(monkeypatch):
    phy.load()
    log = []
    srv = serve.SlotServer(max_cells=4, memory_budget=1 << 40)
    srv.streams = [None]  # host-only: no CUDA streams, events or graphs
    monkeypatch.setattr(srv, "_graph",
                        lambda cfg, n, lane=0: _FakeGraph(log, serve.config_key(cfg)[0], n))
    monkeypatch.setattr(srv, "_event", lambda: _FakeEvent())
    monkeypatch.setattr(srv, "_sync", lambda: None)
    jobs = ([serve.Job(SMALL, None, None, 1.0, arrival=0.5, job_id=i) for i in range(5)] +
            [serve.Job(CARRIER, None, None, 1.0, arrival=0.0, job_id=10 + i) for i in range(3)])
    jobs[5].arrival = -1.0  # the oldest job is a CARRIER one
    done = srv.run(jobs, realtime=False)
    assert sorted(j.job_id for j in done) == sorted(j.job_id for j in jobs)
    # CARRIER first (oldest waiting job), as 2 + 1; SMALL as 4 + 1
    assert [len(b) for _, b in log] == [2, 1, 4, 1]
    assert log[0][1] == [10, 11] and log[1][1] == [12]
    assert log[2][1] == [0, 1, 2, 3] and log[3][1] == [4]


@pytest.mark.gpu
@pytest.mark.parametrize("streams", [1, 2])
def test_mixed_jobs_equal_alone(streams):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_07843_gb300 import build
    build.build()
    phy.load()
    dev = torch.device("cuda:0")
    specs = {"small": (S.spec_small_51prb(), SMALL), "carrier": (S.spec_carrier_273prb(n_prb=25),
                                                                 CARRIER)}
    jobs, rng = [], np.random.default_rng(5)
    for n in range(14):
        name = "small" if rng.random() < 0.5 else "carrier"
        spec, cfg = specs[name]
        sl = S.make_slot(spec, 700 + n, keep_h=False)
        jobs.append(serve.Job(cfg, torch.from_numpy(sl.Y).to(dev),
                              torch.from_numpy(sl.pilots).to(dev), float(sl.sigma2[0]),
                              arrival=0.0, job_id=n))
    srv = serve.SlotServer(device=dev, max_cells=4, streams=streams)
    srv.prepare([SMALL, CARRIER])
    done = srv.run(jobs, realtime=False)
    assert len(done) == len(jobs) and srv.batches < len(jobs)
    for j in jobs:  # each job alone, plain call
        cfg = dataclasses.replace(j.cfg, n_cells=1)
        b = phy.SlotBuffers(cfg, device=dev)
        b.Y.copy_(j.Y)
        b.pilots.copy_(j.pilots)
        b.sigma2.fill_(j.sigma2)
        phy.slot_run(cfg, b.Y, b.pilots, b.sigma2, b.x_hat, b.sinr, b.llr, b.flags, b.workspace)
        torch.cuda.synchronize()
        assert torch.equal(b.llr, j.llr), j.job_id
        assert torch.equal(b.flags, j.flags), j.job_id
    summ = serve.latency_summary(done)
    print("mixed batch latency:", summ)
    assert summ["jobs"] == len(jobs)


@pytest.mark.gpu
def test_zero_copy_batches_equal_alone():
    """Jobs that are consecutive cells of one resident input are read in place (no copies, no
    graph); each result still equals the job run alone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_07843_gb300 import build
    build.build()
    phy.load()
    dev = torch.device("cuda:0")
    spec = S.spec_carrier_273prb(n_prb=25, n_cells=4)
    sl = S.make_slot(spec, 811, keep_h=False)
    Y = torch.from_numpy(sl.Y).to(dev)
    P = torch.from_numpy(sl.pilots).to(dev)
    s2 = torch.from_numpy(sl.sigma2).to(dev)
    jobs = [serve.Job(CARRIER, Y[c:c + 1], P[c:c + 1], float(sl.sigma2[c]), job_id=c,
                      sigma2_dev=s2[c:c + 1]) for c in range(4)]
    assert serve._direct(jobs)
    srv = serve.SlotServer(device=dev, max_cells=4)
    done = srv.run(jobs, realtime=False)
    assert srv.batches == 1 and len(done) == 4
    for j in jobs:
        b = phy.SlotBuffers(CARRIER, device=dev)
        b.Y.copy_(j.Y)
        b.pilots.copy_(j.pilots)
        b.sigma2.copy_(j.sigma2_dev)
        phy.slot_run(CARRIER, b.Y, b.pilots, b.sigma2, b.x_hat, b.sinr, b.llr, b.flags,
                     b.workspace)
        torch.cuda.synchronize()
        assert torch.equal(b.llr, j.llr) and torch.equal(b.flags, j.flags), j.job_id


@pytest.mark.gpu
def test_noise_state_tracked_through_the_server():
    """Four cells of a resident input ring, served twice with noise tracking: each cell's noise
    level lives in its device slot between the rounds, and the served results and states equal
    the same cells run by phy_slot_run_track one at a time on a copy of the state."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_07843_gb300 import build
    build.build()
    phy.load()
    dev = torch.device("cuda:0")
    spec = S.spec_carrier_273prb(n_prb=25, n_cells=4)
    Y = torch.empty((4, 14, spec.n_rx, spec.n_sc), dtype=torch.complex64, device=dev)
    P = torch.empty((4, 2, spec.n_layers, spec.n_sc), dtype=torch.complex64, device=dev)
    state = torch.zeros(4, dtype=torch.float32, device=dev)  # unset: the first round sets it
    ref_state = state.clone()
    srv = serve.SlotServer(device=dev, max_cells=4)
    for rnd in range(2):
        sl = S.make_slot(spec, 900 + rnd, keep_h=False)  # new slot data in the same ring
        Y.copy_(torch.from_numpy(sl.Y))
        P.copy_(torch.from_numpy(sl.pilots))
        jobs = [serve.Job(CARRIER, Y[c:c + 1], P[c:c + 1], 0.0, job_id=c,
                          sigma2_dev=state[c:c + 1], noise_alpha=0.25) for c in range(4)]
        done = srv.run(jobs, realtime=False)
        assert len(done) == 4
        for j in jobs:
            c = j.job_id
            b = phy.SlotBuffers(CARRIER, device=dev)
            phy.slot_run_track(CARRIER, "min", 0.25, j.Y, j.pilots, ref_state[c:c + 1], b.x_hat,
                               b.sinr, b.llr, b.flags, b.workspace)
            torch.cuda.synchronize()
            assert torch.equal(b.llr, j.llr) and torch.equal(b.flags, j.flags), (rnd, c)
        assert torch.equal(state, ref_state)
        assert torch.all(state > 0)


def test_noise_tracking_jobs_batch_apart(monkeypatch):
    """Jobs that track their noise level and jobs with a given one never share a batch (the
    captured receivers differ), even with the same configuration."""
    phy.load()
    log = []
    srv = serve.SlotServer(max_cells=4, memory_budget=1 << 40)
    srv.streams = [None]
    monkeypatch.setattr(srv, "_graph",
                        lambda cfg, n, lane=0: _FakeGraph(log, serve.config_key(cfg)[0], n))
    monkeypatch.setattr(srv, "_event", lambda: _FakeEvent())
    monkeypatch.setattr(srv, "_sync", lambda: None)
    jobs = [serve.Job(SMALL, None, None, 1.0, arrival=0.1 * i, job_id=i,
                      noise_alpha=0.25 if i % 2 else 0.0) for i in range(6)]
    done = srv.run(jobs, realtime=False)
    assert sorted(j.job_id for j in done) == list(range(6))
    for _, ids in log:
        assert len({ids_i % 2 for ids_i in ids}) == 1, ids
    assert sorted(len(b) for _, b in log) == [1, 1, 2, 2]


def test_batch_records_match_the_ctypes_jobs():
    """The serving loop writes phy_job records into a byte buffer; each record equals the
    ctypes phy_job of the same configuration and addresses, and the outputs follow the
    intermediates in the arena, 256-byte aligned and disjoint."""
    import ctypes
    import numpy as np
    from paper_2510_07843_gb300 import synth as S
    phy.load()
    rng = np.random.default_rng(3)
    cfgs = [phy.SlotConfig.from_spec(S.spec_serving_job(rng)) for _ in range(12)]
    lays = [serve._JobLayout(c) for c in cfgs]
    addrs = [(1 << 32) + 4096 * i for i in range(12)]
    base = 1 << 40
    rec = bytearray(12 * phy.JOB_BYTES)
    # every third job tracks its noise level on the device (a state address, alpha, mode)
    tracked = [(a + 48, 0.25, 1) if i % 3 == 0 else (None, 0.0, 2) for i, a in enumerate(addrs)]
    ws, outs, end = serve.write_records(memoryview(rec), lays,
                                        [(a, a + 16, a + 32) + tr for a, tr in zip(addrs, tracked)],
                                        base)
    assert sum(l.ws for l in lays) == phy.batch_workspace_size([(c,) + (None,) * 7 for c in cfgs])
    assert ws == serve._up(sum(l.ws for l in lays))
    spans = []
    for i, (c, a, (lo, fo)) in enumerate(zip(cfgs, addrs, outs)):
        st, alpha, mode = tracked[i]
        want = phy._jobs_array([(c, a, a + 16, a + 32, None, None, base + lo, base + fo, st,
                                 alpha, mode)])
        assert bytes(rec[i * phy.JOB_BYTES:(i + 1) * phy.JOB_BYTES]) == bytes(want[0])
        assert lo % 256 == 0 and fo % 256 == 0 and lo >= ws
        spans += [(lo, lo + lays[i].llr), (fo, fo + lays[i].flags)]
    spans.sort()
    assert all(b[0] >= a[1] for a, b in zip(spans, spans[1:])) and spans[-1][1] <= end
    assert ctypes.sizeof(phy.CJob) == phy.JOB_BYTES


def test_batch_forming_defers_jobs_whose_noise_state_is_busy():
    """BatchServer._take, the host logic that keeps one cell's noise-state updates in arrival
    order: no two jobs of one state in a batch; jobs whose state a batch in flight updates wait
    (keeping their places) while independent jobs go; and when every waiting job waits, they
    form a batch anyway (run() then chains it on the GPU after the batches in flight)."""
    import collections

    class _Job:
        def __init__(self, job_id, state):
            self.job_id, self.cfg = job_id, None
            self._addr = (0, 0, 0, state, 0.5, 0)

    srv = serve.BatchServer.__new__(serve.BatchServer)  # the batch-forming state only
    srv.max_jobs, srv.arena_bytes = 4, 1 << 30
    srv.job_bytes = lambda cfg: 1 << 10

    def take(states, busy=frozenset()):
        waiting = collections.deque(_Job(i, s) for i, s in enumerate(states))
        batch = srv._take(waiting, frozenset(busy))
        return [j.job_id for j in batch], [j.job_id for j in waiting]

    # within a batch: a state's second job waits, later independent jobs still join
    assert take([7, 7, None, 8, 7]) == ([0, 2, 3], [1, 4])
    # a state in flight: its jobs wait in place, the rest fill the batch (up to max_jobs)
    assert take([7, None, 7, 8, 9, 10], busy={7}) == ([1, 3, 4, 5], [0, 2])
    # every waiting job waits on a batch in flight: they form one batch, one job per state
    assert take([7, 8, 7], busy={7, 8}) == ([0, 1], [2])
    # nothing busy, nothing tracked: plain arrival order up to max_jobs
    assert take([None] * 6) == ([0, 1, 2, 3], [4, 5])
    # the arena bounds a batch (jobs' bytes plus one alignment pad): the rest stay waiting
    srv.arena_bytes = 2 * (1 << 10) + serve._ALIGN
    assert take([None] * 5) == ([0, 1], [2, 3, 4])
