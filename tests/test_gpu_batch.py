"""Batched receiver on the GPU: jobs of different shapes in one launch per stage and layer
class, each job's outputs bitwise those of phy_slot_run on that job alone; a captured graph of
the launch serving changing batches; and the gate's bounded wait running out when the host never
posts a table."""
import dataclasses

import numpy as np
import pytest

from paper_2510_07843_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_07843_gb300 import build, phy
    build.build()
    phy.load()
    return torch.device("cuda:0")


# (spec, seed, extra cfg) of a heterogeneous batch: every layer class, one and two DMRS
# symbols, every modulation, both LLR formats, multi-cell jobs, FP64 re-computation enabled,
# FP32 and FP16 tensor-core products
MIX = [
    (S.spec_massive_mimo(n_cells=1, n_prb=24), 501, {}),
    (S.SlotSpec(n_cells=2, n_prb=4, n_rx=4, n_layers=1, qm=2, dmrs_sym=(2,), snr_db=12.0), 502,
     {}),
    (S.spec_carrier_273prb(n_prb=40), 503, {"llr_format": "f16"}),
    (S.SlotSpec(n_prb=17, n_rx=32, n_layers=7, qm=6, dmrs_sym=(3,), snr_db=25.0, n_taps=6), 504,
     {"fp64_refactor": True}),
    (S.SlotSpec(n_prb=9, n_rx=64, n_layers=12, qm=8, dmrs_sym=(2, 11), snr_db=30.0), 505, {}),
    (S.SlotSpec(n_prb=33, n_rx=16, n_layers=3, qm=4, dmrs_sym=(2, 11), snr_db=18.0,
                doppler_hz=300.0), 506, {}),
    (S.SlotSpec(n_prb=1, n_rx=2, n_layers=2, qm=2, dmrs_sym=(0,), n_sym=2), 507, {}),
    # FP16 tensor-core products: every layer class
    (S.spec_massive_mimo(n_cells=2, n_prb=10), 508, {"precision": "fp16"}),
    (S.SlotSpec(n_prb=23, n_rx=32, n_layers=6, qm=6, dmrs_sym=(2, 11), snr_db=25.0), 509,
     {"precision": "fp16", "llr_format": "f16"}),
    (S.SlotSpec(n_prb=14, n_rx=16, n_layers=4, qm=4, dmrs_sym=(2, 11), snr_db=20.0), 510,
     {"precision": "fp16"}),
    (S.SlotSpec(n_prb=5, n_rx=4, n_layers=1, qm=2, dmrs_sym=(2, 11), snr_db=15.0), 511,
     {"precision": "fp16"}),
]


def _prepare(dev, entries):
    """Inputs on the device and two output sets (batched, alone) per job."""
    import torch
    from paper_2510_07843_gb300 import phy
    jobs = []
    for spec, seed, kw in entries:
        sl = S.make_slot(spec, seed, keep_h=False)
        cfg = phy.SlotConfig.from_spec(spec, **kw)
        inp = [torch.from_numpy(a).to(dev) for a in (sl.Y, sl.pilots, sl.sigma2)]
        outs = [phy.SlotBuffers(cfg, device=dev, with_inputs=False) for _ in range(2)]
        for b in outs:
            b.flags.fill_(0xEE)
        jobs.append((cfg, inp, outs))
    return jobs


def _tuples(jobs, which=0):
    return [(cfg, *inp, o[which].x_hat, o[which].sinr, o[which].llr, o[which].flags)
            for cfg, inp, o in jobs]


def _tables(dev):
    import torch
    from paper_2510_07843_gb300 import phy
    n = phy.batch_table_bytes()
    host = torch.zeros(n, dtype=torch.uint8).pin_memory()
    devt = torch.zeros(n, dtype=torch.uint8, device=dev)
    return host, devt


def _alone(jobs):
    from paper_2510_07843_gb300 import phy
    for cfg, (Y, P, s2), o in jobs:
        b = o[1]
        phy.slot_run(cfg, Y, P, s2, b.x_hat, b.sinr, b.llr, b.flags, b.workspace)


def _assert_same(jobs):
    import torch
    for cfg, _, (a, b) in jobs:
        for k in ("x_hat", "sinr", "llr", "flags"):
            va, vb = getattr(a, k), getattr(b, k)
            if not torch.equal(va, vb):
                bad = (va != vb).nonzero()[:5].tolist()
                raise AssertionError((cfg, k, bad, va.flatten()[:16].tolist(),
                                      vb.flatten()[:16].tolist()))
        assert not torch.any(a.flags == 0xEE)


def test_mixed_batch_equals_each_job_alone(dev):
    import torch
    from paper_2510_07843_gb300 import phy
    jobs = _prepare(dev, MIX)
    host, devt = _tables(dev)
    ws = torch.empty(phy.batch_workspace_size(_tuples(jobs)), dtype=torch.uint8, device=dev)
    phy.batch_post(_tuples(jobs), host, ws)
    phy.batch_launch(host, devt)
    _alone(jobs)
    torch.cuda.synchronize()
    assert phy.batch_status(host) == 0
    _assert_same(jobs)


def test_captured_launch_serves_changing_batches(dev):
    """One CUDA graph of phy_batch_launch, replayed for three different posted batches (the
    jobs in another order and mix each time)."""
    import torch
    from paper_2510_07843_gb300 import phy
    jobs = _prepare(dev, MIX)
    host, devt = _tables(dev)
    ws = torch.empty(phy.batch_workspace_size(_tuples(jobs)), dtype=torch.uint8, device=dev)
    st = torch.cuda.Stream(device=dev)
    # a first batch configures the kernels before capture
    phy.batch_post(_tuples(jobs[:1]), host, ws)
    phy.batch_launch(host, devt, stream=st)
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        phy.batch_launch(host, devt, stream=st)
    _alone(jobs)
    for order in ([6, 0, 3, 8], [1, 2, 4, 5, 10], [7, 9], list(range(len(MIX)))[::-1]):
        sub = [jobs[i] for i in order]
        for _, _, o in sub:
            o[0].flags.fill_(0xEE)
        phy.batch_post(_tuples(sub), host, ws)
        with torch.cuda.stream(st):
            g.replay()
        st.synchronize()
        torch.cuda.synchronize()
        assert phy.batch_status(host) == 0
        _assert_same(sub)


def test_gate_times_out_when_nothing_is_posted(dev):
    """The gate's bounded wait runs out (about 2 ms of polls) when the host never rings: the
    stages run on an empty table, no output is touched, the status is PHY_ERR_TIMEOUT; the next
    posted batch runs normally."""
    import torch
    from paper_2510_07843_gb300 import phy
    jobs = _prepare(dev, MIX[:2])
    host, devt = _tables(dev)
    ws = torch.empty(phy.batch_workspace_size(_tuples(jobs)), dtype=torch.uint8, device=dev)
    phy.batch_launch(host, devt, poll_limit=2000)
    torch.cuda.synchronize()
    assert phy.batch_status(host) == 5
    for _, _, o in jobs:
        assert torch.all(o[0].flags == 0xEE)
    # a batch that ran, then a launch without a new post: the old table is not run again
    phy.batch_post(_tuples(jobs), host, ws)
    phy.batch_launch(host, devt, poll_limit=2000)
    torch.cuda.synchronize()
    assert phy.batch_status(host) == 0
    for _, _, o in jobs:
        o[0].flags.fill_(0xEE)
    phy.batch_launch(host, devt, poll_limit=2000)
    torch.cuda.synchronize()
    assert phy.batch_status(host) == 5
    for _, _, o in jobs:
        assert torch.all(o[0].flags == 0xEE)


def test_batch_server_mixed_stream_equals_each_job_alone(dev):
    """The serving loop over the batched receiver: jobs of the serving configuration's shapes
    (4-273 PRB, 4-64 Rx, 1-16 layers, QPSK-256QAM) arriving as a Poisson stream, continuously
    batched on two lanes; every job's LLRs and flags equal phy_slot_run on the job alone."""
    import torch
    from paper_2510_07843_gb300 import phy, serve
    rng = np.random.default_rng(77)
    specs = [S.spec_serving_job(rng) for _ in range(10)]
    specs = [dataclasses.replace(s, n_prb=min(s.n_prb, 60)) for s in specs]  # test-sized
    pool = []
    for i, sp in enumerate(specs):
        sl = S.make_slot(sp, 900 + i, keep_h=False)
        cfg = phy.SlotConfig.from_spec(sp)
        pool.append((cfg, *(torch.from_numpy(a).to(dev) for a in (sl.Y, sl.pilots, sl.sigma2))))
    arrivals = S.serving_arrivals(8, 2000.0, 0.004, 3)
    jobs = [serve.MixedJob(pool[k % len(pool)][0], *pool[k % len(pool)][1:], arrival=t,
                           job_id=k) for k, (t, _) in enumerate(arrivals)]
    srv = serve.BatchServer(device=dev, lanes=2, memory_fraction=0.05)
    srv.prepare(jobs[0])
    done = srv.run(jobs, realtime=False, keep=True)
    assert len(done) == len(jobs) and srv.batches >= 1 and max(srv.batch_sizes) > 1
    ref = {}
    for k, (cfg, Y, P, s2) in enumerate(pool):
        b = phy.SlotBuffers(cfg, device=dev, with_inputs=False)
        phy.slot_run(cfg, Y, P, s2, b.x_hat, b.sinr, b.llr, b.flags, b.workspace)
        ref[k] = b
    torch.cuda.synchronize()
    for j in done:
        r = ref[j.job_id % len(pool)]
        assert torch.equal(j.llr, r.llr) and torch.equal(j.flags, r.flags), j.job_id


# (index into MIX, mode, alpha, prior state or None for a state set to 3x the true level) of the
# jobs that track their noise level on the device; a prior of 0 is an unset state
TRACK = [(0, "min", 0.5, 0.0), (2, "freq", 0.25, None), (3, "freq", 1.0, 0.0),
         (8, "time", 0.5, None), (9, "min", 0.75, 0.0)]


def test_noise_tracking_in_the_batch_equals_slot_run_track(dev):
    """Jobs with a device noise state (phy_job.noise_state) next to plain ones: over two batches
    each tracking job's outputs and state equal phy_slot_run_track on the job alone with the
    same state, bit for bit, and the plain jobs still equal phy_slot_run."""
    import torch
    from paper_2510_07843_gb300 import phy
    jobs = _prepare(dev, MIX)
    host, devt = _tables(dev)
    track = {i: (mode, alpha) for i, mode, alpha, _ in TRACK}
    states = {}
    for i, _, _, prior in TRACK:
        s2 = jobs[i][1][2]
        init = torch.full_like(s2, 0.0) if prior == 0.0 else 3.0 * s2
        states[i] = (init.clone(), init.clone())  # (batched, alone)
    for rnd in range(2):
        tuples = []
        for i, (cfg, inp, o) in enumerate(jobs):
            t = (cfg, *inp, o[0].x_hat, o[0].sinr, o[0].llr, o[0].flags)
            if i in track:
                t = t + (states[i][0], track[i][1], track[i][0])
            tuples.append(t)
        ws = torch.empty(phy.batch_workspace_size(tuples), dtype=torch.uint8, device=dev)
        for _, _, o in jobs:
            o[0].flags.fill_(0xEE)
        phy.batch_post(tuples, host, ws)
        phy.batch_launch(host, devt)
        for i, (cfg, (Y, P, s2), o) in enumerate(jobs):
            b = o[1]
            if i in track:
                phy.slot_run_track(cfg, track[i][0], track[i][1], Y, P, states[i][1], b.x_hat,
                                   b.sinr, b.llr, b.flags, b.workspace)
            else:
                phy.slot_run(cfg, Y, P, s2, b.x_hat, b.sinr, b.llr, b.flags, b.workspace)
        torch.cuda.synchronize()
        assert phy.batch_status(host) == 0
        _assert_same(jobs)
        for i in track:
            a, b = states[i]
            assert torch.equal(a, b), (rnd, i, a.tolist(), b.tolist())
            assert torch.all(torch.isfinite(a)) and torch.all(a > 0)


def test_batch_server_tracks_each_cells_noise_in_arrival_order(dev):
    """Four cells, three slots each, all arriving at once, every job tracking its cell's noise
    level: the server never puts two slots of one cell in one batch, and a batch holding a
    cell's later slot starts on the GPU only after the batch in flight with its earlier slot
    (the lanes' streams are chained, the host does not wait), so each cell's state follows its
    slots in arrival order; outputs and final states equal per-cell sequences of
    phy_slot_run_track."""
    import torch
    from paper_2510_07843_gb300 import phy, serve
    specs = [S.SlotSpec(n_prb=12, n_rx=16, n_layers=4, qm=4, dmrs_sym=(2, 11), snr_db=15.0),
             S.SlotSpec(n_prb=8, n_rx=32, n_layers=8, qm=6, dmrs_sym=(2, 11), snr_db=22.0),
             S.SlotSpec(n_prb=20, n_rx=4, n_layers=2, qm=2, dmrs_sym=(2, 11), snr_db=10.0),
             S.SlotSpec(n_prb=6, n_rx=64, n_layers=16, qm=8, dmrs_sym=(2, 11), snr_db=28.0)]
    slots = []  # (cell, cfg, inputs) in arrival order: slot r of every cell, then r + 1
    for r in range(3):
        for c, sp in enumerate(specs):
            sl = S.make_slot(sp, 1200 + 10 * c + r, keep_h=False)
            cfg = phy.SlotConfig.from_spec(sp, precision="fp16" if sp.n_layers > 4 else "fp32")
            slots.append((c, cfg, [torch.from_numpy(a).to(dev) for a in (sl.Y, sl.pilots,
                                                                         sl.sigma2)]))
    state = [torch.zeros(1, device=dev) for _ in specs]
    jobs = [serve.MixedJob(cfg, *inp, arrival=0.0, job_id=k, noise_state=state[c],
                           noise_alpha=0.5, noise_mode="min")
            for k, (c, cfg, inp) in enumerate(slots)]
    srv = serve.BatchServer(device=dev, lanes=2, memory_fraction=0.05)
    srv.prepare(serve.MixedJob(slots[0][1], *slots[0][2]))
    done = srv.run(jobs, realtime=False, keep=True)
    assert len(done) == len(jobs)
    ref_state = [torch.zeros(1, device=dev) for _ in specs]
    by_id = {j.job_id: j for j in done}
    for k, (c, cfg, (Y, P, s2)) in enumerate(slots):
        b = phy.SlotBuffers(cfg, device=dev, with_inputs=False)
        phy.slot_run_track(cfg, "min", 0.5, Y, P, ref_state[c], b.x_hat, b.sinr, b.llr, b.flags,
                           b.workspace)
        torch.cuda.synchronize()
        assert torch.equal(by_id[k].llr, b.llr) and torch.equal(by_id[k].flags, b.flags), k
    for c in range(len(specs)):
        assert torch.equal(state[c], ref_state[c]), (c, state[c].tolist(), ref_state[c].tolist())
