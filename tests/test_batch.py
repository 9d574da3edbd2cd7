"""Batched receiver (phy_batch_*): host-side validation and the job table the host writes.

phy_batch_post is host-only (it writes the caller's table and lays out intermediates by
arithmetic; no CUDA call), so these tests pass fake device addresses that are never read and a
plain host buffer as the table. The GPU behaviour is in tests/test_gpu_batch.py."""
import ctypes

import numpy as np
import pytest

from paper_2510_07843_gb300 import build, phy

FAKE = 1 << 24  # a 256-byte aligned address that nothing dereferences here


@pytest.fixture(scope="module")
def lib():
    build.build()
    return phy.load()


def _job(cfg, base=FAKE):
    return (cfg, base, base, base, base, base, base, base)


def _table():
    """A zeroed host table, 128-byte aligned (a view into a larger buffer)."""
    n = phy.batch_table_bytes()
    assert n % 128 == 0
    raw = np.zeros(n // 8 + 16, dtype=np.uint64)
    off = (-raw.ctypes.data % 128) // 8
    return raw[off:off + n // 8]


def _post(jobs, table, ws_bytes=1 << 40):
    arr = phy._jobs_array(jobs)
    return phy.load().phy_batch_post(arr, len(jobs), table.ctypes.data, FAKE, ws_bytes)


def _words(table):
    return table.view(np.uint32)


def _items(cfg):
    """(LS, segment, solve) work items of one job and its layer class index."""
    n_sc = 12 * cfg.n_prb
    L = 1
    while L < (cfg.n_layers + 1) // 2:
        L *= 2
    G = -(-(n_sc // 2) // L)
    n_seg = max(G - 1, 1)
    nds = cfg.n_sym - len(cfg.dmrs_sym)
    nlc = next(c for c in (2, 4, 8, 16) if cfg.n_layers <= c)
    # LS items take 128 / (n_rx padded to a power of two) groups each
    nrp = 1
    while nrp < cfg.n_rx:
        nrp *= 2
    ls = -(-G // (128 // nrp)) * len(cfg.dmrs_sym) * cfg.n_cells
    if nlc <= 4:  # the direct form: no segment stage
        return ((ls, 0, -(-n_sc // 128) * nds * cfg.n_cells), (2, 4, 8, 16).index(nlc))
    return ((ls, n_seg * cfg.n_cells, -(-n_sc // 128) * nds * cfg.n_cells),
            (2, 4, 8, 16).index(nlc))


MIX = [phy.SlotConfig(n_cells=1, n_prb=273, n_rx=64, n_layers=16, qm=8, dmrs_sym=(2, 11)),
       phy.SlotConfig(n_cells=2, n_prb=4, n_rx=4, n_layers=1, qm=2, dmrs_sym=(2,)),
       phy.SlotConfig(n_cells=1, n_prb=51, n_rx=16, n_layers=3, qm=6, dmrs_sym=(2, 11),
                      llr_format="f16"),
       phy.SlotConfig(n_cells=1, n_prb=100, n_rx=32, n_layers=7, qm=4, dmrs_sym=(3,),
                      fp64_refactor=True),
       phy.SlotConfig(n_cells=1, n_prb=13, n_rx=64, n_layers=12, qm=8, dmrs_sym=(2, 11))]


def test_post_writes_the_table_and_rings_the_doorbell(lib):
    t = _table()
    assert _post([_job(c) for c in MIX], t) == 0
    w = _words(t)
    assert w[0] == 1 and w[2] == 0 and w[3] == len(MIX)  # seq bumped, status pending, n_jobs
    # stages: LS, FP32 segment, tensor-core segment, solve, direct, noise partial sums, noise
    n_items = w[4:32].reshape(7, 4)
    want = np.zeros((7, 4), dtype=np.int64)
    for c in MIX:
        (ls, seg, solve), cls = _items(c)
        want[0, 0] += ls
        if cls <= 1:
            want[4, cls] += solve
        else:
            want[1, cls] += seg
            want[3, cls] += solve
    assert np.array_equal(n_items, want)
    assert _post([_job(MIX[0])], t) == 0 and w[0] == 2  # every post rings again


def test_workspace_size_is_the_sum_over_jobs(lib):
    one = [phy.batch_workspace_size([_job(c)]) for c in MIX]
    assert all(v > 0 for v in one)
    assert phy.batch_workspace_size([_job(c) for c in MIX]) == sum(one)
    t = _table()
    assert _post([_job(c) for c in MIX], t, ws_bytes=sum(one) - 1) == 3  # PHY_ERR_NO_MEMORY
    assert _post([_job(c) for c in MIX], t, ws_bytes=sum(one)) == 0


@pytest.mark.parametrize("bad,code", [
    (dict(precision="bf16"), 2),          # products in FP32 or FP16 on this path
    (dict(precision="fp16", dmrs_sym=(2,)), 2),  # tensor-core jobs need two DMRS symbols
    (dict(occ_len=16, n_layers=16), 2),   # forced cover length other than the automatic one
    (dict(n_layers=17), 1),
    (dict(qm=5), 1),
])
def test_post_rejects_unsupported_jobs(lib, bad, code):
    base = dict(n_cells=1, n_prb=20, n_rx=16, n_layers=4, qm=4, dmrs_sym=(2, 11))
    base.update(bad)
    t = _table()
    assert _post([_job(MIX[1]), _job(phy.SlotConfig(**base))], t) == code
    assert _words(t)[0] == 0  # nothing rung


def test_post_rejects_bad_counts_and_pointers(lib):
    t = _table()
    arr = phy._jobs_array([_job(MIX[1])])
    assert lib.phy_batch_post(arr, 0, t.ctypes.data, FAKE, 1 << 30) == 1
    many = phy._jobs_array([_job(MIX[1])] * 65)
    assert lib.phy_batch_post(many, 65, t.ctypes.data, FAKE, 1 << 30) == 1
    assert lib.phy_batch_post(arr, 1, None, FAKE, 1 << 30) == 1
    assert lib.phy_batch_post(arr, 1, t.ctypes.data, FAKE + 8, 1 << 30) == 1  # workspace align
    assert lib.phy_batch_post(arr, 1, t.ctypes.data + 8, FAKE, 1 << 30) == 1  # table align
    assert _post([_job(MIX[1], base=FAKE + 8)], t) == 1  # grid not 16-byte aligned
    assert lib.phy_batch_status(None) == 1
    assert lib.phy_batch_status(ctypes.c_void_p(t.ctypes.data)) == 1  # nothing ran


def _noise_blocks(cfg):
    """Partial-sum blocks per cell of the noise estimate: 1024 anchor entries each."""
    n_sc = 12 * cfg.n_prb
    L = 1
    while L < (cfg.n_layers + 1) // 2:
        L *= 2
    G = -(-(n_sc // 2) // L)
    return -(-(G * cfg.n_layers * cfg.n_rx) // 1024)


def _job_track(cfg, state, alpha=0.5, mode="min"):
    return (cfg, FAKE, FAKE, None, None, None, FAKE, FAKE, state, alpha, mode)


def test_noise_tracking_jobs_add_the_noise_stages(lib):
    """Jobs with a device noise state add (partial-sum block, cell) and cell items to the two
    noise stages; other jobs add none, and a tracking job needs no sigma2."""
    t = _table()
    jobs = [_job(MIX[1]), _job_track(MIX[0], FAKE + 4096), _job_track(MIX[3], FAKE + 8192,
                                                                    mode="freq")]
    assert _post(jobs, t) == 0
    n_items = _words(t)[4:32].reshape(7, 4)
    assert n_items[5, 0] == sum(_noise_blocks(c) * c.n_cells for c in (MIX[0], MIX[3]))
    assert n_items[6, 0] == MIX[0].n_cells + MIX[3].n_cells
    assert n_items[5:, 1:].sum() == 0


@pytest.mark.parametrize("alpha,mode,code", [(0.0, "min", 1), (1.5, "min", 1), (0.5, 3, 1),
                                             (0.5, "time", 1), (1.0, "freq", 0)])
def test_noise_tracking_fields_are_validated(lib, alpha, mode, code):
    one_dmrs = phy.SlotConfig(n_cells=1, n_prb=20, n_rx=16, n_layers=4, qm=4, dmrs_sym=(2,))
    t = _table()
    assert _post([_job_track(one_dmrs, FAKE, alpha, mode)], t) == code


def test_tracking_jobs_may_not_share_state(lib):
    two = phy.SlotConfig(n_cells=2, n_prb=20, n_rx=16, n_layers=4, qm=4, dmrs_sym=(2, 11))
    one = phy.SlotConfig(n_cells=1, n_prb=20, n_rx=16, n_layers=4, qm=4, dmrs_sym=(2, 11))
    t = _table()
    # the first job's state covers FAKE and FAKE + 4: a second state at FAKE + 4 overlaps it
    assert _post([_job_track(two, FAKE), _job_track(one, FAKE + 4)], t) == 1
    assert _words(t)[0] == 0
    assert _post([_job_track(two, FAKE), _job_track(one, FAKE + 8)], t) == 0
