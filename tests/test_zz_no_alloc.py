"""phy_slot_run_noalloc: the receiver for callers that may not allocate device memory.

Such callers (a real-time slot loop that must not stall on an allocation, or a plugin whose
host framework owns all device memory) pass only inputs and outputs; the library keeps its
scratch in one fixed device array. These tests check that this entry point gives the same
results as phy_slot_run, call after call, and that it refuses work that does not fit the array.
This file is collected last so that a failure here cannot hide the other tests' results.
"""
import ctypes

import numpy as np
import pytest

from paper_2510_07843_gb300 import synth as S
from parity import LLR_ABS, X_REL, rel_fro


def _slot(seed, n_cells=2, n_prb=8):
    spec = S.spec_massive_mimo(n_cells=n_cells, n_prb=n_prb)
    return spec, S.make_slot(spec, seed, keep_h=False)


def test_noalloc_rejects_configs_beyond_the_fixed_scratch():
    """No GPU work: the size check answers before anything is enqueued. The configuration's LS
    anchors alone (which every chunk schedule keeps for all cells) exceed the array, so the
    rejection does not depend on how small the per-cell detection scratch is."""
    from paper_2510_07843_gb300 import build, phy
    build.build()
    lib = phy.load()
    big = phy.SlotConfig(n_cells=32, n_prb=273, n_rx=64, n_layers=16, qm=8, dmrs_sym=(2, 11))
    anchors = big.n_cells * 2 * phy.n_groups(big) * big.n_layers * big.n_rx * 8
    assert anchors > 1.5 * phy.NOALLOC_SCRATCH_BYTES
    c = big.c()
    fake = ctypes.c_void_p(256)  # never dereferenced
    rc = lib.phy_slot_run_noalloc(ctypes.byref(c), fake, fake, fake, fake, fake, fake, fake, None)
    assert rc == 3  # PHY_ERR_NO_MEMORY


@pytest.mark.gpu
def test_noalloc_matches_slot_run_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_07843_gb300 import build, phy
    build.build()
    phy.load()
    dev = torch.device("cuda:0")
    # two different slots back to back: the second call must not see the first call's scratch;
    # the second is the full 8-cell 273-PRB 64x16 batch, which runs in chunks of cells
    for seed, n_cells, n_prb in ((61, 2, 8), (62, 8, 273)):
        spec, sl = _slot(seed, n_cells, n_prb)
        cfg = phy.SlotConfig.from_spec(spec)
        Y = torch.from_numpy(sl.Y).to(dev)
        P = torch.from_numpy(sl.pilots).to(dev)
        s2 = torch.from_numpy(sl.sigma2).to(dev)
        ref = phy.SlotBuffers(cfg, device=dev, with_inputs=False)
        got = phy.SlotBuffers(cfg, device=dev, with_inputs=False)
        phy.slot_run(cfg, Y, P, s2, ref.x_hat, ref.sinr, ref.llr, ref.flags, ref.workspace)
        phy.slot_run_noalloc(cfg, Y, P, s2, got.x_hat, got.sinr, got.llr, got.flags)
        torch.cuda.synchronize()
        xr, xg = ref.x_hat.cpu().numpy(), got.x_hat.cpu().numpy()
        sr, sg = ref.sinr.cpu().numpy(), got.sinr.cpu().numpy()
        lr, lg = ref.llr.cpu().numpy(), got.llr.cpu().numpy()
        assert rel_fro(xg, xr) <= X_REL
        assert np.max(np.abs(sg - sr) / sr) <= 1e-6
        assert np.max(np.abs(lg - lr) / sr[..., None]) <= LLR_ABS
        assert np.array_equal(got.flags.cpu().numpy(), ref.flags.cpu().numpy())
