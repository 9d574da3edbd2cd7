"""Chunk autotuner (phy_autotune): picks a chunk size that fits the workspace, and a tuned
configuration computes exactly what an untuned one does (chunking does not change arithmetic)."""
import numpy as np
import pytest

from paper_2510_07843_gb300 import synth as S


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_07843_gb300 import build, phy
    build.build()
    phy.load()
    return torch.device("cuda:0")


@pytest.mark.gpu
def test_autotune_picks_a_fitting_chunk_and_keeps_results(dev):
    import torch
    from paper_2510_07843_gb300 import phy
    spec = S.spec_massive_mimo(n_cells=4, n_prb=12)
    sl = S.make_slot(spec, 3100, keep_h=False)
    cfg = phy.SlotConfig.from_spec(spec)
    buf = phy.SlotBuffers(cfg, device=dev)
    buf.Y.copy_(torch.from_numpy(sl.Y))
    buf.pilots.copy_(torch.from_numpy(sl.pilots))
    buf.sigma2.copy_(torch.from_numpy(sl.sigma2))
    args = (buf.Y, buf.pilots, buf.sigma2, buf.x_hat, buf.sinr, buf.llr, buf.flags, buf.workspace)
    phy.autotune_clear()
    phy.slot_run(cfg, *args)
    torch.cuda.synchronize()
    ref = [t.cpu().numpy().copy() for t in (buf.x_hat, buf.sinr, buf.llr, buf.flags)]
    chunk = phy.autotune(cfg, *args)
    assert chunk in (1, 2, 4)
    got = [t.cpu().numpy().copy() for t in (buf.x_hat, buf.sinr, buf.llr, buf.flags)]
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    phy.slot_run(cfg, *args)  # a later call with the same cfg uses the tuned chunk
    torch.cuda.synchronize()
    again = [t.cpu().numpy().copy() for t in (buf.x_hat, buf.sinr, buf.llr, buf.flags)]
    for a, b in zip(ref, again):
        assert np.array_equal(a, b)
    print("tuned cells per chunk:", chunk)
    phy.autotune_clear()
