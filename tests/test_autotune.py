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


def test_tile_pins_are_validated_and_read_back():
    """phy_autotune_set_tiles / phy_autotune_tiles on the host (no GPU work)."""
    from paper_2510_07843_gb300 import build, phy
    build.build()
    phy.load()
    cfg = phy.SlotConfig(n_cells=4, n_prb=12, n_rx=64, n_layers=16, qm=8, dmrs_sym=(2, 11))
    phy.autotune_clear()
    assert phy.autotune_tiles(cfg) == {"chunk": 0, "solve_width": 0, "ring": 0}
    phy.autotune_set_tiles(cfg, 2, 64, 12)
    # the deeper ring reads back only where it applies: tensor-core products whose
    # shared-memory map still fits it (8 layers yes; FP32 products or 16 layers no)
    assert phy.autotune_tiles(cfg) == {"chunk": 2, "solve_width": 64, "ring": 0}
    tc8 = phy.SlotConfig(n_cells=2, n_prb=12, n_rx=64, n_layers=8, qm=8, dmrs_sym=(2, 11),
                         precision="fp16")
    tc16 = phy.SlotConfig(n_cells=2, n_prb=12, n_rx=64, n_layers=16, qm=8, dmrs_sym=(2, 11),
                          precision="fp16")
    for c, ring in ((tc8, 12), (tc16, 0)):
        phy.autotune_set_tiles(c, 1, 128, 12)
        assert phy.autotune_tiles(c) == {"chunk": 1, "solve_width": 128, "ring": ring}
    for bad in ((5, 0, 0), (-1, 0, 0), (0, 96, 0), (0, 0, 10)):
        with pytest.raises(phy.PhyError):
            phy.autotune_set_tiles(cfg, *bad)
    phy.autotune_clear()
    assert phy.autotune_tiles(cfg)["chunk"] == 0


TILE_CASES = {  # (spec, precision): the massive shape with FP16 products, the carrier with FP32
    "massive_2x12prb_fp16": (S.spec_massive_mimo(n_cells=2, n_prb=12), "fp16"),
    "carrier_2x30prb_fp16": (S.spec_carrier_273prb(n_cells=2, n_prb=30), "fp16"),
    "carrier_2x30prb_fp32": (S.spec_carrier_273prb(n_cells=2, n_prb=30), "fp32"),
}


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(TILE_CASES))
def test_every_tile_shape_gives_the_same_bits(dev, name):
    """Each candidate tile (solve CTA width 128 / 64, tensor-core ring default / 12 stages,
    chunk 1 / whole batch) gives bitwise the outputs of the default tiles; then the autotuner
    picks one and the results still match."""
    import torch
    from paper_2510_07843_gb300 import phy
    spec, prec = TILE_CASES[name]
    sl = S.make_slot(spec, 3200, keep_h=False)
    cfg = phy.SlotConfig.from_spec(spec, precision=prec)
    buf = phy.SlotBuffers(cfg, device=dev)
    buf.Y.copy_(torch.from_numpy(sl.Y))
    buf.pilots.copy_(torch.from_numpy(sl.pilots))
    buf.sigma2.copy_(torch.from_numpy(sl.sigma2))
    args = (buf.Y, buf.pilots, buf.sigma2, buf.x_hat, buf.sinr, buf.llr, buf.flags, buf.workspace)
    outs = lambda: [t.clone() for t in (buf.x_hat, buf.sinr, buf.llr, buf.flags)]
    phy.autotune_clear()
    phy.slot_run(cfg, *args)
    ref = outs()
    for chunk in (1, spec.n_cells):
        for w in (128, 64):
            for ring in (0, 12):
                phy.autotune_set_tiles(cfg, chunk, w, ring)
                for t in (buf.x_hat, buf.sinr, buf.llr):
                    t.zero_()
                phy.slot_run(cfg, *args)
                for a, b in zip(ref, outs()):
                    assert torch.equal(a, b), (chunk, w, ring)
    phy.autotune_clear()
    phy.autotune(cfg, *args)
    tiles = phy.autotune_tiles(cfg)
    print(name, "tuned tiles:", tiles)
    for a, b in zip(ref, outs()):
        assert torch.equal(a, b)
    phy.autotune_clear()
