"""Block-floating-point fronthaul input: CUDA decompression and fused LS estimation vs the oracle.

Decompression is integer bit unpacking followed by one FP32 rounding of m 2^e scale (m 2^e is
exact), the same rounding the oracle's exact FP64 product takes when cast to complex64: the bar
is bitwise equality. Everything downstream of the decoded grid runs the unchanged kernels, so the
stream-fed paths must equal the grid-fed ones bit for bit.
"""
import numpy as np
import pytest

from oracle import phy_oracle as O
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


def T(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def decompress_gpu(cfg, c, w, scale, shape, dev, data_only=False, fill=None):
    import torch
    from paper_2510_07843_gb300 import phy
    Y = torch.empty(shape, dtype=torch.complex64, device=dev)
    if fill is not None:
        Y.fill_(fill)
    phy.bfp_decompress(cfg, T(c, dev), w, scale, Y, data_only=data_only)
    torch.cuda.synchronize()
    return Y


CASES = [  # (spec, width, scale, seed); odd widths with odd block counts leave a ragged tail
    (S.SlotSpec(n_prb=5, n_rx=3, n_layers=2, qm=4, dmrs_sym=(2,)), 9, 2.0 ** -10, 1),
    (S.SlotSpec(n_prb=7, n_rx=5, n_layers=3, qm=6, dmrs_sym=(2, 11)), 8, 0.7e-3, 2),
    (S.SlotSpec(n_prb=3, n_rx=2, n_layers=1, qm=2, dmrs_sym=(3,)), 1, 2.0 ** -4, 3),
    (S.SlotSpec(n_prb=4, n_rx=4, n_layers=4, qm=4, dmrs_sym=(2, 11)), 16, 2.0 ** -14, 4),
    (S.SlotSpec(n_prb=6, n_rx=8, n_layers=8, qm=8, dmrs_sym=(2, 11)), 12, 1.3e-4, 5),
    (S.SlotSpec(n_prb=3, n_rx=1, n_layers=1, qm=2, dmrs_sym=(2,)), 4, 0.25, 6),
    (S.SlotSpec(n_prb=1, n_rx=1, n_layers=1, qm=2, dmrs_sym=(2,)), 7, 3.0e-3, 7),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_decompress_bitwise_vs_oracle(dev, case):
    from paper_2510_07843_gb300 import phy
    spec, w, scale, seed = CASES[case]
    sl = S.make_slot(spec, seed, keep_h=False)
    cfg = phy.SlotConfig.from_spec(spec)
    c = S.bfp_compress(sl.Y, w, scale)
    assert c.size == phy.bfp_bytes(cfg, w)
    s32 = float(np.float32(scale))
    want = O.bfp_decompress(c, sl.Y.shape, w, s32).astype(np.complex64)
    got = decompress_gpu(cfg, c, w, scale, sl.Y.shape, dev).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # any byte stream is a valid input: random bytes, junk in the parameter bytes' high nibble
    raw = np.random.default_rng(seed).integers(0, 256, size=c.size, dtype=np.uint8)
    want = O.bfp_decompress(raw, sl.Y.shape, w, s32).astype(np.complex64)
    got = decompress_gpu(cfg, raw, w, scale, sl.Y.shape, dev).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_decompress_data_only_leaves_dmrs_rows(dev):
    from paper_2510_07843_gb300 import phy
    spec, w, scale, seed = CASES[1]
    sl = S.make_slot(spec, seed, keep_h=False)
    cfg = phy.SlotConfig.from_spec(spec)
    c = S.bfp_compress(sl.Y, w, scale)
    full = decompress_gpu(cfg, c, w, scale, sl.Y.shape, dev).cpu().numpy()
    part = decompress_gpu(cfg, c, w, scale, sl.Y.shape, dev, data_only=True,
                          fill=complex(7.0, -7.0)).cpu().numpy()
    for t in range(spec.n_sym):
        if t in spec.dmrs_sym:
            assert np.all(part[:, t] == np.complex64(7.0 - 7.0j))
        else:
            assert np.array_equal(part[:, t], full[:, t])


STREAM_CASES = {
    "small_51prb_4x2_w9": (S.spec_small_51prb(), 9, 2.0 ** -12, 1001, "fp32"),
    "carrier_25prb_16x4_w14": (S.spec_carrier_273prb(n_prb=25), 14, 2.0 ** -13, 2000, "fp32"),
    "massive_6prb_64x16_w9_fp16": (S.spec_massive_mimo(n_cells=2, n_prb=6), 9, 2.0 ** -10,
                                   3000, "fp16"),
    "ragged_7prb_6x3_w5": (S.SlotSpec(n_prb=7, n_rx=6, n_layers=3, qm=6, dmrs_sym=(2, 11),
                                      snr_db=25.0), 5, 2.0 ** -6, 11, "fp32"),
}


@pytest.mark.parametrize("name", list(STREAM_CASES))
def test_stream_fed_paths_equal_grid_fed(dev, name):
    """phy_chest_bfp = phy_chest on the decoded grid, phy_slot_run_bfp = phy_slot_run on it,
    and phy_slot_run_bfp leaves the decoded grid in its buffer."""
    import torch
    from paper_2510_07843_gb300 import phy
    spec, w, scale, seed, prec = STREAM_CASES[name]
    sl = S.make_slot(spec, seed, keep_h=False)
    cfg = phy.SlotConfig.from_spec(spec, precision=prec)
    c = T(S.bfp_compress(sl.Y, w, scale), dev)
    P, s2 = T(sl.pilots, dev), T(sl.sigma2, dev)
    Yd = torch.empty(sl.Y.shape, dtype=torch.complex64, device=dev)
    phy.bfp_decompress(cfg, c, w, scale, Yd)
    G = phy.n_groups(cfg)
    ashape = (spec.n_cells, len(spec.dmrs_sym), G, spec.n_layers, spec.n_rx)
    a0 = torch.empty(ashape, dtype=torch.complex64, device=dev)
    a1 = torch.empty(ashape, dtype=torch.complex64, device=dev)
    phy.chest(cfg, Yd, P, a0)
    phy.chest_bfp(cfg, c, w, scale, P, a1)
    ref = phy.SlotBuffers(cfg, with_inputs=False)
    got = phy.SlotBuffers(cfg, with_inputs=False)
    phy.slot_run(cfg, Yd, P, s2, ref.x_hat, ref.sinr, ref.llr, ref.flags, ref.workspace)
    Ys = torch.zeros_like(Yd)
    phy.slot_run_bfp(cfg, c, w, scale, Ys, P, s2, got.x_hat, got.sinr, got.llr, got.flags,
                     got.workspace)
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(a0), torch.view_as_real(a1))
    for key in ("x_hat", "sinr", "llr", "flags"):
        assert torch.equal(getattr(ref, key), getattr(got, key)), key
    assert torch.equal(torch.view_as_real(Ys), torch.view_as_real(Yd))


def test_full_size_massive_stream(dev):
    """8 cells x 273 PRB x 14 symbols x 64 Rx at 9-bit mantissas (54.8 MB of stream): sampled
    blocks bitwise against the oracle, and the stream-fed receiver equal to the grid-fed one."""
    import torch
    from paper_2510_07843_gb300 import phy
    spec = S.spec_massive_mimo()
    sl = S.make_slot(spec, 3000, keep_h=False)
    w, scale = 9, 2.0 ** -10
    cfg = phy.SlotConfig.from_spec(spec, precision="fp16")
    c_np = S.bfp_compress(sl.Y, w, scale)
    c = T(c_np, dev)
    Yd = torch.empty(sl.Y.shape, dtype=torch.complex64, device=dev)
    phy.bfp_decompress(cfg, c, w, scale, Yd)
    torch.cuda.synchronize()
    nb = O.bfp_block_bytes(w)
    n_blocks = c_np.size // nb
    pick = np.random.default_rng(9).choice(n_blocks, size=1500, replace=False)
    pick = np.concatenate([pick, [0, n_blocks - 1]])
    sample = c_np.reshape(n_blocks, nb)[pick].reshape(-1)
    want = O.bfp_decompress(sample, (1, 1, 1, 12 * pick.size), w, scale).astype(np.complex64)
    flat = Yd.reshape(-1, 12).cpu().numpy()[pick].reshape(-1)
    assert np.array_equal(flat.view(np.uint32), want[0, 0, 0].view(np.uint32))
    P, s2 = T(sl.pilots, dev), T(sl.sigma2, dev)
    ref = phy.SlotBuffers(cfg, with_inputs=False)
    got = phy.SlotBuffers(cfg, with_inputs=False)
    phy.slot_run(cfg, Yd, P, s2, ref.x_hat, ref.sinr, ref.llr, ref.flags, ref.workspace)
    Ys = torch.zeros_like(Yd)
    phy.slot_run_bfp(cfg, c, w, scale, Ys, P, s2, got.x_hat, got.sinr, got.llr, got.flags,
                     got.workspace)
    torch.cuda.synchronize()
    for key in ("x_hat", "sinr", "llr", "flags"):
        assert torch.equal(getattr(ref, key), getattr(got, key)), key


def test_host_buffer_stream_path(dev):
    """phy_slot_run_bfp_host: pinned host stream in, host LLRs and flags out, equal to the device
    path's outputs."""
    import torch
    from paper_2510_07843_gb300 import phy
    spec, w, scale, seed, prec = STREAM_CASES["massive_6prb_64x16_w9_fp16"]
    sl = S.make_slot(spec, seed, keep_h=False)
    cfg = phy.SlotConfig.from_spec(spec, precision=prec)
    c_np = S.bfp_compress(sl.Y, w, scale)
    ref = phy.SlotBuffers(cfg, with_inputs=False)
    P, s2 = T(sl.pilots, dev), T(sl.sigma2, dev)
    c = T(c_np, dev)
    Yd = torch.empty(sl.Y.shape, dtype=torch.complex64, device=dev)
    phy.slot_run_bfp(cfg, c, w, scale, Yd, P, s2, ref.x_hat, ref.sinr, ref.llr, ref.flags,
                     ref.workspace)
    b = phy.SlotBuffers(cfg, device=dev)
    ch = torch.from_numpy(c_np).pin_memory()
    Ph = torch.from_numpy(sl.pilots).pin_memory()
    sh = torch.from_numpy(sl.sigma2).pin_memory()
    lh = torch.empty(b.llr.shape, dtype=b.llr.dtype).pin_memory()
    fh = torch.empty(b.flags.shape, dtype=torch.uint8).pin_memory()
    cd = torch.empty_like(c)
    Y2 = torch.empty_like(Yd)
    phy.slot_run_bfp_host(cfg, ch, w, scale, Ph, sh, lh, fh, cd, Y2, b.pilots, b.sigma2,
                          b.x_hat, b.sinr, b.llr, b.flags, b.workspace)
    torch.cuda.synchronize()
    assert torch.equal(lh, ref.llr.cpu()) and torch.equal(fh, ref.flags.cpu())
