"""CUDA path vs the FP64 oracle, element by element on identical seeded inputs.

Small cases run the oracle on every RE (several segments, ragged PRB counts, every layer class
and modulation); the full-size 8-cell 273-PRB 64x16 workload (the benchmark's launch) is checked
on sampled REs that include the first and last frequency segments.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import phy_oracle as O
from paper_2510_07843_gb300 import synth as S
from parity import assert_parity, check_flags, compare_res, rel_fro

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


def gpu_slot(spec, sl, dev, **kw):
    import torch
    from paper_2510_07843_gb300 import phy
    cfg = phy.SlotConfig.from_spec(spec, **kw)
    buf = phy.SlotBuffers(cfg, with_inputs=False)
    Y, P, s2 = T(sl.Y, dev), T(sl.pilots, dev), T(sl.sigma2, dev)
    phy.slot_run(cfg, Y, P, s2, buf.x_hat, buf.sinr, buf.llr, buf.flags, buf.workspace)
    G = phy.n_groups(cfg)
    anchors = torch.empty((spec.n_cells, len(spec.dmrs_sym), G, spec.n_layers, spec.n_rx),
                          dtype=torch.complex64, device=dev)
    phy.chest(cfg, Y, P, anchors)
    torch.cuda.synchronize()
    return dict(x_hat=buf.x_hat.cpu().numpy(), sinr=buf.sinr.cpu().numpy(),
                llr=buf.llr.cpu().numpy(), flags=buf.flags.cpu().numpy(),
                anchors=anchors.cpu().numpy(), cfg=cfg, buf=buf, Y=Y, P=P, s2=s2)


def oracle_dense(spec, sl):
    ref = O.run_slot(sl.Y, sl.pilots, sl.sigma2, spec.dmrs_sym, spec.n_layers, spec.qm,
                     spec.occ_len)
    sinr = ref["sinr"]
    ref["s2eff"] = 1.0 / sinr
    mu = sinr / (1.0 + sinr)
    ref["x_t"] = ref["x_hat"] / mu
    return ref


def gather_sampled(got, ref, res):
    """GPU outputs at the sampled REs res = {cell: (j, k)} next to the oracle's, flat."""
    keys = ("x_hat", "sinr", "llr", "flags")
    g = {k: np.concatenate([got[k][c, jj, kk] for c, (jj, kk) in res.items()]) for k in keys}
    r = {k: np.concatenate([ref[f"{k}_{c}"] for c in res]) for k in keys + ("pivot_ratio",)}
    return g, r


def compare_sampled(tag, qm, got, ref, res):
    """Flags RE by RE, then the outputs over every sampled RE (none may drop out: the oracle
    flags none of them in these well-conditioned batches)."""
    g, r = gather_sampled(got, ref, res)
    mask = check_flags(tag, g["flags"], r["flags"], r["pivot_ratio"])
    assert mask.all(), (tag, int(mask.sum()), mask.size)
    rs = r["sinr"]
    m = compare_res(tag, dict(x_hat=g["x_hat"], sinr=g["sinr"], llr=g["llr"]),
                    dict(x_hat=r["x_hat"], sinr=rs, llr=r["llr"]), qm, 1.0 / rs,
                    r["x_hat"] / (rs / (1 + rs)), mask)
    return m, g, r


def sample_res(spec, seed, edge=30, n_rand=60):
    """Per cell: the first and last `edge` subcarriers and n_rand random ones, each at a random
    data symbol."""
    rng = np.random.default_rng(seed)
    K, J = spec.n_sc, len(spec.data_sym)
    res = {}
    for c in range(spec.n_cells):
        kk = np.concatenate([np.arange(0, edge), np.arange(K - edge, K),
                             rng.integers(0, K, n_rand)])
        res[c] = (rng.integers(0, J, kk.size), kk)
    return res


CASES = {
    "small_51prb_4x2_16qam": (S.spec_small_51prb(), 1001),
    "carrier_25prb_16x4_64qam_jakes": (S.spec_carrier_273prb(n_prb=25), 2000),
    "ragged_7prb_6x3_64qam": (S.SlotSpec(n_prb=7, n_rx=6, n_layers=3, qm=6, dmrs_sym=(2, 11),
                                         snr_db=25.0, n_taps=6, doppler_hz=300.0), 11),
    "one_layer_3prb_qpsk": (S.SlotSpec(n_prb=3, n_rx=2, n_layers=1, qm=2, dmrs_sym=(3,),
                                       snr_db=10.0), 12),
    "five_layers_5prb_8rx_256qam": (S.SlotSpec(n_prb=5, n_rx=8, n_layers=5, qm=8,
                                               dmrs_sym=(2, 11), snr_db=35.0), 13),
    "nine_layers_4prb_12rx": (S.SlotSpec(n_prb=4, n_rx=12, n_layers=9, qm=4, dmrs_sym=(2, 11),
                                         snr_db=25.0, n_taps=4), 14),
    "massive_6prb_64x16_256qam_2cells": (S.spec_massive_mimo(n_cells=2, n_prb=6), 3000),
    "massive_one_dmrs_5prb_32x16": (S.spec_massive_mimo(n_cells=1, n_prb=5, n_rx=32,
                                                        dmrs_sym=(2,)), 15),
    "one_prb_4x2": (S.SlotSpec(n_prb=1, n_rx=4, n_layers=2, qm=4, dmrs_sym=(2,)), 16),
    "forced_cover_4_single_layer": (S.SlotSpec(n_prb=4, n_rx=4, n_layers=1, qm=4,
                                               dmrs_sym=(2, 11), occ_len=4), 17),
    "minimal_slot_1prb_1x1_two_symbols": (S.SlotSpec(n_prb=1, n_rx=1, n_layers=1, qm=2,
                                                     dmrs_sym=(0,), n_sym=2, snr_db=15.0), 21),
}


@pytest.mark.parametrize("name", list(CASES))
def test_slot_parity_dense(dev, name):
    spec, seed = CASES[name]
    sl = S.make_slot(spec, seed, keep_h=False)
    got = gpu_slot(spec, sl, dev)
    ref = oracle_dense(spec, sl)
    # LS anchors
    a_rel = rel_fro(got["anchors"], ref["anchors"])
    print(name, "anchors rel", a_rel)
    assert a_rel < 2e-7
    # detection outputs over every data RE, flattened to [re][layer]
    nl, qm = spec.n_layers, spec.qm
    flat = lambda a, tail: a.reshape((-1,) + tail)
    fl_got = got["flags"].reshape(-1)
    # flags RE by RE; the oracle flags no RE of these cases, so every RE is compared
    mask = check_flags(name, fl_got, ref["flags"], ref["pivot_ratio"])
    m = compare_res(name,
                    dict(x_hat=flat(got["x_hat"], (nl,)), sinr=flat(got["sinr"], (nl,)),
                         llr=flat(got["llr"], (nl, qm))),
                    dict(x_hat=flat(ref["x_hat"], (nl,)), sinr=flat(ref["sinr"], (nl,)),
                         llr=flat(ref["llr"], (nl, qm))),
                    qm, flat(ref["s2eff"], (nl,)), flat(ref["x_t"], (nl,)), mask)
    assert_parity(m)
    assert not ref["flags"].any() and not fl_got.any()


def test_slot_parity_full_size_sampled(dev):
    """The benchmark's launch: 8 cells x 273 PRB x 64 Rx x 16 layers, 256-QAM; sampled REs
    including both band edges of every cell, every one of them compared."""
    spec = S.spec_massive_mimo()
    sl = S.make_slot(spec, 3000, keep_h=False)
    got = gpu_slot(spec, sl, dev)
    res = sample_res(spec, 0)
    ref = O.run_slot(sl.Y, sl.pilots, sl.sigma2, spec.dmrs_sym, spec.n_layers, spec.qm, res=res)
    assert rel_fro(got["anchors"], ref["anchors"]) < 2e-7
    m, _, _ = compare_sampled("full_size_sampled", spec.qm, got, ref, res)
    assert_parity(m)
    assert m["n"] == 8 * 120


@pytest.mark.parametrize("n_sym,dmrs", [(14, (2, 11)), (12, (1, 9))])
def test_slot_parity_maximum_carrier_sampled(dev, n_sym, dmrs):
    """The largest grid the ABI takes: 275 PRB (3300 subcarriers, the last LS group overlapping),
    64 Rx x 16 layers, 256-QAM, one cell; also with a 12-symbol slot. Sampled REs including both
    band edges against the oracle."""
    spec = S.spec_massive_mimo(n_cells=1, n_prb=275, n_sym=n_sym, dmrs_sym=dmrs)
    sl = S.make_slot(spec, 3300 + n_sym, keep_h=False)
    got = gpu_slot(spec, sl, dev)
    res = sample_res(spec, 1, edge=40)
    ref = O.run_slot(sl.Y, sl.pilots, sl.sigma2, spec.dmrs_sym, spec.n_layers, spec.qm, res=res)
    assert rel_fro(got["anchors"], ref["anchors"]) < 2e-7
    m, _, _ = compare_sampled("max_carrier", spec.qm, got, ref, res)
    assert_parity(m)
    assert m["n"] == 140


def test_mmse_detect_genie_and_zero_forcing(dev):
    import torch
    from paper_2510_07843_gb300 import phy
    spec = S.SlotSpec(n_prb=4, n_rx=8, n_layers=4, qm=4, dmrs_sym=(2, 11), snr_db=20.0)
    for noise, s2 in ((True, spec.sigma2), (False, 0.0)):
        sl = S.make_slot(spec, 21, keep_h=True, noise=noise)
        dsym = list(spec.data_sym)
        H = np.stack([sl.H[0][dsym]])  # [cell][dsym][sc][rx][layer]
        cfg = phy.SlotConfig.from_spec(spec)
        C, J, K, nl = 1, len(dsym), spec.n_sc, spec.n_layers
        x = torch.empty((C, J, K, nl), dtype=torch.complex64, device=dev)
        sn = torch.empty((C, J, K, nl), dtype=torch.float32, device=dev)
        fl = torch.empty((C, J, K), dtype=torch.uint8, device=dev)
        s2t = T(np.array([s2], dtype=np.float32), dev)
        phy.mmse_detect(cfg, T(H.astype(np.complex64), dev), T(sl.Y, dev), s2t, x, sn, fl)
        torch.cuda.synchronize()
        Hc = H.astype(np.complex64).astype(np.complex128)
        y = np.stack([sl.Y[0, t].T for t in dsym])[None].astype(np.complex128)  # [1][J][K][rx]
        xr, d = O.lmmse_gram(Hc, y, s2)
        got = x.cpu().numpy()
        err = rel_fro(got, xr)
        print("mmse_detect noise" if noise else "zero forcing", err)
        assert err < 1e-5
        if not noise:
            assert rel_fro(got, sl.x) < 1e-5  # ZF recovers the transmitted symbols
        else:
            sr, _, _ = O.sinr_unbias(xr, d, s2)
            assert np.max(np.abs(sn.cpu().numpy() - sr) / sr) < 1e-4
        assert not fl.cpu().numpy().any()


def test_llr_demap_standalone_matches_fused_and_oracle(dev):
    import torch
    from paper_2510_07843_gb300 import phy
    spec = S.spec_carrier_273prb(n_prb=10)
    sl = S.make_slot(spec, 31, keep_h=False)
    got = gpu_slot(spec, sl, dev)
    buf = got["buf"]
    llr2 = torch.empty_like(buf.llr)
    phy.llr_demap(got["cfg"], buf.x_hat, buf.sinr, llr2)
    torch.cuda.synchronize()
    l2 = llr2.cpu().numpy()
    sinr = got["sinr"].astype(np.float64)
    s2eff = 1.0 / sinr
    x_t = got["x_hat"].astype(np.complex128) / (sinr / (1 + sinr))
    ref = O.llr_maxlog(x_t, s2eff, spec.qm)
    assert np.max(np.abs(l2 - ref) * s2eff[..., None]) < 1e-4
    assert np.max(np.abs(l2 - got["llr"]) * s2eff[..., None]) < 1e-4


def test_non_finite_input_is_flagged(dev):
    spec = S.SlotSpec(n_prb=3, n_rx=4, n_layers=2, qm=4, dmrs_sym=(2,))
    sl = S.make_slot(spec, 41, keep_h=False)
    clean = gpu_slot(spec, sl, dev)
    Y = sl.Y.copy()
    Y[0, 5, 1, 17] = np.nan  # data symbol 5 (data index 4), subcarrier 17
    sl.Y = Y
    got = gpu_slot(spec, sl, dev)
    j = spec.data_sym.index(5)
    assert got["flags"][0, j, 17] & 4
    assert np.all(np.isfinite(got["llr"])) and np.all(np.isfinite(got["x_hat"]))
    assert np.all(got["llr"][0, j, 17] == 0)
    other = np.ones(got["flags"].shape, dtype=bool)
    other[0, j, 17] = False
    assert np.array_equal(got["llr"][other], clean["llr"][other])


def test_repeatable_bitwise(dev):
    spec = S.spec_massive_mimo(n_cells=1, n_prb=4)
    sl = S.make_slot(spec, 51, keep_h=False)
    a = gpu_slot(spec, sl, dev)
    b = gpu_slot(spec, sl, dev)
    assert np.array_equal(a["llr"], b["llr"]) and np.array_equal(a["x_hat"], b["x_hat"])


def test_errors_enqueue_nothing(dev):
    import torch
    from paper_2510_07843_gb300 import phy
    spec = S.spec_small_51prb(n_prb=4)
    cfg = phy.SlotConfig.from_spec(spec)
    buf = phy.SlotBuffers(cfg)
    small = torch.empty((16,), dtype=torch.uint8, device=dev)
    with pytest.raises(phy.PhyError) as e:
        phy.slot_run(cfg, buf.Y, buf.pilots, buf.sigma2, buf.x_hat, buf.sinr, buf.llr, buf.flags,
                     small)
    assert e.value.code == 3
    bad = dataclasses.replace(cfg, occ_len=3)
    with pytest.raises(phy.PhyError) as e:
        phy.slot_run(bad, buf.Y, buf.pilots, buf.sigma2, buf.x_hat, buf.sinr, buf.llr, buf.flags,
                     buf.workspace)
    assert e.value.code == 1


TC_CASES = {
    "massive_6prb_64x16_256qam_2cells": (S.spec_massive_mimo(n_cells=2, n_prb=6), 3000),
    "carrier_25prb_16x4_64qam_jakes": (S.spec_carrier_273prb(n_prb=25), 2000),
    "massive_one_dmrs_5prb_32x16": (S.spec_massive_mimo(n_cells=1, n_prb=5, n_rx=32,
                                                        dmrs_sym=(2,)), 15),
    "small_51prb_4x2_16qam": (S.spec_small_51prb(), 1001),
}


@pytest.mark.parametrize("prec", ["tf32", "fp16", "bf16"])
@pytest.mark.parametrize("name", list(TC_CASES))
def test_tensor_core_variants_vs_oracle(dev, name, prec):
    """Gram and matched-filter products on tcgen05 with operands rounded to TF32/FP16/BF16."""
    spec, seed = TC_CASES[name]
    sl = S.make_slot(spec, seed, keep_h=False)
    got = gpu_slot(spec, sl, dev, precision=prec)
    ref = oracle_dense(spec, sl)
    nl, qm = spec.n_layers, spec.qm
    flat = lambda a, tail: a.reshape((-1,) + tail)
    mask = check_flags(f"{name}[{prec}]", got["flags"], ref["flags"], ref["pivot_ratio"])
    assert mask.all()
    m = compare_res(f"{name}[{prec}]",
                    dict(x_hat=flat(got["x_hat"], (nl,)), sinr=flat(got["sinr"], (nl,)),
                         llr=flat(got["llr"], (nl, qm))),
                    dict(x_hat=flat(ref["x_hat"], (nl,)), sinr=flat(ref["sinr"], (nl,)),
                         llr=flat(ref["llr"], (nl, qm))),
                    qm, flat(ref["s2eff"], (nl,)), flat(ref["x_t"], (nl,)), mask)
    hard = (got["llr"] < 0).astype(np.uint8)
    hard_ref = (ref["llr"] < 0).astype(np.uint8)
    m["bit_disagree"] = float(np.mean(hard != hard_ref))
    m["ber"] = float(np.mean(hard != sl.bits))
    m["ber_ref"] = float(np.mean(hard_ref != sl.bits))
    print(f"{name}[{prec}] bits:", m["bit_disagree"], m["ber"], m["ber_ref"])
    # Operand rounding u = 2^-11 (TF32, FP16) or 2^-8 (BF16) per product; the Gram and matched
    # filter carry a few u of relative error and the solve multiplies it by the conditioning.
    # Bounds: x_hat 2u / 2.5u aggregate, SINR 6u / 5u, normalised LLR 40u / 25u, hard-bit
    # disagreement with the oracle 1e-3 / 5e-3, uncoded BER within 2% of the oracle's.
    lim = TC_LIMITS[prec]
    assert m["x_rel"] <= lim[0], m
    assert m["sinr_rel_max"] <= lim[1], m
    assert m["llr_norm_max"] <= lim[2], m
    assert m["bit_disagree"] <= lim[3], m
    assert abs(m["ber"] - m["ber_ref"]) <= 0.02 * m["ber_ref"] + 2e-4, m


def test_fp64_refactor_of_ill_conditioned_res(dev):
    """Nearly collinear layers: kappa(H) ~ 3e3, so kappa(A) ~ 1e7 trips the 1e-6 pivot-ratio flag.
    FP32 loses ~kappa(A) u of accuracy; the FP64 recomputation from the (FP32) LS anchors keeps
    ~kappa(H) u. Flag bit 0 marks the REs on both sides; bit 1 marks the FP64 recomputation."""
    rng = np.random.default_rng(71)
    nr, nl = 4, 4
    h = (rng.standard_normal((nr, nl)) + 1j * rng.standard_normal((nr, nl))) / math.sqrt(2)
    h[:, 1] = h[:, 0] + 3e-4 * (rng.standard_normal(nr) + 1j * rng.standard_normal(nr))
    spec = S.SlotSpec(n_prb=4, n_rx=nr, n_layers=nl, qm=4, dmrs_sym=(2, 11), snr_db=120.0)
    ch = np.broadcast_to(h, (1, 14, spec.n_sc, nr, nl))
    sl = S.make_slot(spec, 72, noise=False, channel=ch)
    ref = oracle_dense(spec, sl)
    assert np.all(ref["flags"] & 1)
    plain = gpu_slot(spec, sl, dev)
    fixed = gpu_slot(spec, sl, dev, fp64_refactor=True)
    assert np.all(plain["flags"] & 1) and not np.any(plain["flags"] & 2)
    assert np.all((fixed["flags"] & 3) == 3)
    e32 = rel_fro(plain["x_hat"], ref["x_hat"])
    e64 = rel_fro(fixed["x_hat"], ref["x_hat"])
    # The FP64 recomputation starts from the FP32 LS anchors, whose rounding (a few u32 relative)
    # the noise-free least-squares solution amplifies by kappa(H); the bar is 8 kappa(H) u32.
    kappa = float(np.linalg.cond(h))
    bound = 8.0 * kappa * 2.0 ** -24
    print("ill-conditioned x_hat rel err: fp32", e32, "fp64 refactor", e64, "kappa(H)", kappa,
          "bound", bound)
    assert e64 <= bound and e64 < e32 / 10


def test_host_buffer_entry_point_on_concurrent_streams(dev):
    """phy_slot_run_host (pinned host inputs in, host LLRs and flags out) equals phy_slot_run on
    device buffers, bit for bit, also when three calls on three streams with their own device
    buffers overlap, as the benchmark's end-to-end steps do."""
    import torch
    from paper_2510_07843_gb300 import phy
    spec = S.spec_massive_mimo(n_cells=2, n_prb=8)
    sl = S.make_slot(spec, 3300, keep_h=False)
    cfg = phy.SlotConfig.from_spec(spec, precision="fp16")
    ref = phy.SlotBuffers(cfg, device=dev)
    ref.Y.copy_(torch.from_numpy(sl.Y))
    ref.pilots.copy_(torch.from_numpy(sl.pilots))
    ref.sigma2.copy_(torch.from_numpy(sl.sigma2))
    phy.slot_run(cfg, ref.Y, ref.pilots, ref.sigma2, ref.x_hat, ref.sinr, ref.llr, ref.flags,
                 ref.workspace)
    torch.cuda.synchronize()
    Yh = torch.from_numpy(sl.Y).pin_memory()
    Ph = torch.from_numpy(sl.pilots).pin_memory()
    sh = torch.from_numpy(sl.sigma2).pin_memory()
    sets = []
    for i in range(3):
        b = phy.SlotBuffers(cfg, device=dev)
        lh = torch.full(ref.llr.shape, float("nan"), dtype=ref.llr.dtype).pin_memory()
        fh = torch.full(ref.flags.shape, 255, dtype=torch.uint8).pin_memory()
        sets.append((b, torch.cuda.Stream(device=dev), lh, fh))
    for rep in range(2):
        for b, st, lh, fh in sets:
            phy.slot_run_host(cfg, Yh, Ph, sh, lh, fh, b.Y, b.pilots, b.sigma2, b.x_hat, b.sinr,
                              b.llr, b.flags, b.workspace, stream=st)
    torch.cuda.synchronize()
    for b, st, lh, fh in sets:
        assert torch.equal(lh, ref.llr.cpu()) and torch.equal(fh, ref.flags.cpu())


def test_llr_binary16_output_is_the_rounded_fp32_output(dev):
    """cfg.llr_format = f16: every LLR is the FP32 value rounded to nearest binary16, saturating
    at +-65504; through the full receiver and through the stand-alone demapper."""
    import torch
    from paper_2510_07843_gb300 import phy
    for spec, seed in ((S.spec_massive_mimo(n_cells=2, n_prb=6), 3200),
                       (S.spec_small_51prb(), 1002)):
        sl = S.make_slot(spec, seed, keep_h=False)
        out = {}
        for fmt in ("f32", "f16"):
            cfg = phy.SlotConfig.from_spec(spec, llr_format=fmt)
            b = phy.SlotBuffers(cfg, device=dev)
            b.Y.copy_(torch.from_numpy(sl.Y))
            b.pilots.copy_(torch.from_numpy(sl.pilots))
            b.sigma2.copy_(torch.from_numpy(sl.sigma2))
            phy.slot_run(cfg, b.Y, b.pilots, b.sigma2, b.x_hat, b.sinr, b.llr, b.flags,
                         b.workspace)
            demap = torch.empty_like(b.llr)
            phy.llr_demap(cfg, b.x_hat, b.sinr, demap)
            torch.cuda.synchronize()
            out[fmt] = (b.llr, demap)
        assert out["f16"][0].dtype == torch.float16
        for k in range(2):
            ref = out["f32"][k].clamp(-65504.0, 65504.0).half()
            assert torch.equal(ref, out["f16"][k])


def test_slot_parity_full_size_sampled_tensor_core_fp16(dev):
    """The FP16 tensor-core launch on the benchmark's full batch (8 cells x 273 PRB x 64 Rx x 16
    layers), sampled REs against the oracle with the reduced-precision bounds of the small
    tensor-core cases, and hard decisions nearly all equal to the oracle's."""
    spec = S.spec_massive_mimo()
    sl = S.make_slot(spec, 3001, keep_h=False)
    got = gpu_slot(spec, sl, dev, precision="fp16")
    res = sample_res(spec, 1, edge=24, n_rand=48)
    ref = O.run_slot(sl.Y, sl.pilots, sl.sigma2, spec.dmrs_sym, spec.n_layers, spec.qm, res=res)
    m, g, r = compare_sampled("full_size_sampled[fp16]", spec.qm, got, ref, res)
    assert m["n"] == 8 * 96
    assert m["x_rel"] <= 1e-3, m
    assert m["sinr_rel_max"] <= 3e-3, m
    assert m["llr_norm_max"] <= 2e-2, m
    assert np.mean((g["llr"] < 0) != (r["llr"] < 0)) <= 1e-3


def test_device_wait_timeouts_void_the_solve(dev):
    """Failure detection without a fault. (1) The error word set by hand between the two stages
    makes every RE report flag bit 3 alone. (2) The tensor-core segment kernel's first-level
    waits given no polls (phy_debug_set_wait_polls) run out: its groups agree, leave, drain the
    copies in flight and free tensor memory; the kernel returns, the error word is nonzero and the
    solve voids every RE. (3) The solve kernel's own copy wait given no polls does the same.
    (4) With the default limits restored, the same calls give the clean result bit for bit."""
    import torch
    from paper_2510_07843_gb300 import phy
    spec = S.spec_massive_mimo(n_cells=1, n_prb=6)
    sl = S.make_slot(spec, 3300, keep_h=False)
    cfg = phy.SlotConfig.from_spec(spec, precision="fp16")
    if not phy.stage_supported(cfg):
        pytest.skip("single-chunk stages not supported for this shape")
    b = phy.SlotBuffers(cfg, device=dev)
    b.Y.copy_(torch.from_numpy(sl.Y))
    b.pilots.copy_(torch.from_numpy(sl.pilots))
    b.sigma2.copy_(torch.from_numpy(sl.sigma2))
    args = (b.anchors, b.Y, b.sigma2, b.x_hat, b.sinr, b.llr, b.flags, b.workspace)
    # workspace: anchors | noise-estimate partial sums (one 16-byte float4 per 1024 anchor
    # entries of each cell) | detection scratch, each region 256-byte aligned; the error word
    # is the first word of the detection scratch
    up = lambda v: (v + 255) // 256 * 256
    per_d = phy.n_groups(cfg) * spec.n_layers * spec.n_rx
    a = up(b.anchors.numel() * 8) + up(spec.n_cells * -(-per_d // 1024) * 16)
    word = b.workspace[a:a + 4].view(torch.int32)

    def run(stage=None):
        b.flags.fill_(0)
        phy.chest(cfg, b.Y, b.pilots, b.anchors)
        if stage in (None, phy.STAGE_GRAM_MF):
            phy.detect_stage(cfg, phy.STAGE_GRAM_MF, *args)
        if stage in (None, phy.STAGE_SOLVE):
            phy.detect_stage(cfg, phy.STAGE_SOLVE, *args)
        torch.cuda.synchronize()

    run()
    clean = {k: getattr(b, k).clone() for k in ("x_hat", "sinr", "llr", "flags")}
    assert not torch.any(clean["flags"] & 8) and int(word.item()) == 0
    # (1) by hand
    word.fill_(1)
    run(phy.STAGE_SOLVE)
    assert torch.all(b.flags == 8)
    try:
        # (2) the segment kernel's waits run out
        phy.debug_set_wait_polls("segment", 0)
        run(phy.STAGE_GRAM_MF)
        assert int(word.item()) > 0
        phy.debug_set_wait_polls("segment", -1)
        run(phy.STAGE_SOLVE)
        assert torch.all(b.flags == 8)
        # (3) the solve kernel's wait runs out (the segment kernel is clean)
        phy.debug_set_wait_polls("solve", 0)
        run()
        assert int(word.item()) == 0
        assert torch.all(b.flags == 8)
    finally:
        phy.debug_set_wait_polls("segment", -1)
        phy.debug_set_wait_polls("solve", -1)
    # (4) defaults again: the clean result
    run()
    for k, v in clean.items():
        assert torch.equal(getattr(b, k), v), k


def _ber(dev, spec, seed, precision):
    import torch
    from paper_2510_07843_gb300 import phy
    sl = S.make_slot(spec, seed, keep_h=False)
    cfg = phy.SlotConfig.from_spec(spec, precision=precision)
    b = phy.SlotBuffers(cfg, with_inputs=False)
    phy.slot_run(cfg, T(sl.Y, dev), T(sl.pilots, dev), T(sl.sigma2, dev), b.x_hat, b.sinr,
                 b.llr, b.flags, b.workspace)
    torch.cuda.synchronize()
    hard = (b.llr.cpu().numpy() < 0).astype(np.uint8)
    return float(np.mean(hard != sl.bits.reshape(hard.shape)))


BER_CASES = {  # one 273-PRB 64 x 16 256-QAM cell; noise-limited enough for 0.1 dB to show
    "flat_18dB": dict(n_taps=1, delay_spread_s=0.0, snr_db=18.0),
    "6tap_100ns_20dB": dict(n_taps=6, delay_spread_s=100e-9, snr_db=20.0),
}


@pytest.mark.parametrize("name", list(BER_CASES))
def test_reduced_precision_ber_within_a_tenth_of_a_db(dev, name):
    """Uncoded BER of the tensor-core variants against plain FP32 on the same slot: FP16 and BF16
    products may not need more than 0.1 dB extra SNR to match FP32, i.e. BER_x(s) <=
    BER_fp32(s - 0.1 dB). The slot redrawn at the lower SNR shares bits, channel
    and noise samples (the noise scales with the SNR), so the comparison is deterministic. (On the
    benchmark's 300 ns channel the BER sits on the LS estimation floor, about 24% at 22 dB, where
    a tenth of a dB does not show.)"""
    kw = BER_CASES[name]
    snr = kw["snr_db"]
    mk = lambda s: S.spec_massive_mimo(n_cells=1, **{**kw, "snr_db": s})
    b32, b16, bb = (_ber(dev, mk(snr), 3100, p) for p in ("fp32", "fp16", "bf16"))
    b32_01, b32_05 = (_ber(dev, mk(snr - d), 3100, "fp32") for d in (0.1, 0.5))
    print(name, {"fp32": b32, "fp16": b16, "bf16": bb, "fp32_-0.1dB": b32_01,
                 "fp32_-0.5dB": b32_05})
    assert b32 < b32_01 < b32_05  # the SNR shift is resolvable on this slot
    assert b16 <= b32_01
    assert bb <= b32_01


def test_pivot_flag_per_re_matches_oracle(dev):
    """Flag bit 0 RE by RE on a slot whose conditioning sweeps across the band: layer 1 is
    layer 0 plus eps(k) times an independent direction, eps log-spaced from 1e-5 to 1e-1 over the
    subcarriers, so the oracle's pivot ratios run from about 1e-10 to 1e-2 across the 1e-6
    threshold. Off the ambiguous band the GPU's flags equal the oracle's. Unflagged REs meet the
    per-RE bound 64 u32 kappa(A); with fp64_refactor the flagged ones carry bit 1 and are
    recomputed to within 8 kappa(H) u32 of the oracle."""
    rng = np.random.default_rng(81)
    nr, nl = 4, 4
    spec = S.SlotSpec(n_prb=16, n_rx=nr, n_layers=nl, qm=4, dmrs_sym=(2, 11), snr_db=80.0)
    K = spec.n_sc
    h0 = (rng.standard_normal((nr, nl)) + 1j * rng.standard_normal((nr, nl))) / math.sqrt(2)
    dvec = (rng.standard_normal(nr) + 1j * rng.standard_normal(nr)) / math.sqrt(2)
    eps = 10.0 ** np.linspace(-5.0, -1.0, K)
    ch = np.broadcast_to(h0, (K, nr, nl)).copy()
    ch[:, :, 1] = h0[:, 0][None, :] + eps[:, None] * dvec[None, :]
    ch = np.broadcast_to(ch, (1, 14, K, nr, nl))
    sl = S.make_slot(spec, 82, noise=False, channel=ch)
    ref = oracle_dense(spec, sl)
    ratio = ref["pivot_ratio"]
    n_flag = int(ref["flags"].sum())
    assert 0.2 * ratio.size < n_flag < 0.8 * ratio.size, n_flag  # a mix on both sides
    u32 = 2.0 ** -24
    L = spec.occ
    Hs = np.stack([O.interp_channel(ref["anchors"][0], spec.dmrs_sym, K, L, t, np.arange(K))
                   for t in spec.data_sym])  # [dsym][sc][rx][layer]
    kA = np.linalg.cond(O.gram(Hs, spec.sigma2))
    kH = np.linalg.cond(Hs)
    for refactor in (False, True):
        got = gpu_slot(spec, sl, dev, fp64_refactor=refactor)
        tag = f"conditioning_sweep[refactor={refactor}]"
        mask = check_flags(tag, got["flags"], ref["flags"], ratio).reshape(kA.shape)
        assert mask.sum() > 0.2 * mask.size
        g0 = (got["flags"][0] & 1) != 0
        assert np.array_equal((got["flags"][0] & 2) != 0, g0 if refactor else np.zeros_like(g0))
        err = (np.linalg.norm(got["x_hat"][0] - ref["x_hat"][0], axis=-1)
               / np.linalg.norm(ref["x_hat"][0], axis=-1))
        worst = float(np.max(err[mask] / (kA[mask] * u32)))
        print(tag, "unflagged: max err / (kappa(A) u32) =", worst)
        assert worst <= 64.0
        if refactor:
            sel = g0 & ((ref["flags"][0] & 1) != 0)
            assert sel.sum() > 0
            w64 = float(np.max(err[sel] / (kH[sel] * u32)))
            print(tag, "flagged, FP64 recomputed: max err / (kappa(H) u32) =", w64)
            assert w64 <= 8.0


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_massive_corner_rho07_35db_dense(dev, prec):
    """The massive configuration's hardest corner: Kronecker rho = 0.7 at the receiver and
    35 dB, 64 Rx x 16 layers, 256-QAM, every RE of a 6-PRB two-cell batch, with and without the
    FP64 re-computation (which then never triggers: the outputs must not change)."""
    spec = S.spec_massive_mimo(n_cells=2, n_prb=6, snr_db=35.0)
    sl = S.make_slot(spec, 3500, keep_h=False)
    ref = oracle_dense(spec, sl)
    nl, qm = spec.n_layers, spec.qm
    flat = lambda a, tail: a.reshape((-1,) + tail)
    outs = []
    for refactor in (False, True):
        got = gpu_slot(spec, sl, dev, precision=prec, fp64_refactor=refactor)
        mask = check_flags(f"corner35[{prec}]", got["flags"], ref["flags"], ref["pivot_ratio"])
        assert mask.all()
        m = compare_res(f"corner35[{prec},refactor={refactor}]",
                        dict(x_hat=flat(got["x_hat"], (nl,)), sinr=flat(got["sinr"], (nl,)),
                             llr=flat(got["llr"], (nl, qm))),
                        dict(x_hat=flat(ref["x_hat"], (nl,)), sinr=flat(ref["sinr"], (nl,)),
                             llr=flat(ref["llr"], (nl, qm))),
                        qm, flat(ref["s2eff"], (nl,)), flat(ref["x_t"], (nl,)), mask)
        if prec == "fp32":
            assert_parity(m)
        else:
            lim = TC_LIMITS[prec]
            assert m["n"] == m["n_total"]
            assert m["x_rel"] <= lim[0] and m["sinr_rel_max"] <= lim[1], m
            assert m["llr_norm_max"] <= lim[2], m
        outs.append(got)
    for k in ("x_hat", "sinr", "llr", "flags"):
        assert np.array_equal(outs[0][k], outs[1][k])


def test_massive_corner_rho07_35db_full_size_sampled(dev):
    """The benchmark's 8-cell 273-PRB 64x16 batch at the 35 dB corner with the FP64
    re-computation enabled (as the massive configuration asks): sampled REs, both band edges,
    every one compared with the FP32 bars, and no RE flagged on either side."""
    spec = S.spec_massive_mimo(snr_db=35.0)
    sl = S.make_slot(spec, 3600, keep_h=False)
    got = gpu_slot(spec, sl, dev, fp64_refactor=True)
    res = sample_res(spec, 2)
    ref = O.run_slot(sl.Y, sl.pilots, sl.sigma2, spec.dmrs_sym, spec.n_layers, spec.qm, res=res)
    m, _, _ = compare_sampled("corner35_full_size", spec.qm, got, ref, res)
    assert_parity(m)
    assert not got["flags"].any()


TC_LIMITS = {"tf32": (1e-3, 3e-3, 2e-2, 1e-3), "fp16": (1e-3, 3e-3, 2e-2, 1e-3),
             "bf16": (1e-2, 2e-2, 1e-1, 5e-3)}

SWEEP = [("carrier", snr) for snr in (10.0, 20.0, 30.0)] + \
        [("massive", snr) for snr in (20.0, 25.0, 30.0, 35.0)]


@pytest.mark.parametrize("conf,snr", SWEEP)
def test_snr_sweep_error_vs_oracle(dev, conf, snr):
    """Error against the FP64 oracle across each configuration's SNR range, for the plain FP32
    path and the FP16 / BF16 tensor-core products: the 273-PRB 16x4 64-QAM carrier (Jakes
    100 Hz) at 10, 20, 30 dB on every RE of one slot, and one cell of the 273-PRB 64x16 256-QAM
    massive batch (rho = 0.7) at 20 to 35 dB on 460 sampled REs. Prints one SWEEP row per
    precision (x_hat, SINR, normalised LLR errors, hard-bit disagreement, uncoded BER of the GPU
    and of the oracle); FP32 must meet the parity bars, FP16/BF16 the tensor-core bounds."""
    if conf == "carrier":
        spec = S.spec_carrier_273prb(snr_db=snr)
        sl = S.make_slot(spec, 2000 + int(snr), keep_h=False)
        ref = oracle_dense(spec, sl)
        res = None
    else:
        spec = S.spec_massive_mimo(n_cells=1, snr_db=snr)
        sl = S.make_slot(spec, 3000 + int(snr), keep_h=False)
        res = sample_res(spec, int(snr), n_rand=400)
        ref = O.run_slot(sl.Y, sl.pilots, sl.sigma2, spec.dmrs_sym, spec.n_layers, spec.qm,
                         res=res)
    nl, qm = spec.n_layers, spec.qm
    for prec in ("fp32", "fp16", "bf16"):
        got = gpu_slot(spec, sl, dev, precision=prec)
        ber_gpu = float(np.mean((got["llr"] < 0) != sl.bits.reshape(got["llr"].shape)))
        tag = f"{conf}@{snr:g}dB[{prec}]"
        if res is None:
            flat = lambda a, tail: a.reshape((-1,) + tail)
            mask = check_flags(tag, got["flags"], ref["flags"], ref["pivot_ratio"])
            assert mask.all()
            g = dict(x_hat=flat(got["x_hat"], (nl,)), sinr=flat(got["sinr"], (nl,)),
                     llr=flat(got["llr"], (nl, qm)))
            r = dict(x_hat=flat(ref["x_hat"], (nl,)), sinr=flat(ref["sinr"], (nl,)),
                     llr=flat(ref["llr"], (nl, qm)))
            m = compare_res(tag, g, r, qm, flat(ref["s2eff"], (nl,)), flat(ref["x_t"], (nl,)),
                            mask)
            bits_ref = sl.bits.reshape(ref["llr"].shape).reshape(-1, nl, qm)
        else:
            m, g, r = compare_sampled(tag, qm, got, ref, res)
            bits = sl.bits.reshape(got["llr"].shape)
            bits_ref = np.concatenate([bits[c, jj, kk] for c, (jj, kk) in res.items()])
        ber_ref = float(np.mean((r["llr"] < 0) != bits_ref))
        ber_gpu_same = float(np.mean((g["llr"] < 0) != bits_ref))
        dis = float(np.mean((g["llr"] < 0) != (r["llr"] < 0)))
        print(f"SWEEP {conf} snr={snr:g} prec={prec} n={m['n']} x_rel={m['x_rel']:.2e} "
              f"sinr_rel_max={m['sinr_rel_max']:.2e} llr_norm_max={m['llr_norm_max']:.2e} "
              f"bit_disagree={dis:.2e} ber_gpu_all={ber_gpu:.4e} ber_gpu={ber_gpu_same:.4e} "
              f"ber_oracle={ber_ref:.4e}")
        if prec == "fp32":
            assert_parity(m)
        else:
            lim = TC_LIMITS[prec]
            assert m["n"] == m["n_total"] and m["x_rel"] <= lim[0], m
            assert m["sinr_rel_max"] <= lim[1] and m["llr_norm_max"] <= lim[2], m
            assert dis <= lim[3], dis
