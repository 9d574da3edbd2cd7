"""Noise-variance estimate from the DMRS anchor residuals: CUDA path vs the FP64 oracle.

Tolerances:
  * Same anchors on both sides (the GPU's LS anchors, read back): relative 1e-5 on the estimate.
    The kernels form each residual in FP32 from anchors far larger than the residual (at 35 dB
    and cover 8 the time residual is about 1/100 of the anchors, costing up to ~7 bits per term),
    and sum 10^3..10^6 such terms; the rounding errors average out to well below 1e-5.
  * End to end from the received grid: relative 1e-4, since the FP32 anchors themselves differ
    from the FP64 ones by a few units in the last place, amplified by the same cancellation.
"""
import numpy as np
import pytest

from oracle import phy_oracle as O
from paper_2510_07843_gb300 import synth as S

pytestmark = pytest.mark.gpu

SAME_ANCHORS_REL = 1e-5
END_TO_END_REL = 1e-4


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


def gpu_estimates(spec, sl, dev, modes):
    """GPU anchors and the GPU estimate of every mode in `modes` (dict mode -> [cell])."""
    import torch
    from paper_2510_07843_gb300 import phy
    cfg = phy.SlotConfig.from_spec(spec)
    G = phy.n_groups(cfg)
    Y, P = T(sl.Y, dev), T(sl.pilots, dev)
    anchors = torch.empty((spec.n_cells, len(spec.dmrs_sym), G, spec.n_layers, spec.n_rx),
                          dtype=torch.complex64, device=dev)
    ws = torch.empty(phy.workspace_size(cfg), dtype=torch.uint8, device=dev)
    phy.chest(cfg, Y, P, anchors)
    out = {}
    for mode in modes:
        s2 = torch.full((spec.n_cells,), -1.0, dtype=torch.float32, device=dev)
        phy.noise_est(cfg, mode, anchors, P, s2, ws)
        out[mode] = s2
    torch.cuda.synchronize()
    return anchors.cpu().numpy(), {m: v.cpu().numpy() for m, v in out.items()}


def check_close(got, want, rel, tag):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert np.array_equal(np.isnan(got), np.isnan(want)), (tag, got, want)
    ok = ~np.isnan(want)
    err = np.abs(got[ok] - want[ok]) / np.abs(want[ok])
    print(tag, "max rel", float(err.max()) if err.size else 0.0)
    assert np.all(err <= rel), (tag, got, want)


CASES = {
    "small_51prb_4x2_one_dmrs": (S.spec_small_51prb(), 1001),
    "carrier_25prb_16x4_jakes": (S.spec_carrier_273prb(n_prb=25), 2000),
    "ragged_7prb_6x3": (S.SlotSpec(n_prb=7, n_rx=6, n_layers=3, qm=6, dmrs_sym=(2, 11),
                                   snr_db=25.0, n_taps=6, doppler_hz=300.0), 11),
    "massive_6prb_64x16_2cells": (S.spec_massive_mimo(n_cells=2, n_prb=6), 3000),
    "massive_13prb_32x16_35db": (S.spec_massive_mimo(n_cells=1, n_prb=13, n_rx=32,
                                                     snr_db=35.0), 3001),
    "cover_16_3prb_two_groups": (S.SlotSpec(n_prb=3, n_rx=2, n_layers=2, qm=2,
                                            dmrs_sym=(2, 11), occ_len=16), 5),
    "one_layer_cover_4_ragged": (S.SlotSpec(n_prb=5, n_rx=3, n_layers=1, qm=2,
                                            dmrs_sym=(3, 10), occ_len=4), 6),
}


@pytest.mark.parametrize("name", list(CASES))
def test_noise_estimate_parity_same_anchors(dev, name):
    spec, seed = CASES[name]
    sl = S.make_slot(spec, seed, keep_h=False)
    modes = O.NOISE_MODES if len(spec.dmrs_sym) == 2 else ("freq", "min")
    anchors, got = gpu_estimates(spec, sl, dev, modes)
    for mode in modes:
        want = O.noise_variance_dmrs(sl.pilots, anchors, spec.n_rx, spec.n_layers, spec.occ,
                                     mode)
        check_close(got[mode], want, SAME_ANCHORS_REL, f"{name}/{mode}")


@pytest.mark.parametrize("name", ["carrier_25prb_16x4_jakes", "massive_6prb_64x16_2cells",
                                  "small_51prb_4x2_one_dmrs"])
def test_slot_run_est_end_to_end(dev, name):
    """phy_slot_run_est writes the estimate the oracle derives from the grid, and its outputs are
    bitwise those of phy_slot_run given that estimate."""
    import torch
    from paper_2510_07843_gb300 import phy
    spec, seed = CASES[name]
    sl = S.make_slot(spec, seed, keep_h=False)
    cfg = phy.SlotConfig.from_spec(spec)
    Y, P = T(sl.Y, dev), T(sl.pilots, dev)
    a = phy.SlotBuffers(cfg, with_inputs=False)
    b = phy.SlotBuffers(cfg, with_inputs=False)
    s2 = torch.zeros(spec.n_cells, dtype=torch.float32, device=dev)
    phy.slot_run_est(cfg, "min", Y, P, s2, a.x_hat, a.sinr, a.llr, a.flags, a.workspace)
    phy.slot_run(cfg, Y, P, s2.clone(), b.x_hat, b.sinr, b.llr, b.flags, b.workspace)
    torch.cuda.synchronize()
    anchors = O.ls_anchors(sl.Y, sl.pilots, spec.dmrs_sym, spec.n_layers, spec.occ)
    want = O.noise_variance_dmrs(sl.pilots, anchors, spec.n_rx, spec.n_layers, spec.occ, "min")
    check_close(s2.cpu().numpy(), want, END_TO_END_REL, name)
    for key in ("x_hat", "sinr", "llr", "flags"):
        assert torch.equal(getattr(a, key), getattr(b, key)), key


def test_noise_estimate_full_size_massive(dev):
    """8 cells x 273 PRB, 64 Rx x 16 layers, DMRS 2 and 11 (the benchmark batch): every mode
    against the oracle on the GPU's anchors, and bitwise repeatable."""
    spec = S.spec_massive_mimo()
    sl = S.make_slot(spec, 3000, keep_h=False)
    anchors, got = gpu_estimates(spec, sl, dev, O.NOISE_MODES)
    for mode in O.NOISE_MODES:
        want = O.noise_variance_dmrs(sl.pilots, anchors, spec.n_rx, spec.n_layers, spec.occ,
                                     mode)
        check_close(got[mode], want, SAME_ANCHORS_REL, f"massive/{mode}")
    # static channel: the time residual sees the noise alone
    assert np.all(np.abs(got["time"] / spec.sigma2 - 1.0) < 0.02), got["time"]
    _, again = gpu_estimates(spec, sl, dev, ("min",))
    assert np.array_equal(again["min"], got["min"])


def test_noise_state_tracked_across_slots(dev):
    """phy_noise_track keeps a per-cell noise level on the device from slot to slot: the first
    slot takes its estimate, later ones blend alpha estimate + (1 - alpha) state, a NaN estimate
    leaves the state alone; phy_slot_run_track detects with the updated state."""
    import torch
    from paper_2510_07843_gb300 import phy
    spec, _ = CASES["carrier_25prb_16x4_jakes"]
    alpha = 0.3
    state = torch.zeros(1, dtype=torch.float32, device=dev)
    prev = None
    for k in range(4):
        sl = S.make_slot(spec, 500 + k, keep_h=False)
        cfg = phy.SlotConfig.from_spec(spec)
        _, est = gpu_estimates(spec, sl, dev, ("min",))
        e = float(est["min"][0])
        Y, P = T(sl.Y, dev), T(sl.pilots, dev)
        a = phy.SlotBuffers(cfg, with_inputs=False)
        phy.slot_run_track(cfg, "min", alpha, Y, P, state, a.x_hat, a.sinr, a.llr, a.flags,
                           a.workspace)
        b = phy.SlotBuffers(cfg, with_inputs=False)
        phy.slot_run(cfg, Y, P, state.clone(), b.x_hat, b.sinr, b.llr, b.flags, b.workspace)
        torch.cuda.synchronize()
        s_now = float(state.item())
        want = e if prev is None else alpha * e + (1 - alpha) * prev
        assert s_now == pytest.approx(want, rel=1e-6), (k, s_now, want)
        for key in ("x_hat", "sinr", "llr", "flags"):
            assert torch.equal(getattr(a, key), getattr(b, key)), key
        prev = s_now
    # an undefined estimate (two LS groups: no frequency residual) keeps the state
    spec2, seed2 = CASES["cover_16_3prb_two_groups"]
    sl2 = S.make_slot(spec2, seed2, keep_h=False)
    cfg2 = phy.SlotConfig.from_spec(spec2)
    G = phy.n_groups(cfg2)
    anchors = torch.empty((1, 2, G, spec2.n_layers, spec2.n_rx), dtype=torch.complex64,
                          device=dev)
    phy.chest(cfg2, T(sl2.Y, dev), T(sl2.pilots, dev), anchors)
    ws = torch.empty(phy.workspace_size(cfg2), dtype=torch.uint8, device=dev)
    st2 = torch.full((1,), 0.5, dtype=torch.float32, device=dev)
    phy.noise_track(cfg2, "freq", alpha, anchors, T(sl2.pilots, dev), st2, ws)
    torch.cuda.synchronize()
    assert float(st2.item()) == 0.5
