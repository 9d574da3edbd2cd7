"""Statistical checks of the seeded input generator (channel, pilots, noise)."""
import math

import numpy as np
import pytest
from scipy.special import j0

from paper_2510_07843_gb300 import synth as S


def test_pdp_rms_delay_spread_and_power():
    for n, ds in ((6, 100e-9), (23, 300e-9)):
        tau, p = S.exp_pdp(n, ds)
        assert abs(p.sum() - 1) < 1e-12
        assert abs(S.rms_delay_spread(tau, p) - ds) < 1e-15
        assert np.all(np.diff(p) < 0)


def test_channel_power_is_unit():
    spec = S.spec_carrier_273prb(n_rx=4, n_layers=2, n_prb=20, doppler_hz=0.0)
    rng = np.random.default_rng(0)
    pw = []
    for _ in range(200):
        H = S.tdl_channel(rng, spec)
        pw.append(np.mean(np.abs(H[0]) ** 2))
    assert abs(np.mean(pw) - 1.0) < 0.05


def test_kronecker_rx_correlation():
    spec = S.SlotSpec(n_prb=1, n_rx=6, n_layers=1, n_taps=1, rho_rx=0.7)
    rng = np.random.default_rng(1)
    hs = np.stack([S.tdl_channel(rng, spec)[0, 0, :, 0] for _ in range(20000)])
    R = hs.T @ hs.conj() / len(hs)
    i = np.arange(6)
    np.testing.assert_allclose(R, 0.7 ** np.abs(i[:, None] - i[None, :]), atol=0.04)


def test_jakes_autocorrelation_is_bessel():
    rng = np.random.default_rng(2)
    fd = 100.0
    t = np.linspace(0, 5e-3, 51)
    g = S.jakes_sos(rng, (4000,), t, fd)
    assert abs(np.mean(np.abs(g) ** 2) - 1.0) < 0.03
    for lag in (5, 10, 20, 40):
        r = np.mean(g[:, lag:] * np.conj(g[:, :-lag])).real
        assert abs(r - j0(2 * math.pi * fd * t[lag])) < 0.05, (lag, r)


def test_noise_variance():
    spec = S.SlotSpec(n_prb=10, n_rx=2, n_layers=1, qm=2, snr_db=10.0)
    ch = np.zeros((1, 14, spec.n_sc, 2, 1), dtype=np.complex128)
    sl = S.make_slot(spec, 5, channel=ch)
    v = np.mean(np.abs(sl.Y.astype(np.complex128)) ** 2)
    assert abs(v / spec.sigma2 - 1) < 0.05


def test_pilot_structure():
    rng = np.random.default_rng(3)
    P = S.dmrs_pilots(rng, 48, 6, 2, 4)
    for l in range(6):
        c = l % 2
        on = P[:, l, c::2]
        off = P[:, l, 1 - c::2]
        assert np.allclose(np.abs(on), 1.0) and np.all(off == 0)
    # layers sharing a comb share the base sequence up to the Walsh sign
    ratio = P[0, 2, 0::2] / P[0, 0, 0::2]
    assert np.allclose(np.abs(ratio), 1) and np.allclose(ratio.imag, 0)


def test_seeded_reproducible():
    spec = S.spec_small_51prb(n_prb=3)
    a = S.make_slot(spec, 42)
    b = S.make_slot(spec, 42)
    assert np.array_equal(a.Y, b.Y) and np.array_equal(a.bits, b.bits)


def test_bfp_compressor_rejects_bad_widths_and_sizes_its_stream():
    spec = S.SlotSpec(n_prb=2, n_rx=3, n_layers=1, qm=2, dmrs_sym=(2,))
    sl = S.make_slot(spec, 1, keep_h=False)
    for w in (0, 17):
        with pytest.raises(ValueError):
            S.bfp_compress(sl.Y, w, 1e-3)
    for w in (1, 9, 16):
        c = S.bfp_compress(sl.Y, w, 1e-3)
        assert c.dtype == np.uint8 and c.size == 14 * 3 * 2 * (1 + 3 * w)
        assert np.all((c.reshape(-1, 1 + 3 * w)[:, 0] & 0xF0) == 0)  # exponent byte: low nibble


def test_true_channel_array_layout_is_what_the_kernels_index():
    """The generator's channel arrays may be strided; made C-ordered they index as
    [sym][sc][rx][layer] (Y = H x at every symbol)."""
    spec = S.SlotSpec(n_prb=2, n_rx=3, n_layers=2, qm=2, dmrs_sym=(2,), doppler_hz=300.0,
                      n_taps=3, snr_db=200.0)
    sl = S.make_slot(spec, 4, keep_h=True, noise=False)
    H = np.ascontiguousarray(np.stack(sl.H), dtype=np.complex128)
    t = spec.data_sym[0]
    y = np.einsum("krl,kl->rk", H[0, t], sl.x[0, 0])
    np.testing.assert_allclose(y, sl.Y[0, t], atol=1e-5)


def test_denoiser_initial_parameters_are_the_identity_network():
    from paper_2510_07843_gb300 import denoise as D
    from oracle import phy_oracle as O
    p = D.init_params(3)
    assert p.dtype == np.float32 and p.size == 19682
    assert np.all(p[-(2 * 32 * 9 + 2):] == 0.0)
    x = np.random.default_rng(0).standard_normal((2, 2, 14, 12))
    out, _ = O.cnn_forward(p.astype(np.float64), x)
    np.testing.assert_array_equal(out, x)


def test_serving_stream_shapes_and_rates():
    """The serving workload's job shapes stay in their ranges (layers never above antennas) and
    its arrivals are Poisson at the stated rate per cell (count within 5 sigma)."""
    import numpy as np
    rng = np.random.default_rng(0)
    specs = [S.spec_serving_job(rng) for _ in range(2000)]
    assert all(4 <= s.n_prb <= 273 and s.n_rx in S.SERVING_RX and 1 <= s.n_layers <= s.n_rx
               and s.n_layers <= 16 and s.qm in S.SERVING_QM for s in specs)
    assert {s.n_rx for s in specs} == set(S.SERVING_RX) and min(s.n_prb for s in specs) == 4
    arr = S.serving_arrivals(32, 2000.0, 0.05, 1)
    mean = 32 * 2000.0 * 0.05
    assert abs(len(arr) - mean) < 5 * mean ** 0.5
    assert all(a[0] <= b[0] for a, b in zip(arr, arr[1:]))
    assert {c for _, c in arr} == set(range(32))
