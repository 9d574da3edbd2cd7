"""Pins of the FP64 oracle against closed forms, invariants, hand-worked examples and brute force.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign, a wrong
index, a transposed operand) fails at least one of them. None re-types an oracle formula.
"""
import math

import numpy as np
import pytest
from scipy.special import erfc, j0

from conftest import golden_lines
from oracle import phy_oracle as O
from paper_2510_07843_gb300 import synth as S


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


# ------------------------------------------------------------------ constellation

@pytest.mark.parametrize("qm", [2, 4, 6, 8])
def test_constellation_unit_energy_and_grid(qm):
    pts = O.qam_points(qm)
    assert len(np.unique(np.round(pts, 12))) == 1 << qm
    assert abs(np.mean(np.abs(pts) ** 2) - 1.0) < 1e-12
    # square grid of odd integers scaled by the NR normalisation
    h = qm // 2
    nrm = math.sqrt(2.0 * (4 ** h - 1) / 3.0)
    lv = np.arange(-(2 ** h) + 1, 2 ** h, 2)
    assert set(np.round(pts.real * nrm).astype(int)) == set(lv)
    assert set(np.round(pts.imag * nrm).astype(int)) == set(lv)


@pytest.mark.parametrize("qm", [2, 4, 6, 8])
def test_constellation_gray_neighbours(qm):
    """Horizontally or vertically adjacent points differ in exactly one bit; I bits are even."""
    pts = O.qam_points(qm)
    bt = O.point_bits(qm)
    dmin = 2.0 / math.sqrt(2.0 * (4 ** (qm // 2) - 1) / 3.0)
    for a in range(len(pts)):
        for b in range(len(pts)):
            if abs(abs(pts[a] - pts[b]) - dmin) < 1e-9:
                diff = np.nonzero(bt[a] != bt[b])[0]
                assert len(diff) == 1
                # a horizontal step flips an even (in-phase) bit, a vertical one an odd bit
                horiz = abs(pts[a].imag - pts[b].imag) < 1e-9
                assert (diff[0] % 2 == 0) == horiz


def test_constellation_first_bit_is_sign():
    for qm in (2, 4, 6, 8):
        pts = O.qam_points(qm)
        bt = O.point_bits(qm)
        assert np.all((pts.real > 0) == (bt[:, 0] == 0))
        assert np.all((pts.imag > 0) == (bt[:, 1] == 0))


@pytest.mark.parametrize("qm", [2, 4, 6, 8])
def test_generator_mapper_agrees_with_oracle_slicer(qm):
    """Two independent writings of the NR mapper: the transmitter's and the oracle's."""
    rng = np.random.default_rng(qm)
    bits = rng.integers(0, 2, size=(500, qm), dtype=np.uint8)
    x = S.gray_qam_modulate(bits, qm)
    np.testing.assert_array_equal(O.slice_bits(x, qm), bits)


# ------------------------------------------------------------------ detection

def _golden_lmmse():
    cases, cur = [], None
    for tok in golden_lines("lmmse_handworked.txt"):
        if tok[0] == "case":
            cur = {"s2": float(tok[2])}
            cases.append(cur)
        else:
            cur[tok[0]] = np.array([float(v) for v in tok[1:]])
    return cases


def test_lmmse_handworked():
    for c in _golden_lmmse():
        H = (c["H"][0::2] + 1j * c["H"][1::2]).reshape(2, 2)
        y = c["y"][0::2] + 1j * c["y"][1::2]
        x_ref = c["x"][0::2] + 1j * c["x"][1::2]
        x, d = O.lmmse_gram(H, y, c["s2"])
        np.testing.assert_allclose(x, x_ref, atol=1e-14)
        np.testing.assert_allclose(d, c["d"], atol=1e-14)
        sinr, _, _ = O.sinr_unbias(x, d, c["s2"])
        np.testing.assert_allclose(sinr, c["sinr"], rtol=1e-13)
        xc, _ = O.lmmse_covariance_lu(H, y, c["s2"])
        np.testing.assert_allclose(xc, x_ref, atol=1e-14)


@pytest.mark.parametrize("nr,nl", [(2, 2), (4, 2), (16, 4), (64, 16)])
def test_zero_forcing_recovers_symbols(nr, nl):
    """Noise-free, s2 = 0: the Gram form is zero forcing and returns x exactly."""
    rng = np.random.default_rng(nr * 100 + nl)
    H = crandn(rng, 50, nr, nl)
    x = crandn(rng, 50, nl)
    y = np.einsum("brl,bl->br", H, x)
    xh, _ = O.lmmse_gram(H, y, 0.0)
    np.testing.assert_allclose(xh, x, atol=1e-10)


@pytest.mark.parametrize("nr,nl,s2", [(2, 2, 0.1), (4, 2, 0.01), (16, 4, 0.5), (8, 8, 1e-3)])
def test_push_through_identity(nr, nl, s2):
    """The paper's covariance form (LU on H H^H + s2 I) equals the Gram form."""
    rng = np.random.default_rng(7 + nr)
    for _ in range(10):
        H = crandn(rng, nr, nl)
        y = crandn(rng, nr)
        xc, W = O.lmmse_covariance_lu(H, y, s2)
        xg, _ = O.lmmse_gram(H, y, s2)
        Wg = np.linalg.inv(O.gram(H, s2)) @ np.conj(H.T)
        np.testing.assert_allclose(W, Wg, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(xc, xg, rtol=1e-10, atol=1e-12)


def test_orthogonal_channel_closed_form():
    """H^H H = c I  =>  x_hat = H^H y / (c + s2), (A^-1)_kk = 1/(c + s2)."""
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(crandn(rng, 16, 16))
    c, s2 = 2.5, 0.3
    H = math.sqrt(c) * Q[:, :4]
    y = crandn(rng, 16)
    x, d = O.lmmse_gram(H, y, s2)
    np.testing.assert_allclose(x, np.conj(H.T) @ y / (c + s2), atol=1e-13)
    np.testing.assert_allclose(d, np.full(4, 1.0 / (c + s2)), atol=1e-13)


def test_single_layer_mrc_closed_form():
    """One layer: x_hat = h^H y / (|h|^2 + s2), SINR = |h|^2 / s2."""
    rng = np.random.default_rng(4)
    h = crandn(rng, 8, 1)
    y = crandn(rng, 8)
    s2 = 0.2
    x, d = O.lmmse_gram(h, y, s2)
    nh = float(np.sum(np.abs(h) ** 2))
    np.testing.assert_allclose(x[0], np.vdot(h[:, 0], y) / (nh + s2), rtol=1e-13)
    sinr, _, _ = O.sinr_unbias(x, d, s2)
    np.testing.assert_allclose(sinr[0], nh / s2, rtol=1e-12)


def test_unbiased_error_times_sinr_is_one():
    """E|x~ - x|^2 SINR = 1 per layer for the unbiased LMMSE output (genie channel)."""
    rng = np.random.default_rng(5)
    nb, nr, nl, s2 = 40000, 4, 3, 0.3
    H = crandn(rng, nb, nr, nl)
    bits = rng.integers(0, 2, size=(nb, nl, 4), dtype=np.uint8)
    x = S.gray_qam_modulate(bits, 4)
    y = np.einsum("brl,bl->br", H, x) + math.sqrt(s2) * crandn(rng, nb, nr)
    xh, d = O.lmmse_gram(H, y, s2)
    sinr, xt, _ = O.sinr_unbias(xh, d, s2)
    v = np.abs(xt - x) ** 2 * sinr
    # mean of nb*nl samples of an O(1)-variance variable: 5 sigma ~ 0.02
    assert abs(v.mean() - 1.0) < 0.03, v.mean()


def test_pivot_ratio_closed_forms():
    A = np.diag([4.0, 1.0, 0.5]).astype(np.complex128)
    assert abs(O.pivot_ratio(A) - 0.5 / 4.0) < 1e-15
    a, b, c = 2.0, 1.0 + 1.0j, 3.0
    A2 = np.array([[a, np.conj(b)], [b, c]])
    p1 = c - abs(b) ** 2 / a  # second pivot of [[a, b*], [b, c]]
    assert abs(O.pivot_ratio(A2) - min(a, p1) / max(a, p1)) < 1e-14
    assert O.pivot_ratio(np.array([[1.0, 2.0], [2.0, 1.0]], dtype=np.complex128)) == 0.0


def test_ml_bruteforce_vs_mmse_2x2_qpsk():
    """Exact ML over 16 hypotheses: never more bit errors than MMSE on average, agrees at high
    SNR."""
    rng = np.random.default_rng(6)
    nb = 4000
    for snr_db, agree_min in ((5.0, 0.5), (25.0, 0.98)):
        s2 = 10 ** (-snr_db / 10)
        H = crandn(rng, nb, 2, 2)
        bits = rng.integers(0, 2, size=(nb, 2, 2), dtype=np.uint8)
        x = S.gray_qam_modulate(bits, 2)
        y = np.einsum("brl,bl->br", H, x) + math.sqrt(s2) * crandn(rng, nb, 2)
        ml = O.ml_detect_bruteforce(H, y, 2)
        ml_bits = O.point_bits(2)[ml]
        xh, d = O.lmmse_gram(H, y, s2)
        _, xt, _ = O.sinr_unbias(xh, d, s2)
        mm_bits = O.slice_bits(xt, 2)
        e_ml = np.mean(ml_bits != bits)
        e_mm = np.mean(mm_bits != bits)
        assert e_ml <= e_mm + 0.005, (snr_db, e_ml, e_mm)
        assert np.mean(np.all(ml_bits == mm_bits, axis=(-1, -2))) >= agree_min


def test_siso_awgn_qpsk_ber_matches_q_function():
    """Flat unit channel, genie detection: QPSK bit error rate equals Q(sqrt(SNR))."""
    rng = np.random.default_rng(8)
    nb = 200000
    snr_db = 6.0
    s2 = 10 ** (-snr_db / 10)
    bits = rng.integers(0, 2, size=(nb, 1, 2), dtype=np.uint8)
    x = S.gray_qam_modulate(bits, 2)
    H = np.ones((nb, 1, 1), dtype=np.complex128)
    y = x + math.sqrt(s2) * crandn(rng, nb, 1)
    xh, d = O.lmmse_gram(H, y, s2)
    sinr, xt, s2e = O.sinr_unbias(xh, d, s2)
    llr = O.llr_maxlog(xt, s2e, 2)
    ber = np.mean((llr < 0).astype(np.uint8) != bits)
    p = 0.5 * erfc(math.sqrt(1.0 / s2) / math.sqrt(2.0))
    sd = math.sqrt(p * (1 - p) / (2 * nb))
    assert abs(ber - p) < 5 * sd, (ber, p)


# ------------------------------------------------------------------ LLR

def test_llr_handworked_16qam():
    for tok in golden_lines("llr_handworked.txt"):
        qm = int(tok[0])
        xt = float(tok[1]) + 1j * float(tok[2])
        s2e = float(tok[3])
        ref = np.array([float(v) for v in tok[4:]])
        np.testing.assert_allclose(O.llr_maxlog(np.array([xt]), np.array([s2e]), qm)[0], ref,
                                   atol=1e-12)


def test_llr_qpsk_closed_form():
    rng = np.random.default_rng(9)
    xt = crandn(rng, 200) * 2
    s2e = rng.uniform(0.05, 2.0, 200)
    llr = O.llr_maxlog(xt, s2e, 2)
    np.testing.assert_allclose(llr[:, 0], 2 * math.sqrt(2) * xt.real / s2e, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(llr[:, 1], 2 * math.sqrt(2) * xt.imag / s2e, rtol=1e-12, atol=1e-12)


def test_llr_16qam_inner_outer_closed_form():
    """b2 of 16-QAM (inner/outer level): LLR = 4 (2 - |u|) / (10 s2eff), u = sqrt(10) Re x~."""
    rng = np.random.default_rng(10)
    xt = crandn(rng, 300) * 1.5
    s2e = rng.uniform(0.05, 1.0, 300)
    llr = O.llr_maxlog(xt, s2e, 4)
    u = np.abs(xt.real) * math.sqrt(10)
    np.testing.assert_allclose(llr[:, 2], 4 * (2 - u) / (10 * s2e), rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("qm", [2, 4, 6, 8])
def test_llr_sign_equals_slicer(qm):
    rng = np.random.default_rng(11 + qm)
    xt = crandn(rng, 2000) * 1.3
    llr = O.llr_maxlog(xt, np.full(2000, 0.3), qm)
    hard = (llr < 0).astype(np.uint8)
    np.testing.assert_array_equal(hard, O.slice_bits(xt, qm))


@pytest.mark.parametrize("qm", [4, 6, 8])
def test_llr_separable_equals_bruteforce(qm):
    """Max-log over the 2-D grid equals two 1-D PAM searches (even bits I, odd bits Q)."""
    rng = np.random.default_rng(12 + qm)
    xt = crandn(rng, 500) * 1.3
    s2e = rng.uniform(0.1, 1.0, 500)
    llr = O.llr_maxlog(xt, s2e, qm)
    pts = O.qam_points(qm)
    bt = O.point_bits(qm)
    for i in range(qm):
        comp = pts.real if i % 2 == 0 else pts.imag
        v = xt.real if i % 2 == 0 else xt.imag
        lv1 = np.unique(comp[bt[:, i] == 1])
        lv0 = np.unique(comp[bt[:, i] == 0])
        d1 = np.min((v[:, None] - lv1) ** 2, axis=1)
        d0 = np.min((v[:, None] - lv0) ** 2, axis=1)
        np.testing.assert_allclose(llr[:, i], (d1 - d0) / s2e, rtol=1e-10, atol=1e-10)


# ------------------------------------------------------------------ LS estimation

@pytest.mark.parametrize("n_prb,nl", [(1, 2), (3, 4), (5, 8), (7, 16), (51, 2), (2, 16)])
def test_ls_exact_on_constant_channel(n_prb, nl):
    """Noise-free, frequency-flat channel: every anchor equals the channel (Walsh orthogonality),
    including ragged PRB counts where the last group overlaps its neighbour."""
    rng = np.random.default_rng(n_prb * 31 + nl)
    nr = 3
    Hc = crandn(rng, nr, nl)
    L = O.occ_length(nl)
    if 6 * n_prb < L:
        pytest.skip("cover longer than the comb")
    spec = S.SlotSpec(n_prb=n_prb, n_rx=nr, n_layers=nl, qm=2, dmrs_sym=(2, 11), snr_db=100.0)
    ch = np.broadcast_to(Hc, (1, 14, spec.n_sc, nr, nl))
    sl = S.make_slot(spec, 1, noise=False, channel=ch)
    A = O.ls_anchors(sl.Y, sl.pilots, spec.dmrs_sym, nl, L)
    G = A.shape[2]
    want = np.broadcast_to(Hc.T, (1, 2, G, nl, nr))
    np.testing.assert_allclose(A, want, atol=1e-6)  # complex64 grid


def test_ls_anchor_sits_at_group_mean():
    """One layer, cover length 4 forced, channel linear in k: the LS anchor is the channel at the
    group's mean subcarrier."""
    nr, n_prb, L = 2, 3, 4
    spec = S.SlotSpec(n_prb=n_prb, n_rx=nr, n_layers=1, qm=2, dmrs_sym=(3,), occ_len=L,
                      snr_db=100.0)
    K = spec.n_sc
    a = np.array([1.0 + 0.5j, -0.3 + 0.2j])
    slope = np.array([0.01 - 0.02j, 0.03 + 0.01j])
    k = np.arange(K)
    Hk = (a[None, :] + slope[None, :] * k[:, None])[:, :, None]  # [sc][rx][1]
    ch = np.broadcast_to(Hk, (1, 14, K, nr, 1))
    sl = S.make_slot(spec, 2, noise=False, channel=ch)
    A = O.ls_anchors(sl.Y, sl.pilots, spec.dmrs_sym, 1, L)
    s, pos = O.ls_groups(K, L)
    for g in range(len(s)):
        want = a + slope * pos[0][g]
        np.testing.assert_allclose(A[0, 0, g, 0], want, atol=2e-6)


def test_ls_groups_overlap_rule():
    s, pos = O.ls_groups(3276, 8)  # 1638 comb subcarriers, 204.75 groups of 8
    assert len(s) == 205
    assert s[-1] == 1638 - 8 and s[-2] == 8 * 203
    assert pos[0][0] == 7 and pos[1][0] == 8
    s1, _ = O.ls_groups(24, 4)
    np.testing.assert_array_equal(s1, [0, 4, 8])


# ------------------------------------------------------------------ interpolation

def test_interp_handworked():
    rows = list(golden_lines("interp_handworked.txt"))
    anc = np.array([float(v) for v in rows[0][1:]])
    anc = anc[0::2] + 1j * anc[1::2]
    A = anc.reshape(1, 3, 1, 1)  # [dmrs][group][layer][rx]
    want = {int(r[0]): float(r[1]) + 1j * float(r[2]) for r in rows[1:] if r[0] != "time"}
    H = O.interp_channel(A, (2,), 12, 2, 5, np.arange(12))
    for k, v in want.items():
        assert abs(H[k, 0, 0] - v) < 1e-14, (k, H[k, 0, 0], v)
    for r in rows:
        if r[0] == "time":
            assert abs(O.time_weight((2, 11), int(r[1])) - float(r[2])) < 1e-15


def test_interp_exact_for_linear_time_variation():
    """Anchors that are the channel at the DMRS symbols of a channel linear in t reproduce it
    inside [d0, d1] and hold it outside."""
    rng = np.random.default_rng(13)
    nr, nl, K = 2, 2, 24
    H2, H11 = crandn(rng, nr, nl), crandn(rng, nr, nl)
    L = 1
    s, pos = O.ls_groups(K, L)
    G = len(s)
    A = np.zeros((2, G, nl, nr), dtype=np.complex128)
    A[0] = H2.T[None]
    A[1] = H11.T[None]
    for t in range(14):
        H = O.interp_channel(A, (2, 11), K, L, t, np.arange(K))
        a = min(max((t - 2) / 9, 0.0), 1.0)
        np.testing.assert_allclose(H, np.broadcast_to((1 - a) * H2 + a * H11, H.shape), atol=1e-14)


def test_interp_exact_for_linear_frequency_variation():
    """Single layer, L = 1 (an anchor on every comb subcarrier), channel linear in k: the
    interpolation is exact at every subcarrier between the first and last anchors."""
    rng = np.random.default_rng(14)
    nr, K = 3, 36
    a, slope = crandn(rng, nr), crandn(rng, nr) * 0.05
    s, pos = O.ls_groups(K, 1)
    A = np.zeros((1, len(s), 1, nr), dtype=np.complex128)
    for g in range(len(s)):
        A[0, g, 0] = a + slope * pos[0][g]
    k = np.arange(K)
    H = O.interp_channel(A, (2,), K, 1, 4, k)
    inside = (k >= pos[0][0]) & (k <= pos[0][-1])
    want = a[None, :] + slope[None, :] * k[:, None]
    np.testing.assert_allclose(H[inside, :, 0], want[inside], atol=1e-13)
    np.testing.assert_allclose(H[k > pos[0][-1], :, 0], np.broadcast_to(A[0, -1, 0], (1, nr)),
                               atol=1e-14)


# ------------------------------------------------------------------ whole slot

def test_slot_noise_free_recovers_bits():
    """Noise-free flat channel, full pipeline: LS + interpolation + LMMSE + LLR signs give back
    the transmitted bits on every data RE (tiny s2 keeps the LLR scale finite)."""
    spec = S.SlotSpec(n_prb=4, n_rx=4, n_layers=4, qm=6, dmrs_sym=(2, 11), snr_db=100.0)
    rng = np.random.default_rng(15)
    Hc = crandn(rng, 4, 4)
    ch = np.broadcast_to(Hc, (1, 14, spec.n_sc, 4, 4))
    sl = S.make_slot(spec, 3, noise=False, channel=ch)
    out = O.run_slot(sl.Y, sl.pilots, np.array([1e-10]), spec.dmrs_sym, 4, 6)
    hard = (out["llr"] < 0).astype(np.uint8)
    np.testing.assert_array_equal(hard, sl.bits)
    np.testing.assert_allclose(out["x_hat"], sl.x, atol=1e-4)


def test_slot_sampled_matches_dense():
    spec = S.spec_small_51prb(n_prb=5)
    sl = S.make_slot(spec, 16)
    dense = O.run_slot(sl.Y, sl.pilots, sl.sigma2, spec.dmrs_sym, 2, 4)
    rng = np.random.default_rng(0)
    jj = rng.integers(0, 13, 40)
    kk = rng.integers(0, spec.n_sc, 40)
    samp = O.run_slot(sl.Y, sl.pilots, sl.sigma2, spec.dmrs_sym, 2, 4, res={0: (jj, kk)})
    np.testing.assert_allclose(samp["x_hat_0"], dense["x_hat"][0, jj, kk], rtol=1e-13)
    np.testing.assert_allclose(samp["llr_0"], dense["llr"][0, jj, kk], rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ noise-variance estimate

def _golden_noise():
    return {r[0]: float(r[1]) for r in golden_lines("noise_handworked.txt")}


def test_noise_gain_handworked():
    """Three PRB, cover 4, one comb-0 layer: the gains worked out by hand, overlap included."""
    want = _golden_noise()
    P = S.dmrs_pilots(np.random.default_rng(5), 36, 1, 2, 4)[None]  # complex128, |P| = 1
    assert O.noise_gain(P[:, :1], 1, 4, "freq")[0] == pytest.approx(want["gain_freq"], rel=1e-14)
    assert O.noise_gain(P, 1, 4, "time")[0] == pytest.approx(want["gain_time"], rel=1e-14)
    # both DMRS symbols: the frequency residuals of each symbol
    assert O.noise_gain(P, 1, 4, "freq")[0] == pytest.approx(2 * want["gain_freq"], rel=1e-14)


def test_noise_residual_handworked_quadratic():
    """Anchors p^2 at the anchor subcarriers: the frequency residuals of a quadratic, by hand."""
    want = _golden_noise()
    _, pos = O.ls_groups(36, 4)
    for comb in range(2):
        A = (pos[comb] ** 2).astype(np.complex128).reshape(1, 1, 5, 1, 1)
        got = O.noise_residual_energy(A, 36, 4, "freq")[0]
        assert got == pytest.approx(want["energy_quadratic"], rel=1e-14)


@pytest.mark.parametrize("n_prb,nl,occ,nd", [(3, 1, 4, 2), (2, 4, 0, 2), (3, 8, 0, 1),
                                             (4, 2, 1, 2), (5, 16, 0, 2), (3, 3, 8, 2)])
def test_noise_gain_matches_probed_linear_map(n_prb, nl, occ, nd):
    """The summed gain equals the residual energy of unit impulses sent through the LS estimator:
    one 'antenna' per DMRS RE, carrying 1 on that RE and 0 elsewhere, so that the residual energy
    summed over the antennas is sum over residuals of sum_k |c_k|^2."""
    L = occ if occ else O.occ_length(nl)
    if 6 * n_prb < L:
        pytest.skip("cover longer than the comb")
    dmrs = (2, 11)[:nd]
    spec = S.SlotSpec(n_prb=n_prb, n_rx=1, n_layers=nl, qm=2, dmrs_sym=dmrs, occ_len=L)
    sl = S.make_slot(spec, 17 + nl)
    K = spec.n_sc
    Yp = np.zeros((1, 14, nd * K, K), dtype=np.complex128)
    for d, t in enumerate(dmrs):
        Yp[0, t, d * K + np.arange(K), np.arange(K)] = 1.0
    A = O.ls_anchors(Yp, sl.pilots, dmrs, nl, L)
    for mode in ("freq", "time"):
        probed = O.noise_residual_energy(A, K, L, mode)[0]
        assert O.noise_gain(sl.pilots, nl, L, mode)[0] == pytest.approx(probed, rel=1e-12,
                                                                        abs=1e-12)


@pytest.mark.parametrize("n_prb,nl", [(3, 1), (5, 2), (4, 4), (7, 8), (6, 16)])
def test_noise_residuals_vanish_without_noise(n_prb, nl):
    """Noise-free channel constant over the band: both residuals are zero for any layer count
    (Walsh orthogonality), ragged PRB counts included."""
    rng = np.random.default_rng(100 + nl)
    nr = 3
    Hc = crandn(rng, nr, nl)
    spec = S.SlotSpec(n_prb=n_prb, n_rx=nr, n_layers=nl, qm=2, dmrs_sym=(2, 11))
    ch = np.broadcast_to(Hc, (1, 14, spec.n_sc, nr, nl))
    sl = S.make_slot(spec, 1, noise=False, channel=ch)
    A = O.ls_anchors(sl.Y, sl.pilots, spec.dmrs_sym, nl, spec.occ)
    scale = np.sum(np.abs(A) ** 2)
    for mode in ("freq", "time"):
        assert O.noise_residual_energy(A, spec.n_sc, spec.occ, mode)[0] < 1e-12 * scale


def test_noise_frequency_residual_vanishes_for_linear_channel_one_layer_per_comb():
    """Two layers (one per comb), cover 4 forced, channel linear in k: every anchor is the channel
    at its group's mean subcarrier, so linear prediction from the neighbours is exact."""
    nr, nl, L = 2, 2, 4
    spec = S.SlotSpec(n_prb=5, n_rx=nr, n_layers=nl, qm=2, dmrs_sym=(3,), occ_len=L)
    rng = np.random.default_rng(9)
    a, slope = crandn(rng, nr, nl), 0.02 * crandn(rng, nr, nl)
    k = np.arange(spec.n_sc)
    ch = a[None, None] + slope[None, None] * k[None, :, None, None]
    ch = np.broadcast_to(ch, (14, spec.n_sc, nr, nl))[None]
    sl = S.make_slot(spec, 2, noise=False, channel=ch)
    A = O.ls_anchors(sl.Y, sl.pilots, spec.dmrs_sym, nl, L)
    assert O.noise_residual_energy(A, spec.n_sc, L, "freq")[0] < 1e-11 * np.sum(np.abs(A) ** 2)


def test_noise_time_residual_vanishes_for_static_channel():
    """Noise-free frequency-selective channel that does not change in time: the time residual is
    zero (the frequency one is not)."""
    spec = S.spec_carrier_273prb(n_prb=20, doppler_hz=0.0)
    sl = S.make_slot(spec, 3, noise=False)
    A = O.ls_anchors(sl.Y, sl.pilots, spec.dmrs_sym, spec.n_layers, spec.occ)
    scale = np.sum(np.abs(A) ** 2)
    assert O.noise_residual_energy(A, spec.n_sc, spec.occ, "time")[0] < 1e-12 * scale
    assert O.noise_residual_energy(A, spec.n_sc, spec.occ, "freq")[0] > 1e-6 * scale


@pytest.mark.parametrize("nl", [1, 4, 16])
@pytest.mark.parametrize("mode", ["freq", "time"])
def test_noise_estimate_unbiased_on_flat_channel(nl, mode):
    """Flat channel plus white noise: the mean estimate over independent slots is s2 within the
    spread of the mean (the residual energy is a sum of many chi-square terms)."""
    nr, snr = 8, 12.0
    ests = []
    for seed in range(8):
        rng = np.random.default_rng(1000 * nl + seed)
        spec = S.SlotSpec(n_prb=24, n_rx=nr, n_layers=nl, qm=2, dmrs_sym=(2, 11), snr_db=snr)
        ch = np.broadcast_to(crandn(rng, nr, nl), (1, 14, spec.n_sc, nr, nl))
        sl = S.make_slot(spec, 50 + seed, channel=ch)
        A = O.ls_anchors(sl.Y, sl.pilots, spec.dmrs_sym, nl, spec.occ)
        ests.append(O.noise_variance_dmrs(sl.pilots, A, nr, nl, spec.occ, mode)[0] / spec.sigma2)
    ests = np.array(ests)
    spread = ests.std(ddof=1) / math.sqrt(len(ests))
    assert abs(ests.mean() - 1.0) < max(5.0 * spread, 0.01), (ests.mean(), spread)
    assert spread < 0.05


def test_noise_estimate_pure_noise():
    """No signal at all: the estimate is the noise level (any pilots, any mode)."""
    spec = S.SlotSpec(n_prb=40, n_rx=16, n_layers=4, qm=2, dmrs_sym=(2, 11), snr_db=0.0)
    zero = np.zeros((1, 14, spec.n_sc, spec.n_rx, spec.n_layers))
    sl = S.make_slot(spec, 77, channel=zero)
    A = O.ls_anchors(sl.Y, sl.pilots, spec.dmrs_sym, spec.n_layers, spec.occ)
    for mode in O.NOISE_MODES:
        est = O.noise_variance_dmrs(sl.pilots, A, spec.n_rx, spec.n_layers, spec.occ, mode)[0]
        assert est == pytest.approx(1.0, rel=0.05), mode


def test_noise_estimate_modes_and_undefined_cases():
    """'min' is the smaller estimate; time needs two DMRS symbols, frequency three groups."""
    spec = S.spec_carrier_273prb(n_prb=30)
    sl = S.make_slot(spec, 4)
    A = O.ls_anchors(sl.Y, sl.pilots, spec.dmrs_sym, spec.n_layers, spec.occ)
    est = {m: O.noise_variance_dmrs(sl.pilots, A, spec.n_rx, spec.n_layers, spec.occ, m)[0]
           for m in O.NOISE_MODES}
    assert est["min"] == min(est["freq"], est["time"])
    one = O.noise_variance_dmrs(sl.pilots[:, :1], A[:, :1], spec.n_rx, spec.n_layers, spec.occ,
                                "time")
    assert np.isnan(one[0])
    assert O.noise_variance_dmrs(sl.pilots[:, :1], A[:, :1], spec.n_rx, spec.n_layers, spec.occ,
                                 "min")[0] == est_freq_one(sl, A, spec)
    # 3 PRB with cover 16: two groups only, so no interior anchor
    sp2 = S.SlotSpec(n_prb=3, n_rx=2, n_layers=2, qm=2, dmrs_sym=(2, 11), occ_len=16)
    s2 = S.make_slot(sp2, 1)
    A2 = O.ls_anchors(s2.Y, s2.pilots, sp2.dmrs_sym, 2, 16)
    assert np.isnan(O.noise_variance_dmrs(s2.pilots, A2, 2, 2, 16, "freq")[0])
    assert np.isfinite(O.noise_variance_dmrs(s2.pilots, A2, 2, 2, 16, "min")[0])


def est_freq_one(sl, A, spec):
    return O.noise_variance_dmrs(sl.pilots[:, :1], A[:, :1], spec.n_rx, spec.n_layers, spec.occ,
                                 "freq")[0]


# ------------------------------------------------------------------ BFP fronthaul decompression

def test_bfp_handworked_blocks():
    rows = list(golden_lines("bfp_handworked.txt"))
    for blk, vals in zip(rows[0::2], rows[1::2]):
        assert blk[0] == "block" and vals[0] == "re"
        w, scale = int(blk[1]), float(blk[2])
        raw = np.array([int(b, 16) for b in blk[3:]], dtype=np.uint8)
        assert raw.size == O.bfp_block_bytes(w)
        got = O.bfp_decompress(raw, (1, 1, 1, 12), w, scale)[0, 0, 0]
        want = np.array([float(v) for v in vals[1:]])
        np.testing.assert_array_equal(got.real, want[0::2])
        np.testing.assert_array_equal(got.imag, want[1::2])


@pytest.mark.parametrize("w,dtype", [(16, ">i2"), (8, "i1")])
def test_bfp_byte_aligned_widths_are_plain_integers(w, dtype):
    """At 8 and 16 bits the mantissas are whole (big-endian) integers: numpy reads them directly."""
    rng = np.random.default_rng(w)
    n = 50
    raw = rng.integers(0, 256, size=(n, O.bfp_block_bytes(w)), dtype=np.uint8)
    raw[:, 0] &= 0x3F  # some high-nibble junk stays in the parameter byte
    got = O.bfp_decompress(raw.reshape(-1), (1, 1, 1, 12 * n), w, 0.25)[0, 0, 0]
    for b in range(n):
        m = np.frombuffer(raw[b, 1:].tobytes(), dtype=dtype).astype(np.float64)
        v = m * 2.0 ** (raw[b, 0] & 0xF) * 0.25
        np.testing.assert_array_equal(got[12 * b:12 * b + 12], v[0::2] + 1j * v[1::2])


@pytest.mark.parametrize("w", list(range(1, 17)))
def test_bfp_round_trip_within_the_quantisation_step(w):
    """The sender's compressor (written independently, with numpy bit packing) and the oracle's
    decompressor agree up to half a quantisation step 2^(e-1) scale per block (the mantissas are
    rounded), or the saturation of the one-bit width."""
    spec = S.SlotSpec(n_prb=3, n_rx=3, n_layers=2, qm=4, dmrs_sym=(2,), snr_db=15.0)
    sl = S.make_slot(spec, 100 + w, keep_h=False)
    scale = 2.0 ** -12
    c = S.bfp_compress(sl.Y, w, scale)
    nb = O.bfp_block_bytes(w)
    assert c.size == sl.Y.size // 12 * nb
    got = O.bfp_decompress(c, sl.Y.shape, w, scale)
    e = (c.reshape(-1, nb)[:, 0] & 0xF).astype(np.float64)
    step = (2.0 ** e * scale).reshape(sl.Y.shape[:-1] + (-1,)).repeat(12, axis=-1)
    err = np.maximum(np.abs(got.real - sl.Y.real), np.abs(got.imag - sl.Y.imag))
    if w > 1:
        assert np.all(err <= 0.5 * step + 0.5 * scale + 1e-12)
    else:  # one bit: -1 or 0 times the step
        assert np.all(np.isin(np.round(got.real / step), [-1.0, 0.0]))


# ------------------------------------------------------------------ CNN denoiser

def test_conv3x3_matches_scipy_correlate():
    """Each (out, in) channel pair is scipy's 2-D cross-correlation with zero fill."""
    from scipy.signal import correlate2d
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 3, 14, 12))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    z = O.conv3x3(a, W, b)
    for n in range(2):
        for co in range(4):
            want = b[co] + sum(correlate2d(a[n, ci], W[co, ci], mode="same", boundary="fill")
                               for ci in range(3))
            np.testing.assert_allclose(z[n, co], want, rtol=1e-12, atol=1e-12)


def test_cnn_is_the_identity_with_a_zero_last_layer():
    rng = np.random.default_rng(2)
    p = rng.standard_normal(19682) * 0.1
    p[-(2 * 32 * 9 + 2):] = 0.0  # W4, b4
    x = rng.standard_normal((3, 2, 14, 12))
    out, _ = O.cnn_forward(p, x)
    np.testing.assert_array_equal(out, x)


def test_cnn_backward_matches_finite_differences():
    """Central differences of the FP64 loss, on every parameter tensor and the input. The step
    is small (1e-7) because the ReLUs put kinks within 1e-5 of many parameters; at 1e-7 the
    differences match to 1e-5 (a wrong term or index errs by the size of the gradient)."""
    rng = np.random.default_rng(3)
    p = rng.standard_normal(19682) * 0.2
    x = rng.standard_normal((2, 2, 14, 12))
    lab = rng.standard_normal((2, 2, 14, 12))
    out, acts = O.cnn_forward(p, x)
    g, dx = O.cnn_backward(p, acts, out, lab)
    h = 1e-7
    offs = np.cumsum([0] + [int(np.prod(s)) for s in O.cnn_param_shapes()])
    idx = []
    for a, b in zip(offs[:-1], offs[1:]):  # a few entries of each tensor
        idx += list(rng.choice(np.arange(a, b), size=min(6, b - a), replace=False))
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (O.cnn_loss(O.cnn_forward(p + e, x)[0], lab)
              - O.cnn_loss(O.cnn_forward(p - e, x)[0], lab)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(abs(fd), 0.1), (i, fd, g[i])
    for _ in range(8):
        ii = tuple(rng.integers(0, s) for s in x.shape)
        e = np.zeros_like(x)
        e[ii] = h
        fd = (O.cnn_loss(O.cnn_forward(p, x + e)[0], lab)
              - O.cnn_loss(O.cnn_forward(p, x - e)[0], lab)) / (2 * h)
        assert abs(fd - dx[ii]) <= 1e-5 * max(abs(fd), 0.1), (ii, fd, dx[ii])


def test_adam_first_step_moves_by_the_learning_rate():
    """After one step from zero moments the bias-corrected update is lr * g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m, v = O.adam_step(np.ones(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(p, 1.0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_bf16_rounding_matches_torch():
    """The oracle's bfloat16 rounding equals torch's float -> bfloat16 conversion (to nearest,
    ties to even), including exact ties and values that carry into the exponent."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8),
                                  2.0 - 2.0 ** -9, 0.0, -0.0, 65504.0])]).astype(np.float32)
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    np.testing.assert_array_equal(O.round_bf16(v), want)


def test_cnn_bf16_operands_stay_within_the_rounding_bound():
    """Rounding weights and activations to bfloat16 (relative step 2^-8) moves the output of the
    residual network by far less than the rounding of its largest terms would allow."""
    rng = np.random.default_rng(6)
    p = rng.standard_normal(19682) * 0.1
    x = rng.standard_normal((4, 2, 14, 12))
    out32, _ = O.cnn_forward(p, x)
    out16, _ = O.cnn_forward(p, x, operands="bf16")
    err = np.linalg.norm(out16 - out32) / np.linalg.norm(out32 - x)
    assert 1e-4 < err < 3e-2, err  # rounding visible, and of the size 2^-8 predicts
