"""Seeded synthetic uplink slots: the input side of the receiver, and nothing of it.

This module is the transmitter and the propagation channel of a PUSCH-like uplink slot. It draws
bits, maps them to Gray QAM symbols, places DMRS pilots on a comb with a Walsh cover, passes every
layer through a tapped-delay-line (TDL) channel and adds white Gaussian noise. It holds none of the
receiver's arithmetic (no estimation, interpolation, detection or demapping); both the CUDA
library and the FP64 oracle take its arrays as plain inputs.

The paper evaluates its LMMSE receiver on 3GPP NR slots over TDL-C channels (Sec. IV); the TDL-C
tap table is not reproduced here. Channels are synthetic exponential power-delay profiles with a
stated RMS delay spread, optional Jakes sum-of-sinusoids Doppler and optional Kronecker receive
correlation.

Conventions (shared with the C ABI):
  Y        [cell][sym][rx][sc]          complex64   received grid, all 14 symbols
  pilots   [cell][dmrs][layer][sc]      complex64   0 off the layer's comb
  bits     [cell][dsym][sc][layer][qm]  uint8       data symbols only, codeword order
  x        [cell][dsym][sc][layer]      complex128  transmitted data symbols
  H        [cell][sym][sc][rx][layer]   complex128  true channel per symbol
Layer l sits on comb c = l % 2 (subcarriers k = 2m + c) with Walsh row o = l // 2 of length L,
L the smallest power of two >= ceil(n_layers / 2). The pilot on comb subcarrier m is
r_{d,c}(m) * w_o[m mod L], r a unit-modulus QPSK sequence shared by the layers of one comb.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np

SYMBOLS_PER_SLOT = 14
SCS_HZ_DEFAULT = 30e3


@dataclasses.dataclass(frozen=True)
class SlotSpec:
    """Shape and channel recipe of one batch of uplink slots (one slot per cell)."""

    n_cells: int = 1
    n_prb: int = 51
    n_rx: int = 4
    n_layers: int = 2
    qm: int = 4
    dmrs_sym: Tuple[int, ...] = (2,)
    occ_len: int = 0  # 0: smallest power of two >= ceil(n_layers / 2)
    snr_db: float = 20.0
    n_taps: int = 6
    delay_spread_s: float = 100e-9
    doppler_hz: float = 0.0
    rho_rx: float = 0.0
    scs_hz: float = SCS_HZ_DEFAULT
    n_sym: int = SYMBOLS_PER_SLOT
    slot_index: int = 0

    @property
    def n_sc(self) -> int:
        return 12 * self.n_prb

    @property
    def occ(self) -> int:
        return self.occ_len if self.occ_len > 0 else auto_occ_len(self.n_layers)

    @property
    def data_sym(self) -> Tuple[int, ...]:
        return tuple(t for t in range(self.n_sym) if t not in self.dmrs_sym)

    @property
    def sigma2(self) -> float:
        return 10.0 ** (-self.snr_db / 10.0)


def auto_occ_len(n_layers: int) -> int:
    half = (n_layers + 1) // 2
    L = 1
    while L < half:
        L *= 2
    return L


# Named workloads.  The sizes follow the 30 kHz NR numerology: 273 PRB fill a 100 MHz carrier.
def spec_small_51prb(**kw) -> SlotSpec:
    """51 PRB, 4 Rx x 2 layers, 16-QAM, one DMRS symbol, 6-tap 100 ns PDP, static, 20 dB."""
    base = dict(n_cells=1, n_prb=51, n_rx=4, n_layers=2, qm=4, dmrs_sym=(2,), snr_db=20.0,
                n_taps=6, delay_spread_s=100e-9, doppler_hz=0.0, rho_rx=0.0)
    base.update(kw)
    return SlotSpec(**base)


def spec_carrier_273prb(**kw) -> SlotSpec:
    """273 PRB, 16 Rx x 4 layers, 64-QAM, DMRS 2 and 11, 23-tap 300 ns PDP, Jakes 100 Hz."""
    base = dict(n_cells=1, n_prb=273, n_rx=16, n_layers=4, qm=6, dmrs_sym=(2, 11), snr_db=20.0,
                n_taps=23, delay_spread_s=300e-9, doppler_hz=100.0, rho_rx=0.0)
    base.update(kw)
    return SlotSpec(**base)


def spec_massive_mimo(**kw) -> SlotSpec:
    """273 PRB, 64 Rx x 16 layers, 256-QAM, DMRS 2 and 11, Kronecker rho=0.7, 8 cells."""
    base = dict(n_cells=8, n_prb=273, n_rx=64, n_layers=16, qm=8, dmrs_sym=(2, 11),
                snr_db=30.0, n_taps=23, delay_spread_s=300e-9, doppler_hz=0.0, rho_rx=0.7)
    base.update(kw)
    return SlotSpec(**base)


# Serving workload: a stream of per-cell uplink jobs of uneven shapes.
SERVING_RX = (4, 16, 32, 64)
SERVING_QM = (2, 4, 6, 8)


def spec_serving_job(rng: np.random.Generator) -> SlotSpec:
    """One job of the serving stream: 4-273 PRB (uniform), 4/16/32/64 Rx, 1-16 layers (uniform,
    clamped to the antenna count), QPSK to 256-QAM, DMRS 2 and 11, the 23-tap 300 ns PDP with
    Jakes 100 Hz Doppler, 10-30 dB SNR (uniform)."""
    n_rx = int(rng.choice(SERVING_RX))
    return SlotSpec(n_cells=1, n_prb=int(rng.integers(4, 274)), n_rx=n_rx,
                    n_layers=min(int(rng.integers(1, 17)), n_rx), qm=int(rng.choice(SERVING_QM)),
                    dmrs_sym=(2, 11), snr_db=float(rng.uniform(10.0, 30.0)), n_taps=23,
                    delay_spread_s=300e-9, doppler_hz=100.0, rho_rx=0.0)


def serving_arrivals(n_cells: int, rate_hz: float, duration_s: float, seed: int):
    """Poisson arrivals of every cell (exponential gaps of mean 1/rate_hz) within duration_s:
    a list of (time in seconds, cell), sorted by time."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_cells):
        t = rng.exponential(1.0 / rate_hz)
        while t < duration_s:
            out.append((float(t), c))
            t += rng.exponential(1.0 / rate_hz)
    out.sort()
    return out


# ----------------------------------------------------------------------------------------------
# Transmitter
# ----------------------------------------------------------------------------------------------

def gray_qam_modulate(bits: np.ndarray, qm: int) -> np.ndarray:
    """Map bit groups (last axis, length qm, b0 first) to unit-energy Gray QAM points.

    Even-indexed bits b0, b2, ... set the in-phase PAM level and odd-indexed bits the quadrature
    one, nested as in the NR modulation mapper: for h = qm/2 bits per axis the level is
    (1-2e0)(2^(h-1) - (1-2e1)(2^(h-2) - ... (2 - (1-2e_{h-1})))).
    """
    if qm not in (2, 4, 6, 8):
        raise ValueError(f"qm must be 2, 4, 6 or 8, got {qm}")
    b = bits.astype(np.int64)
    h = qm // 2

    def axis(e):  # e: list of sign-source bit arrays for one axis, outermost first
        inner = np.ones(e[0].shape, dtype=np.float64)
        for i in range(h - 1, 0, -1):
            inner = float(2 ** (h - i)) - (1 - 2 * e[i]) * inner
        return (1 - 2 * e[0]) * inner

    re = axis([b[..., 2 * i] for i in range(h)])
    im = axis([b[..., 2 * i + 1] for i in range(h)])
    norm = math.sqrt(2.0 * (4 ** h - 1) / 3.0)
    return (re + 1j * im) / norm


def walsh_row(o: int, L: int, m: np.ndarray) -> np.ndarray:
    """Sylvester-Hadamard row o of length L evaluated at m mod L (values +-1)."""
    idx = np.asarray(m) % L
    pc = np.zeros(idx.shape, dtype=np.int64)
    v = idx & o
    while np.any(v):
        pc += v & 1
        v = v >> 1
    return np.where(pc % 2 == 0, 1.0, -1.0)


def dmrs_pilots(rng: np.random.Generator, n_sc: int, n_layers: int, n_dmrs: int, L: int
                ) -> np.ndarray:
    """Pilot grid [dmrs][layer][sc] (complex128), comb-2 with a length-L Walsh cover."""
    n_comb = n_sc // 2
    P = np.zeros((n_dmrs, n_layers, n_sc), dtype=np.complex128)
    m = np.arange(n_comb)
    for d in range(n_dmrs):
        # one unit-modulus QPSK base sequence per comb, shared by the layers on that comb
        base = []
        for c in range(2):
            q = rng.integers(0, 2, size=(2, n_comb))
            base.append(((1 - 2 * q[0]) + 1j * (1 - 2 * q[1])) / math.sqrt(2.0))
        for l in range(n_layers):
            c, o = l % 2, l // 2
            P[d, l, 2 * m + c] = base[c] * walsh_row(o, L, m)
    return P


# ----------------------------------------------------------------------------------------------
# Channel
# ----------------------------------------------------------------------------------------------

def exp_pdp(n_taps: int, delay_spread_s: float, span_db: float = 25.0
            ) -> Tuple[np.ndarray, np.ndarray]:
    """Exponential power-delay profile with a given discrete RMS delay spread.

    Tap powers fall by span_db from the first tap to the last one, are normalised to sum 1, and
    sit on a uniform delay grid tau_l = l * delta.  The RMS spread is linear in delta for fixed
    relative powers, so delta is the target divided by the unit-grid spread.
    """
    if n_taps == 1:
        return np.zeros(1), np.ones(1)
    l = np.arange(n_taps, dtype=np.float64)
    p = 10.0 ** (-(span_db / 10.0) * l / (n_taps - 1))
    p /= p.sum()
    mean = (p * l).sum()
    rms_unit = math.sqrt((p * (l - mean) ** 2).sum())
    delta = delay_spread_s / rms_unit
    return l * delta, p


def rms_delay_spread(tau: np.ndarray, p: np.ndarray) -> float:
    p = p / p.sum()
    mean = (p * tau).sum()
    return float(math.sqrt((p * (tau - mean) ** 2).sum()))


def jakes_sos(rng: np.random.Generator, shape: Sequence[int], times_s: np.ndarray,
              doppler_hz: float, n_sin: int = 16) -> np.ndarray:
    """Unit-power Rayleigh fading processes by sum of sinusoids (random arrival angles/phases).

    g(t) = (1/sqrt(M)) sum_n exp(j(2 pi f_D cos(a_n) t + phi_n)), with arrival angles
    a_n = (2 pi n - pi + theta)/M equispaced over the circle under a random rotation theta and
    i.i.d. uniform phases phi_n, so the autocorrelation tends to J0(2 pi f_D tau) (after the
    sum-of-sinusoids construction of Zheng and Xiao, 2003).  Returns shape + (len(times_s),).
    """
    M = n_sin
    shape = tuple(shape)
    theta = rng.uniform(-np.pi, np.pi, size=shape + (1,))
    phi = rng.uniform(-np.pi, np.pi, size=shape + (M,))
    n = np.arange(1, M + 1)
    alpha = (2.0 * np.pi * n - np.pi + theta) / M  # shape + (M,)
    w = 2.0 * np.pi * doppler_hz * np.cos(alpha)  # rad/s
    ph = w[..., None] * times_s[None, :] + phi[..., None]  # shape + (M, T)
    return np.exp(1j * ph).sum(axis=-2) / math.sqrt(M)


def rx_correlation_sqrt(n_rx: int, rho: float) -> np.ndarray:
    """Hermitian square root of R[i,j] = rho^|i-j| (exponential receive correlation)."""
    i = np.arange(n_rx)
    R = rho ** np.abs(i[:, None] - i[None, :])
    w, V = np.linalg.eigh(R)
    return (V * np.sqrt(np.clip(w, 0.0, None))) @ V.conj().T


def tdl_channel(rng: np.random.Generator, spec: SlotSpec) -> np.ndarray:
    """True channel H[sym][sc][rx][layer] (complex128) of one cell over one slot."""
    tau, p = exp_pdp(spec.n_taps, spec.delay_spread_s)
    n_t = spec.n_sym
    shape = (spec.n_taps, spec.n_rx, spec.n_layers)
    g = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)
    if spec.doppler_hz > 0.0:
        sym_dur = 1e-3 * (15e3 / spec.scs_hz) / SYMBOLS_PER_SLOT
        t = (spec.slot_index * SYMBOLS_PER_SLOT + np.arange(n_t)) * sym_dur
        fade = jakes_sos(rng, shape, t, spec.doppler_hz)  # [tap][rx][layer][t]
        taps = fade.transpose(3, 0, 1, 2)  # [t][tap][rx][layer]
    else:
        taps = np.broadcast_to(g, (n_t,) + shape)
    taps = taps * np.sqrt(p)[None, :, None, None]
    if spec.rho_rx > 0.0:
        Rs = rx_correlation_sqrt(spec.n_rx, spec.rho_rx)
        taps = np.einsum("ij,tljk->tlik", Rs, taps)
    k = np.arange(spec.n_sc, dtype=np.float64)
    F = np.exp(-2j * np.pi * spec.scs_hz * np.outer(k, tau))  # [sc][tap]
    if spec.doppler_hz > 0.0:
        H = np.einsum("kl,tlrj->tkrj", F, taps)
    else:
        H0 = (F @ taps[0].reshape(spec.n_taps, -1)).reshape(spec.n_sc, spec.n_rx, spec.n_layers)
        H = np.broadcast_to(H0, (n_t,) + H0.shape)
    return H


# ----------------------------------------------------------------------------------------------
# Slot assembly
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Slot:
    spec: SlotSpec
    Y: np.ndarray        # [cell][sym][rx][sc] complex64
    pilots: np.ndarray   # [cell][dmrs][layer][sc] complex64
    sigma2: np.ndarray   # [cell] float32
    bits: np.ndarray     # [cell][dsym][sc][layer][qm] uint8
    x: np.ndarray        # [cell][dsym][sc][layer] complex128
    H: Optional[list]    # per cell: [sym][sc][rx][layer] complex128 (None if not kept)


def make_slot(spec: SlotSpec, seed: int, keep_h: bool = True, noise: bool = True,
              channel: Optional[np.ndarray] = None) -> Slot:
    """Draw one slot per cell.  channel, if given, replaces the TDL draw: [cell][sym][sc][rx][l]."""
    rng = np.random.default_rng(seed)
    C, S, R, L, K = spec.n_cells, spec.n_sym, spec.n_rx, spec.n_layers, spec.n_sc
    dsym = spec.data_sym
    nd = len(spec.dmrs_sym)
    Y = np.empty((C, S, R, K), dtype=np.complex64)
    P_all = np.empty((C, nd, L, K), dtype=np.complex64)
    bits = np.empty((C, len(dsym), K, L, spec.qm), dtype=np.uint8)
    X = np.empty((C, len(dsym), K, L), dtype=np.complex128)
    H_all = [] if keep_h else None
    s2 = spec.sigma2
    for c in range(C):
        H = tdl_channel(rng, spec) if channel is None else channel[c]
        P = dmrs_pilots(rng, K, L, nd, spec.occ)
        b = rng.integers(0, 2, size=(len(dsym), K, L, spec.qm), dtype=np.uint8)
        x = gray_qam_modulate(b, spec.qm)
        tx = np.zeros((S, K, L), dtype=np.complex128)
        for j, t in enumerate(dsym):
            tx[t] = x[j]
        for d, t in enumerate(spec.dmrs_sym):
            tx[t] = P[d].T
        rx = np.einsum("tkrl,tkl->trk", H, tx)
        if noise and s2 > 0.0:
            n = rng.standard_normal((S, R, K, 2))
            rx = rx + math.sqrt(s2 / 2.0) * (n[..., 0] + 1j * n[..., 1])
        Y[c] = rx.astype(np.complex64)
        P_all[c] = P.astype(np.complex64)
        bits[c] = b
        X[c] = x
        if keep_h:
            H_all.append(H)
    return Slot(spec=spec, Y=Y, pilots=P_all, sigma2=np.full(C, s2, dtype=np.float32),
                bits=bits, x=X, H=H_all)


# ----------------------------------------------------------------------------------------------
# Fronthaul: block-floating-point compression at the radio unit (the sending side)
# ----------------------------------------------------------------------------------------------

def bfp_compress(Y: np.ndarray, iq_width: int, scale: float) -> np.ndarray:
    """Byte stream of the grid Y [cell][sym][rx][sc] as blocks [cell][sym][rx][prb].

    Each block: a parameter byte holding the exponent e (0..15) in its low four bits, then the 24
    values I0, Q0, I1, Q1, ... of the PRB as w-bit two's-complement mantissas, most significant
    bit first. The sender quantises round(Y / scale) to integers, takes the smallest e for which
    every value of the block rounded to a multiple of 2^e fits w bits, and saturates what still
    does not (e capped at 15).
    """
    w = int(iq_width)
    if not 1 <= w <= 16:
        raise ValueError("iq_width must be 1..16")
    Y = np.asarray(Y)
    n_cells, n_sym, n_rx, n_sc = Y.shape
    v = np.empty(Y.shape + (2,), dtype=np.float64)
    v[..., 0], v[..., 1] = Y.real, Y.imag
    q = np.rint(v / np.float64(np.float32(scale))).reshape(-1, 24)  # [block][24]
    lo, hi = -(1 << (w - 1)), (1 << (w - 1)) - 1
    e = np.full(q.shape[0], 15, dtype=np.int64)
    for cand in range(15, -1, -1):  # smallest exponent that fits
        m = np.rint(q / (1 << cand))
        fits = np.all((m >= lo) & (m <= hi), axis=1)
        e = np.where(fits, cand, e)
    m = np.clip(np.rint(q / (1 << e)[:, None]), lo, hi).astype(np.int64)
    u = (m & ((1 << w) - 1)).astype(np.uint32)  # two's complement in w bits
    bits = ((u[:, :, None] >> np.arange(w - 1, -1, -1, dtype=np.uint32)) & 1).astype(np.uint8)
    payload = np.packbits(bits.reshape(q.shape[0], 24 * w), axis=1)  # 3w bytes per block
    out = np.concatenate([e.astype(np.uint8)[:, None], payload], axis=1)
    return out.reshape(-1)
