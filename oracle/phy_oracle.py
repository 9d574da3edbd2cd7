"""FP64 oracle of the uplink PUSCH receiver inner loop (test infrastructure only).

Plain, slow and written to be checked by eye against its definitions. Every array is promoted to
complex128 / float64 on entry; numpy routines (solve, inv, cholesky, LU) serve as single steps.
Vectorisation is over independent resource elements (REs) only; nothing is blocked, fused or
reordered inside one RE's computation.

Steps and where they come from:

* LMMSE detection (Sec. III-B, Fig. 3; Sec. IV). The paper inverts the received-signal covariance
  R with an LU factorisation followed by forward/backward substitution. `lmmse_covariance_lu`
  writes that form out: W = H^H (H H^H + s2 I)^-1. `lmmse_gram` is the same estimator in the
  Gram form x = (H^H H + s2 I)^-1 H^H y, equal by the push-through identity; it is what the
  slot pipeline uses, with the per-layer error diag((H^H H + s2 I)^-1) that the paper's
  "matrix inversion" stage yields.
* Covariance products by multiply-accumulate (Fig. 2(b)): H^H H and H^H y.
* Channel estimation (named as a SIMD target in Sec. III-B, no method given): DMRS least squares
  on a comb of two with a Walsh cover of length L, then linear interpolation in frequency and time.
* Demapping to soft bits (implied by the LDPC decoder that follows detection in Sec. IV; the paper
  gives no method): max-log LLRs over the NR Gray QAM constellation, by brute force over all points.
* Ill-conditioning flag: Cholesky pivot ratio min L_kk^2 / max L_kk^2 below a threshold.
* Noise-variance estimate (the paper treats the noise level as known; no method given): residuals
  of the LS anchors against their prediction from neighbouring anchors in frequency or from the
  other DMRS symbol, normalised by the exact noise gain of each residual (see the section at the
  end of this file).
* Learned channel denoiser (no learned part in the paper): a residual 3x3 CNN on 12 x 14 tiles of
  the interpolated LS estimate, its forward pass, loss, backward pass and Adam written out with
  numpy (see the last section).
* Block-floating-point fronthaul decompression (the grid's arrival format in a split-7 software DU;
  no format in the paper): bit unpacking of per-PRB blocks with a shared exponent, by Python
  integers (see the last section).

Readings where the paper is silent (each also fixed in the C ABI):
  - Layer l uses comb c = l % 2 (k = 2m + c) and Walsh row o = l // 2; L is the smallest power of
    two >= ceil(n_layers/2). LS group g covers comb indices m = s_g .. s_g+L-1 with
    s_g = min(L g, n_comb - L); the last group overlaps its neighbour so that every group is full.
    The group's anchor sits at the mean subcarrier 2 s_g + (L-1) + c.
  - Frequency interpolation is linear between neighbouring anchors of the layer's comb and holds
    the end anchors outside them. Time interpolation holds with one DMRS symbol and, with two
    (d0 < d1), uses a = clamp((t-d0)/(d1-d0), 0, 1). Frequency is applied first.
  - DMRS symbols carry no data. Outputs are indexed by data symbol j (the non-DMRS symbols in
    increasing order).
  - Output x_hat is the biased LMMSE estimate W y. With e_k = s2 (A^-1)_kk (the per-layer MSE),
    mu_k = 1 - e_k, SINR_k = mu_k / e_k, unbiased x~_k = x_hat_k / mu_k and noise
    s2eff_k = e_k / mu_k. e_k is clamped to [1e-30, 1 - 1e-7] so SINR stays finite.
  - LLR sign: positive means bit 0. No clipping.
"""
from __future__ import annotations

import math
from typing import Dict, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg

E_MIN = 1e-30
E_MAX = 1.0 - 1e-7
PIVOT_RATIO_MIN = 1e-6


# ----------------------------------------------------------------------------------------------
# Constellation (NR Gray QAM; the paper names QAM with MCS tables but prints no mapping)
# ----------------------------------------------------------------------------------------------

def qam_points(qm: int) -> np.ndarray:
    """All 2^qm points, index p holding bits b_i = (p >> (qm-1-i)) & 1, b0 the first bit.

    The closed forms of the NR modulation mapper, written per order:
      QPSK : ((1-2b0) + j(1-2b1)) / sqrt(2)
      16QAM: ((1-2b0)(2-(1-2b2)) + j(1-2b1)(2-(1-2b3))) / sqrt(10)
      64QAM: ((1-2b0)(4-(1-2b2)(2-(1-2b4))) + j(1-2b1)(4-(1-2b3)(2-(1-2b5)))) / sqrt(42)
      256QAM: ((1-2b0)(8-(1-2b2)(4-(1-2b4)(2-(1-2b6))))
              + j(1-2b1)(8-(1-2b3)(4-(1-2b5)(2-(1-2b7))))) / sqrt(170)
    """
    pts = np.empty(1 << qm, dtype=np.complex128)
    for p in range(1 << qm):
        b = [(p >> (qm - 1 - i)) & 1 for i in range(qm)]
        s = [1 - 2 * v for v in b]
        if qm == 2:
            re, im, nrm = s[0], s[1], math.sqrt(2.0)
        elif qm == 4:
            re = s[0] * (2 - s[2])
            im = s[1] * (2 - s[3])
            nrm = math.sqrt(10.0)
        elif qm == 6:
            re = s[0] * (4 - s[2] * (2 - s[4]))
            im = s[1] * (4 - s[3] * (2 - s[5]))
            nrm = math.sqrt(42.0)
        elif qm == 8:
            re = s[0] * (8 - s[2] * (4 - s[4] * (2 - s[6])))
            im = s[1] * (8 - s[3] * (4 - s[5] * (2 - s[7])))
            nrm = math.sqrt(170.0)
        else:
            raise ValueError(f"unsupported qm {qm}")
        pts[p] = complex(re, im) / nrm
    return pts


def point_bits(qm: int) -> np.ndarray:
    """[2^qm][qm] bit table matching qam_points."""
    p = np.arange(1 << qm)[:, None]
    i = np.arange(qm)[None, :]
    return ((p >> (qm - 1 - i)) & 1).astype(np.uint8)


# ----------------------------------------------------------------------------------------------
# DMRS least squares with comb and Walsh cover
# ----------------------------------------------------------------------------------------------

def occ_length(n_layers: int) -> int:
    L = 1
    while L < (n_layers + 1) // 2:
        L *= 2
    return L


def ls_groups(n_sc: int, L: int) -> Tuple[np.ndarray, np.ndarray]:
    """Group starts s_g (comb index) and anchor subcarriers pos[c][g] for combs c = 0, 1."""
    n_comb = n_sc // 2
    if n_comb < L:
        raise ValueError("fewer comb subcarriers than the cover length")
    G = -(-n_comb // L)
    s = np.array([min(L * g, n_comb - L) for g in range(G)], dtype=np.int64)
    pos = np.stack([2 * s + (L - 1) + c for c in range(2)]).astype(np.float64)
    return s, pos


def ls_anchors(Y: np.ndarray, pilots: np.ndarray, dmrs_sym: Sequence[int], n_layers: int,
               L: int) -> np.ndarray:
    """LS anchors [cell][dmrs][group][layer][rx] (complex128).

    H_d,l(g) = (1/L) sum_{m in group g} Y[d][:, 2m+c] conj(P_d,l(2m+c)), c = l % 2.
    """
    Y = np.asarray(Y, dtype=np.complex128)
    P = np.asarray(pilots, dtype=np.complex128)
    n_cells, _, n_rx, n_sc = Y.shape
    s, _ = ls_groups(n_sc, L)
    G = len(s)
    out = np.zeros((n_cells, len(dmrs_sym), G, n_layers, n_rx), dtype=np.complex128)
    for cell in range(n_cells):
        for d, t in enumerate(dmrs_sym):
            for l in range(n_layers):
                c = l % 2
                ks = 2 * (s[:, None] + np.arange(L)[None, :]) + c  # [group][i]
                prod = Y[cell, t][:, ks] * np.conj(P[cell, d, l, ks])[None]  # [rx][group][i]
                out[cell, d, :, l, :] = (prod.sum(axis=-1) / L).T
    return out


# ----------------------------------------------------------------------------------------------
# Linear interpolation
# ----------------------------------------------------------------------------------------------

def freq_weights(pos: np.ndarray, k: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """For subcarriers k: lower anchor index g and weight b of anchor g+1 (hold outside)."""
    k = np.asarray(k, dtype=np.float64)
    G = len(pos)
    if G == 1:
        return np.zeros(k.shape, dtype=np.int64), np.zeros(k.shape)
    g = np.searchsorted(pos, k, side="right") - 1
    g = np.clip(g, 0, G - 2)
    b = (k - pos[g]) / (pos[g + 1] - pos[g])
    b = np.clip(b, 0.0, 1.0)
    return g, b


def time_weight(dmrs_sym: Sequence[int], t: int) -> float:
    """Weight of the second DMRS symbol's estimate at symbol t (0 with a single DMRS symbol)."""
    if len(dmrs_sym) == 1:
        return 0.0
    d0, d1 = dmrs_sym
    return min(max((t - d0) / (d1 - d0), 0.0), 1.0)


def interp_channel(anchors_cell: np.ndarray, dmrs_sym: Sequence[int], n_sc: int, L: int,
                   t: int, k: np.ndarray) -> np.ndarray:
    """Interpolated channel [len(k)][rx][layer] at symbol t for one cell's anchors.

    anchors_cell: [dmrs][group][layer][rx]. Frequency first (per layer on its comb), then time.
    """
    A = np.asarray(anchors_cell, dtype=np.complex128)
    nd, G, n_layers, n_rx = A.shape
    _, pos = ls_groups(n_sc, L)
    k = np.asarray(k)
    Hf = np.zeros((nd, len(k), n_rx, n_layers), dtype=np.complex128)
    for l in range(n_layers):
        g, b = freq_weights(pos[l % 2], k)
        g1 = np.minimum(g + 1, G - 1)
        for d in range(nd):
            Hf[d, :, :, l] = (1.0 - b)[:, None] * A[d, g, l, :] + b[:, None] * A[d, g1, l, :]
    a = time_weight(dmrs_sym, t)
    if nd == 1:
        return Hf[0]
    return (1.0 - a) * Hf[0] + a * Hf[1]


# ----------------------------------------------------------------------------------------------
# LMMSE detection
# ----------------------------------------------------------------------------------------------

def gram(H: np.ndarray, sigma2: float) -> np.ndarray:
    """A = H^H H + s2 I for a batch H [..., rx, layer]."""
    H = np.asarray(H, dtype=np.complex128)
    A = np.conj(np.swapaxes(H, -1, -2)) @ H
    n = H.shape[-1]
    return A + sigma2 * np.eye(n)


def lmmse_gram(H: np.ndarray, y: np.ndarray, sigma2: float) -> Tuple[np.ndarray, np.ndarray]:
    """x_hat = (H^H H + s2 I)^-1 H^H y and d = diag((H^H H + s2 I)^-1), batched over REs."""
    H = np.asarray(H, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    A = gram(H, sigma2)
    b = np.conj(np.swapaxes(H, -1, -2)) @ y[..., None]
    x = np.linalg.solve(A, b)[..., 0]
    d = np.real(np.diagonal(np.linalg.inv(A), axis1=-2, axis2=-1))
    return x, d


def lmmse_covariance_lu(H: np.ndarray, y: np.ndarray, sigma2: float
                        ) -> Tuple[np.ndarray, np.ndarray]:
    """The paper's form: R = H H^H + s2 I factored by LU, W = H^H R^-1, x_hat = W y.

    Returns (x_hat, W) for a single RE (H [rx][layer], y [rx]).
    """
    H = np.asarray(H, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    n_rx = H.shape[0]
    R = H @ np.conj(H.T) + sigma2 * np.eye(n_rx)
    lu, piv = scipy.linalg.lu_factor(R)
    # R^-1 H by forward/backward substitution, then W = (R^-1 H)^H since R is Hermitian
    RinvH = scipy.linalg.lu_solve((lu, piv), H)
    W = np.conj(RinvH.T)
    return W @ y, W


def pivot_ratio(A: np.ndarray) -> np.ndarray:
    """min_k L_kk^2 / max_k L_kk^2 of the Cholesky factor of a batch of Hermitian PD matrices.

    Matrices whose factorisation fails (not positive definite) get ratio 0.
    """
    A = np.asarray(A, dtype=np.complex128)
    flat = A.reshape((-1,) + A.shape[-2:])
    out = np.zeros(flat.shape[0])
    for i in range(flat.shape[0]):
        try:
            Lc = np.linalg.cholesky(flat[i])
        except np.linalg.LinAlgError:
            out[i] = 0.0
            continue
        p = np.real(np.diagonal(Lc)) ** 2
        out[i] = p.min() / p.max()
    return out.reshape(A.shape[:-2])


def sinr_unbias(x_hat: np.ndarray, d: np.ndarray, sigma2: float
                ) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Per-layer SINR, unbiased symbols x~ and effective noise s2eff from x_hat and diag(A^-1)."""
    e = np.clip(sigma2 * np.asarray(d, dtype=np.float64), E_MIN, E_MAX)
    mu = 1.0 - e
    sinr = mu / e
    return sinr, np.asarray(x_hat) / mu, e / mu


# ----------------------------------------------------------------------------------------------
# Max-log LLR demapping
# ----------------------------------------------------------------------------------------------

def llr_maxlog(x_t: np.ndarray, s2eff: np.ndarray, qm: int) -> np.ndarray:
    """LLR [..., qm]: (min_{s: b_i=1} |x~-s|^2 - min_{s: b_i=0} |x~-s|^2) / s2eff, brute force."""
    pts = qam_points(qm)
    bt = point_bits(qm)
    x_t = np.asarray(x_t, dtype=np.complex128)
    dist = np.abs(x_t[..., None] - pts) ** 2  # [..., 2^qm]
    out = np.empty(x_t.shape + (qm,))
    for i in range(qm):
        d1 = np.min(dist[..., bt[:, i] == 1], axis=-1)
        d0 = np.min(dist[..., bt[:, i] == 0], axis=-1)
        out[..., i] = (d1 - d0) / np.asarray(s2eff)
    return out


def slice_bits(x_t: np.ndarray, qm: int) -> np.ndarray:
    """Hard bits of the nearest constellation point (ties to the lower point index)."""
    pts = qam_points(qm)
    bt = point_bits(qm)
    dist = np.abs(np.asarray(x_t, dtype=np.complex128)[..., None] - pts) ** 2
    return bt[np.argmin(dist, axis=-1)]


def ml_detect_bruteforce(H: np.ndarray, y: np.ndarray, qm: int) -> np.ndarray:
    """Exhaustive maximum likelihood over all layer symbol vectors (tiny cases only).

    H [..., rx, layer], y [..., rx]; returns the point indices [..., layer].
    """
    pts = qam_points(qm)
    H = np.asarray(H, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    n_l = H.shape[-1]
    M = len(pts)
    idx = np.stack(np.unravel_index(np.arange(M ** n_l), (M,) * n_l), axis=-1)  # [M^n][n_l]
    S = pts[idx]  # [M^n][n_l]
    r = y[..., None, :] - np.einsum("...rl,hl->...hr", H, S)
    cost = np.sum(np.abs(r) ** 2, axis=-1)
    return idx[np.argmin(cost, axis=-1)]


# ----------------------------------------------------------------------------------------------
# Whole slot
# ----------------------------------------------------------------------------------------------

def detect_res(anchors_cell: np.ndarray, Y_cell: np.ndarray, dmrs_sym: Sequence[int],
               n_layers: int, L: int, qm: int, sigma2: float, t: int, k: np.ndarray,
               pivot_min: float = PIVOT_RATIO_MIN) -> Dict[str, np.ndarray]:
    """All outputs for the REs (t, k) of one cell: interpolate, detect, SINR, LLR, flag."""
    n_sc = Y_cell.shape[-1]
    H = interp_channel(anchors_cell, dmrs_sym, n_sc, L, t, k)
    y = np.asarray(Y_cell[t][:, k].T, dtype=np.complex128)  # [len(k)][rx]
    x_hat, d = lmmse_gram(H, y, sigma2)
    sinr, x_t, s2eff = sinr_unbias(x_hat, d, sigma2)
    llr = llr_maxlog(x_t, s2eff, qm)
    ratio = pivot_ratio(gram(H, sigma2))
    flags = (ratio < pivot_min).astype(np.uint8)
    return dict(x_hat=x_hat, sinr=sinr, llr=llr, flags=flags, x_t=x_t, s2eff=s2eff, H=H,
                pivot_ratio=ratio)


def run_slot(Y: np.ndarray, pilots: np.ndarray, sigma2: np.ndarray, dmrs_sym: Sequence[int],
             n_layers: int, qm: int, occ_len: int = 0,
             res: Optional[Dict[int, Tuple[np.ndarray, np.ndarray]]] = None,
             pivot_min: float = PIVOT_RATIO_MIN) -> Dict[str, np.ndarray]:
    """The whole receiver for every data RE of every cell (or a sample of REs).

    Y [cell][sym][rx][sc]; pilots [cell][dmrs][layer][sc]; sigma2 [cell].
    Dense outputs: x_hat [cell][dsym][sc][layer], sinr same, llr [...][qm], flags [cell][dsym][sc],
    pivot_ratio [cell][dsym][sc] (the value the flag thresholds).
    With res = {cell: (j_idx, k_idx)} only those REs (data symbol j, subcarrier k) are computed and
    each output is returned flat in that order per cell (keys 'x_hat_<cell>' etc.).
    """
    Y = np.asarray(Y)
    n_cells, n_sym, n_rx, n_sc = Y.shape
    L = occ_len if occ_len > 0 else occ_length(n_layers)
    anchors = ls_anchors(Y, pilots, dmrs_sym, n_layers, L)
    data_sym = [t for t in range(n_sym) if t not in dmrs_sym]
    out: Dict[str, np.ndarray] = {"anchors": anchors}
    if res is None:
        nj = len(data_sym)
        xh = np.zeros((n_cells, nj, n_sc, n_layers), dtype=np.complex128)
        sn = np.zeros((n_cells, nj, n_sc, n_layers))
        ll = np.zeros((n_cells, nj, n_sc, n_layers, qm))
        fl = np.zeros((n_cells, nj, n_sc), dtype=np.uint8)
        pr = np.zeros((n_cells, nj, n_sc))
        ks = np.arange(n_sc)
        for c in range(n_cells):
            for j, t in enumerate(data_sym):
                r = detect_res(anchors[c], Y[c], dmrs_sym, n_layers, L, qm, float(sigma2[c]), t,
                               ks, pivot_min)
                xh[c, j], sn[c, j], ll[c, j], fl[c, j] = r["x_hat"], r["sinr"], r["llr"], r["flags"]
                pr[c, j] = r["pivot_ratio"]
        out.update(x_hat=xh, sinr=sn, llr=ll, flags=fl, pivot_ratio=pr)
        return out
    for c, (jj, kk) in res.items():
        jj = np.asarray(jj)
        kk = np.asarray(kk)
        parts = {key: [] for key in ("x_hat", "sinr", "llr", "flags", "pivot_ratio")}
        order = []
        for j in np.unique(jj):
            sel = np.nonzero(jj == j)[0]
            r = detect_res(anchors[c], Y[c], dmrs_sym, n_layers, L, qm, float(sigma2[c]),
                           data_sym[j], kk[sel], pivot_min)
            for key in parts:
                parts[key].append(r[key])
            order.append(sel)
        inv = np.argsort(np.concatenate(order))
        for key in parts:
            out[f"{key}_{c}"] = np.concatenate(parts[key], axis=0)[inv]
    return out




# ----------------------------------------------------------------------------------------------
# Noise-variance estimate from the DMRS (the paper takes the noise level as known)
# ----------------------------------------------------------------------------------------------
#
# Reading (no method in the paper): a noise sample is the residual of an LS anchor against a
# prediction of it from other anchors of the same layer, under the receiver's own channel model.
#  * frequency: every interior anchor against the linear interpolation of its two neighbours,
#      e = H_d,l(g) - a_g H_d,l(g-1) - b_g H_d,l(g+1),  g = 1 .. G-2, every DMRS symbol d,
#      a_g = (p_g+1 - p_g) / (p_g+1 - p_g-1), b_g = (p_g - p_g-1) / (p_g+1 - p_g-1), p the anchor
#      subcarriers;
#  * time (two DMRS symbols): every anchor against the same anchor of the other symbol,
#      e = H_0,l(g) - H_1,l(g).
# Each residual is a fixed linear function of the DMRS REs, e = sum_k c_k Y(k), with
# c_k = (1/L) conj(P(k)) times the signed weight of the group(s) holding k, so white noise of
# variance s2 per RE leaves E|e|^2 = s2 gamma with gamma = sum_k |c_k|^2, and
#   s2_hat = sum |e|^2 / (n_rx sum gamma)   (sums over d, l, g and, for |e|^2, the antennas r).
# Without noise the frequency residual vanishes for a channel constant over the three groups (and,
# with one layer per comb, for one linear in frequency), the time residual for a channel that does
# not change between the DMRS symbols; any other channel variation only adds to E|e|^2. Each
# estimate is therefore unbiased or too large, and the "min" mode takes the smaller of the two.
# The frequency estimate needs three groups, the time one two DMRS symbols (NaN otherwise).

NOISE_MODES = ("freq", "time", "min")


def anchor_neighbour_weights(pos: np.ndarray, g: int) -> Tuple[float, float]:
    """(a_g, b_g): weights of anchors g-1 and g+1 in the linear prediction of anchor g."""
    span = pos[g + 1] - pos[g - 1]
    return (pos[g + 1] - pos[g]) / span, (pos[g] - pos[g - 1]) / span


def noise_residual_energy(anchors: np.ndarray, n_sc: int, L: int, mode: str) -> np.ndarray:
    """sum |e|^2 per cell from anchors [cell][dmrs][group][layer][rx] ('freq' or 'time')."""
    A = np.asarray(anchors, dtype=np.complex128)
    n_cells, n_dmrs, G, _, _ = A.shape
    out = np.zeros(n_cells)
    if mode == "time":
        if n_dmrs == 2:
            out += np.sum(np.abs(A[:, 0] - A[:, 1]) ** 2, axis=(1, 2, 3))
        return out
    _, pos = ls_groups(n_sc, L)
    for g in range(1, G - 1):
        a, b = anchor_neighbour_weights(pos[0], g)  # the same on both combs
        e = A[:, :, g] - a * A[:, :, g - 1] - b * A[:, :, g + 1]
        out += np.sum(np.abs(e) ** 2, axis=(1, 2, 3))
    return out


def noise_gain(pilots: np.ndarray, n_layers: int, L: int, mode: str) -> np.ndarray:
    """sum gamma per cell: for each residual the coefficient vector c over the DMRS REs of the
    symbol(s) it uses, written out, and its squared norm."""
    P = np.asarray(pilots, dtype=np.complex128)
    n_cells, n_dmrs, _, n_sc = P.shape
    s, pos = ls_groups(n_sc, L)
    G = len(s)
    out = np.zeros(n_cells)

    def group_coef(cell, d, l, terms):
        coef = np.zeros(n_sc, dtype=np.complex128)
        for grp, w in terms:
            ks = 2 * (s[grp] + np.arange(L)) + l % 2
            coef[ks] += w * np.conj(P[cell, d, l, ks]) / L
        return coef

    for cell in range(n_cells):
        for l in range(n_layers):
            if mode == "time":
                if n_dmrs < 2:
                    continue
                for g in range(G):
                    c0 = group_coef(cell, 0, l, [(g, 1.0)])   # coefficients on symbol 0's REs
                    c1 = group_coef(cell, 1, l, [(g, -1.0)])  # and on symbol 1's
                    out[cell] += np.sum(np.abs(c0) ** 2) + np.sum(np.abs(c1) ** 2)
                continue
            for d in range(n_dmrs):
                for g in range(1, G - 1):
                    a, b = anchor_neighbour_weights(pos[l % 2], g)
                    coef = group_coef(cell, d, l, [(g, 1.0), (g - 1, -a), (g + 1, -b)])
                    out[cell] += np.sum(np.abs(coef) ** 2)
    return out


def noise_variance_dmrs(pilots: np.ndarray, anchors: np.ndarray, n_rx: int, n_layers: int,
                        L: int, mode: str = "min") -> np.ndarray:
    """s2_hat per cell from the LS anchors and the pilots; NaN where the mode has no residual."""
    n_sc = np.asarray(pilots).shape[-1]
    if mode == "min":
        f = noise_variance_dmrs(pilots, anchors, n_rx, n_layers, L, "freq")
        t = noise_variance_dmrs(pilots, anchors, n_rx, n_layers, L, "time")
        return np.fmin(f, t)  # NaN only where both are
    energy = noise_residual_energy(anchors, n_sc, L, mode)
    gain = noise_gain(pilots, n_layers, L, mode)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(gain > 0.0, energy / (n_rx * gain), np.nan)


# ----------------------------------------------------------------------------------------------
# Block-floating-point fronthaul decompression (the step before channel estimation in a split-7
# fronthaul, which the paper's software-DU setting receives the grid over; no format is printed)
# ----------------------------------------------------------------------------------------------
#
# Reading: the grid arrives per (cell, symbol, antenna, PRB) as one block of 1 + 3w bytes: a
# parameter byte whose low four bits are the shared exponent e (high four bits ignored), then the
# 24 mantissas of the PRB's 12 REs in the order I0, Q0, I1, Q1, ..., each a w-bit two's-complement
# integer (1 <= w <= 16), packed most significant bit first across the bytes. The decompressed
# value is mantissa * 2^e * scale.

def bfp_block_bytes(iq_width: int) -> int:
    return 1 + 3 * iq_width


def bfp_decompress(Yc: np.ndarray, shape: Tuple[int, int, int, int], iq_width: int,
                   scale: float) -> np.ndarray:
    """Grid [cell][sym][rx][sc] (complex128) from the byte stream Yc of blocks
    [cell][sym][rx][prb]."""
    n_cells, n_sym, n_rx, n_sc = shape
    n_prb = n_sc // 12
    w = iq_width
    nb = bfp_block_bytes(w)
    raw = np.asarray(Yc, dtype=np.uint8).reshape(n_cells, n_sym, n_rx, n_prb, nb)
    out = np.zeros(shape, dtype=np.complex128)
    for idx in np.ndindex(n_cells, n_sym, n_rx, n_prb):
        blk = raw[idx]
        e = int(blk[0]) & 0xF
        bits = int.from_bytes(bytes(blk[1:]), "big")  # 24 w bits, first mantissa on top
        vals = []
        for i in range(24):
            m = (bits >> (24 * w - (i + 1) * w)) & ((1 << w) - 1)
            if m >= 1 << (w - 1):
                m -= 1 << w
            vals.append(m * (2.0 ** e) * scale)
        c, t, r, p = idx
        out[c, t, r, 12 * p:12 * p + 12] = np.array(vals[0::2]) + 1j * np.array(vals[1::2])
    return out


# ----------------------------------------------------------------------------------------------
# Learned channel denoiser (not in the paper, which has no learned part): a residual CNN on
# 12-subcarrier x 14-symbol tiles of the interpolated LS estimate, one tile per (PRB, Rx, layer)
# ----------------------------------------------------------------------------------------------
#
# Tiles are [2][14][12] (real, imaginary; symbol rows; subcarrier columns). Layers: 3x3
# cross-correlations with zero padding, channels 2 -> 32 -> 32 -> 32 -> 2, ReLU after the first
# three, and the input added to the output (the network predicts the correction). Parameters are
# one flat vector in the order W1 [32][2][3][3], b1 [32], W2 [32][32][3][3], b2, W3, b3,
# W4 [2][32][3][3], b4. Loss: the mean over tiles and tile positions of |out - H|^2 (real and
# imaginary squared errors summed). Optimiser: Adam with bias correction.

CNN_CHANNELS = (2, 32, 32, 32, 2)
TILE_ROWS, TILE_COLS = 14, 12


def cnn_param_shapes():
    shapes = []
    for cin, cout in zip(CNN_CHANNELS[:-1], CNN_CHANNELS[1:]):
        shapes += [(cout, cin, 3, 3), (cout,)]
    return shapes


def cnn_unflatten(params: np.ndarray):
    out, o = [], 0
    for shp in cnn_param_shapes():
        n = int(np.prod(shp))
        out.append(np.asarray(params[o:o + n], dtype=np.float64).reshape(shp))
        o += n
    return out


def conv3x3(a: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """z[n][co][i][j] = b[co] + sum_{ci, di, dj} W[co][ci][di+1][dj+1] a[n][ci][i+di][j+dj]."""
    n, cin, R, C = a.shape
    ap = np.zeros((n, cin, R + 2, C + 2))
    ap[:, :, 1:-1, 1:-1] = a
    z = np.zeros((n, W.shape[0], R, C)) + b[None, :, None, None]
    for di in range(3):
        for dj in range(3):
            z += np.einsum("oc,ncij->noij", W[:, :, di, dj], ap[:, :, di:di + R, dj:dj + C])
    return z


def round_bf16(a: np.ndarray) -> np.ndarray:
    """a rounded to FP32, then to bfloat16 (8-bit significand) to nearest, ties to even."""
    bits = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) >> 16 << 16
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def cnn_forward(params: np.ndarray, x: np.ndarray, operands: str = "fp32"):
    """Output tiles and the post-ReLU activations [a0 = x, a1, a2, a3]. With operands="bf16" the
    weights and every convolution's input are rounded to bfloat16 before the products (the
    tensor-core form; biases, sums and the residual stay exact)."""
    p = cnn_unflatten(params)
    acts = [np.asarray(x, dtype=np.float64)]
    a = acts[0]
    rnd = round_bf16 if operands == "bf16" else (lambda v: v)
    for layer in range(4):
        z = conv3x3(rnd(a), rnd(p[2 * layer]), p[2 * layer + 1])
        if layer < 3:
            a = np.maximum(z, 0.0)
            acts.append(a)
        else:
            return acts[0] + z, acts
    raise AssertionError


def cnn_loss(out: np.ndarray, label: np.ndarray) -> float:
    n = out.shape[0]
    return float(np.sum((out - label) ** 2) / (n * TILE_ROWS * TILE_COLS))


def cnn_backward(params: np.ndarray, acts, out: np.ndarray, label: np.ndarray):
    """(gradient of the loss w.r.t. the flat parameters, gradient w.r.t. the input tiles)."""
    p = cnn_unflatten(params)
    n = out.shape[0]
    dz = 2.0 * (out - label) / (n * TILE_ROWS * TILE_COLS)  # d loss / d out = d loss / d z4
    dx = dz.copy()  # through the residual connection
    grads = [None] * 8
    for layer in (3, 2, 1, 0):
        a = acts[layer]
        W = p[2 * layer]
        _, cin, R, C = a.shape
        ap = np.zeros((n, cin, R + 2, C + 2))
        ap[:, :, 1:-1, 1:-1] = a
        gW = np.zeros_like(W)
        for di in range(3):
            for dj in range(3):
                gW[:, :, di, dj] = np.einsum("noij,ncij->oc", dz, ap[:, :, di:di + R, dj:dj + C])
        grads[2 * layer] = gW
        grads[2 * layer + 1] = dz.sum(axis=(0, 2, 3))
        # d a[ci][i][j] = sum_{co, di, dj} W[co][ci][di][dj] dz[co][i-di+1][j-dj+1]
        dzp = np.zeros((n, W.shape[0], R + 2, C + 2))
        dzp[:, :, 1:-1, 1:-1] = dz
        da = np.zeros_like(a)
        for di in range(3):
            for dj in range(3):
                da += np.einsum("oc,noij->ncij", W[:, :, di, dj],
                                dzp[:, :, 2 - di:2 - di + R, 2 - dj:2 - dj + C])
        if layer > 0:
            dz = da * (a > 0.0)  # through the ReLU that made a
        else:
            dx = dx + da
    return np.concatenate([g.ravel() for g in grads]), dx


def adam_step(params, grad, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (step count t >= 1): returns new (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
