"""Comparison helpers for CUDA-vs-oracle parity tests (no arithmetic of the method here).

Tolerances (FP32 path, complex64 inputs, FP64 oracle on the same inputs):
  * x_hat: aggregate ||x_gpu - x_ref||_F / ||x_ref||_F <= X_REL per slot batch, over REs that
    neither side flags.
  * SINR: per layer, |s_gpu - s_ref| / s_ref <= SINR_REL. Both sides form e = s2 (A^-1)_kk
    directly (no cancellation in 1 - mu), so the SINR carries the relative error of (A^-1)_kk.
  * LLR: normalised by the oracle's effective noise, |l_gpu - l_ref| * s2eff_ref <= LLR_ABS
    (the difference of squared distances in constellation units).
  * Hard bits sign(l): equal, except where the oracle's unbiased symbol lies within BOUNDARY of a
    PAM decision threshold in constellation units.
  * Flag bit 0 (ill-conditioned Gram matrix): equal RE by RE, except where the oracle's pivot
    ratio lies within a factor FLAG_BAND of the threshold. The FP32 pivots carry an absolute
    error of about n_rx n_layers u32 times the largest pivot (the rounding of the Gram entries,
    each a sum of n_rx products, propagated through the factorisation); at a threshold of 1e-6
    and the test shapes that is of the order of the smallest pivot itself, so a ratio within a
    factor of 8 of the threshold may land on either side.
  * Every comparison states how many REs it compared and fails on an empty set.
"""
import math

import numpy as np

X_REL = 1e-5
SINR_REL = 2e-5
LLR_ABS = 2e-4
BOUNDARY = 1e-4
FLAG_BAND = 8.0
PIVOT_RATIO_MIN = 1e-6


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def boundary_distance(x_t, qm):
    """Distance (constellation units) of each axis value to the nearest PAM threshold."""
    h = qm // 2
    nrm = math.sqrt(2.0 * (4 ** h - 1) / 3.0)
    out = []
    for v in (np.real(x_t), np.imag(x_t)):
        u = v * nrm
        top = 2 ** h - 2
        e = np.clip(2.0 * np.round(u / 2.0), -top, top)  # thresholds at even integers within grid
        out.append(np.abs(u - e) / nrm)
    return np.minimum(out[0], out[1])


def check_flags(tag, gpu_flags, ref_flags, ref_ratio, pivot_min=PIVOT_RATIO_MIN,
                band=FLAG_BAND):
    """Flag bit 0 RE by RE against the oracle (outside the ambiguous band around the threshold).

    Returns the mask of REs that neither side flags (bit 0 or the non-finite bit 2), the set the
    output comparisons run on."""
    gf = np.asarray(gpu_flags).reshape(-1)
    rf = np.asarray(ref_flags).reshape(-1)
    ratio = np.asarray(ref_ratio, dtype=np.float64).reshape(-1)
    assert gf.size == rf.size == ratio.size and gf.size > 0, (gf.size, rf.size, ratio.size)
    g0 = (gf & 1) != 0
    r0 = (rf & 1) != 0
    amb = (ratio > pivot_min / band) & (ratio < pivot_min * band)
    mism = (g0 != r0) & ~amb
    print(tag, f"flags: oracle {int(r0.sum())}, gpu {int(g0.sum())}, ambiguous {int(amb.sum())},"
               f" mismatched {int(mism.sum())} of {gf.size} REs")
    assert not mism.any(), (tag, np.nonzero(mism)[0][:10], ratio[mism][:10])
    return ~g0 & ~r0 & ((gf & 4) == 0)


def compare_res(tag, gpu, ref, qm, s2eff_ref, x_t_ref, mask=None):
    """Compare per-RE outputs; arrays are [n_re, n_layers(, qm)]. Returns a metrics dict whose
    'n' is the number of REs compared and 'n_total' the number offered."""
    xg, xr = gpu["x_hat"], ref["x_hat"]
    if mask is None:
        mask = np.ones(xr.shape[0], dtype=bool)
    mask = np.asarray(mask, dtype=bool).reshape(-1)
    assert mask.size == xr.shape[0], (mask.size, xr.shape)
    m = {"n": int(mask.sum()), "n_total": int(mask.size)}
    m["x_rel"] = rel_fro(xg[mask], xr[mask])
    m["x_rel_re_p999"] = float(np.quantile(
        np.linalg.norm(xg[mask] - xr[mask], axis=-1)
        / np.maximum(np.linalg.norm(xr[mask], axis=-1), 1e-30),
        0.999)) if mask.any() else 0.0
    sg, sr = gpu["sinr"][mask], ref["sinr"][mask]
    m["sinr_rel_max"] = float(np.max(np.abs(sg - sr) / sr)) if mask.any() else 0.0
    if "llr" in gpu:
        lg, lr = gpu["llr"][mask], ref["llr"][mask]
        sc = np.asarray(s2eff_ref)[mask][..., None]
        m["llr_norm_max"] = float(np.max(np.abs(lg - lr) * sc)) if mask.any() else 0.0
        near = boundary_distance(np.asarray(x_t_ref)[mask], qm) < BOUNDARY  # [n, layers]
        hard_g = lg < 0
        hard_r = lr < 0
        diff = (hard_g != hard_r) & ~near[..., None]
        m["hard_mismatch"] = int(diff.sum())
        m["near_boundary"] = int(near.sum())
    print(tag, {k: (f"{v:.3e}" if isinstance(v, float) else v) for k, v in m.items()})
    return m


def assert_parity(m, x_rel=X_REL, sinr_rel=SINR_REL, llr_abs=LLR_ABS, min_frac=1.0):
    """The bars above, over a comparison set that is not empty and holds at least min_frac of
    the REs offered (1.0: every one)."""
    assert m["n"] > 0 and m["n"] >= min_frac * m["n_total"], m
    assert m["x_rel"] <= x_rel, m
    assert m["sinr_rel_max"] <= sinr_rel, m
    if "llr_norm_max" in m:
        assert m["llr_norm_max"] <= llr_abs, m
        assert m["hard_mismatch"] == 0, m
