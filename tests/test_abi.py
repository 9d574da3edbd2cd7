"""The C ABI library loads and exports every symbol include/phy.h declares; host-side validation
answers without touching a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT
from paper_2510_07843_gb300 import build, phy


@pytest.fixture(scope="module")
def lib():
    build.build()
    return phy.load()


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(phy_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "phy_slot_run" in names and "phy_chest" in names
    for n in names:
        assert hasattr(lib, n), n
    # and the binding knows every one of them
    assert set(names) <= set(phy._SIGS), set(names) - set(phy._SIGS)


def _cfg(**kw):
    base = dict(n_cells=8, n_prb=273, n_rx=64, n_layers=16, qm=8, dmrs_sym=(2, 11))
    base.update(kw)
    return phy.SlotConfig(**base)


def test_geometry_queries(lib):
    c = _cfg().c()
    assert lib.phy_n_groups(ctypes.byref(c)) == 205
    assert lib.phy_n_data_symbols(ctypes.byref(c)) == 12
    assert lib.phy_workspace_size(ctypes.byref(c)) >= 8 * 2 * 205 * 16 * 64 * 8
    c1 = _cfg(n_cells=1, n_prb=51, n_rx=4, n_layers=2, qm=4, dmrs_sym=(2,)).c()
    assert lib.phy_n_groups(ctypes.byref(c1)) == 306  # L = 1: one group per comb subcarrier
    assert lib.phy_n_data_symbols(ctypes.byref(c1)) == 13


@pytest.mark.parametrize("bad", [
    dict(n_layers=17), dict(n_layers=65, n_rx=64), dict(n_rx=65), dict(qm=3), dict(n_prb=0),
    dict(n_prb=276), dict(dmrs_sym=(11, 2)), dict(dmrs_sym=(2, 14)), dict(occ_len=3),
    dict(occ_len=4), dict(n_layers=16, n_prb=1), dict(n_cells=0), dict(n_layers=8, n_rx=4),
    dict(precision="fp32", pivot_ratio_min=-1.0), dict(llr_format="f8")])
def test_invalid_configs_rejected(lib, bad):
    cfg = _cfg(**bad)
    c = cfg.c()
    assert lib.phy_workspace_size(ctypes.byref(c)) == 0
    assert lib.phy_n_groups(ctypes.byref(c)) == -1
    # validation happens before any CUDA call: null pointers are never dereferenced
    rc = lib.phy_slot_run(ctypes.byref(c), None, None, None, None, None, None, None, None, 0, None)
    assert rc == 1


def test_null_and_small_workspace_rejected(lib):
    c = _cfg().c()
    fake = ctypes.c_void_p(256)  # never dereferenced: the call fails validation first
    rc = lib.phy_slot_run(ctypes.byref(c), fake, fake, fake, None, None, None, None, None, 0, None)
    assert rc == 1  # flags and workspace are required
    rc = lib.phy_slot_run(ctypes.byref(c), fake, fake, fake, None, None, None, fake, fake, 16,
                          None)
    assert rc == 3  # workspace too small
    assert lib.phy_chest(None, fake, fake, fake, None) == 1
    assert lib.phy_status_str(3) == b"workspace too small"


def test_autotune_validates_before_any_cuda_call(lib):
    bad = _cfg(qm=3).c()
    fake = ctypes.c_void_p(256)  # never dereferenced: the call fails validation first
    out = ctypes.c_int32(-7)
    rc = lib.phy_autotune(ctypes.byref(bad), fake, fake, fake, None, None, None, fake, fake, 0,
                          None, ctypes.byref(out))
    assert rc == 1 and out.value == -7
    c = _cfg().c()
    rc = lib.phy_autotune(ctypes.byref(c), fake, fake, fake, None, None, None, fake, fake, 16,
                          None, ctypes.byref(out))
    assert rc == 3 and out.value == -7  # workspace too small, nothing tuned
    lib.phy_autotune_clear()


def test_tensor_core_precision_needs_even_antenna_count(lib):
    c = _cfg(n_cells=1, n_prb=4, n_rx=5, n_layers=2, qm=4, precision="fp16").c()
    assert lib.phy_workspace_size(ctypes.byref(c)) > 0  # a valid shape ...
    ws = lib.phy_workspace_size(ctypes.byref(c))
    fake = ctypes.c_void_p(256)
    rc = lib.phy_slot_run(ctypes.byref(c), fake, fake, fake, None, None, None, fake, fake, ws,
                          None)
    assert rc == 2  # ... that the TMA-fed tensor-core kernel does not support


def test_noise_estimate_validates_before_any_cuda_call(lib):
    fake = ctypes.c_void_p(256)  # never dereferenced: the calls fail validation first
    c = _cfg().c()
    ws = lib.phy_workspace_size(ctypes.byref(c))
    for mode in (-1, 3):  # unknown modes
        assert lib.phy_noise_est(ctypes.byref(c), mode, fake, fake, fake, fake, ws, None) == 1
        assert lib.phy_slot_run_est(ctypes.byref(c), mode, fake, fake, fake, None, None, None,
                                    fake, fake, ws, None) == 1
    one = _cfg(dmrs_sym=(2,)).c()  # the time residual needs two DMRS symbols
    ws1 = lib.phy_workspace_size(ctypes.byref(one))
    assert lib.phy_noise_est(ctypes.byref(one), phy.NOISE_MODE["time"], fake, fake, fake, fake,
                             ws1, None) == 1
    assert lib.phy_noise_est(ctypes.byref(c), 2, None, fake, fake, fake, ws, None) == 1
    assert lib.phy_noise_est(ctypes.byref(c), 2, fake, fake, None, fake, ws, None) == 1
    assert lib.phy_noise_est(ctypes.byref(c), 2, fake, fake, fake, fake, 16, None) == 3
    assert lib.phy_slot_run_est(ctypes.byref(c), 2, fake, fake, fake, None, None, None, fake,
                                fake, 16, None) == 3
    # the estimate's partial sums make the workspace a little larger than anchors + scratch
    assert ws > 8 * 2 * 205 * 16 * 64 * 8


def test_noalloc_scratch_still_holds_the_massive_batch(lib):
    """The fixed scratch of phy_slot_run_noalloc covers 8 cells of 273 PRB at 64x16 with the
    smallest chunk (the call shrinks chunks to fit)."""
    c = _cfg().c()
    one_cell = _cfg(n_cells=1).c()
    per_cell = lib.phy_workspace_size(ctypes.byref(one_cell))
    assert per_cell > 0
    assert lib.phy_workspace_size(ctypes.byref(c)) > 0
    # anchors and partial sums of 8 cells plus one cell's detection scratch
    need = 8 * (2 * 205 * 16 * 64 * 8) + per_cell
    assert need < 64 << 20


def test_bfp_entry_points_validate_before_any_cuda_call(lib):
    fake = ctypes.c_void_p(256)  # never dereferenced: the calls fail validation first
    c = _cfg().c()
    assert lib.phy_bfp_bytes(ctypes.byref(c), 9) == 8 * 14 * 64 * 273 * 28
    assert lib.phy_bfp_bytes(ctypes.byref(c), 16) == 8 * 14 * 64 * 273 * 49
    assert lib.phy_bfp_bytes(ctypes.byref(c), 0) == 0
    assert lib.phy_bfp_bytes(ctypes.byref(c), 17) == 0
    for w, scale in ((0, 1.0), (17, 1.0), (9, 0.0), (9, -1.0), (9, float("nan")),
                     (9, float("inf"))):
        assert lib.phy_bfp_decompress(ctypes.byref(c), fake, w, scale, 0, fake, None) == 1
        assert lib.phy_chest_bfp(ctypes.byref(c), fake, w, scale, fake, fake, None) == 1
    odd = ctypes.c_void_p(257)  # the stream must be 4-byte aligned, the grid 16-byte aligned
    assert lib.phy_bfp_decompress(ctypes.byref(c), odd, 9, 1.0, 0, fake, None) == 1
    assert lib.phy_bfp_decompress(ctypes.byref(c), fake, 9, 1.0, 0, ctypes.c_void_p(264),
                                  None) == 1
    ws = lib.phy_workspace_size(ctypes.byref(c))
    assert lib.phy_slot_run_bfp(ctypes.byref(c), fake, 9, 1.0, fake, fake, fake, None, None,
                                None, fake, fake, 16, None) == 3
    assert lib.phy_slot_run_bfp(ctypes.byref(c), fake, 9, 1.0, None, fake, fake, None, None,
                                None, fake, fake, ws, None) == 1


def test_cnn_entry_points_validate_before_any_cuda_call(lib):
    fake = ctypes.c_void_p(256)  # never dereferenced: the calls fail validation first
    assert lib.phy_cnn_param_count() == 19682
    assert lib.phy_cnn_workspace_size(0) == 0
    ws = lib.phy_cnn_workspace_size(64)
    assert ws >= 64 * 7 * 32 * 168 * 4
    assert lib.phy_cnn_forward(0, fake, fake, fake, fake, ws, None) == 1
    assert lib.phy_cnn_forward(64, fake, fake, fake, fake, ws - 4, None) == 3
    assert lib.phy_cnn_train_step(64, fake, None, None, 1, 1e-3, fake, fake, fake, None, None,
                                  fake, ws, None) == 1  # an update needs the Adam moments
    assert lib.phy_cnn_train_step(64, fake, fake, fake, 1, float("nan"), fake, fake, fake,
                                  None, None, fake, ws, None) == 1
    c = _cfg(n_cells=1, n_rx=32, n_layers=8, qm=6).c()
    assert lib.phy_cnn_n_tiles(ctypes.byref(c)) == 273 * 32 * 8
    assert lib.phy_cnn_denoise_workspace_size(ctypes.byref(c)) > 0
    short = _cfg(n_cells=1, n_sym=12, n_rx=32, n_layers=8, qm=6).c()  # tiles need 14 symbols
    assert lib.phy_cnn_n_tiles(ctypes.byref(short)) == -1
    assert lib.phy_cnn_tiles(ctypes.byref(short), fake, fake, None) == 2
    assert lib.phy_cnn_denoise(ctypes.byref(c), fake, fake, fake, fake, 16, None) == 3


def test_noise_tracking_validates_alpha(lib):
    fake = ctypes.c_void_p(256)
    c = _cfg().c()
    ws = lib.phy_workspace_size(ctypes.byref(c))
    for alpha in (0.0, -0.5, 1.5, float("nan")):
        assert lib.phy_noise_track(ctypes.byref(c), 2, alpha, fake, fake, fake, fake, ws,
                                   None) == 1
        assert lib.phy_slot_run_track(ctypes.byref(c), 2, alpha, fake, fake, fake, None, None,
                                      None, fake, fake, ws, None) == 1
    assert lib.phy_noise_track(ctypes.byref(c), 2, 0.5, fake, fake, fake, fake, 16, None) == 3


def test_wait_poll_hook_validates_its_kernel(lib):
    """phy_debug_set_wait_polls: known kernels accept any limit (and -1 restores the default);
    an unknown kernel is rejected. No GPU work."""
    assert lib.phy_debug_set_wait_polls(0, 5) == 0
    assert lib.phy_debug_set_wait_polls(1, 7) == 0
    assert lib.phy_debug_set_wait_polls(0, -1) == 0
    assert lib.phy_debug_set_wait_polls(1, -1) == 0
    assert lib.phy_debug_set_wait_polls(2, 0) == 1
    assert lib.phy_debug_set_wait_polls(-1, 0) == 1


def test_fma_probe_validates_its_arguments(lib):
    """phy_fma_probe rejects an unknown kind, empty grids or loops and a NULL sink before it
    launches anything (no GPU work here)."""
    sink = ctypes.c_void_p(256)  # never reached: every call below is rejected first
    fl = ctypes.c_double(0.0)
    assert lib.phy_fma_probe(3, 1, 1, sink, ctypes.byref(fl), None) == 1
    assert lib.phy_fma_probe(0, 0, 1, sink, ctypes.byref(fl), None) == 1
    assert lib.phy_fma_probe(0, 1, 0, sink, ctypes.byref(fl), None) == 1
    assert lib.phy_fma_probe(0, 1, 1, None, ctypes.byref(fl), None) == 1
