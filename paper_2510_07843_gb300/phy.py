"""Thin ctypes binding of libphy.so: argument marshalling only.

Tensors are torch CUDA tensors (PyTorch supplies device memory and streams); every step of the
receiver runs in the library's CUDA kernels. The library must be built (build.build()) before
use; loading fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libphy.so")

PHY_OK = 0
PREC = {"fp32": 0, "tf32": 1, "bf16": 2, "fp16": 3}
LLR_FORMAT = {"f32": 0, "f16": 1}
STATUS = {0: "PHY_OK", 1: "PHY_ERR_INVALID_ARG", 2: "PHY_ERR_UNSUPPORTED",
          3: "PHY_ERR_NO_MEMORY", 4: "PHY_ERR_CUDA", 5: "PHY_ERR_TIMEOUT"}


class CSlotCfg(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int32), ("n_prb", ctypes.c_int32),
                ("n_sym", ctypes.c_int32), ("n_rx", ctypes.c_int32),
                ("n_layers", ctypes.c_int32), ("qm", ctypes.c_int32),
                ("n_dmrs", ctypes.c_int32), ("dmrs_sym", ctypes.c_int32 * 2),
                ("occ_len", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("pivot_ratio_min", ctypes.c_float), ("fp64_refactor", ctypes.c_int32),
                ("llr_format", ctypes.c_int32)]


class CJob(ctypes.Structure):
    """phy_job: one job of a batched call (configuration, device buffers and the optional
    device-side noise tracking)."""
    _fields_ = [("cfg", CSlotCfg), ("Y", ctypes.c_void_p), ("pilots", ctypes.c_void_p),
                ("sigma2", ctypes.c_void_p), ("x_hat", ctypes.c_void_p),
                ("sinr", ctypes.c_void_p), ("llr", ctypes.c_void_p), ("flags", ctypes.c_void_p),
                ("noise_state", ctypes.c_void_p), ("noise_alpha", ctypes.c_float),
                ("noise_mode", ctypes.c_int32)]


# Every entry point declared in include/phy.h, with its ctypes signature.
_P = ctypes.c_void_p
_SIGS = {
    "phy_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "phy_debug_set_wait_polls": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64]),
    "phy_fma_probe": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P,
                                     ctypes.POINTER(ctypes.c_double), _P]),
    "phy_n_groups": (ctypes.c_int32, [_P]),
    "phy_n_data_symbols": (ctypes.c_int32, [_P]),
    "phy_workspace_size": (ctypes.c_size_t, [_P]),
    "phy_chest": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "phy_mmse_detect": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "phy_detect_anchors": (ctypes.c_int, [_P] * 9 + [ctypes.c_size_t, _P]),
    "phy_llr_demap": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "phy_slot_run": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "phy_slot_run_host": (ctypes.c_int, [_P] * 14 + [ctypes.c_size_t, _P]),
    "phy_slot_run_noalloc": (ctypes.c_int, [_P] * 9),
    "phy_stage_supported": (ctypes.c_int32, [_P]),
    "phy_detect_stage": (ctypes.c_int, [_P, ctypes.c_int32] + [_P] * 8 + [ctypes.c_size_t, _P]),
    "phy_autotune": (ctypes.c_int, [_P] * 9 + [ctypes.c_size_t, _P, _P]),
    "phy_autotune_clear": (None, []),
    "phy_autotune_set_tiles": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "phy_autotune_tiles": (ctypes.c_int, [_P, _P, _P, _P]),
    "phy_batch_table_bytes": (ctypes.c_size_t, []),
    "phy_batch_workspace_size": (ctypes.c_size_t, [_P, ctypes.c_int32]),
    "phy_batch_post": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_size_t]),
    "phy_batch_launch": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "phy_batch_status": (ctypes.c_int, [_P]),
    "phy_noise_est": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "phy_slot_run_est": (ctypes.c_int, [_P, ctypes.c_int32] + [_P] * 8 + [ctypes.c_size_t, _P]),
    "phy_noise_track": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_float, _P, _P, _P, _P,
                                       ctypes.c_size_t, _P]),
    "phy_slot_run_track": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_float] + [_P] * 8
                           + [ctypes.c_size_t, _P]),
    "phy_bfp_bytes": (ctypes.c_size_t, [_P, ctypes.c_int32]),
    "phy_bfp_decompress": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_float, ctypes.c_int32,
                                          _P, _P]),
    "phy_chest_bfp": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_float, _P, _P, _P]),
    "phy_slot_run_bfp": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_float] + [_P] * 8
                         + [ctypes.c_size_t, _P]),
    "phy_slot_run_bfp_host": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_float] + [_P] * 13
                              + [ctypes.c_size_t, _P]),
    "phy_cnn_param_count": (ctypes.c_int32, []),
    "phy_cnn_workspace_size": (ctypes.c_size_t, [ctypes.c_int32]),
    "phy_cnn_forward": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "phy_cnn_train_step": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, ctypes.c_int32,
                                          ctypes.c_float, _P, _P, _P, _P, _P, _P,
                                          ctypes.c_size_t, _P]),
    "phy_cnn_train_step_bf16": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, ctypes.c_int32,
                                               ctypes.c_float, _P, _P, _P, _P, _P, _P,
                                               ctypes.c_size_t, _P]),
    "phy_cnn_train_error_offset": (ctypes.c_size_t, [ctypes.c_int32]),
    "phy_cnn_n_tiles": (ctypes.c_int32, [_P]),
    "phy_interp_channel": (ctypes.c_int, [_P, _P, _P, _P]),
    "phy_cnn_tiles": (ctypes.c_int, [_P, _P, _P, _P]),
    "phy_cnn_untile": (ctypes.c_int, [_P, _P, _P, _P]),
    "phy_cnn_denoise_workspace_size": (ctypes.c_size_t, [_P]),
    "phy_cnn_denoise": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "phy_cnn_forward_bf16": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, ctypes.c_size_t,
                                            _P]),
    "phy_cnn_denoise_bf16": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "phy_cnn_denoise_error_offset": (ctypes.c_size_t, [_P]),
}

STAGE_GRAM_MF, STAGE_SOLVE = 0, 1

# Bytes of the fixed scratch array behind phy_slot_run_noalloc (PHY_NOALLOC_SCRATCH_BYTES).
NOALLOC_SCRATCH_BYTES = 64 << 20

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libphy.so not built at {path}; "
                           "run paper_2510_07843_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PhyError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} returned {STATUS.get(code, code)}")
        self.code = code


@dataclass
class SlotConfig:
    n_cells: int
    n_prb: int
    n_rx: int
    n_layers: int
    qm: int
    dmrs_sym: Sequence[int] = (2,)
    n_sym: int = 14
    occ_len: int = 0
    precision: str = "fp32"
    pivot_ratio_min: float = 1e-6
    fp64_refactor: bool = False
    llr_format: str = "f32"  # "f16": LLRs as binary16 (saturating at +-65504)

    def c(self) -> CSlotCfg:
        ds = list(self.dmrs_sym) + [0] * (2 - len(self.dmrs_sym))
        return CSlotCfg(self.n_cells, self.n_prb, self.n_sym, self.n_rx, self.n_layers, self.qm,
                        len(self.dmrs_sym), (ctypes.c_int32 * 2)(*ds), self.occ_len,
                        PREC[self.precision], self.pivot_ratio_min, int(self.fp64_refactor),
                        LLR_FORMAT.get(self.llr_format, -1))

    @property
    def n_sc(self) -> int:
        return 12 * self.n_prb

    @property
    def n_dsym(self) -> int:
        return self.n_sym - len(self.dmrs_sym)

    @staticmethod
    def from_spec(spec, **kw) -> "SlotConfig":
        return SlotConfig(n_cells=spec.n_cells, n_prb=spec.n_prb, n_rx=spec.n_rx,
                          n_layers=spec.n_layers, qm=spec.qm, dmrs_sym=tuple(spec.dmrs_sym),
                          n_sym=spec.n_sym, occ_len=spec.occ_len, **kw)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):  # a raw device address
        return t
    if not t.is_contiguous():  # the library indexes dense row-major arrays
        raise ValueError("libphy arguments must be contiguous tensors")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(fn: str, code: int):
    if code != PHY_OK:
        raise PhyError(fn, code)


def n_groups(cfg: SlotConfig) -> int:
    c = cfg.c()
    return load().phy_n_groups(ctypes.byref(c))


def workspace_size(cfg: SlotConfig) -> int:
    c = cfg.c()
    return load().phy_workspace_size(ctypes.byref(c))


def chest(cfg: SlotConfig, Y, pilots, anchors, stream=None):
    c = cfg.c()
    _check("phy_chest", load().phy_chest(ctypes.byref(c), _ptr(Y), _ptr(pilots), _ptr(anchors),
                                         _stream(stream)))


def mmse_detect(cfg: SlotConfig, H, Y, sigma2, x_hat, sinr, flags, stream=None):
    c = cfg.c()
    _check("phy_mmse_detect",
           load().phy_mmse_detect(ctypes.byref(c), _ptr(H), _ptr(Y), _ptr(sigma2), _ptr(x_hat),
                                  _ptr(sinr), _ptr(flags), _stream(stream)))


def detect_anchors(cfg: SlotConfig, anchors, Y, sigma2, x_hat, sinr, llr, flags, workspace,
                   stream=None):
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_detect_anchors",
           load().phy_detect_anchors(ctypes.byref(c), _ptr(anchors), _ptr(Y), _ptr(sigma2),
                                     _ptr(x_hat), _ptr(sinr), _ptr(llr), _ptr(flags),
                                     _ptr(workspace), ws_bytes, _stream(stream)))


def stage_supported(cfg: SlotConfig) -> bool:
    c = cfg.c()
    return bool(load().phy_stage_supported(ctypes.byref(c)))


def detect_stage(cfg: SlotConfig, stage: int, anchors, Y, sigma2, x_hat, sinr, llr, flags,
                 workspace, stream=None):
    """One of the two detection stages (STAGE_GRAM_MF then STAGE_SOLVE) on a shared workspace."""
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_detect_stage",
           load().phy_detect_stage(ctypes.byref(c), stage, _ptr(anchors), _ptr(Y), _ptr(sigma2),
                                   _ptr(x_hat), _ptr(sinr), _ptr(llr), _ptr(flags),
                                   _ptr(workspace), ws_bytes, _stream(stream)))


def llr_demap(cfg: SlotConfig, x_hat, sinr, llr, stream=None):
    c = cfg.c()
    _check("phy_llr_demap", load().phy_llr_demap(ctypes.byref(c), _ptr(x_hat), _ptr(sinr),
                                                 _ptr(llr), _stream(stream)))


def slot_run(cfg: SlotConfig, Y, pilots, sigma2, x_hat, sinr, llr, flags, workspace,
             stream=None):
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_slot_run",
           load().phy_slot_run(ctypes.byref(c), _ptr(Y), _ptr(pilots), _ptr(sigma2), _ptr(x_hat),
                               _ptr(sinr), _ptr(llr), _ptr(flags), _ptr(workspace), ws_bytes,
                               _stream(stream)))


def autotune(cfg: SlotConfig, Y, pilots, sigma2, x_hat, sinr, llr, flags, workspace,
             stream=None) -> int:
    """phy_autotune: times phy_slot_run for each chunk size that fits the workspace and keeps the
    fastest for cfg (process-wide); returns the chosen cells per chunk. Synchronises."""
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    out = ctypes.c_int32(0)
    _check("phy_autotune",
           load().phy_autotune(ctypes.byref(c), _ptr(Y), _ptr(pilots), _ptr(sigma2), _ptr(x_hat),
                               _ptr(sinr), _ptr(llr), _ptr(flags), _ptr(workspace), ws_bytes,
                               _stream(stream), ctypes.byref(out)))
    return int(out.value)


def autotune_clear():
    """phy_autotune_clear: forget every tuned configuration."""
    load().phy_autotune_clear()


def autotune_set_tiles(cfg: SlotConfig, chunk: int = 0, solve_width: int = 0, ring: int = 0):
    """phy_autotune_set_tiles: pin cfg's tile shapes (0: the default)."""
    c = cfg.c()
    _check("phy_autotune_set_tiles",
           load().phy_autotune_set_tiles(ctypes.byref(c), chunk, solve_width, ring))


def autotune_tiles(cfg: SlotConfig) -> dict:
    """phy_autotune_tiles: cfg's tile shapes (chunk, solve_width, ring; 0 = default)."""
    c = cfg.c()
    v = [ctypes.c_int32(0) for _ in range(3)]
    _check("phy_autotune_tiles", load().phy_autotune_tiles(ctypes.byref(c), *map(ctypes.byref, v)))
    return {"chunk": v[0].value, "solve_width": v[1].value, "ring": v[2].value}


PROBE_KIND = {"fp32": 0, "fp32x2": 1, "fp64": 2}  # phy_probe_kind


def fma_probe(kind: str, blocks: int, iters: int, sink, stream=None) -> float:
    """phy_fma_probe: enqueue the FMA-throughput probe; returns the flops the launch performs."""
    fl = ctypes.c_double(0.0)
    _check("phy_fma_probe", load().phy_fma_probe(PROBE_KIND[kind], int(blocks), int(iters),
                                                 _ptr(sink), ctypes.byref(fl), _stream(stream)))
    return float(fl.value)


WAIT_KERNEL = {"segment": 0, "solve": 1}  # phy_wait_kernel


def debug_set_wait_polls(kernel: str, polls: int):
    """phy_debug_set_wait_polls: first-level device wait limit of one detection kernel for the
    calls that follow (polls < 0: the default). A failure-detection test hook."""
    _check("phy_debug_set_wait_polls",
           load().phy_debug_set_wait_polls(WAIT_KERNEL[kernel], int(polls)))


NOISE_MODE = {"freq": 0, "time": 1, "min": 2}  # phy_noise_mode


def noise_est(cfg: SlotConfig, mode: str, anchors, pilots, sigma2_out, workspace, stream=None):
    """phy_noise_est: per-cell noise variance from the DMRS anchor residuals into sigma2_out."""
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_noise_est",
           load().phy_noise_est(ctypes.byref(c), NOISE_MODE[mode], _ptr(anchors), _ptr(pilots),
                                _ptr(sigma2_out), _ptr(workspace), ws_bytes, _stream(stream)))


def slot_run_est(cfg: SlotConfig, mode: str, Y, pilots, sigma2_out, x_hat, sinr, llr, flags,
                 workspace, stream=None):
    """phy_slot_run_est: the receiver with the noise variance estimated into sigma2_out."""
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_slot_run_est",
           load().phy_slot_run_est(ctypes.byref(c), NOISE_MODE[mode], _ptr(Y), _ptr(pilots),
                                   _ptr(sigma2_out), _ptr(x_hat), _ptr(sinr), _ptr(llr),
                                   _ptr(flags), _ptr(workspace), ws_bytes, _stream(stream)))


def bfp_bytes(cfg: SlotConfig, iq_width: int) -> int:
    """phy_bfp_bytes: size of cfg's block-floating-point fronthaul stream."""
    c = cfg.c()
    return load().phy_bfp_bytes(ctypes.byref(c), iq_width)


def bfp_decompress(cfg: SlotConfig, Yc, iq_width: int, scale: float, Y, data_only=False,
                   stream=None):
    """phy_bfp_decompress: the stream Yc (uint8 tensor) decoded into the grid Y."""
    c = cfg.c()
    _check("phy_bfp_decompress",
           load().phy_bfp_decompress(ctypes.byref(c), _ptr(Yc), iq_width, scale,
                                     1 if data_only else 0, _ptr(Y), _stream(stream)))


def chest_bfp(cfg: SlotConfig, Yc, iq_width: int, scale: float, pilots, anchors, stream=None):
    """phy_chest_bfp: LS anchors read straight from the compressed stream."""
    c = cfg.c()
    _check("phy_chest_bfp",
           load().phy_chest_bfp(ctypes.byref(c), _ptr(Yc), iq_width, scale, _ptr(pilots),
                                _ptr(anchors), _stream(stream)))


def slot_run_bfp(cfg: SlotConfig, Yc, iq_width: int, scale: float, Y, pilots, sigma2, x_hat,
                 sinr, llr, flags, workspace, stream=None):
    """phy_slot_run_bfp: the receiver from the compressed stream (Y: the grid buffer it decodes
    into)."""
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_slot_run_bfp",
           load().phy_slot_run_bfp(ctypes.byref(c), _ptr(Yc), iq_width, scale, _ptr(Y),
                                   _ptr(pilots), _ptr(sigma2), _ptr(x_hat), _ptr(sinr), _ptr(llr),
                                   _ptr(flags), _ptr(workspace), ws_bytes, _stream(stream)))


def slot_run_bfp_host(cfg: SlotConfig, Yc_h, iq_width: int, scale: float, pilots_h, sigma2_h,
                      llr_h, flags_h, Yc, Y, pilots, sigma2, x_hat, sinr, llr, flags, workspace,
                      stream=None):
    """phy_slot_run_bfp_host: the compressed stream and pilots from (pinned) host memory in, LLRs
    and flags back to host memory, everything on the stream."""
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_slot_run_bfp_host",
           load().phy_slot_run_bfp_host(ctypes.byref(c), _ptr(Yc_h), iq_width, scale,
                                        _ptr(pilots_h), _ptr(sigma2_h), _ptr(llr_h),
                                        _ptr(flags_h), _ptr(Yc), _ptr(Y), _ptr(pilots),
                                        _ptr(sigma2), _ptr(x_hat), _ptr(sinr), _ptr(llr),
                                        _ptr(flags), _ptr(workspace), ws_bytes, _stream(stream)))


def cnn_param_count() -> int:
    return load().phy_cnn_param_count()


def cnn_workspace_size(n_tiles: int) -> int:
    return load().phy_cnn_workspace_size(n_tiles)


def cnn_forward(n_tiles: int, params, tiles_in, tiles_out, workspace, stream=None):
    """phy_cnn_forward: the denoiser on n tiles [n][2][14][12]."""
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_cnn_forward",
           load().phy_cnn_forward(n_tiles, _ptr(params), _ptr(tiles_in), _ptr(tiles_out),
                                  _ptr(workspace), ws_bytes, _stream(stream)))


def cnn_train_step(n_tiles: int, params, adam_m, adam_v, step: int, lr: float, tiles_in,
                   tiles_label, grad, grad_in=None, loss=None, workspace=None, stream=None,
                   bf16: bool = False):
    """phy_cnn_train_step (or, with bf16, phy_cnn_train_step_bf16: the forward pass on the
    tensor cores): loss, gradients and (step >= 1) one Adam update, on the device."""
    ws_bytes = workspace.numel() * workspace.element_size()
    name = "phy_cnn_train_step_bf16" if bf16 else "phy_cnn_train_step"
    _check(name, getattr(load(), name)(n_tiles, _ptr(params), _ptr(adam_m), _ptr(adam_v), step,
                                       lr, _ptr(tiles_in), _ptr(tiles_label), _ptr(grad),
                                       _ptr(grad_in), _ptr(loss), _ptr(workspace), ws_bytes,
                                       _stream(stream)))


def cnn_train_error_offset(n_tiles: int) -> int:
    """Byte offset of the mixed-precision step's error word in its workspace."""
    return int(load().phy_cnn_train_error_offset(n_tiles))


def cnn_n_tiles(cfg: SlotConfig) -> int:
    c = cfg.c()
    return load().phy_cnn_n_tiles(ctypes.byref(c))


def interp_channel(cfg: SlotConfig, anchors, H, stream=None):
    """phy_interp_channel: interpolated LS channel at every symbol, [cell][sym][sc][rx][layer]."""
    c = cfg.c()
    _check("phy_interp_channel", load().phy_interp_channel(ctypes.byref(c), _ptr(anchors),
                                                           _ptr(H), _stream(stream)))


def cnn_tiles(cfg: SlotConfig, H, tiles, stream=None):
    c = cfg.c()
    _check("phy_cnn_tiles", load().phy_cnn_tiles(ctypes.byref(c), _ptr(H), _ptr(tiles),
                                                 _stream(stream)))


def cnn_untile(cfg: SlotConfig, tiles, H_data, stream=None):
    c = cfg.c()
    _check("phy_cnn_untile", load().phy_cnn_untile(ctypes.byref(c), _ptr(tiles), _ptr(H_data),
                                                   _stream(stream)))


def cnn_denoise_workspace_size(cfg: SlotConfig) -> int:
    c = cfg.c()
    return load().phy_cnn_denoise_workspace_size(ctypes.byref(c))


def cnn_denoise(cfg: SlotConfig, params, anchors, H_data, workspace, stream=None):
    """phy_cnn_denoise: refined channel at the data symbols, [cell][dsym][sc][rx][layer]."""
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_cnn_denoise",
           load().phy_cnn_denoise(ctypes.byref(c), _ptr(params), _ptr(anchors), _ptr(H_data),
                                  _ptr(workspace), ws_bytes, _stream(stream)))


def cnn_forward_bf16(n_tiles: int, params, tiles_in, tiles_out, workspace, stream=None):
    """phy_cnn_forward_bf16: the denoiser on the tensor cores (BF16 operands, FP32 sums);
    workspace word 0 then holds the timed-out CTA count (0 when the outputs are valid)."""
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_cnn_forward_bf16",
           load().phy_cnn_forward_bf16(n_tiles, _ptr(params), _ptr(tiles_in), _ptr(tiles_out),
                                       _ptr(workspace), ws_bytes, _stream(stream)))


def cnn_denoise_bf16(cfg: SlotConfig, params, anchors, H_data, workspace, stream=None):
    """phy_cnn_denoise_bf16: phy_cnn_denoise with the tensor-core forward pass."""
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_cnn_denoise_bf16",
           load().phy_cnn_denoise_bf16(ctypes.byref(c), _ptr(params), _ptr(anchors), _ptr(H_data),
                                       _ptr(workspace), ws_bytes, _stream(stream)))


def cnn_denoise_error_offset(cfg: SlotConfig) -> int:
    c = cfg.c()
    return int(load().phy_cnn_denoise_error_offset(ctypes.byref(c)))


def noise_track(cfg: SlotConfig, mode: str, alpha: float, anchors, pilots, sigma2_state,
                workspace, stream=None):
    """phy_noise_track: blend this slot's noise estimate into the per-cell device state."""
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_noise_track",
           load().phy_noise_track(ctypes.byref(c), NOISE_MODE[mode], alpha, _ptr(anchors),
                                  _ptr(pilots), _ptr(sigma2_state), _ptr(workspace), ws_bytes,
                                  _stream(stream)))


def slot_run_track(cfg: SlotConfig, mode: str, alpha: float, Y, pilots, sigma2_state, x_hat,
                   sinr, llr, flags, workspace, stream=None):
    """phy_slot_run_track: the receiver with the tracked noise state updated and used."""
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_slot_run_track",
           load().phy_slot_run_track(ctypes.byref(c), NOISE_MODE[mode], alpha, _ptr(Y),
                                     _ptr(pilots), _ptr(sigma2_state), _ptr(x_hat), _ptr(sinr),
                                     _ptr(llr), _ptr(flags), _ptr(workspace), ws_bytes,
                                     _stream(stream)))


def slot_run_noalloc(cfg: SlotConfig, Y, pilots, sigma2, x_hat, sinr, llr, flags, stream=None):
    """phy_slot_run without a workspace argument, for callers that may not allocate device
    memory: the library keeps its scratch in a fixed device array (see include/phy.h)."""
    c = cfg.c()
    _check("phy_slot_run_noalloc",
           load().phy_slot_run_noalloc(ctypes.byref(c), _ptr(Y), _ptr(pilots), _ptr(sigma2),
                                       _ptr(x_hat), _ptr(sinr), _ptr(llr), _ptr(flags),
                                       _stream(stream)))


def slot_run_host(cfg: SlotConfig, Y_h, pilots_h, sigma2_h, llr_h, flags_h, Y, pilots, sigma2,
                  x_hat, sinr, llr, flags, workspace, stream=None):
    c = cfg.c()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("phy_slot_run_host",
           load().phy_slot_run_host(ctypes.byref(c), _ptr(Y_h), _ptr(pilots_h), _ptr(sigma2_h),
                                    _ptr(llr_h), _ptr(flags_h), _ptr(Y), _ptr(pilots),
                                    _ptr(sigma2), _ptr(x_hat), _ptr(sinr), _ptr(llr),
                                    _ptr(flags), _ptr(workspace), ws_bytes, _stream(stream)))


class SlotBuffers:
    """Device buffers for one phy_slot_run call (torch tensors, caller-owned)."""

    def __init__(self, cfg: SlotConfig, device="cuda", with_inputs=True):
        import torch
        C, K, nl, nds = cfg.n_cells, cfg.n_sc, cfg.n_layers, cfg.n_dsym
        f32, c64 = torch.float32, torch.complex64
        if with_inputs:
            self.Y = torch.empty((C, cfg.n_sym, cfg.n_rx, K), dtype=c64, device=device)
            self.pilots = torch.empty((C, len(cfg.dmrs_sym), nl, K), dtype=c64, device=device)
            self.sigma2 = torch.empty((C,), dtype=f32, device=device)
        self.x_hat = torch.empty((C, nds, K, nl), dtype=c64, device=device)
        self.sinr = torch.empty((C, nds, K, nl), dtype=f32, device=device)
        self.llr = torch.empty((C, nds, K, nl, cfg.qm),
                               dtype=torch.float16 if cfg.llr_format == "f16" else f32,
                               device=device)
        self.flags = torch.empty((C, nds, K), dtype=torch.uint8, device=device)
        self.anchors = torch.empty((C, len(cfg.dmrs_sym), n_groups(cfg), nl, cfg.n_rx),
                                   dtype=c64, device=device)
        ws = workspace_size(cfg)
        if ws == 0:
            raise PhyError("phy_workspace_size", 1)
        self.workspace = torch.empty((ws,), dtype=torch.uint8, device=device)


# ---------------------------------------------------------------------------------------------
# batched receiver (phy_batch_*)
# ---------------------------------------------------------------------------------------------

BATCH_MAX_JOBS = 64


def _jobs_array(jobs):
    """jobs: sequence of (SlotConfig, Y, pilots, sigma2, x_hat, sinr, llr, flags) tuples, each
    optionally followed by (noise_state, noise_alpha, noise_mode) for device-side noise
    tracking (mode a NOISE_MODE key or code)."""
    arr = (CJob * len(jobs))()
    for i, j in enumerate(jobs):
        cfg, Y, P, s2, x, sn, l, f = j[:8]
        st, alpha, mode = (j[8], j[9], j[10]) if len(j) >= 11 else (None, 0.0, "min")
        arr[i] = CJob(cfg.c(), _ptr(Y), _ptr(P), _ptr(s2), _ptr(x), _ptr(sn), _ptr(l), _ptr(f),
                      _ptr(st), float(alpha), NOISE_MODE.get(mode, mode))
    return arr


# Raw job records for callers that fill them without ctypes objects (a serving loop's hot path):
# the configuration block, then the seven buffer addresses as 64-bit words.
JOB_BYTES = ctypes.sizeof(CJob)
JOB_ADDR_OFFSET = CJob.Y.offset
assert JOB_ADDR_OFFSET == ctypes.sizeof(CSlotCfg) and CJob.noise_state.offset == JOB_ADDR_OFFSET + 56
assert JOB_BYTES == JOB_ADDR_OFFSET + 8 * 8 + 8


def batch_post_records(records, n_jobs: int, table_host: int, workspace: int,
                       workspace_bytes: int) -> int:
    """phy_batch_post on `n_jobs` raw phy_job records (a ctypes char array of JOB_BYTES each)
    and raw addresses; returns the status code."""
    return int(load().phy_batch_post(records, int(n_jobs), table_host, workspace,
                                     workspace_bytes))


def batch_table_bytes() -> int:
    return int(load().phy_batch_table_bytes())


def batch_workspace_size(jobs) -> int:
    """phy_batch_workspace_size for jobs given as (cfg, ...) tuples (only cfg is read)."""
    arr = (CJob * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = CJob(j[0].c(), None, None, None, None, None, None, None)
    return int(load().phy_batch_workspace_size(arr, len(jobs)))


def batch_post(jobs, table_host, workspace):
    """phy_batch_post: lays out the batch in `workspace` and rings the doorbell of the pinned
    host table (a uint8 tensor of batch_table_bytes())."""
    arr = _jobs_array(jobs)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("phy_batch_post", load().phy_batch_post(arr, len(jobs), _ptr(table_host),
                                                   _ptr(workspace), ws_bytes))


def batch_launch(table_host, table_dev, poll_limit: int = -1, stream=None):
    """phy_batch_launch: gate (bounded wait for the doorbell) and stage kernels on `stream`."""
    _check("phy_batch_launch", load().phy_batch_launch(_ptr(table_host), _ptr(table_dev),
                                                       int(poll_limit), _stream(stream)))


def batch_status(table_host) -> int:
    """phy_batch_status as a status code (0 OK, 5 timed out, 1 not finished or not launched)."""
    return int(load().phy_batch_status(_ptr(table_host)))
