"""Learned channel denoiser: data, training loop and evaluation around the library's CNN kernels.

Every forward, backward and optimiser step runs in libphy.so (phy_cnn_forward,
phy_cnn_train_step); this module only prepares device buffers, draws training slots from the
generator, orders the batches and reads metrics back. The network refines the interpolated LS
channel tile of each (PRB, Rx antenna, layer) entry; the plain LS + interpolation estimate stays
both its fallback (the network starts as the identity: last layer zero) and its judge (channel
MSE and detected BER against the true channel and bits).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

from . import phy
from . import synth as S

CHANNELS = (2, 32, 32, 32, 2)


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights for the ReLU layers, zero biases, zero last layer (identity network)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, (cin, cout) in enumerate(zip(CHANNELS[:-1], CHANNELS[1:])):
        if i < 3:
            w = rng.standard_normal((cout, cin, 3, 3)) * math.sqrt(2.0 / (cin * 9))
        else:
            w = np.zeros((cout, cin, 3, 3))
        parts += [w.ravel(), np.zeros(cout)]
    return np.concatenate(parts).astype(np.float32)  # 19,682 = phy_cnn_param_count()


def train_spec(n_prb: int, snr_db: float, doppler_hz: float, n_rx: int = 32,
               n_layers: int = 8) -> S.SlotSpec:
    """A slot of the learned-estimation workload: 64-QAM, DMRS 2 and 11, 23-tap 300 ns PDP."""
    return S.SlotSpec(n_cells=1, n_prb=n_prb, n_rx=n_rx, n_layers=n_layers, qm=6,
                      dmrs_sym=(2, 11), snr_db=snr_db, n_taps=23, delay_spread_s=300e-9,
                      doppler_hz=doppler_hz)


@dataclasses.dataclass
class SlotTiles:
    """One slot on the device: LS-interpolated input tiles, true-channel label tiles, anchors."""
    spec: S.SlotSpec
    cfg: "phy.SlotConfig"
    slot: S.Slot
    x: "object"        # torch float32 [n][2][14][12]
    label: "object"    # torch float32 [n][2][14][12]
    anchors: "object"  # torch complex64 [cell][dmrs][group][layer][rx]
    Y: "object"
    pilots: "object"
    sigma2: "object"


def _make_slot(args):
    """Process-pool entry: one generated slot (numpy only)."""
    spec, seed = args
    return S.make_slot(spec, seed, keep_h=True)


def slot_tiles(spec: S.SlotSpec, seed: int, dev, slot: Optional[S.Slot] = None) -> SlotTiles:
    import torch
    sl = slot if slot is not None else S.make_slot(spec, seed, keep_h=True)
    cfg = phy.SlotConfig.from_spec(spec)
    Y = torch.from_numpy(sl.Y).to(dev)
    P = torch.from_numpy(sl.pilots).to(dev)
    s2 = torch.from_numpy(sl.sigma2).to(dev)
    G = phy.n_groups(cfg)
    anchors = torch.empty((spec.n_cells, len(spec.dmrs_sym), G, spec.n_layers, spec.n_rx),
                          dtype=torch.complex64, device=dev)
    phy.chest(cfg, Y, P, anchors)
    hshape = (spec.n_cells, spec.n_sym, spec.n_sc, spec.n_rx, spec.n_layers)
    H_est = torch.empty(hshape, dtype=torch.complex64, device=dev)
    phy.interp_channel(cfg, anchors, H_est)
    n = phy.cnn_n_tiles(cfg)
    x = torch.empty((n, 2, 14, 12), dtype=torch.float32, device=dev)
    phy.cnn_tiles(cfg, H_est, x)
    # the generator's channel arrays need not be C-ordered: copy into the [cell][sym][sc][rx][l]
    # layout the kernels index
    H_true = torch.from_numpy(np.ascontiguousarray(np.stack(sl.H), dtype=np.complex64)).to(dev)
    label = torch.empty_like(x)
    phy.cnn_tiles(cfg, H_true, label)
    return SlotTiles(spec, cfg, sl, x, label, anchors, Y, P, s2)


def training_set(n_slots: int, n_prb: int, seed: int, dev, snr_range=(0.0, 30.0),
                 doppler_range=(0.0, 500.0), workers: int = 0):
    """Tiles of n_slots slots with SNR and Doppler drawn uniformly (seeded), concatenated. With
    workers > 0 the slots are generated (numpy) in that many spawned processes, in chunks, and
    tiled on the device as they arrive; the tiles are the same either way."""
    import torch
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n_slots):
        snr, doppler = float(rng.uniform(*snr_range)), float(rng.uniform(*doppler_range))
        specs.append((train_spec(n_prb, snr, doppler), seed * 1000 + i))
    xs, ys = [], []
    if workers > 0:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            for (spec, sd), sl in zip(specs, pool.imap(_make_slot, specs, chunksize=4)):
                st = slot_tiles(spec, sd, dev, slot=sl)
                xs.append(st.x)
                ys.append(st.label)
    else:
        for spec, sd in specs:
            st = slot_tiles(spec, sd, dev)
            xs.append(st.x)
            ys.append(st.label)
    return torch.cat(xs), torch.cat(ys)


class Trainer:
    """Adam on the device through phy_cnn_train_step (with bf16: phy_cnn_train_step_bf16, the
    forward pass on the tensor cores with BF16 operands, FP32 backward and master weights);
    batches are contiguous slices of a shuffled copy of the tile set."""

    def __init__(self, params: np.ndarray, batch: int, dev, lr: float = 1e-3, bf16: bool = False):
        import torch
        self.dev = dev
        self.batch = batch
        self.lr = lr
        self.p = torch.from_numpy(params.copy()).to(dev)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.g = torch.zeros_like(self.p)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.ws = torch.empty(phy.cnn_workspace_size(batch), dtype=torch.uint8, device=dev)
        self.step = 0
        self.bf16 = bf16
        self.err_at = phy.cnn_train_error_offset(batch)

    def epoch(self, x, y, seed: int, max_steps: Optional[int] = None) -> List[float]:
        import torch
        gen = torch.Generator(device="cpu").manual_seed(seed)
        perm = torch.randperm(x.shape[0], generator=gen).to(self.dev)
        xs, ys = x.index_select(0, perm), y.index_select(0, perm)
        losses = []
        nb = x.shape[0] // self.batch
        if max_steps is not None:
            nb = min(nb, max_steps)
        for b in range(nb):
            sl = slice(b * self.batch, (b + 1) * self.batch)
            self.step += 1
            phy.cnn_train_step(self.batch, self.p, self.m, self.v, self.step, self.lr, xs[sl],
                               ys[sl], self.g, None, self.loss, self.ws, bf16=self.bf16)
            if b % 50 == 0 or b == nb - 1:
                losses.append(float(self.loss.item()))
                if self.bf16 and self.error_word() != 0:
                    raise RuntimeError("tensor-core forward pass: a bounded wait ran out")
        return losses

    def error_word(self) -> int:
        import torch
        return int(self.ws[self.err_at:self.err_at + 4].view(torch.int32).item())

    def params(self) -> np.ndarray:
        return self.p.cpu().numpy()


def channel_mse(H_data, H_true_data) -> float:
    return float((H_data - H_true_data).abs().pow(2).mean().item())


def evaluate(params_dev, st: SlotTiles, dev, tensor_cores: bool = False) -> Dict[str, float]:
    """Channel MSE at the data symbols and uncoded BER of LMMSE detection on the LS +
    interpolation channel and on the denoised one (explicit-channel detector, same demapper);
    with tensor_cores also for the network run on the tensor cores with BF16 operands
    (phy_cnn_denoise_bf16, keys mse_cnn_bf16 and ber_cnn_bf16)."""
    import torch
    spec, cfg = st.spec, st.cfg
    dshape = (spec.n_cells, len(spec.data_sym), spec.n_sc, spec.n_rx, spec.n_layers)
    H_ls = torch.empty(dshape, dtype=torch.complex64, device=dev)
    phy.cnn_untile(cfg, st.x, H_ls)
    H_cnn = torch.empty_like(H_ls)
    ws = torch.empty(phy.cnn_denoise_workspace_size(cfg), dtype=torch.uint8, device=dev)
    phy.cnn_denoise(cfg, params_dev, st.anchors, H_cnn, ws)
    H_true = torch.empty_like(H_ls)
    phy.cnn_untile(cfg, st.label, H_true)
    out = {"mse_ls": channel_mse(H_ls, H_true), "mse_cnn": channel_mse(H_cnn, H_true)}
    chans = [("ls", H_ls), ("cnn", H_cnn), ("genie", H_true)]
    if tensor_cores:
        H_tc = torch.empty_like(H_ls)
        phy.cnn_denoise_bf16(cfg, params_dev, st.anchors, H_tc, ws)
        off = phy.cnn_denoise_error_offset(cfg)
        if int(ws[off:off + 4].view(torch.int32).item()) != 0:
            raise RuntimeError("tensor-core denoiser: a bounded wait ran out")
        out["mse_cnn_bf16"] = channel_mse(H_tc, H_true)
        chans.append(("cnn_bf16", H_tc))
    bits = torch.from_numpy(st.slot.bits).to(dev)
    for name, H in chans:
        n_re = spec.n_cells * len(spec.data_sym) * spec.n_sc
        x_hat = torch.empty((n_re, spec.n_layers), dtype=torch.complex64, device=dev)
        sinr = torch.empty((n_re, spec.n_layers), dtype=torch.float32, device=dev)
        flags = torch.empty(n_re, dtype=torch.uint8, device=dev)
        llr = torch.empty((n_re, spec.n_layers, spec.qm), dtype=torch.float32, device=dev)
        phy.mmse_detect(cfg, H, st.Y, st.sigma2, x_hat, sinr, flags)
        phy.llr_demap(cfg, x_hat, sinr, llr)
        hard = (llr < 0).to(torch.uint8).reshape(bits.shape)
        out[f"ber_{name}"] = float((hard != bits).float().mean().item())
    return out
