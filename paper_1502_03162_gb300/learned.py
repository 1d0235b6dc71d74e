"""Learned reflection filters and moving sources (Python layer over the C ABI).

The paper fits one non-negative reflection filter per measured direction (Sec. III,
Algorithm 1).  ``FilterNet`` trains the direction -> filter network of the C ABI
(hrir_mlp_forward / hrir_mlp_backward / hrir_mlp_adam, all on the GPU) on such filters, and
turns its outputs into per-segment tap tables (hrir_topk_pack) for ``hrir_render_moving``,
so that sources moving between the measured directions get filters too.  Every step of the
arithmetic runs in the library's kernels; this module only sequences the calls and draws
the initial weights.
"""
from __future__ import annotations

import math

import numpy as np

from . import hrir

HIDDEN = 256
N_IN = 5


def layer_sizes(refl_len: int):
    return [N_IN, HIDDEN, HIDDEN, HIDDEN, refl_len]


def init_params(refl_len: int, seed: int, target_mean: float) -> np.ndarray:
    """Initial weights: every layer U(-1/sqrt(fan_in), 1/sqrt(fan_in)) (weights and biases),
    the output layer's weights scaled by 0.1 and its biases set to softplus^-1 of the mean
    target tap, so that training starts near the mean filter instead of far above it."""
    rng = np.random.default_rng(seed)
    sizes = layer_sizes(refl_len)
    parts = []
    for i in range(len(sizes) - 1):
        fan_in, fan_out = sizes[i], sizes[i + 1]
        bound = 1.0 / math.sqrt(fan_in)
        W = rng.uniform(-bound, bound, (fan_out, fan_in))
        b = rng.uniform(-bound, bound, fan_out)
        if i == len(sizes) - 2:
            W *= 0.1
            m = max(float(target_mean), 1e-12)
            b[:] = math.log(math.expm1(m))
        parts += [W.ravel(), b]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == hrir.hrir_mlp_param_count(refl_len)
    return p


def direction_rows(az, el, ears=(0, 1)) -> np.ndarray:
    """Network input rows {az, el, ear sign}: for every direction, one row per ear (left
    -1, right +1), ordered (direction, ear).  float32 [n * len(ears)][3]."""
    az = np.asarray(az, dtype=np.float64).ravel()
    el = np.asarray(el, dtype=np.float64).ravel()
    rows = np.zeros((az.size, len(ears), 3), np.float32)
    for j, e in enumerate(ears):
        rows[:, j, 0] = az
        rows[:, j, 1] = el
        rows[:, j, 2] = 2.0 * e - 1.0
    return rows.reshape(-1, 3)


class FilterNet:
    """The direction -> reflection-filter network on one device (parameters, Adam moments)."""

    def __init__(self, renderer: "hrir.Renderer", refl_len: int = 200, seed: int = 0):
        import torch
        self.r = renderer
        self.refl_len = refl_len
        self.seed = seed
        self.n_params = hrir.hrir_mlp_param_count(refl_len)
        self.params = torch.zeros(self.n_params, dtype=torch.float32, device="cuda")
        self.step_count = 0

    def set_params(self, p) -> None:
        import torch
        self.params = torch.as_tensor(np.asarray(p, np.float32)).cuda().contiguous()

    def fit(self, rows, targets, steps: int, lr: float = 1e-3, init: bool = True,
            log_every: int = 0):
        """Full-batch Adam on L = 1/(2B) sum ||g - T||^2 with a cosine learning-rate schedule
        (lr_t = lr (1 + cos(pi t / steps)) / 2).  rows [B][3], targets [B][Lg] (numpy or
        CUDA tensors).  Returns the loss trace (one value per step, read back at the end)."""
        import torch
        rows = torch.as_tensor(np.asarray(rows, np.float32)).cuda().contiguous() \
            if not torch.is_tensor(rows) else rows.cuda().float().contiguous()
        tg = torch.as_tensor(np.asarray(targets, np.float32)).cuda().contiguous() \
            if not torch.is_tensor(targets) else targets.cuda().float().contiguous()
        B = rows.shape[0]
        if init:
            self.set_params(init_params(self.refl_len, self.seed, float(tg.mean())))
            self.step_count = 0
        m = torch.zeros_like(self.params)
        v = torch.zeros_like(self.params)
        acts = torch.empty((B, hrir.hrir_mlp_act_stride(self.refl_len)), dtype=torch.float32,
                           device="cuda")
        out = torch.empty((B, self.refl_len), dtype=torch.float32, device="cuda")
        grads = torch.empty_like(self.params)
        losses = torch.empty(steps, dtype=torch.float32, device="cuda")
        for t in range(1, steps + 1):
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * (t - 1) / steps))
            hrir.hrir_mlp_forward(self.r.ctx, rows, self.params, self.refl_len, out=out, acts=acts)
            hrir.hrir_mlp_backward(self.r.ctx, rows, self.params, acts, out, tg, self.refl_len,
                                   grads=grads, loss=losses[t - 1:t])
            hrir.hrir_mlp_adam(self.r.ctx, self.params, grads, m, v, t, lr_t)
        self.step_count += steps
        return losses.cpu().numpy()

    def filters(self, rows, out=None, precision: str = "fp32"):
        """g [n][Lg] (CUDA) for input rows [n][3]; precision "fp32" (the training kernels) or
        "bf16" (tensor-core inference)."""
        import torch
        rows = rows if torch.is_tensor(rows) else torch.as_tensor(np.asarray(rows, np.float32))
        rows = rows.cuda().float().contiguous()
        if precision == "bf16":
            return hrir.hrir_mlp_forward_bf16(self.r.ctx, rows, self.params, self.refl_len, out=out)
        return hrir.hrir_mlp_forward(self.r.ctx, rows, self.params, self.refl_len, out=out)

    def tap_tables(self, az, el, k: int, precision: str = "bf16"):
        """Per-(source, segment) tap tables for hrir_render_moving from directions az, el
        [S][n_seg] (radians): network filters for both ears, then top-k.  Returns CUDA
        (idx [S][n_seg][2][k], w, nnz [S][n_seg][2])."""
        import torch
        az = np.asarray(az)
        S, n_seg = az.shape
        rows = torch.as_tensor(direction_rows(az, el)).cuda()
        g = self.filters(rows, precision=precision).view(S, n_seg, 2, self.refl_len)
        return self.r.topk_pack(g, k)


def nearest_grid_tables(grid_az, grid_el, tap_idx, tap_w, tap_nnz, az, el):
    """The method without the network: each (source, segment) direction takes the tap table
    of the nearest grid direction (largest cosine between unit vectors).  Host numpy in/out:
    tables [n_dirs][2][k] -> [S][n_seg][2][k]."""
    def unit(a, e):
        a, e = np.asarray(a, np.float64), np.asarray(e, np.float64)
        return np.stack([np.cos(e) * np.cos(a), np.cos(e) * np.sin(a), np.sin(e)], -1)
    q = unit(az, el).reshape(-1, 3)
    g = unit(grid_az, grid_el)
    nn = np.argmax(q @ g.T, axis=1).reshape(np.asarray(az).shape)
    return tap_idx[nn], tap_w[nn], tap_nnz[nn], nn
