"""Adam over every base Gaussian and blendshape of the models in a batch (fused kernel in
librgba). Learning rates follow RGBAvatar Supp. A.3: position 8e-4, opacity 0.25, scale 0.025,
rotation 0.005, colour 0.0125; blendshape rates are the base rates scaled by 0.05 (position),
0.5 (rotation) and 0.5 (colour). The paper blends neither scale nor opacity; when log-scale is
blended its delta uses 0.5. beta1, beta2, eps are the usual defaults (0.9, 0.999, 1e-8): the
paper names the optimizer only."""
from __future__ import annotations

import torch

from . import api
from .rasterizer import DeviceBatch, Renderer, stream_ptr

PAPER_LR = [8e-4] * 3 + [0.005] * 4 + [0.025] * 3 + [0.25] + [0.0125] * 3
PAPER_DELTA_SCALE = [0.05] * 3 + [0.5] * 4 + [0.5] * 3 + [0.0] + [0.5] * 3


def paper_cfg(beta1=0.9, beta2=0.999, eps=1e-8) -> api.RgbaAdamCfg:
    cfg = api.RgbaAdamCfg()
    for c in range(api.RGBA_NCH):
        cfg.lr[c] = PAPER_LR[c]
        cfg.lr_delta[c] = PAPER_LR[c] * PAPER_DELTA_SCALE[c]
    cfg.beta1, cfg.beta2, cfg.eps = beta1, beta2, eps
    return cfg


class Adam:
    """Moment buffers for the models of a DeviceBatch, and the fused update."""

    def __init__(self, renderer: Renderer, db: DeviceBatch, cfg: api.RgbaAdamCfg | None = None):
        self.ctx = renderer.ctx
        self.db = db
        self.cfg = cfg or paper_cfg()
        dev = db.psi.device
        self.m = [(torch.zeros_like(m.g0), torch.zeros_like(m.dg)) for m in db.models]
        self.v = [(torch.zeros_like(m.g0), torch.zeros_like(m.dg)) for m in db.models]
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        st = (api.RgbaAdamState * max(1, len(db.models)))()
        for i in range(len(db.models)):
            st[i] = api.RgbaAdamState(self.m[i][0].data_ptr(), self.v[i][0].data_ptr(),
                                      self.m[i][1].data_ptr(), self.v[i][1].data_ptr())
        self.states = st

    def step(self, stream: int | None = None):
        """One update from the gradients the last backward wrote (device-side step count)."""
        api.rgba_adam(self.ctx, self.db.struct(), self.cfg, self.states, 0,
                      self.step_dev.data_ptr(), stream if stream is not None else stream_ptr())

    def train_step(self, ws: torch.Tensor, target: torch.Tensor, loss_kind: int = api.RGBA_LOSS_L1,
                   img: torch.Tensor | None = None, stream: int | None = None,
                   db: DeviceBatch | None = None):
        """A whole training step with this update fused into the backward
        (rgba_step_adam_async): no host synchronisation; the loss and pair count are in the
        workspace counters. db: another batch over the same models (other frames, weights,
        cameras), else the optimizer's own."""
        b = (db or self.db).struct()
        api.rgba_step_adam_async(self.ctx, b, ws.data_ptr(), ws.numel(), target.data_ptr(),
                                 loss_kind, img.data_ptr() if img is not None else None, self.cfg,
                                 self.states, 0, self.step_dev.data_ptr(),
                                 stream if stream is not None else stream_ptr())
