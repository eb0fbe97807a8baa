"""Differentiable rendering as a torch.autograd.Function over the C ABI.

The forward renders B frames (preprocess, bin/sort, compositing) and saves only the per-pixel
final transmittance and contributor count (plus references to its inputs). The backward
re-runs preprocess and bin/sort from the inputs, then walks the compositing in reverse from
T_final and n_contrib (rgba_render_bwd) down to G0, the blendshapes and the weights
(RGBAvatar Sec. 3.2: the image loss is back-propagated to every Gaussian and basis attribute).
"""
from __future__ import annotations

import torch

from . import api
from .rasterizer import DeviceBatch, DeviceModel, Renderer, stream_ptr


class _Frames:
    """Host description of a batch whose tensors come from autograd (no copies)."""

    def __init__(self, frames, k_stride, tile, smem_batch, verts=None):
        self.frames = [(int(m), int(w), int(h)) for m, w, h in frames]
        self.verts = list(verts) if verts is not None else [None] * len(self.frames)
        self.k_stride = k_stride
        self.tile = tile
        self.smem_batch = smem_batch


def _device_batch(spec: _Frames, psi, fparams, models, grads: bool) -> DeviceBatch:
    db = DeviceBatch.__new__(DeviceBatch)
    db.device = psi.device
    db.models = models
    db.frames = spec.frames
    db.verts = spec.verts
    db.k_stride = spec.k_stride
    db.psi = psi
    db.fparams = fparams
    db.grad_psi = torch.zeros_like(psi) if grads else None
    db.tile = spec.tile
    db.smem_batch = spec.smem_batch
    db.loss_frames = 0
    offs, tot = [], 0
    for _, w, h in db.frames:
        offs.append(tot)
        tot += w * h
    db.pix_offsets, db.total_pix = offs, tot
    rec, rt = [], 0
    for mi, _, _ in db.frames:
        rec.append(rt)
        rt += models[mi].n_pad
    db.rec_offsets, db.total_rec = rec, rt
    db._struct = None
    return db


class RasterizeBlendFn(torch.autograd.Function):
    """img = render(G0_m + sum_k psi_bk dG_m,k ; camera_b) for every frame b.

    Inputs (after the non-tensor ones): psi [B][k_stride], fparams [B][20], then for each model
    g0 [14][n_pad] and dg [k][A][n_pad]. Output: the concatenated planar images [sum 3 H_b W_b].
    Gradients flow to psi, g0 and dg (fparams carries no gradient)."""

    @staticmethod
    def forward(ctx, renderer: Renderer, spec: _Frames, model_meta, psi, fparams, *tensors):
        models = [DeviceModel(n, k, mask, tensors[2 * i].contiguous(), tensors[2 * i + 1].contiguous(),
                              binding=bd)
                  for i, (n, k, mask, bd) in enumerate(model_meta)]
        db = _device_batch(spec, psi.contiguous(), fparams.contiguous(), models, grads=False)
        img, T, n = renderer.forward(db)
        ctx.renderer, ctx.spec, ctx.model_meta = renderer, spec, model_meta
        ctx.save_for_backward(T, n, psi, fparams, *tensors)
        return img

    @staticmethod
    def backward(ctx, dl_dimg):
        T, n, psi, fparams, *tensors = ctx.saved_tensors
        models = []
        for i, (nn, k, mask, bd) in enumerate(ctx.model_meta):
            g0, dg = tensors[2 * i].contiguous(), tensors[2 * i + 1].contiguous()
            models.append(DeviceModel(nn, k, mask, g0, dg, torch.empty_like(g0), torch.empty_like(dg),
                                      binding=bd))
        db = _device_batch(ctx.spec, psi.contiguous(), fparams.contiguous(), models, grads=True)
        r: Renderer = ctx.renderer
        ws = r.ensure_workspace(db)
        b = db.struct()
        s = stream_ptr()
        for _ in range(3):  # recompute the splats and tile lists the forward used
            api.rgba_preprocess(r.ctx, b, ws.data_ptr(), ws.numel(), s)
            api.rgba_bin_sort(r.ctx, b, ws.data_ptr(), ws.numel(), s)
            cnt = r.counters(db)
            if not cnt["overflow"]:
                break
            ws = r.ensure_workspace(db, int(cnt["pairs"] * 1.25) + 4096)
            b = db.struct()
        r.backward(db, dl_dimg.contiguous(), T, n)
        grads = []
        for m in models:
            grads += [m.grad_g0, m.grad_dg]
        return (None, None, None, db.grad_psi, None, *grads)


def rasterize(renderer: Renderer, frames, psi, fparams, models, tile=(16, 16), smem_batch=64,
              bindings=None, verts=None):
    """Differentiable batched render.

    frames: list of (model index, width, height); psi [B][k_stride]; fparams [B][20];
    models: list of (n, k, mask, g0, dg) with g0/dg CUDA float32 tensors (may require grad);
    bindings (optional): per model a rasterizer.DeviceBinding or None (tangent space, Supp.
    "Gaussian Transformation"), with verts: per frame the deformed mesh [V][3] (CUDA float32)
    or None. Returns one [3][H][W] view per frame of the concatenated output."""
    spec = _Frames(frames, psi.shape[1], tile, smem_batch, verts)
    bindings = bindings or [None] * len(models)
    meta = [(n, k, mask, bd) for (n, k, mask, _, _), bd in zip(models, bindings)]
    flat = []
    for _, _, _, g0, dg in models:
        flat += [g0, dg]
    img = RasterizeBlendFn.apply(renderer, spec, meta, psi, fparams, *flat)
    out, o = [], 0
    for _, w, h in spec.frames:
        out.append(img[3 * o: 3 * (o + w * h)].view(3, h, w))
        o += w * h
    return out
