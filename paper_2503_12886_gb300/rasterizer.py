"""Device-side batches, workspaces and the training/render calls on top of the C ABI.

PyTorch supplies device memory and streams only; all arithmetic happens in librgba.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import api, synth


@dataclass
class DeviceBinding:
    """A model's tangent-space binding on the device (synth.Binding)."""
    faces: torch.Tensor     # int32 [F][3]
    face_uv: torch.Tensor   # float32 [F][6]
    face_of: torch.Tensor   # int32 [n]
    bary: torch.Tensor      # float32 [3][n_pad]
    n_verts: int

    @staticmethod
    def of(b: synth.Binding | None, device) -> "DeviceBinding | None":
        if b is None:
            return None
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        return DeviceBinding(t(b.faces), t(b.face_uv), t(b.face_of), t(b.bary), b.n_verts)


@dataclass
class DeviceModel:
    n: int
    k: int
    mask: int
    g0: torch.Tensor        # [14][n_pad]
    dg: torch.Tensor        # [k][A][n_pad]
    grad_g0: torch.Tensor | None = None
    grad_dg: torch.Tensor | None = None
    binding: DeviceBinding | None = None

    @property
    def n_pad(self) -> int:
        return self.g0.shape[1]

    def abi(self) -> api.RgbaModel:
        b = self.binding
        return api.RgbaModel(self.n, self.n_pad, self.k, self.mask, self.g0.data_ptr(),
                             self.dg.data_ptr(),
                             self.grad_g0.data_ptr() if self.grad_g0 is not None else None,
                             self.grad_dg.data_ptr() if self.grad_dg is not None else None,
                             b.faces.shape[0] if b else 0, b.n_verts if b else 0,
                             b.faces.data_ptr() if b else None, b.face_uv.data_ptr() if b else None,
                             b.face_of.data_ptr() if b else None, b.bary.data_ptr() if b else None)


class DeviceBatch:
    """A synth.Batch resident on one CUDA device, plus the ABI descriptor that points at it."""

    def __init__(self, batch: synth.Batch, device="cuda", tile=(16, 16), smem_batch=64,
                 grads=True, models: list[DeviceModel] | None = None):
        self.device = torch.device(device)
        if models is None:
            models = [DeviceModel(m.n, m.k, m.mask, torch.from_numpy(m.g0).to(self.device),
                                  torch.from_numpy(m.dg).to(self.device),
                                  binding=DeviceBinding.of(m.binding, self.device))
                      for m in batch.models]
        self.models = models
        if grads:
            for m in self.models:
                if m.grad_g0 is None:
                    m.grad_g0 = torch.zeros_like(m.g0)
                    m.grad_dg = torch.zeros_like(m.dg)
        self.frames = [(f.model, f.width, f.height) for f in batch.frames]
        # each frame's deformed mesh (bound models), one device tensor per frame
        self.verts = [None if f.verts is None else
                      torch.from_numpy(np.ascontiguousarray(f.verts, np.float32)).to(self.device)
                      for f in batch.frames]
        self.k_stride = batch.k_stride
        self.psi = torch.from_numpy(np.ascontiguousarray(batch.psi)).to(self.device)
        self.fparams = torch.from_numpy(np.ascontiguousarray(batch.fparams)).to(self.device)
        self.grad_psi = torch.zeros_like(self.psi) if grads else None
        self.tile = tile
        self.smem_batch = smem_batch
        offs, tot = [], 0
        for _, w, h in self.frames:
            offs.append(tot)
            tot += w * h
        self.pix_offsets = offs
        self.total_pix = tot
        rec, rt = [], 0
        for mi, _, _ in self.frames:
            rec.append(rt)
            rt += self.models[mi].n_pad
        self.rec_offsets = rec
        self.total_rec = rt
        # frames the loss is averaged over (0: this batch's own); a rank of a frame-sharded
        # data-parallel step sets the global batch size (sharding.py)
        self.loss_frames = 0
        self._struct = None

    @property
    def n_frames(self) -> int:
        return len(self.frames)

    def struct(self) -> api.RgbaBatch:
        """ABI descriptor; host arrays are kept alive on this object."""
        ms = (api.RgbaModel * max(1, len(self.models)))()
        for i, m in enumerate(self.models):
            ms[i] = m.abi()
        fs = (api.RgbaFrame * max(1, len(self.frames)))()
        for i, (mi, w, h) in enumerate(self.frames):
            v = self.verts[i]
            fs[i] = api.RgbaFrame(mi, w, h, v.data_ptr() if v is not None else None)
        b = api.RgbaBatch()
        b.n_models = len(self.models)
        b.models = C.cast(ms, C.POINTER(api.RgbaModel))
        b.n_frames = len(self.frames)
        b.frames = C.cast(fs, C.POINTER(api.RgbaFrame))
        b.k_stride = self.k_stride
        b.psi = self.psi.data_ptr()
        b.fparams = self.fparams.data_ptr()
        b.grad_psi = self.grad_psi.data_ptr() if self.grad_psi is not None else None
        b.tile_w, b.tile_h = self.tile
        b.smem_batch = self.smem_batch
        b.loss_frames = self.loss_frames
        self._keep = (ms, fs)
        self._struct = b
        return b

    # views into the concatenated per-frame image arrays
    def image_views(self, flat: torch.Tensor) -> list[torch.Tensor]:
        return [flat[3 * o: 3 * (o + w * h)].view(3, h, w)
                for o, (_, w, h) in zip(self.pix_offsets, self.frames)]

    def pix_views(self, flat: torch.Tensor) -> list[torch.Tensor]:
        return [flat[o: o + w * h].view(h, w) for o, (_, w, h) in zip(self.pix_offsets, self.frames)]

    def pack_images(self, imgs) -> torch.Tensor:
        parts = [torch.as_tensor(np.ascontiguousarray(i), dtype=torch.float32).reshape(-1)
                 for i in imgs]
        if not parts:
            return torch.zeros(0, dtype=torch.float32, device=self.device)
        return torch.cat(parts).to(self.device)


def stream_ptr() -> int:
    return torch.cuda.current_stream().cuda_stream


class Renderer:
    """Owns one librgba context and a growable workspace."""

    def __init__(self, device: int = 0):
        self.device = device
        self.ctx = api.rgba_create(device)
        self.ws: torch.Tensor | None = None

    def close(self):
        if self.ctx:
            api.rgba_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ensure_workspace(self, db: DeviceBatch, pair_capacity: int | None = None) -> torch.Tensor:
        if pair_capacity is None:
            pair_capacity = 4 * db.total_rec + 4096
        need = api.rgba_workspace_size(db.struct(), int(pair_capacity))
        if self.ws is None or self.ws.numel() < need:
            self.ws = torch.empty(need, dtype=torch.uint8, device=f"cuda:{self.device}")
        return self.ws

    def layout(self, db: DeviceBatch) -> api.RgbaWsLayout:
        return api.rgba_workspace_layout(db.struct(), self.ws.numel())

    def counters(self, db: DeviceBatch) -> dict:
        lay = self.layout(db)
        raw = self.ws[lay.counters: lay.counters + 24].cpu().numpy()
        u = raw[:16].view(np.uint32)
        return {"pairs": int(u[0]), "overflow": int(u[1]), "n_work": int(u[2]),
                "device_error": int(u[3]), "loss": float(raw[16:24].view(np.float64)[0])}

    def forward(self, db: DeviceBatch, grow: bool = True):
        """preprocess -> bin/sort -> render; returns (img, T_final, n_contrib) flat tensors.
        Reads the counters once (the one host sync of this path) to detect a pair overflow."""
        dev = f"cuda:{self.device}"
        img = torch.empty(3 * db.total_pix, dtype=torch.float32, device=dev)
        T = torch.empty(db.total_pix, dtype=torch.float32, device=dev)
        n = torch.empty(db.total_pix, dtype=torch.int32, device=dev)
        for _ in range(3):
            ws = self.ensure_workspace(db)
            b = db.struct()
            s = stream_ptr()
            api.rgba_preprocess(self.ctx, b, ws.data_ptr(), ws.numel(), s)
            api.rgba_bin_sort(self.ctx, b, ws.data_ptr(), ws.numel(), s)
            api.rgba_render_fwd(self.ctx, b, ws.data_ptr(), ws.numel(), img.data_ptr(),
                                T.data_ptr(), n.data_ptr(), s)
            cnt = self.counters(db) if db.n_frames else {"overflow": 0}
            if not cnt["overflow"]:
                return img, T, n
            if not grow:
                raise api.RgbaError(api.RGBA_ERR_CAPACITY, f"need {cnt['pairs']} pairs")
            self.ensure_workspace(db, int(cnt["pairs"] * 1.25) + 4096)
        raise api.RgbaError(api.RGBA_ERR_CAPACITY, "workspace growth did not converge")

    def color_init(self, db: DeviceBatch, target: torch.Tensor, done: list, delta: float = 0.1):
        """Colour initialisation (Eq. 3) of every model of the batch from the target images;
        done: per model a CUDA uint8 tensor [n] of flags (or None), updated in place. Regrows the
        workspace and retries on a pair overflow. Returns the pair count."""
        ptrs = [d.data_ptr() if d is not None else None for d in done]
        for _ in range(3):
            ws = self.ensure_workspace(db)
            rc, out = api.rgba_color_init(self.ctx, db.struct(), ws.data_ptr(), ws.numel(),
                                          target.data_ptr(), float(delta), ptrs, stream_ptr())
            if rc == api.RGBA_OK:
                return int(out.pairs)
            self.ensure_workspace(db, int(out.pairs_needed * 1.25) + 4096)
        raise api.RgbaError(api.RGBA_ERR_CAPACITY, "workspace growth did not converge")

    def backward(self, db: DeviceBatch, dl_dimg: torch.Tensor, T: torch.Tensor, n: torch.Tensor,
                 grad_blended: torch.Tensor | None = None):
        """grad_blended (optional, float32 [total_rec * 14] on the device): receives the
        per-frame gradient with respect to the blended Gaussians (layout of blend())."""
        b = db.struct()
        api.rgba_render_bwd(self.ctx, b, self.ws.data_ptr(), self.ws.numel(),
                            dl_dimg.data_ptr(), T.data_ptr(), n.data_ptr(),
                            grad_blended.data_ptr() if grad_blended is not None else None,
                            stream_ptr())

    def blend(self, db: DeviceBatch) -> torch.Tensor:
        out = torch.zeros(db.total_rec * 14, dtype=torch.float32, device=f"cuda:{self.device}")
        api.rgba_blend(self.ctx, db.struct(), out.data_ptr(), stream_ptr())
        return out

    def step(self, db: DeviceBatch, target: torch.Tensor, loss_kind: int = api.RGBA_LOSS_L1,
             img: torch.Tensor | None = None) -> api.RgbaStepOut:
        """One training step with a single host sync; grows the workspace on overflow."""
        for _ in range(3):
            ws = self.ensure_workspace(db)
            rc, out = api.rgba_step(self.ctx, db.struct(), ws.data_ptr(), ws.numel(),
                                    target.data_ptr(), loss_kind,
                                    img.data_ptr() if img is not None else None, stream_ptr())
            if rc == api.RGBA_OK:
                return out
            self.ensure_workspace(db, int(out.pairs_needed * 1.25) + 4096)
        raise api.RgbaError(api.RGBA_ERR_CAPACITY, "workspace growth did not converge")
