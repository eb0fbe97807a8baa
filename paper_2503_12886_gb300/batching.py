"""Batched training steps as CUDA graphs, and the autotuner for tile shape and staging size.

A batch may mix avatars with different Gaussian counts N and blendshape counts K and frames of
different resolutions: every stage of librgba runs once per batch over all (frame, Gaussian)
pairs or all (frame, tile) items, and the compositing kernels are persistent over one flattened
work list, so an uneven batch is one launch per stage (RGBAvatar Sec. 3.2, Fig. 4c: many
samples per step, one synchronisation).
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import api, synth
from .rasterizer import DeviceBatch, Renderer


class GraphStep:
    """One training step (rgba_step_async + the read of its counters) captured as a CUDA graph.

    replay() runs every kernel of the step and returns (loss, pairs) after the step's single
    host synchronisation. If a replay overflows the pair buffer, the workspace grows and the
    graph is re-captured (then the step is replayed once more)."""

    def __init__(self, renderer: Renderer, db: DeviceBatch, target: torch.Tensor,
                 loss_kind: int = api.RGBA_LOSS_L1, img: torch.Tensor | None = None,
                 headroom: float = 1.1, optimizer=None, fused: bool = False):
        self.r, self.db, self.target, self.loss_kind = renderer, db, target, loss_kind
        self.opt = optimizer  # optim.Adam: its update becomes part of the captured step
        # fused: the update runs inside the backward (rgba_step_adam_async), else after it
        self.fused = fused and optimizer is not None
        self.img = img if img is not None else torch.empty(
            3 * db.total_pix, dtype=torch.float32, device=target.device)
        self.headroom = headroom
        self.stream = torch.cuda.Stream(device=target.device)
        self.host = torch.zeros(24, dtype=torch.uint8).pin_memory()
        out = renderer.step(db, target, loss_kind, self.img)  # sizes the workspace
        self._capture(int(out.pairs * headroom) + 4096)

    def _capture(self, pairs: int):
        r, db = self.r, self.db
        b = db.struct()
        self._b = b
        # the graph owns its workspace: exactly the capacity asked for
        self.ws = torch.empty(api.rgba_workspace_size(b, pairs), dtype=torch.uint8,
                              device=self.target.device)
        self.layout = api.rgba_workspace_layout(b, self.ws.numel())
        with torch.cuda.stream(self.stream):
            api.rgba_step_async(r.ctx, b, self.ws.data_ptr(), self.ws.numel(),
                                self.target.data_ptr(), self.loss_kind, self.img.data_ptr(),
                                self.stream.cuda_stream)
            self.stream.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream):
                if self.fused:
                    self.opt.train_step(self.ws, self.target, self.loss_kind, self.img,
                                        self.stream.cuda_stream, db=self.db)
                else:
                    api.rgba_step_async(r.ctx, b, self.ws.data_ptr(), self.ws.numel(),
                                        self.target.data_ptr(), self.loss_kind, self.img.data_ptr(),
                                        self.stream.cuda_stream)
                    if self.opt is not None:
                        self.opt.step(self.stream.cuda_stream)
                c0 = self.layout.counters
                self.host.copy_(self.ws[c0: c0 + 24], non_blocking=True)
        torch.cuda.synchronize()

    def replay(self) -> tuple[float, int]:
        for _ in range(3):
            with torch.cuda.stream(self.stream):
                self.graph.replay()
            self.stream.synchronize()
            raw = self.host.numpy()
            u = raw[:16].view(np.uint32)
            if not u[1]:
                return float(raw[16:24].view(np.float64)[0]), int(u[0])
            self._capture(int(u[0] * max(self.headroom, 1.1)) + 4096)
        raise api.RgbaError(api.RGBA_ERR_CAPACITY, "graph step kept overflowing")


@dataclass
class TuneResult:
    tile: tuple[int, int]
    smem_batch: int
    ms: float
    table: dict


TILES = ((16, 16), (8, 32))
SMEM_BATCHES = (64, 128, 256)


def workload_signature(batch: synth.Batch) -> str:
    ns = sorted({(m.n, m.k) for m in batch.models})
    res = sorted({(f.width, f.height) for f in batch.frames})
    return json.dumps({"models": ns, "res": res, "frames": len(batch.frames)})


def autotune(renderer: Renderer, batch: synth.Batch, targets, steps: int = 5,
             tiles=TILES, smem_batches=SMEM_BATCHES, cache_path: str | None = None) -> TuneResult:
    """Times the whole training step for every (tile shape, staging size) and keeps the fastest.

    Each candidate builds its own device batch (the tile shape changes the binning), runs one
    sizing step, then `steps` timed steps with CUDA events. Results are cached per workload
    signature in cache_path (JSON) when given."""
    sig = workload_signature(batch)
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if sig in cache:
            e = cache[sig]
            return TuneResult(tuple(e["tile"]), e["smem_batch"], e["ms"], e["table"])
    table = {}
    models = None
    for tile in tiles:
        for sb in smem_batches:
            db = DeviceBatch(batch, f"cuda:{renderer.device}", tile=tile, smem_batch=sb,
                             models=models)
            models = db.models
            tg = db.pack_images(targets)
            img = torch.empty(3 * db.total_pix, dtype=torch.float32, device=tg.device)
            renderer.step(db, tg, api.RGBA_LOSS_L1, img)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(steps):
                renderer.step(db, tg, api.RGBA_LOSS_L1, img)
            e1.record()
            torch.cuda.synchronize()
            table[f"{tile[0]}x{tile[1]}/{sb}"] = e0.elapsed_time(e1) / steps
    best = min(table, key=table.get)
    tw, th = (int(x) for x in best.split("/")[0].split("x"))
    res = TuneResult((tw, th), int(best.split("/")[1]), table[best], table)
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        cache[sig] = {"tile": list(res.tile), "smem_batch": res.smem_batch, "ms": res.ms,
                      "table": table, "when": time.time()}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return res
