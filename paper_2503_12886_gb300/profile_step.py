"""Runs eager training steps of a named workload, for profilers (ncu) and quick timing.

    python -m paper_2503_12886_gb300.profile_step [--workload batched|single|uneven|tangent]
        [--steps N] [--tile 16x16|8x32] [--smem-batch 64|128|256] [--train T]
        [--adam none|separate|fused]

With --train T the avatar first fits images of its reference avatar (synth.reference_avatar)
for T training steps with Adam, reaching the state a training benchmark times; the targets are
then those images (else seeded U[0,1] images). One sizing step (grows the workspace to the pair
count), then N rgba_step calls, each one launch sequence of the whole hot path plus its single
host synchronisation. With --adam separate each profiled step is followed by the Adam update
(rgba_adam, timed as "adam"); with --adam fused the profiled steps are rgba_step_adam_async (the
update runs inside the gauss_bwd stage). Prints per-stage device times of the last step (CUDA
events) as one JSON line. The profiled steps run inside the NVTX range "profiled".
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import api, synth
from .optim import Adam
from .rasterizer import DeviceBatch, Renderer


def make(name: str):
    if name == "batched":
        return synth.workload_batched()
    if name == "single":
        return synth.workload_single()
    if name == "uneven":
        return synth.workload_uneven()
    if name == "tangent":
        return synth.workload_tangent()
    raise ValueError(name)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="batched")
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--tile", default="16x16")
    p.add_argument("--smem-batch", type=int, default=64)
    p.add_argument("--train", type=int, default=0)
    p.add_argument("--adam", default="none", choices=("none", "separate", "fused"))
    p.add_argument("--stats", action="store_true",
                   help="after the profiled steps, one more step with the compositing statistics "
                        "counted (profiling mode 2), printed with the stage times")
    a = p.parse_args()
    tw, th = (int(x) for x in a.tile.split("x"))
    batch = make(a.workload)
    r = Renderer(0)
    db = DeviceBatch(batch, "cuda:0", tile=(tw, th), smem_batch=a.smem_batch)
    opt = Adam(r, db)
    if a.train:
        refs = [synth.reference_avatar(m, 3999 + j) for j, m in enumerate(batch.models)]
        rb = synth.Batch(refs, batch.frames, batch.psi, batch.fparams, batch.k_stride)
        tg, _, _ = r.forward(DeviceBatch(rb, "cuda:0", tile=(tw, th), grads=False))
        tg = tg.clone()
        for _ in range(a.train):
            r.step(db, tg, api.RGBA_LOSS_L1)
            opt.step()
    else:
        tg = db.pack_images(synth.make_targets(batch, 5))
    img = torch.empty(3 * db.total_pix, dtype=torch.float32, device="cuda:0")
    out = r.step(db, tg, api.RGBA_LOSS_L1, img)
    wall = []
    ws = r.ensure_workspace(db, int(out.pairs * 1.3) + 4096)
    adam_ms = None
    api.rgba_profile_enable(r.ctx, True)
    torch.cuda.nvtx.range_push("profiled")  # ncu --nvtx --nvtx-include profiled/ selects these steps
    for _ in range(a.steps):
        t0 = time.perf_counter()
        if a.adam == "fused":
            opt.train_step(ws, tg, api.RGBA_LOSS_L1, img)
            torch.cuda.synchronize()
        else:
            out = r.step(db, tg, api.RGBA_LOSS_L1, img)
            if a.adam == "separate":
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                opt.step()
                e1.record()
                torch.cuda.synchronize()
                adam_ms = e0.elapsed_time(e1)
        wall.append(time.perf_counter() - t0)
    torch.cuda.nvtx.range_pop()
    prof = api.rgba_profile_read(r.ctx)
    if adam_ms is not None:
        prof["adam"] = adam_ms
    stats = None
    if a.stats:  # the same step state as the last profiled step (no update in between)
        api.rgba_profile_enable(r.ctx, 2)
        r.step(db, tg, api.RGBA_LOSS_L1, img)
        stats = api.rgba_debug_render_stats(r.ctx, db.struct(), ws.data_ptr(), ws.numel(),
                                            torch.cuda.current_stream().cuda_stream)
        api.rgba_profile_enable(r.ctx, 0)
    r.close()
    print(json.dumps({"workload": a.workload, "frames": db.n_frames, "pairs": out.pairs,
                      "loss": out.loss, "step_ms": [1e3 * w for w in wall], "stages_ms": prof,
                      "render_stats": stats}))


if __name__ == "__main__":
    main()
