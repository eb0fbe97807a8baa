"""Parity at the full workload sizes, in the launch configuration the bench times: all tile
decisions and lists bit-exact, pixels and per-Gaussian 2-D gradients on sampled tile blocks
(the oracle renders only those tiles), sampled frames of the uneven 64-frame batch, and the
final gradients (dG0, ddG, dpsi) of the batched, tangent-space and uneven workloads with every
pixel of every frame."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_12886_gb300 import synth
from paper_2503_12886_gb300.rasterizer import DeviceBatch, Renderer

from gpu_helpers import (GRAD_FLOOR, GRAD_RTOL, PIX_ATOL, backward_errors, compare_decisions,
                         compare_images, grad2d_from_sums, oracle_fwd_bwd, read_intermediates)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    import __graft_entry__
    __graft_entry__.build()
    r = Renderer(0)
    yield r
    r.close()


def _block_mask(fr, ores_f, TW, TH, size=4):
    """A size x size block of tiles centred on the frame's densest tile."""
    tx, ty = (fr.width + TW - 1) // TW, (fr.height + TH - 1) // TH
    counts = np.diff(ores_f.tile_start).reshape(ty, tx)
    cy, cx = np.unravel_index(np.argmax(counts), counts.shape)
    y0, x0 = max(0, min(ty - size, cy - size // 2)), max(0, min(tx - size, cx - size // 2))
    mask = np.zeros(ty * tx, np.uint8)
    pix = np.zeros((fr.height, fr.width), bool)
    for y in range(y0, y0 + size):
        mask[y * tx + x0: y * tx + x0 + size] = 1
    pix[y0 * TH:(y0 + size) * TH, x0 * TW:(x0 + size) * TW] = True
    return mask, pix, (x0, y0, x0 + size, y0 + size)


def test_batched_workload_full_size(renderer):
    batch = synth.workload_batched()           # N=60,000, K=32, B=16, 512x512
    db = DeviceBatch(batch, "cuda:0", tile=(16, 16), smem_batch=64)
    img, T, n = renderer.forward(db)
    torch.cuda.synchronize()
    inter = read_intermediates(renderer, db)
    ores = oracle.forward(batch, do_render=False)
    st = compare_decisions(batch, ores, inter, db)
    assert st["pairs"] > 3_000_000
    # sampled tile blocks of three frames: pixels, then 2-D gradients of the Gaussians that lie
    # entirely inside the block (so the oracle, rendering only the block, sees all of them)
    rng = np.random.default_rng(0)
    dl = torch.from_numpy(rng.standard_normal(3 * db.total_pix).astype(np.float32) * 1e-6).cuda()
    renderer.backward(db, dl, T, n)
    torch.cuda.synchronize()
    inter = read_intermediates(renderer, db)
    g2_gpu = grad2d_from_sums(inter["grad2d"], inter["records"])
    dl_views = [v.cpu().numpy().astype(np.float64) for v in db.image_views(dl)]
    checked = 0
    for b in (0, 7, 15):
        fr = batch.frames[b]
        mask, pix, (x0, y0, x1, y1) = _block_mask(fr, ores[b], 16, 16)
        sub = synth.Batch(batch.models, [fr], batch.psi[b:b + 1], batch.fparams[b:b + 1], batch.k_stride)
        o = oracle.forward(sub, splat="spec", tile_masks={0: mask})
        s = compare_images(sub, o, _view_batch(db, b), img, T, n, tiles_only=[pix])
        assert s["max_err"] <= 1e-4 and s["n_mismatch"] == 0, s
        # the block is the frame's densest (most evaluations per pixel, so more cutoff
        # decisions near their threshold); whole frames stay under 0.1 % flagged
        assert s["flagged"] <= 0.005 * s["pixels"]
        g2 = oracle.render_bwd(fr.width, fr.height, 16, 16, o[0].rec, o[0].tile_start, o[0].lst,
                               batch.fparams[b, 17:20].astype(np.float64), dl_views[b],
                               batch.models[0].n, mask)
        r = o[0].rect
        inside = (r[:, 0] >= x0) & (r[:, 2] <= x1) & (r[:, 1] >= y0) & (r[:, 3] <= y1) & (r[:, 2] > r[:, 0])
        idx = np.nonzero(inside)[0]
        assert len(idx) > 100
        got = g2_gpu[db.rec_offsets[b] + idx]
        ref = g2[idx]
        scale = np.abs(ref).max(0, keepdims=True)
        err = np.abs(got - ref) / (GRAD_RTOL * np.abs(ref) + GRAD_FLOOR * scale + 1e-30)
        assert err.max() <= 1.0, (b, err.max())
        checked += len(idx)
    assert checked > 300


def test_batched_workload_gradients_full_size(renderer):
    """The batched training workload at its full size (N=60,000, K=32, B=16 at 512x512, the
    bench's 16x16 tiles and 64-entry staging): every pixel of every frame, then dG0, ddG, dpsi
    and each frame's gradient with respect to its blended Gaussians against the oracle, from
    the same L1 dL/dimg (zero at the pixels the oracle flags as ambiguous)."""
    batch = synth.workload_batched()
    targets = synth.make_targets(batch, 99)
    ores, L, dls, per_model, dpsi, g2s, dgbs = oracle_fwd_bwd(batch, targets, "l1",
                                                               drop_flagged=True, with_blended=True)
    db = DeviceBatch(batch, "cuda:0", tile=(16, 16), smem_batch=64)
    img, T, n = renderer.forward(db)
    torch.cuda.synchronize()
    st = compare_images(batch, ores, db, img, T, n)
    assert st["max_err"] <= PIX_ATOL and st["n_mismatch"] == 0, st
    assert st["flagged"] <= 0.001 * st["pixels"], st
    dl = db.pack_images([d.astype(np.float32) for d in dls])
    gb = torch.full((db.total_rec * 14,), float("nan"), device="cuda:0")
    renderer.backward(db, dl, T, n, grad_blended=gb)
    torch.cuda.synchronize()
    errs = backward_errors(batch, db, per_model, dpsi, dgbs, gb)
    assert max(errs.values()) <= 1.0, errs


class _view_batch:
    """DeviceBatch-like view of one frame of a batch (for compare_images)."""

    def __init__(self, db, b):
        self.db, self.b = db, b

    def image_views(self, flat):
        return [self.db.image_views(flat)[self.b]]

    def pix_views(self, flat):
        return [self.db.pix_views(flat)[self.b]]


def test_uneven_workload_sampled_frames(renderer):
    batch = synth.workload_uneven()            # 8 avatars N 20k..100k, 64 frames 256/512/1024
    db = DeviceBatch(batch, "cuda:0", tile=(16, 16), smem_batch=64, grads=False)
    img, T, n = renderer.forward(db)
    torch.cuda.synchronize()
    inter = read_intermediates(renderer, db)
    for b in (0, 9, 18, 21, 47, 63):          # 256, 512 and 1024 px frames, all 8 avatars
        fr = batch.frames[b]
        sub = synth.Batch(batch.models, [fr], batch.psi[b:b + 1], batch.fparams[b:b + 1],
                          batch.k_stride)
        o = oracle.forward(sub, do_render=False)
        # decisions of frame b against the oracle (its records and lists inside the batch)
        m = batch.models[fr.model]
        rb = db.rec_offsets[b]
        np.testing.assert_array_equal(inter["rects"][rb: rb + m.n].astype(np.int32), o[0].rect)
        tb = sum(((f.width + 15) // 16) * ((f.height + 15) // 16) for f in batch.frames[:b])
        nt = ((fr.width + 15) // 16) * ((fr.height + 15) // 16)
        ts = inter["tile_start"][tb: tb + nt + 1].astype(np.int64)
        np.testing.assert_array_equal(ts - ts[0], o[0].tile_start)
        np.testing.assert_array_equal(inter["sorted"][ts[0]: ts[-1]].astype(np.int64), o[0].lst)
        mask, pix, _ = _block_mask(fr, o[0], 16, 16, size=3)
        o = oracle.forward(sub, splat="spec", tile_masks={0: mask})
        s = compare_images(sub, o, _view_batch(db, b), img, T, n, tiles_only=[pix])
        assert s["max_err"] <= 1e-4 and s["n_mismatch"] == 0, (b, s)


def test_tangent_workload_full_size(renderer):
    """The bench's tangent-space workload (N=60,000 bound to a 9,024-triangle mesh, K=32,
    B=16 at 512x512): every decision and list bit-exact, pixels of the densest tile block of
    three frames."""
    batch = synth.workload_tangent()
    db = DeviceBatch(batch, "cuda:0", tile=(16, 16), smem_batch=64, grads=False)
    img, T, n = renderer.forward(db)
    torch.cuda.synchronize()
    inter = read_intermediates(renderer, db)
    ores = oracle.forward(batch, do_render=False)
    st = compare_decisions(batch, ores, inter, db)
    assert st["pairs"] > 3_000_000
    for b in (0, 8, 15):
        fr = batch.frames[b]
        mask, pix, _ = _block_mask(fr, ores[b], 16, 16)
        sub = synth.Batch(batch.models, [fr], batch.psi[b:b + 1], batch.fparams[b:b + 1], batch.k_stride)
        o = oracle.forward(sub, splat="spec", tile_masks={0: mask})
        s = compare_images(sub, o, _view_batch(db, b), img, T, n, tiles_only=[pix])
        assert s["max_err"] <= 1e-4 and s["n_mismatch"] == 0, (b, s)
        assert s["flagged"] <= 0.005 * s["pixels"]


def test_tangent_workload_gradients_full_size(renderer):
    """The tangent-space training workload at its full size (N=60,000 bound to a 9,024-triangle
    head mesh with an expression per frame, K=32, B=16 at 512x512; Alg. 1 in the preprocess and
    its derivative in the Gaussian backward): every pixel of every frame, then dG0, ddG, dpsi and
    each frame's gradient with respect to its blended Gaussians against the oracle, from the same
    L1 dL/dimg (zero at the pixels the oracle flags as ambiguous)."""
    batch = synth.workload_tangent()
    targets = synth.make_targets(batch, 97)
    ores, L, dls, per_model, dpsi, g2s, dgbs = oracle_fwd_bwd(batch, targets, "l1",
                                                               drop_flagged=True, with_blended=True)
    db = DeviceBatch(batch, "cuda:0", tile=(16, 16), smem_batch=64)
    img, T, n = renderer.forward(db)
    torch.cuda.synchronize()
    st = compare_images(batch, ores, db, img, T, n)
    assert st["max_err"] <= PIX_ATOL and st["n_mismatch"] == 0, st
    assert st["flagged"] <= 0.001 * st["pixels"], st
    dl = db.pack_images([d.astype(np.float32) for d in dls])
    gb = torch.full((db.total_rec * 14,), float("nan"), device="cuda:0")
    renderer.backward(db, dl, T, n, grad_blended=gb)
    torch.cuda.synchronize()
    errs = backward_errors(batch, db, per_model, dpsi, dgbs, gb)
    assert max(errs.values()) <= 1.0, errs


def test_uneven_workload_full_size(renderer):
    """The uneven batch at its full size (8 avatars, N 20k..100k, K 16/24/32, 64 frames at
    256/512/1024 px, one launch per stage, the bench's 16x16 tiles and 64-entry staging): every
    frame's decisions and lists bit-exact, every pixel, then every avatar's dG0 and ddG and every
    frame's dpsi against the oracle. Both backward passes take the same dL/dimg: the L1 gradient
    of the CUDA image, zero at the pixels the oracle flags as ambiguous. The oracle runs one
    spawned worker per avatar."""
    import multiprocessing as mp
    import os

    import oracle_pool
    from gpu_helpers import AMBIG_EPS, AMBIG_EPS_T, frame_tile_bases, grad_error

    batch = synth.workload_uneven()
    B = len(batch.frames)
    db = DeviceBatch(batch, "cuda:0", tile=(16, 16), smem_batch=64)
    img, T, n = renderer.forward(db)
    torch.cuda.synchronize()
    inter = read_intermediates(renderer, db)
    targets = synth.make_targets(batch, 96)
    imgs, Ts, ns = db.image_views(img), db.pix_views(T), db.pix_views(n)
    bases = frame_tile_bases(batch)
    payload = {a: [] for a in range(len(batch.models))}
    for b, fr in enumerate(batch.frames):
        m = batch.models[fr.model]
        rb = db.rec_offsets[b]
        nt = ((fr.width + 15) // 16) * ((fr.height + 15) // 16)
        ts = inter["tile_start"][bases[b]: bases[b] + nt + 1].astype(np.int64)
        gi = imgs[b].cpu().numpy()
        # L1 over the batch: mean per frame, mean over the frames
        dl = (np.sign(gi.astype(np.float64) - targets[b]) / (3.0 * fr.width * fr.height * B)).astype(np.float32)
        payload[fr.model].append({
            "b": b, "img": gi, "T": Ts[b].cpu().numpy(), "n": ns[b].cpu().numpy(),
            "rect": inter["rects"][rb: rb + m.n].astype(np.int32), "rec": inter["records"][rb: rb + m.n],
            "tile_start": ts - ts[0], "lst": inter["sorted"][ts[0]: ts[-1]].astype(np.int64), "dl": dl})
    jobs = [(a, payload[a], AMBIG_EPS, AMBIG_EPS_T, PIX_ATOL) for a in payload]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(oracle_pool.uneven_avatar, jobs)
    dls = [None] * B
    flagged = pixels = 0
    for r in res:
        flagged += r["stats"]["flagged"]
        pixels += r["stats"]["pixels"]
        for j, b in enumerate(r["idx"]):
            f = payload[r["a"]][j]
            dls[b] = np.where(r["flags"][j][None], np.float32(0), f["dl"])
    assert flagged <= 0.001 * pixels, (flagged, pixels)
    renderer.backward(db, db.pack_images(dls), T, n)
    torch.cuda.synchronize()
    errs = {}
    dpsi = np.zeros_like(db.grad_psi.cpu().numpy(), dtype=np.float64)
    for r in res:
        m = db.models[r["a"]]
        errs[f"g0[{r['a']}]"] = grad_error(m.grad_g0.cpu().numpy()[:, :m.n], r["g0"][:, :m.n])
        errs[f"dg[{r['a']}]"] = grad_error(m.grad_dg.cpu().numpy()[..., :m.n].reshape(-1, m.n),
                                           r["dg"][..., :m.n].reshape(-1, m.n))
        assert np.all(m.grad_g0.cpu().numpy()[:, m.n:] == 0)
        dpsi[r["idx"], :r["dpsi"].shape[1]] = r["dpsi"]
    errs["psi"] = grad_error(db.grad_psi.cpu().numpy(), dpsi, axis_rows=False)
    assert max(errs.values()) <= 1.0, errs
