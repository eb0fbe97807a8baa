"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI, read its
intermediate results out of the workspace, run the oracle on the same seeded inputs, and
compare."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2503_12886_gb300 import api, synth
from paper_2503_12886_gb300.rasterizer import DeviceBatch, Renderer

# Pixels: the workload tolerance. Gradients: relative bound plus a floor of 1e-3 of the
# largest reference entry of the same channel, for entries that cancel to near zero.
PIX_ATOL = 1e-4
GRAD_RTOL = 1e-3
GRAD_FLOOR = 1e-3
# Compositing decisions that the fp32 GPU path and the fp64 oracle may take differently are
# flagged by the oracle within these relative margins: alpha against 1/255 and 0.99 (fp32 exp
# and product error ~1e-6 relative), T (1 - alpha) against 1e-4 (fp32 product of up to a few
# hundred factors, ~1e-5 relative).
AMBIG_EPS = 1e-5
AMBIG_EPS_T = 1e-4


def run_gpu_forward(batch: synth.Batch, tile=(16, 16), smem_batch=64, renderer=None):
    r = renderer or Renderer(0)
    db = DeviceBatch(batch, "cuda:0", tile=tile, smem_batch=smem_batch)
    img, T, n = r.forward(db)
    torch.cuda.synchronize()
    return r, db, img, T, n


def read_intermediates(r: Renderer, db: DeviceBatch) -> dict:
    lay = r.layout(db)
    ws = r.ws
    R, Tt = lay.records_total, lay.tiles_total

    def arr(off, nbytes, dt):
        return ws[off: off + nbytes].cpu().numpy().view(dt)

    rec = arr(lay.records, R * 48, np.float32).reshape(R, 12)
    rects = arr(lay.rects, R * 8, np.uint16).reshape(R, 4)
    ts = arr(lay.tile_start, (Tt + 1) * 4, np.uint32)
    pairs = int(ts[-1])
    srt = arr(lay.sorted, pairs * 4, np.uint32)
    g2 = arr(lay.grad2d, R * 48, np.float32).reshape(R, 12)
    return {"records": rec, "rects": rects, "tile_start": ts, "sorted": srt, "grad2d": g2,
            "layout": lay}


def grad2d_from_sums(sums: np.ndarray, rec: np.ndarray) -> np.ndarray:
    """The 2-D gradients dL/d(u, v, conic a, b, c, opacity, r, g, b) of the records rec [n][12]
    from the compositing backward's per-record sums [n][>=9] (the workspace's grad2d layout:
    S1..S5, S0 of g (dx, dy, dx^2, dx dy, dy^2, 1), g = dL/dpower, then the colour gradients),
    in FP64: power = -(a dx^2 + c dy^2) / 2 - b dx dy with dx = pixel - u, alpha = o e^power."""
    S = np.asarray(sums, np.float64)
    a, b, c, o = (np.asarray(rec[:, k], np.float64) for k in (2, 3, 4, 5))
    out = np.zeros((S.shape[0], 9))
    out[:, 0] = a * S[:, 0] + b * S[:, 1]
    out[:, 1] = b * S[:, 0] + c * S[:, 1]
    out[:, 2] = -0.5 * S[:, 2]
    out[:, 3] = -S[:, 3]
    out[:, 4] = -0.5 * S[:, 4]
    out[:, 5] = np.divide(S[:, 5], o, out=np.zeros_like(o), where=o > 0)
    out[:, 6:9] = S[:, 6:9]
    return out


def frame_tile_bases(batch: synth.Batch, tile=(16, 16)):
    TW, TH = tile
    out, t = [], 0
    for fr in batch.frames:
        out.append(t)
        t += ((fr.width + TW - 1) // TW) * ((fr.height + TH - 1) // TH)
    return out


def compare_decisions(batch, ores, inter, db, tile=(16, 16)):
    """Bit-exact: rectangles, fp32 record values, tile list offsets and every list."""
    bases = frame_tile_bases(batch, tile)
    TW, TH = tile
    stats = {"kept": 0, "pairs": 0}
    for b, fr in enumerate(batch.frames):
        m = batch.models[fr.model]
        o = ores[b]
        rb = db.rec_offsets[b]
        g_rect = inter["rects"][rb: rb + m.n].astype(np.int32)
        np.testing.assert_array_equal(g_rect, o.rect, err_msg=f"frame {b} rects")
        kept = (o.rect[:, 2] > o.rect[:, 0]) & (o.rect[:, 3] > o.rect[:, 1])
        stats["kept"] += int(kept.sum())
        g = inter["records"][rb: rb + m.n]
        # u, v, conic a, b, c, opacity, depth from the fp32 decision spec
        pairs_cols = [(0, 0), (1, 1), (2, 2), (3, 3), (4, 4), (5, 7), (9, 6)]
        for gc, oc in pairs_cols:
            np.testing.assert_array_equal(g[kept, gc].view(np.uint32), o.f32[kept, oc].view(np.uint32),
                                          err_msg=f"frame {b} record column {gc}")
        nt = ((fr.width + TW - 1) // TW) * ((fr.height + TH - 1) // TH)
        ts = inter["tile_start"][bases[b]: bases[b] + nt + 1].astype(np.int64)
        np.testing.assert_array_equal(ts - ts[0], o.tile_start.astype(np.int64),
                                      err_msg=f"frame {b} tile offsets")
        lst = inter["sorted"][ts[0]: ts[-1]].astype(np.int64)
        np.testing.assert_array_equal(lst, o.lst.astype(np.int64), err_msg=f"frame {b} lists")
        stats["pairs"] += len(o.lst)
    return stats


def compare_images(batch, ores, db, img, T, n, tiles_only=None):
    """Pixels within PIX_ATOL and equal contributor counts, except on pixels the oracle flags
    as ambiguous (a cutoff decision within AMBIG_EPS relative); flagged pixels are counted and
    still bounded by the size of one flipped contribution."""
    imgs = db.image_views(img)
    Ts = db.pix_views(T)
    ns = db.pix_views(n)
    out = {"pixels": 0, "flagged": 0, "max_err": 0.0, "max_err_flagged": 0.0, "n_mismatch": 0}
    for b, fr in enumerate(batch.frames):
        o = ores[b]
        if o.img is None:
            continue
        gi = imgs[b].cpu().numpy().astype(np.float64)
        gT = Ts[b].cpu().numpy().astype(np.float64)
        gn = ns[b].cpu().numpy()
        mask = np.ones((fr.height, fr.width), bool) if tiles_only is None else tiles_only[b]
        fl = (o.flags > 0) & mask
        ok = (~fl) & mask
        e = np.abs(gi - o.img).max(0)
        eT = np.abs(gT - o.T)
        out["pixels"] += int(mask.sum())
        out["flagged"] += int(fl.sum())
        if ok.any():
            out["max_err"] = max(out["max_err"], float(e[ok].max()), float(eT[ok].max()))
            out["n_mismatch"] += int((gn[ok] != o.n_contrib[ok]).sum())
        if fl.any():
            out["max_err_flagged"] = max(out["max_err_flagged"], float(e[fl].max()))
    return out


def grad_error(g: np.ndarray, ref: np.ndarray, axis_rows=True):
    """max over entries of |g - ref| / (rtol |ref| + floor * max|ref of its row|) (<= 1 passes)."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0.0
    rows = ref.reshape(ref.shape[0], -1) if axis_rows else ref.reshape(1, -1)
    gr = g.reshape(rows.shape)
    scale = np.abs(rows).max(1, keepdims=True)
    tol = GRAD_RTOL * np.abs(rows) + GRAD_FLOOR * scale + 1e-30
    return float((np.abs(gr - rows) / tol).max())


def oracle_fwd_bwd(batch, targets, kind, tile=(16, 16), drop_flagged=False, with_blended=False):
    """Oracle forward, loss and backward. With drop_flagged, dL/dimg is zeroed at the pixels
    the oracle flags as ambiguous (a compositing cutoff within AMBIG_EPS / AMBIG_EPS_T): there
    the fp32 path may legitimately take the other decision, and the gradient of that pixel is
    discontinuous, so both backward passes then see the same, decision-stable dL/dimg.
    with_blended: also return the per-frame gradients with respect to the blended Gaussians
    ([14][n_pad] per frame)."""
    ores = oracle.forward(batch, tile=tile, eps=AMBIG_EPS, splat="spec", eps_t=AMBIG_EPS_T)
    L, dls = oracle.loss(batch, ores, targets, kind)
    if drop_flagged:
        dls = [np.where(r.flags[None] != 0, 0.0, d) for r, d in zip(ores, dls)]
    per_model, dpsi, g2s, dgbs = oracle.backward(batch, ores, dls, tile=tile)
    if with_blended:
        return ores, L, dls, per_model, dpsi, g2s, dgbs
    return ores, L, dls, per_model, dpsi, g2s


def backward_errors(batch, db, per_model, dpsi, dgbs=None, grad_blended=None):
    """grad_error of every model's dG0 and ddG, of dpsi and (when both are given) of each
    frame's gradient with respect to its blended Gaussians (one row per channel). Also checks
    that padding columns of dG0 stay zero."""
    errs = {}
    for mi, m in enumerate(db.models):
        g0_ref, dg_ref = per_model[mi]
        errs[f"g0[{mi}]"] = grad_error(m.grad_g0.cpu().numpy()[:, :m.n], g0_ref[:, :m.n])
        errs[f"dg[{mi}]"] = grad_error(m.grad_dg.cpu().numpy()[..., :m.n].reshape(-1, m.n),
                                       dg_ref[..., :m.n].reshape(-1, m.n))
        assert np.all(m.grad_g0.cpu().numpy()[:, m.n:] == 0)
    errs["psi"] = grad_error(db.grad_psi.cpu().numpy(), dpsi, axis_rows=False)
    if dgbs is not None and grad_blended is not None:
        gb = grad_blended.cpu().numpy()
        worst = 0.0
        for b, (mi, _, _) in enumerate(db.frames):
            m = db.models[mi]
            got = gb[db.rec_offsets[b] * 14: (db.rec_offsets[b] + m.n_pad) * 14].reshape(14, m.n_pad)
            worst = max(worst, grad_error(got[:, :m.n], dgbs[b][:, :m.n]))
            assert np.all(got[:, m.n:] == 0)
        errs["blended"] = worst
    return errs


def gpu_step(batch, targets, kind, tile=(16, 16), smem_batch=64, renderer=None):
    r = renderer or Renderer(0)
    db = DeviceBatch(batch, "cuda:0", tile=tile, smem_batch=smem_batch)
    tg = db.pack_images(targets)
    img = torch.empty(3 * db.total_pix, dtype=torch.float32, device="cuda:0")
    lk = api.RGBA_LOSS_L1 if kind == "l1" else api.RGBA_LOSS_L2
    out = r.step(db, tg, lk, img)
    torch.cuda.synchronize()
    return r, db, img, out
