"""CUDA path vs the FP64 oracle on the same seeded inputs, through the C ABI.

Bars: bit-exact tile rectangles, fp32 splat values, tile offsets and per-tile sorted lists;
pixels within 1e-4 (pixels the oracle flags as ambiguous at a cutoff are counted and bounded
separately); gradients within 1e-3 relative with a per-channel floor (gpu_helpers.grad_error).
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2503_12886_gb300 import api, synth
from paper_2503_12886_gb300.rasterizer import DeviceBatch, Renderer

from gpu_helpers import (PIX_ATOL, backward_errors, compare_decisions, compare_images,
                         grad_error, oracle_fwd_bwd, read_intermediates, run_gpu_forward)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    import __graft_entry__
    __graft_entry__.build()
    r = Renderer(0)
    yield r
    r.close()


def ragged_batch():
    """Three frames of one avatar at ragged sizes (not multiples of the tile), random bg."""
    m = synth.make_model(77, 3000, 6, log_scale_mu=math.log(5e-3))
    fr = [synth.Frame(0, 100, 75), synth.Frame(0, 37, 129), synth.Frame(0, 64, 64)]
    return synth.make_batch([m], fr, seed=77, jitter_deg=15, random_bg=True)


def uneven_batch():
    """Eight avatars (N 1k..5k, K 16/24/32) over 8 frames at 256/512/1024 pixels."""
    models = [synth.make_model(400 + a, n, k) for a, (n, k) in
              enumerate([(1000, 16), (1750, 24), (2500, 32), (3250, 16), (4000, 24), (4500, 32),
                         (4750, 16), (5000, 24)])]
    res = [256, 512, 1024, 256, 512, 256, 512, 256]
    fr = [synth.Frame(f % 8, res[f], res[f]) for f in range(8)]
    return synth.make_batch(models, fr, seed=4000, jitter_deg=20, random_bg=True)


def ties_batch():
    """Exact depth ties: the means of avatar 0 repeat in groups of 20 and those of avatar 1 in
    groups of 125 (no mean deltas, so blended means and depths stay equal): runs of equal depth
    in a tile list that the tie pass orders by itself, and runs longer than it orders, which
    take the full-key sort."""
    models = []
    for a, grp in enumerate((20, 125)):
        m = synth.make_model(91 + a, 2000, 4, sd_dmean=0.0, log_scale_mu=math.log(5e-3))
        g0 = m.g0.copy()
        for s in range(0, m.n, grp):
            g0[0:3, s:s + grp] = g0[0:3, s:s + 1]
        models.append(dataclasses.replace(m, g0=g0))
    return synth.make_batch(models, [synth.Frame(0, 96, 80), synth.Frame(1, 96, 80)], seed=91,
                            jitter_deg=10, random_bg=True)


def dense_batch():
    """16,000 Gaussians within 4 px of one tile corner: lists of up to ~15,000 keys, longer
    than a shared-memory sort holds, with natural depth ties."""
    m = synth.make_model(93, 16_000, 4, radii=(0.05, 0.05, 0.05), log_scale_mu=math.log(6e-3))
    return synth.make_batch([m], [synth.Frame(0, 64, 64)], seed=93)


def mid_lists_batch():
    """11,000 Gaussians around one tile corner: four tile lists of 8,238 to 10,405 keys, past the
    shared-memory bucket sort's 8,192 and within the position bucket sort's 12,288 (depth
    buckets of at most 16 keys)."""
    m = synth.make_model(93, 11_000, 4, radii=(0.05, 0.05, 0.05), log_scale_mu=math.log(6e-3))
    return synth.make_batch([m], [synth.Frame(0, 64, 64)], seed=93)


def mid_lists_crowded_batch():
    """The same four list lengths, with a cluster of 300 Gaussians at nearly one depth (steps of
    about two ulps) in them: about 250 keys fall into one depth bucket, more than the position
    sort's rank placement takes, so those lists go to the global-memory sort after it."""
    m = synth.make_model(94, 11_000, 4, radii=(0.05, 0.05, 0.05), log_scale_mu=math.log(6e-3), sd_dmean=0.0)
    g0 = m.g0.copy()
    g0[0:2, :300] = 0.0
    g0[2, :300] = 0.02 + 2.4e-7 * np.arange(300)
    return synth.make_batch([dataclasses.replace(m, g0=g0)], [synth.Frame(0, 64, 64)], seed=94)


def cluster_batch():
    """A tight cluster of 300 Gaussians at nearly one depth (steps of about two ulps) among 1,700
    spread ones: the cluster's tile lists put ~150 distinct keys into each of one or two of the
    sort's 4096 depth buckets, more than its rank placement takes, so those segments take the
    full-key fallback; buckets of a few keys take the rank placement."""
    m = synth.make_model(95, 2000, 4, sd_dmean=0.0, log_scale_mu=math.log(5e-3))
    g0 = m.g0.copy()
    g0[0:2, :300] = 0.0
    g0[2, :300] = 0.05 + 2.4e-7 * np.arange(300)
    return synth.make_batch([dataclasses.replace(m, g0=g0)], [synth.Frame(0, 96, 96)], seed=95)


MASK_ALL = sum(1 << c for c in range(14) if c != 10)   # every channel but opacity
MASK_MEAN_COLOR = 0x7 | (0x7 << 11)


def all_channels_batch():
    """The largest blend: K = 64 blendshapes on all 13 blendable channels (a mask without a
    compiled instance: the preprocess reads it at run time), 14 + 832 staged rows per chunk."""
    m = synth.make_model(97, 1500, 64, mask=MASK_ALL)
    return synth.make_batch([m], [synth.Frame(0, 96, 96), synth.Frame(0, 80, 112)], seed=97,
                            jitter_deg=10, random_bg=True)


def mixed_masks_batch():
    """Two avatars with different channel masks in one batch (mean + colour, and the paper's):
    no common mask, so the preprocess takes its run-time-mask instance."""
    ms = [synth.make_model(98, 3000, 12, mask=MASK_MEAN_COLOR), synth.make_model(99, 2500, 8, mask=synth.MASK_PAPER)]
    fr = [synth.Frame(0, 96, 80), synth.Frame(1, 80, 96), synth.Frame(1, 64, 64)]
    return synth.make_batch(ms, fr, seed=98, jitter_deg=15, random_bg=True)


def tangent_batch(mask=synth.MASK_MEAN_SCALE_COLOR, seed=81):
    """Gaussians bound to a head mesh (tangent space, Supp. "Gaussian Transformation"), three
    frames with different mesh expressions, jittered cameras, random background."""
    mesh = synth.make_head_mesh(seed, 24, 48)
    m = synth.make_bound_model(seed, 8000, 8, mesh, mask=mask)
    fr = [synth.Frame(0, 192, 160, synth.frame_verts(mesh, seed, f)) for f in range(3)]
    return synth.make_batch([m], fr, seed, jitter_deg=20, random_bg=True)


def odd_k_batch():
    """Blendshape counts that are not multiples of four (7 and 3, one channel mask: the compiled
    instance; the blend takes the weights four at a time and the rest one by one)."""
    ms = [synth.make_model(83, 2500, 7), synth.make_model(84, 1800, 3)]
    fr = [synth.Frame(0, 96, 96), synth.Frame(1, 80, 112), synth.Frame(0, 64, 64)]
    return synth.make_batch(ms, fr, seed=83, jitter_deg=12, random_bg=True)


def odd_k_mixed_batch():
    """K = 5 and K = 1 with different channel masks (the run-time-mask instance)."""
    ms = [synth.make_model(85, 2200, 5, mask=synth.MASK_PAPER), synth.make_model(86, 2000, 1, mask=MASK_MEAN_COLOR)]
    fr = [synth.Frame(0, 96, 80), synth.Frame(1, 96, 96)]
    return synth.make_batch(ms, fr, seed=85, jitter_deg=12, random_bg=True)


def closeup_batch():
    """The camera 0.25 m and 0.22 m from the avatar's centre: the near plane (0.2 m) culls part
    of the avatar, the rest spans more than the field of view, so the Jacobian's 1.3 x
    half-fov clamp is active for many Gaussians (the decision spec's clamp and the backward's
    blocked gradient on clamped coordinates), and the splats are large."""
    m = synth.make_model(88, 4000, 8)
    b = synth.make_batch([m], [synth.Frame(0, 128, 128), synth.Frame(0, 96, 128)], seed=88, jitter_deg=10,
                         random_bg=True)
    b.fparams[0, 11] = 0.25
    b.fparams[1, 11] = 0.22
    return b


def many_tiles_batch():
    """17 frames of 512x512 at 16x16 tiles: 17,408 tiles over 17 scan CTAs, a batch with more
    tiles than the 16-frame workload, every tile list and pixel compared."""
    m = synth.make_model(87, 3000, 8)
    return synth.make_batch([m], [synth.Frame(0, 512, 512) for _ in range(17)], seed=87, jitter_deg=15,
                            random_bg=True)


CASES = {
    "single_128": (lambda: synth.workload_single(), (16, 16), 64),
    "gradcheck_64": (lambda: synth.workload_gradcheck(), (16, 16), 256),
    "gradcheck_paper_mask": (lambda: synth.workload_gradcheck(mask=synth.MASK_PAPER), (16, 16), 128),
    "batched_reduced": (lambda: synth.workload_batched(n=20_000, k=32, frames=4, res=256), (16, 16), 64),
    "ragged_8x32": (ragged_batch, (8, 32), 64),
    "uneven": (uneven_batch, (16, 16), 128),
    "depth_ties": (ties_batch, (16, 16), 128),
    "depth_cluster": (cluster_batch, (16, 16), 64),
    "all_channels_k64": (all_channels_batch, (16, 16), 64),
    "mixed_masks": (mixed_masks_batch, (8, 32), 128),
    "dense_lists": (dense_batch, (16, 16), 64),
    "mid_lists": (mid_lists_batch, (16, 16), 64),
    "mid_lists_crowded": (mid_lists_crowded_batch, (16, 16), 64),
    "tangent": (tangent_batch, (16, 16), 64),
    "tangent_paper_mask": (lambda: tangent_batch(synth.MASK_PAPER, 82), (8, 32), 128),
    "odd_k": (odd_k_batch, (16, 16), 64),
    "odd_k_mixed": (odd_k_mixed_batch, (8, 32), 64),
    "many_tiles": (many_tiles_batch, (16, 16), 64),
    "closeup": (closeup_batch, (16, 16), 64),
}


@pytest.mark.parametrize("case", list(CASES))
def test_decisions_and_sort_bit_exact(renderer, case):
    make, tile, sb = CASES[case]
    batch = make()
    r, db, img, T, n = run_gpu_forward(batch, tile, sb, renderer)
    ores = oracle.forward(batch, tile=tile, do_render=False)
    st = compare_decisions(batch, ores, read_intermediates(r, db), db, tile)
    assert st["kept"] > 0 and st["pairs"] > 0


@pytest.mark.parametrize("case", list(CASES))
def test_forward_pixels(renderer, case):
    make, tile, sb = CASES[case]
    batch = make()
    r, db, img, T, n = run_gpu_forward(batch, tile, sb, renderer)
    ores = oracle.forward(batch, tile=tile, splat="spec")
    st = compare_images(batch, ores, db, img, T, n)
    assert st["max_err"] <= PIX_ATOL, st
    assert st["n_mismatch"] == 0, st
    assert st["flagged"] <= 0.001 * st["pixels"], st
    assert st["max_err_flagged"] <= 5e-3, st


@pytest.mark.parametrize("case", list(CASES))
def test_backward_gradients(renderer, case):
    """Same dL/dimg (the oracle's, from its own image, zero at the pixels it flags as
    ambiguous) into both backward passes."""
    make, tile, sb = CASES[case]
    batch = make()
    kind = "l2" if case.startswith("gradcheck") else "l1"
    targets = synth.make_targets(batch, 99)
    ores, L, dls, per_model, dpsi, g2s = oracle_fwd_bwd(batch, targets, kind, tile, drop_flagged=True)
    r, db, img, T, n = run_gpu_forward(batch, tile, sb, renderer)
    dl = db.pack_images([d.astype(np.float32) for d in dls])
    r.backward(db, dl, T, n)
    torch.cuda.synchronize()
    errs = {}
    for mi, m in enumerate(db.models):
        g0_ref, dg_ref = per_model[mi]
        errs[f"g0[{mi}]"] = grad_error(m.grad_g0.cpu().numpy()[:, :m.n], g0_ref[:, :m.n])
        errs[f"dg[{mi}]"] = grad_error(m.grad_dg.cpu().numpy()[..., :m.n].reshape(-1, m.n),
                                       dg_ref[..., :m.n].reshape(-1, m.n))
        assert np.all(m.grad_g0.cpu().numpy()[:, m.n:] == 0)
    errs["psi"] = grad_error(db.grad_psi.cpu().numpy(), dpsi, axis_rows=False)
    assert max(errs.values()) <= 1.0, errs


@pytest.mark.parametrize("case", ["single_128", "gradcheck_64", "uneven"])
def test_step_loss_and_grads(renderer, case):
    """rgba_step (fused loss, one sync) against the oracle loss and gradients."""
    make, tile, sb = CASES[case]
    batch = make()
    kind = "l2" if case.startswith("gradcheck") else "l1"
    targets = synth.make_targets(batch, 98)
    ores, L, dls, per_model, dpsi, g2s = oracle_fwd_bwd(batch, targets, kind, tile)
    db = DeviceBatch(batch, "cuda:0", tile=tile, smem_batch=sb)
    tg = db.pack_images(targets)
    img = torch.empty(3 * db.total_pix, dtype=torch.float32, device="cuda:0")
    out = renderer.step(db, tg, api.RGBA_LOSS_L1 if kind == "l1" else api.RGBA_LOSS_L2, img)
    torch.cuda.synchronize()
    assert abs(out.loss - L) <= 1e-5 * abs(L) + 1e-7, (out.loss, L)
    assert out.pairs == sum(len(o.lst) for o in ores) and not out.overflow
    errs = {}
    for mi, m in enumerate(db.models):
        g0_ref, dg_ref = per_model[mi]
        errs[f"g0[{mi}]"] = grad_error(m.grad_g0.cpu().numpy()[:, :m.n], g0_ref[:, :m.n])
        errs[f"dg[{mi}]"] = grad_error(m.grad_dg.cpu().numpy()[..., :m.n].reshape(-1, m.n),
                                       dg_ref[..., :m.n].reshape(-1, m.n))
    errs["psi"] = grad_error(db.grad_psi.cpu().numpy(), dpsi, axis_rows=False)
    assert max(errs.values()) <= 1.0, errs


def test_blend_matches_oracle(renderer):
    batch = uneven_batch()
    db = DeviceBatch(batch, "cuda:0")
    out = renderer.blend(db).cpu().numpy()
    for b, fr in enumerate(batch.frames):
        m = batch.models[fr.model]
        ref = oracle.blend(m.g0, m.dg, batch.psi[b, :m.k], m.n, m.mask)
        got = out[db.rec_offsets[b] * 14: (db.rec_offsets[b] + m.n_pad) * 14].reshape(14, m.n_pad)
        # fp32 fused multiply-add chain over k terms: each step rounds once
        mag = np.abs(m.g0.astype(np.float64)).copy()
        chans = synth.blended_channels(m.mask)
        mag[chans] += np.einsum("k,kan->an", np.abs(batch.psi[b, :m.k].astype(np.float64)),
                                np.abs(m.dg.astype(np.float64)))
        bound = (m.k + 1) * 2.0 ** -24 * mag
        assert (np.abs(got[:, :m.n] - ref[:, :m.n]) <= bound[:, :m.n]).all()


def test_identity_frames_match_the_unbound_path_bit_for_bit(renderer):
    """Every Gaussian bound to a triangle whose tangent frame is the identity at the origin:
    the CUDA path's decisions, lists, image, T and contributor counts equal the unbound run."""
    import dataclasses
    m = synth.make_model(91, 6000, 8)
    n = m.n
    bary = np.zeros((3, m.n_pad), np.float32)
    bary[0, :n] = 1.0
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    b = synth.Binding(np.array([[0, 1, 2]], np.int32), np.array([[0, 0, 1, 0, 0, 1]], np.float32),
                      np.zeros(n, np.int32), bary, 3)
    frames = [synth.Frame(0, 160, 128), synth.Frame(0, 96, 96)]
    plain = synth.make_batch([m], frames, seed=91, jitter_deg=15, random_bg=True)
    bound = synth.Batch([dataclasses.replace(m, binding=b)],
                        [synth.Frame(0, f.width, f.height, verts) for f in frames],
                        plain.psi, plain.fparams, plain.k_stride)
    outs = []
    for batch in (plain, bound):
        r, db, img, T, nc = run_gpu_forward(batch, (16, 16), 64, renderer)
        inter = read_intermediates(r, db)
        outs.append((img.clone(), T.clone(), nc.clone(), inter["rects"].copy(),
                     inter["sorted"].copy(), inter["records"].copy()))
    for a, c in zip(*outs):
        if isinstance(a, torch.Tensor):
            assert torch.equal(a, c)
        else:
            np.testing.assert_array_equal(a, c)


def many_frames_batch(nframes, seed):
    """One avatar rendered by more frames than the kernels take in one group (16): ragged
    sizes, jittered cameras, random backgrounds."""
    m = synth.make_model(seed, 3000, 8, log_scale_mu=math.log(5e-3))
    sizes = [(64, 64), (96, 80), (80, 96)]
    fr = [synth.Frame(0, *sizes[f % 3]) for f in range(nframes)]
    return synth.make_batch([m], fr, seed=seed, jitter_deg=20, random_bg=True)


def two_avatars_many_frames():
    """50 frames interleaved over two avatars (33 and 17 frames): both past one frame group."""
    ms = [synth.make_model(611, 3000, 8, log_scale_mu=math.log(5e-3)),
          synth.make_model(612, 2500, 12, log_scale_mu=math.log(5e-3))]
    fr = [synth.Frame(1 if f % 3 == 2 else 0, 64 + 16 * (f % 2), 80) for f in range(50)]
    return synth.make_batch(ms, fr, seed=613, jitter_deg=20, random_bg=True)


MANY = {"17": lambda: many_frames_batch(17, 601), "33": lambda: many_frames_batch(33, 602),
        "40": lambda: many_frames_batch(40, 603), "33+17": two_avatars_many_frames}


@pytest.mark.parametrize("case", list(MANY))
def test_more_than_sixteen_frames_per_avatar(renderer, case):
    """The preprocess runs a model's frames in rounds of 16 and the projection/blend backward
    reduces them in groups of 16: decisions, pixels, dG0, ddG, dpsi and each frame's gradient
    with respect to its blended Gaussians against the oracle when a model has 17 to 40."""
    batch = MANY[case]()
    targets = synth.make_targets(batch, 97)
    ores, L, dls, per_model, dpsi, g2s, dgbs = oracle_fwd_bwd(batch, targets, "l1",
                                                               drop_flagged=True, with_blended=True)
    r, db, img, T, n = run_gpu_forward(batch, (16, 16), 64, renderer)
    compare_decisions(batch, oracle.forward(batch, do_render=False), read_intermediates(r, db), db)
    st = compare_images(batch, ores, db, img, T, n)
    assert st["max_err"] <= PIX_ATOL and st["n_mismatch"] == 0, st
    assert st["flagged"] <= 0.001 * st["pixels"], st
    dl = db.pack_images([d.astype(np.float32) for d in dls])
    gb = torch.full((db.total_rec * 14,), float("nan"), device="cuda:0")
    r.backward(db, dl, T, n, grad_blended=gb)
    torch.cuda.synchronize()
    errs = backward_errors(batch, db, per_model, dpsi, dgbs, gb)
    assert max(errs.values()) <= 1.0, errs

