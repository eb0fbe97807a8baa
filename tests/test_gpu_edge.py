"""Edge cases of the CUDA path through the C ABI: empty batches, empty models, everything
culled, the near-plane boundary, tiny and ragged images, the largest frame and K, pair-buffer overflow with retry, and
tangent-space bindings with degenerate triangles or out-of-range indices."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2503_12886_gb300 import api, synth
from paper_2503_12886_gb300.rasterizer import DeviceBatch, Renderer

from gpu_helpers import compare_decisions, compare_images, read_intermediates, run_gpu_forward

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    import __graft_entry__
    __graft_entry__.build()
    r = Renderer(0)
    yield r
    r.close()


def test_empty_batch_is_a_noop(renderer):
    b = api.RgbaBatch()
    b.n_models, b.n_frames, b.k_stride = 0, 0, 1
    ws = torch.empty(api.rgba_workspace_size(b, 16), dtype=torch.uint8, device="cuda:0")
    s = torch.cuda.current_stream().cuda_stream
    api.rgba_preprocess(renderer.ctx, b, ws.data_ptr(), ws.numel(), s)
    api.rgba_bin_sort(renderer.ctx, b, ws.data_ptr(), ws.numel(), s)
    rc, out = api.rgba_step(renderer.ctx, b, ws.data_ptr(), ws.numel(), 16, 1, None, s)
    assert rc == api.RGBA_OK and out.pairs == 0 and out.loss == 0.0


def test_model_without_gaussians_renders_background(renderer):
    full = synth.make_model(1, 500, 4)
    empty = synth.Model(n=0, k=4, mask=full.mask, g0=np.zeros((14, 4), np.float32),
                        dg=np.zeros((4, 9, 4), np.float32))
    batch = synth.make_batch([empty, full], [synth.Frame(0, 48, 40), synth.Frame(1, 48, 40)],
                             seed=1, random_bg=True)
    r, db, img, T, n = run_gpu_forward(batch, renderer=renderer)
    im0 = db.image_views(img)[0].cpu().numpy()
    bg = batch.fparams[0, 17:20]
    np.testing.assert_array_equal(im0, np.broadcast_to(bg[:, None, None], im0.shape))
    assert (db.pix_views(T)[0] == 1).all() and (db.pix_views(n)[0] == 0).all()
    ores = oracle.forward(batch, splat="spec")
    st = compare_images(batch, ores, db, img, T, n)
    assert st["max_err"] <= 1e-4 and st["n_mismatch"] == 0
    tg = db.pack_images(synth.make_targets(batch, 2))
    out = renderer.step(db, tg, api.RGBA_LOSS_L1)
    assert out.pairs > 0
    assert float(db.models[0].grad_g0.abs().max()) == 0.0
    assert float(db.models[1].grad_g0.abs().max()) > 0.0


def test_everything_culled(renderer):
    m = synth.make_model(2, 800, 4)
    batch = synth.make_batch([m], [synth.Frame(0, 64, 64)], seed=2, random_bg=True)
    batch.fparams[0, :12] = synth.camera_params(64, 64, yaw=math.pi)[:12]  # facing away
    batch.fparams[0, 11] = -1.0  # the avatar sits behind the camera
    r, db, img, T, n = run_gpu_forward(batch, renderer=renderer)
    bg = batch.fparams[0, 17:20]
    im = db.image_views(img)[0].cpu().numpy()
    np.testing.assert_array_equal(im, np.broadcast_to(bg[:, None, None], im.shape))
    out = renderer.step(db, db.pack_images(synth.make_targets(batch, 3)), api.RGBA_LOSS_L1)
    assert out.pairs == 0
    assert float(db.models[0].grad_g0.abs().max()) == 0.0
    assert float(db.grad_psi.abs().max()) == 0.0


def test_near_plane_boundary_matches_the_oracle(renderer):
    """Gaussians exactly at, just in front of, just behind and well behind the near distance
    (camera depths 0.25, 0.2501, 0.24, 0.5 against near = 0.25, exact in binary32): the kernel
    culls the same ones as the oracle, bit for bit."""
    n = 4
    g0 = np.zeros((14, n), np.float32)
    g0[2] = [-0.75, -0.7499, -0.76, -0.5]
    g0[0] = [-0.01, 0.01, 0.0, 0.02]
    g0[3] = 1.0
    g0[7:10] = math.log(0.01)
    g0[10] = 1.0
    g0[11:14] = 0.5
    m = synth.Model(n=n, k=1, mask=synth.MASK_MEAN_SCALE_COLOR, g0=g0, dg=np.zeros((1, 9, n), np.float32))
    fp = synth.camera_params(64, 64, bg=(0.1, 0.2, 0.3))
    fp[16] = 0.25
    batch = synth.Batch(models=[m], frames=[synth.Frame(0, 64, 64)], psi=np.zeros((1, 1), np.float32),
                        fparams=fp[None, :], k_stride=1)
    r, db, img, T, nc = run_gpu_forward(batch, renderer=renderer)
    ores = oracle.forward(batch, do_render=False)
    compare_decisions(batch, ores, read_intermediates(r, db), db)
    rect = ores[0].rect
    kept = (rect[:, 2] > rect[:, 0]) & (rect[:, 3] > rect[:, 1])
    assert kept.tolist() == [False, True, False, True]


@pytest.mark.parametrize("W,H,tile", [(1, 1, (16, 16)), (17, 1, (16, 16)), (1, 33, (8, 32)),
                                      (129, 3, (8, 32))])
def test_tiny_and_ragged_images(renderer, W, H, tile):
    m = synth.make_model(3, 600, 4, radii=(0.3, 0.3, 0.2), log_scale_mu=math.log(0.05))
    batch = synth.make_batch([m], [synth.Frame(0, W, H)], seed=3, random_bg=True)
    r, db, img, T, n = run_gpu_forward(batch, tile=tile, renderer=renderer)
    ores = oracle.forward(batch, tile=tile, splat="spec")
    compare_decisions(batch, ores, read_intermediates(r, db), db, tile)
    st = compare_images(batch, ores, db, img, T, n)
    assert st["max_err"] <= 1e-4 and st["n_mismatch"] == 0


def test_largest_frame_and_one_beyond(renderer):
    m = synth.make_model(4, 3000, 4)
    batch = synth.make_batch([m], [synth.Frame(0, 4096, 4096)], seed=4)
    r, db, img, T, n = run_gpu_forward(batch, renderer=renderer)
    ores = oracle.forward(batch, do_render=False)
    compare_decisions(batch, ores, read_intermediates(r, db), db)
    # pixels of a 3x3 block of tiles around the centre
    mask = np.zeros(256 * 256, np.uint8)
    for ty in range(127, 130):
        mask[ty * 256 + 127: ty * 256 + 130] = 1
    ores = oracle.forward(batch, splat="spec", tile_masks={0: mask})
    pix = np.zeros((4096, 4096), bool)
    pix[127 * 16:130 * 16, 127 * 16:130 * 16] = True
    st = compare_images(batch, ores, db, img, T, n, tiles_only=[pix])
    assert st["max_err"] <= 1e-4 and st["n_mismatch"] == 0 and st["pixels"] == 48 * 48
    big = synth.make_batch([m], [synth.Frame(0, 4097, 16)], seed=4)
    with pytest.raises(api.RgbaError) as e:
        api.rgba_workspace_size(DeviceBatch(big, "cuda:0", grads=False).struct(), 0)
    assert e.value.code == api.RGBA_ERR_INVALID_ARG


def test_largest_k(renderer):
    """K = 64 blendshapes with the paper's blended set (10 channels): the preprocess stages
    14 + 640 rows per chunk."""
    m = synth.make_model(5, 1500, 64, mask=synth.MASK_PAPER)
    batch = synth.make_batch([m], [synth.Frame(0, 96, 96)] * 2, seed=5, jitter_deg=10)
    r, db, img, T, n = run_gpu_forward(batch, renderer=renderer)
    ores = oracle.forward(batch, splat="spec")
    compare_decisions(batch, ores, read_intermediates(r, db), db)
    st = compare_images(batch, ores, db, img, T, n)
    assert st["max_err"] <= 1e-4 and st["n_mismatch"] == 0


def test_pair_overflow_reports_and_retries(renderer):
    batch = synth.workload_batched(n=6_000, k=8, frames=2, res=128)
    db = DeviceBatch(batch, "cuda:0")
    tg = db.pack_images(synth.make_targets(batch, 6))
    small = torch.empty(api.rgba_workspace_size(db.struct(), 100), dtype=torch.uint8, device="cuda:0")
    s = torch.cuda.current_stream().cuda_stream
    rc, out = api.rgba_step(renderer.ctx, db.struct(), small.data_ptr(), small.numel(),
                            tg.data_ptr(), api.RGBA_LOSS_L1, None, s)
    assert rc == api.RGBA_ERR_CAPACITY and out.overflow == 1 and out.pairs_needed > 100
    big = torch.empty(api.rgba_workspace_size(db.struct(), out.pairs_needed), dtype=torch.uint8,
                      device="cuda:0")
    rc, out2 = api.rgba_step(renderer.ctx, db.struct(), big.data_ptr(), big.numel(),
                             tg.data_ptr(), api.RGBA_LOSS_L1, None, s)
    assert rc == api.RGBA_OK and out2.pairs == out.pairs_needed
    ref = Renderer(0).step(DeviceBatch(batch, "cuda:0"), tg, api.RGBA_LOSS_L1)
    assert abs(out2.loss - ref.loss) <= 1e-6 * ref.loss


def _bound_batch(seed=301, n=2000):
    import dataclasses
    mesh = synth.make_head_mesh(seed, 12, 24)
    m = synth.make_bound_model(seed, n, 4, mesh)
    fr = [synth.Frame(0, 96, 80, synth.frame_verts(mesh, seed, f)) for f in range(2)]
    return synth.make_batch([m], fr, seed, jitter_deg=10, random_bg=True), mesh, dataclasses


def test_degenerate_triangles_cull_like_the_oracle(renderer):
    """Gaussians on zero-area triangles (collapsed in the mesh) or on triangles with a
    degenerate UV map get a non-finite frame and are culled, the same way by both paths."""
    batch, mesh, dataclasses = _bound_batch()
    m = batch.models[0]
    faces = m.binding.faces
    hit = np.unique(m.binding.face_of[:200])
    uv = m.binding.face_uv.copy()
    uv[hit[::2], 4:6] = uv[hit[::2], 0:2]         # UV triangle collapsed onto a segment
    frames = []
    for fr in batch.frames:
        v = fr.verts.copy()
        for f in hit[1::2]:
            v[faces[f, 2]] = v[faces[f, 0]]           # a corner on top of another: zero area
        frames.append(synth.Frame(fr.model, fr.width, fr.height, v))
    mb = dataclasses.replace(m, binding=dataclasses.replace(m.binding, face_uv=uv))
    b2 = synth.Batch([mb], frames, batch.psi, batch.fparams, batch.k_stride)
    r, db, img, T, n = run_gpu_forward(b2, (16, 16), 64, renderer)
    ores = oracle.forward(b2, do_render=False)
    compare_decisions(b2, ores, read_intermediates(r, db), db)
    culled = (ores[0].rect[:200, 2] <= ores[0].rect[:200, 0])
    assert culled.sum() > 50


def test_binding_index_out_of_range_is_reported(renderer):
    """A face index past n_faces culls that Gaussian (the kernels check every index before
    reading) and rgba_step reports RGBA_ERR_INVALID_ARG."""
    batch, mesh, dataclasses = _bound_batch(seed=303)
    m = batch.models[0]
    face_of = m.binding.face_of.copy()
    face_of[5] = m.binding.faces.shape[0] + 7
    mb = dataclasses.replace(m, binding=dataclasses.replace(m.binding, face_of=face_of))
    b2 = synth.Batch([mb], batch.frames, batch.psi, batch.fparams, batch.k_stride)
    db = DeviceBatch(b2, "cuda:0")
    ws = renderer.ensure_workspace(db)
    tg = db.pack_images(synth.make_targets(b2, 3))
    img = torch.empty(3 * db.total_pix, device="cuda:0")
    with pytest.raises(api.RgbaError) as e:
        api.rgba_step(renderer.ctx, db.struct(), ws.data_ptr(), ws.numel(), tg.data_ptr(),
                      api.RGBA_LOSS_L1, img.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.code == api.RGBA_ERR_INVALID_ARG and "binding index" in str(e.value)
    rects = read_intermediates(renderer, db)["rects"]
    assert (rects[5] == 0).all() and (rects[db.rec_offsets[1] + 5] == 0).all()
