"""The three forms built on the per-frame path: differentiation (autograd.Function), batching
(uneven batches, CUDA-graph replay, autotuner) and serving (continuous batching)."""

import numpy as np
import pytest
import torch

import oracle
from paper_2503_12886_gb300 import api, synth
from paper_2503_12886_gb300.autograd import rasterize
from paper_2503_12886_gb300.batching import GraphStep, autotune
from paper_2503_12886_gb300.rasterizer import DeviceBatch, Renderer
from paper_2503_12886_gb300.serving import Server, requests_from_trace

from gpu_helpers import grad_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    import __graft_entry__
    __graft_entry__.build()
    r = Renderer(0)
    yield r
    r.close()


def _autograd_inputs(batch):
    dev = "cuda:0"
    models = []
    for m in batch.models:
        g0 = torch.from_numpy(m.g0).to(dev).requires_grad_(True)
        dg = torch.from_numpy(m.dg).to(dev).requires_grad_(True)
        models.append((m.n, m.k, m.mask, g0, dg))
    psi = torch.from_numpy(batch.psi).to(dev).requires_grad_(True)
    fp = torch.from_numpy(batch.fparams).to(dev)
    frames = [(f.model, f.width, f.height) for f in batch.frames]
    return frames, psi, fp, models


# -------------------------------------------------------------------------------- autograd

@pytest.mark.parametrize("mask", [synth.MASK_MEAN_SCALE_COLOR, synth.MASK_PAPER])
def test_autograd_matches_oracle_gradient(renderer, mask):
    batch = synth.workload_gradcheck(mask=mask)
    targets = synth.make_targets(batch, 31)
    frames, psi, fp, models = _autograd_inputs(batch)
    imgs = rasterize(renderer, frames, psi, fp, models)
    tg = torch.from_numpy(targets[0]).cuda()
    loss = 0.5 * ((imgs[0] - tg) ** 2).mean()
    loss.backward()
    ores = oracle.forward(batch, splat="spec")
    L, dls = oracle.loss(batch, ores, targets, "l2")
    per_model, dpsi, _, _ = oracle.backward(batch, ores, dls)
    assert abs(loss.item() - L) <= 1e-5 * L
    m = batch.models[0]
    g0, dg = models[0][3].grad, models[0][4].grad
    errs = {"g0": grad_error(g0.cpu().numpy()[:, :m.n], per_model[0][0][:, :m.n]),
            "dg": grad_error(dg.cpu().numpy()[..., :m.n].reshape(-1, m.n),
                             per_model[0][1][..., :m.n].reshape(-1, m.n)),
            "psi": grad_error(psi.grad.cpu().numpy(), dpsi, axis_rows=False)}
    assert max(errs.values()) <= 1.0, errs


def test_autograd_tangent_space_matches_oracle_gradient(renderer):
    """The autograd path with a tangent-space binding and a deformed mesh per frame: the
    oracle's dL/dimg (zero at the pixels it flags as ambiguous) back through rasterize() gives
    the oracle's gradients of G0, the blendshapes and the weights."""
    from gpu_helpers import oracle_fwd_bwd
    from paper_2503_12886_gb300.rasterizer import DeviceBinding
    from test_gpu_parity import tangent_batch
    batch = tangent_batch()
    targets = synth.make_targets(batch, 41)
    ores, L, dls, per_model, dpsi, _ = oracle_fwd_bwd(batch, targets, "l1", drop_flagged=True)
    frames, psi, fp, models = _autograd_inputs(batch)
    bindings = [DeviceBinding.of(m.binding, "cuda:0") for m in batch.models]
    verts = [torch.from_numpy(f.verts).cuda() for f in batch.frames]
    imgs = rasterize(renderer, frames, psi, fp, models, bindings=bindings, verts=verts)
    torch.autograd.backward(imgs, [torch.from_numpy(d.astype(np.float32)).cuda() for d in dls])
    m = batch.models[0]
    g0, dg = models[0][3].grad, models[0][4].grad
    errs = {"g0": grad_error(g0.cpu().numpy()[:, :m.n], per_model[0][0][:, :m.n]),
            "dg": grad_error(dg.cpu().numpy()[..., :m.n].reshape(-1, m.n),
                             per_model[0][1][..., :m.n].reshape(-1, m.n)),
            "psi": grad_error(psi.grad.cpu().numpy(), dpsi, axis_rows=False)}
    assert max(errs.values()) <= 1.0, errs


def test_autograd_central_differences(renderer):
    """dL/dtheta from the backward against central differences of the fp32 forward itself,
    for a weighted sum of pixels (steps sized for fp32, Gaussians with large gradients)."""
    batch = synth.workload_gradcheck()
    frames, psi, fp, models = _autograd_inputs(batch)
    w = torch.from_numpy(synth.make_targets(batch, 77)[0]).cuda()
    imgs = rasterize(renderer, frames, psi, fp, models)
    (imgs[0] * w).sum().backward()
    g0_grad = models[0][3].grad.clone()
    m = batch.models[0]
    rng = np.random.default_rng(3)
    checked = 0
    with torch.no_grad():
        for ch, h in [(0, 2e-4), (1, 2e-4), (7, 2e-3), (11, 2e-3), (10, 2e-3)]:
            row = g0_grad[ch, :m.n].abs()
            cand = torch.argsort(row, descending=True)[:40].cpu().numpy()
            for i in rng.choice(cand, 4, replace=False):
                g0 = models[0][3]
                orig = g0[ch, i].item()
                fds = []
                for hh in (h, h / 2):
                    vals = []
                    for sgn in (1, -1):
                        g0[ch, i] = orig + sgn * hh
                        im = rasterize(renderer, frames, psi, fp, models)[0]
                        vals.append(float((im * w).sum(dtype=torch.float64)))
                    fds.append((vals[0] - vals[1]) / (2 * hh))
                g0[ch, i] = orig
                an = float(g0_grad[ch, i])
                if abs(fds[0] - fds[1]) > 0.02 * abs(an) + 1e-3:
                    continue  # a compositing decision flipped inside the step: no derivative
                assert abs(fds[1] - an) <= 0.03 * abs(an) + 1e-3, (ch, i, fds, an)
                checked += 1
    assert checked >= 12


# -------------------------------------------------------------------------------- batching

def test_uneven_batch_frames_equal_frames_alone(renderer):
    """Each frame of an uneven batch (8 avatars, N 1k..4.5k, K 16/24/32, 256/512/1024 px) is
    bit-identical to the same frame rendered alone."""
    models = [synth.make_model(900 + a, 1000 + 500 * a, (16, 24, 32)[a % 3]) for a in range(8)]
    res = [256, 512, 1024, 256, 512, 256, 512, 256]
    batch = synth.make_batch(models, [synth.Frame(f, res[f], res[f]) for f in range(8)],
                             seed=901, jitter_deg=20, random_bg=True)
    db = DeviceBatch(batch, "cuda:0", grads=False)
    img, T, n = renderer.forward(db)
    imgs, Ts, ns = db.image_views(img), db.pix_views(T), db.pix_views(n)
    for f in range(8):
        one = synth.Batch([models[f]], [synth.Frame(0, res[f], res[f])], batch.psi[f:f + 1],
                          batch.fparams[f:f + 1], batch.k_stride)
        d1 = DeviceBatch(one, "cuda:0", grads=False)
        i1, T1, n1 = renderer.forward(d1)
        assert torch.equal(imgs[f], d1.image_views(i1)[0]), f
        assert torch.equal(Ts[f], d1.pix_views(T1)[0]) and torch.equal(ns[f], d1.pix_views(n1)[0])


def test_graph_replay_equals_eager(renderer):
    batch = synth.workload_batched(n=20_000, k=16, frames=4, res=256)
    tg_np = synth.make_targets(batch, 5)
    db = DeviceBatch(batch, "cuda:0")
    tg = db.pack_images(tg_np)
    img_e = torch.empty(3 * db.total_pix, device="cuda:0")
    out = renderer.step(db, tg, api.RGBA_LOSS_L1, img_e)
    g_e = db.models[0].grad_g0.clone()
    psi_e = db.grad_psi.clone()
    gs = GraphStep(Renderer(0), db, tg)
    for _ in range(3):
        loss, pairs = gs.replay()
    assert pairs == out.pairs
    # the loss is a sum of per-CTA fp32 partials whose tile sets depend on scheduling
    assert abs(loss - out.loss) <= 1e-6 * abs(out.loss)
    assert torch.equal(gs.img, img_e)
    n = batch.models[0].n
    assert grad_error(db.models[0].grad_g0.cpu().numpy()[:, :n], g_e.cpu().numpy()[:, :n]) <= 0.1
    assert grad_error(db.grad_psi.cpu().numpy(), psi_e.cpu().numpy(), axis_rows=False) <= 0.1


def test_graph_step_grows_workspace_on_overflow(renderer):
    batch = synth.workload_batched(n=5_000, k=8, frames=2, res=128)
    db = DeviceBatch(batch, "cuda:0")
    tg = db.pack_images(synth.make_targets(batch, 6))
    gs = GraphStep(Renderer(0), db, tg, headroom=0.5)  # capture with too few pairs
    loss, pairs = gs.replay()
    ref = Renderer(0).step(DeviceBatch(batch, "cuda:0"), tg, api.RGBA_LOSS_L1)
    assert pairs == ref.pairs and abs(loss - ref.loss) <= 1e-6 * ref.loss


def test_autotune_returns_a_candidate(renderer, tmp_path):
    models = [synth.make_model(950 + a, 2000 * (a + 1), (16, 24)[a % 2]) for a in range(2)]
    batch = synth.make_batch(models, [synth.Frame(f % 2, 256 * (1 + f % 2), 256 * (1 + f % 2))
                                      for f in range(4)], seed=951, random_bg=True)
    targets = synth.make_targets(batch, 9)
    cache = str(tmp_path / "tune.json")
    res = autotune(renderer, batch, targets, steps=2, cache_path=cache)
    assert res.tile in ((16, 16), (8, 32)) and res.smem_batch in (64, 128, 256)
    assert len(res.table) == 6 and res.ms == min(res.table.values())
    again = autotune(renderer, batch, targets, steps=2, cache_path=cache)
    assert again.tile == res.tile and again.smem_batch == res.smem_batch


# -------------------------------------------------------------------------------- serving

def _small_server(budget=40e9, slots=2):
    avatars = [synth.make_model(960 + a, 3000 + 700 * a, 8) for a in range(4)]
    return avatars, Server(avatars, 0, hbm_budget=budget, max_frames=8, slots=slots, max_res=512)


def _requests(avatars, n, seed=5):
    rng = np.random.default_rng(seed)
    trace = [(0.0005 * i, int(rng.integers(4)), int(rng.choice([256, 512])),
              (0.3 * rng.standard_normal(8)).astype(np.float32)) for i in range(n)]
    return requests_from_trace(trace, avatars, seed)


def test_serving_results_same_alone_and_in_the_mix():
    avatars, srv = _small_server()
    reqs = _requests(avatars, 24)
    st = srv.run(reqs, realtime=False, keep_images=True)
    assert st["served"] == 24 and st["batches"] < 24  # requests were batched together
    mixed = {q.rid: q.image for q in reqs}
    alone = _requests(avatars, 24)
    for q in alone:
        srv._launch(srv.slots[0], [q])
        srv.slots[0].event.synchronize()
        srv._finish(srv.slots[0], 0.0, True)
        assert np.abs(q.image - mixed[q.rid]).max() <= 1e-4, q.rid
    srv.close()


def test_serving_realtime_overlap_and_latency():
    avatars, srv = _small_server()
    reqs = _requests(avatars, 60)
    st = srv.run(reqs, realtime=True)
    assert st["served"] == 60 and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_serving_admission_budget_and_rejections():
    avatars, srv = _small_server(slots=2)
    srv.budget = srv.fixed_bytes + 30e6       # 30 MB for requests beside the slots' memory
    reqs = _requests(avatars, 10)
    reqs[3].avatar = 99                         # injected host-side failure: unknown avatar
    reqs[5].width = reqs[5].height = 4096       # larger than the whole budget
    st = srv.run(reqs, realtime=False)
    assert reqs[3].status == "rejected" and reqs[5].status == "rejected"
    done = [q for q in reqs if q.status == "done"]
    assert len(done) == 8 and st["served"] == 8 and st["regrowths"] == 0
    assert srv.used == pytest.approx(0.0, abs=1.0)
    srv.close()


def test_serving_slots_sized_from_measured_pairs():
    """The slot workspaces hold a full batch of the largest avatar at the largest resolution
    (pairs per Gaussian measured at start-up): a batch of max_frames such requests renders
    without a regrowth, and a budget smaller than the slots' own memory is refused."""
    avatars, srv = _small_server()
    assert srv.ppg > 1.0 and srv.pair_capacity >= srv.max_frames * max(m.n for m in avatars)
    big = int(np.argmax([m.n for m in avatars]))
    trace = [(0.0, big, 512, (0.3 * np.random.default_rng(i).standard_normal(8)).astype(np.float32))
             for i in range(srv.max_frames)]
    st = srv.run(requests_from_trace(trace, avatars, 7), realtime=False)
    assert st["served"] == srv.max_frames and st["regrowths"] == 0
    with pytest.raises(ValueError):
        Server(avatars, 0, hbm_budget=srv.fixed_bytes / 2, max_frames=8, slots=2, max_res=512)
    srv.close()
