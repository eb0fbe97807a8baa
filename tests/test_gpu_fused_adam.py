"""rgba_step_adam_async (the Adam update fused into the projection/blend backward) against the
separate calls rgba_step_async + rgba_adam, and its fallback for batches it cannot fuse.

The compositing backward sums 2-D gradients with atomics, so two runs differ in the last bits
of each gradient; the comparison is therefore on the update itself: after one step from zero
moments every parameter moves by lr g / (|g| + eps') (Kingma & Ba), which the two paths must
agree on wherever |g| is not within rounding noise of 0 (elements with |g| below 1e-4 of the
tensor's largest are skipped, where the sign can flip): the parameters to 1e-6 absolute (far
below any learning rate, so a wrong rate, index or moment fails), the first moments to 1e-3
relative. After three steps all parameters agree to 1e-5 absolute."""
import numpy as np
import pytest
import torch

from paper_2503_12886_gb300 import api, synth
from paper_2503_12886_gb300.optim import Adam
from paper_2503_12886_gb300.rasterizer import DeviceBatch, Renderer, stream_ptr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    import __graft_entry__
    __graft_entry__.build()
    r = Renderer(0)
    yield r
    r.close()


def two_models():
    models = [synth.make_model(110, 6000, 8, mask=synth.MASK_MEAN_SCALE_COLOR),
              synth.make_model(111, 5000, 6, mask=synth.MASK_PAPER)]
    fr = [synth.Frame(0, 128, 96), synth.Frame(1, 96, 128), synth.Frame(0, 96, 96), synth.Frame(1, 128, 128)]
    return synth.make_batch(models, fr, seed=110, jitter_deg=15, random_bg=True)


def seventeen_frames():
    """One model rendered by 17 frames: more than one frame group, so the update is not fused."""
    m = synth.make_model(112, 3000, 4)
    return synth.make_batch([m], [synth.Frame(0, 64, 64) for _ in range(17)], seed=112, jitter_deg=20)


def _workspace(db, pairs=None):
    b = db.struct()
    cap = pairs if pairs is not None else 8 * db.total_rec + 4096
    return torch.empty(api.rgba_workspace_size(b, cap), dtype=torch.uint8, device="cuda:0")


def _counters(db, ws):
    lay = api.rgba_workspace_layout(db.struct(), ws.numel())
    raw = ws[lay.counters: lay.counters + 24].cpu().numpy()
    u = raw[:16].view(np.uint32)
    return int(u[1]), float(raw[16:24].view(np.float64)[0])


def _separate(r, db, opt, ws, tg, img):
    api.rgba_step_async(r.ctx, db.struct(), ws.data_ptr(), ws.numel(), tg.data_ptr(), api.RGBA_LOSS_L1,
                        img.data_ptr(), stream_ptr())
    opt.step()


@pytest.mark.parametrize("make", [two_models, seventeen_frames])
def test_fused_step_matches_separate_calls(renderer, make):
    batch = make()
    targets = synth.make_targets(batch, 3)
    dbA, dbB = DeviceBatch(batch, "cuda:0"), DeviceBatch(batch, "cuda:0")
    optA, optB = Adam(renderer, dbA), Adam(renderer, dbB)
    tgA, tgB = dbA.pack_images(targets), dbB.pack_images(targets)
    wsA, wsB = _workspace(dbA), _workspace(dbB)
    imgA = torch.empty(3 * dbA.total_pix, device="cuda:0")
    imgB = torch.empty_like(imgA)
    p0 = [(m.g0.clone(), m.dg.clone()) for m in dbA.models]
    for step in range(3):
        _separate(renderer, dbA, optA, wsA, tgA, imgA)
        optB.train_step(wsB, tgB, api.RGBA_LOSS_L1, imgB)
        torch.cuda.synchronize()
        (ovA, lossA), (ovB, lossB) = _counters(dbA, wsA), _counters(dbB, wsB)
        assert ovA == 0 and ovB == 0
        assert abs(lossA - lossB) <= 1e-5 * abs(lossA)
        if step == 0:  # same parameters: same images, and weight gradients up to summation order
            torch.testing.assert_close(imgB, imgA, rtol=0, atol=1e-5)
            torch.testing.assert_close(dbB.grad_psi, dbA.grad_psi, rtol=1e-3, atol=1e-7)
            for mi, (mA, mB) in enumerate(zip(dbA.models, dbB.models)):
                for pA, pB, g, momA, momB in ((mA.g0, mB.g0, mA.grad_g0, optA.m[mi][0], optB.m[mi][0]),
                                              (mA.dg, mB.dg, mA.grad_dg, optA.m[mi][1], optB.m[mi][1])):
                    sig = g.abs() > 1e-4 * g.abs().max()
                    assert int(sig.sum()) > 0
                    # a wrong learning rate, index or moment moves a parameter by ~lr >= 4e-5
                    torch.testing.assert_close(pB[sig], pA[sig], rtol=0, atol=1e-6)
                    assert not torch.equal(pB, p0[mi][0] if pB is mB.g0 else p0[mi][1])
                    # first moment (1 - b1) g, up to the gradients' summation order
                    torch.testing.assert_close(momB[sig], momA[sig], rtol=1e-3, atol=1e-6 * float(g.abs().max()))
    for mA, mB in zip(dbA.models, dbB.models):
        torch.testing.assert_close(mB.g0, mA.g0, rtol=0, atol=1e-5)
        torch.testing.assert_close(mB.dg, mA.dg, rtol=0, atol=1e-5)
    assert int(optA.step_dev.item()) == int(optB.step_dev.item()) == 3


def test_fused_step_needs_no_gradient_arrays(renderer):
    """A batch that fuses runs without grad_g0 / grad_dg; one that cannot fuse refuses them."""
    batch = two_models()
    db = DeviceBatch(batch, "cuda:0", grads=False)
    opt = Adam(renderer, db)
    ws = _workspace(db)
    tg = db.pack_images(synth.make_targets(batch, 4))
    g0 = [m.g0.clone() for m in db.models]
    opt.train_step(ws, tg)
    torch.cuda.synchronize()
    assert int(opt.step_dev.item()) == 1
    assert all(not torch.equal(m.g0, a) for m, a in zip(db.models, g0))
    b17 = seventeen_frames()
    db17 = DeviceBatch(b17, "cuda:0", grads=False)
    opt17 = Adam(renderer, db17)
    with pytest.raises(api.RgbaError) as e:
        opt17.train_step(_workspace(db17), db17.pack_images(synth.make_targets(b17, 5)))
    assert e.value.code == api.RGBA_ERR_INVALID_ARG


def test_graph_step_with_fused_update_trains(renderer):
    """GraphStep(fused=True) captures rgba_step_adam_async: replays advance the step count and
    fit the targets (images of a reference avatar)."""
    from paper_2503_12886_gb300.batching import GraphStep
    batch = two_models()
    refs = [synth.reference_avatar(m, 130 + j) for j, m in enumerate(batch.models)]
    rb = synth.Batch(refs, batch.frames, batch.psi, batch.fparams, batch.k_stride)
    tg, _, _ = renderer.forward(DeviceBatch(rb, "cuda:0", grads=False))
    tg = tg.clone()
    db = DeviceBatch(batch, "cuda:0", grads=False)
    opt = Adam(renderer, db)
    gs = GraphStep(renderer, db, tg, optimizer=opt, headroom=1.6, fused=True)
    losses = [gs.replay()[0] for _ in range(30)]
    assert int(opt.step_dev.item()) == 30
    assert losses[-1] < 0.7 * losses[0], losses
