"""Fused Adam (librgba rgba_adam) against the FP64 definition, and inside a captured step."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_12886_gb300 import synth
from paper_2503_12886_gb300.batching import GraphStep
from paper_2503_12886_gb300.optim import PAPER_DELTA_SCALE, PAPER_LR, Adam
from paper_2503_12886_gb300.rasterizer import DeviceBatch, Renderer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    import __graft_entry__
    __graft_entry__.build()
    r = Renderer(0)
    yield r
    r.close()


def test_adam_matches_definition(renderer):
    models = [synth.make_model(70 + a, 1000 + 13 * a, 4 + a, mask=(synth.MASK_PAPER if a else synth.MASK_MEAN_SCALE_COLOR))
              for a in range(2)]
    batch = synth.make_batch(models, [synth.Frame(0, 64, 64), synth.Frame(1, 64, 64)], seed=70)
    db = DeviceBatch(batch, "cuda:0")
    rng = np.random.default_rng(0)
    opt = Adam(renderer, db)
    ref = [(m.g0.astype(np.float64), m.dg.astype(np.float64)) for m in batch.models]
    mom = [[np.zeros_like(a) for a in r] for r in ref]
    vel = [[np.zeros_like(a) for a in r] for r in ref]
    for t in range(1, 4):
        for mi, m in enumerate(db.models):
            g0 = rng.normal(size=m.g0.shape).astype(np.float32)
            dg = rng.normal(size=m.dg.shape).astype(np.float32)
            g0[:, m.n:] = 0
            dg[..., m.n:] = 0
            m.grad_g0.copy_(torch.from_numpy(g0))
            m.grad_dg.copy_(torch.from_numpy(dg))
            # the kernel receives learning rates and betas as fp32: the definition takes the same
            lr0 = np.array(PAPER_LR, np.float32).astype(np.float64)[:, None]
            chans = synth.blended_channels(m.mask)
            lrd = np.array([np.float32(PAPER_LR[c] * PAPER_DELTA_SCALE[c]) for c in chans],
                           np.float64)[None, :, None]
            b = dict(beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)),
                     eps=float(np.float32(1e-8)))
            ref[mi] = list(ref[mi])
            ref[mi][0], mom[mi][0], vel[mi][0] = oracle.adam(ref[mi][0], g0.astype(np.float64),
                                                             mom[mi][0], vel[mi][0], lr0, t, **b)
            ref[mi][1], mom[mi][1], vel[mi][1] = oracle.adam(ref[mi][1], dg.astype(np.float64),
                                                             mom[mi][1], vel[mi][1], lrd, t, **b)
        opt.step()
        torch.cuda.synchronize()
        for mi, m in enumerate(db.models):
            np.testing.assert_allclose(m.g0.cpu().numpy(), ref[mi][0], rtol=1e-6, atol=1e-6)
            np.testing.assert_allclose(m.dg.cpu().numpy(), ref[mi][1], rtol=1e-6, atol=1e-6)
    assert int(opt.step_dev.item()) == 3


def test_training_graph_with_adam_lowers_the_loss(renderer):
    """A captured step with the Adam tail: replaying it trains (the loss falls) and the step
    count advances on the device."""
    batch = synth.workload_batched(n=8_000, k=8, frames=4, res=128)
    db = DeviceBatch(batch, "cuda:0")
    tg = db.pack_images(synth.make_targets(batch, 8))
    opt = Adam(renderer, db)
    gs = GraphStep(renderer, db, tg, optimizer=opt)
    losses = [gs.replay()[0] for _ in range(30)]
    assert losses[-1] < losses[0] * 0.98, losses[::6]
    assert int(opt.step_dev.item()) >= 30
