"""The frame-sharded data-parallel step on the GPU, with its ranks run one after the other on
one device: each rank's rgba_step over its share of the frames, with the loss averaged over the
whole batch (rgba_batch.loss_frames), writes its share of dG0 and ddG into a flat buffer laid out
by sharding.attach_flat_grads; the sum of the ranks' buffers (what the step's all-reduce computes)
equals the gradient of one step over the whole batch, their losses sum to its loss and their dpsi
rows are its rows (Sec. 3.2: the batch loss is the mean over the batch's frames). The whole-batch
step itself is held to the oracle by the parity tests."""
import numpy as np
import pytest
import torch

from paper_2503_12886_gb300 import api, sharding, synth
from paper_2503_12886_gb300.rasterizer import DeviceBatch, Renderer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    import __graft_entry__
    __graft_entry__.build()
    r = Renderer(0)
    yield r
    r.close()


def _step(renderer, batch, targets, loss_frames):
    db = DeviceBatch(batch, "cuda:0")
    db.loss_frames = loss_frames
    flat = sharding.attach_flat_grads(db.models)
    out = renderer.step(db, db.pack_images(targets), api.RGBA_LOSS_L1)
    torch.cuda.synchronize()
    return flat.clone(), out.loss, db.grad_psi.clone()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_steps_sum_to_the_whole_batch(renderer, world):
    ms = [synth.make_model(71, 5000, 8), synth.make_model(72, 4000, 6, mask=synth.MASK_PAPER)]
    fr = [synth.Frame(f % 2, 96 + 16 * (f % 3), 80) for f in range(7)]
    batch = synth.make_batch(ms, fr, seed=73, jitter_deg=20, random_bg=True)
    targets = synth.make_targets(batch, 74)
    B = len(fr)
    full, loss_full, psi_full = _step(renderer, batch, targets, 0)
    total, loss_sum, psi_rows = torch.zeros_like(full), 0.0, []
    for rank in range(world):
        sh = sharding.shard(B, world, rank)
        sub = synth.Batch(batch.models, batch.frames[sh.start:sh.stop], batch.psi[sh.start:sh.stop],
                          batch.fparams[sh.start:sh.stop], batch.k_stride)
        flat, loss, psi = _step(renderer, sub, targets[sh.start:sh.stop], B)
        total += flat
        loss_sum += loss
        psi_rows.append(psi)
    # the ranks' sums meet in another order than the whole batch's fp32 atomics: equal up to it
    scale = float(full.abs().max())
    assert scale > 0 and float((total - full).abs().max()) <= 1e-5 * scale
    assert abs(loss_sum - loss_full) <= 1e-5 * loss_full
    psi = torch.cat(psi_rows, 0)
    assert float((psi - psi_full).abs().max()) <= 1e-5 * float(psi_full.abs().max())

