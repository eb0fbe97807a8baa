"""Pins of the oracle's loss (Sec. 3.2 "Loss Function": L1; 1/2 L2 for the gradient-check
workload) and of its normalisation (a mean over each frame's 3 H W values, then a mean over the
frames of the batch).

What pins it: with the near plane beyond the avatar every Gaussian is culled and each frame's
image is its background, so against a constant target the loss has a closed form per frame,
and frames of different sizes weigh the same; dL/dimg is sign(d) / (3 H W B) for L1 and
d / (3 H W B) for L2."""
import numpy as np
import pytest

import oracle
from paper_2503_12886_gb300 import synth


def _background_batch():
    m = synth.make_model(31, 400, 4)
    fr = [synth.Frame(0, 16, 8), synth.Frame(0, 32, 32)]
    batch = synth.make_batch([m], fr, seed=31, random_bg=True)
    for b, f in enumerate(fr):  # a near plane behind the avatar: every Gaussian is culled
        bg = batch.fparams[b, 17:20].copy()
        batch.fparams[b] = synth.camera_params(f.width, f.height, bg=tuple(bg), near=5.0)
    return batch


@pytest.mark.parametrize("kind", ["l1", "l2"])
def test_loss_of_background_images_against_constant_targets(kind):
    batch = _background_batch()
    res = oracle.forward(batch)
    t = [0.25, 0.8]
    targets = [np.full((3, f.height, f.width), t[b], np.float32) for b, f in enumerate(batch.frames)]
    L, grads = oracle.loss(batch, res, targets, kind)
    per_frame = []
    for b, f in enumerate(batch.frames):
        bg = batch.fparams[b, 17:20].astype(np.float64)
        np.testing.assert_array_equal(res[b].img, np.broadcast_to(bg[:, None, None], res[b].img.shape))
        d = bg - np.float64(np.float32(t[b]))
        per_frame.append(np.abs(d).mean() if kind == "l1" else 0.5 * (d * d).mean())
        npx = 3 * f.width * f.height
        want = (np.sign(d) if kind == "l1" else d)[:, None, None] / (npx * len(batch.frames))
        np.testing.assert_allclose(grads[b], np.broadcast_to(want, grads[b].shape), rtol=1e-15, atol=0)
    np.testing.assert_allclose(L, np.mean(per_frame), rtol=1e-14, atol=0)
