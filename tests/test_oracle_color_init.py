"""Pins of the oracle's colour initialisation (Sec. 3.2 "Initialization", Eq. 3, delta = 0.1).

What pins it: the weighted mean of a constant image is that constant; the weighted mean of a
linear ramp under a weight symmetric about a point is the ramp's value there (a centred
isotropic Gaussian, whose tile rectangle and alpha cutoff are symmetric too); the threshold
admits exactly the Gaussians whose total weight exceeds delta; a done flag is never revisited;
the sums over the frames of a batch are the sums of the per-frame sums.
"""
import numpy as np

import oracle
from paper_2503_12886_gb300 import synth

from test_oracle_pins import one_gaussian_model, single_frame_batch


def _const_targets(batch, rgb):
    return [np.broadcast_to(np.asarray(rgb, np.float32)[:, None, None],
                            (3, f.height, f.width)).copy() for f in batch.frames]


def test_constant_target_gives_its_colour():
    batch = synth.workload_gradcheck()
    res = oracle.forward(batch)
    targets = _const_targets(batch, (0.2, 0.5, 0.9))
    col, done, W = oracle.color_init(batch, res, targets, [np.zeros(batch.models[0].n, bool)])[0]
    assert done.sum() > 100
    np.testing.assert_allclose(col[:, done], np.array([[0.2], [0.5], [0.9]], np.float32).astype(np.float64)
                               .repeat(done.sum(), 1), rtol=0, atol=1e-12)
    assert np.isnan(col[:, ~done]).all()
    assert (W[done] > 0.1).all() and (W[~done] <= 0.1).all()


def test_linear_ramp_under_a_centred_symmetric_gaussian():
    """An isotropic Gaussian on the optical axis of a 32x32 frame: its screen mean is the
    image centre (16, 16), pixel centres and its 2x2-tile rectangle are symmetric about it, so
    the weighted mean of I = a + b x + c y is a + 16 b + 16 c."""
    m = one_gaussian_model([0, 0, 1.5], [1, 0, 0, 0], np.log([0.02] * 3), 3.0, [0.5] * 3)
    batch = single_frame_batch(m, 32, 32)
    res = oracle.forward(batch)
    assert res[0].rect[0].tolist() == [0, 0, 2, 2]
    ys, xs = np.mgrid[0:32, 0:32] + 0.5
    a = np.array([0.1, 0.7, 0.3])
    bx = np.array([0.01, -0.02, 0.005])
    cy = np.array([-0.004, 0.003, 0.02])
    tg = (a[:, None, None] + bx[:, None, None] * xs + cy[:, None, None] * ys).astype(np.float32)
    col, done, W = oracle.color_init(batch, res, [tg], [np.zeros(1, bool)])[0]
    assert done[0] and W[0] > 1.0
    ref = a + 16.0 * bx + 16.0 * cy
    # the target is stored in fp32: each pixel carries up to 2^-24 relative rounding
    np.testing.assert_allclose(col[:, 0], ref, rtol=0, atol=3e-8)


def test_threshold_and_done_flags():
    batch = synth.workload_gradcheck()
    res = oracle.forward(batch)
    targets = synth.make_targets(batch, 5)
    n = batch.models[0].n
    _, done1, W = oracle.color_init(batch, res, targets, [np.zeros(n, bool)])[0]
    assert ((W > 0.1) == done1).all()
    lo = np.sort(W[W > 0])[len(W[W > 0]) // 4]  # a threshold that admits three quarters
    _, done_lo, _ = oracle.color_init(batch, res, targets, [np.zeros(n, bool)], delta=lo)[0]
    assert ((W > lo) == done_lo).all() and done_lo.sum() > done1.sum()
    # already initialised Gaussians keep their colour
    col2, done2, _ = oracle.color_init(batch, res, targets, [done1.copy()])[0]
    assert (done2 == done1).all() and np.isnan(col2).all()


def test_batch_sums_are_sums_over_frames():
    m = synth.make_model(41, 1500, 4)
    fr = [synth.Frame(0, 64, 48), synth.Frame(0, 48, 64), synth.Frame(0, 64, 64)]
    batch = synth.make_batch([m], fr, seed=41, jitter_deg=15, random_bg=True)
    res = oracle.forward(batch)
    targets = synth.make_targets(batch, 42)
    acc = sum(oracle.color_accum(f.width, f.height, 16, 16, r.rec, r.tile_start, r.lst, t, m.n)
              for f, r, t in zip(fr, res, targets))
    col, done, W = oracle.color_init(batch, res, targets, [np.zeros(m.n, bool)])[0]
    np.testing.assert_allclose(W, acc[:, 0], rtol=1e-15, atol=0)
    np.testing.assert_allclose(col[:, done], (acc[done, 1:] / acc[done, :1]).T, rtol=1e-15)


def test_weights_are_alpha_times_transmittance():
    """Two isotropic Gaussians with the same screen footprint on the optical axis, one behind
    the other (sigma / z equal): at every pixel the front one has weight alpha and the back one
    alpha (1 - alpha), with alpha = o exp(-rho^2 / 2 s^2), s^2 = (f sigma / z)^2 + 0.3 (the EWA
    closed form), so W_front = sum alpha and W_back = sum alpha (1 - alpha) over the pixels with
    alpha >= 1/255."""
    g0 = np.zeros((14, 4), np.float32)
    z = np.array([1.5, 2.0])          # world z; the camera sits at z = -1, so depths 2.5, 3.0
    sig = 0.12 * (z + 1.0) / 2.5
    g0[2, :2] = z
    g0[3, :2] = 1.0
    g0[7:10, :2] = np.log(sig)[None, :]
    g0[10, :2] = 0.4
    g0[11:14, :2] = 0.5
    m = synth.Model(n=2, k=1, mask=synth.MASK_MEAN_SCALE_COLOR, g0=g0, dg=np.zeros((1, 9, 4), np.float32))
    batch = single_frame_batch(m, 32, 32)
    res = oracle.forward(batch)
    targets = _const_targets(batch, (1.0, 1.0, 1.0))
    _, _, W = oracle.color_init(batch, res, targets, [np.zeros(2, bool)])[0]
    f = 150.0 * 32 / 128
    s2 = (f * 0.12 / 2.5) ** 2 + 0.3
    ys, xs = np.mgrid[0:32, 0:32] + 0.5
    rho2 = (xs - 16.0) ** 2 + (ys - 16.0) ** 2
    o = 1.0 / (1.0 + np.exp(-np.float64(np.float32(0.4))))
    al = np.minimum(0.99, o * np.exp(-rho2 / (2 * s2)))
    al = np.where(al >= 1 / 255, al, 0.0)
    assert W[0] > 5.0
    np.testing.assert_allclose(W[0], al.sum(), rtol=1e-6)
    np.testing.assert_allclose(W[1], (al * (1 - al)).sum(), rtol=1e-6)
