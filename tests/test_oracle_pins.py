"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what pins it: a library routine (numpy einsum, scipy rotations, linear algebra),
a closed form of EWA splatting, an invariant of alpha compositing, a brute-force untiled
renderer on tiny inputs, or central finite differences. The method follows RGBAvatar Eq. 1
(blend), Supp. Sec. A.3 (activations after blending, 3DGS renderer) and Sec. 3.2 (compositing
and back-propagation of the image loss).
"""
import math
import struct

import numpy as np
import pytest

import oracle
from paper_2503_12886_gb300 import synth

ALPHA_MIN = 1.0 / 255.0


def one_gaussian_model(mean, quat, logscale, logit, color, k=1):
    g0 = np.zeros((14, 4), np.float32)
    g0[0:3, 0] = mean
    g0[3:7, 0] = quat
    g0[7:10, 0] = logscale
    g0[10, 0] = logit
    g0[11:14, 0] = color
    dg = np.zeros((k, 9, 4), np.float32)
    return synth.Model(n=1, k=k, mask=synth.MASK_MEAN_SCALE_COLOR, g0=g0, dg=dg)


def single_frame_batch(model, W, H, bg=(0.0, 0.0, 0.0)):
    fp = synth.camera_params(W, H, bg=bg)
    return synth.Batch(models=[model], frames=[synth.Frame(0, W, H)],
                       psi=np.zeros((1, model.k), np.float32), fparams=fp[None, :],
                       k_stride=model.k)


def f32(x):
    return float(np.float32(x))


# --------------------------------------------------------------------------------------------
# Decision-path exp: Cody-Waite + Taylor, checked against libm's exp rounded to binary32.

def test_exp_spec_within_one_ulp_of_libm():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(-87, 88, 4000), rng.uniform(-9, 1, 4000),
                         np.array([0.0, -1e-7, 1e-7, 0.5, -0.5, 1.0, -1.0, 10.0, -10.0])])
    xs = xs.astype(np.float32)
    exact = 0
    for x in xs:
        got = np.float32(oracle.exp_spec(float(x)))
        ref = np.float32(math.exp(float(x)))
        gi = struct.unpack("<i", struct.pack("<f", got))[0]
        ri = struct.unpack("<i", struct.pack("<f", ref))[0]
        assert abs(gi - ri) <= 1, (x, got, ref)
        exact += gi == ri
    assert exact / len(xs) > 0.9
    assert oracle.exp_spec(0.0) == 1.0
    assert oracle.exp_spec(-100.0) == 0.0
    assert math.isinf(oracle.exp_spec(100.0))


# --------------------------------------------------------------------------------------------
# Eq. 1 blend against numpy einsum; blend adjoint against einsum and the inner-product identity.

@pytest.mark.parametrize("mask", [synth.MASK_MEAN_SCALE_COLOR, synth.MASK_PAPER])
def test_blend_matches_einsum(mask):
    rng = np.random.default_rng(1)
    n, npad, k = 37, 40, 5
    chans = synth.blended_channels(mask)
    g0 = rng.normal(size=(14, npad))
    dg = rng.normal(size=(k, len(chans), npad))
    psi = rng.normal(size=k)
    got = oracle.blend(g0, dg, psi, n, mask)
    ref = g0.copy()
    ref[chans] += np.einsum("k,kan->an", psi, dg)
    np.testing.assert_allclose(got[:, :n], ref[:, :n], rtol=0, atol=1e-12)


def test_blend_bwd_is_adjoint():
    rng = np.random.default_rng(2)
    n, npad, k, nb = 29, 32, 6, 3
    mask = synth.MASK_PAPER
    chans = synth.blended_channels(mask)
    A = len(chans)
    g0 = rng.normal(size=(14, npad))
    dg = rng.normal(size=(k, A, npad))
    psi = rng.normal(size=(nb, k))
    dY = rng.normal(size=(nb, 14, npad))
    dY[:, :, n:] = 0
    dg0, ddg, dpsi = oracle.blend_bwd(g0.shape, dg, mask, n, psi, dY)
    # <dY, blend(g0', dg')> == <dg0, g0'> + <ddg, dg'> for the linear part in (g0, dg)
    g0p = rng.normal(size=(14, npad))
    dgp = rng.normal(size=(k, A, npad))
    lhs = sum((dY[b, :, :n] * oracle.blend(g0p, dgp, psi[b], n, mask)[:, :n]).sum()
              for b in range(nb))
    rhs = (dg0[:, :n] * g0p[:, :n]).sum() + (ddg[:, :, :n] * dgp[:, :, :n]).sum()
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))
    # dpsi[b][k] = sum over channels/Gaussians of dG_k * dY_b, by einsum
    ref = np.einsum("kan,ban->bk", dg[:, :, :n], dY[:, chans, :n])
    np.testing.assert_allclose(dpsi, ref, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------------------------
# EWA closed forms: one Gaussian seen by the default camera (view = identity, depth 1 m).

def pinhole(p, fx, fy, cx, cy):
    return np.array([fx * p[0] / p[2] + cx, fy * p[1] / p[2] + cy])


def jacobian_fd(p, fx, fy, cx, cy, h=1e-6):
    J = np.zeros((2, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        J[:, j] = (pinhole(p + e, fx, fy, cx, cy) - pinhole(p - e, fx, fy, cx, cy)) / (2 * h)
    return J


def closed_form_image(W, H, mean_px, cov2, o, color, bg, rect, TW=16, TH=16):
    """Image of one Gaussian: alpha = min(.99, o exp(-d^T cov2^-1 d / 2)) inside its tile
    rectangle, background elsewhere."""
    inv = np.linalg.inv(cov2)
    img = np.zeros((3, H, W))
    for py in range(H):
        for px in range(W):
            tx, ty = px // TW, py // TH
            val = np.asarray(bg, float)
            if rect[0] <= tx < rect[2] and rect[1] <= ty < rect[3]:
                d = np.array([px + 0.5, py + 0.5]) - mean_px
                a = min(0.99, o * math.exp(-0.5 * d @ inv @ d))
                if a >= ALPHA_MIN:
                    val = np.asarray(color) * a + (1 - a) * val
            img[:, py, px] = val
    return img


@pytest.mark.parametrize("z,near,kept", [(-0.75, 0.25, False), (-0.75, 0.2499, True),
                                         (-0.7499, 0.25, True), (-0.76, 0.25, False)])
def test_near_plane_culls_at_and_behind_it(z, near, kept):
    """The near-plane reading: a Gaussian whose camera depth p_z = z + 1 m (the default camera)
    is at or in front of the near distance is culled, one just past it is kept (0.75 and 0.25
    are exact in binary32, so p_z == near holds exactly in the first case)."""
    m = one_gaussian_model((0.0, 0.0, z), (1.0, 0.0, 0.0, 0.0), np.log((0.01, 0.01, 0.01)), 1.0,
                           (0.5, 0.5, 0.5))
    batch = single_frame_batch(m, 64, 64)
    batch.fparams[0, 16] = near
    rect = oracle.forward(batch, do_render=False)[0].rect[0]
    assert ((rect[2] > rect[0]) and (rect[3] > rect[1])) == kept


@pytest.mark.parametrize("case", ["isotropic_axis", "rotated_axis", "offaxis_general"])
def test_single_gaussian_closed_form(case):
    from scipy.spatial.transform import Rotation
    W, H = 80, 64
    o_logit, color, bg = 1.2, (0.3, 0.6, 0.9), (0.2, 0.1, 0.05)
    if case == "isotropic_axis":
        mean, s = (0.0, 0.0, 0.0), (0.02, 0.02, 0.02)
        q = (1.0, 0.0, 0.0, 0.0)
    elif case == "rotated_axis":
        th = math.radians(30)
        mean, s = (0.0, 0.0, 0.0), (0.03, 0.01, 0.02)
        q = (math.cos(th / 2), 0.0, 0.0, math.sin(th / 2))
    else:
        mean, s = (0.05, -0.03, 0.1), (0.03, 0.012, 0.02)
        q = (0.8, 0.2, -0.4, 0.3)
    m = one_gaussian_model(mean, q, np.log(s), o_logit, color)
    batch = single_frame_batch(m, W, H, bg)
    res = oracle.forward(batch)[0]
    fp = batch.fparams[0].astype(np.float64)
    fx, fy, cx, cy = fp[12], fp[13], fp[14], fp[15]
    x = m.g0[0:3, 0].astype(np.float64)
    p = x + np.array([0.0, 0.0, 1.0])
    qq = m.g0[3:7, 0].astype(np.float64)
    Rm = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()  # scipy is (x, y, z, w)
    sc = np.exp(m.g0[7:10, 0].astype(np.float64))
    Sig = Rm @ np.diag(sc ** 2) @ Rm.T
    J = jacobian_fd(p, fx, fy, cx, cy)
    cov2 = J @ Sig @ J.T + 0.3 * np.eye(2)
    mean_px = pinhole(p, fx, fy, cx, cy)
    o = 1 / (1 + math.exp(-float(np.float32(o_logit))))
    rect = res.rect[0]
    assert (rect[2] - rect[0]) * (rect[3] - rect[1]) > 0
    ref = closed_form_image(W, H, mean_px, cov2, o, color=m.g0[11:14, 0].astype(float),
                            bg=fp[17:20], rect=rect)
    np.testing.assert_allclose(res.img, ref, rtol=0, atol=2e-8)
    # the 3-sigma screen radius covers the largest eigen-direction
    lam = np.linalg.eigvalsh(cov2).max()
    r = res.f32[0, 5]
    assert 3 * math.sqrt(lam) <= r <= 3 * math.sqrt(lam + 0.32) + 1
    # one Gaussian: T_final is 1 - alpha where it contributes
    contributes = res.n_contrib == 1
    assert contributes.any()
    np.testing.assert_allclose((res.img[0] - fp[17] * res.T)[contributes],
                               (color[0] * (1 - res.T))[contributes], atol=1e-7)


def test_isotropic_is_rotation_invariant():
    W = H = 48
    imgs = []
    rng = np.random.default_rng(3)
    for _ in range(4):
        q = rng.normal(size=4)
        m = one_gaussian_model((0.01, 0.02, 0.0), q, np.log([0.02] * 3), 0.5, (1.0, 0.5, 0.2))
        imgs.append(oracle.forward(single_frame_batch(m, W, H))[0].img)
    for im in imgs[1:]:
        np.testing.assert_allclose(im, imgs[0], rtol=0, atol=1e-7)


# --------------------------------------------------------------------------------------------
# Compositing invariant: sum_i alpha_i T_i + T_final = 1 (white Gaussians, black background).

def test_weights_plus_final_transmittance_is_one():
    m = synth.make_model(7, 3000, 4)
    m.g0[11:14, :] = 1.0
    m.dg[:, 6:9, :] = 0.0  # colour deltas (blended channels 6..8 of the default mask)
    batch = synth.make_batch([m], [synth.Frame(0, 96, 80)], seed=7)
    r = oracle.forward(batch)[0]
    for c in range(3):
        np.testing.assert_allclose(r.img[c] + r.T, 1.0, rtol=0, atol=1e-12)
    assert (r.T < 0.5).sum() > 300  # the scene is dense enough for the check to bite
    assert r.T.min() >= 1e-4


# --------------------------------------------------------------------------------------------
# Brute force on tiny inputs: one global depth order, every Gaussian tested at every pixel with
# membership "pixel's tile lies in the Gaussian's rectangle"; equals the tiled renderer.

def depth_bits(x):
    return struct.unpack("<I", struct.pack("<f", float(x)))[0]


def brute_force_render(W, H, TW, TH, rec, rect, depth, bg):
    n = rect.shape[0]
    kept = [i for i in range(n) if (rect[i, 2] - rect[i, 0]) * (rect[i, 3] - rect[i, 1]) > 0]
    order = sorted(kept, key=lambda i: (depth_bits(depth[i]), i))
    img = np.zeros((3, H, W))
    T_out = np.zeros((H, W))
    n_out = np.zeros((H, W), np.int32)
    for py in range(H):
        for px in range(W):
            tx, ty = px // TW, py // TH
            T, Cc, last, pos = 1.0, np.zeros(3), 0, 0
            for i in order:
                if not (rect[i, 0] <= tx < rect[i, 2] and rect[i, 1] <= ty < rect[i, 3]):
                    continue
                pos += 1
                g = rec[i]
                dx, dy = px + 0.5 - g[0], py + 0.5 - g[1]
                pw = -0.5 * (g[2] * dx * dx + g[4] * dy * dy) - g[3] * dx * dy
                if pw > 0:
                    continue
                a = min(0.99, g[5] * math.exp(pw))
                if a < ALPHA_MIN:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                Cc += g[6:9] * a * T
                T *= 1 - a
                last = pos
            img[:, py, px] = Cc + T * np.asarray(bg)
            T_out[py, px] = T
            n_out[py, px] = last
    return img, T_out, n_out


@pytest.mark.parametrize("W,H,TW,TH", [(32, 32, 16, 16), (37, 29, 16, 16), (40, 40, 8, 32)])
def test_tiled_equals_brute_force(W, H, TW, TH):
    m = synth.make_model(11, 48, 3, radii=(0.35, 0.35, 0.2), log_scale_mu=math.log(0.04))
    batch = synth.make_batch([m], [synth.Frame(0, W, H)], seed=11)
    batch.fparams[0, 17:20] = (0.1, 0.2, 0.3)
    r = oracle.forward(batch, tile=(TW, TH))[0]
    img, T, n = brute_force_render(W, H, TW, TH, r.rec, r.rect, r.f32[:, 6],
                                  batch.fparams[0, 17:20].astype(np.float64))
    np.testing.assert_allclose(r.img, img, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.T, T, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(r.n_contrib, n)
    assert (r.n_contrib > 1).mean() > 0.2
    # and the per-tile lists equal a comparison sort of (tile, depth bits, index)
    tx = (W + TW - 1) // TW
    pairs = []
    for i in range(m.n):
        x0, y0, x1, y1 = r.rect[i]
        for y in range(y0, y1):
            for x in range(x0, x1):
                pairs.append((y * tx + x, depth_bits(r.f32[i, 6]), i))
    pairs.sort()
    assert [p[2] for p in pairs] == list(r.lst)
    counts = np.bincount([p[0] for p in pairs], minlength=len(r.tile_start) - 1)
    np.testing.assert_array_equal(np.diff(r.tile_start), counts)


# --------------------------------------------------------------------------------------------
# Central finite differences (h = 1e-5, FP64) for every parameter class.

def fd_setup(batch, targets, kind):
    params = {"g0": [m.g0.astype(np.float64) for m in batch.models],
              "dg": [m.dg.astype(np.float64) for m in batch.models],
              "psi": batch.psi.astype(np.float64)}

    def run(p):
        res = oracle.forward(batch, params=p)
        L, _ = oracle.loss(batch, res, targets, kind)
        return L, oracle.decision_signature(res)

    res = oracle.forward(batch, params=params)
    L0, grads = oracle.loss(batch, res, targets, kind)
    per_model, dpsi, _, _ = oracle.backward(batch, res, grads, params=params)
    return params, run, per_model, dpsi, oracle.decision_signature(res)


def check_fd(params, run, sig0, slot, idx, analytic, h=1e-5):
    import copy
    p_plus = copy.deepcopy(params)
    p_minus = copy.deepcopy(params)

    def at(p):
        if slot[0] == "psi":
            return p["psi"]
        return p[slot[0]][slot[1]]

    at(p_plus)[idx] += h
    at(p_minus)[idx] -= h
    Lp, sp = run(p_plus)
    Lm, sm = run(p_minus)
    if sp != sig0 or sm != sig0:
        return None  # a discrete decision changed inside [-h, h]: no derivative to compare
    return (Lp - Lm) / (2 * h), analytic


def _fd_classes(batch, per_model, dpsi, rng, per_class):
    m = batch.models[0]
    chans = synth.blended_channels(m.mask)
    dg0, ddg = per_model[0]
    # visible, contributing Gaussians: rank by |d loss / d colour|
    score = np.abs(dg0[11:14, :m.n]).sum(0)
    cand = np.argsort(-score)[: max(10, m.n // 4)]
    classes = {"mean": (0, 1, 2), "quat": (3, 4, 5, 6), "logscale": (7, 8, 9),
               "opacity": (10,), "color": (11, 12, 13)}
    out = []
    for name, chs in classes.items():
        for _ in range(per_class):
            i = int(rng.choice(cand))
            ch = int(rng.choice(chs))
            out.append((name, ("g0", 0), (ch, i), dg0[ch, i]))
    for _ in range(per_class):
        i = int(rng.choice(cand))
        a = int(rng.integers(len(chans)))
        kk = int(rng.integers(m.k))
        out.append(("basis", ("dg", 0), (kk, a, i), ddg[kk, a, i]))
    for _ in range(per_class):
        b = int(rng.integers(len(batch.frames)))
        kk = int(rng.integers(batch.models[batch.frames[b].model].k))
        out.append(("psi", ("psi",), (b, kk), dpsi[b, kk]))
    return out


def _run_fd(batch, kind, per_class, seed):
    targets = synth.make_targets(batch, seed)
    params, run, per_model, dpsi, sig0 = fd_setup(batch, targets, kind)
    rng = np.random.default_rng(seed)
    results = {}
    for name, slot, idx, an in _fd_classes(batch, per_model, dpsi, rng, per_class):
        r = check_fd(params, run, sig0, slot, idx, an)
        results.setdefault(name, []).append(r)
    return results


def _assert_fd(results, rel=2e-4, min_checked=0.5, fd_noise=5e-12):
    # fd_noise: rounding floor of a central difference of an O(0.1) loss at h = 1e-5
    for name, rs in results.items():
        ok = [r for r in rs if r is not None]
        assert len(ok) >= min_checked * len(rs), (name, len(ok), len(rs))
        scale = max(abs(a) for _, a in ok)
        assert scale > 100 * fd_noise, name
        for fd, an in ok:
            assert abs(fd - an) <= rel * abs(an) + fd_noise, (name, fd, an)


def test_fd_gradients_gradcheck_workload():
    """N=2,000, K=8, 64x64, L2 loss: every parameter class against central differences."""
    batch = synth.workload_gradcheck()
    _assert_fd(_run_fd(batch, "l2", per_class=6, seed=21))


def test_fd_gradients_multiframe_paper_mask_ragged():
    """Three frames of one avatar with the paper's blended set (mean, rotation, colour),
    a ragged 52x41 image, jittered cameras, random background and L1 loss."""
    m = synth.make_model(31, 400, 4, mask=synth.MASK_PAPER, log_scale_mu=math.log(6e-3))
    batch = synth.make_batch([m], [synth.Frame(0, 52, 41)] * 3, seed=31, jitter_deg=15,
                             random_bg=True)
    _assert_fd(_run_fd(batch, "l1", per_class=5, seed=31))


def test_fd_gradients_clamps_active():
    """Gaussians beyond 1.3x the half field of view (Jacobian clamp) and opaque ones (alpha
    clamp at 0.99) still match finite differences, i.e. the clamps pass the exact derivative."""
    n = 6
    g0 = np.zeros((14, 8), np.float32)
    g0[0, :n] = [0.75, -0.8, 0.0, 0.02, -0.03, 0.43]   # x: the first two sit outside 1.3 fov
    g0[1, :n] = [0.0, 0.1, 0.0, 0.01, 0.02, -0.46]
    g0[2, :n] = [0.2, 0.3, 0.0, 0.05, -0.05, 0.25]
    g0[3, :n] = 1.0
    g0[4:7, :n] = np.array([[0.1, 0.2, 0.0, 0.3, -0.2, 0.4]] * 3) * [[1], [-0.5], [0.7]]
    g0[7:10, :n] = np.log([[0.15, 0.2, 0.02, 0.01, 0.012, 0.2]] * 3)
    g0[10, :n] = [2.0, 1.0, 6.0, 5.0, 0.5, 1.5]         # o = 0.9975 saturates the clamp
    g0[11:14, :n] = np.array([[0.9, 0.1, 0.5, 0.3, 0.7, 0.2]] * 3)
    dg = (np.random.default_rng(5).normal(size=(2, 9, 8)) * 1e-3).astype(np.float32)
    dg[:, :, n:] = 0
    m = synth.Model(n=n, k=2, mask=synth.MASK_MEAN_SCALE_COLOR, g0=g0, dg=dg)
    batch = synth.make_batch([m], [synth.Frame(0, 40, 40)], seed=5, random_bg=True)
    res = oracle.forward(batch)[0]
    fpx = batch.fparams[0]
    lim = 1.3 * 20 / fpx[12]
    assert (res.rect[:2, 2] > res.rect[:2, 0]).all()  # both clamped Gaussians reach the image
    assert abs(0.75 / 1.2) > lim and abs(-0.8 / 1.3) > lim  # ... with their Jacobian clamped
    assert (res.n_contrib > 0).any()
    targets = synth.make_targets(batch, 5)
    params, run, per_model, dpsi, sig0 = fd_setup(batch, targets, "l2")
    dg0, ddg = per_model[0]
    checked = 0
    for i in range(n):
        for ch in range(14):
            r = check_fd(params, run, sig0, ("g0", 0), (ch, i), dg0[ch, i])
            if r is None:
                continue
            fd, an = r
            checked += 1
            assert abs(fd - an) <= 2e-4 * abs(an) + 1e-9, (i, ch, fd, an)
    assert checked > 60


# --------------------------------------------------------------------------------------------
# The FP32 decision spec tracks the FP64 projection it stands in for.

@pytest.mark.parametrize("res", [128, 1024])
def test_decision_spec_tracks_fp64_projection(res):
    m = synth.make_model(13, 4000, 8)
    batch = synth.make_batch([m], [synth.Frame(0, res, res)], seed=13, jitter_deg=20)
    r = oracle.forward(batch, do_render=False)[0]
    kept = (r.rect[:, 2] > r.rect[:, 0]) & (r.rect[:, 3] > r.rect[:, 1])
    assert kept.sum() > 3000
    f, d = r.f32[kept].astype(np.float64), r.rec[kept]
    np.testing.assert_allclose(f[:, 0:2], d[:, 0:2], rtol=0, atol=4 * res * 2.0 ** -24 * 2)
    for c in range(2, 5):  # conic a, b, c relative to the conic's scale
        scale = np.abs(d[:, [2, 4]]).max(1)
        assert (np.abs(f[:, c] - d[:, c]) <= 1e-5 * scale).all(), c
    np.testing.assert_allclose(f[:, 6], d[:, 9], rtol=1e-6)
    np.testing.assert_allclose(f[:, 7], d[:, 5], rtol=0, atol=1e-6)
