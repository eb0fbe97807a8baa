"""Pins of the oracle's tangent-space transform (Supp. "Gaussian Transformation", Alg. 1).

What pins it, none of it taken from the oracle itself: the defining relations of the tangent
frame (the triangle's edges are the UV differences applied to T and B; N is the unit normal),
the closed form for a right-angled isometric UV triangle (R = identity, or the rotation that
moved the triangle, from scipy), bit-exact agreement with the unbound path when every frame
is the identity, invariance of the projected splats under a rigid motion of the mesh paired
with the opposite motion of the camera, and central finite differences through the transform.
"""
import dataclasses

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2503_12886_gb300 import synth

from test_oracle_pins import _assert_fd, _run_fd


def _binding(verts, faces, face_uv, face_of, bary_rows):
    n = len(face_of)
    npad = synth.pad4(n)
    bary = np.zeros((3, npad), np.float32)
    bary[:, :n] = np.asarray(bary_rows, np.float32).T
    return synth.Binding(np.asarray(faces, np.int32), np.asarray(face_uv, np.float32),
                         np.asarray(face_of, np.int32), bary, len(verts))


def _random_triangles(rng, n):
    verts = rng.normal(size=(3 * n, 3)).astype(np.float32)
    faces = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    face_uv = rng.uniform(size=(n, 6)).astype(np.float32)
    bary = rng.dirichlet([1, 1, 1], size=n)
    return verts, faces, face_uv, bary


def test_tbn_satisfies_its_defining_relations():
    """e1 = du1 T + dv1 B and e2 = du2 T + dv2 B (T, B the derivatives of position along u and
    v over the triangle); N is unit, orthogonal to both edges and along e1 x e2; t is the
    barycentric point."""
    rng = np.random.default_rng(7)
    n = 200
    verts, faces, face_uv, bary = _random_triangles(rng, n)
    b = _binding(verts, faces, face_uv, np.arange(n), bary)
    out = oracle.tbn(b, verts, n)
    v = verts.astype(np.float64)
    uv = face_uv.astype(np.float64)
    for i in range(n):
        R = out[i, :9].reshape(3, 3)
        T, B, N = R[:, 0], R[:, 1], R[:, 2]
        a, p, q = v[faces[i]]
        e1, e2 = p - a, q - a
        du1, dv1 = uv[i, 2] - uv[i, 0], uv[i, 3] - uv[i, 1]
        du2, dv2 = uv[i, 4] - uv[i, 0], uv[i, 5] - uv[i, 1]
        scale = np.abs(du1 * T).max() + np.abs(dv1 * B).max() + np.abs(e1).max()
        np.testing.assert_allclose(du1 * T + dv1 * B, e1, rtol=0, atol=1e-12 * scale)
        scale = np.abs(du2 * T).max() + np.abs(dv2 * B).max() + np.abs(e2).max()
        np.testing.assert_allclose(du2 * T + dv2 * B, e2, rtol=0, atol=1e-12 * scale)
        assert abs(np.linalg.norm(N) - 1.0) < 1e-14
        assert abs(N @ e1) < 1e-13 * np.linalg.norm(e1) and abs(N @ e2) < 1e-13 * np.linalg.norm(e2)
        assert N @ np.cross(e1, e2) > 0
        bb = bary[i].astype(np.float32).astype(np.float64)
        np.testing.assert_allclose(out[i, 9:], bb[0] * a + bb[1] * p + bb[2] * q, rtol=0, atol=1e-14)


@pytest.mark.parametrize("rotated", [False, True])
def test_tbn_right_angled_isometric_triangle(rotated):
    """A right-angled triangle whose UV map is an isometry has R = [T B N] = I; moved by a
    rotation Q (scipy) and a translation, R = Q."""
    s = 0.25
    base = np.array([[0, 0, 0], [s, 0, 0], [0, s, 0]], np.float64)
    Q = Rotation.from_rotvec([0.3, -1.1, 0.7]).as_matrix() if rotated else np.eye(3)
    c = np.array([0.1, -0.2, 0.5]) if rotated else np.zeros(3)
    verts = (base @ Q.T + c).astype(np.float32)
    b = _binding(verts, [[0, 1, 2]], [[0, 0, s, 0, 0, s]], [0], [[0.2, 0.3, 0.5]])
    out = oracle.tbn(b, verts, 1)[0]
    np.testing.assert_allclose(out[:9].reshape(3, 3), Q, rtol=0, atol=2e-7)


def _identity_mesh_binding(n):
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    return verts, _binding(verts, [[0, 1, 2]], [[0, 0, 1, 0, 0, 1]], np.zeros(n, np.int32),
                           np.tile([1.0, 0.0, 0.0], (n, 1)))


@pytest.mark.parametrize("mask", [synth.MASK_MEAN_SCALE_COLOR, synth.MASK_PAPER])
def test_identity_frames_reproduce_the_unbound_path(mask):
    """Every Gaussian on a triangle whose tangent frame is the identity at the origin: the
    FP32 decisions are bit-identical and the FP64 splats and gradients equal the unbound ones."""
    m = synth.make_model(61, 3000, 6, mask=mask)
    verts, b = _identity_mesh_binding(m.n)
    mb = dataclasses.replace(m, binding=b)
    frames = [synth.Frame(0, 96, 80), synth.Frame(0, 64, 64)]
    plain = synth.make_batch([m], frames, seed=61, jitter_deg=15, random_bg=True)
    bound = synth.Batch([mb], [synth.Frame(0, f.width, f.height, verts) for f in frames],
                        plain.psi, plain.fparams, plain.k_stride)
    r0, r1 = oracle.forward(plain), oracle.forward(bound)
    targets = synth.make_targets(plain, 62)
    for a, c in zip(r0, r1):
        np.testing.assert_array_equal(a.rect, c.rect)
        np.testing.assert_array_equal(a.f32.view(np.uint32), c.f32.view(np.uint32))
        np.testing.assert_array_equal(a.lst, c.lst)
        np.testing.assert_allclose(c.rec, a.rec, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(c.img, a.img, rtol=0, atol=1e-12)
    _, g0 = oracle.loss(plain, r0, targets, "l1")
    _, g1 = oracle.loss(bound, r1, targets, "l1")
    pm0, dpsi0, _, _ = oracle.backward(plain, r0, g0)
    pm1, dpsi1, _, _ = oracle.backward(bound, r1, g1)
    for x, y in zip(pm0[0], pm1[0]):
        np.testing.assert_allclose(y, x, rtol=1e-9, atol=1e-12 * np.abs(x).max())
    np.testing.assert_allclose(dpsi1, dpsi0, rtol=1e-9, atol=1e-12 * np.abs(dpsi0).max())


def test_rigid_motion_of_mesh_and_camera_leaves_splats_unchanged():
    """Moving every frame mesh by x -> Q x + c and the camera by the same motion (view
    R_v Q^T, translation t_v - R_v Q^T c) maps T, B, N to Q T, Q B, Q N, so every screen mean,
    conic and depth is unchanged (FP64 path, scipy rotation)."""
    batch = synth.workload_tangent(seed=71, n=2000, k=6, frames=2, res=128)
    Q = Rotation.from_rotvec([0.4, 0.2, -0.5]).as_matrix()
    c = np.array([0.03, -0.05, 0.02])
    fr2, fp2 = [], batch.fparams.astype(np.float64).copy()
    for f, fr in enumerate(batch.frames):
        fr2.append(synth.Frame(fr.model, fr.width, fr.height,
                               (fr.verts.astype(np.float64) @ Q.T + c).astype(np.float32)))
        V = batch.fparams[f, :12].astype(np.float64).reshape(3, 4)
        Rv, tv = V[:, :3], V[:, 3]
        fp2[f, :12] = np.concatenate([Rv @ Q.T, (tv - Rv @ Q.T @ c)[:, None]], 1).reshape(12)
    m = batch.models[0]
    for f, fr in enumerate(batch.frames):
        bl = oracle.blend(m.g0, m.dg, batch.psi[f, :m.k], m.n, m.mask)
        rect = np.tile([0, 0, 1, 1], (m.n, 1)).astype(np.int32)
        a = oracle.project(bl, batch.fparams[f].astype(np.float64), m.n, fr.width, fr.height, rect,
                           oracle.tbn(m.binding, fr.verts, m.n))
        b_ = oracle.project(bl, fp2[f], m.n, fr.width, fr.height, rect,
                            oracle.tbn(m.binding, fr2[f].verts, m.n))
        # the moved mesh is stored in fp32 (vertex rounding ~1e-8 m): tolerances cover it
        np.testing.assert_allclose(b_[:, 0:2], a[:, 0:2], rtol=0, atol=2e-4)   # px
        np.testing.assert_allclose(b_[:, 9], a[:, 9], rtol=2e-6)               # depth
        sc = np.abs(a[:, [2, 4]]).max(1, keepdims=True)
        np.testing.assert_allclose(b_[:, 2:5] / sc, a[:, 2:5] / sc, rtol=0, atol=2e-4)


def test_decision_spec_tracks_fp64_projection_bound():
    """The FP32 spec with the tangent transform stays within a few ulp of the FP64 path."""
    batch = synth.workload_tangent(seed=73, n=4000, k=8, frames=1, res=512)
    r = oracle.forward(batch, do_render=False)[0]
    kept = (r.rect[:, 2] > r.rect[:, 0]) & (r.rect[:, 3] > r.rect[:, 1])
    assert kept.sum() > 3000
    f, d = r.f32[kept].astype(np.float64), r.rec[kept]
    np.testing.assert_allclose(f[:, 0:2], d[:, 0:2], rtol=0, atol=16 * 512 * 2.0 ** -24)
    scale = np.abs(d[:, [2, 4]]).max(1)
    for col in range(2, 5):
        assert (np.abs(f[:, col] - d[:, col]) <= 1e-4 * scale).all(), col
    np.testing.assert_allclose(f[:, 6], d[:, 9], rtol=2e-6)


def test_fd_gradients_through_the_tangent_transform():
    """Central differences for every parameter class of a bound avatar (tangent-space means,
    rotations and scales, opacity, colour, blendshape deltas, psi), two frames with different
    mesh expressions, L1 loss."""
    batch = synth.workload_tangent(seed=75, n=600, k=4, frames=2, res=64)
    _assert_fd(_run_fd(batch, "l1", per_class=5, seed=75))
