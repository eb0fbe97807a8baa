"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no arithmetic of the method: it only draws random numbers and lays them out.
Both the FP64 oracle and the CUDA library consume exactly these arrays (the oracle reads the
float32 values widened to float64), so parity compares the two implementations on identical
inputs.

Random numbers: a counter-based splitmix64 stream (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), one stream per (seed, stream id), uniform doubles
from the top 53 bits, normals by the Box-Muller transform.

Workload shapes follow the paper's avatars: fewer than 100k Gaussians per head (Sec. 1), about
60k at UV resolution 256 (Supp. Sec. A.3), 512x512 frames, K reduced blendshapes (Sec. 3.1,
Eq. 1). The per-attribute distributions are the synthetic recipe stated with each function.

Channel layout of one Gaussian (14 fp32 channels, planar [14][n_pad]):
    0..2  mean x, y, z (world, metres)
    3..6  rotation quaternion (w, x, y, z), unnormalised
    7..9  log-scale per axis
    10    opacity logit
    11..13 RGB colour (identity activation)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NCH = 14
CH_MEAN = (0, 1, 2)
CH_QUAT = (3, 4, 5, 6)
CH_LOGSCALE = (7, 8, 9)
CH_OPACITY = 10
CH_COLOR = (11, 12, 13)

# Blended-channel masks (bit c set: channel c carries blendshape deltas).
# MASK_MEAN_SCALE_COLOR: mean, log-scale and colour are blended (the synthetic workloads).
# MASK_PAPER: position, rotation and colour are blended, scale and opacity are not (Supp. A.3).
MASK_MEAN_SCALE_COLOR = sum(1 << c for c in CH_MEAN + CH_LOGSCALE + CH_COLOR)
MASK_PAPER = sum(1 << c for c in CH_MEAN + CH_QUAT + CH_COLOR)

# Per-frame parameter block [FP_STRIDE] fp32: view matrix (3x4 row-major world->camera,
# OpenCV axes: x right, y down, z forward), fx, fy, cx, cy, near plane, background RGB.
FP_STRIDE = 20
FP_VIEW = 0
FP_FX, FP_FY, FP_CX, FP_CY, FP_NEAR = 12, 13, 14, 15, 16
FP_BG = 17

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser on uint64 arrays (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based generator: value j of stream (seed, sid) is mix64(base + (j+1)*golden)."""

    def __init__(self, seed: int, sid: int):
        with np.errstate(over="ignore"):
            key = np.uint64((seed * 0x100000001B3 + sid * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF)
            self.base = _mix64(np.array([key], dtype=np.uint64))[0]
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        j = np.arange(self.pos + 1, self.pos + 1 + n, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            return _mix64(self.base + j * _GOLDEN)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller (two uniforms per pair, cosine branch only)."""
        u1 = 1.0 - self.uniform(n)  # (0, 1]
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def pad4(n: int) -> int:
    return max(4, (n + 3) // 4 * 4)


def blended_channels(mask: int) -> list[int]:
    return [c for c in range(NCH) if (mask >> c) & 1]


@dataclass
class Binding:
    """Tangent-space binding of a model's Gaussians to a triangle mesh with a UV atlas (Supp.
    "Gaussian Transformation", Alg. 1). Each Gaussian stays on one triangle, at the barycentric
    point of its UV sample; its mean (channels 0..2) and rotation live in that triangle's
    tangent space (u, v, normal)."""
    faces: np.ndarray    # int32 [F][3] vertex indices
    face_uv: np.ndarray  # float32 [F][6] (u, v) of corners 0, 1, 2
    face_of: np.ndarray  # int32 [n] triangle of each Gaussian
    bary: np.ndarray     # float32 [3][n_pad] barycentric weights of each Gaussian's UV sample
    n_verts: int


@dataclass
class Model:
    """One avatar: base Gaussians G0 and K blendshape deltas (Eq. 1)."""
    n: int
    k: int
    mask: int
    g0: np.ndarray      # float32 [14][n_pad]
    dg: np.ndarray      # float32 [k][A][n_pad]
    binding: Binding | None = None

    @property
    def n_pad(self) -> int:
        return self.g0.shape[1]

    @property
    def a(self) -> int:
        return len(blended_channels(self.mask))


@dataclass
class Frame:
    model: int
    width: int
    height: int
    verts: np.ndarray | None = None  # float32 [V][3]: this frame's deformed mesh (bound models)


@dataclass
class Batch:
    """B frames, each rendering one model with its own weights psi_b and camera (Sec. 3.2)."""
    models: list[Model]
    frames: list[Frame]
    psi: np.ndarray       # float32 [B][k_stride]
    fparams: np.ndarray   # float32 [B][FP_STRIDE]
    k_stride: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_frames(self) -> int:
        return len(self.frames)


def make_model(seed: int, n: int, k: int, mask: int = MASK_MEAN_SCALE_COLOR,
               radii=(0.09, 0.12, 0.10), log_scale_mu=math.log(3e-3), log_scale_sd=0.3,
               sd_dmean=1e-3, sd_dlogscale=1e-3, sd_dcolor=0.05, sd_dquat=1e-2) -> Model:
    """Synthetic head avatar.

    Means uniform in the ellipsoid with the given radii (rejection sampling from its bounding
    box), log-scales N(log 3e-3, 0.3) per axis, rotations uniform (normalised 4-D normal),
    opacity logits N(0, 1), colours U[0,1]. Deltas N(0, 1e-3) on mean and log-scale, N(0, 0.05)
    on colour, N(0, 1e-2) on the quaternion when it is blended; opacity is never blended.
    """
    npad = pad4(n)
    g0 = np.zeros((NCH, npad), np.float64)
    st = Stream(seed, 1)
    pts = np.zeros((0, 3))
    r = np.asarray(radii, np.float64)
    while pts.shape[0] < n:
        m = max(64, 2 * (n - pts.shape[0]))
        cand = (st.uniform(3 * m).reshape(m, 3) * 2.0 - 1.0)
        keep = cand[(cand ** 2).sum(1) <= 1.0]
        pts = np.concatenate([pts, keep * r], 0)
    g0[0:3, :n] = pts[:n].T
    q = Stream(seed, 3).normal(4 * n).reshape(n, 4)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    g0[3:7, :n] = q.T
    g0[7:10, :n] = (log_scale_mu + log_scale_sd * Stream(seed, 2).normal(3 * n)).reshape(n, 3).T
    g0[10, :n] = Stream(seed, 4).normal(n)
    g0[11:14, :n] = Stream(seed, 5).uniform(3 * n).reshape(n, 3).T
    chans = blended_channels(mask)
    dg = np.zeros((k, len(chans), npad), np.float64)
    sd = {}
    for c in CH_MEAN:
        sd[c] = sd_dmean
    for c in CH_QUAT:
        sd[c] = sd_dquat
    for c in CH_LOGSCALE:
        sd[c] = sd_dlogscale
    for c in CH_COLOR:
        sd[c] = sd_dcolor
    sd[CH_OPACITY] = 0.0
    dst = Stream(seed, 6)
    for a, c in enumerate(chans):
        dg[:, a, :n] = sd[c] * dst.normal(k * n).reshape(k, n)
    return Model(n=n, k=k, mask=mask, g0=g0.astype(np.float32), dg=dg.astype(np.float32))


def _rot_y(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def _rot_x(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def camera_params(width: int, height: int, yaw: float = 0.0, pitch: float = 0.0,
                  bg=(0.0, 0.0, 0.0), f128: float = 150.0, dist: float = 1.0,
                  near: float = 0.2) -> np.ndarray:
    """Per-frame block: a pinhole camera orbiting the origin at `dist` metres.

    With yaw = pitch = 0 the camera sits at z = -dist looking at the origin (view rotation I,
    translation (0, 0, dist)). The orbit rotates the camera centre by R_y(yaw) R_x(pitch).
    fx = fy = f128 * width / 128, principal point at the image centre.
    """
    ro = _rot_y(yaw) @ _rot_x(pitch)
    rv = ro.T
    t = np.array([0.0, 0.0, dist])
    fp = np.zeros(FP_STRIDE, np.float64)
    fp[0:12] = np.concatenate([rv, t[:, None]], 1).reshape(12)
    f = f128 * width / 128.0
    fp[FP_FX] = f
    fp[FP_FY] = f128 * width / 128.0
    fp[FP_CX] = width / 2.0
    fp[FP_CY] = height / 2.0
    fp[FP_NEAR] = near
    fp[FP_BG:FP_BG + 3] = bg
    return fp.astype(np.float32)


def make_batch(models: list[Model], frames: list[Frame], seed: int, psi_sd: float = 0.3,
               jitter_deg: float = 0.0, random_bg: bool = False) -> Batch:
    """Weights psi ~ N(0, psi_sd), optional yaw/pitch jitter U[-j, j] degrees, optional U[0,1] bg."""
    b = len(frames)
    ks = max([m.k for m in models] + [1])
    psi = np.zeros((b, ks), np.float32)
    pst = Stream(seed, 10)
    jst = Stream(seed, 13)
    bst = Stream(seed, 12)
    fps = np.zeros((b, FP_STRIDE), np.float32)
    for f, fr in enumerate(frames):
        k = models[fr.model].k
        psi[f, :k] = (psi_sd * pst.normal(k)).astype(np.float32)
        yaw = pitch = 0.0
        if jitter_deg > 0:
            yp = (jst.uniform(2) * 2.0 - 1.0) * math.radians(jitter_deg)
            yaw, pitch = float(yp[0]), float(yp[1])
        bg = tuple(bst.uniform(3)) if random_bg else (0.0, 0.0, 0.0)
        fps[f] = camera_params(fr.width, fr.height, yaw, pitch, bg)
    return Batch(models=models, frames=frames, psi=psi, fparams=fps, k_stride=ks)


def reference_avatar(model: Model, seed: int) -> Model:
    """The avatar a training benchmark fits: `model` with colours perturbed by N(0, 0.1) and
    means by N(0, 1 mm) (its images are rendered and used as targets)."""
    g0 = model.g0.copy()
    n = model.n
    g0[11:14, :n] += (0.1 * Stream(seed, 40).normal(3 * n)).reshape(3, n).astype(np.float32)
    g0[0:3, :n] += (1e-3 * Stream(seed, 41).normal(3 * n)).reshape(3, n).astype(np.float32)
    return Model(n=model.n, k=model.k, mask=model.mask, g0=g0, dg=model.dg.copy(), binding=model.binding)


def make_targets(batch: Batch, seed: int) -> list[np.ndarray]:
    """Seeded U[0,1] target images, one float32 [3][H][W] array per frame."""
    st = Stream(seed, 11)
    out = []
    for fr in batch.frames:
        out.append(st.uniform(3 * fr.height * fr.width).reshape(3, fr.height, fr.width)
                   .astype(np.float32))
    return out


# ---------------------------------------------------------------------------------------------
# The five workloads (synthetic stand-ins for the paper's INSTA / GaussianBlendShapes captures).

@dataclass
class Mesh:
    """A head mesh with a UV atlas and an expression basis (stands in for the tracked 3DMM mesh
    of the paper, Sec. 3.1 and Supp. "Gaussian Transformation")."""
    verts: np.ndarray    # float32 [V][3] neutral shape
    faces: np.ndarray    # int32 [F][3]
    face_uv: np.ndarray  # float32 [F][6]
    dverts: np.ndarray   # float32 [E][V][3] expression displacement basis


def make_head_mesh(seed: int, n_lat: int = 48, n_lon: int = 96, radii=(0.09, 0.12, 0.10),
                   n_expr: int = 10, amp: float = 4e-3, theta=(0.06 * math.pi, 0.94 * math.pi)) -> Mesh:
    """Ellipsoid head mesh (radii as the volume avatars) with a latitude-longitude UV atlas.

    Vertex rows at polar angles theta_i in [theta0, theta1] from the +y axis, n_lon + 1 columns
    at azimuth phi_j = 2 pi j / n_lon (the seam column is duplicated so UVs stay continuous):
    position (rx sin th cos ph, ry cos th, rz sin th sin ph), UV (phi / 2 pi, (th - th0) /
    (th1 - th0)); two triangles per grid quad. 48 x 96 gives 4,656 vertices and 9,024 triangles
    (the FLAME head has 5,023 and 9,976). Expression basis: E smooth normal displacements
    amp cos(k_e . x + phase_e) n(x), wave vectors with |k| U[20, 60] rad/m, random direction.
    """
    rx, ry, rz = radii
    th = theta[0] + (theta[1] - theta[0]) * np.arange(n_lat) / (n_lat - 1)
    ph = 2.0 * math.pi * np.arange(n_lon + 1) / n_lon
    T, P = np.meshgrid(th, ph, indexing="ij")
    pos = np.stack([rx * np.sin(T) * np.cos(P), ry * np.cos(T), rz * np.sin(T) * np.sin(P)], -1)
    uv = np.stack([P / (2.0 * math.pi), (T - theta[0]) / (theta[1] - theta[0])], -1)
    pos = pos.reshape(-1, 3)
    uv = uv.reshape(-1, 2)
    cols = n_lon + 1
    faces = []
    for i in range(n_lat - 1):
        for j in range(n_lon):
            a = i * cols + j
            b, c = a + 1, a + cols
            faces.append((a, c, b))
            faces.append((b, c, c + 1))
    faces = np.asarray(faces, np.int32)
    face_uv = uv[faces].reshape(-1, 6)
    nrm = pos / np.asarray(radii) ** 2
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    st = Stream(seed, 40)
    d = st.normal(3 * n_expr).reshape(n_expr, 3)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    kmag = 20.0 + 40.0 * st.uniform(n_expr)
    phase = 2.0 * math.pi * st.uniform(n_expr)
    dverts = np.stack([amp * np.cos(pos @ (kmag[e] * d[e]) + phase[e])[:, None] * nrm
                       for e in range(n_expr)])
    return Mesh(pos.astype(np.float32), faces, face_uv.astype(np.float32), dverts.astype(np.float32))


def frame_verts(mesh: Mesh, seed: int, frame: int) -> np.ndarray:
    """A frame's deformed mesh: neutral + sum_e w_e dverts_e with w ~ N(0, 1) per frame."""
    w = Stream(seed, 1000 + frame).normal(mesh.dverts.shape[0])
    return (mesh.verts.astype(np.float64) +
            np.tensordot(w, mesh.dverts.astype(np.float64), 1)).astype(np.float32)


def make_bound_model(seed: int, n: int, k: int, mesh: Mesh, mask: int = MASK_MEAN_SCALE_COLOR,
                     sd_mean=(2e-3, 3e-3, 1e-3), log_scale_mu=math.log(4e-3), log_scale_sd=0.3) -> Model:
    """Synthetic avatar in the tangent space of `mesh` (Sec. 3.1 "Initialization": positions
    sampled across the UV map). Each Gaussian takes a uniformly random triangle (all triangles
    of the grid atlas have the same UV area, so this is uniform over the UV map) and a uniform
    point in it (barycentric weights 1 - sqrt(r1), sqrt(r1)(1 - r2), sqrt(r1) r2). Tangent-space
    mean offsets N(0, sd_mean) in (u, v, normal) units, log-scales N(log 4e-3, 0.3) in the same
    units; rotations, opacity, colours and deltas as make_model."""
    m = make_model(seed, n, k, mask=mask, log_scale_mu=log_scale_mu, log_scale_sd=log_scale_sd)
    npad = m.n_pad
    st = Stream(seed, 50)
    face_of = (st.uniform(n) * mesh.faces.shape[0]).astype(np.int32)
    r1, r2 = st.uniform(n), st.uniform(n)
    sq = np.sqrt(r1)
    bary = np.zeros((3, npad), np.float32)
    bary[0, :n] = 1.0 - sq
    bary[1, :n] = sq * (1.0 - r2)
    bary[2, :n] = sq * r2
    g0 = m.g0.copy()
    off = Stream(seed, 51).normal(3 * n).reshape(3, n)
    for c in range(3):
        g0[c, :n] = (sd_mean[c] * off[c]).astype(np.float32)
    b = Binding(mesh.faces, mesh.face_uv, face_of, bary, mesh.verts.shape[0])
    return Model(n=n, k=k, mask=mask, g0=g0, dg=m.dg, binding=b)


def workload_single(seed: int = 1000) -> Batch:
    """N=10,000, K=20, one 128x128 frame, fx=fy=150, camera at z=-1 m, bg 0."""
    m = make_model(seed, 10_000, 20)
    return make_batch([m], [Frame(0, 128, 128)], seed)


def workload_gradcheck(seed: int = 2000, mask: int = MASK_MEAN_SCALE_COLOR) -> Batch:
    """N=2,000, K=8, one 64x64 frame (fx=fy=75), bg 0."""
    m = make_model(seed, 2_000, 8, mask=mask)
    return make_batch([m], [Frame(0, 64, 64)], seed)


def workload_batched(seed: int = 3000, n: int = 60_000, k: int = 32, frames: int = 16,
                     res: int = 512) -> Batch:
    """N=60,000, K=32, B=16 frames at 512x512, yaw/pitch jitter U[-20,20] deg, random bg."""
    m = make_model(seed, n, k)
    return make_batch([m], [Frame(0, res, res) for _ in range(frames)], seed,
                      jitter_deg=20.0, random_bg=True)


def workload_tangent(seed: int = 6000, n: int = 60_000, k: int = 32, frames: int = 16,
                     res: int = 512, n_lat: int = 48, n_lon: int = 96) -> Batch:
    """The batched workload in tangent space: N Gaussians bound to a head mesh (48 x 96 grid:
    9,024 triangles) whose expression changes per frame; K blendshapes, B frames, yaw/pitch
    jitter U[-20,20] deg, random bg."""
    mesh = make_head_mesh(seed, n_lat, n_lon)
    m = make_bound_model(seed, n, k, mesh)
    fr = [Frame(0, res, res, frame_verts(mesh, seed, f)) for f in range(frames)]
    return make_batch([m], fr, seed, jitter_deg=20.0, random_bg=True)


UNEVEN_N = (20_000, 35_000, 50_000, 65_000, 80_000, 90_000, 95_000, 100_000)
UNEVEN_K = (16, 24, 32)
UNEVEN_RES = (256, 512, 1024)


def workload_uneven(seed: int = 4000, frames: int = 64, scale: float = 1.0) -> Batch:
    """8 avatars with N in UNEVEN_N (times `scale`), K cycling 16/24/32, 64 frames: frame f
    renders avatar f mod 8 at resolution UNEVEN_RES[(f // 8) mod 3]."""
    models = [make_model(seed + 17 * a, max(1, int(UNEVEN_N[a] * scale)), UNEVEN_K[a % 3])
              for a in range(8)]
    fr = [Frame(f % 8, UNEVEN_RES[(f // 8) % 3], UNEVEN_RES[(f // 8) % 3])
          for f in range(frames)]
    return make_batch(models, fr, seed, jitter_deg=20.0, random_bg=True)


def serving_avatars(seed: int = 5000, count: int = 32, k: int = 32, n_lo: int = 30_000,
                    n_hi: int = 100_000) -> list[Model]:
    """Resident avatars with N ~ U[n_lo, n_hi], K=32."""
    st = Stream(seed, 20)
    ns = (n_lo + st.uniform(count) * (n_hi - n_lo)).astype(np.int64)
    return [make_model(seed + 31 * a, int(ns[a]), k) for a in range(count)]


def serving_requests(seed: int = 5000, rate_hz: float = 2000.0, duration_s: float = 10.0,
                     n_avatars: int = 32, k: int = 32, frac_1024: float = 0.2):
    """Poisson arrivals: list of (t_arrival_s, avatar, res, psi[k] float32)."""
    st = Stream(seed, 21)
    n = int(rate_hz * duration_s * 1.2) + 16
    gaps = -np.log(1.0 - st.uniform(n)) / rate_hz
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    av = (st.uniform(len(t)) * n_avatars).astype(np.int64)
    res = np.where(st.uniform(len(t)) < frac_1024, 1024, 512)
    psi = (0.3 * Stream(seed, 22).normal(len(t) * k)).reshape(len(t), k).astype(np.float32)
    return [(float(t[i]), int(av[i]), int(res[i]), psi[i]) for i in range(len(t))]
