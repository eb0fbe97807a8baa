"""FP64 CPU oracle of the batch-parallel Gaussian blendshape rasterizer (RGBAvatar, Sec. 3.2).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the bench's CPU-baseline leg,
never by the product path. The arithmetic lives in oracle.c (plain C, FP64, single-threaded);
this module composes its steps per frame in the paper's order and computes the image loss in
numpy. It shares nothing with the CUDA path except the seeded inputs of the synth module.

    forward:  Eq. 1 blend -> activations (Supp. A.3) -> EWA projection -> tile binning and
              depth sort -> front-to-back compositing (3DGS, as cited in Supp. A.3)
    loss:     L1 (Sec. 3.2 "Loss Function") or L2 (1/2 squared error), mean per frame, averaged
              over the frames of the batch
    backward: exact reverse of every step above down to G0, the blendshapes and psi

Every discrete decision that the GPU must reproduce bit for bit (cull, tile rectangle, depth key)
comes from the FP32 decision spec in oracle.c; all continuous values are FP64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4


def build(force: bool = False) -> str:
    """Compile oracle.c with contraction off (the FP32 decision spec needs unfused ops)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            i32, u32, f64 = C.c_int, C.c_uint, C.c_double
            L.orc_blend.argtypes = [i32, i32, i32, u32, P, P, P, P]
            L.orc_blend_bwd.argtypes = [i32, i32, i32, u32, P, i32, P, P, P, P, P]
            L.orc_exp_spec.argtypes = [C.c_float]
            L.orc_exp_spec.restype = C.c_float
            L.orc_decide.argtypes = [i32, i32, i32, u32, P, P, P, P, i32, i32, i32, i32, P, P,
                                     P, P, P, P, P]
            L.orc_project.argtypes = [i32, i32, P, P, i32, i32, P, P, P]
            L.orc_project_bwd.argtypes = [i32, i32, P, P, i32, i32, P, P, P, P]
            L.orc_tbn_all.argtypes = [i32, i32, P, P, P, P, P, P]
            L.orc_color_accum.argtypes = [i32, i32, i32, i32, P, P, P, P, P]
            L.orc_bin.argtypes = [i32, P, P, i32, i32, P, P]
            L.orc_bin.restype = C.c_int64
            L.orc_render.argtypes = [i32, i32, i32, i32, P, P, P, P, P, f64, f64, P, P, P, P, P]
            L.orc_render.restype = C.c_uint64
            L.orc_render_bwd.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P]
            _lib = L
    return _lib


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def exp_spec(x: float) -> float:
    """The decision-path exp (Cody-Waite reduction + degree-7 Taylor), fp32 in and out."""
    return float(lib().orc_exp_spec(C.c_float(np.float32(x))))


def blend(g0: np.ndarray, dg: np.ndarray, psi: np.ndarray, n: int, mask: int) -> np.ndarray:
    """Eq. 1 in FP64: [14][n_pad] blended channels for one weight vector psi[k]."""
    g0 = np.ascontiguousarray(g0, np.float64)
    dg = np.ascontiguousarray(dg, np.float64)
    psi = np.ascontiguousarray(psi, np.float64)
    out = np.zeros_like(g0)
    lib().orc_blend(n, g0.shape[1], dg.shape[0], mask, _p(g0), _p(dg), _p(psi), _p(out))
    return out


def _bind_args(binding, verts):
    if binding is None:
        return [None] * 5, None
    arrs = [np.ascontiguousarray(binding.faces, np.int32), np.ascontiguousarray(binding.face_uv, np.float32),
            np.ascontiguousarray(binding.face_of, np.int32), np.ascontiguousarray(binding.bary, np.float32),
            np.ascontiguousarray(verts, np.float32)]
    return [_p(a) for a in arrs], arrs


def tbn(binding, verts, n):
    """FP64 TBN matrix and barycentric point per Gaussian (Alg. 1): [n][12] = R row-major
    (columns T, B, N), then t."""
    ptrs, keep = _bind_args(binding, verts)
    out = np.zeros((n, 12), np.float64)
    lib().orc_tbn_all(n, binding.bary.shape[1], *ptrs, _p(out))
    return out


def decide(g0, dg, psi, fp, n, mask, W, H, TW=16, TH=16, binding=None, verts=None):
    """FP32 decision spec per Gaussian: rect[n][4] (int32) and f32[n][8] =
    (u, v, conic a, b, c, radius, depth, opacity). With a binding the mean and covariance are
    first mapped from tangent space by the frame mesh `verts`."""
    ptrs, keep = _bind_args(binding, verts)
    g0 = np.ascontiguousarray(g0, np.float32)
    dg = np.ascontiguousarray(dg, np.float32)
    psi = np.ascontiguousarray(psi, np.float32)
    fp = np.ascontiguousarray(fp, np.float32)
    rect = np.zeros((n, 4), np.int32)
    f32 = np.zeros((n, 8), np.float32)
    lib().orc_decide(n, g0.shape[1], dg.shape[0], mask, _p(g0), _p(dg), _p(psi), _p(fp), W, H,
                     TW, TH, _p(rect), _p(f32), *ptrs)
    return rect, f32


def project(blended, fp, n, W, H, rect, tbn64=None):
    """FP64 render records [n][12] = (u, v, conic a, b, c, opacity, r, g, b, depth, 0, 0);
    tbn64 ([n][12] from tbn()) maps bound Gaussians from tangent space."""
    out = np.zeros((n, 12), np.float64)
    fp64 = np.ascontiguousarray(fp, np.float64)
    lib().orc_project(n, blended.shape[1], _p(blended), _p(fp64), W, H, _p(rect), _p(out),
                      _p(tbn64))
    return out


def project_bwd(blended, fp, n, W, H, rect, grad2d, tbn64=None):
    dG = np.zeros_like(blended)
    fp64 = np.ascontiguousarray(fp, np.float64)
    g2 = np.ascontiguousarray(grad2d, np.float64)
    lib().orc_project_bwd(n, blended.shape[1], _p(blended), _p(fp64), W, H, _p(rect), _p(g2),
                          _p(dG), _p(tbn64))
    return dG


def bin_sort(rect, depth, tiles_x, tiles_y):
    """Per-tile lists ordered by (fp32 depth bits, index): (tile_start[nt+1], list[P])."""
    n = rect.shape[0]
    depth = np.ascontiguousarray(depth, np.float32)
    ts = np.zeros(tiles_x * tiles_y + 1, np.int32)
    total = lib().orc_bin(n, _p(rect), _p(depth), tiles_x, tiles_y, _p(ts), None)
    lst = np.zeros(max(total, 1), np.int32)
    lib().orc_bin(n, _p(rect), _p(depth), tiles_x, tiles_y, _p(ts), _p(lst))
    return ts, lst[:total]


def render(W, H, TW, TH, rec, tile_start, lst, bg, tile_mask=None, eps=1e-5, eps_t=1e-4):
    img = np.zeros((3, H, W), np.float64)
    T = np.ones((H, W), np.float64)
    nc = np.zeros((H, W), np.int32)
    flags = np.zeros((H, W), np.uint8)
    stats = np.zeros(2, np.float64)
    bg = np.ascontiguousarray(bg, np.float64)
    lst = np.ascontiguousarray(lst if len(lst) else np.zeros(1, np.int32), np.int32)
    tm = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8)
    h = lib().orc_render(W, H, TW, TH, _p(rec), _p(tile_start), _p(lst), _p(bg), _p(tm), eps,
                         eps_t, _p(img), _p(T), _p(nc), _p(flags), _p(stats))
    return img, T, nc, flags, int(h), stats


def render_bwd(W, H, TW, TH, rec, tile_start, lst, bg, dL_dimg, n, tile_mask=None):
    g2 = np.zeros((n, 9), np.float64)
    bg = np.ascontiguousarray(bg, np.float64)
    lst = np.ascontiguousarray(lst if len(lst) else np.zeros(1, np.int32), np.int32)
    dl = np.ascontiguousarray(dL_dimg, np.float64)
    tm = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8)
    lib().orc_render_bwd(W, H, TW, TH, _p(rec), _p(tile_start), _p(lst), _p(bg), _p(dl),
                         _p(tm), _p(g2))
    return g2


def blend_bwd(g0_shape, dg, mask, n, psi_frames, dGb_frames):
    """Adjoint of Eq. 1 over the frames that render one model."""
    dg = np.ascontiguousarray(dg, np.float64)
    k, A, npad = dg.shape
    nb = len(dGb_frames)
    psi = np.ascontiguousarray(np.asarray(psi_frames, np.float64).reshape(nb, k))
    dgb = np.ascontiguousarray(np.asarray(dGb_frames, np.float64).reshape(nb, 14, npad))
    dg0 = np.zeros((14, npad), np.float64)
    ddg = np.zeros((k, A, npad), np.float64)
    dpsi = np.zeros((nb, k), np.float64)
    lib().orc_blend_bwd(n, npad, k, mask, _p(dg), nb, _p(psi), _p(dgb), _p(dg0), _p(ddg),
                        _p(dpsi))
    return dg0, ddg, dpsi


# ------------------------------------------------------------------------------------------
# Whole-batch composition

@dataclass
class FrameResult:
    rect: np.ndarray
    f32: np.ndarray
    blended: np.ndarray
    rec: np.ndarray
    tile_start: np.ndarray
    lst: np.ndarray
    img: np.ndarray | None = None
    T: np.ndarray | None = None
    n_contrib: np.ndarray | None = None
    flags: np.ndarray | None = None
    hash: int = 0
    stats: np.ndarray | None = None
    tbn64: np.ndarray | None = None


def forward(batch, tile=(16, 16), render_frames=None, tile_masks=None, eps=1e-5,
            params=None, do_render=True, splat="f64", eps_t=1e-4):
    """Run the forward for every frame of a synth.Batch.

    params (optional, FP64 overrides for finite differences): {"g0": [per model], "dg": [...],
    "psi": [B][k_stride]}. The FP32 decision spec reads the same values rounded to fp32.

    splat: "f64" composites the FP64 projection of every Gaussian (the pure FP64 function of
    the parameters, used by the closed-form and finite-difference pins); "spec" composites the
    mean, conic and opacity that the FP32 decision spec computes (the same values that define
    the tile rectangles), widened to FP64, with FP64 colours. Parity with the fp32 GPU path
    uses "spec": at 1024 px the fp32 rounding of a screen mean alone (up to 7e-5 px) moves
    alpha by more than the ambiguity margin around the 1/255 cutoff.
    """
    TW, TH = tile
    params = params or {}
    out = []
    for b, fr in enumerate(batch.frames):
        m = batch.models[fr.model]
        g0 = params["g0"][fr.model] if "g0" in params else m.g0.astype(np.float64)
        dg = params["dg"][fr.model] if "dg" in params else m.dg.astype(np.float64)
        psi = (params["psi"][b] if "psi" in params else batch.psi[b].astype(np.float64))[:m.k]
        fp = batch.fparams[b]
        W, H = fr.width, fr.height
        rect, f32 = decide(g0.astype(np.float32), dg.astype(np.float32), psi.astype(np.float32),
                           fp, m.n, m.mask, W, H, TW, TH, m.binding, fr.verts)
        bl = blend(g0, dg, psi, m.n, m.mask)
        t64 = None if m.binding is None else tbn(m.binding, fr.verts, m.n)
        rec = project(bl, fp, m.n, W, H, rect, t64)
        if splat == "spec":
            kept = (rect[:, 2] > rect[:, 0]) & (rect[:, 3] > rect[:, 1])
            rec[kept, 0:5] = f32[kept, 0:5]
            rec[kept, 5] = f32[kept, 7]
        elif splat != "f64":
            raise ValueError(splat)
        tx, ty = (W + TW - 1) // TW, (H + TH - 1) // TH
        ts, lst = bin_sort(rect, f32[:, 6], tx, ty)
        fr_res = FrameResult(rect, f32, bl, rec, ts, lst, tbn64=t64)
        if do_render and (render_frames is None or b in render_frames):
            tm = None if tile_masks is None else tile_masks.get(b)
            bg = fp[17:20].astype(np.float64)
            (fr_res.img, fr_res.T, fr_res.n_contrib, fr_res.flags, fr_res.hash,
             fr_res.stats) = render(W, H, TW, TH, rec, ts, lst, bg, tm, eps, eps_t)
        out.append(fr_res)
    return out


def loss(batch, res, targets, kind="l1", n_total=None):
    """Mean per frame, averaged over frames; returns (L, [dL/dimg per frame]). n_total: the
    frame count of the whole batch when `batch` holds only some of its frames (one rank's share
    of a frame-sharded batch): L and its gradients are then this share's part of the whole
    batch's mean, and the sum over the shares is the whole batch's."""
    B = len(batch.frames) if n_total is None else n_total
    total = 0.0
    grads = []
    for b, fr in enumerate(batch.frames):
        d = res[b].img - targets[b].astype(np.float64)
        npx = d.size
        if kind == "l1":
            total += np.abs(d).sum() / npx
            grads.append(np.sign(d) / (npx * B))
        elif kind == "l2":
            total += 0.5 * (d * d).sum() / npx
            grads.append(d / (npx * B))
        else:
            raise ValueError(kind)
    return total / B, grads


def backward(batch, res, dL_dimg, tile=(16, 16), tile_masks=None, params=None):
    """Returns per-model (dG0 [14][n_pad], ddG [k][A][n_pad]), dpsi [B][k_stride] and the
    per-frame grad2d [n][9] and dGb [14][n_pad]."""
    TW, TH = tile
    params = params or {}
    g2s, dgbs = [], []
    for b, fr in enumerate(batch.frames):
        m = batch.models[fr.model]
        r = res[b]
        fp = batch.fparams[b]
        tm = None if tile_masks is None else tile_masks.get(b)
        g2 = render_bwd(fr.width, fr.height, TW, TH, r.rec, r.tile_start, r.lst,
                        fp[17:20].astype(np.float64), dL_dimg[b], m.n, tm)
        dgb = project_bwd(r.blended, fp, m.n, fr.width, fr.height, r.rect, g2, r.tbn64)
        g2s.append(g2)
        dgbs.append(dgb)
    per_model = []
    dpsi = np.zeros((len(batch.frames), batch.k_stride), np.float64)
    for mi, m in enumerate(batch.models):
        fids = [b for b, fr in enumerate(batch.frames) if fr.model == mi]
        dg = params["dg"][mi] if "dg" in params else m.dg.astype(np.float64)
        psi = [(params["psi"][b] if "psi" in params else batch.psi[b].astype(np.float64))[:m.k]
               for b in fids]
        if not fids:
            per_model.append((np.zeros((14, m.n_pad)), np.zeros_like(dg)))
            continue
        dg0, ddg, dps = blend_bwd(m.g0.shape, dg, m.mask, m.n, psi, [dgbs[b] for b in fids])
        per_model.append((dg0, ddg))
        for j, b in enumerate(fids):
            dpsi[b, :m.k] = dps[j]
    return per_model, dpsi, g2s, dgbs


def color_accum(W, H, TW, TH, rec, tile_start, lst, target, n):
    """Per Gaussian of one frame: [n][4] = (sum w, sum w I_r, sum w I_g, sum w I_b) over the
    pixels that blend it, w = alpha T its splatting weight there, I the target (Eq. 3)."""
    acc = np.zeros((n, 4), np.float64)
    lst = np.ascontiguousarray(lst if len(lst) else np.zeros(1, np.int32), np.int32)
    tg = np.ascontiguousarray(target, np.float64)
    lib().orc_color_accum(W, H, TW, TH, _p(np.ascontiguousarray(rec, np.float64)), _p(tile_start),
                          _p(lst), _p(tg), _p(acc))
    return acc


def color_init(batch, res, targets, done, delta=0.1, tile=(16, 16)):
    """Colour initialisation (Sec. 3.2 "Initialization", Eq. 3) over one batch: for every model,
    W_i and C_i = sums over all pixels of all its frames of w and w I; a Gaussian whose done flag
    is clear and whose W_i exceeds delta gets colour C_i / W_i and its flag set (once only).
    done: per model a bool array [n]. Returns per model (colour [3][n] or None where unchanged,
    new done flags, W [n])."""
    TW, TH = tile
    out = []
    for mi, m in enumerate(batch.models):
        acc = np.zeros((m.n, 4), np.float64)
        for b, fr in enumerate(batch.frames):
            if fr.model != mi:
                continue
            r = res[b]
            acc += color_accum(fr.width, fr.height, TW, TH, r.rec, r.tile_start, r.lst, targets[b], m.n)
        W = acc[:, 0]
        take = (~done[mi]) & (W > delta)
        col = np.full((3, m.n), np.nan)
        col[:, take] = (acc[take, 1:] / W[take, None]).T
        out.append((col, done[mi] | take, W))
    return out


def decision_signature(res) -> int:
    """Hash of every discrete decision of a forward: rectangles plus compositing outcomes."""
    h = 0
    for r in res:
        h = hash((h, r.rect.tobytes(), r.hash))
    return h


def adam(p, g, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, ICLR 2015, Algorithm 1) in FP64; lr broadcasts against p."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
