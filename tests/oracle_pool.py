"""Per-avatar oracle work of the full-size uneven-workload parity test, run in spawned worker
processes so that the 64 frames' FP64 oracle runs in parallel (test infrastructure: numpy, the
oracle and the seeded inputs only; no torch, no GPU).

A worker rebuilds the seeded workload, takes one avatar and the frames that render it, and
compares the CUDA path's results for those frames (passed in as arrays) with the oracle:
rectangles, the FP32 decision-spec record columns, tile offsets and lists bit for bit, pixels
and contributor counts within the pixel tolerance except at the pixels the oracle flags as
ambiguous. It then runs the oracle backward from the dL/dimg the caller passes in, zeroed at
those flagged pixels, and returns the avatar's dG0 and ddG (the adjoint of Eq. 1 summed over its
frames), its frames' dpsi rows and the flag maps, so that the caller can feed the same dL/dimg
to the CUDA backward and compare."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2503_12886_gb300 import synth

# record columns of the CUDA path's render record and of the oracle's FP32 decision spec that
# must agree bit for bit: u, v, conic a, b, c, opacity, depth
_REC_COLS = [(0, 0), (1, 1), (2, 2), (3, 3), (4, 4), (5, 7), (9, 6)]


def uneven_avatar(args):
    a, frames, eps, eps_t, pix_atol = args
    batch = synth.workload_uneven()
    m = batch.models[a]
    idx = [f["b"] for f in frames]
    assert all(batch.frames[b].model == a for b in idx)
    sub = synth.Batch([m], [synth.Frame(0, batch.frames[b].width, batch.frames[b].height) for b in idx],
                      batch.psi[idx], batch.fparams[idx], batch.k_stride)
    ores = oracle.forward(sub, eps=eps, splat="spec", eps_t=eps_t)
    st = {"pairs": 0, "pixels": 0, "flagged": 0, "max_err": 0.0, "n_mismatch": 0}
    flags, dls = [], []
    for f, o in zip(frames, ores):
        b = f["b"]
        np.testing.assert_array_equal(f["rect"], o.rect, err_msg=f"frame {b} rects")
        kept = (o.rect[:, 2] > o.rect[:, 0]) & (o.rect[:, 3] > o.rect[:, 1])
        for gc, oc in _REC_COLS:
            np.testing.assert_array_equal(f["rec"][kept, gc].view(np.uint32), o.f32[kept, oc].view(np.uint32),
                                          err_msg=f"frame {b} record column {gc}")
        np.testing.assert_array_equal(f["tile_start"], o.tile_start.astype(np.int64), err_msg=f"frame {b} offsets")
        np.testing.assert_array_equal(f["lst"], o.lst.astype(np.int64), err_msg=f"frame {b} lists")
        st["pairs"] += len(o.lst)
        fl = o.flags > 0
        ok = ~fl
        e = np.abs(f["img"].astype(np.float64) - o.img).max(0)
        eT = np.abs(f["T"].astype(np.float64) - o.T)
        st["pixels"] += fl.size
        st["flagged"] += int(fl.sum())
        if ok.any():
            st["max_err"] = max(st["max_err"], float(e[ok].max()), float(eT[ok].max()))
            st["n_mismatch"] += int((f["n"][ok] != o.n_contrib[ok]).sum())
        flags.append(fl)
        dls.append(np.where(fl[None], 0.0, f["dl"].astype(np.float64)))
    assert st["max_err"] <= pix_atol and st["n_mismatch"] == 0, (a, st)
    per_model, dpsi, _, _ = oracle.backward(sub, ores, dls)
    g0, dg = per_model[0]
    return {"a": a, "idx": idx, "flags": flags, "stats": st, "g0": np.asarray(g0, np.float32),
            "dg": np.asarray(dg, np.float32), "dpsi": np.asarray(dpsi, np.float64)}
