"""The frame-sharded data-parallel step's exchange on CPU (gloo, world size 2): each rank runs
the oracle's forward, loss and backward on its share of a batch, with the loss averaged over the
whole batch, and the step's one all-reduce of the flat dG0 / ddG buffer (plus the loss sum and
the dpsi gather for reporting) must give exactly the single-process oracle gradients of the
whole batch (Eq. 1's adjoint sums over the batch's frames; Sec. 3.2). The batch has two avatars
with ragged frame sizes and an odd frame count, so the shards are uneven and one avatar has no
frame on one rank."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    from paper_2503_12886_gb300 import synth
    ms = [synth.make_model(41, 700, 6), synth.make_model(42, 500, 4, mask=synth.MASK_PAPER)]
    fr = [synth.Frame(0, 48, 40), synth.Frame(0, 40, 48), synth.Frame(0, 32, 32),
          synth.Frame(1, 48, 48), synth.Frame(1, 40, 32)]
    return synth.make_batch(ms, fr, seed=43, jitter_deg=15, random_bg=True)


def _flat(models, per_model):
    from paper_2503_12886_gb300.sharding import grad_layout
    lay = grad_layout(models)
    out = np.zeros(lay[-1][2], np.float64)
    for (a, b, c), (g0, dg) in zip(lay, per_model):
        out[a:b] = np.asarray(g0, np.float64).ravel()
        out[b:c] = np.asarray(dg, np.float64).ravel()
    return out


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2503_12886_gb300 import sharding, synth
        batch = _batch()
        B = len(batch.frames)
        targets = synth.make_targets(batch, 44)
        mine = sharding.shard(B, world, rank)
        sub = synth.Batch(batch.models, batch.frames[mine.start:mine.stop],
                          batch.psi[mine.start:mine.stop], batch.fparams[mine.start:mine.stop],
                          batch.k_stride)
        res = oracle.forward(sub)
        L, dls = oracle.loss(sub, res, targets[mine.start:mine.stop], "l1", n_total=B)
        per_model, dpsi, _, _ = oracle.backward(sub, res, dls)
        flat = torch.from_numpy(_flat(batch.models, per_model))
        sharding.all_reduce_grads(flat)
        loss = sharding.all_reduce_loss(L, "cpu")
        psi = sharding.gather_psi_grads(torch.from_numpy(dpsi), B)
        q.put((rank, len(mine), flat.numpy(), loss, psi.numpy(), None))
    except Exception as e:  # report, do not hang the other rank's collectives
        q.put((rank, 0, None, None, None, repr(e)))
        raise
    finally:
        dist.destroy_process_group()


def test_sharded_gradients_equal_the_whole_batch_gloo():
    import oracle
    batch = _batch()
    from paper_2503_12886_gb300 import synth
    targets = synth.make_targets(batch, 44)
    res = oracle.forward(batch)
    L, dls = oracle.loss(batch, res, targets, "l1")
    per_model, dpsi, _, _ = oracle.backward(batch, res, dls)
    ref = _flat(batch.models, per_model)

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
    assert all(o[5] is None for o in out), [o[5] for o in out]
    assert all(p.exitcode == 0 for p in procs)
    assert [o[1] for o in out] == [3, 2]
    scale = np.abs(ref).max()
    for rank, _, flat, loss, psi, _ in out:
        np.testing.assert_allclose(flat, ref, rtol=1e-12, atol=1e-12 * scale)
        assert loss == pytest.approx(L, rel=1e-12)
        np.testing.assert_allclose(psi, dpsi, rtol=1e-12, atol=1e-12 * np.abs(dpsi).max())
    np.testing.assert_array_equal(out[0][2], out[1][2])    # replicas see identical gradients


def test_shard_splits_every_frame_once():
    from paper_2503_12886_gb300.sharding import shard
    for n in (0, 1, 5, 16, 17):
        for world in (1, 2, 3, 8):
            parts = [shard(n, world, r) for r in range(world)]
            assert [f for p in parts for f in p] == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
