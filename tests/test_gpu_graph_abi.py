"""The C ABI's captured training step (rgba_step_capture / rgba_step_replay) and its debug getter
for the binned lists (rgba_debug_keys).

Bars: a replayed step (with the captured Adam update) follows the eager rgba_step + rgba_adam
sequence: losses to 1e-5 relative, parameters after three steps to 1e-5 absolute (the
compositing backward's atomics sum in another order in the two runs); a graph whose workspace
is too small returns RGBA_ERR_CAPACITY with the pair count it needs; the debug getter returns
exactly the tile starts and sorted lists of the oracle's binning (bit-exact)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_12886_gb300 import api, synth
from paper_2503_12886_gb300.optim import Adam
from paper_2503_12886_gb300.rasterizer import DeviceBatch, Renderer, stream_ptr

from gpu_helpers import frame_tile_bases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    import __graft_entry__
    __graft_entry__.build()
    r = Renderer(0)
    yield r
    r.close()


def small_batch():
    models = [synth.make_model(120, 4000, 6), synth.make_model(121, 3000, 4, mask=synth.MASK_PAPER)]
    fr = [synth.Frame(0, 96, 80), synth.Frame(1, 80, 96), synth.Frame(0, 64, 64)]
    return synth.make_batch(models, fr, seed=120, jitter_deg=15, random_bg=True)


def test_replayed_step_follows_eager_steps(renderer):
    batch = small_batch()
    targets = synth.make_targets(batch, 6)
    dbA, dbB = DeviceBatch(batch, "cuda:0"), DeviceBatch(batch, "cuda:0")
    optA, optB = Adam(renderer, dbA), Adam(renderer, dbB)
    tgA, tgB = dbA.pack_images(targets), dbB.pack_images(targets)
    bB = dbB.struct()
    ws = torch.empty(api.rgba_workspace_size(bB, 8 * dbB.total_rec + 4096), dtype=torch.uint8, device="cuda:0")
    img = torch.empty(3 * dbB.total_pix, device="cuda:0")
    s = torch.cuda.Stream()
    g0_init = [m.g0.clone() for m in dbB.models]
    g = api.rgba_step_capture(renderer.ctx, bB, ws.data_ptr(), ws.numel(), tgB.data_ptr(), api.RGBA_LOSS_L1,
                              img.data_ptr(), optB.cfg, optB.states, optB.step_dev.data_ptr(), s.cuda_stream)
    try:
        for _ in range(3):
            outA = renderer.step(dbA, tgA, api.RGBA_LOSS_L1)
            optA.step()
            rc, outB = api.rgba_step_replay(g)
            assert rc == api.RGBA_OK and outB.overflow == 0
            assert abs(outA.loss - outB.loss) <= 1e-5 * abs(outA.loss)
            assert outA.pairs == outB.pairs
    finally:
        api.rgba_graph_destroy(g)
    torch.cuda.synchronize()
    assert int(optB.step_dev.item()) == 3
    for mA, mB, init in zip(dbA.models, dbB.models, g0_init):
        torch.testing.assert_close(mB.g0, mA.g0, rtol=0, atol=1e-5)
        torch.testing.assert_close(mB.dg, mA.dg, rtol=0, atol=1e-5)
        assert not torch.equal(mB.g0, init)  # the captured update ran


def test_replay_reports_capacity(renderer):
    batch = small_batch()
    db = DeviceBatch(batch, "cuda:0")
    tg = db.pack_images(synth.make_targets(batch, 7))
    b = db.struct()
    ws = torch.empty(api.rgba_workspace_size(b, 1000), dtype=torch.uint8, device="cuda:0")
    s = torch.cuda.Stream()
    g = api.rgba_step_capture(renderer.ctx, b, ws.data_ptr(), ws.numel(), tg.data_ptr(), api.RGBA_LOSS_L2,
                              None, None, None, None, s.cuda_stream)
    try:
        rc, out = api.rgba_step_replay(g)
    finally:
        api.rgba_graph_destroy(g)
    assert rc == api.RGBA_ERR_CAPACITY
    assert out.overflow == 1 and out.pairs_needed > out.pair_capacity >= 1000


def test_debug_keys_equal_oracle_lists(renderer):
    batch = small_batch()
    db = DeviceBatch(batch, "cuda:0", grads=False)
    renderer.forward(db)
    ws = renderer.ws
    lay = renderer.layout(db)
    T = lay.tiles_total
    ts = torch.empty(T + 1, dtype=torch.int32, device="cuda:0")
    n = api.rgba_debug_keys(renderer.ctx, db.struct(), ws.data_ptr(), ws.numel(), ts.data_ptr(), None, 0,
                            stream_ptr())
    srt = torch.empty(max(1, n), dtype=torch.int32, device="cuda:0")
    assert api.rgba_debug_keys(renderer.ctx, db.struct(), ws.data_ptr(), ws.numel(), None, srt.data_ptr(), n,
                               stream_ptr()) == n
    with pytest.raises(api.RgbaError):
        api.rgba_debug_keys(renderer.ctx, db.struct(), ws.data_ptr(), ws.numel(), None, srt.data_ptr(), n - 1,
                            stream_ptr())
    ts, srt = ts.cpu().numpy().astype(np.int64), srt.cpu().numpy().astype(np.int64)
    assert ts[-1] == n
    ores = oracle.forward(batch, splat="spec")
    bases = frame_tile_bases(batch)
    for b, (fr, o) in enumerate(zip(batch.frames, ores)):
        nt = len(o.tile_start) - 1
        t = ts[bases[b]: bases[b] + nt + 1]
        np.testing.assert_array_equal(t - t[0], o.tile_start.astype(np.int64))
        np.testing.assert_array_equal(srt[t[0]: t[-1]], o.lst.astype(np.int64))


def test_render_stats_count_blends_without_changing_results(renderer):
    """Profiling mode 2 runs counting instances of the two compositing kernels: their images
    equal the plain kernels' bit for bit and their loss and gradients up to the order of the
    atomic sums (same arithmetic, only counters added), the backward takes a gradient of exactly the (pixel, entry) pairs the forward
    blended, and that count lies between the pixels with a contributor and the sum of the
    contributor counts (the entries scanned up to each pixel's last blend)."""
    batch = synth.workload_batched(n=20_000, k=16, frames=3, res=256)
    db = DeviceBatch(batch, "cuda:0")
    tg = db.pack_images(synth.make_targets(batch, 12))
    ws = renderer.ensure_workspace(db)
    lay = renderer.layout(db)
    s = stream_ptr()
    outs = []
    for mode in (0, 2):
        api.rgba_profile_enable(renderer.ctx, mode)
        img = torch.empty(3 * db.total_pix, device="cuda:0")
        rc, out = api.rgba_step(renderer.ctx, db.struct(), ws.data_ptr(), ws.numel(), tg.data_ptr(),
                                api.RGBA_LOSS_L1, img.data_ptr(), s)
        assert rc == api.RGBA_OK
        st = api.rgba_debug_render_stats(renderer.ctx, db.struct(), ws.data_ptr(), ws.numel(), s)
        n = ws[lay.pix_n: lay.pix_n + 4 * db.total_pix].view(torch.int32).clone()
        outs.append((img, out.loss, db.models[0].grad_g0.clone(), db.models[0].grad_dg.clone(),
                     db.grad_psi.clone(), n, st))
    api.rgba_profile_enable(renderer.ctx, 0)
    (i0, l0, g0, d0, p0, n0, s0), (i2, l2, g2, d2, p2, n2, s2) = outs
    assert all(v == 0 for v in s0.values())
    assert torch.equal(i0, i2) and torch.equal(n0, n2)
    assert abs(l0 - l2) <= 1e-6 * l0  # fp32 per-CTA loss partials are added by atomics, in any order
    # the compositing backward's atomics may sum in another order: equal up to that
    for a, b in ((g0, g2), (d0, d2), (p0, p2)):
        assert float((a - b).abs().max()) <= 1e-5 * float(a.abs().max())
    assert s2["fwd_blends"] == s2["bwd_pairs"] > 0
    assert 0 < s2["fwd_visits"] <= s2["fwd_hits"] <= s2["fwd_staged"]
    assert 0 < s2["bwd_visits"] <= s2["bwd_hits"] <= s2["bwd_staged"]
    assert int((n2 > 0).sum()) <= s2["fwd_blends"] <= int(n2.to(torch.int64).sum())
