"""The forward render that allocates nothing (rgba_render_fwd_noalloc), called through the C ABI.

Callers that cannot use cudaMalloc (inside another framework's memory pool, plugins whose host
forbids device allocation) get the forward render with the library's fixed 64 MiB scratch
block. This file runs last so that a run stopping at the first failure has run everything else.
"""
import pytest
import torch

from paper_2503_12886_gb300 import api, synth
from paper_2503_12886_gb300.rasterizer import DeviceBatch, Renderer

pytestmark = pytest.mark.gpu

PIX_ATOL = 1e-4  # the pixel tolerance of the parity tests


@pytest.fixture(scope="module")
def renderer():
    import __graft_entry__
    __graft_entry__.build()
    r = Renderer(0)
    yield r
    r.close()


def small_batch():
    return synth.workload_batched(n=20_000, k=16, frames=3, res=256)


def test_noalloc_matches_workspace_path_twice(renderer):
    batch = small_batch()
    db = DeviceBatch(batch, "cuda:0", grads=False)
    img_ref, T_ref, n_ref = renderer.forward(db)
    torch.cuda.synchronize()
    b = db.struct()
    for call in range(2):  # two calls in a row share the block
        img = torch.full_like(img_ref, float("nan"))
        T = torch.full_like(T_ref, float("nan"))
        n = torch.full_like(n_ref, -1)
        rc, out = api.rgba_render_fwd_noalloc(renderer.ctx, b, img.data_ptr(), T.data_ptr(),
                                              n.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert rc == api.RGBA_OK, (call, api.last_error())
        assert out.pairs > 0 and not out.overflow
        torch.cuda.synchronize()
        assert torch.isfinite(img).all() and torch.isfinite(T).all()
        assert float((img - img_ref).abs().max()) <= PIX_ATOL, call
        assert float((T - T_ref).abs().max()) <= PIX_ATOL, call
        assert torch.equal(n, n_ref), call


def test_noalloc_rejects_batches_beyond_its_block(renderer):
    m = synth.make_model(1, 1000, 4)
    big = synth.make_batch([m], [synth.Frame(0, 1024, 1024)] * 64, seed=1)
    db = DeviceBatch(big, "cuda:0", grads=False)
    with pytest.raises(api.RgbaError) as e:
        api.rgba_render_fwd_noalloc(renderer.ctx, db.struct(), 0, 0, 0,
                                    torch.cuda.current_stream().cuda_stream)
    assert e.value.code == api.RGBA_ERR_INVALID_ARG
    assert "no-alloc scratch block" in str(e.value)
