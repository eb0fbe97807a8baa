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


def test_noalloc_reports_a_pair_overflow_then_recovers(renderer):
    """A batch whose records and pixels fit the block but whose (Gaussian, tile) pairs do not:
    large splats over a 1024x1024 frame. The call returns RGBA_ERR_CAPACITY with the pair count
    it needed; the next call with a batch that fits still matches the workspace path."""
    import math
    m = synth.make_model(11, 8000, 4, radii=(0.3, 0.3, 0.2), log_scale_mu=math.log(0.05))
    big = synth.make_batch([m], [synth.Frame(0, 1024, 1024)], seed=11)
    db = DeviceBatch(big, "cuda:0", grads=False)
    img = torch.empty(3 * db.total_pix, device="cuda:0")
    T = torch.empty(db.total_pix, device="cuda:0")
    n = torch.empty(db.total_pix, dtype=torch.int32, device="cuda:0")
    s = torch.cuda.current_stream().cuda_stream
    rc, out = api.rgba_render_fwd_noalloc(renderer.ctx, db.struct(), img.data_ptr(), T.data_ptr(),
                                          n.data_ptr(), s)
    assert rc == api.RGBA_ERR_CAPACITY, api.last_error()
    assert out.overflow == 1 and out.pair_capacity > 0
    assert out.pairs_needed > out.pair_capacity and out.pairs_needed == out.pairs
    test_noalloc_matches_workspace_path_twice(renderer)


def test_noalloc_reports_a_binding_index_out_of_range(renderer):
    """A tangent-space binding whose face index is past the mesh: the Gaussian is culled and
    the call returns RGBA_ERR_INVALID_ARG after its synchronisation, like rgba_step."""
    import dataclasses
    mesh = synth.make_head_mesh(303, 12, 24)
    m = synth.make_bound_model(303, 2000, 4, mesh)
    face_of = m.binding.face_of.copy()
    face_of[5] = m.binding.faces.shape[0] + 7
    m = dataclasses.replace(m, binding=dataclasses.replace(m.binding, face_of=face_of))
    fr = [synth.Frame(0, 96, 80, synth.frame_verts(mesh, 303, f)) for f in range(2)]
    batch = synth.make_batch([m], fr, 303, jitter_deg=10, random_bg=True)
    db = DeviceBatch(batch, "cuda:0", grads=False)
    img = torch.empty(3 * db.total_pix, device="cuda:0")
    T = torch.empty(db.total_pix, device="cuda:0")
    n = torch.empty(db.total_pix, dtype=torch.int32, device="cuda:0")
    with pytest.raises(api.RgbaError) as e:
        api.rgba_render_fwd_noalloc(renderer.ctx, db.struct(), img.data_ptr(), T.data_ptr(),
                                    n.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.code == api.RGBA_ERR_INVALID_ARG and "binding index" in str(e.value)


def test_noalloc_rejects_null_outputs_before_enqueueing(renderer):
    db = DeviceBatch(small_batch(), "cuda:0", grads=False)
    T = torch.empty(db.total_pix, device="cuda:0")
    n = torch.empty(db.total_pix, dtype=torch.int32, device="cuda:0")
    with pytest.raises(api.RgbaError) as e:
        api.rgba_render_fwd_noalloc(renderer.ctx, db.struct(), None, T.data_ptr(), n.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert e.value.code == api.RGBA_ERR_INVALID_ARG and "NULL" in str(e.value)
