"""C ABI checks that need no GPU: the library loads, exports every symbol include/rgba.h
declares, and rejects invalid batches on the host before anything is enqueued."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_12886_gb300 import api as a
    a.lib()
    return a


def header_functions():
    src = open(os.path.join(ROOT, "include", "rgba.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rgba_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(api):
    names = header_functions()
    assert set(names) == set(api.EXPORTS), names
    L = api.lib()
    for n in names:
        assert hasattr(L, n), n


def _batch(api, **kw):
    m = api.RgbaModel(10, 12, 4, 0x3B87, 0x1000, 0x2000, None, None)
    ms = (api.RgbaModel * 1)(m)
    fs = (api.RgbaFrame * 1)(api.RgbaFrame(0, 64, 48))
    b = api.RgbaBatch(1, C.cast(ms, C.POINTER(api.RgbaModel)), 1,
                      C.cast(fs, C.POINTER(api.RgbaFrame)), 4, 0x3000, 0x4000, None, 16, 16, 256)
    for k, v in kw.items():
        setattr(b, k, v)
    b._keep = (ms, fs)
    return b, ms, fs


def test_workspace_size_grows_with_capacity(api):
    b, _, _ = _batch(api)
    s0 = api.rgba_workspace_size(b, 0)
    s1 = api.rgba_workspace_size(b, 1000)
    assert s1 >= s0 + 12 * 1000 and s0 > 0
    lay = api.rgba_workspace_layout(b, s1)
    assert lay.pair_capacity >= 1000 and lay.records_total == 12
    assert lay.tiles_total == 4 * 3


@pytest.mark.parametrize("mutate,msg", [
    (lambda b, ms, fs: setattr(b, "tile_w", 32), "tile"),
    (lambda b, ms, fs: setattr(b, "smem_batch", 100), "smem_batch"),
    (lambda b, ms, fs: setattr(ms[0], "mask", 0x3B87 | (1 << 10)), "opacity"),
    (lambda b, ms, fs: setattr(ms[0], "n_pad", 10), "n_pad"),
    (lambda b, ms, fs: setattr(ms[0], "k", 0), "k out of range"),
    (lambda b, ms, fs: setattr(fs[0], "model", 3), "model index"),
    (lambda b, ms, fs: setattr(fs[0], "width", 0), "size"),
    (lambda b, ms, fs: setattr(b, "k_stride", 2), "k_stride"),
    (lambda b, ms, fs: setattr(b, "psi", None), "psi"),
    (lambda b, ms, fs: setattr(ms[0], "g0", None), "g0"),
    (lambda b, ms, fs: setattr(ms[0], "g0", 0x1004), "aligned"),
    (lambda b, ms, fs: setattr(ms[0], "n_faces", 5), "tangent-space binding"),
    (lambda b, ms, fs: (setattr(ms[0], "n_faces", 5), setattr(ms[0], "n_verts", 9),
                        setattr(ms[0], "faces", 0x5000), setattr(ms[0], "face_uv", 0x6000),
                        setattr(ms[0], "face_of", 0x7000), setattr(ms[0], "bary", 0x8000)), "verts"),
    (lambda b, ms, fs: setattr(ms[0], "n_faces", -1), "tangent-space binding"),
    (lambda b, ms, fs: setattr(b, "loss_frames", -1), "loss_frames"),
])
def test_invalid_batches_rejected_on_host(api, mutate, msg):
    b, ms, fs = _batch(api)
    mutate(b, ms, fs)
    with pytest.raises(api.RgbaError) as e:
        api.rgba_workspace_size(b, 100)
    assert e.value.code == api.RGBA_ERR_INVALID_ARG
    assert msg in str(e.value)


def test_loss_frames_of_a_shard_accepted(api):
    """A data-parallel rank's batch averages its loss over the global batch: loss_frames at or
    above the batch's own frame count is valid and changes no buffer size."""
    b, _, _ = _batch(api, loss_frames=16)
    assert api.rgba_workspace_size(b, 100) == api.rgba_workspace_size(_batch(api)[0], 100)


def test_complete_binding_accepted(api):
    b, ms, fs = _batch(api)
    for k, v in (("n_faces", 5), ("n_verts", 9), ("faces", 0x5000), ("face_uv", 0x6000),
                 ("face_of", 0x7000), ("bary", 0x8000)):
        setattr(ms[0], k, v)
    fs[0].verts = 0x9000
    assert api.rgba_workspace_size(b, 100) == api.rgba_workspace_size(_batch(api)[0], 100)


def test_null_arguments(api):
    L = api.lib()
    assert L.rgba_workspace_size(None, 10, None) == api.RGBA_ERR_INVALID_ARG
    assert L.rgba_create(0, None) == api.RGBA_ERR_INVALID_ARG
    b, _, _ = _batch(api)
    n = C.c_size_t()
    assert L.rgba_workspace_size(C.byref(b), -1, C.byref(n)) == api.RGBA_ERR_INVALID_ARG
    assert L.rgba_workspace_layout(C.byref(b), 16, C.byref(api.RgbaWsLayout())) == \
        api.RGBA_ERR_INVALID_ARG
    assert L.rgba_step(None, C.byref(b), None, 0, None, 1, None, None, None) == \
        api.RGBA_ERR_INVALID_ARG


def test_empty_batch_is_a_noop_size(api):
    b, _, _ = _batch(api, n_frames=0)
    assert api.rgba_workspace_size(b, 0) > 0


def test_null_arguments_of_the_step_variants(api):
    """The fused step, the captured step and the debug getter reject missing arguments on the
    host, before touching a device (no GPU is needed to run this)."""
    L = api.lib()
    b, _, _ = _batch(api)
    cfg = api.RgbaAdamCfg()
    cfg.beta1, cfg.beta2, cfg.eps = 0.9, 0.999, 1e-8
    st = (api.RgbaAdamState * 1)()
    E = api.RGBA_ERR_INVALID_ARG
    # no context / no configuration / no states
    assert L.rgba_step_adam_async(None, C.byref(b), None, 0, None, 1, None, C.byref(cfg), st, 1, None, None) == E
    assert L.rgba_step_adam_async(C.c_void_p(1), C.byref(b), None, 0, None, 1, None, None, st, 1, None, None) == E
    # step count must start at 1 without a device counter; betas in [0, 1), eps > 0
    assert L.rgba_step_adam_async(C.c_void_p(1), C.byref(b), None, 0, None, 1, None, C.byref(cfg), st, 0,
                                  None, None) == E
    bad = api.RgbaAdamCfg()
    bad.beta1, bad.beta2, bad.eps = 1.0, 0.999, 1e-8
    assert L.rgba_step_adam_async(C.c_void_p(1), C.byref(b), None, 0, None, 1, None, C.byref(bad), st, 1,
                                  None, None) == E
    # capture: no output slot / no context
    assert L.rgba_step_capture(None, C.byref(b), None, 0, None, 1, None, None, None, None, None, None) == E
    g = C.c_void_p(123)
    assert L.rgba_step_capture(None, C.byref(b), None, 0, None, 1, None, None, None, None, None, C.byref(g)) == E
    assert g.value is None  # cleared on failure
    assert L.rgba_step_replay(None, C.byref(api.RgbaStepOut())) == E
    L.rgba_graph_destroy(None)  # a no-op
    # debug getter: no pair-count slot
    assert L.rgba_debug_keys(None, C.byref(b), None, 0, None, None, 0, None, None) == E
