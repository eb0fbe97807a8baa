// Forward render for callers that cannot allocate device memory.
//
// Some callers have no device allocator they may use: code running inside another framework's
// memory pool, plugins whose host forbids cudaMalloc, or processes that must never grow their
// device footprint after start-up. rgba_render_fwd_noalloc gives them the forward render
// (preprocess, bin/sort, compositing) with all scratch taken from one fixed block of device
// memory that is part of this library's image: every GPU that loads the library holds the
// block until the process exits, and no call allocates or frees device memory.
#include <cstring>
#include <mutex>

#include "rgba_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(RGBA_NOALLOC_SCRATCH_BYTES);

// The scratch block. In host code this name is only a host-side stand-in for the symbol; its
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_dev[kMaxDevices] = {};

// With the context's device current: the device address of g_scratch on that device.
int scratch_address(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return RGBA_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return RGBA_ERR_CUDA;
        g_scratch_dev[device] = p;
    }
    *out = g_scratch_dev[device];
    return RGBA_OK;
}

}  // namespace

extern "C" int rgba_render_fwd_noalloc(rgba_ctx_t ctx, const rgba_batch *batch, float *img,
                                       float *T_final, int32_t *n_contrib, rgba_step_out *out,
                                       void *stream) {
    if (!ctx || !batch || !out) return rgba::set_error(RGBA_ERR_INVALID_ARG, "ctx/batch/out is NULL");
    memset(out, 0, sizeof(*out));
    // every host-side check comes before the first enqueue
    size_t fixed = 0;
    int rc = rgba_workspace_size(batch, 0, &fixed);
    if (rc) return rc;
    // the batch must leave room in the block for at least one pair per Gaussian record
    rgba_ws_layout lay;
    if (fixed > kScratchBytes || (rc = rgba_workspace_layout(batch, kScratchBytes, &lay)) != RGBA_OK ||
        lay.pair_capacity < lay.records_total)
        return rgba::set_error(RGBA_ERR_INVALID_ARG,
                               "batch too large for the 64 MiB no-alloc scratch block (its workspace "
                               "with one pair per Gaussian record must fit); use rgba_render_fwd "
                               "with a caller-allocated workspace");
    if (batch->n_frames == 0) return RGBA_OK;
    if (!img || !T_final || !n_contrib)
        return rgba::set_error(RGBA_ERR_INVALID_ARG, "img/T_final/n_contrib is NULL");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return rgba::set_error(RGBA_ERR_CUDA, "cudaSetDevice failed");
    void *ws = nullptr;
    if ((rc = scratch_address(ctx->device, &ws)) != RGBA_OK)
        return rgba::set_error(rc, "could not resolve the scratch block's device address");
    // rgba_preprocess clears the counters and tile counts that must start at zero; every other
    // region is written before it is read.
    if ((rc = rgba_preprocess(ctx, batch, ws, kScratchBytes, stream)) != RGBA_OK) return rc;
    if ((rc = rgba_bin_sort(ctx, batch, ws, kScratchBytes, stream)) != RGBA_OK) return rc;
    if ((rc = rgba_render_fwd(ctx, batch, ws, kScratchBytes, img, T_final, n_contrib, stream)) != RGBA_OK)
        return rc;
    // the same counter read as the other synchronous entry points: a pair overflow gives
    // RGBA_ERR_CAPACITY (out->pairs_needed set), an out-of-range tangent-space binding index
    // RGBA_ERR_INVALID_ARG
    return rgba::read_out(ctx, batch, ws, kScratchBytes, out, stream);
}
