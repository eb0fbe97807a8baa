// Colour initialisation (RGBAvatar Sec. 3.2 "Initialization", Eq. 3): the second half of
// rgba_color_init. The forward compositing pass in accumulation mode has left, per (frame,
// Gaussian) record, the sums W = sum w and C = sum w I over the pixels that blend it (w its
// splatting weight alpha T there, I the target colour) in the record's first four 2-D gradient
// slots. Here every Gaussian whose done flag is clear sums them over the frames that render its
// model, in frame-list order; if W exceeds delta its base colour becomes C / W and its flag is
// set, so each Gaussian is initialised once.
#include "rgba_internal.cuh"

namespace rgba {
namespace {

struct DonePtrs {
    uint8_t *p[RGBA_MAX_MODELS];
};

constexpr int kFinishThreads = 256;

__global__ void __launch_bounds__(kFinishThreads) k_color_finish(Ctx c, float delta, DonePtrs done) {
    const ModelInfo &m = c.models[blockIdx.y];
    uint8_t *d = done.p[blockIdx.y];
    const int i = blockIdx.x * kFinishThreads + threadIdx.x;
    if (!d || i >= m.n || m.nb == 0 || d[i]) return;
    float W = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    for (int q = 0; q < m.nb; ++q) {
        const int b = c.mframes[m.frame_off + q];
        const float *a = c.grad2d + ((size_t)c.frames[b].rec_base + i) * kG2Floats;
        W += a[0];
        C0 += a[1];
        C1 += a[2];
        C2 += a[3];
    }
    if (W > delta) {
        float *g0 = const_cast<float *>(m.g0);  // the caller's model, written in place
        g0[(size_t)11 * m.n_pad + i] = C0 / W;
        g0[(size_t)12 * m.n_pad + i] = C1 / W;
        g0[(size_t)13 * m.n_pad + i] = C2 / W;
        d[i] = 1;
    }
}

}  // namespace

cudaError_t launch_color_finish(const Ctx &c, int max_n, float delta, const uint8_t *const *done_host,
                                int n_models, cudaStream_t s) {
    if (n_models == 0 || max_n == 0) return cudaSuccess;
    DonePtrs d;
    for (int m = 0; m < RGBA_MAX_MODELS; ++m) d.p[m] = m < n_models ? const_cast<uint8_t *>(done_host[m]) : nullptr;
    dim3 grid((max_n + kFinishThreads - 1) / kFinishThreads, n_models);
    k_color_finish<<<grid, kFinishThreads, 0, s>>>(c, delta, d);
    return cudaGetLastError();
}

}  // namespace rgba
