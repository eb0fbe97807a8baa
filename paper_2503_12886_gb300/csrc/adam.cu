// Fused Adam update of every base Gaussian and blendshape of every model in a batch (RGBAvatar
// Supp. A.3: Adam with per-attribute learning rates; blendshape rates scaled per attribute).
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
// (Kingma & Ba, ICLR 2015). Rows are n_pad floats (a multiple of 4), so every thread moves
// float4s; padding slots carry zero gradients and stay unchanged.
#include "rgba_internal.cuh"

namespace rgba {
namespace {

struct AdamModel {
    float *p0, *g0, *m0, *v0;  // [14][n_pad]
    float *pd, *gd, *md, *vd;  // [k][A][n_pad]
    int n_pad, k, A, pad_;
    float lr0[kNch];
    float lrd[kNch];           // per blended slot a (first A used)
};

constexpr int kAdamModels = 16;
struct AdamChunk {
    AdamModel m[kAdamModels];
};

__device__ __forceinline__ void adam4(float4 &p, const float4 g, float4 &m, float4 &v, float lr,
                                      float b1, float b2, float eps, float ibc1, float ibc2) {
    const float gs[4] = {g.x, g.y, g.z, g.w};
    float ps[4] = {p.x, p.y, p.z, p.w}, ms[4] = {m.x, m.y, m.z, m.w}, vs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) adam_update(ps[q], gs[q], ms[q], vs[q], lr, b1, b2, eps, ibc1, ibc2);
    p = make_float4(ps[0], ps[1], ps[2], ps[3]);
    m = make_float4(ms[0], ms[1], ms[2], ms[3]);
    v = make_float4(vs[0], vs[1], vs[2], vs[3]);
}

__global__ void k_adam(AdamChunk ch, float b1, float b2, float eps, float ibc1, float ibc2,
                       const int *step_dev) {
    pdl_enter();
    if (step_dev) {  // t = completed steps + 1, read from the device (graph replays advance it)
        ibc1 = adam_ibc(step_dev, b1);
        ibc2 = adam_ibc(step_dev, b2);
    }
    const AdamModel &M = ch.m[blockIdx.y];
    const long long rows0 = kNch, rowsd = (long long)M.k * M.A;
    const long long q4 = M.n_pad / 4;                  // float4s per row
    const long long total = (rows0 + rowsd) * q4;
    const bool narrow = total + (long long)gridDim.x * blockDim.x < 0xffffffffLL;  // 32-bit division
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long row = narrow ? (long long)((unsigned)e / (unsigned)q4) : e / q4;
        if (row < rows0) {
            if (!M.p0) continue;
            float4 *p = reinterpret_cast<float4 *>(M.p0) + e;
            float4 *m = reinterpret_cast<float4 *>(M.m0) + e;
            float4 *v = reinterpret_cast<float4 *>(M.v0) + e;
            const float4 g = reinterpret_cast<const float4 *>(M.g0)[e];
            float4 pp = *p, mm = *m, vv = *v;
            adam4(pp, g, mm, vv, M.lr0[row], b1, b2, eps, ibc1, ibc2);
            *p = pp;
            *m = mm;
            *v = vv;
        } else {
            if (!M.pd) continue;
            const long long ed = e - rows0 * q4;
            const int a = (int)((unsigned)(row - rows0) % (unsigned)M.A);
            float4 *p = reinterpret_cast<float4 *>(M.pd) + ed;
            float4 *m = reinterpret_cast<float4 *>(M.md) + ed;
            float4 *v = reinterpret_cast<float4 *>(M.vd) + ed;
            const float4 g = reinterpret_cast<const float4 *>(M.gd)[ed];
            float4 pp = *p, mm = *m, vv = *v;
            adam4(pp, g, mm, vv, M.lrd[a], b1, b2, eps, ibc1, ibc2);
            *p = pp;
            *m = mm;
            *v = vv;
        }
    }
}

__global__ void k_step_advance(int *step_dev) {
    pdl_enter();
    *step_dev += 1;
}

}  // namespace

// 1 / (1 - b^step) on the host, for updates without a device step counter.
static float host_ibc(float b, int step) { return (float)(1.0 / (1.0 - pow((double)b, step))); }

bool make_fused_adam(const ModelInfo *models, int n_models, const rgba_adam_cfg &cfg, const rgba_adam_state *st,
                     int step, const int *step_dev, FusedAdam &fa) {
    if (n_models > kFusedAdamModels) return false;
    memset(&fa, 0, sizeof(fa));
    for (int j = 0; j < n_models; ++j) {
        const ModelInfo &mi = models[j];
        FusedAdamModel &M = fa.m[j];
        if (st[j].m_g0 && st[j].v_g0) {
            M.p0 = const_cast<float *>(mi.g0);
            M.m0 = st[j].m_g0;
            M.v0 = st[j].v_g0;
        }
        if (mi.A > 0 && st[j].m_dg && st[j].v_dg) {
            M.pd = const_cast<float *>(mi.dg);
            M.md = st[j].m_dg;
            M.vd = st[j].v_dg;
        }
        for (int c = 0; c < kNch; ++c) M.lr0[c] = cfg.lr[c];
        for (int a = 0; a < mi.A; ++a) M.lrd[a] = cfg.lr_delta[mi.chans[a]];
    }
    fa.b1 = cfg.beta1;
    fa.b2 = cfg.beta2;
    fa.eps = cfg.eps;
    fa.ibc1 = host_ibc(cfg.beta1, step < 1 ? 1 : step);
    fa.ibc2 = host_ibc(cfg.beta2, step < 1 ? 1 : step);
    fa.step_dev = step_dev;
    return true;
}

cudaError_t launch_step_advance(int *step_dev, cudaStream_t s) {
    return launch_pdl(k_step_advance, dim3(1), dim3(1), 0, s, step_dev);
}

cudaError_t launch_adam(const ModelInfo *models, int n_models, const rgba_adam_cfg &cfg,
                        const rgba_adam_state *st, int step, int *step_dev, int sms, cudaStream_t s) {
    const float ibc1 = host_ibc(cfg.beta1, step), ibc2 = host_ibc(cfg.beta2, step);
    for (int m0 = 0; m0 < n_models; m0 += kAdamModels) {
        const int nm = n_models - m0 < kAdamModels ? n_models - m0 : kAdamModels;
        AdamChunk ch;
        memset(&ch, 0, sizeof(ch));
        for (int j = 0; j < nm; ++j) {
            const ModelInfo &mi = models[m0 + j];
            const rgba_adam_state &sj = st[m0 + j];
            AdamModel &M = ch.m[j];
            M.n_pad = mi.n_pad;
            M.k = mi.k;
            M.A = mi.A;
            if (mi.gg0 && sj.m_g0 && sj.v_g0) {
                M.p0 = const_cast<float *>(mi.g0);
                M.g0 = mi.gg0;
                M.m0 = sj.m_g0;
                M.v0 = sj.v_g0;
            }
            if (mi.A > 0 && mi.gdg && sj.m_dg && sj.v_dg) {
                M.pd = const_cast<float *>(mi.dg);
                M.gd = mi.gdg;
                M.md = sj.m_dg;
                M.vd = sj.v_dg;
            }
            for (int c = 0; c < kNch; ++c) M.lr0[c] = cfg.lr[c];
            for (int a = 0; a < mi.A; ++a) M.lrd[a] = cfg.lr_delta[mi.chans[a]];
        }
        dim3 grid(sms * 4, nm);
        cudaError_t e = launch_pdl(k_adam, grid, dim3(256), 0, s, ch, cfg.beta1, cfg.beta2, cfg.eps, ibc1, ibc2,
                                   (const int *)step_dev);
        if (e != cudaSuccess) return e;
    }
    if (step_dev) return launch_step_advance(step_dev, s);
    return cudaSuccess;
}

}  // namespace rgba
