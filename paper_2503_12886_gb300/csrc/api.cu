// C ABI of librgba: argument validation, workspace layout and the launch sequence of every entry
// point declared in include/rgba.h.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rgba_internal.cuh"

using namespace rgba;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(RGBA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int popcount14(unsigned m) {
    int c = 0;
    for (int i = 0; i < kNch; ++i) c += (m >> i) & 1u;
    return c;
}

struct Plan {
    std::vector<ModelInfo> models;
    std::vector<FrameInfo> frames;
    std::vector<int> mframes;
    Layout L{};
    int max_n = 0, max_k = 1, max_chunks = 0, max_nb = 0;
};

// Host-side checks and tables; sizes of everything except the pair buffers.
int make_plan(const rgba_batch *b, Plan &p) {
    if (!b) return fail(RGBA_ERR_INVALID_ARG, "batch is NULL");
    if (b->n_frames < 0 || b->n_frames > RGBA_MAX_FRAMES)
        return fail(RGBA_ERR_INVALID_ARG, "n_frames out of range");
    if (b->n_models < 0 || b->n_models > RGBA_MAX_MODELS)
        return fail(RGBA_ERR_INVALID_ARG, "n_models out of range");
    if (b->n_frames > 0 && (!b->frames || !b->models || b->n_models == 0))
        return fail(RGBA_ERR_INVALID_ARG, "frames/models arrays missing");
    int tw = b->tile_w, th = b->tile_h;
    if (tw == 0 && th == 0) tw = th = 16;
    if (!((tw == 16 && th == 16) || (tw == 8 && th == 32)))
        return fail(RGBA_ERR_INVALID_ARG, "tile shape must be 16x16 or 8x32");
    int sb = b->smem_batch == 0 ? 64 : b->smem_batch;
    if (sb != 64 && sb != 128 && sb != 256)
        return fail(RGBA_ERR_INVALID_ARG, "smem_batch must be 64, 128 or 256");
    const int M = b->n_frames > 0 ? b->n_models : 0;
    p.models.assign(M, ModelInfo{});
    for (int m = 0; m < M; ++m) {
        const rgba_model &src = b->models[m];
        ModelInfo &mi = p.models[m];
        if (src.n < 0 || src.n_pad < src.n || (src.n_pad & 3))
            return fail(RGBA_ERR_INVALID_ARG, "model " + std::to_string(m) + ": need 0 <= n <= n_pad, n_pad % 4 == 0");
        if (src.k < 1 || src.k > RGBA_MAX_K)
            return fail(RGBA_ERR_INVALID_ARG, "model " + std::to_string(m) + ": k out of range");
        if (src.mask & ~0x3FFFu) return fail(RGBA_ERR_INVALID_ARG, "mask has bits above channel 13");
        if (src.mask & (1u << 10)) return fail(RGBA_ERR_INVALID_ARG, "opacity (channel 10) cannot be blended");
        const int A = popcount14(src.mask);
        if (src.n > 0 && (!src.g0 || (A > 0 && !src.dg)))
            return fail(RGBA_ERR_INVALID_ARG, "model " + std::to_string(m) + ": g0/dg is NULL");
        if ((reinterpret_cast<uintptr_t>(src.g0) | reinterpret_cast<uintptr_t>(src.dg) |
             reinterpret_cast<uintptr_t>(src.grad_g0) | reinterpret_cast<uintptr_t>(src.grad_dg)) & 15)
            return fail(RGBA_ERR_INVALID_ARG, "model arrays must be 16-byte aligned");
        mi.g0 = src.g0;
        mi.dg = src.dg;
        mi.gg0 = src.grad_g0;
        mi.gdg = src.grad_dg;
        mi.n = src.n;
        mi.n_pad = src.n_pad;
        mi.k = src.k;
        mi.A = A;
        mi.mask = src.mask;
        int a = 0;
        for (int ch = 0; ch < kNch; ++ch)
            if ((src.mask >> ch) & 1u) mi.chans[a++] = ch;
        if (src.n_faces < 0 || (src.n_faces > 0 && (src.n_verts < 3 || !src.faces || !src.face_uv ||
                                                     (src.n > 0 && (!src.face_of || !src.bary)))))
            return fail(RGBA_ERR_INVALID_ARG, "model " + std::to_string(m) + ": incomplete tangent-space binding");
        mi.n_faces = src.n_faces;
        mi.n_verts = src.n_faces > 0 ? src.n_verts : 0;
        mi.faces = src.n_faces > 0 ? src.faces : nullptr;
        mi.face_uv = src.n_faces > 0 ? src.face_uv : nullptr;
        mi.face_of = src.n_faces > 0 ? src.face_of : nullptr;
        mi.bary = src.n_faces > 0 ? src.bary : nullptr;
        mi.n_chunks = (src.n_pad + kBwdChunk - 1) / kBwdChunk;
        p.max_n = std::max(p.max_n, src.n_pad);
        p.max_chunks = std::max(p.max_chunks, mi.n_chunks);
    }
    const int B = b->n_frames;
    p.frames.assign(B, FrameInfo{});
    long long R = 0, T = 0, P = 0;
    std::vector<std::vector<int>> by_model(M);
    for (int f = 0; f < B; ++f) {
        const rgba_frame &fr = b->frames[f];
        if (fr.model < 0 || fr.model >= M) return fail(RGBA_ERR_INVALID_ARG, "frame " + std::to_string(f) + ": bad model index");
        if (fr.width < 1 || fr.height < 1 || fr.width > RGBA_MAX_DIM || fr.height > RGBA_MAX_DIM)
            return fail(RGBA_ERR_INVALID_ARG, "frame " + std::to_string(f) + ": size out of range");
        const ModelInfo &mi = p.models[fr.model];
        if (mi.k > b->k_stride) return fail(RGBA_ERR_INVALID_ARG, "k_stride smaller than a model's k");
        if (mi.n_faces > 0 && !fr.verts)
            return fail(RGBA_ERR_INVALID_ARG, "frame " + std::to_string(f) + ": its model is bound to a mesh but verts is NULL");
        FrameInfo &fi = p.frames[f];
        fi.verts = mi.n_faces > 0 ? fr.verts : nullptr;
        fi.model = fr.model;
        fi.W = fr.width;
        fi.H = fr.height;
        fi.tiles_x = (fr.width + tw - 1) / tw;
        fi.tiles_y = (fr.height + th - 1) / th;
        fi.tile_base = (int)T;
        fi.rec_base = (int)R;
        fi.n = mi.n;
        fi.n_pad = mi.n_pad;
        fi.k = mi.k;
        fi.pix_base = P;
        R += mi.n_pad;
        T += (long long)fi.tiles_x * fi.tiles_y;
        P += (long long)fr.width * fr.height;
        if (R > 0x7fffffffLL || T > 0x7fffffffLL) return fail(RGBA_ERR_INVALID_ARG, "batch too large");
        by_model[fr.model].push_back(f);
        p.max_k = std::max(p.max_k, mi.k);
    }
    if (B > 0 && (!b->psi || !b->fparams)) return fail(RGBA_ERR_INVALID_ARG, "psi/fparams is NULL");
    if (b->loss_frames != 0 && b->loss_frames < B)
        return fail(RGBA_ERR_INVALID_ARG, "loss_frames must be 0 or at least n_frames");
    long long dpsi = 0;
    for (int m = 0; m < M; ++m) {
        ModelInfo &mi = p.models[m];
        mi.nb = (int)by_model[m].size();
        mi.frame_off = (int)p.mframes.size();
        for (int f : by_model[m]) p.mframes.push_back(f);
        mi.dpsi_off = dpsi;
        dpsi += (long long)mi.nb * mi.k * mi.n_chunks;
        p.max_nb = std::max(p.max_nb, mi.nb);
    }
    Layout &L = p.L;
    L.R = R;
    L.T = T;
    L.P = P;
    L.B = B;
    L.M = M;
    L.k_stride = b->k_stride;
    L.tw = tw;
    L.th = th;
    L.smem_batch = sb;
    L.loss_frames = b->loss_frames ? b->loss_frames : B;
    L.dpsi_floats = dpsi;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    L.counters = take(256);
    L.models = take(sizeof(ModelInfo) * (size_t)M);
    L.frames = take(sizeof(FrameInfo) * (size_t)B);
    L.mframes = take(sizeof(int) * (size_t)B);
    L.tile_count = take((size_t)tc_bytes(T));
    L.tile_start = take(4 * (size_t)(T + 1));
    L.cursor = take(4 * (size_t)T * kSubCounters);
    L.work = take(4 * (size_t)T);
    L.scan_aux = take(scan_aux_bytes(T));
    L.records = take(sizeof(float) * kRecFloats * (size_t)R);
    L.rects = take(8 * (size_t)R);
    L.cache = take(sizeof(float) * kCacheFloats * (size_t)R);
    L.grad2d = take(sizeof(float) * kG2Floats * (size_t)R);
    L.ranks = take(4 * kRankSlots * (size_t)R);
    L.depth = take(4 * (size_t)R);
    L.pix_T = take(4 * (size_t)P);
    L.pix_n = take(4 * (size_t)P);
    L.pix_dl = take(12 * (size_t)P);
    L.pix_img = take(12 * (size_t)P);
    L.dpsi_part = take(4 * (size_t)dpsi);
    L.keys = o;  // pair buffers follow: 8 + 8 + 4 bytes per pair
    return RGBA_OK;
}

void finish_layout(Layout &L, long long cap) {
    L.cap = cap;
    size_t o = L.keys;
    o = align256(o + 8 * (size_t)cap);
    L.keys2 = o;
    o = align256(o + 8 * (size_t)cap);
    L.sorted = o;
    o = align256(o + 4 * (size_t)cap);
    L.total = o;
}

long long cap_for_bytes(const Layout &L, size_t bytes) {
    Layout t = L;
    finish_layout(t, 0);
    if (bytes < t.total) return -1;
    long long c = (long long)((bytes - L.keys) / 20);
    while (c > 0) {
        finish_layout(t, c);
        if (t.total <= bytes) break;
        c -= (long long)((t.total - bytes + 19) / 20);
    }
    return c < 0 ? 0 : c;
}

Ctx make_ctx(const Layout &L, unsigned char *ws, const rgba_batch *b) {
    Ctx c{};
    c.models = reinterpret_cast<const ModelInfo *>(ws + L.models);
    c.frames = reinterpret_cast<const FrameInfo *>(ws + L.frames);
    c.mframes = reinterpret_cast<const int *>(ws + L.mframes);
    c.psi = b->psi;
    c.fparams = b->fparams;
    c.grad_psi = b->grad_psi;
    c.cnt = reinterpret_cast<Counters *>(ws + L.counters);
    c.tile_count = reinterpret_cast<unsigned *>(ws + L.tile_count);
    c.tc_mask = (unsigned)(tc_pow2(L.T) - 1);
    c.tile_start = reinterpret_cast<unsigned *>(ws + L.tile_start);
    c.cursor = reinterpret_cast<unsigned *>(ws + L.cursor);
    c.work = reinterpret_cast<unsigned *>(ws + L.work);
    c.scan_aux = ws + L.scan_aux;
    c.records = reinterpret_cast<float4 *>(ws + L.records);
    c.rects = reinterpret_cast<ushort4 *>(ws + L.rects);
    c.cache = reinterpret_cast<float4 *>(ws + L.cache);
    c.grad2d = reinterpret_cast<float *>(ws + L.grad2d);
    c.keys = reinterpret_cast<unsigned long long *>(ws + L.keys);
    c.keys2 = reinterpret_cast<unsigned long long *>(ws + L.keys2);
    c.sorted = reinterpret_cast<unsigned *>(ws + L.sorted);
    c.dpsi_part = reinterpret_cast<float *>(ws + L.dpsi_part);
    c.ranks = reinterpret_cast<unsigned *>(ws + L.ranks);
    c.depth = reinterpret_cast<float *>(ws + L.depth);
    c.R = L.R;
    c.T = L.T;
    c.cap = L.cap;
    c.B = L.B;
    c.M = L.M;
    c.k_stride = L.k_stride;
    c.tw = L.tw;
    c.th = L.th;
    c.loss_frames = L.loss_frames;
    return c;
}

// Common prologue of the workspace-taking entry points.
struct Call {
    Plan p;
    Ctx c;
    unsigned char *ws = nullptr;
    cudaStream_t s = nullptr;
};

int prologue(rgba_ctx_t ctx, const rgba_batch *b, void *ws, size_t ws_bytes, void *stream, Call &call) {
    if (!ctx) return fail(RGBA_ERR_INVALID_ARG, "ctx is NULL");
    int rc = make_plan(b, call.p);
    if (rc) return rc;
    if (!ws) return fail(RGBA_ERR_INVALID_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(RGBA_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    long long cap = cap_for_bytes(call.p.L, ws_bytes);
    if (cap < 0) return fail(RGBA_ERR_INVALID_ARG, "workspace smaller than the fixed part of the layout");
    finish_layout(call.p.L, cap);
    call.ws = static_cast<unsigned char *>(ws);
    call.c = make_ctx(call.p.L, call.ws, b);
    call.s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return RGBA_OK;
}

enum Stage { ST_UPLOAD, ST_PRE, ST_SCAN, ST_SCATTER, ST_SORT, ST_FWD, ST_BWD, ST_GBWD, ST_DPSI };

// Brackets one stage with events when profiling is on; counts the kernels it launches.
struct StageScope {
    rgba_ctx_t c;
    int st;
    cudaStream_t s;
    StageScope(rgba_ctx_t c_, int st_, cudaStream_t s_, int kernels) : c(c_), st(st_), s(s_) {
        c->launches += kernels;
        if (c->prof) cudaEventRecord(c->ev0[st], s);
    }
    ~StageScope() {
        if (c->prof) {
            cudaEventRecord(c->ev1[st], s);
            c->recorded[st] = true;
        }
    }
};

int upload_kernels(size_t bytes) { return (int)((bytes + 3839) / 3840); }

int upload_tables(rgba_ctx_t ctx, Call &k) {
    const Layout &L = k.p.L;
    StageScope sc(ctx, ST_UPLOAD, k.s,
                  upload_kernels(sizeof(ModelInfo) * k.p.models.size()) +
                      upload_kernels(sizeof(FrameInfo) * k.p.frames.size()) +
                      upload_kernels(sizeof(int) * k.p.mframes.size()));
    cudaError_t e;
    if (!k.p.models.empty() &&
        (e = launch_upload(k.ws + L.models, k.p.models.data(), sizeof(ModelInfo) * k.p.models.size(), k.s)) != cudaSuccess)
        return cuda_fail(e, "upload models");
    if (!k.p.frames.empty() &&
        (e = launch_upload(k.ws + L.frames, k.p.frames.data(), sizeof(FrameInfo) * k.p.frames.size(), k.s)) != cudaSuccess)
        return cuda_fail(e, "upload frames");
    if (!k.p.mframes.empty() &&
        (e = launch_upload(k.ws + L.mframes, k.p.mframes.data(), sizeof(int) * k.p.mframes.size(), k.s)) != cudaSuccess)
        return cuda_fail(e, "upload model frames");
    return RGBA_OK;
}

int memset_async(void *p, size_t bytes, cudaStream_t s, const char *what) {
    if (bytes == 0) return RGBA_OK;
    cudaError_t e = cudaMemsetAsync(p, 0, bytes, s);
    return e == cudaSuccess ? RGBA_OK : cuda_fail(e, what);
}




int do_preprocess(rgba_ctx_t ctx, Call &k) {
    int rc;
    const size_t count_bytes = (size_t)tc_bytes(k.p.L.T);
    {  // tables, counters and tile counts in one launch when the tables fit its parameters
        const Layout &L = k.p.L;
        PrologueArgs a{};
        const void *src[3] = {k.p.models.data(), k.p.frames.data(), k.p.mframes.data()};
        const size_t bytes[3] = {sizeof(ModelInfo) * k.p.models.size(), sizeof(FrameInfo) * k.p.frames.size(),
                                 sizeof(int) * k.p.mframes.size()};
        const size_t off[3] = {L.models, L.frames, L.mframes};
        for (int t = 0; t < 3; ++t) {
            a.dst[t] = reinterpret_cast<uint4 *>(k.ws + off[t]);
            a.nbytes[t] = (int)std::min(bytes[t], (size_t)1 << 30);
            a.n16[t] = (int)((bytes[t] + 15) / 16);
        }
        a.zero_a = reinterpret_cast<uint4 *>(k.ws + L.counters);
        a.zero_a16 = 256 / 16;
        a.zero_b = reinterpret_cast<uint4 *>(k.ws + L.tile_count);  // regions are 256-byte aligned
        a.zero_b16 = (long long)((count_bytes + 15) / 16);
        if ((bytes[0] + 15) / 16 + (bytes[1] + 15) / 16 + (bytes[2] + 15) / 16 <= (size_t)kPrologueBlob16) {
            cudaError_t e;
            {
                StageScope sc(ctx, ST_UPLOAD, k.s, 1);
                e = launch_prologue(a, src, k.s);
            }
            if (e != cudaSuccess) return cuda_fail(e, "step prologue");
        } else {
            if ((rc = upload_tables(ctx, k))) return rc;
            if ((rc = memset_async(k.ws + L.counters, 256, k.s, "memset counters"))) return rc;
            if ((rc = memset_async(k.ws + L.tile_count, count_bytes, k.s, "memset tile counts"))) return rc;
        }
    }
    StageScope sc(ctx, ST_PRE, k.s, 1);
    int max_rows = 0;
    unsigned common_mask = k.p.models.empty() ? 0u : k.p.models[0].mask;
    for (const ModelInfo &m : k.p.models) {
        max_rows = std::max(max_rows, kNch + m.k * m.A);
        if (m.mask != common_mask) common_mask = 0u;
    }
    cudaError_t e = launch_preprocess(k.c, k.p.max_n, k.p.max_k, max_rows, common_mask, k.s);
    return e == cudaSuccess ? RGBA_OK : cuda_fail(e, "preprocess");
}

int do_bin_sort(rgba_ctx_t ctx, Call &k) {
    cudaError_t e;
    {
        StageScope sc(ctx, ST_SCAN, k.s, 3);
        if ((e = launch_scan(k.c, k.s)) != cudaSuccess) return cuda_fail(e, "scan");
    }
    {
        StageScope sc(ctx, ST_SCATTER, k.s, 1);
        if ((e = launch_scatter(k.c, k.p.max_n, k.s)) != cudaSuccess) return cuda_fail(e, "scatter");
    }
    StageScope sc(ctx, ST_SORT, k.s, 1);
    if ((e = launch_tile_sort(k.c, ctx->sms, k.s)) != cudaSuccess) return cuda_fail(e, "tile sort");
    return RGBA_OK;
}

int do_render_fwd(rgba_ctx_t ctx, Call &k, float *img, float *T, int *n, const float *target, int loss_kind, float *dl,
                  const float *acc_target = nullptr) {
    StageScope sc(ctx, ST_FWD, k.s, 1);
    cudaError_t e = launch_render_fwd(k.c, ctx->sms, k.p.L.smem_batch, img, T, n, target, loss_kind, dl, acc_target,
                                      ctx->stats, k.s);
    return e == cudaSuccess ? RGBA_OK : cuda_fail(e, "render fwd");
}

// The projection and blend backward after the compositing backward: zeroes the gradients of
// models no frame renders, then the Gaussian backward (optionally with the fused Adam update)
// and the weight-gradient reduction.
int do_gauss_bwd(rgba_ctx_t ctx, Call &k, const FusedAdam *fa) {
    int rc;
    cudaError_t e;
    for (const ModelInfo &m : k.p.models) {
        if (m.nb) continue;  // no frame renders it: zero gradient
        if (m.gg0 && (rc = memset_async(m.gg0, sizeof(float) * kNch * (size_t)m.n_pad, k.s, "memset grad_g0"))) return rc;
        if (m.gdg && (rc = memset_async(m.gdg, sizeof(float) * (size_t)m.k * m.A * m.n_pad, k.s, "memset grad_dg"))) return rc;
    }
    {
        StageScope sc(ctx, ST_GBWD, k.s, 1);
        int max_ka = 0;
        bool any_bound = false;
        for (const ModelInfo &m : k.p.models) {
            max_ka = std::max(max_ka, m.k * m.A);
            any_bound = any_bound || m.n_faces > 0;
        }
        if ((e = launch_gauss_bwd(k.c, k.p.max_chunks, k.p.max_k, max_ka, fa, any_bound, k.s)) != cudaSuccess)
            return cuda_fail(e, "gauss bwd");
    }
    if (k.c.grad_psi) {
        StageScope sc(ctx, ST_DPSI, k.s, 1);
        if ((e = launch_dpsi_reduce(k.c, k.p.max_k, k.s)) != cudaSuccess) return cuda_fail(e, "dpsi reduce");
    }
    if (fa && fa->step_dev) {  // after every reader of the step count
        ctx->launches += 1;
        if ((e = launch_step_advance(const_cast<int *>(fa->step_dev), k.s)) != cudaSuccess)
            return cuda_fail(e, "step advance");
    }
    return RGBA_OK;
}

// g2_zeroed: the preprocess of the same call zeroed the 2-D gradients (the fused step); a
// standalone backward clears them itself.
int do_render_bwd(rgba_ctx_t ctx, Call &k, const float *dl, const float *T, const int *n, bool g2_zeroed = false,
                  const FusedAdam *fa = nullptr) {
    int rc;
    const Layout &L = k.p.L;
    if (!g2_zeroed &&
        (rc = memset_async(k.ws + L.grad2d, sizeof(float) * kG2Floats * (size_t)L.R, k.s, "memset grad2d")))
        return rc;
    {
        StageScope sc(ctx, ST_BWD, k.s, 1);
        cudaError_t e = launch_render_bwd(k.c, ctx->sms, L.smem_batch, dl, T, n, ctx->stats, k.s);
        if (e != cudaSuccess) return cuda_fail(e, "render bwd");
    }
    return do_gauss_bwd(ctx, k, fa);
}

// The training step's compositing and backward: the forward with the fused loss (dL/dimg into
// the workspace), the compositing backward, then the projection and blend backward.
int do_render_step(rgba_ctx_t ctx, Call &k, float *img, float *T, int *n, const float *target, int loss_kind,
                   const FusedAdam *fa = nullptr) {
    float *dl = reinterpret_cast<float *>(k.ws + k.p.L.pix_dl);
    int rc = do_render_fwd(ctx, k, img, T, n, target, loss_kind, dl);
    if (rc) return rc;
    return do_render_bwd(ctx, k, dl, T, n, true, fa);
}

}  // namespace

int rgba::set_error(int code, const char *msg) { return fail(code, msg); }

extern "C" {

const char *rgba_last_error(void) { return g_err.c_str(); }

int rgba_create(int device, rgba_ctx_t *out) {
    if (!out) return fail(RGBA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(RGBA_ERR_INVALID_ARG, "no such device");
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    if (prop.major < 10) return fail(RGBA_ERR_UNSUPPORTED, "needs a Blackwell-class GPU (sm_100 or newer)");
    rgba_ctx *c = new rgba_ctx{};
    c->device = device;
    c->sms = prop.multiProcessorCount;
    if ((e = cudaHostAlloc(reinterpret_cast<void **>(&c->pinned), sizeof(rgba_counters), cudaHostAllocDefault)) != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaHostAlloc");
    }
    *out = c;
    return RGBA_OK;
}

void rgba_destroy(rgba_ctx_t ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->ev0[0]) {
        for (int i = 0; i < RGBA_N_STAGES; ++i) {
            cudaEventDestroy(ctx->ev0[i]);
            cudaEventDestroy(ctx->ev1[i]);
        }
    }
    cudaFreeHost(ctx->pinned);
    delete ctx;
}

int rgba_profile_enable(rgba_ctx_t ctx, int on) {
    if (!ctx) return fail(RGBA_ERR_INVALID_ARG, "ctx is NULL");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if (on && !ctx->ev0[0]) {
        for (int i = 0; i < RGBA_N_STAGES; ++i) {
            if ((e = cudaEventCreate(&ctx->ev0[i])) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
            if ((e = cudaEventCreate(&ctx->ev1[i])) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        }
    }
    ctx->prof = on != 0;
    ctx->stats = on == 2;
    for (int i = 0; i < RGBA_N_STAGES; ++i) ctx->recorded[i] = false;
    return RGBA_OK;
}

int rgba_profile_read(rgba_ctx_t ctx, rgba_profile *out) {
    if (!ctx || !out) return fail(RGBA_ERR_INVALID_ARG, "ctx/out is NULL");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    for (int i = 0; i < RGBA_N_STAGES; ++i) {
        out->ms[i] = -1.0f;
        if (!ctx->recorded[i]) continue;
        if ((e = cudaEventSynchronize(ctx->ev1[i])) != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, ctx->ev0[i], ctx->ev1[i])) != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        out->ms[i] = ms;
    }
    out->launches = ctx->launches;
    out->pad_ = 0;
    ctx->launches = 0;
    return RGBA_OK;
}

int rgba_workspace_size(const rgba_batch *batch, int64_t pair_capacity, size_t *bytes) {
    if (!bytes) return fail(RGBA_ERR_INVALID_ARG, "bytes is NULL");
    if (pair_capacity < 0 || pair_capacity > 0xfffffff0LL) return fail(RGBA_ERR_INVALID_ARG, "pair_capacity out of range");
    Plan p;
    int rc = make_plan(batch, p);
    if (rc) return rc;
    finish_layout(p.L, pair_capacity);
    *bytes = p.L.total;
    return RGBA_OK;
}

int rgba_workspace_layout(const rgba_batch *batch, size_t ws_bytes, rgba_ws_layout *out) {
    if (!out) return fail(RGBA_ERR_INVALID_ARG, "out is NULL");
    Plan p;
    int rc = make_plan(batch, p);
    if (rc) return rc;
    long long cap = cap_for_bytes(p.L, ws_bytes);
    if (cap < 0) return fail(RGBA_ERR_INVALID_ARG, "workspace smaller than the fixed part of the layout");
    finish_layout(p.L, cap);
    out->counters = p.L.counters;
    out->records = p.L.records;
    out->rects = p.L.rects;
    out->tile_start = p.L.tile_start;
    out->sorted = p.L.sorted;
    out->grad2d = p.L.grad2d;
    out->pix_T = p.L.pix_T;
    out->pix_n = p.L.pix_n;
    out->pix_dl = p.L.pix_dl;
    out->pix_img = p.L.pix_img;
    out->total_bytes = p.L.total;
    out->records_total = p.L.R;
    out->tiles_total = p.L.T;
    out->pair_capacity = p.L.cap;
    return RGBA_OK;
}

int rgba_blend(rgba_ctx_t ctx, const rgba_batch *batch, float *out, void *stream) {
    if (!ctx) return fail(RGBA_ERR_INVALID_ARG, "ctx is NULL");
    Plan p;
    int rc = make_plan(batch, p);
    if (rc) return rc;
    if (p.L.B == 0) return RGBA_OK;
    if (!out) return fail(RGBA_ERR_INVALID_ARG, "out is NULL");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    Ctx c{};
    c.models = p.models.data();  // host tables: launch_blend packs them into kernel parameters
    c.frames = p.frames.data();
    c.psi = batch->psi;
    c.k_stride = batch->k_stride;
    c.B = p.L.B;
    ctx->launches += (p.L.B + 63) / 64;
    e = launch_blend(c, p.max_n, out, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RGBA_OK : cuda_fail(e, "blend");
}

int rgba_preprocess(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes, void *stream) {
    Call k;
    int rc = prologue(ctx, batch, ws, ws_bytes, stream, k);
    if (rc || k.p.L.B == 0) return rc;
    return do_preprocess(ctx, k);
}

int rgba_bin_sort(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes, void *stream) {
    Call k;
    int rc = prologue(ctx, batch, ws, ws_bytes, stream, k);
    if (rc || k.p.L.B == 0) return rc;
    return do_bin_sort(ctx, k);
}

int rgba_render_fwd(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes, float *img,
                    float *T_final, int32_t *n_contrib, void *stream) {
    Call k;
    int rc = prologue(ctx, batch, ws, ws_bytes, stream, k);
    if (rc || k.p.L.B == 0) return rc;
    if (!img || !T_final || !n_contrib) return fail(RGBA_ERR_INVALID_ARG, "img/T_final/n_contrib is NULL");
    return do_render_fwd(ctx, k, img, T_final, n_contrib, nullptr, 0, nullptr);
}

int rgba_render_bwd(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes, const float *dL_dimg,
                    const float *T_final, const int32_t *n_contrib, float *grad_blended, void *stream) {
    Call k;
    int rc = prologue(ctx, batch, ws, ws_bytes, stream, k);
    if (rc || k.p.L.B == 0) return rc;
    if (!dL_dimg || !T_final || !n_contrib) return fail(RGBA_ERR_INVALID_ARG, "dL_dimg/T_final/n_contrib is NULL");
    if (reinterpret_cast<uintptr_t>(grad_blended) & 15) return fail(RGBA_ERR_INVALID_ARG, "grad_blended must be 16-byte aligned");
    k.c.grad_blended = grad_blended;
    return do_render_bwd(ctx, k, dL_dimg, T_final, n_contrib);
}

int rgba_adam(rgba_ctx_t ctx, const rgba_batch *batch, const rgba_adam_cfg *cfg,
              const rgba_adam_state *states, int step, int32_t *step_dev, void *stream) {
    if (!ctx || !cfg || !states) return fail(RGBA_ERR_INVALID_ARG, "ctx/cfg/states is NULL");
    if (!step_dev && step < 1) return fail(RGBA_ERR_INVALID_ARG, "Adam step count starts at 1");
    if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps > 0.f))
        return fail(RGBA_ERR_INVALID_ARG, "Adam betas must lie in [0, 1) and eps be positive");
    Plan p;
    int rc = make_plan(batch, p);
    if (rc) return rc;
    if (p.models.empty()) return RGBA_OK;
    for (size_t m = 0; m < p.models.size(); ++m) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(states[m].m_g0) | reinterpret_cast<uintptr_t>(states[m].v_g0) |
                            reinterpret_cast<uintptr_t>(states[m].m_dg) | reinterpret_cast<uintptr_t>(states[m].v_dg);
        if (a & 15) return fail(RGBA_ERR_INVALID_ARG, "Adam moment buffers must be 16-byte aligned");
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    ctx->launches += ((int)p.models.size() + 15) / 16 + (step_dev ? 1 : 0);
    e = launch_adam(p.models.data(), (int)p.models.size(), *cfg, states, step < 1 ? 1 : step, step_dev,
                    ctx->sms, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RGBA_OK : cuda_fail(e, "adam");
}

int rgba_step_async(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes, const float *target,
                    int loss_kind, float *img, void *stream) {
    Call k;
    int rc = prologue(ctx, batch, ws, ws_bytes, stream, k);
    if (rc || k.p.L.B == 0) return rc;
    if (!target) return fail(RGBA_ERR_INVALID_ARG, "target is NULL");
    if (loss_kind != RGBA_LOSS_L1 && loss_kind != RGBA_LOSS_L2) return fail(RGBA_ERR_INVALID_ARG, "bad loss kind");
    const Layout &L = k.p.L;
    float *im = img ? img : reinterpret_cast<float *>(k.ws + L.pix_img);
    float *T = reinterpret_cast<float *>(k.ws + L.pix_T);
    int *n = reinterpret_cast<int *>(k.ws + L.pix_n);
    if ((rc = do_preprocess(ctx, k))) return rc;
    if ((rc = do_bin_sort(ctx, k))) return rc;
    return do_render_step(ctx, k, im, T, n, target, loss_kind);
}

int rgba_step_adam_async(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes, const float *target,
                         int loss_kind, float *img, const rgba_adam_cfg *cfg, const rgba_adam_state *states,
                         int step, int32_t *step_dev, void *stream) {
    if (!ctx || !cfg || !states) return fail(RGBA_ERR_INVALID_ARG, "ctx/cfg/states is NULL");
    if (!step_dev && step < 1) return fail(RGBA_ERR_INVALID_ARG, "Adam step count starts at 1");
    if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps > 0.f))
        return fail(RGBA_ERR_INVALID_ARG, "Adam betas must lie in [0, 1) and eps be positive");
    Call k;
    int rc = prologue(ctx, batch, ws, ws_bytes, stream, k);
    if (rc || k.p.L.B == 0) return rc;
    if (!target) return fail(RGBA_ERR_INVALID_ARG, "target is NULL");
    if (loss_kind != RGBA_LOSS_L1 && loss_kind != RGBA_LOSS_L2) return fail(RGBA_ERR_INVALID_ARG, "bad loss kind");
    for (size_t m = 0; m < k.p.models.size(); ++m) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(states[m].m_g0) | reinterpret_cast<uintptr_t>(states[m].v_g0) |
                            reinterpret_cast<uintptr_t>(states[m].m_dg) | reinterpret_cast<uintptr_t>(states[m].v_dg);
        if (a & 15) return fail(RGBA_ERR_INVALID_ARG, "Adam moment buffers must be 16-byte aligned");
    }
    // fused when every model is rendered by 1..16 frames (one frame group in the backward)
    bool fuse = true;
    for (const ModelInfo &m : k.p.models) fuse = fuse && m.nb >= 1 && m.nb <= 16;
    FusedAdam fa;
    fuse = fuse && make_fused_adam(k.p.models.data(), (int)k.p.models.size(), *cfg, states, step, step_dev, fa);
    if (!fuse) {  // the two calls; the separate update reads the gradient arrays
        for (const ModelInfo &m : k.p.models)
            if ((states[&m - k.p.models.data()].m_g0 && !m.gg0) || (m.A > 0 && states[&m - k.p.models.data()].m_dg && !m.gdg))
                return fail(RGBA_ERR_INVALID_ARG,
                            "this batch cannot fuse the update (a model rendered by 0 or more than 16 frames, "
                            "or more than 16 models): grad_g0 / grad_dg are needed");
        if ((rc = rgba_step_async(ctx, batch, ws, ws_bytes, target, loss_kind, img, stream))) return rc;
        return rgba_adam(ctx, batch, cfg, states, step, step_dev, stream);
    }
    const Layout &L = k.p.L;
    float *im = img ? img : reinterpret_cast<float *>(k.ws + L.pix_img);
    float *T = reinterpret_cast<float *>(k.ws + L.pix_T);
    int *n = reinterpret_cast<int *>(k.ws + L.pix_n);
    if ((rc = do_preprocess(ctx, k))) return rc;
    if ((rc = do_bin_sort(ctx, k))) return rc;
    return do_render_step(ctx, k, im, T, n, target, loss_kind, &fa);
}

}  // extern "C"

// The one host synchronisation of a synchronous entry point: reads the counters into out.
int rgba::read_out(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes, rgba_step_out *out,
                   void *stream) {
    Plan p;
    make_plan(batch, p);
    const long long cap = cap_for_bytes(p.L, ws_bytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(ctx->pinned, static_cast<unsigned char *>(ws) + p.L.counters, sizeof(rgba_counters),
                                    cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "read counters");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const rgba_counters &h = *ctx->pinned;
    out->loss = h.loss;
    out->pairs = h.pairs;
    out->pair_capacity = cap;
    out->overflow = h.overflow;
    out->device_error = h.device_error;
    if (h.overflow) {
        out->pairs_needed = h.pairs;
        return fail(RGBA_ERR_CAPACITY, "pair buffer too small: need " + std::to_string(h.pairs) + " pairs");
    }
    if (h.device_error & 1u) return fail(RGBA_ERR_TIMEOUT, "device loop gave up");
    if (h.device_error & 2u) return fail(RGBA_ERR_INVALID_ARG, "tangent-space binding index out of range");
    return RGBA_OK;
}

extern "C" {

int rgba_step(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes, const float *target,
              int loss_kind, float *img, rgba_step_out *out, void *stream) {
    if (!out) return fail(RGBA_ERR_INVALID_ARG, "out is NULL");
    memset(out, 0, sizeof(*out));
    int rc = rgba_step_async(ctx, batch, ws, ws_bytes, target, loss_kind, img, stream);
    if (rc) return rc;
    if (batch->n_frames == 0) return RGBA_OK;
    return read_out(ctx, batch, ws, ws_bytes, out, stream);
}

int rgba_step_capture(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes, const float *target,
                      int loss_kind, float *img, const rgba_adam_cfg *cfg, const rgba_adam_state *states,
                      int32_t *step_dev, void *stream, rgba_graph_t *out) {
    if (!out) return fail(RGBA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx) return fail(RGBA_ERR_INVALID_ARG, "ctx is NULL");
    if (ctx->prof) return fail(RGBA_ERR_INVALID_ARG, "stage profiling is on: it cannot be captured");
    if (cfg && (!states || !step_dev))
        return fail(RGBA_ERR_INVALID_ARG, "a captured Adam update needs states and the device step counter");
    if (!stream) return fail(RGBA_ERR_INVALID_ARG, "capture needs a non-default stream");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // one eager step first: validates the arguments and sets every kernel attribute outside
    // the capture (the update is not applied)
    int rc = rgba_step_async(ctx, batch, ws, ws_bytes, target, loss_kind, img, stream);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    Plan p;
    make_plan(batch, p);
    rgba_graph *g = new rgba_graph();
    g->ctx = ctx;
    g->stream = s;
    g->ws = static_cast<unsigned char *>(ws);
    g->ws_bytes = ws_bytes;
    g->counters_off = p.L.counters;
    g->cap = cap_for_bytes(p.L, ws_bytes);
    if ((e = cudaMallocHost(reinterpret_cast<void **>(&g->host), sizeof(rgba_counters))) != cudaSuccess) {
        delete g;
        return cuda_fail(e, "cudaMallocHost");
    }
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        cudaFreeHost(g->host);
        delete g;
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    rc = rgba_step_async(ctx, batch, ws, ws_bytes, target, loss_kind, img, stream);
    if (!rc && cfg) rc = rgba_adam(ctx, batch, cfg, states, 0, step_dev, stream);
    if (!rc && (e = cudaMemcpyAsync(g->host, g->ws + g->counters_off, sizeof(rgba_counters), cudaMemcpyDeviceToHost,
                                    s)) != cudaSuccess)
        rc = cuda_fail(e, "read counters");
    cudaGraph_t graph = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(s, &graph);
    if (!rc && e_end != cudaSuccess) rc = cuda_fail(e_end, "cudaStreamEndCapture");
    if (!rc && (e = cudaGraphInstantiate(&g->exec, graph, 0)) != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
    if (graph) cudaGraphDestroy(graph);
    if (rc) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        cudaFreeHost(g->host);
        delete g;
        return rc;
    }
    *out = g;
    return RGBA_OK;
}

int rgba_step_replay(rgba_graph_t g, rgba_step_out *out) {
    if (!g || !out) return fail(RGBA_ERR_INVALID_ARG, "graph/out is NULL");
    memset(out, 0, sizeof(*out));
    cudaError_t e = cudaSetDevice(g->ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if ((e = cudaGraphLaunch(g->exec, g->stream)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const rgba_counters &h = *g->host;
    out->loss = h.loss;
    out->pairs = h.pairs;
    out->pair_capacity = g->cap;
    out->overflow = h.overflow;
    out->device_error = h.device_error;
    if (h.overflow) {
        out->pairs_needed = h.pairs;
        return fail(RGBA_ERR_CAPACITY, "pair buffer too small: need " + std::to_string(h.pairs) + " pairs");
    }
    if (h.device_error & 2u) return fail(RGBA_ERR_INVALID_ARG, "tangent-space binding index out of range");
    return RGBA_OK;
}

void rgba_graph_destroy(rgba_graph_t g) {
    if (!g) return;
    cudaSetDevice(g->ctx->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->host) cudaFreeHost(g->host);
    delete g;
}

int rgba_debug_keys(rgba_ctx_t ctx, const rgba_batch *batch, const void *ws, size_t ws_bytes, uint32_t *tile_start,
                    uint32_t *sorted, size_t sorted_cap, int64_t *n_pairs, void *stream) {
    if (!n_pairs) return fail(RGBA_ERR_INVALID_ARG, "n_pairs is NULL");
    Call k;
    int rc = prologue(ctx, batch, const_cast<void *>(ws), ws_bytes, stream, k);
    if (rc) return rc;
    const Layout &L = k.p.L;
    rgba_counters h;
    cudaError_t e = cudaMemcpyAsync(&h, k.ws + L.counters, sizeof(h), cudaMemcpyDeviceToHost, k.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(k.s);
    if (e != cudaSuccess) return cuda_fail(e, "read counters");
    *n_pairs = h.pairs;
    if (h.overflow) return fail(RGBA_ERR_CAPACITY, "the last binning overflowed: its lists are incomplete");
    if (tile_start &&
        (e = cudaMemcpyAsync(tile_start, k.ws + L.tile_start, 4 * (size_t)(L.T + 1), cudaMemcpyDeviceToDevice, k.s)) !=
            cudaSuccess)
        return cuda_fail(e, "copy tile starts");
    if (sorted) {
        if (sorted_cap < (size_t)h.pairs) return fail(RGBA_ERR_INVALID_ARG, "sorted_cap is smaller than the pair count");
        if (h.pairs &&
            (e = cudaMemcpyAsync(sorted, k.ws + L.sorted, 4 * (size_t)h.pairs, cudaMemcpyDeviceToDevice, k.s)) != cudaSuccess)
            return cuda_fail(e, "copy sorted lists");
    }
    if ((e = cudaStreamSynchronize(k.s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return RGBA_OK;
}

int rgba_debug_render_stats(rgba_ctx_t ctx, const rgba_batch *batch, const void *ws, size_t ws_bytes,
                            rgba_render_stats *out, void *stream) {
    if (!out) return fail(RGBA_ERR_INVALID_ARG, "out is NULL");
    memset(out, 0, sizeof(*out));
    Call k;
    int rc = prologue(ctx, batch, const_cast<void *>(ws), ws_bytes, stream, k);
    if (rc) return rc;
    Counters h;
    cudaError_t e = cudaMemcpyAsync(&h, k.ws + k.p.L.counters, sizeof(h), cudaMemcpyDeviceToHost, k.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(k.s);
    if (e != cudaSuccess) return cuda_fail(e, "read counters");
    out->fwd_staged = (int64_t)h.st_fwd[0];
    out->fwd_hits = (int64_t)h.st_fwd[1];
    out->fwd_visits = (int64_t)h.st_fwd[2];
    out->fwd_blends = (int64_t)h.st_fwd[3];
    out->bwd_staged = (int64_t)h.st_bwd[0];
    out->bwd_hits = (int64_t)h.st_bwd[1];
    out->bwd_visits = (int64_t)h.st_bwd[2];
    out->bwd_pairs = (int64_t)h.st_bwd[3];
    return RGBA_OK;
}

int rgba_color_init(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes, const float *target,
                    float delta, uint8_t *const *done, rgba_step_out *out, void *stream) {
    if (!out) return fail(RGBA_ERR_INVALID_ARG, "out is NULL");
    memset(out, 0, sizeof(*out));
    Call k;
    int rc = prologue(ctx, batch, ws, ws_bytes, stream, k);
    if (rc || k.p.L.B == 0) return rc;
    if (!target || !done) return fail(RGBA_ERR_INVALID_ARG, "target/done is NULL");
    if (!(delta >= 0.f)) return fail(RGBA_ERR_INVALID_ARG, "delta must be >= 0");
    const Layout &L = k.p.L;
    if ((rc = do_preprocess(ctx, k))) return rc;
    if ((rc = do_bin_sort(ctx, k))) return rc;
    // the accumulators (the records' 2-D gradient slots) were zeroed by the preprocess
    if ((rc = do_render_fwd(ctx, k, reinterpret_cast<float *>(k.ws + L.pix_img), reinterpret_cast<float *>(k.ws + L.pix_T),
                            reinterpret_cast<int *>(k.ws + L.pix_n), nullptr, 0, nullptr, target)))
        return rc;
    ctx->launches += 1;
    cudaError_t e = launch_color_finish(k.c, k.p.max_n, delta, done, (int)k.p.models.size(), k.s);
    if (e != cudaSuccess) return cuda_fail(e, "colour finish");
    return read_out(ctx, batch, ws, ws_bytes, out, stream);
}

}  // extern "C"
