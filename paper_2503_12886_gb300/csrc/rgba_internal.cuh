// Internal declarations shared by the CUDA translation units of librgba.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rgba.h"

// Context behind rgba_ctx_t.
struct rgba_ctx {
    int device;
    int sms;
    rgba_counters *pinned;  // host-pinned landing spot of rgba_step's single read
    bool prof;
    bool stats;             // compositing kernels run their counting instances
    bool recorded[RGBA_N_STAGES];
    cudaEvent_t ev0[RGBA_N_STAGES], ev1[RGBA_N_STAGES];
    int launches;
};

// A captured training step (rgba_step_capture): the instantiated graph, the stream it replays
// on, and its own pinned landing spot for the counters.
struct rgba_graph {
    rgba_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0, counters_off = 0;
    long long cap = 0;
    rgba_counters *host = nullptr;
};

namespace rgba {

constexpr int kNch = 14;
constexpr int kRecFloats = 12;   // render record: u, v, a, b, c, o, r, g, b, depth, -, -
constexpr int kCacheFloats = 12; // backward cache: mean(3), quat(4), log-scale(3), opacity, kept
constexpr int kG2Floats = 12;    // 2-D gradient: du, dv, da, db, dc, dopacity, dr, dg, db, -
constexpr int kTilePix = 256;    // pixels per screen tile (16x16 or 8x32)
constexpr int kBwdChunk = 32;    // Gaussians per CTA in the fused preprocess/blend backward
constexpr int kRankSlots = 8;    // tiles per Gaussian whose in-tile slot preprocess records
constexpr int kSubCounters = 8;  // per-tile counters for larger rectangles (by Gaussian index)
// The per-tile counts of the preprocess take millions of atomics on the few thousand counters of
// the tiles a face covers. Stored side by side, those counters share a few L2 slices, whose
// atomic units then set the preprocess's pace (it varied by 30 % with the counters' offset). So
// each tile's ranked count has its own 32-byte sector, at a slot given by an odd multiplier
// modulo a power of two (Knuth's multiplicative hashing with the golden-ratio constant: a
// bijection that scatters neighbouring tiles), and the sub-counters follow the slots.
constexpr int kTcWords = 8;
__host__ __device__ inline long long tc_pow2(long long T) {
    long long p = 1;
    while (p < T) p <<= 1;
    return p;
}
__host__ __device__ inline long long tc_word(unsigned mask, long long t) {
    return (long long)kTcWords * (long long)(((unsigned)t * 0x9E3779B1u) & mask);
}
__host__ __device__ inline long long tc_sub_base(unsigned mask) { return (long long)kTcWords * ((long long)mask + 1); }
__host__ __device__ inline long long tc_bytes(long long T) {
    return 4 * ((long long)kTcWords * tc_pow2(T) + T * kSubCounters);
}

// Per-model table (device copy in the workspace).
struct ModelInfo {
    const float *g0;
    const float *dg;
    float *gg0;
    float *gdg;
    int n, n_pad, k, A;
    unsigned mask;
    int nb;          // frames that render this model
    int frame_off;   // into the model-frame list
    int n_chunks;    // ceil(n / kBwdChunk)
    long long dpsi_off;  // float offset of this model's [n_chunks][nb][k] dpsi partials
    int chans[kNch]; // blended channel ids, ascending (first A used)
    int n_faces;     // tangent-space binding (0: unbound)
    int n_verts;
    const int *faces;      // [n_faces][3]
    const float *face_uv;  // [n_faces][6]
    const int *face_of;    // [n]
    const float *bary;     // [3][n_pad]
};

// Per-frame table (device copy in the workspace).
struct FrameInfo {
    int model, W, H, tiles_x;
    int tiles_y, tile_base, rec_base, n;
    long long pix_base;  // first pixel of this frame in the concatenated image arrays
    int n_pad, k;
    const float *verts;  // [n_verts][3] deformed mesh (bound models) or nullptr
};

struct Counters {
    unsigned pairs;       // pairs needed (saturating)
    unsigned overflow;
    unsigned n_work;      // non-empty tiles
    unsigned device_error;
    double loss;
    unsigned next_sort;   // dynamic work counters of the persistent kernels
    unsigned next_fwd;
    unsigned next_bwd;
    unsigned done_sort;   // CTAs / warps of each persistent kernel that ran out of work: the
    unsigned done_fwd;    // last one to leave puts its kernel's counters back to zero, so
    unsigned done_bwd;    // every launch starts from zero without a memset
    // compositing statistics, counted only by the counting instances of the compositing kernels
    // (rgba_profile_enable(ctx, 2)); zeroed with the rest at the start of every preprocess
    // per direction: list entries staged, box hits, (entry, pixel block) visits that evaluated
    // the entry, (pixel, entry) pairs that blended (forward) or took a gradient (backward)
    unsigned long long st_fwd[4];
    unsigned long long st_bwd[4];
};
static_assert(sizeof(Counters) <= 256, "counters fit in one 256-byte block");

struct Layout {
    size_t counters, models, frames, mframes, tile_count, tile_start, cursor, work;
    size_t records, rects, cache, grad2d, ranks, depth, pix_T, pix_n, pix_dl, pix_img, dpsi_part;
    size_t keys, keys2, sorted, scan_aux, total;
    long long R, T, P;     // records, tiles, pixels
    long long dpsi_floats;
    long long cap;
    int B, M, k_stride, tw, th, smem_batch;
    int loss_frames;       // the loss's frame count (rgba_batch.loss_frames, or B)
    int max_n_pad;
};

// Everything a kernel needs to find its data (passed by value).
struct Ctx {
    const ModelInfo *models;
    const FrameInfo *frames;
    const int *mframes;
    const float *psi;
    const float *fparams;
    float *grad_psi;
    float *grad_blended;   // [sum over frames of 14 n_pad] or nullptr: dL/dG^psi_b per frame
    Counters *cnt;
    unsigned *tile_count;  // ranked counts (<= kRankSlots tiles; at tc_word), then [T][kSubCounters] the others
    unsigned tc_mask;      // tc_pow2(T) - 1: the ranked counts' slot hash range
    unsigned *tile_start;
    unsigned *cursor;      // [T][kSubCounters]: fill positions of the larger rectangles
    unsigned *work;
    unsigned char *scan_aux;  // the tile scan's per-CTA partials
    float4 *records;   // [R][3]
    ushort4 *rects;    // [R]
    float4 *cache;     // [R][3]
    float *grad2d;     // [R][12]
    unsigned long long *keys;
    unsigned long long *keys2;  // [cap]: second buffer of the global-memory radix passes
    unsigned *sorted;
    float *dpsi_part;
    unsigned *ranks;   // [R][kRankSlots]: slot of the Gaussian in each tile of its rectangle
    float *depth;      // [R]: view-space depth of each kept record (the scatter's sort key)
    long long R, T, cap;
    int B, M, k_stride, tw, th;
    int loss_frames;       // the loss is averaged over this many frames (>= B)
};

// Programmatic dependent launch (Hopper/Blackwell): a kernel launched with launch_pdl may be
// scheduled while the previous kernel in its stream drains; every kernel starts with pdl_wait(),
// which returns once the previous grid has completed and its writes are visible (a no-op for
// kernels launched without the attribute), then releases its own dependents (pdl_release).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_release();
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Records msg as the calling thread's rgba_last_error() text and returns code.
int set_error(int code, const char *msg);

// The one host synchronisation of a synchronous entry point: reads the workspace counters on
// `stream`, waits, fills out (pair capacity from ws_bytes) and maps the overflow flag and the
// device error bits to RGBA_ERR_CAPACITY, RGBA_ERR_TIMEOUT and RGBA_ERR_INVALID_ARG.
int read_out(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes, rgba_step_out *out,
             void *stream);

// Launch wrappers (each returns the cudaError_t of its launch).
cudaError_t launch_upload(void *dst, const void *src, size_t bytes, cudaStream_t s);
// One launch for the start of a step: n16[t] 16-byte units of table t from host src[t] to dst[t]
// (src16 is filled in), zero_a16 units zeroed at zero_a and zero_b16 at zero_b. The tables
// travel as kernel parameters, at most kPrologueBlob16 units in all.
constexpr int kPrologueBlob16 = 240;
struct PrologueArgs {
    uint4 *dst[3];
    int nbytes[3];  // table sizes; n16 = ceil(nbytes / 16)
    int n16[3];
    int src16[3];
    uint4 *zero_a;
    int zero_a16;
    uint4 *zero_b;
    long long zero_b16;
};
cudaError_t launch_prologue(const PrologueArgs &a, const void *const src[3], cudaStream_t s);
// common_mask: the channel mask every model of the batch shares (0 when they differ); the two
// masks of the RGBA_MASK_* constants run a blend specialised at compile time.
cudaError_t launch_preprocess(const Ctx &c, int max_n, int max_k, int max_rows, unsigned common_mask,
                              cudaStream_t s);
cudaError_t launch_blend(const Ctx &c, int max_n, float *out, cudaStream_t s);
cudaError_t launch_scan(const Ctx &c, cudaStream_t s);
size_t scan_aux_bytes(long long T);
cudaError_t launch_scatter(const Ctx &c, int max_n, cudaStream_t s);
cudaError_t launch_tile_sort(const Ctx &c, int sms, cudaStream_t s);
// stats: run the counting instance (16 x 16 tiles, 64-entry staging only), which adds the
// compositing statistics of Counters
cudaError_t launch_render_fwd(const Ctx &c, int grid, int smem_batch, float *img, float *T_final,
                              int *n_contrib, const float *target, int loss_kind,
                              float *dl_dimg, const float *acc_target, bool stats, cudaStream_t s);
cudaError_t launch_color_finish(const Ctx &c, int max_n, float delta, const uint8_t *const *done_host,
                                int n_models, cudaStream_t s);
cudaError_t launch_render_bwd(const Ctx &c, int grid, int smem_batch, const float *dl_dimg,
                              const float *T_final, const int *n_contrib, bool stats, cudaStream_t s);
// One Adam update (Kingma & Ba, ICLR 2015) of parameter p with gradient g:
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
// with ibc = 1 / (1 - b^t). The separate and the fused update both call this, so they agree
// bit for bit.
__device__ __forceinline__ void adam_update(float &p, float g, float &m, float &v, float lr, float b1, float b2,
                                            float eps, float ibc1, float ibc2) {
    m = fmaf(b1, m, (1.f - b1) * g);
    v = fmaf(b2, v, (1.f - b2) * g * g);
    p -= lr * (m * ibc1) / (sqrtf(v * ibc2) + eps);
}

// 1 / (1 - b^t) for t = *step_dev + 1 (completed steps + 1, read on the device so that graph
// replays advance it): 1 - b^t = -expm1(t log1p(b - 1)), no cancellation when b^t is close to 1
// (1 - b is exact in binary32 for b in [0.5, 1]).
__device__ __forceinline__ float adam_ibc(const int *step_dev, float b) {
    const float t = (float)(*step_dev + 1);
    return -1.0f / expm1f(t * log1pf(-(1.0f - b)));
}

// The Adam update fused into the projection/blend backward (rgba_step_adam_async): per model
// the parameters, moments and learning rates (NULL parameters: not updated).
constexpr int kFusedAdamModels = 16;
struct FusedAdamModel {
    float *p0, *m0, *v0;  // [14][n_pad]
    float *pd, *md, *vd;  // [k][A][n_pad]
    float lr0[kNch];
    float lrd[kNch];      // per blended slot a (first A used)
};
struct FusedAdam {
    FusedAdamModel m[kFusedAdamModels];
    float b1, b2, eps, ibc1, ibc2;  // ibc from the host when step_dev is NULL
    const int *step_dev;
};
// Fills fa for the batch's models; false when the update cannot be fused (too many models).
bool make_fused_adam(const ModelInfo *models, int n_models, const rgba_adam_cfg &cfg, const rgba_adam_state *st,
                     int step, const int *step_dev, FusedAdam &fa);

// max_ka: the largest k * A over the models (rows of blendshapes a chunk stages). fa (may be
// NULL): apply Adam to G0 and the blendshapes where their gradients are reduced, instead of
// writing the gradients (every model must be rendered by 1..16 frames).
// any_bound: some model has a tangent-space binding (else the instance without the TBN mapping).
cudaError_t launch_gauss_bwd(const Ctx &c, int max_chunks, int max_k, int max_ka, const FusedAdam *fa,
                             bool any_bound, cudaStream_t s);
cudaError_t launch_dpsi_reduce(const Ctx &c, int max_k, cudaStream_t s);
cudaError_t launch_adam(const ModelInfo *models, int n_models, const rgba_adam_cfg &cfg,
                        const rgba_adam_state *st, int step, int *step_dev, int sms, cudaStream_t s);
cudaError_t launch_step_advance(int *step_dev, cudaStream_t s);

}  // namespace rgba
