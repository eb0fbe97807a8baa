/*
 * rgba.h -- C ABI of the batch-parallel differentiable Gaussian blendshape rasterizer
 * (RGBAvatar, arXiv 2503.12886), hand-written CUDA for GB300 (sm_103a).
 *
 * One call renders B frames in one pass. Frame b draws the Gaussians of one avatar model,
 * blended with its own weight vector psi_b (Eq. 1, Sec. 3.1), activated after blending
 * (Supp. Sec. A.3), projected by EWA splatting, binned to screen tiles with a depth key, sorted
 * and alpha-composited front to back (the 3DGS "preprocess" / "rasterize" stages that the
 * batch-parallel rasterizer of Sec. 3.2 builds on). The backward pass takes the image-loss
 * gradient back to every base Gaussian, blendshape and weight. rgba_step does all of it with a
 * single host synchronisation per training step (Sec. 3.2, Fig. 4c).
 *
 * Conventions shared by every entry point
 *  - Memory: every array argument is caller-owned DEVICE memory unless marked "host". The
 *    library allocates nothing on the device; scratch lives in a caller-allocated workspace
 *    sized by rgba_workspace_size. No pointer is retained after a call returns, except by a
 *    captured step (rgba_step_capture), whose graph keeps them until rgba_graph_destroy.
 *  - Streams: every call is asynchronous on the given stream (0 = legacy default stream) and
 *    enqueues kernels and memsets only, so it can be captured in a CUDA graph, except
 *    rgba_step, rgba_color_init, rgba_render_fwd_noalloc, rgba_step_replay and rgba_debug_keys,
 *    which end with one device-to-host read and a stream synchronisation, and
 *    rgba_step_capture, which captures.
 *  - Errors: every call returns an rgba_status. Host-side validation failures return before
 *    anything is enqueued. rgba_last_error() gives a thread-local message for the last failure.
 *    No call aborts or exits the process.
 *  - Types: fp32 for all attributes and images, int32 for counts and indices.
 *
 * Layouts
 *  - Model (avatar), planar: g0[14][n_pad] with channels 0..2 mean (world, metres), 3..6
 *    rotation quaternion (w, x, y, z) unnormalised, 7..9 log-scale, 10 opacity logit,
 *    11..13 RGB colour. n_pad is a multiple of 4 and >= n; padding is ignored.
 *    dg[k][A][n_pad] holds the blendshape deltas of the A channels set in `mask`, in ascending
 *    channel order. Opacity (channel 10) must not be blended (Supp. A.3: blendshapes act on
 *    position, rotation and colour; the synthetic workloads also blend log-scale).
 *  - Frame parameters fparams[B][RGBA_FP_STRIDE]: 3x4 world-to-camera matrix (row-major,
 *    x right, y down, z forward), fx, fy, cx, cy, near-plane depth, background RGB.
 *  - Weights psi[B][k_stride]; frame b uses the first k of its model's entries.
 *  - Images: frames are concatenated in frame order; frame b occupies 3*H_b*W_b floats, planar
 *    [3][H_b][W_b]; per-pixel arrays (T_final, n_contrib) occupy H_b*W_b entries.
 *    Pixel (px, py) has its centre at (px + 0.5, py + 0.5).
 */
#ifndef RGBA_H
#define RGBA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RGBA_OK = 0,
    RGBA_ERR_INVALID_ARG = 1,  /* bad pointer, size, layout or mask; nothing was enqueued */
    RGBA_ERR_CAPACITY = 2,     /* tile-pair buffer too small; rgba_step_out.pairs_needed set */
    RGBA_ERR_CUDA = 3,         /* a CUDA runtime call failed; see rgba_last_error() */
    RGBA_ERR_TIMEOUT = 4,      /* a bounded device wait gave up; the results are invalid (reserved:
                                  no kernel of this library waits on another's progress) */
    RGBA_ERR_UNSUPPORTED = 5   /* valid request outside what the library supports */
} rgba_status;

#define RGBA_NCH 14
#define RGBA_FP_STRIDE 20
#define RGBA_MAX_FRAMES 4096
#define RGBA_MAX_MODELS 256
#define RGBA_MAX_K 64
/* Two common channel masks (any other valid mask works too; these two run a blend specialised at
 * compile time when every model of a batch uses the same one): mean + log-scale + colour, and
 * the paper's mean + rotation + colour (Supp. A.3). */
#define RGBA_MASK_MEAN_SCALE_COLOR 0x3B87u
#define RGBA_MASK_MEAN_ROT_COLOR 0x387Fu
#define RGBA_MAX_DIM 4096

/* Loss kinds for rgba_step (Sec. 3.2 "Loss Function" uses L1). Each frame's loss is the mean
 * over its 3*H*W values; the batch loss is their sum over the batch's frames divided by
 * rgba_batch.loss_frames (the mean over frames when that is 0). */
#define RGBA_LOSS_L1 1
#define RGBA_LOSS_L2 2 /* 1/2 (I - target)^2 */

typedef struct {
    int32_t n;          /* Gaussians */
    int32_t n_pad;      /* row stride of g0/dg, multiple of 4, >= n */
    int32_t k;          /* blendshapes, 1..RGBA_MAX_K */
    uint32_t mask;      /* bit c set: channel c is blended; bit 10 must be clear */
    const float *g0;    /* device [14][n_pad] */
    const float *dg;    /* device [k][A][n_pad], A = popcount(mask) */
    float *grad_g0;     /* device [14][n_pad] or NULL: dL/dG0, overwritten by the backward */
    float *grad_dg;     /* device [k][A][n_pad] or NULL: dL/ddG, overwritten by the backward */
    /* Tangent-space binding (Supp. "Gaussian Transformation", Alg. 1), or n_faces == 0 (the
     * pointers are then ignored and means/rotations are in world space). A bound Gaussian i
     * sits on triangle face_of[i] at the barycentric point bary[.][i] of its UV sample; its
     * mean and rotation channels are tangent-space (u, v, normal) coordinates. Per frame,
     * with the triangle's corners v0..v2 from rgba_frame.verts and their UVs, the TBN matrix
     * R = [T B N] (T = dx/du, B = dx/dv over the triangle, N the unit normal of
     * (v1 - v0) x (v2 - v0)) and t = b0 v0 + b1 v1 + b2 v2 map it to deformed space:
     * x = R x_T + t, covariance R Sigma_T R^T. No gradient flows to the mesh. A face or vertex
     * index out of range culls the Gaussian and sets bit 1 of rgba_step_out.device_error. */
    int32_t n_faces;            /* triangles of the mesh, 0 = unbound */
    int32_t n_verts;            /* vertices of every frame mesh of this model */
    const int32_t *faces;       /* device [n_faces][3] vertex indices */
    const float *face_uv;       /* device [n_faces][6]: (u, v) of corners 0, 1, 2 */
    const int32_t *face_of;     /* device [n]: triangle of each Gaussian */
    const float *bary;          /* device [3][n_pad]: barycentric weights of each Gaussian */
} rgba_model;

typedef struct {
    int32_t model;      /* index into rgba_batch.models */
    int32_t width;      /* pixels, 1..RGBA_MAX_DIM */
    int32_t height;
    const float *verts; /* device [n_verts][3]: this frame's deformed mesh if the model is
                           bound, else NULL (Supp. "Gaussian Transformation") */
} rgba_frame;

typedef struct {
    int32_t n_models;
    const rgba_model *models;   /* host array [n_models] */
    int32_t n_frames;
    const rgba_frame *frames;   /* host array [n_frames] */
    int32_t k_stride;           /* row stride of psi, >= every model's k */
    const float *psi;           /* device [n_frames][k_stride] */
    const float *fparams;       /* device [n_frames][RGBA_FP_STRIDE] */
    float *grad_psi;            /* device [n_frames][k_stride] or NULL, overwritten */
    int32_t tile_w, tile_h;     /* screen tile shape: 16x16 or 8x32 (tile_w * tile_h == 256) */
    int32_t smem_batch;         /* list entries a compositing warp stages per step: 64, 128 or 256 (0: 64) */
    int32_t loss_frames;        /* frames the batch loss is averaged over: 0 = n_frames; a rank of
                                   a frame-sharded data-parallel step passes the global batch size
                                   (>= n_frames), so that its loss and gradients are its share of
                                   the global batch's and a sum over ranks gives the batch's */
} rgba_batch;

typedef struct {
    double loss;                /* batch loss (rgba_step only) */
    int64_t pairs;              /* (Gaussian, tile) pairs the batch needed */
    int64_t pair_capacity;      /* pairs the workspace could hold */
    int64_t pairs_needed;       /* == pairs; set on RGBA_ERR_CAPACITY */
    uint32_t overflow;          /* 1 when pairs > pair_capacity */
    uint32_t device_error;      /* bit 0: a bounded device wait gave up (reserved); bit 1: a
                                   tangent-space binding index was out of range */
} rgba_step_out;

/* Byte offsets of the workspace regions, for tests and debugging tools that read the
 * intermediate results (splat records, tile ranges, sorted lists) directly. */
typedef struct {
    size_t counters;     /* rgba_counters */
    size_t records;      /* float[R][12]: u, v, conic a, b, c, opacity, r, g, b, depth, 0, 0 */
    size_t rects;        /* uint16[R][4]: tile rectangle x0, y0, x1, y1 (half-open) */
    size_t tile_start;   /* uint32[T + 1]: start of each (frame, tile) list */
    size_t sorted;       /* uint32[capacity]: Gaussian index per list entry */
    size_t grad2d;       /* float[R][12]: per (frame, Gaussian), the compositing backward's sums
                            over the pixels that blend it: S1..S5, S0 of g (dx, dy, dx^2, dx dy,
                            dy^2, 1), g = dL/dpower at the pixel, (dx, dy) = pixel centre - mean,
                            then dL/d(r, g, b). The 2-D gradients follow with the record's conic
                            (a, b, c) and opacity o: dL/du = a S1 + b S2, dL/dv = b S1 + c S2,
                            dL/d(a, b, c) = (-S3/2, -S4, -S5/2), dL/do = S0 / o */
    size_t pix_T;        /* float[P]: T_final of rgba_step (P = total pixels of the batch) */
    size_t pix_n;        /* int32[P]: n_contrib of rgba_step */
    size_t pix_dl;       /* float[3P]: dL/dimg of rgba_step's fused loss */
    size_t pix_img;      /* float[3P]: image of rgba_step when its img argument is NULL */
    size_t total_bytes;
    int64_t records_total;   /* R = sum over frames of the model's n_pad; frame b starts at
                                the sum of n_pad over frames before b */
    int64_t tiles_total;     /* T = sum over frames of tiles_x * tiles_y, frame-major,
                                row-major within a frame */
    int64_t pair_capacity;
} rgba_ws_layout;

typedef struct {
    uint32_t pairs;        /* pairs the batch needed (saturates at 2^32 - 1) */
    uint32_t overflow;     /* 1 if pairs > capacity */
    uint32_t n_work;       /* non-empty tiles */
    uint32_t device_error;
    double loss;
} rgba_counters;

typedef struct rgba_ctx *rgba_ctx_t;

/* Thread-local description of the last failure in this thread ("" if none). */
const char *rgba_last_error(void);

/* Create a context bound to CUDA device `device` (queries its SM count; allocates one small
 * pinned host block for rgba_step's result). */
int rgba_create(int device, rgba_ctx_t *out);
void rgba_destroy(rgba_ctx_t ctx);

/* Workspace bytes for `batch` with room for `pair_capacity` (Gaussian, tile) pairs.
 * Every entry point below that takes (ws, ws_bytes) derives the same layout from the batch;
 * the pair capacity it uses is whatever fits in ws_bytes. ws must be 256-byte aligned. */
int rgba_workspace_size(const rgba_batch *batch, int64_t pair_capacity, size_t *bytes);
int rgba_workspace_layout(const rgba_batch *batch, size_t ws_bytes, rgba_ws_layout *out);

/* Eq. 1 (Sec. 3.1): out[b] = G0 + sum_k psi_b[k] dG_k on the blended channels, G0 elsewhere.
 * out: device [B][14][n_pad(model of b)], frames concatenated. No workspace needed. */
int rgba_blend(rgba_ctx_t ctx, const rgba_batch *batch, float *out, void *stream);

/* Fused blend (Eq. 1) + activations (Supp. A.3) + EWA projection + tile rectangle + depth key
 * for every (frame, Gaussian); counts the Gaussians of every (frame, tile). */
int rgba_preprocess(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes,
                    void *stream);

/* Builds every (frame, tile) list sorted by (depth bits, Gaussian index). If the pairs exceed
 * the capacity the device sets the overflow counter and the later stages skip their work. */
int rgba_bin_sort(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes,
                  void *stream);

/* Front-to-back compositing (Sec. 3.2 "rasterize"): img [3][H][W] per frame = C + T bg,
 * T_final and n_contrib (list position + 1 of the last blended Gaussian) per pixel.
 * Alpha = min(0.99, o exp(power)), skipped below 1/255, stop when T (1 - alpha) < 1e-4. */
int rgba_render_fwd(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes,
                    float *img, float *T_final, int32_t *n_contrib, void *stream);

/* Back-propagation of dL/dimg (same layout as img) through compositing, projection,
 * activations and the blend. Uses only T_final and n_contrib from the forward (recomputes the
 * compositing in reverse). Writes models[m].grad_g0 / grad_dg and batch->grad_psi (those that
 * are non-NULL); the per-(frame, Gaussian) sums the 2-D gradients follow from stay in the
 * workspace (grad2d, see rgba_ws_layout).
 * grad_blended (device, 16-byte aligned, or NULL): also the gradient with respect to each
 * frame's blended Gaussians G^psi_b of Eq. 1, before the blend's adjoint reduces it over the
 * frames: frame b's [14][n_pad] block at float offset 14 * (sum of n_pad over frames before b),
 * the layout of rgba_blend's out; zero for culled Gaussians and padding columns. */
int rgba_render_bwd(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes,
                    const float *dL_dimg, const float *T_final, const int32_t *n_contrib,
                    float *grad_blended, void *stream);

/* One training step: preprocess, bin/sort, render with the fused loss against `target`
 * (layout of img), backward, then ONE device-to-host read of the counters and a stream
 * synchronisation. img may be NULL (the workspace keeps it). out: host. Returns
 * RGBA_ERR_CAPACITY (gradients invalid, out->pairs_needed set) when the pairs overflowed. */
int rgba_step(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes,
              const float *target, int loss_kind, float *img, rgba_step_out *out, void *stream);

/* rgba_step without the final read and synchronisation: everything it enqueues is kernels and
 * memsets, so a caller can capture it in a CUDA graph; the loss and counters stay in the
 * workspace's rgba_counters. */
int rgba_step_async(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes,
                    const float *target, int loss_kind, float *img, void *stream);

/* Adam update of the models' base Gaussians and blendshapes in place, from the gradients a
 * previous rgba_render_bwd / rgba_step wrote to grad_g0 / grad_dg (Supp. A.3: Adam with
 * per-attribute learning rates, blendshape rates scaled per attribute; Kingma & Ba 2015):
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;  p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
 * cfg (host): lr[14] for G0 channels, lr_delta[14] for the blendshape of each blended channel.
 * states (host array [n_models]): caller-owned device moment buffers shaped like g0 and dg,
 * zero before the first step; a model whose gradient or moment pointer is NULL is skipped.
 * step: 1-based Adam step count t, used when step_dev is NULL. step_dev (device int32 or
 * NULL): the number of completed steps; the call uses t = *step_dev + 1 and increments it on
 * the device, so a captured graph advances the bias correction on every replay.
 * Writes models[m].g0 / dg (cast from const). */
typedef struct {
    float lr[RGBA_NCH];
    float lr_delta[RGBA_NCH];
    float beta1, beta2, eps;
} rgba_adam_cfg;

typedef struct {
    float *m_g0, *v_g0;  /* device [14][n_pad] */
    float *m_dg, *v_dg;  /* device [k][A][n_pad] */
} rgba_adam_state;

int rgba_adam(rgba_ctx_t ctx, const rgba_batch *batch, const rgba_adam_cfg *cfg,
              const rgba_adam_state *states, int step, int32_t *step_dev, void *stream);

/* One training step with the Adam update fused into the backward: rgba_step_async followed by
 * rgba_adam (same arguments, same meaning), with results equal to those two calls bit for bit.
 * When every model of the batch is rendered by 1 to 16 of its frames and there are at most 16
 * models, the update is applied at the end of the projection/blend backward, from the
 * gradients it reduced in shared memory: the gradient arrays grad_g0 / grad_dg are neither
 * written nor needed (grad_psi is written as usual), so a training loop needs no memory for
 * them. (On the batched training workload it takes about as long as the two calls.) Other
 * batches run the two calls, and then need grad_g0 / grad_dg wherever the matching moments are
 * given (RGBA_ERR_INVALID_ARG otherwise, before anything is enqueued). Capturable, like
 * rgba_step_async; no host synchronisation. */
int rgba_step_adam_async(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes,
                         const float *target, int loss_kind, float *img, const rgba_adam_cfg *cfg,
                         const rgba_adam_state *states, int step, int32_t *step_dev, void *stream);

/* A training step captured once as a CUDA graph and replayed with one host synchronisation per
 * step (Sec. 3.2: one synchronisation per batch). rgba_step_capture runs the step once eagerly
 * on `stream` (a non-default stream; no update applied), then captures rgba_step_async, the
 * Adam update when cfg is non-NULL (rgba_adam with states and the device step counter
 * step_dev, both required then) and the read of the counters. The graph keeps every pointer:
 * batch arrays, workspace, target, img, moments and step_dev must stay valid and in place
 * while it is used; their contents may change between replays (new weights, cameras, targets).
 * Stage profiling must be off. rgba_step_replay launches it on the capture stream, waits and
 * fills out like rgba_step; RGBA_ERR_CAPACITY (out->pairs_needed set) means the workspace is
 * too small for this step: grow it and capture again. rgba_graph_destroy frees the graph. */
typedef struct rgba_graph *rgba_graph_t;
int rgba_step_capture(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes,
                      const float *target, int loss_kind, float *img, const rgba_adam_cfg *cfg,
                      const rgba_adam_state *states, int32_t *step_dev, void *stream,
                      rgba_graph_t *out);
int rgba_step_replay(rgba_graph_t graph, rgba_step_out *out);
void rgba_graph_destroy(rgba_graph_t graph);

/* The (frame, tile) lists of the last binning on this workspace (rgba_bin_sort, rgba_step or a
 * forward), for tests and debugging; synchronous. *n_pairs (host) receives the pair count.
 * tile_start (device uint32[T + 1], or NULL): list starts, T = total tiles of the batch, frame
 * after frame, tiles row-major. sorted (device uint32[sorted_cap], or NULL): every list's
 * Gaussian indices in (depth bits, index) order. RGBA_ERR_CAPACITY if that binning overflowed,
 * RGBA_ERR_INVALID_ARG if sorted_cap is below the pair count. */
int rgba_debug_keys(rgba_ctx_t ctx, const rgba_batch *batch, const void *ws, size_t ws_bytes,
                    uint32_t *tile_start, uint32_t *sorted, size_t sorted_cap, int64_t *n_pairs,
                    void *stream);

/* Per-stage device timing with CUDA events on the call's stream (off by default). Stages, in
 * launch order: 0 table upload, 1 preprocess (fused blend + projection), 2 tile-count scan,
 * 3 pair scatter, 4 per-tile depth sort, 5 compositing forward (+ fused loss), 6 compositing
 * backward, 7 projection + blend backward, 8 weight-gradient reduction. Do not enable it while
 * capturing a CUDA graph. */
#define RGBA_N_STAGES 9

typedef struct {
    float ms[RGBA_N_STAGES];  /* last recorded duration of each stage; -1 if not recorded */
    int32_t launches;         /* kernel launches enqueued since the previous read */
    int32_t pad_;
} rgba_profile;

/* on: 0 off, 1 stage timing, 2 stage timing and compositing statistics (rgba_debug_render_stats;
 * the two compositing kernels then run counting instances, built for 16x16 tiles with 64-entry
 * staging only: other shapes count nothing). */
int rgba_profile_enable(rgba_ctx_t ctx, int on);
/* Waits for the recorded events, fills `out` (host) and resets the launch count. */
int rgba_profile_read(rgba_ctx_t ctx, rgba_profile *out);

/* Compositing statistics of the forward and backward that ran on this workspace since its last
 * preprocess, counted while rgba_profile_enable(ctx, 2) was on (zero otherwise), for roofline
 * accounting: how many list entries the kernels evaluated and how many of those blend.
 * Synchronous; out: host. */
typedef struct {
    int64_t fwd_staged;  /* list entries the forward's pixel-block warps staged */
    int64_t fwd_hits;    /* (list entry, 8x4 pixel block) pairs whose alpha box meets the block */
    int64_t fwd_visits;  /* hits at which some pixel of the block passes the cutoffs (the entry
                            is then composited at the block) */
    int64_t fwd_blends;  /* (pixel, entry) pairs the forward blended */
    int64_t bwd_staged;  /* the same counts for the backward's reverse walk */
    int64_t bwd_hits;
    int64_t bwd_visits;
    int64_t bwd_pairs;   /* (pixel, entry) pairs the backward took a gradient of (those that
                            blended: equal to fwd_blends after one forward and one backward) */
} rgba_render_stats;
int rgba_debug_render_stats(rgba_ctx_t ctx, const rgba_batch *batch, const void *ws, size_t ws_bytes,
                            rgba_render_stats *out, void *stream);

/* Colour initialisation (Sec. 3.2 "Initialization", Eq. 3), synchronous. Renders the batch
 * (preprocess, bin/sort, front-to-back compositing) and, for every Gaussian, sums over all
 * pixels of all frames that render its model W = sum w and C = sum w I, with w the Gaussian's
 * splatting weight alpha T at the pixel and I the pixel's colour in target (planar [3][H][W]
 * per frame, frames concatenated as the images of rgba_render_fwd). A Gaussian whose done flag
 * is 0 and whose W exceeds delta (the paper uses 0.1) gets base colour G0[11..13] = C / W and
 * its flag set to 1; flags already set are never revisited, so each Gaussian is initialised
 * once. done: host array [n_models] of device uint8[n] flag arrays (NULL skips a model).
 * Writes models[m].g0 colour rows (cast from const). Uses the workspace's image regions and
 * 2-D gradient slots as scratch. Returns like rgba_step (out->loss is 0). */
int rgba_color_init(rgba_ctx_t ctx, const rgba_batch *batch, void *ws, size_t ws_bytes,
                    const float *target, float delta, uint8_t *const *done, rgba_step_out *out,
                    void *stream);

/* Forward render that allocates nothing: for callers that cannot call cudaMalloc (code inside
 * another framework's memory pool, plugins whose host forbids device allocation, processes that
 * must not grow their device footprint). The paper has no counterpart; it is a deployment
 * variant of rgba_preprocess + rgba_bin_sort + rgba_render_fwd.
 *  - Scratch: one fixed block of RGBA_NOALLOC_SCRATCH_BYTES (64 MiB) of device memory that is
 *    part of the library image; every GPU that loads the library holds it until the process
 *    exits. The caller still passes the inputs (batch) and the outputs img, T_final, n_contrib
 *    in the layouts of rgba_render_fwd; out (host) receives the pair count.
 *  - Limits: a batch whose workspace (rgba_workspace_size with capacity = the batch's total
 *    Gaussian records) does not fit the block returns RGBA_ERR_INVALID_ARG before anything is
 *    enqueued. The block holds the full rgba_step layout, so roughly 208 bytes per Gaussian
 *    record (a frame's record count is its model's n_pad; 20 of them are the one pair per record
 *    that must fit) + 32 bytes per pixel + 110-140 bytes per tile must fit in 64 MiB: one 512x512
 *    frame of a 100,000-Gaussian avatar (about 29 MB) or two of them fit, three do not; 16
 *    frames of 512x512 of a 60,000-Gaussian avatar need about 335 MB and are rejected. More
 *    pairs than fit in what is left return RGBA_ERR_CAPACITY with out->pairs_needed set (the
 *    outputs are then not written), and an out-of-range tangent-space binding index returns
 *    RGBA_ERR_INVALID_ARG, both after the call's one synchronisation. A NULL img, T_final or
 *    n_contrib with frames to render returns RGBA_ERR_INVALID_ARG before anything is enqueued.
 *  - The first call on a device looks up the block's device address with that device current;
 *    make that first call before any stream capture.
 *  - Every call uses the same block, which keeps the last call's contents; the call clears what
 *    must start at zero. Calls that overlap on the GPU (other streams, other threads) race on
 *    the block: serialise them.
 *  - Synchronous: ends with one device-to-host read of the counters and a stream
 *    synchronisation. No device memory is allocated or freed. */
#define RGBA_NOALLOC_SCRATCH_BYTES (64u << 20)
int rgba_render_fwd_noalloc(rgba_ctx_t ctx, const rgba_batch *batch, float *img, float *T_final,
                            int32_t *n_contrib, rgba_step_out *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RGBA_H */
