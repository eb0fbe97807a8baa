// Front-to-back alpha compositing ("rasterize", RGBAvatar Sec. 3.2 on the 3DGS renderer) and
// its exact reverse. The binning tile (16x16 or 8x32 pixels) fixes the lists; the compositing
// work is split finer: every warp is an independent persistent worker that takes (tile, pixel
// block) items from one counter, so the few heavy tiles of a face-centred frame spread over
// many warps and no warp ever waits at a CTA barrier. A block is 8 x 4 pixels, one per lane. A
// warp walks its tile's list in steps of BATCH entries: each lane stages BATCH / 32 of them into
// the warp's shared-memory slots together with the box of the entry's alpha >= 1/255 ellipse, a
// ballot marks the entries whose box meets the warp's block, and only those are visited, in
// list order (in reverse in the backward). A visit evaluates the power at every pixel, skips
// the entry when no lane passes the cutoff, and otherwise runs the pixel step without branches
// (lanes that do not take part keep their state). The forward stops once every pixel of the
// block is saturated.
//
// Per pixel, with d = pixel centre - mean:
//   power = -(a dx^2 + c dy^2) / 2 - b dx dy  (skip if > 0)
//   alpha = min(0.99, o exp(power))            (skip if < 1/255)
//   stop, without blending, once T (1 - alpha) < 1e-4
// The backward recomputes each alpha with the same instruction sequence as the forward, walks
// the list backwards from the stored contributor count, and recovers T by division by
// (1 - alpha). Per-Gaussian gradient sums are reduced across the warp (reduce-scatter) to four
// partials per component, which reach global memory as atomic reductions.
#include "rgba_internal.cuh"

namespace rgba {
namespace {

constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

__device__ __forceinline__ int find_frame(const Ctx &c, long long t) {
    int lo = 0, hi = c.B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (c.frames[mid].tile_base <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// A Gaussian as the compositing loops read it from shared memory:
//   a = (u, v, -a/2, -b)   q = (-c/2, tau)   c = (opacity, r, g, b)
// tau = -ln(255 o): alpha = o e^power < 1/255 exactly when power < tau, so most pairs (the far
// tail of a splat, 90 % of all evaluations) are rejected from a and q alone, before the
// exponential and before the colour is read. Both kernels stage and evaluate through these
// functions, so their decisions agree bit for bit.
__device__ __forceinline__ void splat_from_record(const float4 &r0, const float4 &r1, float r2x, float4 &sa,
                                                  float2 &sq, float4 &sc, float4 &sb) {
    sa = make_float4(r0.x, r0.y, -0.5f * r0.z, -r0.w);
    const float tau = -__logf(255.0f * r1.y);
    sq = make_float2(-0.5f * r1.x, tau);
    sc = make_float4(r1.y, r1.z, r1.w, r2x);
    // bounding box of the ellipse power >= tau, i.e. d^T conic d <= -2 tau: half-extents
    // sqrt(-2 tau Sigma'_xx) and sqrt(-2 tau Sigma'_yy) with Sigma' = conic^-1, widened by 1 %
    // + 0.05 px so that everything it excludes fails the per-pixel test with room to spare
    const float det = r0.z * r1.x - r0.w * r0.w;
    if (tau < 0.0f && det > 0.0f) {
        const float s = -2.0f * tau / det;
        const float hx = 1.01f * sqrtf(s * r1.x) + 0.05f, hy = 1.01f * sqrtf(s * r0.z) + 0.05f;
        sb = make_float4(r0.x - hx, r0.x + hx, r0.y - hy, r0.y + hy);
    } else {
        sb = make_float4(1.0f, -1.0f, 1.0f, -1.0f);  // empty: the splat never reaches 1/255
    }
}

// Whether a staged splat's box misses a block of pixel centres [x0, x1] x [y0, y1].
__device__ __forceinline__ bool box_misses(const float4 &b, float x0, float x1, float y0, float y1) {
    return b.y < x0 || b.x > x1 || b.w < y0 || b.z > y1;
}

// power = -(a dx^2 + c dy^2)/2 - b dx dy = dx ((-a/2) dx + (-b) dy) + (-c/2) dy dy
__device__ __forceinline__ float power_of(float dx, float dy, const float4 &A, const float2 &Q) {
    return __fmaf_rn(dx, __fmaf_rn(A.z, dx, __fmul_rn(A.w, dy)), __fmul_rn(__fmul_rn(Q.x, dy), dy));
}

// the skip decision: a positive power (never, for a positive definite conic, but kept as the
// definition) or alpha below 1/255
__device__ __forceinline__ bool skip(float power, float tau) { return power > 0.0f || power < tau; }

struct PixF {
    float pxc, pyc, T, C0, C1, C2;
    int last;
    bool inside, done;
};

// One list entry for one pixel (forward), once the caller has evaluated the entry's power at
// the pixel: live = the pixel is still compositing and the entry passes the alpha cutoff. A live
// entry that would take T (1 - alpha) below 1e-4 marks the pixel done without blending;
// otherwise it blends. Branch-free, so a warp whose lanes disagree runs it once: a lane that is
// not live keeps its state whatever its exponential gives (alpha is capped at 0.99 and its
// weight is 0). Returns the splatting weight alpha T at the pixel (0 when the entry does not
// blend).
__device__ __forceinline__ float composite(PixF &p, bool live, float power, const float4 &Cc, int pos) {
    const float alpha = fminf(kAlphaMax, __fmul_rn(Cc.x, __expf(power)));
    const float testT = p.T * (1.0f - alpha);
    const bool sat = testT < kTMin;
    p.done = p.done || (live && sat);
    const bool blend = live && !sat;
    const float w = blend ? alpha * p.T : 0.0f;
    p.C0 = fmaf(Cc.y, w, p.C0);
    p.C1 = fmaf(Cc.z, w, p.C1);
    p.C2 = fmaf(Cc.w, w, p.C2);
    p.T = blend ? testT : p.T;
    p.last = blend ? pos : p.last;
    return w;
}

constexpr int kWarpsPerCta = 4;  // independent warps per CTA (they share nothing but the loss sum)

// A warp's staging of BATCH list entries [lo, lo + BATCH) (those in [0, hi)), lane l taking
// slots l, l + 32, ...: first the entries' Gaussian indices, then their records, then the
// staged form in the warp's shared-memory slots with, per 32-slot word, the ballot of entries
// whose box meets the block. The three steps run one and two batches ahead of the compositing,
// so the loads of the next batch are in flight while the current one is composited.
template <int S>
struct Stage {
    unsigned idx[S];
    float4 r0[S], r1[S];
    float r2[S];
};

template <int S>
__device__ __forceinline__ void load_idx(const Ctx &c, int lo, int hi, unsigned st, unsigned idx[S]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        const int e = lo + lane + 32 * q;
        idx[q] = (e >= 0 && e < hi) ? c.sorted[st + e] : 0u;
    }
}

template <int S>
__device__ __forceinline__ void load_rec(const float4 *rec, int lo, int hi, const unsigned idx[S], Stage<S> &g) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        g.idx[q] = idx[q];
        if (lo + lane + 32 * q >= 0 && lo + lane + 32 * q < hi) {
            const float4 *r = rec + (size_t)idx[q] * 3;
            g.r0[q] = r[0];
            g.r1[q] = r[1];
            g.r2[q] = r[2].x;
        }
    }
}

template <int S>
__device__ __forceinline__ void commit(const Stage<S> &g, int lo, int hi, float4 *wa, float2 *wq, float4 *wc,
                                       unsigned *widx, float bx0, float bx1, float by0, float by1, unsigned hit[S]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        bool h = false;
        if (lo + lane + 32 * q >= 0 && lo + lane + 32 * q < hi) {
            float4 sa, sc, sb;
            float2 sq;
            splat_from_record(g.r0[q], g.r1[q], g.r2[q], sa, sq, sc, sb);
            const int k = lane + 32 * q;
            wa[k] = sa;
            wq[k] = sq;
            wc[k] = sc;
            if (widx) widx[k] = g.idx[q];
            h = !box_misses(sb, bx0, bx1, by0, by1);
        }
        hit[q] = __ballot_sync(0xffffffffu, h);
    }
}

// A fire-and-forget global float add by the lanes where p holds, written as one predicated
// instruction: a branch around the atomic made the compiler reconverge the warp at every visit
// (0.53 -> 0.48 ms for the compositing backward of the batched training workload).
__device__ __forceinline__ void red_add_if(bool p, float *addr, float v) {
    asm volatile("{ .reg .pred q; setp.ne.b32 q, %2, 0; @q red.global.add.f32 [%0], %1; }"
                 :: "l"(addr), "f"(v), "r"((int)p) : "memory");
}

// The same reduction by every lane.
__device__ __forceinline__ void red_add(float *addr, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" :: "l"(addr), "f"(v) : "memory");
}

// Warp sum of v[0..3] as a reduce-scatter: lane l ends with the total of value (l >> 3) & 3.
__device__ __forceinline__ float warp_reduce4(const float v[4], int lane) {
    const unsigned F = 0xffffffffu;
    const bool h16 = lane & 16, h8 = lane & 8;
    float a[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = h16 ? v[i] : v[i + 2];
        const float keep = h16 ? v[i + 2] : v[i];
        a[i] = keep + __shfl_xor_sync(F, send, 16);
    }
    float m = (h8 ? a[1] : a[0]) + __shfl_xor_sync(F, h8 ? a[0] : a[1], 8);
    m += __shfl_xor_sync(F, m, 4);
    m += __shfl_xor_sync(F, m, 2);
    m += __shfl_xor_sync(F, m, 1);
    return m;
}

// Writes one finished pixel (colour over the background, T, contributor count) and, with a
// target, adds its loss term and returns dL/dpixel in g (also stored to dl_dimg unless that is
// NULL: the fused training-step kernel keeps it in registers).
__device__ __forceinline__ void finish_pixel(const Ctx &c, const FrameInfo &f, int b, int px, int py,
                                             const PixF &p, float *img, float *T_final, int *n_contrib,
                                             const float *target, int loss_kind, float *dl_dimg,
                                             float &loss_acc, float g[3]) {
    const float *bg = c.fparams + (size_t)b * RGBA_FP_STRIDE + 17;
    const long long hw = (long long)f.W * f.H;
    const long long pix = (long long)py * f.W + px;
    float *im = img + f.pix_base * 3 + pix;
    const float o0 = fmaf(p.T, bg[0], p.C0), o1 = fmaf(p.T, bg[1], p.C1), o2 = fmaf(p.T, bg[2], p.C2);
    im[0] = o0;
    im[hw] = o1;
    im[2 * hw] = o2;
    T_final[f.pix_base + pix] = p.T;
    n_contrib[f.pix_base + pix] = p.last;
    g[0] = g[1] = g[2] = 0.0f;
    if (target) {
        const float *tg = target + f.pix_base * 3 + pix;
        const float scale = 1.0f / (3.0f * (float)hw * (float)c.loss_frames);
        const float d0 = o0 - tg[0], d1 = o1 - tg[hw], d2 = o2 - tg[2 * hw];
        if (loss_kind == RGBA_LOSS_L1) {
            loss_acc += (fabsf(d0) + fabsf(d1) + fabsf(d2)) * scale;
            g[0] = d0 > 0.f ? scale : (d0 < 0.f ? -scale : 0.f);
            g[1] = d1 > 0.f ? scale : (d1 < 0.f ? -scale : 0.f);
            g[2] = d2 > 0.f ? scale : (d2 < 0.f ? -scale : 0.f);
        } else {
            loss_acc += 0.5f * (d0 * d0 + d1 * d1 + d2 * d2) * scale;
            g[0] = d0 * scale;
            g[1] = d1 * scale;
            g[2] = d2 * scale;
        }
        if (dl_dimg) {
            float *dl = dl_dimg + f.pix_base * 3 + pix;
            dl[0] = g[0];
            dl[hw] = g[1];
            dl[2 * hw] = g[2];
        }
    }
}

// One compositing warp's view of a (tile, pixel block) item: the frame, the tile's list, the
// block's pixel-centre box and the warp's shared-memory slots.
struct Walk {
    unsigned st;        // first list entry of the tile
    int len;            // list length
    const float4 *rec;  // the frame's render records
    float bx0, bx1, by0, by1;
    float4 *wa, *wc;
    float2 *wq;
    unsigned *widx;     // Gaussian index per slot, or nullptr when no caller needs it
};

// An empty tile's item: the background, T = 1, no contributors, eight pixels per lane.
template <int TW>
__device__ __forceinline__ void empty_tile(const Ctx &c, long long t, float *img, float *T_final, int *n_contrib,
                                           const float *target, int loss_kind, float *dl_dimg, float &loss_acc) {
    constexpr int TH = kTilePix / TW;
    const int lane = threadIdx.x & 31;
    const int b = find_frame(c, t);
    const FrameInfo &f = c.frames[b];
    const int lt = (int)(t - f.tile_base);
    const int ty = lt / f.tiles_x, tx = lt - ty * f.tiles_x;
#pragma unroll 1
    for (int k = lane; k < kTilePix; k += 32) {
        const int px = tx * TW + (k % TW), py = ty * TH + (k / TW);
        if (px < f.W && py < f.H) {
            const PixF p{(float)px + 0.5f, (float)py + 0.5f, 1.f, 0.f, 0.f, 0.f, 0, true, true};
            float g[3];
            finish_pixel(c, f, b, px, py, p, img, T_final, n_contrib, target, loss_kind, dl_dimg, loss_acc, g);
        }
    }
}

// Compositing statistics of one warp (counting instances only): entries staged, box hits,
// visits that evaluated an entry (a hit with some pixel past the cutoffs; warp-uniform), and the
// (pixel, entry) pairs that blend or take a gradient (this lane's).
struct WalkStats {
    unsigned long long staged, hits, visits;
    unsigned lanes;
};

// The forward walk of one pixel block: the tile's list staged BATCH = 32 S entries at a time
// (each batch's loads one and two batches ahead), the hits of each batch composited front to
// back, until every pixel of the block is done or the list ends. The last committed batch
// stays in the warp's slots: its first list position in lo_last (-1 if none), its hit words in
// hit[]. ACC: colour-initialisation accumulation into acc (see k_render_fwd).
template <int S, bool ACC, bool STATS>
__device__ __forceinline__ void fwd_walk(const Ctx &c, const Walk &w, PixF &p, float I0, float I1, float I2,
                                         float *acc, unsigned hit[S], int &lo_last, WalkStats &st) {
    constexpr int BATCH = 32 * S;
    const int lane = threadIdx.x & 31;
    Stage<S> g;
    unsigned nidx[S];
    load_idx<S>(c, 0, w.len, w.st, nidx);
    load_rec<S>(w.rec, 0, w.len, nidx, g);
    load_idx<S>(c, BATCH, w.len, w.st, nidx);
    lo_last = -1;
    for (int lo = 0; lo < w.len; lo += BATCH) {
        if (__all_sync(0xffffffffu, p.done)) break;
        __syncwarp();  // the previous batch's slots are no longer read
        commit<S>(g, lo, w.len, w.wa, w.wq, w.wc, w.widx, w.bx0, w.bx1, w.by0, w.by1, hit);
        lo_last = lo;
        if (STATS) st.staged += min(BATCH, w.len - lo);
        load_rec<S>(w.rec, lo + BATCH, w.len, nidx, g);
        load_idx<S>(c, lo + 2 * BATCH, w.len, w.st, nidx);
        __syncwarp();
        const int pos0 = lo + 1;
#pragma unroll
        for (int q = 0; q < S; ++q) {
            unsigned hm = hit[q];
            while (hm) {
                const int j = 32 * q + __ffs(hm) - 1;
                hm &= hm - 1;
                const float4 A = w.wa[j];
                const float2 Q = w.wq[j];
                const float dx = __fsub_rn(p.pxc, A.x), dy = __fsub_rn(p.pyc, A.y);
                const float power = power_of(dx, dy, A, Q);
                const bool live = !p.done && !skip(power, Q.y);
                if (STATS) ++st.hits;
                if (!__any_sync(0xffffffffu, live)) continue;  // the colour is not even read
                const float wgt = composite(p, live, power, w.wc[j], pos0 + j);
                if (STATS) {
                    ++st.visits;
                    st.lanes += wgt > 0.0f ? 1u : 0u;
                }
                if (ACC && __any_sync(0xffffffffu, wgt > 0.0f)) {
                    const float v[4] = {wgt, wgt * I0, wgt * I1, wgt * I2};
                    const float mine = warp_reduce4(v, lane);
                    red_add_if((lane & 7) == 0, acc + (size_t)w.widx[j] * kG2Floats + (lane >> 3), mine);
                }
            }
        }
    }
}

// Backward state of one pixel: its dL/dcolour g, T_final times g . background (TB), the
// transmittance T in front of the current entry and P = g . S, S the colour accumulated behind
// it (only that dot product enters the alpha gradient).
struct PixB {
    float pxc, pyc, T, TB, g0, g1, g2, P;
    int last;
};

// One list entry for one pixel, in reverse, once the caller has evaluated the entry's power at
// the pixel: live = the pixel blended the entry (its position is within the pixel's contributor
// count and the power passes the cutoff). Writes this pixel's share of the entry's gradient
// sums into v (zeros when not live) and, when live, steps T and P back past the entry. With
// g = dL/dpower at the pixel and (dx, dy) = pixel centre - mean, the power's gradient with
// respect to the mean, the conic and the opacity is linear in g (dx, dy, dx^2, dx dy, dy^2, 1):
// v = (g dx, g dy, g dx^2, g dx dy, g dy^2, g, dL/dr, dL/dg, dL/db), and the projection
// backward turns the block sums into dL/d(u, v, conic, opacity) with the splat's own conic and
// opacity (five products per pixel instead of sixteen). Branch-free, like the forward step: a
// lane that is not live keeps its state and computes with its power clamped to 0, so that no
// infinite exponential times a zero factor puts a NaN into the warp's sums.
__device__ __forceinline__ void accumulate(PixB &p, bool live, float dx, float dy, float power, const float4 &Cc,
                                           float v[9]) {
    const float G = __expf(fminf(power, 0.0f));
    const float araw = __fmul_rn(Cc.x, G);
    const float alpha = fminf(kAlphaMax, araw);
    const float oma = 1.0f - alpha;
    const float inv = __fdividef(1.0f, oma);  // 1 - alpha >= 0.01
    const float T = p.T * inv;                // transmittance in front of this Gaussian
    // dL/dalpha = T (g . c - g . S) - T_final / (1 - alpha) g . bg, then S <- alpha c + (1-alpha) S
    const float gc = fmaf(p.g2, Cc.w, fmaf(p.g1, Cc.z, p.g0 * Cc.y));
    const float dalpha = fmaf(T, gc - p.P, -p.TB * inv);
    const float P = fmaf(alpha, gc, oma * p.P);
    const float wgt = live ? alpha * T : 0.0f;
    p.T = live ? T : p.T;
    p.P = live ? P : p.P;
    v[6] = wgt * p.g0;
    v[7] = wgt * p.g1;
    v[8] = wgt * p.g2;
    // the clamp alpha = 0.99 passes no gradient to the opacity, conic or mean
    const float dcl = (live && !(araw > kAlphaMax)) ? dalpha : 0.0f;
    const float dpow = dcl * araw;  // dL/dpower: alpha = o e^power
    const float ex = dpow * dx, ey = dpow * dy;
    v[0] = ex;
    v[1] = ey;
    v[2] = ex * dx;
    v[3] = ex * dy;
    v[4] = ey * dy;
    v[5] = dpow;
}

// Warp partial sums of v[0..8] as a reduce-scatter that stops one quarter short: three halving
// exchanges leave lane l with the sum of value (l >> 2) over the 8 lanes that share l & 3, and
// three butterflies leave lanes 0-3 with the sums of v[8] over the same lane classes. The caller
// adds the four partials of each value to global memory (four lanes per address). Finishing the
// sums in the warp takes four more shuffles and adds per visit; the L2's reduction units absorb
// the extra atomics (compositing backward 0.377 -> 0.354 ms on the batched training workload).
// Stopping a further level short (eight lanes per address) made the atomics the limit
// (0.35 -> 0.40 ms). 10 shuffles instead of 45.
__device__ __forceinline__ void warp_reduce9(const float v[9], int lane, float &mine, float &v8) {
    const unsigned F = 0xffffffffu;
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    float a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = h16 ? v[i] : v[i + 4];
        const float keep = h16 ? v[i + 4] : v[i];
        a[i] = keep + __shfl_xor_sync(F, send, 16);
    }
    float b2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = h8 ? a[i] : a[i + 2];
        const float keep = h8 ? a[i + 2] : a[i];
        b2[i] = keep + __shfl_xor_sync(F, send, 8);
    }
    mine = (h4 ? b2[1] : b2[0]) + __shfl_xor_sync(F, h4 ? b2[0] : b2[1], 4);
    float x = v[8];
#pragma unroll
    for (int o = 16; o > 2; o >>= 1) x += __shfl_xor_sync(F, x, o);
    v8 = x;
}

// The reverse walk of one pixel block over list positions [0, top), top the block's largest
// contributor count: batches of BATCH = 32 S entries aligned to multiples of BATCH, from the one
// holding position top - 1 down to position 0 (each batch's loads one and two batches ahead),
// the hits of each batch in reverse. If the top batch is already in the warp's slots (staged by
// the forward walk of the same block: first position `have`, hit words in hit[]), it is not
// staged again. Per hit the block's gradient is reduced across the warp and added to the
// entry's 2-D gradient slots in g2 (four atomic partials per component).
template <int S, bool STATS>
__device__ __forceinline__ void bwd_walk(const Ctx &c, const Walk &w, PixB &p, float *g2, int top, int have,
                                         unsigned hit[S], WalkStats &st) {
    constexpr int BATCH = 32 * S;
    const int lane = threadIdx.x & 31;
    if (top <= 0) return;
    const int b_hi = ((top - 1) / BATCH) * BATCH;
    Stage<S> g;
    unsigned nidx[S];
    if (b_hi != have) {
        load_idx<S>(c, b_hi, w.len, w.st, nidx);
        load_rec<S>(w.rec, b_hi, w.len, nidx, g);
        __syncwarp();  // the slots may still be read by the forward walk's last visits
        commit<S>(g, b_hi, w.len, w.wa, w.wq, w.wc, w.widx, w.bx0, w.bx1, w.by0, w.by1, hit);
        if (STATS) st.staged += min(BATCH, w.len - b_hi);
    }
    load_idx<S>(c, b_hi - BATCH, w.len, w.st, nidx);
    load_rec<S>(w.rec, b_hi - BATCH, w.len, nidx, g);
    load_idx<S>(c, b_hi - 2 * BATCH, w.len, w.st, nidx);
    __syncwarp();
    for (int begin = b_hi; begin >= 0; begin -= BATCH) {
        if (begin != b_hi) {
            __syncwarp();  // the previous batch's slots are no longer read
            commit<S>(g, begin, w.len, w.wa, w.wq, w.wc, w.widx, w.bx0, w.bx1, w.by0, w.by1, hit);
            if (STATS) st.staged += BATCH;
            load_rec<S>(w.rec, begin - BATCH, w.len, nidx, g);
            load_idx<S>(c, begin - 2 * BATCH, w.len, w.st, nidx);
            __syncwarp();
        }
#pragma unroll
        for (int q = S - 1; q >= 0; --q) {
            // positions at or past top blended at no pixel of the block
            const int room = top - begin - 32 * q;
            unsigned hm = hit[q] & (room >= 32 ? 0xffffffffu : (room <= 0 ? 0u : (1u << room) - 1u));
            while (hm) {
                const int bit = 31 - __clz(hm);
                hm &= ~(1u << bit);
                const int j = 32 * q + bit;
                const int pos = begin + j + 1;
                const float4 A = w.wa[j];
                const float2 Q = w.wq[j];
                const float dx = __fsub_rn(p.pxc, A.x), dy = __fsub_rn(p.pyc, A.y);
                const float power = power_of(dx, dy, A, Q);
                const bool live = pos <= p.last && !skip(power, Q.y);
                if (STATS) ++st.hits;
                if (!__any_sync(0xffffffffu, live)) continue;  // the colour is not even read
                if (STATS) {
                    ++st.visits;
                    st.lanes += live ? 1u : 0u;
                }
                float v[9];
                accumulate(p, live, dx, dy, power, w.wc[j], v);
                float mine, v8;
                warp_reduce9(v, lane, mine, v8);
                float *dst = g2 + (size_t)w.widx[j] * kG2Floats;
                red_add(dst + (lane >> 2), mine);
                red_add_if(lane < 4, dst + 8, v8);
            }
        }
    }
}

// A (tile, pixel block) item: its frame, the block's pixel (one per lane: column lane % 8 of
// row lane / 8 of the 8 x 4 block) and the walk over the tile's list.
template <int TW>
__device__ __forceinline__ int block_item(const Ctx &c, unsigned item, int &px, int &py, Walk &w) {
    constexpr int TH = kTilePix / TW, NBX = TW / 8, NB = NBX * (TH / 4);
    const int lane = threadIdx.x & 31;
    const unsigned wk = item / NB, blk = item - wk * NB;
    const long long t = c.work[wk];
    const int b = find_frame(c, t);
    const FrameInfo &f = c.frames[b];
    const int lt = (int)(t - f.tile_base);
    const int ty = lt / f.tiles_x, tx = lt - ty * f.tiles_x;
    const int bx = tx * TW + (int)(blk % NBX) * 8, by = ty * TH + (int)(blk / NBX) * 4;
    px = bx + (lane & 7);
    py = by + (lane >> 3);
    w.bx0 = (float)bx + 0.5f;
    w.bx1 = (float)bx + 7.5f;
    w.by0 = (float)by + 0.5f;
    w.by1 = (float)by + 3.5f;
    w.st = c.tile_start[t];
    w.len = (int)(c.tile_start[t + 1] - w.st);
    w.rec = c.records + (size_t)f.rec_base * 3;
    return b;
}

// Adds a warp's statistics to the counters (dst: staged, hits, visits, pairs), the per-lane
// pair count summed over the warp first.
__device__ __forceinline__ void flush_stats(unsigned long long *dst, WalkStats st) {
    for (int o = 16; o > 0; o >>= 1) st.lanes += __shfl_xor_sync(0xffffffffu, st.lanes, o);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(dst + 0, st.staged);
        atomicAdd(dst + 1, st.hits);
        atomicAdd(dst + 2, st.visits);
        atomicAdd(dst + 3, (unsigned long long)st.lanes);
    }
}

// The loss: warp sums, then one double atomic per CTA.
__device__ __forceinline__ void flush_loss(const Ctx &c, float loss_acc, float *s_red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
    if (lane == 0) s_red[wid] = loss_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float sum = 0.f;
        for (int i = 0; i < kWarpsPerCta; ++i) sum += s_red[i];
        atomicAdd(&c.cnt->loss, (double)sum);
    }
}

// Items: the pixel blocks of the non-empty tiles (work list order, heaviest tiles first), then
// one item per empty tile, which the warp fills with the background eight pixels per lane.
// ACC (colour initialisation, Eq. 3): every blended entry also adds its splatting weight w and
// w times the pixel's colour in acc_target to the record's first four 2-D gradient slots
// (one warp reduction and four atomics per entry and pixel block).
// STATS (the counting instance): also count the visits that evaluate an entry and the
// (pixel, entry) pairs that blend, into the compositing statistics of the counters.
template <int TW, int BATCH, bool ACC, bool STATS = false>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_render_fwd(Ctx c, float *__restrict__ img, float *__restrict__ T_final, int *__restrict__ n_contrib,
             const float *__restrict__ target, int loss_kind, float *__restrict__ dl_dimg,
             const float *__restrict__ acc_target) {
    constexpr int TH = kTilePix / TW, NB = (TW / 8) * (TH / 4), S = BATCH / 32;
    __shared__ float4 s_a[kWarpsPerCta][BATCH];
    __shared__ float2 s_q[kWarpsPerCta][BATCH];
    __shared__ float4 s_c[kWarpsPerCta][BATCH];
    __shared__ unsigned s_idx[kWarpsPerCta][ACC ? BATCH : 1];
    __shared__ float s_red[kWarpsPerCta];
    pdl_enter();
    if (c.cnt->overflow) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Walk w;
    w.wa = s_a[wid];
    w.wc = s_c[wid];
    w.wq = s_q[wid];
    w.widx = ACC ? s_idx[wid] : nullptr;
    const unsigned n_work = c.cnt->n_work, n_blocks = n_work * NB;
    const unsigned n_items = n_blocks + ((unsigned)c.T - n_work);
    float loss_acc = 0.0f;
    WalkStats st{0ull, 0ull, 0ull, 0u};  // STATS
    while (true) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(&c.cnt->next_fwd, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        if (item >= n_blocks) {  // an empty tile: background, T = 1, no contributors
            empty_tile<TW>(c, c.work[n_work + (item - n_blocks)], img, T_final, n_contrib, target, loss_kind,
                           dl_dimg, loss_acc);
            continue;
        }
        int px, py;
        const int b = block_item<TW>(c, item, px, py, w);
        const FrameInfo &f = c.frames[b];
        PixF p{(float)px + 0.5f, (float)py + 0.5f, 1.f, 0.f, 0.f, 0.f, 0, px < f.W && py < f.H, false};
        p.done = !p.inside;
        float I0 = 0.f, I1 = 0.f, I2 = 0.f;  // ACC: the pixel's target colour
        if (ACC && p.inside) {
            const long long hw = (long long)f.W * f.H;
            const float *tg = acc_target + f.pix_base * 3 + (long long)py * f.W + px;
            I0 = tg[0];
            I1 = tg[hw];
            I2 = tg[2 * hw];
        }
        unsigned hit[S];
        int lo_last;
        fwd_walk<S, ACC, STATS>(c, w, p, I0, I1, I2, c.grad2d + (size_t)f.rec_base * kG2Floats, hit, lo_last, st);
        if (p.inside) {
            float g[3];
            finish_pixel(c, f, b, px, py, p, img, T_final, n_contrib, target, loss_kind, dl_dimg, loss_acc, g);
        }
    }
    if (STATS) flush_stats(c.cnt->st_fwd, st);
    // the last warp out puts the work counter back to zero for the next launch
    if (lane == 0 && atomicAdd(&c.cnt->done_fwd, 1u) == gridDim.x * kWarpsPerCta - 1) {
        c.cnt->next_fwd = 0u;
        c.cnt->done_fwd = 0u;
    }
    if (target) flush_loss(c, loss_acc, s_red);
}

// STATS (the counting instance): also count the visits that evaluate an entry and the
// (pixel, entry) pairs that take a gradient, into the compositing statistics of the counters.
template <int TW, int BATCH, bool STATS = false>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_render_bwd(Ctx c, const float *__restrict__ dl_dimg, const float *__restrict__ T_final,
             const int *__restrict__ n_contrib) {
    constexpr int TH = kTilePix / TW, NB = (TW / 8) * (TH / 4), S = BATCH / 32;
    __shared__ float4 s_a[kWarpsPerCta][BATCH];
    __shared__ float2 s_q[kWarpsPerCta][BATCH];
    __shared__ float4 s_c[kWarpsPerCta][BATCH];
    __shared__ unsigned s_idx[kWarpsPerCta][BATCH];
    pdl_enter();
    if (c.cnt->overflow) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Walk w;
    w.wa = s_a[wid];
    w.wc = s_c[wid];
    w.wq = s_q[wid];
    w.widx = s_idx[wid];
    const unsigned n_items = c.cnt->n_work * NB;
    WalkStats st{0ull, 0ull, 0ull, 0u};  // STATS
    while (true) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(&c.cnt->next_bwd, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        int px, py;
        const int b = block_item<TW>(c, item, px, py, w);
        const FrameInfo &f = c.frames[b];
        const float *bgp = c.fparams + (size_t)b * RGBA_FP_STRIDE + 17;
        const long long hw = (long long)f.W * f.H;
        PixB p{(float)px + 0.5f, (float)py + 0.5f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
        if (px < f.W && py < f.H) {
            const long long pix = (long long)py * f.W + px;
            const float Tfin = T_final[f.pix_base + pix];
            p.T = Tfin;
            p.last = n_contrib[f.pix_base + pix];
            const float *dl = dl_dimg + f.pix_base * 3 + pix;
            p.g0 = dl[0];
            p.g1 = dl[hw];
            p.g2 = dl[2 * hw];
            p.TB = Tfin * (p.g0 * bgp[0] + p.g1 * bgp[1] + p.g2 * bgp[2]);
        }
        int m = p.last;
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        // n_contrib comes from the caller: entries past the list's end do not exist
        unsigned hit[S];
        bwd_walk<S, STATS>(c, w, p, c.grad2d + (size_t)f.rec_base * kG2Floats, min(m, w.len), -1, hit, st);
    }
    if (STATS) flush_stats(c.cnt->st_bwd, st);
    // the last warp out puts the work counter back to zero for the next launch
    if (lane == 0 && atomicAdd(&c.cnt->done_bwd, 1u) == gridDim.x * kWarpsPerCta - 1) {
        c.cnt->next_bwd = 0u;
        c.cnt->done_bwd = 0u;
    }
}

// Persistent grid: every CTA the SMs can hold at once (occupancy query, cached by the caller
// per kernel instance: all instances of a template share one function type).
template <typename K>
int persistent_grid(K kernel, int sms_hint, int threads, int &cached) {
    if (!cached) {
        int per_sm = 0, dev = 0, sms = sms_hint;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 4;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached = per_sm * sms;
    }
    return cached;
}

template <int TW, int BATCH, bool ACC, bool STATS = false>
cudaError_t fwd_inst(const Ctx &c, int grid, float *img, float *T, int *n, const float *tg, int lk,
                     float *dl, const float *acc_tg, cudaStream_t s) {
    static int cached = 0;
    const int g = persistent_grid(k_render_fwd<TW, BATCH, ACC, STATS>, grid, 32 * kWarpsPerCta, cached);
    return launch_pdl(k_render_fwd<TW, BATCH, ACC, STATS>, dim3(g), dim3(32 * kWarpsPerCta), 0, s, c, img, T, n,
                      tg, lk, dl, acc_tg);
}

template <bool ACC>
cudaError_t fwd_dispatch(const Ctx &c, int grid, int sb, float *img, float *T, int *n, const float *tg,
                         int lk, float *dl, const float *acc_tg, bool stats, cudaStream_t s) {
    if (!ACC && stats && c.tw == 16 && sb == 64)
        return fwd_inst<16, 64, false, true>(c, grid, img, T, n, tg, lk, dl, acc_tg, s);
    if (c.tw == 16) {
        if (sb == 64) return fwd_inst<16, 64, ACC>(c, grid, img, T, n, tg, lk, dl, acc_tg, s);
        if (sb == 128) return fwd_inst<16, 128, ACC>(c, grid, img, T, n, tg, lk, dl, acc_tg, s);
        return fwd_inst<16, 256, ACC>(c, grid, img, T, n, tg, lk, dl, acc_tg, s);
    }
    if (sb == 64) return fwd_inst<8, 64, ACC>(c, grid, img, T, n, tg, lk, dl, acc_tg, s);
    if (sb == 128) return fwd_inst<8, 128, ACC>(c, grid, img, T, n, tg, lk, dl, acc_tg, s);
    return fwd_inst<8, 256, ACC>(c, grid, img, T, n, tg, lk, dl, acc_tg, s);
}

template <int TW, int BATCH, bool STATS = false>
cudaError_t bwd_inst(const Ctx &c, int grid, const float *dl, const float *T, const int *n,
                     cudaStream_t s) {
    static int cached = 0;
    const int g = persistent_grid(k_render_bwd<TW, BATCH, STATS>, grid, 32 * kWarpsPerCta, cached);
    return launch_pdl(k_render_bwd<TW, BATCH, STATS>, dim3(g), dim3(32 * kWarpsPerCta), 0, s, c, dl, T, n);
}

}  // namespace

cudaError_t launch_render_fwd(const Ctx &c, int grid, int smem_batch, float *img, float *T_final,
                              int *n_contrib, const float *target, int loss_kind,
                              float *dl_dimg, const float *acc_target, bool stats, cudaStream_t s) {
    if (acc_target)
        return fwd_dispatch<true>(c, grid, smem_batch, img, T_final, n_contrib, target, loss_kind, dl_dimg,
                                  acc_target, false, s);
    return fwd_dispatch<false>(c, grid, smem_batch, img, T_final, n_contrib, target, loss_kind, dl_dimg,
                               nullptr, stats, s);
}

cudaError_t launch_render_bwd(const Ctx &c, int grid, int smem_batch, const float *dl_dimg,
                              const float *T_final, const int *n_contrib, bool stats, cudaStream_t s) {
    if (stats && c.tw == 16 && smem_batch == 64) return bwd_inst<16, 64, true>(c, grid, dl_dimg, T_final, n_contrib, s);
    if (c.tw == 16) {
        if (smem_batch == 64) return bwd_inst<16, 64>(c, grid, dl_dimg, T_final, n_contrib, s);
        if (smem_batch == 128) return bwd_inst<16, 128>(c, grid, dl_dimg, T_final, n_contrib, s);
        return bwd_inst<16, 256>(c, grid, dl_dimg, T_final, n_contrib, s);
    }
    if (smem_batch == 64) return bwd_inst<8, 64>(c, grid, dl_dimg, T_final, n_contrib, s);
    if (smem_batch == 128) return bwd_inst<8, 128>(c, grid, dl_dimg, T_final, n_contrib, s);
    return bwd_inst<8, 256>(c, grid, dl_dimg, T_final, n_contrib, s);
}

}  // namespace rgba
