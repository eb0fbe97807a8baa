// Front-to-back alpha compositing ("rasterize", RGBAvatar Sec. 3.2 on the 3DGS renderer) and
// its exact reverse. One 256-thread CTA owns one screen tile (16x16 or 8x32 pixels) at a time;
// persistent CTAs pull (frame, tile) items from the device work list, so every frame of every
// avatar in the batch shares one launch. Gaussians are staged in shared memory in rounds of
// BATCH entries, each with the box of its alpha >= 1/255 ellipse; every warp owns a compact
// block of pixels (8 x 4 in the forward, 8 x 8 with two pixels per lane in the backward) and
// skips, with one uniform test, the entries whose box misses its block. A CTA stops as soon as
// every pixel of its tile is saturated.
//
// Per pixel, with d = pixel centre - mean:
//   power = -(a dx^2 + c dy^2) / 2 - b dx dy  (skip if > 0)
//   alpha = min(0.99, o exp(power))            (skip if < 1/255)
//   stop, without blending, once T (1 - alpha) < 1e-4
// The backward recomputes each alpha with the same instruction sequence as the forward, walks
// the list backwards from the stored contributor count, and recovers T by division by
// (1 - alpha). Per-Gaussian gradients are reduced across the warp (reduce-scatter), then
// across the CTA in shared memory, and reach global memory as one atomic per Gaussian, tile
// and component.
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
__device__ __forceinline__ void stage_splat(const float4 *rec, unsigned idx, float4 &sa, float2 &sq,
                                            float4 &sc, float4 &sb) {
    const float4 r0 = rec[(size_t)idx * 3 + 0], r1 = rec[(size_t)idx * 3 + 1];
    const float r2 = rec[(size_t)idx * 3 + 2].x;
    sa = make_float4(r0.x, r0.y, -0.5f * r0.z, -r0.w);
    const float tau = -__logf(255.0f * r1.y);
    sq = make_float2(-0.5f * r1.x, tau);
    sc = make_float4(r1.y, r1.z, r1.w, r2);
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

constexpr int kThreads = kTilePix / 2;  // backward: two pixels per thread, rows y and y + TH/2

struct PixF {
    float pxc, pyc, T, C0, C1, C2;
    int last;
    bool inside, done;
};

// One list entry for one pixel (forward); marks the pixel done when it saturates.
__device__ __forceinline__ void composite(PixF &p, const float4 *s_a, const float2 *s_q,
                                          const float4 *s_c, int j, int pos) {
    const float4 A = s_a[j];
    const float2 Q = s_q[j];
    const float dx = __fsub_rn(p.pxc, A.x), dy = __fsub_rn(p.pyc, A.y);
    const float power = power_of(dx, dy, A, Q);
    if (skip(power, Q.y)) return;
    const float4 Cc = s_c[j];
    const float alpha = fminf(kAlphaMax, __fmul_rn(Cc.x, __expf(power)));
    const float testT = p.T * (1.0f - alpha);
    if (testT < kTMin) {
        p.done = true;
        return;
    }
    const float wgt = alpha * p.T;
    p.C0 = fmaf(Cc.y, wgt, p.C0);
    p.C1 = fmaf(Cc.z, wgt, p.C1);
    p.C2 = fmaf(Cc.w, wgt, p.C2);
    p.T = testT;
    p.last = pos;
}

template <int TW, int BATCH>
__global__ void __launch_bounds__(kTilePix)
k_render_fwd(Ctx c, float *__restrict__ img, float *__restrict__ T_final, int *__restrict__ n_contrib,
             const float *__restrict__ target, int loss_kind, float *__restrict__ dl_dimg) {
    constexpr int TH = kTilePix / TW;
    __shared__ float4 s_a[BATCH];
    __shared__ float2 s_q[BATCH];
    __shared__ float4 s_c[BATCH];
    __shared__ float4 s_box[BATCH];
    __shared__ unsigned s_w;
    __shared__ float s_red[kTilePix / 32];
    if (c.cnt->overflow) return;
    const int tid = threadIdx.x;
    float loss_acc = 0.0f;
    while (true) {
        if (tid == 0) s_w = atomicAdd(&c.cnt->next_fwd, 1u);
        __syncthreads();
        const unsigned w = s_w;
        __syncthreads();
        if (w >= (unsigned)c.T) break;
        const long long t = c.work[w];
        const int b = find_frame(c, t);
        const FrameInfo &f = c.frames[b];
        const int lt = (int)(t - f.tile_base);
        const int ty = lt / f.tiles_x, tx = lt - ty * f.tiles_x;
        // warp w owns an 8 x 4 block of the tile: column block w % (TW / 8), row block w / (TW / 8)
        const int warp = tid >> 5, lane = tid & 31;
        const int bx = tx * TW + (warp % (TW / 8)) * 8, by = ty * TH + (warp / (TW / 8)) * 4;
        const int px = bx + (lane & 7), py = by + (lane >> 3);
        const float bx0 = (float)bx + 0.5f, bx1 = (float)bx + 7.5f, by0 = (float)by + 0.5f, by1 = (float)by + 3.5f;
        PixF p{(float)px + 0.5f, (float)py + 0.5f, 1.f, 0.f, 0.f, 0.f, 0, px < f.W && py < f.H, false};
        p.done = !p.inside;
        const unsigned st = c.tile_start[t], en = c.tile_start[t + 1];
        const float4 *rec = c.records + (size_t)f.rec_base * 3;
        for (unsigned base = st; base < en; base += BATCH) {
            if (__syncthreads_count(p.done) == kTilePix) break;
            if (tid < BATCH && base + tid < en)
                stage_splat(rec, c.sorted[base + tid], s_a[tid], s_q[tid], s_c[tid], s_box[tid]);
            __syncthreads();
            const int cnt = min(BATCH, (int)(en - base));
            const int pos0 = (int)(base - st) + 1;
            // 32 entries at a time: each lane tests one box against the warp's block, and the
            // warp then visits only the entries that hit, in list order
            for (int j0 = 0; j0 < cnt; j0 += 32) {
                if (__all_sync(0xffffffffu, p.done)) break;
                const int jl = j0 + lane;
                unsigned hits = __ballot_sync(0xffffffffu, jl < cnt && !box_misses(s_box[jl], bx0, bx1, by0, by1));
                while (hits) {
                    const int j = j0 + __ffs(hits) - 1;
                    hits &= hits - 1;
                    if (!p.done) composite(p, s_a, s_q, s_c, j, pos0 + j);
                }
            }
        }
        if (p.inside) {
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
            if (target) {
                const float *tg = target + f.pix_base * 3 + pix;
                const float scale = 1.0f / (3.0f * (float)hw * (float)c.B);
                const float d0 = o0 - tg[0], d1 = o1 - tg[hw], d2 = o2 - tg[2 * hw];
                float *dl = dl_dimg + f.pix_base * 3 + pix;
                if (loss_kind == RGBA_LOSS_L1) {
                    loss_acc += (fabsf(d0) + fabsf(d1) + fabsf(d2)) * scale;
                    dl[0] = d0 > 0.f ? scale : (d0 < 0.f ? -scale : 0.f);
                    dl[hw] = d1 > 0.f ? scale : (d1 < 0.f ? -scale : 0.f);
                    dl[2 * hw] = d2 > 0.f ? scale : (d2 < 0.f ? -scale : 0.f);
                } else {
                    loss_acc += 0.5f * (d0 * d0 + d1 * d1 + d2 * d2) * scale;
                    dl[0] = d0 * scale;
                    dl[hw] = d1 * scale;
                    dl[2 * hw] = d2 * scale;
                }
            }
        }
    }
    if (target) {
        for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
        if ((tid & 31) == 0) s_red[tid >> 5] = loss_acc;
        __syncthreads();
        if (tid == 0) {
            float sum = 0.f;
            for (int i = 0; i < kTilePix / 32; ++i) sum += s_red[i];
            atomicAdd(&c.cnt->loss, (double)sum);
        }
    }
}

struct PixB {
    float pxc, pyc, T, Tfin, g0, g1, g2, bgdot, S0, S1, S2;
    int last;
};

// One list entry for one pixel, in reverse; adds this pixel's share of the entry's gradient
// dL/d(u, v, conic a, b, c, opacity, r, g, b) into v. Returns whether the pixel blended it.
__device__ __forceinline__ bool accumulate(PixB &p, int pos, const float4 &A, const float2 &Q,
                                           const float4 &Cc, float v[9]) {
    if (pos > p.last) return false;
    const float dx = __fsub_rn(p.pxc, A.x), dy = __fsub_rn(p.pyc, A.y);
    const float power = power_of(dx, dy, A, Q);
    if (skip(power, Q.y)) return false;
    const float4 Bv = make_float4(Q.x, Cc.x, Cc.y, Cc.z);  // -c/2, opacity, r, g
    const float cb = Cc.w;
    const float G = __expf(power);
    const float araw = __fmul_rn(Bv.y, G);
    const float alpha = fminf(kAlphaMax, araw);
    const float oma = 1.0f - alpha;
    const float inv = __fdividef(1.0f, oma);  // 1 - alpha >= 0.01
    p.T = p.T * inv;  // transmittance in front of this Gaussian
    const float wgt = alpha * p.T;
    v[6] = fmaf(wgt, p.g0, v[6]);
    v[7] = fmaf(wgt, p.g1, v[7]);
    v[8] = fmaf(wgt, p.g2, v[8]);
    float dalpha = p.T * (p.g0 * (Bv.z - p.S0) + p.g1 * (Bv.w - p.S1) + p.g2 * (cb - p.S2));
    dalpha -= p.Tfin * inv * p.bgdot;
    p.S0 = fmaf(alpha, Bv.z, oma * p.S0);
    p.S1 = fmaf(alpha, Bv.w, oma * p.S1);
    p.S2 = fmaf(alpha, cb, oma * p.S2);
    if (!(araw > kAlphaMax)) {
        v[5] = fmaf(dalpha, G, v[5]);
        const float dpow = dalpha * Bv.y * G;
        v[2] = fmaf(-0.5f * dx * dx, dpow, v[2]);
        v[3] = fmaf(-dx * dy, dpow, v[3]);
        v[4] = fmaf(-0.5f * dy * dy, dpow, v[4]);
        // conic a = -2 A.z, b = -A.w, c = -2 B.x
        v[0] = fmaf(-dpow, 2.0f * A.z * dx + A.w * dy, v[0]);
        v[1] = fmaf(-dpow, 2.0f * Bv.x * dy + A.w * dx, v[1]);
    }
    return true;
}

// Warp sum of v[0..8] as a reduce-scatter: three halving exchanges leave lane l with the partial
// sum of value (l >> 2) over the 8 lanes that share l & 3, two more butterflies finish it;
// v[8] takes a plain butterfly. 14 shuffles instead of 45.
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
    float m = (h4 ? b2[1] : b2[0]) + __shfl_xor_sync(F, h4 ? b2[0] : b2[1], 4);
    m += __shfl_xor_sync(F, m, 2);
    m += __shfl_xor_sync(F, m, 1);
    mine = m;
    float x = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(F, x, o);
    v8 = x;
}

template <int TW, int BATCH>
__global__ void __launch_bounds__(kThreads)
k_render_bwd(Ctx c, const float *__restrict__ dl_dimg, const float *__restrict__ T_final,
             const int *__restrict__ n_contrib) {
    constexpr int TH = kTilePix / TW;
    __shared__ float4 s_a[BATCH];
    __shared__ float2 s_q[BATCH];
    __shared__ float4 s_c[BATCH];
    __shared__ float4 s_box[BATCH];
    __shared__ unsigned s_idx[BATCH];
    __shared__ float s_g[BATCH][9];  // per entry: stride 9 keeps lanes on distinct banks
    __shared__ unsigned s_w;
    __shared__ int s_max;
    if (c.cnt->overflow) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned n_work = c.cnt->n_work;
    while (true) {
        if (tid == 0) {
            s_w = atomicAdd(&c.cnt->next_bwd, 1u);
            s_max = 0;
        }
        __syncthreads();
        const unsigned w = s_w;
        if (w >= n_work) break;
        const long long t = c.work[w];
        const int b = find_frame(c, t);
        const FrameInfo &f = c.frames[b];
        const int lt = (int)(t - f.tile_base);
        const int ty = lt / f.tiles_x, tx = lt - ty * f.tiles_x;
        // warp w owns an 8 x 8 block: column block w % (TW / 8), row block w / (TW / 8); each
        // lane two pixels of the block, rows lane / 8 and lane / 8 + 4
        const int warp = tid >> 5;
        const int bx = tx * TW + (warp % (TW / 8)) * 8, by = ty * TH + (warp / (TW / 8)) * 8;
        const int px = bx + (lane & 7), py0 = by + (lane >> 3);
        const float bx0 = (float)bx + 0.5f, bx1 = (float)bx + 7.5f, by0 = (float)by + 0.5f, by1 = (float)by + 7.5f;
        const unsigned st = c.tile_start[t], list_len = c.tile_start[t + 1] - st;
        const float4 *rec = c.records + (size_t)f.rec_base * 3;
        float *g2 = c.grad2d + (size_t)f.rec_base * kG2Floats;
        const float *bgp = c.fparams + (size_t)b * RGBA_FP_STRIDE + 17;
        const long long hw = (long long)f.W * f.H;
        PixB p[2];
        int m = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int py = py0 + h * 4;
            p[h] = PixB{(float)px + 0.5f, (float)py + 0.5f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
            if (px < f.W && py < f.H) {
                const long long pix = (long long)py * f.W + px;
                p[h].Tfin = T_final[f.pix_base + pix];
                p[h].T = p[h].Tfin;
                p[h].last = n_contrib[f.pix_base + pix];
                const float *dl = dl_dimg + f.pix_base * 3 + pix;
                p[h].g0 = dl[0];
                p[h].g1 = dl[hw];
                p[h].g2 = dl[2 * hw];
                p[h].bgdot = p[h].g0 * bgp[0] + p[h].g1 * bgp[1] + p[h].g2 * bgp[2];
                m = max(m, p[h].last);
            }
        }
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) atomicMax(&s_max, m);
        __syncthreads();
        const int max_last = min(s_max, (int)list_len);  // n_contrib comes from the caller
        const int warp_last = m;  // entries past it are skipped by the whole warp
        for (int end = max_last; end > 0; end -= BATCH) {
            const int begin = max(0, end - BATCH);
            const int cnt = end - begin;
            for (int e = tid; e < cnt; e += kThreads) {
                const unsigned idx = c.sorted[st + begin + e];
                s_idx[e] = idx;
                stage_splat(rec, idx, s_a[e], s_q[e], s_c[e], s_box[e]);
            }
            for (int e = tid; e < 9 * BATCH; e += kThreads) (&s_g[0][0])[e] = 0.f;
            __syncthreads();
            // 32 entries at a time from the top: each lane tests one box against the warp's
            // block, and the warp then visits only the entries that hit, in reverse list order
            const int jtop = min(cnt, warp_last - begin);
            for (int j0 = (jtop - 1) & ~31; j0 >= 0; j0 -= 32) {
                const int jl = j0 + lane;
                unsigned hits = __ballot_sync(0xffffffffu, jl < jtop && !box_misses(s_box[jl], bx0, bx1, by0, by1));
                while (hits) {
                    const int bit = 31 - __clz(hits);
                    hits &= ~(1u << bit);
                    const int j = j0 + bit;
                    const int pos = begin + j + 1;
                    const float4 A = s_a[j], Cc = s_c[j];
                    const float2 Q = s_q[j];
                    float v[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) v[q] = 0.f;
                    bool any = accumulate(p[0], pos, A, Q, Cc, v);
                    any |= accumulate(p[1], pos, A, Q, Cc, v);
                    if (__any_sync(0xffffffffu, any)) {
                        float mine, v8;
                        warp_reduce9(v, lane, mine, v8);
                        if ((lane & 3) == 0) atomicAdd(&s_g[j][lane >> 2], mine);
                        if (lane == 0) atomicAdd(&s_g[j][8], v8);
                    }
                }
            }
            __syncthreads();
            for (int e = tid; e < cnt; e += kThreads) {
                float *dst = g2 + (size_t)s_idx[e] * kG2Floats;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const float x = s_g[e][q];
                    if (x != 0.f) atomicAdd(dst + q, x);
                }
            }
            __syncthreads();
        }
    }
}

// Persistent grid: every CTA the SMs can hold at once (occupancy query, cached per kernel).
template <typename K>
int persistent_grid(K kernel, int sms_hint, int threads) {
    static int cached = 0;
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

template <int TW, int BATCH>
cudaError_t fwd_inst(const Ctx &c, int grid, float *img, float *T, int *n, const float *tg, int lk,
                     float *dl, cudaStream_t s) {
    const int g = persistent_grid(k_render_fwd<TW, BATCH>, grid, kTilePix);
    k_render_fwd<TW, BATCH><<<g, kTilePix, 0, s>>>(c, img, T, n, tg, lk, dl);
    return cudaGetLastError();
}

template <int TW, int BATCH>
cudaError_t bwd_inst(const Ctx &c, int grid, const float *dl, const float *T, const int *n,
                     cudaStream_t s) {
    const int g = persistent_grid(k_render_bwd<TW, BATCH>, grid, kThreads);
    k_render_bwd<TW, BATCH><<<g, kThreads, 0, s>>>(c, dl, T, n);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render_fwd(const Ctx &c, int grid, int smem_batch, float *img, float *T_final,
                              int *n_contrib, const float *target, int loss_kind,
                              float *dl_dimg, const long long *, cudaStream_t s) {
    if (c.tw == 16) {
        if (smem_batch == 64) return fwd_inst<16, 64>(c, grid, img, T_final, n_contrib, target, loss_kind, dl_dimg, s);
        if (smem_batch == 128) return fwd_inst<16, 128>(c, grid, img, T_final, n_contrib, target, loss_kind, dl_dimg, s);
        return fwd_inst<16, 256>(c, grid, img, T_final, n_contrib, target, loss_kind, dl_dimg, s);
    }
    if (smem_batch == 64) return fwd_inst<8, 64>(c, grid, img, T_final, n_contrib, target, loss_kind, dl_dimg, s);
    if (smem_batch == 128) return fwd_inst<8, 128>(c, grid, img, T_final, n_contrib, target, loss_kind, dl_dimg, s);
    return fwd_inst<8, 256>(c, grid, img, T_final, n_contrib, target, loss_kind, dl_dimg, s);
}

cudaError_t launch_render_bwd(const Ctx &c, int grid, int smem_batch, const float *dl_dimg,
                              const float *T_final, const int *n_contrib, cudaStream_t s) {
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
