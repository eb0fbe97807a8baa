// Front-to-back alpha compositing ("rasterize", RGBAvatar Sec. 3.2 on the 3DGS renderer) and
// its exact reverse. One 256-thread CTA owns one screen tile (16x16 or 8x32 pixels) at a time;
// persistent CTAs pull (frame, tile) items from the device work list, so every frame of every
// avatar in the batch shares one launch. Gaussians are staged in shared memory in rounds of
// BATCH entries; a CTA stops as soon as every pixel of its tile is saturated.
//
// Per pixel, with d = pixel centre - mean:
//   power = -(a dx^2 + c dy^2) / 2 - b dx dy  (skip if > 0)
//   alpha = min(0.99, o exp(power))            (skip if < 1/255)
//   stop, without blending, once T (1 - alpha) < 1e-4
// The backward recomputes each alpha with the same instruction sequence as the forward, walks
// the list backwards from the stored contributor count, and recovers T by division by
// (1 - alpha). Per-Gaussian gradients are reduced across the warp, then across the CTA in
// shared memory, and reach global memory as one atomic per Gaussian, tile and component.
#include "rgba_internal.cuh"

namespace rgba {
namespace {

constexpr float kAlphaMin = 1.0f / 255.0f;
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

// power and raw alpha; both kernels call this so their decisions agree bit for bit
__device__ __forceinline__ float eval_power(float dx, float dy, float a, float b, float cc) {
    float q = __fmaf_rn(cc, __fmul_rn(dy, dy), __fmul_rn(__fmul_rn(a, dx), dx));
    return __fmaf_rn(-0.5f, q, -__fmul_rn(__fmul_rn(b, dx), dy));
}

template <int TW, int BATCH>
__global__ void __launch_bounds__(kTilePix)
k_render_fwd(Ctx c, float *__restrict__ img, float *__restrict__ T_final, int *__restrict__ n_contrib,
             const float *__restrict__ target, int loss_kind, float *__restrict__ dl_dimg) {
    constexpr int TH = kTilePix / TW;
    __shared__ float4 s_a[BATCH];  // u, v, conic a, conic b
    __shared__ float4 s_b[BATCH];  // conic c, opacity, r, g
    __shared__ float s_c[BATCH];   // b
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
        const int px = tx * TW + (tid % TW), py = ty * TH + (tid / TW);
        const bool inside = px < f.W && py < f.H;
        const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
        const unsigned st = c.tile_start[t], en = c.tile_start[t + 1];
        const float4 *rec = c.records + (size_t)f.rec_base * 3;
        float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        int last = 0;
        bool done = !inside;
        for (unsigned base = st; base < en; base += BATCH) {
            if (__syncthreads_count(done) == kTilePix) break;
            if (tid < BATCH && base + tid < en) {
                const unsigned idx = c.sorted[base + tid];
                s_a[tid] = rec[(size_t)idx * 3 + 0];
                s_b[tid] = rec[(size_t)idx * 3 + 1];
                s_c[tid] = rec[(size_t)idx * 3 + 2].x;
            }
            __syncthreads();
            const int cnt = min(BATCH, (int)(en - base));
            if (!done) {
                for (int j = 0; j < cnt; ++j) {
                    const float4 A = s_a[j];
                    const float dx = __fsub_rn(pxc, A.x), dy = __fsub_rn(pyc, A.y);
                    const float4 Bv = s_b[j];
                    const float power = eval_power(dx, dy, A.z, A.w, Bv.x);
                    if (power > 0.0f) continue;
                    const float alpha = fminf(kAlphaMax, __fmul_rn(Bv.y, __expf(power)));
                    if (alpha < kAlphaMin) continue;
                    const float testT = T * (1.0f - alpha);
                    if (testT < kTMin) {
                        done = true;
                        break;
                    }
                    const float wgt = alpha * T;
                    C0 = fmaf(Bv.z, wgt, C0);
                    C1 = fmaf(Bv.w, wgt, C1);
                    C2 = fmaf(s_c[j], wgt, C2);
                    T = testT;
                    last = (int)(base - st) + j + 1;
                }
            }
        }
        if (inside) {
            const float *bg = c.fparams + (size_t)b * RGBA_FP_STRIDE + 17;
            const long long hw = (long long)f.W * f.H;
            const long long pix = (long long)py * f.W + px;
            float *im = img + f.pix_base * 3 + pix;
            const float o0 = fmaf(T, bg[0], C0), o1 = fmaf(T, bg[1], C1), o2 = fmaf(T, bg[2], C2);
            im[0] = o0;
            im[hw] = o1;
            im[2 * hw] = o2;
            T_final[f.pix_base + pix] = T;
            n_contrib[f.pix_base + pix] = last;
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
            float s = 0.f;
            for (int i = 0; i < kTilePix / 32; ++i) s += s_red[i];
            atomicAdd(&c.cnt->loss, (double)s);
        }
    }
}

template <int TW, int BATCH>
__global__ void __launch_bounds__(kTilePix)
k_render_bwd(Ctx c, const float *__restrict__ dl_dimg, const float *__restrict__ T_final,
             const int *__restrict__ n_contrib) {
    constexpr int TH = kTilePix / TW;
    __shared__ float4 s_a[BATCH];
    __shared__ float4 s_b[BATCH];
    __shared__ float s_c[BATCH];
    __shared__ unsigned s_idx[BATCH];
    __shared__ float s_g[9][BATCH];
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
        const int px = tx * TW + (tid % TW), py = ty * TH + (tid / TW);
        const bool inside = px < f.W && py < f.H;
        const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
        const unsigned st = c.tile_start[t], list_len = c.tile_start[t + 1] - st;
        const float4 *rec = c.records + (size_t)f.rec_base * 3;
        float *g2 = c.grad2d + (size_t)f.rec_base * kG2Floats;
        const float *bgp = c.fparams + (size_t)b * RGBA_FP_STRIDE + 17;
        float T = 0.f, Tfin = 0.f, g0 = 0.f, g1 = 0.f, gb2 = 0.f, bgdot = 0.f;
        int last = 0;
        if (inside) {
            const long long hw = (long long)f.W * f.H;
            const long long pix = (long long)py * f.W + px;
            Tfin = T_final[f.pix_base + pix];
            T = Tfin;
            last = n_contrib[f.pix_base + pix];
            const float *dl = dl_dimg + f.pix_base * 3 + pix;
            g0 = dl[0];
            g1 = dl[hw];
            gb2 = dl[2 * hw];
            bgdot = g0 * bgp[0] + g1 * bgp[1] + gb2 * bgp[2];
        }
        int m = last;
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) atomicMax(&s_max, m);
        __syncthreads();
        const int max_last = min(s_max, (int)list_len);  // n_contrib comes from the caller
        float S0 = 0.f, S1 = 0.f, S2 = 0.f;  // normalised colour behind the current entry
        for (int end = max_last; end > 0; end -= BATCH) {
            const int begin = max(0, end - BATCH);
            const int cnt = end - begin;
            if (tid < cnt) {
                const unsigned idx = c.sorted[st + begin + tid];
                s_idx[tid] = idx;
                s_a[tid] = rec[(size_t)idx * 3 + 0];
                s_b[tid] = rec[(size_t)idx * 3 + 1];
                s_c[tid] = rec[(size_t)idx * 3 + 2].x;
            }
            for (int e = tid; e < 9 * BATCH; e += kTilePix) (&s_g[0][0])[e] = 0.f;
            __syncthreads();
            for (int j = cnt - 1; j >= 0; --j) {
                const int pos = begin + j + 1;
                float v[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) v[q] = 0.f;
                bool contrib = false;
                if (pos <= last) {
                    const float4 A = s_a[j];
                    const float dx = __fsub_rn(pxc, A.x), dy = __fsub_rn(pyc, A.y);
                    const float4 Bv = s_b[j];
                    const float power = eval_power(dx, dy, A.z, A.w, Bv.x);
                    if (power <= 0.0f) {
                        const float G = __expf(power);
                        const float araw = __fmul_rn(Bv.y, G);
                        const float alpha = fminf(kAlphaMax, araw);
                        if (alpha >= kAlphaMin) {
                            contrib = true;
                            const float oma = 1.0f - alpha;
                            T = T / oma;  // transmittance in front of this Gaussian
                            const float wgt = alpha * T;
                            const float cb = s_c[j];
                            v[6] = wgt * g0;
                            v[7] = wgt * g1;
                            v[8] = wgt * gb2;
                            float dalpha = T * (g0 * (Bv.z - S0) + g1 * (Bv.w - S1) + gb2 * (cb - S2));
                            dalpha -= Tfin / oma * bgdot;
                            S0 = fmaf(alpha, Bv.z, oma * S0);
                            S1 = fmaf(alpha, Bv.w, oma * S1);
                            S2 = fmaf(alpha, cb, oma * S2);
                            if (!(araw > kAlphaMax)) {
                                v[5] = dalpha * G;
                                const float dpow = dalpha * Bv.y * G;
                                v[2] = -0.5f * dx * dx * dpow;
                                v[3] = -dx * dy * dpow;
                                v[4] = -0.5f * dy * dy * dpow;
                                v[0] = dpow * (A.z * dx + A.w * dy);
                                v[1] = dpow * (Bv.x * dy + A.w * dx);
                            }
                        }
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        float x = v[q];
                        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                        v[q] = x;
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int q = 0; q < 9; ++q) atomicAdd(&s_g[q][j], v[q]);
                    }
                }
            }
            __syncthreads();
            if (tid < cnt) {
                float *dst = g2 + (size_t)s_idx[tid] * kG2Floats;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const float x = s_g[q][tid];
                    if (x != 0.f) atomicAdd(dst + q, x);
                }
            }
            __syncthreads();
        }
    }
}

template <int TW, int BATCH>
cudaError_t fwd_inst(const Ctx &c, int grid, float *img, float *T, int *n, const float *tg, int lk,
                     float *dl, cudaStream_t s) {
    k_render_fwd<TW, BATCH><<<grid, kTilePix, 0, s>>>(c, img, T, n, tg, lk, dl);
    return cudaGetLastError();
}

template <int TW, int BATCH>
cudaError_t bwd_inst(const Ctx &c, int grid, const float *dl, const float *T, const int *n,
                     cudaStream_t s) {
    k_render_bwd<TW, BATCH><<<grid, kTilePix, 0, s>>>(c, dl, T, n);
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
