// Fused blend + activation + EWA projection + tile binning count (the "preprocess" stage of
// the batch-parallel rasterizer, RGBAvatar Sec. 3.2 / Supp. A.3, built on 3DGS), and the
// standalone Eq. 1 blend.
//
// The base Gaussians and blendshapes are read from HBM once per step: a CTA stages its chunk's
// rows in shared memory with asynchronous copies and blends every frame of the model from
// there.
//
// Every value that decides a discrete outcome (cull, tile rectangle, depth key) is computed by
// a fixed sequence of correctly rounded binary32 operations written with explicit-rounding
// intrinsics, so the compiler can neither contract nor reorder them: any other IEEE-754
// implementation of the same sequence reproduces the tile lists bit for bit.
#include <algorithm>
#include <cstring>

#include "rgba_internal.cuh"

namespace rgba {
namespace {

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }

// exp for the decision path: Cody & Waite (1980) range reduction with ln 2 split into a short
// head and a tail, the degree-7 Taylor polynomial of e^r in Horner form (|r| <= ln2 / 2),
// and an exact scaling by 2^n. x < -87 -> 0, x > 88 -> +inf.
__device__ float exp_spec(float x) {
    if (x != x) return x;
    if (x < -87.0f) return 0.0f;
    if (x > 88.0f) return __int_as_float(0x7f800000);
    const float log2e = 1.44269504088896341f;
    const float ln2_hi = 0.693145751953125f;
    const float ln2_lo = 1.428606765330187045e-06f;
    float n = rintf(fmul(x, log2e));
    float r = ffma(-n, ln2_hi, x);
    r = ffma(-n, ln2_lo, r);
    float p = 1.0f / 5040.0f;
    p = ffma(p, r, 1.0f / 720.0f);
    p = ffma(p, r, 1.0f / 120.0f);
    p = ffma(p, r, 1.0f / 24.0f);
    p = ffma(p, r, 1.0f / 6.0f);
    p = ffma(p, r, 0.5f);
    p = ffma(p, r, 1.0f);
    p = ffma(p, r, 1.0f);
    int e = (int)n;
    return fmul(p, __int_as_float((e + 127) << 23));
}

struct UploadBlob {
    uint4 data[240];  // 3840 bytes per launch
};

// The step's prologue in one launch: CTA 0 copies up to three host tables (packed in the blob
// at 16-byte offsets) to the workspace and zeroes the counters; every CTA zeroes its share of
// the per-tile counts, which the preprocess then counts into.
__global__ void k_prologue(PrologueArgs a, UploadBlob blob) {
    pdl_enter();  // the previous step's kernels may still read the tables and counts
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    if (blockIdx.x == 0) {
#pragma unroll
        for (int t = 0; t < 3; ++t)
            for (int i = threadIdx.x; i < a.n16[t]; i += blockDim.x) a.dst[t][i] = blob.data[a.src16[t] + i];
        for (int i = threadIdx.x; i < a.zero_a16; i += blockDim.x) a.zero_a[i] = z;
    }
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.zero_b16;
         i += (long long)gridDim.x * blockDim.x)
        a.zero_b[i] = z;
}

__global__ void k_upload_param(uint4 *dst, UploadBlob blob, int n16) {
    pdl_enter();  // the previous step's kernels may still read the tables
    int i = threadIdx.x;
    if (i < n16) dst[i] = blob.data[i];
}

// Blends the 14 channels of Gaussian i for frame b: v = g0; v = fma(psi_k, dG_k, v), k ascending.
__device__ __forceinline__ void blend14(const ModelInfo &m, const float *__restrict__ psi, int i,
                                        float v[kNch]) {
    int a = 0;
#pragma unroll
    for (int ch = 0; ch < kNch; ++ch) {
        float x = __ldg(m.g0 + (size_t)ch * m.n_pad + i);
        if ((m.mask >> ch) & 1u) {
            const float *d = m.dg + (size_t)a * m.n_pad + i;
            const size_t kstep = (size_t)m.A * m.n_pad;
            for (int kk = 0; kk < m.k; ++kk) x = ffma(psi[kk], __ldg(d + kk * kstep), x);
            ++a;
        }
        v[ch] = x;
    }
}

// What the decision spec needs of a frame, staged in shared memory once per round. limx/limy
// are the Jacobian clamp bounds 1.3 tan(fov/2), computed by the same operation sequence the
// per-Gaussian spec would use, so staging them changes no bit.
struct FrameConst {
    float limx, limy;
    int tiles_x, tiles_y, tile_base, rec_base;
    const float *verts;  // the frame's deformed mesh (bound models)
};

// The TBN matrix of Gaussian i's triangle (Supp. "Gaussian Transformation", Alg. 1) and the
// barycentric point of its UV sample, as a fixed sequence of correctly rounded operations:
// e1 = v1 - v0, e2 = v2 - v0; with UV differences (du1, dv1), (du2, dv2) and
// det = du1 dv2 - dv1 du2: T = (dv2 e1 - dv1 e2) / det, B = (du1 e2 - du2 e1) / det (so that
// e1 = du1 T + dv1 B and e2 = du2 T + dv2 B), N = (e1 x e2) / |e1 x e2|; t = (b0 v0 + b1 v1) +
// b2 v2. R[c] = (T_c, B_c, N_c). False when an index is out of range.
__device__ __forceinline__ bool tbn_spec(const ModelInfo &m, const float *__restrict__ verts, int i,
                                         float R[3][3], float t[3]) {
    const int f = __ldg(m.face_of + i);
    if ((unsigned)f >= (unsigned)m.n_faces) return false;
    const int i0 = __ldg(m.faces + 3 * f), i1 = __ldg(m.faces + 3 * f + 1), i2 = __ldg(m.faces + 3 * f + 2);
    if ((unsigned)i0 >= (unsigned)m.n_verts || (unsigned)i1 >= (unsigned)m.n_verts ||
        (unsigned)i2 >= (unsigned)m.n_verts)
        return false;
    float a[3], b[3], c[3], e1[3], e2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a[k] = __ldg(verts + 3 * i0 + k);
        b[k] = __ldg(verts + 3 * i1 + k);
        c[k] = __ldg(verts + 3 * i2 + k);
        e1[k] = fsub(b[k], a[k]);
        e2[k] = fsub(c[k], a[k]);
    }
    const float *uv = m.face_uv + 6 * f;
    const float u0 = __ldg(uv), v0 = __ldg(uv + 1);
    const float du1 = fsub(__ldg(uv + 2), u0), dv1 = fsub(__ldg(uv + 3), v0);
    const float du2 = fsub(__ldg(uv + 4), u0), dv2 = fsub(__ldg(uv + 5), v0);
    const float det = fsub(fmul(du1, dv2), fmul(dv1, du2));
    const float rd = fdiv(1.0f, det);
    float n[3];
    n[0] = fsub(fmul(e1[1], e2[2]), fmul(e1[2], e2[1]));
    n[1] = fsub(fmul(e1[2], e2[0]), fmul(e1[0], e2[2]));
    n[2] = fsub(fmul(e1[0], e2[1]), fmul(e1[1], e2[0]));
    float l2 = fmul(n[0], n[0]);
    l2 = fadd(l2, fmul(n[1], n[1]));
    l2 = fadd(l2, fmul(n[2], n[2]));
    const float len = fsqrt(l2);
    const float b0 = __ldg(m.bary + i), b1 = __ldg(m.bary + m.n_pad + i), b2 = __ldg(m.bary + 2 * m.n_pad + i);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R[k][0] = fmul(fsub(fmul(dv2, e1[k]), fmul(dv1, e2[k])), rd);
        R[k][1] = fmul(fsub(fmul(du1, e2[k]), fmul(du2, e1[k])), rd);
        R[k][2] = fdiv(n[k], len);
        t[k] = fadd(fadd(fmul(b0, a[k]), fmul(b1, b[k])), fmul(b2, c[k]));
    }
    return true;
}

__device__ __forceinline__ float sigmoid_spec(float x) { return fdiv(1.0f, fadd(1.0f, exp_spec(-x))); }

// The FP32 decision spec for one (frame, Gaussian) from its blended channels v and activated
// opacity op: view transform, activations, EWA covariance, conic, radius, tile rectangle, depth.
// Writes the render record, the rectangle and the backward cache, and counts the Gaussian in
// every tile it touches.
__device__ __forceinline__ void decide_and_write(const Ctx &c, const ModelInfo &m, const FrameConst &f,
                                                 const float *V, const float v[kNch], float op, int i,
                                                 long long r) {
    c.cache[r * 3 + 0] = make_float4(v[0], v[1], v[2], v[3]);
    c.cache[r * 3 + 1] = make_float4(v[4], v[5], v[6], v[7]);
    {  // the record's 2-D gradient slots start at zero for the compositing backward's atomics
        float4 *g = reinterpret_cast<float4 *>(c.grad2d + r * kG2Floats);
        g[0] = g[1] = g[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
    ushort4 rc = make_ushort4(0, 0, 0, 0);
    do {
        // tangent space -> deformed space: x_c = fma(N_c, x2, fma(B_c, x1, fma(T_c, x0, t_c)))
        const bool bound = m.n_faces > 0;
        float Rt[3][3], xm[3] = {v[0], v[1], v[2]};
        if (bound) {
            float tt[3];
            if (!tbn_spec(m, f.verts, i, Rt, tt)) {
                atomicOr(&c.cnt->device_error, 2u);
                break;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) xm[k] = ffma(Rt[k][2], v[2], ffma(Rt[k][1], v[1], ffma(Rt[k][0], v[0], tt[k])));
        }
        // view transform
        float p[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
            p[j] = ffma(V[4 * j + 2], xm[2], ffma(V[4 * j + 1], xm[1], ffma(V[4 * j + 0], xm[0], V[4 * j + 3])));
        if (!(p[2] > V[16])) break;
        // scales
        float s[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) s[q] = exp_spec(v[7 + q]);
        // quaternion
        float qw = v[3], qx = v[4], qy = v[5], qz = v[6];
        float n2 = ffma(qz, qz, ffma(qy, qy, ffma(qx, qx, fmul(qw, qw))));
        if (!(n2 > 0.0f)) break;
        float inv = fdiv(1.0f, fsqrt(n2));
        float w = fmul(qw, inv), x = fmul(qx, inv), y = fmul(qy, inv), z = fmul(qz, inv);
        float xx = fmul(x, x), yy = fmul(y, y), zz = fmul(z, z);
        float xy = fmul(x, y), xz = fmul(x, z), yz = fmul(y, z);
        float wx = fmul(w, x), wy = fmul(w, y), wz = fmul(w, z);
        float R[3][3];
        R[0][0] = fsub(1.0f, fmul(2.0f, fadd(yy, zz)));
        R[0][1] = fmul(2.0f, fsub(xy, wz));
        R[0][2] = fmul(2.0f, fadd(xz, wy));
        R[1][0] = fmul(2.0f, fadd(xy, wz));
        R[1][1] = fsub(1.0f, fmul(2.0f, fadd(xx, zz)));
        R[1][2] = fmul(2.0f, fsub(yz, wx));
        R[2][0] = fmul(2.0f, fsub(xz, wy));
        R[2][1] = fmul(2.0f, fadd(yz, wx));
        R[2][2] = fsub(1.0f, fmul(2.0f, fadd(xx, yy)));
        // world covariance
        float d[3] = {fmul(s[0], s[0]), fmul(s[1], s[1]), fmul(s[2], s[2])};
        float Mm[3][3], Sg[3][3];
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
            for (int q = 0; q < 3; ++q) Mm[ii][q] = fmul(R[ii][q], d[q]);
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
                Sg[ii][jj] = ffma(Mm[ii][2], R[jj][2], ffma(Mm[ii][1], R[jj][1], fmul(Mm[ii][0], R[jj][0])));
        // deformed-space covariance Rt Sigma Rt^T (P = Rt Sigma, then P Rt^T)
        if (bound) {
            float P[3][3];
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
#pragma unroll
                for (int jj = 0; jj < 3; ++jj)
                    P[ii][jj] = ffma(Rt[ii][2], Sg[2][jj], ffma(Rt[ii][1], Sg[1][jj], fmul(Rt[ii][0], Sg[0][jj])));
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
#pragma unroll
                for (int jj = 0; jj < 3; ++jj)
                    Sg[ii][jj] = ffma(P[ii][2], Rt[jj][2], ffma(P[ii][1], Rt[jj][1], fmul(P[ii][0], Rt[jj][0])));
        }
        // camera covariance W Sigma W^T
        float Tm[3][3], Cm[3][3];
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
                Tm[ii][jj] = ffma(V[4 * ii + 2], Sg[2][jj], ffma(V[4 * ii + 1], Sg[1][jj], fmul(V[4 * ii + 0], Sg[0][jj])));
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
                Cm[ii][jj] = ffma(Tm[ii][2], V[4 * jj + 2], ffma(Tm[ii][1], V[4 * jj + 1], fmul(Tm[ii][0], V[4 * jj + 0])));
        // EWA Jacobian with the 1.3 x half-fov ratio clamp
        const float fx = V[12], fy = V[13];
        const float limx = f.limx, limy = f.limy;
        float rx = fdiv(p[0], p[2]), ry = fdiv(p[1], p[2]);
        rx = fminf(limx, fmaxf(-limx, rx));
        ry = fminf(limy, fmaxf(-limy, ry));
        float J[2][3];
        J[0][0] = fdiv(fx, p[2]);
        J[0][1] = 0.0f;
        J[0][2] = fdiv(-fmul(fx, rx), p[2]);
        J[1][0] = 0.0f;
        J[1][1] = fdiv(fy, p[2]);
        J[1][2] = fdiv(-fmul(fy, ry), p[2]);
        float Km[2][3], Sp[2][2];
#pragma unroll
        for (int ii = 0; ii < 2; ++ii)
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
                Km[ii][jj] = ffma(J[ii][2], Cm[2][jj], ffma(J[ii][1], Cm[1][jj], fmul(J[ii][0], Cm[0][jj])));
#pragma unroll
        for (int ii = 0; ii < 2; ++ii)
#pragma unroll
            for (int jj = 0; jj < 2; ++jj)
                Sp[ii][jj] = ffma(Km[ii][2], J[jj][2], ffma(Km[ii][1], J[jj][1], fmul(Km[ii][0], J[jj][0])));
        float cA = fadd(Sp[0][0], 0.3f), cB = Sp[0][1], cC = fadd(Sp[1][1], 0.3f);
        float det = fsub(fmul(cA, cC), fmul(cB, cB));
        if (!(det > 0.0f)) break;
        float ca = fdiv(cC, det), cb = fdiv(-cB, det), cc = fdiv(cA, det);
        float mid = fmul(0.5f, fadd(cA, cC));
        float lam = fadd(mid, fsqrt(fmaxf(0.1f, fsub(fmul(mid, mid), det))));
        float rad = ceilf(fmul(3.0f, fsqrt(lam)));
        float u = fadd(fmul(fx, fdiv(p[0], p[2])), V[14]);
        float vv = fadd(fmul(fy, fdiv(p[1], p[2])), V[15]);
        // the tile sides are powers of two (16 x 16 or 8 x 32), so each division by a side is
        // the product with its exact reciprocal: the same correctly rounded quotient
        const float ftw = (float)c.tw, fth = (float)c.th, rtw = 1.0f / ftw, rth = 1.0f / fth;
        float x0 = floorf(fmul(fsub(u, rad), rtw));
        float x1 = floorf(fmul(fadd(fadd(u, rad), fsub(ftw, 1.0f)), rtw));
        float y0 = floorf(fmul(fsub(vv, rad), rth));
        float y1 = floorf(fmul(fadd(fadd(vv, rad), fsub(fth, 1.0f)), rth));
        x0 = fminf((float)f.tiles_x, fmaxf(0.0f, x0));
        x1 = fminf((float)f.tiles_x, fmaxf(0.0f, x1));
        y0 = fminf((float)f.tiles_y, fmaxf(0.0f, y0));
        y1 = fminf((float)f.tiles_y, fmaxf(0.0f, y1));
        if (x0 != x0 || y0 != y0 || x1 != x1 || y1 != y1) break;
        int ix0 = (int)x0, ix1 = (int)x1, iy0 = (int)y0, iy1 = (int)y1;
        if ((ix1 - ix0) * (iy1 - iy0) <= 0) break;
        r0 = make_float4(u, vv, ca, cb);
        r1 = make_float4(cc, op, v[11], v[12]);
        r2 = make_float4(v[13], p[2], 0.f, 0.f);
        rc = make_ushort4((unsigned short)ix0, (unsigned short)iy0, (unsigned short)ix1, (unsigned short)iy1);
        // count the Gaussian in every tile of its rectangle; for rectangles of up to kRankSlots
        // tiles keep the slot each count returns, so the scatter needs no atomics
        const int rw = ix1 - ix0, area = rw * (iy1 - iy0);
        if (area <= kRankSlots) {
            const long long t0 = (long long)f.tile_base + iy0 * f.tiles_x + ix0;
            unsigned rk[kRankSlots];
            int ox = 0, off = 0;  // slot q is tile (ix0 + ox, iy0 + q / rw), off its offset from t0
#pragma unroll
            for (int q = 0; q < kRankSlots; ++q) {
                rk[q] = 0u;
                if (q < area) {
                    rk[q] = atomicAdd(c.tile_count + tc_word(c.tc_mask, t0 + off), 1u);
                    ++off;
                    if (++ox == rw) {
                        ox = 0;
                        off += f.tiles_x - rw;
                    }
                }
            }
            uint4 *rp = reinterpret_cast<uint4 *>(c.ranks + r * kRankSlots);
            rp[0] = make_uint4(rk[0], rk[1], rk[2], rk[3]);
            rp[1] = make_uint4(rk[4], rk[5], rk[6], rk[7]);
        } else {  // spread over kSubCounters counters per tile, chosen by the Gaussian index
            unsigned *tb = c.tile_count + tc_sub_base(c.tc_mask) + (size_t)f.tile_base * kSubCounters +
                           (r & (kSubCounters - 1));
            for (int ty = iy0; ty < iy1; ++ty)
                for (int tx = ix0; tx < ix1; ++tx) atomicAdd(tb + (size_t)(ty * f.tiles_x + tx) * kSubCounters, 1u);
        }
    } while (0);
    c.records[r * 3 + 0] = r0;
    c.records[r * 3 + 1] = r1;
    c.records[r * 3 + 2] = r2;
    c.rects[r] = rc;
    c.depth[r] = r2.y;  // compact copy for the scatter (0 when culled; never read then)
    // the cache's last slot also carries the activated opacity and whether the Gaussian was
    // kept (1) or culled (0), so the backward reads one array per (frame, Gaussian)
    c.cache[r * 3 + 2] = make_float4(v[8], v[9], op, rc.z > rc.x && rc.w > rc.y ? 1.f : 0.f);
}

constexpr int kPreThreads = 128;  // standalone blend
// the row stride of the staged weights: max_k rounded up to a multiple of 4
__host__ __device__ constexpr int psi_stride(int max_k) { return (max_k + 3) & ~3; }
constexpr int kPreG = 32;         // Gaussians per CTA
constexpr int kPreSlots = 8;      // frame slots per Gaussian
constexpr int kPreFB = 2;         // frames per thread per round (register block)
constexpr int kPreRound = kPreSlots * kPreFB;
constexpr int kPreBlock = kPreG * kPreSlots;

__host__ __device__ constexpr int popcount_c(unsigned x) { return x ? (int)(x & 1u) + popcount_c(x >> 1) : 0; }

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Asynchronous 16-byte copy global -> shared (both addresses 16-byte aligned), completed by
// cp.async.wait_all.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_u32(dst)), "l"(src) : "memory");
}

// One CTA = kPreG (32) Gaussians of one model and every frame that renders it. The model's G0
// rows and blendshape rows for the chunk arrive once in shared memory by 16-byte asynchronous
// copies from all threads (39 KB at K = 32 with 9 blended channels, so several CTAs share an
// SM; 128-byte bulk copies issued by one warp were 20 % slower); its kPreSlots (8)
// thread slots per Gaussian then each blend kPreFB (2) frames at a time from shared memory
// (each blendshape value read once per 2 frames) and run the decision spec per frame.
// MASK != 0: every model of the batch blends exactly the channels in MASK, so the channel
// selection of the blend loop is resolved at compile time (a runtime mask costs a test, a
// branch and an index update per channel and blendshape); MASK = 0 reads each model's mask.
template <unsigned MASK>
__global__ void __launch_bounds__(kPreBlock, 3)
k_preprocess(Ctx c, int max_k) {
    extern __shared__ float4 smem4[];
    __shared__ FrameConst s_fc[kPreRound];
    pdl_enter();
    const ModelInfo &m = c.models[blockIdx.y];
    const int i0 = blockIdx.x * kPreG;
    if (i0 >= m.n || m.nb == 0) return;
    const unsigned mask = MASK ? MASK : m.mask;
    const int K = m.k, A = MASK ? popcount_c(MASK) : m.A, rows = kNch + K * A;
    float *s_rows = reinterpret_cast<float *>(smem4);      // [rows][kPreG]: G0 then blendshapes
    const int kp = psi_stride(max_k);                      // 16-byte rows of weights
    float *s_psi = s_rows + (size_t)rows * kPreG;          // [16][kp]
    float *s_fp = s_psi + kPreRound * kp;                  // [16][20]
    const int tid = threadIdx.x;
    const int cols = min(kPreG, m.n_pad - i0);
    {  // 16-byte asynchronous copies of the chunk's rows by every thread; the first round's
       // frame tables below are gathered while they are in flight, then one wait
        const int per_row = cols >> 2;  // n_pad and i0 are multiples of 4
        auto copy = [&](int rr, int q) {
            const float *src = (rr < kNch ? m.g0 + (size_t)rr * m.n_pad : m.dg + (size_t)(rr - kNch) * m.n_pad) + i0 + 4 * q;
            cp_async16(s_rows + (size_t)rr * kPreG + 4 * q, src);
        };
        if (per_row == kPreG / 4) {  // a full chunk: thread t copies quad t % 8 of every 32nd row
            for (int rr = tid / (kPreG / 4); rr < rows; rr += kPreBlock / (kPreG / 4)) copy(rr, tid % (kPreG / 4));
        } else {
            for (int e = tid; e < rows * per_row; e += kPreBlock) copy(e / per_row, e % per_row);
        }
    }
    const int g = tid % kPreG, slot = tid / kPreG;
    const int i = i0 + g;
    const bool valid = i < m.n;
    // opacity is the same for every frame unless it is blended
    const bool op_blended = (mask >> 10) & 1u;
    float op0 = 0.0f;
    for (int round = 0; round < m.nb; round += kPreRound) {
        const int nr = min(kPreRound, m.nb - round);
        for (int e = tid; e < nr * K; e += kPreBlock) {
            const int fl = e / K, kk = e - fl * K;
            const int b = c.mframes[m.frame_off + round + fl];
            s_psi[fl * kp + kk] = c.psi[(size_t)b * c.k_stride + kk];
        }
        for (int e = tid; e < nr * RGBA_FP_STRIDE; e += kPreBlock) {
            const int fl = e / RGBA_FP_STRIDE, q = e - fl * RGBA_FP_STRIDE;
            const int b = c.mframes[m.frame_off + round + fl];
            s_fp[e] = c.fparams[(size_t)b * RGBA_FP_STRIDE + q];
        }
        if (tid < nr) {
            const int b = c.mframes[m.frame_off + round + tid];
            const FrameInfo &f = c.frames[b];
            const float *fp = c.fparams + (size_t)b * RGBA_FP_STRIDE;
            FrameConst fc;
            fc.limx = fmul(1.3f, fdiv(fmul(0.5f, (float)f.W), fp[12]));
            fc.limy = fmul(1.3f, fdiv(fmul(0.5f, (float)f.H), fp[13]));
            fc.tiles_x = f.tiles_x;
            fc.tiles_y = f.tiles_y;
            fc.tile_base = f.tile_base;
            fc.rec_base = f.rec_base;
            fc.verts = f.verts;
            s_fc[tid] = fc;
        }
        if (round == 0) asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        if (round == 0) op0 = sigmoid_spec(s_rows[10 * kPreG + g]);
        const int f0 = slot * kPreFB;
        if (valid && f0 < nr) {
            // Eq. 1 for kPreFB frames: v = g0, then v = fma(psi_k, dG_k, v) for k ascending in
            // every blended channel (the order of the loops over k and channels is free)
            float v[kPreFB][kNch];
#pragma unroll
            for (int ch = 0; ch < kNch; ++ch) {
                const float x = s_rows[ch * kPreG + g];
#pragma unroll
                for (int q = 0; q < kPreFB; ++q) v[q][ch] = x;
            }
            auto term = [&](int kk, const float ps[kPreFB]) {
                const float *d = s_rows + (size_t)(kNch + kk * A) * kPreG + g;
                int a = 0;
#pragma unroll
                for (int ch = 0; ch < kNch; ++ch) {
                    if ((mask >> ch) & 1u) {
                        const float dv = d[a * kPreG];
#pragma unroll
                        for (int q = 0; q < kPreFB; ++q) v[q][ch] = __fmaf_rn(ps[q], dv, v[q][ch]);
                        ++a;
                    }
                }
            };
            int kk = 0;
            for (; kk + 4 <= K; kk += 4) {  // the weights four at a time (one 16-byte load per frame)
                float4 w4[kPreFB];
#pragma unroll
                for (int q = 0; q < kPreFB; ++q) w4[q] = *reinterpret_cast<const float4 *>(s_psi + (f0 + q) * kp + kk);
                float ps[kPreFB];
#pragma unroll
                for (int q = 0; q < kPreFB; ++q) ps[q] = w4[q].x;
                term(kk, ps);
#pragma unroll
                for (int q = 0; q < kPreFB; ++q) ps[q] = w4[q].y;
                term(kk + 1, ps);
#pragma unroll
                for (int q = 0; q < kPreFB; ++q) ps[q] = w4[q].z;
                term(kk + 2, ps);
#pragma unroll
                for (int q = 0; q < kPreFB; ++q) ps[q] = w4[q].w;
                term(kk + 3, ps);
            }
            for (; kk < K; ++kk) {
                float ps[kPreFB];
#pragma unroll
                for (int q = 0; q < kPreFB; ++q) ps[q] = s_psi[(f0 + q) * kp + kk];
                term(kk, ps);
            }
            // one frame at a time through v[0] (a rolled loop keeps the code small)
#pragma unroll 1
            for (int q = 0; q < kPreFB; ++q) {
                if (f0 + q < nr) {
                    const FrameConst &fc = s_fc[f0 + q];
                    decide_and_write(c, m, fc, s_fp + (f0 + q) * RGBA_FP_STRIDE, v[0],
                                     op_blended ? sigmoid_spec(v[0][10]) : op0, i, fc.rec_base + i);
                }
#pragma unroll
                for (int q2 = 0; q2 + 1 < kPreFB; ++q2)
#pragma unroll
                    for (int ch = 0; ch < kNch; ++ch) v[q2][ch] = v[q2 + 1][ch];
            }
        }
        __syncthreads();
    }
}

// Standalone Eq. 1 for up to kBlendFrames frames per launch; the frame table travels as a
// kernel parameter so this entry point needs no workspace.
constexpr int kBlendFrames = 64;
struct BlendFrame {
    const float *g0;
    const float *dg;
    const float *psi;
    float *out;
    int n, n_pad, k, A;
    unsigned mask;
    int pad_;
};
struct BlendChunk {
    BlendFrame f[kBlendFrames];
};

__global__ void __launch_bounds__(kPreThreads)
k_blend(BlendChunk ch) {
    __shared__ float s_psi[RGBA_MAX_K];
    const BlendFrame &f = ch.f[blockIdx.y];
    for (int t = threadIdx.x; t < f.k; t += blockDim.x) s_psi[t] = f.psi[t];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f.n) return;
    ModelInfo m;
    m.g0 = f.g0;
    m.dg = f.dg;
    m.n = f.n;
    m.n_pad = f.n_pad;
    m.k = f.k;
    m.A = f.A;
    m.mask = f.mask;
    float v[kNch];
    blend14(m, s_psi, i, v);
#pragma unroll
    for (int q = 0; q < kNch; ++q) f.out[(size_t)q * f.n_pad + i] = v[q];
}

}  // namespace

cudaError_t launch_prologue(const PrologueArgs &a0, const void *const src[3], cudaStream_t s) {
    static_assert(sizeof(UploadBlob) == 16 * kPrologueBlob16, "one blob per prologue");
    PrologueArgs a = a0;
    UploadBlob blob;
    memset(&blob, 0, sizeof(blob));
    int at = 0;
    for (int t = 0; t < 3; ++t) {
        if (at + a.n16[t] > kPrologueBlob16) return cudaErrorInvalidValue;
        if (a.nbytes[t]) memcpy(&blob.data[at], src[t], (size_t)a.nbytes[t]);  // the blob is zeroed
        a.src16[t] = at;
        at += a.n16[t];
    }
    const long long per = 256LL * 8;  // uint4 stores per CTA
    const unsigned grid = (unsigned)std::max(1LL, std::min((a.zero_b16 + per - 1) / per, 1024LL));
    return launch_pdl(k_prologue, dim3(grid), dim3(256), 0, s, a, blob);
}

cudaError_t launch_upload(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    // src is host memory: it travels as kernel parameters (captured by value in graphs).
    const unsigned char *p = static_cast<const unsigned char *>(src);
    unsigned char *d = static_cast<unsigned char *>(dst);
    size_t off = 0;
    while (off < bytes) {
        UploadBlob blob;
        size_t n = bytes - off;
        if (n > sizeof(blob.data)) n = sizeof(blob.data);
        size_t n16 = (n + 15) / 16;
        memset(&blob, 0, sizeof(blob));
        memcpy(&blob, p + off, n);
        cudaError_t e = launch_pdl(k_upload_param, dim3(1), dim3(256), 0, s, reinterpret_cast<uint4 *>(d + off),
                                   blob, (int)n16);
        if (e != cudaSuccess) return e;
        off += n16 * 16;
    }
    return cudaSuccess;
}

int preprocess_smem(int max_k, int max_rows) {
    return (max_rows * kPreG + kPreRound * psi_stride(max_k) + kPreRound * RGBA_FP_STRIDE) * (int)sizeof(float);
}

namespace {
template <unsigned MASK>
cudaError_t preprocess_inst(const Ctx &c, int max_n, int max_k, int max_rows, cudaStream_t s) {
    static int attr_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_device != dev) {  // once, at the largest size (K = 64, 13 blended channels)
        e = cudaFuncSetAttribute(k_preprocess<MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 preprocess_smem(RGBA_MAX_K, kNch + RGBA_MAX_K * 13));
        if (e != cudaSuccess) return e;
        attr_device = dev;
    }
    dim3 grid((max_n + kPreG - 1) / kPreG, c.M);
    return launch_pdl(k_preprocess<MASK>, grid, dim3(kPreBlock), preprocess_smem(max_k, max_rows), s, c, max_k);
}
}  // namespace

cudaError_t launch_preprocess(const Ctx &c, int max_n, int max_k, int max_rows, unsigned common_mask,
                              cudaStream_t s) {
    if (c.B == 0 || max_n == 0) return cudaSuccess;
    if (common_mask == RGBA_MASK_MEAN_SCALE_COLOR)
        return preprocess_inst<RGBA_MASK_MEAN_SCALE_COLOR>(c, max_n, max_k, max_rows, s);
    if (common_mask == RGBA_MASK_MEAN_ROT_COLOR)
        return preprocess_inst<RGBA_MASK_MEAN_ROT_COLOR>(c, max_n, max_k, max_rows, s);
    return preprocess_inst<0u>(c, max_n, max_k, max_rows, s);
}

cudaError_t launch_blend(const Ctx &c, int max_n, float *out, cudaStream_t s) {
    // c.models / c.frames are HOST tables here (rgba_blend has no workspace)
    for (int f0 = 0; f0 < c.B; f0 += kBlendFrames) {
        const int nf = min(kBlendFrames, c.B - f0);
        BlendChunk ch;
        memset(&ch, 0, sizeof(ch));
        int mx = 0;
        for (int j = 0; j < nf; ++j) {
            const FrameInfo &fi = c.frames[f0 + j];
            const ModelInfo &m = c.models[fi.model];
            BlendFrame &bf = ch.f[j];
            bf.g0 = m.g0;
            bf.dg = m.dg;
            bf.psi = c.psi + (size_t)(f0 + j) * c.k_stride;
            bf.out = out + (size_t)fi.rec_base * kNch;
            bf.n = m.n;
            bf.n_pad = m.n_pad;
            bf.k = m.k;
            bf.A = m.A;
            bf.mask = m.mask;
            mx = max(mx, m.n);
        }
        if (mx == 0) continue;
        dim3 grid((mx + kPreThreads - 1) / kPreThreads, nf);
        k_blend<<<grid, kPreThreads, 0, s>>>(ch);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    (void)max_n;
    return cudaSuccess;
}

}  // namespace rgba
