// Backward through the projection (EWA splatting, activations) and the linear blend (Eq. 1).
//
//   k_gauss_bwd  one CTA per 32 Gaussians of one model, lane = Gaussian, frames 16 at a time:
//                first, per (frame, Gaussian), the 2-D gradients dL/d(u, v, conic, opacity,
//                colour) from the compositing backward's sums -> dL/dG_b over the 14 channels
//                (chain rule through conic inversion, J W Sigma W^T J^T, R diag(s^2) R^T,
//                quaternion normalisation, exp and sigmoid) into shared memory; then the
//                adjoint of Eq. 1:
//                dG0[ch][i]    += sum_b dG_b[ch][i]
//                ddG[k][a][i]  += sum_b psi_b[k] dG_b[ch_a][i]
//                dpsi_b[k]     partial = sum_{a, i in chunk} dG_k[a][i] dG_b[ch_a][i]
//                the last two as TF32 tensor-core products at FP32 accuracy (three products
//                of split operands).
// Every sum runs in a fixed order (dG0 in registers, the products tile by tile, the warps'
// dpsi sums in warp order), so the results are deterministic; dpsi partials go to a
// [frame][k][chunk] buffer that a second kernel sums.
#include <type_traits>

#include "rgba_internal.cuh"

namespace rgba {
namespace {

constexpr int kBwdThreads = 256;

// The backward needs no bit-exact replay of the forward decisions (those come from the
// records), only fp32 values to the gradient tolerance, so it uses the hardware's fast
// reciprocal, reciprocal square root and exponential.
struct Fwd {
    float p[3], qn[4], il, s[3], R[3][3], M[3][3], J[2][3], rx, ry, ipz;
    bool clx, cly;
    float A, B, C, det;
};

// BOUND: Rt [12] = TBN matrix row-major (columns T, B, N), then t (the identity and zero for an
// unbound model of a batch that also has bound ones); the Gaussian is mapped from tangent space
// by x = R x_T + t, covariance R Sigma R^T. !BOUND: no mapping (Rt is not read).
template <bool BOUND>
__device__ __forceinline__ void recompute(const float v[10], const float *V, int W, int H, const float *Rt, Fwd &f) {
    float xm[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        xm[c] = BOUND ? Rt[3 * c] * v[0] + Rt[3 * c + 1] * v[1] + Rt[3 * c + 2] * v[2] + Rt[9 + c] : v[c];
#pragma unroll
    for (int j = 0; j < 3; ++j) f.p[j] = V[4 * j] * xm[0] + V[4 * j + 1] * xm[1] + V[4 * j + 2] * xm[2] + V[4 * j + 3];
#pragma unroll
    for (int m = 0; m < 3; ++m) f.s[m] = __expf(v[7 + m]);
    f.il = rsqrtf(v[3] * v[3] + v[4] * v[4] + v[5] * v[5] + v[6] * v[6]);
#pragma unroll
    for (int m = 0; m < 4; ++m) f.qn[m] = v[3 + m] * f.il;
    const float w = f.qn[0], x = f.qn[1], y = f.qn[2], z = f.qn[3];
    f.R[0][0] = 1.f - 2.f * (y * y + z * z);
    f.R[0][1] = 2.f * (x * y - w * z);
    f.R[0][2] = 2.f * (x * z + w * y);
    f.R[1][0] = 2.f * (x * y + w * z);
    f.R[1][1] = 1.f - 2.f * (x * x + z * z);
    f.R[1][2] = 2.f * (y * z - w * x);
    f.R[2][0] = 2.f * (x * z - w * y);
    f.R[2][1] = 2.f * (y * z + w * x);
    f.R[2][2] = 1.f - 2.f * (x * x + y * y);
    float Sg[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float a = 0.f;
#pragma unroll
            for (int m = 0; m < 3; ++m) a += f.R[i][m] * f.s[m] * f.s[m] * f.R[j][m];
            Sg[i][j] = a;
        }
    if (BOUND) {
        float P[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) P[i][j] = Rt[3 * i] * Sg[0][j] + Rt[3 * i + 1] * Sg[1][j] + Rt[3 * i + 2] * Sg[2][j];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Sg[i][j] = P[i][0] * Rt[3 * j] + P[i][1] * Rt[3 * j + 1] + P[i][2] * Rt[3 * j + 2];
    }
    float Tm[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Tm[i][j] = V[4 * i] * Sg[0][j] + V[4 * i + 1] * Sg[1][j] + V[4 * i + 2] * Sg[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) f.M[i][j] = Tm[i][0] * V[4 * j] + Tm[i][1] * V[4 * j + 1] + Tm[i][2] * V[4 * j + 2];
    const float fx = V[12], fy = V[13], pz = f.p[2];
    const float limx = 1.3f * __fdividef(0.5f * W, fx), limy = 1.3f * __fdividef(0.5f * H, fy);
    f.ipz = __frcp_rn(pz);
    const float rx = f.p[0] * f.ipz, ry = f.p[1] * f.ipz;
    f.clx = rx > limx || rx < -limx;
    f.cly = ry > limy || ry < -limy;
    f.rx = fminf(limx, fmaxf(-limx, rx));
    f.ry = fminf(limy, fmaxf(-limy, ry));
    f.J[0][0] = fx * f.ipz;
    f.J[0][1] = 0.f;
    f.J[0][2] = -fx * f.rx * f.ipz;
    f.J[1][0] = 0.f;
    f.J[1][1] = fy * f.ipz;
    f.J[1][2] = -fy * f.ry * f.ipz;
    float S2[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float a = 0.f;
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) a += f.J[i][p] * f.M[p][q] * f.J[j][q];
            S2[i][j] = a;
        }
    f.A = S2[0][0] + 0.3f;
    f.B = S2[0][1];
    f.C = S2[1][1] + 0.3f;
    f.det = f.A * f.C - f.B * f.B;
}

// dG[14]: gradient w.r.t. the blended channels of one (frame, Gaussian). g2: the compositing
// backward's sums over the pixels that blend the Gaussian, S = (S1, S2, S3, S4, S5, S0) of
// g (dx, dy, dx^2, dx dy, dy^2, 1) with g = dL/dpower and (dx, dy) = pixel centre - mean, then
// dL/d(r, g, b). As power = -(a dx^2 + c dy^2) / 2 - b dx dy and alpha = o e^power:
// dL/du = a S1 + b S2, dL/dv = b S1 + c S2, dL/d(a, b, c) = (-S3 / 2, -S4, -S5 / 2) and
// dL/do = S0 / o, with the conic (a, b, c) = Sigma'^-1 recomputed here.
template <bool BOUND>
__device__ __forceinline__ void chain(const float v[10], float op, const float *V, int W, int H,
                                      const float *Rt, const float g2[9], float dG[kNch]) {
    Fwd f;
    recompute<BOUND>(v, V, W, H, Rt, f);
    const float A = f.A, B = f.B, C = f.C, D = f.det, iD = __frcp_rn(D), iD2 = iD * iD;
    const float ca = C * iD, cb = -B * iD, cc = A * iD;
    const float du = ca * g2[0] + cb * g2[1], dv = cb * g2[0] + cc * g2[1];
    const float dca = -0.5f * g2[2], dcb = -g2[3], dcc = -0.5f * g2[4];
    dG[10] = g2[5] * (1.f - op);  // dL/do times the sigmoid's o (1 - o)
    dG[11] = g2[6];
    dG[12] = g2[7];
    dG[13] = g2[8];
    const float dA = dca * (-C * C * iD2) + dcb * (B * C * iD2) + dcc * (iD - A * C * iD2);
    const float dC = dca * (iD - A * C * iD2) + dcb * (A * B * iD2) + dcc * (-A * A * iD2);
    const float dB = dca * (2.f * B * C * iD2) + dcb * (-iD - 2.f * B * B * iD2) + dcc * (2.f * A * B * iD2);
    const float G2[2][2] = {{dA, 0.5f * dB}, {0.5f * dB, dC}};
    // dJ = 2 G2 J M ; dM = J^T G2 J
    float GJ[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) GJ[r][c] = G2[r][0] * f.J[0][c] + G2[r][1] * f.J[1][c];
    float dJ[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) dJ[r][c] = 2.f * (GJ[r][0] * f.M[0][c] + GJ[r][1] * f.M[1][c] + GJ[r][2] * f.M[2][c]);
    float dM[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) dM[r][c] = f.J[0][r] * GJ[0][c] + f.J[1][r] * GJ[1][c];
    // dSigma = V^T dM V
    float tmp[3][3], dS[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) tmp[r][c] = V[r] * dM[0][c] + V[4 + r] * dM[1][c] + V[8 + r] * dM[2][c];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) dS[r][c] = tmp[r][0] * V[c] + tmp[r][1] * V[4 + c] + tmp[r][2] * V[8 + c];
    if (BOUND) {  // Sigma = R Sigma_T R^T: dSigma_T = R^T dSigma R
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) tmp[r][c] = Rt[r] * dS[0][c] + Rt[3 + r] * dS[1][c] + Rt[6 + r] * dS[2][c];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) dS[r][c] = tmp[r][0] * Rt[c] + tmp[r][1] * Rt[3 + c] + tmp[r][2] * Rt[6 + c];
    }
    // Sigma = R diag(s^2) R^T
    float dSR[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int m = 0; m < 3; ++m) dSR[r][m] = dS[r][0] * f.R[0][m] + dS[r][1] * f.R[1][m] + dS[r][2] * f.R[2][m];
    float dR[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int m = 0; m < 3; ++m) dR[r][m] = 2.f * dSR[r][m] * f.s[m] * f.s[m];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const float q = f.R[0][m] * dSR[0][m] + f.R[1][m] * dSR[1][m] + f.R[2][m] * dSR[2][m];
        dG[7 + m] = 2.f * f.s[m] * q * f.s[m];  // ds * s (s = exp(log-scale))
    }
    const float w = f.qn[0], x = f.qn[1], y = f.qn[2], z = f.qn[3];
    const float dw = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    const float dx = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] +
                            z * dR[2][0] + w * dR[2][1] - 2.f * x * dR[2][2]);
    const float dy = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] -
                            w * dR[2][0] + z * dR[2][1] - 2.f * y * dR[2][2]);
    const float dz = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2.f * z * dR[1][1] +
                            y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    const float dot = w * dw + x * dx + y * dy + z * dz;
    const float il = f.il;
    dG[3] = (dw - w * dot) * il;
    dG[4] = (dx - x * dot) * il;
    dG[5] = (dy - y * dot) * il;
    dG[6] = (dz - z * dot) * il;
    // mean
    const float fx = V[12], fy = V[13], ipz = f.ipz, ipz2 = ipz * ipz;
    float dp0 = du * fx * ipz, dp1 = dv * fy * ipz;
    float dp2 = -du * fx * f.p[0] * ipz2 - dv * fy * f.p[1] * ipz2;
    dp2 += -(dJ[0][0] * fx + dJ[1][1] * fy) * ipz2;
    if (!f.clx) {
        dp0 += -dJ[0][2] * fx * ipz2;
        dp2 += dJ[0][2] * 2.f * fx * f.p[0] * ipz2 * ipz;
    } else {
        dp2 += dJ[0][2] * fx * f.rx * ipz2;
    }
    if (!f.cly) {
        dp1 += -dJ[1][2] * fy * ipz2;
        dp2 += dJ[1][2] * 2.f * fy * f.p[1] * ipz2 * ipz;
    } else {
        dp2 += dJ[1][2] * fy * f.ry * ipz2;
    }
    float dxw[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dxw[c] = V[c] * dp0 + V[4 + c] * dp1 + V[8 + c] * dp2;
#pragma unroll
    for (int c = 0; c < 3; ++c)  // x = R x_T + t: dx_T = R^T dx
        dG[c] = BOUND ? Rt[c] * dxw[0] + Rt[3 + c] * dxw[1] + Rt[6 + c] * dxw[2] : dxw[c];
}

// TBN matrix and barycentric point of Gaussian i in one frame (the same definitions as the
// preprocess, fp32 without its fixed rounding order): out[12] as recompute() reads it.
__device__ __forceinline__ bool tbn_fast(const ModelInfo &m, const float *__restrict__ verts, int i, float out[12]) {
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
        e1[k] = b[k] - a[k];
        e2[k] = c[k] - a[k];
    }
    const float *uv = m.face_uv + 6 * f;
    const float du1 = __ldg(uv + 2) - __ldg(uv), dv1 = __ldg(uv + 3) - __ldg(uv + 1);
    const float du2 = __ldg(uv + 4) - __ldg(uv), dv2 = __ldg(uv + 5) - __ldg(uv + 1);
    const float rd = __frcp_rn(du1 * dv2 - dv1 * du2);
    const float n0 = e1[1] * e2[2] - e1[2] * e2[1], n1 = e1[2] * e2[0] - e1[0] * e2[2],
                n2 = e1[0] * e2[1] - e1[1] * e2[0];
    const float il = rsqrtf(n0 * n0 + n1 * n1 + n2 * n2);
    const float nn[3] = {n0 * il, n1 * il, n2 * il};
    const float b0 = __ldg(m.bary + i), b1 = __ldg(m.bary + m.n_pad + i), b2 = __ldg(m.bary + 2 * m.n_pad + i);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        out[3 * k] = (dv2 * e1[k] - dv1 * e2[k]) * rd;
        out[3 * k + 1] = (du1 * e2[k] - du2 * e1[k]) * rd;
        out[3 * k + 2] = nn[k];
        out[9 + k] = b0 * a[k] + b1 * b[k] + b2 * c[k];
    }
    return true;
}

// The backward of one model chunk. One CTA = 32 Gaussians (lane = Gaussian) of one model; the
// frames that render it go 16 at a time. The chunk's blendshape rows are copied to shared
// memory asynchronously at the start. Meanwhile the chain rule per (frame, Gaussian) turns the
// 2-D gradients into dL/dG_b over the 14 channels, straight into shared memory (each item
// reads only its cache and 2-D gradients: the cache carries the opacity and whether the
// Gaussian was kept); then the adjoint of Eq. 1 reduces them over the frames: dG0 by plain
// sums, ddG and the dpsi partials as tensor-core products (below).
// Asynchronous 16-byte copy global -> shared (both addresses 16-byte aligned), completed by
// cp.async.wait_all.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))), "l"(src) : "memory");
}

constexpr int kFG2 = 16;
constexpr int kWarps = kBwdThreads / 32;
// Shared-memory strides in floats: a frame's 14 x 32 blended-channel gradients, and a staged
// blendshape row of 32 Gaussians, each padded by 4 so that the tensor-core fragment loads,
// which step over frames or blendshapes, fall in different banks (stride = 4 mod 32).
constexpr int kDGF = kNch * kBwdChunk + 4;
constexpr int kDgRow = kBwdChunk + 4;

// The adjoint of Eq. 1 is two small dense products per chunk and group of frames (ddG: the
// K x 16 weights times the 16 x (A 32) blended-channel gradients; dpsi: the 16 x (A 32)
// gradients times the (A 32) x K blendshape rows), done on the tensor cores as
// m16n8k8 TF32 matrix multiply-accumulates with FP32 accumulators. Each FP32 operand x is split
// into x_hi = tf32(x) and x_lo = tf32(x - x_hi), and a b is accumulated as
// a_lo b_hi + a_hi b_lo + a_hi b_hi (the a_lo b_lo term is below FP32 rounding), which keeps
// the products at FP32 accuracy (the split-operand scheme of Ootomo and Yokota, "Recovering
// single precision accuracy from Tensor Cores", 2022). Fragment layout (m16n8k8, A row-major,
// B column-major), with g = lane / 4 and t = lane % 4: A elements (g, t), (g + 8, t), (g, t + 4), (g + 8, t + 4);
// B elements (t, g), (t + 4, g); C elements (g, 2t), (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1).
__device__ __forceinline__ void split_tf32(float x, unsigned &hi, unsigned &lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    const float r = x - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

__device__ __forceinline__ void mma_tf32(float d[4], const unsigned a[4], const unsigned b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// d += a b at FP32 accuracy from split operands (small terms first)
__device__ __forceinline__ void mma_3xtf32(float d[4], const unsigned ah[4], const unsigned al[4],
                                           const unsigned bh[2], const unsigned bl[2]) {
    mma_tf32(d, al, bh);
    mma_tf32(d, ah, bl);
    mma_tf32(d, ah, bh);
}

// 2 CTAs per SM: without the TBN mapping (unbound batches) the chain rule fits without spills
// at up to 128 registers, and that beat 3 CTAs at 80 registers with spills (0.120 vs 0.127 ms
// on the batched training workload).
// ADAM: the fused Adam update of rgba_step_adam_async; every model is rendered by at most kFG2
// frames, so the reductions below are complete after one group. Their results are parked in
// shared memory (G0's in s_g0, the blendshapes' in the slots of the staged rows, whose values
// are read again from memory) and the CTA then streams the update over the chunk's rows; the
// gradient arrays are not written.
// The plain instance's stand-in for FusedAdam: the same members, one model, never read.
struct NoAdam {
    FusedAdamModel m[1];
    float b1, b2, eps, ibc1, ibc2;
    const int *step_dev;
};
template <bool ADAM>
using AdamArg = typename std::conditional<ADAM, FusedAdam, NoAdam>::type;

// BOUND: some model of the batch has a tangent-space binding (the chain rule then maps through
// each bound Gaussian's TBN frame); otherwise that mapping is compiled out.
template <bool ADAM, bool BOUND>
__global__ void __launch_bounds__(kBwdThreads, 2)
k_gauss_bwd(Ctx c, int max_k, AdamArg<ADAM> fa) {
    extern __shared__ float smem[];
    float *s_dG = smem;                                   // [16][kDGF]: [14][32] per frame
    float *s_psi = s_dG + kFG2 * kDGF;                    // [16][max_k]
    float *s_dgc = s_psi + kFG2 * max_k;                  // [k][A][kDgRow]: the chunk's blendshapes
    __shared__ __align__(16) float s_g0[ADAM ? kNch * kBwdChunk : 1];  // ADAM: the G0 gradients
    __shared__ long long s_rec[kFG2];
    __shared__ int s_wh[kFG2][2];
    __shared__ const float *s_verts[kFG2];
    pdl_enter();
    __shared__ float s_fp[kFG2][RGBA_FP_STRIDE];
    __shared__ int s_ch[kNch];               // the model's blended channels, by slot
    __shared__ __align__(16) float s_red[kWarps * kFG2 * 32];  // dpsi: each warp's sums, 32 blendshapes
    const ModelInfo &m = c.models[blockIdx.y];
    const int chunk = blockIdx.x;
    const int i0 = chunk * kBwdChunk;
    if (i0 >= m.n_pad || m.nb == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = i0 + lane;
    const bool valid = i < m.n;      // real Gaussian
    const bool in_pad = i < m.n_pad; // row slot (padding slots receive zeros)
    const int K = m.k, A = m.A;
    float ibc1 = 0.f, ibc2 = 0.f;
    if (ADAM) {
        ibc1 = fa.step_dev ? adam_ibc(fa.step_dev, fa.b1) : fa.ibc1;
        ibc2 = fa.step_dev ? adam_ibc(fa.step_dev, fa.b2) : fa.ibc2;
    }
    const FusedAdamModel &am = fa.m[ADAM ? blockIdx.y : 0];
    {  // the chunk's blendshape rows travel to shared memory while the chain rule runs
        const int per_row = min(kBwdChunk, m.n_pad - i0) >> 2;  // n_pad, i0 multiples of 4
        auto copy = [&](int rr, int q) {
            cp_async16(s_dgc + rr * kDgRow + 4 * q, m.dg + (size_t)rr * m.n_pad + i0 + 4 * q);
        };
        if (per_row == kBwdChunk / 4) {  // a full chunk: thread t copies quad t % 8 of every 32nd row
            for (int rr = threadIdx.x / (kBwdChunk / 4); rr < K * A; rr += kBwdThreads / (kBwdChunk / 4))
                copy(rr, threadIdx.x % (kBwdChunk / 4));
        } else {
            for (int e = threadIdx.x; e < K * A * per_row; e += kBwdThreads) copy(e / per_row, e % per_row);
        }
    }
    if (threadIdx.x < A) s_ch[threadIdx.x] = m.chans[threadIdx.x];
    for (int g0 = 0; g0 < m.nb; g0 += kFG2) {
        const int ng = min(kFG2, m.nb - g0);
        if (threadIdx.x < ng) {
            const FrameInfo &f = c.frames[c.mframes[m.frame_off + g0 + threadIdx.x]];
            s_rec[threadIdx.x] = f.rec_base;
            s_wh[threadIdx.x][0] = f.W;
            s_wh[threadIdx.x][1] = f.H;
            s_verts[threadIdx.x] = f.verts;
        }
        for (int e = threadIdx.x; e < ng * RGBA_FP_STRIDE; e += kBwdThreads) {
            const int fl = e / RGBA_FP_STRIDE, q = e - fl * RGBA_FP_STRIDE;
            s_fp[fl][q] = c.fparams[(size_t)c.mframes[m.frame_off + g0 + fl] * RGBA_FP_STRIDE + q];
        }
        for (int e = threadIdx.x; e < kFG2 * max_k; e += kBwdThreads) {
            const int fl = e / max_k, kk = e % max_k;
            s_psi[e] = (fl < ng && kk < K) ? c.psi[(size_t)c.mframes[m.frame_off + g0 + fl] * c.k_stride + kk] : 0.f;
        }
        __syncthreads();
        // dL/dG_b per (frame, Gaussian) of the chunk (zero for culled Gaussians and for frames
        // past the group's end, which the loops below run over too); a warp takes 32
        // consecutive Gaussians of one frame
        {
            constexpr int kItems = kFG2 * kBwdChunk / kBwdThreads;
            float4 c0[kItems], c1[kItems], c2[kItems], ga[kItems], gb[kItems], gc[kItems];
            bool live[kItems];
#pragma unroll
            for (int u = 0; u < kItems; ++u) {  // every load of both items in flight at once
                const int e = threadIdx.x + u * kBwdThreads;
                const int fl = e / kBwdChunk, gi = i0 + (e & (kBwdChunk - 1));
                live[u] = fl < ng && gi < m.n;
                const long long r = live[u] ? s_rec[fl] + gi : 0;
                c0[u] = c1[u] = c2[u] = ga[u] = gb[u] = gc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (live[u]) {
                    c0[u] = c.cache[r * 3 + 0];
                    c1[u] = c.cache[r * 3 + 1];
                    c2[u] = c.cache[r * 3 + 2];  // (log-scale z, -, opacity, kept)
                    const float4 *gp = reinterpret_cast<const float4 *>(c.grad2d + r * kG2Floats);
                    ga[u] = gp[0];
                    gb[u] = gp[1];
                    gc[u] = gp[2];
                }
            }
#pragma unroll 1
            for (int u = 0; u < kItems; ++u) {
                const int e = threadIdx.x + u * kBwdThreads;
                const int fl = e / kBwdChunk, li = e & (kBwdChunk - 1);
                float dG[kNch];
#pragma unroll
                for (int q = 0; q < kNch; ++q) dG[q] = 0.f;
                if (live[0] && c2[0].w != 0.f) {  // item u sits in slot 0 (a rolled loop keeps the code small)
                    const float v[10] = {c0[0].x, c0[0].y, c0[0].z, c0[0].w, c1[0].x, c1[0].y, c1[0].z, c1[0].w, c2[0].x, c2[0].y};
                    const float g2[9] = {ga[0].x, ga[0].y, ga[0].z, ga[0].w, gb[0].x, gb[0].y, gb[0].z, gb[0].w, gc[0].x};
                    if (BOUND) {
                        float Rt[12] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f};
                        if (m.n_faces == 0 || tbn_fast(m, s_verts[fl], i0 + li, Rt))
                            chain<true>(v, c2[0].z, s_fp[fl], s_wh[fl][0], s_wh[fl][1], Rt, g2, dG);
                    } else {
                        chain<false>(v, c2[0].z, s_fp[fl], s_wh[fl][0], s_wh[fl][1], nullptr, g2, dG);
                    }
                }
#pragma unroll
                for (int q = 0; q < kNch; ++q) s_dG[fl * kDGF + q * kBwdChunk + li] = dG[q];
                if (c.grad_blended && fl < ng && i0 + li < m.n_pad) {  // rgba_render_bwd's optional output
                    float *o = c.grad_blended + s_rec[fl] * kNch + i0 + li;
#pragma unroll
                    for (int q = 0; q < kNch; ++q) o[(size_t)q * m.n_pad] = dG[q];
                }
#pragma unroll
                for (int w = 0; w + 1 < kItems; ++w) {
                    c0[w] = c0[w + 1];
                    c1[w] = c1[w + 1];
                    c2[w] = c2[w + 1];
                    ga[w] = ga[w + 1];
                    gb[w] = gb[w + 1];
                    gc[w] = gc[w + 1];
                    live[w] = live[w + 1];
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        // dG0[ch][i] = sum_b dG_b[ch][i]
        if ((ADAM ? am.p0 != nullptr : m.gg0 != nullptr) && in_pad) {
            for (int ch = warp; ch < kNch; ch += kWarps) {
                float a = 0.f;
                for (int fl = 0; fl < ng; ++fl) a += s_dG[fl * kDGF + ch * kBwdChunk + lane];
                const size_t o = (size_t)ch * m.n_pad + i;
                if (ADAM) {  // parked for the update below, exactly as the separate update reads it
                    s_g0[ch * kBwdChunk + lane] = 0.f + a;
                } else {
                    m.gg0[o] = (g0 == 0 ? 0.f : m.gg0[o]) + a;
                }
            }
        }
        const int grp = lane >> 2, tig = lane & 3;
        // dpsi_b[k] partial = sum over a, i of dG_k[a][i] dG_b[ch_a][i]: D (frames x k) =
        // A (frames x columns) B (columns x k), a column being (channel slot a, Gaussian i) and
        // 8 columns one k-step; the warps split the k-steps, their sums meet in s_red
        if (c.grad_psi) {
            const int KS = A * (kBwdChunk / 8);
            for (int kb = 0; kb < K; kb += 32) {
                float acc[4][4];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
                for (int ks = warp; ks < KS; ks += kWarps) {
                    const int sa = ks / (kBwdChunk / 8), ib = (ks % (kBwdChunk / 8)) * 8;
                    const float *dg = s_dG + s_ch[sa] * kBwdChunk + ib;  // + frame * kDGF
                    unsigned ah[4], al[4];
                    split_tf32(dg[grp * kDGF + tig], ah[0], al[0]);
                    split_tf32(dg[(grp + 8) * kDGF + tig], ah[1], al[1]);
                    split_tf32(dg[grp * kDGF + tig + 4], ah[2], al[2]);
                    split_tf32(dg[(grp + 8) * kDGF + tig + 4], ah[3], al[3]);
                    // padding columns hold whatever the caller left there: zero them
                    const bool v0 = i0 + ib + tig < m.n, v1 = i0 + ib + tig + 4 < m.n;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int kk = kb + j * 8 + grp;
                        const float *bs = s_dgc + ((size_t)kk * A + sa) * kDgRow + ib + tig;
                        unsigned bh[2], bl[2];
                        split_tf32(kk < K && v0 ? bs[0] : 0.f, bh[0], bl[0]);
                        split_tf32(kk < K && v1 ? bs[4] : 0.f, bh[1], bl[1]);
                        mma_3xtf32(acc[j], ah, al, bh, bl);
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {  // this warp's sums, then the warps' in a fixed order
                    float *r = s_red + warp * (kFG2 * 32) + grp * 32 + j * 8 + 2 * tig;
                    *reinterpret_cast<float2 *>(r) = make_float2(acc[j][0], acc[j][1]);
                    *reinterpret_cast<float2 *>(r + 8 * 32) = make_float2(acc[j][2], acc[j][3]);
                }
                __syncthreads();
                for (int e = threadIdx.x; e < kFG2 * 32; e += kBwdThreads) {
                    const int fl = e >> 5, kk = kb + (e & 31);
                    float t = 0.f;
#pragma unroll
                    for (int w = 0; w < kWarps; ++w) t += s_red[w * (kFG2 * 32) + e];
                    if (fl < ng && kk < K)
                        c.dpsi_part[m.dpsi_off + ((long long)(g0 + fl) * K + kk) * m.n_chunks + chunk] = t;
                }
                __syncthreads();
            }
        }
        // ddG[k][a][i] = sum_b psi_b[k] dG_b[ch_a][i]: D (k x columns) = A (k x frames)
        // B (frames x columns), two k-steps of 8 frames; the warps split the 8-column tiles
        if (ADAM ? true : m.gdg != nullptr) {
            const int NT = A * (kBwdChunk / 8);
            for (int mb = 0; mb < K; mb += 16) {
                const int k0 = mb + grp, k1 = k0 + 8;
                unsigned ah[2][4], al[2][4];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int f0 = q * 8 + tig, f1 = f0 + 4;
                    split_tf32(k0 < K ? s_psi[f0 * max_k + k0] : 0.f, ah[q][0], al[q][0]);
                    split_tf32(k1 < K ? s_psi[f0 * max_k + k1] : 0.f, ah[q][1], al[q][1]);
                    split_tf32(k0 < K ? s_psi[f1 * max_k + k0] : 0.f, ah[q][2], al[q][2]);
                    split_tf32(k1 < K ? s_psi[f1 * max_k + k1] : 0.f, ah[q][3], al[q][3]);
                }
                for (int nt = warp; nt < NT; nt += kWarps) {
                    const int sa = nt / (kBwdChunk / 8), ib = (nt % (kBwdChunk / 8)) * 8;
                    const float *dg = s_dG + s_ch[sa] * kBwdChunk + ib + grp;
                    float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        unsigned bh[2], bl[2];
                        split_tf32(dg[(q * 8 + tig) * kDGF], bh[0], bl[0]);
                        split_tf32(dg[(q * 8 + tig + 4) * kDGF], bh[1], bl[1]);
                        mma_3xtf32(d, ah[q], al[q], bh, bl);
                    }
                    const int i = ib + 2 * tig;  // columns i, i + 1 of rows k0 and k1
                    if (ADAM) {
                        // s_dgc is no longer read (dpsi is done): its slots park the gradients
                        if (k0 < K) {
                            s_dgc[((size_t)k0 * A + sa) * kDgRow + i] = 0.f + d[0];
                            s_dgc[((size_t)k0 * A + sa) * kDgRow + i + 1] = 0.f + d[1];
                        }
                        if (k1 < K) {
                            s_dgc[((size_t)k1 * A + sa) * kDgRow + i] = 0.f + d[2];
                            s_dgc[((size_t)k1 * A + sa) * kDgRow + i + 1] = 0.f + d[3];
                        }
                    } else if (i0 + i < m.n_pad) {  // n_pad - i0 is a multiple of 4: i + 1 too
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int kk = h ? k1 : k0;
                            if (kk >= K) continue;
                            float2 *o = reinterpret_cast<float2 *>(m.gdg + ((size_t)kk * A + sa) * m.n_pad + i0 + i);
                            const float2 old = g0 == 0 ? make_float2(0.f, 0.f) : *o;
                            *o = make_float2(old.x + d[2 * h], old.y + d[2 * h + 1]);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (ADAM) {
        // the update, streamed over the chunk's rows (G0 rows, then blendshape rows) by the whole
        // CTA, float4 by float4, with the loads of several float4s in flight per thread
        const int cols4 = min(kBwdChunk, m.n_pad - i0) >> 2;
        const int rows0 = am.p0 ? kNch : 0, rowsd = am.pd ? K * A : 0;
        const int total = (rows0 + rowsd) * cols4;
        constexpr int kU = 4;
        for (int e0 = threadIdx.x; e0 < total; e0 += kU * kBwdThreads) {
            float4 pp[kU], mm[kU], vv[kU];
            int rows[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {  // every load first
                const int e = e0 + u * kBwdThreads;
                rows[u] = e < total ? e / cols4 : -1;
                if (rows[u] >= 0) {
                    const int row = rows[u], c4 = e - row * cols4;
                    const bool base = row < rows0;
                    const size_t off = (size_t)(base ? row : row - rows0) * m.n_pad + i0 + 4 * c4;
                    pp[u] = *reinterpret_cast<const float4 *>((base ? am.p0 : am.pd) + off);
                    mm[u] = *reinterpret_cast<const float4 *>((base ? am.m0 : am.md) + off);
                    vv[u] = *reinterpret_cast<const float4 *>((base ? am.v0 : am.vd) + off);
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                if (rows[u] < 0) continue;
                const int e = e0 + u * kBwdThreads, row = rows[u], c4 = e - row * cols4;
                const bool base = row < rows0;
                const int rr = base ? row : row - rows0;
                const size_t off = (size_t)rr * m.n_pad + i0 + 4 * c4;
                const float4 g = *reinterpret_cast<const float4 *>((base ? s_g0 + rr * kBwdChunk : s_dgc + rr * kDgRow) + 4 * c4);
                const float lr = base ? am.lr0[rr] : am.lrd[rr % A];
                float p4[4] = {pp[u].x, pp[u].y, pp[u].z, pp[u].w}, m4[4] = {mm[u].x, mm[u].y, mm[u].z, mm[u].w},
                      v4[4] = {vv[u].x, vv[u].y, vv[u].z, vv[u].w};
                const float g4[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) adam_update(p4[q], g4[q], m4[q], v4[q], lr, fa.b1, fa.b2, fa.eps, ibc1, ibc2);
                *reinterpret_cast<float4 *>((base ? am.p0 : am.pd) + off) = make_float4(p4[0], p4[1], p4[2], p4[3]);
                *reinterpret_cast<float4 *>((base ? am.m0 : am.md) + off) = make_float4(m4[0], m4[1], m4[2], m4[3]);
                *reinterpret_cast<float4 *>((base ? am.v0 : am.vd) + off) = make_float4(v4[0], v4[1], v4[2], v4[3]);
            }
        }
    }
}

// dpsi[b][k] = sum over chunks of the partials; zero for k >= the model's k.
constexpr int kDpsiThreads = 256;

// One CTA per (blendshape k, frame b): the CTA's threads stride over the chunk partials, then
// a warp-shuffle and shared-memory sum.
__global__ void __launch_bounds__(kDpsiThreads) k_dpsi_reduce(Ctx c) {
    __shared__ float s_w[kDpsiThreads / 32];
    pdl_enter();
    const int kk = blockIdx.x, b = blockIdx.y;
    const FrameInfo &f = c.frames[b];
    const ModelInfo &m = c.models[f.model];
    float s = 0.f;
    if (kk < m.k) {
        // position of frame b in its model's frame list
        int j = 0;
        for (int q = 0; q < m.nb; ++q)
            if (c.mframes[m.frame_off + q] == b) j = q;
        const float *p = c.dpsi_part + m.dpsi_off + ((long long)j * m.k + kk) * m.n_chunks;
        for (int q = threadIdx.x; q < m.n_chunks; q += kDpsiThreads) s += p[q];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < kDpsiThreads / 32; ++w) t += s_w[w];
        c.grad_psi[(size_t)b * c.k_stride + kk] = t;
    }
}

}  // namespace

namespace {
template <bool ADAM, bool BOUND>
cudaError_t gauss_bwd_inst(const Ctx &c, int max_chunks, int max_k, int max_ka, const AdamArg<ADAM> &fa,
                           cudaStream_t s) {
    auto bytes = [](int k, int ka) { return (kFG2 * kDGF + kFG2 * k + ka * kDgRow) * (int)sizeof(float); };
    // set once, at the largest size any batch can ask for, so no attribute call happens while
    // a stream is being captured
    static int attr_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_device != dev) {
        e = cudaFuncSetAttribute(k_gauss_bwd<ADAM, BOUND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes(RGBA_MAX_K, RGBA_MAX_K * 13));
        if (e != cudaSuccess) return e;
        attr_device = dev;
    }
    dim3 g2(max_chunks, c.M);
    return launch_pdl(k_gauss_bwd<ADAM, BOUND>, g2, dim3(kBwdThreads), (size_t)bytes(max_k, max_ka), s, c, max_k,
                      fa);
}
}  // namespace

cudaError_t launch_gauss_bwd(const Ctx &c, int max_chunks, int max_k, int max_ka, const FusedAdam *fa,
                             bool any_bound, cudaStream_t s) {
    if (c.M == 0 || max_chunks == 0) return cudaSuccess;
    if (fa)
        return any_bound ? gauss_bwd_inst<true, true>(c, max_chunks, max_k, max_ka, *fa, s)
                         : gauss_bwd_inst<true, false>(c, max_chunks, max_k, max_ka, *fa, s);
    const NoAdam none{};
    return any_bound ? gauss_bwd_inst<false, true>(c, max_chunks, max_k, max_ka, none, s)
                     : gauss_bwd_inst<false, false>(c, max_chunks, max_k, max_ka, none, s);
}

cudaError_t launch_dpsi_reduce(const Ctx &c, int max_k, cudaStream_t s) {
    (void)max_k;
    if (!c.grad_psi || c.B == 0 || c.k_stride == 0) return cudaSuccess;
    return launch_pdl(k_dpsi_reduce, dim3(c.k_stride, c.B), dim3(kDpsiThreads), 0, s, c);
}

}  // namespace rgba
