/*
 * oracle.c -- plain, slow FP64 CPU oracle for the batch-parallel Gaussian blendshape rasterizer
 * of RGBAvatar (arXiv 2503.12886).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's CPU-baseline leg may
 * load this library. It shares no code, header, table or constant generator with the CUDA path;
 * both sides read the same seeded inputs and nothing else.
 *
 * What it computes, in the paper's order:
 *   Eq. 1 (Sec. 3.1)       linear blending  G^psi = G0 + sum_k psi_k dG_k on the blended channels
 *   Supp. Sec. A.3         activations after blending: exp scale, sigmoid opacity, normalised
 *                          quaternion, identity colour ("only RGB colour")
 *   Sec. 3.2 + Supp. A.3   the 3DGS "preprocess" the batch-parallel rasterizer builds on: EWA
 *                          projection of the 3-D covariance to a 2-D conic, screen radius, 16x16
 *                          tile rectangle, depth key (Kerbl et al. 2023; Zwicker et al. 2001)
 *   Sec. 3.2               binning into (frame, tile) lists sorted by depth, then front-to-back
 *                          alpha compositing per pixel ("rasterize")
 *   Sec. 3.2 "Loss"        the image loss gradient is back-propagated through compositing,
 *                          projection, activations and the blend to G0, dG and psi
 * The paper prints none of the projection or compositing formulas; they are the standard 3DGS
 * forms it cites (Supp. A.3 "builds upon the 3DGS renderer"). Constants it does not print:
 * alpha cutoff 1/255, alpha clamp 0.99, transmittance cutoff 1e-4, low-pass dilation 0.3 px^2,
 * 3-sigma radius, Jacobian clamp at 1.3x the half field of view, pixel centres at (px+0.5, py+0.5).
 *
 * Precision. Continuous values are FP64. Every DISCRETE quantity that the GPU must reproduce
 * bit for bit (cull, tile rectangle, depth sort key) is taken from the FP32 decision spec in
 * section 2 below: a fixed sequence of correctly rounded IEEE-754 binary32 operations (+ - * /,
 * sqrt, fused multiply-add where written, floor/ceil/rint), so that any conforming
 * implementation of the same sequence produces the same bits. Build with -ffp-contract=off.
 *
 * Tangent space (Supp. "Gaussian Transformation", Alg. 1), optional per model: a Gaussian bound
 * to triangle f of a mesh with UV atlas has its mean and rotation in the triangle's tangent
 * space. Per frame the mesh is deformed; the triangle's TBN matrix R = [T B N] (T and B the
 * derivatives of position along u and v, N the unit normal) and the barycentric point t of the
 * Gaussian's UV sample map the Gaussian to deformed space: x^D = R x^T + t, covariance
 * R Sigma^T R^T (the image of the Gaussian under x -> R x + t; this is the rotation q^D = R q^T
 * whenever R is orthonormal).
 *
 * Channel layout (planar [14][n_pad]): 0..2 mean, 3..6 quaternion (w,x,y,z), 7..9 log-scale,
 * 10 opacity logit, 11..13 RGB. Frame block [20]: 3x4 world->camera view matrix (row-major),
 * fx, fy, cx, cy, near, background RGB.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NCH 14
#define FP_FX 12
#define FP_FY 13
#define FP_CX 14
#define FP_CY 15
#define FP_NEAR 16
#define FP_BG 17

/* Compositing constants (3DGS defaults; the two cutoffs are fixed by the workload spec). */
#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_MIN 1e-4
#define DILATION 0.3
#define JCLAMP 1.3

static int popcount14(unsigned m) {
    int c = 0;
    for (int i = 0; i < NCH; ++i) c += (m >> i) & 1u;
    return c;
}

/* ============================================================================================
 * 1. Linear blending, Eq. 1:  G^psi[ch][i] = G0[ch][i] + sum_k psi[k] * dG[k][a(ch)][i]
 *    for every blended channel ch (a(ch) = rank of ch among the blended channels); the other
 *    channels are copied from G0.
 * ========================================================================================== */
void orc_blend(int n, int n_pad, int k, unsigned mask, const double *g0, const double *dg,
               const double *psi, double *out) {
    int a = 0;
    for (int ch = 0; ch < NCH; ++ch) {
        int blended = (mask >> ch) & 1u;
        for (int i = 0; i < n; ++i) {
            double v = g0[(size_t)ch * n_pad + i];
            if (blended) {
                int A = popcount14(mask);
                for (int kk = 0; kk < k; ++kk)
                    v += psi[kk] * dg[((size_t)kk * A + a) * n_pad + i];
            }
            out[(size_t)ch * n_pad + i] = v;
        }
        if (blended) ++a;
    }
}

/* Adjoint of Eq. 1 over the frames b that render this model:
 *   dG0[ch][i]    = sum_b dGb[b][ch][i]
 *   ddG[k][a][i]  = sum_b psi[b][k] * dGb[b][ch_a][i]
 *   dpsi[b][k]    = sum_i sum_a dG[k][a][i] * dGb[b][ch_a][i]                                  */
void orc_blend_bwd(int n, int n_pad, int k, unsigned mask, const double *dg, int nb,
                   const double *psi, const double *dgb, double *dg0, double *ddg,
                   double *dpsi) {
    int A = popcount14(mask);
    memset(dg0, 0, sizeof(double) * NCH * (size_t)n_pad);
    memset(ddg, 0, sizeof(double) * (size_t)k * A * n_pad);
    memset(dpsi, 0, sizeof(double) * (size_t)nb * k);
    for (int b = 0; b < nb; ++b) {
        const double *d = dgb + (size_t)b * NCH * n_pad;
        for (int ch = 0; ch < NCH; ++ch)
            for (int i = 0; i < n; ++i) dg0[(size_t)ch * n_pad + i] += d[(size_t)ch * n_pad + i];
        int a = 0;
        for (int ch = 0; ch < NCH; ++ch) {
            if (!((mask >> ch) & 1u)) continue;
            for (int kk = 0; kk < k; ++kk) {
                double s = 0.0;
                for (int i = 0; i < n; ++i) {
                    double gi = d[(size_t)ch * n_pad + i];
                    ddg[((size_t)kk * A + a) * n_pad + i] += psi[(size_t)b * k + kk] * gi;
                    s += dg[((size_t)kk * A + a) * n_pad + i] * gi;
                }
                dpsi[(size_t)b * k + kk] += s;
            }
            ++a;
        }
    }
}

/* ============================================================================================
 * 2. FP32 decision spec. Every operation below is one correctly rounded binary32 operation in
 *    the order written; fmaf is a single-rounding fused multiply-add.
 * ========================================================================================== */

/* exp for the decision path: Cody & Waite range reduction (Cody & Waite, "Software Manual for
 * the Elementary Functions", 1980) with ln 2 split into a short head and a tail, then the
 * degree-7 Taylor polynomial of e^r in Horner form (|r| <= ln2/2, truncation < 8e-9 relative),
 * then an exact scaling by 2^n.  x < -87 gives 0, x > 88 gives +inf.                           */
float orc_exp_spec(float x) {
    if (x != x) return x;
    if (x < -87.0f) return 0.0f;
    if (x > 88.0f) return INFINITY;
    const float log2e = 1.44269504088896341f;
    const float ln2_hi = 0.693145751953125f;      /* 0x3F317200 */
    const float ln2_lo = 1.428606765330187045e-06f; /* ln2 - ln2_hi */
    float n = rintf(x * log2e);
    float r = fmaf(-n, ln2_hi, x);
    r = fmaf(-n, ln2_lo, r);
    float p = 1.0f / 5040.0f;
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int e = (int)n; /* in [-126, 127] for x in [-87, 88] */
    union { uint32_t u; float f; } sc;
    sc.u = (uint32_t)(e + 127) << 23;
    return p * sc.f;
}

/* The decision spec for one (frame, Gaussian). Inputs are the fp32 model, weights and frame
 * block. Outputs: rect[4] = (x0, y0, x1, y1) half-open tile rectangle, all zero when culled;
 * f32[8] = (u, v, conic a, conic b, conic c, radius, depth, opacity) as computed by the spec
 * (radius = 0 when culled). Returns 1 when the Gaussian is kept.                               */
/* S1b (bound models only) the TBN matrix of Gaussian i's triangle (Alg. 1) and its barycentric
 * point, FP32 spec. With e1 = v1 - v0, e2 = v2 - v0 and UV differences (du1, dv1), (du2, dv2):
 * e1 = du1 T + dv1 B, e2 = du2 T + dv2 B, so T = (dv2 e1 - dv1 e2) / det and
 * B = (du1 e2 - du2 e1) / det with det = du1 dv2 - dv1 du2; N = (e1 x e2) / |e1 x e2|.
 * R[c] = (T_c, B_c, N_c); t_c = (b0 v0_c + b1 v1_c) + b2 v2_c. Every product and sum is
 * rounded separately, in the order written.                                                    */
static void tbn_spec(int i, int n_pad, const int32_t *faces, const float *face_uv,
                     const int32_t *face_of, const float *bary, const float *verts,
                     float R[3][3], float t[3]) {
    int f = face_of[i];
    const float *a = verts + 3 * (size_t)faces[3 * (size_t)f + 0];
    const float *b = verts + 3 * (size_t)faces[3 * (size_t)f + 1];
    const float *c = verts + 3 * (size_t)faces[3 * (size_t)f + 2];
    const float *uv = face_uv + 6 * (size_t)f;
    float e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = b[k] - a[k];
        e2[k] = c[k] - a[k];
    }
    float du1 = uv[2] - uv[0], dv1 = uv[3] - uv[1], du2 = uv[4] - uv[0], dv2 = uv[5] - uv[1];
    float p1 = du1 * dv2, p2 = dv1 * du2;
    float det = p1 - p2;
    float rd = 1.0f / det;
    float n[3];
    {
        float q1 = e1[1] * e2[2], q2 = e1[2] * e2[1];
        n[0] = q1 - q2;
        q1 = e1[2] * e2[0];
        q2 = e1[0] * e2[2];
        n[1] = q1 - q2;
        q1 = e1[0] * e2[1];
        q2 = e1[1] * e2[0];
        n[2] = q1 - q2;
    }
    float l2 = n[0] * n[0];
    l2 = l2 + n[1] * n[1];
    l2 = l2 + n[2] * n[2];
    float len = sqrtf(l2);
    float b0 = bary[i], b1 = bary[(size_t)n_pad + i], b2 = bary[2 * (size_t)n_pad + i];
    for (int k = 0; k < 3; ++k) {
        float x1 = dv2 * e1[k], x2 = dv1 * e2[k];
        R[k][0] = (x1 - x2) * rd;
        x1 = du1 * e2[k];
        x2 = du2 * e1[k];
        R[k][1] = (x1 - x2) * rd;
        R[k][2] = n[k] / len;
        float y = b0 * a[k];
        y = y + b1 * b[k];
        t[k] = y + b2 * c[k];
    }
}

int orc_decide_one(int i, int n_pad, int k, unsigned mask, const float *g0, const float *dg,
                   const float *psi, const float *fp, int W, int H, int TW, int TH,
                   int32_t *rect, float *f32, const int32_t *faces, const float *face_uv,
                   const int32_t *face_of, const float *bary, const float *verts) {
    int A = popcount14(mask);
    float v[NCH];
    int a = 0;
    /* S1 blend: v = g0; v = fmaf(psi_k, dG_k, v) for k = 0..K-1 */
    for (int ch = 0; ch < NCH; ++ch) {
        float x = g0[(size_t)ch * n_pad + i];
        if ((mask >> ch) & 1u) {
            for (int kk = 0; kk < k; ++kk)
                x = fmaf(psi[kk], dg[((size_t)kk * A + a) * n_pad + i], x);
            ++a;
        }
        v[ch] = x;
    }
    rect[0] = rect[1] = rect[2] = rect[3] = 0;
    for (int j = 0; j < 8; ++j) f32[j] = 0.0f;
    /* S1b tangent -> deformed space: x_c = fmaf(N_c, x2, fmaf(B_c, x1, fmaf(T_c, x0, t_c))) */
    float Rt[3][3], tt[3];
    const int bound = faces != NULL;
    if (bound) {
        tbn_spec(i, n_pad, faces, face_uv, face_of, bary, verts, Rt, tt);
        float xd[3];
        for (int c = 0; c < 3; ++c) xd[c] = fmaf(Rt[c][2], v[2], fmaf(Rt[c][1], v[1], fmaf(Rt[c][0], v[0], tt[c])));
        v[0] = xd[0];
        v[1] = xd[1];
        v[2] = xd[2];
    }
    /* S2 view transform p_j = fmaf(V_j2, x2, fmaf(V_j1, x1, fmaf(V_j0, x0, V_j3))) */
    float p[3];
    for (int j = 0; j < 3; ++j)
        p[j] = fmaf(fp[4 * j + 2], v[2], fmaf(fp[4 * j + 1], v[1], fmaf(fp[4 * j + 0], v[0],
                                                                        fp[4 * j + 3])));
    if (!(p[2] > fp[FP_NEAR])) return 0;
    /* S3 scales */
    float s[3];
    for (int m = 0; m < 3; ++m) s[m] = orc_exp_spec(v[7 + m]);
    /* S4 quaternion normalisation */
    float qw = v[3], qx = v[4], qy = v[5], qz = v[6];
    float n2 = fmaf(qz, qz, fmaf(qy, qy, fmaf(qx, qx, qw * qw)));
    if (!(n2 > 0.0f)) return 0;
    float inv = 1.0f / sqrtf(n2);
    float w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
    /* S5 rotation matrix */
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (yy + zz);
    R[0][1] = 2.0f * (xy - wz);
    R[0][2] = 2.0f * (xz + wy);
    R[1][0] = 2.0f * (xy + wz);
    R[1][1] = 1.0f - 2.0f * (xx + zz);
    R[1][2] = 2.0f * (yz - wx);
    R[2][0] = 2.0f * (xz - wy);
    R[2][1] = 2.0f * (yz + wx);
    R[2][2] = 1.0f - 2.0f * (xx + yy);
    /* S6 world covariance Sigma = R diag(s^2) R^T: M_im = R_im * d_m,
     *    Sigma_ij = fmaf(M_i2, R_j2, fmaf(M_i1, R_j1, M_i0 * R_j0))                              */
    float d[3] = {s[0] * s[0], s[1] * s[1], s[2] * s[2]};
    float Mm[3][3], Sg[3][3];
    for (int ii = 0; ii < 3; ++ii)
        for (int m = 0; m < 3; ++m) Mm[ii][m] = R[ii][m] * d[m];
    for (int ii = 0; ii < 3; ++ii)
        for (int jj = 0; jj < 3; ++jj)
            Sg[ii][jj] = fmaf(Mm[ii][2], R[jj][2], fmaf(Mm[ii][1], R[jj][1], Mm[ii][0] * R[jj][0]));
    /* S6b (bound) deformed-space covariance Rt Sigma Rt^T with P = Rt Sigma:
     *    P_ij = fmaf(Rt_i2, S_2j, fmaf(Rt_i1, S_1j, Rt_i0 * S_0j)); S_ij = fmaf(P_i2, Rt_j2, ...) */
    if (bound) {
        float P[3][3];
        for (int ii = 0; ii < 3; ++ii)
            for (int jj = 0; jj < 3; ++jj)
                P[ii][jj] = fmaf(Rt[ii][2], Sg[2][jj], fmaf(Rt[ii][1], Sg[1][jj], Rt[ii][0] * Sg[0][jj]));
        for (int ii = 0; ii < 3; ++ii)
            for (int jj = 0; jj < 3; ++jj)
                Sg[ii][jj] = fmaf(P[ii][2], Rt[jj][2], fmaf(P[ii][1], Rt[jj][1], P[ii][0] * Rt[jj][0]));
    }
    /* S7 camera covariance C = W Sigma W^T with T = W Sigma:
     *    T_ij = fmaf(W_i2, S_2j, fmaf(W_i1, S_1j, W_i0 * S_0j)); C_ij = fmaf(T_i2, W_j2, ...)    */
    float Tm[3][3], Cm[3][3];
    for (int ii = 0; ii < 3; ++ii)
        for (int jj = 0; jj < 3; ++jj)
            Tm[ii][jj] = fmaf(fp[4 * ii + 2], Sg[2][jj],
                              fmaf(fp[4 * ii + 1], Sg[1][jj], fp[4 * ii + 0] * Sg[0][jj]));
    for (int ii = 0; ii < 3; ++ii)
        for (int jj = 0; jj < 3; ++jj)
            Cm[ii][jj] = fmaf(Tm[ii][2], fp[4 * jj + 2],
                              fmaf(Tm[ii][1], fp[4 * jj + 1], Tm[ii][0] * fp[4 * jj + 0]));
    /* S8 EWA Jacobian with the ratio clamp at 1.3 x tan(half fov) */
    float fx = fp[FP_FX], fy = fp[FP_FY];
    float limx = 1.3f * ((0.5f * (float)W) / fx);
    float limy = 1.3f * ((0.5f * (float)H) / fy);
    float rx = p[0] / p[2], ry = p[1] / p[2];
    rx = fminf(limx, fmaxf(-limx, rx));
    ry = fminf(limy, fmaxf(-limy, ry));
    float J[2][3];
    J[0][0] = fx / p[2];
    J[0][1] = 0.0f;
    J[0][2] = -(fx * rx) / p[2];
    J[1][0] = 0.0f;
    J[1][1] = fy / p[2];
    J[1][2] = -(fy * ry) / p[2];
    /* S9 Sigma' = J C J^T + 0.3 I: K = J C, S'_ij = fmaf(K_i2, J_j2, fmaf(K_i1, J_j1, K_i0*J_j0)) */
    float Km[2][3], Sp[2][2];
    for (int ii = 0; ii < 2; ++ii)
        for (int jj = 0; jj < 3; ++jj)
            Km[ii][jj] = fmaf(J[ii][2], Cm[2][jj], fmaf(J[ii][1], Cm[1][jj], J[ii][0] * Cm[0][jj]));
    for (int ii = 0; ii < 2; ++ii)
        for (int jj = 0; jj < 2; ++jj)
            Sp[ii][jj] = fmaf(Km[ii][2], J[jj][2], fmaf(Km[ii][1], J[jj][1], Km[ii][0] * J[jj][0]));
    float cA = Sp[0][0] + 0.3f, cB = Sp[0][1], cC = Sp[1][1] + 0.3f;
    /* S10 determinant and conic */
    float det = cA * cC - cB * cB;
    if (!(det > 0.0f)) return 0;
    float conic_a = cC / det, conic_b = -cB / det, conic_c = cA / det;
    /* S11 radius from the larger eigenvalue */
    float mid = 0.5f * (cA + cC);
    float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
    float r = ceilf(3.0f * sqrtf(lam));
    /* S12 screen-space mean (pixel centres sit at integer + 0.5) */
    float u = fx * (p[0] / p[2]) + fp[FP_CX];
    float vv = fy * (p[1] / p[2]) + fp[FP_CY];
    /* S13 tile rectangle, half-open, clamped to the grid */
    int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH;
    float ftw = (float)TW, fth = (float)TH;
    float x0 = floorf((u - r) / ftw), x1 = floorf(((u + r) + (ftw - 1.0f)) / ftw);
    float y0 = floorf((vv - r) / fth), y1 = floorf(((vv + r) + (fth - 1.0f)) / fth);
    x0 = fminf((float)tx, fmaxf(0.0f, x0));
    x1 = fminf((float)tx, fmaxf(0.0f, x1));
    y0 = fminf((float)ty, fmaxf(0.0f, y0));
    y1 = fminf((float)ty, fmaxf(0.0f, y1));
    if (x0 != x0 || y0 != y0 || x1 != x1 || y1 != y1) return 0;
    int ix0 = (int)x0, ix1 = (int)x1, iy0 = (int)y0, iy1 = (int)y1;
    if ((ix1 - ix0) * (iy1 - iy0) <= 0) return 0;
    rect[0] = ix0;
    rect[1] = iy0;
    rect[2] = ix1;
    rect[3] = iy1;
    f32[0] = u;
    f32[1] = vv;
    f32[2] = conic_a;
    f32[3] = conic_b;
    f32[4] = conic_c;
    f32[5] = r;
    f32[6] = p[2];
    /* opacity (not a decision; reported for reference) */
    f32[7] = 1.0f / (1.0f + orc_exp_spec(-v[10]));
    return 1;
}

void orc_decide(int n, int n_pad, int k, unsigned mask, const float *g0, const float *dg,
                const float *psi, const float *fp, int W, int H, int TW, int TH, int32_t *rect,
                float *f32, const int32_t *faces, const float *face_uv, const int32_t *face_of,
                const float *bary, const float *verts) {
    for (int i = 0; i < n; ++i)
        orc_decide_one(i, n_pad, k, mask, g0, dg, psi, fp, W, H, TW, TH, rect + 4 * (size_t)i,
                       f32 + 8 * (size_t)i, faces, face_uv, face_of, bary, verts);
}

/* FP64 TBN matrix and barycentric point of Gaussian i (Alg. 1; same definitions as tbn_spec):
 * out[0..8] = R row-major (columns T, B, N), out[9..11] = t.                                   */
void orc_tbn(int i, int n_pad, const int32_t *faces, const float *face_uv, const int32_t *face_of,
             const float *bary, const float *verts, double *out) {
    int f = face_of[i];
    double a[3], b[3], c[3], e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = verts[3 * (size_t)faces[3 * (size_t)f + 0] + k];
        b[k] = verts[3 * (size_t)faces[3 * (size_t)f + 1] + k];
        c[k] = verts[3 * (size_t)faces[3 * (size_t)f + 2] + k];
        e1[k] = b[k] - a[k];
        e2[k] = c[k] - a[k];
    }
    const float *uv = face_uv + 6 * (size_t)f;
    double du1 = (double)uv[2] - uv[0], dv1 = (double)uv[3] - uv[1];
    double du2 = (double)uv[4] - uv[0], dv2 = (double)uv[5] - uv[1];
    double det = du1 * dv2 - dv1 * du2;
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                   e1[0] * e2[1] - e1[1] * e2[0]};
    double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double bb[3] = {bary[i], bary[(size_t)n_pad + i], bary[2 * (size_t)n_pad + i]};
    for (int k = 0; k < 3; ++k) {
        out[3 * k + 0] = (dv2 * e1[k] - dv1 * e2[k]) / det;
        out[3 * k + 1] = (du1 * e2[k] - du2 * e1[k]) / det;
        out[3 * k + 2] = n[k] / len;
        out[9 + k] = bb[0] * a[k] + bb[1] * b[k] + bb[2] * c[k];
    }
}

void orc_tbn_all(int n, int n_pad, const int32_t *faces, const float *face_uv, const int32_t *face_of,
                 const float *bary, const float *verts, double *out) {
    for (int i = 0; i < n; ++i) orc_tbn(i, n_pad, faces, face_uv, face_of, bary, verts, out + 12 * (size_t)i);
}

/* ============================================================================================
 * 3. FP64 projection (3DGS preprocess; EWA splatting of Zwicker et al. 2001).
 * ========================================================================================== */
typedef struct {
    double p[3], qn[4], qlen, s[3], R[3][3], Sig[3][3], Mc[3][3], J[2][3], Rt[3][3];
    int bound;
    double rx, ry;
    int clx, cly;
    double A, B, C, det, conic[3], u, v, o, col[3];
} fwd64;

/* tbn (bound models): [12] = TBN matrix R row-major, then t (orc_tbn); NULL when unbound.      */
static void project64(const double *g, const double *fp, int W, int H, const double *tbn, fwd64 *f) {
    const double *V = fp;
    double x[3] = {g[0], g[1], g[2]};
    f->bound = tbn != NULL;
    if (f->bound) { /* x^D = R x^T + t */
        double xd[3];
        for (int c = 0; c < 3; ++c) {
            for (int k = 0; k < 3; ++k) f->Rt[c][k] = tbn[3 * c + k];
            xd[c] = tbn[3 * c] * x[0] + tbn[3 * c + 1] * x[1] + tbn[3 * c + 2] * x[2] + tbn[9 + c];
        }
        for (int c = 0; c < 3; ++c) x[c] = xd[c];
    }
    for (int j = 0; j < 3; ++j)
        f->p[j] = V[4 * j] * x[0] + V[4 * j + 1] * x[1] + V[4 * j + 2] * x[2] + V[4 * j + 3];
    /* activations applied after blending (Supp. A.3) */
    for (int m = 0; m < 3; ++m) f->s[m] = exp(g[7 + m]);
    f->qlen = sqrt(g[3] * g[3] + g[4] * g[4] + g[5] * g[5] + g[6] * g[6]);
    for (int m = 0; m < 4; ++m) f->qn[m] = g[3 + m] / f->qlen;
    f->o = 1.0 / (1.0 + exp(-g[10]));
    for (int c = 0; c < 3; ++c) f->col[c] = g[11 + c];
    double w = f->qn[0], qx = f->qn[1], qy = f->qn[2], qz = f->qn[3];
    double (*R)[3] = f->R;
    R[0][0] = 1 - 2 * (qy * qy + qz * qz);
    R[0][1] = 2 * (qx * qy - w * qz);
    R[0][2] = 2 * (qx * qz + w * qy);
    R[1][0] = 2 * (qx * qy + w * qz);
    R[1][1] = 1 - 2 * (qx * qx + qz * qz);
    R[1][2] = 2 * (qy * qz - w * qx);
    R[2][0] = 2 * (qx * qz - w * qy);
    R[2][1] = 2 * (qy * qz + w * qx);
    R[2][2] = 1 - 2 * (qx * qx + qy * qy);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int m = 0; m < 3; ++m) acc += R[i][m] * f->s[m] * f->s[m] * R[j][m];
            f->Sig[i][j] = acc;
        }
    if (f->bound) { /* deformed-space covariance Rt Sigma Rt^T */
        double S[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) acc += f->Rt[i][a] * f->Sig[a][b] * f->Rt[j][b];
                S[i][j] = acc;
            }
        memcpy(f->Sig, S, sizeof(S));
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += V[4 * i + a] * f->Sig[a][b] * V[4 * j + b];
            f->Mc[i][j] = acc;
        }
    double fx = fp[FP_FX], fy = fp[FP_FY];
    double limx = JCLAMP * (0.5 * W / fx), limy = JCLAMP * (0.5 * H / fy);
    double rx = f->p[0] / f->p[2], ry = f->p[1] / f->p[2];
    f->clx = (rx > limx || rx < -limx);
    f->cly = (ry > limy || ry < -limy);
    f->rx = rx > limx ? limx : (rx < -limx ? -limx : rx);
    f->ry = ry > limy ? limy : (ry < -limy ? -limy : ry);
    double z = f->p[2];
    f->J[0][0] = fx / z;
    f->J[0][1] = 0;
    f->J[0][2] = -fx * f->rx / z;
    f->J[1][0] = 0;
    f->J[1][1] = fy / z;
    f->J[1][2] = -fy * f->ry / z;
    double S2[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += f->J[i][a] * f->Mc[a][b] * f->J[j][b];
            S2[i][j] = acc;
        }
    f->A = S2[0][0] + DILATION;
    f->B = S2[0][1];
    f->C = S2[1][1] + DILATION;
    f->det = f->A * f->C - f->B * f->B;
    f->conic[0] = f->C / f->det;
    f->conic[1] = -f->B / f->det;
    f->conic[2] = f->A / f->det;
    f->u = fx * f->p[0] / z + fp[FP_CX];
    f->v = fy * f->p[1] / z + fp[FP_CY];
}

/* Per-Gaussian render record: out[n][12] = (u, v, conic a, b, c, opacity, r, g, b, depth, 0, 0)
 * for Gaussians kept by the decision spec (rect area > 0); zeros otherwise.                    */
void orc_project(int n, int n_pad, const double *blended, const double *fp, int W, int H,
                 const int32_t *rect, double *out, const double *tbn) {
    double g[NCH];
    for (int i = 0; i < n; ++i) {
        double *o = out + 12 * (size_t)i;
        for (int j = 0; j < 12; ++j) o[j] = 0.0;
        const int32_t *rc = rect + 4 * (size_t)i;
        if ((rc[2] - rc[0]) * (rc[3] - rc[1]) <= 0) continue;
        for (int ch = 0; ch < NCH; ++ch) g[ch] = blended[(size_t)ch * n_pad + i];
        fwd64 f;
        project64(g, fp, W, H, tbn ? tbn + 12 * (size_t)i : NULL, &f);
        o[0] = f.u;
        o[1] = f.v;
        o[2] = f.conic[0];
        o[3] = f.conic[1];
        o[4] = f.conic[2];
        o[5] = f.o;
        o[6] = f.col[0];
        o[7] = f.col[1];
        o[8] = f.col[2];
        o[9] = f.p[2];
    }
}

/* Chain rule of the projection: grad2d[n][9] = dL/d(u, v, conic a, b, c, opacity, r, g, b)
 * -> dG[14][n_pad], the gradient w.r.t. the blended (pre-activation) channels.                 */
void orc_project_bwd(int n, int n_pad, const double *blended, const double *fp, int W, int H,
                     const int32_t *rect, const double *grad2d, double *dG, const double *tbn) {
    double g[NCH];
    for (int i = 0; i < n; ++i) {
        for (int ch = 0; ch < NCH; ++ch) dG[(size_t)ch * n_pad + i] = 0.0;
        const int32_t *rc = rect + 4 * (size_t)i;
        if ((rc[2] - rc[0]) * (rc[3] - rc[1]) <= 0) continue;
        for (int ch = 0; ch < NCH; ++ch) g[ch] = blended[(size_t)ch * n_pad + i];
        fwd64 f;
        project64(g, fp, W, H, tbn ? tbn + 12 * (size_t)i : NULL, &f);
        const double *gg = grad2d + 9 * (size_t)i;
        double du = gg[0], dv = gg[1], dca = gg[2], dcb = gg[3], dcc = gg[4], dop = gg[5];
        /* opacity: o = sigmoid(logit) */
        dG[(size_t)10 * n_pad + i] = dop * f.o * (1.0 - f.o);
        /* colour: identity */
        for (int c = 0; c < 3; ++c) dG[(size_t)(11 + c) * n_pad + i] = gg[6 + c];
        /* conic = inverse of [[A, B], [B, C]] */
        double A = f.A, B = f.B, C = f.C, D = f.det, D2 = D * D;
        double dA = dca * (-C * C / D2) + dcb * (B * C / D2) + dcc * (1.0 / D - A * C / D2);
        double dC = dca * (1.0 / D - A * C / D2) + dcb * (A * B / D2) + dcc * (-A * A / D2);
        double dB = dca * (2.0 * B * C / D2) + dcb * (-1.0 / D - 2.0 * B * B / D2) +
                    dcc * (2.0 * A * B / D2);
        double G2[2][2] = {{dA, 0.5 * dB}, {0.5 * dB, dC}};
        /* Sigma' = J Mc J^T:  dJ = 2 G2 J Mc,  dMc = J^T G2 J */
        double dJ[2][3], dM[3][3];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 3; ++b) acc += G2[r][a] * f.J[a][b] * f.Mc[b][c];
                dJ[r][c] = 2.0 * acc;
            }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) acc += f.J[a][r] * G2[a][b] * f.J[b][c];
                dM[r][c] = acc;
            }
        /* Mc = V Sig V^T:  dSig = V^T dM V */
        const double *V = fp;
        double dS[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) acc += V[4 * a + r] * dM[a][b] * V[4 * b + c];
                dS[r][c] = acc;
            }
        if (f.bound) { /* Sigma^D = Rt Sigma^T Rt^T:  dSigma^T = Rt^T dSigma^D Rt */
            double dT[3][3];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    double acc = 0;
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) acc += f.Rt[a][r] * dS[a][b] * f.Rt[b][c];
                    dT[r][c] = acc;
                }
            memcpy(dS, dT, sizeof(dT));
        }
        /* Sig = R diag(s^2) R^T:  dR = 2 dS R diag(s^2),  ds_m = 2 s_m (R^T dS R)_mm */
        double dR[3][3], ds[3];
        for (int r = 0; r < 3; ++r)
            for (int m = 0; m < 3; ++m) {
                double acc = 0;
                for (int a = 0; a < 3; ++a) acc += dS[r][a] * f.R[a][m];
                dR[r][m] = 2.0 * acc * f.s[m] * f.s[m];
            }
        for (int m = 0; m < 3; ++m) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += f.R[a][m] * dS[a][b] * f.R[b][m];
            ds[m] = 2.0 * f.s[m] * acc;
            dG[(size_t)(7 + m) * n_pad + i] = ds[m] * f.s[m]; /* s = exp(log-scale) */
        }
        /* R(q) for the unit quaternion (w, x, y, z) */
        double w = f.qn[0], x = f.qn[1], y = f.qn[2], z = f.qn[3];
        double dw = dR[0][1] * (-2 * z) + dR[0][2] * (2 * y) + dR[1][0] * (2 * z) +
                    dR[1][2] * (-2 * x) + dR[2][0] * (-2 * y) + dR[2][1] * (2 * x);
        double dx = dR[0][1] * (2 * y) + dR[0][2] * (2 * z) + dR[1][0] * (2 * y) +
                    dR[1][1] * (-4 * x) + dR[1][2] * (-2 * w) + dR[2][0] * (2 * z) +
                    dR[2][1] * (2 * w) + dR[2][2] * (-4 * x);
        double dy = dR[0][0] * (-4 * y) + dR[0][1] * (2 * x) + dR[0][2] * (2 * w) +
                    dR[1][0] * (2 * x) + dR[1][2] * (2 * z) + dR[2][0] * (-2 * w) +
                    dR[2][1] * (2 * z) + dR[2][2] * (-4 * y);
        double dz = dR[0][0] * (-4 * z) + dR[0][1] * (-2 * w) + dR[0][2] * (2 * x) +
                    dR[1][0] * (2 * w) + dR[1][1] * (-4 * z) + dR[1][2] * (2 * y) +
                    dR[2][0] * (2 * x) + dR[2][1] * (2 * y);
        double dqn[4] = {dw, dx, dy, dz};
        double dot = 0;
        for (int m = 0; m < 4; ++m) dot += f.qn[m] * dqn[m];
        for (int m = 0; m < 4; ++m)
            dG[(size_t)(3 + m) * n_pad + i] = (dqn[m] - f.qn[m] * dot) / f.qlen;
        /* mean: u = fx px/pz + cx, v = fy py/pz + cy, and J(p) */
        double fx = fp[FP_FX], fy = fp[FP_FY], pz = f.p[2];
        double dp[3] = {0, 0, 0};
        dp[0] += du * fx / pz;
        dp[1] += dv * fy / pz;
        dp[2] += -du * fx * f.p[0] / (pz * pz) - dv * fy * f.p[1] / (pz * pz);
        dp[2] += dJ[0][0] * (-fx / (pz * pz)) + dJ[1][1] * (-fy / (pz * pz));
        if (!f.clx) {
            dp[0] += dJ[0][2] * (-fx / (pz * pz));
            dp[2] += dJ[0][2] * (2.0 * fx * f.p[0] / (pz * pz * pz));
        } else {
            dp[2] += dJ[0][2] * (fx * f.rx / (pz * pz));
        }
        if (!f.cly) {
            dp[1] += dJ[1][2] * (-fy / (pz * pz));
            dp[2] += dJ[1][2] * (2.0 * fy * f.p[1] / (pz * pz * pz));
        } else {
            dp[2] += dJ[1][2] * (fy * f.ry / (pz * pz));
        }
        double dxw[3];
        for (int c = 0; c < 3; ++c) dxw[c] = V[c] * dp[0] + V[4 + c] * dp[1] + V[8 + c] * dp[2];
        for (int c = 0; c < 3; ++c) /* x^D = Rt x^T + t:  dx^T = Rt^T dx^D */
            dG[(size_t)c * n_pad + i] =
                f.bound ? f.Rt[0][c] * dxw[0] + f.Rt[1][c] * dxw[1] + f.Rt[2][c] * dxw[2] : dxw[c];
    }
}

/* ============================================================================================
 * 4. Binning and depth sort (Sec. 3.2 "preprocess" output feeding "rasterize"):
 *    every kept Gaussian is listed in every tile of its rectangle; each tile's list is ordered
 *    by (fp32 depth bits ascending, Gaussian index ascending).
 * ========================================================================================== */
typedef struct { uint32_t key; int32_t idx; } kv;

static int kv_cmp(const void *a, const void *b) {
    const kv *x = (const kv *)a, *y = (const kv *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* tile_start[tiles_x*tiles_y + 1]; list may be NULL (count only). Returns the pair count. */
int64_t orc_bin(int n, const int32_t *rect, const float *depth, int tiles_x, int tiles_y,
                int32_t *tile_start, int32_t *list) {
    int nt = tiles_x * tiles_y;
    int64_t *cnt = (int64_t *)calloc((size_t)nt + 1, sizeof(int64_t));
    for (int i = 0; i < n; ++i) {
        const int32_t *r = rect + 4 * (size_t)i;
        for (int y = r[1]; y < r[3]; ++y)
            for (int x = r[0]; x < r[2]; ++x) cnt[y * tiles_x + x]++;
    }
    int64_t total = 0;
    for (int t = 0; t < nt; ++t) {
        tile_start[t] = (int32_t)total;
        total += cnt[t];
    }
    tile_start[nt] = (int32_t)total;
    if (list) {
        kv *buf = (kv *)malloc(sizeof(kv) * (size_t)(total > 0 ? total : 1));
        int64_t *fill = (int64_t *)calloc((size_t)nt + 1, sizeof(int64_t));
        for (int i = 0; i < n; ++i) {
            const int32_t *r = rect + 4 * (size_t)i;
            uint32_t bits;
            memcpy(&bits, &depth[i], 4);
            for (int y = r[1]; y < r[3]; ++y)
                for (int x = r[0]; x < r[2]; ++x) {
                    int t = y * tiles_x + x;
                    kv e = {bits, i};
                    buf[tile_start[t] + fill[t]++] = e;
                }
        }
        for (int t = 0; t < nt; ++t)
            qsort(buf + tile_start[t], (size_t)cnt[t], sizeof(kv), kv_cmp);
        for (int64_t p = 0; p < total; ++p) list[p] = buf[p].idx;
        free(buf);
        free(fill);
    }
    free(cnt);
    return total;
}

/* ============================================================================================
 * 5. Front-to-back compositing per pixel (3DGS "rasterize"):
 *      power = -(a dx^2 + c dy^2)/2 - b dx dy,  skip if power > 0
 *      alpha = min(0.99, o e^power),           skip if alpha < 1/255
 *      stop (without blending) when T (1 - alpha) < 1e-4
 *      C += colour alpha T;  T *= 1 - alpha;   n_contrib = list position + 1
 *    output C + T bg, T_final, n_contrib.  d = pixel centre - mean, centre = (px+0.5, py+0.5).
 * ========================================================================================== */
#define FLAG_ALPHA_MIN 1u
#define FLAG_ALPHA_MAX 2u
#define FLAG_T_MIN 4u

static inline uint64_t fnv(uint64_t h, uint64_t v) {
    for (int i = 0; i < 8; ++i) {
        h ^= (v >> (8 * i)) & 0xFFu;
        h *= 0x100000001B3ull;
    }
    return h;
}

/* tile_mask (may be NULL): render only tiles with a non-zero byte.  eps / eps_t: relative
 * distance to an alpha cutoff / to the transmittance cutoff below which a pixel is flagged
 * ambiguous.  stats[0] += list entries evaluated, stats[1] += pixels rendered.  Returns the
 * decision hash of the rendered pixels.                                                        */
uint64_t orc_render(int W, int H, int TW, int TH, const double *rec, const int32_t *tile_start,
                    const int32_t *list, const double *bg, const uint8_t *tile_mask, double eps,
                    double eps_t, double *img, double *T_out, int32_t *n_out, uint8_t *flags,
                    double *stats) {
    int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    uint64_t hash = 0xCBF29CE484222325ull;
    for (int ty = 0; ty < tiles_y; ++ty)
        for (int tx = 0; tx < tiles_x; ++tx) {
            int t = ty * tiles_x + tx;
            if (tile_mask && !tile_mask[t]) continue;
            for (int py = ty * TH; py < (ty + 1) * TH && py < H; ++py)
                for (int px = tx * TW; px < (tx + 1) * TW && px < W; ++px) {
                    double T = 1.0, C[3] = {0, 0, 0};
                    int32_t last = 0;
                    uint8_t fl = 0;
                    double ev = 0;
                    for (int32_t j = tile_start[t]; j < tile_start[t + 1]; ++j) {
                        const double *g = rec + 12 * (size_t)list[j];
                        double dx = px + 0.5 - g[0], dy = py + 0.5 - g[1];
                        double power = -0.5 * (g[2] * dx * dx + g[4] * dy * dy) - g[3] * dx * dy;
                        ev += 1;
                        if (power > 0.0) {
                            hash = fnv(hash, ((uint64_t)j << 4) | 1u);
                            continue;
                        }
                        double araw = g[5] * exp(power);
                        double alpha = araw < ALPHA_MAX ? araw : ALPHA_MAX;
                        if (fabs(araw - ALPHA_MAX) <= eps * ALPHA_MAX) fl |= FLAG_ALPHA_MAX;
                        if (fabs(alpha - ALPHA_MIN) <= eps * ALPHA_MIN) fl |= FLAG_ALPHA_MIN;
                        if (alpha < ALPHA_MIN) {
                            hash = fnv(hash, ((uint64_t)j << 4) | 2u);
                            continue;
                        }
                        double testT = T * (1.0 - alpha);
                        if (fabs(testT - T_MIN) <= eps_t * T_MIN) fl |= FLAG_T_MIN;
                        if (testT < T_MIN) {
                            hash = fnv(hash, ((uint64_t)j << 4) | 3u);
                            break;
                        }
                        for (int c = 0; c < 3; ++c) C[c] += g[6 + c] * alpha * T;
                        T = testT;
                        last = j - tile_start[t] + 1;
                        hash = fnv(hash, ((uint64_t)j << 4) | (araw > ALPHA_MAX ? 5u : 4u));
                    }
                    size_t pix = (size_t)py * W + px;
                    for (int c = 0; c < 3; ++c) img[(size_t)c * W * H + pix] = C[c] + T * bg[c];
                    T_out[pix] = T;
                    n_out[pix] = last;
                    flags[pix] = fl;
                    if (stats) {
                        stats[0] += ev;
                        stats[1] += 1;
                    }
                }
        }
    return hash;
}

/* Colour initialisation (Sec. 3.2 "Initialization", Eq. 3), the sums of one frame: the same
 * front-to-back compositing as orc_render, and for every Gaussian that a pixel blends, with its
 * splatting weight w = alpha T at that pixel and the target colour I of the pixel,
 *   acc[g][0] += w,  acc[g][1 + c] += w I_c        (target planar [3][H][W]).              */
void orc_color_accum(int W, int H, int TW, int TH, const double *rec, const int32_t *tile_start,
                     const int32_t *list, const double *target, double *acc) {
    int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    for (int ty = 0; ty < tiles_y; ++ty)
        for (int tx = 0; tx < tiles_x; ++tx) {
            int t = ty * tiles_x + tx;
            for (int py = ty * TH; py < (ty + 1) * TH && py < H; ++py)
                for (int px = tx * TW; px < (tx + 1) * TW && px < W; ++px) {
                    size_t pix = (size_t)py * W + px;
                    double T = 1.0;
                    for (int32_t j = tile_start[t]; j < tile_start[t + 1]; ++j) {
                        const double *g = rec + 12 * (size_t)list[j];
                        double dx = px + 0.5 - g[0], dy = py + 0.5 - g[1];
                        double power = -0.5 * (g[2] * dx * dx + g[4] * dy * dy) - g[3] * dx * dy;
                        if (power > 0.0) continue;
                        double araw = g[5] * exp(power);
                        double alpha = araw < ALPHA_MAX ? araw : ALPHA_MAX;
                        if (alpha < ALPHA_MIN) continue;
                        double testT = T * (1.0 - alpha);
                        if (testT < T_MIN) break;
                        double w = alpha * T;
                        double *a = acc + 4 * (size_t)list[j];
                        a[0] += w;
                        for (int c = 0; c < 3; ++c) a[1 + c] += w * target[(size_t)c * W * H + pix];
                        T = testT;
                    }
                }
        }
}

/* Exact derivative of the compositing above (reverse sweep over the contributors).
 * dL_dimg[3][H][W] -> grad2d[n][9] += dL/d(u, v, conic a, b, c, opacity, r, g, b).
 * The oracle keeps each pixel's contributors in a local list; the clamp at 0.99 passes no
 * gradient while it is active; skipped Gaussians and the stopping decision carry none.         */
typedef struct { int32_t g; double alpha, G, T, dx, dy; int clamped; } contrib;

void orc_render_bwd(int W, int H, int TW, int TH, const double *rec, const int32_t *tile_start,
                    const int32_t *list, const double *bg, const double *dL_dimg,
                    const uint8_t *tile_mask, double *grad2d) {
    int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    size_t cap = 1024;
    contrib *cs = (contrib *)malloc(sizeof(contrib) * cap);
    for (int ty = 0; ty < tiles_y; ++ty)
        for (int tx = 0; tx < tiles_x; ++tx) {
            int t = ty * tiles_x + tx;
            if (tile_mask && !tile_mask[t]) continue;
            for (int py = ty * TH; py < (ty + 1) * TH && py < H; ++py)
                for (int px = tx * TW; px < (tx + 1) * TW && px < W; ++px) {
                    size_t nc = 0;
                    double T = 1.0;
                    for (int32_t j = tile_start[t]; j < tile_start[t + 1]; ++j) {
                        const double *g = rec + 12 * (size_t)list[j];
                        double dx = px + 0.5 - g[0], dy = py + 0.5 - g[1];
                        double power = -0.5 * (g[2] * dx * dx + g[4] * dy * dy) - g[3] * dx * dy;
                        if (power > 0.0) continue;
                        double G = exp(power);
                        double araw = g[5] * G;
                        double alpha = araw < ALPHA_MAX ? araw : ALPHA_MAX;
                        if (alpha < ALPHA_MIN) continue;
                        double testT = T * (1.0 - alpha);
                        if (testT < T_MIN) break;
                        if (nc == cap) {
                            cap *= 2;
                            cs = (contrib *)realloc(cs, sizeof(contrib) * cap);
                        }
                        contrib e = {list[j], alpha, G, T, dx, dy, araw > ALPHA_MAX};
                        cs[nc++] = e;
                        T = testT;
                    }
                    double Tfin = T;
                    size_t pix = (size_t)py * W + px;
                    double gC[3], bgdot = 0;
                    for (int c = 0; c < 3; ++c) {
                        gC[c] = dL_dimg[(size_t)c * W * H + pix];
                        bgdot += gC[c] * bg[c];
                    }
                    double S[3] = {0, 0, 0}; /* normalised colour behind the current Gaussian */
                    for (size_t q = nc; q-- > 0;) {
                        const contrib *e = &cs[q];
                        const double *g = rec + 12 * (size_t)e->g;
                        double *gr = grad2d + 9 * (size_t)e->g;
                        double dalpha = 0;
                        for (int c = 0; c < 3; ++c) {
                            gr[6 + c] += e->alpha * e->T * gC[c];
                            dalpha += gC[c] * e->T * (g[6 + c] - S[c]);
                        }
                        dalpha += -Tfin / (1.0 - e->alpha) * bgdot;
                        for (int c = 0; c < 3; ++c)
                            S[c] = e->alpha * g[6 + c] + (1.0 - e->alpha) * S[c];
                        if (e->clamped) continue;
                        gr[5] += dalpha * e->G;
                        double dpow = dalpha * g[5] * e->G;
                        double dx = e->dx, dy = e->dy;
                        gr[2] += dpow * (-0.5 * dx * dx);
                        gr[3] += dpow * (-dx * dy);
                        gr[4] += dpow * (-0.5 * dy * dy);
                        gr[0] += dpow * (g[2] * dx + g[3] * dy);
                        gr[1] += dpow * (g[4] * dy + g[3] * dx);
                    }
                }
        }
    free(cs);
}
