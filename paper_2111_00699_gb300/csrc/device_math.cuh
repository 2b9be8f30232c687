// Device-side math for the MLS-MPM kernels: Morton codes, quadratic B-spline
// weights, the 3x3 SVD and the constitutive models (fixed-corotated, snow,
// fluid, Drucker-Prager sand, NACC snow, neo-Hookean sand).  FP32 throughout,
// compiled with fast-math intrinsics as the paper does (Sec. 4.3).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mpm {

// ---- Morton codes (Sec. 4: interleaved integer indices) --------------------
// Bit i of the x index goes to bit 3i, y to 3i+1, z to 3i+2 (10 bits/axis).
__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__host__ __device__ __forceinline__ uint32_t compact3(uint32_t v)
{
    v &= 0x09249249u;
    v = (v ^ (v >> 2)) & 0x030c30c3u;
    v = (v ^ (v >> 4)) & 0x0300f00fu;
    v = (v ^ (v >> 8)) & 0x030000ffu;
    v = (v ^ (v >> 16)) & 0x000003ffu;
    return v;
}

__host__ __device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z)
{
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// Base node and fraction along one axis: base = floor(x/dx - 1/2) (the
// particle block's -dx/2 shift of Sec. 4.2.1), f = x/dx - base in [0.5, 1.5).
// The product and the difference are rounded separately (no FMA) so the
// integer decision matches a plain FP32 evaluation.
__device__ __forceinline__ int base_of(float x, float inv_dx)
{
    return __float2int_rd(__fsub_rn(__fmul_rn(x, inv_dx), 0.5f));
}

// Quadratic B-spline weights at offsets f, f-1, f-2 (Sec. 3.1).
__device__ __forceinline__ void bspline(float f, float w[3])
{
    float a = 1.5f - f, b = f - 1.0f, c = f - 0.5f;
    w[0] = 0.5f * a * a;
    w[1] = 0.75f - b * b;
    w[2] = 0.5f * c * c;
}

// ---- stencil addressing and the G2P gather ------------------------------------
// Grid index of the 27 nodes of a stencil at base b, from the (up to) 8
// blocks stencil_blocks returned.  Node (i, j, k) lies in candidate block
// (dx, dy, dz) with dx = ((b_x & 3) + i) >> 2 and so on; the block is picked
// by one select per axis (z, then y, then x), so that after unrolling a row
// of 3 nodes costs 2 selects and each node 1 more.
struct StencilIndex {
    int pb64[8];   // candidate block slot * 64 (0 where unused)
    int bx, by, bz;

    __device__ __forceinline__ int operator()(int i, int j, int k) const
    {
        const int nx = bx + i, ny = by + j, nz = bz + k;
        const bool dz = nz >= 4, dy = ny >= 4, dx = nx >= 4;
        const int q0 = dz ? pb64[4] : pb64[0], q1 = dz ? pb64[5] : pb64[1];
        const int q2 = dz ? pb64[6] : pb64[2], q3 = dz ? pb64[7] : pb64[3];
        const int r0 = dy ? q2 : q0, r1 = dy ? q3 : q1;
        return (dx ? r1 : r0) + (nx & 3) + 4 * (ny & 3) + 16 * (nz & 3);
    }
};

// vp = sum w v_i, Bm = sum w v_i (node - f)^T over the 27 stencil nodes,
// node velocities given by vel(i, j, k) -> float3.  With centred offsets
// e = (i, j, k) - 1 in {-1, 0, 1}, sum w v (node - f)^T = sum w v e^T - vp (f - 1)^T,
// and both weighted sums factor axis by axis: each row of 3 nodes along x is
// reduced first (its sum and its e_x moment), then the rows along y, then z.
template <class Vel>
__device__ __forceinline__ void g2p_accumulate(const float* f, const float (*w)[3], Vel vel, float* vp, float* Bm)
{
    float M[3][3];   // M[a][d] = sum w v_a e_d
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        vp[a] = 0.0f;
        M[a][0] = M[a][1] = M[a][2] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float s[3] = {0.f, 0.f, 0.f}, sx[3] = {0.f, 0.f, 0.f}, sy[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float3 g0 = vel(0, j, k), g1 = vel(1, j, k), g2 = vel(2, j, k);
            const float a0[3] = {w[0][0] * g0.x, w[0][0] * g0.y, w[0][0] * g0.z};
            const float a2[3] = {w[0][2] * g2.x, w[0][2] * g2.y, w[0][2] * g2.z};
            const float g1v[3] = {g1.x, g1.y, g1.z};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float r = a0[a] + w[0][1] * g1v[a] + a2[a];   // row sum
                const float rx = a2[a] - a0[a];                       // row e_x moment
                s[a] += w[1][j] * r;
                sx[a] += w[1][j] * rx;
                if (j == 0) sy[a] -= w[1][0] * r;
                if (j == 2) sy[a] += w[1][2] * r;
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            vp[a] += w[2][k] * s[a];
            M[a][0] += w[2][k] * sx[a];
            M[a][1] += w[2][k] * sy[a];
            if (k == 0) M[a][2] -= w[2][0] * s[a];
            if (k == 2) M[a][2] += w[2][2] * s[a];
        }
    }
    const float fm[3] = {f[0] - 1.0f, f[1] - 1.0f, f[2] - 1.0f};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d)
            Bm[3 * a + d] = M[a][d] - vp[a] * fm[d];
}

// ---- 3x3 SVD helpers -------------------------------------------------------------
// The SVD (svd_h below) diagonalises the symmetric F^T F - I by cyclic Jacobi
// rotations with exact angles (V and the singular values), as in McAdams et
// al. 2011, then orthonormalises the columns of F V (U).

// 1/sqrt(x) to ~1 ulp: the fast-math rsqrt plus one Newton step.  The
// orthogonality of a rotation (c^2 + s^2 = 1 with s = t c) depends only on
// the accuracy of c = 1/sqrt(1 + t^2), and errors in it feed straight into
// sigma - 1, i.e. into the stress.
__device__ __forceinline__ float rsqrt_nr(float x)
{
    float y = rsqrtf(x);
    return y * (1.5f - 0.5f * x * y * y);
}

__device__ __forceinline__ void jacobi_pair(float& spp, float& sqq, float& spq, float& srp, float& srq,
                                            float* V, int p, int q)
{
    // An off-diagonal below FP32 resolution of the diagonal is already zero to
    // working precision; rotating it away (by up to 45 degrees when the
    // diagonal is degenerate, as for F = I) would only add rounding.
    float mag = fabsf(spp) + fabsf(sqq);
    if (!(fabsf(spq) > 6e-8f * mag + 1e-35f))
        return;
    float theta = (sqq - spp) / (2.0f * spq);
    float at = fabsf(theta);
    float t = at > 1e15f ? 0.5f / theta : copysignf(1.0f, theta) / (at + sqrtf(theta * theta + 1.0f));
    float c = rsqrt_nr(t * t + 1.0f);
    float s = t * c;
    spp -= t * spq;
    sqq += t * spq;
    spq = 0.0f;
    float a = srp, b = srq;
    srp = c * a - s * b;
    srq = s * a + c * b;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float vp = V[3 * r + p], vq = V[3 * r + q];
        V[3 * r + p] = c * vp - s * vq;
        V[3 * r + q] = s * vp + c * vq;
    }
}

__device__ __forceinline__ void swap_neg_cols(float* V, float& la, float& lb, int a, int b)
{
    float t = la;
    la = lb;
    lb = t;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float va = V[3 * r + a];
        V[3 * r + a] = V[3 * r + b];
        V[3 * r + b] = -va;   // keep det V = +1
    }
}

__device__ __forceinline__ float det3(const float* M)
{
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// ---- constitutive models (Sec. 4.1: SVD, projection and stress merged) --------
// The deformation gradient is held as H = F - I, the displacement gradient,
// and the snow/fluid volume ratios as Jp - 1 and J - 1: near the rest shape
// F is I plus a strain of 1e-3 or less, which an FP32 F resolves to ~1e-4
// relative (an FP32 SVD of F then returns sigma - 1 with ~1e-7 absolute
// error, i.e. 1e-4 relative stress error).  All quantities below that are
// small near the rest shape are computed from small quantities only.

// prod(1 + a_i) - 1, without forming the products near 1.
__device__ __forceinline__ float prod_m1(const float* a)
{
    return a[0] + a[1] + a[2] + a[0] * a[1] + a[0] * a[2] + a[1] * a[2] + a[0] * a[1] * a[2];
}

// det(I + H) - 1 = tr H + ((tr H)^2 - tr(H^2)) / 2 + det H.
__device__ __forceinline__ float det_m1(const float* H)
{
    float tr = H[0] + H[4] + H[8];
    float trHH = H[0] * H[0] + H[4] * H[4] + H[8] * H[8] + 2.0f * (H[1] * H[3] + H[2] * H[6] + H[5] * H[7]);
    return tr + 0.5f * (tr * tr - trHH) + det3(H);
}

// Rotation-variant SVD of F = I + H: F = U diag(s) V^T, det U = det V = +1,
// s sorted descending with only s[2] possibly negative (inverted F), and
// sm1 = s - 1 to full relative precision.  V and the s come from Jacobi
// rotations of the small symmetric E = F^T F - I = H + H^T + H^T H, with
// s_i - 1 = l_i / (sqrt(1 + l_i) + 1) for its eigenvalues l_i.
struct SVDH {
    float U[9], V[9], s[3], sm1[3];
    float Jm1;      // det F - 1
    bool inverted;  // det F < 0 (s[2] negated, U's last column flipped)
};

__device__ __forceinline__ void svd_h(const float* H, SVDH& d)
{
    float e00 = 2.f * H[0] + H[0] * H[0] + H[3] * H[3] + H[6] * H[6];
    float e11 = 2.f * H[4] + H[1] * H[1] + H[4] * H[4] + H[7] * H[7];
    float e22 = 2.f * H[8] + H[2] * H[2] + H[5] * H[5] + H[8] * H[8];
    float e01 = H[1] + H[3] + H[0] * H[1] + H[3] * H[4] + H[6] * H[7];
    float e02 = H[2] + H[6] + H[0] * H[2] + H[3] * H[5] + H[6] * H[8];
    float e12 = H[5] + H[7] + H[1] * H[2] + H[4] * H[5] + H[7] * H[8];
#pragma unroll
    for (int i = 0; i < 9; ++i)
        d.V[i] = (i % 4 == 0) ? 1.0f : 0.0f;
#pragma unroll
    for (int sweep = 0; sweep < 3; ++sweep) {
        jacobi_pair(e00, e11, e01, e02, e12, d.V, 0, 1);
        jacobi_pair(e00, e22, e02, e01, e12, d.V, 0, 2);
        jacobi_pair(e11, e22, e12, e01, e02, d.V, 1, 2);
    }
    if (e00 < e11) swap_neg_cols(d.V, e00, e11, 0, 1);
    if (e00 < e22) swap_neg_cols(d.V, e00, e22, 0, 2);
    if (e11 < e22) swap_neg_cols(d.V, e11, e22, 1, 2);
    const float l[3] = {e00, e11, e22};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float r = sqrtf(fmaxf(1.0f + l[i], 0.0f));
        d.sm1[i] = l[i] / (r + 1.0f);
        d.s[i] = 1.0f + d.sm1[i];
    }
    // U by Gram-Schmidt on the columns b_c = (I + H) v_c, closed by a cross
    // product so that det U = +1 even when F is singular or inverted.
    float b[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c)
            b[3 * r + c] = d.V[3 * r + c] + H[3 * r] * d.V[c] + H[3 * r + 1] * d.V[3 + c] + H[3 * r + 2] * d.V[6 + c];
    float n0 = b[0] * b[0] + b[3] * b[3] + b[6] * b[6];
    float u0[3], u1[3];
    if (n0 > 1e-30f) {
        float in0 = rsqrt_nr(n0);
        u0[0] = b[0] * in0; u0[1] = b[3] * in0; u0[2] = b[6] * in0;
    } else {
        u0[0] = 1.0f; u0[1] = 0.0f; u0[2] = 0.0f;
    }
    float pr = u0[0] * b[1] + u0[1] * b[4] + u0[2] * b[7];
    float w[3] = {b[1] - pr * u0[0], b[4] - pr * u0[1], b[7] - pr * u0[2]};
    float n1 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const float s1_qr = sqrtf(n1);
    if (!(n1 > 1e-12f * n0 + 1e-30f)) {
        // rank <= 1: any unit vector orthogonal to u0
        // u0 x e_k for the axis k along which u0 is smallest
        float ax = fabsf(u0[0]), ay = fabsf(u0[1]), az = fabsf(u0[2]);
        if (ax <= ay && ax <= az) {
            w[0] = 0.0f; w[1] = u0[2]; w[2] = -u0[1];
        } else if (ay <= az) {
            w[0] = -u0[2]; w[1] = 0.0f; w[2] = u0[0];
        } else {
            w[0] = u0[1]; w[1] = -u0[0]; w[2] = 0.0f;
        }
        n1 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    }
    float in1 = rsqrt_nr(n1);
    u1[0] = w[0] * in1; u1[1] = w[1] * in1; u1[2] = w[2] * in1;
    d.U[0] = u0[0]; d.U[3] = u0[1]; d.U[6] = u0[2];
    d.U[1] = u1[0]; d.U[4] = u1[1]; d.U[7] = u1[2];
    d.U[2] = u0[1] * u1[2] - u0[2] * u1[1];
    d.U[5] = u0[2] * u1[0] - u0[0] * u1[2];
    d.U[8] = u0[0] * u1[1] - u0[1] * u1[0];
    d.Jm1 = det_m1(H);
    // A singular value far below 1 is ill-determined by the eigenvalue
    // 1 + l = s^2 of F^T F; there the projections of F V on U (the diagonal
    // of the QR factor of F V) give it to FP32 absolute accuracy instead.
    if (l[1] < -0.75f) {
        d.s[1] = s1_qr;
        d.sm1[1] = d.s[1] - 1.0f;
    }
    if (l[2] < -0.75f) {
        float b2[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            b2[r] = d.V[3 * r + 2] + H[3 * r] * d.V[2] + H[3 * r + 1] * d.V[5] + H[3 * r + 2] * d.V[8];
        d.s[2] = d.U[2] * b2[0] + d.U[5] * b2[1] + d.U[8] * b2[2];   // signed: det U = det V = +1
        d.sm1[2] = d.s[2] - 1.0f;
        d.inverted = d.s[2] < 0.0f;
    } else {
        d.inverted = d.Jm1 < -1.0f;
        if (d.inverted) {
            d.s[2] = -d.s[2];
            d.sm1[2] = d.s[2] - 1.0f;
        }
    }
}

// tau = U diag(dg) U^T + vol I, as (xx, yy, zz, xy, xz, yz).
__device__ __forceinline__ void tau6(const float* U, const float* dg, float vol, float* t6)
{
    t6[0] = U[0] * U[0] * dg[0] + U[1] * U[1] * dg[1] + U[2] * U[2] * dg[2] + vol;
    t6[1] = U[3] * U[3] * dg[0] + U[4] * U[4] * dg[1] + U[5] * U[5] * dg[2] + vol;
    t6[2] = U[6] * U[6] * dg[0] + U[7] * U[7] * dg[1] + U[8] * U[8] * dg[2] + vol;
    t6[3] = U[0] * U[3] * dg[0] + U[1] * U[4] * dg[1] + U[2] * U[5] * dg[2];
    t6[4] = U[0] * U[6] * dg[0] + U[1] * U[7] * dg[1] + U[2] * U[8] * dg[2];
    t6[5] = U[3] * U[6] * dg[0] + U[4] * U[7] * dg[1] + U[5] * U[8] * dg[2];
}

// H of F' = U diag(1 + t) V^T, written as U diag(t) V^T + (R - I) with
// R - I = (H V - V diag(s - 1)) diag(1/s) V^T (the rotation of the polar
// decomposition), so that H' keeps its precision near the rest shape.
__device__ __forceinline__ void rebuild_h(const SVDH& d, const float* H, const float* t, float* Hout)
{
    if (d.inverted || d.s[2] < 0.25f) {
        // far from the rest shape: F' - I directly
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Hout[3 * r + c] = d.U[3 * r] * (1.0f + t[0]) * d.V[3 * c] + d.U[3 * r + 1] * (1.0f + t[1]) * d.V[3 * c + 1] +
                                  d.U[3 * r + 2] * (1.0f + t[2]) * d.V[3 * c + 2] - (r == c ? 1.0f : 0.0f);
        return;
    }
    float Wm[9];   // (H V - V diag(s - 1)) diag(1/s), so that R - I = Wm V^T
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float hv = H[3 * r] * d.V[k] + H[3 * r + 1] * d.V[3 + k] + H[3 * r + 2] * d.V[6 + k];
            Wm[3 * r + k] = (hv - d.V[3 * r + k] * d.sm1[k]) / d.s[k];
        }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                acc += (d.U[3 * r + k] * t[k] + Wm[3 * r + k]) * d.V[3 * c + k];
            Hout[3 * r + c] = acc;
        }
}

// Fluid pressure term: tau = -p J I, p = K (J^-gamma - 1), from jm1 = J - 1.
__device__ __forceinline__ void fluid_tau6(const MatParams& m, float jm1, float* t6)
{
    float Jg_m1 = expm1f(-m.gamma * log1pf(jm1));   // J^-gamma - 1
    float pj = m.K * Jg_m1 * (1.0f + jm1);
    t6[0] = t6[1] = t6[2] = -pj;
    t6[3] = t6[4] = t6[5] = 0.0f;
}

// Hencky strain of a singular value (floored at 1e-4 for collapsed or
// inverted directions).
__device__ __forceinline__ float hencky(float s, float sm1)
{
    return s > 1e-4f ? log1pf(sm1) : logf(1e-4f);
}

// ---- small-strain path without an SVD ----------------------------------------
// Near the rest shape every quantity the models need is an isotropic function
// of the left Cauchy-Green tensor B = F F^T = I + G, G = H + H^T + H H^T, and
// so a power series in G (all such series commute with G and with each other):
//   fixed-corotated:  (F - R) F^T = B - sqrt(B)
//                     = G/2 + G^2/8 - G^3/16 + 5 G^4/128 - 7 G^5/256 + ...
//   Hencky strain:    eps = ln(B)/2 = (G - G^2/2 + G^3/3 - G^4/4 + G^5/5 - G^6/6 + ...)/2
//   Drucker-Prager:   F' = exp(-X) F (X = eps for case II, the radial return
//                     of case III for case III), exp(-X) - I by its series.
// With |G|_F <= 0.1 the first omitted terms are below 1e-6 of the leading
// one.  Snow takes this path only when no singular value reaches the clamp
// (G - lo I and hi I - G both positive definite), and no model takes it for
// an inverted F.  Everything else goes through the SVD below.

struct Sym {   // symmetric 3x3
    float xx, yy, zz, xy, xz, yz;
};

// A B for commuting symmetric A, B (then A B is symmetric).
__device__ __forceinline__ Sym sym_mul(const Sym& a, const Sym& b)
{
    Sym r;
    r.xx = a.xx * b.xx + a.xy * b.xy + a.xz * b.xz;
    r.yy = a.xy * b.xy + a.yy * b.yy + a.yz * b.yz;
    r.zz = a.xz * b.xz + a.yz * b.yz + a.zz * b.zz;
    r.xy = a.xx * b.xy + a.xy * b.yy + a.xz * b.yz;
    r.xz = a.xx * b.xz + a.xy * b.yz + a.xz * b.zz;
    r.yz = a.xy * b.xz + a.yy * b.yz + a.yz * b.zz;
    return r;
}

__device__ __forceinline__ Sym sym_scale(const Sym& a, float c)
{
    return {a.xx * c, a.yy * c, a.zz * c, a.xy * c, a.xz * c, a.yz * c};
}

__device__ __forceinline__ Sym sym_add_diag(const Sym& a, float c)
{
    return {a.xx + c, a.yy + c, a.zz + c, a.xy, a.xz, a.yz};
}

// sum_{k=1..N} c[k-1] G^k by Horner.
template <int N>
__device__ __forceinline__ Sym sym_series(const Sym& g, const float (&c)[N])
{
    Sym q = sym_add_diag(sym_scale(g, c[N - 1]), c[N - 2]);
#pragma unroll
    for (int k = N - 3; k >= 0; --k)
        q = sym_add_diag(sym_mul(g, q), c[k]);
    return sym_mul(g, q);
}

__device__ __forceinline__ float sym_frob2(const Sym& a)
{
    return a.xx * a.xx + a.yy * a.yy + a.zz * a.zz + 2.0f * (a.xy * a.xy + a.xz * a.xz + a.yz * a.yz);
}

__device__ __forceinline__ float sym_trace(const Sym& a) { return a.xx + a.yy + a.zz; }

// a positive definite (leading principal minors)
__device__ __forceinline__ bool sym_pd(const Sym& a)
{
    float m2 = a.xx * a.yy - a.xy * a.xy;
    float m3 = a.xx * (a.yy * a.zz - a.yz * a.yz) - a.xy * (a.xy * a.zz - a.yz * a.xz) +
               a.xz * (a.xy * a.yz - a.yy * a.xz);
    return a.xx > 0.0f && m2 > 0.0f && m3 > 0.0f;
}

// G = F F^T - I = H + H^T + H H^T
__device__ __forceinline__ Sym left_cg_m1(const float* H)
{
    Sym g;
    g.xx = 2.f * H[0] + H[0] * H[0] + H[1] * H[1] + H[2] * H[2];
    g.yy = 2.f * H[4] + H[3] * H[3] + H[4] * H[4] + H[5] * H[5];
    g.zz = 2.f * H[8] + H[6] * H[6] + H[7] * H[7] + H[8] * H[8];
    g.xy = H[1] + H[3] + H[0] * H[3] + H[1] * H[4] + H[2] * H[5];
    g.xz = H[2] + H[6] + H[0] * H[6] + H[1] * H[7] + H[2] * H[8];
    g.yz = H[5] + H[7] + H[3] * H[6] + H[4] * H[7] + H[5] * H[8];
    return g;
}

constexpr float kSeriesMaxG2 = 0.01f;   // |G|_F^2 bound of the series path

__device__ __forceinline__ void sym_to_t6(const Sym& a, float* t6)
{
    t6[0] = a.xx; t6[1] = a.yy; t6[2] = a.zz; t6[3] = a.xy; t6[4] = a.xz; t6[5] = a.yz;
}

// fixed-corotated: tau = 2 mu (B - sqrt B) + lambda J (J - 1) I
__device__ __forceinline__ void fc_tau_series(const Sym& g, float mu, float la, float Jm1, float* t6)
{
    const float c[5] = {0.5f, 0.125f, -0.0625f, 0.0390625f, -0.02734375f};
    Sym t = sym_add_diag(sym_scale(sym_series(g, c), 2.0f * mu), la * (1.0f + Jm1) * Jm1);
    sym_to_t6(t, t6);
}

// Hencky strain eps = ln(I + G) / 2
__device__ __forceinline__ Sym hencky_series(const Sym& g)
{
    const float c[6] = {0.5f, -0.25f, 1.0f / 6.0f, -0.125f, 0.1f, -1.0f / 12.0f};
    return sym_series(g, c);
}

// H <- H + (exp(-X) - I)(I + H), i.e. F <- exp(-X) F
__device__ __forceinline__ void left_exp_update(const Sym& x, float* H)
{
    const float c[5] = {-1.0f, 0.5f, -1.0f / 6.0f, 1.0f / 24.0f, -1.0f / 120.0f};
    const Sym e = sym_series(x, c);
    const float E[9] = {e.xx, e.xy, e.xz, e.xy, e.yy, e.yz, e.xz, e.yz, e.zz};
    float Hn[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c2 = 0; c2 < 3; ++c2)
            Hn[3 * r + c2] = H[3 * r + c2] + E[3 * r + c2] + E[3 * r] * H[c2] + E[3 * r + 1] * H[3 + c2] +
                             E[3 * r + 2] * H[6 + c2];
#pragma unroll
    for (int q = 0; q < 9; ++q)
        H[q] = Hn[q];
}

// The series path of constitutive_update / stress_h; false if the state is
// outside its range (the caller then takes the SVD path).  With
// `project` the return maps run (snow: none needed on this path; sand:
// cases II and III update H).
// NACC return map on the Hencky strain, given its trace tr and the norm nd
// of its deviator: with p = -kappa tr and q = sqrt(3/2) 2 mu nd, a state
// outside the ellipse (1 + 2 beta) q^2 + M^2 (p + beta p0)(p - p0) <= 0,
// p0 = kappa sinh(xi max(-alpha, 0)), alpha = alpha0 + ln Jp, keeps p and
// takes the q on the ellipse, or moves to a tip beyond p0 or -beta p0.
// Returns false if the state is inside; else the new trace trn and the
// factor s on the deviator.
__device__ __forceinline__ bool nacc_return(const MatParams& m, float jm1, float tr, float nd, float& trn, float& s)
{
    const float kappa = m.K;
    const float p = -kappa * tr;
    const float q = 1.22474487f * 2.0f * m.mu * nd;   // sqrt(3/2) |dev tau|
    const float alpha = m.alpha0 + log1pf(jm1);
    const float p0 = kappa * sinhf(m.xi * fmaxf(-alpha, 0.0f));
    float pn = p, qn = q;
    if (p > p0) {
        pn = p0;
        qn = 0.0f;
    } else if (p < -m.beta * p0) {
        pn = -m.beta * p0;
        qn = 0.0f;
    } else {
        const float y = (1.0f + 2.0f * m.beta) * q * q + m.M2 * (p + m.beta * p0) * (p - p0);
        if (!(y > 0.0f))
            return false;
        qn = sqrtf(m.M2 * (p + m.beta * p0) * (p0 - p) / (1.0f + 2.0f * m.beta));
    }
    trn = -pn / kappa;
    s = q > 0.0f ? qn / q : 0.0f;
    return true;
}

__device__ __forceinline__ bool small_strain_update(const MatParams& m, float* H, float& jm1, bool project, float* t6)
{
    const Sym g = left_cg_m1(H);
    const float Jm1 = det_m1(H);
    if (!(sym_frob2(g) <= kSeriesMaxG2) || !(Jm1 > -1.0f))
        return false;
    if (m.kind == MPM_SNOW) {
        // elastic only if every sigma^2 - 1 (eigenvalue of G) lies strictly inside the clamp
        if (!sym_pd(sym_add_diag(g, -m.lo_b)) || !sym_pd(sym_add_diag(sym_scale(g, -1.0f), m.hi_b)))
            return false;
        const float h = __expf(-m.xi * jm1);
        fc_tau_series(g, m.mu * h, m.la * h, Jm1, t6);
        return true;
    }
    if (m.kind == MPM_ELASTIC) {
        fc_tau_series(g, m.mu, m.la, Jm1, t6);
        return true;
    }
    // sand and NACC: Hencky strain in the current (left) frame
    Sym eps = hencky_series(g);
    const float tr = sym_trace(eps);
    if (project && m.kind == MPM_NACC) {
        const Sym dev = sym_add_diag(eps, -tr * (1.0f / 3.0f));
        float trn, sc;
        if (nacc_return(m, jm1, tr, sqrtf(sym_frob2(dev)), trn, sc)) {
            // eps <- trn/3 I + sc dev, F <- exp(eps_new - eps) F, Jp <- Jp exp(tr - trn)
            const Sym en = sym_add_diag(sym_scale(dev, sc), trn * (1.0f / 3.0f));
            const Sym x = {eps.xx - en.xx, eps.yy - en.yy, eps.zz - en.zz, eps.xy - en.xy, eps.xz - en.xz,
                           eps.yz - en.yz};
            left_exp_update(x, H);
            const float r = expm1f(tr - trn);
            jm1 = jm1 * (1.0f + r) + r;
            eps = en;
        }
        const Sym t = sym_add_diag(sym_scale(eps, 2.0f * m.mu), m.la * sym_trace(eps));
        sym_to_t6(t, t6);
        return true;
    }
    bool moved = false;
    if (project) {
        if (tr >= 0.0f) {
            // case II: project to the cone tip, F <- R = exp(-eps) F, tau = 0
            left_exp_update(eps, H);
            t6[0] = t6[1] = t6[2] = t6[3] = t6[4] = t6[5] = 0.0f;
            return true;
        }
        const Sym dev = sym_add_diag(eps, -tr * (1.0f / 3.0f));
        const float nd = sqrtf(sym_frob2(dev));
        const float dgm = nd + m.dp_coef * tr * m.alpha;
        if (dgm > 0.0f) {
            // case III: eps <- eps - dgm dev / |dev|, F <- exp(-X) F with X = dgm dev / |dev|
            const Sym x = sym_scale(dev, dgm / nd);
            left_exp_update(x, H);
            eps = {eps.xx - x.xx, eps.yy - x.yy, eps.zz - x.zz, -x.xy + eps.xy, eps.xz - x.xz, eps.yz - x.yz};
            moved = true;
        }
    }
    if (m.kind == MPM_NHSAND) {
        // neo-Hookean: tau = mu (B - I) + lambda ln J I; the projection keeps tr eps = ln J
        const Sym gb = moved ? left_cg_m1(H) : g;
        sym_to_t6(sym_add_diag(sym_scale(gb, m.mu), m.la * tr), t6);
        return true;
    }
    const Sym t = sym_add_diag(sym_scale(eps, 2.0f * m.mu), m.la * tr);
    sym_to_t6(t, t6);
    return true;
}

// Kirchhoff stress of a stored state (no return map): used when the stress
// channels must be rebuilt from (H, Jp - 1), e.g. after mpm_write_state.
//   fixed-corotated: tau = U diag(2 mu (s - 1) s) U^T + lambda J (J - 1) I,
//     mu, lambda scaled by exp(xi (1 - Jp)) for snow [Stomakhin 2013];
//   sand: tau = U diag(2 mu e + lambda tr e) U^T, e = ln s [Klar 2016];
//   neo-Hookean sand: tau = U diag(mu (s^2 - 1) + lambda ln J) U^T [Yue 2018];
//   fluid: tau = -p J I, p = K (J^-gamma - 1) [Tampubolon 2017].
__device__ __forceinline__ void stress_h(const MatParams& m, const float* H, float jm1, float* t6)
{
    if (m.kind == MPM_FLUID) {
        fluid_tau6(m, jm1, t6);
        return;
    }
    {
        float Hc[9];
#pragma unroll
        for (int q = 0; q < 9; ++q)
            Hc[q] = H[q];
        float jc = jm1;
        if (small_strain_update(m, Hc, jc, false, t6))
            return;
    }
    SVDH d;
    svd_h(H, d);
    float dg[3];
    if (m.kind == MPM_SAND || m.kind == MPM_NACC || m.kind == MPM_NHSAND) {
        float e[3] = {hencky(d.s[0], d.sm1[0]), hencky(d.s[1], d.sm1[1]), hencky(d.s[2], d.sm1[2])};
        float tr = e[0] + e[1] + e[2];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dg[k] = m.kind == MPM_NHSAND ? m.mu * d.sm1[k] * (d.s[k] + 1.0f) + m.la * tr
                                         : 2.0f * m.mu * e[k] + m.la * tr;
        tau6(d.U, dg, 0.0f, t6);
        return;
    }
    float mu = m.mu, la = m.la;
    if (m.kind == MPM_SNOW) {
        float h = __expf(-m.xi * jm1);
        mu *= h;
        la *= h;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        dg[k] = 2.0f * mu * d.sm1[k] * d.s[k];
    tau6(d.U, dg, la * (1.0f + d.Jm1) * d.Jm1, t6);
}

// End-of-G2P constitutive update with one SVD (Sec. 4.1 merges "SVD,
// plasticity projection, stress computation"): the return map on the trial
// state H (snow singular-value clamp with the Jp update [Stomakhin 2013];
// Drucker-Prager cases I-III [Klar 2016]), then the stress of the projected
// state for the next P2G.  jm1 is Jp - 1 (snow) or J - 1 (fluid, already
// advanced by the caller).
__device__ __forceinline__ void constitutive_update(const MatParams& m, float* H, float& jm1, float* t6)
{
    if (m.kind == MPM_FLUID) {
        fluid_tau6(m, jm1, t6);
        return;
    }
    if (small_strain_update(m, H, jm1, true, t6))
        return;
    SVDH d;
    svd_h(H, d);
    float dg[3];
    if (m.kind == MPM_SNOW) {
        float t[3];
        bool changed = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            t[k] = fminf(fmaxf(d.sm1[k], m.lo_m1), m.hi_m1);
            changed = changed || t[k] != d.sm1[k];
        }
        if (changed) {
            float P = prod_m1(d.sm1), Ph = prod_m1(t);
            float r_m1 = (P - Ph) / (1.0f + Ph);           // det(F)/det(F_clamped) - 1
            jm1 = jm1 * (1.0f + r_m1) + r_m1;              // Jp <- Jp det(F) / det(F_clamped)
            float Hn[9];
            rebuild_h(d, H, t, Hn);
#pragma unroll
            for (int e = 0; e < 9; ++e)
                H[e] = Hn[e];
        }
        float h = __expf(-m.xi * jm1);
        float mu = m.mu * h, la = m.la * h;
        float Jm1 = changed ? prod_m1(t) : d.Jm1;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dg[k] = 2.0f * mu * t[k] * (1.0f + t[k]);
        tau6(d.U, dg, la * (1.0f + Jm1) * Jm1, t6);
        return;
    }
    if (m.kind == MPM_NACC) {
        float e[3] = {hencky(d.s[0], d.sm1[0]), hencky(d.s[1], d.sm1[1]), hencky(d.s[2], d.sm1[2])};
        const float tr = e[0] + e[1] + e[2];
        const float dv[3] = {e[0] - tr * (1.0f / 3.0f), e[1] - tr * (1.0f / 3.0f), e[2] - tr * (1.0f / 3.0f)};
        float trn, sc;
        if (nacc_return(m, jm1, tr, sqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]), trn, sc)) {
            float t[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                e[k] = trn * (1.0f / 3.0f) + sc * dv[k];
                t[k] = expm1f(e[k]);
            }
            float Hn[9];
            rebuild_h(d, H, t, Hn);
#pragma unroll
            for (int q = 0; q < 9; ++q)
                H[q] = Hn[q];
            const float r = expm1f(tr - trn);
            jm1 = jm1 * (1.0f + r) + r;
        }
        const float tr2 = e[0] + e[1] + e[2];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dg[k] = 2.0f * m.mu * e[k] + m.la * tr2;
        tau6(d.U, dg, 0.0f, t6);
        return;
    }
    if (m.kind == MPM_SAND || m.kind == MPM_NHSAND) {
        float e[3] = {hencky(d.s[0], d.sm1[0]), hencky(d.s[1], d.sm1[1]), hencky(d.s[2], d.sm1[2])};
        float tr = e[0] + e[1] + e[2];
        if (tr >= 0.0f) {
            // case II: expansion, project to the cone tip (sigma = 1)
            const float zero[3] = {0.0f, 0.0f, 0.0f};
            float Hn[9];
            rebuild_h(d, H, zero, Hn);
#pragma unroll
            for (int q = 0; q < 9; ++q)
                H[q] = Hn[q];
            e[0] = e[1] = e[2] = 0.0f;
        } else {
            float third = tr * (1.0f / 3.0f);
            float d0 = e[0] - third, d1 = e[1] - third, d2 = e[2] - third;
            float nd = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            float dgm = nd + m.dp_coef * tr * m.alpha;
            if (dgm > 0.0f) {
                // case III: radial return onto the cone surface
                float k = dgm / nd;
                e[0] -= k * d0;
                e[1] -= k * d1;
                e[2] -= k * d2;
                float t[3] = {expm1f(e[0]), expm1f(e[1]), expm1f(e[2])};
                float Hn[9];
                rebuild_h(d, H, t, Hn);
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    H[q] = Hn[q];
            }
        }
        float tr2 = e[0] + e[1] + e[2];
#pragma unroll
        for (int k = 0; k < 3; ++k)   // neo-Hookean: s^2 - 1 = expm1(2 e)
            dg[k] = m.kind == MPM_NHSAND ? m.mu * expm1f(2.0f * e[k]) + m.la * tr2 : 2.0f * m.mu * e[k] + m.la * tr2;
        tau6(d.U, dg, 0.0f, t6);
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        dg[k] = 2.0f * m.mu * d.sm1[k] * d.s[k];
    tau6(d.U, dg, m.la * (1.0f + d.Jm1) * d.Jm1, t6);
}

}  // namespace mpm
