// Device-side math for the MLS-MPM kernels: Morton codes, quadratic B-spline
// weights, the 3x3 SVD and the four constitutive models.  FP32 throughout,
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

// ---- 3x3 SVD -----------------------------------------------------------------
// Eigen-decomposition of the symmetric F^T F by cyclic Jacobi rotations
// (V), then a Givens QR of F V, whose triangular factor is diagonal up to
// rounding (U, sigma); the approach of McAdams et al. 2011, written with
// exact Jacobi angles.  Result: F = U diag(sig) V^T, det U = det V = +1,
// sig[0] >= sig[1] >= |sig[2]|, sig[2] < 0 for inverted F.

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

__device__ __forceinline__ void givens_rows(float* B, float* U, int i, int j)
{
    float a = B[3 * i + i], b = B[3 * j + i];
    if (!(fabsf(b) > 6e-8f * fabsf(a))) {
        // b is zero to working precision: the rotation is the identity, or a
        // half turn (exact sign flips of rows i, j) when the pivot is negative.
        if (a < 0.0f) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                B[3 * i + k] = -B[3 * i + k];
                B[3 * j + k] = -B[3 * j + k];
                U[3 * k + i] = -U[3 * k + i];
                U[3 * k + j] = -U[3 * k + j];
            }
        }
        return;
    }
    float r2 = a * a + b * b;
    float ir = rsqrt_nr(r2);
    float c = a * ir, s = b * ir;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float bi = B[3 * i + k], bj = B[3 * j + k];
        B[3 * i + k] = c * bi + s * bj;
        B[3 * j + k] = -s * bi + c * bj;
        float ui = U[3 * k + i], uj = U[3 * k + j];
        U[3 * k + i] = c * ui + s * uj;
        U[3 * k + j] = -s * ui + c * uj;
    }
}

__device__ __forceinline__ void svd3(const float* F, float* U, float* sig, float* V)
{
    // S = F^T F
    float s00 = F[0] * F[0] + F[3] * F[3] + F[6] * F[6];
    float s01 = F[0] * F[1] + F[3] * F[4] + F[6] * F[7];
    float s02 = F[0] * F[2] + F[3] * F[5] + F[6] * F[8];
    float s11 = F[1] * F[1] + F[4] * F[4] + F[7] * F[7];
    float s12 = F[1] * F[2] + F[4] * F[5] + F[7] * F[8];
    float s22 = F[2] * F[2] + F[5] * F[5] + F[8] * F[8];
#pragma unroll
    for (int i = 0; i < 9; ++i)
        V[i] = (i % 4 == 0) ? 1.0f : 0.0f;
#pragma unroll
    for (int sweep = 0; sweep < 5; ++sweep) {
        jacobi_pair(s00, s11, s01, s02, s12, V, 0, 1);
        jacobi_pair(s00, s22, s02, s01, s12, V, 0, 2);
        jacobi_pair(s11, s22, s12, s01, s02, V, 1, 2);
    }
    // order eigenvalues descending
    if (s00 < s11) swap_neg_cols(V, s00, s11, 0, 1);
    if (s00 < s22) swap_neg_cols(V, s00, s22, 0, 2);
    if (s11 < s22) swap_neg_cols(V, s11, s22, 1, 2);
    // B = F V, then B = U R by Givens rotations
    float B[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            B[3 * r + c] = F[3 * r] * V[c] + F[3 * r + 1] * V[3 + c] + F[3 * r + 2] * V[6 + c];
#pragma unroll
    for (int i = 0; i < 9; ++i)
        U[i] = (i % 4 == 0) ? 1.0f : 0.0f;
    givens_rows(B, U, 0, 1);
    givens_rows(B, U, 0, 2);
    givens_rows(B, U, 1, 2);
    sig[0] = B[0];
    sig[1] = B[4];
    sig[2] = B[8];
}

__device__ __forceinline__ float det3(const float* M)
{
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// out = U diag(d) W^T
__device__ __forceinline__ void udwt(const float* U, const float* d, const float* W, float* out)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            out[3 * i + j] = U[3 * i] * d[0] * W[3 * j] + U[3 * i + 1] * d[1] * W[3 * j + 1] +
                             U[3 * i + 2] * d[2] * W[3 * j + 2];
}

// ---- constitutive models (Sec. 4.1: SVD, projection and stress merged) --------
// Kirchhoff stress tau = P F^T.  Fixed-corotated, written through the SVD:
// (F - R) F^T = U (Sigma - I) Sigma U^T, so tau = U diag(2 mu (s - 1) s) U^T
// + lambda J (J - 1) I.  Sand: tau = U diag(2 mu eps + lambda tr eps) U^T with
// eps = ln(max(s, 1e-4)).  Fluid: tau = -p J I, p = K (J^-gamma - 1).
__device__ __forceinline__ void kirchhoff(const MatParams& m, const float* F, float Jp, float* tau)
{
    if (m.kind == MPM_FLUID) {
        float J = Jp;
        float p = m.K * (__powf(J, -m.gamma) - 1.0f);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            tau[i] = 0.0f;
        tau[0] = tau[4] = tau[8] = -p * J;
        return;
    }
    float U[9], s[3], V[9], d[3];
    svd3(F, U, s, V);
    if (m.kind == MPM_SAND) {
        float e0 = __logf(fmaxf(s[0], 1e-4f)), e1 = __logf(fmaxf(s[1], 1e-4f)), e2 = __logf(fmaxf(s[2], 1e-4f));
        float tr = e0 + e1 + e2;
        d[0] = 2.0f * m.mu * e0 + m.la * tr;
        d[1] = 2.0f * m.mu * e1 + m.la * tr;
        d[2] = 2.0f * m.mu * e2 + m.la * tr;
        udwt(U, d, U, tau);
        return;
    }
    float mu = m.mu, la = m.la;
    if (m.kind == MPM_SNOW) {
        float h = __expf(m.xi * (1.0f - Jp));
        mu *= h;
        la *= h;
    }
    float J = s[0] * s[1] * s[2];
    d[0] = 2.0f * mu * (s[0] - 1.0f) * s[0];
    d[1] = 2.0f * mu * (s[1] - 1.0f) * s[1];
    d[2] = 2.0f * mu * (s[2] - 1.0f) * s[2];
    udwt(U, d, U, tau);
    float vol = la * J * (J - 1.0f);
    tau[0] += vol;
    tau[4] += vol;
    tau[8] += vol;
}

// Return mapping on the trial F at the end of G2P: snow singular-value clamp
// with the Jp update [Stomakhin 2013]; Drucker-Prager projection (cases I-III)
// [Klar 2016].  Elastic and fluid: nothing to do here.
__device__ __forceinline__ void plasticity(const MatParams& m, float* F, float& Jp)
{
    if (m.kind != MPM_SNOW && m.kind != MPM_SAND)
        return;
    float U[9], s[3], V[9], t[3];
    svd3(F, U, s, V);
    if (m.kind == MPM_SNOW) {
        t[0] = fminf(fmaxf(s[0], m.lo), m.hi);
        t[1] = fminf(fmaxf(s[1], m.lo), m.hi);
        t[2] = fminf(fmaxf(s[2], m.lo), m.hi);
        Jp *= (s[0] * s[1] * s[2]) / (t[0] * t[1] * t[2]);
        udwt(U, t, V, F);
        return;
    }
    float e0 = __logf(fmaxf(s[0], 1e-4f)), e1 = __logf(fmaxf(s[1], 1e-4f)), e2 = __logf(fmaxf(s[2], 1e-4f));
    float tr = e0 + e1 + e2;
    if (tr >= 0.0f) {
        t[0] = t[1] = t[2] = 1.0f;
        udwt(U, t, V, F);
        return;
    }
    float third = tr * (1.0f / 3.0f);
    float d0 = e0 - third, d1 = e1 - third, d2 = e2 - third;
    float nd = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    float dg = nd + m.dp_coef * tr * m.alpha;
    if (dg <= 0.0f)
        return;
    float k = dg / nd;
    t[0] = __expf(e0 - k * d0);
    t[1] = __expf(e1 - k * d1);
    t[2] = __expf(e2 - k * d2);
    udwt(U, t, V, F);
}

// End-of-G2P constitutive update with a single SVD (Sec. 4.1 merges "SVD,
// plasticity projection, stress computation"): the return map on the trial
// F (snow clamp + Jp, Drucker-Prager projection), then the Kirchhoff stress
// of the projected state, which the next P2G needs.  Output t6 = (xx, yy, zz,
// xy, xz, yz) of the symmetric tau = U diag(d) U^T + vol I.
__device__ __forceinline__ void constitutive_update(const MatParams& m, float* F, float& Jp, float* t6)
{
    if (m.kind == MPM_FLUID) {
        float p = m.K * (__powf(Jp, -m.gamma) - 1.0f);
        t6[0] = t6[1] = t6[2] = -p * Jp;
        t6[3] = t6[4] = t6[5] = 0.0f;
        return;
    }
    float U[9], s[3], V[9], d[3];
    float vol = 0.0f;
    svd3(F, U, s, V);
    if (m.kind == MPM_SNOW) {
        float t[3];
        t[0] = fminf(fmaxf(s[0], m.lo), m.hi);
        t[1] = fminf(fmaxf(s[1], m.lo), m.hi);
        t[2] = fminf(fmaxf(s[2], m.lo), m.hi);
        Jp *= (s[0] * s[1] * s[2]) / (t[0] * t[1] * t[2]);
        udwt(U, t, V, F);
        float h = __expf(m.xi * (1.0f - Jp));
        float mu = m.mu * h, la = m.la * h;
        float J = t[0] * t[1] * t[2];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            d[k] = 2.0f * mu * (t[k] - 1.0f) * t[k];
        vol = la * J * (J - 1.0f);
    } else if (m.kind == MPM_SAND) {
        float e[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            e[k] = __logf(fmaxf(s[k], 1e-4f));
        float tr = e[0] + e[1] + e[2];
        if (tr >= 0.0f) {
            float one[3] = {1.0f, 1.0f, 1.0f};
            udwt(U, one, V, F);
            e[0] = e[1] = e[2] = 0.0f;
        } else {
            float third = tr * (1.0f / 3.0f);
            float d0 = e[0] - third, d1 = e[1] - third, d2 = e[2] - third;
            float nd = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            float dg = nd + m.dp_coef * tr * m.alpha;
            if (dg > 0.0f) {
                float k = dg / nd;
                e[0] -= k * d0;
                e[1] -= k * d1;
                e[2] -= k * d2;
                float t[3] = {__expf(e[0]), __expf(e[1]), __expf(e[2])};
                udwt(U, t, V, F);
            }
        }
        float tr2 = e[0] + e[1] + e[2];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            d[k] = 2.0f * m.mu * e[k] + m.la * tr2;
    } else {
        float J = s[0] * s[1] * s[2];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            d[k] = 2.0f * m.mu * (s[k] - 1.0f) * s[k];
        vol = m.la * J * (J - 1.0f);
    }
    t6[0] = U[0] * U[0] * d[0] + U[1] * U[1] * d[1] + U[2] * U[2] * d[2] + vol;
    t6[1] = U[3] * U[3] * d[0] + U[4] * U[4] * d[1] + U[5] * U[5] * d[2] + vol;
    t6[2] = U[6] * U[6] * d[0] + U[7] * U[7] * d[1] + U[8] * U[8] * d[2] + vol;
    t6[3] = U[0] * U[3] * d[0] + U[1] * U[4] * d[1] + U[2] * U[5] * d[2];
    t6[4] = U[0] * U[6] * d[0] + U[1] * U[7] * d[1] + U[2] * U[8] * d[2];
    t6[5] = U[3] * U[6] * d[0] + U[4] * U[7] * d[1] + U[5] * U[8] * d[2];
}

}  // namespace mpm
