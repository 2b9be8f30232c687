// Differentiable elastic substep: forward and hand-written adjoint kernels.
//
// Not in the paper: a differentiable form of the same substep (Sec. 4 phases
// P2G -> grid update -> G2P) for gradient-based control and inverse problems.
// Model: fixed-corotated elasticity with a per-particle Young's modulus E_p
// (mu_p, lambda_p from E_p and a common nu), common density, MLS-MPM
// transfers with quadratic B-splines, sticky or slip walls.
//
// The grid is dense (res0 x res1 x res2 nodes): the differentiable rollouts
// this serves are small (tens of thousands of particles on 64^3), so mapping
// and sorting would only add state to differentiate through.  The two grid
// sums (P2G momentum and mass, and the scattered velocity adjoint) are
// accumulated in FP64 (4 doubles per node): in FP32 their order-dependent
// rounding made a 200-substep gradient vary by ~1e-3 from run to run.
//
// State of one particle: 24 floats x[3] v[3] C[9] H[9], with H = F - I the
// displacement gradient (row-major).  The
// adjoint of one substep runs the forward P2G and grid update again, then
// the reverse of G2P (scatter of the velocity adjoint to the grid), of the
// grid update, and of P2G (gather), by the chain rule.  The stress adjoint
// differentiates tau = 2 mu (F - R) F^T + lambda J (J - 1) I through the
// polar rotation R with the closed form
//   <M, dR> = < U Z V^T, dF >,  Z_ij = (G_ij - G_ji) / (s_i + s_j),
//   G = U^T M V,  F = U diag(s) V^T.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <string>

#include "device_math.cuh"
#include "internal.h"

using namespace mpm;

namespace {

struct DiffParams {
    int res[3];
    float dx, inv_dx;
    int boundary, wall;
    float g[3];
    float mu1, la1;   // mu and lambda per unit E (from nu)
    float rho;
};

constexpr int kDT = 128;

inline unsigned dblk(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

struct DStencil {
    int b[3];
    float f[3], w[3][3], dw[3][3];
};

__device__ __forceinline__ bool d_stencil(const DiffParams& dp, const float* x, DStencil& s)
{
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        s.b[a] = base_of(x[a], dp.inv_dx);
        float f = __fmul_rn(x[a], dp.inv_dx) - (float)s.b[a];
        s.f[a] = f;
        bspline(f, s.w[a]);
        s.dw[a][0] = -(1.5f - f);
        s.dw[a][1] = -2.0f * (f - 1.0f);
        s.dw[a][2] = f - 0.5f;
        ok = ok && isfinite(x[a]) && s.b[a] >= 0 && s.b[a] + 2 < dp.res[a];
    }
    return ok;
}

__device__ __forceinline__ int64_t d_node(const DiffParams& dp, const DStencil& s, int i, int j, int k)
{
    return (int64_t)(s.b[0] + i) + (int64_t)dp.res[0] * ((int64_t)(s.b[1] + j) + (int64_t)dp.res[1] * (s.b[2] + k));
}

// Fixed-corotated stress from the displacement gradient H = F - I, keeping
// full FP32 relative precision for small strains (F itself in FP32 resolves
// a strain of 1e-4 to only ~6e-4 relative).  With E = F^T F - I = H + H^T +
// H^T H = V diag(l) V^T (Jacobi on the small matrix E):
//   sigma_i - 1 = l_i / (sqrt(1 + l_i) + 1),
//   F - R = F (I - S^-1) = F V diag((sigma_i - 1) / sigma_i) V^T,
//   J - 1 = tr H + ((tr H)^2 - tr(H^2)) / 2 + det H,
//   tau = 2 mu (F - R) F^T + lambda J (J - 1) I,
// and U = F V diag(1 / sigma) for the rotation adjoint.  (Polar form: for an
// inverted F, det F < 0, R would be a reflection; the rollouts this serves
// stay far from inversion.)
struct FCDecomp {
    float F[9], U[9], V[9], sg[3], FmR[9], J, Jm1;
};

__device__ __forceinline__ void fc_decomp(const float* H, FCDecomp& d)
{
#pragma unroll
    for (int e = 0; e < 9; ++e)
        d.F[e] = H[e] + ((e % 4 == 0) ? 1.0f : 0.0f);
    // E = H + H^T + H^T H
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
    for (int sweep = 0; sweep < 5; ++sweep) {
        jacobi_pair(e00, e11, e01, e02, e12, d.V, 0, 1);
        jacobi_pair(e00, e22, e02, e01, e12, d.V, 0, 2);
        jacobi_pair(e11, e22, e12, e01, e02, d.V, 1, 2);
    }
    if (e00 < e11) swap_neg_cols(d.V, e00, e11, 0, 1);
    if (e00 < e22) swap_neg_cols(d.V, e00, e22, 0, 2);
    if (e11 < e22) swap_neg_cols(d.V, e11, e22, 1, 2);
    const float l[3] = {e00, e11, e22};
    float q[3], inv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float s = sqrtf(fmaxf(1.0f + l[i], 1e-12f));
        d.sg[i] = s;
        float sm1 = l[i] / (s + 1.0f);
        inv[i] = 1.0f / s;
        q[i] = sm1 * inv[i];          // (sigma - 1) / sigma
    }
    float FV[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            FV[3 * r + c] = d.F[3 * r] * d.V[c] + d.F[3 * r + 1] * d.V[3 + c] + d.F[3 * r + 2] * d.V[6 + c];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            d.U[3 * r + c] = FV[3 * r + c] * inv[c];
            d.FmR[3 * r + c] = FV[3 * r] * q[0] * d.V[3 * c] + FV[3 * r + 1] * q[1] * d.V[3 * c + 1] +
                               FV[3 * r + 2] * q[2] * d.V[3 * c + 2];
        }
    float trH = H[0] + H[4] + H[8];
    float trHH = H[0] * H[0] + H[4] * H[4] + H[8] * H[8] + 2.f * (H[1] * H[3] + H[2] * H[6] + H[5] * H[7]);
    d.Jm1 = trH + 0.5f * (trH * trH - trHH) + det3(H);
    d.J = 1.0f + d.Jm1;
}

__device__ __forceinline__ void fc_tau(const DiffParams& dp, float E, const FCDecomp& d, float* tau)
{
    float mu = E * dp.mu1, la = E * dp.la1;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float acc = d.FmR[3 * i] * d.F[3 * j] + d.FmR[3 * i + 1] * d.F[3 * j + 1] + d.FmR[3 * i + 2] * d.F[3 * j + 2];
            tau[3 * i + j] = 2.0f * mu * acc + (i == j ? la * d.J * d.Jm1 : 0.0f);
        }
}

// P2G of the differentiable substep.  A thread takes kRun consecutive
// particles; while they share a base cell their node contributions add up in
// 27 float4 registers, and each such run goes to the grid as FP64 atomics.
// The FP32 partial sums are formed in a fixed order, so the grid sums do not
// depend on the order of the atomics beyond FP64 rounding.
constexpr int kRun = 4;
constexpr int kRunThreads = 64;
constexpr int kRunMinBlocks = 4;

__global__ void __launch_bounds__(kRunThreads, kRunMinBlocks) dk_p2g(DiffParams dp, int64_t n, const float* __restrict__ s,
                                                 const float* __restrict__ E, const float* __restrict__ vol, float dt,
                                                 double* __restrict__ grid, uint32_t* err)
{
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kRun;
    if (p0 >= n)
        return;
    float4 acc[27];
    DStencil run;          // stencil of the open run (its base cell addresses the flush)
    bool open = false;
    auto flush = [&]() {
#pragma unroll
        for (int kk = 0; kk < 3; ++kk)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float4 v = acc[i + 3 * j + 9 * kk];
                    double* g = grid + 4 * d_node(dp, run, i, j, kk);
                    atomicAdd(g + 0, (double)v.x);
                    atomicAdd(g + 1, (double)v.y);
                    atomicAdd(g + 2, (double)v.z);
                    atomicAdd(g + 3, (double)v.w);
                }
    };
#pragma unroll 1
    for (int c = 0; c < kRun; ++c) {
        const int64_t p = p0 + c;
        if (p >= n)
            break;
        const float* q = s + 24 * p;
        DStencil S;
        if (!d_stencil(dp, q, S)) {
            atomicOr(err, ST_EDOMAIN);
            continue;
        }
        FCDecomp dec;
        fc_decomp(q + 15, dec);
        float tau[9];
        fc_tau(dp, E[p], dec, tau);
        const float mp = dp.rho * vol[p];
        const float k = 4.0f * dt * vol[p] * dp.inv_dx * dp.inv_dx;
        float A[9];
#pragma unroll
        for (int e = 0; e < 9; ++e)
            A[e] = (mp * q[6 + e] - k * tau[e]) * dp.dx;
        const bool same = open && S.b[0] == run.b[0] && S.b[1] == run.b[1] && S.b[2] == run.b[2];
        if (open && !same)
            flush();
        if (!same) {
            run = S;
#pragma unroll
            for (int m = 0; m < 27; ++m)
                acc[m] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            open = true;
        }
#pragma unroll
        for (int kk = 0; kk < 3; ++kk)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float wt = S.w[0][i] * S.w[1][j] * S.w[2][kk];
                    const float d0 = (float)i - S.f[0], d1 = (float)j - S.f[1], d2 = (float)kk - S.f[2];
                    float4& a = acc[i + 3 * j + 9 * kk];
                    a.x += wt * (mp * q[3] + A[0] * d0 + A[1] * d1 + A[2] * d2);
                    a.y += wt * (mp * q[4] + A[3] * d0 + A[4] * d1 + A[5] * d2);
                    a.z += wt * (mp * q[5] + A[6] * d0 + A[7] * d1 + A[8] * d2);
                    a.w += wt * mp;
                }
    }
    if (open)
        flush();
}

// v = P / m + dt g with the wall condition; Pm keeps (P, m), vel gets (v, m).
__global__ void dk_grid(DiffParams dp, int64_t nodes, float dt, const double* __restrict__ Pm, float4* __restrict__ vel)
{
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nodes)
        return;
    const double2 pa = reinterpret_cast<const double2*>(Pm)[2 * id], pb = reinterpret_cast<const double2*>(Pm)[2 * id + 1];
    const double P[3] = {pa.x, pa.y, pb.x}, m = pb.y;
    double v[3] = {0.0, 0.0, 0.0};
    if (m > 0.0) {
        int c[3] = {(int)(id % dp.res[0]), (int)((id / dp.res[0]) % dp.res[1]), (int)(id / ((int64_t)dp.res[0] * dp.res[1]))};
        v[0] = P[0] / m + (double)(dt * dp.g[0]);
        v[1] = P[1] / m + (double)(dt * dp.g[1]);
        v[2] = P[2] / m + (double)(dt * dp.g[2]);
        if (dp.boundary == MPM_STICKY) {
            bool wall = false;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                wall = wall || c[a] < dp.wall || c[a] >= dp.res[a] - dp.wall;
            if (wall)
                v[0] = v[1] = v[2] = 0.f;
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (c[a] < dp.wall && v[a] < 0.f)
                    v[a] = 0.f;
                if (c[a] >= dp.res[a] - dp.wall && v[a] > 0.f)
                    v[a] = 0.f;
            }
        }
    }
    vel[id] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)m);
}

__global__ void dk_g2p(DiffParams dp, int64_t n, const float* __restrict__ s, const float4* __restrict__ vel, float dt,
                       float* __restrict__ out)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    const float* q = s + 24 * p;
    float* o = out + 24 * p;
    DStencil S;
    if (!d_stencil(dp, q, S)) {
        for (int e = 0; e < 24; ++e)
            o[e] = q[e];
        return;
    }
    float vp[3] = {0.f, 0.f, 0.f}, B[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 3; ++kk)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float wt = S.w[0][i] * S.w[1][j] * S.w[2][kk];
                float d[3] = {(float)i - S.f[0], (float)j - S.f[1], (float)kk - S.f[2]};
                float4 g = vel[d_node(dp, S, i, j, kk)];
                float gv[3] = {wt * g.x, wt * g.y, wt * g.z};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    vp[a] += gv[a];
#pragma unroll
                    for (int b = 0; b < 3; ++b)
                        B[3 * a + b] += gv[a] * d[b];
                }
            }
    float C[9];
#pragma unroll
    for (int e = 0; e < 9; ++e)
        C[e] = 4.0f * dp.inv_dx * B[e];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = q[a] + dt * vp[a];
        o[3 + a] = vp[a];
    }
#pragma unroll
    for (int e = 0; e < 9; ++e)
        o[6 + e] = C[e];
    // F' = (I + dt C) F with F = I + H:  H' = H + dt (C + C H)
    const float* H = q + 15;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            o[15 + 3 * r + c] = H[3 * r + c] + dt * (C[3 * r + c] + C[3 * r] * H[c] + C[3 * r + 1] * H[3 + c] +
                                                      C[3 * r + 2] * H[6 + c]);
}

// ---- adjoint ------------------------------------------------------------------------

// Reverse of G2P: writes xbar (partial) and Fbar (partial) of the input state
// and scatters the velocity adjoint to the grid.
__global__ void dk_g2p_adj(DiffParams dp, int64_t n, const float* __restrict__ s, const float4* __restrict__ vel,
                           const float* __restrict__ gout, float dt, float* __restrict__ gin, double* __restrict__ vbar)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    const float* q = s + 24 * p;
    const float* g1 = gout + 24 * p;
    float* gi = gin + 24 * p;
    DStencil S;
    if (!d_stencil(dp, q, S)) {
        for (int e = 0; e < 24; ++e)
            gi[e] = 0.0f;
        return;
    }
    const float D = 4.0f * dp.inv_dx * dp.inv_dx;
    const float h = dp.dx;
    // recompute C'
    float Cn[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 3; ++kk)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float wt = S.w[0][i] * S.w[1][j] * S.w[2][kk];
                float d[3] = {((float)i - S.f[0]) * h, ((float)j - S.f[1]) * h, ((float)kk - S.f[2]) * h};
                float4 g = vel[d_node(dp, S, i, j, kk)];
                float gv[3] = {g.x, g.y, g.z};
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b)
                        Cn[3 * a + b] += D * wt * gv[a] * d[b];
            }
    float F[9];
#pragma unroll
    for (int e = 0; e < 9; ++e)
        F[e] = q[15 + e] + ((e % 4 == 0) ? 1.0f : 0.0f);
    const float* Fb1 = g1 + 15;
    // F' = (I + dt C') F
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                acc += ((c == a ? 1.0f : 0.0f) + dt * Cn[3 * c + a]) * Fb1[3 * c + b];
            gi[15 + 3 * a + b] = acc;
        }
    float Ct[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Ct[3 * a + b] = g1[6 + 3 * a + b] +
                            dt * (Fb1[3 * a] * F[3 * b] + Fb1[3 * a + 1] * F[3 * b + 1] + Fb1[3 * a + 2] * F[3 * b + 2]);
    float vt[3], xb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xb[a] = g1[a];
        vt[a] = g1[3 + a] + dt * g1[a];
    }
#pragma unroll
    for (int kk = 0; kk < 3; ++kk)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float wt = S.w[0][i] * S.w[1][j] * S.w[2][kk];
                float gw[3] = {dp.inv_dx * S.dw[0][i] * S.w[1][j] * S.w[2][kk],
                               dp.inv_dx * S.w[0][i] * S.dw[1][j] * S.w[2][kk],
                               dp.inv_dx * S.w[0][i] * S.w[1][j] * S.dw[2][kk]};
                float d[3] = {((float)i - S.f[0]) * h, ((float)j - S.f[1]) * h, ((float)kk - S.f[2]) * h};
                int64_t id = d_node(dp, S, i, j, kk);
                float4 g = vel[id];
                float v[3] = {g.x, g.y, g.z};
                float Cd[3], CtTv[3];
                float vCd = 0.f, vtv = 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Cd[a] = Ct[3 * a] * d[0] + Ct[3 * a + 1] * d[1] + Ct[3 * a + 2] * d[2];
                    CtTv[a] = Ct[a] * v[0] + Ct[3 + a] * v[1] + Ct[6 + a] * v[2];
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    vtv += vt[a] * v[a];
                    vCd += v[a] * Cd[a];
                }
                atomicAdd(vbar + 4 * id + 0, (double)(wt * (vt[0] + D * Cd[0])));
                atomicAdd(vbar + 4 * id + 1, (double)(wt * (vt[1] + D * Cd[1])));
                atomicAdd(vbar + 4 * id + 2, (double)(wt * (vt[2] + D * Cd[2])));
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    xb[a] += gw[a] * (vtv + D * vCd) - D * wt * CtTv[a];
            }
#pragma unroll
    for (int a = 0; a < 3; ++a)
        gi[a] = xb[a];
#pragma unroll
    for (int e = 3; e < 15; ++e)
        gi[e] = 0.0f;
}

// Reverse of the grid update: (Pbar, mbar) from vbar.
__global__ void dk_grid_adj(DiffParams dp, int64_t nodes, float dt, const double* __restrict__ Pm,
                            const double* __restrict__ vbar, float4* __restrict__ Pmbar)
{
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nodes)
        return;
    const double2 pa = reinterpret_cast<const double2*>(Pm)[2 * id], pq = reinterpret_cast<const double2*>(Pm)[2 * id + 1];
    const double P[3] = {pa.x, pa.y, pq.x}, m = pq.y;
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m > 0.0) {
        const double2 ba = reinterpret_cast<const double2*>(vbar)[2 * id], bb = reinterpret_cast<const double2*>(vbar)[2 * id + 1];
        int c[3] = {(int)(id % dp.res[0]), (int)((id / dp.res[0]) % dp.res[1]), (int)(id / ((int64_t)dp.res[0] * dp.res[1]))};
        const double b[3] = {ba.x, ba.y, bb.x};
        double keep[3] = {1.0, 1.0, 1.0};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bool low = c[a] < dp.wall, high = c[a] >= dp.res[a] - dp.wall;
            double vfree = P[a] / m + (double)(dt * dp.g[a]);   // as dk_grid computes it
            if (dp.boundary == MPM_STICKY) {
                if (low || high)
                    keep[0] = keep[1] = keep[2] = 0.0;
            } else if ((low && vfree < 0.0) || (high && vfree > 0.0)) {
                keep[a] = 0.0;
            }
        }
        const double im = 1.0 / m;
        double mb = 0.0;
        double pb[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double v = keep[a] * b[a];
            pb[a] = v * im;
            mb -= v * P[a] * im * im;
        }
        out = make_float4((float)pb[0], (float)pb[1], (float)pb[2], (float)mb);
    }
    Pmbar[id] = out;
}

// Fbar += d tau / dF contracted with taubar (fixed-corotated, closed form):
//   Fbar = 2 mu [taubar F + taubar^T (F - R) - U Z V^T] + lambda (2J - 1) tr(taubar) cof(F)
// with Z_ij = (G_ij - G_ji) / (s_i + s_j), G = U^T (taubar F) V.
__device__ __forceinline__ void fc_tau_vjp(float mu, float la, const FCDecomp& d, const float* tb, float* Fb)
{
    const float* F = d.F;
    const float* U = d.U;
    const float* V = d.V;
    float M[9], G[9], Z[9], UZ[9], MV[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            M[3 * i + j] = tb[3 * i] * F[j] + tb[3 * i + 1] * F[3 + j] + tb[3 * i + 2] * F[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            MV[3 * i + j] = M[3 * i] * V[j] + M[3 * i + 1] * V[3 + j] + M[3 * i + 2] * V[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            G[3 * i + j] = U[i] * MV[j] + U[3 + i] * MV[3 + j] + U[6 + i] * MV[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float den = d.sg[i] + d.sg[j];
            den = fabsf(den) < 1e-6f ? copysignf(1e-6f, den) : den;
            Z[3 * i + j] = (i == j) ? 0.0f : (G[3 * i + j] - G[3 * j + i]) / den;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            UZ[3 * i + j] = U[3 * i] * Z[j] + U[3 * i + 1] * Z[3 + j] + U[3 * i + 2] * Z[6 + j];
    float tr = tb[0] + tb[4] + tb[8];
    float cof[9] = {F[4] * F[8] - F[5] * F[7], F[5] * F[6] - F[3] * F[8], F[3] * F[7] - F[4] * F[6],
                    F[2] * F[7] - F[1] * F[8], F[0] * F[8] - F[2] * F[6], F[1] * F[6] - F[0] * F[7],
                    F[1] * F[5] - F[2] * F[4], F[2] * F[3] - F[0] * F[5], F[0] * F[4] - F[1] * F[3]};
    float cj = la * (2.0f * d.J - 1.0f) * tr;
    const float* FmR = d.FmR;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float t2 = tb[i] * FmR[j] + tb[3 + i] * FmR[3 + j] + tb[6 + i] * FmR[6 + j];
            float ZV = UZ[3 * i] * V[3 * j] + UZ[3 * i + 1] * V[3 * j + 1] + UZ[3 * i + 2] * V[3 * j + 2];
            Fb[3 * i + j] += 2.0f * mu * (M[3 * i + j] + t2 - ZV) + cj * cof[3 * i + j];
        }
}

// Reverse of P2G: gathers (Pbar, mbar) and completes the input adjoint.
__global__ void dk_p2g_adj(DiffParams dp, int64_t n, const float* __restrict__ s, const float* __restrict__ E,
                           const float* __restrict__ vol, float dt, const float4* __restrict__ Pmbar,
                           float* __restrict__ gin, float* __restrict__ gE)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    const float* q = s + 24 * p;
    float* gi = gin + 24 * p;
    DStencil S;
    if (!d_stencil(dp, q, S))
        return;
    const float h = dp.dx;
    const float Ep = E[p];
    FCDecomp dec;
    fc_decomp(q + 15, dec);
    float tau[9];
    fc_tau(dp, Ep, dec, tau);
    float mp = dp.rho * vol[p];
    float k = 4.0f * dt * vol[p] * dp.inv_dx * dp.inv_dx;
    float A[9];
#pragma unroll
    for (int e = 0; e < 9; ++e)
        A[e] = mp * q[6 + e] - k * tau[e];
    float Ab[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float xb[3] = {0.f, 0.f, 0.f}, vb[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 3; ++kk)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float wt = S.w[0][i] * S.w[1][j] * S.w[2][kk];
                float gw[3] = {dp.inv_dx * S.dw[0][i] * S.w[1][j] * S.w[2][kk],
                               dp.inv_dx * S.w[0][i] * S.dw[1][j] * S.w[2][kk],
                               dp.inv_dx * S.w[0][i] * S.w[1][j] * S.dw[2][kk]};
                float d[3] = {((float)i - S.f[0]) * h, ((float)j - S.f[1]) * h, ((float)kk - S.f[2]) * h};
                float4 pm = Pmbar[d_node(dp, S, i, j, kk)];
                float Pb[3] = {pm.x, pm.y, pm.z};
                float contrib = mp * pm.w;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float Ad = A[3 * a] * d[0] + A[3 * a + 1] * d[1] + A[3 * a + 2] * d[2];
                    contrib += Pb[a] * (mp * q[3 + a] + Ad);
                    vb[a] += wt * mp * Pb[a];
#pragma unroll
                    for (int b = 0; b < 3; ++b)
                        Ab[3 * a + b] += wt * Pb[a] * d[b];
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float ATPb = A[a] * Pb[0] + A[3 + a] * Pb[1] + A[6 + a] * Pb[2];
                    xb[a] += gw[a] * contrib - wt * ATPb;
                }
            }
    float tb[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        gi[6 + e] += mp * Ab[e];
        tb[e] = -k * Ab[e];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gi[a] += xb[a];
        gi[3 + a] += vb[a];
    }
    float Fb[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    fc_tau_vjp(Ep * dp.mu1, Ep * dp.la1, dec, tb, Fb);
#pragma unroll
    for (int e = 0; e < 9; ++e)
        gi[15 + e] += Fb[e];
    // tau is linear in E: dL/dE = <taubar, tau / E>
    float s1 = 0.f;
#pragma unroll
    for (int e = 0; e < 9; ++e)
        s1 += tb[e] * tau[e];
    gE[p] += s1 / Ep;
}

}  // namespace

struct mpm_diff {
    DiffParams dp{};
    int64_t n = 0, nodes = 0;
    cudaStream_t stream = nullptr;
    mpm_allocator alloc{};
    bool have_alloc = false;
    float* vol = nullptr;
    double *Pm = nullptr, *vbar = nullptr;   // 4 doubles per node
    float4 *vel = nullptr, *Pmbar = nullptr;
    uint32_t* err = nullptr;
    int64_t launches = 0;
};

static void* dd_alloc(mpm_diff* d, size_t b)
{
    if (d->have_alloc)
        return d->alloc.alloc(b, (void*)d->stream, d->alloc.user);
    void* p = nullptr;
    return cudaMallocAsync(&p, b, d->stream) == cudaSuccess ? p : nullptr;
}

static void dd_free(mpm_diff* d, void* p, size_t b)
{
    if (!p)
        return;
    if (d->have_alloc)
        d->alloc.free(p, b, (void*)d->stream, d->alloc.user);
    else
        cudaFreeAsync(p, d->stream);
}

static void forward_grid(mpm_diff* d, float dt, const float* E, const float* s)
{
    cudaStream_t st = d->stream;
    cudaMemsetAsync(d->Pm, 0, (size_t)d->nodes * 32, st);
    dk_p2g<<<dblk((d->n + kRun - 1) / kRun, kRunThreads), kRunThreads, 0, st>>>(d->dp, d->n, s, E, d->vol, dt, d->Pm,
                                                                              d->err);
    dk_grid<<<dblk(d->nodes, 256), 256, 0, st>>>(d->dp, d->nodes, dt, d->Pm, d->vel);
    d->launches += 2;
}

extern "C" {

mpm_status mpm_diff_create(const mpm_config* cfg, float nu, float rho, int64_t n, const float* vol0,
                           const mpm_allocator* allocator, void* cuda_stream, mpm_diff** out)
{
    if (!cfg || !out || n <= 0 || !(rho > 0.f) || !(nu > -1.f && nu < 0.5f) || !(cfg->dx > 0.f))
        return MPM_EINVAL;
    if (cfg->transfer != MPM_APIC)
        return MPM_EINVAL;   // the differentiable substep is APIC only
    for (int a = 0; a < 3; ++a)
        if (cfg->res[a] < 8 || cfg->res[a] > 512)
            return MPM_EINVAL;
    *out = nullptr;
    mpm_diff* d = new (std::nothrow) mpm_diff();
    if (!d)
        return MPM_ENOMEM;
    d->stream = (cudaStream_t)cuda_stream;
    if (allocator) {
        d->alloc = *allocator;
        d->have_alloc = true;
    }
    DiffParams& dp = d->dp;
    for (int a = 0; a < 3; ++a) {
        dp.res[a] = cfg->res[a];
        dp.g[a] = cfg->gravity[a];
    }
    dp.dx = cfg->dx;
    dp.inv_dx = 1.0f / cfg->dx;
    dp.boundary = cfg->boundary;
    dp.wall = cfg->wall;
    dp.mu1 = (float)(1.0 / (2.0 * (1.0 + nu)));
    dp.la1 = (float)(nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
    dp.rho = rho;
    d->n = n;
    d->nodes = (int64_t)cfg->res[0] * cfg->res[1] * cfg->res[2];
    size_t gb = (size_t)d->nodes * 16;
    d->vol = (float*)dd_alloc(d, (size_t)n * 4);
    d->Pm = (double*)dd_alloc(d, 2 * gb);
    d->vel = (float4*)dd_alloc(d, gb);
    d->vbar = (double*)dd_alloc(d, 2 * gb);
    d->Pmbar = (float4*)dd_alloc(d, gb);
    d->err = (uint32_t*)dd_alloc(d, 256);
    if (!d->vol || !d->Pm || !d->vel || !d->vbar || !d->Pmbar || !d->err) {
        mpm_diff_destroy(d);
        return MPM_ENOMEM;
    }
    cudaStream_t st = d->stream;
    cudaMemsetAsync(d->err, 0, 256, st);
    if (vol0) {
        cudaMemcpyAsync(d->vol, vol0, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
    } else {
        float v = cfg->dx * cfg->dx * cfg->dx / 8.0f;
        float* h = new (std::nothrow) float[(size_t)n];
        if (!h) {
            mpm_diff_destroy(d);
            return MPM_ENOMEM;
        }
        for (int64_t i = 0; i < n; ++i)
            h[i] = v;
        cudaMemcpyAsync(d->vol, h, (size_t)n * 4, cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
        delete[] h;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        mpm_diff_destroy(d);
        return MPM_ECUDA;
    }
    *out = d;
    return MPM_OK;
}

mpm_status mpm_diff_forward(mpm_diff* d, float dt, const float* E, const float* s_in, float* s_out)
{
    TraceRange trace("mpm_diff_forward");
    if (!d || !E || !s_in || !s_out || !(dt > 0.f) || s_in == s_out)
        return MPM_EINVAL;
    forward_grid(d, dt, E, s_in);
    dk_g2p<<<dblk(d->n, kDT), kDT, 0, d->stream>>>(d->dp, d->n, s_in, d->vel, dt, s_out);
    d->launches += 1;
    return cudaGetLastError() == cudaSuccess ? MPM_OK : MPM_ECUDA;
}

mpm_status mpm_diff_adjoint(mpm_diff* d, float dt, const float* E, const float* s_in, const float* g_out,
                            float* g_in, float* gE)
{
    TraceRange trace("mpm_diff_adjoint");
    if (!d || !E || !s_in || !g_out || !g_in || !gE || !(dt > 0.f) || g_in == g_out)
        return MPM_EINVAL;
    cudaStream_t st = d->stream;
    forward_grid(d, dt, E, s_in);
    cudaMemsetAsync(d->vbar, 0, (size_t)d->nodes * 32, st);
    dk_g2p_adj<<<dblk(d->n, kDT), kDT, 0, st>>>(d->dp, d->n, s_in, d->vel, g_out, dt, g_in, d->vbar);
    dk_grid_adj<<<dblk(d->nodes, 256), 256, 0, st>>>(d->dp, d->nodes, dt, d->Pm, d->vbar, d->Pmbar);
    dk_p2g_adj<<<dblk(d->n, kDT), kDT, 0, st>>>(d->dp, d->n, s_in, E, d->vol, dt, d->Pmbar, g_in, gE);
    d->launches += 3;
    return cudaGetLastError() == cudaSuccess ? MPM_OK : MPM_ECUDA;
}

mpm_status mpm_diff_sync(mpm_diff* d)
{
    if (!d)
        return MPM_EINVAL;
    uint32_t e = 0;
    if (cudaMemcpyAsync(&e, d->err, 4, cudaMemcpyDeviceToHost, d->stream) != cudaSuccess ||
        cudaStreamSynchronize(d->stream) != cudaSuccess)
        return MPM_ECUDA;
    return (e & ST_EDOMAIN) ? MPM_EDOMAIN : MPM_OK;
}

void mpm_diff_destroy(mpm_diff* d)
{
    if (!d)
        return;
    cudaStreamSynchronize(d->stream);
    size_t gb = (size_t)d->nodes * 16;
    dd_free(d, d->vol, (size_t)d->n * 4);
    dd_free(d, d->Pm, 2 * gb);
    dd_free(d, d->vel, gb);
    dd_free(d, d->vbar, 2 * gb);
    dd_free(d, d->Pmbar, gb);
    dd_free(d, d->err, 256);
    cudaStreamSynchronize(d->stream);
    delete d;
}

}  // extern "C"
