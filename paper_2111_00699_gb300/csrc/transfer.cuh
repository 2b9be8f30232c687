// Device routines shared by the transfer kernels of one MLS-MPM substep
// (p2g.cu, g2p.cu, g2p2g.cu): stencil addressing in the blocked grid, the
// per-particle P2G record and its 27 node contributions, the register and
// shared-memory node accumulators, the warp-level reduction of Sec. 4.2.2,
// and everything G2P does after its gather (C, x, v, the F update with the
// return map and the stress, the free-zone test of Sec. 4.2.1).
//
// Layout: particles are SoA float channels (coalesced per warp); grid nodes
// are float4 (p_x, p_y, p_z, m) -- after the update (v_x, v_y, v_z, m) -- in
// physical blocks of 4x4x4 = 64 nodes, node (i, j, k) of a block at
// (i & 3) + 4 (j & 3) + 16 (k & 3).  A node's block index comes from the
// direct-mapped Morton table.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "async_copy.cuh"
#include "device_math.cuh"
#include "internal.h"

namespace mpm {

namespace {

constexpr int kTransferThreads = 128;  // 4 warps per CUDA block (Sec. 6.2)

// The physical blocks a 3-node stencil starting at base b touches: per axis
// the block b >> 2 and, when (b & 3) >= 2, also the next one.  pb[dz][dy][dx]
// (flattened dx + 2 dy + 4 dz) receives the block indices; returns false if
// one of them is not mapped.
__device__ __forceinline__ bool stencil_blocks(const GridView& gv, const int* b, int* pb)
{
    uint32_t sx[2], sy[2], sz[2];
    int B0 = b[0] >> 2, B1 = b[1] >> 2, B2 = b[2] >> 2;
    // Morton codes of B and B + 1 per axis; the +1 is done on the dilated
    // bits directly (fill the other axes' bits with ones, add, mask).
    constexpr uint32_t kMx = 0x09249249u, kMy = kMx << 1, kMz = kMx << 2;
    sx[0] = spread3((uint32_t)B0);
    sx[1] = ((sx[0] | ~kMx) + 1u) & kMx;
    sy[0] = spread3((uint32_t)B1) << 1;
    sy[1] = ((sy[0] | ~kMy) + 1u) & kMy;
    sz[0] = spread3((uint32_t)B2) << 2;
    sz[1] = ((sz[0] | ~kMz) + 1u) & kMz;
    int cx = (b[0] & 3) >= 2, cy = (b[1] & 3) >= 2, cz = (b[2] & 3) >= 2;
    bool ok = true;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                int v = 0;
                if ((dx <= cx) && (dy <= cy) && (dz <= cz)) {
                    v = __ldg(&gv.table[sx[dx] | sy[dy] | sz[dz]]);
                    ok = ok && v >= 0;
                }
                pb[dx + 2 * dy + 4 * dz] = v;
            }
    return ok;
}

__device__ __forceinline__ bool stencil_index(const GridView& gv, const int* b, StencilIndex& si)
{
    int pb[8];
    bool ok = stencil_blocks(gv, b, pb);
#pragma unroll
    for (int c = 0; c < 8; ++c)
        si.pb64[c] = pb[c] * 64;
    si.bx = b[0] & 3;
    si.by = b[1] & 3;
    si.bz = b[2] & 3;
    return ok;
}

// The 3x3x3 stencil at base b lies inside the grid.
__device__ __forceinline__ bool in_grid(const SimParams& sp, const int* b, const float* x)
{
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        ok = ok && isfinite(x[a]) && b[a] >= 0 && b[a] + 2 < sp.res[a];
    return ok;
}

// Everything P2G needs of one particle: stencil base and weights, mass, the
// momentum m v and the affine matrix A = (m C - 4 dt V / dx^2 tau) dx, so that
// node (i, j, k) of the stencil receives w (m v + A (node - f)) and w m.
struct P2GParticle {
    int b[3];
    float f[3], w[3][3];
    float mp, mv[3], A[9];
};

// get(c) returns channel c of the particle (global channel numbering).
template <class Get>
__device__ __forceinline__ bool make_p2g_particle(const SimParams& sp, Get get, int mat, float dt, P2GParticle& q,
                                                  uint32_t* err)
{
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x[a] = get(CH_X + a);
        q.b[a] = base_of(x[a], sp.inv_dx);
        q.f[a] = __fmul_rn(x[a], sp.inv_dx) - (float)q.b[a];
        bspline(q.f[a], q.w[a]);
    }
    if (!in_grid(sp, q.b, x)) {
        atomicOr(err, ST_EDOMAIN);
        return false;
    }
    const float rho = sp.mat[mat].rho;
    float vol = get(CH_VOL);
    q.mp = rho * vol;
    float kst = 4.0f * dt * vol * sp.inv_dx * sp.inv_dx;
    float t[6];
#pragma unroll
    for (int e = 0; e < 6; ++e)
        t[e] = kst * get(CH_TAU + e);
    // symmetric tau: (xx, yy, zz, xy, xz, yz)
    const float tm[9] = {t[0], t[3], t[4], t[3], t[1], t[5], t[4], t[5], t[2]};
#pragma unroll
    for (int e = 0; e < 9; ++e)
        q.A[e] = (q.mp * get(CH_C + e) - tm[e]) * sp.dx;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        q.mv[a] = q.mp * get(CH_V + a);
    return true;
}

template <bool kAoS = false>
__device__ __forceinline__ bool load_p2g_particle(const SimParams& sp, const PartView& pv, int64_t p, float dt,
                                                  P2GParticle& q, uint32_t* err)
{
    // a single-material scene needs no per-particle material index
    return make_p2g_particle(sp, [&](int c) { return pch<kAoS>(pv, c, p); }, sp.n_mats == 1 ? 0 : (int)pv.mat[p], dt,
                             q, err);
}

__device__ __forceinline__ float4 node_contribution(const P2GParticle& q, int i, int j, int k)
{
    float dxo = (float)i - q.f[0], dy = (float)j - q.f[1], dz = (float)k - q.f[2];
    float wt = q.w[0][i] * q.w[1][j] * q.w[2][k];
    float4 val;
    val.x = wt * (q.mv[0] + q.A[0] * dxo + q.A[1] * dy + q.A[2] * dz);
    val.y = wt * (q.mv[1] + q.A[3] * dxo + q.A[4] * dy + q.A[5] * dz);
    val.z = wt * (q.mv[2] + q.A[6] * dxo + q.A[7] * dy + q.A[8] * dz);
    val.w = wt * q.mp;
    return val;
}

// 27 float4 global atomics (native vector reductions on sm_90+) into `target`
// (a grid buffer with the mapping of gv).
__device__ __forceinline__ void scatter_to(const GridView& gv, float4* target, const P2GParticle& q, uint32_t* err)
{
    StencilIndex si;
    if (!stencil_index(gv, q.b, si)) {
        atomicOr(err, ST_MISSED);
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                atomicAdd(&target[si(i, j, k)], node_contribution(q, i, j, k));
}

__device__ __forceinline__ void scatter_global(const GridView& gv, const P2GParticle& q, uint32_t* err)
{
    scatter_to(gv, gv.cur, q, err);
}

// P2G_CHUNK4 / P2G_CHUNK8: a thread walks K consecutive particles of the
// cell-sorted storage order.  Particles with the same base cell (about 8 per
// cell after the sort of Sec. 4.2.2) add into 27 node accumulators held in
// registers; the accumulators go to global memory (27 float4 reductions)
// only when the base cell changes and at the end of the chunk.  Reductions
// per particle drop from 27 to 27 x (runs per chunk) / K.
struct NodeAcc {
    float4 a[27];
};

__device__ __forceinline__ void acc_zero(NodeAcc& acc)
{
#pragma unroll
    for (int n = 0; n < 27; ++n)
        acc.a[n] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// The contributions of particle q to its 27 nodes: add(n, wt, vx, vy, vz, m)
// for node n = i + 3 j + 9 k receives w (m v + A (node - f)) as wt * (vx, vy,
// vz) and w m as wt * m.  The affine term is split per axis: (mv + A d) =
// (mv + A_y dy + A_z dz) + A_x dx, with the (j, k) part computed once per row.
template <class Add>
__device__ __forceinline__ void p2g_contributions(const P2GParticle& q, Add add)
{
    float dxo[3], dyo[3], dzo[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dxo[i] = (float)i - q.f[0];
        dyo[i] = (float)i - q.f[1];
        dzo[i] = (float)i - q.f[2];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float wyz = q.w[1][j] * q.w[2][k];
            float bx = q.mv[0] + q.A[1] * dyo[j] + q.A[2] * dzo[k];
            float by = q.mv[1] + q.A[4] * dyo[j] + q.A[5] * dzo[k];
            float bz = q.mv[2] + q.A[7] * dyo[j] + q.A[8] * dzo[k];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                add(i + 3 * j + 9 * k, q.w[0][i] * wyz, bx + q.A[0] * dxo[i], by + q.A[3] * dxo[i],
                    bz + q.A[6] * dxo[i], q.mp);
        }
}

// The same contributions from centred offsets (fewer instructions, more
// values live at once: used where no accumulators compete for registers).
template <class Add>
__device__ __forceinline__ void p2g_contributions_centred(const P2GParticle& q, Add add)
{
    // With centred offsets e = (i, j, k) - 1 in {-1, 0, 1}, node - f =
    // e - (f - 1), so mv + A (node - f) = u + A e with u = mv - A (f - 1):
    // per row of 3 nodes along x the value is u + A_y e_j + A_z e_k, and
    // the three nodes of the row differ from it by -A_x, 0 and +A_x.
    const float g0 = q.f[0] - 1.0f, g1 = q.f[1] - 1.0f, g2 = q.f[2] - 1.0f;
    float u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        u[a] = q.mv[a] - (q.A[3 * a] * g0 + q.A[3 * a + 1] * g1 + q.A[3 * a + 2] * g2);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float wyz = q.w[1][j] * q.w[2][k];
            float b[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float r = u[a];
                if (j == 0) r -= q.A[3 * a + 1];
                if (j == 2) r += q.A[3 * a + 1];
                if (k == 0) r -= q.A[3 * a + 2];
                if (k == 2) r += q.A[3 * a + 2];
                b[a] = r;
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float v[3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    v[a] = i == 0 ? b[a] - q.A[3 * a] : (i == 2 ? b[a] + q.A[3 * a] : b[a]);
                add(i + 3 * j + 9 * k, q.w[0][i] * wyz, v[0], v[1], v[2], q.mp);
            }
        }
}

// acc += contributions of particle q (same base cell as the accumulator).
__device__ __forceinline__ void acc_add(NodeAcc& acc, const P2GParticle& q)
{
    p2g_contributions(q, [&](int n, float wt, float vx, float vy, float vz, float m) {
        float4& a = acc.a[n];
        a.x = fmaf(wt, vx, a.x);
        a.y = fmaf(wt, vy, a.y);
        a.z = fmaf(wt, vz, a.z);
        a.w = fmaf(wt, m, a.w);
    });
}

// acc_add with Blackwell's paired FP32 arithmetic (__ffma2_rn: two fused
// multiply-adds in one instruction): the accumulator float4 is two pairs,
// (p_x, p_y) and (p_z, m), and the affine value's x and y rows are formed as
// one pair.
__device__ __forceinline__ void acc_add_x2(NodeAcc& acc, const P2GParticle& q)
{
    const float2 mvxy = make_float2(q.mv[0], q.mv[1]);
    const float2 ax = make_float2(q.A[0], q.A[3]), ay = make_float2(q.A[1], q.A[4]), az = make_float2(q.A[2], q.A[5]);
    float dxo[3], dyo[3], dzo[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dxo[i] = (float)i - q.f[0];
        dyo[i] = (float)i - q.f[1];
        dzo[i] = (float)i - q.f[2];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float wyz = q.w[1][j] * q.w[2][k];
            const float2 bxy = __ffma2_rn(az, make_float2(dzo[k], dzo[k]),
                                          __ffma2_rn(ay, make_float2(dyo[j], dyo[j]), mvxy));
            const float bz = q.mv[2] + q.A[7] * dyo[j] + q.A[8] * dzo[k];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float wt = q.w[0][i] * wyz;
                const float2 w2 = make_float2(wt, wt);
                const float2 vxy = __ffma2_rn(ax, make_float2(dxo[i], dxo[i]), bxy);
                const float vz = fmaf(q.A[6], dxo[i], bz);
                float4& a = acc.a[i + 3 * j + 9 * k];
                const float2 axy = __ffma2_rn(w2, vxy, make_float2(a.x, a.y));
                const float2 azw = __ffma2_rn(w2, make_float2(vz, q.mp), make_float2(a.z, a.w));
                a = make_float4(axy.x, axy.y, azw.x, azw.y);
            }
        }
}

// The same 27 accumulators held in shared memory, private to one thread:
// node n at base[n * kTransferThreads] (a warp touches 32 consecutive float4
// per node: no bank conflicts, no atomics).  Frees ~108 registers per thread
// for occupancy at the cost of a shared load and store per node.
struct SmemAcc {
    float4* base;
};

__device__ __forceinline__ void acc_zero(SmemAcc acc)
{
#pragma unroll
    for (int n = 0; n < 27; ++n)
        acc.base[n * kTransferThreads] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

__device__ __forceinline__ void acc_add(SmemAcc acc, const P2GParticle& q)
{
    p2g_contributions(q, [&](int n, float wt, float vx, float vy, float vz, float m) {
        float4 a = acc.base[n * kTransferThreads];
        a.x = fmaf(wt, vx, a.x);
        a.y = fmaf(wt, vy, a.y);
        a.z = fmaf(wt, vz, a.z);
        a.w = fmaf(wt, m, a.w);
        acc.base[n * kTransferThreads] = a;
        // one row of 3 nodes at a time: keeps the compiler from hoisting all
        // 27 shared loads (and their registers) ahead of the arithmetic
        if (n % 3 == 2)
            asm volatile("" ::: "memory");
    });
}

__device__ __forceinline__ void acc_flush(const GridView& gv, float4* target, SmemAcc acc, const int* b,
                                          uint32_t* err)
{
    StencilIndex si;
    if (!stencil_index(gv, b, si)) {
        atomicOr(err, ST_MISSED);
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                atomicAdd(&target[si(i, j, k)], acc.base[(i + 3 * j + 9 * k) * kTransferThreads]);
}

constexpr size_t kSmemAccBytes = (size_t)27 * kTransferThreads * sizeof(float4);

__device__ __forceinline__ void acc_flush(const GridView& gv, float4* target, const NodeAcc& acc, const int* b,
                                          uint32_t* err)
{
    StencilIndex si;
    if (!stencil_index(gv, b, si)) {
        atomicOr(err, ST_MISSED);
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                atomicAdd(&target[si(i, j, k)], acc.a[i + 3 * j + 9 * k]);
}

// ---- node-parallel runs (P2G_NODE and its fused form) -----------------------
// A warp walks 32 * NB consecutive particles of the cell-sorted order, 32 at
// a time: each lane prepares one particle of the batch with prep(p, q) into
// a 16-float record in shared memory (fraction f, mass, and the node value's
// affine form m v + A (n - f) = c + A n with c = m v - A f, n = (i, j, k) the
// node's offset from the base cell); then the warp takes the batch's
// particles in order, and lane l < 27 adds each particle's contribution to
// stencil node (l % 3, l / 3 % 3, l / 9) -- its weight, three quadratic
// B-spline factors each written as a polynomial in f with the lane's
// coefficients, times (c + A n, m) -- into one float4.  At a change of base
// cell the node lanes issue one float4 reduction each into `target` (27
// reductions in one warp instruction) and look up the new cell's node
// addresses, which arrive while the next run is summed.  Runs carry over
// from batch to batch: a warp reduces once per distinct cell of its range.
constexpr int kNodeWarps = kTransferThreads / 32;

template <int NB, class Prep>
__device__ __forceinline__ void node_runs(const GridView& gv, float4* target, int64_t n, Prep prep,
                                          uint32_t* __restrict__ err)
{
    __shared__ float4 s_rec[kNodeWarps][4][32];   // [warp][quarter of the record][particle of the batch]
    __shared__ int s_key[kNodeWarps][32];          // base cell, x | y << 10 | z << 20 (res <= 1024); -1: skip
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t begin = ((int64_t)blockIdx.x * kNodeWarps + w) * (32 * NB);
    if (begin >= n)
        return;
    const int64_t end = begin + 32 * NB < n ? begin + 32 * NB : n;
    const int ni = lane % 3, nj = (lane / 3) % 3, nk = lane / 9;   // lanes 27-31: nk = 3, no node
    const bool node_lane = lane < 27;
    const float fi = (float)ni, fj = (float)nj, fk = (float)nk;
    // weight of offset index i at fraction f: N_i(f) = (c2 f + c1) f + c0, the quadratic B-spline
    // pieces 0.5 (1.5 - f)^2, 0.75 - (f - 1)^2 and 0.5 (f - 0.5)^2 expanded in f
    auto coef = [](int i, float& c2, float& c1, float& c0) {
        c2 = i == 1 ? -1.0f : 0.5f;
        c1 = i == 0 ? -1.5f : (i == 1 ? 2.0f : -0.5f);
        c0 = i == 0 ? 1.125f : (i == 1 ? -0.25f : 0.125f);
    };
    float cx2, cx1, cx0, cy2, cy1, cy0, cz2, cz1, cz0;
    coef(ni, cx2, cx1, cx0);
    coef(nj, cy2, cy1, cy0);
    coef(nk, cz2, cz1, cz0);
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int cur = -1;          // base cell of the open run, -1: none
    int pblk = -1, loc = 0; // the lane's node: physical block (from the table) and index in it
    auto flush = [&]() {
        if (node_lane) {
            if (pblk < 0)
                atomicOr(err, ST_MISSED);
            else
                atomicAdd(&target[(int64_t)pblk * 64 + loc], acc);
        }
    };
#pragma unroll 1
    for (int64_t base = begin; base < end; base += 32) {
        const int64_t p = base + lane;
        int key = -1;
        float4 r0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), r1 = r0, r2 = r0, r3 = r0;
        if (p < end) {
            P2GParticle q;
            if (prep(p, q)) {
                key = q.b[0] | (q.b[1] << 10) | (q.b[2] << 20);
                float c[3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    c[a] = q.mv[a] - (q.A[3 * a] * q.f[0] + q.A[3 * a + 1] * q.f[1] + q.A[3 * a + 2] * q.f[2]);
                r0 = make_float4(q.f[0], q.f[1], q.f[2], q.mp);
                r1 = make_float4(c[0], c[1], c[2], q.A[0]);
                r2 = make_float4(q.A[1], q.A[2], q.A[3], q.A[4]);
                r3 = make_float4(q.A[5], q.A[6], q.A[7], q.A[8]);
            }
        }
        __syncwarp();   // the previous batch is read
        s_rec[w][0][lane] = r0;
        s_rec[w][1][lane] = r1;
        s_rec[w][2][lane] = r2;
        s_rec[w][3][lane] = r3;
        s_key[w][lane] = key;
        __syncwarp();
        const int cnt = end - base < 32 ? (int)(end - base) : 32;
#pragma unroll 1
        for (int j = 0; j < cnt; ++j) {
            const int k = s_key[w][j];
            if (k < 0)
                continue;
            if (k != cur) {
                if (cur >= 0)
                    flush();
                cur = k;
                acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (node_lane) {
                    const int x = (k & 1023) + ni, y = ((k >> 10) & 1023) + nj, z = (k >> 20) + nk;
                    const uint32_t slot = spread3((uint32_t)(x >> 2)) | (spread3((uint32_t)(y >> 2)) << 1) |
                                          (spread3((uint32_t)(z >> 2)) << 2);
                    pblk = __ldg(&gv.table[slot]);
                    loc = (x & 3) + 4 * (y & 3) + 16 * (z & 3);
                }
            }
            const float4 a = s_rec[w][0][j], b = s_rec[w][1][j], c = s_rec[w][2][j], d = s_rec[w][3][j];
            const float wx = fmaf(fmaf(cx2, a.x, cx1), a.x, cx0);
            const float wy = fmaf(fmaf(cy2, a.y, cy1), a.y, cy0);
            const float wz = fmaf(fmaf(cz2, a.z, cz1), a.z, cz0);
            const float wt = wx * wy * wz;
            // A = (b.w, c.x, c.y; c.z, c.w, d.x; d.y, d.z, d.w), node value c + A n
            const float vx = fmaf(c.y, fk, fmaf(c.x, fj, fmaf(b.w, fi, b.x)));
            const float vy = fmaf(d.x, fk, fmaf(c.w, fj, fmaf(c.z, fi, b.y)));
            const float vz = fmaf(d.w, fk, fmaf(d.z, fj, fmaf(d.y, fi, b.z)));
            acc.x = fmaf(wt, vx, acc.x);
            acc.y = fmaf(wt, vy, acc.y);
            acc.z = fmaf(wt, vz, acc.z);
            acc.w = fmaf(wt, a.w, acc.w);
        }
    }
    if (cur >= 0)
        flush();
}

constexpr int kStageWaitIter = 1 << 16;

// ---- warp-level reduction before the global reductions (Sec. 4.2.2) ----------
// P2G_WARP: a warp takes 32 consecutive particles, one per lane, and groups
// the lanes whose particles share a base cell (and so the same 27 nodes).
// The paper sorts each warp's particles by a 10-bit cell key so that equal
// cells sit on consecutive lanes; here __match_any_sync finds the groups and
// each lane gets a position in a virtual order in which every group is
// contiguous (groups ordered by their lowest lane), so no particle data
// moves between lanes.  For each node the 32 contributions are reduced per
// group by a shuffle tree over those positions (log2 of the largest group
// steps, each lane adding the value of the lane d positions further on
// while that one is in its group); the group's first position then holds
// the sum and issues the one float4 reduction.  P2G_WARPRUN is the paper's
// "no sort" case: groups are only runs of equal cells on consecutive lanes.
constexpr uint32_t kFull = 0xffffffffu;

// Positions of the warp's lanes in the grouped order: pos (this lane's),
// end (one past its group), the source lane of position pos + 2^s for the
// tree steps s = 0..4 (6 bits each), and the largest group of the warp.
struct WarpGroups {
    int pos, end, lmax;
    bool head;      // pos is the group's first position
    uint32_t src;   // 5 x 6-bit lane indices
    __device__ __forceinline__ int src_of(int s) const { return (int)((src >> (6 * s)) & 63u); }
};

template <bool kGroup>
__device__ __forceinline__ WarpGroups warp_groups(uint32_t key, uint8_t* s_lane)
{
    const int lane = threadIdx.x & 31;
    WarpGroups g;
    if (kGroup) {
        const uint32_t eq = __match_any_sync(kFull, key);
        const int leader = __ffs(eq) - 1;
        const int size = __popc(eq);
        const int rank = __popc(eq & ((1u << lane) - 1u));
        // exclusive prefix, in lane order, of the group sizes held by the leaders
        const int mine = lane == leader ? size : 0;
        int incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, d);
            if (lane >= d)
                incl += t;
        }
        const int start = __shfl_sync(kFull, incl - mine, leader);
        g.pos = start + rank;
        g.end = start + size;
        g.head = rank == 0;
        s_lane[g.pos] = (uint8_t)lane;
        __syncwarp();
        uint32_t src = 0;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const int q = g.pos + (1 << s);
            src |= (uint32_t)(q < 32 ? s_lane[q] : lane) << (6 * s);
        }
        g.src = src;
        g.lmax = (int)__reduce_max_sync(kFull, (unsigned)size);
        __syncwarp();   // s_lane may be rewritten by the caller's next group
    } else {
        const uint32_t prev = __shfl_up_sync(kFull, key, 1);
        const uint32_t heads = __ballot_sync(kFull, lane == 0 || prev != key);
        const uint32_t le = lane == 31 ? kFull : ((2u << lane) - 1u);
        const int start = 31 - __clz(heads & le);
        const uint32_t above = heads & ~le;
        g.pos = lane;
        g.end = above ? __ffs(above) - 1 : 32;
        g.head = start == lane;
        uint32_t src = 0;
#pragma unroll
        for (int s = 0; s < 5; ++s)
            src |= (uint32_t)min(lane + (1 << s), 31) << (6 * s);
        g.src = src;
        g.lmax = (int)__reduce_max_sync(kFull, (unsigned)(g.end - start));
    }
    return g;
}

// Sum of v over this lane's group, left at the group's first position.
__device__ __forceinline__ float4 group_sum(float4 v, const WarpGroups& g)
{
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        if (g.lmax > (1 << s)) {   // warp-uniform
            const int src = g.src_of(s);
            float4 o;
            o.x = __shfl_sync(kFull, v.x, src);
            o.y = __shfl_sync(kFull, v.y, src);
            o.z = __shfl_sync(kFull, v.z, src);
            o.w = __shfl_sync(kFull, v.w, src);
            if (g.pos + (1 << s) < g.end) {
                v.x += o.x;
                v.y += o.y;
                v.z += o.z;
                v.w += o.w;
            }
        }
    }
    return v;
}

// The 27 contributions of q (zero for an invalid lane), reduced per group;
// the group's first position adds each sum into `target`.
__device__ __forceinline__ void warp_scatter(const GridView& gv, float4* target, const P2GParticle& q, bool ok,
                                             const WarpGroups& g, uint32_t* err)
{
    StencilIndex si;
    bool write = g.head && ok;
    if (write && !stencil_index(gv, q.b, si)) {
        atomicOr(err, ST_MISSED);
        write = false;
    }
    const float scale = ok ? 1.0f : 0.0f;
    p2g_contributions_centred(q, [&](int nidx, float wt, float vx, float vy, float vz, float m) {
        const float ws = wt * scale;
        float4 v = make_float4(ws * vx, ws * vy, ws * vz, ws * m);
        v = group_sum(v, g);
        if (write)
            atomicAdd(&target[si(nidx % 3, (nidx / 3) % 3, nidx / 9)], v);
    });
}

// A P2G record with zero weights and mass, for lanes without a particle.
__device__ __forceinline__ void clear_p2g_particle(P2GParticle& q)
{
    q.b[0] = q.b[1] = q.b[2] = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        q.f[a] = 1.0f;
        q.w[a][0] = q.w[a][1] = q.w[a][2] = 0.0f;
        q.mv[a] = 0.0f;
    }
    q.mp = 0.0f;
#pragma unroll
    for (int e = 0; e < 9; ++e)
        q.A[e] = 0.0f;
}

// Key of a particle's base cell (10 bits per axis: res <= 1024), or a key
// no valid particle has for an invalid lane.
__device__ __forceinline__ uint32_t cell_key(const int* b, bool ok, int lane)
{
    return ok ? ((uint32_t)b[0] | ((uint32_t)b[1] << 10) | ((uint32_t)b[2] << 20)) : (0x80000000u | (uint32_t)lane);
}

// Opts kernel `Kernel` into `bytes` of dynamic shared memory, once per
// kernel and device (the flag set is per instantiation, i.e. per kernel).
template <auto Kernel>
void smem_opt_in(size_t bytes)
{
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {
        cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        done.fetch_or(bit);
    }
}

// True if every node in [lo, hi] (per axis, clipped to the grid) lies in a
// mapped block.
__device__ __forceinline__ bool range_mapped(const SimParams& sp, const GridView& gv, const int* lo, const int* hi)
{
    int B0[3], B1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int l = max(lo[a], 0), h = min(hi[a], sp.res[a] - 1);
        B0[a] = l >> 2;
        B1[a] = h >> 2;
    }
    bool ok = true;
    for (int z = B0[2]; z <= B1[2]; ++z)
        for (int y = B0[1]; y <= B1[1]; ++y)
            for (int x = B0[0]; x <= B1[0]; ++x)
                ok = ok && __ldg(&gv.table[morton3((uint32_t)x, (uint32_t)y, (uint32_t)z)]) >= 0;
    return ok;
}

// Weights of one particle for G2P; false if its stencil left the grid.
template <class Get>
__device__ __forceinline__ bool g2p_weights_from(const SimParams& sp, Get get, float* x, int* b, float* f,
                                                 float (*w)[3], uint32_t* err)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x[a] = get(CH_X + a);
        b[a] = base_of(x[a], sp.inv_dx);
        f[a] = __fmul_rn(x[a], sp.inv_dx) - (float)b[a];
        bspline(f[a], w[a]);
    }
    if (!in_grid(sp, b, x)) {
        atomicOr(err, ST_EDOMAIN);
        return false;
    }
    return true;
}

template <bool kAoS = false>
__device__ __forceinline__ bool g2p_weights(const SimParams& sp, const PartView& pv, int64_t p, float* x, int* b,
                                            float* f, float (*w)[3], uint32_t* err)
{
    return g2p_weights_from(sp, [&](int c) { return pch<kAoS>(pv, c, p); }, x, b, f, w, err);
}

// Everything after the gather: C, x, v, the F update with the return map and
// the stress for the next P2G (or the fluid J update), and the free-zone test
// of Sec. 4.2.1.
// The particle after G2P, as the fused G2P2G kernel scatters it.
struct G2POut {
    float xn[3], vp[3], C[9], t6[6];
};

// get(c) reads input channel c (F - I, Jp - 1) of particle p; mat is its
// material.  Kind >= 0 asserts that every particle has a material of that
// kind (a single-material scene), so the constitutive code of the others
// drops out of the kernel.
template <bool kFused, int Kind, bool kAoS, class Get>
__device__ __forceinline__ bool g2p_finish_from(const SimParams& sp, const PartView& pv, const GridView& gv,
                                                int64_t p, Get get, int mat, const float* x, const int* b,
                                                int own_rank, const float* vp, const float* Bm, float dt,
                                                uint32_t* __restrict__ flags, uint32_t* __restrict__ err,
                                                G2POut* out, const float* va = nullptr)
{
    // va: the velocity that moves the particle, if not vp (ASFLIP)
    const float* adv = va ? va : vp;
    // C = (4 / dx^2) sum w v (x_i - x_p)^T = (4 / dx) sum w v (node - f)^T
    float C[9];
    float c4 = 4.0f * sp.inv_dx;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        C[e] = c4 * Bm[e];
        pch<kAoS>(pv, CH_C + e, p) = C[e];
    }
    float xn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xn[a] = x[a] + dt * adv[a];
        pch<kAoS>(pv, CH_X + a, p) = xn[a];
        pch<kAoS>(pv, CH_V + a, p) = vp[a];
    }
    MatParams m = sp.mat[mat];
    if (Kind >= 0)
        m.kind = Kind;
    float jm1 = get(CH_JP);
    float t6[6];
    if (m.kind == MPM_FLUID) {
        // J <- (1 + dt tr C) J, held as J - 1
        jm1 += dt * (C[0] + C[4] + C[8]) * (1.0f + jm1);
        pch<kAoS>(pv, CH_JP, p) = jm1;
        float Hdummy[9];
        constitutive_update(m, Hdummy, jm1, t6);
    } else {
        // F <- (I + dt C) F, i.e. H <- H + dt (C + C H)
        float H[9], Hn[9];
#pragma unroll
        for (int e = 0; e < 9; ++e)
            H[e] = get(CH_F + e);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Hn[3 * r + c] = H[3 * r + c] + dt * (C[3 * r + c] + C[3 * r] * H[c] + C[3 * r + 1] * H[3 + c] +
                                                     C[3 * r + 2] * H[6 + c]);
        float jn = jm1;
        constitutive_update(m, Hn, jn, t6);
#pragma unroll
        for (int e = 0; e < 9; ++e)
            pch<kAoS>(pv, CH_F + e, p) = Hn[e];
        if (m.kind == MPM_SNOW || m.kind == MPM_NACC)
            pch<kAoS>(pv, CH_JP, p) = jn;
    }
    if (kFused) {
        // the fused kernel scatters the new state at once: tau is not stored
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            out->xn[a] = xn[a];
            out->vp[a] = vp[a];
        }
#pragma unroll
        for (int e = 0; e < 9; ++e)
            out->C[e] = C[e];
#pragma unroll
        for (int e = 0; e < 6; ++e)
            out->t6[e] = t6[e];
    } else {
#pragma unroll
        for (int e = 0; e < 6; ++e)
            pch<kAoS>(pv, CH_TAU + e, p) = t6[e];
    }
    // Free-zone test (Sec. 4.2.1): while every particle's stencil stays in
    // mapped blocks no rebuild is needed.  A particle that changed cell
    // checks the stencil widened by kM cells per side; failing that asks for
    // a rebuild before the substep after next.  kM = 1 when the next P2G is
    // a separate launch (one substep of travel before it); kM = 2 for the
    // fused G2P2G, whose scatter already happens at the new position.  A new
    // base cell in an interior block (all 26 neighbours mapped) passes at
    // once; own_rank is the physical index of the old base cell's block
    // (-1 if the caller does not have it).
    int bn[3];
    bool moved = false, bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        bad = bad || !isfinite(xn[a]);
        bn[a] = base_of(xn[a], sp.inv_dx);
        moved = moved || bn[a] != b[a];
    }
    if (bad) {
        atomicOr(err, ST_ENONFINITE);
        return false;
    }
    if (moved) {
        constexpr int kM = kFused ? 2 : 1;
        bool dom = true;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            dom = dom && bn[a] >= 0 && bn[a] + 2 < sp.res[a] && ((bn[a] + 2) >> 2) < (1 << sp.L);
        if (!dom) {
            atomicOr(err, ST_EDOMAIN);
            return false;
        }
        const bool same_block = (bn[0] >> 2) == (b[0] >> 2) && (bn[1] >> 2) == (b[1] >> 2) && (bn[2] >> 2) == (b[2] >> 2);
        int rank = same_block ? own_rank : -1;
        if (rank < 0)
            rank = __ldg(&gv.table[morton3((uint32_t)bn[0] >> 2, (uint32_t)bn[1] >> 2, (uint32_t)bn[2] >> 2)]);
        int lo[3] = {bn[0] - kM, bn[1] - kM, bn[2] - kM}, hi[3] = {bn[0] + 2 + kM, bn[1] + 2 + kM, bn[2] + 2 + kM};
        if (!(rank >= 0 && __ldg(&gv.interior[rank])) && !range_mapped(sp, gv, lo, hi)) {
            int lo2[3] = {bn[0], bn[1], bn[2]}, hi2[3] = {bn[0] + 2, bn[1] + 2, bn[2] + 2};
            atomicOr(flags, range_mapped(sp, gv, lo2, hi2) ? ST_REBUILD_SOFT : (ST_REBUILD_SOFT | ST_REBUILD_HARD));
        }
    }
    return true;
}

template <bool kFused, int Kind = -1, bool kAoS = false>
__device__ __forceinline__ bool g2p_finish_t(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t p,
                                             const float* x, const int* b, int own_rank, const float* vp,
                                             const float* Bm, float dt, uint32_t* __restrict__ flags,
                                             uint32_t* __restrict__ err, G2POut* out)
{
    return g2p_finish_from<kFused, Kind, kAoS>(sp, pv, gv, p, [&](int c) { return pch<kAoS>(pv, c, p); }, pv.mat[p], x, b,
                                         own_rank, vp, Bm, dt, flags, err, out);
}

__device__ __forceinline__ void g2p_finish(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t p,
                                           const float* x, const int* b, int own_rank, const float* vp,
                                           const float* Bm, float dt, uint32_t* __restrict__ flags,
                                           uint32_t* __restrict__ err)
{
    g2p_finish_t<false>(sp, pv, gv, p, x, b, own_rank, vp, Bm, dt, flags, err, nullptr);
}

inline unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

}  // namespace mpm
