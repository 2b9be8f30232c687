// The three essential phases of one MLS-MPM substep (Sec. 4): P2G, which
// scatters the Kirchhoff stress the previous G2P stored; the grid update
// with the boundary condition and the clearing of the next buffer merged in
// (Sec. 4.1); and G2P with the F update, the return mapping, the stress of
// the projected state and the free-zone test merged in (the SVD, projection
// and stress of Sec. 4.1 done once per substep).
//
// Layout: particles are SoA float channels (coalesced per warp); grid nodes
// are float4 (p_x, p_y, p_z, m) -- after the update (v_x, v_y, v_z, m) -- in
// physical blocks of 4x4x4 = 64 nodes, node (i, j, k) of a block at
// (i & 3) + 4 (j & 3) + 16 (k & 3).  A node's block index comes from the
// direct-mapped Morton table.  The default P2G adds into the grid with
// native global float4 reductions (Sec. 4.3 prefers native atomics to
// shared-memory float atomics); the shared-memory variants are kept for the
// ablation.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>
#include <type_traits>

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

__device__ __forceinline__ bool load_p2g_particle(const SimParams& sp, const PartView& pv, int64_t p, float dt,
                                                  P2GParticle& q, uint32_t* err)
{
    // a single-material scene needs no per-particle material index
    return make_p2g_particle(sp, [&](int c) { return pv.ch(c)[p]; }, sp.n_mats == 1 ? 0 : (int)pv.mat[p], dt, q, err);
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

constexpr int kTileThreads = 256;       // particles per CTA in the strided / tile variants
constexpr int kTileNodes = 2048;        // shared-memory tile capacity (nodes), 32 KB

// P2G_DIRECT: thread per particle in storage order.
__global__ void __launch_bounds__(kTransferThreads) k_p2g_direct(SimParams sp, PartView pv, GridView gv,
                                                                 int64_t n, float dt, uint32_t* __restrict__ err)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    P2GParticle q;
    if (load_p2g_particle(sp, pv, p, dt, q, err))
        scatter_global(gv, q, err);
}

// Lane L of warp w takes particle 8 L + w of the CTA's 256: after the cell
// sort, consecutive particles share cells (8 per cell), so this puts the 32
// lanes of a warp on ~32 different cells and their atomics on different
// addresses.
__device__ __forceinline__ int64_t strided_particle(int64_t base)
{
    return base + (int64_t)((threadIdx.x & 31) * 8 + (threadIdx.x >> 5));
}

__global__ void __launch_bounds__(kTileThreads) k_p2g_strided(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                              float dt, uint32_t* __restrict__ err)
{
    int64_t p = strided_particle((int64_t)blockIdx.x * kTileThreads);
    if (p >= n)
        return;
    P2GParticle q;
    if (load_p2g_particle(sp, pv, p, dt, q, err))
        scatter_global(gv, q, err);
}

// P2G_TILE: the CTA's 256 consecutive (cell-sorted) particles accumulate
// into a shared-memory tile spanning the bounding box of their stencils,
// then the touched nodes are flushed with one float4 global atomic each.
// A CTA whose box exceeds the tile falls back to direct atomics.
__global__ void __launch_bounds__(kTileThreads) k_p2g_tile(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                           float dt, uint32_t* __restrict__ err)
{
    __shared__ float tile[4][kTileNodes];
    __shared__ int box[6];
    const int tid = threadIdx.x;
    if (tid < 3) {
        box[tid] = 0x7fffffff;
        box[3 + tid] = -0x7fffffff;
    }
    __syncthreads();
    int64_t p = strided_particle((int64_t)blockIdx.x * kTileThreads);
    P2GParticle q;
    bool ok = p < n && load_p2g_particle(sp, pv, p, dt, q, err);
    if (ok) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&box[a], q.b[a]);
            atomicMax(&box[3 + a], q.b[a]);
        }
    }
    __syncthreads();
    const int lo0 = box[0], lo1 = box[1], lo2 = box[2];
    const int d0 = box[3] - lo0 + 3, d1 = box[4] - lo1 + 3, d2 = box[5] - lo2 + 3;
    const bool empty = box[3] < lo0;
    const int nodes = empty ? 0 : d0 * d1 * d2;
    if (nodes > kTileNodes) {
        if (ok)
            scatter_global(gv, q, err);
        return;   // uniform across the CTA: no barrier follows
    }
    for (int i = tid; i < nodes; i += kTileThreads) {
        tile[0][i] = 0.0f;
        tile[1][i] = 0.0f;
        tile[2][i] = 0.0f;
        tile[3][i] = 0.0f;
    }
    __syncthreads();
    if (ok) {
        const int o0 = q.b[0] - lo0, o1 = q.b[1] - lo1, o2 = q.b[2] - lo2;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    int idx = (o0 + i) + d0 * ((o1 + j) + d1 * (o2 + k));
                    float4 v = node_contribution(q, i, j, k);
                    atomicAdd(&tile[0][idx], v.x);
                    atomicAdd(&tile[1][idx], v.y);
                    atomicAdd(&tile[2][idx], v.z);
                    atomicAdd(&tile[3][idx], v.w);
                }
    }
    __syncthreads();
    for (int i = tid; i < nodes; i += kTileThreads) {
        float m = tile[3][i];
        if (!(m != 0.0f))
            continue;
        int x = lo0 + i % d0, y = lo1 + (i / d0) % d1, z = lo2 + i / (d0 * d1);
        int blk = __ldg(&gv.table[morton3((uint32_t)x >> 2, (uint32_t)y >> 2, (uint32_t)z >> 2)]);
        if (blk < 0) {
            atomicOr(err, ST_MISSED);
            continue;
        }
        int local = (x & 3) + 4 * (y & 3) + 16 * (z & 3);
        atomicAdd(&gv.cur[(int64_t)blk * 64 + local], make_float4(tile[0][i], tile[1][i], tile[2][i], m));
    }
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

template <int K, bool kSmem>
__global__ void __launch_bounds__(kTransferThreads, kSmem ? 4 : 3) k_p2g_chunk(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                                float dt, uint32_t* __restrict__ err)
{
    extern __shared__ float4 sacc[];
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * K;
    if (p0 >= n)
        return;
    typename std::conditional<kSmem, SmemAcc, NodeAcc>::type acc;
    if constexpr (kSmem)
        acc.base = sacc + threadIdx.x;
    acc_zero(acc);
    int cb[3] = {0, 0, 0};
    bool open = false;
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
        int64_t p = p0 + j;
        if (p >= n)
            break;
        P2GParticle q;
        if (!load_p2g_particle(sp, pv, p, dt, q, err))
            continue;
        if (open && (q.b[0] != cb[0] || q.b[1] != cb[1] || q.b[2] != cb[2])) {
            acc_flush(gv, gv.cur, acc, cb, err);
            acc_zero(acc);
            open = false;
        }
        if (!open) {
            cb[0] = q.b[0];
            cb[1] = q.b[1];
            cb[2] = q.b[2];
            open = true;
        }
        acc_add(acc, q);
    }
    if (open)
        acc_flush(gv, gv.cur, acc, cb, err);
}

// P2G_SLAB4: the register runs of k_p2g_chunk<4> split over three threads,
// one per z-slab of the stencil: 9 node accumulators (36 registers) instead
// of 27, so about twice the warps fit on an SM to hide the latency of the
// loads and reductions, for the price of evaluating each particle's weights
// and affine matrix three times.  CTA b takes chunk group b / 3 and slab
// b % 3: the three CTAs reading one group are launched back to back, so the
// second and third reads of the particles hit L2.
template <int K>
__global__ void __launch_bounds__(kTransferThreads, 5) k_p2g_slab(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                                  float dt, uint32_t* __restrict__ err)
{
    const int slab = (int)(blockIdx.x % 3u);
    const int64_t p0 = ((int64_t)(blockIdx.x / 3u) * blockDim.x + threadIdx.x) * K;
    if (p0 >= n)
        return;
    float4 acc[9];
#pragma unroll
    for (int m = 0; m < 9; ++m)
        acc[m] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int cb[3] = {0, 0, 0};
    bool open = false;
    auto flush = [&]() {
        StencilIndex si;
        if (!stencil_index(gv, cb, si)) {
            atomicOr(err, ST_MISSED);
            return;
        }
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                atomicAdd(&gv.cur[si(i, j, slab)], acc[i + 3 * j]);
    };
#pragma unroll 1
    for (int c = 0; c < K; ++c) {
        const int64_t p = p0 + c;
        if (p >= n)
            break;
        P2GParticle q;
        if (!load_p2g_particle(sp, pv, p, dt, q, err))
            continue;
        if (open && (q.b[0] != cb[0] || q.b[1] != cb[1] || q.b[2] != cb[2])) {
            flush();
#pragma unroll
            for (int m = 0; m < 9; ++m)
                acc[m] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            open = false;
        }
        if (!open) {
            cb[0] = q.b[0];
            cb[1] = q.b[1];
            cb[2] = q.b[2];
            open = true;
        }
        // this thread's slab k = slab: node (i, j, slab) receives
        // w (m v + A (node - f)) and w m, the affine term split per axis
        const float wz = slab == 0 ? q.w[2][0] : (slab == 1 ? q.w[2][1] : q.w[2][2]);
        const float dz = (float)slab - q.f[2];
        const float cx = q.mv[0] + q.A[2] * dz, cy = q.mv[1] + q.A[5] * dz, cz = q.mv[2] + q.A[8] * dz;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float dy = (float)j - q.f[1];
            const float wyz = q.w[1][j] * wz;
            const float bx = cx + q.A[1] * dy, by = cy + q.A[4] * dy, bz = cz + q.A[7] * dy;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float dx = (float)i - q.f[0];
                const float wt = q.w[0][i] * wyz;
                float4& a = acc[i + 3 * j];
                a.x = fmaf(wt, bx + q.A[0] * dx, a.x);
                a.y = fmaf(wt, by + q.A[3] * dx, a.y);
                a.z = fmaf(wt, bz + q.A[6] * dx, a.z);
                a.w = fmaf(wt, q.mp, a.w);
            }
        }
    }
    if (open)
        flush();
}

// P2G_STAGE4 / P2G_STAGE8: the chunked scatter of k_p2g_chunk, with the
// CTA's 128 K consecutive particles brought into shared memory first by one
// bulk asynchronous copy per channel (the TMA engine's 1-D form), issued by
// one thread and completed on an mbarrier.  The channel arrays are read
// once, fully coalesced and with all copies in flight together, and the
// per-particle loop then reads shared memory only.
constexpr int kStageThreads = 128;
constexpr int kStageCh = 22;   // x 3, v 3, C 9 (channels 0..14), vol, tau 6 (channels 25..31)
constexpr int kStageWaitIter = 1 << 16;

__host__ __device__ constexpr int stage_slot(int c) { return c < 15 ? c : c - 10; }
__host__ __device__ constexpr int stage_channel(int i) { return i < 15 ? i : i + 10; }

template <int K>
constexpr size_t stage_smem_bytes() { return (size_t)kStageThreads * K * (kStageCh * 4 + 1); }

template <int K>
__global__ void __launch_bounds__(kStageThreads) k_p2g_stage(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                             float dt, uint32_t* __restrict__ err)
{
    static_assert(stage_slot(CH_VOL) == 15 && stage_slot(CH_TAU) == 16 && stage_channel(21) == CH_TAU + 5, "slots");
    constexpr int T = kStageThreads * K;
    extern __shared__ __align__(128) float sm[];   // kStageCh x T floats, then T material bytes
    __shared__ __align__(8) uint64_t bar;
    uint8_t* smat = reinterpret_cast<uint8_t*>(sm + kStageCh * T);
    const int tid = threadIdx.x;
    const int64_t p0 = (int64_t)blockIdx.x * T;
    if (tid == 0)
        mbar_init(&bar, 1);
    __syncthreads();
    if (tid == 0) {
        // p0 + T <= cap (the capacity is a multiple of kCapQuantum): every
        // copy stays inside its channel array; entries past n are not used.
        mbar_arrive_expect_tx(&bar, (uint32_t)(T * (kStageCh * 4 + 1)));
#pragma unroll 1
        for (int i = 0; i < kStageCh; ++i)
            bulk_copy_g2s(sm + i * T, pv.ch(stage_channel(i)) + p0, T * 4, &bar);
        bulk_copy_g2s(smat, pv.mat + p0, T, &bar);
    }
    if (!mbar_wait(&bar, 0, kStageWaitIter)) {
        if (tid == 0)
            atomicOr(err, ST_TIMEOUT);
        mbar_wait(&bar, 0, kStageWaitIter);   // let copies still in flight land before the CTA exits
        return;
    }
    const int l0 = tid * K;
    if (p0 + l0 >= n)
        return;
    NodeAcc acc;
    acc_zero(acc);
    int cb[3] = {0, 0, 0};
    bool open = false;
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
        const int l = l0 + j;
        if (p0 + l >= n)
            break;
        P2GParticle q;
        if (!make_p2g_particle(sp, [&](int c) { return sm[stage_slot(c) * T + l]; }, smat[l], dt, q, err))
            continue;
        if (open && (q.b[0] != cb[0] || q.b[1] != cb[1] || q.b[2] != cb[2])) {
            acc_flush(gv, gv.cur, acc, cb, err);
            acc_zero(acc);
            open = false;
        }
        if (!open) {
            cb[0] = q.b[0];
            cb[1] = q.b[1];
            cb[2] = q.b[2];
            open = true;
        }
        acc_add(acc, q);
    }
    if (open)
        acc_flush(gv, gv.cur, acc, cb, err);
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

template <int K>
void launch_p2g_stage(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt,
                      uint32_t* err, cudaStream_t s)
{
    constexpr size_t bytes = stage_smem_bytes<K>();
    smem_opt_in<k_p2g_stage<K>>(bytes);
    constexpr int T = kStageThreads * K;
    k_p2g_stage<K><<<(unsigned)((n + T - 1) / T), kStageThreads, bytes, s>>>(sp, pv, gv, n, dt, err);
}

// Kirchhoff stress of the stored H = F - I and Jp - 1, for states P2G has
// not seen yet (after mpm_write_state).
__global__ void k_prepare_stress(SimParams sp, PartView pv, int64_t n)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    const MatParams m = sp.mat[pv.mat[p]];
    float H[9], t6[6];
#pragma unroll
    for (int e = 0; e < 9; ++e)
        H[e] = pv.ch(CH_F + e)[p];
    stress_h(m, H, pv.ch(CH_JP)[p], t6);
#pragma unroll
    for (int e = 0; e < 6; ++e)
        pv.ch(CH_TAU + e)[p] = t6[e];
}

__global__ void k_grid(SimParams sp, GridView gv, float dt)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx == 0 && gv.slot) {
        // clear this substep's status words before the G2P that sets them
        gv.slot[0] = 0u;
        gv.slot[1] = 0u;
    }
    if (idx >= (int64_t)gv.n_pblocks * 64)
        return;
    float4 g = gv.cur[idx];
    gv.nxt[idx] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float v[3] = {0.0f, 0.0f, 0.0f};
    if (g.w > 0.0f) {
        float im = 1.0f / g.w;
        v[0] = g.x * im + dt * sp.g[0];
        v[1] = g.y * im + dt * sp.g[1];
        v[2] = g.z * im + dt * sp.g[2];
        uint32_t s = (uint32_t)gv.pslot[idx >> 6];
        int l = (int)(idx & 63);
        int c[3] = {4 * (int)compact3(s) + (l & 3), 4 * (int)compact3(s >> 1) + ((l >> 2) & 3),
                    4 * (int)compact3(s >> 2) + (l >> 4)};
        if (sp.boundary == MPM_STICKY) {
            bool wall = false;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                wall = wall || c[a] < sp.wall || c[a] >= sp.res[a] - sp.wall;
            if (wall)
                v[0] = v[1] = v[2] = 0.0f;
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (c[a] < sp.wall && v[a] < 0.0f)
                    v[a] = 0.0f;
                if (c[a] >= sp.res[a] - sp.wall && v[a] > 0.0f)
                    v[a] = 0.0f;
            }
        }
    }
    gv.cur[idx] = make_float4(v[0], v[1], v[2], g.w);
    if (gv.old) {
        // ASFLIP: the grid velocity before forces and walls
        const float im = g.w > 0.0f ? 1.0f / g.w : 0.0f;
        gv.old[idx] = make_float4(g.x * im, g.y * im, g.z * im, 0.0f);
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

__device__ __forceinline__ bool g2p_weights(const SimParams& sp, const PartView& pv, int64_t p, float* x, int* b,
                                            float* f, float (*w)[3], uint32_t* err)
{
    return g2p_weights_from(sp, [&](int c) { return pv.ch(c)[p]; }, x, b, f, w, err);
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
template <bool kFused, int Kind, class Get>
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
        pv.ch(CH_C + e)[p] = C[e];
    }
    float xn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xn[a] = x[a] + dt * adv[a];
        pv.ch(CH_X + a)[p] = xn[a];
        pv.ch(CH_V + a)[p] = vp[a];
    }
    MatParams m = sp.mat[mat];
    if (Kind >= 0)
        m.kind = Kind;
    float jm1 = get(CH_JP);
    float t6[6];
    if (m.kind == MPM_FLUID) {
        // J <- (1 + dt tr C) J, held as J - 1
        jm1 += dt * (C[0] + C[4] + C[8]) * (1.0f + jm1);
        pv.ch(CH_JP)[p] = jm1;
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
            pv.ch(CH_F + e)[p] = Hn[e];
        if (m.kind == MPM_SNOW || m.kind == MPM_NACC)
            pv.ch(CH_JP)[p] = jn;
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
            pv.ch(CH_TAU + e)[p] = t6[e];
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

template <bool kFused, int Kind = -1>
__device__ __forceinline__ bool g2p_finish_t(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t p,
                                             const float* x, const int* b, int own_rank, const float* vp,
                                             const float* Bm, float dt, uint32_t* __restrict__ flags,
                                             uint32_t* __restrict__ err, G2POut* out)
{
    return g2p_finish_from<kFused, Kind>(sp, pv, gv, p, [&](int c) { return pv.ch(c)[p]; }, pv.mat[p], x, b,
                                         own_rank, vp, Bm, dt, flags, err, out);
}

__device__ __forceinline__ void g2p_finish(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t p,
                                           const float* x, const int* b, int own_rank, const float* vp,
                                           const float* Bm, float dt, uint32_t* __restrict__ flags,
                                           uint32_t* __restrict__ err)
{
    g2p_finish_t<false>(sp, pv, gv, p, x, b, own_rank, vp, Bm, dt, flags, err, nullptr);
}

__global__ void __launch_bounds__(kTransferThreads) k_g2p(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                          float dt, uint32_t* __restrict__ flags,
                                                          uint32_t* __restrict__ err)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    float x[3], f[3], w[3][3];
    int b[3];
    if (!g2p_weights(sp, pv, p, x, b, f, w, err))
        return;
    StencilIndex si;
    if (!stencil_index(gv, b, si)) {
        atomicOr(err, ST_MISSED);
        return;
    }
    float vp[3], Bm[9];
    g2p_accumulate(f, w, [&](int i, int j, int k) {
        const float4 g = gv.cur[si(i, j, k)];
        return make_float3(g.x, g.y, g.z);
    }, vp, Bm);
    g2p_finish(sp, pv, gv, p, x, b, si.pb64[0] >> 6, vp, Bm, dt, flags, err);
}

// G2P_OCC / G2P_OCC10: the thread-per-particle G2P capped at 64 (48)
// registers, 8 (10) CTAs of 128 per SM, trading register spills for
// occupancy.  Kind >= 0: the scene has one material, of that kind.
template <int MinBlocks, int Kind = -1>
__global__ void __launch_bounds__(kTransferThreads, MinBlocks) k_g2p_occ(SimParams sp, PartView pv, GridView gv,
                                                                        int64_t n, float dt,
                                                                        uint32_t* __restrict__ flags,
                                                                        uint32_t* __restrict__ err)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    float x[3], f[3], w[3][3];
    int b[3];
    if (!g2p_weights(sp, pv, p, x, b, f, w, err))
        return;
    StencilIndex si;
    if (!stencil_index(gv, b, si)) {
        atomicOr(err, ST_MISSED);
        return;
    }
    float vp[3], Bm[9];
    g2p_accumulate(f, w, [&](int i, int j, int k) {
        const float4 g = gv.cur[si(i, j, k)];
        return make_float3(g.x, g.y, g.z);
    }, vp, Bm);
    g2p_finish_t<false, Kind>(sp, pv, gv, p, x, b, si.pb64[0] >> 6, vp, Bm, dt, flags, err, nullptr);
}

// ASFLIP G2P (Fei et al. 2021, the integrator of the paper's fountain,
// Sec. 6.5).  Besides the APIC gather of the new grid velocity (vbar, C) it
// gathers v0, the grid velocity before forces, and blends in the particle's
// own deviation from it: v <- vbar + alpha (v - v0), and the particle moves
// with vbar + beta alpha (v - v0), beta = beta_min when the particle is
// compressed (J < 1 - m, m the configured margin, 0 by default) and beta_max
// otherwise.  J - 1 is formed from the small H = F - I (or is the fluid's
// tracked J - 1), so it carries the rounding of H, not of F.  C, F, J and the
// free-zone test are those of APIC.  One thread per particle at 64
// registers.
__global__ void __launch_bounds__(kTransferThreads, 8) k_g2p_asflip(SimParams sp, PartView pv, GridView gv,
                                                                   int64_t n, float dt,
                                                                   uint32_t* __restrict__ flags,
                                                                   uint32_t* __restrict__ err)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    float x[3], f[3], w[3][3];
    int b[3];
    if (!g2p_weights(sp, pv, p, x, b, f, w, err))
        return;
    StencilIndex si;
    if (!stencil_index(gv, b, si)) {
        atomicOr(err, ST_MISSED);
        return;
    }
    float vp[3], Bm[9];
    g2p_accumulate(f, w, [&](int i, int j, int k) {
        const float4 g = gv.cur[si(i, j, k)];
        return make_float3(g.x, g.y, g.z);
    }, vp, Bm);
    float v0[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float wjk = w[1][j] * w[2][k];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float4 g = gv.old[si(i, j, k)];
                const float wt = w[0][i] * wjk;
                v0[0] = fmaf(wt, g.x, v0[0]);
                v0[1] = fmaf(wt, g.y, v0[1]);
                v0[2] = fmaf(wt, g.z, v0[2]);
            }
        }
    // J - 1 before this G2P: the fluid's tracked J, else det(I + H) - 1
    // formed from H, so that its sign is that of the small quantity itself
    const int mat = pv.mat[p];
    float jm1;
    if (sp.mat[mat].kind == MPM_FLUID) {
        jm1 = pv.ch(CH_JP)[p];
    } else {
        float H[9];
#pragma unroll
        for (int e = 0; e < 9; ++e)
            H[e] = pv.ch(CH_F + e)[p];
        jm1 = det_m1(H);
    }
    const float beta = jm1 < -sp.flip_margin ? sp.flip_beta_min : sp.flip_beta_max;
    float vn[3], va[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float dv = pv.ch(CH_V + a)[p] - v0[a];
        vn[a] = fmaf(sp.flip_alpha, dv, vp[a]);
        va[a] = fmaf(beta * sp.flip_alpha, dv, vp[a]);
    }
    g2p_finish_from<false, -1>(sp, pv, gv, p, [&](int c) { return pv.ch(c)[p]; }, mat, x, b, si.pb64[0] >> 6, vn, Bm,
                           dt, flags, err, nullptr, va);
}

// G2P_TILE: shared-memory staging of the block-local grid tile.  The CTA's
// 128 consecutive (cell-sorted) particles span a small box of nodes; the CTA
// loads that box once, coalesced, into shared memory, and each particle then
// gathers its 27 nodes from shared memory (tens of cycles) instead of L2
// (hundreds).  A CTA whose box exceeds the tile gathers from global memory.
constexpr int kG2PTileNodes = 1024;   // 16 KB of float4

__global__ void __launch_bounds__(kTransferThreads) k_g2p_tile(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                               float dt, uint32_t* __restrict__ flags,
                                                               uint32_t* __restrict__ err)
{
    __shared__ float4 tile[kG2PTileNodes];
    __shared__ int box[6];
    __shared__ int tile_ok;
    const int tid = threadIdx.x;
    if (tid < 3) {
        box[tid] = 0x7fffffff;
        box[3 + tid] = -0x7fffffff;
    }
    if (tid == 0)
        tile_ok = 1;
    __syncthreads();
    int64_t p = (int64_t)blockIdx.x * blockDim.x + tid;
    float x[3], f[3], w[3][3];
    int b[3];
    bool ok = p < n && g2p_weights(sp, pv, p, x, b, f, w, err);
    if (ok) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&box[a], b[a]);
            atomicMax(&box[3 + a], b[a]);
        }
    }
    __syncthreads();
    const int lo0 = box[0], lo1 = box[1], lo2 = box[2];
    const int d0 = box[3] - lo0 + 3, d1 = box[4] - lo1 + 3, d2 = box[5] - lo2 + 3;
    const bool empty = box[3] < lo0;
    const int nodes = empty ? 0 : d0 * d1 * d2;
    const bool use_tile = nodes > 0 && nodes <= kG2PTileNodes;   // uniform across the CTA
    if (use_tile) {
        for (int i = tid; i < nodes; i += kTransferThreads) {
            int xx = lo0 + i % d0, yy = lo1 + (i / d0) % d1, zz = lo2 + i / (d0 * d1);
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            if (xx < sp.res[0] && yy < sp.res[1] && zz < sp.res[2]) {
                int blk = __ldg(&gv.table[morton3((uint32_t)xx >> 2, (uint32_t)yy >> 2, (uint32_t)zz >> 2)]);
                if (blk >= 0)
                    g = gv.cur[(int64_t)blk * 64 + (xx & 3) + 4 * (yy & 3) + 16 * (zz & 3)];
                else
                    tile_ok = 0;   // a node no particle should need is unmapped: checked per particle below
            }
            tile[i] = g;
        }
        __syncthreads();
    }
    if (!ok)
        return;
    float vp[3], Bm[9];
    if (use_tile) {
        // the particle's own stencil must be mapped (the tile holds zeros elsewhere)
        int pb[8];
        if (!tile_ok && !stencil_blocks(gv, b, pb)) {
            atomicOr(err, ST_MISSED);
            return;
        }
        const int o0 = b[0] - lo0, o1 = b[1] - lo1, o2 = b[2] - lo2;
        g2p_accumulate(f, w, [&](int i, int j, int k) {
            float4 g = tile[(o0 + i) + d0 * ((o1 + j) + d1 * (o2 + k))];
            return make_float3(g.x, g.y, g.z);
        }, vp, Bm);
    } else {
        StencilIndex si;
        if (!stencil_index(gv, b, si)) {
            atomicOr(err, ST_MISSED);
            return;
        }
        g2p_accumulate(f, w, [&](int i, int j, int k) {
            const float4 g = gv.cur[si(i, j, k)];
            return make_float3(g.x, g.y, g.z);
        }, vp, Bm);
    }
    g2p_finish(sp, pv, gv, p, x, b, -1, vp, Bm, dt, flags, err);
}

// G2P_STAGE: thread per particle, with the CTA's inputs brought into shared
// memory by bulk asynchronous copies (the TMA engine's 1-D form): the 128
// particles' x, F - I and Jp - 1 (one copy per channel) and the 2x2x2 grid
// blocks around the first particle's block (one 1 KB copy per block).  The
// particles are block-sorted, so most of a CTA gathers its 27 nodes from that
// tile; a particle whose stencil leaves it gathers from global memory.
constexpr int kG2PStageIn = 13;   // x (channels 0..2), F - I and Jp - 1 (channels 15..24)
__host__ __device__ constexpr int g2p_in_slot(int c) { return c < 3 ? c : c - 12; }
__host__ __device__ constexpr int g2p_in_channel(int i) { return i < 3 ? i : i + 12; }

__global__ void __launch_bounds__(kTransferThreads, 8) k_g2p_stage(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                                  float dt, uint32_t* __restrict__ flags,
                                                                  uint32_t* __restrict__ err)
{
    static_assert(g2p_in_slot(CH_F) == 3 && g2p_in_slot(CH_JP) == 12 && g2p_in_channel(12) == CH_JP, "slots");
    constexpr int T = kTransferThreads;
    __shared__ __align__(128) float sin[kG2PStageIn * T];
    __shared__ __align__(128) float4 tile[8 * 64];
    __shared__ __align__(16) uint8_t smat[T];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int home[3], home_mask, home_slot[8];
    const int tid = threadIdx.x;
    const int64_t p0 = (int64_t)blockIdx.x * T;
    const int64_t p = p0 + tid;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    if (tid == 0) {
        // particles: p0 + T <= cap (capacity is a multiple of kCapQuantum)
        mbar_arrive_expect_tx(&bar[0], (uint32_t)(T * (kG2PStageIn * 4 + 1)));
#pragma unroll 1
        for (int i = 0; i < kG2PStageIn; ++i)
            bulk_copy_g2s(sin + i * T, pv.ch(g2p_in_channel(i)) + p0, T * 4, &bar[0]);
        bulk_copy_g2s(smat, pv.mat + p0, T, &bar[0]);
        // grid tile: the 2x2x2 mapped blocks starting at the first particle's block
        float x0[3];
        int b0[3];
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x0[a] = pv.ch(CH_X + a)[p0];
            b0[a] = base_of(x0[a], sp.inv_dx);
        }
        ok = in_grid(sp, b0, x0);
        int mask = 0;
        if (ok) {
#pragma unroll 1
            for (int c = 0; c < 8; ++c) {
                int B[3] = {(b0[0] >> 2) + (c & 1), (b0[1] >> 2) + ((c >> 1) & 1), (b0[2] >> 2) + (c >> 2)};
                bool in = true;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    in = in && 4 * B[a] < sp.res[a] && B[a] < (1 << sp.L);
                int slot = in ? __ldg(&gv.table[morton3((uint32_t)B[0], (uint32_t)B[1], (uint32_t)B[2])]) : -1;
                home_slot[c] = slot;
                if (slot >= 0)
                    mask |= 1 << c;
            }
        }
        home[0] = b0[0] >> 2;
        home[1] = b0[1] >> 2;
        home[2] = b0[2] >> 2;
        home_mask = mask;
        mbar_arrive_expect_tx(&bar[1], (uint32_t)(__popc(mask) * 1024));
#pragma unroll 1
        for (int c = 0; c < 8; ++c)
            if (mask & (1 << c))
                bulk_copy_g2s(tile + 64 * c, gv.cur + (int64_t)home_slot[c] * 64, 1024, &bar[1]);
    }
    __syncthreads();
    bool ok = mbar_wait(&bar[0], 0, kStageWaitIter);
    if (ok && p < n) {
        const int l = tid;
        auto get = [&](int c) { return sin[g2p_in_slot(c) * T + l]; };
        float x[3], f[3], w[3][3];
        int b[3];
        if (g2p_weights_from(sp, get, x, b, f, w, err)) {
            int o[3];
            bool use_tile = true;
            int need = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = b[a] - 4 * home[a];
                use_tile = use_tile && o[a] >= 0 && o[a] <= 5;
            }
            if (use_tile) {
                // candidate blocks the stencil touches: per axis o >> 2 .. (o + 2) >> 2
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int d[3] = {c & 1, (c >> 1) & 1, c >> 2};
                    bool t = true;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        t = t && d[a] >= (o[a] >> 2) && d[a] <= ((o[a] + 2) >> 2);
                    need |= t ? (1 << c) : 0;
                }
                use_tile = (need & ~home_mask) == 0;
            }
            float vp[3], Bm[9];
            int own_rank = -1;
            bool have = true;
            if (use_tile && (ok = mbar_wait(&bar[1], 0, kStageWaitIter))) {
                StencilIndex ti;
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    ti.pb64[c] = 64 * c;
                ti.bx = o[0];
                ti.by = o[1];
                ti.bz = o[2];
                g2p_accumulate(f, w, [&](int i, int j, int k) {
                    const float4 g = tile[ti(i, j, k)];
                    return make_float3(g.x, g.y, g.z);
                }, vp, Bm);
                own_rank = home_slot[(o[0] >> 2) + 2 * (o[1] >> 2) + 4 * (o[2] >> 2)];
            } else if (ok) {
                StencilIndex si;
                if (!stencil_index(gv, b, si)) {
                    atomicOr(err, ST_MISSED);
                    have = false;
                } else {
                    g2p_accumulate(f, w, [&](int i, int j, int k) {
                        const float4 g = gv.cur[si(i, j, k)];
                        return make_float3(g.x, g.y, g.z);
                    }, vp, Bm);
                    own_rank = si.pb64[0] >> 6;
                }
            }
            if (ok && have)
                g2p_finish_from<false, -1>(sp, pv, gv, p, get, smat[l], x, b, own_rank, vp, Bm, dt, flags, err, nullptr);
        }
    }
    // no CTA exits with copies into its shared memory still in flight
    bool done0 = ok || mbar_wait(&bar[0], 0, kStageWaitIter);
    bool done1 = mbar_wait(&bar[1], 0, kStageWaitIter);
    if (!(ok && done0 && done1) && tid == 0)
        atomicOr(err, ST_TIMEOUT);
}

// A thread walks K consecutive particles (cell-sorted storage order) and keeps
// the 27 node velocities of the current base cell in registers, loading them
// again only when the base cell changes (about once per 8 particles after the
// sort), instead of 27 gathers per particle.
template <int K>
__global__ void __launch_bounds__(kTransferThreads) k_g2p_chunk(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                                float dt, uint32_t* __restrict__ flags,
                                                                uint32_t* __restrict__ err)
{
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * K;
    if (p0 >= n)
        return;
    float3 cache[27];
    int cb[3] = {-1, -1, -1};
    int own_rank = -1;
    bool have = false;
#pragma unroll 1
    for (int jj = 0; jj < K; ++jj) {
        int64_t p = p0 + jj;
        if (p >= n)
            break;
        float x[3], f[3], w[3][3];
        int b[3];
        if (!g2p_weights(sp, pv, p, x, b, f, w, err))
            continue;
        if (!have || b[0] != cb[0] || b[1] != cb[1] || b[2] != cb[2]) {
            StencilIndex si;
            if (!stencil_index(gv, b, si)) {
                atomicOr(err, ST_MISSED);
                have = false;
                continue;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const float4 g = gv.cur[si(i, j, k)];
                        cache[i + 3 * j + 9 * k] = make_float3(g.x, g.y, g.z);
                    }
            own_rank = si.pb64[0] >> 6;
            cb[0] = b[0];
            cb[1] = b[1];
            cb[2] = b[2];
            have = true;
        }
        float vp[3], Bm[9];
        g2p_accumulate(f, w, [&](int i, int j, int k) { return cache[i + 3 * j + 9 * k]; }, vp, Bm);
        g2p_finish(sp, pv, gv, p, x, b, own_rank, vp, Bm, dt, flags, err);
    }
}

// Fused G2P2G (Sec. 4.1: G2P of substep n and P2G of substep n + 1 in one
// kernel, the paper's choice below ~100K particles without particle
// addition): gather from gv.cur at x_n, update the particle (one SVD for the
// return map and the stress), write x, v, C, F, Jp, and build the new
// particle's P2G record at x_{n+1} for the scatter into gv.nxt, which must be
// zero (the grid update of this substep cleared it).
__device__ __forceinline__ bool g2p2g_particle(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t p,
                                               float dt, uint32_t* __restrict__ flags, uint32_t* __restrict__ err,
                                               P2GParticle& q)
{
    float x[3], f[3], w[3][3];
    int b[3];
    if (!g2p_weights(sp, pv, p, x, b, f, w, err))
        return false;
    StencilIndex si;
    if (!stencil_index(gv, b, si)) {
        atomicOr(err, ST_MISSED);
        return false;
    }
    float vp[3], Bm[9];
    g2p_accumulate(f, w, [&](int i, int j, int k) {
        const float4 g = gv.cur[si(i, j, k)];
        return make_float3(g.x, g.y, g.z);
    }, vp, Bm);
    G2POut o;
    if (!g2p_finish_t<true>(sp, pv, gv, p, x, b, si.pb64[0] >> 6, vp, Bm, dt, flags, err, &o))
        return false;
    // P2G record of the new state (same arithmetic as load_p2g_particle)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        q.b[a] = base_of(o.xn[a], sp.inv_dx);
        q.f[a] = __fmul_rn(o.xn[a], sp.inv_dx) - (float)q.b[a];
        bspline(q.f[a], q.w[a]);
    }
    if (!in_grid(sp, q.b, o.xn)) {
        atomicOr(err, ST_EDOMAIN);
        return false;
    }
    const float rho = sp.mat[pv.mat[p]].rho;
    float vol = pv.ch(CH_VOL)[p];
    q.mp = rho * vol;
    float kst = 4.0f * dt * vol * sp.inv_dx * sp.inv_dx;
    const float tm[9] = {o.t6[0], o.t6[3], o.t6[4], o.t6[3], o.t6[1], o.t6[5], o.t6[4], o.t6[5], o.t6[2]};
#pragma unroll
    for (int e = 0; e < 9; ++e)
        q.A[e] = (q.mp * o.C[e] - kst * tm[e]) * sp.dx;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        q.mv[a] = q.mp * o.vp[a];
    return true;
}

// Thread per particle, 27 float4 reductions per particle.
__global__ void __launch_bounds__(kTransferThreads) k_g2p2g(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                            float dt, uint32_t* __restrict__ flags,
                                                            uint32_t* __restrict__ err)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    P2GParticle q;
    if (g2p2g_particle(sp, pv, gv, p, dt, flags, err, q))
        scatter_to(gv, gv.nxt, q, err);
}

// The scatter of k_p2g_chunk inside the fused kernel: a thread walks K
// consecutive particles and accumulates the new particles' contributions in
// registers while their new base cells agree (particles move less than a
// cell per substep, so the cell sort still groups them), flushing 27 float4
// reductions into gv.nxt per run.
template <int K, bool kSmem>
__global__ void __launch_bounds__(kTransferThreads, kSmem ? 4 : 2) k_g2p2g_chunk(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                                  float dt, uint32_t* __restrict__ flags,
                                                                  uint32_t* __restrict__ err)
{
    extern __shared__ float4 sacc[];
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * K;
    if (p0 >= n)
        return;
    typename std::conditional<kSmem, SmemAcc, NodeAcc>::type acc;
    if constexpr (kSmem)
        acc.base = sacc + threadIdx.x;
    acc_zero(acc);
    int cb[3] = {0, 0, 0};
    bool open = false;
#pragma unroll 1
    for (int jj = 0; jj < K; ++jj) {
        int64_t p = p0 + jj;
        if (p >= n)
            break;
        P2GParticle q;
        if (!g2p2g_particle(sp, pv, gv, p, dt, flags, err, q))
            continue;
        if (open && (q.b[0] != cb[0] || q.b[1] != cb[1] || q.b[2] != cb[2])) {
            acc_flush(gv, gv.nxt, acc, cb, err);
            acc_zero(acc);
            open = false;
        }
        if (!open) {
            cb[0] = q.b[0];
            cb[1] = q.b[1];
            cb[2] = q.b[2];
            open = true;
        }
        acc_add(acc, q);
    }
    if (open)
        acc_flush(gv, gv.nxt, acc, cb, err);
}

// Debug kernels take F and Jp (or fluid J) as a user holds them and run the
// product's H = F - I formulation on them.
__global__ void k_debug_svd(const float* __restrict__ F, float* U, float* sig, float* V, int64_t n)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    float h[9];
#pragma unroll
    for (int e = 0; e < 9; ++e)
        h[e] = F[9 * p + e] - ((e % 4 == 0) ? 1.0f : 0.0f);
    SVDH d;
    svd_h(h, d);
    for (int e = 0; e < 9; ++e) {
        if (U) U[9 * p + e] = d.U[e];
        if (V) V[9 * p + e] = d.V[e];
    }
    if (sig)
        for (int e = 0; e < 3; ++e)
            sig[3 * p + e] = d.s[e];
}

__global__ void k_debug_stress(MatParams m, const float* __restrict__ F, const float* __restrict__ Jp,
                               float* __restrict__ tau, int64_t n)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    float h[9], t[6];
#pragma unroll
    for (int e = 0; e < 9; ++e)
        h[e] = F[9 * p + e] - ((e % 4 == 0) ? 1.0f : 0.0f);
    stress_h(m, h, Jp ? Jp[p] - 1.0f : 0.0f, t);
    const float full[9] = {t[0], t[3], t[4], t[3], t[1], t[5], t[4], t[5], t[2]};
#pragma unroll
    for (int e = 0; e < 9; ++e)
        tau[9 * p + e] = full[e];
}

__global__ void k_debug_plasticity(MatParams m, float* __restrict__ F, float* __restrict__ Jp, int64_t n)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    float h[9], t[6];
#pragma unroll
    for (int e = 0; e < 9; ++e)
        h[e] = F[9 * p + e] - ((e % 4 == 0) ? 1.0f : 0.0f);
    float jm1 = Jp ? Jp[p] - 1.0f : 0.0f;
    if (m.kind == MPM_SNOW || m.kind == MPM_SAND || m.kind == MPM_NACC || m.kind == MPM_NHSAND)
        constitutive_update(m, h, jm1, t);
#pragma unroll
    for (int e = 0; e < 9; ++e)
        F[9 * p + e] = h[e] + ((e % 4 == 0) ? 1.0f : 0.0f);
    if (Jp)
        Jp[p] = 1.0f + jm1;
}

inline unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

MatParams make_mat_params(const mpm_material& m)
{
    MatParams q{};
    q.kind = m.kind;
    q.rho = m.rho;
    double E = m.E, nu = m.nu;
    q.mu = (float)(E / (2.0 * (1.0 + nu)));
    q.la = (float)(E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
    if (m.kind == MPM_NACC) {
        // E is the bulk modulus kappa
        const double mu = 3.0 * E * (1.0 - 2.0 * nu) / (2.0 * (1.0 + nu));
        q.mu = (float)mu;
        q.la = (float)(E - 2.0 * mu / 3.0);
        q.M2 = m.friction_M * m.friction_M;
        q.beta = m.cohesion;
        q.alpha0 = m.alpha0;
    }
    q.K = m.E;
    q.gamma = m.gamma;
    q.lo_m1 = -m.theta_c;
    q.hi_m1 = m.theta_s;
    q.lo_b = (float)((1.0 - (double)m.theta_c) * (1.0 - (double)m.theta_c) - 1.0);
    q.hi_b = (float)((1.0 + (double)m.theta_s) * (1.0 + (double)m.theta_s) - 1.0);
    q.xi = m.hardening;
    double sphi = sin((double)m.friction_deg * 3.14159265358979323846 / 180.0);
    q.alpha = (float)(sqrt(2.0 / 3.0) * 2.0 * sphi / (3.0 - sphi));
    q.dp_coef = (float)((3.0 * q.la + 2.0 * q.mu) / (2.0 * q.mu));
    return q;
}

void launch_p2g(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt, uint32_t* err,
                int variant, cudaStream_t s)
{
    if (n <= 0)
        return;
    if ((variant == P2G_STAGE4 || variant == P2G_STAGE8) && pv.cap % kCapQuantum != 0)
        variant = variant == P2G_STAGE8 ? P2G_CHUNK8 : P2G_CHUNK4;   // staging needs whole tiles inside the arrays
    if (variant == P2G_STAGE8)
        launch_p2g_stage<8>(sp, pv, gv, n, dt, err, s);
    else if (variant == P2G_STAGE4)
        launch_p2g_stage<4>(sp, pv, gv, n, dt, err, s);
    else if (variant == P2G_SACC4) {
        smem_opt_in<k_p2g_chunk<4, true>>(kSmemAccBytes);
        k_p2g_chunk<4, true><<<blocks_for((n + 3) / 4, kTransferThreads), kTransferThreads, kSmemAccBytes, s>>>(
            sp, pv, gv, n, dt, err);
    } else if (variant == P2G_CHUNK8)
        k_p2g_chunk<8, false><<<blocks_for((n + 7) / 8, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt,
                                                                                                   err);
    else if (variant == P2G_CHUNK4)
        k_p2g_chunk<4, false><<<blocks_for((n + 3) / 4, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt,
                                                                                                   err);
    else if (variant == P2G_SLAB4)
        k_p2g_slab<4><<<3 * blocks_for((n + 3) / 4, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, err);
    else if (variant == P2G_STRIDED)
        k_p2g_strided<<<blocks_for(n, kTileThreads), kTileThreads, 0, s>>>(sp, pv, gv, n, dt, err);
    else if (variant == P2G_TILE)
        k_p2g_tile<<<blocks_for(n, kTileThreads), kTileThreads, 0, s>>>(sp, pv, gv, n, dt, err);
    else
        k_p2g_direct<<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, err);
}

void launch_prepare_stress(const SimParams& sp, const PartView& pv, int64_t n, cudaStream_t s)
{
    if (n > 0)
        k_prepare_stress<<<blocks_for(n, 128), 128, 0, s>>>(sp, pv, n);
}

void launch_grid_update(const SimParams& sp, const GridView& gv, float dt, cudaStream_t s)
{
    if (gv.n_pblocks > 0)
        k_grid<<<blocks_for((int64_t)gv.n_pblocks * 64, 256), 256, 0, s>>>(sp, gv, dt);
}

// G2P_OCC, specialised to the material kind when the scene has only one.
static void launch_g2p_occ8(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt,
                            uint32_t* flags, uint32_t* err, cudaStream_t s)
{
    const unsigned g = blocks_for(n, kTransferThreads);
    switch (sp.n_mats == 1 ? sp.mat[0].kind : -1) {
    case MPM_ELASTIC: k_g2p_occ<8, MPM_ELASTIC><<<g, kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    case MPM_FLUID: k_g2p_occ<8, MPM_FLUID><<<g, kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    case MPM_SNOW: k_g2p_occ<8, MPM_SNOW><<<g, kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    case MPM_SAND: k_g2p_occ<8, MPM_SAND><<<g, kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    case MPM_NACC: k_g2p_occ<8, MPM_NACC><<<g, kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    case MPM_NHSAND: k_g2p_occ<8, MPM_NHSAND><<<g, kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    default: k_g2p_occ<8><<<g, kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    }
}

void launch_g2p(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt, uint32_t* flags,
                uint32_t* err, int variant, cudaStream_t s)
{
    if (n > 0)
    {
        if (sp.transfer == MPM_ASFLIP)
            k_g2p_asflip<<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
        else if (variant == G2P_STAGE && pv.cap % kCapQuantum == 0)
            k_g2p_stage<<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
        else if (variant == G2P_TILE)
            k_g2p_tile<<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
        else if (variant == G2P_OCC)
            launch_g2p_occ8(sp, pv, gv, n, dt, flags, err, s);
        else if (variant == G2P_OCC10)
            k_g2p_occ<10><<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
        else if (variant == G2P_CHUNK8)
            k_g2p_chunk<8><<<blocks_for((n + 7) / 8, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt,
                                                                                                 flags, err);
        else if (variant == G2P_CHUNK4)
            k_g2p_chunk<4><<<blocks_for((n + 3) / 4, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt,
                                                                                                 flags, err);
        else
            k_g2p<<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
    }
}

void launch_debug_svd(const float* F, float* U, float* sig, float* V, int64_t n, cudaStream_t s)
{
    if (n > 0)
        k_debug_svd<<<blocks_for(n, 128), 128, 0, s>>>(F, U, sig, V, n);
}

void launch_debug_stress(const MatParams& mp, const float* F, const float* Jp, float* tau, int64_t n, cudaStream_t s)
{
    if (n > 0)
        k_debug_stress<<<blocks_for(n, 128), 128, 0, s>>>(mp, F, Jp, tau, n);
}

void launch_debug_plasticity(const MatParams& mp, float* F, float* Jp, int64_t n, cudaStream_t s)
{
    if (n > 0)
        k_debug_plasticity<<<blocks_for(n, 128), 128, 0, s>>>(mp, F, Jp, n);
}

}  // namespace mpm

namespace mpm {
void launch_g2p2g(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt, uint32_t* flags,
                  uint32_t* err, int p2g_variant, cudaStream_t s)
{
    if (n <= 0)
        return;
    // the scatter follows the P2G variant: register runs of 4 or 8 particles,
    // else one thread per particle
    if (p2g_variant == P2G_SACC4) {
        smem_opt_in<k_g2p2g_chunk<4, true>>(kSmemAccBytes);
        k_g2p2g_chunk<4, true><<<blocks_for((n + 3) / 4, kTransferThreads), kTransferThreads, kSmemAccBytes, s>>>(
            sp, pv, gv, n, dt, flags, err);
    } else if (p2g_variant == P2G_CHUNK8 || p2g_variant == P2G_STAGE8)
        k_g2p2g_chunk<8, false><<<blocks_for((n + 7) / 8, kTransferThreads), kTransferThreads, 0, s>>>(
            sp, pv, gv, n, dt, flags, err);
    else if (p2g_variant == P2G_CHUNK4 || p2g_variant == P2G_STAGE4)
        k_g2p2g_chunk<4, false><<<blocks_for((n + 3) / 4, kTransferThreads), kTransferThreads, 0, s>>>(
            sp, pv, gv, n, dt, flags, err);
    else
        k_g2p2g<<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
}
}  // namespace mpm
