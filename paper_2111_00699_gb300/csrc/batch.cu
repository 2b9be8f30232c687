// Batched substep: many small independent scenes advanced together.
//
// The paper's motivation for fewer, larger kernels (Sec. 3.1: minimise the
// kernels per step; Sec. 4.1: small kernels leave SMs idle, the tail effect)
// applied across scenes: S scenes of a few thousand particles each cost S x 3
// launches per substep when run one by one, and each of those launches is too
// small to fill the GPU.  Here every phase of the substep is one launch over
// the particles (or grid blocks) of all scenes, and the whole substep is
// replayed from a CUDA graph.
//
// Layout:
//  - particles of all scenes in one SoA store (the single-scene channel
//    layout), scene-contiguous; sid[p] names the scene of particle p;
//  - grid blocks are slot-indexed: scene s owns the block range
//    [slot_base_s, slot_base_s + 8^L_s) (one 1 KiB block per Morton code of
//    its domain), so remapping one scene never moves another scene's data;
//    mapped[slot] != 0 for the blocks of the current mapping;
//  - active[] lists the mapped blocks of all scenes (device-side count), the
//    grid update's work list.
// Rebuild-mapping (Sec. 4.2.1) is per scene: G2P sets the scene's bit when a
// particle's widened stencil reaches an unmapped block; the host acts on the
// bit two substeps later (the same lag argument as the single-scene path)
// and remaps only the flagged scenes.  Particles are sorted by (scene, block,
// cell) once, when they are added; remapping does not re-sort.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "device_math.cuh"
#include "internal.h"

using namespace mpm;

namespace mpm {
namespace {

struct SceneParams {
    int res[3];
    float dx, inv_dx;
    int boundary, wall;
    float g[3];
    int L;
    uint32_t slot_base;
    float dt;
    int64_t p_begin, p_end;
};

struct BatchView {
    const SceneParams* scenes;
    const MatParams* mats;
    const uint16_t* sid;
    const uint8_t* mapped;   // per slot
    float4* cur;             // slot-indexed grid, 64 nodes per slot
    float4* nxt;
    const int32_t* active;   // active slots
    const int32_t* n_active;
};

constexpr int kT = 128;
constexpr uint32_t kBatchFlagRing = 4;

inline unsigned nblk(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

__device__ __forceinline__ bool b_in_grid(const SceneParams& sc, const int* b, const float* x)
{
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        ok = ok && isfinite(x[a]) && b[a] >= 0 && b[a] + 2 < sc.res[a];
    return ok;
}

// Node indices of the stencil at base b in a scene's slot range: the 8
// candidate blocks B + {0,1}^3 (B = b >> 2) sit at slot_base + Morton(B + d);
// the +1 per axis is done on the dilated Morton bits.
__device__ __forceinline__ StencilIndex scene_stencil_index(const SceneParams& sc, const int* b)
{
    constexpr uint32_t kMx = 0x09249249u, kMy = kMx << 1, kMz = kMx << 2;
    const uint32_t sx0 = spread3((uint32_t)b[0] >> 2), sy0 = spread3((uint32_t)b[1] >> 2) << 1,
                   sz0 = spread3((uint32_t)b[2] >> 2) << 2;
    const uint32_t sx[2] = {sx0, ((sx0 | ~kMx) + 1u) & kMx}, sy[2] = {sy0, ((sy0 | ~kMy) + 1u) & kMy},
                   sz[2] = {sz0, ((sz0 | ~kMz) + 1u) & kMz};
    StencilIndex si;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        si.pb64[c] = (int)((sc.slot_base + (sx[c & 1] | sy[(c >> 1) & 1] | sz[c >> 2])) * 64u);
    si.bx = b[0] & 3;
    si.by = b[1] & 3;
    si.bz = b[2] & 3;
    return si;
}

__device__ __forceinline__ bool b_stencil_mapped(const SceneParams& sc, const BatchView& bv, const int* lo,
                                                 const int* hi)
{
    bool ok = true;
    int B0[3], B1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        B0[a] = max(lo[a], 0) >> 2;
        B1[a] = min(hi[a], sc.res[a] - 1) >> 2;
    }
    for (int z = B0[2]; z <= B1[2]; ++z)
        for (int y = B0[1]; y <= B1[1]; ++y)
            for (int x = B0[0]; x <= B1[0]; ++x)
                ok = ok && bv.mapped[sc.slot_base + morton3((uint32_t)x, (uint32_t)y, (uint32_t)z)] != 0;
    return ok;
}

// ---- rebuild-mapping ---------------------------------------------------------

// key = (global slot of the particle's block) << 6 | Morton(cell)
__global__ void bk_keys(const SceneParams* __restrict__ scenes, PartView pv, const uint16_t* __restrict__ sid,
                        int64_t n, uint32_t* __restrict__ keys, int32_t* __restrict__ vals, uint32_t* err)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    const SceneParams sc = scenes[sid[p]];
    int b[3];
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x[a] = pv.ch(CH_X + a)[p];
        b[a] = base_of(x[a], sc.inv_dx);
    }
    uint32_t key = 0xffffffffu;
    if (b_in_grid(sc, b, x)) {
        uint32_t slot = sc.slot_base + morton3((uint32_t)b[0] >> 2, (uint32_t)b[1] >> 2, (uint32_t)b[2] >> 2);
        key = (slot << 6) | morton3((uint32_t)b[0] & 3u, (uint32_t)b[1] & 3u, (uint32_t)b[2] & 3u);
    } else {
        atomicOr(err, ST_EDOMAIN);
    }
    keys[p] = key;
    vals[p] = (int32_t)p;
}

// Clear the mapping of the scenes listed in `which` (scene-per-CTA-row).
__global__ void bk_clear_mapped(const SceneParams* __restrict__ scenes, const int32_t* __restrict__ which,
                                uint8_t* __restrict__ mapped)
{
    const SceneParams sc = scenes[which[blockIdx.y]];
    int64_t slots = (int64_t)1 << (3 * sc.L);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += (int64_t)gridDim.x * blockDim.x)
        mapped[sc.slot_base + i] = 0;
}

// Mark the 3x3x3 neighbourhood of every particle's block, for the particles
// of the listed scenes (a particle whose block equals the previous
// particle's skips the marking).
__global__ void bk_mark(const SceneParams* __restrict__ scenes, const int32_t* __restrict__ which, PartView pv,
                        uint8_t* __restrict__ mapped)
{
    const SceneParams sc = scenes[which[blockIdx.y]];
    const int side = 1 << sc.L;
    for (int64_t p = sc.p_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < sc.p_end;
         p += (int64_t)gridDim.x * blockDim.x) {
        int B[3], P[3];
        bool ok = true, same = p > sc.p_begin;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float x = pv.ch(CH_X + a)[p];
            int b = base_of(x, sc.inv_dx);
            ok = ok && isfinite(x) && b >= 0 && b + 2 < sc.res[a];
            B[a] = b >> 2;
            if (same) {
                int bp = base_of(pv.ch(CH_X + a)[p - 1], sc.inv_dx);
                P[a] = bp >> 2;
                same = same && P[a] == B[a];
            }
        }
        if (!ok || same)
            continue;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int x = B[0] + dx, y = B[1] + dy, z = B[2] + dz;
                    if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side)
                        continue;
                    mapped[sc.slot_base + morton3((uint32_t)x, (uint32_t)y, (uint32_t)z)] = 1;
                }
    }
}

__global__ void bk_flags_to_int(const uint8_t* __restrict__ mapped, int64_t n_slots, int32_t* __restrict__ f)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n_slots)
        f[s] = mapped[s] ? 1 : 0;
}

__global__ void bk_active(const int32_t* __restrict__ f, const int32_t* __restrict__ rank, int64_t n_slots,
                          int32_t* __restrict__ active, int32_t* __restrict__ n_active)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slots)
        return;
    if (f[s])
        active[rank[s]] = (int32_t)s;
    if (s == n_slots - 1)
        *n_active = rank[s] + f[s];
}

// Zero both grid buffers on the mapped blocks of the listed scenes.
__global__ void bk_zero_scene_grid(const SceneParams* __restrict__ scenes, const int32_t* __restrict__ which,
                                   const uint8_t* __restrict__ mapped, float4* g0, float4* g1)
{
    const SceneParams sc = scenes[which[blockIdx.y]];
    int64_t nodes = ((int64_t)1 << (3 * sc.L)) * 64;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t slot = sc.slot_base + (i >> 6);
        if (mapped[slot]) {
            g0[slot * 64 + (i & 63)] = make_float4(0.f, 0.f, 0.f, 0.f);
            g1[slot * 64 + (i & 63)] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// ---- the substep ----------------------------------------------------------------

struct BParticle {
    int b[3];
    float f[3], w[3][3];
    float mp, mv[3], A[9];
};

__device__ __forceinline__ bool b_load(const SceneParams& sc, const BatchView& bv, const PartView& pv, int64_t p,
                                       BParticle& q, uint32_t* err)
{
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x[a] = pv.ch(CH_X + a)[p];
        q.b[a] = base_of(x[a], sc.inv_dx);
        q.f[a] = __fmul_rn(x[a], sc.inv_dx) - (float)q.b[a];
        bspline(q.f[a], q.w[a]);
    }
    if (!b_in_grid(sc, q.b, x)) {
        atomicOr(err, ST_EDOMAIN);
        return false;
    }
    float vol = pv.ch(CH_VOL)[p];
    q.mp = bv.mats[pv.mat[p]].rho * vol;
    float kst = 4.0f * sc.dt * vol * sc.inv_dx * sc.inv_dx;
    float t[6];
#pragma unroll
    for (int e = 0; e < 6; ++e)
        t[e] = kst * pv.ch(CH_TAU + e)[p];
    const float tm[9] = {t[0], t[3], t[4], t[3], t[1], t[5], t[4], t[5], t[2]};
#pragma unroll
    for (int e = 0; e < 9; ++e)
        q.A[e] = (q.mp * pv.ch(CH_C + e)[p] - tm[e]) * sc.dx;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        q.mv[a] = q.mp * pv.ch(CH_V + a)[p];
    return true;
}

// The chunk of K consecutive particles starting at p0 (< n): register runs
// per base cell, as the single-scene k_p2g_chunk, with the scene id part of
// the run key.
template <int K>
__device__ __forceinline__ void bk_p2g_chunk(const BatchView& bv, const PartView& pv, int64_t n, int64_t p0,
                                             uint32_t* __restrict__ err)
{
    if constexpr (K == 1) {
        // one particle: its 27 contributions go straight to the grid (no accumulators)
        const SceneParams sc = bv.scenes[bv.sid[p0]];
        BParticle q;
        if (!b_load(sc, bv, pv, p0, q, err))
            return;
        int lo[3] = {q.b[0], q.b[1], q.b[2]}, hi[3] = {q.b[0] + 2, q.b[1] + 2, q.b[2] + 2};
        if (!b_stencil_mapped(sc, bv, lo, hi)) {
            atomicOr(err, ST_MISSED);
            return;
        }
        const StencilIndex si = scene_stencil_index(sc, q.b);
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float dxo = (float)i - q.f[0], dyo = (float)jj - q.f[1], dzo = (float)k - q.f[2];
                    const float wt = q.w[0][i] * q.w[1][jj] * q.w[2][k];
                    float4 v;
                    v.x = wt * (q.mv[0] + q.A[0] * dxo + q.A[1] * dyo + q.A[2] * dzo);
                    v.y = wt * (q.mv[1] + q.A[3] * dxo + q.A[4] * dyo + q.A[5] * dzo);
                    v.z = wt * (q.mv[2] + q.A[6] * dxo + q.A[7] * dyo + q.A[8] * dzo);
                    v.w = wt * q.mp;
                    atomicAdd(&bv.cur[si(i, jj, k)], v);
                }
        return;
    } else {
        float4 acc[27];
    #pragma unroll
        for (int i = 0; i < 27; ++i)
            acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        int cb[3] = {0, 0, 0}, cs = -1;
        SceneParams sc;
    #pragma unroll 1
        for (int j = 0; j < K; ++j) {
            int64_t p = p0 + j;
            if (p >= n)
                break;
            int s = bv.sid[p];
            const SceneParams sp = bv.scenes[s];
            BParticle q;
            if (!b_load(sp, bv, pv, p, q, err))
                continue;
            bool change = cs >= 0 && (s != cs || q.b[0] != cb[0] || q.b[1] != cb[1] || q.b[2] != cb[2]);
            if (change) {
                int lo[3] = {cb[0], cb[1], cb[2]}, hi[3] = {cb[0] + 2, cb[1] + 2, cb[2] + 2};
                if (b_stencil_mapped(sc, bv, lo, hi)) {
                    const StencilIndex si = scene_stencil_index(sc, cb);
    #pragma unroll
                    for (int k = 0; k < 3; ++k)
    #pragma unroll
                        for (int jj = 0; jj < 3; ++jj)
    #pragma unroll
                            for (int i = 0; i < 3; ++i)
                                atomicAdd(&bv.cur[si(i, jj, k)], acc[i + 3 * jj + 9 * k]);
                } else {
                    atomicOr(err, ST_MISSED);
                }
    #pragma unroll
                for (int i = 0; i < 27; ++i)
                    acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            cs = s;
            sc = sp;
            cb[0] = q.b[0];
            cb[1] = q.b[1];
            cb[2] = q.b[2];
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
                for (int jj = 0; jj < 3; ++jj) {
                    float wyz = q.w[1][jj] * q.w[2][k];
                    float bx = q.mv[0] + q.A[1] * dyo[jj] + q.A[2] * dzo[k];
                    float by = q.mv[1] + q.A[4] * dyo[jj] + q.A[5] * dzo[k];
                    float bz = q.mv[2] + q.A[7] * dyo[jj] + q.A[8] * dzo[k];
    #pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        float wt = q.w[0][i] * wyz;
                        float4& a = acc[i + 3 * jj + 9 * k];
                        a.x += wt * (bx + q.A[0] * dxo[i]);
                        a.y += wt * (by + q.A[3] * dxo[i]);
                        a.z += wt * (bz + q.A[6] * dxo[i]);
                        a.w += wt * q.mp;
                    }
                }
        }
        if (cs >= 0) {
            int lo[3] = {cb[0], cb[1], cb[2]}, hi[3] = {cb[0] + 2, cb[1] + 2, cb[2] + 2};
            if (b_stencil_mapped(sc, bv, lo, hi)) {
                const StencilIndex si = scene_stencil_index(sc, cb);
    #pragma unroll
                for (int k = 0; k < 3; ++k)
    #pragma unroll
                    for (int jj = 0; jj < 3; ++jj)
    #pragma unroll
                        for (int i = 0; i < 3; ++i)
                            atomicAdd(&bv.cur[si(i, jj, k)], acc[i + 3 * jj + 9 * k]);
            } else {
                atomicOr(err, ST_MISSED);
            }
        }
    }
}

// CTAs of T threads at the same registers per thread for each T (168 with
// the register runs, 80 for one particle per thread).
template <int K, int T>
__global__ void __launch_bounds__(T, (K == 1 ? 6 : 3) * kT / T) bk_p2g(BatchView bv, PartView pv, int64_t n,
                                                                      uint32_t* __restrict__ err)
{
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * K;
    if (p0 < n)
        bk_p2g_chunk<K>(bv, pv, n, p0, err);
}

template <int K>
__global__ void __maxnreg__(K == 1 ? 80 : 168) bk_p2g_w8(BatchView bv, PartView pv, int64_t n,
                                                         uint32_t* __restrict__ err)
{
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * K;
    if (p0 < n)
        bk_p2g_chunk<K>(bv, pv, n, p0, err);
}

// Grid update over the active blocks of all scenes; the count lives on the
// device (set by the last remap), so the launch covers a capacity bound and
// surplus threads exit.
__device__ __forceinline__ void bk_grid_node(const BatchView& bv, const int32_t* __restrict__ ascene, int64_t idx)
{
    {
        int ai = (int)(idx >> 6);
        int l = (int)(idx & 63);
        int64_t slot = bv.active[ai];
        const SceneParams sc = bv.scenes[ascene[ai]];
        int64_t g = slot * 64 + l;
        float4 m = bv.cur[g];
        bv.nxt[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        float v[3] = {0.f, 0.f, 0.f};
        if (m.w > 0.0f) {
            float im = 1.0f / m.w;
            v[0] = m.x * im + sc.dt * sc.g[0];
            v[1] = m.y * im + sc.dt * sc.g[1];
            v[2] = m.z * im + sc.dt * sc.g[2];
            uint32_t loc = (uint32_t)(slot - sc.slot_base);
            int c[3] = {4 * (int)compact3(loc) + (l & 3), 4 * (int)compact3(loc >> 1) + ((l >> 2) & 3),
                        4 * (int)compact3(loc >> 2) + (l >> 4)};
            if (sc.boundary == MPM_STICKY) {
                bool wall = false;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    wall = wall || c[a] < sc.wall || c[a] >= sc.res[a] - sc.wall;
                if (wall)
                    v[0] = v[1] = v[2] = 0.0f;
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (c[a] < sc.wall && v[a] < 0.0f)
                        v[a] = 0.0f;
                    if (c[a] >= sc.res[a] - sc.wall && v[a] > 0.0f)
                        v[a] = 0.0f;
                }
            }
        }
        bv.cur[g] = make_float4(v[0], v[1], v[2], m.w);
    }
}

__global__ void bk_grid(BatchView bv, const int32_t* __restrict__ ascene)
{
    const int64_t na = *bv.n_active;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < na * 64;
         idx += (int64_t)gridDim.x * blockDim.x)
        bk_grid_node(bv, ascene, idx);
}

__global__ void bk_active_scene(const SceneParams* __restrict__ scenes, int n_scenes, const int32_t* __restrict__ active,
                                const int32_t* __restrict__ n_active, int32_t* __restrict__ ascene)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *n_active)
        return;
    uint32_t slot = (uint32_t)active[i];
    int lo = 0, hi = n_scenes - 1;
    while (lo < hi) {   // last scene whose slot_base <= slot
        int mid = (lo + hi + 1) >> 1;
        if (scenes[mid].slot_base <= slot)
            lo = mid;
        else
            hi = mid - 1;
    }
    ascene[i] = lo;
}

// G2P of particle p with the constitutive update of its scene's material.
__device__ __forceinline__ void bk_g2p_particle(const BatchView& bv, const PartView& pv, int64_t p,
                                                uint32_t* __restrict__ flags, uint32_t* __restrict__ err)
{
    const int s = bv.sid[p];
    const SceneParams sc = bv.scenes[s];
    float x[3], f[3], w[3][3];
    int b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x[a] = pv.ch(CH_X + a)[p];
        b[a] = base_of(x[a], sc.inv_dx);
        f[a] = __fmul_rn(x[a], sc.inv_dx) - (float)b[a];
        bspline(f[a], w[a]);
    }
    if (!b_in_grid(sc, b, x)) {
        atomicOr(err, ST_EDOMAIN);
        return;
    }
    int lo0[3] = {b[0], b[1], b[2]}, hi0[3] = {b[0] + 2, b[1] + 2, b[2] + 2};
    if (!b_stencil_mapped(sc, bv, lo0, hi0)) {
        atomicOr(err, ST_MISSED);
        return;
    }
    const StencilIndex si = scene_stencil_index(sc, b);
    float vp[3], Bm[9];
    g2p_accumulate(f, w, [&](int i, int j, int k) {
        const float4 g = bv.cur[si(i, j, k)];
        return make_float3(g.x, g.y, g.z);
    }, vp, Bm);
    float C[9];
    const float c4 = 4.0f * sc.inv_dx;
    const float dt = sc.dt;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        C[e] = c4 * Bm[e];
        pv.ch(CH_C + e)[p] = C[e];
    }
    float xn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xn[a] = x[a] + dt * vp[a];
        pv.ch(CH_X + a)[p] = xn[a];
        pv.ch(CH_V + a)[p] = vp[a];
    }
    const MatParams m = bv.mats[pv.mat[p]];
    float jm1 = pv.ch(CH_JP)[p];   // Jp - 1 (snow) or J - 1 (fluid)
    float t6[6];
    if (m.kind == MPM_FLUID) {
        jm1 += dt * (C[0] + C[4] + C[8]) * (1.0f + jm1);
        pv.ch(CH_JP)[p] = jm1;
        float Hd[9];
        constitutive_update(m, Hd, jm1, t6);
    } else {
        // H = F - I: F <- (I + dt C) F is H <- H + dt (C + C H)
        float H[9], Hn[9];
#pragma unroll
        for (int e = 0; e < 9; ++e)
            H[e] = pv.ch(CH_F + e)[p];
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
#pragma unroll
    for (int e = 0; e < 6; ++e)
        pv.ch(CH_TAU + e)[p] = t6[e];
    int bn[3];
    bool moved = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(xn[a])) {
            atomicOr(err, ST_ENONFINITE);
            return;
        }
        bn[a] = base_of(xn[a], sc.inv_dx);
        moved = moved || bn[a] != b[a];
    }
    if (moved) {
        bool dom = true;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            dom = dom && bn[a] >= 0 && bn[a] + 2 < sc.res[a];
        if (!dom) {
            atomicOr(err, ST_EDOMAIN);
            return;
        }
        int lo[3] = {bn[0] - 1, bn[1] - 1, bn[2] - 1}, hi[3] = {bn[0] + 3, bn[1] + 3, bn[2] + 3};
        if (!b_stencil_mapped(sc, bv, lo, hi))
            atomicOr(&flags[s >> 5], 1u << (s & 31));
    }
}

// Thread per particle, capped at 72 registers (7 CTAs of 128 per SM; the same
// cap for CTAs of 64 or 256 threads): with every material's constitutive code
// in one kernel this cap measured faster than 64 (8 CTAs) or 80 (6 CTAs)
// registers on the 256-scene batch.
template <int T>
__global__ void __launch_bounds__(T, 7 * kT / T) bk_g2p(BatchView bv, PartView pv, int64_t n,
                                                       uint32_t* __restrict__ flags, uint32_t* __restrict__ err)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n)
        bk_g2p_particle(bv, pv, p, flags, err);
}

__global__ void __maxnreg__(72) bk_g2p_w8(BatchView bv, PartView pv, int64_t n, uint32_t* __restrict__ flags,
                                          uint32_t* __restrict__ err)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n)
        bk_g2p_particle(bv, pv, p, flags, err);
}

// ---- the persistent form: one launch per substep ------------------------------
// A cooperative launch (every CTA resident at once) runs the three phases of
// the substep over all scenes: CTAs take work items (tiles of particles, or
// of active grid nodes) from a device counter per phase, so that tiles of
// uneven scenes spread over the SMs, and meet at a grid-wide barrier between
// the phases.  The barrier's wait is bounded: after kBarrierSpin polls a CTA
// records ST_TIMEOUT and returns (the others then time out at their next
// barrier), and the host reports MPM_ETIMEOUT.  The counters are zeroed
// before each launch.
struct PersistCtl {
    unsigned count, gen;   // grid barrier: arrivals, generation
    unsigned q[3];         // next tile of each phase
    unsigned pad[3];
};

constexpr int kBarrierSpin = 1 << 22;   // polls of ~256 ns: ~1 s

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* a)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(PersistCtl* c, uint32_t* err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire_gpu(&c->gen);
        __threadfence();
        if (atomicAdd(&c->count, 1u) == gridDim.x - 1) {
            atomicExch(&c->count, 0u);
            __threadfence();
            atomicAdd(&c->gen, 1u);
        } else {
            int it = 0;
            while (ld_acquire_gpu(&c->gen) == g) {
                if (++it > kBarrierSpin) {
                    ok = 0;
                    atomicOr(err, ST_TIMEOUT);
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The next tile of a phase for this CTA (uniform across the CTA).
__device__ __forceinline__ int64_t next_tile(unsigned* q)
{
    __shared__ unsigned s_t;
    __syncthreads();   // the previous tile's s_t has been read by every thread
    if (threadIdx.x == 0)
        s_t = atomicAdd(q, 1u);
    __syncthreads();
    return (int64_t)s_t;
}

template <int K>
__global__ void __launch_bounds__(kT, K == 1 ? 7 : 3) bk_persist(BatchView bv, PartView pv, int64_t n,
                                                               const int32_t* __restrict__ ascene,
                                                               uint32_t* __restrict__ flags, int words,
                                                               uint32_t* __restrict__ err, PersistCtl* ctl)
{
    // this substep's flag words (cleared here instead of by a memset)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x)
        flags[i] = 0u;
    // P2G: tiles of kT chunks of K particles
    const int64_t chunks = (n + K - 1) / K;
    for (int64_t t = next_tile(&ctl->q[0]); t * kT < chunks; t = next_tile(&ctl->q[0])) {
        const int64_t c = t * kT + threadIdx.x;
        if (c < chunks)
            bk_p2g_chunk<K>(bv, pv, n, c * K, err);
    }
    if (!grid_barrier(ctl, err))
        return;
    // grid update: tiles of 8 kT nodes
    const int64_t nodes = (int64_t)*bv.n_active * 64;
    for (int64_t t = next_tile(&ctl->q[1]); t * 8 * kT < nodes; t = next_tile(&ctl->q[1])) {
#pragma unroll 1
        for (int r = 0; r < 8; ++r) {
            const int64_t idx = (t * 8 + r) * kT + threadIdx.x;
            if (idx < nodes)
                bk_grid_node(bv, ascene, idx);
        }
    }
    if (!grid_barrier(ctl, err))
        return;
    // G2P: tiles of kT particles
    for (int64_t t = next_tile(&ctl->q[2]); t * kT < n; t = next_tile(&ctl->q[2])) {
        const int64_t p = t * kT + threadIdx.x;
        if (p < n)
            bk_g2p_particle(bv, pv, p, flags, err);
    }
}

}  // namespace
}  // namespace mpm

// ---- host side ----------------------------------------------------------------------

struct mpm_batch {
    int S = 0;
    cudaStream_t stream = nullptr;
    mpm_allocator alloc{};
    bool have_alloc = false;
    std::vector<mpm::SceneParams> hscenes;
    std::vector<mpm::MatParams> hmats;
    std::vector<std::vector<float>> pend_x, pend_v, pend_vol;   // particles added, per scene
    std::vector<int> pend_mat;
    mpm::SceneParams* dscenes = nullptr;
    mpm::MatParams* dmats = nullptr;
    int64_t n = 0, n_slots = 0;
    int key_bits = 0;
    void* pbuf[2] = {nullptr, nullptr};
    size_t pbuf_bytes = 0;
    mpm::PartView pv[2]{};
    int cur = 0;
    uint16_t* sid = nullptr;
    uint8_t* mapped = nullptr;
    int32_t *fl = nullptr, *rank = nullptr, *active = nullptr, *ascene = nullptr, *n_active = nullptr;
    int32_t* which = nullptr;   // device list of scenes to remap
    void* scan_scr = nullptr;
    size_t scan_bytes = 0;
    float4* grid[2] = {nullptr, nullptr};
    int gcur = 0;
    uint32_t* keys = nullptr;
    int32_t* vals = nullptr;
    uint32_t* skeys = nullptr;
    int32_t* svals = nullptr;
    void* sort_scr = nullptr;
    size_t sort_bytes = 0;
    uint32_t* dstat = nullptr;   // [0] errors, then kBatchFlagRing x words flag masks
    uint32_t* hstat = nullptr;
    int words = 0;
    cudaEvent_t ev[mpm::kBatchFlagRing] = {};
    int64_t step = 0, last_remap = -1;
    bool built = false;
    std::vector<int> need;       // scenes to remap before the next substep
    bool graphs = false;
    cudaGraphExec_t gexec[mpm::kBatchFlagRing] = {};
    int p2g_k = 4;
    int cta_warps = 4;            // CTA size of the per-phase P2G and G2P launches (2, 4 or 8 warps)
    bool persistent = false;      // one cooperative launch per substep instead of one per phase
    mpm::PersistCtl* ctl = nullptr;
    int persist_grid[3] = {0, 0, 0};   // CTAs of the cooperative launch, per chunk length 1 / 4 / 8
    int64_t launches = 0, remaps = 0, graph_launches = 0;
    std::string err;
    std::vector<std::pair<void*, size_t>> owned;
};

namespace {

using namespace mpm;

void* balloc(mpm_batch* b, size_t bytes)
{
    if (bytes == 0)
        bytes = 256;
    void* p = nullptr;
    if (b->have_alloc)
        p = b->alloc.alloc(bytes, (void*)b->stream, b->alloc.user);
    else if (cudaMallocAsync(&p, bytes, b->stream) != cudaSuccess)
        p = nullptr;
    if (p)
        b->owned.push_back({p, bytes});
    return p;
}

void bfree_all(mpm_batch* b)
{
    for (auto& o : b->owned) {
        if (b->have_alloc)
            b->alloc.free(o.first, o.second, (void*)b->stream, b->alloc.user);
        else
            cudaFreeAsync(o.first, b->stream);
    }
    b->owned.clear();
}

#define BCK(call)                                                                \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            b->err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
            return MPM_ECUDA;                                                    \
        }                                                                        \
    } while (0)

BatchView batch_view(mpm_batch* b)
{
    BatchView v;
    v.scenes = b->dscenes;
    v.mats = b->dmats;
    v.sid = b->sid;
    v.mapped = b->mapped;
    v.cur = b->grid[b->gcur];
    v.nxt = b->grid[1 - b->gcur];
    v.active = b->active;
    v.n_active = b->n_active;
    return v;
}

// Remap the scenes in `list` (all of them at the first build).
mpm_status remap(mpm_batch* b, const std::vector<int>& list)
{
    if (list.empty())
        return MPM_OK;
    cudaStream_t s = b->stream;
    BCK(cudaMemcpyAsync(b->which, list.data(), list.size() * 4, cudaMemcpyHostToDevice, s));
    dim3 g(64, (unsigned)list.size());
    bk_clear_mapped<<<g, 256, 0, s>>>(b->dscenes, b->which, b->mapped);
    bk_mark<<<g, 256, 0, s>>>(b->dscenes, b->which, b->pv[b->cur], b->mapped);
    bk_flags_to_int<<<nblk(b->n_slots, 256), 256, 0, s>>>(b->mapped, b->n_slots, b->fl);
    BCK(exclusive_scan(b->fl, b->rank, b->n_slots, b->scan_scr, s, &b->launches));
    bk_active<<<nblk(b->n_slots, 256), 256, 0, s>>>(b->fl, b->rank, b->n_slots, b->active, b->n_active);
    bk_active_scene<<<nblk(b->n_slots, 256), 256, 0, s>>>(b->dscenes, b->S, b->active, b->n_active, b->ascene);
    bk_zero_scene_grid<<<g, 256, 0, s>>>(b->dscenes, b->which, b->mapped, b->grid[0], b->grid[1]);
    b->launches += 7;
    BCK(cudaGetLastError());
    b->last_remap = b->step;
    b->remaps += 1;
    return MPM_OK;
}

// First build: upload the particles, sort them by (scene, block, cell), map all scenes.
mpm_status build(mpm_batch* b)
{
    cudaStream_t s = b->stream;
    int64_t n = 0;
    std::vector<int64_t> off(b->S + 1, 0);
    for (int i = 0; i < b->S; ++i) {
        off[i] = n;
        n += (int64_t)b->pend_x[i].size() / 3;
    }
    off[b->S] = n;
    if (n == 0)
        return MPM_EINVAL;
    b->n = n;
    int64_t cap = (n + 255) / 256 * 256;
    size_t pb = (size_t)cap * (kChannels * 4 + 1 + 4) + 512;
    for (int k = 0; k < 2; ++k) {
        b->pbuf[k] = balloc(b, pb);
        if (!b->pbuf[k])
            return MPM_ENOMEM;
        PartView v;
        v.soa = (float*)b->pbuf[k];
        v.cap = cap;
        v.id = (int32_t*)((char*)b->pbuf[k] + (size_t)cap * kChannels * 4);
        v.mat = (uint8_t*)((char*)v.id + (size_t)cap * 4);
        b->pv[k] = v;
    }
    b->pbuf_bytes = pb;
    b->sid = (uint16_t*)balloc(b, (size_t)cap * 2);
    b->keys = (uint32_t*)balloc(b, (size_t)cap * 4);
    b->vals = (int32_t*)balloc(b, (size_t)cap * 4);
    b->skeys = (uint32_t*)balloc(b, (size_t)cap * 4);
    b->svals = (int32_t*)balloc(b, (size_t)cap * 4);
    b->sort_bytes = radix_sort_scratch_bytes(cap);
    b->sort_scr = balloc(b, b->sort_bytes);
    if (!b->sid || !b->keys || !b->vals || !b->skeys || !b->svals || !b->sort_scr)
        return MPM_ENOMEM;
    // upload scene by scene (append kernel), then the scene ids
    std::vector<uint16_t> hsid((size_t)n);
    float* stage = (float*)balloc(b, (size_t)n * 7 * 4);
    if (!stage)
        return MPM_ENOMEM;
    for (int i = 0; i < b->S; ++i) {
        int64_t m = off[i + 1] - off[i];
        for (int64_t j = 0; j < m; ++j)
            hsid[(size_t)(off[i] + j)] = (uint16_t)i;
        b->hscenes[i].p_begin = off[i];
        b->hscenes[i].p_end = off[i + 1];
        if (m == 0)
            continue;
        float* sx = stage + 7 * off[i];
        BCK(cudaMemcpyAsync(sx, b->pend_x[i].data(), (size_t)m * 12, cudaMemcpyHostToDevice, s));
        BCK(cudaMemcpyAsync(sx + 3 * m, b->pend_v[i].data(), (size_t)m * 12, cudaMemcpyHostToDevice, s));
        BCK(cudaMemcpyAsync(sx + 6 * m, b->pend_vol[i].data(), (size_t)m * 4, cudaMemcpyHostToDevice, s));
        launch_append(b->pv[0], off[i], m, sx, sx + 3 * m, sx + 6 * m, 0.0f, b->pend_mat[i], s);
        b->launches += 1;
    }
    BCK(cudaMemcpyAsync(b->sid, hsid.data(), (size_t)n * 2, cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(b->dscenes, b->hscenes.data(), b->hscenes.size() * sizeof(SceneParams),
                        cudaMemcpyHostToDevice, s));
    // sort by (scene, block, cell): scene-contiguous, cell-sorted within
    bk_keys<<<nblk(n, 256), 256, 0, s>>>(b->dscenes, b->pv[0], b->sid, n, b->keys, b->vals, b->dstat);
    BCK(cudaMemcpyAsync(b->hstat, b->dstat, 4, cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    if (b->hstat[0] & ST_EDOMAIN) {
        b->err = "a particle's stencil lies outside its scene's grid";
        return MPM_EDOMAIN;   // an invalid key would break the scene-contiguous order
    }
    BCK(radix_sort_pairs(b->keys, b->vals, b->skeys, b->svals, n, b->key_bits, b->sort_scr, s, &b->launches));
    launch_permute(b->pv[0], b->pv[1], b->svals, n, s);
    b->launches += 2;
    b->cur = 1;
    BCK(cudaStreamSynchronize(s));
    for (auto& v : b->pend_x) std::vector<float>().swap(v);
    for (auto& v : b->pend_v) std::vector<float>().swap(v);
    for (auto& v : b->pend_vol) std::vector<float>().swap(v);
    std::vector<int> all(b->S);
    for (int i = 0; i < b->S; ++i)
        all[i] = i;
    mpm_status st = remap(b, all);
    if (st != MPM_OK)
        return st;
    b->built = true;
    return MPM_OK;
}

template <int T>
void enqueue_phases(mpm_batch* b, const BatchView& bv, uint32_t* flags, cudaStream_t s)
{
    const int64_t n = b->n;
    const PartView& pv = b->pv[b->cur];
    if constexpr (T == 256) {
        if (b->p2g_k == 8)
            bk_p2g_w8<8><<<nblk((n + 7) / 8, T), T, 0, s>>>(bv, pv, n, b->dstat);
        else if (b->p2g_k == 1)
            bk_p2g_w8<1><<<nblk(n, T), T, 0, s>>>(bv, pv, n, b->dstat);
        else
            bk_p2g_w8<4><<<nblk((n + 3) / 4, T), T, 0, s>>>(bv, pv, n, b->dstat);
    } else {
        if (b->p2g_k == 8)
            bk_p2g<8, T><<<nblk((n + 7) / 8, T), T, 0, s>>>(bv, pv, n, b->dstat);
        else if (b->p2g_k == 1)
            bk_p2g<1, T><<<nblk(n, T), T, 0, s>>>(bv, pv, n, b->dstat);
        else
            bk_p2g<4, T><<<nblk((n + 3) / 4, T), T, 0, s>>>(bv, pv, n, b->dstat);
    }
    bk_grid<<<152 * 8, 256, 0, s>>>(bv, b->ascene);
    if constexpr (T == 256)
        bk_g2p_w8<<<nblk(n, T), T, 0, s>>>(bv, pv, n, flags, b->dstat);
    else
        bk_g2p<T><<<nblk(n, T), T, 0, s>>>(bv, pv, n, flags, b->dstat);
}

// The cooperative launch of the persistent substep: as many CTAs of kT
// threads as fit on the device at once (all co-resident, as the grid
// barrier requires).
template <int K>
cudaError_t launch_persist(mpm_batch* b, const BatchView& bv, uint32_t* flags, cudaStream_t s)
{
    const int ki = K == 1 ? 0 : (K == 4 ? 1 : 2);
    if (b->persist_grid[ki] == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bk_persist<K>, kT, 0);
        if (e != cudaSuccess)
            return e;
        if (per_sm < 1)
            return cudaErrorCooperativeLaunchTooLarge;
        b->persist_grid[ki] = per_sm * sms;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)b->persist_grid[ki]);
    cfg.blockDim = dim3(kT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, bk_persist<K>, bv, b->pv[b->cur], b->n, (const int32_t*)b->ascene, flags,
                              b->words, b->dstat, b->ctl);
}

cudaError_t enqueue_step(mpm_batch* b, int slot)
{
    cudaStream_t s = b->stream;
    BatchView bv = batch_view(b);
    uint32_t* flags = &b->dstat[1 + slot * b->words];
    cudaError_t e = cudaSuccess;
    if (b->persistent) {
        // the kernel clears this substep's flag words itself
        e = cudaMemsetAsync(b->ctl, 0, sizeof(PersistCtl), s);
        if (e == cudaSuccess)
            e = b->p2g_k == 8 ? launch_persist<8>(b, bv, flags, s)
                              : (b->p2g_k == 1 ? launch_persist<1>(b, bv, flags, s) : launch_persist<4>(b, bv, flags, s));
        b->launches += 1;
    } else {
        e = cudaMemsetAsync(flags, 0, (size_t)b->words * 4, s);
        if (b->cta_warps == 2)
            enqueue_phases<64>(b, bv, flags, s);
        else if (b->cta_warps == 8)
            enqueue_phases<256>(b, bv, flags, s);
        else
            enqueue_phases<kT>(b, bv, flags, s);
        b->launches += 3;
    }
    cudaError_t e2 = cudaMemcpyAsync(&b->hstat[slot * b->words], flags, (size_t)b->words * 4, cudaMemcpyDeviceToHost, s);
    return e != cudaSuccess ? e : e2;
}

void drop_graphs(mpm_batch* b)
{
    for (int i = 0; i < (int)kBatchFlagRing; ++i)
        if (b->gexec[i]) {
            cudaGraphExecDestroy(b->gexec[i]);
            b->gexec[i] = nullptr;
        }
}

}  // namespace

extern "C" {

mpm_status mpm_batch_create(int n_scenes, const mpm_scene_desc* scenes, const mpm_material* mats, int n_mats,
                            const mpm_allocator* allocator, void* cuda_stream, mpm_batch** out)
{
    if (!out || !scenes || !mats || n_scenes < 1 || n_scenes > 65535 || n_mats < 1 || n_mats > 255)
        return MPM_EINVAL;
    *out = nullptr;
    if (allocator && (!allocator->alloc || !allocator->free))
        return MPM_EINVAL;
    for (int i = 0; i < n_mats; ++i) {
        const mpm_material& m = mats[i];
        if (m.kind < MPM_ELASTIC || m.kind > MPM_NHSAND || !(m.rho > 0.f) || !(m.E > 0.f) ||
            (m.kind != MPM_FLUID && !(m.nu > -1.f && m.nu < 0.5f)))
            return MPM_EINVAL;
    }
    mpm_batch* b = new (std::nothrow) mpm_batch();
    if (!b)
        return MPM_ENOMEM;
    b->S = n_scenes;
    b->stream = (cudaStream_t)cuda_stream;
    if (allocator) {
        b->alloc = *allocator;
        b->have_alloc = true;
    }
    b->hscenes.resize(n_scenes);
    uint64_t slots = 0;
    for (int i = 0; i < n_scenes; ++i) {
        const mpm_scene_desc& d = scenes[i];
        int maxres = 0;
        bool ok = d.dx > 0.f && d.wall >= 0 && (d.boundary == MPM_STICKY || d.boundary == MPM_SLIP) &&
                  d.material >= 0 && d.material < n_mats;
        for (int a = 0; a < 3; ++a) {
            ok = ok && d.res[a] >= 8 && d.res[a] <= 512;
            maxres = d.res[a] > maxres ? d.res[a] : maxres;
        }
        if (!ok) {
            delete b;
            return MPM_EINVAL;
        }
        SceneParams& sc = b->hscenes[i];
        memset(&sc, 0, sizeof(sc));
        for (int a = 0; a < 3; ++a) {
            sc.res[a] = d.res[a];
            sc.g[a] = d.gravity[a];
        }
        sc.dx = d.dx;
        sc.inv_dx = 1.0f / d.dx;
        sc.boundary = d.boundary;
        sc.wall = d.wall;
        int L = 0;
        while ((4 << L) < maxres)
            ++L;
        sc.L = L;
        sc.slot_base = (uint32_t)slots;
        sc.dt = 0.0f;
        slots += (uint64_t)1 << (3 * L);
    }
    int bits = 0;
    while (((uint64_t)1 << bits) < slots)
        ++bits;
    if (bits + 6 > 31) {   // sort keys (slot << 6 | cell) and node indices (slot * 64) stay below 2^31
        delete b;
        return MPM_ECAPACITY;
    }
    b->key_bits = bits + 6;
    b->n_slots = (int64_t)slots;
    for (int i = 0; i < n_mats; ++i)
        b->hmats.push_back(make_mat_params(mats[i]));
    b->pend_x.resize(n_scenes);
    b->pend_v.resize(n_scenes);
    b->pend_vol.resize(n_scenes);
    b->pend_mat.resize(n_scenes);
    for (int i = 0; i < n_scenes; ++i)
        b->pend_mat[i] = scenes[i].material;
    b->words = (n_scenes + 31) / 32;
    size_t ss = (size_t)slots;
    b->dscenes = (SceneParams*)balloc(b, sizeof(SceneParams) * n_scenes);
    b->dmats = (MatParams*)balloc(b, sizeof(MatParams) * n_mats);
    b->mapped = (uint8_t*)balloc(b, ss);
    b->fl = (int32_t*)balloc(b, ss * 4);
    b->rank = (int32_t*)balloc(b, ss * 4);
    b->active = (int32_t*)balloc(b, ss * 4);
    b->ascene = (int32_t*)balloc(b, ss * 4);
    b->n_active = (int32_t*)balloc(b, 256);
    b->which = (int32_t*)balloc(b, (size_t)n_scenes * 4);
    b->scan_bytes = scan_scratch_bytes((int64_t)slots);
    b->scan_scr = balloc(b, b->scan_bytes);
    b->grid[0] = (float4*)balloc(b, ss * 1024);
    b->grid[1] = (float4*)balloc(b, ss * 1024);
    b->dstat = (uint32_t*)balloc(b, (size_t)(1 + kBatchFlagRing * b->words) * 4);
    if (!b->dscenes || !b->dmats || !b->mapped || !b->fl || !b->rank || !b->active || !b->ascene || !b->n_active ||
        !b->which || !b->scan_scr || !b->grid[0] || !b->grid[1] || !b->dstat) {
        mpm_batch_destroy(b);
        return MPM_ENOMEM;
    }
    if (cudaMallocHost(&b->hstat, (size_t)kBatchFlagRing * b->words * 4 + 64) != cudaSuccess) {
        b->hstat = nullptr;
        mpm_batch_destroy(b);
        return MPM_ENOMEM;
    }
    memset(b->hstat, 0, (size_t)kBatchFlagRing * b->words * 4 + 64);
    for (int i = 0; i < (int)kBatchFlagRing; ++i)
        cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming);
    cudaStream_t s = b->stream;
    if (cudaMemcpyAsync(b->dmats, b->hmats.data(), sizeof(MatParams) * n_mats, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemsetAsync(b->dstat, 0, (size_t)(1 + kBatchFlagRing * b->words) * 4, s) != cudaSuccess ||
        cudaMemsetAsync(b->mapped, 0, ss, s) != cudaSuccess || cudaMemsetAsync(b->n_active, 0, 4, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        mpm_batch_destroy(b);
        return MPM_ECUDA;
    }
    *out = b;
    return MPM_OK;
}

void mpm_batch_destroy(mpm_batch* b)
{
    if (!b)
        return;
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    bfree_all(b);
    cudaStreamSynchronize(b->stream);
    if (b->hstat)
        cudaFreeHost(b->hstat);
    for (int i = 0; i < (int)kBatchFlagRing; ++i)
        if (b->ev[i])
            cudaEventDestroy(b->ev[i]);
    delete b;
}

mpm_status mpm_batch_add_particles(mpm_batch* b, int scene, int64_t n, const float* x, const float* v,
                                   const float* vol0)
{
    if (!b || scene < 0 || scene >= b->S || n < 0 || (n > 0 && !x))
        return MPM_EINVAL;
    if (b->built)
        return MPM_ENOTSUP;   // scenes are filled before the first substep
    const SceneParams& sc = b->hscenes[scene];
    auto& X = b->pend_x[scene];
    auto& V = b->pend_v[scene];
    auto& W = b->pend_vol[scene];
    X.insert(X.end(), x, x + 3 * n);
    if (v)
        V.insert(V.end(), v, v + 3 * n);
    else
        V.insert(V.end(), (size_t)3 * n, 0.0f);
    float dv = sc.dx * sc.dx * sc.dx / 8.0f;
    if (vol0)
        W.insert(W.end(), vol0, vol0 + n);
    else
        W.insert(W.end(), (size_t)n, dv);
    return MPM_OK;
}

mpm_status mpm_batch_substep(mpm_batch* b, const float* dt)
{
    TraceRange trace("mpm_batch_substep");
    if (!b || !dt)
        return MPM_EINVAL;
    bool dt_changed = false;
    for (int i = 0; i < b->S; ++i) {
        if (!(dt[i] > 0.f))
            return MPM_EINVAL;
        if (dt[i] != b->hscenes[i].dt) {
            b->hscenes[i].dt = dt[i];
            dt_changed = true;
        }
    }
    if (!b->built) {
        mpm_status st = build(b);   // uploads the scene table, dt included
        if (st != MPM_OK)
            return st;
    } else if (dt_changed) {
        // kernels (and captured graphs) read dt from the device scene table
        BCK(cudaMemcpyAsync(b->dscenes, b->hscenes.data(), b->hscenes.size() * sizeof(SceneParams),
                            cudaMemcpyHostToDevice, b->stream));
    }
    // per-scene flags of substep step - 2
    if (b->step >= 2 && b->step - 2 >= b->last_remap) {
        int slot = (int)((b->step - 2) % kBatchFlagRing);
        BCK(cudaEventSynchronize(b->ev[slot]));
        std::vector<int> list;
        for (int w = 0; w < b->words; ++w) {
            uint32_t m = b->hstat[slot * b->words + w];
            while (m) {
                int bit = __builtin_ctz(m);
                m &= m - 1;
                list.push_back(32 * w + bit);
            }
        }
        if (!list.empty()) {
            mpm_status st = remap(b, list);
            if (st != MPM_OK)
                return st;
        }
    }
    int slot = (int)(b->step % kBatchFlagRing);
    if (b->graphs) {
        // One graph per flag slot.  The grid buffers swap every substep and
        // the ring length is even, so the slot also fixes which buffer is
        // current; every pointer a graph captures is fixed after the build.
        static_assert(kBatchFlagRing % 2 == 0, "grid parity must repeat with the flag ring");
        int gi = slot;
        cudaGraph_t graph;
        if (!b->gexec[gi]) {
            BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            const cudaError_t ce = enqueue_step(b, slot);
            const cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
            BCK(ce);
            BCK(ee);
            cudaError_t e = cudaGraphInstantiate(&b->gexec[gi], graph, 0);
            cudaGraphDestroy(graph);
            BCK(e);
        }
        BCK(cudaGraphLaunch(b->gexec[gi], b->stream));
        b->graph_launches += 1;
        b->launches += b->persistent ? 1 : 3;
    } else {
        BCK(enqueue_step(b, slot));
    }
    BCK(cudaEventRecord(b->ev[slot], b->stream));
    BCK(cudaGetLastError());
    b->gcur = 1 - b->gcur;
    b->step += 1;
    return MPM_OK;
}

mpm_status mpm_batch_use_graphs(mpm_batch* b, int on)
{
    if (!b)
        return MPM_EINVAL;
    if (on && b->stream == nullptr) {
        b->err = "CUDA graphs need a stream other than the legacy default stream";
        return MPM_EINVAL;
    }
    if (!on)
        drop_graphs(b);
    b->graphs = on != 0;
    return MPM_OK;
}

mpm_status mpm_batch_set_cta_warps(mpm_batch* b, int warps)
{
    if (!b || (warps != 2 && warps != 4 && warps != 8))
        return MPM_EINVAL;
    if (warps != b->cta_warps)
        drop_graphs(b);
    b->cta_warps = warps;
    return MPM_OK;
}

mpm_status mpm_batch_set_persistent(mpm_batch* b, int on)
{
    if (!b || (on != 0 && on != 1))
        return MPM_EINVAL;
    if (on && !b->ctl) {
        b->ctl = (PersistCtl*)balloc(b, sizeof(PersistCtl));
        if (!b->ctl)
            return MPM_ENOMEM;
    }
    if ((on != 0) != b->persistent)
        drop_graphs(b);
    b->persistent = on != 0;
    return MPM_OK;
}

mpm_status mpm_batch_set_p2g_chunk(mpm_batch* b, int k)
{
    if (!b || (k != 1 && k != 4 && k != 8))
        return MPM_EINVAL;
    if (k != b->p2g_k)
        drop_graphs(b);
    b->p2g_k = k;
    return MPM_OK;
}

mpm_status mpm_batch_read_state(mpm_batch* b, int scene, float* x, float* v, float* C, float* F, float* Jp)
{
    if (!b || scene < 0 || scene >= b->S)
        return MPM_EINVAL;
    if (!b->built)
        return MPM_EINVAL;
    BCK(cudaStreamSynchronize(b->stream));
    const SceneParams& sc = b->hscenes[scene];
    int64_t m = sc.p_end - sc.p_begin;
    float* outs[5] = {x, v, C, F, Jp};
    static const int first[5] = {CH_X, CH_V, CH_C, CH_F, CH_JP};
    static const int width[5] = {3, 3, 9, 9, 1};
    static const int bias_step[5] = {0, 0, 0, 4, 1};   // F and Jp are held as F - I and Jp - 1
    // particles of a scene are stored contiguously; ids give insertion order
    std::vector<int32_t> id((size_t)m);
    const PartView& pv = b->pv[b->cur];
    if (m > 0)
        BCK(cudaMemcpy(id.data(), pv.id + sc.p_begin, (size_t)m * 4, cudaMemcpyDeviceToHost));
    std::vector<float> ch((size_t)m);
    for (int f = 0; f < 5; ++f) {
        if (!outs[f] || m == 0)
            continue;
        for (int e = 0; e < width[f]; ++e) {
            BCK(cudaMemcpy(ch.data(), pv.ch(first[f] + e) + sc.p_begin, (size_t)m * 4, cudaMemcpyDeviceToHost));
            const float bias = (bias_step[f] && e % bias_step[f] == 0) ? 1.0f : 0.0f;
            for (int64_t j = 0; j < m; ++j)
                outs[f][(int64_t)(id[(size_t)j] - sc.p_begin) * width[f] + e] = ch[(size_t)j] + bias;
        }
    }
    uint32_t errw = 0;
    BCK(cudaMemcpy(&errw, b->dstat, 4, cudaMemcpyDeviceToHost));
    if (errw & ST_TIMEOUT) {
        b->err = "a grid-wide barrier of the persistent substep gave up waiting";
        return MPM_ETIMEOUT;
    }
    if (errw & ST_ENONFINITE)
        return MPM_ENONFINITE;
    if (errw & (ST_EDOMAIN | ST_MISSED))
        return MPM_EDOMAIN;
    return MPM_OK;
}

mpm_status mpm_batch_sync(mpm_batch* b)
{
    if (!b)
        return MPM_EINVAL;
    BCK(cudaStreamSynchronize(b->stream));
    uint32_t errw = 0;
    BCK(cudaMemcpy(&errw, b->dstat, 4, cudaMemcpyDeviceToHost));
    if (errw & ST_TIMEOUT) {
        b->err = "a grid-wide barrier of the persistent substep gave up waiting";
        return MPM_ETIMEOUT;
    }
    if (errw & ST_ENONFINITE)
        return MPM_ENONFINITE;
    if (errw & (ST_EDOMAIN | ST_MISSED))
        return MPM_EDOMAIN;
    return MPM_OK;
}

mpm_status mpm_batch_get_stats(const mpm_batch* b, int64_t* out4)
{
    if (!b || !out4)
        return MPM_EINVAL;
    out4[0] = b->step;
    out4[1] = b->remaps;
    out4[2] = b->launches;
    out4[3] = b->graph_launches;
    return MPM_OK;
}

int64_t mpm_batch_num_particles(const mpm_batch* b, int scene)
{
    if (!b || scene < -1 || scene >= b->S)
        return 0;
    if (scene == -1) {
        if (b->built)
            return b->n;
        int64_t n = 0;
        for (auto& v : b->pend_x)
            n += (int64_t)v.size() / 3;
        return n;
    }
    if (b->built)
        return b->hscenes[scene].p_end - b->hscenes[scene].p_begin;
    return (int64_t)b->pend_x[scene].size() / 3;
}

const char* mpm_batch_last_error(const mpm_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
