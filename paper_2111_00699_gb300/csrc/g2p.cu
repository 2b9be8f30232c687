// G2P of one MLS-MPM substep (Sec. 4): the gather of the updated grid
// velocities with the F update, the return mapping, the stress of the
// projected state and the free-zone test merged in (the SVD, projection and
// stress of Sec. 4.1 done once per substep), in the launch forms the
// autotuner chooses from; the ASFLIP form of the fountain scene (Sec. 6.5);
// and the stand-alone constitutive kernels used by the tests.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>
#include <type_traits>

#include "async_copy.cuh"
#include "device_math.cuh"
#include "internal.h"
#include "transfer.cuh"

namespace mpm {

namespace {


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
// occupancy.  Kind >= 0: the scene has one material, of that kind.  T: the
// CTA size (the same register cap for 64 or 256 threads per CTA).
// kSmemW: the particle's nine B-spline weights live in shared memory instead
// of registers (the paper's weight spilling, Sec. 3.2 / Sec. 6.2): each
// thread's 9 floats at stride 9 (no bank conflicts), read by the gather.
template <int MinBlocks, int Kind = -1, int T = kTransferThreads, bool kSmemW = false, bool kAoS = false>
__global__ void __launch_bounds__(T, MinBlocks * kTransferThreads / T) k_g2p_occ(SimParams sp, PartView pv, GridView gv,
                                                                        int64_t n, float dt,
                                                                        uint32_t* __restrict__ flags,
                                                                        uint32_t* __restrict__ err)
{
    __shared__ float s_w[kSmemW ? 9 * T : 1];
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    float x[3], f[3], wr[3][3];
    float (*w)[3] = kSmemW ? reinterpret_cast<float (*)[3]>(s_w + 9 * threadIdx.x) : wr;
    int b[3];
    if (!g2p_weights<kAoS>(sp, pv, p, x, b, f, w, err))
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
    g2p_finish_t<false, Kind, kAoS>(sp, pv, gv, p, x, b, si.pb64[0] >> 6, vp, Bm, dt, flags, err, nullptr);
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
    g2p_finish_from<false, -1, false>(sp, pv, gv, p, [&](int c) { return pv.ch(c)[p]; }, mat, x, b, si.pb64[0] >> 6, vn, Bm,
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
                g2p_finish_from<false, -1, false>(sp, pv, gv, p, get, smat[l], x, b, own_rank, vp, Bm, dt, flags, err, nullptr);
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


// G2P_OCC, specialised to the material kind when the scene has only one.
template <int T, bool kSmemW = false, bool kAoS = false, int MinBlocks = 8>
static void launch_g2p_occ_t(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt,
                             uint32_t* flags, uint32_t* err, cudaStream_t s)
{
    constexpr int B = MinBlocks;
    const unsigned g = blocks_for(n, T);
    switch (sp.n_mats == 1 ? sp.mat[0].kind : -1) {
    case MPM_ELASTIC: k_g2p_occ<B, MPM_ELASTIC, T, kSmemW, kAoS><<<g, T, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    case MPM_FLUID: k_g2p_occ<B, MPM_FLUID, T, kSmemW, kAoS><<<g, T, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    case MPM_SNOW: k_g2p_occ<B, MPM_SNOW, T, kSmemW, kAoS><<<g, T, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    case MPM_SAND: k_g2p_occ<B, MPM_SAND, T, kSmemW, kAoS><<<g, T, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    case MPM_NACC: k_g2p_occ<B, MPM_NACC, T, kSmemW, kAoS><<<g, T, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    case MPM_NHSAND: k_g2p_occ<B, MPM_NHSAND, T, kSmemW, kAoS><<<g, T, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    default: k_g2p_occ<B, -1, T, kSmemW, kAoS><<<g, T, 0, s>>>(sp, pv, gv, n, dt, flags, err); break;
    }
}

// G2P_OCC, specialised to the material kind when the scene has only one, in
// CTAs of sp.cta_warps warps (2, 4 or 8; 64 registers per thread in each).
static void launch_g2p_occ8(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt,
                            uint32_t* flags, uint32_t* err, cudaStream_t s)
{
    if (sp.cta_warps == 2)
        launch_g2p_occ_t<64>(sp, pv, gv, n, dt, flags, err, s);
    else if (sp.cta_warps == 8)
        launch_g2p_occ_t<256>(sp, pv, gv, n, dt, flags, err, s);
    else
        launch_g2p_occ_t<kTransferThreads>(sp, pv, gv, n, dt, flags, err, s);
}

void launch_g2p(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt, uint32_t* flags,
                uint32_t* err, int variant, cudaStream_t s)
{
    if (n > 0)
    {
        if (pv.aosoa) {   // the AoSoA store has the thread-per-particle forms 4, 6 and 7 only
            if (variant == G2P_OCC10)   // 48 registers, 10 CTAs of 128 per SM
                launch_g2p_occ_t<kTransferThreads, false, true, 10>(sp, pv, gv, n, dt, flags, err, s);
            else if (sp.cta_warps == 2) {
                if (variant == G2P_OCCSW)
                    launch_g2p_occ_t<64, true, true>(sp, pv, gv, n, dt, flags, err, s);
                else
                    launch_g2p_occ_t<64, false, true>(sp, pv, gv, n, dt, flags, err, s);
            } else if (variant == G2P_OCCSW) {
                launch_g2p_occ_t<kTransferThreads, true, true>(sp, pv, gv, n, dt, flags, err, s);
            } else {
                launch_g2p_occ_t<kTransferThreads, false, true>(sp, pv, gv, n, dt, flags, err, s);
            }
        }
        else if (sp.transfer == MPM_ASFLIP)
            k_g2p_asflip<<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
        else if (variant == G2P_STAGE && pv.cap % kCapQuantum == 0)
            k_g2p_stage<<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
        else if (variant == G2P_TILE)
            k_g2p_tile<<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
        else if (variant == G2P_OCC)
            launch_g2p_occ8(sp, pv, gv, n, dt, flags, err, s);
        else if (variant == G2P_OCCSW)
            launch_g2p_occ_t<kTransferThreads, true>(sp, pv, gv, n, dt, flags, err, s);
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
