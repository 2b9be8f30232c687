// The fused G2P2G transfer (Sec. 4.1): G2P of substep n and the P2G of
// substep n + 1 in one kernel, with each of the scatter forms of p2g.cu
// (thread per particle, register runs, shared-memory runs, the warp-level
// reduction of Sec. 4.2.2).
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

// The fused kernel with the warp-level reduction of k_p2g_warp as its
// scatter: each lane updates its own particle (G2P), then the lanes whose
// new base cells agree are grouped and their contributions to the 27 nodes
// reduced by the shuffle tree, one float4 reduction into gv.nxt per group
// and node.  No accumulators are held across particles, so the G2P state
// and the scatter share a register budget of 128.
template <bool kGroup>
__global__ void __launch_bounds__(kTransferThreads, 4) k_g2p2g_warp(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                                   float dt, uint32_t* __restrict__ flags,
                                                                   uint32_t* __restrict__ err)
{
    __shared__ uint8_t s_lane[kTransferThreads];
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    if (w0 >= n)
        return;   // whole warps
    const int64_t p = w0 + lane;
    P2GParticle q;
    const bool ok = p < n && g2p2g_particle(sp, pv, gv, p, dt, flags, err, q);
    if (!ok)
        clear_p2g_particle(q);
    const WarpGroups g = warp_groups<kGroup>(cell_key(q.b, ok, lane), s_lane + (threadIdx.x & ~31));
    warp_scatter(gv, gv.nxt, q, ok, g, err);
}


}  // namespace

void launch_g2p2g(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt, uint32_t* flags,
                  uint32_t* err, int p2g_variant, cudaStream_t s)
{
    if (n <= 0)
        return;
    // the scatter follows the P2G variant: register runs of 4 or 8 particles,
    // else one thread per particle
    if (p2g_variant == P2G_WARP || p2g_variant == P2G_WARPRUN) {
        const unsigned g = blocks_for(n, kTransferThreads);
        if (p2g_variant == P2G_WARP)
            k_g2p2g_warp<true><<<g, kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
        else
            k_g2p2g_warp<false><<<g, kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
    } else if (p2g_variant == P2G_SACC4) {
        smem_opt_in<k_g2p2g_chunk<4, true>>(kSmemAccBytes);
        k_g2p2g_chunk<4, true><<<blocks_for((n + 3) / 4, kTransferThreads), kTransferThreads, kSmemAccBytes, s>>>(
            sp, pv, gv, n, dt, flags, err);
    } else if (p2g_variant == P2G_CHUNK8 || p2g_variant == P2G_STAGE8 || p2g_variant == P2G_WTILE8)
        k_g2p2g_chunk<8, false><<<blocks_for((n + 7) / 8, kTransferThreads), kTransferThreads, 0, s>>>(
            sp, pv, gv, n, dt, flags, err);
    else if (p2g_variant == P2G_CHUNK4 || p2g_variant == P2G_STAGE4)
        k_g2p2g_chunk<4, false><<<blocks_for((n + 3) / 4, kTransferThreads), kTransferThreads, 0, s>>>(
            sp, pv, gv, n, dt, flags, err);
    else
        k_g2p2g<<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, flags, err);
}
}  // namespace mpm
