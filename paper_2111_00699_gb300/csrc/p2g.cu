// P2G of one MLS-MPM substep (Sec. 4): the scatter of each particle's
// mass and momentum, with the Kirchhoff stress the previous G2P stored
// (Sec. 4.1), into the blocked sparse grid, in the launch forms the
// autotuner chooses from; and the grid update with the boundary condition
// and the clearing of the next buffer merged in (Sec. 4.1).  The default
// P2G adds into the grid with native global float4 reductions (Sec. 4.3
// prefers native atomics to shared-memory float atomics); the shared-memory
// forms are kept for the ablations.
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


// With kSort, the order in which a thread takes its K particles, packed 4 bits
// per step: sorted by base cell (a bitonic network over the K keys), so that
// particles that drifted into a cell since the last sort join its run instead
// of splitting it.  Without kSort the storage order is taken (and 0 returned).
template <int K, bool kSort, bool kAoS>
__device__ __forceinline__ uint32_t chunk_order(const SimParams& sp, const PartView& pv, int64_t p0, int64_t n)
{
    static_assert(K <= 8, "4 bits per step");
    uint32_t order = 0;
    if constexpr (kSort) {
        uint32_t key[K];
        int idx[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            idx[j] = j;
            key[j] = 0xffffffffu;   // past the end: last
            if (p0 + j < n) {
                int b[3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    b[a] = base_of(pch<kAoS>(pv, CH_X + a, p0 + j), sp.inv_dx);
                key[j] = ((uint32_t)b[0] & 1023u) | (((uint32_t)b[1] & 1023u) << 10) | (((uint32_t)b[2] & 1023u) << 20);
            }
        }
#pragma unroll
        for (int size = 2; size <= K; size <<= 1)
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const int l = i ^ stride;
                    if (l > i) {
                        const bool up = (i & size) == 0;
                        if ((key[i] > key[l]) == up) {
                            const uint32_t tk = key[i];
                            key[i] = key[l];
                            key[l] = tk;
                            const int ti = idx[i];
                            idx[i] = idx[l];
                            idx[l] = ti;
                        }
                    }
                }
        order = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            order |= (uint32_t)idx[j] << (4 * j);
    }
    return order;
}

template <int K, bool kSmem, bool kAoS = false, bool kX2 = false, bool kSort = false>
__device__ __forceinline__ void p2g_chunk_body(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n,
                                               float dt, uint32_t* __restrict__ err)
{
    extern __shared__ float4 sacc[];
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * K;
    if (p0 >= n)
        return;
    const uint32_t order = chunk_order<K, kSort, kAoS>(sp, pv, p0, n);
    typename std::conditional<kSmem, SmemAcc, NodeAcc>::type acc;
    if constexpr (kSmem)
        acc.base = sacc + threadIdx.x;
    acc_zero(acc);
    int cb[3] = {0, 0, 0};
    bool open = false;
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
        int64_t p = p0 + (kSort ? (int)((order >> (4 * j)) & 15u) : j);
        if (p >= n)
            break;
        P2GParticle q;
        if (!load_p2g_particle<kAoS>(sp, pv, p, dt, q, err))
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
        if constexpr (kX2)
            acc_add_x2(acc, q);
        else
            acc_add(acc, q);
    }
    if (open)
        acc_flush(gv, gv.cur, acc, cb, err);
}

template <int K, bool kSmem, bool kAoS = false, bool kX2 = false>
__global__ void __launch_bounds__(kTransferThreads, kSmem ? 4 : 3) k_p2g_chunk(SimParams sp, PartView pv, GridView gv,
                                                                              int64_t n, float dt,
                                                                              uint32_t* __restrict__ err)
{
    p2g_chunk_body<K, kSmem, kAoS, kX2>(sp, pv, gv, n, dt, err);
}

// P2G_CHUNK8S: the register runs of 8 with each thread's chunk taken in the
// order of its particles' base cells.  Between sorts particles drift across
// cell faces, so the storage order interleaves a cell's particles with a few
// that moved in from next door and each of those splits a run; sorting the 8
// keys in registers (a bitonic network, about 100 instructions per chunk)
// makes every cell of the chunk one run.
template <int K, bool kAoS>
__global__ void __launch_bounds__(kTransferThreads, 3) k_p2g_chunks(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                                    float dt, uint32_t* __restrict__ err)
{
    p2g_chunk_body<K, false, kAoS, false, true>(sp, pv, gv, n, dt, err);
}

// The same register runs in CTAs of 2 or 8 warps instead of 4 (the paper's
// warps-per-block study, Sec. 6.2), at the same register budget per thread
// (168), so that only the CTA shape changes: 6 CTAs of 64 or one CTA of 256
// threads per SM (12 and 8 warps; 4 warps give 3 CTAs, 12 warps).
template <int K, bool kAoS = false>
__global__ void __launch_bounds__(64, 6) k_p2g_chunk_w2(SimParams sp, PartView pv, GridView gv, int64_t n, float dt,
                                                        uint32_t* __restrict__ err)
{
    p2g_chunk_body<K, false, kAoS>(sp, pv, gv, n, dt, err);
}

template <int K>
__global__ void __maxnreg__(168) k_p2g_chunk_w8(SimParams sp, PartView pv, GridView gv, int64_t n, float dt,
                                               uint32_t* __restrict__ err)
{
    p2g_chunk_body<K, false>(sp, pv, gv, n, dt, err);
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



template <bool kGroup>
__global__ void __launch_bounds__(kTransferThreads, 8) k_p2g_warp(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                                 float dt, uint32_t* __restrict__ err)
{
    __shared__ uint8_t s_lane[kTransferThreads];
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    if (w0 >= n)
        return;   // whole warps only: the lanes past n of the last warp take part as invalid lanes
    const int64_t p = w0 + lane;
    P2GParticle q;
    const bool ok = p < n && load_p2g_particle(sp, pv, p, dt, q, err);
    if (!ok)
        clear_p2g_particle(q);   // defined values for an invalid lane (its contributions are 0)
    const WarpGroups g = warp_groups<kGroup>(cell_key(q.b, ok, lane), s_lane + (threadIdx.x & ~31));
    warp_scatter(gv, gv.cur, q, ok, g, err);
}

// ---- node-parallel runs ----------------------------------------------------
// P2G_NODE: the work of a run spread over the stencil's nodes instead of its
// particles (node_runs in transfer.cuh): a warp takes its particles one at a
// time, lane l < 27 adding the particle's share of node l into one float4, so
// a lane holds one accumulator (64 registers, 8 CTAs per SM, against 168 and
// 3 for the register runs of one particle per thread), and a run ends in one
// warp instruction of 27 float4 reductions.  The price is separability: each
// lane forms its node's weight and value from scratch, about 21 arithmetic
// instructions per particle and node lane, where a register run shares the
// axis weights and row sums among a thread's 27 nodes (about 8 per node).
template <int NB, bool kAoS>
__global__ void __launch_bounds__(kTransferThreads, 8) k_p2g_node(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                                  float dt, uint32_t* __restrict__ err)
{
    node_runs<NB>(gv, gv.cur, n, [&](int64_t p, P2GParticle& q) { return load_p2g_particle<kAoS>(sp, pv, p, dt, q, err); },
                  err);
}

// ---- group sums through shared memory ---------------------------------------
// P2G_WXPOSE: a warp takes 32 consecutive particles, one per lane (the loads
// are one full line per channel, with no reuse to keep in L1), and groups
// the lanes whose particles share a base cell (__match_any_sync).  A lane
// alone in its group adds its 27 contributions to the grid directly.  The
// lanes of a group write theirs to a warp-private buffer, one z-slab of the
// stencil (9 nodes) at a time, and then split the slab's nodes among them:
// the member of rank r sums node r, r + s, ... over the s members and issues
// the one float4 reduction of that node.  The sums are plain shared-memory
// loads and adds (no shuffle tree, no shared atomics); each group's nodes
// reach L2 once, as with the paper's warp-level reduction.
constexpr int kXSlots = 9;   // nodes per pass (one z-slab); row stride 36 words: no bank conflicts

__global__ void __launch_bounds__(kTransferThreads, 8) k_p2g_wxpose(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                                   float dt, uint32_t* __restrict__ err)
{
    __shared__ float4 xbuf[kTransferThreads * kXSlots];
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    if (w0 >= n)
        return;   // whole warps
    const int64_t p = w0 + lane;
    P2GParticle q;
    const bool ok = p < n && load_p2g_particle(sp, pv, p, dt, q, err);
    if (!ok)
        clear_p2g_particle(q);
    const uint32_t eq = __match_any_sync(kFull, cell_key(q.b, ok, lane));
    const int gs = __popc(eq);
    const int rank = __popc(eq & ((1u << lane) - 1u));
    const bool single = gs == 1;
    StencilIndex si;
    bool mapped = ok;
    if (ok && !stencil_index(gv, q.b, si)) {
        atomicOr(err, ST_MISSED);
        mapped = false;
    }
    float4* rows = xbuf + (threadIdx.x & ~31) * kXSlots;   // this warp's 32 rows of 9 nodes
    const float scale = ok ? 1.0f : 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p2g_contributions_centred(q, [&](int nidx, float wt, float vx, float vy, float vz, float m) {
            if (nidx / 9 != k)
                return;   // another slab's node (resolved at compile time)
            const float ws = wt * scale;
            const float4 v = make_float4(ws * vx, ws * vy, ws * vz, ws * m);
            if (single) {
                if (mapped)
                    atomicAdd(&gv.cur[si(nidx % 3, (nidx / 3) % 3, k)], v);
            } else {
                rows[lane * kXSlots + nidx % 9] = v;
            }
        });
        __syncwarp();
        if (!single) {
#pragma unroll 1
            for (int t = rank; t < kXSlots; t += gs) {
                float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                uint32_t mm = eq;
#pragma unroll 1
                while (mm) {
                    const int m = __ffs(mm) - 1;
                    mm &= mm - 1u;
                    const float4 v = rows[m * kXSlots + t];
                    acc.x += v.x;
                    acc.y += v.y;
                    acc.z += v.z;
                    acc.w += v.w;
                }
                if (mapped)
                    atomicAdd(&gv.cur[si(t % 3, t / 3, k)], acc);
            }
        }
        __syncwarp();   // the slab's sums are read before the next slab overwrites the rows
    }
}

// ---- register runs into a warp-private node tile -----------------------------
// P2G_WTILE8: the register runs of k_p2g_chunk<8>, flushed into a node tile
// in shared memory private to the warp instead of into global memory; the
// warp then adds each touched node of its tile to the grid with one float4
// reduction.  A warp's 256 consecutive particles (cell-sorted) cover a few
// dozen cells, whose stencils share most of their nodes, so the global
// reductions per particle drop from ~6 (one set of 27 per run) to ~1, and a
// flush needs no block-table lookups.  Lanes flushing runs of different
// base cells reach distinct tile nodes at one node offset (i, j, k); lanes
// whose runs share a base cell (a cell split between two lanes' chunks)
// take turns; and the offsets follow one another with __syncwarp between
// them (a node can be another lane's other offset), so plain shared loads
// and stores suffice.  A warp whose box of base cells does not fit the tile
// flushes to global memory as k_p2g_chunk does.
constexpr int kWTileNodes = 512;   // 8 KB of float4 per warp

struct WarpTile {
    float4* t;       // this warp's tile
    int lo[3];       // smallest base cell of the warp's particles
    int d0, d01;     // tile extents: x, x * y
};

// Adds the 27 accumulators of the runs that end now (lanes with `flush`)
// into the warp's tile.  Called by every lane of the warp.
__device__ __forceinline__ void tile_flush(const WarpTile& wt, const NodeAcc& acc, const int* b, bool flush)
{
    const int lane = threadIdx.x & 31;
    const uint32_t key = cell_key(b, flush, lane);
    const uint32_t eq = __match_any_sync(kFull, key);
    const int rank = __popc(eq & ((1u << lane) - 1u));
    const int rounds = (int)__reduce_max_sync(kFull, flush ? (unsigned)rank + 1u : 0u);
    const int t0 = (b[0] - wt.lo[0]) + wt.d0 * (b[1] - wt.lo[1]) + wt.d01 * (b[2] - wt.lo[2]);
#pragma unroll 1
    for (int r = 0; r < rounds; ++r) {
        const bool go = flush && rank == r;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    if (go) {
                        float4* c = wt.t + (t0 + i + wt.d0 * j + wt.d01 * k);
                        float4 a = *c;
                        const float4 v = acc.a[i + 3 * j + 9 * k];
                        a.x += v.x;
                        a.y += v.y;
                        a.z += v.z;
                        a.w += v.w;
                        *c = a;
                    }
                    __syncwarp();
                }
    }
}

template <int K>
__global__ void __launch_bounds__(kTransferThreads, 3) k_p2g_wtile(SimParams sp, PartView pv, GridView gv, int64_t n,
                                                                  float dt, uint32_t* __restrict__ err)
{
    extern __shared__ float4 wtiles[];
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * K;
    if (w0 >= n)
        return;   // whole warps
    const int64_t p0 = w0 + (int64_t)lane * K;
    WarpTile wt;
    wt.t = wtiles + (threadIdx.x >> 5) * kWTileNodes;
    // box of the base cells of the warp's particles (positions outside the
    // grid or non-finite are left to the scatter's own checks: they make the
    // box too large, and the warp takes the global path)
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
    bool finite = true;
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
        const int64_t p = p0 + j;
        if (p >= n)
            break;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float xa = pv.ch(CH_X + a)[p];
            finite = finite && isfinite(xa);
            const int ba = isfinite(xa) ? base_of(xa, sp.inv_dx) : 0;
            lo[a] = min(lo[a], ba);
            hi[a] = max(hi[a], ba);
        }
    }
    int nodes = 1;
    bool fits = __all_sync(kFull, finite);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = __reduce_min_sync(kFull, lo[a]);
        hi[a] = __reduce_max_sync(kFull, hi[a]);
        const int dim = hi[a] - lo[a] + 3;   // the box of base cells widened by the stencil
        fits = fits && lo[a] >= 0 && dim > 0 && dim <= kWTileNodes;
        nodes = fits ? nodes * dim : 0;
    }
    const bool use_tile = fits && nodes <= kWTileNodes;   // warp-uniform
    if (use_tile) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            wt.lo[a] = lo[a];
        wt.d0 = hi[0] - lo[0] + 3;
        wt.d01 = wt.d0 * (hi[1] - lo[1] + 3);
        for (int i = lane; i < nodes; i += 32)
            wt.t[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        __syncwarp();
    }
    NodeAcc acc;
    acc_zero(acc);
    int cb[3] = {0, 0, 0};
    bool open = false;
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
        const int64_t p = p0 + j;
        P2GParticle q;
        const bool ok = p < n && load_p2g_particle(sp, pv, p, dt, q, err);
        const bool flush = ok && open && (q.b[0] != cb[0] || q.b[1] != cb[1] || q.b[2] != cb[2]);
        if (use_tile) {
            if (__any_sync(kFull, flush))
                tile_flush(wt, acc, cb, flush);
        } else if (flush) {
            acc_flush(gv, gv.cur, acc, cb, err);
        }
        if (flush) {
            acc_zero(acc);
            open = false;
        }
        if (ok) {
            if (!open) {
                cb[0] = q.b[0];
                cb[1] = q.b[1];
                cb[2] = q.b[2];
                open = true;
            }
            acc_add(acc, q);
        }
    }
    if (use_tile) {
        tile_flush(wt, acc, cb, open);
        // every touched node of the tile to the grid, one float4 reduction each
        const int d1 = wt.d01 / wt.d0;
        for (int i = lane; i < nodes; i += 32) {
            const float4 a = wt.t[i];
            if (!(a.w != 0.0f))
                continue;   // no particle weight reached this node
            const int x = wt.lo[0] + i % wt.d0, y = wt.lo[1] + (i / wt.d0) % d1, z = wt.lo[2] + i / wt.d01;
            const int blk = (x < sp.res[0] && y < sp.res[1] && z < sp.res[2])
                                ? __ldg(&gv.table[morton3((uint32_t)x >> 2, (uint32_t)y >> 2, (uint32_t)z >> 2)])
                                : -1;
            if (blk < 0) {
                atomicOr(err, ST_MISSED);
                continue;
            }
            atomicAdd(&gv.cur[(int64_t)blk * 64 + (x & 3) + 4 * (y & 3) + 16 * (z & 3)], a);
        }
    } else if (open) {
        acc_flush(gv, gv.cur, acc, cb, err);
    }
}

constexpr size_t kWTileBytes = (size_t)(kTransferThreads / 32) * kWTileNodes * sizeof(float4);



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
        H[e] = pv.at(CH_F + e, p);
    stress_h(m, H, pv.at(CH_JP, p), t6);
#pragma unroll
    for (int e = 0; e < 6; ++e)
        pv.at(CH_TAU + e, p) = t6[e];
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


}  // namespace

void launch_p2g(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt, uint32_t* err,
                int variant, cudaStream_t s)
{
    if (n <= 0)
        return;
    if (variant == P2G_CHUNK8S) {
        if (pv.aosoa)
            k_p2g_chunks<8, true><<<blocks_for((n + 7) / 8, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, err);
        else
            k_p2g_chunks<8, false><<<blocks_for((n + 7) / 8, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, err);
        return;
    }
    if (variant == P2G_NODE) {
        constexpr int NB = 4;
        const unsigned blocks = (unsigned)((n + 32 * NB * kNodeWarps - 1) / (32 * NB * kNodeWarps));
        if (pv.aosoa)
            k_p2g_node<NB, true><<<blocks, kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, err);
        else
            k_p2g_node<NB, false><<<blocks, kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, err);
        return;
    }
    if (pv.aosoa) {
        // the AoSoA store has register-run forms only besides P2G_NODE (the context allows no other
        // variant with it),
        // in CTAs of 4 or 2 warps
        if (sp.cta_warps == 2) {
            const unsigned g = variant == P2G_CHUNK8 ? blocks_for((n + 7) / 8, 64) : blocks_for((n + 3) / 4, 64);
            if (variant == P2G_CHUNK8)
                k_p2g_chunk_w2<8, true><<<g, 64, 0, s>>>(sp, pv, gv, n, dt, err);
            else
                k_p2g_chunk_w2<4, true><<<g, 64, 0, s>>>(sp, pv, gv, n, dt, err);
            return;
        }
        if (variant == P2G_CHUNK8)
            k_p2g_chunk<8, false, true><<<blocks_for((n + 7) / 8, kTransferThreads), kTransferThreads, 0, s>>>(
                sp, pv, gv, n, dt, err);
        else
            k_p2g_chunk<4, false, true><<<blocks_for((n + 3) / 4, kTransferThreads), kTransferThreads, 0, s>>>(
                sp, pv, gv, n, dt, err);
        return;
    }
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
    } else if ((variant == P2G_CHUNK8 || variant == P2G_CHUNK4) && sp.cta_warps != 4) {
        const int T = 32 * sp.cta_warps;
        const int K = variant == P2G_CHUNK8 ? 8 : 4;
        const unsigned g = blocks_for((n + K - 1) / K, T);
        if (sp.cta_warps == 2)
            (K == 8 ? k_p2g_chunk_w2<8> : k_p2g_chunk_w2<4>)<<<g, T, 0, s>>>(sp, pv, gv, n, dt, err);
        else
            (K == 8 ? k_p2g_chunk_w8<8> : k_p2g_chunk_w8<4>)<<<g, T, 0, s>>>(sp, pv, gv, n, dt, err);
    } else if (variant == P2G_CHUNK8)
        k_p2g_chunk<8, false><<<blocks_for((n + 7) / 8, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt,
                                                                                                   err);
    else if (variant == P2G_CHUNK4)
        k_p2g_chunk<4, false><<<blocks_for((n + 3) / 4, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt,
                                                                                                   err);
    else if (variant == P2G_SLAB4)
        k_p2g_slab<4><<<3 * blocks_for((n + 3) / 4, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, err);
    else if (variant == P2G_WARP)
        k_p2g_warp<true><<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, err);
    else if (variant == P2G_WARPRUN)
        k_p2g_warp<false><<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, err);
    else if (variant == P2G_CHUNK8X2)
        k_p2g_chunk<8, false, false, true><<<blocks_for((n + 7) / 8, kTransferThreads), kTransferThreads, 0, s>>>(
            sp, pv, gv, n, dt, err);
    else if (variant == P2G_WXPOSE)
        k_p2g_wxpose<<<blocks_for(n, kTransferThreads), kTransferThreads, 0, s>>>(sp, pv, gv, n, dt, err);
    else if (variant == P2G_WTILE8) {
        smem_opt_in<k_p2g_wtile<8>>(kWTileBytes);
        k_p2g_wtile<8><<<blocks_for((n + 7) / 8, kTransferThreads), kTransferThreads, kWTileBytes, s>>>(sp, pv, gv, n,
                                                                                                      dt, err);
    }
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


}  // namespace mpm
