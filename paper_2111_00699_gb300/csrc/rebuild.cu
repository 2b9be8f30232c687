// Rebuild-mapping (Sec. 4 and Sec. 4.2.1) and particle bookkeeping kernels.
//
// The block "hash" is direct-mapped: a table with one int32 per block of
// the whole domain, indexed by the block's Morton code.  On a GB300 (288 GB
// HBM, 129 MB L2) that table is 1 MB for a 256^3 grid and stays in L2, so a
// lookup is one cached load with no probing.  Physical-block indices are the
// ranks of the Morton codes of the marked blocks (a scan over the table),
// which makes the mapping deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "async_copy.cuh"
#include "device_math.cuh"
#include "internal.h"

namespace mpm {

namespace {

constexpr int kBlock = 256;

inline unsigned blocks_for(int64_t n, int per = kBlock) { return (unsigned)((n + per - 1) / per); }

// Particle code (Sec. 4): base node per axis with the -dx/2 shift of the
// particle blocks; key = Morton(block) << 6 | Morton(cell within block).
// Key of particle p (0xffffffff if its stencil leaves the grid or the table).
__device__ __forceinline__ uint32_t particle_key(const SimParams& sp, const PartView& pv, int64_t p)
{
    int b[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float x = pv.at(CH_X + a, p);
        b[a] = base_of(x, sp.inv_dx);
        ok = ok && isfinite(x) && b[a] >= 0 && b[a] + 2 < sp.res[a] && (b[a] >> 2) < (1 << sp.L);
    }
    if (!ok)
        return 0xffffffffu;
    uint32_t blk = morton3((uint32_t)b[0] >> 2, (uint32_t)b[1] >> 2, (uint32_t)b[2] >> 2);
    uint32_t cell = morton3((uint32_t)b[0] & 3u, (uint32_t)b[1] & 3u, (uint32_t)b[2] & 3u);
    return (blk << 6) | cell;
}

__global__ void k_keys(SimParams sp, PartView pv, int64_t n, uint32_t* __restrict__ keys,
                       int32_t* __restrict__ vals, uint32_t* __restrict__ err)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    const uint32_t key = particle_key(sp, pv, p);
    if (key == 0xffffffffu)
        atomicOr(err, ST_EDOMAIN);
    keys[p] = key;
    vals[p] = (int32_t)p;
}

// Window re-sort between rebuilds: the particles of each window of
// kResortWindow consecutive storage slots are ordered by their current key
// (block code, cell code) and copied, permuted, to the other particle
// buffer.  Particles drift across cell faces long before they leave the
// mapped blocks, and P2G merges only runs of consecutive particles in one
// cell; this restores the runs without a global sort or a host round trip.
// Equal keys keep their storage order (the sort key is (key, slot)).
//
// The sort is a bitonic network over (key << 32 | slot) with 4 elements per
// thread in registers: the compare-exchanges at strides 1 and 2 stay inside a
// thread, those at strides 4 to 64 pair lanes of one warp (shuffles), and
// only the 6 steps at strides 128 to 512 go through shared memory and a
// barrier (against 55 barrier steps for a network held in shared memory).
constexpr int kResortThreads = 256;
constexpr int kResortPer = kResortWindow / kResortThreads;   // elements per thread

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int mask)
{
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, mask);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), mask);
    return ((uint64_t)hi << 32) | lo;
}

__global__ void __launch_bounds__(kResortThreads, 4) k_resort_window(SimParams sp, PartView src, PartView dst, int64_t n)
{
    static_assert(kResortPer == 4 && kResortThreads % 32 == 0, "4 elements per thread");
    __shared__ uint64_t xch[kResortWindow];
    __shared__ uint16_t idx[kResortWindow];
    const int tid = threadIdx.x;
    const int64_t p0 = (int64_t)blockIdx.x * kResortWindow;
    uint64_t v[kResortPer];
#pragma unroll
    for (int e = 0; e < kResortPer; ++e) {
        const int i = kResortPer * tid + e;
        const int64_t p = p0 + i;
        uint32_t k = 0xffffffffu;                       // padding past n sorts last
        if (p < n)
            k = min(particle_key(sp, src, p), 0xfffffffeu);
        v[e] = ((uint64_t)k << 32) | (uint32_t)i;
    }
    // element i = 4 tid + e is compared with i ^ stride; blocks of `size` with (i & size) == 0 ascend
#pragma unroll
    for (int size = 2; size <= kResortWindow; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride < kResortPer) {
#pragma unroll
                for (int e = 0; e < kResortPer; ++e) {
                    const int l = e ^ stride;
                    if (l > e) {
                        const bool up = ((kResortPer * tid + e) & size) == 0;
                        if ((v[e] > v[l]) == up) {
                            const uint64_t t = v[e];
                            v[e] = v[l];
                            v[l] = t;
                        }
                    }
                }
            } else {
                const int tmask = stride / kResortPer;          // partner thread: tid ^ tmask
                const bool keep_min = ((tid & tmask) == 0) == (((kResortPer * tid) & size) == 0);
                if (tmask < 32) {
#pragma unroll
                    for (int e = 0; e < kResortPer; ++e) {
                        const uint64_t o = shfl_xor_u64(v[e], tmask);
                        v[e] = keep_min ? (o < v[e] ? o : v[e]) : (o > v[e] ? o : v[e]);
                    }
                } else {
                    __syncthreads();   // the previous exchange is read
#pragma unroll
                    for (int e = 0; e < kResortPer; ++e)
                        xch[kResortPer * tid + e] = v[e];
                    __syncthreads();
#pragma unroll
                    for (int e = 0; e < kResortPer; ++e) {
                        const uint64_t o = xch[kResortPer * (tid ^ tmask) + e];
                        v[e] = keep_min ? (o < v[e] ? o : v[e]) : (o > v[e] ? o : v[e]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < kResortPer; ++e)
        idx[kResortPer * tid + e] = (uint16_t)(uint32_t)v[e];
    __syncthreads();
    const int m = (int)min((int64_t)kResortWindow, n - p0);
    // permutation: each thread moves its 4 slots; 8 channels' loads in flight at a time
    constexpr int kPer = kResortWindow / kResortThreads;
    int src_i[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = tid + k * kResortThreads;
        src_i[k] = i < m ? idx[i] : -1;
    }
#pragma unroll 1
    for (int c0 = 0; c0 < kChannels; c0 += 8) {
        float val[8][kPer];
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
            for (int k = 0; k < kPer; ++k)
                val[c][k] = src_i[k] >= 0 ? src.at(c0 + c, p0 + src_i[k]) : 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
            for (int k = 0; k < kPer; ++k)
                if (src_i[k] >= 0)
                    dst.at(c0 + c, p0 + tid + k * kResortThreads) = val[c][k];
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        if (src_i[k] < 0)
            continue;
        const int64_t o = p0 + tid + k * kResortThreads;
        dst.mat[o] = src.mat[p0 + src_i[k]];
        dst.id[o] = src.id[p0 + src_i[k]];
    }
}

// Mark the 3x3x3 neighbourhood of every gblock (the first particle of each
// run of equal block codes in the sorted keys does the marking).
__global__ void k_mark(const uint32_t* __restrict__ skeys, int64_t n, int L, int32_t* __restrict__ flags)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    uint32_t k = skeys[i];
    if (k == 0xffffffffu)
        return;
    uint32_t code = k >> 6;
    if (i > 0 && (skeys[i - 1] >> 6) == code)
        return;
    int bx = (int)compact3(code), by = (int)compact3(code >> 1), bz = (int)compact3(code >> 2);
    int side = 1 << L;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int x = bx + dx, y = by + dy, z = bz + dz;
                if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side)
                    continue;
                flags[morton3((uint32_t)x, (uint32_t)y, (uint32_t)z)] = 1;
            }
}

__global__ void k_table(const int32_t* __restrict__ flags, const int32_t* __restrict__ ranks, int64_t n_slots,
                        int32_t* __restrict__ table, int32_t* __restrict__ pslot, int32_t* __restrict__ n_pblocks)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slots)
        return;
    int f = flags[s];
    int r = ranks[s];
    table[s] = f ? r : -1;
    if (f)
        pslot[r] = (int32_t)s;
    if (s == n_slots - 1)
        *n_pblocks = r + f;
}

// Interior blocks: a physical block whose 26 neighbours that lie in the grid
// are all mapped.  A base cell in an interior block keeps the particle's
// stencil, widened by up to 4 cells per side, inside mapped blocks.
__global__ void k_interior(SimParams sp, const int32_t* __restrict__ table, const int32_t* __restrict__ pslot,
                           int32_t n_pblocks, uint8_t* __restrict__ interior)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pblocks)
        return;
    uint32_t s = (uint32_t)pslot[r];
    int B[3] = {(int)compact3(s), (int)compact3(s >> 1), (int)compact3(s >> 2)};
    bool ok = true;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int N[3] = {B[0] + dx, B[1] + dy, B[2] + dz};
                bool in = true;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    in = in && N[a] >= 0 && N[a] <= (sp.res[a] - 1) >> 2;
                if (in)
                    ok = ok && table[morton3((uint32_t)N[0], (uint32_t)N[1], (uint32_t)N[2])] >= 0;
            }
    interior[r] = ok ? 1 : 0;
}

// dst[i] = src[perm[i]] for every channel, the material and the id.
__global__ void k_permute(PartView src, PartView dst, const int32_t* __restrict__ perm, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int64_t j = perm[i];
#pragma unroll 2
    for (int c = 0; c < kChannels; ++c)
        dst.at(c, i) = src.at(c, j);
    dst.mat[i] = src.mat[j];
    dst.id[i] = src.id[j];
}

// The same particles in another store layout (src and dst differ in aosoa).
__global__ void k_relayout(PartView src, PartView dst, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
#pragma unroll 4
    for (int c = 0; c < kChannels; ++c)
        dst.at(c, i) = src.at(c, i);
    dst.mat[i] = src.mat[i];
    dst.id[i] = src.id[i];
}

__global__ void k_append(PartView pv, int64_t n0, int64_t n, const float* __restrict__ x,
                         const float* __restrict__ v, const float* __restrict__ vol, float default_vol, int material)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int64_t p = n0 + i;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        pv.at(CH_X + a, p) = x[3 * i + a];
        pv.at(CH_V + a, p) = v ? v[3 * i + a] : 0.0f;
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        pv.at(CH_C + e, p) = 0.0f;
        pv.at(CH_F + e, p) = 0.0f;   // F - I
    }
    pv.at(CH_JP, p) = 0.0f;          // Jp - 1 (J - 1 for fluids)
    pv.at(CH_VOL, p) = vol ? vol[i] : default_vol;
#pragma unroll
    for (int e = 0; e < 6; ++e)
        pv.at(CH_TAU + e, p) = 0.0f;   // stress of F = I, Jp = J = 1 is zero for every model
    pv.mat[p] = (uint8_t)material;
    pv.id[p] = (int32_t)p;
}

// out[id[i] * width + e] = channel(first + e)[i]: storage order -> insertion order.
// F and Jp are held as F - I and Jp - 1 (J - 1 for fluids): the fields
// with a unit bias add it on the way out and remove it on the way in.
// bias_step: 4 for F (diagonal entries 0, 4, 8), 1 for Jp, 0 for none.
__device__ __forceinline__ float unit_bias(int e, int bias_step)
{
    return (bias_step && e % bias_step == 0) ? 1.0f : 0.0f;
}

__global__ void k_gather_out(PartView pv, int64_t n, int first, int width, int bias_step, float* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int64_t q = pv.id[i];
    for (int e = 0; e < width; ++e)
        out[q * width + e] = pv.at(first + e, i) + unit_bias(e, bias_step);
}

__global__ void k_scatter_in(PartView pv, int64_t n, int first, int width, int bias_step, const float* __restrict__ in)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int64_t q = pv.id[i];
    for (int e = 0; e < width; ++e)
        pv.at(first + e, i) = in[q * width + e] - unit_bias(e, bias_step);
}

__global__ void k_grid_to_dense(SimParams sp, const float4* __restrict__ grid, const int32_t* __restrict__ pslot,
                                int32_t n_pblocks, float* __restrict__ dense)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_pblocks * 64)
        return;
    int pb = (int)(idx >> 6), l = (int)(idx & 63);
    uint32_t s = (uint32_t)pslot[pb];
    int i = 4 * (int)compact3(s) + (l & 3);
    int j = 4 * (int)compact3(s >> 1) + ((l >> 2) & 3);
    int k = 4 * (int)compact3(s >> 2) + (l >> 4);
    if (i >= sp.res[0] || j >= sp.res[1] || k >= sp.res[2])
        return;
    float4 g = grid[idx];
    int64_t o = 4 * ((int64_t)i + (int64_t)sp.res[0] * ((int64_t)j + (int64_t)sp.res[1] * k));
    dense[o + 0] = g.w;
    dense[o + 1] = g.x;
    dense[o + 2] = g.y;
    dense[o + 3] = g.z;
}

}  // namespace

void launch_keys(const SimParams& sp, const PartView& pv, int64_t n, uint32_t* keys, int32_t* vals, uint32_t* err,
                 cudaStream_t s)
{
    if (n > 0)
        k_keys<<<blocks_for(n), kBlock, 0, s>>>(sp, pv, n, keys, vals, err);
}

void launch_mark_pblocks(const uint32_t* skeys, int64_t n, int L, int32_t* flags, cudaStream_t s)
{
    if (n > 0)
        k_mark<<<blocks_for(n), kBlock, 0, s>>>(skeys, n, L, flags);
}

void launch_build_table(const int32_t* flags, const int32_t* ranks, int64_t n_slots, int32_t* table,
                        int32_t* pslot, int32_t* n_pblocks, cudaStream_t s)
{
    k_table<<<blocks_for(n_slots), kBlock, 0, s>>>(flags, ranks, n_slots, table, pslot, n_pblocks);
}

void launch_relayout(const PartView& src, const PartView& dst, int64_t n, cudaStream_t s)
{
    if (n > 0)
        k_relayout<<<blocks_for(n), kBlock, 0, s>>>(src, dst, n);
}

void launch_permute(const PartView& src, const PartView& dst, const int32_t* perm, int64_t n, cudaStream_t s)
{
    if (n > 0)
        k_permute<<<blocks_for(n), kBlock, 0, s>>>(src, dst, perm, n);
}

void launch_resort_window(const SimParams& sp, const PartView& src, const PartView& dst, int64_t n, cudaStream_t s)
{
    if (n > 0)
        k_resort_window<<<(unsigned)((n + kResortWindow - 1) / kResortWindow), kResortThreads, 0, s>>>(sp, src, dst, n);
}

void launch_interior(const SimParams& sp, const int32_t* table, const int32_t* pslot, int32_t n_pblocks,
                     uint8_t* interior, cudaStream_t s)
{
    if (n_pblocks > 0)
        k_interior<<<blocks_for(n_pblocks), kBlock, 0, s>>>(sp, table, pslot, n_pblocks, interior);
}

void launch_append(const PartView& pv, int64_t n0, int64_t n, const float* x, const float* v, const float* vol,
                   float default_vol, int material, cudaStream_t s)
{
    if (n > 0)
        k_append<<<blocks_for(n), kBlock, 0, s>>>(pv, n0, n, x, v, vol, default_vol, material);
}

// field: 0 x, 1 v, 2 C, 3 F, 4 Jp
static void field_range(int field, int& first, int& width, int& bias_step)
{
    static const int F0[5] = {CH_X, CH_V, CH_C, CH_F, CH_JP};
    static const int W[5] = {3, 3, 9, 9, 1};
    static const int B[5] = {0, 0, 0, 4, 1};
    first = F0[field];
    width = W[field];
    bias_step = B[field];
}

void launch_gather_out(const PartView& pv, int64_t n, int field, float* out, cudaStream_t s)
{
    int first, width, bias_step;
    field_range(field, first, width, bias_step);
    if (n > 0)
        k_gather_out<<<blocks_for(n), kBlock, 0, s>>>(pv, n, first, width, bias_step, out);
}

void launch_scatter_in(const PartView& pv, int64_t n, int field, const float* in, cudaStream_t s)
{
    int first, width, bias_step;
    field_range(field, first, width, bias_step);
    if (n > 0)
        k_scatter_in<<<blocks_for(n), kBlock, 0, s>>>(pv, n, first, width, bias_step, in);
}

void launch_grid_to_dense(const SimParams& sp, const float4* grid, const int32_t* pslot, int32_t n_pblocks,
                          float* dense, cudaStream_t s)
{
    if (n_pblocks > 0)
        k_grid_to_dense<<<blocks_for((int64_t)n_pblocks * 64), kBlock, 0, s>>>(sp, grid, pslot, n_pblocks, dense);
}

}  // namespace mpm

// ---- largest particle speed (adaptive dt) -----------------------------------

namespace mpm {
namespace {
// The maximum is taken over the bit patterns: for |v|^2 >= 0 they order as
// the floats do, and every NaN pattern (either sign) lies above +Inf's, so a
// NaN speed reaches the host as NaN (fmaxf would drop it).
__global__ void k_max_speed2(PartView pv, int64_t n, uint32_t* __restrict__ word)
{
    uint32_t best = 0u;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const float a = pv.at(CH_V, p), b = pv.at(CH_V + 1, p), c = pv.at(CH_V + 2, p);
        best = max(best, __float_as_uint(a * a + b * b + c * c));
    }
    const unsigned m = __reduce_max_sync(0xffffffffu, best);
    if ((threadIdx.x & 31) == 0)
        atomicMax(word, m);
}
}  // namespace

void launch_max_speed2(const PartView& pv, int64_t n, uint32_t* word, cudaStream_t s)
{
    if (n > 0) {
        int64_t blocks = (n + kBlock - 1) / kBlock;
        k_max_speed2<<<(unsigned)(blocks < 1216 ? blocks : 1216), kBlock, 0, s>>>(pv, n, word);
    }
}
}  // namespace mpm

// ---- bounded-wait check -----------------------------------------------------
// One warp waits on an mbarrier that expects 1024 bytes no copy ever delivers,
// with the same bounded poll the staged transfer kernels use; when the poll
// gives up it records ST_TIMEOUT and the kernel returns normally.

namespace mpm {
namespace {
__global__ void k_debug_wait_timeout(int max_iter, uint32_t* __restrict__ err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_arrive_expect_tx(&bar, 1024u);
    }
    __syncthreads();
    if (!mbar_wait(&bar, 0, max_iter) && threadIdx.x == 0)
        atomicOr(err, ST_TIMEOUT);
}
}  // namespace

void launch_debug_wait_timeout(int max_iter, uint32_t* err, cudaStream_t s)
{
    k_debug_wait_timeout<<<1, 32, 0, s>>>(max_iter, err);
}
}  // namespace mpm
