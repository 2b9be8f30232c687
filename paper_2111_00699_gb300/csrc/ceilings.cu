// Micro-benchmark kernels for the second ceilings of the substep: the rate at
// which the L2 cache applies float4 reductions, which bounds P2G's scatter
// (Sec. 4.2.2 reduces per warp precisely to spend fewer of them).  Not part
// of the substep.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mpm {

namespace {

// Each warp applies `reds` float4 reductions of (1, 1, 1, 1) per lane to
// 32-node spans of `grid` chosen by a per-warp linear congruential sequence:
// pattern 0, lane l adds to node span + l (32 distinct 16-byte nodes in 4
// consecutive 128-byte lines, as lanes flushing neighbouring cells' runs);
// pattern 1, lane l adds to node span + l / 4 (four lanes per node); pattern
// 2, lane l adds to node 0 of its own span (32 lines per warp instruction, as
// lanes flushing unrelated cells); pattern 3, all lanes add to one node.
// nodes and threads are multiples of 32.
__global__ void k_red_rate(float4* __restrict__ grid, int64_t nodes, int64_t threads, int reds, int pattern)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= threads)
        return;   // whole warps: threads is a multiple of 32
    const int lane = threadIdx.x & 31;
    uint32_t h = (uint32_t)(t >> 5) * 2654435761u + 12345u;
    const int64_t spans = nodes / 32;
    const int off = pattern == 0 ? lane : (pattern == 1 ? (lane >> 2) : 0);
    const uint32_t lane_mix = pattern == 2 ? (uint32_t)lane * 2246822519u : 0u;
#pragma unroll 4
    for (int r = 0; r < reds; ++r) {
        h = h * 1664525u + 1013904223u;
        const int64_t span = (int64_t)((h ^ lane_mix) >> 6) % spans;
        atomicAdd(&grid[span * 32 + off], make_float4(1.0f, 1.0f, 1.0f, 1.0f));
    }
}

}  // namespace

cudaError_t launch_debug_red_rate(float4* grid, int64_t nodes, int64_t threads, int reds, int pattern, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    k_red_rate<<<blocks, 256, 0, s>>>(grid, nodes, threads, reds, pattern);
    return cudaGetLastError();
}

}  // namespace mpm
