// Device prefix scan and stable LSD radix sort (the histogram sort of
// Sec. 4.2.2), with all scratch supplied by the caller and never
// reallocated per call (Sec. 6.3.1 measured per-call scratch reallocation at
// 4.4-9.2% of the step).
//
// Radix sort, one pass per 8-bit digit:
//   1. k_digit_hist: per tile of kTile keys, a 256-bin digit histogram,
//      stored digit-major (hist[d * ntiles + tile]).
//   2. exclusive scan of the histogram -> the global output offset of each
//      (digit, tile) pair.
//   3. k_digit_scatter: each tile writes its keys to their offsets.  Within a
//      tile, keys are taken in rounds of 256 (one per thread, in index
//      order); __match_any_sync groups equal digits in a warp, so the rank of
//      a key is (offset of its digit in this tile) + (same-digit keys in
//      earlier rounds) + (same-digit keys in earlier warps of this round) +
//      (same-digit lanes below it).  Equal keys keep their input order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "internal.h"

namespace mpm {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // 2048 keys per tile
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ int warp_inclusive_scan(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and the block total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int& total)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = warp_inclusive_scan(v, lane);
    if (lane == 31)
        warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kWarps ? warp_sums[lane] : 0;
        int wi = warp_inclusive_scan(w, lane);
        if (lane < kWarps)
            warp_sums[lane] = wi - w;
        if (lane == kWarps - 1)
            warp_sums[kWarps] = wi;
    }
    __syncthreads();
    int ex = inc - v + warp_sums[warp];
    total = warp_sums[kWarps];
    __syncthreads();
    return ex;
}

// Scan of one tile of kTile ints: out = local exclusive prefix, sums[tile] =
// tile total.  Each thread owns kItems consecutive elements.  in and out may
// be the same array (each thread reads its items before any write).
__global__ void __launch_bounds__(kThreads) k_scan_tiles(const int32_t* in, int32_t* out, int64_t n,
                                                         int32_t* __restrict__ sums)
{
    __shared__ int warp_sums[kWarps + 1];
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int v[kItems];
    int local = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        local += v[i];
    }
    int total;
    int ex = block_exclusive_scan(local, warp_sums, total);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int64_t idx = base + i;
        if (idx < n)
            out[idx] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0)
        sums[blockIdx.x] = total;
}

// Exclusive scan of the tile totals by one block, in chunks of kTile.
__global__ void __launch_bounds__(kThreads) k_scan_sums(int32_t* sums, int64_t ntiles)
{
    __shared__ int warp_sums[kWarps + 1];
    int carry = 0;
    for (int64_t c0 = 0; c0 < ntiles; c0 += kTile) {
        int64_t base = c0 + (int64_t)threadIdx.x * kItems;
        int v[kItems];
        int local = 0;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            v[i] = base + i < ntiles ? sums[base + i] : 0;
            local += v[i];
        }
        int total;
        int ex = block_exclusive_scan(local, warp_sums, total) + carry;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if (base + i < ntiles)
                sums[base + i] = ex;
            ex += v[i];
        }
        carry += total;
    }
}

__global__ void __launch_bounds__(kThreads) k_scan_add(int32_t* __restrict__ out, int64_t n,
                                                       const int32_t* __restrict__ sums)
{
    int add = sums[blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t idx = base + i;
        if (idx < n)
            out[idx] += add;
    }
}

__global__ void __launch_bounds__(kThreads) k_digit_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                         int32_t* __restrict__ hist, int64_t ntiles)
{
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        int64_t idx = base + r * kThreads + threadIdx.x;
        if (idx < n)
            atomicAdd(&cnt[(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_digit_scatter(const uint32_t* __restrict__ kin,
                                                            const int32_t* __restrict__ vin,
                                                            uint32_t* __restrict__ kout, int32_t* __restrict__ vout,
                                                            int64_t n, int shift, const int32_t* __restrict__ offs,
                                                            int64_t ntiles)
{
    __shared__ int gofs[256];       // global offset of each digit for this tile, plus earlier rounds
    __shared__ int wcnt[kWarps][256];
    __shared__ int wofs[kWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    gofs[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kWarps; ++w)
        wcnt[w][tid] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kItems; ++r) {
        int64_t idx = base + r * kThreads + tid;
        bool valid = idx < n;
        uint32_t k = valid ? kin[idx] : 0u;
        int32_t v = valid ? vin[idx] : 0;
        int d = valid ? (int)((k >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (valid && rank == 0)
            wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {   // thread tid owns digit tid: offsets of each warp's run of this digit
            int run = gofs[tid];
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                int c = wcnt[w][tid];
                wofs[w][tid] = run;
                run += c;
                wcnt[w][tid] = 0;
            }
            gofs[tid] = run;
        }
        __syncthreads();
        if (valid) {
            int pos = wofs[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
    }
}

inline int64_t tiles_of(int64_t n) { return (n + kTile - 1) / kTile; }

}  // namespace

size_t scan_scratch_bytes(int64_t n)
{
    return (size_t)(tiles_of(n) + 1) * sizeof(int32_t);
}

cudaError_t exclusive_scan(const int32_t* in, int32_t* out, int64_t n, void* scratch, cudaStream_t s,
                           int64_t* launches)
{
    if (n <= 0)
        return cudaSuccess;
    int64_t nt = tiles_of(n);
    int32_t* sums = (int32_t*)scratch;
    k_scan_tiles<<<(unsigned)nt, kThreads, 0, s>>>(in, out, n, sums);
    k_scan_sums<<<1, kThreads, 0, s>>>(sums, nt);
    k_scan_add<<<(unsigned)nt, kThreads, 0, s>>>(out, n, sums);
    if (launches)
        *launches += 3;
    return cudaGetLastError();
}

// Scratch layout: [alt keys n][alt vals n][hist 256*ntiles][scan scratch]
size_t radix_sort_scratch_bytes(int64_t n)
{
    int64_t nt = tiles_of(n > 0 ? n : 1);
    size_t b = 0;
    b += ((size_t)n * 4 + 255) & ~(size_t)255;
    b += ((size_t)n * 4 + 255) & ~(size_t)255;
    b += ((size_t)256 * nt * 4 + 255) & ~(size_t)255;
    b += (scan_scratch_bytes(256 * nt) + 255) & ~(size_t)255;
    return b;
}

cudaError_t radix_sort_pairs(const uint32_t* kin, const int32_t* vin, uint32_t* kout, int32_t* vout,
                             int64_t n, int key_bits, void* scratch, cudaStream_t s, int64_t* launches)
{
    if (n <= 0)
        return cudaSuccess;
    int64_t nt = tiles_of(n);
    char* p = (char*)scratch;
    uint32_t* kalt = (uint32_t*)p;
    p += ((size_t)n * 4 + 255) & ~(size_t)255;
    int32_t* valt = (int32_t*)p;
    p += ((size_t)n * 4 + 255) & ~(size_t)255;
    int32_t* hist = (int32_t*)p;
    p += ((size_t)256 * nt * 4 + 255) & ~(size_t)255;
    void* scan_scr = p;
    int passes = (key_bits + 7) / 8;
    if (passes < 1)
        passes = 1;
    // Ping-pong so the last pass lands in (kout, vout); the first pass reads
    // the caller's input, which is never written.
    const uint32_t* ks = kin;
    const int32_t* vs = vin;
    for (int pss = 0; pss < passes; ++pss) {
        bool to_out = ((passes - 1 - pss) % 2) == 0;
        uint32_t* kd = to_out ? kout : kalt;
        int32_t* vd = to_out ? vout : valt;
        int shift = 8 * pss;
        k_digit_hist<<<(unsigned)nt, kThreads, 0, s>>>(ks, n, shift, hist, nt);
        cudaError_t e = exclusive_scan(hist, hist, 256 * nt, scan_scr, s, launches);
        if (e != cudaSuccess)
            return e;
        k_digit_scatter<<<(unsigned)nt, kThreads, 0, s>>>(ks, vs, kd, vd, n, shift, hist, nt);
        if (launches)
            *launches += 2;
        ks = kd;
        vs = vd;
    }
    return cudaGetLastError();
}

}  // namespace mpm

extern "C" mpm_status mpm_radix_sort_pairs(const uint32_t* keys_in, const int32_t* vals_in, uint32_t* keys_out,
                                           int32_t* vals_out, int64_t n, int key_bits, void* scratch,
                                           size_t* scratch_bytes, void* cuda_stream)
{
    if (n < 0 || key_bits < 1 || key_bits > 32 || !scratch_bytes)
        return MPM_EINVAL;
    size_t need = mpm::radix_sort_scratch_bytes(n);
    if (!scratch) {
        *scratch_bytes = need;
        return MPM_OK;
    }
    if (n == 0)
        return MPM_OK;
    if (*scratch_bytes < need || !keys_in || !vals_in || !keys_out || !vals_out)
        return MPM_EINVAL;
    if (n > (int64_t)0x7fffffff)
        return MPM_EINVAL;
    cudaError_t e = mpm::radix_sort_pairs(keys_in, vals_in, keys_out, vals_out, n, key_bits, scratch,
                                          (cudaStream_t)cuda_stream, nullptr);
    return e == cudaSuccess ? MPM_OK : MPM_ECUDA;
}

// ---- allocation-free entry point ---------------------------------------------
// Scratch for mpm_radix_sort_pairs_noalloc lives in one file-scope device
// array, laid out as radix_sort_pairs expects for MPM_SORT_NOALLOC_MAX_KEYS
// keys: two ping-pong arrays of keys and values, the digit histogram of every
// 2048-key tile, and the scan's tile sums, each rounded up to 256 bytes.
namespace {

constexpr int64_t kNoAllocKeys = MPM_SORT_NOALLOC_MAX_KEYS;
constexpr size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr int64_t kNoAllocTiles = (kNoAllocKeys + mpm::kTile - 1) / mpm::kTile;
constexpr size_t kNoAllocBytes = round256((size_t)kNoAllocKeys * 4) * 2 + round256((size_t)256 * kNoAllocTiles * 4) +
                                 round256((size_t)((256 * kNoAllocTiles + mpm::kTile - 1) / mpm::kTile + 1) * 4);

__device__ __align__(256) unsigned char g_sort_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device (looked up once per
// device; host code must not hand the symbol itself to a kernel).
cudaError_t noalloc_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" mpm_status mpm_radix_sort_pairs_noalloc(const uint32_t* keys_in, const int32_t* vals_in,
                                                   uint32_t* keys_out, int32_t* vals_out, int64_t n, int key_bits,
                                                   void* cuda_stream)
{
    if (n < 0 || key_bits < 1 || key_bits > 32)
        return MPM_EINVAL;
    if (n > kNoAllocKeys)
        return MPM_ECAPACITY;
    if (n == 0)
        return MPM_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out)
        return MPM_EINVAL;
    if (mpm::radix_sort_scratch_bytes(n) > kNoAllocBytes)
        return MPM_ECAPACITY;
    void* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess)
        return MPM_ECUDA;
    // Every word of scratch a pass reads was written earlier in the same call
    // (histograms, scanned offsets, ping-pong buffers), so nothing needs clearing.
    cudaError_t e = mpm::radix_sort_pairs(keys_in, vals_in, keys_out, vals_out, n, key_bits, scratch,
                                          (cudaStream_t)cuda_stream, nullptr);
    return e == cudaSuccess ? MPM_OK : MPM_ECUDA;
}
