// Internal types shared by the libmpm translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "mpm.h"

namespace mpm {

constexpr int kMaxMaterials = 8;

// Particle SoA channels: one float array of `cap` entries per channel.
enum Channel : int {
    CH_X = 0,    // x, y, z
    CH_V = 3,    // velocity
    CH_C = 6,    // affine velocity C (row-major 3x3)
    CH_F = 15,   // displacement gradient H = F - I (row-major 3x3)
    CH_JP = 24,  // snow Jp - 1 / fluid J - 1 (0 for the other models)
    CH_VOL = 25, // rest volume
    CH_TAU = 26, // Kirchhoff stress of the current F: xx, yy, zz, xy, xz, yz
    kChannels = 32
};

// P2G scatter variants (tuning knob mpm_config.p2g_variant).
enum P2GVariant : int {
    P2G_DIRECT = 0,   // thread per particle in storage order, float4 global atomics
    P2G_STRIDED = 1,  // lanes take every 8th particle of a 256-particle tile (distinct cells), float4 atomics
    P2G_TILE = 2,     // CTA accumulates its 256 particles into a shared-memory node tile, one flush
    P2G_CHUNK4 = 3,   // thread walks 4 consecutive particles, register accumulation per base-cell run
    P2G_CHUNK8 = 4,   // same with 8 particles per thread
    P2G_STAGE4 = 5,   // CHUNK4 reading a CTA's 512 particles from shared memory, staged by bulk async copies
    P2G_STAGE8 = 6,   // same with 8 particles per thread (1024 per CTA)
    P2G_SACC4 = 7,    // CHUNK4 with the 27 node accumulators in (thread-private) shared memory
    P2G_SLAB4 = 8,    // CHUNK4 split over three threads, one per z-slab of 9 nodes
    P2G_WARP = 9,     // thread per particle, lanes grouped by base cell, shuffle-tree reduction per group (Sec. 4.2.2)
    P2G_WARPRUN = 10, // WARP with groups limited to runs on consecutive lanes (the paper's "no sort" case)
    P2G_WTILE8 = 11,  // CHUNK8 flushing its runs into a warp-private shared-memory node tile, one reduction per node
    P2G_WXPOSE = 12,  // thread per particle, lanes grouped by base cell, group sums through shared memory
    P2G_CHUNK8X2 = 13, // CHUNK8 accumulating with paired FP32 fused multiply-adds
    P2G_NODE = 14,    // warp per run of particles, one lane per stencil node
    P2G_CHUNK8S = 15, // CHUNK8 with each thread's particles taken in base-cell order
    kP2GVariants = 16
};

// Particle capacity is a multiple of this, so that a staged tile of
// particles never reads past the end of a channel array.
constexpr int64_t kCapQuantum = 1024;

// G2P gather variants (tuning knob mpm_config.g2p_variant).
enum G2PVariant : int {
    G2P_DIRECT = 0,   // thread per particle, 27 gathers
    G2P_CHUNK4 = 1,   // thread walks 4 consecutive particles, node velocities cached per base cell
    G2P_CHUNK8 = 2,   // same with 8 particles per thread
    G2P_TILE = 3,     // CTA stages its grid tile in shared memory, gathers from there
    G2P_OCC = 4,      // thread per particle capped at 64 registers (occupancy)
    G2P_STAGE = 5,    // OCC with particle inputs and a 2x2x2-block grid tile staged by bulk async copies
    G2P_OCC10 = 6,    // thread per particle capped at 48 registers (10 CTAs of 128 per SM)
    G2P_OCCSW = 7,    // OCC with the B-spline weights in shared memory (the paper's weight spilling)
    kG2PVariants = 8
};

// Device status word bits.
enum : uint32_t {
    ST_REBUILD_SOFT = 1u,  // a particle's next stencil may reach an unmapped block
    ST_REBUILD_HARD = 2u,  // a particle's stencil reached an unmapped block
    ST_EDOMAIN = 4u,       // a stencil left the grid
    ST_ENONFINITE = 8u,    // a position became non-finite
    ST_MISSED = 16u,       // P2G/G2P found an unmapped block (CFL violated)
    ST_TIMEOUT = 32u,      // an asynchronous copy did not complete within its wait limit
};

struct MatParams {
    int kind;
    float mu, la, rho;
    float K, gamma;          // fluid
    float lo_m1, hi_m1, xi;  // snow clamp bounds of sigma - 1 (-theta_c, theta_s), hardening
    float lo_b, hi_b;        // the same bounds on sigma^2 - 1: (1 - theta_c)^2 - 1, (1 + theta_s)^2 - 1
    float M2, beta, alpha0;  // NACC: M^2, cohesion, initial alpha (K holds the bulk modulus, xi the hardening)
    float alpha, dp_coef;    // sand: cone slope, (3 la + 2 mu) / (2 mu)
};

struct SimParams {
    int res[3];
    float dx, inv_dx;
    int boundary, wall;
    float g[3];
    int L;                   // Morton bits per axis of the block table
    int transfer;            // MPM_APIC or MPM_ASFLIP
    float flip_alpha, flip_beta_min, flip_beta_max, flip_margin;
    int n_mats;
    int cta_warps;           // warps per CTA of the register-run P2G and the 64-register G2P: 2, 4 or 8
    MatParams mat[kMaxMaterials];
};

// The particle store: kChannels x cap floats in one of two layouts.
//  - SoA (aosoa = 0): one array of cap floats per channel; channel c of
//    particle p at c * cap + p.
//  - AoSoA (aosoa = 1): packets of 32 particles, each packet holding its 32
//    floats of channel 0, then of channel 1, ..., then 32 unused floats;
//    channel c of particle p at (p / 32) * kPacketFloats + 32 c + p % 32.  A
//    warp's 32 consecutive particles then read one 128-byte line per
//    channel as in SoA, but all their channels lie in one 4 KB span (the
//    paper's AoSoA, Sec. 6.2).  The unused line makes consecutive packets
//    4224 bytes apart, so that the same channel of neighbouring packets does
//    not fall into one L1 set (4 KB strides alias).
// ch() is the SoA channel pointer (SoA only); at() serves both layouts.
constexpr int kPacketFloats = 32 * kChannels + 32;

struct PartView {
    float* soa;     // the store: (cap / 32) * kPacketFloats floats (SoA uses the first kChannels * cap)
    int64_t cap;    // a multiple of kCapQuantum (so of 32)
    uint8_t* mat;
    int32_t* id;
    int aosoa = 0;
    __host__ __device__ float* ch(int c) const { return soa + (int64_t)c * cap; }
    __host__ __device__ int64_t idx(int c, int64_t p) const
    {
        return aosoa ? (p >> 5) * kPacketFloats + 32 * c + (p & 31) : (int64_t)c * cap + p;
    }
    __host__ __device__ float& at(int c, int64_t p) const { return soa[idx(c, p)]; }
};

// Channel c of particle p with the layout fixed at compile time (the
// kernels instantiated per layout).
template <bool kAoS>
__device__ __forceinline__ float& pch(const PartView& pv, int c, int64_t p)
{
    if (kAoS)
        return pv.soa[(p >> 5) * kPacketFloats + 32 * c + (p & 31)];
    return pv.soa[(int64_t)c * pv.cap + p];
}

struct GridView {
    float4* cur;          // (p or v, m) per node, 64 nodes per physical block
    float4* nxt;          // buffer for the next substep (cleared by the grid update)
    const int32_t* table; // Morton slot -> physical block index, or -1
    const int32_t* pslot; // physical block index -> Morton slot
    const uint8_t* interior; // physical block index -> 1 if its 26 neighbours (in the grid) are mapped
    float4* old;          // ASFLIP: grid velocity before forces (p / m, 0) per node; else null
    uint32_t* slot;       // null, or the substep's two status words (flags, speed), zeroed by the grid update
    int32_t n_pblocks;
};

// NVTX range over a host call (visible in Nsight Systems timelines; a no-op
// unless a tool is attached).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// ---- launchers implemented in the .cu files -------------------------------

// sort.cu
size_t radix_sort_scratch_bytes(int64_t n);
size_t scan_scratch_bytes(int64_t n);
cudaError_t radix_sort_pairs(const uint32_t* kin, const int32_t* vin, uint32_t* kout, int32_t* vout,
                             int64_t n, int key_bits, void* scratch, cudaStream_t s, int64_t* launches);
cudaError_t exclusive_scan(const int32_t* in, int32_t* out, int64_t n, void* scratch, cudaStream_t s,
                           int64_t* launches);

// rebuild.cu
void launch_keys(const SimParams& sp, const PartView& pv, int64_t n, uint32_t* keys, int32_t* vals,
                 uint32_t* err, cudaStream_t s);
void launch_mark_pblocks(const uint32_t* skeys, int64_t n, int L, int32_t* flags, cudaStream_t s);
void launch_build_table(const int32_t* flags, const int32_t* ranks, int64_t n_slots, int32_t* table,
                        int32_t* pslot, int32_t* n_pblocks, cudaStream_t s);
void launch_permute(const PartView& src, const PartView& dst, const int32_t* perm, int64_t n, cudaStream_t s);
void launch_relayout(const PartView& src, const PartView& dst, int64_t n, cudaStream_t s);
constexpr int kResortWindow = 1024;
void launch_resort_window(const SimParams& sp, const PartView& src, const PartView& dst, int64_t n, cudaStream_t s);
void launch_interior(const SimParams& sp, const int32_t* table, const int32_t* pslot, int32_t n_pblocks,
                     uint8_t* interior, cudaStream_t s);
void launch_append(const PartView& pv, int64_t n0, int64_t n, const float* x, const float* v,
                   const float* vol, float default_vol, int material, cudaStream_t s);
void launch_gather_out(const PartView& pv, int64_t n, int field, float* out, cudaStream_t s);
void launch_scatter_in(const PartView& pv, int64_t n, int field, const float* in, cudaStream_t s);
void launch_grid_to_dense(const SimParams& sp, const float4* grid, const int32_t* pslot, int32_t n_pblocks,
                          float* dense, cudaStream_t s);
// *word (zeroed by the caller) <- max over particles of |v|^2, as float bits
void launch_max_speed2(const PartView& pv, int64_t n, uint32_t* word, cudaStream_t s);

// p2g.cu, g2p.cu, g2p2g.cu
void launch_p2g(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt,
                uint32_t* err, int variant, cudaStream_t s);
void launch_prepare_stress(const SimParams& sp, const PartView& pv, int64_t n, cudaStream_t s);
void launch_g2p2g(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt,
                  uint32_t* flags, uint32_t* err, int p2g_variant, cudaStream_t s);
void launch_grid_update(const SimParams& sp, const GridView& gv, float dt, cudaStream_t s);
void launch_g2p(const SimParams& sp, const PartView& pv, const GridView& gv, int64_t n, float dt,
                uint32_t* flags, uint32_t* err, int variant, cudaStream_t s);
MatParams make_mat_params(const mpm_material& m);
void launch_debug_svd(const float* F, float* U, float* sig, float* V, int64_t n, cudaStream_t s);
void launch_debug_stress(const MatParams& mp, const float* F, const float* Jp, float* tau, int64_t n,
                         cudaStream_t s);
void launch_debug_plasticity(const MatParams& mp, float* F, float* Jp, int64_t n, cudaStream_t s);

}  // namespace mpm
