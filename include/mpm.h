/*
 * libmpm -- one explicit MLS-MPM substep on a GB300 (sm_103a), behind a C ABI.
 *
 * Method: "Principles towards Real-Time Simulation of Material Point Method
 * on Modern GPUs" (Fei, Huang, Gao).  One time step is the five phases of
 * Sec. 4: rebuild-mapping (particle codes, block hash with the 3x3x3
 * neighbour blocks, Sec. 4 and Sec. 4.2.1), particle sort to cell
 * granularity (Sec. 4.2.2), particle-to-grid transfer with the stress
 * computation merged in (Sec. 4.1), grid update with the boundary condition
 * merged in (Sec. 4.1), and grid-to-particle transfer.  The first two phases
 * run only when some particle is about to leave the blocks mapped at the
 * last rebuild (the "free zone" of Sec. 4.2.1).  Transfers are MLS-MPM with
 * quadratic B-splines (Sec. 6, [Hu et al. 2018]).
 *
 * Conventions for every call:
 *   - Every entry point returns mpm_status (or a plain value where stated);
 *     no C++ exception and no abort crosses this boundary.
 *   - Pointers are plain host or device addresses; a call that takes
 *     `on_device` reads/writes device memory when it is non-zero and host
 *     memory when it is zero.  The library never keeps a caller pointer
 *     beyond the call: inputs are copied in, outputs copied out.
 *   - Work is enqueued on the CUDA stream given to mpm_create.  Calls marked
 *     "syncs" wait for that stream; the others return before the GPU is done.
 *   - Device-side failures (a particle leaving the domain, a non-finite
 *     value) set a sticky error word; the next syncing call returns it and
 *     mpm_last_error() describes it.
 *   - All particle arrays crossing the ABI are in insertion order (the
 *     order of mpm_add_particles calls), row-major FP32:
 *     x, v: n x 3;  C, F: n x 3 x 3 with element (a, b) at 9 p + 3 a + b;
 *     Jp: n (snow plastic volume ratio, or J for fluid particles).
 */
#ifndef MPM_H
#define MPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_ctx mpm_ctx; /* opaque; owned by the library */

typedef enum {
    MPM_OK = 0,
    MPM_EINVAL = 1,     /* bad argument (null pointer, bad size, bad material) */
    MPM_ENOMEM = 2,     /* the allocator returned NULL */
    MPM_ECAPACITY = 3,  /* a fixed capacity (max_particles) would be exceeded */
    MPM_EDOMAIN = 4,    /* a particle's 3x3x3 stencil left the grid, or outran the mapped blocks */
    MPM_ENONFINITE = 5, /* a particle position became NaN or infinite */
    MPM_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
    MPM_ECUDA = 7,      /* a CUDA runtime call failed; see mpm_last_error */
    MPM_ENOTSUP = 8     /* the request is valid but not supported by this build */
} mpm_status;

typedef enum { MPM_ELASTIC = 0, MPM_FLUID = 1, MPM_SNOW = 2, MPM_SAND = 3, MPM_NACC = 4, MPM_NHSAND = 5 } mpm_kind;
typedef enum { MPM_STICKY = 0, MPM_SLIP = 1 } mpm_boundary;

/* One material.  E is Young's modulus (for MPM_FLUID and MPM_NACC: the bulk
 * modulus).  Fixed-corotated elastic [Stomakhin 2012]; snow = fixed-corotated
 * on F_E with exp(hardening (1 - Jp)) and singular values clamped to
 * [1 - theta_c, 1 + theta_s] [Stomakhin 2013]; fluid p = K (J^-gamma - 1)
 * [Tampubolon 2017]; sand = Hencky-strain St. Venant-Kirchhoff with the
 * Drucker-Prager return map for friction angle friction_deg [Klar 2016];
 * NACC snow (the paper's snow model, Sec. 6.5, after Wolper et al. 2019) =
 * the same Hencky elasticity from the bulk modulus E and nu, the Cam-Clay
 * yield ellipse (1 + 2 beta) q^2 + M^2 (p + beta p0)(p - p0) <= 0 with
 * p0 = E sinh(hardening * max(-alpha, 0)), alpha = alpha0 + ln Jp, and a
 * non-associative return map (q scaled at fixed p, or the tips); neo-Hookean
 * sand (the sand of the paper's sand benchmark, Sec. 6, after Yue et al.
 * 2018) = tau = mu (F F^T - I) + lambda ln(J) I with the sand's
 * Drucker-Prager return map on the Hencky strain. */
typedef struct {
    int32_t kind;          /* mpm_kind */
    float E, nu, rho;
    float gamma;           /* fluid exponent */
    float theta_c, theta_s, hardening;
    float friction_deg;
    float friction_M;      /* NACC: slope M of the critical state line */
    float cohesion;        /* NACC: cohesion beta */
    float alpha0;          /* NACC: initial alpha (< 0 gives the material strength at rest) */
} mpm_material;

/* Grid and scene.  Nodes i = 0..res[a]-1 sit at i * dx.  Nodes with
 * i < wall or i >= res - wall are wall nodes: sticky walls zero their
 * velocity, slip walls zero the component pointing into the wall.
 * Particle keys need 3L + 6 <= 32 bits with 4 * 2^L >= max(res):
 * res up to 1024 per axis. */
typedef struct {
    int32_t res[3];
    float dx;
    int32_t boundary;      /* mpm_boundary */
    int32_t wall;          /* wall layer thickness in nodes (3 is usual) */
    float gravity[3];
    int64_t max_particles; /* 0: grow without bound (4x when half full) */
    int32_t use_g2p2g;     /* 1: fused G2P2G transfer (Sec. 4.1) -- per substep the grid
                              update and one kernel doing G2P and the next P2G, whose
                              scatter follows p2g_variant (3/4: register runs of 4/8
                              particles, 7: runs of 4 accumulated in shared memory,
                              9/10: the warp-level reduction of p2g_variant 9/10, 11: as 4,
                              else one thread per particle);
                              0: separate P2G, grid update, G2P */
    int32_t p2g_variant;   /* tuning: 0 direct float4 atomics, 1 cell-strided lanes,
                              2 shared-memory node tile per CTA, 3/4 register
                              accumulation over runs of 4/8 particles, 5/6 the same with
                              each CTA's 512/1024 particles staged in shared memory by
                              bulk asynchronous copies, 7 as 3 with the accumulators in
                              thread-private shared memory, 8 as 3 split over three threads
                              per particle run, one per z-slab of 9 nodes, 9 thread per
                              particle with the warp-level reduction of Sec. 4.2.2 (lanes
                              grouped by base cell, a shuffle tree per group, one float4
                              reduction per group and node), 10 the same over runs of equal
                              cells on consecutive lanes only (the paper's no-sort case),
                              11 as 4 with the runs flushed into a shared-memory node tile
                              private to each warp and one reduction per touched node,
                              12 thread per particle with lanes grouped by base cell whose
                              members sum the group's node values through shared memory, one
                              float4 reduction per group and node, 13 as 4 accumulating with
                              paired FP32 fused multiply-adds, 14 a warp per run of particles
                              with one lane per stencil node, taking the particles one at a
                              time into one float4 per lane and reducing the 27 nodes at each
                              change of cell, 15 as 4 with each thread's 8 particles taken
                              in the order of their base cells (see the autotuner) */
    int32_t g2p_variant;   /* tuning: 0 thread per particle, 1/2 node velocities cached in
                              registers over runs of 4/8 particles, 3 grid tile staged
                              in shared memory per CTA, 4 thread per particle at 64
                              registers, 5 the same with each CTA's particle inputs and
                              2x2x2-block grid tile staged by bulk asynchronous copies,
                              6 thread per particle at 48 registers, 7 as 4 with the nine
                              B-spline weights in shared memory (weight spilling, Sec. 3.2) */
    int32_t no_sort;       /* ablation (Sec. 6 sorting study): 1 = a rebuild maps the blocks
                              but leaves the particles in their storage order (no sort, no
                              permutation; mpm_read_order then returns MPM_EINVAL); results
                              are the same up to floating-point summation order.  0: sort */
    int32_t resort_interval; /* > 0: every this many substeps between rebuilds, re-order the
                              particles of each window of 1024 storage slots by their current
                              (block, cell) key, so that P2G keeps merging runs of particles
                              in one cell; 0: only the sort at rebuild (Sec. 4.2.2).  Same
                              results up to floating-point summation order. */
    int32_t transfer;      /* MPM_APIC (0): G2P sets v_p to the interpolated new grid velocity
                              vbar_p and moves x_p by dt vbar_p.  MPM_ASFLIP (1): the
                              integrator of the paper's fountain (Sec. 6.5, after Fei et al.
                              2021): with v0_p the interpolated grid velocity before forces,
                              v_p <- vbar_p + flip_alpha (v_p - v0_p) and
                              x_p <- x_p + dt (vbar_p + beta flip_alpha (v_p(old) - v0_p)),
                              beta = flip_beta_min if J < 1 - flip_compress_margin (J = det F
                              before this G2P; the fluid's tracked J) else flip_beta_max.
                              C, F and J update as in APIC.  ASFLIP keeps a
                              third grid buffer, always gathers with one thread per particle
                              (g2p_variant is ignored) and needs use_g2p2g = 0. */
    float flip_alpha;      /* ASFLIP, in [0, 1] */
    float flip_beta_min;   /* ASFLIP, in [0, 1] */
    float flip_beta_max;   /* ASFLIP, in [0, 1] */
    float flip_compress_margin; /* ASFLIP: m in [0, 1) of the compressed-state test J < 1 - m.
                              0 (the default) is the plain test J < 1.  A particle the sand
                              return map left at J = 1 exactly (in tension) sits on the plain
                              test's threshold, where the rounding of det F decides; m > 0
                              counts such particles as not compressed. */
    int32_t reserved[1];
} mpm_config;

enum { MPM_APIC = 0, MPM_ASFLIP = 1 };

/* Device memory provider.  alloc returns device memory usable on `stream`
 * or NULL; free releases it.  Pass NULL to mpm_create to use
 * cudaMallocAsync / cudaFreeAsync on the context's stream. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void (*free)(void* ptr, size_t bytes, void* stream, void* user);
    void* user;
} mpm_allocator;

/* Create a simulation context (Sec. 4: the grid of 4x4x4 blocks and the
 * empty particle set).  mats[0..n_mats-1] (n_mats <= 8) are copied.
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream). */
mpm_status mpm_create(const mpm_config* cfg, const mpm_material* mats, int n_mats,
                      const mpm_allocator* allocator, void* cuda_stream, mpm_ctx** out);

/* Append n particles at rest-state F = I, C = 0, Jp = 1.  x: n x 3 positions;
 * v: n x 3 velocities or NULL for zero; vol0: n rest volumes or NULL for
 * dx^3 / 8 each; material: index into the context's materials.  Capacity
 * grows to 4x the needed size when more than half full (Sec. 3.1, GPU
 * container).  Marks the mapping for a rebuild.  Syncs. */
mpm_status mpm_add_particles(mpm_ctx* ctx, int64_t n, const float* x, const float* v,
                             const float* vol0, int material, int on_device);

/* Particle source between substeps (Sec. 4.1: particle addition happens
 * between G2P and P2G; Sec. 6.4 Fountain).  Same arguments as
 * mpm_add_particles, but asynchronous: host data is staged through pinned
 * memory and appended on the context's stream, with no host wait unless the
 * particle capacity must grow (4x when half full).  New particles are not
 * sorted until the next rebuild; a rebuild is requested only if some new
 * particle's stencil, widened by one cell per side, reaches a block that
 * the last rebuild did not map (device-side input always requests one). */
mpm_status mpm_emit_particles(mpm_ctx* ctx, int64_t n, const float* x, const float* v,
                              const float* vol0, int material, int on_device);

/* Advance by one substep of size dt: [rebuild-mapping and sort, when some
 * particle neared the edge of its mapped blocks two substeps ago] ->
 * P2G (stress merged in) -> grid update (boundary merged in, next buffer
 * cleared) -> G2P (F update and return mapping merged in).  Asynchronous;
 * a rebuild costs one host wait for the new block count. */
mpm_status mpm_substep(mpm_ctx* ctx, float dt);

/* Advance by `duration` seconds of simulated time in adaptive substeps (the
 * paper's scenes take their step sizes from Fang et al. 2018, Sec. 6.5):
 * each substep uses dt = min(dt_max, cfl dx / (v + c)), c the largest
 * dilatational wave speed of the context's materials (sqrt((lambda + 2 mu) /
 * rho); sqrt(K gamma / rho) for the fluid) and v a bound on the particle
 * speed; the last steps of the interval are made equal so that they end on
 * it exactly.  v is the largest |v| after substep s - 2, reduced on the
 * device at the end of that substep (no stall: the host already waits for
 * it), grown by |g| dt per substep of age; after particles were added or
 * velocities written, one reduction with a stream sync supplies it instead.  cfl in (0, 1],
 * dt_max > 0.  dts: NULL, or room for max_substeps floats that receive each
 * substep's dt; n_substeps (may be NULL) receives the count.  MPM_ECAPACITY
 * if the interval needs more than max_substeps substeps (those ran);
 * MPM_ENONFINITE if the speed bound is not finite.  The
 * first call turns on the per-substep speed reduction for the context (one
 * small kernel reading v after G2P). */
mpm_status mpm_advance(mpm_ctx* ctx, double duration, float cfl, float dt_max, int64_t max_substeps,
                       float* dts, int64_t* n_substeps);

/* Copy the particle state out in insertion order; any pointer may be NULL
 * to skip that field.  Syncs; returns the sticky device error, if any. */
mpm_status mpm_read_state(mpm_ctx* ctx, float* x, float* v, float* C, float* F, float* Jp,
                          int on_device);

/* Overwrite the particle state (insertion order); NULL fields are kept.
 * Marks the mapping for a rebuild.  Syncs. */
mpm_status mpm_write_state(mpm_ctx* ctx, const float* x, const float* v, const float* C,
                           const float* F, const float* Jp, int on_device);

/* Wait for the stream and return the sticky device error, if any. */
mpm_status mpm_sync(mpm_ctx* ctx);

/* Run rebuild-mapping and the full sort now (Sec. 4.2.1, Sec. 4.2.2). Syncs. */
mpm_status mpm_rebuild(mpm_ctx* ctx);

int64_t mpm_num_particles(const mpm_ctx* ctx);
const char* mpm_last_error(const mpm_ctx* ctx); /* never NULL; owned by ctx */
void mpm_destroy(mpm_ctx* ctx);                  /* NULL is a no-op; syncs */

/* ---- batched scenes ---------------------------------------------------- */
/* Many small independent scenes advanced together: each phase of a substep
 * is one launch over all scenes, and the substep can be replayed from a CUDA
 * graph (the paper's principle of few kernels per substep, Sec. 3.1, and its
 * tail-effect argument, Sec. 4.1; the batching itself is not in the paper).
 * Grid blocks are indexed by (scene, Morton code) without compaction, and
 * rebuild-mapping runs per scene, only for the scenes whose free-zone test
 * fired.  Transfers are APIC (no ASFLIP form). */
typedef struct mpm_batch mpm_batch; /* opaque */

typedef struct {
    int32_t res[3];        /* 8..512 per axis */
    float dx;
    int32_t boundary;      /* mpm_boundary */
    int32_t wall;
    float gravity[3];
    int32_t material;      /* index into the batch's materials */
} mpm_scene_desc;

/* n_scenes <= 65535 scenes and n_mats <= 255 materials are copied.  Fails
 * with MPM_ECAPACITY if the scenes' block slots need more than 25 bits. */
mpm_status mpm_batch_create(int n_scenes, const mpm_scene_desc* scenes, const mpm_material* mats, int n_mats,
                            const mpm_allocator* allocator, void* cuda_stream, mpm_batch** out);
/* Host arrays (x, v: n x 3; vol0: n, NULL = dx^3/8; v NULL = 0), before the
 * first mpm_batch_substep (MPM_ENOTSUP afterwards). */
mpm_status mpm_batch_add_particles(mpm_batch* b, int scene, int64_t n, const float* x, const float* v,
                                   const float* vol0);
/* One substep of every scene; dt: n_scenes host floats.  The first call
 * uploads and sorts the particles (syncs).  Asynchronous afterwards. */
mpm_status mpm_batch_substep(mpm_batch* b, const float* dt);
/* Capture the substep in CUDA graphs and replay them (one graph launch per
 * substep instead of five stream operations).  Default off; needs a stream
 * other than the legacy default stream (MPM_EINVAL otherwise). */
mpm_status mpm_batch_use_graphs(mpm_batch* b, int on);
/* Tuning: particles per thread in the batched P2G (1, 4 or 8). */
mpm_status mpm_batch_set_p2g_chunk(mpm_batch* b, int k);
/* Tuning: warps per CTA (2, 4 or 8) of the per-phase P2G and G2P launches. */
mpm_status mpm_batch_set_cta_warps(mpm_batch* b, int warps);
/* Persistent form (on = 1): the whole substep of all scenes is one
 * cooperative launch of as many CTAs as the device holds at once; the CTAs
 * take tiles of particles (P2G chunks of mpm_batch_set_p2g_chunk particles
 * per thread, G2P one per thread) and of active grid nodes from a device
 * counter per phase, and meet at a grid-wide barrier between P2G, the grid
 * update and G2P.  A barrier wait gives up after about a second; the next
 * syncing call then returns MPM_ETIMEOUT.  Replayed from CUDA graphs like
 * the per-phase form.  Off (0, the default): one launch per phase.  Results
 * are identical up to float summation order. */
mpm_status mpm_batch_set_persistent(mpm_batch* b, int on);
/* Host copies of one scene's state in that scene's insertion order; any
 * pointer may be NULL.  Syncs; returns the sticky device error, if any. */
mpm_status mpm_batch_read_state(mpm_batch* b, int scene, float* x, float* v, float* C, float* F, float* Jp);
mpm_status mpm_batch_sync(mpm_batch* b);
/* out4: substeps, per-scene remaps, kernel launches, graph launches. */
mpm_status mpm_batch_get_stats(const mpm_batch* b, int64_t* out4);
/* Particles of one scene, or of all scenes for scene == -1. */
int64_t mpm_batch_num_particles(const mpm_batch* b, int scene);
const char* mpm_batch_last_error(const mpm_batch* b);
void mpm_batch_destroy(mpm_batch* b);

/* ---- differentiable substep -------------------------------------------- */
/* A differentiable form of the substep (not in the paper): fixed-corotated
 * elasticity with a per-particle Young's modulus E_p, a common Poisson ratio
 * and density, MLS-MPM transfers on a dense grid (res0 x res1 x res2 nodes,
 * walls as in mpm_config).  State of one particle: 24 floats x[3] v[3] C[9]
 * H[9], row-major, where H = F - I is the displacement gradient (kept instead
 * of F so that FP32 resolves small strains to full relative precision; the
 * adjoint with respect to H equals the adjoint with respect to F).  All
 * arrays are device pointers with n rows.  The caller keeps the states
 * (checkpointing is the caller's choice). */
typedef struct mpm_diff mpm_diff; /* opaque */

/* vol0: n device floats, or NULL for dx^3/8 each.  cfg->transfer must be
 * MPM_APIC (else MPM_EINVAL). */
mpm_status mpm_diff_create(const mpm_config* cfg, float nu, float rho, int64_t n, const float* vol0,
                           const mpm_allocator* allocator, void* cuda_stream, mpm_diff** out);
/* s_out = one substep of s_in with moduli E (n floats); s_out must not alias s_in. */
mpm_status mpm_diff_forward(mpm_diff* d, float dt, const float* E, const float* s_in, float* s_out);
/* Hand-written adjoint of mpm_diff_forward at s_in: given g_out = dL/ds_out,
 * writes g_in = dL/ds_in and adds dL/dE into gE (n floats).  Re-runs the
 * forward P2G and grid update, then the reverse G2P, grid update and P2G. */
mpm_status mpm_diff_adjoint(mpm_diff* d, float dt, const float* E, const float* s_in, const float* g_out,
                            float* g_in, float* gE);
/* Wait for the stream; MPM_EDOMAIN if a particle's stencil left the grid. */
mpm_status mpm_diff_sync(mpm_diff* d);
void mpm_diff_destroy(mpm_diff* d);

/* ---- introspection (tests, benchmarks) ------------------------------- */

typedef struct {
    int64_t substeps;      /* substeps run */
    int64_t rebuilds;      /* rebuild-mapping runs */
    int64_t n_pblocks;     /* physical blocks at the last rebuild */
    int64_t grid_capacity; /* blocks the grid buffers can hold */
    int64_t particle_capacity;
    int64_t kernel_launches; /* kernels this context has launched */
} mpm_stats;

mpm_status mpm_get_stats(const mpm_ctx* ctx, mpm_stats* out);

/* Sort keys of the particles in storage order after the last rebuild
 * (Sec. 4.2.2: Morton(block) << 6 | Morton(cell), ascending) and the
 * insertion index of each stored particle.  keys, ids: n entries each;
 * either may be NULL.  Syncs. */
mpm_status mpm_read_order(mpm_ctx* ctx, uint32_t* keys, int32_t* ids, int on_device);

/* Physical blocks of the last rebuild (Sec. 4: gblocks and their 3x3x3
 * neighbours) as Morton slots in block-index order (ascending).  Writes
 * min(count, cap) entries to slots (may be NULL) and the count.  Syncs. */
mpm_status mpm_read_blocks(mpm_ctx* ctx, int32_t* slots, int64_t cap, int64_t* count);

/* Run the P2G phase for the current state with step dt into a fresh grid
 * and copy the result out as a dense res0 x res1 x res2 array of
 * (m, p_x, p_y, p_z) float quadruples, node (i, j, k) at
 * 4 * (i + res0 * (j + res1 * k)).  Does not advance the simulation.
 * Rebuilds first if needed.  Syncs. */
mpm_status mpm_debug_p2g(mpm_ctx* ctx, float dt, float* grid_out, int on_device);

/* Switch the P2G scatter variant (mpm_config.p2g_variant) between substeps;
 * used by the autotuner.  Results are identical up to float summation order. */
mpm_status mpm_set_p2g_variant(mpm_ctx* ctx, int variant);
/* Same for the G2P gather variant (mpm_config.g2p_variant). */
mpm_status mpm_set_g2p_variant(mpm_ctx* ctx, int variant);
/* Particle store layout (the paper's SoA / AoSoA study, Sec. 6.2): 0 = SoA,
 * one array per state channel (the default); 1 = AoSoA, packets of 32
 * particles with each channel's 32 floats contiguous inside the packet, so a
 * warp's particles keep their whole state in one 4 KB span.  The current
 * particles are converted on the stream.  AoSoA runs P2G variants 3, 4, 14 and 15,
 * G2P variants 4, 6 and 7, 2 or 4 warps per CTA and separate APIC transfers only: switching
 * to it from another configuration, or to another configuration under it,
 * returns MPM_EINVAL.  Results are identical up to float summation order. */
mpm_status mpm_set_layout(mpm_ctx* ctx, int aosoa);
/* Warps per CTA of the register-run P2G (p2g_variant 3 and 4) and of the
 * 64-register G2P (g2p_variant 4): 2, 4 (the default) or 8, at the same
 * registers per thread (the paper's warps-per-block study, Sec. 6.2).  The
 * other variants keep their own CTA sizes.  Results are identical up to float
 * summation order.  MPM_EINVAL for other values. */
mpm_status mpm_set_cta_warps(mpm_ctx* ctx, int warps);
/* Change mpm_config.resort_interval between substeps (the window re-sort that
 * restores P2G's runs of equal cells between the sorts of Sec. 4.2.2; 0 turns
 * it off); used by the autotuner.  Results are identical up to float
 * summation order.  MPM_EINVAL for a negative interval. */
mpm_status mpm_set_resort_interval(mpm_ctx* ctx, int interval);
/* Switch between separate phases (0) and the fused G2P2G transfer (1)
 * between substeps (mpm_config.use_g2p2g).  MPM_EINVAL for on = 1 when the
 * context uses MPM_ASFLIP.  The fused kernel scatters the next substep's
 * momentum with the current dt, so a substep whose dt differs from the
 * previous one first repeats that P2G with its own dt (one extra launch). */
mpm_status mpm_set_g2p2g(mpm_ctx* ctx, int on);

/* Replay the steady-state substep (P2G, grid update, G2P and the flag copy;
 * in fused mode the grid update and G2P2G) from CUDA graphs (on = 1): one
 * graph per mode, flag-ring slot, current grid buffer and current particle
 * buffer, captured on first use and dropped at every rebuild, particle
 * addition or variant change (the substep of a drop launches directly).  A
 * change of dt re-captures the substep and updates the instantiated graph in
 * place, so adaptive steps (mpm_advance) replay too.  Removes the launch gaps
 * between the phases, which dominate small scenes.  The paper launches
 * kernels directly; this is a GB300-side choice with the same results.
 * EINVAL if the context runs on the legacy default stream (it cannot be
 * captured).  Not used while profiling is on.  mpm_graph_launches returns
 * the number of graph replays so far. */
mpm_status mpm_use_graphs(mpm_ctx* ctx, int on);
int64_t mpm_graph_launches(const mpm_ctx* ctx);

/* Per-phase timing with CUDA events on the context's stream.  Phase ids:
 * 0 rebuild, 1 P2G, 2 grid update, 3 G2P.  mpm_profile_read syncs and
 * writes total milliseconds and launch counts per phase since the last
 * read (n_phases <= 4 entries each). */
#define MPM_PHASES 4
mpm_status mpm_profile_enable(mpm_ctx* ctx, int on);
mpm_status mpm_profile_read(mpm_ctx* ctx, double* ms, int64_t* launches, int n_phases);

/* ---- stand-alone kernels ---------------------------------------------- */

/* Stable LSD radix sort of (key, value) pairs on the device (the histogram
 * sort of Sec. 4.2.2 with 8-bit digits over the low key_bits bits).
 * keys_in/vals_in: n entries (read only); keys_out/vals_out: n entries.
 * Scratch: call with scratch == NULL to get the byte count in
 * *scratch_bytes; then pass a device buffer of at least that size (the
 * preallocated scratch of Sec. 6.3.1).  Asynchronous on cuda_stream. */
mpm_status mpm_radix_sort_pairs(const uint32_t* keys_in, const int32_t* vals_in,
                                uint32_t* keys_out, int32_t* vals_out, int64_t n, int key_bits,
                                void* scratch, size_t* scratch_bytes, void* cuda_stream);

/* Allocation-free variant of mpm_radix_sort_pairs.  The paper has no
 * counterpart; it exists for callers that must not allocate device memory
 * themselves or through the library: a host engine or plugin that owns every
 * device allocation and gives libraries no allocator hook, or a per-frame
 * callback in a real-time loop where an allocation may synchronize the device
 * and blow the frame budget.  Such a caller passes only its inputs and
 * outputs (device pointers, same layout and meaning as in
 * mpm_radix_sort_pairs, which must not alias); the scratch lives in one
 * fixed array of device memory inside the library, sized for
 * MPM_SORT_NOALLOC_MAX_KEYS keys (about 8.5 MB), which every GPU that loads
 * the library holds until the process exits.
 *   - n > MPM_SORT_NOALLOC_MAX_KEYS returns MPM_ECAPACITY and launches nothing.
 *   - The first call on each device looks up that device's address of the
 *     array (a one-time set-up with that device current); make that first
 *     call before any CUDA stream capture.  The address is kept for the life
 *     of the process: after cudaDeviceReset (or any teardown of the device's
 *     primary context) it may be stale, so do not call this entry point on a
 *     device that was reset after its first call.
 *   - No call allocates or frees memory (no cudaMalloc / cudaFree, no
 *     allocating library routine).
 *   - All calls share the one array and it keeps whatever the last call left
 *     there: every call overwrites what it reads, so nothing carries over, but
 *     two calls whose GPU work overlaps (different streams, or different
 *     host threads) race on it and corrupt each other's result.
 * Asynchronous on cuda_stream. */
#define MPM_SORT_NOALLOC_MAX_KEYS (1 << 20)
mpm_status mpm_radix_sort_pairs_noalloc(const uint32_t* keys_in, const int32_t* vals_in,
                                        uint32_t* keys_out, int32_t* vals_out, int64_t n,
                                        int key_bits, void* cuda_stream);

/* Batched SVD / stress evaluation of the constitutive model (Sec. 4.1:
 * SVD, plasticity projection and stress computation), for testing the
 * device routines in isolation.  F: n x 9, Jp: n; outputs U, V: n x 9,
 * sig: n x 3, tau: n x 9 (any output may be NULL).  Device pointers.
 * Syncs. */
mpm_status mpm_debug_svd(const float* F, float* U, float* sig, float* V, int64_t n);
mpm_status mpm_debug_stress(const mpm_material* mat, const float* F, const float* Jp,
                            float* tau, int64_t n);
/* Apply the end-of-G2P return map to n trial F (in place) and Jp. */
mpm_status mpm_debug_plasticity(const mpm_material* mat, float* F, float* Jp, int64_t n);

/* Failure-detection check of the bounded device waits (no counterpart in
 * the paper): one CTA waits on a shared-memory mbarrier that expects bytes no
 * copy will deliver, gives up after max_iter polls (1..65536, each at most
 * ~1 us) and records the time-out as the staged kernels do.  Returns
 * MPM_ETIMEOUT when the wait gave up (the expected result), MPM_OK if it
 * did not, MPM_EINVAL for max_iter out of range.  The device stays usable:
 * nothing faults, nothing is left in flight.  Synchronous. */
mpm_status mpm_debug_wait_timeout(int max_iter);

/* Measurement of a second ceiling of P2G (not part of the substep): the rate
 * at which L2 applies float4 reductions, the operation P2G's scatter ends in
 * (Sec. 4.2.2 aggregates per warp to issue fewer of them).  Launches `threads`
 * threads (a multiple of 32) on `stream`; each applies `reds_per_thread`
 * reductions of (1, 1, 1, 1) to the device array `grid` of `nodes` float4
 * (caller-owned, 16-byte aligned, nodes a multiple of 32; a few MB keeps it
 * resident in L2 like the P2G grid).  Each step picks spans of 32 consecutive
 * nodes by a pseudo-random sequence: pattern 0 gives each lane of a warp its
 * own node of one span (32 distinct nodes in 4 lines), pattern 1 four lanes per
 * node of one span, pattern 2 each lane node 0 of its own span (32 lines per
 * warp instruction), pattern 3 one node for the whole warp.  The caller times
 * it (events on `stream`) and may check that the
 * fourth components sum to threads * reds_per_thread.  Asynchronous.
 * MPM_EINVAL for a null or misaligned grid or sizes out of range (1 to 4096
 * reductions per thread), MPM_ECUDA if the launch fails. */
mpm_status mpm_debug_red_rate(void* grid, int64_t nodes, int64_t threads, int32_t reds_per_thread, int32_t pattern,
                              void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MPM_H */
